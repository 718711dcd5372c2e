// Image-formation kernels interface.
#pragma once

#include "usrt_device.cuh"

namespace usrt {

// DAS; with a device status word the TMA-staged kernel is used when the shape allows
void launch_das(const Acq& q, const Img& im, const float* rf, float* irf, int grid, cudaStream_t st,
                int* status = nullptr);
// transposed DAS, deterministic (64-bit fixed-point accumulation): acc is scratch of
// ntx * ne * ns words, maxbits one word
void launch_das_adj(const Acq& q, const Img& im, const float* gi, float* grf, int grid, cudaStream_t st,
                    unsigned long long* acc, unsigned int* maxbits);
// DAS derivative in (c_bf, pitch, steering angles) contracted with gi: das_acq_blocks(im)
// partial rows of 2 + ntx floats into part (reduce them with launch_grad_reduce_split)
int das_acq_blocks(const Img& im);
void launch_das_acq(const Acq& q, const Img& im, const float* rf, const float* gi, float* part, cudaStream_t st);
// envelope + log compression.  key points to 2 words (packed (E_max, argmax), barrier counter).
// With bmode: one cooperative fused kernel when the image fits (env untouched) and the fused
// path is enabled (us_set_envlog_fused), else envelope -> env then log compression.  Without
// bmode: envelope -> env and the key only.  status (may be null) receives ST_TIMEOUT if the
// fused kernel's grid barrier expires; fault_barrier != 0 makes that barrier wait for an
// arrival no block makes (1 ms limit), to test the report.  Returns the number of kernels
// launched; launch_err (may be null) the first launch error of this call alone.
int launch_envlog(const Img& im, const float* irf, float* env, unsigned long long* key, float* bmode, int grid,
                  cudaStream_t st, int* status = nullptr, int fault_barrier = 0, cudaError_t* launch_err = nullptr);
void launch_loss(const Img& im, const float* b, const float* bref, float* gb, float* part, int nparts, float* loss,
                 cudaStream_t st);
void launch_envlog_vjp(const Img& im, const float* irf, const float* gb, float* env, unsigned long long* key,
                       float* part, int nparts, float* live_sum, float* gi, int grid, cudaStream_t st);
cudaError_t image_set_attrs(int nd);

}  // namespace usrt
