// Optimiser step of the inverse problem (Sec. 3.4 parameterisation, Sec. 3.7 optimiser, Alg. 1):
// the unconstrained variables theta_u are clipped to [0, 1] (Eq. clip01) and scaled into the
// admissible physical ranges (Eq. scale_phys); the physical gradient is carried back through the
// scale and the clip (Eq. clip_grad), clipped by its global L2 norm, and Adam with per-parameter
// learning rates (parameter groups) and bias corrections updates theta_u (Eq. adam).
// One block handles the whole (short) parameter vector, so the norm needs no second launch.
#include <cuda_runtime.h>

#include <cstdint>

namespace usrt {

constexpr int OPT_THREADS = 256;

__global__ void k_param_map(int n, const float* __restrict__ theta_u, const float* __restrict__ lo,
                            const float* __restrict__ hi, float* __restrict__ theta) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float tn = fminf(fmaxf(theta_u[j], 0.0f), 1.0f);
    theta[j] = fmaf(tn, hi[j] - lo[j], lo[j]);
  }
}

__global__ void __launch_bounds__(OPT_THREADS) k_adam_step(int n, float* __restrict__ theta_u,
                                                           const float* __restrict__ grad, const float* __restrict__ lo,
                                                           const float* __restrict__ hi, const float* __restrict__ lr,
                                                           float beta1, float beta2, float eps, float clip_norm,
                                                           float bc1, float bc2, float* __restrict__ m,
                                                           float* __restrict__ v) {
  __shared__ float red[OPT_THREADS / 32];
  __shared__ float scale_s;
  // gradient with respect to theta_u: chain through the scale, zero where the clip saturates
  float ss = 0.0f;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float tu = theta_u[j];
    const float g = (tu > 0.0f && tu < 1.0f) ? grad[j] * (hi[j] - lo[j]) : 0.0f;
    ss = fmaf(g, g, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];  // fixed order
    const float norm = sqrtf(t);
    scale_s = (clip_norm > 0.0f && norm > clip_norm) ? clip_norm / norm : 1.0f;
  }
  __syncthreads();
  const float sc = scale_s;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float tu = theta_u[j];
    const float g = ((tu > 0.0f && tu < 1.0f) ? grad[j] * (hi[j] - lo[j]) : 0.0f) * sc;
    const float mj = fmaf(beta1, m[j], (1.0f - beta1) * g);
    const float vj = fmaf(beta2, v[j], (1.0f - beta2) * g * g);
    m[j] = mj;
    v[j] = vj;
    const float mh = mj / bc1, vh = vj / bc2;
    theta_u[j] = tu - lr[j] * mh / (sqrtf(vh) + eps);
  }
}

void launch_param_map(int n, const float* theta_u, const float* lo, const float* hi, float* theta, cudaStream_t st) {
  k_param_map<<<1, OPT_THREADS, 0, st>>>(n, theta_u, lo, hi, theta);
}

void launch_adam_step(int n, float* theta_u, const float* grad, const float* lo, const float* hi, const float* lr,
                      float beta1, float beta2, float eps, float clip_norm, float bc1, float bc2, float* m, float* v,
                      cudaStream_t st) {
  k_adam_step<<<1, OPT_THREADS, 0, st>>>(n, theta_u, grad, lo, hi, lr, beta1, beta2, eps, clip_norm, bc1, bc2, m, v);
}

}  // namespace usrt
