// Adjoint kernels interface.
#pragma once

#include "transport.cuh"
#include "usrt_device.cuh"

namespace usrt {

constexpr int MAX_P = 4 * MAX_MEDIA + 2;  // with a roughness per medium
constexpr int MAX_P_ACQ = MAX_P + 2 + MAX_TX;  // with the acquisition slots (c_bf, pitch, steering angles)

struct PulseP {
  float f0, sig, fs, half;  // half = 4 sqrt(sigma) fs (support in samples)
  int ns;
  // per-sample steps of the gather's recurrences: the carrier phase advances by 2 pi f0 / fs
  // (cos, sin), and the Gaussian's ratio E(x + 1/fs) / E(x) is multiplied by
  // exp(-2 / (fs^2 sigma)) every sample
  float rot_c, rot_s, env_qq;
};

struct AdjArgs {
  SceneDev S;
  Media med;
  Acq acq;
  PulseP pulse;
  const uint32_t* record;  // (path - path_base) * (kmax + 1) + k
  long long path_base;
  uint32_t n_paths;
  const float* grf;        // dL/dRF [ntx][ne][ns]
  float* gpart;            // [gridDim.x][P] per-block partial gradients
  int P;                   // gradient slots: 3M + 2 scene parameters (+ 2 + ntx with acq_slot)
  int acq_slot;            // >= 0: slot of dL/dc_bf, then dL/dpitch, then dL/dth_t for every transmit t
  int accumulate;          // add into gpart instead of overwriting
  float* g_tris;           // non-null: dL/d(triangle vertices) [n_tris][9], accumulated atomically
  NeeQ nee;                // the pass's secondary-ray jobs
  NeeRes nres;             // their stored results (null members: trace them again)
  const Counters* cnt;     // job counts per round
  float2* seeds;           // per (path - path_base, k): (dL/da, dL/dtau) seeded by secondary rays
  float4* seedv;           // with secondary rays at rough events, per (path - path_base, k) two entries:
                           // (dL/d(event point), 0), (dL/d(incident direction), 0)
  const uint32_t* active;  // paths with an arrival, grouped by event count
  const uint32_t* n_active;
};

// secondary-ray adjoint (job-parallel): seeds + direct parameter derivatives
void launch_nee_adjoint(const AdjArgs& a, int grid, cudaStream_t st);
// active paths of the record grouped by event count: work = 2 counters + 17 offsets + n entries;
// pclass: n_paths bytes of scratch (each path's class)
// rough_mask: media whose interface events send secondary rays (their paths are active too)
void launch_active_paths(const uint32_t* record, uint32_t n_paths, int kmax, uint32_t* work, uint8_t* pclass,
                         uint32_t* active, int grid, cudaStream_t st, uint32_t rough_mask = 0u,
                         const float4* tri_nrm = nullptr);
void launch_path_adjoint(const AdjArgs& a, int grid, cudaStream_t st);
cudaError_t adjoint_set_attrs();
void launch_grad_reduce(const float* gpart, int nblocks, int P, float* g, cudaStream_t st);
// columns [0, Ps) of gpart to g, the others to g2 (added to it when acc2)
void launch_grad_reduce_split(const float* gpart, int nblocks, int P, int Ps, float* g, float* g2, int acc2,
                              cudaStream_t st);
// dL/dq_j = sum_i g[i] * tan[j * n + i] for j < n_param (one block per parameter, fixed order)
void launch_tangent_dot(long long n, const float* g, int n_param, const float* tan, float* out, cudaStream_t st);
void launch_splat_adjoint(const Acq& q, const PulseP& P, const int32_t* tx, const int32_t* e, const float* tau,
                          const float* a, long long n, const float* grf, float* ga, float* gt, float* gf, int grid,
                          cudaStream_t st);
void launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, long long n,
                        uint32_t* out, int grid, cudaStream_t st);

}  // namespace usrt
