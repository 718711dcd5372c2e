// Sort-based splat interface.
#pragma once

#include "usrt_device.cuh"

namespace usrt {

typedef uint4 Arrival;  // (row, tq, bits(a), path id)

constexpr int ROW_THREADS = 512;
constexpr int ROW_MAX_R = 8;   // samples per thread: n_samples <= ROW_THREADS * ROW_MAX_R
constexpr int HALO = 64;       // bins kept on each side of the record (>= pulse half-width)
constexpr int MAX_SPLAT_NS = ROW_THREADS * ROW_MAX_R;

struct SplatGeom {
  int nrows, ns, nbins;  // nbins = ns + 2 * HALO
  int dlo, ntaps;        // taps d = dlo .. dlo + ntaps - 1 (d = n - bin)
  float Sig, Om;         // sigma * fs^2, 2 pi f0 / fs
};

// moments of a row live in shared memory with one spare slot after every 8 (slot of x: x + x/8),
// bins shifted so that each thread's convolution window starts on a multiple of 8
__host__ __device__ inline int mom_slot(int x) { return x + (x >> 3); }
__host__ __device__ inline int row_mom_stride(int ns) {
  const int xn = ns + 2 * HALO + 16;
  return mom_slot(xn) + 8;
}
__host__ __device__ inline int row_mom_shift(const SplatGeom& g) { return (((g.dlo - HALO + 7) % 8) + 8) % 8; }

struct SplatWork {
  uint32_t* row_cnt;     // [nrows]
  uint32_t* row_off;     // [nrows + 1]
  uint32_t* row_cursor;  // [nrows]
  uint2* bucket;         // [cap] (tq, bits(a)) in row order
  uint2* scratch;        // [cap] (tq, bits(a)) in (row, bin) order
};

size_t row_splat_smem(const SplatGeom& g);
int row_splat_threads(const SplatGeom& g);  // 8 output samples per thread
void launch_pulse_table(const SplatGeom& g, float* G, cudaStream_t st);
// row bucketing (3 kernels), then the per-row sort / reduction / convolution (1 kernel)
void launch_splat_sort(const SplatGeom& g, const Arrival* arr, const uint32_t* n_arr, uint32_t cap, SplatWork w,
                       int grid, cudaStream_t st);
void launch_splat_rows(const SplatGeom& g, SplatWork w, const float* G, float* rf, cudaStream_t st);
void launch_pack_arrivals(const int32_t* tx, const int32_t* e, const float* tau, const float* a, long long n, int ne,
                          float fs, Arrival* out, uint32_t* n_out, int grid, cudaStream_t st);
cudaError_t splat_set_attrs(const SplatGeom& g);
// exclusive scan of n counts (one block): off[n] = total, cursor zeroed
void launch_count_scan(const uint32_t* cnt, uint32_t* off, uint32_t* cursor, int n, cudaStream_t st);
cudaError_t row_scatter_set_attrs(int nrows);
cudaError_t row_hist_set_attrs(int nrows);

}  // namespace usrt
