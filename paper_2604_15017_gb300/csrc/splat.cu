// Sort-based RF splat (Sec. 2.3.4, Eq. axial_sig): RF[row][n] = sum_i a_i s(n / fs - tau_i).
//
// No scatter of pulse taps with atomics.  Instead:
//   1. rows:   counting sort of the arrivals by row = tx * n_elem + e (histogram, scan, scatter);
//   2. per row (one CTA): counting sort by time bin b = floor(tau fs) into an L2-resident
//      scratch, then a segmented warp reduction of the Taylor moments
//        M_j(b) = sum_{i in b} a_i (-delta_i)^j,  delta_i = tau_i fs - (b + 1/2),  j < 8,
//      and finally the convolution RF[n] = sum_j sum_d G_j(d) M_j(n - d) with the table
//        G_j(d) = g^(j)(d - 1/2) / j!,  g(x) = s(x / fs)
//      (truncation after 8 moments: |delta| <= 1/2 sample gives < 1e-7 relative error).
#include <cooperative_groups.h>

#include "splat.cuh"

namespace cg = cooperative_groups;

namespace usrt {

// ------------------------------------------------------------------------------------------
// pulse-derivative table: g(x) = Im h(x), h(x) = exp(-x^2 / S + i W x) with S = sigma fs^2 and
// W = 2 pi f0 / fs; with y = (x - i W S / 2) / sqrt(S),  h^(j)(x) = h(x) (-1/sqrt(S))^j H_j(y)
// (physicists' Hermite polynomials, H_{j+1} = 2 y H_j - 2 j H_{j-1}).
// ------------------------------------------------------------------------------------------
__global__ void k_pulse_table(SplatGeom g, float* G) {
  const int d = threadIdx.x;
  if (d >= g.ntaps) return;
  const float x = (float)(g.dlo + d) - 0.5f;
  const float S = g.Sig, W = g.Om;
  const float rs = rsqrtf(S);
  const float yr = x * rs, yi = -0.5f * W * S * rs;
  float e_s, e_c;
  const float mag = expf(-x * x / S);
  sincosf(W * x, &e_s, &e_c);
  const float hr = mag * e_c, hi = mag * e_s;  // h(x)
  float Hr0 = 1.0f, Hi0 = 0.0f, Hr1 = 2.0f * yr, Hi1 = 2.0f * yi;
  float fact = 1.0f, sc = 1.0f;
  for (int j = 0; j < K_MOM; ++j) {
    float Hr, Hi;
    if (j == 0) {
      Hr = Hr0;
      Hi = Hi0;
    } else if (j == 1) {
      Hr = Hr1;
      Hi = Hi1;
    } else {
      const float nr = 2.0f * (yr * Hr1 - yi * Hi1) - 2.0f * (j - 1) * Hr0;
      const float ni = 2.0f * (yr * Hi1 + yi * Hr1) - 2.0f * (j - 1) * Hi0;
      Hr0 = Hr1;
      Hi0 = Hi1;
      Hr1 = nr;
      Hi1 = ni;
      Hr = nr;
      Hi = ni;
    }
    if (j > 0) {
      fact *= (float)j;
      sc *= -rs;
    }
    // Im(h * H) * sc / j!
    G[j * g.ntaps + d] = (hr * Hi + hi * Hr) * sc / fact;
  }
}

// ------------------------------------------------------------------------------------------
// 1. bucket by row
// ------------------------------------------------------------------------------------------
__global__ void k_row_hist(const Arrival* arr, const uint32_t* n_arr, uint32_t cap, uint32_t* row_cnt, int nrows) {
  extern __shared__ uint32_t h[];
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) h[r] = 0;
  __syncthreads();
  const uint32_t n = min(*n_arr, cap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&h[arr[i].x], 1u);
  __syncthreads();
  for (int r = threadIdx.x; r < nrows; r += blockDim.x)
    if (h[r]) atomicAdd(&row_cnt[r], h[r]);
}

// exclusive scan of the row counts (one block of 1024 threads); off[nrows] = total
// exclusive scan of nrows counts by one block: warp w owns a contiguous segment, read and written
// 32 entries at a time (coalesced) with a shuffle scan per chunk; the 32 segment totals are
// scanned by warp 0
__global__ void k_row_scan(const uint32_t* cnt, uint32_t* off, uint32_t* cursor, int nrows) {
  __shared__ uint32_t seg_total[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = (nrows + nw - 1) / nw;
  const int lo = warp * seg, hi = min(nrows, lo + seg);
  uint32_t run = 0;
  for (int b = lo; b < hi; b += 32) {
    const int r = b + lane;
    uint32_t v = r < hi ? cnt[r] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += u;
    }
    run += __shfl_sync(0xFFFFFFFFu, v, 31);
  }
  if (lane == 0) seg_total[warp] = run;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? seg_total[lane] : 0u;
    const uint32_t own = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) seg_total[lane] = v - own;  // exclusive
    if (lane == 31) off[nrows] = v;
  }
  __syncthreads();
  run = seg_total[warp];
  for (int b = lo; b < hi; b += 32) {
    const int r = b + lane;
    const uint32_t c = r < hi ? cnt[r] : 0u;
    uint32_t v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += u;
    }
    if (r < hi) {
      off[r] = run + v - c;
      cursor[r] = 0;
    }
    run += __shfl_sync(0xFFFFFFFFu, v, 31);
  }
}

// scatter into row buckets: each block takes chunks of CH arrivals, ranks them per row in
// shared memory and reserves one range per (chunk, row) with a single global atomic
constexpr int SC_THREADS = 512;
constexpr int SC_PER = 16;
constexpr int SC_CH = SC_THREADS * SC_PER;
__global__ void __launch_bounds__(SC_THREADS) k_row_scatter(const Arrival* arr, const uint32_t* n_arr, uint32_t cap,
                                                            const uint32_t* off, uint32_t* cursor, uint2* out,
                                                            int nrows) {
  extern __shared__ uint32_t sm[];
  uint32_t* h = sm;           // per-row count in this chunk
  uint32_t* base = sm + nrows;
  const uint32_t n = min(*n_arr, cap);
  for (uint32_t c0 = blockIdx.x * SC_CH; c0 < n; c0 += gridDim.x * SC_CH) {
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) h[r] = 0;
    __syncthreads();
    uint32_t row[SC_PER], rank[SC_PER];
    uint2 val[SC_PER];
#pragma unroll
    for (int k = 0; k < SC_PER; ++k) {
      const uint32_t i = c0 + k * SC_THREADS + threadIdx.x;
      row[k] = 0xFFFFFFFFu;
      if (i < n) {
        const Arrival A = arr[i];
        row[k] = A.x;
        val[k] = make_uint2(A.y, A.z);
        rank[k] = atomicAdd(&h[A.x], 1u);
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x)
      if (h[r]) base[r] = off[r] + atomicAdd(&cursor[r], h[r]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SC_PER; ++k)
      if (row[k] != 0xFFFFFFFFu) out[base[row[k]] + rank[k]] = val[k];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// 2. per row: sort by bin, segmented moment reduction, convolution
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(ROW_THREADS) k_row_splat(SplatGeom g, const uint2* bucket, const uint32_t* off,
                                                           uint2* scratch, const float* Gtab, float* rf) {
  extern __shared__ float smf[];
  const int row = blockIdx.x;
  const int NB = g.nbins;         // bins -HALO .. ns + HALO - 1
  const int MS = row_mom_stride(g.ns);
  const int sh = row_mom_shift(g);  // bin x is stored at mom_slot(x + sh)
  float* M = smf;                 // [K_MOM][MS], padded: one spare slot after every 8
  uint32_t* hist = reinterpret_cast<uint32_t*>(M + K_MOM * MS);  // [NB + 1]
  float* G = reinterpret_cast<float*>(hist + NB + 1);            // [K_MOM][MAX_TAPS], zero past ntaps
  const uint32_t a0 = off[row], a1 = off[row + 1];
  for (int i = threadIdx.x; i < K_MOM * MS; i += blockDim.x) M[i] = 0.0f;
  for (int i = threadIdx.x; i <= NB; i += blockDim.x) hist[i] = 0;
  for (int i = threadIdx.x; i < K_MOM * MAX_TAPS; i += blockDim.x) {
    const int j = i / MAX_TAPS, d = i - j * MAX_TAPS;
    G[i] = d < g.ntaps ? Gtab[j * g.ntaps + d] : 0.0f;
  }
  __syncthreads();
  const uint32_t mask = (1u << TQ_FRAC) - 1u;
  // pass 1: histogram of bins
  for (uint32_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    const int b = (int)(bucket[i].x >> TQ_FRAC) - TQ_OFFSET + HALO;
    if (b >= 0 && b < NB) atomicAdd(&hist[b], 1u);
  }
  __syncthreads();
  // exclusive scan of hist (NB entries) in place: per-thread serial chunk + block scan
  {
    __shared__ uint32_t part[ROW_THREADS];
    const int per = (NB + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(NB, lo + per);
    uint32_t s = 0;
    for (int b = lo; b < hi; ++b) s += hist[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      uint32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int b = lo; b < hi; ++b) {
      const uint32_t c = hist[b];
      hist[b] = run;
      run += c;
    }
    if (threadIdx.x == blockDim.x - 1) hist[NB] = part[threadIdx.x];
  }
  __syncthreads();
  // pass 2: scatter into bin order (scratch shares the row's index range)
  for (uint32_t i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    const uint2 v = bucket[i];
    const int b = (int)(v.x >> TQ_FRAC) - TQ_OFFSET + HALO;
    if (b >= 0 && b < NB) scratch[a0 + atomicAdd(&hist[b], 1u)] = v;
  }
  __syncthreads();
  // after pass 2 hist[b] = end of bin b; total kept arrivals:
  const uint32_t nk = hist[NB];
  __syncthreads();
  // pass 3: segmented warp reduction of the moments over the bin-sorted arrivals
  const int lane = threadIdx.x & 31;
  for (uint32_t base = (threadIdx.x & ~31u); base < nk; base += blockDim.x) {
    const uint32_t i = base + lane;
    int b = -1;
    float m[K_MOM];
#pragma unroll
    for (int j = 0; j < K_MOM; ++j) m[j] = 0.0f;
    if (i < nk) {
      const uint2 v = scratch[a0 + i];
      b = (int)(v.x >> TQ_FRAC) - TQ_OFFSET + HALO;
      const float delta = (float)(v.x & mask) * (1.0f / (float)(1u << TQ_FRAC)) - 0.5f;
      float p = __uint_as_float(v.y);
      m[0] = p;
#pragma unroll
      for (int j = 1; j < K_MOM; ++j) {
        p = p * (-delta);  // the 1/j! of the Taylor term lives in the pulse table
        m[j] = p;
      }
    }
    // inclusive segmented scan: lanes of one bin are contiguous (sorted)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int bu = __shfl_up_sync(0xFFFFFFFFu, b, o);
#pragma unroll
      for (int j = 0; j < K_MOM; ++j) {
        const float mu = __shfl_up_sync(0xFFFFFFFFu, m[j], o);
        if (lane >= o && bu == b) m[j] += mu;
      }
    }
    const int bn = __shfl_down_sync(0xFFFFFFFFu, b, 1);
    const bool tail = (b >= 0) && (lane == 31 || bn != b);
    if (tail) {
#pragma unroll
      for (int j = 0; j < K_MOM; ++j) atomicAdd(&M[j * MS + mom_slot(b + sh)], m[j]);
    }
  }
  __syncthreads();
  // convolution: each thread produces 8 consecutive samples n0 .. n0 + 7 of the row,
  // out[n] = sum_j sum_d G_j[d] M_j[bin n - dlo - d].  Taps go in blocks of 8: the 15 moments a
  // block touches are read once into registers (a sliding window) and feed 64 FMAs.  The
  // shift sh puts every window start on a multiple of 8, so the padded slots of the window are
  // fixed offsets and the lanes of a warp read addresses 9 apart: no bank conflicts.
  const int n0 = 8 * threadIdx.x;
  if (n0 < g.ns) {
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.0f;
    const int xs0 = n0 - g.dlo + HALO + sh - 7;  // window start for taps 0..7, a multiple of 8
    const int ntp = (g.ntaps + 7) & ~7;
    for (int j = 0; j < K_MOM; ++j) {
      const float* Mj = M + j * MS;
      const float* Gj = G + j * MAX_TAPS;
      for (int d0 = 0; d0 < ntp; d0 += 8) {
        const float* W = Mj + 9 * ((xs0 - d0) >> 3);
        float w[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) w[k] = W[k + (k >= 8 ? 1 : 0)];
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
          const float gv = Gj[d0 + dd];
#pragma unroll
          for (int r = 0; r < 8; ++r) acc[r] = fmaf(gv, w[r - dd + 7], acc[r]);
        }
      }
    }
    float* out = rf + (size_t)row * g.ns + n0;
    if (n0 + 8 <= g.ns) {
      reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (n0 + r < g.ns) out[r] = acc[r];
    }
  }
}

// standalone arrival list -> packed arrivals
__global__ void k_pack_arrivals(const int32_t* tx, const int32_t* e, const float* tau, const float* a, long long n,
                                int ne, float fs, Arrival* out, uint32_t* n_out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t tq = time_to_tq(tau[i], 0.0f, fs);
    if (tq == 0xFFFFFFFFu) continue;
    cg::coalesced_group grp = cg::coalesced_threads();
    uint32_t s = 0;
    if (grp.thread_rank() == 0) s = atomicAdd(n_out, (uint32_t)grp.size());
    s = grp.shfl(s, 0) + grp.thread_rank();
    out[s] = make_uint4((uint32_t)(tx[i] * ne + e[i]), tq, __float_as_uint(a[i]), (uint32_t)i);
  }
}

// ------------------------------------------------------------------------------------------
size_t row_splat_smem(const SplatGeom& g) {
  return sizeof(float) * (size_t)K_MOM * row_mom_stride(g.ns) + sizeof(uint32_t) * (g.nbins + 1) +
         sizeof(float) * (size_t)K_MOM * MAX_TAPS;
}
int row_splat_threads(const SplatGeom& g) { return ((g.ns + 7) / 8 + 31) / 32 * 32; }

void launch_pulse_table(const SplatGeom& g, float* G, cudaStream_t st) { k_pulse_table<<<1, 128, 0, st>>>(g, G); }

void launch_splat_sort(const SplatGeom& g, const Arrival* arr, const uint32_t* n_arr, uint32_t cap, SplatWork w,
                       int grid, cudaStream_t st) {
  const int nrows = g.nrows;
  cudaMemsetAsync(w.row_cnt, 0, sizeof(uint32_t) * nrows, st);
  k_row_hist<<<grid, 256, sizeof(uint32_t) * nrows, st>>>(arr, n_arr, cap, w.row_cnt, nrows);
  k_row_scan<<<1, 1024, 0, st>>>(w.row_cnt, w.row_off, w.row_cursor, nrows);
  k_row_scatter<<<grid, SC_THREADS, 2 * sizeof(uint32_t) * nrows, st>>>(arr, n_arr, cap, w.row_off, w.row_cursor,
                                                                         w.bucket, nrows);
}
void launch_splat_rows(const SplatGeom& g, SplatWork w, const float* G, float* rf, cudaStream_t st) {
  k_row_splat<<<g.nrows, row_splat_threads(g), row_splat_smem(g), st>>>(g, w.bucket, w.row_off, w.scratch, G, rf);
}

void launch_pack_arrivals(const int32_t* tx, const int32_t* e, const float* tau, const float* a, long long n, int ne,
                          float fs, Arrival* out, uint32_t* n_out, int grid, cudaStream_t st) {
  k_pack_arrivals<<<grid, 256, 0, st>>>(tx, e, tau, a, n, ne, fs, out, n_out);
}

void launch_count_scan(const uint32_t* cnt, uint32_t* off, uint32_t* cursor, int n, cudaStream_t st) {
  k_row_scan<<<1, 1024, 0, st>>>(cnt, off, cursor, n);
}

cudaError_t splat_set_attrs(const SplatGeom& g) {
  return cudaFuncSetAttribute(k_row_splat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_splat_smem(g));
}
cudaError_t row_scatter_set_attrs(int nrows) {
  return cudaFuncSetAttribute(k_row_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * sizeof(uint32_t) * nrows));
}
cudaError_t row_hist_set_attrs(int nrows) {
  return cudaFuncSetAttribute(k_row_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(uint32_t) * nrows));
}

}  // namespace usrt
