// Image formation and its adjoint: delay-and-sum (Eq. das) and its transpose (Eq.
// das_adjoint), the Hilbert envelope along depth, log compression with the dynamic-range clip
// (Sec. 2.3.4), the l1/l2 loss (Eq. weighted_l1_l2_loss) and the envelope/log VJP.
#include <atomic>

#include "image.cuh"

namespace usrt {

// ------------------------------------------------------------------------------------------
// DAS delays (Eq. das), in samples, evaluated in float-float so that the interpolation
// position of a ~4000-sample delay is resolved to ~1e-6 samples:
//   u = (x sin(th) + z cos(th) + W/2 |sin(th)|) fs / c_bf + sqrt((x - x_e)^2 + z^2) fs / c_bf
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ ff ff_div_f(ff a, float b) {
  const float q = __fdiv_rn(a.hi, b);
  const float r = __fmaf_rn(-q, b, a.hi);
  return ff_fast(q, __fdiv_rn(__fadd_rn(r, a.lo), b));
}
// coordinate v0 + (v1 - v0) i / (n - 1)
__device__ __forceinline__ ff grid_coord(float v0, float v1, int i, int n) {
  if (n <= 1) return ff{v0, 0.0f};
  const ff span = ff_div_f(ff_two_sum(v1, -v0), (float)(n - 1));
  const ff off = ff_mulf(span, (float)i);
  return ff_addx(ff{v0, 0.0f}, off);
}
struct DasGeo {
  ff k;       // fs / c_bf
  ff half_w;  // (n_elem - 1) pitch / 2
};
__device__ __forceinline__ DasGeo das_geo(const Acq& q) {
  DasGeo g;
  g.k = ff_divf(q.fs, q.cbf);
  g.half_w = ff_mulf(ff{0.5f * (float)(q.ne - 1), 0.0f}, q.pitch);
  return g;
}
__device__ __forceinline__ ff das_utx(const Acq& q, const DasGeo& g, ff x, ff z, int t) {
  const float st = q.sin_tx[t];
  ff p = ff_mulf(x, st);
  p = ff_addx(p, ff_mul(z, ff{q.cos_tx[t], q.cos_lo[t]}));
  p = ff_addx(p, ff_mulf(g.half_w, fabsf(st)));
  return ff_mul(p, g.k);
}
__device__ __forceinline__ ff das_urx(const Acq& q, const DasGeo& g, ff x, ff z, int e) {
  const ff xe = ff_mulf(ff{(float)e - 0.5f * (float)(q.ne - 1), 0.0f}, q.pitch);
  const ff dx = ff_addx(x, ff{-xe.hi, -xe.lo});
  const ff r2 = ff_addx(ff_mul(dx, dx), ff_mul(z, z));
  return ff_mul(ff_sqrt(r2), g.k);
}
__device__ __forceinline__ float hann_w(int e, int ne) {
  return 0.5f * (1.0f - cospif(2.0f * (float)(e + 1) / (float)(ne + 1)));
}
// Element weight w_e(x, z) of Eq. das: F-number <= 0, the Hann window over the array; F > 0,
// the dynamic receive aperture: cos^2(pi xi / 2) for |xi| < 1, xi = (x_e - x) / a, half-width
// a = max(z / 2F, pitch).  dw_dp (optional): its derivative in the pitch (x_e = p (e - (N_e -
// 1)/2), and a = p where clamped).
__device__ __forceinline__ float apod_w(const Acq& q, const Img& im, float x, float z, int e,
                                        float* dw_dp = nullptr) {
  if (dw_dp) *dw_dp = 0.0f;
  if (!(im.fnum > 0.0f)) return hann_w(e, q.ne);
  const float ce = (float)e - 0.5f * (float)(q.ne - 1);
  const float ad = z / (2.0f * im.fnum);
  const bool clamped = ad < q.pitch;
  const float a = clamped ? q.pitch : ad;
  const float xi = (ce * q.pitch - x) / a;
  if (fabsf(xi) >= 1.0f) return 0.0f;
  const float c = cospif(0.5f * xi);
  if (dw_dp) *dw_dp = -0.5f * PI_F * sinpif(xi) * (ce - (clamped ? xi : 0.0f)) / a;
  return c * c;
}
// The transmit and receive delays of a pixel are each split once into whole samples and a
// fraction in [0, 1) (exactly, from their float-float values); a tap then adds the two parts:
// the one float addition of the fractions rounds by at most 2^-24 samples.
__device__ __forceinline__ float2 das_split(ff u) {
  int i;
  float f;
  ff_floor(u, i, f);
  return make_float2(__int_as_float(i), f);
}
__device__ __forceinline__ void das_tap(float2 a, float2 b, int& i, float& f) {
  f = __fadd_rn(a.y, b.y);
  i = __float_as_int(a.x) + __float_as_int(b.x);
  if (f >= 1.0f) {
    f = __fsub_rn(f, 1.0f);  // exact on [1, 2)
    ++i;
  }
}

// DAS: one pixel per thread; transmit delays staged per pixel in shared memory, the receive
// delay computed once per (pixel, element) and reused for every transmit; channel data read
// through the read-only path (rows stay L2-resident)
constexpr int DAS_THREADS = 256;
__global__ void __launch_bounds__(DAS_THREADS) k_das(Acq q, Img im, const float* __restrict__ rf,
                                                     float* __restrict__ irf) {
  extern __shared__ float2 utx_s[];  // [ntx][DAS_THREADS]
  const int npx = im.nl * im.nd;
  const DasGeo g = das_geo(q);
  for (int base = blockIdx.x * DAS_THREADS; base < npx; base += gridDim.x * DAS_THREADS) {
    const int p = base + threadIdx.x;
    const bool valid = p < npx;
    const int l = valid ? p / im.nd : 0, d = valid ? p - l * im.nd : 0;
    const ff x = grid_coord(im.x0, im.x1, l, im.nl), z = grid_coord(im.z0, im.z1, d, im.nd);
    for (int t = 0; t < q.ntx; ++t) utx_s[t * DAS_THREADS + threadIdx.x] = das_split(das_utx(q, g, x, z, t));
    float acc = 0.0f;
    if (valid) {
      const size_t tstride = (size_t)q.ne * q.ns;  // between one element's rows of two transmits
      for (int e = 0; e < q.ne; ++e) {
        const float2 ur = das_split(das_urx(q, g, x, z, e));
        const float* row = rf + (size_t)e * q.ns;
        float s = 0.0f;
#pragma unroll 4
        for (int t = 0; t < q.ntx; ++t, row += tstride) {
          int i;
          float f;
          das_tap(utx_s[t * DAS_THREADS + threadIdx.x], ur, i, f);
          float a, b;
          if ((unsigned)i < (unsigned)(q.ns - 1)) {  // both samples inside the record
            a = __ldg(&row[i]);
            b = __ldg(&row[i + 1]);
          } else {
            a = (i >= 0 && i < q.ns) ? __ldg(&row[i]) : 0.0f;
            b = (i + 1 >= 0 && i + 1 < q.ns) ? __ldg(&row[i + 1]) : 0.0f;
          }
          s += fmaf(f, b - a, a);
        }
        acc = fmaf(apod_w(q, im, x.hi, z.hi, e), s, acc);
      }
      irf[p] = acc;
    }
  }
}

// ------------------------------------------------------------------------------------------
// DAS with the channel-data windows staged in shared memory by TMA bulk copies.
// A CTA owns a 4-line x 128-depth pixel tile (two pixels per thread).  For every (element,
// transmit) the samples the tile can touch form one contiguous window of the row (the delay
// grows monotonically with depth along each line).  One pipeline stage holds the windows of
// all transmits of one element: an elected thread issues them as cp.async.bulk copies that
// complete on the stage's mbarrier, the CTA interpolates from shared memory, and the stage is
// refilled with a later element once the CTA has moved on.  Every wait is bounded in time:
// on expiry the CTA records the timeout, stops using the staged buffers and reads the channel
// data directly (same result).
// ------------------------------------------------------------------------------------------
constexpr int DT_THREADS = 256, DT_DEPTHS = 128, DT_LINES = 4, DT_PX = 2;
constexpr int DT_SMEM_MAX = 200 * 1024;
constexpr int DT_STAGES = 3;
constexpr int DT_WIN = 512;            // floats per staged window
constexpr int DT_MAX_WINDOWS = 4096;   // (element, transmit) windows per tile
constexpr long long DT_WAIT_CYCLES = 2000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// bounded wait for phase `parity` of a stage's barrier; false on expiry
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > DT_WAIT_CYCLES) return false;
  return true;
}

// plain FP32 delay of pixel (l, d) for (element e, transmit t), in samples
__device__ __forceinline__ float das_delay_f32(const Acq& q, const Img& im, int l, int d, int e, int t) {
  const float k = q.fs / q.cbf;
  const float st = q.sin_tx[t], ct = q.cos_tx[t];
  const float hw = 0.5f * (q.ne - 1) * q.pitch * fabsf(st);
  const float xe = (e - 0.5f * (q.ne - 1)) * q.pitch;
  const float x = im.nl > 1 ? im.x0 + (im.x1 - im.x0) * (float)l / (float)(im.nl - 1) : im.x0;
  const float z = im.nd > 1 ? im.z0 + (im.z1 - im.z0) * (float)d / (float)(im.nd - 1) : im.z0;
  return (x * st + z * ct + hw) * k + sqrtf((x - xe) * (x - xe) + z * z) * k;
}
// sample window [start, start + len) covering delays in [lo, hi], padded by 2 samples and
// aligned to 4 (len 0: nothing in the record; -1: longer than max_len)
__device__ __forceinline__ int2 das_window_of(int ns, float lo, float hi, int max_len) {
  int a = (int)floorf(lo) - 2, b = (int)ceilf(hi) + 3;
  a = max(0, a) & ~3;
  b = min(ns, (b + 3) & ~3);
  if (b <= a) return make_int2(0, 0);
  if (b - a > max_len) return make_int2(a, -1);
  return make_int2(a, b - a);
}
// sample window of (element e, transmit t) for the tile: the delays at the tile's corners (the
// delay grows monotonically with depth along each line)
__device__ int2 das_window(const Acq& q, const Img& im, int l0, int l1, int d0, int d1, int e, int t) {
  float lo = 3.0e38f, hi = -3.0e38f;
  for (int l = l0; l <= l1; ++l)
    for (int r = 0; r < 2; ++r) {
      const float u = das_delay_f32(q, im, l, r ? d1 : d0, e, t);
      lo = fminf(lo, u);
      hi = fmaxf(hi, u);
    }
  return das_window_of(q.ns, lo, hi, DT_WIN);
}

__global__ void __launch_bounds__(DT_THREADS) k_das_tma(Acq q, Img im, const float* __restrict__ rf,
                                                        float* __restrict__ irf, int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const int ntx = q.ntx;
  float* win = reinterpret_cast<float*>(smraw);                                // [DT_STAGES][ntx][DT_WIN]
  uint64_t* bar = reinterpret_cast<uint64_t*>(win + (size_t)DT_STAGES * ntx * DT_WIN);  // [DT_STAGES]
  int2* table = reinterpret_cast<int2*>(bar + DT_STAGES);                     // [ne][ntx]
  float2* utx_s = reinterpret_cast<float2*>(table + q.ne * ntx);              // [ntx][DT_PX][DT_THREADS]
  __shared__ int use_tma;
  const int tiles_d = (im.nd + DT_DEPTHS - 1) / DT_DEPTHS;
  const int l0 = (blockIdx.x / tiles_d) * DT_LINES, d0 = (blockIdx.x % tiles_d) * DT_DEPTHS;
  const int l1 = min(l0 + DT_LINES - 1, im.nl - 1), d1 = min(d0 + DT_DEPTHS - 1, im.nd - 1);
  const int d = d0 + (threadIdx.x % DT_DEPTHS);
  int lp[DT_PX];
  bool valid[DT_PX];
  ff x[DT_PX], z[DT_PX];
  const DasGeo g = das_geo(q);
#pragma unroll
  for (int p = 0; p < DT_PX; ++p) {
    lp[p] = l0 + (threadIdx.x / DT_DEPTHS) + 2 * p;
    valid[p] = lp[p] < im.nl && d < im.nd;
    x[p] = grid_coord(im.x0, im.x1, valid[p] ? lp[p] : l0, im.nl);
    z[p] = grid_coord(im.z0, im.z1, valid[p] ? d : d0, im.nd);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < DT_STAGES; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    use_tma = 1;
  }
  for (int w = threadIdx.x; w < q.ne * ntx; w += blockDim.x)
    table[w] = das_window(q, im, l0, l1, d0, d1, w / ntx, w % ntx);
  for (int t = 0; t < ntx; ++t)
#pragma unroll
    for (int p = 0; p < DT_PX; ++p)
      utx_s[(t * DT_PX + p) * DT_THREADS + threadIdx.x] = das_split(das_utx(q, g, x[p], z[p], t));
  __syncthreads();
  int issued[DT_STAGES];  // uses issued per stage (meaningful in thread 0, the only issuer)
  for (int k = 0; k < DT_STAGES; ++k) issued[k] = 0;
  auto issue = [&](int e) {  // all transmit windows of element e into stage e % DT_STAGES
    if (e >= q.ne) return;
    const int s = e % DT_STAGES;
    ++issued[s];
    uint32_t bytes = 0;
    for (int t = 0; t < ntx; ++t) {
      const int2 b = table[e * ntx + t];
      if (b.y > 0) bytes += (uint32_t)b.y * 4u;
    }
    mbar_arrive_tx(&bar[s], bytes);  // arrival + expected bytes; phase completes when all land
    for (int t = 0; t < ntx; ++t) {
      const int2 b = table[e * ntx + t];
      if (b.y > 0)
        bulk_g2s(win + ((size_t)s * ntx + t) * DT_WIN, rf + ((size_t)t * q.ne + e) * q.ns + b.x, (uint32_t)b.y * 4u,
                 &bar[s]);
    }
  };
  if (threadIdx.x == 0)
    for (int e = 0; e < DT_STAGES; ++e) issue(e);
  float acc[DT_PX];
#pragma unroll
  for (int p = 0; p < DT_PX; ++p) acc[p] = 0.0f;
  for (int e = 0; e < q.ne; ++e) {
    const int s = e % DT_STAGES;
    bool staged = use_tma;
    if (staged && !mbar_wait_bounded(&bar[s], (uint32_t)((e / DT_STAGES) & 1))) {
      use_tma = 0;  // benign race: every writer stores 0
      atomicOr(status, ST_TIMEOUT);
      staged = false;
    }
    float2 ur[DT_PX];
#pragma unroll
    for (int p = 0; p < DT_PX; ++p) ur[p] = das_split(das_urx(q, g, x[p], z[p], e));
    float se[DT_PX];
#pragma unroll
    for (int p = 0; p < DT_PX; ++p) se[p] = 0.0f;
    for (int t = 0; t < ntx; ++t) {
      const int2 b = table[e * ntx + t];
      const float* row = rf + ((size_t)t * q.ne + e) * q.ns;
      const float* sw = win + ((size_t)s * ntx + t) * DT_WIN;
#pragma unroll
      for (int p = 0; p < DT_PX; ++p) {
        int i;
        float f;
        das_tap(utx_s[(t * DT_PX + p) * DT_THREADS + threadIdx.x], ur[p], i, f);
        const int rel = i - b.x;
        float a0, a1;
        if (staged && b.y > 0 && rel >= 0 && rel + 1 < b.y) {
          a0 = sw[rel];
          a1 = sw[rel + 1];
        } else {
          a0 = (i >= 0 && i < q.ns) ? __ldg(&row[i]) : 0.0f;
          a1 = (i + 1 >= 0 && i + 1 < q.ns) ? __ldg(&row[i + 1]) : 0.0f;
        }
        se[p] += fmaf(f, a1 - a0, a0);
      }
    }
#pragma unroll
    for (int p = 0; p < DT_PX; ++p) acc[p] = fmaf(apod_w(q, im, x[p].hi, z[p].hi, e), se[p], acc[p]);
    __syncthreads();  // the CTA is done with stage s
    if (threadIdx.x == 0 && use_tma) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(e + DT_STAGES);
    }
  }
  // drain: every issued copy was waited on above unless a wait expired; then wait (bounded)
  // once more for the last use issued into each stage before the CTA's shared memory goes away
  if (threadIdx.x == 0 && !use_tma)
    for (int s = 0; s < DT_STAGES; ++s)
      if (issued[s] > 0) (void)mbar_wait_bounded(&bar[s], (uint32_t)((issued[s] - 1) & 1));
#pragma unroll
  for (int p = 0; p < DT_PX; ++p)
    if (valid[p]) irf[(size_t)lp[p] * im.nd + d] = acc[p];
}

size_t das_tma_smem(const Acq& q) {
  return sizeof(float) * DT_STAGES * (size_t)q.ntx * DT_WIN + sizeof(uint64_t) * DT_STAGES +
         sizeof(int2) * (size_t)q.ne * q.ntx + sizeof(float2) * (size_t)q.ntx * DT_PX * DT_THREADS;
}

// transposed DAS: every tap scatters w_e (1 - f) g and w_e f g to its two samples
// The transposed DAS accumulates in 64-bit fixed point so that its sums do not depend on the
// order of the atomics (integer addition is associative, and wraps harmlessly in between).  A
// pixel's weighted gradient w_e dL/dI becomes the integer W nearest w_e dL/dI 2^k, with 2^k the
// largest power of two for which max |dL/dI| 2^k < 2^40 and (pixel count) x max |dL/dI| 2^k
// < 2^62; a tap then splits W exactly into its two samples' shares, s1 = floor(W F / 2^23) and
// s0 = W - s1, F the interpolation fraction in units of 2^-23.  The second bound holds every
// entry's sum, since a pixel adds at most |W| to one row (w_e <= 1); the first keeps W F below
// 2^63 and lets the tiled kernel hold a tile's partial sums in two 32-bit words (below).  The
// quantum is 2^-40 of the largest pixel's contribution (2^-43 for 2^22 pixels), far below FP32
// rounding.  max |dL/dI| comes from an integer atomicMax on the float bits of |dL/dI|
// (order-independent too); a non-finite dL/dI makes every entry NaN.
__global__ void k_das_adj_max(const float* __restrict__ gi, int n, unsigned int* maxbits) {
  unsigned int m = 0u;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(gi[i])));  // NaN's bits lie above +inf's
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(maxbits, m);
}
constexpr unsigned int F32_INF_BITS = 0x7F800000u;
constexpr int DAS_ADJ_V_BITS = 40;  // |W| < 2^40 in fixed point
constexpr int DAS_ADJ_F_BITS = 23;  // interpolation fraction in units of 2^-23
static_assert(DAS_ADJ_V_BITS + DAS_ADJ_F_BITS <= 63, "W F fits a signed 64-bit integer");
// the exponent k: max |dL/dI| < 2^e and npx <= 2^c give npx max |dL/dI| < 2^(e + c)
__device__ __forceinline__ int das_adj_kexp(int npx, unsigned int maxbits) {
  if (maxbits == 0u) return 0;
  const int e = ilogbf(__uint_as_float(maxbits)) + 1;
  const int c = 32 - __clz(max(npx - 1, 1));
  return min(DAS_ADJ_V_BITS, 62 - c) - e;
}
// v (|v| < 2^43) rounded to the nearest integer (ties to even, as __float2ll_rn) and split as
// hi 2^22 + lo with lo in [0, 2^22), by FP32 additions only: a float -> 64-bit integer
// conversion runs on the FP64 pipe, a small fraction of the FP32 rate on this part.  Adding
// 2^23 (same sign as v) leaves an integer, exactly when |v| < 2^23 (larger v are integers
// already); 1.5 2^23 added with rounding toward -inf gives floor(v / 2^22) in the float's low
// mantissa bits; the remainder is an exact subtraction.
constexpr int DAS_ADJ_LO_BITS = 22;
__device__ __forceinline__ void das_adj_fixed(float v, int& hi, uint32_t& lo) {
  const float c = copysignf(8388608.0f, v);
  const float vr = fabsf(v) < 8388608.0f ? __fsub_rn(__fadd_rn(v, c), c) : v;
  const float h = __fadd_rd(vr * (1.0f / 4194304.0f), 12582912.0f);  // 1.5 2^23 + floor(vr / 2^22)
  hi = __float_as_int(h) - 0x4B400000;
  const float hf = __fsub_rn(h, 12582912.0f);
  const float lf = __fsub_rn(vr, hf * 4194304.0f);  // in [0, 2^22), exact
  lo = __float_as_uint(__fadd_rn(lf, 8388608.0f)) - 0x4B000000u;
}
__device__ __forceinline__ long long das_adj_fixed64(float v) {
  int hi;
  uint32_t lo;
  das_adj_fixed(v, hi, lo);
  return (long long)hi * (1ll << DAS_ADJ_LO_BITS) + (long long)lo;
}
// the two samples' shares of W at interpolation fraction f in [0, 1): 1 + f rounded to the
// float grid of [1, 2) puts F = round(f 2^23) in the mantissa; s0 + s1 = W exactly
__device__ __forceinline__ void das_adj_shares(long long W, float f, long long& s0, long long& s1) {
  const long long F = (long long)(__float_as_int(__fadd_rn(1.0f, f)) - 0x3F800000);
  s1 = (W * F) >> DAS_ADJ_F_BITS;  // arithmetic shift: floor
  s0 = W - s1;
}
// a share as the tiled kernel's two words: hi 2^22 + lo, lo in [0, 2^22)
__device__ __forceinline__ void das_adj_words(long long v, int& hi, uint32_t& lo) {
  hi = (int)(v >> DAS_ADJ_LO_BITS);
  lo = (uint32_t)v & ((1u << DAS_ADJ_LO_BITS) - 1u);
}
__global__ void k_das_adj_finish(const unsigned long long* __restrict__ acc, long long n, int npx,
                                 const unsigned int* maxbits, float* grf) {
  const unsigned int mb = *maxbits;
  const int k = das_adj_kexp(npx, mb);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    grf[j] = mb >= F32_INF_BITS ? __int_as_float(0x7FC00000) : ldexpf(__ll2float_rn((long long)acc[j]), -k);
}

__global__ void __launch_bounds__(DAS_THREADS) k_das_adj(Acq q, Img im, const float* __restrict__ gi,
                                                         unsigned long long* acc, const unsigned int* maxbits) {
  extern __shared__ float2 utx_s[];
  const int npx = im.nl * im.nd;
  const DasGeo g = das_geo(q);
  const unsigned int mb = *maxbits;
  if (mb >= F32_INF_BITS) return;  // k_das_adj_finish writes NaN
  const int kexp = das_adj_kexp(npx, mb);
  for (int base = blockIdx.x * DAS_THREADS; base < npx; base += gridDim.x * DAS_THREADS) {
    const int p = base + threadIdx.x;
    const bool valid = p < npx;
    const int l = valid ? p / im.nd : 0, d = valid ? p - l * im.nd : 0;
    const ff x = grid_coord(im.x0, im.x1, l, im.nl), z = grid_coord(im.z0, im.z1, d, im.nd);
    for (int t = 0; t < q.ntx; ++t) utx_s[t * DAS_THREADS + threadIdx.x] = das_split(das_utx(q, g, x, z, t));
    const float gv = valid ? gi[p] : 0.0f;
    if (gv != 0.0f) {
      for (int e = 0; e < q.ne; ++e) {
        const float2 ur = das_split(das_urx(q, g, x, z, e));
        const long long W = das_adj_fixed64(ldexpf(apod_w(q, im, x.hi, z.hi, e) * gv, kexp));
        for (int t = 0; t < q.ntx; ++t) {
          int i;
          float f;
          das_tap(utx_s[t * DAS_THREADS + threadIdx.x], ur, i, f);
          long long s0, s1;
          das_adj_shares(W, f, s0, s1);
          unsigned long long* row = acc + ((size_t)t * q.ne + e) * q.ns;
          if (i >= 0 && i < q.ns) atomicAdd(&row[i], (unsigned long long)s0);
          if (i + 1 >= 0 && i + 1 < q.ns) atomicAdd(&row[i + 1], (unsigned long long)s1);
        }
      }
    }
  }
}

// Tiled transposed DAS.  A CTA owns a 16-line x 32-depth pixel tile (one pixel per thread; a
// warp holds 32 consecutive depths of one line).  Element by element, the taps of all transmits
// go into per-transmit sample windows in shared memory, the window of (e, t) being the samples
// the tile's delays can reach (FP32 delays at the tile's corners, padded); then every nonzero
// window entry goes to its row with one global atomic.  A window spans ~100-200 samples against
// the tile's 1024 taps per (e, t), so the global atomics drop several-fold.  A tap outside its
// window (an underestimated window, or one longer than DJ_WIN) goes to the row directly.
// A window entry is two 32-bit words with native shared atomics: a share v (|v| <= |W| < 2^40)
// splits into v >> 22 (signed, |.| <= 2^18) and its low 22 bits (unsigned); at most 512 pixels
// add to one entry, so neither word can overflow (2^27 and 2^31), and the flush rebuilds
// hi 2^22 + lo exactly.  The shares and their sums are those of k_das_adj, so the two kernels
// give the same bits.
constexpr int DJ_THREADS = 512, DJ_LINES = 16, DJ_DEPTHS = 32, DJ_WIN = 192;  // 256: +0.07 ms
constexpr int DJ_SMEM_MAX = 200 * 1024;
static_assert(DJ_DEPTHS == 32 && DJ_LINES == 16 && DJ_THREADS / 32 == DJ_LINES, "a warp is one line's 32 depths");
static_assert(DAS_ADJ_V_BITS - DAS_ADJ_LO_BITS + 9 < 31 && DAS_ADJ_LO_BITS + 9 < 32,
              "the tile's 512 contributions per entry fit both words");
__host__ __device__ constexpr size_t das_adj_tile_smem(int ntx) {
  return (2 * sizeof(uint32_t) * DJ_WIN + sizeof(float2) * DJ_THREADS + 2 * sizeof(int2)) * (size_t)ntx;
}
// windows of element e for all transmits: warp w takes transmits w, w + 16, ...; its lanes
// evaluate the 32 corner delays (16 lines x the two depth ends) and reduce them
__device__ __forceinline__ void dj_windows(const Acq& q, const Img& im, int l0, int l1, int d0, int d1, int e,
                                           int2* out, int lane, int warp) {
  for (int t = warp; t < q.ntx; t += DJ_THREADS / 32) {  // warp-uniform
    const float u = das_delay_f32(q, im, min(l0 + (lane & 15), l1), (lane & 16) ? d1 : d0, e, t);
    float lo = u, hi = u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if (lane == 0) out[t] = das_window_of(q.ns, lo, hi, DJ_WIN);
  }
}
__global__ void __launch_bounds__(DJ_THREADS) k_das_adj_tile(Acq q, Img im, const float* __restrict__ gi,
                                                             unsigned long long* acc, const unsigned int* maxbits) {
  extern __shared__ __align__(16) unsigned char dj_sm[];
  const int ntx = q.ntx;
  int* hi_s = reinterpret_cast<int*>(dj_sm);                                   // [ntx][DJ_WIN]
  uint32_t* lo_s = reinterpret_cast<uint32_t*>(hi_s + (size_t)ntx * DJ_WIN);   // [ntx][DJ_WIN]
  float2* utx_s = reinterpret_cast<float2*>(lo_s + (size_t)ntx * DJ_WIN);      // [ntx][DJ_THREADS]
  int2* win_s = reinterpret_cast<int2*>(utx_s + (size_t)ntx * DJ_THREADS);     // [2][ntx]
  const unsigned int mb = *maxbits;
  if (mb >= F32_INF_BITS) return;  // k_das_adj_finish writes NaN
  const int kexp = das_adj_kexp(im.nl * im.nd, mb);
  const int tiles_d = (im.nd + DJ_DEPTHS - 1) / DJ_DEPTHS;
  const int l0 = (blockIdx.x / tiles_d) * DJ_LINES, d0 = (blockIdx.x % tiles_d) * DJ_DEPTHS;
  const int l1 = min(l0 + DJ_LINES - 1, im.nl - 1), d1 = min(d0 + DJ_DEPTHS - 1, im.nd - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = l0 + warp, d = d0 + lane;
  const bool valid = l < im.nl && d < im.nd;
  const DasGeo g = das_geo(q);
  const ff x = grid_coord(im.x0, im.x1, valid ? l : l0, im.nl);
  const ff z = grid_coord(im.z0, im.z1, valid ? d : d0, im.nd);
  const float gv = valid ? gi[(size_t)l * im.nd + d] : 0.0f;
  for (int t = 0; t < ntx; ++t) utx_s[t * DJ_THREADS + threadIdx.x] = das_split(das_utx(q, g, x, z, t));
  for (int j = threadIdx.x; j < ntx * DJ_WIN; j += DJ_THREADS) {
    hi_s[j] = 0;
    lo_s[j] = 0u;
  }
  dj_windows(q, im, l0, l1, d0, d1, 0, win_s, lane, warp);
  __syncthreads();
  for (int e = 0; e < q.ne; ++e) {
    const int2* wcur = win_s + (e & 1) * ntx;
    // the other buffer was last read by the previous element's flush, before its barrier
    if (e + 1 < q.ne) dj_windows(q, im, l0, l1, d0, d1, e + 1, win_s + ((e + 1) & 1) * ntx, lane, warp);
    const long long W = gv != 0.0f ? das_adj_fixed64(ldexpf(apod_w(q, im, x.hi, z.hi, e) * gv, kexp)) : 0ll;
    if (W != 0ll) {
      const float2 ur = das_split(das_urx(q, g, x, z, e));
#pragma unroll 4
      for (int t = 0; t < ntx; ++t) {
        int i;
        float f;
        das_tap(utx_s[t * DJ_THREADS + threadIdx.x], ur, i, f);
        long long s0, s1;
        das_adj_shares(W, f, s0, s1);
        const int2 w = wcur[t];
        const int rel = i - w.x;
        if (w.y > 0 && rel >= 0 && rel + 1 < w.y) {
          const int j = t * DJ_WIN + rel;
          int h0, h1;
          uint32_t o0, o1;
          das_adj_words(s0, h0, o0);
          das_adj_words(s1, h1, o1);
          atomicAdd(&hi_s[j], h0);
          atomicAdd(&lo_s[j], o0);
          atomicAdd(&hi_s[j + 1], h1);
          atomicAdd(&lo_s[j + 1], o1);
        } else {
          unsigned long long* row = acc + ((size_t)t * q.ne + e) * q.ns;
          if (i >= 0 && i < q.ns) atomicAdd(&row[i], (unsigned long long)s0);
          if (i + 1 >= 0 && i + 1 < q.ns) atomicAdd(&row[i + 1], (unsigned long long)s1);
        }
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ntx * DJ_WIN; j += DJ_THREADS) {
      const int t = j / DJ_WIN, r = j - t * DJ_WIN;
      const int2 w = wcur[t];
      if (r < w.y) {
        const long long v = (long long)hi_s[j] * (1ll << DAS_ADJ_LO_BITS) + (long long)lo_s[j];
        if (v) atomicAdd(acc + ((size_t)t * q.ne + e) * q.ns + w.x + r, (unsigned long long)v);
        hi_s[j] = 0;  // both words, also when they cancel (v = 0 with hi = -lo / 2^22)
        lo_s[j] = 0u;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// shared-memory radix-2 FFT of one line (N = n_depth, power of two)
// ------------------------------------------------------------------------------------------
__device__ void fft_smem(float2* z, const float2* tw, int N, int logN, bool inverse) {
  for (int len = 2, s = 1; len <= N; len <<= 1, ++s) {
    const int half = len >> 1;
    const int step = N >> s;
    for (int b = threadIdx.x; b < (N >> 1); b += blockDim.x) {
      const int grp = b >> (s - 1);
      const int kk = b & (half - 1);
      const int i = grp * len + kk, j = i + half;
      float2 w = tw[kk * step];
      if (inverse) w.y = -w.y;
      const float2 xj = z[j], xi = z[i];
      const float2 t = make_float2(w.x * xj.x - w.y * xj.y, w.x * xj.y + w.y * xj.x);
      z[j] = make_float2(xi.x - t.x, xi.y - t.y);
      z[i] = make_float2(xi.x + t.x, xi.y + t.y);
    }
    __syncthreads();
  }
}

__device__ void twiddles(float2* tw, int N) {
  for (int kk = threadIdx.x; kk < N / 2; kk += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)kk / (float)N, &s, &c);
    tw[kk] = make_float2(c, s);
  }
}

// analytic signal of a real line (already bit-reversed into z): X = FFT(x); X *= h; IFFT / N
__device__ void analytic_smem(float2* z, const float2* tw, int N, int logN) {
  fft_smem(z, tw, N, logN, false);
  for (int kk = threadIdx.x; kk < N; kk += blockDim.x) {
    const float h = (kk == 0 || 2 * kk == N) ? 1.0f : (2 * kk < N ? 2.0f : 0.0f);
    const float sc = h / (float)N;
    z[kk] = make_float2(z[kk].x * sc, z[kk].y * sc);
  }
  __syncthreads();
  // bit-reverse in place for the inverse transform
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - logN));
    if (i < j) {
      const float2 t = z[i];
      z[i] = z[j];
      z[j] = t;
    }
  }
  __syncthreads();
  fft_smem(z, tw, N, logN, true);
}

// envelope of each line: E = |x + i H x|; per-image maximum (value, first index) into a
// packed 64-bit key (float bits << 32 | ~index) with atomicMax
__global__ void k_envelope(Img im, const float* __restrict__ irf, float* env, unsigned long long* emax_key) {
  extern __shared__ float2 sz[];
  const int N = im.nd;
  const int logN = 31 - __clz(N);
  float2* z = sz;
  float2* tw = sz + N;
  twiddles(tw, N);
  __shared__ unsigned long long best;
  if (threadIdx.x == 0) best = 0ull;
  for (int l = blockIdx.x; l < im.nl; l += gridDim.x) {
    const float* x = irf + (size_t)l * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int j = (int)(__brev((unsigned)i) >> (32 - logN));
      z[j] = make_float2(__ldg(&x[i]), 0.0f);
    }
    __syncthreads();
    analytic_smem(z, tw, N, logN);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float e = sqrtf(z[i].x * z[i].x + z[i].y * z[i].y);
      env[(size_t)l * N + i] = e;
      const unsigned long long key =
          ((unsigned long long)__float_as_uint(e) << 32) | (0xFFFFFFFFu - (uint32_t)(l * N + i));
      atomicMax(&best, key);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(emax_key, best);
}

__device__ __forceinline__ float key_emax(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int key_argmax(unsigned long long k) { return (int)(0xFFFFFFFFu - (uint32_t)k); }

// ------------------------------------------------------------------------------------------
// Fused envelope + log compression: one cooperative launch whose blocks keep the envelope of
// their lines in shared memory, meet at one grid-wide barrier once every block has folded its
// maximum into the packed key, then write B = max(20 log10(E / E_max), -DR).  The barrier's
// wait is bounded in time (cooperative launches are co-resident, so it never expires in
// practice); should it expire, the block writes NaN instead of a wrong image and raises
// ST_TIMEOUT in the status word (when one is given).  `extra` arrivals beyond the grid are
// awaited as well: 0 in normal use; 1 injects the fault (an arrival no block makes) so that
// the timeout report can be tested, with the short limit `limit` (clock cycles).
// keyw[0] = packed maximum, keyw[1] = arrival counter (both zeroed before the launch).
// ------------------------------------------------------------------------------------------
constexpr long long BARRIER_CYCLES = 4000000000ll;     // ~2 s at the maximum SM clock
constexpr long long FAULT_BARRIER_CYCLES = 2000000ll;  // ~1 ms: the injected fault's wait

__global__ void k_envlog_fused(Img im, const float* __restrict__ irf, unsigned long long* keyw, float* b, int* status,
                               int extra, long long limit) {
  extern __shared__ float2 sz[];
  const int N = im.nd;
  const int logN = 31 - __clz(N);
  float2* z = sz;
  float2* tw = sz + N;
  float* ev = reinterpret_cast<float*>(tw + N / 2);  // envelopes of this block's lines
  twiddles(tw, N);
  __shared__ unsigned long long best;
  if (threadIdx.x == 0) best = 0ull;
  int j = 0;
  for (int l = blockIdx.x; l < im.nl; l += gridDim.x, ++j) {
    const float* x = irf + (size_t)l * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int r = (int)(__brev((unsigned)i) >> (32 - logN));
      z[r] = make_float2(__ldg(&x[i]), 0.0f);
    }
    __syncthreads();
    analytic_smem(z, tw, N, logN);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float e = sqrtf(z[i].x * z[i].x + z[i].y * z[i].y);
      ev[j * N + i] = e;
      atomicMax(&best, ((unsigned long long)__float_as_uint(e) << 32) | (0xFFFFFFFFu - (uint32_t)(l * N + i)));
    }
    __syncthreads();
  }
  bool ok = true;
  if (threadIdx.x == 0) {
    atomicMax(&keyw[0], best);
    __threadfence();
    atomicAdd(&keyw[1], 1ull);
    const long long t0 = clock64();
    while (atomicAdd(&keyw[1], 0ull) < (unsigned long long)gridDim.x + (unsigned long long)extra) {
      if (clock64() - t0 > limit) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    best = ok ? atomicAdd(&keyw[0], 0ull) : 0xFFFFFFFFFFFFFFFFull;
    if (!ok && status) atomicOr(status, ST_TIMEOUT);
  }
  __syncthreads();
  const unsigned long long kk = best;
  const float emax = __uint_as_float((uint32_t)(kk >> 32));
  const bool valid = kk != 0xFFFFFFFFFFFFFFFFull;
  j = 0;
  for (int l = blockIdx.x; l < im.nl; l += gridDim.x, ++j) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float e = ev[j * N + i];
      float v = -im.dr;
      if (!valid) v = __int_as_float(0x7FC00000);
      else if (emax > 0.0f && e > 0.0f) v = fmaxf(20.0f * log10f(e / emax), -im.dr);
      b[(size_t)l * N + i] = v;
    }
  }
}

// B = max(20 log10(E / E_max), -DR); E = 0 or E_max = 0 -> -DR
__global__ void k_logc(Img im, const float* __restrict__ env, const unsigned long long* emax_key, float* b) {
  const int n = im.nl * im.nd;
  const float emax = key_emax(*emax_key);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float e = env[i];
    float v = -im.dr;
    if (emax > 0.0f && e > 0.0f) v = fmaxf(20.0f * log10f(e / emax), -im.dr);
    b[i] = v;
  }
}

// ------------------------------------------------------------------------------------------
// loss: L = (l1 sum |r| + l2 sum r^2) / N, dL/dB = (l1 sign(r) + 2 l2 r) / N
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float block_sum(float v) {
  __shared__ float ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  }
  __syncthreads();
  return s;  // valid in thread 0
}

__global__ void k_loss_partial(Img im, const float* __restrict__ b, const float* __restrict__ bref, float* gb,
                               float* part) {
  const int n = im.nl * im.nd;
  const float inv = 1.0f / (float)n;
  float s = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float r = b[i] - bref[i];
    s += im.l1 * fabsf(r) + im.l2 * r * r;
    if (gb) gb[i] = (im.l1 * (r > 0.0f ? 1.0f : (r < 0.0f ? -1.0f : 0.0f)) + 2.0f * im.l2 * r) * inv;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_final(const float* part, int n, float scale, float* out) {
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[0] = s * scale;
}

// sum over unclipped pixels of dL/dB (the E_max share of the log-compression derivative)
__global__ void k_live_sum(Img im, const float* __restrict__ env, const unsigned long long* emax_key,
                           const float* __restrict__ gb, float* part) {
  const int n = im.nl * im.nd;
  const float emax = key_emax(*emax_key);
  float s = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float e = env[i];
    if (emax > 0.0f && e > 0.0f && 20.0f * log10f(e / emax) > -im.dr) s += gb[i];
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// per line: g_E = dL/dB * (20/ln10) / E on unclipped pixels, minus (20/ln10) S / E_max at the
// argmax; then g_x = (x/E) g_E - H((y/E) g_E) (the Hilbert matrix is skew-symmetric)
__global__ void k_envlog_vjp(Img im, const float* __restrict__ irf, const float* __restrict__ gb,
                             const unsigned long long* emax_key, const float* live_sum, float* gi) {
  extern __shared__ float2 sz[];
  const int N = im.nd;
  const int logN = 31 - __clz(N);
  float2* z = sz;
  float2* v = sz + N;
  float2* tw = sz + 2 * N;
  twiddles(tw, N);
  const float emax = key_emax(*emax_key);
  const int am = key_argmax(*emax_key);
  const float c = 8.685889638065036f;  // 20 / ln(10)
  const float S = *live_sum;
  for (int l = blockIdx.x; l < im.nl; l += gridDim.x) {
    const float* x = irf + (size_t)l * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const int j = (int)(__brev((unsigned)i) >> (32 - logN));
      z[j] = make_float2(__ldg(&x[i]), 0.0f);
    }
    __syncthreads();
    analytic_smem(z, tw, N, logN);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const float xi = __ldg(&x[i]), yi = z[i].y;
      const float e = sqrtf(xi * xi + yi * yi);
      const int p = l * N + i;
      float ge = 0.0f;
      if (emax > 0.0f && e > 0.0f && 20.0f * log10f(e / emax) > -im.dr) ge = gb[p] * c / e;
      if (p == am && emax > 0.0f) ge -= c * S / emax;
      const float vv = e > 0.0f ? yi / e * ge : 0.0f;
      z[i] = make_float2(e > 0.0f ? xi / e * ge : 0.0f, 0.0f);  // keep (x/E) g_E in z.x
      const int j = (int)(__brev((unsigned)i) >> (32 - logN));
      v[j] = make_float2(vv, 0.0f);
    }
    __syncthreads();
    analytic_smem(v, tw, N, logN);
    for (int i = threadIdx.x; i < N; i += blockDim.x) gi[(size_t)l * N + i] = z[i].x - v[i].y;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// DAS derivative in the acquisition parameters (Eq. das with the delays of Sec. 2.3.1),
// contracted with an image gradient gi, the RF held fixed:
//   out[0] = sum_p gi(p) dI(p)/dc_bf,  out[1] = .../dpitch,  out[2 + t] = .../dth_t.
// A tap at u = i + f has dI/du = w_e (rf[i + 1] - rf[i]) (the slope of its interpolation
// interval); du/dc_bf = -u / c_bf; du/dpitch = (W/2 |sin th| / p - (x - x_e) / r (e - (N_e -
// 1)/2)) fs / c_bf (transmit aperture and receive distance r); only the transmit delay holds
// th_t: du/dth = (x cos th - z sin th + W/2 sgn(sin th) cos th) fs / c_bf, sgn(0) = 0.  So a
// pixel needs, per transmit, S1 = sum_e w_e slope, and over all its taps sum w_e slope u and
// sum w_e slope du/dp.  One pixel per thread (one pass, no grid stride), elements outer and
// transmits inner as in k_das, so the receive delay, its pitch derivative and the element
// weight are evaluated once per (pixel, element); the transmit delays and the per-transmit
// sums S1 sit in shared memory in thread-major rows; the other two sums are per-pixel scalars
// (their transmit weights are known before the sum).  Each block writes one
// row of 2 + ntx sums, reduced in a fixed order (deterministic).
// ------------------------------------------------------------------------------------------
constexpr int DA_THREADS = 256;
__host__ __device__ constexpr size_t das_acq_smem(int ntx) { return (sizeof(float2) + sizeof(float)) * DA_THREADS * ntx; }
__global__ void __launch_bounds__(DA_THREADS) k_das_acq(Acq q, Img im, const float* __restrict__ rf,
                                                        const float* __restrict__ gi, float* part) {
  extern __shared__ float2 da_sm[];
  float2* ut_s = da_sm;                                              // [ntx][DA_THREADS]
  float* s1_s = reinterpret_cast<float*>(da_sm + q.ntx * DA_THREADS);  // [ntx][DA_THREADS]
  const int npx = im.nl * im.nd;
  const DasGeo g = das_geo(q);
  const int p = blockIdx.x * DA_THREADS + threadIdx.x;
  const bool valid = p < npx;
  const int l = valid ? p / im.nd : 0, d = valid ? p - l * im.nd : 0;
  const ff x = grid_coord(im.x0, im.x1, l, im.nl), z = grid_coord(im.z0, im.z1, d, im.nd);
  const float gp = valid ? __ldg(&gi[p]) : 0.0f;
  const float kfs = q.fs / q.cbf, hn = 0.5f * (float)(q.ne - 1), hw = hn * q.pitch;
  for (int t = 0; t < q.ntx; ++t) {
    ut_s[t * DA_THREADS + threadIdx.x] = das_split(das_utx(q, g, x, z, t));
    s1_s[t * DA_THREADS + threadIdx.x] = 0.0f;
  }
  float c0 = 0.0f, cp = 0.0f;  // sum slope u; sum slope du/dp
  if (gp != 0.0f) {
    for (int e = 0; e < q.ne; ++e) {
      const float2 ur = das_split(das_urx(q, g, x, z, e));
      float dwp;
      const float w = apod_w(q, im, x.hi, z.hi, e, &dwp);
      const float ce = (float)e - hn;
      const float dx = x.hi - ce * q.pitch;
      const float drp = -dx * ce * kfs / sqrtf(fmaf(dx, dx, z.hi * z.hi));  // d(receive delay)/dp
      for (int t = 0; t < q.ntx; ++t) {
        int i;
        float f;
        das_tap(ut_s[t * DA_THREADS + threadIdx.x], ur, i, f);
        const float* row = rf + ((size_t)t * q.ne + e) * q.ns;
        const float a = (i >= 0 && i < q.ns) ? __ldg(&row[i]) : 0.0f;
        const float b = (i + 1 >= 0 && i + 1 < q.ns) ? __ldg(&row[i + 1]) : 0.0f;
        const float sl = w * (b - a);
        s1_s[t * DA_THREADS + threadIdx.x] += sl;
        c0 = fmaf(sl, (float)i + f, c0);
        cp = fmaf(sl, fmaf(hn * fabsf(q.sin_tx[t]), kfs, drp), cp);
        cp = fmaf(dwp, fmaf(f, b - a, a), cp);  // the weight's own pitch term (dynamic aperture)
      }
    }
  }
  float* out = part + (size_t)blockIdx.x * (2 + q.ntx);
  for (int t = 0; t < q.ntx; ++t) {
    const float st = q.sin_tx[t], ct = q.cos_tx[t];
    const float sg = st > 0.0f ? 1.0f : (st < 0.0f ? -1.0f : 0.0f);
    const float du = (x.hi * ct - z.hi * st + hw * sg * ct) * kfs;
    const float v = block_sum(gp * du * s1_s[t * DA_THREADS + threadIdx.x]);
    if (threadIdx.x == 0) out[2 + t] = v;
  }
  const float v0 = block_sum(gp * c0);
  if (threadIdx.x == 0) out[0] = -v0 / q.cbf;
  const float v1 = block_sum(gp * cp);
  if (threadIdx.x == 0) out[1] = v1;
}

// ------------------------------------------------------------------------------------------
void launch_das(const Acq& q, const Img& im, const float* rf, float* irf, int grid, cudaStream_t st, int* status) {
  if (status && q.ne * q.ntx <= DT_MAX_WINDOWS && das_tma_smem(q) <= (size_t)DT_SMEM_MAX &&
      ((uintptr_t)rf & 15u) == 0) {
    const int tiles = ((im.nl + DT_LINES - 1) / DT_LINES) * ((im.nd + DT_DEPTHS - 1) / DT_DEPTHS);
    k_das_tma<<<tiles, DT_THREADS, das_tma_smem(q), st>>>(q, im, rf, irf, status);
    return;
  }
  k_das<<<grid, DAS_THREADS, sizeof(float2) * DAS_THREADS * q.ntx, st>>>(q, im, rf, irf);
}
int das_acq_blocks(const Img& im) { return (im.nl * im.nd + DA_THREADS - 1) / DA_THREADS; }
void launch_das_acq(const Acq& q, const Img& im, const float* rf, const float* gi, float* part, cudaStream_t st) {
  k_das_acq<<<das_acq_blocks(im), DA_THREADS, das_acq_smem(q.ntx), st>>>(q, im, rf, gi, part);
}
static std::atomic<int> g_das_adj_tiled{1};
void launch_das_adj(const Acq& q, const Img& im, const float* gi, float* grf, int grid, cudaStream_t st,
                    unsigned long long* acc, unsigned int* maxbits) {
  const long long n = (long long)q.ntx * q.ne * q.ns;
  const int npx = im.nl * im.nd;
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)n, st);
  cudaMemsetAsync(maxbits, 0, sizeof(unsigned int), st);
  k_das_adj_max<<<min(grid, (npx + 255) / 256), 256, 0, st>>>(gi, npx, maxbits);
  if (das_adj_tile_smem(q.ntx) <= (size_t)DJ_SMEM_MAX && g_das_adj_tiled.load()) {
    const int tiles = ((im.nl + DJ_LINES - 1) / DJ_LINES) * ((im.nd + DJ_DEPTHS - 1) / DJ_DEPTHS);
    k_das_adj_tile<<<tiles, DJ_THREADS, das_adj_tile_smem(q.ntx), st>>>(q, im, gi, acc, maxbits);
  } else {
    k_das_adj<<<grid, DAS_THREADS, sizeof(float2) * DAS_THREADS * q.ntx, st>>>(q, im, gi, acc, maxbits);
  }
  k_das_adj_finish<<<grid, 256, 0, st>>>(acc, n, npx, maxbits, grf);
}
constexpr int FUSED_SMEM_MAX = 200 * 1024;
static std::atomic<int> g_envlog_fused{1};

}  // namespace usrt

extern "C" void us_set_envlog_fused(int enable) { usrt::g_envlog_fused.store(enable ? 1 : 0); }
extern "C" void us_set_das_adj_tiled(int enable) { usrt::g_das_adj_tiled.store(enable ? 1 : 0); }

namespace usrt {

int launch_envlog(const Img& im, const float* irf, float* env, unsigned long long* key, float* bmode, int grid,
                  cudaStream_t st, int* status, int fault_barrier, cudaError_t* launch_err) {
  // every launch reports its own status: no cudaGetLastError, which would also take (and
  // clear) an error left by unrelated earlier work
  cudaError_t err = cudaMemsetAsync(key, 0, 2 * sizeof(unsigned long long), st);
  int launched = 0;
  if (bmode && g_envlog_fused.load() && err == cudaSuccess) {
    // fused path: every line's envelope stays in the shared memory of a co-resident block
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t base = sizeof(float2) * (size_t)(im.nd + im.nd / 2);
    for (int lpb = 1; lpb <= 8; ++lpb) {
      const size_t smem = base + sizeof(float) * (size_t)lpb * im.nd;
      if (smem > (size_t)FUSED_SMEM_MAX) break;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_envlog_fused, 256, smem) != cudaSuccess) break;
      const int nb = (im.nl + lpb - 1) / lpb;
      if (per_sm > 0 && nb <= per_sm * sms) {
        int extra = fault_barrier ? 1 : 0;
        long long limit = fault_barrier ? FAULT_BARRIER_CYCLES : BARRIER_CYCLES;
        void* args[] = {(void*)&im, (void*)&irf, (void*)&key, (void*)&bmode, (void*)&status, (void*)&extra,
                        (void*)&limit};
        if (cudaLaunchCooperativeKernel((const void*)k_envlog_fused, dim3(nb), dim3(256), args, smem, st) ==
            cudaSuccess) {
          if (launch_err) *launch_err = cudaSuccess;
          return 1;
        }
        cudaGetLastError();  // the refused cooperative launch: fall back to two kernels
        break;
      }
    }
  }
  const int nb = min(im.nl, grid);
  if (err == cudaSuccess) {
    void* args[] = {(void*)&im, (void*)&irf, (void*)&env, (void*)&key};
    err = cudaLaunchKernel((const void*)k_envelope, dim3(nb), dim3(256), args,
                           sizeof(float2) * (size_t)(im.nd + im.nd / 2), st);
    launched += err == cudaSuccess;
  }
  if (bmode && err == cudaSuccess) {
    const unsigned long long* ckey = key;
    void* args[] = {(void*)&im, (void*)&env, (void*)&ckey, (void*)&bmode};
    err = cudaLaunchKernel((const void*)k_logc, dim3(grid), dim3(256), args, 0, st);
    launched += err == cudaSuccess;
  }
  if (launch_err) *launch_err = err;
  return launched;
}
void launch_loss(const Img& im, const float* b, const float* bref, float* gb, float* part, int nparts, float* loss,
                 cudaStream_t st) {
  k_loss_partial<<<nparts, 256, 0, st>>>(im, b, bref, gb, part);
  k_sum_final<<<1, 1024, 0, st>>>(part, nparts, 1.0f / (float)(im.nl * im.nd), loss);
}
void launch_envlog_vjp(const Img& im, const float* irf, const float* gb, float* env, unsigned long long* key,
                       float* part, int nparts, float* live_sum, float* gi, int grid, cudaStream_t st) {
  launch_envlog(im, irf, env, key, nullptr, grid, st);
  k_live_sum<<<nparts, 256, 0, st>>>(im, env, key, gb, part);
  k_sum_final<<<1, 1024, 0, st>>>(part, nparts, 1.0f, live_sum);
  const int nb = min(im.nl, grid);
  k_envlog_vjp<<<nb, 256, sizeof(float2) * (size_t)(2 * im.nd + im.nd / 2), st>>>(im, irf, gb, key, live_sum, gi);
}
cudaError_t image_set_attrs(int nd) {
  cudaError_t ea = cudaFuncSetAttribute(k_das_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, DT_SMEM_MAX);
  if (ea != cudaSuccess) return ea;
  cudaError_t e0 = cudaFuncSetAttribute(k_envlog_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, FUSED_SMEM_MAX);
  if (e0 != cudaSuccess) return e0;
  cudaError_t e = cudaFuncSetAttribute(k_das, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float2) * DAS_THREADS * MAX_TX));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_das_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float2) * DAS_THREADS * MAX_TX));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_das_adj_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, DJ_SMEM_MAX);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_das_acq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)das_acq_smem(MAX_TX));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_envelope, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float2) * (size_t)(nd + nd / 2)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_envlog_vjp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float2) * (size_t)(2 * nd + nd / 2)));
}

}  // namespace usrt
