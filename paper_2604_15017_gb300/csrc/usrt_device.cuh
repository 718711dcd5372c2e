// Device-side building blocks shared by the usrt kernels: Philox4x32-10, launch parameters,
// scene layout, float-float time accumulation, the interface event and the pulse.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace usrt {

constexpr int MAX_MEDIA = 32;
constexpr int MAX_TX = 64;
constexpr int MAX_ELEM = 256;
constexpr int MAX_KMAX = 15;
constexpr int K_MOM = 8;         // Taylor moments of the sort-based splat
constexpr int MAX_TAPS = 96;     // pulse support in samples (both sides)
constexpr int MAX_XINGS = 32;    // interface crossings of one secondary ray
constexpr float T_MIN = 1e-7f;   // minimum hit distance [m]: no re-hit of the surface just left
constexpr float PI_F = 3.14159265358979f;
// amplitude attenuation per (dB/cm/MHz * Hz * m): ln(10)/20 * 1e-6 * 100
constexpr float KAPPA_F = 1.1512925464970229e-05f;
// arrival times are carried as fixed point in samples: tq = (u + TQ_OFFSET) * 2^TQ_FRAC
constexpr int TQ_FRAC = 18;
constexpr int TQ_OFFSET = 64;

// primitive / event codes (record word): id bits 0-19, class 20-21, choice 22-23, aux 24-31
enum : uint32_t { CLS_NONE = 0, CLS_XDCR = 1, CLS_TRI = 2, CLS_SCAT = 3 };
enum : uint32_t { CH_NONE = 0, CH_REFLECT = 1, CH_TRANSMIT = 2, CH_TIR = 3 };
__host__ __device__ __forceinline__ uint32_t prim_code(uint32_t cls, uint32_t id) { return (cls << 20) | id; }
__host__ __device__ __forceinline__ uint32_t code_cls(uint32_t c) { return (c >> 20) & 3u; }
__host__ __device__ __forceinline__ uint32_t code_id(uint32_t c) { return c & 0xFFFFFu; }

// device status word bits
enum : int { ST_OVERFLOW = 1, ST_TIMEOUT = 2 };

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = c.x * 0xD2511F53u, hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u, hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------------------------------------
// Launch parameters (passed by value)
// ------------------------------------------------------------------------------------------
struct Media {
  int M;
  float c[MAX_MEDIA], rho[MAX_MEDIA], al[MAX_MEDIA];
  float As, f0;
  float rough[MAX_MEDIA];  // GGX roughness of the interfaces bounding each medium (0: smooth)
  int has_rough;           // theta carries the roughness values (4M + 2 parameters)
};
// parameters in theta: 3M + 2, and M roughness values after them in a rough scene
__host__ __device__ __forceinline__ int n_theta(const Media& m) { return 3 * m.M + 2 + (m.has_rough ? m.M : 0); }

struct Acq {
  int ne, ntx, ns, kmax, nr, n_emit, tx_elem, split_mode;
  int rough_nee;  // secondary rays at rough interface events too
  float pitch, hel, fs, bw, alpha_m, alpha_c, cbf, split_q;
  uint32_t stream, key0, key1;
  long long rays_per_tx;
  float sin_tx[MAX_TX], cos_tx[MAX_TX];
  float cos_lo[MAX_TX];  // cos(angle) - cos_tx (float-float steering cosine for the delays)
};

struct Img {
  int nl, nd;
  float x0, x1, z0, z1, dr, l1, l2;
  float fnum;  // receive F-number of the dynamic aperture (<= 0: the whole array)
};

// device-resident scene: triangle BVH2 (nodes of 4 float4, triangles in leaf order, 3 float4
// each) and the uniform grid over the scatterer spheres
struct SceneDev {
  const float4* tri_nrm;     // by triangle id: (unit normal, bits(m_front | m_back << 16))
  const float4* tri_v0;      // by triangle id: (v0, 0)
  const float4* tri_e1;      // by triangle id: (v1 - v0, |(v1 - v0) x (v2 - v0)|)  (shape adjoint)
  const float4* tri_e2;      // by triangle id: (v2 - v0, 0)
  const float4* scat;        // by scatterer id: (p, amplitude)
  const float4* nodes_t;     // triangle BVH2: n0=(c0.lo.x,c0.hi.x,c0.lo.y,c0.hi.y) n1=(same, c1)
                             // n2=(c0 z, c1 z) n3=int4(child0, child1, count0, count1)
  const float4* prims_t;     // triangles in leaf order: (v0, code) (e1, -) (e2, -)
  const float4* nodes4;      // the triangle tree as a 4-wide BVH (8 float4 per node, same leaves)
  const uint32_t* cell;        // scatterer grid, per cell (z * gny + y) * gnx + x: first entry << 8 | count
  const float4* cell_sph;      // per (cell, sphere): (centre, bits(code))
  const float4* cell2;         // per cell its first two entries; code 0: empty, bit 31: more follow
  float3 glo;                  // grid origin and cell edge
  float gh;
  int gnx, gny, gnz;
  int n_tris, n_scat;
  float rs2;
};

// ------------------------------------------------------------------------------------------
// small vector helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 xyz(float4 v) { return f3(v.x, v.y, v.z); }

// ------------------------------------------------------------------------------------------
// float-float accumulation of the path time (error-free TwoSum, Knuth)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// ------------------------------------------------------------------------------------------
// float-float arithmetic (Dekker / Knuth error-free transformations) for delays that must be
// resolved to ~1e-6 samples out of ~4000
// ------------------------------------------------------------------------------------------
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
__device__ __forceinline__ ff ff_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_addx(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return ff_fast(p, __fmaf_rn(a.lo, b, e));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return ff_fast(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.0f)) return ff{0.0f, 0.0f};
  const float s = sqrtf(a.hi);
  const float r = __fmaf_rn(-s, s, a.hi);  // exact residual
  return ff_fast(s, __fdiv_rn(__fadd_rn(r, a.lo), __fmul_rn(2.0f, s)));
}
__device__ __forceinline__ ff ff_divf(float a, float b) {  // a / b
  const float q = __fdiv_rn(a, b);
  const float r = __fmaf_rn(-q, b, a);
  return ff_fast(q, __fdiv_rn(r, b));
}
// split x = i + f, 0 <= f < 1, from a float-float
__device__ __forceinline__ void ff_floor(ff u, int& i, float& f) {
  const float fl = floorf(u.hi);
  float fr = __fadd_rn(__fsub_rn(u.hi, fl), u.lo);
  int ii = (int)fl;
  if (fr < 0.0f) {
    fr = __fadd_rn(fr, 1.0f);
    ii -= 1;
  } else if (fr >= 1.0f) {
    fr = __fsub_rn(fr, 1.0f);
    ii += 1;
  }
  if (fr >= 1.0f) fr = 0.99999994f;
  i = ii;
  f = fr;
}

// time (hi, lo) [s] -> fixed-point samples tq, or 0xFFFFFFFF outside [-TQ_OFFSET, 2^(32-TQ_FRAC) - TQ_OFFSET)
__device__ __forceinline__ uint32_t time_to_tq(float hi, float lo, float fs) {
  const float u = __fmul_rn(hi, fs);
  const float e = __fmaf_rn(hi, fs, -u);  // exact product error
  const float fl = floorf(u);
  const float frac = (u - fl) + (e + lo * fs);  // u - fl is exact
  const float base = fl + (float)TQ_OFFSET;
  if (!(base >= 0.0f) || base >= (float)(1u << (32 - TQ_FRAC)) - 2.0f) return 0xFFFFFFFFu;
  const long long q = (long long)base * (1ll << TQ_FRAC) + __float2ll_rn(frac * (float)(1 << TQ_FRAC));
  if (q < 0 || q >= 0xFFFFFFFFll) return 0xFFFFFFFFu;
  return (uint32_t)q;
}

// receive directivity, Eq. cutoff; cosd = cos of the angle to the element normal
__device__ __forceinline__ float f_rx(float cosd, float am, float ac) {
  const float th = acosf(fminf(1.0f, fmaxf(-1.0f, cosd)));
  if (th <= am) return 1.0f;
  if (th > ac) return 0.0f;
  return (ac - th) / (ac - am);
}

// ------------------------------------------------------------------------------------------
// Interface event (Sec. 2.3.2): w incident, nin unit normal back into medium 1.
// R = (Z2 ci - Z1 ct)/(Z2 ci + Z1 ct), T = 2 Z2 ci/(Z2 ci + Z1 ct); Snell with sound speeds.
// ------------------------------------------------------------------------------------------
struct Iface {
  bool tir;
  float ci, ct, r, R, T;
};
__device__ __forceinline__ Iface iface(float3 w, float3 nin, float c1, float c2, float rho1, float rho2) {
  Iface f;
  f.ci = -dot3(w, nin);
  f.r = c2 / c1;
  const float si2 = fmaxf(0.0f, 1.0f - f.ci * f.ci);
  const float st2 = f.r * f.r * si2;
  f.tir = st2 >= 1.0f;
  if (f.tir) {
    f.ct = 0.0f;
    f.R = 1.0f;
    f.T = 0.0f;
    return f;
  }
  f.ct = sqrtf(1.0f - st2);
  const float A = rho2 * c2 * f.ci, B = rho1 * c1 * f.ct;
  const float inv = 1.0f / (A + B);
  f.R = (A - B) * inv;
  f.T = 2.0f * A * inv;
  return f;
}

// ------------------------------------------------------------------------------------------
// Rough interfaces (Sec. 2.3.2, Eq. GGX_PDF): a microfacet normal h drawn with density
// D(h) (h.n) around the macro normal n, D the GGX distribution of roughness alpha.  Inverting
// its cumulative distribution: tan(theta_h) = alpha s with s = sqrt(u / (1 - u)), and a uniform
// azimuth phi about n, in the tangent frame of Duff et al. (2017, branch-free orthonormal basis).
// The event reflects or refracts about h; the amplitude takes the microfacet weight of this
// sampling, |w_i.h| G1(w_i) G1(w_o) / (|w_i.n| |h.n|) with the Smith masking of GGX,
// G1(v) = 2 |v.n| / (|v.n| + sqrt(alpha^2 + (1 - alpha^2) (v.n)^2)).
// ------------------------------------------------------------------------------------------
struct GgxSample {
  float3 h;         // microfacet normal
  float3 b;         // unit tangent direction of the tilt (h = cos(theta) n + sin(theta) b)
  float s;          // tan(theta_h) / alpha
  float cphi, sphi;  // azimuth: b = cos(phi) t1 + sin(phi) t2
};
__device__ __forceinline__ GgxSample ggx_sample(float3 n, float alpha, float u2, float u3) {
  const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sg + n.z);
  const float bb = n.x * n.y * a;
  const float3 t1 = make_float3(1.0f + sg * n.x * n.x * a, sg * bb, -sg * n.x);
  const float3 t2 = make_float3(bb, sg + n.y * n.y * a, -n.y);
  float sp, cp;
  sincospif(2.0f * u3, &sp, &cp);
  GgxSample g;
  g.cphi = cp;
  g.sphi = sp;
  g.b = make_float3(cp * t1.x + sp * t2.x, cp * t1.y + sp * t2.y, cp * t1.z + sp * t2.z);
  g.s = sqrtf(u2 / (1.0f - u2));
  const float tn = alpha * g.s;
  const float ct = rsqrtf(1.0f + tn * tn), st = tn * ct;
  g.h = make_float3(ct * n.x + st * g.b.x, ct * n.y + st * g.b.y, ct * n.z + st * g.b.z);
  return g;
}
// adjoint of the macro normal n from the adjoint hb of h = ct n + st (cos(phi) t1 + sin(phi) t2),
// t1 and t2 the tangent frame of ggx_sample (its sign choice held fixed)
__device__ __forceinline__ float3 ggx_normal_adjoint(float3 n, const GgxSample& g, float alpha, float3 hb) {
  const float tn = alpha * g.s, ct = rsqrtf(1.0f + tn * tn), st = tn * ct;
  const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sg + n.z);
  const float3 t1b = make_float3(st * g.cphi * hb.x, st * g.cphi * hb.y, st * g.cphi * hb.z);
  const float3 t2b = make_float3(st * g.sphi * hb.x, st * g.sphi * hb.y, st * g.sphi * hb.z);
  // t1 = (1 + sg nx^2 a, sg nx ny a, -sg nx), t2 = (nx ny a, sg + ny^2 a, -ny), a = -1 / (sg + nz)
  const float a2 = a * a;
  float3 nb;
  nb.x = ct * hb.x + t1b.x * 2.0f * sg * n.x * a + t1b.y * sg * n.y * a - t1b.z * sg + t2b.x * n.y * a;
  nb.y = ct * hb.y + t1b.y * sg * n.x * a + t2b.x * n.x * a + t2b.y * 2.0f * n.y * a - t2b.z;
  nb.z = ct * hb.z + (t1b.x * sg * n.x * n.x + t1b.y * sg * n.x * n.y + t2b.x * n.x * n.y + t2b.y * n.y * n.y) * a2;
  return nb;
}
__device__ __forceinline__ float smith_g1(float vn, float alpha) {
  const float c = fabsf(vn);
  return 2.0f * c / (c + sqrtf(fmaf(1.0f - alpha * alpha, c * c, alpha * alpha)));
}

// GGX distribution of microfacet normals, Eq. GGX_PDF
__device__ __forceinline__ float ggx_d(float nh, float alpha) {
  const float a2 = alpha * alpha;
  const float k = fmaf(nh * nh, a2 - 1.0f, 1.0f);
  return a2 / (PI_F * k * k);
}

// Forward-mode dual number with N derivative slots (the local derivatives of the rough-event
// secondary ray's BSDF factor in the adjoint), and the few operations that factor needs; the
// same code instantiated with float is the forward pass's.
template <int N>
struct DualN {
  float v;
  float d[N];
  __device__ __forceinline__ DualN() {}
  __device__ __forceinline__ DualN(float x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0f;
  }
};
template <int N>
__device__ __forceinline__ DualN<N> dual_const(float v) {
  DualN<N> r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = 0.0f;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> dual_var(float v, int slot) {
  DualN<N> r = dual_const<N>(v);
  r.d[slot] = 1.0f;
  return r;
}
__device__ __forceinline__ float dval(float x) { return x; }
template <int N>
__device__ __forceinline__ float dval(const DualN<N>& x) { return x.v; }
template <int N>
__device__ __forceinline__ DualN<N> operator+(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator-(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(const DualN<N>& a, const DualN<N>& b) {
  DualN<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator*(const DualN<N>& a, float b) {
  DualN<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> operator/(const DualN<N>& a, const DualN<N>& b) {
  const float ib = 1.0f / b.v, q = a.v * ib;
  DualN<N> r;
  r.v = q;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - q * b.d[i]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ DualN<N> dsqrt(const DualN<N>& a) {
  const float s = sqrtf(a.v), k = s > 0.0f ? 0.5f / s : 0.0f;
  DualN<N> r;
  r.v = s;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k;
  return r;
}
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
template <class T>
__device__ __forceinline__ T dabs(const T& a) {
  return dval(a) < 0.0f ? a * -1.0f : a;
}
template <class T>
struct V3 {
  T x, y, z;
};
template <class T>
__device__ __forceinline__ V3<T> v3(const T& x, const T& y, const T& z) {
  V3<T> r;
  r.x = x;
  r.y = y;
  r.z = z;
  return r;
}
template <class T>
__device__ __forceinline__ T vdot(const V3<T>& a, const V3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class T>
__device__ __forceinline__ V3<T> vscale(const V3<T>& a, const T& k) {
  return v3(a.x * k, a.y * k, a.z * k);
}
template <class T>
__device__ __forceinline__ V3<T> vadd(const V3<T>& a, const V3<T>& b) {
  return v3(a.x + b.x, a.y + b.y, a.z + b.z);
}

// Secondary ray from a rough interface event (Sec. 2.3.3) toward unit direction o (distance^2
// r2 to the element's centre): the microfacet BSDF's amplitude per solid angle toward o for the
// incident direction w (i = -w; nin the macro normal on the incident side), with the half vector
// of reflection (o on the incident side) or of refraction (Snell with sound speeds),
// g = D(h) G1(i) G1(o) C(h) |i.h| |dh/do| / |i.n| (C the facet's pressure reflection or
// transmission coefficient; |dh/do| = 1 / (4 |o.h|), or |o.h| / (c2^2 (i.h / c1 + o.h / c2)^2)),
// combined with the primary's own direct hits by the balance heuristic: the ray carries
// g / (p_nee + p_bsdf), p_nee = 1 / (N_e Omega) the density of a uniform element and direction
// within it (Omega its face's solid angle), p_bsdf = D(h) (h.n) |dh/do| P(choice) the primary's.
// Returns false when nothing is sent that way; else fac = that weight / N_e (the segment's
// shading multiplies by N_e) and whether o reflects (the segment starts in m1) or refracts (m2).
// T is float, or a DualN carrying the derivatives in the inputs.
template <class T>
__device__ __forceinline__ T ggx_d_t(const T& nh, const T& alpha) {
  const T a2 = alpha * alpha;
  const T k = nh * nh * (a2 - T(1.0f)) + T(1.0f);
  return a2 / (k * k * PI_F);
}
template <class T>
__device__ __forceinline__ T smith_g1_t(const T& vn, const T& alpha) {
  const T c = dabs(vn);
  const T a2 = alpha * alpha;
  return c * 2.0f / (c + dsqrt(a2 + (T(1.0f) - a2) * c * c));
}
template <class T>
__device__ __forceinline__ bool rough_nee_factor_t(const Acq& q, const T& c1, const T& c2, const T& r1, const T& r2,
                                                   const T& alpha, const V3<T>& w, const V3<T>& nin, const V3<T>& o,
                                                   const T& dist2, const T& pitch, T& fac, bool& reflect) {
  const V3<T> i = vscale(w, T(-1.0f));
  const T in = vdot(i, nin), on = vdot(o, nin);
  reflect = dval(on) > 0.0f;
  V3<T> hv = reflect ? vadd(i, o) : vscale(vadd(vscale(i, T(1.0f) / c1), vscale(o, T(1.0f) / c2)), T(-1.0f));
  T hl = T(1.0f) / dsqrt(vdot(hv, hv));
  if (!reflect && dval(vdot(hv, nin)) < 0.0f) hl = hl * -1.0f;  // the facet faces the incident side
  const V3<T> h = vscale(hv, hl);
  const T ih = vdot(i, h), oh = vdot(o, h), nh = vdot(nin, h);
  if (!(dval(ih) > 0.0f) || !(dval(nh) > 0.0f) || (!reflect && !(dval(oh) < 0.0f))) return false;
  // pressure coefficients of the facet h (Snell with sound speeds), incidence cosine ih
  const T rr = c2 / c1;
  T si2 = T(1.0f) - ih * ih;
  if (dval(si2) < 0.0f) si2 = T(0.0f);
  const T st2 = rr * rr * si2;
  const bool tir = dval(st2) >= 1.0f;
  T R, C, J;
  if (tir) {
    if (!reflect) return false;
    R = T(1.0f);
    C = R;
  } else {
    const T ct = dsqrt(T(1.0f) - st2);
    const T Av = r2 * c2 * ih, Bv = r1 * c1 * ct;
    R = (Av - Bv) / (Av + Bv);
    C = reflect ? R : Av * 2.0f / (Av + Bv);
  }
  if (reflect) {
    J = T(1.0f) / (ih * 4.0f);
  } else {
    const T den = ih / c1 + oh / c2;
    J = oh * -1.0f / (c2 * c2 * den * den);
  }
  const T D = ggx_d_t(nh, alpha);
  const T g = D * smith_g1_t(in, alpha) * smith_g1_t(on, alpha) * C * ih * J / in;
  const T omega = pitch * dabs(o.z) * q.hel / dist2;
  const T p_nee = T(1.0f) / (omega * (float)q.ne);
  const T pr = tir ? T(1.0f) : (q.split_mode == 0 ? R * R : T(q.split_q));
  const T p_bsdf = D * nh * J * (reflect ? pr : T(1.0f) - pr);
  fac = g / ((p_nee + p_bsdf) * (float)q.ne);
  return true;
}

__device__ __forceinline__ bool rough_nee_factor(const Acq& q, const Media& med, float3 w, float3 nin, int m1, int m2,
                                                 float alpha, float3 o, float r2, float& fac, int& m_start) {
  bool reflect = false;
  if (!rough_nee_factor_t<float>(q, med.c[m1], med.c[m2], med.rho[m1], med.rho[m2], alpha, v3(w.x, w.y, w.z),
                                 v3(nin.x, nin.y, nin.z), v3(o.x, o.y, o.z), r2, q.pitch, fac, reflect))
    return false;
  m_start = reflect ? m1 : m2;
  return true;
}

// the primary's direction density at a rough event for its sampled facet fn and choice:
// D(h) (h.n) |dh/dw'| P(choice), w_in the incident and w_out the outgoing direction
__device__ __forceinline__ float rough_bsdf_pdf(const Acq& q, const Media& med, float3 w_in, float3 w_out, float3 fn,
                                                float3 nin, int m1, int m2, float alpha, const Iface& f,
                                                bool transmit) {
  const float ih = -dot3(w_in, fn), nh = dot3(fn, nin);
  float J;
  if (transmit) {
    const float oh = dot3(w_out, fn), c1 = med.c[m1], c2 = med.c[m2];
    const float den = ih / c1 + oh / c2;
    J = -oh / (c2 * c2 * den * den);
  } else {
    J = 1.0f / (4.0f * ih);
  }
  const float pr = f.tir ? 1.0f : (q.split_mode == 0 ? f.R * f.R : q.split_q);
  return ggx_d(nh, alpha) * nh * J * (transmit ? 1.0f - pr : pr);
}

// balance weight of a primary's direct hit on the array after a rough event: its direction
// density pdf there, against the secondary ray's 1 / (N_e Omega) for the element face seen from
// distance r along w
__device__ __forceinline__ float rough_hit_weight(const Acq& q, float pdf, float r, float3 w) {
  const float p_nee = r * r / ((float)q.ne * q.pitch * q.hel * fabsf(w.z));
  return pdf / (pdf + p_nee);
}

}  // namespace usrt
