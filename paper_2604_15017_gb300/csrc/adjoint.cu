// Fixed-sample adjoint of the transport and splat (Sec. 3.2, Eq. chain_rule).
//
// One thread per path replays the path from its record (primitive, interface choice and
// secondary-ray element per event are frozen; hit distances are re-solved on the frozen
// primitive: its plane, the closest approach to the scatterer centre, or the transducer
// plane).  For every arrival the splat adjoint is gathered on the fly from dL/dRF (S11), then
// a reverse sweep over the events propagates the adjoints of amplitude, time, position and
// direction through attenuation, Fresnel weights, Snell directions, hit distances and the
// receive directivity, accumulating dL/dtheta in shared memory.
#include "adjoint.cuh"
#include "bvh_query.cuh"

namespace usrt {

// ------------------------------------------------------------------------------------------
// S11: splat adjoint of one arrival (time t_hi + t_lo [s], amplitude a) against the row g:
//   ga = sum_n g[n] s(x_n),  gt = -a sum_n g[n] s'(x_n),  gf = a sum_n g[n] ds(x_n)/df0,
// x_n = n / fs - tau, s(x) = sin(2 pi f0 x) exp(-x^2 / sigma), sigma = 4 ln2 / (pi bw f0)^2.
// The taps are consecutive samples, so the carrier and the Gaussian are stepped by recurrences
// from the first tap (a rotation by 2 pi f0 / fs; E_{n+1} = E_n q_n, q_{n+1} = q_n exp(-2 /
// (fs^2 sigma))) instead of a sin/cos and an exp per tap; over the <= 96 taps of the support
// their rounding grows to a few 1e-6 relative.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void splat_adj_gather(const float* __restrict__ g, float t_hi, float t_lo, float a,
                                                 const PulseP& P, float& ga, float& gt, float& gf) {
  const float u = __fmul_rn(t_hi, P.fs);
  const float e = __fmaf_rn(t_hi, P.fs, -u);
  const float n0f = floorf(u);
  const float fr = (u - n0f) + (e + t_lo * P.fs);  // tau fs = n0 + fr
  const int n0 = (int)n0f;
  const int lo = max(0, n0 + (int)ceilf(fr - P.half));
  const int hi = min(P.ns - 1, n0 + (int)floorf(fr + P.half));
  float sa = 0.0f, st = 0.0f, sf = 0.0f;
  if (lo <= hi) {
    const float w = 2.0f * PI_F * P.f0;
    const float inv_sig = 1.0f / P.sig;
    const float dt = 1.0f / P.fs;
    const float x0 = ((float)(lo - n0) - fr) / P.fs;
    float sn, cs;
    sincosf(w * x0, &sn, &cs);
    float E = expf(-x0 * x0 * inv_sig);
    float q = expf(-(2.0f * x0 + dt) * dt * inv_sig);  // E(x0 + dt) / E(x0)
    for (int n = lo; n <= hi; ++n) {
      const float gn = __ldg(&g[n]);
      const float x = fmaf((float)(n - lo), dt, x0);
      const float s = sn * E;
      const float ds_dx = (w * cs - 2.0f * x * inv_sig * sn) * E;
      const float ds_df = (2.0f * PI_F * x * cs - sn * 2.0f * x * x * inv_sig / P.f0) * E;
      sa = fmaf(gn, s, sa);
      st = fmaf(gn, -ds_dx, st);
      sf = fmaf(gn, ds_df, sf);
      const float sn1 = fmaf(sn, P.rot_c, cs * P.rot_s);
      cs = fmaf(cs, P.rot_c, -sn * P.rot_s);
      sn = sn1;
      E *= q;
      q *= P.env_qq;
    }
  }
  ga = sa;
  gt = a * st;
  gf = a * sf;
}

__global__ void k_splat_adjoint(Acq q, PulseP P, const int32_t* tx, const int32_t* e, const float* tau, const float* a,
                                long long n, const float* grf, float* ga, float* gt, float* gf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float x, y, z;
    splat_adj_gather(grf + ((size_t)tx[i] * q.ne + e[i]) * q.ns, tau[i], 0.0f, a[i], P, x, y, z);
    ga[i] = x;
    gt[i] = y;
    gf[i] = z;
  }
}

// ------------------------------------------------------------------------------------------
// frozen hit distance and its gradient w.r.t. (o, w)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float frozen_t(const SceneDev& S, uint32_t cls, uint32_t id, float3 o, float3 w) {
  if (cls == CLS_XDCR) return -o.z / w.z;
  if (cls == CLS_TRI) {
    const float3 n = xyz(__ldg(&S.tri_nrm[id]));
    const float3 v0 = xyz(__ldg(&S.tri_v0[id]));
    return dot3(v0 - o, n) / dot3(w, n);
  }
  const float3 p = xyz(__ldg(&S.scat[id]));
  return dot3(p - o, w);
}

// Shape adjoint of one triangle (fixed-sample: the same triangle is hit or crossed, its plane
// and normal move with its vertices): from the adjoint nhb of its unit normal n = N / |N|,
// N = e1 x e2 (e1 = v1 - v0, e2 = v2 - v0), and the adjoint v0b of its first vertex through
// the plane offset, the adjoints of its three vertices are added to g[9 id, 9 id + 9).
__device__ __forceinline__ void tri_shape_add(const SceneDev& S, uint32_t id, float3 n, float3 nhb, float3 v0b,
                                              float* g) {
  const float4 E1 = __ldg(&S.tri_e1[id]);
  const float3 e1 = xyz(E1), e2 = xyz(__ldg(&S.tri_e2[id]));
  const float3 Nb = (nhb - n * dot3(n, nhb)) * (1.0f / E1.w);
  const float3 e1b = cross3(e2, Nb), e2b = cross3(Nb, e1);
  const float3 a = v0b - e1b - e2b;
  float* r = g + 9 * (size_t)id;
  atomicAdd(r + 0, a.x);
  atomicAdd(r + 1, a.y);
  atomicAdd(r + 2, a.z);
  atomicAdd(r + 3, e1b.x);
  atomicAdd(r + 4, e1b.y);
  atomicAdd(r + 5, e1b.z);
  atomicAdd(r + 6, e2b.x);
  atomicAdd(r + 7, e2b.y);
  atomicAdd(r + 8, e2b.z);
}

// ------------------------------------------------------------------------------------------
// S12: path adjoint
// ------------------------------------------------------------------------------------------
// slot of the secondary-ray seeds of event k of the pass's path p: event-major, so that the
// path sweep's lanes (consecutive active paths) read neighbouring words at each event
__device__ __forceinline__ size_t seed_slot(const AdjArgs& A, uint32_t p, int k) {
  return (size_t)k * A.n_paths + p;
}
constexpr int ADJ_THREADS = 128;
constexpr int ADJ_EV_SHARED = 4;  // events per path whose sweep state sits in shared memory

// each thread accumulates dL/dtheta in a private shared-memory row (odd stride: no bank
// conflicts, no atomics); the block sums the rows once at the end
#define ADD(slot, v) ((slot) += (v))
__host__ __device__ constexpr int adj_row_stride(int P) { return P | 1; }

// Options compiled in, so that the plain adjoint carries none of their code: bit 0 = the
// acquisition slots (acq_slot), bit 1 = the vertex gradient (g_tris).
constexpr int ADJ_ACQ = 1, ADJ_SHAPE = 2, ADJ_ROUGH = 4;  // bit 2: a rough scene (GGX events)
constexpr int ADJ_RNEE = 8;  // bit 3: secondary rays at rough events (and the balance weights)

// d log G1 / d(v.n) and d log G1 / d alpha of the Smith masking G1 of GGX (see smith_g1)
__device__ __forceinline__ void g1_log_grad(float vn, float alpha, float& d_vn, float& d_alpha) {
  const float c = fabsf(vn);
  const float q = sqrtf(fmaf(1.0f - alpha * alpha, c * c, alpha * alpha));
  const float dc = 1.0f / c - (1.0f + (1.0f - alpha * alpha) * c / q) / (c + q);
  d_vn = vn < 0.0f ? -dc : dc;
  d_alpha = -(alpha * (1.0f - c * c) / q) / (c + q);
}

template <int OPT>
__global__ void __launch_bounds__(ADJ_THREADS) k_path_adjoint(AdjArgs A) {
  extern __shared__ float gsm[];
  const Acq& q = A.acq;
  const Media& med = A.med;
  const int P = A.P;
  const int PS = adj_row_stride(P);
  float* acc = gsm + threadIdx.x * PS;
  const int iAs = 3 * med.M, iF0 = 3 * med.M + 1;
  for (int p = 0; p < P; ++p) acc[p] = 0.0f;
  const int K1 = q.kmax + 1;
  // per-event state kept for the reverse sweep: origin, direction, amplitude.  The first
  // ADJ_EV_SHARED events of a path (most paths have no more) sit in shared memory after the
  // gradient rows, 7 words per event, word-major so that a warp's accesses hit 32 banks; later
  // events go to local memory.  The record word, the medium and the secondary-ray seeds are read
  // or derived again in the sweep.
  float* ev = gsm + ADJ_THREADS * PS + threadIdx.x;
  float evl[7 * (MAX_KMAX + 1 - ADJ_EV_SHARED)];
  auto ev_word = [&](int k, int f) -> float& {
    return k < ADJ_EV_SHARED ? ev[(7 * k + f) * ADJ_THREADS] : evl[7 * (k - ADJ_EV_SHARED) + f];
  };
  auto ev_put = [&](int k, float3 o_, float3 w_, float a_) {
    ev_word(k, 0) = o_.x;
    ev_word(k, 1) = o_.y;
    ev_word(k, 2) = o_.z;
    ev_word(k, 3) = w_.x;
    ev_word(k, 4) = w_.y;
    ev_word(k, 5) = w_.z;
    ev_word(k, 6) = a_;
  };
  const float kap = KAPPA_F;
  const uint32_t n_act = *A.n_active;
  for (uint32_t ai = blockIdx.x * blockDim.x + threadIdx.x; ai < n_act; ai += gridDim.x * blockDim.x) {
    const uint32_t i = A.active[ai];
    const long long path = A.path_base + i;
    const int tx = (int)(path / q.rays_per_tx);
    const long long local = path - (long long)tx * q.rays_per_tx;
    const uint32_t ray = (uint32_t)(q.tx_elem < 0 ? local : (long long)q.tx_elem * q.nr + local);
    // emission (identical to the forward pass)
    const uint4 u = philox4x32_10(make_uint4(ray, (uint32_t)tx, q.stream, 0u), make_uint2(q.key0, q.key1));
    const int e = (int)(ray / (uint32_t)q.nr);
    const float xe = (e - 0.5f * (q.ne - 1)) * q.pitch;
    float sp, cp;
    sincospif(2.0f * u01(u.w), &sp, &cp);
    const float r0 = sqrtf(u01(u.z));
    float3 o = f3(xe + (u01(u.x) - 0.5f) * q.pitch, (u01(u.y) - 0.5f) * q.hel, 0.0f);
    float3 w = f3(r0 * cp, r0 * sp, sqrtf(1.0f - u01(u.z)));
    float a = PI_F / q.nr;
    const float st0 = q.sin_tx[tx];
    const float tau0 = (xe * st0 + 0.5f * (q.ne - 1) * q.pitch * fabsf(st0)) / q.cbf;
    float th = tau0, tl = 0.0f;
    int m = 0, m_last = 0;
    int nseg = 0;
    float gxa = 0.0f, gxt = 0.0f;
    // secondary rays at rough events: the direction density of the last rough event and the
    // distance since (the balance weight of a direct hit on the array), as in the forward pass
    float mis_pdf = 0.0f, mis_since = 0.0f, hit_pdf = 0.0f, hit_since = 0.0f;
    const uint32_t* rec = A.record + (size_t)i * K1;
    // ---- forward replay ----
    for (int k = 0; k <= q.kmax; ++k) {
      const uint32_t r = rec[k];
      const uint32_t cls = code_cls(r), id = code_id(r);
      if (cls == CLS_NONE) break;
      ev_put(k, o, w, a);
      m_last = m;
      nseg = k + 1;
      const float t = frozen_t(A.S, cls, id, o, w);
      const float a1 = a * expf(-kap * med.al[m] * med.f0 * t);
      ff_add(th, tl, t / med.c[m]);
      const float3 x = o + w * t;
      if (cls == CLS_XDCR) {
        float frx = f_rx(-w.z, q.alpha_m, q.alpha_c);
        if ((OPT & ADJ_RNEE) && mis_pdf > 0.0f) {
          hit_pdf = mis_pdf;
          hit_since = mis_since;
          frx *= rough_hit_weight(q, mis_pdf, mis_since + t, w);
        }
        if (frx > 0.0f) {
          float ga, gt, gf;
          splat_adj_gather(A.grf + ((size_t)tx * q.ne + id) * q.ns, th, tl, a1 * frx, A.pulse, ga, gt, gf);
          ADD(acc[iF0], gf);
          gxa = ga;
          gxt = gt;
        }
        break;
      }
      if (k == q.kmax) break;
      if (cls == CLS_TRI) {
        const float4 nr = __ldg(&A.S.tri_nrm[id]);
        const uint32_t mm = __float_as_uint(nr.w);
        const float3 nn = xyz(nr);
        const bool front = dot3(w, nn) < 0.0f;
        const float3 nin = front ? nn : nn * -1.0f;
        const int m1 = front ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
        const int m2 = front ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
        float3 fn = nin;  // facet normal (a GGX microfacet normal at a rough event)
        float alpha = 0.0f;
        if (OPT & ADJ_ROUGH) {
          alpha = med.rough[mm >> 16];
          if (alpha > 0.0f) {
            const uint4 uk = philox4x32_10(make_uint4(ray, (uint32_t)tx, q.stream, (uint32_t)(k + 1)),
                                           make_uint2(q.key0, q.key1));
            fn = ggx_sample(nin, alpha, u01(uk.z), u01(uk.w)).h;
          }
        }
        const float3 w_in = w;
        const Iface f = iface(w, fn, med.c[m1], med.c[m2], med.rho[m1], med.rho[m2]);
        const uint32_t choice = (r >> 22) & 3u;
        const float pr = q.split_mode == 0 ? f.R * f.R : q.split_q;
        if (choice == CH_TIR || f.tir) {
          w = w + fn * (2.0f * f.ci);
          m = m1;
          a = a1;
        } else if (choice == CH_REFLECT) {
          a = a1 * (f.R / pr);
          w = w + fn * (2.0f * f.ci);
          m = m1;
        } else {
          a = a1 * (f.T / (1.0f - pr));
          w = w * f.r + fn * (f.r * f.ci - f.ct);
          m = m2;
        }
        if ((OPT & ADJ_ROUGH) && alpha > 0.0f) {  // microfacet weight (a killed event has no successor)
          const float inn = dot3(w_in, nin), on = dot3(w, nin);
          a *= -dot3(w_in, fn) * smith_g1(inn, alpha) * smith_g1(on, alpha) / (-inn * dot3(fn, nin));
          if (OPT & ADJ_RNEE) {
            const bool transmit = !(choice == CH_TIR || f.tir || choice == CH_REFLECT);
            mis_pdf = rough_bsdf_pdf(q, med, w_in, w, fn, nin, m1, m2, alpha, f, transmit);
            mis_since = 0.0f;
          }
        } else {
          mis_pdf = 0.0f;
        }
      } else {  // scatterer: Born pass-through (amplitude after the segment, direction unchanged)
        a = a1;
        mis_since += t;
      }
      o = x;
    }
    // ---- reverse sweep ----
    float ab = 0.0f, tb = 0.0f;
    float3 ob = f3(0.f, 0.f, 0.f), wb = f3(0.f, 0.f, 0.f);
    int m_next = m_last;  // medium of segment k + 1 (of the last segment to start with)
    // the balance weight's adjoints on their way back to the rough event they came from: that of
    // its direction density, and that of the distance travelled since (every segment after it)
    float g_pdf = 0.0f, g_since = 0.0f;
    for (int k = nseg - 1; k >= 0; --k) {
      const float3 ok = f3(ev_word(k, 0), ev_word(k, 1), ev_word(k, 2));
      const float3 wk = f3(ev_word(k, 3), ev_word(k, 4), ev_word(k, 5));
      const float ak = ev_word(k, 6);
      const uint32_t r = rec[k];
      const uint32_t cls = code_cls(r), id = code_id(r);
      // medium of segment k: the incident side of a hit triangle, else that of segment k + 1
      // (a scatterer keeps the medium; the last segment's was kept)
      int mk = m_next;
      if (cls == CLS_TRI && k < nseg - 1) {
        const float4 nr = __ldg(&A.S.tri_nrm[id]);
        const uint32_t mm = __float_as_uint(nr.w);
        mk = dot3(wk, xyz(nr)) < 0.0f ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
      }
      m_next = mk;
      const float t = frozen_t(A.S, cls, id, ok, wk);
      const float att = expf(-kap * med.al[mk] * med.f0 * t);
      const float a1 = ak * att;
      float a1b, t1b;
      float3 xb, wpb;
      float3 nhb = f3(0.f, 0.f, 0.f);  // shape adjoint: dL/d(unit normal) of a hit triangle
      float t_extra = 0.0f;  // further adjoint of this segment's length (the balance weight's)
      if (cls == CLS_XDCR) {
        const float cosd = -wk.z;
        const float frx = f_rx(cosd, q.alpha_m, q.alpha_c);
        float wm = 1.0f;
        if ((OPT & ADJ_RNEE) && hit_pdf > 0.0f) wm = rough_hit_weight(q, hit_pdf, hit_since + t, wk);
        a1b = gxa * frx * wm;
        t1b = gxt;
        xb = f3(0.f, 0.f, 0.f);
        wpb = f3(0.f, 0.f, 0.f);
        const float thd = acosf(fminf(1.0f, fmaxf(-1.0f, cosd)));
        if (thd > q.alpha_m && thd <= q.alpha_c && frx > 0.0f) {
          const float s = sqrtf(fmaxf(1e-30f, 1.0f - wk.z * wk.z));
          wpb.z = gxa * a1 * wm * (-1.0f / ((q.alpha_c - q.alpha_m) * s));
        }
        if ((OPT & ADJ_RNEE) && hit_pdf > 0.0f && frx > 0.0f) {
          // wm = pdf / (pdf + pn), pn = r^2 / (N_e pitch h_el |w.z|), r = since + t
          const float r = hit_since + t;
          const float pn = r * r / ((float)q.ne * q.pitch * q.hel * fabsf(wk.z));
          const float sden = hit_pdf + pn;
          const float gw = gxa * a1 * frx;
          g_pdf = gw * pn / (sden * sden);
          const float gpn = -gw * hit_pdf / (sden * sden);
          g_since = gpn * 2.0f * pn / r;
          t_extra = g_since;
          wpb.z += gpn * (-pn / wk.z);
          if (OPT & ADJ_ACQ) ADD(acc[A.acq_slot + 1], gpn * (-pn / q.pitch));
        }
      } else if (cls == CLS_TRI) {
        const float4 nr = __ldg(&A.S.tri_nrm[id]);
        const uint32_t mm = __float_as_uint(nr.w);
        const float3 nn = xyz(nr);
        const bool front = dot3(wk, nn) < 0.0f;
        const float3 nin = front ? nn : nn * -1.0f;
        const int m1 = front ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
        const int m2 = front ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
        const float c1 = med.c[m1], c2 = med.c[m2], r1 = med.rho[m1], r2 = med.rho[m2];
        float3 fn = nin;  // facet normal (a GGX microfacet normal at a rough event)
        float alpha = 0.0f;
        GgxSample gs;
        if (OPT & ADJ_ROUGH) {
          alpha = med.rough[mm >> 16];
          if (alpha > 0.0f) {
            const uint4 uk = philox4x32_10(make_uint4(ray, (uint32_t)tx, q.stream, (uint32_t)(k + 1)),
                                           make_uint2(q.key0, q.key1));
            gs = ggx_sample(nin, alpha, u01(uk.z), u01(uk.w));
            fn = gs.h;
          }
        }
        const Iface f = iface(wk, fn, c1, c2, r1, r2);
        const uint32_t choice = (r >> 22) & 3u;
        const bool refl = choice == CH_TIR || f.tir || choice == CH_REFLECT;
        // microfacet weight W = -(w.h) G1(w.n) G1(w'.n) / (-(w.n) (h.n)): a' W leaves the event,
        // so the smooth event below sees ab W and wb + dW/dw' terms; log W's adjoint goes to
        // w, h and alpha
        float abx = ab, ihb = 0.0f, inb = 0.0f, hnb = 0.0f, alb = 0.0f, onb = 0.0f;
        float3 wbx = wb, wo = wb;
        float Rb_pdf = 0.0f;                      // the balance weight's density through P(choice)
        float3 hb_pdf = f3(0.f, 0.f, 0.f);        // ... and through o.h (refraction), into the facet
        if ((OPT & ADJ_ROUGH) && alpha > 0.0f) {
          wo = refl ? wk + fn * (2.0f * f.ci) : wk * f.r + fn * (f.r * f.ci - f.ct);
          const float ih = dot3(wk, fn), inn = dot3(wk, nin), on = dot3(wo, nin), hn = dot3(fn, nin);
          if (ih < 0.0f && refl == (on > 0.0f)) {  // a live event (a killed one passes no adjoint)
            const float Wv = -ih * smith_g1(inn, alpha) * smith_g1(on, alpha) / (-inn * hn);
            const float pr = q.split_mode == 0 ? f.R * f.R : q.split_q;
            const float ap = (choice == CH_TIR || f.tir) ? a1 : (choice == CH_REFLECT ? a1 * f.R / pr
                                                                                      : a1 * f.T / (1.0f - pr));
            const float Wl = ab * ap * Wv;  // adjoint of log W
            abx = ab * Wv;
            float gi_n, gi_a, go_n, go_a;
            g1_log_grad(inn, alpha, gi_n, gi_a);
            g1_log_grad(on, alpha, go_n, go_a);
            ihb = Wl / ih;
            inb = Wl * (gi_n - 1.0f / inn);
            hnb = -Wl / hn;
            alb = Wl * (gi_a + go_a);
            onb = Wl * go_n;
            wbx = wb + nin * onb;
            if ((OPT & ADJ_RNEE) && g_pdf != 0.0f) {
              // the direction density D(h) (h.n) J P(choice) of this event's sampled direction,
              // whose balance weight a later direct hit on the array took
              const bool transmit = !refl;
              const float pdf = rough_bsdf_pdf(q, med, wk, wo, fn, nin, m1, m2, alpha, f, transmit);
              const float gl = g_pdf * pdf;  // adjoint of log pdf
              const float a2 = alpha * alpha, kk = fmaf(hn * hn, a2 - 1.0f, 1.0f);
              hnb += gl * (-4.0f * hn * (a2 - 1.0f) / kk + 1.0f / hn);
              alb += gl * (2.0f / alpha - 4.0f * alpha * hn * hn / kk);
              if (!transmit) {
                ihb += gl * (-1.0f / ih);  // J = 1 / (4 (-w.h))
              } else {  // J = -o.h / (c2^2 den^2), den = (-w.h) / c1 + o.h / c2
                const float ihp = -ih, oh = dot3(wo, fn), c1v = med.c[m1], c2v = med.c[m2];
                const float den = ihp / c1v + oh / c2v;
                ihb += gl * (2.0f / (c1v * den));
                const float goh = gl * (1.0f / oh - 2.0f / (c2v * den));
                wbx = wbx + fn * goh;
                hb_pdf = wo * goh;
                ADD(acc[3 * m1 + 0], gl * 2.0f * ihp / (c1v * c1v * den));
                ADD(acc[3 * m2 + 0], gl * (-2.0f / c2v + 2.0f * oh / (c2v * c2v * den)));
              }
              if (q.split_mode == 0 && !(choice == CH_TIR || f.tir))
                Rb_pdf = gl * (transmit ? -2.0f * f.R / (1.0f - f.R * f.R) : 2.0f / f.R);
            }
          }
        }
        t1b = tb;
        xb = ob;
        float cib = 0.0f, ctb = 0.0f, rb = 0.0f, Rb = 0.0f, Tb = 0.0f;
        if (choice == CH_TIR || f.tir) {
          a1b = abx;
          wpb = wbx;
          cib += 2.0f * dot3(wbx, fn);
        } else if (choice == CH_REFLECT) {
          if (q.split_mode == 0) {
            a1b = abx / f.R;
            Rb = abx * a1 * (-1.0f / (f.R * f.R));
          } else {
            a1b = abx * (f.R / q.split_q);
            Rb = abx * a1 / q.split_q;
          }
          wpb = wbx;
          cib += 2.0f * dot3(wbx, fn);
        } else {
          if (q.split_mode == 0) {
            const float om = 1.0f - f.R;
            a1b = abx / om;
            Rb = abx * a1 / (om * om);
          } else {
            a1b = abx * (f.T / (1.0f - q.split_q));
            Tb = abx * a1 / (1.0f - q.split_q);
          }
          wpb = wbx * f.r;
          rb += dot3(wbx, wk + fn * f.ci);
          const float wn = dot3(wbx, fn);
          cib += f.r * wn;
          ctb -= wn;
        }
        Rb += Rb_pdf;
        if (!f.tir && choice != CH_TIR) {
          const float Av = r2 * c2 * f.ci, Bv = r1 * c1 * f.ct;
          const float den = Av + Bv;
          const float den2 = den * den;
          const float Ab = (Rb + Tb) * 2.0f * Bv / den2;
          const float Bb = -(Rb + Tb) * 2.0f * Av / den2;
          ADD(acc[3 * m2 + 1], Ab * c2 * f.ci);
          float c2b = Ab * r2 * f.ci;
          cib += Ab * r2 * c2;
          ADD(acc[3 * m1 + 1], Bb * c1 * f.ct);
          float c1b = Bb * r1 * f.ct;
          ctb += Bb * r1 * c1;
          if (f.ct > 0.0f) {
            const float si2 = fmaxf(0.0f, 1.0f - f.ci * f.ci);
            rb += ctb * (-f.r * si2 / f.ct);
            cib += ctb * (-f.r * f.r / (2.0f * f.ct)) * (-2.0f * f.ci);
          }
          c2b += rb / c1;
          c1b += -rb * c2 / (c1 * c1);
          ADD(acc[3 * m2 + 0], c2b);
          ADD(acc[3 * m1 + 0], c1b);
        }
        wpb = wpb + fn * (-cib);
        bool rough_ev = false;
        float3 hb;
        if ((OPT & ADJ_ROUGH) && alpha > 0.0f) {
          // h = cos(theta) n + sin(theta) b with tan(theta) = alpha s: dh/dalpha = s cos^3 (b - tan n)
          rough_ev = true;
          wpb = wpb + fn * ihb + nin * inb;
          hb = wk * (ihb - cib) + wbx * (refl ? 2.0f * f.ci : f.r * f.ci - f.ct) + nin * hnb + hb_pdf;
          const float tn = alpha * gs.s, ct = rsqrtf(1.0f + tn * tn);
          alb += dot3(hb, (gs.b - nin * tn) * (gs.s * ct * ct * ct));
          ADD(acc[3 * med.M + 2 + (int)(mm >> 16)], alb);
        }
        if (OPT & ADJ_SHAPE) {  // nin enters through ci = -w.nin and the outgoing direction
          float3 nb;
          if ((OPT & ADJ_ROUGH) && rough_ev)  // through the sampled facet normal and the weight
            nb = ggx_normal_adjoint(nin, gs, alpha, hb) + wk * inb + wo * onb + fn * hnb;
          else
            nb = wk * (-cib) + wb * (refl ? 2.0f * f.ci : f.r * f.ci - f.ct);
          nhb = front ? nb : nb * -1.0f;
        }
        if ((OPT & ADJ_RNEE) && alpha > 0.0f && k < q.kmax) {  // this rough event's secondary ray
          const size_t si = seed_slot(A, i, k);
          const float2 sd = A.seeds[si];
          a1b += sd.x;
          t1b += sd.y;
          xb = xb + xyz(A.seedv[2 * si]);
          wpb = wpb + xyz(A.seedv[2 * si + 1]);
        }
        g_pdf = 0.0f;  // a triangle event ends the straight run a balance weight belongs to
        g_since = 0.0f;
      } else {  // scatterer
        // the secondary ray's adjoint seeds; an event at k_max started none (the interaction
        // budget was spent), so its slot was never written
        const float2 sd = k < q.kmax ? A.seeds[seed_slot(A, i, k)] : make_float2(0.0f, 0.0f);
        a1b = ab + sd.x;
        t1b = tb + sd.y;
        xb = ob;
        wpb = wb;
        if (OPT & ADJ_RNEE) t_extra = g_since;  // a segment after the rough event
      }
      // segment x = o + w t, a1 = a att(t), tau1 = tau + t / c
      float ttb = dot3(xb, wk) + t_extra;
      float3 obn = xb;
      float3 wbn = wpb + xb * t;
      const float attb = a1b * ak;
      const float gatt = attb * att * (-kap);
      ADD(acc[3 * mk + 2], gatt * med.f0 * t);
      ADD(acc[iF0], gatt * med.al[mk] * t);
      ttb += gatt * med.al[mk] * med.f0;
      const float cm = med.c[mk];
      ttb += t1b / cm;
      ADD(acc[3 * mk + 0], -t1b * t / (cm * cm));
      if (cls == CLS_TRI) {
        const float3 n = xyz(__ldg(&A.S.tri_nrm[id]));
        const float den = dot3(wk, n);
        obn = obn + n * (-ttb / den);
        wbn = wbn + n * (-ttb * t / den);
        if (OPT & ADJ_SHAPE) {  // t = (v0 - o).n / (w.n): d/dn = (v0 - x) / (w.n), d/dv0 = n / (w.n)
          const float3 xk = ok + wk * t;
          const float3 v0 = xyz(__ldg(&A.S.tri_v0[id]));
          tri_shape_add(A.S, id, n, nhb + (v0 - xk) * (ttb / den), n * (ttb / den), A.g_tris);
        }
      } else if (cls == CLS_SCAT) {
        const float3 pp = xyz(__ldg(&A.S.scat[id]));
        obn = obn + wk * (-ttb);
        wbn = wbn + (pp - ok) * ttb;
      } else {
        obn.z += -ttb / wk.z;
        wbn.z += ttb * ok.z / (wk.z * wk.z);
      }
      ab = a1b * att;
      tb = t1b;
      ob = obn;
      wb = wbn;
    }
    if (OPT & ADJ_ACQ) {
      // tb = dL/dtau0 and ob = dL/do0 at emission (Sec. 2.3.1).  tau0 = (x_e sin th + W/2 |sin th|)
      // / c_bf: d/dc_bf = -tau0 / c_bf; x_e, W and the origin's x are proportional to the pitch p,
      // so d/dp = tau0 / p and o0.x / p; d/dth with d|sin th|/dth = sgn(sin th) cos th, sgn(0) = 0
      const float sg = st0 > 0.0f ? 1.0f : (st0 < 0.0f ? -1.0f : 0.0f);
      ADD(acc[A.acq_slot], tb * (-tau0 / q.cbf));
      ADD(acc[A.acq_slot + 1], (tb * tau0 + ob.x * ev[0]) / q.pitch);
      ADD(acc[A.acq_slot + 2 + tx], tb * (xe + 0.5f * (q.ne - 1) * q.pitch * sg) * q.cos_tx[tx] / q.cbf);
    }
  }
  __syncthreads();
  float* out = A.gpart + (size_t)blockIdx.x * P;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float s = 0.0f;
    for (int t = 0; t < (int)blockDim.x; ++t) s += gsm[t * PS + p];
    out[p] = (A.accumulate ? out[p] : 0.0f) + s;
  }
}

// ------------------------------------------------------------------------------------------
// Secondary-ray adjoint, one thread per job of the forward pass: the ray's geometry is fixed,
// so its crossings are recomputed, the splat adjoint is gathered for its arrival, the direct
// derivatives of a_n = a' A_s s_j prod T exp(-kappa f0 sum alpha l) f_rx N_e and of
// tau_n = tau' + sum l / c go to theta, and the seeds (dL/da', dL/dtau') are left for the
// path's reverse sweep.
// ------------------------------------------------------------------------------------------
// The rows hold only the slots a secondary ray touches (nee_row_len): the 3M + 2 material
// parameters and, with the acquisition option, the pitch at 3M + 2; no roughness slots (the
// crossings are smooth), so a rough scene costs no more shared memory (and L1) than a smooth one.
// With secondary rays at rough events the rows also hold the M roughness slots (3M + 2 ..
// 4M + 1), and the pitch follows them.
__host__ __device__ inline int nee_row_len(int M, bool acq, bool rnee = false) {
  return 3 * M + 2 + (rnee ? M : 0) + (acq ? 1 : 0);
}

// local derivatives of a rough event's secondary-ray BSDF factor: dual slots of its inputs
constexpr int RN_C1 = 0, RN_C2 = 1, RN_R1 = 2, RN_R2 = 3, RN_AL = 4, RN_W = 5, RN_N = 8, RN_O = 11, RN_D2 = 14,
              RN_P = 15, RN_SLOTS = 16;

template <int OPT>
__global__ void __launch_bounds__(ADJ_THREADS) k_nee_adjoint(AdjArgs A) {
  extern __shared__ float gsm[];
  const Acq& q = A.acq;
  const Media& med = A.med;
  const int P = A.P;
  constexpr bool rnee = (OPT & ADJ_RNEE) != 0;
  const int R = nee_row_len(med.M, (OPT & ADJ_ACQ) != 0, rnee);
  const int iPitch = 3 * med.M + 2 + (rnee ? med.M : 0);  // the pitch's row slot (acquisition option)
  const int PS = adj_row_stride(R);
  float* acc = gsm + threadIdx.x * PS;
  const int iAs = 3 * med.M, iF0 = 3 * med.M + 1;
  for (int p = 0; p < R; ++p) acc[p] = 0.0f;
  const int K1 = q.kmax + 1;
  const float kap = KAPPA_F;
  uint32_t total = 0;
  for (int k = 0; k <= q.kmax; ++k) total += A.cnt->nee[k];
  float xt[MAX_XINGS];
  uint32_t xid[MAX_XINGS];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const float4 job = A.nee.job[i];
    const uint32_t jm = A.nee.jm[i];
    const uint32_t jid = __float_as_uint(job.w);
    int m = (int)(jm & 0xFF);
    const int e2 = (int)((jm >> 8) & 0xFF), tx = (int)((jm >> 16) & 0xFF);
    const int k = (int)(jm >> 24);
    const long long path = A.nee.jpath[i];
    float2* seed = &A.seeds[seed_slot(A, (uint32_t)(path - A.path_base), k)];
    const float a1 = job.x;
    float nh = job.y, nl = job.z;
    // the ray's start: a scatterer's centre, or (rough events) the event point on triangle tri
    const bool rough_job = rnee && (jid & NEE_ROUGH) != 0u;
    const uint32_t tri = jid & ~NEE_ROUGH;
    float4 sc = make_float4(0.f, 0.f, 0.f, 0.f);
    float3 p0, wi = f3(0.f, 0.f, 0.f), nin = wi, nn = wi;
    int m2 = m;
    bool front = true;
    if (rough_job) {
      p0 = xyz(A.nee.jx[i]);
      wi = xyz(A.nee.jw[i]);
      const float4 nr = __ldg(&A.S.tri_nrm[tri]);
      const uint32_t mm = __float_as_uint(nr.w);
      nn = xyz(nr);
      front = dot3(wi, nn) < 0.0f;
      nin = front ? nn : nn * -1.0f;
      m2 = front ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
      const float3 dv0 = f3(elem_x(q, e2), 0.0f, 0.0f) - p0;
      const float r2v = dot3(dv0, dv0);
      float fac0;
      int ms;
      if (!rough_nee_factor(q, med, wi, nin, m, m2, med.rough[mm >> 16], dv0 * rsqrtf(r2v), r2v, fac0, ms)) {
        *seed = make_float2(0.0f, 0.0f);
        A.seedv[2 * seed_slot(A, (uint32_t)(path - A.path_base), k)] = make_float4(0.f, 0.f, 0.f, 0.f);
        A.seedv[2 * seed_slot(A, (uint32_t)(path - A.path_base), k) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      m = ms;  // the medium the segment starts in
    } else {
      sc = __ldg(&A.S.scat[jid]);
      p0 = xyz(sc);
    }
    float3 d;
    float D;
    NeeOut no;
    const uint2 xo = A.nres.xo ? A.nres.xo[i] : make_uint2(0u, NEE_UNSTORED);
    if (xo.y == NEE_UNSTORED) {  // trace the secondary ray again
      no = nee_eval(A.S, med, q, p0, e2, m, nh, nl, xt, xid, &d, &D, rough_job ? tri : 0xFFFFFFFFu);
    } else {  // the forward pass's result: same arithmetic, read back
      no.ok = xo.y != NEE_NONE;
      no.overflow = false;
      no.n = no.ok ? (int)xo.y : 0;
      if (no.ok) {
        const float4 rs = A.nres.res[i];
        nh = rs.x;
        nl = rs.y;
        no.gain = rs.z;
        no.sum_al = rs.w;
        for (int c = 0; c < no.n; ++c) {
          const uint2 x = A.nres.xing[xo.x + c];
          xt[c] = __uint_as_float(x.x);
          xid[c] = x.y;
        }
        const float3 dv = f3(elem_x(q, e2), 0.0f, 0.0f) - p0;
        D = sqrtf(dot3(dv, dv));
        d = dv * (1.0f / D);
      }
    }
    if (!no.ok) {
      *seed = make_float2(0.0f, 0.0f);
      if (rough_job) {
        A.seedv[2 * seed_slot(A, (uint32_t)(path - A.path_base), k)] = make_float4(0.f, 0.f, 0.f, 0.f);
        A.seedv[2 * seed_slot(A, (uint32_t)(path - A.path_base), k) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    // a rough event's BSDF factor with its derivatives in its 16 local inputs
    DualN<RN_SLOTS> fd(0.0f);
    if (rough_job) {
      const uint32_t mm = __float_as_uint(__ldg(&A.S.tri_nrm[tri]).w);
      const int m1 = (int)(jm & 0xFF);
      typedef DualN<RN_SLOTS> DT;
      const V3<DT> wv = v3(dual_var<RN_SLOTS>(wi.x, RN_W), dual_var<RN_SLOTS>(wi.y, RN_W + 1),
                           dual_var<RN_SLOTS>(wi.z, RN_W + 2));
      const V3<DT> nv = v3(dual_var<RN_SLOTS>(nin.x, RN_N), dual_var<RN_SLOTS>(nin.y, RN_N + 1),
                           dual_var<RN_SLOTS>(nin.z, RN_N + 2));
      const V3<DT> ov = v3(dual_var<RN_SLOTS>(d.x, RN_O), dual_var<RN_SLOTS>(d.y, RN_O + 1),
                           dual_var<RN_SLOTS>(d.z, RN_O + 2));
      bool refl;
      rough_nee_factor_t<DT>(q, dual_var<RN_SLOTS>(med.c[m1], RN_C1), dual_var<RN_SLOTS>(med.c[m2], RN_C2),
                             dual_var<RN_SLOTS>(med.rho[m1], RN_R1), dual_var<RN_SLOTS>(med.rho[m2], RN_R2),
                             dual_var<RN_SLOTS>(med.rough[mm >> 16], RN_AL), wv, nv, ov,
                             dual_var<RN_SLOTS>(D * D, RN_D2), dual_var<RN_SLOTS>(q.pitch, RN_P), fd, refl);
    }
    const float k_n = (rough_job ? fd.v : med.As * sc.w) * no.gain;
    const float a_n = a1 * k_n;
    float ga, gt, gf;
    splat_adj_gather(A.grf + ((size_t)tx * q.ne + e2) * q.ns, nh, nl, a_n, A.pulse, ga, gt, gf);
    const float Ga = ga * a_n;  // adjoint of log a_n
    ADD(acc[iF0], gf + Ga * (-kap * no.sum_al));
    if (!rough_job) ADD(acc[iAs], ga * a1 * sc.w * no.gain);
    // rough events: the segment's direction d, length D and start point p0 take adjoints too
    float3 gd = f3(0.f, 0.f, 0.f), gP0 = gd;
    float gD = 0.0f;
    if (rough_job) {
      const float Gf = Ga / fd.v;  // adjoint of the factor (log)
      const uint32_t mm = __float_as_uint(__ldg(&A.S.tri_nrm[tri]).w);
      const int m1 = (int)(jm & 0xFF);
      ADD(acc[3 * m1 + 0], Gf * fd.d[RN_C1]);
      ADD(acc[3 * m2 + 0], Gf * fd.d[RN_C2]);
      ADD(acc[3 * m1 + 1], Gf * fd.d[RN_R1]);
      ADD(acc[3 * m2 + 1], Gf * fd.d[RN_R2]);
      ADD(acc[3 * med.M + 2 + (int)(mm >> 16)], Gf * fd.d[RN_AL]);
      gd = f3(Gf * fd.d[RN_O], Gf * fd.d[RN_O + 1], Gf * fd.d[RN_O + 2]);
      gD = Gf * fd.d[RN_D2] * 2.0f * D;
      if (OPT & ADJ_ACQ) ADD(acc[iPitch], Gf * fd.d[RN_P]);
      if (OPT & ADJ_SHAPE) {  // the macro normal of the event's triangle
        const float3 gn = f3(Gf * fd.d[RN_N], Gf * fd.d[RN_N + 1], Gf * fd.d[RN_N + 2]);
        tri_shape_add(A.S, tri, nn, front ? gn : gn * -1.0f, f3(0.f, 0.f, 0.f), A.g_tris);
      }
      // receive directivity f_rx(-d.z) on its ramp
      const float frx = f_rx(-d.z, q.alpha_m, q.alpha_c);
      const float thd = acosf(fminf(1.0f, fmaxf(-1.0f, -d.z)));
      if (thd > q.alpha_m && frx > 0.0f)
        gd.z += Ga * (-1.0f / ((q.alpha_c - q.alpha_m) * frx * sqrtf(fmaxf(1e-30f, 1.0f - d.z * d.z))));
    }
    // pitch: the target x_e = p (e2 - (N_e - 1)/2) moves along x; dX below are derivatives in x_e
    // (direction dd = (e_x - d d.x) / D, crossing distances t_c = A_c / (d.n_c), lengths, cosines)
    // the pitch moves the target x_e (scatterers: dX below; rough events: the general endpoint
    // adjoints gd, gD, gP0 above, converted after the loop)
    const bool acq = (OPT & ADJ_ACQ) != 0 && !rough_job;
    float gX = 0.0f, dt_prev = 0.0f;
    if (acq) {  // receive directivity: d log f_rx / dX on its ramp
      const float frx = f_rx(-d.z, q.alpha_m, q.alpha_c);
      const float thd = acosf(fminf(1.0f, fmaxf(-1.0f, -d.z)));
      if (thd > q.alpha_m && frx > 0.0f) {
        const float ddz = -d.x * d.z / D;
        gX += Ga * (-(ddz / sqrtf(fmaxf(1e-30f, 1.0f - d.z * d.z))) / (q.alpha_c - q.alpha_m)) / frx;
      }
    }
    float tprev = 0.0f;
    int mm_cur = m;
    for (int c = 0; c <= no.n; ++c) {
      const float tc = c < no.n ? xt[c] : D;
      const float l = tc - tprev;
      ADD(acc[3 * mm_cur + 2], Ga * (-kap * med.f0 * l));
      ADD(acc[3 * mm_cur + 0], gt * (-l / (med.c[mm_cur] * med.c[mm_cur])));
      if (rough_job && c == no.n) gD += Ga * (-kap * med.f0 * med.al[mm_cur]) + gt / med.c[mm_cur];
      if (acq) {
        float dtc = d.x;  // dD/dX
        if (c < no.n) {
          const float3 nn = xyz(__ldg(&A.S.tri_nrm[xid[c]]));
          const float dn = dot3(d, nn);
          dtc = -tc * ((nn.x - d.x * dn) / D) / dn;
        }
        gX += (Ga * (-kap * med.f0 * med.al[mm_cur]) + gt / med.c[mm_cur]) * (dtc - dt_prev);
        dt_prev = dtc;
      }
      if (c == no.n) break;
      const float4 nr = __ldg(&A.S.tri_nrm[xid[c]]);
      const uint32_t mm = __float_as_uint(nr.w);
      const float dn = dot3(d, xyz(nr));
      const int m1 = dn < 0.0f ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
      const int m2 = dn < 0.0f ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
      const float ci = fabsf(dn);
      const float c1 = med.c[m1], c2 = med.c[m2], r1 = med.rho[m1], r2 = med.rho[m2];
      const float rr = c2 / c1;
      const float si2 = fmaxf(0.0f, 1.0f - ci * ci);
      const float ct = sqrtf(fmaxf(0.0f, 1.0f - rr * rr * si2));
      const float Av = r2 * c2 * ci, Bv = r1 * c1 * ct;
      const float Ab = Ga * Bv / (Av * (Av + Bv));
      const float Bb = -Ga / (Av + Bv);
      ADD(acc[3 * m2 + 1], Ab * c2 * ci);
      float c2b = Ab * r2 * ci;
      ADD(acc[3 * m1 + 1], Bb * c1 * ct);
      float c1b = Bb * r1 * ct;
      const float ctb = Bb * r1 * c1;
      if (ct > 0.0f) {
        const float rb = ctb * (-rr * si2 / ct);
        c2b += rb / c1;
        c1b += -rb * c2 / (c1 * c1);
      }
      ADD(acc[3 * m2 + 0], c2b);
      ADD(acc[3 * m1 + 0], c1b);
      if (acq) {  // the transmission coefficient through its incidence cosine ci = |d.n|
        const float dci = (dn < 0.0f ? -1.0f : 1.0f) * (nr.x - d.x * dn) / D;
        const float dct = ct > 0.0f ? rr * rr * ci / ct : 0.0f;
        gX += (Ab * r2 * c2 + Bb * r1 * c1 * dct) * dci;
      }
      if (rough_job) {  // t_c = (v0 - p0).n / (d.n) and the incidence cosine |d.n|
        const float3 n = xyz(nr);
        const float tcb = (Ga * (-kap * med.f0 * med.al[mm_cur]) + gt / med.c[mm_cur]) -
                          (Ga * (-kap * med.f0 * med.al[m2]) + gt / med.c[m2]);  // dL/dt_c
        const float dct = ct > 0.0f ? rr * rr * ci / ct : 0.0f;
        const float cib = Ab * r2 * c2 + Bb * r1 * c1 * dct;
        gP0 = gP0 + n * (-tcb / dn);
        gd = gd + n * (-tcb * tc / dn + (dn < 0.0f ? -cib : cib));
      }
      if (OPT & ADJ_SHAPE) {  // the crossed triangle: its plane (crossing distance) and normal (ci)
        const float3 n = xyz(nr);
        const float tcb = (Ga * (-kap * med.f0 * med.al[mm_cur]) + gt / med.c[mm_cur]) -
                          (Ga * (-kap * med.f0 * med.al[m2]) + gt / med.c[m2]);  // dL/dt_c
        const float dct = ct > 0.0f ? rr * rr * ci / ct : 0.0f;
        const float cib = Ab * r2 * c2 + Bb * r1 * c1 * dct;
        const float3 xc = p0 + d * tc;
        const float3 v0 = xyz(__ldg(&A.S.tri_v0[xid[c]]));
        const float3 nhb = d * (dn < 0.0f ? -cib : cib) + (v0 - xc) * (tcb / dn);
        tri_shape_add(A.S, xid[c], n, nhb, n * (tcb / dn), A.g_tris);
      }
      mm_cur = m2;
      tprev = tc;
    }
    if (acq) ADD(acc[iPitch], gX * ((float)e2 - 0.5f * (float)(q.ne - 1)));  // the pitch
    *seed = make_float2(ga * k_n, gt);
    if (rough_job) {
      // d = (x_e - p0) / D, D = |x_e - p0|: the adjoint of the target point is
      // (gd - d (d.gd)) / D + gD d, that of p0 its negative plus the crossings' direct terms
      const float3 gT = (gd - d * dot3(d, gd)) * (1.0f / D) + d * gD;
      gP0 = gP0 - gT;
      if (OPT & ADJ_ACQ) ADD(acc[iPitch], gT.x * ((float)e2 - 0.5f * (float)(q.ne - 1)));
      const float Gf = Ga / fd.v;
      const size_t sv = 2 * seed_slot(A, (uint32_t)(path - A.path_base), k);
      A.seedv[sv] = make_float4(gP0.x, gP0.y, gP0.z, 0.0f);
      A.seedv[sv + 1] = make_float4(Gf * fd.d[RN_W], Gf * fd.d[RN_W + 1], Gf * fd.d[RN_W + 2], 0.0f);
    }
  }
  __syncthreads();
  float* out = A.gpart + (size_t)blockIdx.x * P;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    // the row slot of gradient slot p (-1: a slot secondary rays do not touch)
    const int rp = p < 3 * med.M + 2 ? p
                   : (rnee && p < 4 * med.M + 2) ? p
                   : (((OPT & ADJ_ACQ) && p == A.acq_slot + 1) ? iPitch : -1);
    float s = 0.0f;
    if (rp >= 0)
      for (int t = 0; t < (int)blockDim.x; ++t) s += gsm[t * PS + rp];
    out[p] = (A.accumulate ? out[p] : 0.0f) + s;
  }
}

// ------------------------------------------------------------------------------------------
// Paths that produced an arrival (a transducer hit, or a scatterer event before the
// interaction budget ran out), grouped by their number of events so that the lanes of a warp
// sweep paths of equal length.  work: [0, 17) counts, [17, 34) offsets, [34, 51) cursors,
// [51] total.
// ------------------------------------------------------------------------------------------
// rough_mask: bit m set when medium m is rough and its interfaces' events send secondary rays
// (a triangle's roughness is its back-side medium's), read through the triangle's media
__device__ __forceinline__ int path_class(const uint32_t* rec, int kmax, uint32_t rough_mask, const float4* tri_nrm) {
  int nseg = 0;
  bool active = false;
  for (int k = 0; k <= kmax; ++k) {
    const uint32_t c = code_cls(rec[k]);
    if (c == CLS_NONE) break;
    nseg = k + 1;
    if (c == CLS_XDCR || (c == CLS_SCAT && k < kmax)) active = true;
    if (rough_mask && c == CLS_TRI && k < kmax &&
        ((rough_mask >> (__float_as_uint(__ldg(&tri_nrm[code_id(rec[k])]).w) >> 16)) & 1u))
      active = true;
  }
  return active ? nseg : -1;
}

// One tile of ACT_TILE paths per block iteration: the tile's record rows are read into shared
// memory with coalesced loads, each thread classifies its path from there, and the per-class
// counts go through shared memory to one global atomic per class and block.
constexpr int ACT_TILE = 256;
__global__ void __launch_bounds__(ACT_TILE) k_active_count(const uint32_t* record, uint32_t n, int kmax,
                                                           uint32_t* work, uint8_t* pclass, uint32_t rough_mask,
                                                           const float4* tri_nrm) {
  extern __shared__ uint32_t rows[];  // [ACT_TILE][kmax + 1]
  __shared__ uint32_t cnt[17];
  const int K1 = kmax + 1;
  if (threadIdx.x < 17) cnt[threadIdx.x] = 0u;
  for (uint32_t base = blockIdx.x * ACT_TILE; base < n; base += gridDim.x * ACT_TILE) {
    const uint32_t m = min((uint32_t)ACT_TILE, n - base);
    __syncthreads();
    const uint32_t* src = record + (size_t)base * K1;
    for (uint32_t j = threadIdx.x; j < m * (uint32_t)K1; j += ACT_TILE) rows[j] = __ldg(&src[j]);
    __syncthreads();
    if (threadIdx.x < m) {
      const int c = path_class(rows + threadIdx.x * K1, kmax, rough_mask, tri_nrm);
      pclass[base + threadIdx.x] = (uint8_t)(c < 0 ? 0xFF : c);  // read back by k_active_fill
      if (c >= 0) {
        const unsigned same = __match_any_sync(__activemask(), c);  // lanes of this class
        if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[c], (uint32_t)__popc(same));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 17 && cnt[threadIdx.x]) atomicAdd(&work[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void k_active_scan(uint32_t* work) {
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int c = 16; c >= 0; --c) {  // longest paths first
      work[17 + c] = run;
      work[34 + c] = 0;
      run += work[c];
    }
    work[51] = run;
  }
}

// Per block iteration: the tile's paths are counted per class in shared memory, one global
// atomic per class reserves the tile's range in that class, and the tile's paths take slots
// in it through shared-memory counters (the order inside a class is free).
__global__ void __launch_bounds__(ACT_TILE) k_active_fill(const uint8_t* pclass, uint32_t n, uint32_t* work,
                                                          uint32_t* active) {
  __shared__ uint32_t cnt[17], at[17];
  for (uint32_t base = blockIdx.x * ACT_TILE; base < n; base += gridDim.x * ACT_TILE) {
    if (threadIdx.x < 17) cnt[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t i = base + threadIdx.x;
    const int c = i < n && pclass[i] != 0xFF ? (int)pclass[i] : -1;
    uint32_t off = 0u;
    if (c >= 0) {
      const unsigned same = __match_any_sync(__activemask(), c);
      const int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
      uint32_t b = 0u;
      if (lane == leader) b = atomicAdd(&cnt[c], (uint32_t)__popc(same));
      off = __shfl_sync(same, b, leader) + __popc(same & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (threadIdx.x < 17)
      at[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&work[34 + threadIdx.x], cnt[threadIdx.x]) : 0u;
    __syncthreads();
    if (c >= 0) active[work[17 + c] + at[c] + off] = i;
    __syncthreads();
  }
}

// column sums of gpart [nblocks][P] in block order: columns [0, Ps) to g, the rest to g2
// (added to it when acc2)
__global__ void k_grad_reduce(const float* gpart, int nblocks, int P, int Ps, float* g, float* g2, int acc2) {
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += gpart[(size_t)b * P + p];
    if (p < Ps)
      g[p] = s;
    else
      g2[p - Ps] = (acc2 ? g2[p - Ps] : 0.0f) + s;
  }
}

// chain rule to shape parameters: out[j] = sum_i g[i] tan[j n + i], one block per parameter,
// block-strided partial sums combined in a fixed order
__global__ void k_tangent_dot(long long n, const float* __restrict__ g, const float* __restrict__ tan, float* out) {
  __shared__ float red[256];
  const float* t = tan + (size_t)blockIdx.x * n;
  float s = 0.0f;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s = fmaf(g[i], t[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// S1 as a standalone stream: Philox blocks with consecutive first counter words
__global__ void k_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                              long long n, uint32_t* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(make_uint4(c0 + (uint32_t)i, c1, c2, c3), make_uint2(k0, k1));
    reinterpret_cast<uint4*>(out)[i] = r;
  }
}

static int adj_opt(const AdjArgs& a) {
  return (a.acq_slot >= 0 ? ADJ_ACQ : 0) | (a.g_tris ? ADJ_SHAPE : 0) | (a.med.has_rough ? ADJ_ROUGH : 0);
}
void launch_nee_adjoint(const AdjArgs& a, int grid, cudaStream_t st) {
  const bool rnee = a.med.has_rough && a.acq.rough_nee;
  const size_t sm = sizeof(float) * ADJ_THREADS * adj_row_stride(nee_row_len(a.med.M, a.acq_slot >= 0, rnee));
  // secondary rays cross rough interfaces as smooth ones; they start at rough events with rnee
  switch ((adj_opt(a) & (ADJ_ACQ | ADJ_SHAPE)) | (rnee ? ADJ_RNEE : 0)) {
    case 0: k_nee_adjoint<0><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 1: k_nee_adjoint<1><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 2: k_nee_adjoint<2><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 3: k_nee_adjoint<3><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 8: k_nee_adjoint<8><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 9: k_nee_adjoint<9><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 10: k_nee_adjoint<10><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    default: k_nee_adjoint<11><<<grid, ADJ_THREADS, sm, st>>>(a); break;
  }
}
void launch_active_paths(const uint32_t* record, uint32_t n_paths, int kmax, uint32_t* work, uint8_t* pclass,
                         uint32_t* active, int grid, cudaStream_t st, uint32_t rough_mask, const float4* tri_nrm) {
  cudaMemsetAsync(work, 0, sizeof(uint32_t) * 52, st);
  k_active_count<<<grid, ACT_TILE, sizeof(uint32_t) * ACT_TILE * (kmax + 1), st>>>(record, n_paths, kmax, work,
                                                                                  pclass, rough_mask, tri_nrm);
  k_active_scan<<<1, 32, 0, st>>>(work);
  k_active_fill<<<grid, ACT_TILE, 0, st>>>(pclass, n_paths, work, active);
}
// the path sweep's shared memory: the gradient rows, then 7 words per event and thread for
// the first ADJ_EV_SHARED events
__host__ __device__ constexpr size_t path_adj_smem(int P, int kmax) {
  return sizeof(float) * ADJ_THREADS * (size_t)(adj_row_stride(P) + 7 * (kmax + 1 < ADJ_EV_SHARED ? kmax + 1 : ADJ_EV_SHARED));
}
void launch_path_adjoint(const AdjArgs& a, int grid, cudaStream_t st) {
  const size_t sm = path_adj_smem(a.P, a.acq.kmax);
  const bool rnee = a.med.has_rough && a.acq.rough_nee;
  switch (adj_opt(a) | (rnee ? ADJ_RNEE : 0)) {
    case 12: k_path_adjoint<12><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 13: k_path_adjoint<13><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 14: k_path_adjoint<14><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 15: k_path_adjoint<15><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 0: k_path_adjoint<0><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 1: k_path_adjoint<1><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 2: k_path_adjoint<2><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 3: k_path_adjoint<3><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 4: k_path_adjoint<4><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 5: k_path_adjoint<5><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    case 6: k_path_adjoint<6><<<grid, ADJ_THREADS, sm, st>>>(a); break;
    default: k_path_adjoint<7><<<grid, ADJ_THREADS, sm, st>>>(a); break;
  }
}
cudaError_t adjoint_set_attrs() {
  const int sm = (int)path_adj_smem(MAX_P_ACQ, MAX_KMAX);
  static_assert(path_adj_smem(MAX_P_ACQ, MAX_KMAX) <= 227 * 1024, "path sweep shared memory");
  const void* ks[] = {(const void*)k_path_adjoint<0>,  (const void*)k_path_adjoint<1>,
                      (const void*)k_path_adjoint<2>,  (const void*)k_path_adjoint<3>,
                      (const void*)k_path_adjoint<4>,  (const void*)k_path_adjoint<5>,
                      (const void*)k_path_adjoint<6>,  (const void*)k_path_adjoint<7>,
                      (const void*)k_path_adjoint<12>, (const void*)k_path_adjoint<13>,
                      (const void*)k_path_adjoint<14>, (const void*)k_path_adjoint<15>,
                      (const void*)k_nee_adjoint<0>,   (const void*)k_nee_adjoint<1>,
                      (const void*)k_nee_adjoint<2>,   (const void*)k_nee_adjoint<3>,
                      (const void*)k_nee_adjoint<8>,   (const void*)k_nee_adjoint<9>,
                      (const void*)k_nee_adjoint<10>,  (const void*)k_nee_adjoint<11>};
  for (const void* k : ks) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
void launch_grad_reduce(const float* gpart, int nblocks, int P, float* g, cudaStream_t st) {
  k_grad_reduce<<<1, 128, 0, st>>>(gpart, nblocks, P, P, g, nullptr, 0);
}
void launch_grad_reduce_split(const float* gpart, int nblocks, int P, int Ps, float* g, float* g2, int acc2,
                              cudaStream_t st) {
  k_grad_reduce<<<1, 128, 0, st>>>(gpart, nblocks, P, Ps, g, g2, acc2);
}
void launch_tangent_dot(long long n, const float* g, int n_param, const float* tan, float* out, cudaStream_t st) {
  k_tangent_dot<<<n_param, 256, 0, st>>>(n, g, tan, out);
}
void launch_splat_adjoint(const Acq& q, const PulseP& P, const int32_t* tx, const int32_t* e, const float* tau,
                          const float* a, long long n, const float* grf, float* ga, float* gt, float* gf, int grid,
                          cudaStream_t st) {
  k_splat_adjoint<<<grid, 256, 0, st>>>(q, P, tx, e, tau, a, n, grf, ga, gt, gf);
}
void launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, long long n,
                        uint32_t* out, int grid, cudaStream_t st) {
  k_philox_fill<<<grid, 256, 0, st>>>(c0, c1, c2, c3, k0, k1, n, out);
}

}  // namespace usrt
