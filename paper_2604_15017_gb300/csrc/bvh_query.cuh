// BVH queries (Sec. 2.3.2 traversal, Sec. 2.3.3 secondary rays), header-only so that the
// transport and adjoint kernels inline them.
#pragma once

#include "usrt_device.cuh"

namespace usrt {

constexpr int BVH_STACK = 64;

struct RayInv {
  float3 inv, oi;
};
__device__ __forceinline__ float safe_inv(float d) {
  return 1.0f / (fabsf(d) > 1e-20f ? d : copysignf(1e-20f, d));
}
__device__ __forceinline__ RayInv ray_inv(float3 o, float3 w) {
  RayInv r;
  r.inv = f3(safe_inv(w.x), safe_inv(w.y), safe_inv(w.z));
  r.oi = f3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
  return r;
}

// slab test of both children of a node; tmin returned, hit when tmin <= tmax'.  tmax is
// widened by 2 ulp-ish (robust traversal) so that rounding never culls a box that holds a hit.
__device__ __forceinline__ void node_boxes(const RayInv& r, float4 n0, float4 n1, float4 n2, float tlimit, bool& h0,
                                           bool& h1, float& t0, float& t1) {
  const float ax0 = fmaf(n0.x, r.inv.x, -r.oi.x), bx0 = fmaf(n0.y, r.inv.x, -r.oi.x);
  const float ay0 = fmaf(n0.z, r.inv.y, -r.oi.y), by0 = fmaf(n0.w, r.inv.y, -r.oi.y);
  const float az0 = fmaf(n2.x, r.inv.z, -r.oi.z), bz0 = fmaf(n2.y, r.inv.z, -r.oi.z);
  const float ax1 = fmaf(n1.x, r.inv.x, -r.oi.x), bx1 = fmaf(n1.y, r.inv.x, -r.oi.x);
  const float ay1 = fmaf(n1.z, r.inv.y, -r.oi.y), by1 = fmaf(n1.w, r.inv.y, -r.oi.y);
  const float az1 = fmaf(n2.z, r.inv.z, -r.oi.z), bz1 = fmaf(n2.w, r.inv.z, -r.oi.z);
  const float lo0 = fmaxf(fmaxf(fminf(ax0, bx0), fminf(ay0, by0)), fmaxf(fminf(az0, bz0), 0.0f));
  const float hi0 = fminf(fminf(fmaxf(ax0, bx0), fmaxf(ay0, by0)), fminf(fmaxf(az0, bz0), tlimit));
  const float lo1 = fmaxf(fmaxf(fminf(ax1, bx1), fminf(ay1, by1)), fmaxf(fminf(az1, bz1), 0.0f));
  const float hi1 = fminf(fminf(fmaxf(ax1, bx1), fmaxf(ay1, by1)), fminf(fmaxf(az1, bz1), tlimit));
  h0 = lo0 <= hi0 * 1.0000004f;
  h1 = lo1 <= hi1 * 1.0000004f;
  t0 = lo0;
  t1 = lo1;
}

// Moller-Trumbore ray/triangle test; returns t > T_MIN or -1
__device__ __forceinline__ float tri_test(float3 o, float3 w, float3 v0, float3 e1, float3 e2) {
  const float3 p = cross3(w, e2);
  const float det = dot3(e1, p);
  if (det == 0.0f) return -1.0f;
  const float inv = 1.0f / det;
  const float3 tv = o - v0;
  const float u = dot3(tv, p) * inv;
  if (u < 0.0f || u > 1.0f) return -1.0f;
  const float3 qv = cross3(tv, e1);
  const float v = dot3(w, qv) * inv;
  if (v < 0.0f || u + v > 1.0f) return -1.0f;
  const float t = dot3(e2, qv) * inv;
  return t > T_MIN ? t : -1.0f;
}

// point scatterer: event at the closest approach t = (p - o).w when within r_s of the centre
__device__ __forceinline__ float scat_test(float3 o, float3 w, float3 p, float rs2) {
  const float3 d = p - o;
  const float t = dot3(d, w);
  if (!(t > T_MIN)) return -1.0f;
  const float3 q = w * t - d;
  return dot3(q, q) <= rs2 ? t : -1.0f;
}

__device__ __forceinline__ bool hit_better(float t, uint32_t c, float tb, uint32_t cb) {
  return t < tb || (t == tb && c < cb);
}

// transducer face z = 0, |x| <= n_elem pitch / 2, |y| <= h_el / 2, approached from z > 0
__device__ __forceinline__ void xdcr_test(const Acq& q, float3 o, float3 w, float& tbest, uint32_t& cbest) {
  if (!(w.z < 0.0f)) return;
  const float t = -o.z / w.z;
  const float x = fmaf(t, w.x, o.x), y = fmaf(t, w.y, o.y);
  const float half = 0.5f * q.ne * q.pitch;
  if (t > T_MIN && fabsf(x) <= half && fabsf(y) <= 0.5f * q.hel) {
    int e = (int)floorf((x + half) / q.pitch);
    e = min(q.ne - 1, max(0, e));
    if (hit_better(t, prim_code(CLS_XDCR, e), tbest, cbest)) {
      tbest = t;
      cbest = prim_code(CLS_XDCR, (uint32_t)e);
    }
  }
}

__device__ __forceinline__ void leaf_closest(const SceneDev& S, int first, int count, float3 o, float3 w,
                                             uint32_t prev, float& tbest, uint32_t& cbest) {
  for (int i = first; i < first + count; ++i) {
    const float4 A = __ldg(&S.prims_t[3 * i]);
    const uint32_t code = __float_as_uint(A.w);
    if (code == prev) continue;
    const float4 B = __ldg(&S.prims_t[3 * i + 1]);
    const float4 C = __ldg(&S.prims_t[3 * i + 2]);
    const float t = tri_test(o, w, xyz(A), xyz(B), xyz(C));
    if (t > 0.0f && hit_better(t, code, tbest, cbest)) {
      tbest = t;
      cbest = code;
    }
  }
}

// closest triangle hit: BVH2 traversal, nearer child first; the far child is pushed with its
// entry distance and skipped once a closer hit has been found.  The stack holds at most one
// entry per tree level below the root, and us_scene_upload refuses trees deeper than 60, so it
// cannot fill up; should it ever, the far child is dropped and `overflow` is set so that the
// caller reports it (the hit may then be missed).
__device__ __forceinline__ void tri_closest(const SceneDev& S, float3 o, float3 w, uint32_t prev, float& tbest,
                                            uint32_t& cbest, bool& overflow) {
  const RayInv r = ray_inv(o, w);
  int stack[BVH_STACK];
  float stt[BVH_STACK];
  int sp = 0, node = 0;
  float node_t = 0.0f;
  while (true) {
    if (node_t <= tbest) {
      const float4 n0 = __ldg(&S.nodes_t[4 * node]);
      const float4 n1 = __ldg(&S.nodes_t[4 * node + 1]);
      const float4 n2 = __ldg(&S.nodes_t[4 * node + 2]);
      const int4 n3 = __ldg(reinterpret_cast<const int4*>(&S.nodes_t[4 * node + 3]));
      bool h0, h1;
      float t0, t1;
      node_boxes(r, n0, n1, n2, tbest, h0, h1, t0, t1);
      if (h0 && n3.z > 0) {
        leaf_closest(S, n3.x, n3.z, o, w, prev, tbest, cbest);
        h0 = false;
      }
      if (h1 && n3.w > 0) {
        leaf_closest(S, n3.y, n3.w, o, w, prev, tbest, cbest);
        h1 = false;
      }
      h0 = h0 && n3.x >= 0;
      h1 = h1 && n3.y >= 0;
      if (h0 && h1) {
        const bool first0 = t0 <= t1;
        if (sp < BVH_STACK) {
          stack[sp] = first0 ? n3.y : n3.x;
          stt[sp] = first0 ? t1 : t0;
          ++sp;
        } else {
          overflow = true;
        }
        node = first0 ? n3.x : n3.y;
        node_t = first0 ? t0 : t1;
        continue;
      }
      if (h0 || h1) {
        node = h0 ? n3.x : n3.y;
        node_t = h0 ? t0 : t1;
        continue;
      }
    }
    if (sp == 0) break;
    --sp;
    node = stack[sp];
    node_t = stt[sp];
  }
}

// closest hit over the transducer face and the triangles, excluding the primitive `prev` the
// ray leaves from; cbest = 0xFFFFFFFF when there is none.  The scatterers are searched after
// it (grid march) below the distance found here; the order (t, class, id) decides ties, so the
// result is the closest hit over the union whichever structure reports a candidate first.
__device__ __forceinline__ void surface_hit(const SceneDev& S, const Acq& q, float3 o, float3 w, uint32_t prev,
                                            float& tbest, uint32_t& cbest, bool& overflow) {
  tbest = 3.0e38f;
  cbest = 0xFFFFFFFFu;
  xdcr_test(q, o, w, tbest, cbest);
  tri_closest(S, o, w, prev, tbest, cbest, overflow);
}

// ---- 4-wide BVH (the secondary rays' all-crossings queries) ----------------------------
// Closest hits walk the binary tree: measured, the 4-wide one halved their node visits but was
// not faster (their cost is the scattered node reads, not the count); for all-crossings queries,
// which visit every node the segment overlaps, it is.  A node is 8 float4 (128 bytes): lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of its 4 children, then
// int4 child and int4 count (count > 0: a leaf of count triangles from child; count 0: an inner
// node, or an empty slot with child -1 and an inverted box).
struct Node4 {
  float4 lx, hx, ly, hy, lz, hz;
  int4 ch, cn;
};
__device__ __forceinline__ Node4 load_node4(const float4* nodes, int node) {
  const float4* p = nodes + 8 * node;
  Node4 n;
  n.lx = __ldg(p);
  n.hx = __ldg(p + 1);
  n.ly = __ldg(p + 2);
  n.hy = __ldg(p + 3);
  n.lz = __ldg(p + 4);
  n.hz = __ldg(p + 5);
  n.ch = __ldg(reinterpret_cast<const int4*>(p + 6));
  n.cn = __ldg(reinterpret_cast<const int4*>(p + 7));
  return n;
}
// slab test of one child box; entry distance returned, hit when entry <= exit (robust, as
// node_boxes)
__device__ __forceinline__ bool box_hit(const RayInv& r, float lx, float hx, float ly, float hy, float lz, float hz,
                                        float tlimit, float& tn) {
  const float ax = fmaf(lx, r.inv.x, -r.oi.x), bx = fmaf(hx, r.inv.x, -r.oi.x);
  const float ay = fmaf(ly, r.inv.y, -r.oi.y), by = fmaf(hy, r.inv.y, -r.oi.y);
  const float az = fmaf(lz, r.inv.z, -r.oi.z), bz = fmaf(hz, r.inv.z, -r.oi.z);
  const float lo = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.0f));
  const float hi = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), tlimit));
  tn = lo;
  return lo <= hi * 1.0000004f;
}
__device__ __forceinline__ void node4_boxes(const RayInv& r, const Node4& n, float tlimit, float* tn, bool* h) {
  h[0] = box_hit(r, n.lx.x, n.hx.x, n.ly.x, n.hy.x, n.lz.x, n.hz.x, tlimit, tn[0]);
  h[1] = box_hit(r, n.lx.y, n.hx.y, n.ly.y, n.hy.y, n.lz.y, n.hz.y, tlimit, tn[1]);
  h[2] = box_hit(r, n.lx.z, n.hx.z, n.ly.z, n.hy.z, n.lz.z, n.hz.z, tlimit, tn[2]);
  h[3] = box_hit(r, n.lx.w, n.hx.w, n.ly.w, n.hy.w, n.lz.w, n.hz.w, tlimit, tn[3]);
}
// all triangle crossings T_MIN < t < tmax of the segment o + t d (secondary rays), as a
// resumable traversal: xtrav_step visits one node of the 4-wide triangle BVH (testing the
// triangles of leaf children) and returns false once the traversal is complete; xtrav_finish sorts the
// crossings by t (ties by id) and returns their count, or -1 when more than MAX_XINGS were found.
struct XTrav {
  RayInv r;
  float tmax;
  int node, sp, n;
  bool overflow;
  uint32_t skip;  // a triangle the segment starts on (not a crossing), or 0xFFFFFFFF
};

__device__ __forceinline__ void xtrav_init(float3 o, float3 d, float tmax, XTrav& T, uint32_t skip = 0xFFFFFFFFu) {
  T.r = ray_inv(o, d);
  T.tmax = tmax;
  T.node = 0;
  T.sp = 0;
  T.n = 0;
  T.overflow = false;
  T.skip = skip;
}

__device__ __forceinline__ bool xtrav_step(const SceneDev& S, float3 o, float3 d, XTrav& T, int* stack, float* xt,
                                           uint32_t* xid) {
  const Node4 n = load_node4(S.nodes4, T.node);
  float tn[4];
  bool h[4];
  node4_boxes(T.r, n, T.tmax, tn, h);
  const int ch[4] = {n.ch.x, n.ch.y, n.ch.z, n.ch.w}, cn[4] = {n.cn.x, n.cn.y, n.cn.z, n.cn.w};
  int next = -1;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!h[c]) continue;
    if (cn[c] > 0) {
      for (int i = ch[c]; i < ch[c] + cn[c]; ++i) {
        const float4 A = __ldg(&S.prims_t[3 * i]);
        const uint32_t code = __float_as_uint(A.w);
        const float4 B = __ldg(&S.prims_t[3 * i + 1]);
        const float4 C = __ldg(&S.prims_t[3 * i + 2]);
        const float t = tri_test(o, d, xyz(A), xyz(B), xyz(C));
        if (t > 0.0f && t < T.tmax && code_id(code) != T.skip) {
          if (T.n < MAX_XINGS) {
            xt[T.n] = t;
            xid[T.n] = code_id(code);
            ++T.n;
          } else {
            T.overflow = true;
          }
        }
      }
    } else if (ch[c] >= 0) {
      if (next < 0) {
        next = ch[c];
      } else if (T.sp < BVH_STACK) {
        stack[T.sp++] = ch[c];
      }
    }
  }
  if (next >= 0) {
    T.node = next;
    return true;
  }
  if (T.sp == 0) return false;
  T.node = stack[--T.sp];
  return true;
}

__device__ __forceinline__ int xtrav_finish(const XTrav& T, float* xt, uint32_t* xid) {
  if (T.overflow) return -1;
  const int n = T.n;
  for (int i = 1; i < n; ++i) {  // insertion sort by t (ties by id)
    const float t = xt[i];
    const uint32_t id = xid[i];
    int j = i - 1;
    while (j >= 0 && (xt[j] > t || (xt[j] == t && xid[j] > id))) {
      xt[j + 1] = xt[j];
      xid[j + 1] = xid[j];
      --j;
    }
    xt[j + 1] = t;
    xid[j + 1] = id;
  }
  return n;
}

__device__ __forceinline__ int all_crossings(const SceneDev& S, float3 o, float3 d, float tmax, float* xt,
                                             uint32_t* xid, uint32_t skip = 0xFFFFFFFFu) {
  XTrav T;
  int stack[BVH_STACK];
  xtrav_init(o, d, tmax, T, skip);
  while (xtrav_step(S, o, d, T, stack, xt, xid)) {
  }
  return xtrav_finish(T, xt, xid);
}

// result of one secondary ray (Sec. 2.3.3)
struct NeeOut {
  bool ok;        // false: no contribution (directivity cutoff, TIR or overflow)
  bool overflow;
  float gain;     // prod T * exp(-kappa f0 sum alpha l) * f_rx * n_elem
  float sum_al;   // sum alpha_m l_m
  int n;          // crossings
};

__device__ __forceinline__ float elem_x(const Acq& q, int e) { return (e - 0.5f * (q.ne - 1)) * q.pitch; }

// secondary-ray geometry: unit direction d and length D from p to the centre of element e2;
// the receive directivity (Eq. cutoff) of that direction
__device__ __forceinline__ float nee_setup(const Acq& q, float3 p, int e2, float3& d, float& D) {
  const float3 tgt = f3(elem_x(q, e2), 0.0f, 0.0f);
  const float3 dv = tgt - p;
  D = sqrtf(dot3(dv, dv));
  d = dv * (1.0f / D);
  return f_rx(-d.z, q.alpha_m, q.alpha_c);
}

// weight of a secondary ray from its sorted crossings (n of them; -1: overflow): product of
// the transmission coefficients (zero under total internal reflection), attenuation and time
// per sub-segment in the medium tracked across the crossings
__device__ __forceinline__ NeeOut nee_shade(const SceneDev& S, const Media& med, const Acq& q, float3 d, float D,
                                            float frx, int n, int m_start, float& t_hi, float& t_lo, const float* xt,
                                            const uint32_t* xid) {
  NeeOut r;
  r.ok = false;
  r.overflow = false;
  r.gain = 0.0f;
  r.sum_al = 0.0f;
  r.n = 0;
  if (n < 0) {
    r.overflow = true;
    return r;
  }
  r.n = n;
  float prodT = 1.0f, sa = 0.0f, tprev = 0.0f;
  int m = m_start;
  for (int i = 0; i < n; ++i) {
    const float l = xt[i] - tprev;
    sa = fmaf(med.al[m], l, sa);
    ff_add(t_hi, t_lo, l / med.c[m]);
    const float4 nr = __ldg(&S.tri_nrm[xid[i]]);
    const uint32_t mm = __float_as_uint(nr.w);
    const float3 nn = xyz(nr);
    const float dn = dot3(d, nn);
    const int m1 = dn < 0.0f ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
    const int m2 = dn < 0.0f ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
    const float3 nin = dn < 0.0f ? nn : nn * -1.0f;
    const Iface f = iface(d, nin, med.c[m1], med.c[m2], med.rho[m1], med.rho[m2]);
    if (f.tir) return r;
    prodT *= f.T;
    m = m2;
    tprev = xt[i];
  }
  const float l = D - tprev;
  sa = fmaf(med.al[m], l, sa);
  ff_add(t_hi, t_lo, l / med.c[m]);
  r.sum_al = sa;
  r.gain = prodT * expf(-KAPPA_F * med.f0 * sa) * frx * (float)q.ne;
  r.ok = true;
  return r;
}

// secondary ray from a scatterer centre to element e (Sec. 2.3.3): straight segment, weight
// as in nee_shade, receive directivity (Eq. cutoff)
__device__ __forceinline__ NeeOut nee_eval(const SceneDev& S, const Media& med, const Acq& q, float3 p, int e2,
                                           int m_start, float& t_hi, float& t_lo, float* xt, uint32_t* xid,
                                           float3* dir_out, float* D_out, uint32_t skip = 0xFFFFFFFFu) {
  float3 d;
  float D;
  const float frx = nee_setup(q, p, e2, d, D);
  if (dir_out) *dir_out = d;
  if (D_out) *D_out = D;
  if (frx == 0.0f) {
    NeeOut r;
    r.ok = false;
    r.overflow = false;
    r.gain = 0.0f;
    r.sum_al = 0.0f;
    r.n = 0;
    return r;
  }
  const int n = all_crossings(S, p, d, D, xt, xid, skip);
  return nee_shade(S, med, q, d, D, frx, n, m_start, t_hi, t_lo, xt, xid);
}

}  // namespace usrt
