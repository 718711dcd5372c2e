// Wavefront transport kernels (Sec. 2.3.1-2.3.3): generate, traverse, interact, secondary rays.
//
// Every kernel is a grid-stride loop whose trip count is read from a device counter written by
// the previous kernel, so a whole forward pass is a fixed launch sequence (no host round trip,
// capturable in a CUDA graph).  Live paths are compacted after every interaction with
// warp-aggregated appends (one atomic per coalesced group).
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "bvh_query.cuh"
#include "splat.cuh"
#include "transport.cuh"

namespace cg = cooperative_groups;

namespace usrt {

// one atomic per group of coalesced lanes; returns this lane's slot
__device__ __forceinline__ uint32_t append_slot(uint32_t* counter) {
  cg::coalesced_group g = cg::coalesced_threads();
  uint32_t base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (uint32_t)g.size());
  base = g.shfl(base, 0);
  return base + g.thread_rank();
}

__device__ __forceinline__ void path_tx_ray(const Acq& q, long long path, int& tx, uint32_t& ray) {
  tx = (int)(path / q.rays_per_tx);
  const long long local = path - (long long)tx * q.rays_per_tx;
  ray = (uint32_t)(q.tx_elem < 0 ? local : (long long)q.tx_elem * q.nr + local);
}

// coherence-sort key of a ray (RaySort): origin cell and direction bin; rays that carry their
// surface hit go to the coarser buckets after RAY_KEY_BUCKETS
__device__ __forceinline__ uint32_t ray_key(const RaySort& rs, float3 o, float3 w, bool carried) {
  // origin: 8 x 8 cells over the scene's x and z extent
  const int cx = min(7, max(0, (int)((o.x - rs.lo.x) * rs.inv_ext.x * 8.0f)));
  const int cz = min(7, max(0, (int)((o.z - rs.lo.z) * rs.inv_ext.z * 8.0f)));
  // direction: octahedral map of the unit sphere onto [-1, 1]^2, 16 x 16 bins
  const float l1 = fabsf(w.x) + fabsf(w.y) + fabsf(w.z);
  float u = w.x / l1, v = w.y / l1;
  if (w.z < 0.0f) {
    const float uu = (1.0f - fabsf(v)) * copysignf(1.0f, u);
    const float vv = (1.0f - fabsf(u)) * copysignf(1.0f, v);
    u = uu;
    v = vv;
  }
  const int bu = min(15, max(0, (int)((u + 1.0f) * 8.0f)));
  const int bv = min(15, max(0, (int)((v + 1.0f) * 8.0f)));
  if (carried)  // 4 x 4 origin cells, 8 x 8 direction bins, after the rays that need a query
    return (uint32_t)RAY_KEY_BUCKETS + (uint32_t)(((((cz >> 1) << 2) | (cx >> 1)) << 6) | ((bu >> 1) << 3) | (bv >> 1));
  return (uint32_t)((((cz << 3) | cx) << 8) | (bu << 4) | bv);
}

// the interaction kernel keys each ray it appends for the next round's coherence sort and
// counts it: one atomic per key among the lanes appending together
__device__ __forceinline__ void ray_key_count(const RaySort& rs, uint32_t slot, float3 o, float3 w, bool carried) {
  const uint32_t key = ray_key(rs, o, w, carried);
  rs.key[slot] = key;
  const uint32_t peers = __match_any_sync(__activemask(), key);
  if ((int)(threadIdx.x & 31u) == __ffs(peers) - 1) atomicAdd(&rs.cnt[key], (uint32_t)__popc(peers));
}

// ------------------------------------------------------------------------------------------
// Emission (Sec. 2.3.1, Eq. directivity, Eq. pressure_mc): origin uniform over the element
// face, cosine-weighted direction (f_d / p = pi), weight pi / N_r, steering delay as a time
// stamp tau_tx = (x_e sin(theta) + W/2 |sin(theta)|) / c_bf.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void emit_path(const Acq& q, long long path, float3& o0, float3& w0, float& tau0) {
  int tx;
  uint32_t ray;
  path_tx_ray(q, path, tx, ray);
  const uint4 u = philox4x32_10(make_uint4(ray, (uint32_t)tx, q.stream, 0u), make_uint2(q.key0, q.key1));
  const int e = (int)(ray / (uint32_t)q.nr);
  const float xe = (e - 0.5f * (q.ne - 1)) * q.pitch;
  const float u0 = u01(u.x), u1 = u01(u.y), u2 = u01(u.z), u3 = u01(u.w);
  const float r = sqrtf(u2);
  float sp, cp;
  sincospif(2.0f * u3, &sp, &cp);
  const float st = q.sin_tx[tx];
  tau0 = (xe * st + 0.5f * (q.ne - 1) * q.pitch * fabsf(st)) / q.cbf;
  o0 = f3(xe + (u0 - 0.5f) * q.pitch, (u1 - 0.5f) * q.hel, 0.0f);
  w0 = f3(r * cp, r * sp, sqrtf(1.0f - u2));
}
// The emitted rays go straight into coherence-sorted order: this pass counts their sort keys
// (they share few, all starting on the probe face, so the block counts in shared memory and adds
// the nonzero counts once) and keeps each ray's key; k_generate_sorted emits them again, after
// the scan of the counts, into the slots their kept keys give.  Recomputing an emission costs
// less than writing a ray and moving it.
constexpr int GEN_THREADS = 512;
__global__ void __launch_bounds__(GEN_THREADS) k_generate_count(TransportArgs A, long long path0, uint32_t n) {
  extern __shared__ uint32_t gen_h[];  // [RAY_BUCKETS]
  for (int b = threadIdx.x; b < RAY_BUCKETS; b += blockDim.x) gen_h[b] = 0u;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float3 o0, w0;
    float tau0;
    emit_path(A.acq, path0 + i, o0, w0, tau0);
    const uint32_t key = ray_key(A.rk, o0, w0, false);
    A.rk.key[i] = key;  // the second pass takes the key from here, so that both passes agree
    atomicAdd(&gen_h[key], 1u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) A.cnt->live[0] = n;
  __syncthreads();
  for (int b = threadIdx.x; b < RAY_BUCKETS; b += blockDim.x)
    if (gen_h[b]) atomicAdd(&A.rk.cnt[b], gen_h[b]);
}

// ------------------------------------------------------------------------------------------
// Closest surface hit (transducer face, triangle BVH) of every live path, one ray per thread,
// grid-stride.  The lanes of a warp start their rays at the root together, so the upper levels
// of the BVH are fetched once per warp.  The scatterers are searched next by k_march below the
// distance written here.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(TRAV_THREADS) k_traverse(TransportArgs A) {
  if (blockIdx.x == 0 && threadIdx.x == 0)  // secondary jobs of this round follow the previous rounds'
    A.cnt->nee_off[A.k] = A.k ? A.cnt->nee_off[A.k - 1] + A.cnt->nee[A.k - 1] : 0u;
  const uint32_t n = *A.trav_n;  // the rest of the queue carries its surface hit
  bool overflow = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 pa = A.qin.pa[i];
    const float4 wt = A.qin.wt[i];
    const uint32_t prev = A.qin.meta[i].y;
    float t;
    uint32_t c;
    surface_hit(A.S, A.acq, xyz(pa), xyz(wt), prev, t, c, overflow);
    A.hits[i] = make_float2(t, __uint_as_float(c == 0xFFFFFFFFu ? prim_code(CLS_NONE, 0) : c));
  }
  if (overflow) atomicOr(&A.cnt->status, ST_OVERFLOW);
}

// ------------------------------------------------------------------------------------------
// Closest scatterer event of every live path before its surface hit: a 3D DDA through the
// uniform sphere grid, cells in the order the ray crosses them.  Every sphere whose
// closest-approach point lies on the ray at parameter t is listed in the cell holding that
// point, and that cell is entered at a parameter <= t, so a ray stops at the first cell it
// would enter beyond its best hit.  Cell faces are computed from the grid origin at every step
// (no accumulated increments).
//
// Path lengths to the first event are spread roughly exponentially, so with one ray per thread
// a warp would run as long as its longest ray with most lanes idle.  Instead every loop
// iteration does the same work in every lane: enter one cell, test the two entries its 32-byte
// record holds inline, step the DDA and read the next cell's record (entries past the second,
// in crowded cells, take one iteration each).  Lanes whose rays have finished take the next
// rays, once MARCH_REFILL_MIN of them wait, from a pool the warp claims in chunks of MARCH_CHUNK
// consecutive (coherence-sorted) queue slots.
// ------------------------------------------------------------------------------------------
constexpr int MARCH_CHUNK = 64;
constexpr int MARCH_REFILL_MIN = 8;

__global__ void __launch_bounds__(MARCH_THREADS) k_march(TransportArgs A) {
  const SceneDev& S = A.S;
  const uint32_t n = A.cnt->live[A.k];
  if (S.n_scat == 0 || n == 0) return;
  uint32_t* claim = &A.cnt->march[A.k];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  const float h = S.gh, inv_h = 1.0f / h;
  const float3 lo = S.glo;
  const int nx = S.gnx, ny = S.gny, nz = S.gnz;
  const int dy = nx, dz = nx * ny;
  // lane state
  uint32_t ray = 0xFFFFFFFFu;  // queue slot of the current ray; none when 0xFFFFFFFF
  float3 o = f3(0.0f, 0.0f, 0.0f), w = o;
  float ix = 0.0f, iy = 0.0f, iz = 0.0f, tnx = 0.0f, tny = 0.0f, tnz = 0.0f, tbest = 0.0f, t0hit = 0.0f;
  uint32_t prev = 0u, cbest = 0u, code0 = 0u, e = 0u, e_end = 0u;
  int cx = 0, cy = 0, cz = 0, idx = 0, sx = 1, sy = 1, sz = 1, ux = 0, uy = 0, uz = 0;
  // The DDA runs one cell ahead: (cx, cy, cz, idx) is the next cell to enter, at t_ahead, and
  // its inline record (first two entries) is read as soon as the DDA gets there, so the read has
  // an iteration to arrive.  It is read only while t_ahead <= tbest; tbest only decreases, so a
  // record not read is a record never needed.
  float t_ahead = 0.0f;
  bool ahead_ok = false;
  float4 slot_a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), slot_b = slot_a;
  auto fetch_ahead = [&]() {
    if (ahead_ok && t_ahead <= tbest) {
      slot_a = __ldg(&S.cell2[2 * idx]);
      slot_b = __ldg(&S.cell2[2 * idx + 1]);
    } else {
      slot_a.w = slot_b.w = 0.0f;
    }
  };
  auto step_ahead = [&]() {
    if (tnx <= tny && tnx <= tnz) {
      t_ahead = tnx;
      cx += sx;
      idx += sx;
      ahead_ok = (unsigned)cx < (unsigned)nx;
      tnx = (fmaf((float)(cx + ux), h, lo.x) - o.x) * ix;
    } else if (tny <= tnz) {
      t_ahead = tny;
      cy += sy;
      idx += sy * dy;
      ahead_ok = (unsigned)cy < (unsigned)ny;
      tny = (fmaf((float)(cy + uy), h, lo.y) - o.y) * iy;
    } else {
      t_ahead = tnz;
      cz += sz;
      idx += sz * dz;
      ahead_ok = (unsigned)cz < (unsigned)nz;
      tnz = (fmaf((float)(cz + uz), h, lo.z) - o.z) * iz;
    }
    fetch_ahead();
  };
  auto test = [&](float4 sp) {
    const uint32_t code = __float_as_uint(sp.w) & 0x7FFFFFFFu;
    const float t = code == 0u || code == prev ? -1.0f : scat_test(o, w, xyz(sp), S.rs2);
    if (t > 0.0f && hit_better(t, code, tbest, cbest)) {
      tbest = t;
      cbest = code;
    }
  };
  uint32_t pool = 0u, pool_end = 0u;  // warp-uniform
  bool exhausted = false;             // warp-uniform
  while (true) {
    // hand the pool's rays to idle lanes once MARCH_REFILL_MIN of them wait, so that the setup
    // of new rays runs on many lanes at once; rays that miss the grid leave their lane idle
    uint32_t idle = __ballot_sync(0xFFFFFFFFu, ray == 0xFFFFFFFFu);
    if (__popc(idle) < MARCH_REFILL_MIN) idle = 0u;
    while (idle && !exhausted) {
      if (pool == pool_end) {
        uint32_t b = 0u;
        if (lane == 0) b = atomicAdd(claim, (uint32_t)MARCH_CHUNK);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (b >= n) {
          exhausted = true;
          break;
        }
        pool = b;
        pool_end = min(b + (uint32_t)MARCH_CHUNK, n);
      }
      const uint32_t take = min((uint32_t)__popc(idle), pool_end - pool);
      const uint32_t rank = __popc(idle & below);
      if (((idle >> lane) & 1u) && rank < take) {
        ray = pool + rank;
        const float4 pa = A.qin.pa[ray];
        const float4 wt = A.qin.wt[ray];
        const float2 hit = A.hits[ray];
        o = xyz(pa);
        w = xyz(wt);
        prev = A.qin.meta[ray].y;
        tbest = t0hit = hit.x;
        cbest = code0 = __float_as_uint(hit.y);
        ix = safe_inv(w.x);
        iy = safe_inv(w.y);
        iz = safe_inv(w.z);
        const float ax = (lo.x - o.x) * ix, bx = (fmaf((float)nx, h, lo.x) - o.x) * ix;
        const float ay = (lo.y - o.y) * iy, by = (fmaf((float)ny, h, lo.y) - o.y) * iy;
        const float az = (lo.z - o.z) * iz, bz = (fmaf((float)nz, h, lo.z) - o.z) * iz;
        const float t0 = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.0f));
        const float t1 = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), tbest));
        if (t0 > t1) {
          ray = 0xFFFFFFFFu;  // misses the grid before its surface hit: nothing to do
        } else {
          cx = min(nx - 1, max(0, (int)floorf((fmaf(w.x, t0, o.x) - lo.x) * inv_h)));
          cy = min(ny - 1, max(0, (int)floorf((fmaf(w.y, t0, o.y) - lo.y) * inv_h)));
          cz = min(nz - 1, max(0, (int)floorf((fmaf(w.z, t0, o.z) - lo.z) * inv_h)));
          sx = w.x > 0.0f ? 1 : -1;
          sy = w.y > 0.0f ? 1 : -1;
          sz = w.z > 0.0f ? 1 : -1;
          ux = w.x > 0.0f;
          uy = w.y > 0.0f;
          uz = w.z > 0.0f;
          tnx = w.x == 0.0f ? 3.0e38f : (fmaf((float)(cx + ux), h, lo.x) - o.x) * ix;
          tny = w.y == 0.0f ? 3.0e38f : (fmaf((float)(cy + uy), h, lo.y) - o.y) * iy;
          tnz = w.z == 0.0f ? 3.0e38f : (fmaf((float)(cz + uz), h, lo.z) - o.z) * iz;
          idx = (cz * ny + cy) * nx + cx;
          t_ahead = t0;  // the first cell is the one ahead
          ahead_ok = true;
          e = e_end = 0u;
          fetch_ahead();
        }
      }
      pool += take;
      idle = __ballot_sync(0xFFFFFFFFu, ray == 0xFFFFFFFFu);
    }
    if (__all_sync(0xFFFFFFFFu, ray == 0xFFFFFFFFu)) break;  // pool exhausted, every lane idle
    if (ray == 0xFFFFFFFFu) continue;
    if (e < e_end) {  // entries past the first two of a crowded cell
      test(__ldg(&S.cell_sph[e]));
      ++e;
      continue;
    }
    if (!(ahead_ok && t_ahead <= tbest)) {  // no cell left to enter below tbest: done
      if (cbest != code0) {  // a scatterer comes first; its pass-through carries the surface hit on
        A.keep[ray] = make_float2(t0hit, __uint_as_float(code0));  // the hit this ray came with
        A.hits[ray] = make_float2(tbest, __uint_as_float(cbest));
      }
      ray = 0xFFFFFFFFu;
      continue;
    }
    // enter the cell ahead: test its inline entries, then step the DDA past it
    const float4 a = slot_a, b = slot_b;
    const int cell = idx;
    test(a);
    test(b);
    if (__float_as_uint(b.w) >> 31) {
      const uint32_t word = __ldg(&S.cell[cell]);
      e = (word >> 8) + 2u;
      e_end = (word >> 8) + (word & 0xFFu);
    }
    step_ahead();
  }
}

// ------------------------------------------------------------------------------------------
// Interaction: attenuation and travel time over the segment, then the event at its end:
// transducer arrival, interface split (Fresnel / Snell, Sec. 2.3.2), or a scatterer (queue a
// secondary ray, pass through).  Survivors are compacted into the output queue.
// ------------------------------------------------------------------------------------------
// What the interaction of one queue slot emits: the surviving ray, a secondary-ray job, an
// arrival (each at most once).  The kernel appends a block's emissions with one atomic per
// counter: per-warp atomics on the three queue counters, which every warp of the grid shares,
// are serialised in the L2 (2.46 -> 2.01 ms per frame with three blocks of 256 per SM, their
// registers capped at 80).
struct Emit {
  bool ray, job, arr;
  uint32_t path;   // the slot's path id
  float4 pa, wt;   // the surviving ray
  uint4 meta;
  float2 surf, mis;
  float4 job4;     // the job: (a, tau_hi, tau_lo, bits(job id word)), medium | element << 8 | ...
  uint32_t jm;
  float3 jx, jw;   // a rough event's point and incident direction
  uint4 arr4;      // the arrival
};
__device__ __forceinline__ void interact_one(const TransportArgs& A, uint32_t i, Emit& E) {
  const Acq& q = A.acq;
  const Media& med = A.med;
  const int K1 = q.kmax + 1;
  const float2 h = A.hits[i];
  const uint32_t code = __float_as_uint(h.y);
  const uint32_t cls = code_cls(code);
  const uint4 meta = A.qin.meta[i];
  const float4 pa = A.qin.pa[i];  // read with the slot's other words, before the escape test
  const float4 wt = A.qin.wt[i];
  const float2 ks = A.keep[i];  // used at scatterer events; read with the rest, not after the hit's class
  const long long path = meta.x;
  E.path = meta.x;
  uint32_t* rec = A.record ? &A.record[(size_t)(path - A.path_base) * K1 + A.k] : nullptr;
  if (cls == CLS_NONE) {  // escape
    if (rec) *rec = 0u;
    return;
  }
  float2 mis = A.mis_on ? A.qin.mis[i] : make_float2(0.0f, 0.0f);
  int m = (int)(meta.z & 0xFF);
  float tau_lo = __uint_as_float(meta.w);
  const float t = h.x;
  float3 w = xyz(wt);
  float a = pa.w * expf(-KAPPA_F * med.al[m] * med.f0 * t);
  float tau_hi = wt.w;
  ff_add(tau_hi, tau_lo, t / med.c[m]);
  const float3 x = xyz(pa) + w * t;
  int tx;
  uint32_t ray;
  path_tx_ray(q, path, tx, ray);
  if (cls == CLS_XDCR) {  // arrival at the receiving element (Sec. 2.3.4)
    if (rec) *rec = code;
    float frx = f_rx(-w.z, q.alpha_m, q.alpha_c);
    // straight on from a rough event: balance weight against that event's secondary ray
    if (mis.x > 0.0f) frx *= rough_hit_weight(q, mis.x, mis.y + t, w);
    if (frx > 0.0f && A.arr) {
      const uint32_t tq = time_to_tq(tau_hi, tau_lo, q.fs);
      if (tq != 0xFFFFFFFFu) {
        E.arr = true;
        E.arr4 = make_uint4((uint32_t)(tx * q.ne) + code_id(code), tq, __float_as_uint(a * frx), (uint32_t)path);
      }
    }
    return;
  }
  if (A.k == q.kmax) {  // interaction budget spent
    if (rec) *rec = code;
    return;
  }
  const uint4 u = philox4x32_10(make_uint4(ray, (uint32_t)tx, q.stream, (uint32_t)(A.k + 1)),
                                make_uint2(q.key0, q.key1));
  uint32_t word = code;
  if (cls == CLS_TRI) {
    const float4 nr = __ldg(&A.S.tri_nrm[code_id(code)]);
    const uint32_t mm = __float_as_uint(nr.w);
    const float3 nn = xyz(nr);
    const bool front = dot3(w, nn) < 0.0f;
    const float3 nin = front ? nn : nn * -1.0f;
    const int m1 = front ? (int)(mm & 0xFFFF) : (int)(mm >> 16);
    const int m2 = front ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
    // facet normal: the macro normal, or a GGX microfacet normal (roughness of the medium the
    // triangle bounds, its back side)
    const float alpha = med.rough[mm >> 16];
    float3 fn = nin;
    if (alpha > 0.0f && q.rough_nee) {  // secondary ray to a uniformly chosen element (Sec. 2.3.3)
      const int e2 = min(q.ne - 1, (int)floorf(u01(u.y) * (float)q.ne));
      word |= (uint32_t)e2 << 24;
      E.job = true;
      E.job4 = make_float4(a, tau_hi, tau_lo, __uint_as_float(code_id(code) | NEE_ROUGH));
      E.jm = (uint32_t)m1 | ((uint32_t)e2 << 8) | ((uint32_t)tx << 16) | ((uint32_t)A.k << 24);
      E.jx = x;
      E.jw = w;
    }
    if (alpha > 0.0f) {
      fn = ggx_sample(nin, alpha, u01(u.z), u01(u.w)).h;
      if (dot3(w, fn) >= 0.0f) {  // facet met from behind: the path ends here
        if (rec) {
          *rec = word;
          rec[1] = 0u;
        }
        return;
      }
    }
    const float3 w_in = w;
    const Iface f = iface(w, fn, med.c[m1], med.c[m2], med.rho[m1], med.rho[m2]);
    uint32_t choice;
    if (f.tir) {
      choice = CH_TIR;
    } else {
      const float pr = q.split_mode == 0 ? f.R * f.R : q.split_q;
      choice = u01(u.x) < pr ? CH_REFLECT : CH_TRANSMIT;
    }
    if (choice == CH_TIR) {
      w = w + fn * (2.0f * f.ci);
      m = m1;
    } else if (choice == CH_REFLECT) {
      const float pr = q.split_mode == 0 ? f.R * f.R : q.split_q;
      a = a * (f.R / pr);
      w = w + fn * (2.0f * f.ci);
      m = m1;
    } else {
      const float pr = q.split_mode == 0 ? f.R * f.R : q.split_q;
      a = a * (f.T / (1.0f - pr));
      w = w * f.r + fn * (f.r * f.ci - f.ct);
      m = m2;
    }
    word |= choice << 22;
    if (alpha > 0.0f) {
      const float on = dot3(w, nin), inn = dot3(w_in, nin);
      if ((m == m1) != (on > 0.0f)) {  // outgoing direction on the wrong side: the path ends
        if (rec) {
          *rec = word;
          rec[1] = 0u;
        }
        return;
      }
      a *= -dot3(w_in, fn) * smith_g1(inn, alpha) * smith_g1(on, alpha) / (-inn * dot3(fn, nin));
      if (A.mis_on) mis = make_float2(rough_bsdf_pdf(q, med, w_in, w, fn, nin, m1, m2, alpha, f, choice == CH_TRANSMIT), 0.0f);
    } else {
      mis = make_float2(0.0f, 0.0f);
    }
  } else {  // scatterer: secondary ray to a uniformly chosen element; Born pass-through
    mis.y += t;  // straight on: still the last rough event's direction
    const int e2 = min(q.ne - 1, (int)floorf(u01(u.y) * (float)q.ne));
    word |= (uint32_t)e2 << 24;
    E.job = true;
    E.job4 = make_float4(a, tau_hi, tau_lo, __uint_as_float(code_id(code)));
    E.jm = (uint32_t)m | ((uint32_t)e2 << 8) | ((uint32_t)tx << 16) | ((uint32_t)A.k << 24);
  }
  if (rec) *rec = word;
  // past a scatterer the ray goes on unchanged, so the surface hit found this round is the
  // next one: it is carried, at its distance from the new origin, unless it lies within the
  // minimum hit distance (a fresh query would pass over it)
  float2 carry = make_float2(-1.0f, 0.0f);
  if (cls == CLS_SCAT) {
    const float t_rem = ks.x - t;
    if (t_rem > 2.0f * T_MIN) carry = make_float2(t_rem, ks.y);
  }
  E.ray = true;
  E.pa = make_float4(x.x, x.y, x.z, a);
  E.wt = make_float4(w.x, w.y, w.z, tau_hi);
  E.meta = make_uint4(meta.x, code, (uint32_t)m | ((uint32_t)(A.k + 1) << 8), __float_as_uint(tau_lo));
  E.surf = carry;
  E.mis = mis;
}

constexpr int IA_THREADS = 256, IA_WARPS = IA_THREADS / 32;
__global__ void __launch_bounds__(IA_THREADS, 3) k_interact(TransportArgs A) {
  __shared__ uint32_t s_pre[3][IA_WARPS];  // per warp: emissions, then the warp's first offset
  __shared__ uint32_t s_base[3];           // the block's first slot per counter
  const uint32_t n = A.cnt->live[A.k];
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (uint32_t b0 = blockIdx.x * IA_THREADS; b0 < n; b0 += gridDim.x * IA_THREADS) {  // block-uniform
    const uint32_t i = b0 + threadIdx.x;
    Emit E;
    E.ray = E.job = E.arr = false;
    if (i < n) interact_one(A, i, E);
    const unsigned mr = __ballot_sync(0xFFFFFFFFu, E.ray);
    const unsigned mj = __ballot_sync(0xFFFFFFFFu, E.job);
    const unsigned ma = __ballot_sync(0xFFFFFFFFu, E.arr);
    if (lane == 0) {
      s_pre[0][wid] = __popc(mr);
      s_pre[1][wid] = __popc(mj);
      s_pre[2][wid] = __popc(ma);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      const int c = threadIdx.x;
      uint32_t run = 0u;
      for (int w = 0; w < IA_WARPS; ++w) {
        const uint32_t v = s_pre[c][w];
        s_pre[c][w] = run;
        run += v;
      }
      uint32_t* ctr = c == 0 ? &A.cnt->live[A.k + 1] : (c == 1 ? &A.cnt->nee[A.k] : &A.cnt->n_arr);
      s_base[c] = run ? atomicAdd(ctr, run) : 0u;
    }
    __syncthreads();
    if (E.ray) {
      const uint32_t o = s_base[0] + s_pre[0][wid] + __popc(mr & below);
      A.qout.pa[o] = E.pa;
      A.qout.wt[o] = E.wt;
      A.qout.meta[o] = E.meta;
      A.qout.surf[o] = E.surf;
      if (A.mis_on) A.qout.mis[o] = E.mis;
      ray_key_count(A.rk, o, xyz(E.pa), xyz(E.wt), E.surf.x >= 0.0f);
    }
    if (E.job) {
      const uint32_t slot = A.cnt->nee_off[A.k] + s_base[1] + s_pre[1][wid] + __popc(mj & below);
      A.nee.job[slot] = E.job4;
      A.nee.jm[slot] = E.jm;
      A.nee.jpath[slot] = E.path;
      if (__float_as_uint(E.job4.w) & NEE_ROUGH) {
        A.nee.jx[slot] = make_float4(E.jx.x, E.jx.y, E.jx.z, 0.0f);
        A.nee.jw[slot] = make_float4(E.jw.x, E.jw.y, E.jw.z, 0.0f);
      }
    }
    if (E.arr) {
      const uint32_t slot = s_base[2] + s_pre[2][wid] + __popc(ma & below);
      if (slot < A.arr_cap) A.arr[slot] = E.arr4;
    }
    __syncthreads();  // s_pre and s_base are rewritten by the next iteration
  }
}

// ------------------------------------------------------------------------------------------
// Secondary rays of the scatterer events of segment k (Sec. 2.3.3)
//
// The lengths of the all-crossings traversals differ a lot within a warp, so lanes are refilled:
// a lane whose traversal is complete waits until at most NEE_REFILL_AT lanes of its warp still
// trace, then every waiting lane weighs its ray (nee_shade), stores and appends the arrival
// together, and takes the next job from a pool the warp claims in chunks of NEE_CHUNK
// consecutive (sorted) job slots.  Jobs the receive directivity cuts off finish at the claim.
// ------------------------------------------------------------------------------------------
constexpr int NEE_CHUNK = 64;
constexpr int NEE_REFILL_AT = 16;

__device__ __forceinline__ void nee_store(const TransportArgs& A, uint32_t i, const NeeOut& r, float th, float tl,
                                          const float* xt, const uint32_t* xid) {
  uint2 xo = make_uint2(0u, NEE_NONE);
  if (r.ok) {
    cg::coalesced_group g = cg::coalesced_threads();
    const uint32_t before = cg::exclusive_scan(g, (uint32_t)r.n);
    unsigned long long base = 0ull;
    if (g.thread_rank() == g.size() - 1) base = atomicAdd(&A.cnt->n_xing, (unsigned long long)(before + r.n));
    base = g.shfl(base, g.size() - 1) + before;
    if (base + (unsigned)r.n <= A.nres.xcap) {
      for (int c = 0; c < r.n; ++c) A.nres.xing[base + c] = make_uint2(__float_as_uint(xt[c]), xid[c]);
      xo = make_uint2((uint32_t)base, (uint32_t)r.n);
    } else {
      xo = make_uint2(0u, NEE_UNSTORED);
    }
    A.nres.res[i] = make_float4(th, tl, r.gain, r.sum_al);
  }
  A.nres.xo[i] = xo;
}

__global__ void __launch_bounds__(NEE_THREADS) k_nee(TransportArgs A) {
  const Acq& q = A.acq;
  const Media& med = A.med;
  const uint32_t n = A.cnt->nee[A.k];
  const uint32_t off = A.cnt->nee_off[A.k];
  if (n == 0) return;
  uint32_t* claim = &A.cnt->nee_claim[A.k];
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  float xt[MAX_XINGS];
  uint32_t xid[MAX_XINGS];
  int stack[BVH_STACK];
  uint32_t job = 0xFFFFFFFFu;  // job slot (from off) of this lane; none when 0xFFFFFFFF
  bool tracing = false;
  float3 p = f3(0.0f, 0.0f, 0.0f), d = p;
  float D = 0.0f, frx = 0.0f;
  float jfac = 0.0f;  // a rough event's BSDF factor (its medium in m_start); unused at scatterers
  int m_start = 0;
  XTrav T;
  xtrav_init(p, f3(0.0f, 0.0f, 1.0f), 0.0f, T);
  uint32_t pool = 0u, pool_end = 0u;  // warp-uniform
  bool exhausted = false;             // warp-uniform
  while (true) {
    uint32_t idle = __ballot_sync(0xFFFFFFFFu, job == 0xFFFFFFFFu);
    while (idle && !exhausted) {
      if (pool == pool_end) {
        uint32_t b = 0u;
        if (lane == 0) b = atomicAdd(claim, (uint32_t)NEE_CHUNK);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (b >= n) {
          exhausted = true;
          break;
        }
        pool = b;
        pool_end = min(b + (uint32_t)NEE_CHUNK, n);
      }
      const uint32_t take = min((uint32_t)__popc(idle), pool_end - pool);
      const uint32_t rank = __popc(idle & below);
      if (((idle >> lane) & 1u) && rank < take) {
        job = pool + rank;
        const uint32_t jm = A.nee.jm[off + job];
        const uint32_t jid = __float_as_uint(A.nee.job[off + job].w);
        const bool rough = (jid & NEE_ROUGH) != 0u;
        p = rough ? xyz(A.nee.jx[off + job]) : xyz(__ldg(&A.S.scat[jid]));
        frx = nee_setup(q, p, (int)((jm >> 8) & 0xFF), d, D);
        m_start = (int)(jm & 0xFF);
        if (rough && frx != 0.0f) {  // the microfacet BSDF toward the element
          const uint32_t tri = jid & ~NEE_ROUGH;
          const float4 nr = __ldg(&A.S.tri_nrm[tri]);
          const uint32_t mm = __float_as_uint(nr.w);
          const float3 wi = xyz(A.nee.jw[off + job]);
          const bool front = dot3(wi, xyz(nr)) < 0.0f;
          const float3 nin = front ? xyz(nr) : xyz(nr) * -1.0f;
          const int m2 = front ? (int)(mm >> 16) : (int)(mm & 0xFFFF);
          if (!rough_nee_factor(q, med, wi, nin, m_start, m2, med.rough[mm >> 16], d, D * D, jfac, m_start)) frx = 0.0f;
        }
        if (frx == 0.0f) {  // cut off: no contribution
          if (A.nres.res) A.nres.xo[off + job] = make_uint2(0u, NEE_NONE);
          job = 0xFFFFFFFFu;
        } else {
          xtrav_init(p, d, D, T, rough ? (jid & ~NEE_ROUGH) : 0xFFFFFFFFu);
          tracing = true;
        }
      }
      pool += take;
      idle = __ballot_sync(0xFFFFFFFFu, job == 0xFFFFFFFFu);
    }
    if (__all_sync(0xFFFFFFFFu, job == 0xFFFFFFFFu)) break;
    // trace until at most NEE_REFILL_AT lanes still trace (until none, once the pool is empty)
    while (true) {
      const int still = __popc(__ballot_sync(0xFFFFFFFFu, tracing));
      if (still == 0 || (!exhausted && still <= NEE_REFILL_AT)) break;
      if (tracing) tracing = xtrav_step(A.S, p, d, T, stack, xt, xid);
    }
    if (job == 0xFFFFFFFFu || tracing) continue;
    // weigh the finished rays, keep them for the adjoint, append their arrivals
    const uint32_t i = off + job;
    job = 0xFFFFFFFFu;
    const float4 jb = A.nee.job[i];
    const uint32_t jm = A.nee.jm[i];
    const int e2 = (int)((jm >> 8) & 0xFF), tx = (int)((jm >> 16) & 0xFF);
    const uint32_t jid = __float_as_uint(jb.w);
    float th = jb.y, tl = jb.z;
    const NeeOut r = nee_shade(A.S, med, q, d, D, frx, xtrav_finish(T, xt, xid), m_start, th, tl, xt, xid);
    if (A.nres.res) nee_store(A, i, r, th, tl, xt, xid);
    if (r.overflow) {
      atomicOr(&A.cnt->status, ST_OVERFLOW);
      atomicAdd(&A.cnt->dropped, 1u);
      continue;
    }
    if (!r.ok || !A.arr) continue;
    const uint32_t tq = time_to_tq(th, tl, q.fs);
    if (tq == 0xFFFFFFFFu) continue;
    const float amp = jb.x * ((jid & NEE_ROUGH) ? jfac : med.As * __ldg(&A.S.scat[jid]).w) * r.gain;
    const uint32_t slot = append_slot(&A.cnt->n_arr);
    if (slot < A.arr_cap) A.arr[slot] = make_uint4((uint32_t)(tx * q.ne + e2), tq, __float_as_uint(amp), A.nee.jpath[i]);
  }
}

// ------------------------------------------------------------------------------------------
// Coherence sort of a ray queue (one counting-sort pass over the keys ray_key gave the rays)
// ------------------------------------------------------------------------------------------

constexpr int RS_THREADS = 512;
constexpr int JOB_BUCKETS = 4096;  // <= RAY_BUCKETS (the job sort's scratch is sized as the ray sort's)
// items per thread and chunk, measured: 1024-ray chunks for the rays (512: +0.25 ms of sort per
// frame, 2048: +0.12 ms, 8192: +0.5 ms), 2048-job chunks for the jobs
constexpr int RAY_PER = 2, RS_PER = 4;
constexpr int RAY_CH = RS_THREADS * RAY_PER, RS_CH = RS_THREADS * RS_PER;
// One block sorts a chunk of RAY_CH rays: shared-memory counts of the chunk's keys (in place
// then the chunk's first slot per key; 72 KB with the touched-key list, so that two blocks fit
// an SM), then every ray is
// copied to its slot.  The keys the chunk touches are listed as they first occur, so that only
// they are turned into slots and cleared again (a chunk touches at most RAY_CH of the
// RAY_BUCKETS counters).  Key and rank travel packed in one word (key < 2^15, rank < 2^13).
// The copies go RS_BATCH rays at a time, all loads before the stores, so that each thread
// keeps several reads in flight.
constexpr int RS_BATCH = 2;
static_assert(RAY_BUCKETS < (1 << 19) && RAY_CH <= (1 << 13) && RS_CH <= (1 << 13) && RAY_PER % RS_BATCH == 0,
              "key and rank packing");
__host__ __device__ constexpr size_t scatter_smem(int buckets, int chunk) { return sizeof(uint32_t) * ((size_t)buckets + chunk); }
__global__ void __launch_bounds__(RS_THREADS, 2) k_ray_scatter(TransportArgs A, PathQ from, PathQ to, RaySort rs) {
  extern __shared__ uint32_t sm[];  // [RAY_BUCKETS] counts, then [RAY_CH] touched keys
  uint32_t* touched = sm + RAY_BUCKETS;
  __shared__ uint32_t n_touched;
  const uint32_t n = A.cnt->live[A.k];
  constexpr uint32_t NONE = 0xFFFFFFFFu;
  for (int b = threadIdx.x; b < RAY_BUCKETS; b += blockDim.x) sm[b] = 0;
  if (threadIdx.x == 0) n_touched = 0;
  __syncthreads();
  for (uint32_t c0 = blockIdx.x * RAY_CH; c0 < n; c0 += gridDim.x * RAY_CH) {
    uint32_t kr[RAY_PER];
#pragma unroll
    for (int j = 0; j < RAY_PER; ++j) {
      const uint32_t i = c0 + j * RS_THREADS + threadIdx.x;
      kr[j] = NONE;
      if (i < n) {
        const uint32_t key = rs.key[i];
        const uint32_t rank = atomicAdd(&sm[key], 1u);
        if (rank == 0u) touched[atomicAdd(&n_touched, 1u)] = key;
        kr[j] = (key << 13) | rank;
      }
    }
    __syncthreads();
    const uint32_t nt = n_touched;
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
      const uint32_t b = touched[t];
      sm[b] = rs.off[b] + atomicAdd(&rs.cursor[b], sm[b]);
    }
    __syncthreads();
#pragma unroll
    for (int j0 = 0; j0 < RAY_PER; j0 += RS_BATCH) {
      float4 pa[RS_BATCH], wt[RS_BATCH];
      uint4 me[RS_BATCH];
      float2 sf[RS_BATCH], mi[RS_BATCH];
#pragma unroll
      for (int u = 0; u < RS_BATCH; ++u) {
        if (kr[j0 + u] == NONE) continue;
        const uint32_t i = c0 + (j0 + u) * RS_THREADS + threadIdx.x;
        pa[u] = __ldg(&from.pa[i]);
        wt[u] = __ldg(&from.wt[i]);
        me[u] = __ldg(&from.meta[i]);
        sf[u] = __ldg(&from.surf[i]);
        if (A.mis_on) mi[u] = __ldg(&from.mis[i]);
      }
#pragma unroll
      for (int u = 0; u < RS_BATCH; ++u) {
        const uint32_t v = kr[j0 + u];
        if (v == NONE) continue;
        const uint32_t key = v >> 13;
        const uint32_t o = sm[key] + (v & 0x1FFFu);
        to.pa[o] = pa[u];
        to.wt[o] = wt[u];
        to.meta[o] = me[u];
        if (key >= (uint32_t)RAY_KEY_BUCKETS) A.hits[o] = sf[u];  // the carried surface hit
        if (A.mis_on) to.mis[o] = mi[u];
      }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) sm[touched[t]] = 0;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
  }
}

// the second emission pass: chunks of RAY_CH paths, ranked per key as in k_ray_scatter, each
// ray written once, to its sorted slot of A.qout
__global__ void __launch_bounds__(RS_THREADS, 2) k_generate_sorted(TransportArgs A, long long path0, uint32_t n,
                                                                  RaySort rs) {
  extern __shared__ uint32_t sm[];  // [RAY_BUCKETS] counts, then [RAY_CH] touched keys
  uint32_t* touched = sm + RAY_BUCKETS;
  __shared__ uint32_t n_touched;
  const Acq& q = A.acq;
  constexpr uint32_t NONE = 0xFFFFFFFFu;
  for (int b = threadIdx.x; b < RAY_BUCKETS; b += blockDim.x) sm[b] = 0;
  if (threadIdx.x == 0) n_touched = 0;
  __syncthreads();
  for (uint32_t c0 = blockIdx.x * RAY_CH; c0 < n; c0 += gridDim.x * RAY_CH) {
    uint32_t kr[RAY_PER];
    float3 o[RAY_PER], w[RAY_PER];
    float tau[RAY_PER];
#pragma unroll
    for (int j = 0; j < RAY_PER; ++j) {
      const uint32_t i = c0 + j * RS_THREADS + threadIdx.x;
      kr[j] = NONE;
      if (i < n) {
        emit_path(q, path0 + i, o[j], w[j], tau[j]);
        const uint32_t key = rs.key[i];  // as counted
        const uint32_t rank = atomicAdd(&sm[key], 1u);
        if (rank == 0u) touched[atomicAdd(&n_touched, 1u)] = key;
        kr[j] = (key << 13) | rank;
      }
    }
    __syncthreads();
    const uint32_t nt = n_touched;
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
      const uint32_t b = touched[t];
      sm[b] = rs.off[b] + atomicAdd(&rs.cursor[b], sm[b]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RAY_PER; ++j) {
      const uint32_t v = kr[j];
      if (v == NONE) continue;
      const uint32_t i = c0 + j * RS_THREADS + threadIdx.x;
      const uint32_t slot = sm[v >> 13] + (v & 0x1FFFu);
      A.qout.pa[slot] = make_float4(o[j].x, o[j].y, o[j].z, 3.14159265358979f / q.nr);
      A.qout.wt[slot] = make_float4(w[j].x, w[j].y, w[j].z, tau[j]);
      A.qout.meta[slot] = make_uint4((uint32_t)(path0 + i), 0xFFFFFFFFu, 0u, __float_as_uint(0.0f));
      if (A.mis_on) A.qout.mis[slot] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) sm[touched[t]] = 0;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
  }
}

// key of a secondary-ray job: target element and origin cell, 4 in depth x 8 across (jobs aimed
// at one element from nearby scatterers share a warp); a job the receive directivity cuts off
// (Eq. cutoff) ends at once: those go to the last bucket so that they do not share warps with
// jobs that trace.  4096 buckets measured best (1024 with depth cells only: +0.3 ms per frame,
// 8192: +0.5 ms, its sort's writes scattered into runs too short)
__device__ __forceinline__ uint32_t job_key(const RaySort& rs, const SceneDev& S, const Acq& q, float4 job,
                                            uint32_t jm, float4 jx) {
  const uint32_t jid = __float_as_uint(job.w);
  const float3 p = (jid & NEE_ROUGH) ? xyz(jx) : xyz(__ldg(&S.scat[jid]));
  const uint32_t e2 = (jm >> 8) & 0xFF;
  const float3 dv = f3(elem_x(q, (int)e2), 0.0f, 0.0f) - p;
  if (f_rx(-dv.z * rsqrtf(dot3(dv, dv)), q.alpha_m, q.alpha_c) == 0.0f) return JOB_BUCKETS - 1;
  const int cz = min(3, max(0, (int)((p.z - rs.lo.z) * rs.inv_ext.z * 4.0f)));
  const int cx = min(7, max(0, (int)((p.x - rs.lo.x) * rs.inv_ext.x * 8.0f)));
  return ((e2 << 5) | ((uint32_t)cz << 3) | (uint32_t)cx) & (JOB_BUCKETS - 1);
}

__global__ void __launch_bounds__(256) k_job_keys(TransportArgs A, NeeQ from, RaySort rs) {
  extern __shared__ uint32_t h[];
  for (int b = threadIdx.x; b < JOB_BUCKETS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const uint32_t n = A.cnt->nee[A.k], off = A.cnt->nee_off[A.k];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 jb = from.job[off + i];
    const uint32_t key = job_key(rs, A.S, A.acq, jb, from.jm[off + i],
                                 (__float_as_uint(jb.w) & NEE_ROUGH) ? from.jx[off + i] : make_float4(0.f, 0.f, 0.f, 0.f));
    rs.key[i] = key;
    atomicAdd(&h[key], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < JOB_BUCKETS; b += blockDim.x)
    if (h[b]) atomicAdd(&rs.cnt[b], h[b]);
}

// as k_ray_scatter: key and rank packed, the copies JOB_BATCH jobs at a time with all loads
// ahead of the stores
constexpr int JOB_BATCH = 4;
static_assert(RS_PER % JOB_BATCH == 0 && JOB_BUCKETS <= (1 << 19), "job batches, key and rank packing");
__global__ void __launch_bounds__(RS_THREADS, 2) k_job_scatter(TransportArgs A, NeeQ from, NeeQ to, RaySort rs) {
  extern __shared__ uint32_t sm[];  // [JOB_BUCKETS] counts, then the chunk's first slot per key; [RS_CH] touched keys
  uint32_t* touched = sm + JOB_BUCKETS;
  __shared__ uint32_t n_touched;
  const uint32_t n = A.cnt->nee[A.k], off = A.cnt->nee_off[A.k];
  constexpr uint32_t NONE = 0xFFFFFFFFu;
  for (int b = threadIdx.x; b < JOB_BUCKETS; b += blockDim.x) sm[b] = 0;
  if (threadIdx.x == 0) n_touched = 0;
  __syncthreads();
  for (uint32_t c0 = blockIdx.x * RS_CH; c0 < n; c0 += gridDim.x * RS_CH) {
    uint32_t kr[RS_PER];
#pragma unroll
    for (int j = 0; j < RS_PER; ++j) {
      const uint32_t i = c0 + j * RS_THREADS + threadIdx.x;
      kr[j] = NONE;
      if (i < n) {
        const uint32_t key = rs.key[i];
        const uint32_t rank = atomicAdd(&sm[key], 1u);
        if (rank == 0u) touched[atomicAdd(&n_touched, 1u)] = key;
        kr[j] = (key << 13) | rank;
      }
    }
    __syncthreads();
    const uint32_t nt = n_touched;
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
      const uint32_t b = touched[t];
      sm[b] = rs.off[b] + atomicAdd(&rs.cursor[b], sm[b]);
    }
    __syncthreads();
#pragma unroll
    for (int j0 = 0; j0 < RS_PER; j0 += JOB_BATCH) {
      float4 jb[JOB_BATCH];
      uint32_t jm[JOB_BATCH], jp[JOB_BATCH];
#pragma unroll
      for (int u = 0; u < JOB_BATCH; ++u) {
        if (kr[j0 + u] == NONE) continue;
        const uint32_t i = off + c0 + (j0 + u) * RS_THREADS + threadIdx.x;
        jb[u] = __ldg(&from.job[i]);
        jm[u] = __ldg(&from.jm[i]);
        jp[u] = __ldg(&from.jpath[i]);
      }
#pragma unroll
      for (int u = 0; u < JOB_BATCH; ++u) {
        const uint32_t v = kr[j0 + u];
        if (v == NONE) continue;
        const uint32_t i = off + c0 + (j0 + u) * RS_THREADS + threadIdx.x;
        const uint32_t o = off + sm[v >> 13] + (v & 0x1FFFu);
        to.job[o] = jb[u];
        to.jm[o] = jm[u];
        to.jpath[o] = jp[u];
        if (__float_as_uint(jb[u].w) & NEE_ROUGH) {
          to.jx[o] = __ldg(&from.jx[i]);
          to.jw[o] = __ldg(&from.jw[i]);
        }
      }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) sm[touched[t]] = 0;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
  }
}

void launch_job_sort(const TransportArgs& a, const NeeQ& from, const NeeQ& to, const RaySort& rs, int grid,
                     cudaStream_t st) {
  cudaMemsetAsync(rs.cnt, 0, sizeof(uint32_t) * JOB_BUCKETS, st);
  k_job_keys<<<grid, 256, sizeof(uint32_t) * JOB_BUCKETS, st>>>(a, from, rs);
  launch_count_scan(rs.cnt, rs.off, rs.cursor, JOB_BUCKETS, st);
  k_job_scatter<<<grid, RS_THREADS, scatter_smem(JOB_BUCKETS, RS_CH), st>>>(a, from, to, rs);
}

void launch_ray_sort(const TransportArgs& a, const PathQ& from, const PathQ& to, const RaySort& rs, int grid,
                     cudaStream_t st) {
  launch_count_scan(rs.cnt, rs.off, rs.cursor, RAY_BUCKETS, st);
  k_ray_scatter<<<grid, RS_THREADS, scatter_smem(RAY_BUCKETS, RAY_CH), st>>>(a, from, to, rs);
}

cudaError_t ray_sort_set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_generate_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(uint32_t) * RAY_BUCKETS));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_generate_sorted, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)scatter_smem(RAY_BUCKETS, RAY_CH));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_job_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(uint32_t) * RAY_BUCKETS));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_job_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)scatter_smem(JOB_BUCKETS, RS_CH));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ray_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)scatter_smem(RAY_BUCKETS, RAY_CH));
}

void launch_generate(const TransportArgs& a, long long path0, uint32_t n, const RaySort& rs, int grid,
                     cudaStream_t st) {
  k_generate_count<<<grid, GEN_THREADS, sizeof(uint32_t) * RAY_BUCKETS, st>>>(a, path0, n);
  launch_count_scan(rs.cnt, rs.off, rs.cursor, RAY_BUCKETS, st);
  k_generate_sorted<<<grid, RS_THREADS, scatter_smem(RAY_BUCKETS, RAY_CH), st>>>(a, path0, n, rs);
}
void launch_traverse(const TransportArgs& a, int grid, cudaStream_t st) { k_traverse<<<grid, TRAV_THREADS, 0, st>>>(a); }
void launch_march(const TransportArgs& a, int grid, cudaStream_t st) { k_march<<<grid, MARCH_THREADS, 0, st>>>(a); }
int march_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_march, MARCH_THREADS, 0) != cudaSuccess || b < 1) b = 4;
  return b;  // one wave of resident blocks: lanes refill from the pool until it is empty
}
int traverse_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_traverse, TRAV_THREADS, 0) != cudaSuccess || b < 1) b = 4;
  return 2 * b;  // two waves of resident blocks: a short tail without a long grid-stride loop
}
void launch_interact(const TransportArgs& a, int grid, cudaStream_t st) { k_interact<<<grid, IA_THREADS, 0, st>>>(a); }
void launch_nee(const TransportArgs& a, int grid, cudaStream_t st) { k_nee<<<grid, NEE_THREADS, 0, st>>>(a); }
int nee_blocks_per_sm() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_nee, NEE_THREADS, 0) != cudaSuccess || b < 1) b = 4;
  return b;  // one wave of resident blocks: lanes refill from the pool until it is empty
}

}  // namespace usrt
