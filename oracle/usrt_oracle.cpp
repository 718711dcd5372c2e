// usrt oracle: a plain, slow, FP64 CPU implementation of the differentiable full-path
// Monte Carlo ultrasound ray-tracing hot path (arXiv 2604.15017).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this
// file; it shares no code, header, table or constant generator with the CUDA path.  Only the
// tests, the package's smoke check and the benchmark's CPU-baseline leg load it.
//
// Every function names the passage of the paper it follows.  Where the paper is silent the
// reading taken is stated beside the code (the same readings are listed in the design notes).
//
// Units: SI throughout (metres, seconds, hertz, kg/m^3); attenuation in dB/cm/MHz.
// Parameter vector theta = [c_0, rho_0, alpha_0, ..., c_{M-1}, rho_{M-1}, alpha_{M-1}, A_s, f0].
//
// Pieces:
//   * Philox4x32-10 counter-based generator (Salmon et al., SC'11): 10 rounds, multipliers
//     0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
//   * scene: triangles with (m_front, m_back) media, point scatterers, brute force or a simple
//     median-split BVH for closest-hit and all-crossings queries (textbook Moller-Trumbore).
//   * forward transport (Sec. 2.3.1-2.3.3): emission, traversal, Fresnel/Snell interface,
//     receiver-guided secondary rays at scatterers, receive directivity (Eq. cutoff).
//   * replay of frozen decisions, templated on the scalar so that the same code runs in double
//     (finite differences, Sec. 3.2 / Sec. 4.2.1) and in forward-mode dual numbers (gradient).
//   * splat with the axial pulse (Eq. axial_sig), delay-and-sum (Eq. das), Hilbert envelope,
//     log compression and dynamic-range clip (Sec. 2.3.4), the l1+l2 loss (Eq.
//     weighted_l1_l2_loss) and the vector-Jacobian products of the image chain (Eq.
//     das_adjoint and the envelope/log derivative).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double PI = 3.14159265358979323846;
// amplitude attenuation exponent per (dB/cm/MHz) * Hz * m: ln(10)/20 [Np/dB] * 1e-6 [MHz/Hz] * 100 [cm/m]
const double KAPPA = std::log(10.0) / 20.0 * 1e-4;
// minimum hit distance [m] of every ray query (reading: a ray leaving a surface must not re-hit
// that surface or its neighbour at the shared edge; 0.1 um is far below a wavelength)
const double T_MIN = 1e-7;

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3",
// SC'11).  One round maps (c0,c1,c2,c3) with key (k0,k1) to
//   (hi(B*c2) ^ c1 ^ k0, lo(B*c2), hi(A*c0) ^ c3 ^ k1, lo(A*c0)),  A=0xD2511F53, B=0xCD9E8D57,
// and the key is bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------------
struct U4 {
  uint32_t v[4];
};

U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int round = 0; round < 10; ++round) {
    uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)pb;
    uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)pa;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  U4 r = {{c0, c1, c2, c3}};
  return r;
}

// top 24 bits as a uniform in [0, 1): exactly representable in float and double
double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// ------------------------------------------------------------------------------------------
// Forward-mode dual numbers: value + gradient w.r.t. up to NP parameters.
// ------------------------------------------------------------------------------------------
const int NP = 48;

struct Dual {
  double v;
  double d[NP];
  Dual() : v(0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }
};

Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < NP; ++i) r.d[i] = -a.d[i];
  return r;
}
Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  for (int i = 0; i < NP; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
Dual operator-(double b, const Dual& a) { return -a + b; }
Dual operator*(const Dual& a, double b) {
  Dual r(a.v * b);
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b;
  return r;
}
Dual operator*(double b, const Dual& a) { return a * b; }
Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
Dual operator/(double a, const Dual& b) {
  Dual r(a / b.v);
  for (int i = 0; i < NP; ++i) r.d[i] = -a * b.d[i] / (b.v * b.v);
  return r;
}
// chain rule helper: f(a) with derivative df
Dual chain(const Dual& a, double f, double df) {
  Dual r(f);
  for (int i = 0; i < NP; ++i) r.d[i] = df * a.d[i];
  return r;
}
Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, s > 0 ? 0.5 / s : 0.0); }
Dual exp(const Dual& a) { double e = std::exp(a.v); return chain(a, e, e); }
Dual sin(const Dual& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
Dual acos(const Dual& a) {
  double q = 1.0 - a.v * a.v;
  return chain(a, std::acos(a.v), q > 0 ? -1.0 / std::sqrt(q) : 0.0);
}

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::acos;
using std::exp;
using std::fabs;
using std::log;
using std::sin;
using std::cos;
using std::sqrt;

template <class S>
struct V3 {
  S x, y, z;
};
template <class S> V3<S> mk3(S x, S y, S z) { V3<S> r; r.x = x; r.y = y; r.z = z; return r; }
template <class S, class T> V3<S> add(const V3<S>& a, const V3<T>& b) { return mk3<S>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class S, class T> V3<S> sub(const V3<S>& a, const V3<T>& b) { return mk3<S>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class S, class K> V3<S> scale(const V3<S>& a, const K& k) { return mk3<S>(a.x * k, a.y * k, a.z * k); }
template <class S, class T> S dot(const V3<S>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

typedef V3<double> D3;
D3 d3(double x, double y, double z) { return mk3<double>(x, y, z); }
D3 cross(const D3& a, const D3& b) { return d3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
double dotd(const D3& a, const D3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
D3 subd(const D3& a, const D3& b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }

// ------------------------------------------------------------------------------------------
// Acquisition and image descriptors (flat double arrays; layout mirrored in oracle.py)
// ------------------------------------------------------------------------------------------
enum {
  A_NE = 0, A_PITCH, A_HEL, A_NTX, A_FS, A_NS, A_KMAX, A_NR, A_BW, A_ALPHA_M, A_ALPHA_C, A_CBF,
  A_SPLIT_MODE, A_SPLIT_Q, A_STREAM, A_TX_ELEM, A_N_TX_ELEM, A_ROUGH_NEE, A_COUNT
};
enum { I_NL = 0, I_ND, I_X0, I_X1, I_Z0, I_Z1, I_DR, I_L1, I_L2, I_FNUM, I_COUNT };

struct Acq {
  int ne, ntx, ns, kmax, nr, split_mode, tx_elem, n_tx_elem;
  int rough_nee;  // secondary rays at rough interface events too (else at scatterers only);
                  // 2 (tests of the estimator): the secondary ray alone estimates the rough
                  // event's direct contribution (no balance weights, primary direct hits dropped)
  double pitch, hel, fs, bw, alpha_m, alpha_c, cbf, split_q;
  uint32_t stream;
  std::vector<double> angles;
  // emitting elements: all, or tx_elem .. tx_elem + max(1, n_tx_elem) - 1 (a sub-aperture)
  int n_emit() const { return tx_elem < 0 ? ne : std::max(1, n_tx_elem); }
  long long rays_per_tx() const { return (long long)n_emit() * nr; }
  long long n_paths() const { return rays_per_tx() * ntx; }
  double elem_x(int e) const { return (e - 0.5 * (ne - 1)) * pitch; }
  double aperture() const { return (ne - 1) * pitch; }
};

Acq make_acq(const double* a, const double* angles) {
  Acq q;
  q.ne = (int)a[A_NE];
  q.pitch = a[A_PITCH];
  q.hel = a[A_HEL];
  q.ntx = (int)a[A_NTX];
  q.fs = a[A_FS];
  q.ns = (int)a[A_NS];
  q.kmax = (int)a[A_KMAX];
  q.nr = (int)a[A_NR];
  q.bw = a[A_BW];
  q.alpha_m = a[A_ALPHA_M];
  q.alpha_c = a[A_ALPHA_C];
  q.cbf = a[A_CBF];
  q.split_mode = (int)a[A_SPLIT_MODE];
  q.split_q = a[A_SPLIT_Q];
  q.stream = (uint32_t)a[A_STREAM];
  q.tx_elem = (int)a[A_TX_ELEM];
  q.n_tx_elem = (int)a[A_N_TX_ELEM];
  q.rough_nee = (int)a[A_ROUGH_NEE];
  q.angles.assign(angles, angles + q.ntx);
  return q;
}

struct Img {
  int nl, nd;
  double x0, x1, z0, z1, dr, l1, l2;
  double fnum;  // receive F-number of the dynamic aperture (<= 0: the whole array)
};
Img make_img(const double* p) {
  Img m;
  m.nl = (int)p[I_NL];
  m.nd = (int)p[I_ND];
  m.x0 = p[I_X0];
  m.x1 = p[I_X1];
  m.z0 = p[I_Z0];
  m.z1 = p[I_Z1];
  m.dr = p[I_DR];
  m.l1 = p[I_L1];
  m.l2 = p[I_L2];
  m.fnum = p[I_FNUM];
  return m;
}
double line_x(const Img& m, int l) { return m.nl > 1 ? m.x0 + (m.x1 - m.x0) * l / (m.nl - 1) : m.x0; }
double depth_z(const Img& m, int d) { return m.nd > 1 ? m.z0 + (m.z1 - m.z0) * d / (m.nd - 1) : m.z0; }

// ------------------------------------------------------------------------------------------
// Scene: triangles (v0,v1,v2; front medium = side the normal (v1-v0)x(v2-v0) points to),
// point scatterers (centre, amplitude s_j, common radius r_s), optional median-split BVH.
// ------------------------------------------------------------------------------------------
enum { CLS_NONE = 0, CLS_XDCR = 1, CLS_TRI = 2, CLS_SCAT = 3 };

struct Hit {
  double t;
  int cls, id;
};
bool hit_before(const Hit& a, const Hit& b) {  // (t, class, id) lexicographic
  if (a.t != b.t) return a.t < b.t;
  if (a.cls != b.cls) return a.cls < b.cls;
  return a.id < b.id;
}

struct BNode {
  double lo[3], hi[3];
  int left, right;  // children (inner) or -1
  int first, count; // primitive range in order[] for leaves
};

struct Scene {
  int nt = 0, nsct = 0;
  bool rough = false;  // theta carries a roughness per medium after A_s and f0
  std::vector<D3> v0, v1, v2;
  std::vector<int> mfront, mback;
  std::vector<D3> sp;
  std::vector<double> samp;
  double rs = 0;
  bool use_bvh = false;
  std::vector<BNode> nodes;
  std::vector<int> order;  // primitive ids: 0..nt-1 triangles, nt.. scatterers

  void prim_box(int p, double lo[3], double hi[3]) const {
    if (p < nt) {
      const D3* v[3] = {&v0[p], &v1[p], &v2[p]};
      for (int a = 0; a < 3; ++a) {
        double mn = 1e300, mx = -1e300;
        for (int k = 0; k < 3; ++k) {
          double c = a == 0 ? v[k]->x : a == 1 ? v[k]->y : v[k]->z;
          mn = std::min(mn, c);
          mx = std::max(mx, c);
        }
        lo[a] = mn;
        hi[a] = mx;
      }
    } else {
      const D3& c = sp[p - nt];
      lo[0] = c.x - rs; hi[0] = c.x + rs;
      lo[1] = c.y - rs; hi[1] = c.y + rs;
      lo[2] = c.z - rs; hi[2] = c.z + rs;
    }
  }

  // simple recursive median split on the longest centroid axis, leaves of <= 4 primitives
  int build(int first, int count, std::vector<double>& cen) {
    BNode n;
    for (int a = 0; a < 3; ++a) { n.lo[a] = 1e300; n.hi[a] = -1e300; }
    double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
    for (int i = first; i < first + count; ++i) {
      double lo[3], hi[3];
      prim_box(order[i], lo, hi);
      for (int a = 0; a < 3; ++a) {
        n.lo[a] = std::min(n.lo[a], lo[a]);
        n.hi[a] = std::max(n.hi[a], hi[a]);
        double c = cen[3 * order[i] + a];
        clo[a] = std::min(clo[a], c);
        chi[a] = std::max(chi[a], c);
      }
    }
    int idx = (int)nodes.size();
    nodes.push_back(n);
    if (count <= 4) {
      nodes[idx].left = nodes[idx].right = -1;
      nodes[idx].first = first;
      nodes[idx].count = count;
      return idx;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
      if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    int mid = first + count / 2;
    std::nth_element(order.begin() + first, order.begin() + mid, order.begin() + first + count,
                     [&](int p, int q) { return cen[3 * p + axis] < cen[3 * q + axis]; });
    int l = build(first, mid - first, cen);
    int r = build(mid, first + count - mid, cen);
    nodes[idx].left = l;
    nodes[idx].right = r;
    nodes[idx].first = nodes[idx].count = 0;
    return idx;
  }

  void build_bvh() {
    int n = nt + nsct;
    order.resize(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::vector<double> cen(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
      double lo[3], hi[3];
      prim_box(i, lo, hi);
      for (int a = 0; a < 3; ++a) cen[3 * i + a] = 0.5 * (lo[a] + hi[a]);
    }
    nodes.clear();
    if (n) build(0, n, cen);
    use_bvh = true;
  }
};

// Moller-Trumbore ray/triangle test (Moller & Trumbore 1997); returns t > 0 or -1
double tri_hit(const Scene& s, int i, const D3& o, const D3& w) {
  D3 e1 = subd(s.v1[i], s.v0[i]), e2 = subd(s.v2[i], s.v0[i]);
  D3 p = cross(w, e2);
  double det = dotd(e1, p);
  if (det == 0.0) return -1;
  double inv = 1.0 / det;
  D3 tv = subd(o, s.v0[i]);
  double u = dotd(tv, p) * inv;
  if (u < 0.0 || u > 1.0) return -1;
  D3 q = cross(tv, e1);
  double v = dotd(w, q) * inv;
  if (v < 0.0 || u + v > 1.0) return -1;
  double t = dotd(e2, q) * inv;
  return t > T_MIN ? t : -1;
}

// point scatterer: event at the closest approach t = (p - o).w, if within r_s of the centre
double scat_hit(const Scene& s, int j, const D3& o, const D3& w) {
  D3 d = subd(s.sp[j], o);
  double t = dotd(d, w);
  if (!(t > T_MIN)) return -1;
  D3 q = d3(o.x + t * w.x - s.sp[j].x, o.y + t * w.y - s.sp[j].y, o.z + t * w.z - s.sp[j].z);
  return dotd(q, q) <= s.rs * s.rs ? t : -1;
}

// slab test of a ray against a box, interval [t0, t1] clipped to [0, tmax]
bool box_hit(const BNode& n, const D3& o, const D3& w, double tmax) {
  double t0 = 0.0, t1 = tmax;
  double oo[3] = {o.x, o.y, o.z}, ww[3] = {w.x, w.y, w.z};
  for (int a = 0; a < 3; ++a) {
    if (ww[a] == 0.0) {
      if (oo[a] < n.lo[a] || oo[a] > n.hi[a]) return false;
      continue;
    }
    double ta = (n.lo[a] - oo[a]) / ww[a], tb = (n.hi[a] - oo[a]) / ww[a];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1) return false;
  }
  return true;
}

void test_prim(const Scene& s, int p, const D3& o, const D3& w, int xcls, int xid, Hit& best) {
  Hit h;
  if (p < s.nt) {
    if (xcls == CLS_TRI && xid == p) return;
    h.t = tri_hit(s, p, o, w);
    h.cls = CLS_TRI;
    h.id = p;
  } else {
    int j = p - s.nt;
    if (xcls == CLS_SCAT && xid == j) return;
    h.t = scat_hit(s, j, o, w);
    h.cls = CLS_SCAT;
    h.id = j;
  }
  if (h.t > 0 && hit_before(h, best)) best = h;
}

// closest hit over triangles and scatterers (transducer handled by the caller), excluding
// the primitive (xcls, xid) the ray leaves from.  [Sec. 2.3.2]
void closest_scene(const Scene& s, const D3& o, const D3& w, int xcls, int xid, Hit& best) {
  if (!s.use_bvh) {
    for (int p = 0; p < s.nt + s.nsct; ++p) test_prim(s, p, o, w, xcls, xid, best);
    return;
  }
  if (s.nodes.empty()) return;
  int stack[128];
  int sp = 0;
  stack[sp++] = 0;
  while (sp) {
    const BNode& n = s.nodes[stack[--sp]];
    if (!box_hit(n, o, w, best.t)) continue;
    if (n.left < 0) {
      for (int i = n.first; i < n.first + n.count; ++i) test_prim(s, s.order[i], o, w, xcls, xid, best);
    } else {
      stack[sp++] = n.left;
      stack[sp++] = n.right;
    }
  }
}

// all triangle crossings of the segment o + t w, 0 < t < tmax (secondary rays) [Sec. 2.3.3]
void all_crossings(const Scene& s, const D3& o, const D3& w, double tmax, std::vector<std::pair<double, int>>& out) {
  out.clear();
  if (!s.use_bvh) {
    for (int i = 0; i < s.nt; ++i) {
      double t = tri_hit(s, i, o, w);
      if (t > 0 && t < tmax) out.push_back(std::make_pair(t, i));  // tri_hit already has t > T_MIN
    }
  } else if (!s.nodes.empty()) {
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
      const BNode& n = s.nodes[stack[--sp]];
      if (!box_hit(n, o, w, tmax)) continue;
      if (n.left < 0) {
        for (int i = n.first; i < n.first + n.count; ++i) {
          int p = s.order[i];
          if (p >= s.nt) continue;
          double t = tri_hit(s, p, o, w);
          if (t > 0 && t < tmax) out.push_back(std::make_pair(t, p));
        }
      } else {
        stack[sp++] = n.left;
        stack[sp++] = n.right;
      }
    }
  }
  std::sort(out.begin(), out.end());
}

// ------------------------------------------------------------------------------------------
// Physics parameters in scalar type S
// ------------------------------------------------------------------------------------------
template <class S>
struct Phys {
  int M;
  std::vector<S> c, rho, al;
  S As, f0;
  std::vector<S> rough;  // GGX roughness alpha per medium (empty: every interface smooth)
  int acq_base = -1;  // >= 0: duals also carry the acquisition parameters: d/d c_bf (slot
                      // acq_base), d/d pitch (acq_base + 1), d/d steering angle of transmit t
                      // (acq_base + 2 + t)
  int shape_base = -1;          // >= 0: slots shape_base + j carry d/d q_j of n_shape shape parameters,
  int n_shape = 0;              // whose vertex tangents d v / d q_j are vtan[(j * n_tris + tri) * 9 + 3 k + a]
  const double* vtan = nullptr;  // (vertex k of triangle tri, coordinate a)
};

// Emission (Sec. 2.3.1) in the acquisition parameters.  The time stamp tau_tx = (x_e sin th +
// W/2 |sin th|) / c_bf with W = (N_e - 1) p: d/dc_bf = -tau_tx / c_bf, d/dp = tau_tx / p (x_e
// and W are both proportional to p), d/dth with d|sin th|/dth = sgn(sin th) cos th, sgn(0) = 0.
// The origin's x = x_e + (u - 1/2) p = p (e - (N_e - 1)/2 + u - 1/2): d/dp = x / p.
void emit_acq(double&, double&, int, int, double, double, double, double, const Acq&) {}
void emit_acq(Dual& ox, Dual& tau, int base, int tx, double ox0, double tau0, double xe, double th, const Acq& q) {
  if (base < 0) return;
  const double st = std::sin(th), ct = std::cos(th), sg = st > 0 ? 1.0 : (st < 0 ? -1.0 : 0.0);
  tau.d[base] += -tau0 / q.cbf;
  tau.d[base + 1] += tau0 / q.pitch;
  tau.d[base + 2 + tx] += (xe * ct + 0.5 * q.aperture() * sg * ct) / q.cbf;
  ox.d[base + 1] += ox0 / q.pitch;
}
// Vertex k of triangle tri; with shape slots its dual parts are the tangents d v / d q_j.
void shape_dual(double&, const Phys<double>&, int, int, int, int) {}
void shape_dual(Dual& x, const Phys<Dual>& P, int nt, int tri, int k, int a) {
  for (int j = 0; j < P.n_shape; ++j) x.d[P.shape_base + j] += P.vtan[((size_t)j * nt + tri) * 9 + 3 * k + a];
}
template <class S>
V3<S> tri_vtx(const Scene& sc, const Phys<S>& P, int tri, int k) {
  const D3& v = k == 0 ? sc.v0[tri] : (k == 1 ? sc.v1[tri] : sc.v2[tri]);
  V3<S> r = mk3<S>(S(v.x), S(v.y), S(v.z));
  if (P.shape_base >= 0) {
    shape_dual(r.x, P, sc.nt, tri, k, 0);
    shape_dual(r.y, P, sc.nt, tri, k, 1);
    shape_dual(r.z, P, sc.nt, tri, k, 2);
  }
  return r;
}
template <class S>
V3<S> cross3(const V3<S>& a, const V3<S>& b) {
  return mk3<S>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// unnormalised normal (v1 - v0) x (v2 - v0) of a triangle, and its first vertex
template <class S>
V3<S> tri_normal(const Scene& sc, const Phys<S>& P, int tri, V3<S>& v0) {
  v0 = tri_vtx(sc, P, tri, 0);
  return cross3(sub(tri_vtx(sc, P, tri, 1), v0), sub(tri_vtx(sc, P, tri, 2), v0));
}

// an element centre x_e = p (e - (N_e - 1)/2) with its pitch derivative x_e / p
void elem_acq(double&, int, double, const Acq&) {}
void elem_acq(Dual& x, int base, double xe, const Acq& q) {
  if (base >= 0) x.d[base + 1] += xe / q.pitch;
}

// theta = [c, rho, alpha] x M, A_s, f0 (3M + 2), then with rough a GGX roughness per medium
// (4M + 2 in all)
Phys<double> phys_double(const double* th, int M, bool rough = false) {
  Phys<double> p;
  p.M = M;
  for (int m = 0; m < M; ++m) {
    p.c.push_back(th[3 * m]);
    p.rho.push_back(th[3 * m + 1]);
    p.al.push_back(th[3 * m + 2]);
  }
  p.As = th[3 * M];
  p.f0 = th[3 * M + 1];
  if (rough)
    for (int m = 0; m < M; ++m) p.rough.push_back(th[3 * M + 2 + m]);
  return p;
}

Phys<Dual> phys_dual(const double* th, int M, bool rough = false) {
  Phys<Dual> p;
  p.M = M;
  for (int m = 0; m < M; ++m) {
    Dual c(th[3 * m]), r(th[3 * m + 1]), a(th[3 * m + 2]);
    c.d[3 * m] = 1;
    r.d[3 * m + 1] = 1;
    a.d[3 * m + 2] = 1;
    p.c.push_back(c);
    p.rho.push_back(r);
    p.al.push_back(a);
  }
  Dual as(th[3 * M]), f(th[3 * M + 1]);
  as.d[3 * M] = 1;
  f.d[3 * M + 1] = 1;
  p.As = as;
  p.f0 = f;
  if (rough)
    for (int m = 0; m < M; ++m) {
      Dual r(th[3 * M + 2 + m]);
      r.d[3 * M + 2 + m] = 1;
      p.rough.push_back(r);
    }
  return p;
}

// receive directivity, Eq. cutoff (trapezoid in the angle to the element normal)
template <class S>
S f_rx(const S& theta, double am, double ac) {
  double th = val(theta);
  if (th <= am) return S(1.0);
  if (th > ac) return S(0.0);
  return (ac - theta) / (ac - am);
}

// ------------------------------------------------------------------------------------------
// Per-path record of discrete decisions (frozen for replay / differentiation)
// ------------------------------------------------------------------------------------------
enum { CH_NONE = 0, CH_REFLECT = 1, CH_TRANSMIT = 2, CH_TIR = 3 };

struct Rec {  // one per segment
  int cls, id;   // primitive hit (CLS_NONE = escape)
  int choice;    // interface decision, or CH_NONE
  int aux;       // NEE element (scatterer events) / receiving element (transducer)
};

template <class S>
struct Arrival {
  int tx, e, kind, ev;  // kind 0 = transducer hit, 1 = secondary (NEE) ray; ev = segment index
  long long path;
  S tau, a;
};

struct Counters {
  long long segments = 0, nee = 0;
};

// ------------------------------------------------------------------------------------------
// Interface event [Sec. 2.3.2]: incident unit direction w, unit normal nin pointing back into
// the incident medium 1.  Specular reflection w_r = w + 2 cos(theta_i) nin; Snell's law with
// sound speeds sin(theta_t) / c2 = sin(theta_i) / c1 (the impedance ratio Z1/Z2 the paper
// defines is not a refractive index); total internal reflection when sin(theta_t) >= 1.
// Pressure coefficients (reading of the printed Fresnel form, which at normal incidence gives
// the opposite sign to (Z2 - Z1)/(Z2 + Z1)):
//   R = (Z2 cos_i - Z1 cos_t) / (Z2 cos_i + Z1 cos_t),   T = 2 Z2 cos_i / (Z2 cos_i + Z1 cos_t).
// clamp_ct forces cos_t = 0 (a frozen transmit/reflect branch replayed past the critical angle).
// ------------------------------------------------------------------------------------------
template <class S>
struct Iface {
  bool tir;
  S ci, ct, r, R, T;
  V3<S> wr, wt;
};

template <class S>
Iface<S> interface_event(const V3<S>& w, const V3<S>& nin, const S& c1, const S& c2, const S& rho1,
                         const S& rho2, bool clamp_ct = false) {
  Iface<S> f;
  f.ci = -dot(w, nin);
  f.r = c2 / c1;
  S si2 = 1.0 - f.ci * f.ci;
  if (val(si2) < 0) si2 = S(0.0);
  S st2 = f.r * f.r * si2;
  f.tir = val(st2) >= 1.0;
  f.wr = add(w, scale(nin, 2.0 * f.ci));
  if (f.tir && !clamp_ct) {
    f.ct = S(0.0);
    f.R = S(1.0);
    f.T = S(0.0);
    f.wt = f.wr;
    return f;
  }
  f.ct = clamp_ct ? S(0.0) : sqrt(1.0 - st2);
  S A = rho2 * c2 * f.ci, B = rho1 * c1 * f.ct;
  f.R = (A - B) / (A + B);
  f.T = 2.0 * A / (A + B);
  f.wt = add(scale(w, f.r), scale(nin, f.r * f.ci - f.ct));
  return f;
}

// ------------------------------------------------------------------------------------------
// Secondary (receiver-directed) rays [Sec. 2.3.3]: a straight segment from the event to the
// chosen element's centre, the transmission coefficient at every crossed interface (zero under
// total internal reflection), attenuation and travel time per sub-segment in the medium tracked
// across the crossings, receive directivity (Eq. cutoff) at the element.
// ------------------------------------------------------------------------------------------
// The target element centre carries the pitch derivative and the triangles their shape
// tangents (when the duals hold them), so the geometry below (length, direction, crossing
// distances on the crossed triangles' planes, incidence cosines, directivity) is evaluated in
// S; which triangles are crossed is decided in double.  `skip` is a triangle the segment starts
// on (it is not a crossing).  Returns false when nothing arrives (directivity cutoff, total
// internal reflection at a crossing); else trans = prod T * attenuation * f_rx and the time.
template <class S>
bool secondary_segment(const Scene& sc, const Phys<S>& P, const Acq& q, const V3<S>& ps, int skip, int e2, int m_start,
                       S& trans, S& dt, V3<S>& dir, S& dist, std::vector<std::pair<double, int>>& xs,
                       double* frx_out) {
  S xt(q.elem_x(e2));
  elem_acq(xt, P.acq_base, q.elem_x(e2), q);
  V3<S> dv = mk3<S>(xt + (-1.0 * ps.x), -1.0 * ps.y, -1.0 * ps.z);
  S D = sqrt(dot(dv, dv));
  V3<S> d = scale(dv, 1.0 / D);
  dir = d;
  dist = D;
  S cosd = -1.0 * d.z;
  double cv = std::max(-1.0, std::min(1.0, val(cosd)));
  S th = (cv == val(cosd)) ? acos(cosd) : S(std::acos(cv));
  S frx = f_rx<S>(th, q.alpha_m, q.alpha_c);
  *frx_out = val(frx);
  if (val(frx) == 0.0) return false;
  all_crossings(sc, d3(val(ps.x), val(ps.y), val(ps.z)), d3(val(d.x), val(d.y), val(d.z)), val(D), xs);
  if (skip >= 0) xs.erase(std::remove_if(xs.begin(), xs.end(), [&](const std::pair<double, int>& c) { return c.second == skip; }),
                          xs.end());
  S prodT(1.0), path_alpha(0.0);
  S time(0.0);
  int m = m_start;
  S tprev(0.0);
  for (size_t i = 0; i < xs.size(); ++i) {
    int tri = xs[i].second;
    V3<S> v0;
    V3<S> N = tri_normal(sc, P, tri, v0);
    S t = dot(sub(v0, ps), N) / dot(d, N);  // the crossing on the triangle's plane
    S l = t - tprev;
    path_alpha = path_alpha + P.al[m] * l;
    time = time + l / P.c[m];
    V3<S> n = scale(N, 1.0 / sqrt(dot(N, N)));
    double dn = val(dot(d, n));
    int m1 = dn < 0 ? sc.mfront[tri] : sc.mback[tri];
    int m2 = dn < 0 ? sc.mback[tri] : sc.mfront[tri];
    V3<S> nin = dn < 0 ? n : scale(n, -1.0);
    Iface<S> f = interface_event<S>(d, nin, P.c[m1], P.c[m2], P.rho[m1], P.rho[m2]);
    if (f.tir) return false;  // total internal reflection: no transmitted pressure
    prodT = prodT * f.T;
    m = m2;
    tprev = t;
  }
  S l = D - tprev;
  path_alpha = path_alpha + P.al[m] * l;
  time = time + l / P.c[m];
  trans = prodT * exp(-KAPPA * P.f0 * path_alpha) * frx;
  dt = time;
  return true;
}

// At a scatterer [Sec. 2.3.3]: the segment from the scatterer's centre; the element is chosen
// uniformly, so the weight carries N_e.  gain = N_e * prod T * attenuation * f_rx.
template <class S>
bool nee_weight(const Scene& sc, const Phys<S>& P, const Acq& q, int j, int e2, int m_start, S& gain, S& dt,
                std::vector<std::pair<double, int>>& xs, double* frx_out) {
  const D3 p = sc.sp[j];
  const V3<S> ps = mk3<S>(S(p.x), S(p.y), S(p.z));
  S trans, D;
  V3<S> d;
  if (!secondary_segment<S>(sc, P, q, ps, -1, e2, m_start, trans, dt, d, D, xs, frx_out)) return false;
  gain = trans * (double)q.ne;
  return true;
}

template <class S>
S smith_g1(const S& vn, const S& alpha);  // Smith masking of GGX, defined with the sampling below

// |dh/do| of refraction about the facet h (Walter et al. 2007) with indices 1 / c: o.h < 0
template <class S>
S refract_jacobian(const S& ih, const S& oh, const S& c1, const S& c2) {
  const S den = ih / c1 + oh / c2;
  return (-1.0 * oh) / (c2 * c2 * den * den);
}

// solid angle of an element face (pitch x h_el) seen along unit direction o from distance^2 r2
template <class S>
S element_solid_angle(const Phys<S>& P, const Acq& q, const V3<S>& o, const S& r2) {
  S pitch(q.pitch);
  if (P.acq_base >= 0) elem_acq(pitch, P.acq_base, q.pitch, q);  // d pitch / d pitch = 1
  return pitch * q.hel * (val(o.z) < 0.0 ? -1.0 * o.z : o.z) / r2;
}

// GGX distribution of microfacet normals, Eq. GGX_PDF
template <class S>
S ggx_d(const S& nh, const S& alpha) {
  const S a2 = alpha * alpha;
  const S k = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (PI * k * k);
}

// Direction density of the primary's own sampling at a rough event (reading of Sec. 2.3.2): the
// facet normal h ~ D(h) (h.n), then reflection with probability P_r(h) (R(h)^2, or the fixed
// split q; 1 under total internal reflection) or refraction: toward o it is D(h) (h.n) |dh/do|
// P(choice), with h the facet that maps the incident direction onto o.
template <class S>
S bsdf_pdf(const Acq& q, const S& nh, const S& alpha, const S& J, const Iface<S>& f, bool reflect) {
  const S pr = f.tir ? S(1.0) : (q.split_mode == 0 ? f.R * f.R : S(q.split_q));
  return ggx_d(nh, alpha) * nh * J * (reflect ? pr : 1.0 - pr);
}

// At a rough interface [Sec. 2.3.2-2.3.3, Eq. GGX_PDF] (reading): the secondary ray leaves the
// event point x toward the chosen element's centre, direction o.  The microfacet BSDF gives the
// amplitude the interface sends per unit solid angle toward o, for the incident direction w (i =
// -w points back to the side it came from, n the macro normal on that side): with the half
// vector h of reflection (h ~ i + o, o on the incident side) or of refraction (h ~ -(i / c1 +
// o / c2), o on the far side; Snell with sound speeds), the density the primary sampling
// itself has there, g = D(h) G1(i) G1(o) C(h) |i.h| |dh/do| / |i.n|, with C the pressure
// reflection or transmission coefficient of the facet h and |dh/do| = 1 / (4 |o.h|) for
// reflection, |o.h| / (c2^2 (i.h / c1 + o.h / c2)^2) for refraction (Walter et al. 2007).  The
// primary itself reaches the array from the event too, so the two estimates are combined by
// multiple importance sampling (balance heuristic) over the element's solid angle Omega (face
// pitch x h_el, cosine at the element, 1 / r^2): the secondary ray's density is that of a
// uniform element and direction within it, 1 / (N_e Omega), the primary's is bsdf_pdf, and the
// secondary ray carries g / (1 / (N_e Omega) + bsdf_pdf) times the transmissions, attenuation
// and f_rx of the segment; the primary's own direct arrival takes the complementary weight.
// A facet toward o that is met from behind, or that reflects totally where o asks for
// transmission, sends nothing.
template <class S>
bool rough_nee_weight(const Scene& sc, const Phys<S>& P, const Acq& q, int tri, const V3<S>& x, const V3<S>& w,
                      const V3<S>& nin, int m1, int m2, const S& alpha, int e2, S& gain, S& dt,
                      std::vector<std::pair<double, int>>& xs, double* frx_out) {
  S xt(q.elem_x(e2));
  elem_acq(xt, P.acq_base, q.elem_x(e2), q);
  V3<S> dv = mk3<S>(xt + (-1.0 * x.x), -1.0 * x.y, -1.0 * x.z);
  const S r2 = dot(dv, dv);
  const V3<S> o = scale(dv, 1.0 / sqrt(r2));
  const V3<S> i = scale(w, -1.0);
  const S in = dot(i, nin), on = dot(o, nin);
  const bool reflect = val(on) > 0.0;
  const S c1 = P.c[m1], c2 = P.c[m2];
  V3<S> h;
  if (reflect) {
    V3<S> hv = add(i, o);
    h = scale(hv, 1.0 / sqrt(dot(hv, hv)));
  } else {
    V3<S> hv = scale(add(scale(i, 1.0 / c1), scale(o, 1.0 / c2)), -1.0);
    h = scale(hv, 1.0 / sqrt(dot(hv, hv)));
    if (val(dot(h, nin)) < 0.0) h = scale(h, -1.0);
  }
  const S ih = dot(i, h), oh = dot(o, h), nh = dot(nin, h);
  if (!(val(ih) > 0.0) || !(val(nh) > 0.0)) return false;  // facet met from behind
  if (!reflect && !(val(oh) < 0.0)) return false;
  Iface<S> f = interface_event<S>(w, h, c1, c2, P.rho[m1], P.rho[m2]);
  S C, J;
  if (reflect) {
    C = f.R;
    J = 1.0 / (4.0 * ih);
  } else {
    if (f.tir) return false;
    C = f.T;
    J = refract_jacobian(ih, oh, c1, c2);
  }
  const S g = ggx_d(nh, alpha) * smith_g1(in, alpha) * smith_g1(on, alpha) * C * ih * J / in;
  const S p_nee = 1.0 / ((double)q.ne * element_solid_angle(P, q, o, r2));
  S trans, D;
  V3<S> d;
  if (!secondary_segment<S>(sc, P, q, x, tri, e2, reflect ? m1 : m2, trans, dt, d, D, xs, frx_out)) return false;
  gain = q.rough_nee == 2 ? g * trans / p_nee : g * trans / (p_nee + bsdf_pdf(q, nh, alpha, J, f, reflect));
  return true;
}

// ------------------------------------------------------------------------------------------
// One path.  FORWARD (S = double, rec_in == nullptr): closest-hit search, decisions drawn from
// Philox and written to rec_out.  REPLAY (rec_in != nullptr): the primitive sequence and
// decisions are read from rec_in; hit distances are re-solved on the frozen primitive (its
// plane, the closest approach to the scatterer centre, or the transducer plane), so the result
// is the smooth function of theta that fixed-sample differentiation differentiates
// [Sec. 3.2, Eq. chain_rule].
// Emission [Sec. 2.3.1, Eq. directivity, Eq. pressure_mc]: origin uniform on the element face,
// direction cosine-weighted, so f_d / p = pi; weight pi / N_r; transmit delay as a time stamp.
// Interface [Sec. 2.3.2]: specular reflection, Snell refraction with sound speeds, Fresnel
// pressure coefficients R, T = 1 + R; split probability P_r = R^2 (or a fixed q), weight
// amplitude / selection probability.  Attenuation per segment (exp(-kappa alpha f0 L)).
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// Rough interfaces [Sec. 2.3.2, Eq. GGX_PDF].  A microfacet normal h is drawn with density
// D(h) (h.n) over the hemisphere around n, D the GGX distribution of roughness alpha: inverting
// its cumulative distribution gives tan^2(theta_h) = alpha^2 u / (1 - u) and a uniform azimuth.
// The event then reflects or refracts about h with the pressure coefficients of h (Fresnel and
// Snell as at a smooth interface), and the amplitude takes the microfacet weight of this
// sampling (Walter et al. 2007): |w_i.h| G(w_i, w_o) / (|w_i.n| |h.n|), G the separable Smith
// masking-shadowing of GGX, G1(v) = 2 |v.n| / (|v.n| + sqrt(alpha^2 + (1 - alpha^2) (v.n)^2)).
// A facet the ray meets from behind (w_i.h >= 0), or an outgoing direction on the wrong side
// of the macro surface, ends the path.  alpha -> 0 gives h = n and weight 1: the smooth event.
// ------------------------------------------------------------------------------------------
// orthonormal tangents of a unit normal (the branch-free construction of Duff et al., 2017)
template <class S>
void tangent_frame(const V3<S>& n, V3<S>& t1, V3<S>& t2) {
  const double sg = val(n.z) >= 0.0 ? 1.0 : -1.0;
  const S a = -1.0 / (n.z + sg);
  const S b = n.x * n.y * a;
  t1 = mk3<S>(1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x);
  t2 = mk3<S>(b, sg + n.y * n.y * a, -1.0 * n.y);
}
template <class S>
V3<S> ggx_normal(const V3<S>& n, const S& alpha, double u2, double u3) {
  V3<S> t1, t2;
  tangent_frame(n, t1, t2);
  const S tn = alpha * std::sqrt(u2 / (1.0 - u2));  // tan(theta_h)
  const S ct = 1.0 / sqrt(1.0 + tn * tn);
  const S st = tn * ct;
  const double ph = 2.0 * PI * u3;
  return add(scale(n, ct), add(scale(t1, st * std::cos(ph)), scale(t2, st * std::sin(ph))));
}
template <class S>
S smith_g1(const S& vn, const S& alpha) {
  const S c = vn * (val(vn) < 0 ? -1.0 : 1.0);
  return 2.0 * c / (c + sqrt(alpha * alpha + (1.0 - alpha * alpha) * c * c));
}

// Emission [Sec. 2.3.1, Eq. directivity, Eq. pressure_mc] of ray `ray` (= element x N_r +
// index) of transmit tx from its Philox block (ray, tx, stream, 0): the origin uniform over the
// element face (u0 across the pitch, u1 along the element height); the direction drawn with the
// density p(w) = cos(theta) / pi over the hemisphere around the element normal +z (r = sqrt(u2)
// is sin(theta), u3 the azimuth), so that the directivity f_d = n.w over that density is the
// constant pi and, with the 1/N average over the element's rays, the weight is pi / N_r; the
// steering delay as a time stamp at the element centre.
void emit_ray(const Acq& q, uint32_t k0, uint32_t k1, int tx, long long ray, D3& o0, D3& w0, double& a0,
              double& tau0, double& xe) {
  U4 u = philox((uint32_t)ray, (uint32_t)tx, q.stream, 0u, k0, k1);
  int e = (int)(ray / q.nr);
  xe = q.elem_x(e);
  double u0 = u01(u.v[0]), u1 = u01(u.v[1]), u2 = u01(u.v[2]), u3 = u01(u.v[3]);
  o0 = d3(xe + (u0 - 0.5) * q.pitch, (u1 - 0.5) * q.hel, 0.0);
  double r = std::sqrt(u2), ph = 2.0 * PI * u3;
  w0 = d3(r * std::cos(ph), r * std::sin(ph), std::sqrt(1.0 - u2));
  a0 = PI / q.nr;
  double st = std::sin(q.angles[tx]);
  tau0 = (xe * st + 0.5 * q.aperture() * std::fabs(st)) / q.cbf;
}

struct PathIO {
  // injected emission (tests); when inject is false the emission is sampled from Philox
  bool inject = false;
  D3 o0, w0;
  double a0 = 0, tau0 = 0;
  int tx = 0;
  long long ray = 0;
  // forced interface choices (tests); nullptr = from Philox
  const int* forced = nullptr;
  int n_forced = 0;
  bool physical = false;  // weight interface by R or T instead of amplitude / probability
  double* last_state = nullptr;  // tests: position and direction at the last hit (6 doubles)
};

template <class S>
void trace_path(const Scene& sc, const Phys<S>& P, const Acq& q, uint32_t k0, uint32_t k1, const PathIO& io,
                long long path, const Rec* rec_in, Rec* rec_out, std::vector<Arrival<S>>& arr, Counters& cnt) {
  const bool replay = rec_in != nullptr;
  const uint32_t ray32 = (uint32_t)io.ray;
  D3 o0, w0;
  double a0, tau0, xe_emit = 0.0;
  if (io.inject) {
    o0 = io.o0;
    w0 = io.w0;
    a0 = io.a0;
    tau0 = io.tau0;
  } else {
    emit_ray(q, k0, k1, io.tx, io.ray, o0, w0, a0, tau0, xe_emit);
  }
  V3<S> o = mk3<S>(S(o0.x), S(o0.y), S(o0.z));
  V3<S> w = mk3<S>(S(w0.x), S(w0.y), S(w0.z));
  S a(a0), tau(tau0);
  if (!io.inject) emit_acq(o.x, tau, P.acq_base, io.tx, o0.x, tau0, xe_emit, q.angles[io.tx], q);
  int m = 0;
  int xcls = CLS_NONE, xid = -1;
  std::vector<std::pair<double, int>> xs;
  // the primary's direction density at its last rough event (0: the last event was not rough)
  // and the distance travelled since, straight on through scatterer pass-throughs: a primary
  // that reaches the array from there takes the balance weight against that event's secondary
  // ray
  S last_pdf(0.0), since(0.0);
  for (int k = 0; k <= q.kmax; ++k) {
    Hit h;
    if (!replay) {
      cnt.segments++;
      D3 od = d3(val(o.x), val(o.y), val(o.z)), wd = d3(val(w.x), val(w.y), val(w.z));
      h.t = 1e300;
      h.cls = CLS_NONE;
      h.id = -1;
      if (wd.z < 0.0) {  // transducer face z = 0, |x| <= N_e p / 2, |y| <= h_el / 2
        double t = -od.z / wd.z;
        double x = od.x + t * wd.x, y = od.y + t * wd.y;
        if (t > T_MIN && std::fabs(x) <= 0.5 * q.ne * q.pitch && std::fabs(y) <= 0.5 * q.hel) {
          h.t = t;
          h.cls = CLS_XDCR;
          h.id = std::min(q.ne - 1, std::max(0, (int)std::floor((x + 0.5 * q.ne * q.pitch) / q.pitch)));
        }
      }
      closest_scene(sc, od, wd, xcls, xid, h);
      if (rec_out) {
        rec_out[k].cls = h.cls;
        rec_out[k].id = h.id;
        rec_out[k].choice = CH_NONE;
        rec_out[k].aux = h.cls == CLS_XDCR ? h.id : -1;
      }
    } else {
      h.cls = rec_in[k].cls;
      h.id = rec_in[k].id;
      h.t = 0;
    }
    if (h.cls == CLS_NONE) break;  // escape
    // hit distance on the frozen primitive
    S t;
    if (!replay) {
      t = S(h.t);
    } else if (h.cls == CLS_XDCR) {
      t = -o.z / w.z;
    } else if (h.cls == CLS_TRI) {
      V3<S> v0;
      V3<S> N = tri_normal(sc, P, h.id, v0);
      t = dot(sub(v0, o), N) / dot(w, N);
    } else {
      V3<S> d = sub(mk3<S>(S(sc.sp[h.id].x), S(sc.sp[h.id].y), S(sc.sp[h.id].z)), o);
      t = dot(d, w);
    }
    a = a * exp(-KAPPA * P.al[m] * P.f0 * t);
    tau = tau + t / P.c[m];
    V3<S> x = add(o, scale(w, t));
    if (io.last_state) {
      double st[6] = {val(x.x), val(x.y), val(x.z), val(w.x), val(w.y), val(w.z)};
      std::memcpy(io.last_state, st, sizeof st);
    }
    if (h.cls == CLS_XDCR) {  // arrival at the receiving element [Sec. 2.3.4]
      S cosd = -w.z;
      double cv = std::max(-1.0, std::min(1.0, val(cosd)));
      S th = (cv == val(cosd)) ? acos(cosd) : S(std::acos(cv));
      S f = f_rx<S>(th, q.alpha_m, q.alpha_c);
      int e = replay ? rec_in[k].aux : h.id;
      if (val(last_pdf) > 0.0) {  // balance weight against the last rough event's secondary ray
        const S r = since + t;
        const S p_nee = 1.0 / ((double)q.ne * element_solid_angle(P, q, w, r * r));
        f = q.rough_nee == 2 ? S(0.0) : f * last_pdf / (last_pdf + p_nee);
      }
      if (val(f) != 0.0) {
        Arrival<S> A;
        A.tx = io.tx;
        A.e = e;
        A.kind = 0;
        A.ev = k;
        A.path = path;
        A.tau = tau;
        A.a = a * f;
        arr.push_back(A);
      }
      break;
    }
    if (k == q.kmax) {  // interaction budget spent
      break;
    }
    U4 u = philox(ray32, (uint32_t)io.tx, q.stream, (uint32_t)(k + 1), k0, k1);
    if (h.cls == CLS_TRI) {
      V3<S> v0;
      V3<S> N = tri_normal(sc, P, h.id, v0);
      V3<S> n = scale(N, 1.0 / sqrt(dot(N, N)));
      bool front = val(dot(w, n)) < 0;  // arriving from the side the normal points to
      V3<S> nn = front ? n : scale(n, -1.0);  // unit normal pointing back into medium 1
      int m1 = front ? sc.mfront[h.id] : sc.mback[h.id];
      int m2 = front ? sc.mback[h.id] : sc.mfront[h.id];
      // the facet normal: the macro normal, or a GGX microfacet normal (roughness of the
      // medium the triangle bounds, its back side)
      const bool rough = !P.rough.empty() && val(P.rough[sc.mback[h.id]]) > 0.0;
      if (rough && q.rough_nee) {  // secondary ray to a uniformly chosen element [Sec. 2.3.3]
        const int e2 = replay ? rec_in[k].aux : std::min(q.ne - 1, (int)std::floor(u01(u.v[1]) * q.ne));
        if (rec_out) rec_out[k].aux = e2;
        if (!replay) cnt.nee++;
        S gain, dt;
        double frx;
        if (rough_nee_weight<S>(sc, P, q, h.id, x, w, nn, m1, m2, P.rough[sc.mback[h.id]], e2, gain, dt, xs, &frx)) {
          Arrival<S> A;
          A.tx = io.tx;
          A.e = e2;
          A.kind = 1;
          A.ev = k;
          A.path = path;
          A.tau = tau + dt;
          A.a = a * gain;
          arr.push_back(A);
        }
      }
      V3<S> hf = nn;
      if (rough) hf = ggx_normal<S>(nn, P.rough[sc.mback[h.id]], u01(u.v[2]), u01(u.v[3]));
      const V3<S> w_in = w;
      if (rough && !replay && val(dot(w, hf)) >= 0.0) break;  // facet met from behind: the path ends
      Iface<S> f = interface_event<S>(w, hf, P.c[m1], P.c[m2], P.rho[m1], P.rho[m2]);
      int choice;
      if (replay) {
        choice = rec_in[k].choice;
        if (choice != CH_TIR && f.tir) f = interface_event<S>(w, hf, P.c[m1], P.c[m2], P.rho[m1], P.rho[m2], true);
      } else if (f.tir) {
        choice = CH_TIR;
      } else {
        double pr = q.split_mode == 0 ? val(f.R) * val(f.R) : q.split_q;
        double u0 = u01(u.v[0]);
        if (io.forced && k < io.n_forced) choice = io.forced[k];
        else choice = u0 < pr ? CH_REFLECT : CH_TRANSMIT;
      }
      if (rec_out) rec_out[k].choice = choice;
      S pr = q.split_mode == 0 ? f.R * f.R : S(q.split_q);
      if (choice == CH_TIR) {
        w = f.wr;
        m = m1;
      } else if (choice == CH_REFLECT) {
        a = io.physical ? a * f.R : a * f.R / pr;
        w = f.wr;
        m = m1;
      } else {
        a = io.physical ? a * f.T : a * f.T / (1.0 - pr);
        w = f.wt;
        m = m2;
      }
      if (rough) {
        const S on = dot(w, nn);  // > 0: back into medium 1
        if (!replay && ((m == m1) != (val(on) > 0.0))) break;  // wrong side of the macro surface: the path ends
        const S inn = dot(w_in, nn), hn = dot(hf, nn), ih = dot(w_in, hf);
        const S alpha = P.rough[sc.mback[h.id]];
        a = a * (-1.0 * ih) * smith_g1(inn, alpha) * smith_g1(on, alpha) / ((-1.0 * inn) * hn);
        if (q.rough_nee) {  // the density of the direction just sampled, for the balance weight
          const S J = choice == CH_TRANSMIT ? refract_jacobian(-1.0 * ih, dot(w, hf), P.c[m1], P.c[m2])
                                            : 1.0 / (4.0 * (-1.0 * ih));
          last_pdf = bsdf_pdf(q, hn, alpha, J, f, choice != CH_TRANSMIT);
          since = S(0.0);
        }
      } else {
        last_pdf = S(0.0);
      }
      o = x;
      xcls = CLS_TRI;
      xid = h.id;
    } else {  // scatterer: secondary ray to a uniformly chosen element, Born pass-through
      since = since + t;  // the ray goes on straight: still the last rough event's direction
      int e2 = replay ? rec_in[k].aux : std::min(q.ne - 1, (int)std::floor(u01(u.v[1]) * q.ne));
      if (rec_out) rec_out[k].aux = e2;
      if (!replay) cnt.nee++;
      S gain, dt;
      double frx;
      if (nee_weight<S>(sc, P, q, h.id, e2, m, gain, dt, xs, &frx)) {
        Arrival<S> A;
        A.tx = io.tx;
        A.e = e2;
        A.kind = 1;
        A.ev = k;
        A.path = path;
        A.tau = tau + dt;
        A.a = a * P.As * sc.samp[h.id] * gain;
        arr.push_back(A);
      }
      o = x;
      xcls = CLS_SCAT;
      xid = h.id;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Axial pulse, Eq. axial_sig: s(t) = sin(2 pi f0 t) exp(-t^2 / sigma).  Reading of the
// bandwidth: -6 dB fractional bandwidth bw, i.e. the Gaussian envelope's spectrum falls to one
// half at f0 +- bw f0 / 2, which gives sigma = 4 ln 2 / (pi^2 (bw f0)^2).  Support |t| <= 4 sqrt(sigma).
// ------------------------------------------------------------------------------------------
template <class S>
S pulse_sigma(const S& f0, double bw) {
  return 4.0 * std::log(2.0) / (PI * PI * bw * bw) / (f0 * f0);
}
template <class S>
S pulse(const S& t, const S& f0, const S& sigma) {
  return sin(2.0 * PI * f0 * t) * exp(-(t * t) / sigma);
}
// sample window [n0, n1] of an arrival at tau
void pulse_window(double tau, double sigma, const Acq& q, int& n0, int& n1) {
  double half = 4.0 * std::sqrt(sigma);
  n0 = std::max(0, (int)std::ceil((tau - half) * q.fs));
  n1 = std::min(q.ns - 1, (int)std::floor((tau + half) * q.fs));
}

// ------------------------------------------------------------------------------------------
// Runs over all paths of an acquisition (std::thread over contiguous blocks of paths; every
// block writes its own arrival list, concatenated in path order: deterministic).
// ------------------------------------------------------------------------------------------
struct Run {
  Acq q;
  int M = 0;
  long long path_lo = 0;  // first path index of the run
  long long n_paths = 0;
  int K1 = 0;
  std::vector<Rec> rec;  // n_paths * K1
  std::vector<Arrival<double>> arr;
  Counters cnt;
};

int host_threads() { return std::max(1, (int)std::thread::hardware_concurrency()); }

template <class F>
void parallel_blocks(long long n, int nthreads, F f) {
  if (nthreads <= 1 || n < 2) {
    f(0, 0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int b = 0; b < nthreads; ++b) {
    long long lo = n * b / nthreads, hi = n * (b + 1) / nthreads;
    th.emplace_back([=]() { f(b, lo, hi); });
  }
  for (auto& t : th) t.join();
}

PathIO path_io(const Acq& q, long long path) {
  PathIO io;
  long long rpt = q.rays_per_tx();
  io.tx = (int)(path / rpt);
  long long local = path % rpt;
  io.ray = q.tx_elem < 0 ? local : (long long)q.tx_elem * q.nr + local;
  return io;
}

void forward_run(const Scene& sc, const double* th, Run& run, uint64_t seed, int nthreads,
                 long long path_lo, long long path_hi) {
  const Acq& q = run.q;
  Phys<double> P = phys_double(th, run.M, sc.rough);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  long long n = path_hi - path_lo;
  std::vector<std::vector<Arrival<double>>> parts(std::max(1, nthreads));
  std::vector<Counters> cnts(std::max(1, nthreads));
  parallel_blocks(n, nthreads, [&](int b, long long lo, long long hi) {
    for (long long i = lo; i < hi; ++i) {
      long long p = path_lo + i;
      PathIO io = path_io(q, p);
      Rec* ro = &run.rec[(size_t)i * run.K1];
      for (int k = 0; k < run.K1; ++k) ro[k].cls = CLS_NONE, ro[k].id = -1, ro[k].choice = CH_NONE, ro[k].aux = -1;
      trace_path<double>(sc, P, q, k0, k1, io, p, nullptr, ro, parts[b], cnts[b]);
    }
  });
  for (size_t b = 0; b < parts.size(); ++b) {
    run.arr.insert(run.arr.end(), parts[b].begin(), parts[b].end());
    run.cnt.segments += cnts[b].segments;
    run.cnt.nee += cnts[b].nee;
  }
}

// Splat [Sec. 2.3.4]: RF[tx][e][n] += a s(n / fs - tau), summed in arrival (path) order.
void splat_direct(const Acq& q, double f0, const Arrival<double>* arr, long long n, double* rf) {
  double sig = pulse_sigma<double>(f0, q.bw);
  for (long long i = 0; i < n; ++i) {
    const Arrival<double>& A = arr[i];
    int n0, n1;
    pulse_window(A.tau, sig, q, n0, n1);
    double* row = rf + ((size_t)A.tx * q.ne + A.e) * q.ns;
    for (int s = n0; s <= n1; ++s) row[s] += A.a * pulse<double>(s / q.fs - A.tau, f0, sig);
  }
}

// ------------------------------------------------------------------------------------------
// Image formation
// ------------------------------------------------------------------------------------------
double hann(int e, int ne) { return 0.5 * (1.0 - std::cos(2.0 * PI * (e + 1) / (ne + 1))); }

// Element weight w_e(x, z) of Eq. das.  F-number <= 0: the pixel-independent Hann window over
// the array.  F-number F > 0 (dynamic receive aperture): a Hann window cos^2(pi xi / 2), |xi| < 1,
// of the element's lateral offset from the pixel, xi = (x_e - x) / a, over the half-width
// a = max(z / (2 F), p) (at least one pitch, so that shallow pixels keep an aperture).
// dw_dp: the weight's derivative in the pitch p (x_e = p (e - (N_e - 1)/2); a = p when clamped).
double apod(const Acq& q, const Img& im, double x, double z, int e, double* dw_dp = nullptr) {
  if (dw_dp) *dw_dp = 0.0;
  if (!(im.fnum > 0)) return hann(e, q.ne);
  const double ce = e - 0.5 * (q.ne - 1);
  const bool clamped = z / (2.0 * im.fnum) < q.pitch;
  const double a = clamped ? q.pitch : z / (2.0 * im.fnum);
  const double xi = (ce * q.pitch - x) / a;
  if (std::fabs(xi) >= 1.0) return 0.0;
  const double c = std::cos(0.5 * PI * xi);
  if (dw_dp) *dw_dp = -0.5 * PI * std::sin(PI * xi) * (ce - (clamped ? xi : 0.0)) / a;
  return c * c;
}

// two-way plane-wave delay in samples for pixel (x, z), element e, steering angle th  [Eq. das]
double das_delay_samples(const Acq& q, double x, double z, int e, double th) {
  double st = std::sin(th), ct = std::cos(th);
  double ttx = (x * st + z * ct + 0.5 * q.aperture() * std::fabs(st)) / q.cbf;
  double dx = x - q.elem_x(e);
  double trx = std::sqrt(dx * dx + z * z) / q.cbf;
  return (ttx + trx) * q.fs;
}

// Eq. das: I_rf(x,z) = sum_tx sum_e w_e P(e, tau_e(x,z)), P read by linear interpolation,
// samples outside [0, N_s - 1] count as zero; transmits compounded coherently.
// Lines are independent outputs: they are computed on the host's threads, each line's sums in
// the same order as one thread would take them.
void das(const Acq& q, const Img& im, const double* rf, double* irf) {
  parallel_blocks(im.nl, host_threads(), [&](int, long long l_lo, long long l_hi) {
  for (int l = (int)l_lo; l < (int)l_hi; ++l)
    for (int d = 0; d < im.nd; ++d) {
      double x = line_x(im, l), z = depth_z(im, d), acc = 0;
      for (int tx = 0; tx < q.ntx; ++tx)
        for (int e = 0; e < q.ne; ++e) {
          double u = das_delay_samples(q, x, z, e, q.angles[tx]);
          double fl = std::floor(u);
          long long i = (long long)fl;
          double f = u - fl;
          const double* row = rf + ((size_t)tx * q.ne + e) * q.ns;
          double a = (i >= 0 && i < q.ns) ? row[i] : 0.0;
          double b = (i + 1 >= 0 && i + 1 < q.ns) ? row[i + 1] : 0.0;
          acc += apod(q, im, x, z, e) * ((1.0 - f) * a + f * b);
        }
      irf[(size_t)l * im.nd + d] = acc;
    }
  });
}

// Derivative of the beamformed image in the acquisition parameters, contracted with an image
// gradient, the RF held fixed: out[0] = sum_p gi(p) dI(p)/d c_bf, out[1] = .../d pitch,
// out[2 + t] = .../d th_t.  With u the delay in samples: d u/d c_bf = -u / c_bf; d u/d pitch =
// (W/2 |sin th| / p - (x - x_e) / r (e - (N_e - 1)/2)) fs / c_bf (the transmit term's aperture
// and the receive distance r to x_e = p (e - (N_e - 1)/2)); the transmit delay's d u/d th =
// (x cos th - z sin th + W/2 sgn(sin th) cos th) fs / c_bf (sgn(0) = 0).  dI/du is the slope of
// the linear-interpolation interval [floor(u), floor(u) + 1] holding u.  With a dynamic aperture
// the element weights depend on the pitch too: that term multiplies the interpolated sample.
void das_acq_vjp(const Acq& q, const Img& im, const double* rf, const double* gi, double* out) {
  for (int t = 0; t < 2 + q.ntx; ++t) out[t] = 0.0;
  for (int l = 0; l < im.nl; ++l)
    for (int d = 0; d < im.nd; ++d) {
      double x = line_x(im, l), z = depth_z(im, d), g = gi[(size_t)l * im.nd + d];
      if (g == 0.0) continue;
      for (int tx = 0; tx < q.ntx; ++tx) {
        const double th = q.angles[tx], st = std::sin(th), ct = std::cos(th);
        const double sg = st > 0 ? 1.0 : (st < 0 ? -1.0 : 0.0);
        const double du_dth = (x * ct - z * st + 0.5 * q.aperture() * sg * ct) * q.fs / q.cbf;
        for (int e = 0; e < q.ne; ++e) {
          double u = das_delay_samples(q, x, z, e, th);
          double fl = std::floor(u);
          long long i = (long long)fl;
          const double* row = rf + ((size_t)tx * q.ne + e) * q.ns;
          double a = (i >= 0 && i < q.ns) ? row[i] : 0.0;
          double b = (i + 1 >= 0 && i + 1 < q.ns) ? row[i + 1] : 0.0;
          const double dx = x - q.elem_x(e), r = std::sqrt(dx * dx + z * z);
          const double du_dp = (0.5 * (q.ne - 1) * std::fabs(st) - dx / r * (e - 0.5 * (q.ne - 1))) * q.fs / q.cbf;
          double dw_dp;
          const double w = apod(q, im, x, z, e, &dw_dp);
          const double gs = g * w * (b - a);
          out[1] += g * dw_dp * ((1.0 - (u - fl)) * a + (u - fl) * b);  // the weight's own pitch term
          out[0] += gs * (-u / q.cbf);
          out[1] += gs * du_dp;
          out[2 + tx] += gs * du_dth;
        }
      }
    }
}

// Eq. das_adjoint: scatter the image gradient back to the two interpolation samples.  Channel
// rows (transmit, element) are independent outputs, computed on the host's threads; every row
// takes its pixels in line-then-depth order.
void das_adjoint(const Acq& q, const Img& im, const double* gi, double* grf) {
  parallel_blocks((long long)q.ntx * q.ne, host_threads(), [&](int, long long r_lo, long long r_hi) {
    for (long long r = r_lo; r < r_hi; ++r) {
      const int tx = (int)(r / q.ne), e = (int)(r % q.ne);
      double* row = grf + (size_t)r * q.ns;
      for (int l = 0; l < im.nl; ++l)
        for (int d = 0; d < im.nd; ++d) {
          double x = line_x(im, l), z = depth_z(im, d), g = gi[(size_t)l * im.nd + d];
          double u = das_delay_samples(q, x, z, e, q.angles[tx]);
          double fl = std::floor(u);
          long long i = (long long)fl;
          double f = u - fl;
          double w = apod(q, im, x, z, e);
          if (i >= 0 && i < q.ns) row[i] += w * (1.0 - f) * g;
          if (i + 1 >= 0 && i + 1 < q.ns) row[i + 1] += w * f * g;
        }
    }
  });
}

// discrete Fourier transform, sign -1 forward / +1 inverse (unnormalised).  Radix-2
// Cooley-Tukey for powers of two, the O(N^2) definition otherwise.
void dft(std::vector<double>& re, std::vector<double>& im, int sign) {
  size_t n = re.size();
  if (n && (n & (n - 1)) == 0) {
    for (size_t i = 1, j = 0; i < n; ++i) {  // bit reversal
      size_t bit = n >> 1;
      for (; j & bit; bit >>= 1) j ^= bit;
      j ^= bit;
      if (i < j) {
        std::swap(re[i], re[j]);
        std::swap(im[i], im[j]);
      }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
      for (size_t i = 0; i < n; i += len)
        for (size_t k = 0; k < len / 2; ++k) {
          double ang = sign * 2.0 * PI * (double)k / (double)len;
          double wr = std::cos(ang), wi = std::sin(ang);
          size_t a = i + k, b = i + k + len / 2;
          double xr = re[b] * wr - im[b] * wi, xi = re[b] * wi + im[b] * wr;
          re[b] = re[a] - xr;
          im[b] = im[a] - xi;
          re[a] += xr;
          im[a] += xi;
        }
    }
    return;
  }
  std::vector<double> r2(n), i2(n);
  for (size_t k = 0; k < n; ++k) {
    double sr = 0, si = 0;
    for (size_t j = 0; j < n; ++j) {
      double ang = sign * 2.0 * PI * (double)((k * j) % n) / (double)n;
      sr += re[j] * std::cos(ang) - im[j] * std::sin(ang);
      si += re[j] * std::sin(ang) + im[j] * std::cos(ang);
    }
    r2[k] = sr;
    i2[k] = si;
  }
  re = r2;
  im = i2;
}

// Hilbert transform of a real line via the analytic signal: X = DFT(x), multiply by
// h = [1, 2 ... 2, (1 at N/2 for even N), 0 ...], inverse DFT; returns Im(analytic) in y.
void hilbert(const double* x, int n, double* y) {
  std::vector<double> re(x, x + n), im(n, 0.0);
  dft(re, im, -1);
  for (int k = 0; k < n; ++k) {
    double h;
    if (k == 0) h = 1;
    else if (2 * k < n) h = 2;
    else if (2 * k == n) h = 1;
    else h = 0;
    re[k] *= h;
    im[k] *= h;
  }
  dft(re, im, +1);
  for (int k = 0; k < n; ++k) y[k] = im[k] / n;
}

// envelope |x + i H(x)| per line along depth (the baseband demodulation of Sec. 2.3.4)
void envelope(const Img& im, const double* irf, double* env) {
  std::vector<double> y(im.nd);
  for (int l = 0; l < im.nl; ++l) {
    const double* x = irf + (size_t)l * im.nd;
    hilbert(x, im.nd, y.data());
    for (int d = 0; d < im.nd; ++d) env[(size_t)l * im.nd + d] = std::sqrt(x[d] * x[d] + y[d] * y[d]);
  }
}

// log compression with dynamic-range limit: B = max(20 log10(E / E_max), -DR)
long long log_compress(const Img& im, const double* env, double* b) {
  size_t n = (size_t)im.nl * im.nd;
  long long am = 0;
  for (size_t i = 1; i < n; ++i)
    if (env[i] > env[am]) am = (long long)i;
  double emax = n ? env[am] : 0.0;
  for (size_t i = 0; i < n; ++i) {
    double v = -im.dr;
    if (emax > 0 && env[i] > 0) v = std::max(20.0 * std::log10(env[i] / emax), -im.dr);
    b[i] = v;
  }
  return am;
}

// Eq. weighted_l1_l2_loss and its exact gradient (sign(0) = 0)
double loss_grad(const Img& im, const double* b, const double* bref, double* gb) {
  size_t n = (size_t)im.nl * im.nd;
  double s1 = 0, s2 = 0;
  for (size_t i = 0; i < n; ++i) {
    double r = b[i] - bref[i];
    s1 += std::fabs(r);
    s2 += r * r;
    if (gb) gb[i] = (im.l1 * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) + 2.0 * im.l2 * r) / (double)n;
  }
  return (im.l1 * s1 + im.l2 * s2) / (double)n;
}

// VJP of B(irf): log (20/ln10 / E on unclipped pixels, E_max's share to the first argmax),
// then the envelope E = |x + i H x|: g_x = (x/E) g_E + H^T((y/E) g_E), with H^T = -H.
void envlog_vjp(const Img& im, const double* irf, const double* gb, double* gi) {
  size_t n = (size_t)im.nl * im.nd;
  std::vector<double> env(n), b(n), y(n), ge(n, 0.0);
  for (int l = 0; l < im.nl; ++l) hilbert(irf + (size_t)l * im.nd, im.nd, &y[(size_t)l * im.nd]);
  for (size_t i = 0; i < n; ++i) env[i] = std::sqrt(irf[i] * irf[i] + y[i] * y[i]);
  long long am = log_compress(im, env.data(), b.data());
  double emax = env[am];
  const double c = 20.0 / std::log(10.0);
  double smax = 0;
  for (size_t i = 0; i < n; ++i) {
    bool live = emax > 0 && env[i] > 0 && 20.0 * std::log10(env[i] / emax) > -im.dr;
    if (!live) continue;
    ge[i] += gb[i] * c / env[i];
    smax += gb[i] * c / emax;
  }
  ge[am] -= smax;
  std::vector<double> v(im.nd), hv(im.nd);
  for (int l = 0; l < im.nl; ++l) {
    size_t o = (size_t)l * im.nd;
    for (int d = 0; d < im.nd; ++d) {
      double e = env[o + d];
      v[d] = e > 0 ? y[o + d] / e * ge[o + d] : 0.0;
    }
    hilbert(v.data(), im.nd, hv.data());
    for (int d = 0; d < im.nd; ++d) {
      double e = env[o + d];
      gi[o + d] = (e > 0 ? irf[o + d] / e * ge[o + d] : 0.0) - hv[d];
    }
  }
}

}  // namespace

// ==========================================================================================
// C ABI used by oracle/oracle.py (ctypes)
// ==========================================================================================
extern "C" {

void ora_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, uint32_t* out) {
  U4 r = philox(c0, c1, c2, c3, k0, k1);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

// n blocks with counters (c0_base + i, c1, c2, c3); out[4 i + j]
void ora_philox_fill(uint32_t c0_base, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, long long n,
                     uint32_t* out) {
  for (long long i = 0; i < n; ++i) {
    U4 r = philox(c0_base + (uint32_t)i, c1, c2, c3, k0, k1);
    for (int j = 0; j < 4; ++j) out[4 * i + j] = r.v[j];
  }
}

void* ora_scene_create(int nt, const double* tri, const int* media, int ns, const double* sp, const double* samp,
                       double rs, int use_bvh, int rough) {
  Scene* s = new Scene();
  s->nt = nt;
  s->rough = rough != 0;
  for (int i = 0; i < nt; ++i) {
    const double* t = tri + 9 * (size_t)i;
    s->v0.push_back(d3(t[0], t[1], t[2]));
    s->v1.push_back(d3(t[3], t[4], t[5]));
    s->v2.push_back(d3(t[6], t[7], t[8]));
    s->mfront.push_back(media[2 * i]);
    s->mback.push_back(media[2 * i + 1]);
  }
  s->nsct = ns;
  for (int j = 0; j < ns; ++j) {
    s->sp.push_back(d3(sp[3 * j], sp[3 * j + 1], sp[3 * j + 2]));
    s->samp.push_back(samp[j]);
  }
  s->rs = rs;
  if (use_bvh) s->build_bvh();
  return s;
}

void ora_scene_free(void* s) { delete (Scene*)s; }

// GGX microfacet normal around the unit normal n for the uniforms (u2, u3) (tests)
void ora_ggx_normal(const double* n, double alpha, double u2, double u3, double* h) {
  D3 r = ggx_normal<double>(d3(n[0], n[1], n[2]), alpha, u2, u3);
  h[0] = r.x;
  h[1] = r.y;
  h[2] = r.z;
}

// emission of n consecutive rays ray_lo .. ray_lo + n - 1 of transmit tx (tests):
// out[8 i ..] = {o0 (3), w0 (3), a0, tau0}
void ora_emit(const double* acq, const double* angles, uint64_t seed, int tx, long long ray_lo, long long n,
              double* out) {
  Acq q = make_acq(acq, angles);
  for (long long i = 0; i < n; ++i) {
    D3 o0, w0;
    double a0, tau0, xe;
    emit_ray(q, (uint32_t)seed, (uint32_t)(seed >> 32), tx, ray_lo + i, o0, w0, a0, tau0, xe);
    double* r = out + 8 * i;
    r[0] = o0.x; r[1] = o0.y; r[2] = o0.z;
    r[3] = w0.x; r[4] = w0.y; r[5] = w0.z;
    r[6] = a0;
    r[7] = tau0;
  }
}

// interface event (tests): out = {tir, cos_i, cos_t, R, T, wr[3], wt[3]}
void ora_interface(const double* w, const double* nin, double c1, double c2, double rho1, double rho2, double* out) {
  Iface<double> f = interface_event<double>(d3(w[0], w[1], w[2]), d3(nin[0], nin[1], nin[2]), c1, c2, rho1, rho2);
  out[0] = f.tir;
  out[1] = f.ci;
  out[2] = f.ct;
  out[3] = f.R;
  out[4] = f.T;
  out[5] = f.wr.x; out[6] = f.wr.y; out[7] = f.wr.z;
  out[8] = f.wt.x; out[9] = f.wt.y; out[10] = f.wt.z;
}

// closest hit (tests): out = {t, cls, id}
void ora_closest(void* sp, const double* o, const double* w, int xcls, int xid, double* out) {
  const Scene& s = *(Scene*)sp;
  Hit h;
  h.t = 1e300;
  h.cls = CLS_NONE;
  h.id = -1;
  closest_scene(s, d3(o[0], o[1], o[2]), d3(w[0], w[1], w[2]), xcls, xid, h);
  out[0] = h.cls == CLS_NONE ? -1 : h.t;
  out[1] = h.cls;
  out[2] = h.id;
}

// forward transport over paths [path_lo, path_hi) of the acquisition
void* ora_trace(void* scene, const double* theta, int M, const double* acq, const double* angles, uint64_t seed,
                int nthreads, long long path_lo, long long path_hi) {
  Run* r = new Run();
  r->q = make_acq(acq, angles);
  r->M = M;
  if (path_hi < 0) path_hi = r->q.n_paths();
  r->path_lo = path_lo;
  r->n_paths = path_hi - path_lo;
  r->K1 = r->q.kmax + 1;
  r->rec.resize((size_t)r->n_paths * r->K1);
  forward_run(*(Scene*)scene, theta, *r, seed, nthreads, path_lo, path_hi);
  return r;
}

void ora_run_free(void* r) { delete (Run*)r; }
long long ora_run_n_arrivals(void* r) { return (long long)((Run*)r)->arr.size(); }
void ora_run_counters(void* r, long long* out) {
  out[0] = ((Run*)r)->cnt.segments;
  out[1] = ((Run*)r)->cnt.nee;
}
void ora_run_arrivals(void* rp, int* tx, int* e, double* tau, double* a, long long* path, int* kind, int* ev) {
  Run* r = (Run*)rp;
  for (size_t i = 0; i < r->arr.size(); ++i) {
    const Arrival<double>& A = r->arr[i];
    tx[i] = A.tx;
    e[i] = A.e;
    tau[i] = A.tau;
    a[i] = A.a;
    path[i] = A.path;
    kind[i] = A.kind;
    ev[i] = A.ev;
  }
}
// per-path records: cls, id, choice, aux arrays of n_paths * (kmax + 1)
void ora_run_records(void* rp, int* cls, int* id, int* choice, int* aux) {
  Run* r = (Run*)rp;
  for (size_t i = 0; i < r->rec.size(); ++i) {
    cls[i] = r->rec[i].cls;
    id[i] = r->rec[i].id;
    choice[i] = r->rec[i].choice;
    aux[i] = r->rec[i].aux;
  }
}

// splat of the run's arrivals into rf[ntx][ne][ns] (zeroed by the caller)
void ora_splat_run(void* rp, const double* theta, double* rf) {
  Run* r = (Run*)rp;
  splat_direct(r->q, theta[3 * r->M + 1], r->arr.data(), (long long)r->arr.size(), rf);
}

// splat of an explicit arrival list (stage tests)
void ora_splat(const double* acq, const double* angles, double f0, long long n, const int* tx, const int* e,
               const double* tau, const double* a, double* rf) {
  Acq q = make_acq(acq, angles);
  std::vector<Arrival<double>> arr(n);
  for (long long i = 0; i < n; ++i) {
    arr[i].tx = tx[i];
    arr[i].e = e[i];
    arr[i].tau = tau[i];
    arr[i].a = a[i];
  }
  splat_direct(q, f0, arr.data(), n, rf);
}

// splat adjoint per arrival: ga = sum_n g s(t_n - tau), gt = -a sum_n g s'(t_n - tau),
// gf = a sum_n g ds/df0 (sigma follows f0), by forward-mode duals of the pulse.
void ora_splat_adjoint(const double* acq, const double* angles, double f0, long long n, const int* tx, const int* e,
                       const double* tau, const double* a, const double* grf, double* ga, double* gt, double* gf) {
  Acq q = make_acq(acq, angles);
  double sig = pulse_sigma<double>(f0, q.bw);
  for (long long i = 0; i < n; ++i) {
    int n0, n1;
    pulse_window(tau[i], sig, q, n0, n1);
    Dual T(tau[i]), F(f0);
    T.d[0] = 1;
    F.d[1] = 1;
    Dual S = pulse_sigma<Dual>(F, q.bw);
    double sa = 0, st = 0, sf = 0;
    const double* row = grf + ((size_t)tx[i] * q.ne + e[i]) * q.ns;
    for (int s = n0; s <= n1; ++s) {
      Dual p = pulse<Dual>(Dual(s / q.fs) - T, F, S);
      sa += row[s] * p.v;
      st += row[s] * p.d[0];
      sf += row[s] * p.d[1];
    }
    ga[i] = sa;
    gt[i] = a[i] * st;
    gf[i] = a[i] * sf;
  }
}

void ora_das(const double* acq, const double* angles, const double* img, const double* rf, double* irf) {
  das(make_acq(acq, angles), make_img(img), rf, irf);
}
void ora_das_adjoint(const double* acq, const double* angles, const double* img, const double* gi, double* grf) {
  das_adjoint(make_acq(acq, angles), make_img(img), gi, grf);
}
void ora_das_acq_vjp(const double* acq, const double* angles, const double* img, const double* rf, const double* gi,
                     double* out) {
  das_acq_vjp(make_acq(acq, angles), make_img(img), rf, gi, out);
}
void ora_hilbert(const double* x, int n, double* y) { hilbert(x, n, y); }
void ora_envelope(const double* img, const double* irf, double* env) { envelope(make_img(img), irf, env); }
long long ora_log_compress(const double* img, const double* env, double* b) { return log_compress(make_img(img), env, b); }
double ora_loss(const double* img, const double* b, const double* bref, double* gb) {
  return loss_grad(make_img(img), b, bref, gb);
}
void ora_envlog_vjp(const double* img, const double* irf, const double* gb, double* gi) {
  envlog_vjp(make_img(img), irf, gb, gi);
}

// replay of a run's frozen decisions at (possibly perturbed) theta -> rf (double), for
// finite differences on the same frozen realisation
void ora_replay_rf(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, double* rf) {
  Run* r = (Run*)rp;
  const Scene& sc = *(Scene*)scene;
  const Acq& q = r->q;
  Phys<double> P = phys_double(theta, r->M, ((Scene*)scene)->rough);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  std::vector<std::vector<Arrival<double>>> parts(std::max(1, nthreads));
  std::vector<Counters> cnts(std::max(1, nthreads));
  parallel_blocks(r->n_paths, nthreads, [&](int b, long long lo, long long hi) {
    for (long long i = lo; i < hi; ++i) {
      PathIO io = path_io(q, r->path_lo + i);
      trace_path<double>(sc, P, q, k0, k1, io, r->path_lo + i, &r->rec[(size_t)i * r->K1], nullptr, parts[b],
                         cnts[b]);
    }
  });
  for (auto& p : parts) splat_direct(q, P.f0, p.data(), (long long)p.size(), rf);
}

// gradient of sum_{tx,e,n} grf[tx][e][n] * RF[tx][e][n] w.r.t. theta on the run's frozen
// realisation (forward-mode duals through replay and the pulse; Eq. chain_rule)
// gradient of sum(grf * RF) on the frozen realisation; with_acq: also in c_bf, the pitch and the
// steering angles (emission and secondary-ray targets), appended after the 3M + 2 scene
// parameters.
// Returns -1 when the duals cannot hold that many parameters.
// n_shape > 0: also in n_shape shape parameters whose vertex tangents are vtan
// [n_shape][n_tris][9], appended after the others.
// gabs (may be null): per component the sum over arrivals of |contribution|, the scale below
// which a sum of those terms in finite precision cannot be resolved (its condition)
static int gradient_impl(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, const double* grf,
                         double* gtheta, bool with_acq, int n_shape = 0, const double* vtan = nullptr,
                         double* gabs = nullptr) {
  Run* r = (Run*)rp;
  const Scene& sc = *(Scene*)scene;
  const Acq& q = r->q;
  Phys<Dual> P = phys_dual(theta, r->M, sc.rough);
  int np = 3 * r->M + 2 + (sc.rough ? r->M : 0);
  if (with_acq) {
    P.acq_base = np;
    np += 2 + q.ntx;
  }
  if (n_shape > 0) {
    P.shape_base = np;
    P.n_shape = n_shape;
    P.vtan = vtan;
    np += n_shape;
  }
  if (np > NP) return -1;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  int nb = std::max(1, nthreads);
  std::vector<std::vector<double>> acc(nb, std::vector<double>(np, 0.0)), aabs(nb, std::vector<double>(np, 0.0));
  parallel_blocks(r->n_paths, nthreads, [&](int b, long long lo, long long hi) {
    std::vector<Arrival<Dual>> arr;
    Counters c;
    for (long long i = lo; i < hi; ++i) {
      arr.clear();
      PathIO io = path_io(q, r->path_lo + i);
      trace_path<Dual>(sc, P, q, k0, k1, io, r->path_lo + i, &r->rec[(size_t)i * r->K1], nullptr, arr, c);
      for (const Arrival<Dual>& A : arr) {
        Dual sig = pulse_sigma<Dual>(P.f0, q.bw);
        int n0, n1;
        pulse_window(A.tau.v, sig.v, q, n0, n1);
        const double* row = grf + ((size_t)A.tx * q.ne + A.e) * q.ns;
        Dual s(0.0);
        for (int n = n0; n <= n1; ++n) {
          if (row[n] == 0.0) continue;
          s = s + row[n] * pulse<Dual>(Dual(n / q.fs) - A.tau, P.f0, sig);
        }
        Dual contrib = A.a * s;
        for (int k = 0; k < np; ++k) {
          acc[b][k] += contrib.d[k];
          aabs[b][k] += std::fabs(contrib.d[k]);
        }
      }
    }
  });
  for (int k = 0; k < np; ++k) {
    double s = 0, sa = 0;
    for (int b = 0; b < nb; ++b) {
      s += acc[b][k];
      sa += aabs[b][k];
    }
    gtheta[k] = s;
    if (gabs) gabs[k] = sa;
  }
  return 0;
}

// the gradient and, per component, the sum over arrivals of |contribution|
void ora_gradient_cond(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, const double* grf,
                       double* gtheta, double* gabs) {
  gradient_impl(scene, rp, theta, seed, nthreads, grf, gtheta, false, 0, nullptr, gabs);
}

void ora_gradient(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, const double* grf,
                  double* gtheta) {
  gradient_impl(scene, rp, theta, seed, nthreads, grf, gtheta, false);
}

int ora_gradient_acq(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, const double* grf,
                     double* gtheta) {
  return gradient_impl(scene, rp, theta, seed, nthreads, grf, gtheta, true);
}

// gradient in the scene parameters followed by the derivatives along n_shape vertex tangent
// fields vtan [n_shape][n_tris][9] (fixed-sample: the hit and crossed triangles held fixed)
int ora_gradient_shape(void* scene, void* rp, const double* theta, uint64_t seed, int nthreads, const double* grf,
                       int n_shape, const double* vtan, double* gtheta) {
  if (n_shape < 1) return -1;
  return gradient_impl(scene, rp, theta, seed, nthreads, grf, gtheta, false, n_shape, vtan);
}

// n injected paths (tests): origins o[3 n], unit directions w[3 n], weight 1, time 0, ray
// index = path index.  Per element: the sum of what each path deposits there and the sum of
// the squares of those per-path amounts (sum_e[n_elem], sq_e[n_elem], zeroed here).
void ora_inject_sums(void* scene, const double* theta, int M, const double* acq, const double* angles, uint64_t seed,
                     long long n, const double* o, const double* w, int nthreads, double* sum_e, double* sq_e) {
  Acq q = make_acq(acq, angles);
  const Scene& sc = *(Scene*)scene;
  Phys<double> P = phys_double(theta, M, sc.rough);
  const int nb = std::max(1, nthreads);
  std::vector<std::vector<double>> s(nb, std::vector<double>(q.ne, 0.0)), s2(nb, std::vector<double>(q.ne, 0.0));
  parallel_blocks(n, nthreads, [&](int b, long long lo, long long hi) {
    std::vector<Arrival<double>> arr;
    std::vector<double> per(q.ne);
    Counters c;
    for (long long i = lo; i < hi; ++i) {
      PathIO io;
      io.inject = true;
      io.o0 = d3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
      io.w0 = d3(w[3 * i], w[3 * i + 1], w[3 * i + 2]);
      io.a0 = 1.0;
      io.tau0 = 0.0;
      io.ray = i;
      arr.clear();
      trace_path<double>(sc, P, q, (uint32_t)seed, (uint32_t)(seed >> 32), io, i, nullptr, nullptr, arr, c);
      std::fill(per.begin(), per.end(), 0.0);
      for (const auto& A : arr) per[A.e] += A.a;
      for (int e = 0; e < q.ne; ++e) {
        s[b][e] += per[e];
        s2[b][e] += per[e] * per[e];
      }
    }
  });
  for (int e = 0; e < q.ne; ++e) {
    sum_e[e] = sq_e[e] = 0.0;
    for (int b = 0; b < nb; ++b) {
      sum_e[e] += s[b][e];
      sq_e[e] += s2[b][e];
    }
  }
}

// single injected path (tests): emission state given, optional forced interface choices,
// optional physical (R / T) weights.  Returns the number of arrivals written (<= cap).
int ora_trace_injected(void* scene, const double* theta, int M, const double* acq, const double* angles, uint64_t seed,
                       const double* o, const double* w, double a0, double tau0, int tx, long long ray,
                       const int* forced, int n_forced, int physical, int cap, int* e_out, double* tau_out,
                       double* a_out, int* kind_out, int* rec_out, double* last_state) {
  Acq q = make_acq(acq, angles);
  Phys<double> P = phys_double(theta, M, ((Scene*)scene)->rough);
  PathIO io;
  io.inject = true;
  io.o0 = d3(o[0], o[1], o[2]);
  io.w0 = d3(w[0], w[1], w[2]);
  io.a0 = a0;
  io.tau0 = tau0;
  io.tx = tx;
  io.ray = ray;
  io.forced = forced;
  io.n_forced = n_forced;
  io.physical = physical != 0;
  io.last_state = last_state;
  std::vector<Rec> rec(q.kmax + 1);
  for (auto& x : rec) x.cls = CLS_NONE, x.id = -1, x.choice = CH_NONE, x.aux = -1;
  std::vector<Arrival<double>> arr;
  Counters c;
  trace_path<double>(*(Scene*)scene, P, q, (uint32_t)seed, (uint32_t)(seed >> 32), io, 0, nullptr, rec.data(), arr, c);
  int n = std::min(cap, (int)arr.size());
  for (int i = 0; i < n; ++i) {
    e_out[i] = arr[i].e;
    tau_out[i] = arr[i].tau;
    a_out[i] = arr[i].a;
    kind_out[i] = arr[i].kind;
  }
  if (rec_out)
    for (int k = 0; k <= q.kmax; ++k) {
      rec_out[4 * k] = rec[k].cls;
      rec_out[4 * k + 1] = rec[k].id;
      rec_out[4 * k + 2] = rec[k].choice;
      rec_out[4 * k + 3] = rec[k].aux;
    }
  return n;
}

}  // extern "C"
