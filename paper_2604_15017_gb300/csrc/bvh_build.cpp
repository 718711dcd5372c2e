// Host-side acceleration structures of the usrt scene.
//
// Triangles: a BVH2 built by binned surface-area heuristic, used by both closest-hit queries and
// the all-crossings queries of secondary rays.  Scatterer spheres (tiny, spread through whole
// regions of tissue) go into a uniform grid instead: a ray marches its cells front to back (3D
// DDA), so finding the nearest sphere costs a short sequence of independent cell reads rather
// than a long chain of dependent BVH node reads through a dense cloud of tiny boxes.  The
// device layout of the BVH2 is one whose
// inner nodes hold both children's boxes in four 16-byte words, so a traversal step is four
// 128-bit loads of one 64-byte (32-byte aligned) node:
//   n0 = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)   n1 = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   n2 = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)   n3 = int4(child0, child1, count0, count1)
// count_i == 0: child_i is an inner node index (or -1 = empty); count_i > 0: child_i is the
// first primitive of a leaf in the leaf-ordered primitive array.
#include "bvh_build.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace usrt {

namespace {

struct Box {
  double lo[3], hi[3];
  void empty() {
    for (int a = 0; a < 3; ++a) {
      lo[a] = 1e300;
      hi[a] = -1e300;
    }
  }
  void grow(const Box& b) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], b.lo[a]);
      hi[a] = std::max(hi[a], b.hi[a]);
    }
  }
  void grow(const double p[3]) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], p[a]);
      hi[a] = std::max(hi[a], p[a]);
    }
  }
  double area() const {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = std::max(0.0, hi[a] - lo[a]);
    return 2.0 * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
  }
  bool valid() const { return lo[0] <= hi[0]; }
};

struct TNode {
  Box box;
  int left = -1, right = -1;  // tree children (inner)
  int first = 0, count = 0;   // leaf range (count > 0)
};

const int LEAF_MAX = 8;    // a node with more primitives is always split
const int BINS = 16;
const double C_TRAV = 1.0;  // cost of visiting a node relative to one primitive test (SAH)

struct Builder {
  std::vector<Box> pbox;
  std::vector<double> cen;  // 3 per prim
  std::vector<int> idx;
  std::vector<TNode> tree;

  int make_leaf(const Box& b, int first, int count) {
    TNode n;
    n.box = b;
    n.first = first;
    n.count = count;
    tree.push_back(n);
    return (int)tree.size() - 1;
  }

  int build(int first, int count) {
    Box b, cb;
    b.empty();
    cb.empty();
    for (int i = first; i < first + count; ++i) {
      b.grow(pbox[idx[i]]);
      cb.grow(&cen[3 * (size_t)idx[i]]);
    }
    if (count <= 1) return make_leaf(b, first, count);
    // binned SAH over the three axes
    int best_axis = -1, best_split = -1;
    double best_cost = 1e300;
    for (int a = 0; a < 3; ++a) {
      double ext = cb.hi[a] - cb.lo[a];
      if (!(ext > 0)) continue;
      Box bins[BINS];
      int cnt[BINS];
      for (int k = 0; k < BINS; ++k) {
        bins[k].empty();
        cnt[k] = 0;
      }
      double scale = BINS / ext;
      for (int i = first; i < first + count; ++i) {
        int k = std::min(BINS - 1, (int)((cen[3 * (size_t)idx[i] + a] - cb.lo[a]) * scale));
        bins[k].grow(pbox[idx[i]]);
        cnt[k]++;
      }
      double rarea[BINS];
      int rcnt[BINS];
      Box acc;
      acc.empty();
      int c = 0;
      for (int k = BINS - 1; k > 0; --k) {
        if (cnt[k]) acc.grow(bins[k]);
        c += cnt[k];
        rarea[k] = acc.valid() ? acc.area() : 0.0;
        rcnt[k] = c;
      }
      acc.empty();
      c = 0;
      for (int k = 0; k < BINS - 1; ++k) {
        if (cnt[k]) acc.grow(bins[k]);
        c += cnt[k];
        if (c == 0 || rcnt[k + 1] == 0) continue;
        double cost = (acc.valid() ? acc.area() : 0.0) * c + rarea[k + 1] * rcnt[k + 1];
        if (cost < best_cost) {
          best_cost = cost;
          best_axis = a;
          best_split = k;
        }
      }
    }
    // surface-area heuristic termination: a leaf costs `count` primitive tests, a split one node
    // visit plus the children's tests weighted by the probability of entering them
    const double area = b.area();
    if (count <= LEAF_MAX) {
      const double split_cost = best_axis < 0 || !(area > 0) ? 1e300 : C_TRAV + best_cost / area;
      if ((double)count <= split_cost) return make_leaf(b, first, count);
    }
    int mid;
    if (best_axis < 0) {
      // all centroids coincide: split the range in half
      mid = first + count / 2;
    } else {
      double ext = cb.hi[best_axis] - cb.lo[best_axis];
      double scale = BINS / ext;
      auto it = std::partition(idx.begin() + first, idx.begin() + first + count, [&](int p) {
        int k = std::min(BINS - 1, (int)((cen[3 * (size_t)p + best_axis] - cb.lo[best_axis]) * scale));
        return k <= best_split;
      });
      mid = (int)(it - idx.begin());
      if (mid == first || mid == first + count) mid = first + count / 2;
    }
    int me = (int)tree.size();
    tree.push_back(TNode());
    tree[me].box = b;
    int l = build(first, mid - first);
    int r = build(mid, first + count - mid);
    tree[me].left = l;
    tree[me].right = r;
    return me;
  }
};

float round_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
float round_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}
float bits_f(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

// BVH over the triangles: device nodes and triangles in leaf order
static void build_tri_bvh(const HostSceneIn& in, std::vector<float>& nodes_out, std::vector<float>& prims_out,
                          int& n_nodes_out, int& depth_out, std::vector<float>& nodes4_out, int& n_nodes4_out,
                          int& depth4_out) {
  const int n = in.n_tris;
  Builder B;
  B.pbox.resize(n);
  B.cen.resize(3 * (size_t)n);
  B.idx.resize(n);
  for (int k = 0; k < n; ++k) {
    Box b;
    b.empty();
    for (int v = 0; v < 3; ++v) {
      double p[3] = {in.tris[9 * (size_t)k + 3 * v], in.tris[9 * (size_t)k + 3 * v + 1], in.tris[9 * (size_t)k + 3 * v + 2]};
      b.grow(p);
    }
    B.pbox[k] = b;
    for (int a = 0; a < 3; ++a) B.cen[3 * (size_t)k + a] = 0.5 * (b.lo[a] + b.hi[a]);
    B.idx[k] = k;
  }
  B.tree.reserve(2 * (size_t)n + 2);
  int root = n ? B.build(0, n) : -1;

  // device nodes: one per inner tree node, DFS order; a leaf root gets a wrapper node
  std::vector<int> gpu_index(B.tree.size(), -1);
  std::vector<int> depth(B.tree.size(), 0);
  std::vector<int> order;  // inner tree nodes in DFS order
  int maxd = 1;
  if (root >= 0) {
    std::vector<int> st(1, root);
    depth[root] = 1;
    while (!st.empty()) {
      int t = st.back();
      st.pop_back();
      maxd = std::max(maxd, depth[t]);
      if (B.tree[t].count > 0) continue;
      gpu_index[t] = (int)order.size();
      order.push_back(t);
      depth[B.tree[t].left] = depth[B.tree[t].right] = depth[t] + 1;
      st.push_back(B.tree[t].right);
      st.push_back(B.tree[t].left);
    }
  }
  depth_out = maxd;
  auto child_fields = [&](int c, float* lo, float* hi, int& ci, int& cnt) {
    if (c < 0) {
      for (int a = 0; a < 3; ++a) {
        lo[a] = 1.0f;
        hi[a] = -1.0f;  // never traversed: count 0 and index -1
      }
      ci = -1;
      cnt = 0;
      return;
    }
    const TNode& t = B.tree[c];
    for (int a = 0; a < 3; ++a) {
      lo[a] = round_down(t.box.lo[a]);
      hi[a] = round_up(t.box.hi[a]);
    }
    if (t.count > 0) {
      ci = t.first;
      cnt = t.count;
    } else {
      ci = gpu_index[c];
      cnt = 0;
    }
  };
  nodes_out.clear();
  auto emit = [&](int c0, int c1) {
    float lo0[3], hi0[3], lo1[3], hi1[3];
    int i0, i1, n0, n1;
    child_fields(c0, lo0, hi0, i0, n0);
    child_fields(c1, lo1, hi1, i1, n1);
    float w[16] = {lo0[0], hi0[0], lo0[1], hi0[1], lo1[0], hi1[0], lo1[1], hi1[1],
                   lo0[2], hi0[2], lo1[2], hi1[2], bits_f((uint32_t)i0), bits_f((uint32_t)i1),
                   bits_f((uint32_t)n0), bits_f((uint32_t)n1)};
    nodes_out.insert(nodes_out.end(), w, w + 16);
  };
  if (root < 0) {
    emit(-1, -1);
  } else if (B.tree[root].count > 0) {
    emit(root, -1);
  } else {
    for (int t : order) emit(B.tree[t].left, B.tree[t].right);
  }
  n_nodes_out = (int)(nodes_out.size() / 16);

  // 4-wide BVH by collapsing the binary tree: a node's children are found by repeatedly
  // replacing its inner child of largest surface area with that child's two children, until
  // there are four or only leaves remain.  Device layout, 32 floats (128 bytes) per node:
  // lo.x[4], hi.x[4], lo.y[4], hi.y[4], lo.z[4], hi.z[4], int child[4], int count[4]; count > 0:
  // a leaf of `count` triangles from `child`; count 0: an inner node (child >= 0) or an empty
  // slot (child -1, inverted box).
  nodes4_out.clear();
  depth4_out = 1;
  std::vector<int> work;  // binary inner nodes waiting to become 4-wide nodes
  std::vector<int> id4(B.tree.size(), -1), dep4(B.tree.size(), 1);
  auto children4 = [&](int t, int* ch) {
    int nc = 2;
    ch[0] = B.tree[t].left;
    ch[1] = B.tree[t].right;
    while (nc < 4) {
      int best = -1;
      double area = -1.0;
      for (int i = 0; i < nc; ++i)
        if (B.tree[ch[i]].count == 0 && B.tree[ch[i]].box.area() > area) {
          area = B.tree[ch[i]].box.area();
          best = i;
        }
      if (best < 0) break;
      const int c = ch[best];
      ch[best] = B.tree[c].left;
      ch[nc++] = B.tree[c].right;
    }
    for (int i = nc; i < 4; ++i) ch[i] = -1;
    return nc;
  };
  std::vector<int> order4;
  if (root >= 0 && B.tree[root].count == 0) {
    // number the 4-wide nodes in DFS order
    std::vector<int> st(1, root);
    while (!st.empty()) {
      const int t = st.back();
      st.pop_back();
      id4[t] = (int)order4.size();
      order4.push_back(t);
      depth4_out = std::max(depth4_out, dep4[t]);
      int ch[4];
      children4(t, ch);
      for (int i = 3; i >= 0; --i)
        if (ch[i] >= 0 && B.tree[ch[i]].count == 0) {
          dep4[ch[i]] = dep4[t] + 1;
          st.push_back(ch[i]);
        }
    }
  }
  auto emit4 = [&](const int* ch) {
    float w[32];
    for (int i = 0; i < 4; ++i) {
      float lo[3], hi[3];
      int ci, cnt;
      child_fields(ch[i], lo, hi, ci, cnt);
      if (ch[i] >= 0 && B.tree[ch[i]].count == 0) ci = id4[ch[i]];
      w[0 + i] = lo[0];
      w[4 + i] = hi[0];
      w[8 + i] = lo[1];
      w[12 + i] = hi[1];
      w[16 + i] = lo[2];
      w[20 + i] = hi[2];
      w[24 + i] = bits_f((uint32_t)ci);
      w[28 + i] = bits_f((uint32_t)cnt);
    }
    nodes4_out.insert(nodes4_out.end(), w, w + 32);
  };
  if (root < 0) {
    const int ch[4] = {-1, -1, -1, -1};
    emit4(ch);
  } else if (B.tree[root].count > 0) {
    const int ch[4] = {root, -1, -1, -1};
    emit4(ch);
  } else {
    for (int t : order4) {
      int ch[4];
      children4(t, ch);
      emit4(ch);
    }
  }
  n_nodes4_out = (int)(nodes4_out.size() / 32);

  // triangles in leaf order: (v0, code) (e1, -) (e2, -)
  prims_out.assign(12 * (size_t)n, 0.0f);
  for (int k = 0; k < n; ++k) {
    const int p = B.idx[k];
    float* o = &prims_out[12 * (size_t)k];
    const float* t = &in.tris[9 * (size_t)p];
    o[0] = t[0];
    o[1] = t[1];
    o[2] = t[2];
    o[3] = bits_f((2u << 20) | (uint32_t)p);
    for (int a = 0; a < 3; ++a) {
      o[4 + a] = (float)((double)t[3 + a] - (double)t[a]);
      o[8 + a] = (float)((double)t[6 + a] - (double)t[a]);
    }
  }
}

// Uniform grid over the scatterer spheres.  The cell edge targets GRID_CELLS_PER_SPHERE cells
// per sphere over the spheres' bounding box (a ray then tests about as many spheres as it
// crosses cells: cell steps and sphere tests cost about the same, and measured on the
// inclusion phantom 2 cells per sphere was faster than 1, 4, 8 or 16), but is never below the sphere diameter (each sphere then overlaps at most
// 2 x 2 x 2 cells); it is raised until the grid has at most GRID_MAX_CELLS cells and no cell
// holds more than 255 spheres (clustered scatterers).  Boxes are inflated by GRID_PAD cell
// edges so that a closest-approach point within float rounding of a cell face is listed on
// both sides.
const double GRID_CELLS_PER_SPHERE = 2.0;
const double GRID_MAX_CELLS = 16.0 * 1024 * 1024;
const double GRID_PAD = 1e-2;

static void build_scatter_grid(const HostSceneIn& in, HostSceneOut& out) {
  const int ns = in.n_scat;
  out.cell.clear();
  out.cell_sph.clear();
  if (ns == 0) {
    out.gn[0] = out.gn[1] = out.gn[2] = 0;
    return;
  }
  const double rs = in.r_s;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int j = 0; j < ns; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], (double)in.scat_pos[3 * (size_t)j + a] - rs);
      hi[a] = std::max(hi[a], (double)in.scat_pos[3 * (size_t)j + a] + rs);
    }
  double ext[3], vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    ext[a] = std::max(hi[a] - lo[a], 1e-9);
    vol *= ext[a];
  }
  double h = std::max(std::max(std::cbrt(vol / (GRID_CELLS_PER_SPHERE * ns)), 2.0 * rs), 1e-9);
  for (int attempt = 0; attempt < 200; ++attempt, h *= 1.25) {
    int n[3];
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) {
      n[a] = std::max(1, (int)std::ceil(ext[a] / h));
      cells *= n[a];
    }
    if (cells > GRID_MAX_CELLS || n[0] > 4096 || n[1] > 4096 || n[2] > 4096) continue;
    // the device marches the float description; cells of a coordinate are taken from it here too
    for (int a = 0; a < 3; ++a) {
      out.glo[a] = round_down(lo[a]);
      out.gn[a] = n[a];
    }
    out.gh = (float)h;
    const double pad = GRID_PAD * h;
    auto cell_range = [&](double c, int a, int& c0, int& c1) {
      c0 = std::max(0, std::min(n[a] - 1, (int)std::floor((c - rs - pad - out.glo[a]) / out.gh)));
      c1 = std::max(0, std::min(n[a] - 1, (int)std::floor((c + rs + pad - out.glo[a]) / out.gh)));
    };
    const size_t n_cells = (size_t)n[0] * n[1] * n[2];
    std::vector<uint32_t> count(n_cells, 0), first(n_cells, 0);
    auto for_cells = [&](int j, auto&& fn) {
      int r0[3], r1[3];
      for (int a = 0; a < 3; ++a) cell_range(in.scat_pos[3 * (size_t)j + a], a, r0[a], r1[a]);
      for (int z = r0[2]; z <= r1[2]; ++z)
        for (int y = r0[1]; y <= r1[1]; ++y)
          for (int x = r0[0]; x <= r1[0]; ++x) fn(((uint32_t)z * n[1] + y) * n[0] + x);
    };
    for (int j = 0; j < ns; ++j) for_cells(j, [&](uint32_t c) { count[c]++; });
    uint64_t acc = 0;
    uint32_t most = 0;
    for (size_t c = 0; c < n_cells; ++c) {
      first[c] = (uint32_t)acc;
      acc += count[c];
      most = std::max(most, count[c]);
    }
    if (most > 255 || acc >= (1u << 24)) continue;
    out.cell.resize(n_cells);
    for (size_t c = 0; c < n_cells; ++c) out.cell[c] = first[c] << 8 | count[c];
    out.cell_sph.assign(4 * (size_t)acc, 0.0f);
    for (int j = 0; j < ns; ++j)
      for_cells(j, [&](uint32_t c) {
        float* e = &out.cell_sph[4 * (size_t)first[c]++];
        e[0] = in.scat_pos[3 * (size_t)j];
        e[1] = in.scat_pos[3 * (size_t)j + 1];
        e[2] = in.scat_pos[3 * (size_t)j + 2];
        e[3] = bits_f((3u << 20) | (uint32_t)j);
      });
    // the first two entries of every cell inline, so that a ray reads one 32-byte record per
    // cell: code 0 marks an empty slot, bit 31 of the second code that the cell holds more
    out.cell2.assign(8 * n_cells, 0.0f);
    for (size_t c = 0; c < n_cells; ++c) {
      const uint32_t f0 = out.cell[c] >> 8, k = out.cell[c] & 0xFFu;
      for (uint32_t slot = 0; slot < 2 && slot < k; ++slot) {
        const float* e = &out.cell_sph[4 * (size_t)(f0 + slot)];
        float* o = &out.cell2[8 * c + 4 * slot];
        o[0] = e[0];
        o[1] = e[1];
        o[2] = e[2];
        uint32_t code;
        std::memcpy(&code, &e[3], 4);
        o[3] = bits_f(code | (slot == 1 && k > 2 ? 0x80000000u : 0u));
      }
    }
    return;
  }
  // unreachable for scenes the upload accepts (< 2^20 spheres): an empty grid would lose hits
  out.gn[0] = out.gn[1] = out.gn[2] = -1;
}

void build_scene_host(const HostSceneIn& in, HostSceneOut& out) {
  const int nt = in.n_tris, ns = in.n_scat;
  build_tri_bvh(in, out.nodes_t, out.prims_t, out.n_nodes_t, out.depth_t, out.nodes4, out.n_nodes4, out.depth4);
  build_scatter_grid(in, out);

  // per-triangle normal + media, vertex 0; per-scatterer centre + amplitude
  out.tri_nrm.assign(4 * (size_t)nt, 0.0f);
  out.tri_v0.assign(4 * (size_t)nt, 0.0f);
  out.tri_e1.assign(4 * (size_t)nt, 0.0f);
  out.tri_e2.assign(4 * (size_t)nt, 0.0f);
  for (int i = 0; i < nt; ++i) {
    const float* t = &in.tris[9 * (size_t)i];
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
      e1[a] = (double)t[3 + a] - t[a];
      e2[a] = (double)t[6 + a] - t[a];
    }
    double nn[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double l = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    if (l == 0) l = 1;
    uint32_t med = (uint32_t)(in.media[2 * (size_t)i] & 0xFFFF) | ((uint32_t)(in.media[2 * (size_t)i + 1] & 0xFFFF) << 16);
    out.tri_nrm[4 * (size_t)i] = (float)(nn[0] / l);
    out.tri_nrm[4 * (size_t)i + 1] = (float)(nn[1] / l);
    out.tri_nrm[4 * (size_t)i + 2] = (float)(nn[2] / l);
    out.tri_nrm[4 * (size_t)i + 3] = bits_f(med);
    out.tri_v0[4 * (size_t)i] = t[0];
    out.tri_v0[4 * (size_t)i + 1] = t[1];
    out.tri_v0[4 * (size_t)i + 2] = t[2];
    for (int a = 0; a < 3; ++a) {
      out.tri_e1[4 * (size_t)i + a] = (float)e1[a];
      out.tri_e2[4 * (size_t)i + a] = (float)e2[a];
    }
    out.tri_e1[4 * (size_t)i + 3] = (float)l;
  }
  out.scat.assign(4 * (size_t)ns, 0.0f);
  for (int j = 0; j < ns; ++j) {
    out.scat[4 * (size_t)j] = in.scat_pos[3 * (size_t)j];
    out.scat[4 * (size_t)j + 1] = in.scat_pos[3 * (size_t)j + 1];
    out.scat[4 * (size_t)j + 2] = in.scat_pos[3 * (size_t)j + 2];
    out.scat[4 * (size_t)j + 3] = in.scat_amp[j];
  }
}

}  // namespace usrt
