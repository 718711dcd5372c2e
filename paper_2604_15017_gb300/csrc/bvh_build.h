// Host BVH builder interface (see bvh_build.cpp for the device layout).
#pragma once

#include <cstdint>
#include <vector>

namespace usrt {

struct HostSceneIn {
  int n_tris;
  const float* tris;      // n_tris * 9
  const int32_t* media;   // n_tris * 2
  int n_scat;
  const float* scat_pos;  // n_scat * 3
  const float* scat_amp;  // n_scat
  float r_s;
};

struct HostSceneOut {
  int n_nodes_t = 0, depth_t = 0;  // BVH over the triangles (closest hits, secondary-ray crossings)
  std::vector<float> nodes_t;      // 16 floats per node
  std::vector<float> prims_t;      // 12 floats per triangle, leaf order
  int n_nodes4 = 0, depth4 = 0;    // the same tree collapsed to 4-wide nodes (same leaves)
  std::vector<float> nodes4;       // 32 floats per node
  // uniform grid over the scatterer spheres: cell (x, y, z) covers glo + h [x, x+1) x [y, y+1) x
  // [z, z+1).  cell[(z * gn[1] + y) * gn[0] + x] = first << 8 | count names the (centre, code)
  // entries of every sphere whose (slightly inflated) bounding box overlaps the cell:
  // cell_sph[first .. first + count)
  float glo[3] = {0, 0, 0}, gh = 1.0f;
  int gn[3] = {0, 0, 0};
  std::vector<uint32_t> cell;
  std::vector<float> cell_sph;  // 4 floats per entry
  std::vector<float> cell2;     // per cell its first two entries (8 floats); see build_scatter_grid
  std::vector<float> tri_nrm;  // 4 per triangle
  std::vector<float> tri_v0;   // 4 per triangle
  std::vector<float> tri_e1;   // 4 per triangle: (v1 - v0, |(v1 - v0) x (v2 - v0)|)
  std::vector<float> tri_e2;   // 4 per triangle: (v2 - v0, 0)
  std::vector<float> scat;     // 4 per scatterer
};

void build_scene_host(const HostSceneIn& in, HostSceneOut& out);

}  // namespace usrt
