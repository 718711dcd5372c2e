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
  int n_nodes = 0, depth = 0;      // BVH over triangles and scatterers (closest hits)
  std::vector<float> nodes;        // 16 floats per node
  std::vector<float> prims;        // 12 floats per primitive, leaf order
  int n_nodes_t = 0, depth_t = 0;  // BVH over triangles only (secondary-ray crossings)
  std::vector<float> nodes_t;
  std::vector<float> prims_t;
  std::vector<float> tri_nrm;  // 4 per triangle
  std::vector<float> tri_v0;   // 4 per triangle
  std::vector<float> scat;     // 4 per scatterer
};

void build_scene_host(const HostSceneIn& in, HostSceneOut& out);

}  // namespace usrt
