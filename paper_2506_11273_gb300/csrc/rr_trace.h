// Host-side BVH representation shared by the builder and the upload/trace code.
#pragma once

#include <string>
#include <vector>

#include "rr_common.cuh"

namespace rr {

// Traversal stack entries per thread: one node group per level descended.
// rr_build_bvh refuses deeper trees.
constexpr uint32_t kTraceStack = 32;

struct HostBVH {
    std::vector<RRNode8> nodes;
    std::vector<RRTri> tris;
    std::vector<float4> planes;  // two per triangle: the normal (v1-v0)x(v2-v0) as hi + lo floats
    float lo[3], hi[3];
    uint32_t depth = 0;
    uint32_t stack_need = 0;
    uint32_t n_leaves = 0;
};

rr_status build_wide_bvh(const float *tris, uint32_t n, HostBVH *out, std::string *err);

}  // namespace rr
