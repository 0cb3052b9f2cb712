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

// Serialized form of a BVH (rr_bvh_serialize): a 64-byte header (magic
// "RRBVH8", format version, node size, node and triangle counts, depth, leaf
// count, scene box) followed by the node, triangle and plane arrays exactly as
// they sit in device memory (little-endian).
constexpr size_t kBvhHeaderBytes = 64;
size_t serialized_bvh_bytes(size_t n_nodes, size_t n_tris);
void serialize_bvh(const HostBVH &h, void *out);

// Parses and checks a serialized BVH: sizes consistent with `bytes`, every
// node's children after it (so the tree has no cycle) and inside the node
// array, its triangles inside the triangle array, leaf bits well formed,
// depth within the trace kernel's stack, triangle ids below the count.  A
// buffer that fails any check is refused with RR_ERR_INVALID_ARG.
rr_status deserialize_bvh(const void *buf, size_t bytes, HostBVH *out, std::string *err);

}  // namespace rr
