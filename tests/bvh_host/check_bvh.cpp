// Host-side checks of the wide-BVH builder (no GPU): reads a triangle soup
// (float32 [n][9]) from a file, builds the compressed 8-wide BVH and verifies
// its invariants.  Prints "OK ..." and exits 0, or "FAIL ..." and exits 1.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rr_trace.h"

using namespace rr;

static int fails = 0;
static void fail_msg(const std::string &m) {
    if (fails++ < 10) std::printf("FAIL %s\n", m.c_str());
}

struct Ctx {
    const std::vector<float> *tris;
    const HostBVH *h;
    std::vector<int> seen;
};

// Triangles (original ids) under slot s of node `ni`, checked on the way.
static void subtree_ids(Ctx &c, uint32_t ni, uint32_t depth, std::vector<uint32_t> &out);

static void slot_ids(Ctx &c, const RRNode8 &nd, int s, uint32_t depth, std::vector<uint32_t> &out) {
    const HostBVH &h = *c.h;
    if ((nd.imask >> s) & 1u) {
        const uint32_t child = nd.child_base + __builtin_popcount(nd.imask & ((1u << s) - 1u));
        if (child >= h.nodes.size()) {
            fail_msg("inner child index out of range");
            return;
        }
        subtree_ids(c, child, depth + 1, out);
    } else {
        const uint32_t nib = (nd.tribits >> (4 * s)) & 15u;
        const int cnt = __builtin_popcount(nib);
        if (cnt < 1 || cnt > 4 || nib != ((1u << cnt) - 1u)) fail_msg("leaf triangle bits malformed");
        const uint32_t first = nd.tri_base + __builtin_popcount(nd.tribits & ((1u << (4 * s)) - 1u));
        for (int k = 0; k < cnt; ++k) {
            if (first + k >= h.tris.size()) {
                fail_msg("leaf triangle index out of range");
                return;
            }
            uint32_t id;
            std::memcpy(&id, &h.tris[first + k].v0_id.w, 4);
            out.push_back(id);
        }
    }
}

static void subtree_ids(Ctx &c, uint32_t ni, uint32_t depth, std::vector<uint32_t> &out) {
    const HostBVH &h = *c.h;
    if (depth > h.depth) fail_msg("node deeper than the reported depth");
    const RRNode8 &nd = h.nodes[ni];
    if ((nd.imask & ~nd.valid) != 0) fail_msg("inner-child mask outside the used slots");
    const uint8_t *qlo[3] = {nd.qlo_x, nd.qlo_y, nd.qlo_z}, *qhi[3] = {nd.qhi_x, nd.qhi_y, nd.qhi_z};
    const double p[3] = {nd.px, nd.py, nd.pz};
    const int e[3] = {(int)nd.ex - 127, (int)nd.ey - 127, (int)nd.ez - 127};
    for (int s = 0; s < 8; ++s) {
        const bool used = (nd.valid >> s) & 1u;
        if (!used) {
            if (((nd.tribits >> (4 * s)) & 15u) != 0u) fail_msg("triangle bits in an unused slot");
            for (int a = 0; a < 3; ++a)
                if (!(qlo[a][s] > qhi[a][s])) fail_msg("unused slot with a non-empty box");
            continue;
        }
        std::vector<uint32_t> ids;
        slot_ids(c, nd, s, depth, ids);
        for (uint32_t id : ids) {
            if (id >= c.seen.size()) {
                fail_msg("triangle id out of range");
                continue;
            }
            if (!((nd.imask >> s) & 1u)) c.seen[id]++;  // counted once, at its leaf
            for (int v = 0; v < 3; ++v)
                for (int a = 0; a < 3; ++a) {
                    const double x = (*c.tris)[9 * (size_t)id + 3 * v + a];
                    const double step = std::ldexp(1.0, e[a]);
                    const double lo = p[a] + qlo[a][s] * step, hi = p[a] + qhi[a][s] * step;
                    // every box is at least one step wider than what it bounds
                    if (!(x >= lo + step * (1.0 - 1e-9) && x <= hi - step * (1.0 - 1e-9)))
                        fail_msg("a vertex is not inside its slot's widened box");
                }
        }
        out.insert(out.end(), ids.begin(), ids.end());
    }
}

// The serialized form: a round trip gives back the same arrays, box, depth and
// leaf count; buffers damaged in each way the loader checks are refused.
static bool refused(const std::vector<unsigned char> &buf) {
    HostBVH back;
    std::string err;
    return deserialize_bvh(buf.data(), buf.size(), &back, &err) == RR_ERR_INVALID_ARG && !err.empty();
}

static void check_serialized(const HostBVH &h) {
    std::vector<unsigned char> buf(serialized_bvh_bytes(h.nodes.size(), h.tris.size()));
    serialize_bvh(h, buf.data());
    HostBVH back;
    std::string err;
    if (deserialize_bvh(buf.data(), buf.size(), &back, &err) != RR_OK) {
        fail_msg("round trip refused: " + err);
        return;
    }
    if (back.nodes.size() != h.nodes.size() || back.tris.size() != h.tris.size() ||
        back.planes.size() != h.planes.size() ||
        std::memcmp(back.nodes.data(), h.nodes.data(), sizeof(RRNode8) * h.nodes.size()) ||
        std::memcmp(back.tris.data(), h.tris.data(), sizeof(RRTri) * h.tris.size()) ||
        std::memcmp(back.planes.data(), h.planes.data(), sizeof(float4) * h.planes.size()))
        fail_msg("round trip changed the arrays");
    if (back.depth != h.depth || back.stack_need != h.stack_need || back.n_leaves != h.n_leaves ||
        std::memcmp(back.lo, h.lo, sizeof(h.lo)) || std::memcmp(back.hi, h.hi, sizeof(h.hi)))
        fail_msg("round trip changed depth, leaf count or box");
    auto node_at = [&](std::vector<unsigned char> &b, size_t i) {
        return reinterpret_cast<RRNode8 *>(b.data() + kBvhHeaderBytes + sizeof(RRNode8) * i);
    };
    {
        auto b = buf;
        b[0] ^= 1u;
        if (!refused(b)) fail_msg("bad magic accepted");
    }
    {
        auto b = buf;
        b.pop_back();
        if (!refused(b)) fail_msg("truncated buffer accepted");
    }
    if (h.nodes.empty()) return;
    {
        auto b = buf;
        node_at(b, 0)->tri_base = (uint32_t)h.tris.size();
        if (node_at(b, 0)->tribits && !refused(b)) fail_msg("triangle range past the end accepted");
    }
    {
        auto b = buf;
        node_at(b, 0)->valid |= 1u << 9;
        if (!refused(b)) fail_msg("slot mask above eight slots accepted");
    }
    {
        auto b = buf;
        const uint32_t bad = (uint32_t)h.tris.size();
        std::memcpy(b.data() + kBvhHeaderBytes + sizeof(RRNode8) * h.nodes.size() + 12, &bad, 4);
        if (!refused(b)) fail_msg("triangle id out of range accepted");
    }
    // a leaf slot of the root with malformed bits (two triangles, not the low ones)
    for (int s = 0; s < 8; ++s) {
        const RRNode8 &r = h.nodes[0];
        if (((r.valid >> s) & 1u) && !((r.imask >> s) & 1u)) {
            auto b = buf;
            RRNode8 *nd = node_at(b, 0);
            nd->tribits = (nd->tribits & ~(15u << (4 * s))) | (5u << (4 * s));
            if (!refused(b)) fail_msg("malformed leaf bits accepted");
            break;
        }
    }
    if (h.nodes[0].imask) {
        {
            auto b = buf;
            node_at(b, 0)->child_base = 0;  // the root as its own child: a cycle
            if (!refused(b)) fail_msg("cycle accepted");
        }
        {
            auto b = buf;
            node_at(b, 0)->child_base = (uint32_t)h.nodes.size();
            if (!refused(b)) fail_msg("child index past the end accepted");
        }
        {
            auto b = buf;
            node_at(b, 0)->imask |= (uint8_t)~h.nodes[0].valid;
            if ((uint8_t)~h.nodes[0].valid && !refused(b)) fail_msg("inner child in an unused slot accepted");
        }
    }
}

// A chain of single-child nodes deeper than the trace kernel's stack, ending
// in a one-triangle leaf: well formed in every other respect, refused for its
// depth; one level shorter than the stack it loads.
static void check_deep_chain() {
    for (uint32_t levels : {kTraceStack, kTraceStack + 1}) {
        HostBVH h;
        h.nodes.resize(levels);
        for (uint32_t i = 0; i < levels; ++i) {
            RRNode8 &nd = h.nodes[i];
            std::memset(&nd, 0, sizeof(nd));
            nd.ex = nd.ey = nd.ez = 127;
            nd.valid = 1u;
            if (i + 1 < levels) {
                nd.imask = 1u;
                nd.child_base = i + 1;
            } else {
                nd.tribits = 1u;
            }
        }
        h.tris.resize(1);
        std::memset(h.tris.data(), 0, sizeof(RRTri));
        h.planes.resize(2);
        std::memset(h.planes.data(), 0, 2 * sizeof(float4));
        for (int c = 0; c < 3; ++c) {
            h.lo[c] = 0.0f;
            h.hi[c] = 1.0f;
        }
        h.depth = levels;
        h.n_leaves = 1;
        std::vector<unsigned char> buf(serialized_bvh_bytes(h.nodes.size(), 1));
        serialize_bvh(h, buf.data());
        const bool ok = !refused(buf);
        if (ok != (levels <= kTraceStack)) fail_msg("chain of " + std::to_string(levels) + " levels: wrong verdict");
    }
}

int main(int argc, char **argv) {
    if (argc >= 2 && std::string(argv[1]) == "--deep-chain") {
        check_deep_chain();
        if (fails) return 1;
        std::printf("OK deep chain\n");
        return 0;
    }
    if (argc < 2) return 2;
    std::vector<float> tris;
    if (FILE *f = std::fopen(argv[1], "rb")) {
        float buf[9];
        while (std::fread(buf, 4, 9, f) == 9) tris.insert(tris.end(), buf, buf + 9);
        std::fclose(f);
    } else {
        return 2;
    }
    const uint32_t n = (uint32_t)(tris.size() / 9);
    HostBVH h;
    std::string err;
    const rr_status st = build_wide_bvh(tris.data(), n, &h, &err);
    if (st != RR_OK) {
        std::printf("FAIL build status %d: %s\n", (int)st, err.c_str());
        return 1;
    }
    if (h.tris.size() != n) fail_msg("BVH triangle count differs from the input");
    if (h.planes.size() != 2 * (size_t)n) fail_msg("plane count differs");
    if (h.stack_need > kTraceStack) fail_msg("stack need above the kernel's stack");
    Ctx c{&tris, &h, std::vector<int>(n, 0)};
    if (n > 0) {
        if (h.nodes.empty()) fail_msg("no root node");
        std::vector<uint32_t> all;
        subtree_ids(c, 0, 1, all);
        for (uint32_t t = 0; t < n; ++t)
            if (c.seen[t] != 1) {
                fail_msg("triangle " + std::to_string(t) + " referenced " + std::to_string(c.seen[t]) + " times");
                break;
            }
        // plane normals: hi + lo is the binary64 cross product to ~2^-48 relative
        for (uint32_t k = 0; k < n; ++k) {
            uint32_t id;
            std::memcpy(&id, &h.tris[k].v0_id.w, 4);
            const float *v = &tris[9 * (size_t)id];
            double a[3], b[3];
            for (int q = 0; q < 3; ++q) {
                a[q] = (double)v[3 + q] - v[q];
                b[q] = (double)v[6 + q] - v[q];
            }
            const double nn[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            const float4 p0 = h.planes[2 * k], p1 = h.planes[2 * k + 1];
            const double got[3] = {(double)p0.x + p0.w, (double)p0.y + p1.x, (double)p0.z + p1.y};
            const double mag = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            for (int q = 0; q < 3; ++q)
                if (std::fabs(got[q] - nn[q]) > 1e-13 * mag + 1e-300) {
                    fail_msg("plane normal hi + lo differs from the binary64 cross product");
                    q = 3;
                    k = n;
                }
        }
    }
    check_serialized(h);
    if (fails) return 1;
    std::printf("OK n=%u nodes=%zu leaves=%u depth=%u\n", n, h.nodes.size(), h.n_leaves, h.depth);
    return 0;
}
