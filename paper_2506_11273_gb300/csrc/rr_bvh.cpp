// Host BVH builder: binned-SAH binary BVH collapsed into 8-wide nodes with
// quantised child boxes (compressed wide BVH after Ylitie, Karras and Laine,
// HPG 2017), uploaded once per scene.  The paper traces with RTX hardware
// whose BVH is not described; this BVH serves the software trace kernel.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <limits>
#include <vector>

#include "rr_common.cuh"
#include "rr_trace.h"

namespace rr {
namespace {

struct Box3 {
    float lo[3] = {std::numeric_limits<float>::infinity(), std::numeric_limits<float>::infinity(),
                   std::numeric_limits<float>::infinity()};
    float hi[3] = {-std::numeric_limits<float>::infinity(), -std::numeric_limits<float>::infinity(),
                   -std::numeric_limits<float>::infinity()};
    void grow(const Box3 &b) {
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], b.lo[c]);
            hi[c] = std::max(hi[c], b.hi[c]);
        }
    }
    void grow(const float p[3]) {
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], p[c]);
            hi[c] = std::max(hi[c], p[c]);
        }
    }
    bool empty() const { return !(lo[0] <= hi[0]); }
    double area() const {
        if (empty()) return 0.0;
        double x = (double)hi[0] - lo[0], y = (double)hi[1] - lo[1], z = (double)hi[2] - lo[2];
        return 2.0 * (x * y + y * z + z * x);
    }
};

struct BNode {
    Box3 box;
    uint32_t left = 0, right = 0;  // children (inner node)
    uint32_t first = 0, count = 0; // triangle range in `order` (leaf: count > 0)
};

constexpr int kBins = 16;
constexpr uint32_t kMaxLeaf = 4;

struct Builder {
    const float *tris;
    uint32_t n;
    std::vector<Box3> tbox;
    std::vector<float> cen;  // 3 per triangle
    std::vector<uint32_t> order;
    std::vector<BNode> nodes;

    uint32_t build_range(uint32_t first, uint32_t count) {
        uint32_t id = (uint32_t)nodes.size();
        nodes.emplace_back();
        Box3 box, cb;
        for (uint32_t k = first; k < first + count; ++k) {
            box.grow(tbox[order[k]]);
            cb.grow(&cen[3 * (size_t)order[k]]);
        }
        nodes[id].box = box;
        if (count <= 1) {
            nodes[id].first = first;
            nodes[id].count = count;
            return id;
        }
        // binned SAH over the centroid bounds
        double best_cost = std::numeric_limits<double>::infinity();
        int best_axis = -1, best_split = -1;
        for (int axis = 0; axis < 3; ++axis) {
            const float cmin = cb.lo[axis], cext = cb.hi[axis] - cb.lo[axis];
            if (!(cext > 0.0f)) continue;
            const float scale = kBins / cext;
            Box3 bb[kBins];
            uint32_t bc[kBins] = {0};
            for (uint32_t k = first; k < first + count; ++k) {
                const uint32_t t = order[k];
                int b = (int)((cen[3 * (size_t)t + axis] - cmin) * scale);
                b = std::min(std::max(b, 0), kBins - 1);
                bb[b].grow(tbox[t]);
                bc[b]++;
            }
            double rarea[kBins];
            uint32_t rcnt[kBins];
            Box3 acc;
            uint32_t c = 0;
            for (int b = kBins - 1; b > 0; --b) {
                acc.grow(bb[b]);
                c += bc[b];
                rarea[b] = acc.area();
                rcnt[b] = c;
            }
            Box3 lacc;
            uint32_t lc = 0;
            for (int b = 0; b < kBins - 1; ++b) {
                lacc.grow(bb[b]);
                lc += bc[b];
                if (lc == 0 || rcnt[b + 1] == 0) continue;
                const double cost = lacc.area() * lc + rarea[b + 1] * rcnt[b + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = axis;
                    best_split = b;
                }
            }
        }
        const double parea = box.area();
        const double split_cost = parea > 0.0 ? 1.0 + best_cost / parea : std::numeric_limits<double>::infinity();
        if (count <= kMaxLeaf && (best_axis < 0 || (double)count <= split_cost)) {
            nodes[id].first = first;
            nodes[id].count = count;
            return id;
        }
        uint32_t mid;
        if (best_axis < 0) {
            mid = first + count / 2;  // identical centroids: split by index
        } else {
            const float cmin = cb.lo[best_axis], scale = kBins / (cb.hi[best_axis] - cb.lo[best_axis]);
            uint32_t *p = std::partition(order.data() + first, order.data() + first + count, [&](uint32_t t) {
                int b = (int)((cen[3 * (size_t)t + best_axis] - cmin) * scale);
                b = std::min(std::max(b, 0), kBins - 1);
                return b <= best_split;
            });
            mid = (uint32_t)(p - order.data());
            if (mid == first || mid == first + count) mid = first + count / 2;
        }
        const uint32_t l = build_range(first, mid - first);
        const uint32_t r = build_range(mid, first + count - mid);
        nodes[id].left = l;
        nodes[id].right = r;
        nodes[id].count = 0;
        return id;
    }
};

// Smallest power-of-two step s with 253*s >= ext and s >= 16 ulp of the
// coordinates; returns the exponent (s = 2^e).
int quant_exponent(float lo, float hi) {
    const double ext = (double)hi - (double)lo;
    const double mag = std::max(std::fabs((double)lo), std::fabs((double)hi));
    int e = -126;
    if (mag > 0.0) {
        int me;
        std::frexp(mag, &me);         // mag in [2^(me-1), 2^me)
        e = std::max(e, me - 24 + 4);  // 16 ulp
    }
    while (e < 127 && std::ldexp(253.0, e) < ext) ++e;
    return e;
}

float round_down_float(double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -std::numeric_limits<float>::infinity());
    return f;
}

struct WideTask {
    uint32_t bnode;
    uint32_t wnode;
    uint32_t depth;
};

}  // namespace

rr_status build_wide_bvh(const float *tris, uint32_t n, HostBVH *out, std::string *err) {
    Builder b;
    b.tris = tris;
    b.n = n;
    out->nodes.clear();
    out->tris.clear();
    out->planes.clear();
    out->depth = 0;
    out->stack_need = 0;
    out->n_leaves = 0;
    Box3 scene;
    b.tbox.resize(n);
    b.cen.resize(3 * (size_t)n);
    b.order.resize(n);
    for (uint32_t t = 0; t < n; ++t) {
        Box3 bx;
        for (int v = 0; v < 3; ++v) {
            const float *p = &tris[9 * (size_t)t + 3 * v];
            for (int c = 0; c < 3; ++c)
                if (!std::isfinite(p[c])) {
                    *err = "rr_build_bvh: non-finite vertex";
                    return RR_ERR_INVALID_ARG;
                }
            bx.grow(p);
        }
        b.tbox[t] = bx;
        for (int c = 0; c < 3; ++c) b.cen[3 * (size_t)t + c] = 0.5f * bx.lo[c] + 0.5f * bx.hi[c];
        b.order[t] = t;
        scene.grow(bx);
    }
    for (int c = 0; c < 3; ++c) {
        out->lo[c] = n ? scene.lo[c] : 0.0f;
        out->hi[c] = n ? scene.hi[c] : 0.0f;
    }
    if (n == 0) return RR_OK;
    b.nodes.reserve(2 * (size_t)n);
    const uint32_t root = b.build_range(0, n);

    // collapse into 8-wide nodes, breadth first so that the inner children
    // of a node are contiguous
    std::deque<WideTask> q;
    out->nodes.emplace_back();
    q.push_back({root, 0u, 1u});
    while (!q.empty()) {
        WideTask task = q.front();
        q.pop_front();
        out->depth = std::max(out->depth, task.depth);
        std::vector<uint32_t> ch;
        const BNode &bn = b.nodes[task.bnode];
        if (bn.count > 0) {
            ch.push_back(task.bnode);  // a root that is a single leaf
        } else {
            ch.push_back(bn.left);
            ch.push_back(bn.right);
        }
        while (ch.size() < 8) {
            int pick = -1;
            double best = -1.0;
            for (size_t i = 0; i < ch.size(); ++i) {
                const BNode &c = b.nodes[ch[i]];
                if (c.count == 0 && c.box.area() > best) {
                    best = c.box.area();
                    pick = (int)i;
                }
            }
            if (pick < 0) break;
            const BNode &c = b.nodes[ch[pick]];
            const uint32_t l = c.left, r = c.right;
            ch[pick] = l;
            ch.push_back(r);
        }
        // node box and octant slot assignment (greedy on direction alignment)
        Box3 nb;
        for (uint32_t c : ch) nb.grow(b.nodes[c].box);
        double ncen[3];
        for (int c = 0; c < 3; ++c) ncen[c] = 0.5 * ((double)nb.lo[c] + nb.hi[c]);
        struct Cand {
            double score;
            int child, slot;
        };
        std::vector<Cand> cands;
        for (size_t i = 0; i < ch.size(); ++i) {
            const Box3 &cb = b.nodes[ch[i]].box;
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = 0.5 * ((double)cb.lo[c] + cb.hi[c]) - ncen[c];
            for (int s = 0; s < 8; ++s) {
                double sc = 0.0;
                for (int c = 0; c < 3; ++c) sc += ((s >> c) & 1) ? d[c] : -d[c];
                cands.push_back({sc, (int)i, s});
            }
        }
        std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &c) {
            if (a.score != c.score) return a.score > c.score;
            if (a.child != c.child) return a.child < c.child;
            return a.slot < c.slot;
        });
        int slot_of[8];
        bool used[8] = {false};
        for (int i = 0; i < 8; ++i) slot_of[i] = -1;
        size_t assigned = 0;
        for (const Cand &c : cands) {
            if (assigned == ch.size()) break;
            if (slot_of[c.child] >= 0 || used[c.slot]) continue;
            slot_of[c.child] = c.slot;
            used[c.slot] = true;
            ++assigned;
        }

        RRNode8 node;
        std::memset(&node, 0, sizeof(node));
        // quantisation frame: p = lo - s (rounded down), boxes widened by one step
        int e[3];
        float p[3];
        for (int c = 0; c < 3; ++c) {
            e[c] = quant_exponent(nb.lo[c], nb.hi[c]);
            p[c] = round_down_float((double)nb.lo[c] - std::ldexp(1.0, e[c]));
        }
        node.px = p[0];
        node.py = p[1];
        node.pz = p[2];
        node.ex = (uint8_t)(e[0] + 127);
        node.ey = (uint8_t)(e[1] + 127);
        node.ez = (uint8_t)(e[2] + 127);
        uint8_t *qlo[3] = {node.qlo_x, node.qlo_y, node.qlo_z};
        uint8_t *qhi[3] = {node.qhi_x, node.qhi_y, node.qhi_z};
        for (int s = 0; s < 8; ++s)
            for (int c = 0; c < 3; ++c) {
                qlo[c][s] = 255;  // empty slot: inverted box
                qhi[c][s] = 0;
            }
        uint32_t n_inner = 0;
        for (uint32_t c : ch)
            if (b.nodes[c].count == 0) ++n_inner;
        node.child_base = (uint32_t)out->nodes.size();
        node.tri_base = (uint32_t)out->tris.size();
        // children in slot order: inner children get consecutive node indices in
        // slot order (rank = inner children in lower slots), leaf triangles are
        // appended in slot order
        int child_in_slot[8];
        for (int k = 0; k < 8; ++k) child_in_slot[k] = -1;
        for (size_t i = 0; i < ch.size(); ++i) child_in_slot[slot_of[i]] = (int)i;
        uint32_t inner_rank = 0;
        for (int s = 0; s < 8; ++s) {
            if (child_in_slot[s] < 0) continue;
            const size_t i = (size_t)child_in_slot[s];
            const BNode &cn = b.nodes[ch[i]];
            for (int c = 0; c < 3; ++c) {
                const double step = std::ldexp(1.0, e[c]);
                double ql = std::floor(((double)cn.box.lo[c] - p[c]) / step) - 1.0;
                double qh = std::ceil(((double)cn.box.hi[c] - p[c]) / step) + 1.0;
                if (ql < 0.0 || qh > 255.0) {
                    *err = "rr_build_bvh: child box outside the node's quantisation frame";
                    return RR_ERR_UNSUPPORTED;
                }
                qlo[c][s] = (uint8_t)ql;
                qhi[c][s] = (uint8_t)qh;
            }
            node.valid |= 1u << s;
            if (cn.count == 0) {
                node.imask |= (uint8_t)(1u << s);
                const uint32_t wid = node.child_base + inner_rank;
                q.push_back({ch[i], wid, task.depth + 1});
                ++inner_rank;
            } else {
                node.tribits |= ((1u << cn.count) - 1u) << (4 * s);
                for (uint32_t k = cn.first; k < cn.first + cn.count; ++k) {
                    const uint32_t t = b.order[k];
                    const float *v = &tris[9 * (size_t)t];
                    RRTri rt;
                    rt.v0_id = make_float4(v[0], v[1], v[2], 0.0f);
                    uint32_t id = t;
                    std::memcpy(&rt.v0_id.w, &id, 4);
                    rt.e1 = make_float4(v[3] - v[0], v[4] - v[1], v[5] - v[2], 0.0f);
                    rt.e2 = make_float4(v[6] - v[0], v[7] - v[1], v[8] - v[2], 0.0f);
                    out->tris.push_back(rt);
                    // exact-ish normal from the original vertices, kept as hi + lo floats
                    double a[3], c2[3], nn[3];
                    for (int c = 0; c < 3; ++c) {
                        a[c] = (double)v[3 + c] - v[c];
                        c2[c] = (double)v[6 + c] - v[c];
                    }
                    nn[0] = a[1] * c2[2] - a[2] * c2[1];
                    nn[1] = a[2] * c2[0] - a[0] * c2[2];
                    nn[2] = a[0] * c2[1] - a[1] * c2[0];
                    float hi3[3], lo3[3];
                    for (int c = 0; c < 3; ++c) {
                        hi3[c] = (float)nn[c];
                        lo3[c] = (float)(nn[c] - (double)hi3[c]);
                    }
                    out->planes.push_back(make_float4(hi3[0], hi3[1], hi3[2], lo3[0]));
                    out->planes.push_back(make_float4(lo3[1], lo3[2], 0.0f, 0.0f));
                }
                out->n_leaves++;
            }
        }
        for (uint32_t k = 0; k < n_inner; ++k) out->nodes.emplace_back();
        out->nodes[task.wnode] = node;
    }
    // the traversal pushes at most one node group per level it descends
    out->stack_need = out->depth;
    return RR_OK;
}

namespace {

constexpr char kBvhMagic[8] = {'R', 'R', 'B', 'V', 'H', '8', 0, 0};
constexpr uint32_t kBvhVersion = 1;

struct BvhHeader {
    char magic[8];
    uint32_t version;
    uint32_t node_bytes;
    uint32_t n_nodes;
    uint32_t n_tris;
    uint32_t depth;
    uint32_t n_leaves;
    float lo[3], hi[3];
    uint32_t reserved[2];
};
static_assert(sizeof(BvhHeader) == kBvhHeaderBytes, "header layout");

}  // namespace

size_t serialized_bvh_bytes(size_t n_nodes, size_t n_tris) {
    return kBvhHeaderBytes + sizeof(RRNode8) * n_nodes + sizeof(RRTri) * n_tris + 2 * sizeof(float4) * n_tris;
}

void serialize_bvh(const HostBVH &h, void *out) {
    BvhHeader hd{};
    std::memcpy(hd.magic, kBvhMagic, sizeof(kBvhMagic));
    hd.version = kBvhVersion;
    hd.node_bytes = (uint32_t)sizeof(RRNode8);
    hd.n_nodes = (uint32_t)h.nodes.size();
    hd.n_tris = (uint32_t)h.tris.size();
    hd.depth = h.depth;
    hd.n_leaves = h.n_leaves;
    for (int c = 0; c < 3; ++c) {
        hd.lo[c] = h.lo[c];
        hd.hi[c] = h.hi[c];
    }
    unsigned char *p = static_cast<unsigned char *>(out);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    std::memcpy(p, h.nodes.data(), sizeof(RRNode8) * h.nodes.size());
    p += sizeof(RRNode8) * h.nodes.size();
    std::memcpy(p, h.tris.data(), sizeof(RRTri) * h.tris.size());
    p += sizeof(RRTri) * h.tris.size();
    std::memcpy(p, h.planes.data(), sizeof(float4) * h.planes.size());
}

rr_status deserialize_bvh(const void *buf, size_t bytes, HostBVH *out, std::string *err) {
    auto refuse = [&](const char *why) {
        *err = std::string("rr_bvh_deserialize: ") + why;
        return RR_ERR_INVALID_ARG;
    };
    if (!buf || bytes < kBvhHeaderBytes) return refuse("buffer shorter than the header");
    BvhHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kBvhMagic, sizeof(kBvhMagic)) != 0) return refuse("not a serialized BVH");
    if (hd.version != kBvhVersion) return refuse("unknown format version");
    if (hd.node_bytes != sizeof(RRNode8)) return refuse("node size differs from this library's");
    if (hd.n_tris >= (1u << 28)) return refuse("too many triangles");
    if ((hd.n_tris == 0) != (hd.n_nodes == 0)) return refuse("node and triangle counts disagree");
    if (bytes != serialized_bvh_bytes(hd.n_nodes, hd.n_tris)) return refuse("size does not match the header");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(hd.lo[c]) || !std::isfinite(hd.hi[c]) || hd.lo[c] > hd.hi[c]) return refuse("bad box");
    const unsigned char *p = static_cast<const unsigned char *>(buf) + kBvhHeaderBytes;
    out->nodes.resize(hd.n_nodes);
    out->tris.resize(hd.n_tris);
    out->planes.resize(2 * (size_t)hd.n_tris);
    std::memcpy(out->nodes.data(), p, sizeof(RRNode8) * hd.n_nodes);
    p += sizeof(RRNode8) * hd.n_nodes;
    std::memcpy(out->tris.data(), p, sizeof(RRTri) * hd.n_tris);
    p += sizeof(RRTri) * hd.n_tris;
    std::memcpy(out->planes.data(), p, sizeof(float4) * 2 * (size_t)hd.n_tris);
    // structure: children after their parent (no cycle), indices in range,
    // leaf bits well formed; the depth is recomputed, not trusted
    std::vector<uint32_t> depth(hd.n_nodes, 0);
    if (hd.n_nodes) depth[0] = 1;
    uint32_t max_depth = hd.n_nodes ? 1u : 0u;
    for (uint32_t i = 0; i < hd.n_nodes; ++i) {
        const RRNode8 &nd = out->nodes[i];
        if (i > 0 && depth[i] == 0) return refuse("a node no parent references");
        if (nd.imask & ~nd.valid & 0xFFu) return refuse("inner child in an unused slot");
        if (nd.valid & ~0xFFu) return refuse("slot mask above eight slots");
        const uint32_t inner = (uint32_t)__builtin_popcount(nd.imask);
        if (inner) {
            if (nd.child_base <= i || (uint64_t)nd.child_base + inner > hd.n_nodes)
                return refuse("child index out of order or out of range");
            for (uint32_t k = 0; k < inner; ++k) {
                uint32_t &dc = depth[nd.child_base + k];
                dc = std::max(dc, depth[i] + 1u);
                max_depth = std::max(max_depth, dc);
            }
        }
        for (int s = 0; s < 8; ++s) {
            const uint32_t nib = (nd.tribits >> (4 * s)) & 15u;
            const bool leaf = ((nd.valid >> s) & 1u) && !((nd.imask >> s) & 1u);
            if (!leaf && nib != 0u) return refuse("triangle bits in a slot that is not a leaf");
            if (leaf && nib != 1u && nib != 3u && nib != 7u && nib != 15u) return refuse("leaf triangle bits malformed");
        }
        if ((uint64_t)nd.tri_base + (uint32_t)__builtin_popcount(nd.tribits) > hd.n_tris)
            return refuse("triangle index out of range");
    }
    if (max_depth > kTraceStack) return refuse("tree deeper than the trace kernel's stack");
    for (uint32_t k = 0; k < hd.n_tris; ++k) {
        uint32_t id;
        std::memcpy(&id, &out->tris[k].v0_id.w, 4);
        if (id >= hd.n_tris) return refuse("triangle id out of range");
    }
    for (int c = 0; c < 3; ++c) {
        out->lo[c] = hd.lo[c];
        out->hi[c] = hd.hi[c];
    }
    out->depth = max_depth;
    out->stack_need = max_depth;
    out->n_leaves = hd.n_leaves;
    return RR_OK;
}

}  // namespace rr
