/*
 * CPU oracle for the ray-reordering hot path (Meister, Boksansky, Guthe,
 * Bittner: "On Ray Reordering Techniques for Faster GPU Ray Tracing", I3D 2020).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path, and it never reads anything that the
 * CUDA path produced.
 *
 * Everything here is plain, single-threaded and written in the order of the
 * definitions it follows, so that it can be checked against the paper by eye:
 *   - quantisation and Morton interleaving: Section 3 and Section 3.1,
 *     Figure 2 (bit layouts of the 32-bit keys);
 *   - origin-direction interleaved key (Aila): Section 3.1.4;
 *   - compacted Aila key: Section 3.1.4, Figure 2;
 *   - Two Point (origin-termination) key: Section 3.1.5, Figure 2;
 *   - termination estimate, fixed / adaptive / real: Section 3.1.6;
 *   - origin, origin-direction (Reis), direction-origin (Costa) and
 *     octahedron keys: Sections 3.1.1-3.1.4, Figure 2;
 *   - stable sort of key-index pairs and the ray reorder pass: Section 3.2;
 *   - closest-hit trace: brute force over all triangles (Moller-Trumbore
 *     1997) in double precision, plus a binary BVH that must give the same
 *     answer (it is checked against the brute force in the tests).
 *
 * Floating point that decides an integer (a quantised coordinate, a table
 * cell, a fixed-point length) is evaluated in IEEE binary32, one correctly
 * rounded operation at a time, in the order written; the library is built
 * with -ffp-contract=off so that no multiply-add is fused.  The trace is
 * evaluated in binary64.
 *
 * Where the paper is silent the oracle takes these readings:
 *   - quantisation is per axis of the scene box, by truncation to 32 bits;
 *     values outside the box (and NaN) clamp to its faces;
 *   - the direction is normalised, mapped from [-1,1] to [0,1] and quantised
 *     like a position; its three leading zero bits are a right shift by 3;
 *   - keys longer or shorter than 32 bits are prefixes of the 192-bit
 *     interleaved string (Section 3.1.4 mentions Aila and Karras' 192-bit
 *     keys); x is the most significant component of every triple;
 *   - the termination point p = o + t*dhat is clamped into the box by the
 *     quantiser; a non-finite estimate is replaced by 4*E;
 *   - Reis and Costa keys of b bits give floor(b*10/32) and floor(b*8/32)
 *     bits to the direction (the 32-bit split of Figure 2) and the rest to
 *     the origin, each part a prefix of its own 3D Morton string;
 *   - the octahedron key maps the direction to the square with the
 *     octahedral parametrisation (Meyer et al. 2010), quantises both
 *     coordinates like a position and interleaves them after the origin in
 *     every level, with four leading zero bits removed as in the compact
 *     Aila key (Figure 2 starts with 15 origin bits);
 *   - the length table holds fixed-point sums (units of E/2^24) in 64 bits and
 *     32-bit counts, so that accumulation is exact in any order; only rays that
 *     hit accumulate; the length of a ray is t*|d|, clamped to [0, 64*E].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MISS 0xFFFFFFFFu

enum { OR_AILA = 0, OR_AILA_COMPACT = 1, OR_TWO_POINT = 2, OR_ORIGIN = 3, OR_REIS = 4, OR_COSTA = 5,
       OR_OCTAHEDRON = 6 };
enum { OR_T_FIXED = 0, OR_T_ADAPTIVE = 1, OR_T_GIVEN = 2 };

/* ------------------------------------------------------------------------ */
/* Quantisation                                                              */
/* ------------------------------------------------------------------------ */

/* x in [0,1] -> 32-bit cell index by truncation; x >= 1 -> all ones; x <= 0 or NaN -> 0. */
uint32_t or_quantise_unit(float x)
{
    if (!(x > 0.0f))
        return 0u;
    if (x >= 1.0f)
        return 0xFFFFFFFFu;
    float s = x * 4294967296.0f; /* times 2^32: exact */
    return (uint32_t)s;          /* truncation toward zero */
}

/* Largest extent of the box (Section 3.1.6: "largest extent of the scene bounding box"). */
float or_largest_extent(const float lo[3], const float hi[3])
{
    float e = hi[0] - lo[0];
    float ey = hi[1] - lo[1];
    float ez = hi[2] - lo[2];
    if (ey > e)
        e = ey;
    if (ez > e)
        e = ez;
    return e;
}

/* A point quantised per axis inside the box. */
void or_quantise_point(const float p[3], const float lo[3], const float hi[3], uint32_t q[3])
{
    for (int c = 0; c < 3; ++c) {
        float ext = hi[c] - lo[c];
        float inv = ext > 0.0f ? 1.0f / ext : 0.0f;
        float x = (p[c] - lo[c]) * inv;
        q[c] = or_quantise_unit(x);
    }
}

/* |d| summed left to right, one rounding per operation. */
float or_length(const float d[3])
{
    float s = d[0] * d[0];
    s = s + d[1] * d[1];
    s = s + d[2] * d[2];
    return sqrtf(s);
}

/* Normalised direction (zero for a zero or non-finite length). */
void or_normalise(const float d[3], float dh[3])
{
    float len = or_length(d);
    for (int c = 0; c < 3; ++c)
        dh[c] = len > 0.0f ? d[c] / len : 0.0f;
}

/* The normalised direction mapped from [-1,1] to [0,1] and quantised. */
void or_quantise_direction(const float d[3], uint32_t q[3])
{
    float dh[3];
    or_normalise(d, dh);
    for (int c = 0; c < 3; ++c) {
        float x = (dh[c] + 1.0f) * 0.5f;
        q[c] = or_quantise_unit(x);
    }
}

/* ------------------------------------------------------------------------ */
/* Interleaving: the 192-bit string and its prefixes                         */
/* ------------------------------------------------------------------------ */

/*
 * comp[0..2] = first point (the origin), comp[3..5] = second component
 * (direction with its three leading zeros, or the termination point).  Level
 * L = 0..31 contributes, from the most significant end, bit 31-L of comp[0],
 * comp[1], ..., comp[5].  The compact layout drops the direction slots of
 * levels 0..2 (always zero in the Aila key).  The key is the first `bits`
 * bits of the string read as an unsigned integer (bits <= 64).
 */
uint64_t or_interleave(int layout, const uint32_t comp[6], uint32_t bits)
{
    uint64_t key = 0;
    uint32_t taken = 0;
    for (int L = 0; L < 32 && taken < bits; ++L) {
        for (int s = 0; s < 6 && taken < bits; ++s) {
            if (layout == OR_AILA_COMPACT && s >= 3 && L < 3)
                continue;
            uint32_t bit = (comp[s] >> (31 - L)) & 1u;
            key = (key << 1) | bit;
            taken++;
        }
    }
    return key;
}

/*
 * Prefix of `bits` bits of the Morton string of three 32-bit components: level
 * L holds bit 31-L of c0, c1, c2 in that order.
 */
uint64_t or_morton3_prefix(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t bits)
{
    const uint32_t c[3] = {c0, c1, c2};
    uint64_t key = 0;
    uint32_t taken = 0;
    for (int L = 0; L < 32 && taken < bits; ++L)
        for (int s = 0; s < 3 && taken < bits; ++s) {
            key = (key << 1) | ((c[s] >> (31 - L)) & 1u);
            taken++;
        }
    return key;
}

/*
 * Octahedral parametrisation of a direction (Meyer et al. 2010): project onto
 * the octahedron |x|+|y|+|z| = 1, fold the lower half (z < 0) over the
 * diagonals, and map the square [-1,1]^2 to [0,1]^2.  Sign of 0 is +1.
 */
void or_octahedral(const float d[3], float *u, float *v)
{
    float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    float sum = ax + ay;
    sum = sum + az;
    float px = 0.0f, py = 0.0f;
    if (sum > 0.0f) {
        px = d[0] / sum;
        py = d[1] / sum;
    }
    if (d[2] < 0.0f) {
        float sx = px >= 0.0f ? 1.0f : -1.0f;
        float sy = py >= 0.0f ? 1.0f : -1.0f;
        float qx = (1.0f - fabsf(py)) * sx;
        float qy = (1.0f - fabsf(px)) * sy;
        px = qx;
        py = qy;
    }
    *u = (px + 1.0f) * 0.5f;
    *v = (py + 1.0f) * 0.5f;
}

/*
 * Interleaving of the other key families from their quantised components:
 * ORIGIN reads comp[0..2]; REIS and COSTA read the origin comp[0..2] and the
 * direction comp[3..5]; OCTAHEDRON reads the origin comp[0..2] and the two
 * octahedral coordinates comp[3], comp[4] (already shifted right by 4).
 */
uint64_t or_interleave_od(int layout, const uint32_t comp[6], uint32_t bits)
{
    if (layout == OR_ORIGIN)
        return or_morton3_prefix(comp[0], comp[1], comp[2], bits);
    if (layout == OR_REIS || layout == OR_COSTA) {
        uint32_t db = layout == OR_REIS ? (bits * 10u) / 32u : (bits * 8u) / 32u;
        uint32_t ob = bits - db;
        uint64_t ko = or_morton3_prefix(comp[0], comp[1], comp[2], ob);
        uint64_t kd = or_morton3_prefix(comp[3], comp[4], comp[5], db);
        if (layout == OR_REIS)
            return db ? (ko << db) | kd : ko;
        return ob ? (kd << ob) | ko : kd;
    }
    /* OCTAHEDRON: levels of (ox, oy, oz, u, v), direction slots of levels 0..3 dropped */
    uint64_t key = 0;
    uint32_t taken = 0;
    for (int L = 0; L < 32 && taken < bits; ++L)
        for (int s = 0; s < 5 && taken < bits; ++s) {
            if (s >= 3 && L < 4)
                continue;
            key = (key << 1) | ((comp[s] >> (31 - L)) & 1u);
            taken++;
        }
    return key;
}

/*
 * Keys that read the origin and the direction only (Sections 3.1.1-3.1.4,
 * Figure 2): ORIGIN, REIS, COSTA and OCTAHEDRON.
 */
uint64_t or_key_od(int layout, uint32_t bits, const float o[3], const float d[3], const float lo[3],
                   const float hi[3])
{
    uint32_t qo[3], qd[3], comp[6] = {0, 0, 0, 0, 0, 0};
    or_quantise_point(o, lo, hi, qo);
    for (int c = 0; c < 3; ++c)
        comp[c] = qo[c];
    if (layout == OR_REIS || layout == OR_COSTA) {
        or_quantise_direction(d, qd);
        for (int c = 0; c < 3; ++c)
            comp[3 + c] = qd[c];
    } else if (layout == OR_OCTAHEDRON) {
        float u, v;
        or_octahedral(d, &u, &v);
        comp[3] = or_quantise_unit(u) >> 4;
        comp[4] = or_quantise_unit(v) >> 4;
    }
    return or_interleave_od(layout, comp, bits);
}

/* The 20-bit compacted Aila code of a ray: the length-table cell (Section 3.1.6). */
uint32_t or_table_cell(const float o[3], const float d[3], const float lo[3], const float hi[3])
{
    uint32_t qo[3], qd[3], comp[6];
    or_quantise_point(o, lo, hi, qo);
    or_quantise_direction(d, qd);
    for (int c = 0; c < 3; ++c) {
        comp[c] = qo[c];
        comp[3 + c] = qd[c] >> 3;
    }
    return (uint32_t)or_interleave(OR_AILA_COMPACT, comp, 20);
}

/* ------------------------------------------------------------------------ */
/* Ray-length table (Section 3.1.6)                                          */
/* ------------------------------------------------------------------------ */

#define OR_TABLE_CELLS (1u << 20)
#define OR_FIX_ONE 16777216.0f /* 2^24 fixed-point units per E */

/* Every cell starts with one dummy ray of length 0.25*E. */
void or_table_init(uint64_t *sum, uint32_t *cnt)
{
    for (uint32_t i = 0; i < OR_TABLE_CELLS; ++i) {
        sum[i] = 4194304u; /* 0.25 * 2^24 */
        cnt[i] = 1u;
    }
}

/* Fixed-point length of a hit: trunc(clamp(t*|d|/E, 0, 64) * 2^24). */
uint32_t or_fixed_length(float t, const float d[3], float E)
{
    float len = t * or_length(d);
    float invE = 1.0f / E;
    float x = len * invE;
    if (!(x > 0.0f))
        x = 0.0f;
    if (x > 64.0f)
        x = 64.0f;
    return (uint32_t)(x * OR_FIX_ONE);
}

/* After a trace pass: every ray that hit adds its length to its cell. */
void or_table_accumulate(uint64_t *sum, uint32_t *cnt, const float lo[3], const float hi[3],
                         float E, const float *o_tmin, const float *d_tmax, const float *hits,
                         uint32_t n)
{
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t tri;
        memcpy(&tri, &hits[4 * i + 3], 4);
        float t = hits[4 * i + 0];
        if (tri == OR_MISS || !isfinite(t))
            continue;
        const float *o = &o_tmin[4 * i];
        const float *d = &d_tmax[4 * i];
        uint32_t cell = or_table_cell(o, d, lo, hi);
        sum[cell] += or_fixed_length(t, d, E);
        cnt[cell] += 1u;
    }
}

/* Average length of a cell in world units: (sum / cnt) * 2^-24 * E. */
float or_table_estimate(const uint64_t *sum, const uint32_t *cnt, uint32_t cell, float E)
{
    if (cnt[cell] == 0u)
        return 0.25f * E;
    uint64_t mean = sum[cell] / cnt[cell];
    float m = (float)mean;
    return (m * (1.0f / OR_FIX_ONE)) * E;
}

/* ------------------------------------------------------------------------ */
/* Sorting keys (Section 3.1, Figure 2)                                      */
/* ------------------------------------------------------------------------ */

/* One ray's key.  t_est is only read by the Two Point layout. */
uint64_t or_key(int layout, uint32_t bits, const float o[3], const float d[3], float t_est,
                const float lo[3], const float hi[3])
{
    uint32_t comp[6];
    uint32_t qo[3];
    or_quantise_point(o, lo, hi, qo);
    for (int c = 0; c < 3; ++c)
        comp[c] = qo[c];
    if (layout == OR_TWO_POINT) {
        float E = or_largest_extent(lo, hi);
        if (!isfinite(t_est))
            t_est = 4.0f * E;
        float dh[3], p[3];
        uint32_t qp[3];
        or_normalise(d, dh);
        for (int c = 0; c < 3; ++c) {
            float step = dh[c] * t_est;
            p[c] = o[c] + step;
        }
        or_quantise_point(p, lo, hi, qp);
        for (int c = 0; c < 3; ++c)
            comp[3 + c] = qp[c];
    } else {
        uint32_t qd[3];
        or_quantise_direction(d, qd);
        for (int c = 0; c < 3; ++c)
            comp[3 + c] = qd[c] >> 3; /* three leading zero bits per component */
    }
    return or_interleave(layout, comp, bits);
}

/*
 * Keys of a wavefront.  tsrc selects the termination estimate of the Two
 * Point key: FIXED ratio*E, ADAPTIVE from the table, GIVEN t_given[i].
 */
void or_compute_keys(int layout, uint32_t bits, int tsrc, float ratio, const float lo[3],
                     const float hi[3], const float *t_given, const uint64_t *tab_sum,
                     const uint32_t *tab_cnt, float tab_E, const float *o_tmin,
                     const float *d_tmax, uint32_t n, uint64_t *keys)
{
    float E = or_largest_extent(lo, hi);
    for (uint32_t i = 0; i < n; ++i) {
        const float *o = &o_tmin[4 * i];
        const float *d = &d_tmax[4 * i];
        float t_est = 0.0f;
        if (layout == OR_TWO_POINT) {
            if (tsrc == OR_T_FIXED)
                t_est = ratio * E;
            else if (tsrc == OR_T_GIVEN)
                t_est = t_given[i];
            else
                t_est = or_table_estimate(tab_sum, tab_cnt, or_table_cell(o, d, lo, hi), tab_E);
        }
        keys[i] = layout >= OR_ORIGIN ? or_key_od(layout, bits, o, d, lo, hi)
                                      : or_key(layout, bits, o, d, t_est, lo, hi);
    }
}

/* ------------------------------------------------------------------------ */
/* Stable sort of (key, index) pairs and the reorder pass (Section 3.2)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    uint32_t idx;
} or_pair;

static int or_pair_cmp(const void *a, const void *b)
{
    const or_pair *x = (const or_pair *)a;
    const or_pair *y = (const or_pair *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* perm[i] = index of the i-th smallest key; equal keys keep their input order. */
int or_stable_sort(const uint64_t *keys, uint32_t n, uint32_t *perm, uint64_t *sorted_keys)
{
    or_pair *p = (or_pair *)malloc((size_t)(n ? n : 1) * sizeof(or_pair));
    if (!p)
        return 1;
    for (uint32_t i = 0; i < n; ++i) {
        p[i].key = keys[i];
        p[i].idx = i;
    }
    qsort(p, n, sizeof(or_pair), or_pair_cmp); /* (key, index) is a total order */
    for (uint32_t i = 0; i < n; ++i) {
        perm[i] = p[i].idx;
        if (sorted_keys)
            sorted_keys[i] = p[i].key;
    }
    free(p);
    return 0;
}

/*
 * Local (block-wise) sort, Section 3.2: the rays are cut into consecutive
 * segments of `segment` rays (the last one may be shorter) and each segment is
 * sorted stably on its own.  perm holds global ray indices; segment s occupies
 * perm[s*segment ...] and holds exactly the indices of its own range.
 */
int or_segment_sort(const uint64_t *keys, uint32_t n, uint32_t segment, uint32_t *perm)
{
    if (segment == 0)
        return 1;
    for (uint32_t s = 0; s < n; s += segment) {
        uint32_t m = n - s < segment ? n - s : segment;
        if (or_stable_sort(keys + s, m, perm + s, NULL))
            return 1;
        for (uint32_t i = 0; i < m; ++i)
            perm[s + i] += s;
        if (n - s <= segment)
            break;
    }
    return 0;
}

/* out[i] = in[perm[i]] for every field of the ray SoA, bit for bit. */
void or_permute(const float *o_tmin, const float *d_tmax, const uint32_t *payload,
                const uint32_t *perm, uint32_t n, float *o_out, float *d_out, uint32_t *p_out)
{
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t j = perm[i];
        memcpy(&o_out[4 * i], &o_tmin[4 * j], 16);
        memcpy(&d_out[4 * i], &d_tmax[4 * j], 16);
        p_out[i] = payload[j];
    }
}

/* ------------------------------------------------------------------------ */
/* Closest-hit trace (binary64)                                              */
/* ------------------------------------------------------------------------ */

/*
 * Moller-Trumbore (1997).  Two-sided.  Returns 1 and (t, u, v) when the ray
 * meets the triangle's plane inside the closed triangle; a zero determinant
 * (ray parallel to the plane, or a zero-area triangle) never hits.
 */
int or_ray_triangle(const double o[3], const double d[3], const float *tri, double *t_out,
                    double *u_out, double *v_out)
{
    double v0[3], e1[3], e2[3], pv[3], tv[3], qv[3];
    for (int c = 0; c < 3; ++c) {
        v0[c] = tri[c];
        e1[c] = (double)tri[3 + c] - v0[c];
        e2[c] = (double)tri[6 + c] - v0[c];
    }
    pv[0] = d[1] * e2[2] - d[2] * e2[1];
    pv[1] = d[2] * e2[0] - d[0] * e2[2];
    pv[2] = d[0] * e2[1] - d[1] * e2[0];
    double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0)
        return 0;
    double inv = 1.0 / det;
    for (int c = 0; c < 3; ++c)
        tv[c] = o[c] - v0[c];
    double u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
    if (u < 0.0 || u > 1.0)
        return 0;
    qv[0] = tv[1] * e1[2] - tv[2] * e1[1];
    qv[1] = tv[2] * e1[0] - tv[0] * e1[2];
    qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
    double v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
    if (v < 0.0 || u + v > 1.0)
        return 0;
    *t_out = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
    *u_out = u;
    *v_out = v;
    return 1;
}

/*
 * The same quantities without the inside test: barycentrics (u, v) and t of the
 * ray's meeting point with the triangle's plane.  Returns 0 for a zero
 * determinant.  Used by the tests to tell how close a ray passes to an edge.
 */
int or_ray_triangle_uv(const double o[3], const double d[3], const float *tri, double *t_out,
                       double *u_out, double *v_out)
{
    double v0[3], e1[3], e2[3], pv[3], tv[3], qv[3];
    for (int c = 0; c < 3; ++c) {
        v0[c] = tri[c];
        e1[c] = (double)tri[3 + c] - v0[c];
        e2[c] = (double)tri[6 + c] - v0[c];
    }
    pv[0] = d[1] * e2[2] - d[2] * e2[1];
    pv[1] = d[2] * e2[0] - d[0] * e2[2];
    pv[2] = d[0] * e2[1] - d[1] * e2[0];
    double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0)
        return 0;
    double inv = 1.0 / det;
    for (int c = 0; c < 3; ++c)
        tv[c] = o[c] - v0[c];
    qv[0] = tv[1] * e1[2] - tv[2] * e1[1];
    qv[1] = tv[2] * e1[0] - tv[0] * e1[2];
    qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
    *u_out = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
    *v_out = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
    *t_out = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
    return 1;
}

static void or_write_hit(float *hits, double *info, uint32_t i, uint32_t tri, double t, double u,
                         double v)
{
    float *h = &hits[4 * i];
    if (tri == OR_MISS) {
        h[0] = INFINITY;
        h[1] = 0.0f;
        h[2] = 0.0f;
    } else {
        h[0] = (float)t;
        h[1] = (float)u;
        h[2] = (float)v;
    }
    memcpy(&h[3], &tri, 4);
    if (info) {
        double w = 1.0 - u - v;
        double m = u < v ? u : v;
        info[2 * i + 0] = tri == OR_MISS ? INFINITY : t;
        info[2 * i + 1] = tri == OR_MISS ? INFINITY : (w < m ? w : m);
    }
}

/*
 * The definition: for each ray, the smallest t with tmin < t < tmax over all
 * triangles; on equal t the lowest triangle id.  hits[i] = (t, u, v, tri).
 * info (optional) receives (t in binary64, min(u, v, 1-u-v)) per ray.
 */
void or_trace_brute(const float *tris, uint32_t ntris, const float *o_tmin, const float *d_tmax,
                    uint32_t n, float *hits, double *info)
{
    for (uint32_t i = 0; i < n; ++i) {
        double o[3], d[3];
        for (int c = 0; c < 3; ++c) {
            o[c] = o_tmin[4 * i + c];
            d[c] = d_tmax[4 * i + c];
        }
        double tmin = o_tmin[4 * i + 3];
        double best = d_tmax[4 * i + 3];
        double bu = 0.0, bv = 0.0;
        uint32_t best_tri = OR_MISS;
        for (uint32_t k = 0; k < ntris; ++k) {
            double t, u, v;
            if (!or_ray_triangle(o, d, &tris[9 * k], &t, &u, &v))
                continue;
            if (t > tmin && t < best) {
                best = t;
                bu = u;
                bv = v;
                best_tri = k;
            }
        }
        or_write_hit(hits, info, i, best_tri, best, bu, bv);
    }
}

/*
 * Binary BVH over the triangles (median split of centroids on the longest
 * axis, leaves of at most 4 triangles).  Boxes are exact min/max of the
 * vertices, widened by a relative 1e-9 so that the binary64 slab test can only
 * err toward visiting a node.  A node is skipped only when the ray's interval
 * inside its box starts strictly after the best hit so far, and a triangle
 * replaces the best hit when its t is smaller or equal with a lower id: the
 * result is the brute-force definition above.
 */
typedef struct {
    double lo[3], hi[3];
    uint32_t left;  /* first child node, or first index into order[] for a leaf */
    uint32_t count; /* 0 for an inner node */
} or_node;

typedef struct {
    const float *tris;
    uint32_t ntris;
    or_node *nodes;
    uint32_t nnodes;
    uint32_t *order;
    double *cent;
} or_bvh;

static void or_box_of(const or_bvh *b, uint32_t first, uint32_t count, double lo[3], double hi[3])
{
    for (int c = 0; c < 3; ++c) {
        lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    for (uint32_t k = first; k < first + count; ++k) {
        const float *t = &b->tris[9 * (size_t)b->order[k]];
        for (int v = 0; v < 3; ++v)
            for (int c = 0; c < 3; ++c) {
                double x = t[3 * v + c];
                if (x < lo[c])
                    lo[c] = x;
                if (x > hi[c])
                    hi[c] = x;
            }
    }
    for (int c = 0; c < 3; ++c) {
        double pad = 1e-9 * (fabs(lo[c]) + fabs(hi[c]) + (hi[c] - lo[c])) + 1e-30;
        lo[c] -= pad;
        hi[c] += pad;
    }
}

static int or_cmp_axis;
static const double *or_cmp_cent;
static int or_cent_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    double cx = or_cmp_cent[3 * (size_t)x + or_cmp_axis];
    double cy = or_cmp_cent[3 * (size_t)y + or_cmp_axis];
    if (cx != cy)
        return cx < cy ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static void or_build_node(or_bvh *b, uint32_t node, uint32_t first, uint32_t count)
{
    or_node *nd = &b->nodes[node];
    or_box_of(b, first, count, nd->lo, nd->hi);
    if (count <= 4) {
        nd->left = first;
        nd->count = count;
        return;
    }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t k = first; k < first + count; ++k)
        for (int c = 0; c < 3; ++c) {
            double x = b->cent[3 * (size_t)b->order[k] + c];
            if (x < clo[c])
                clo[c] = x;
            if (x > chi[c])
                chi[c] = x;
        }
    int axis = 0;
    for (int c = 1; c < 3; ++c)
        if (chi[c] - clo[c] > chi[axis] - clo[axis])
            axis = c;
    or_cmp_axis = axis;
    or_cmp_cent = b->cent;
    qsort(&b->order[first], count, sizeof(uint32_t), or_cent_cmp);
    uint32_t half = count / 2;
    uint32_t l = b->nnodes;
    b->nnodes += 2;
    nd = &b->nodes[node];
    nd->left = l;
    nd->count = 0;
    or_build_node(b, l, first, half);
    or_build_node(b, l + 1, first + half, count - half);
}

void *or_bvh_build(const float *tris, uint32_t ntris)
{
    or_bvh *b = (or_bvh *)calloc(1, sizeof(or_bvh));
    if (!b)
        return NULL;
    b->tris = tris;
    b->ntris = ntris;
    b->nodes = (or_node *)calloc(2 * (size_t)(ntris ? ntris : 1), sizeof(or_node));
    b->order = (uint32_t *)malloc((size_t)(ntris ? ntris : 1) * sizeof(uint32_t));
    b->cent = (double *)malloc(3 * (size_t)(ntris ? ntris : 1) * sizeof(double));
    if (!b->nodes || !b->order || !b->cent) {
        free(b->nodes);
        free(b->order);
        free(b->cent);
        free(b);
        return NULL;
    }
    for (uint32_t k = 0; k < ntris; ++k) {
        b->order[k] = k;
        for (int c = 0; c < 3; ++c)
            b->cent[3 * (size_t)k + c] =
                ((double)tris[9 * (size_t)k + c] + tris[9 * (size_t)k + 3 + c] +
                 tris[9 * (size_t)k + 6 + c]) / 3.0;
    }
    b->nnodes = 1;
    if (ntris)
        or_build_node(b, 0, 0, ntris);
    else
        b->nodes[0].count = 0, b->nodes[0].left = 0;
    free(b->cent);
    b->cent = NULL;
    return b;
}

void or_bvh_free(void *h)
{
    or_bvh *b = (or_bvh *)h;
    if (!b)
        return;
    free(b->nodes);
    free(b->order);
    free(b);
}

/* Entry distance of the ray into the box over [tmin, tmax]; returns 0 when disjoint. */
static int or_ray_box(const double o[3], const double d[3], const double lo[3], const double hi[3],
                      double tmin, double tmax, double *tenter)
{
    double a = tmin, z = tmax;
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.0) {
            if (o[c] < lo[c] || o[c] > hi[c])
                return 0;
            continue;
        }
        double t0 = (lo[c] - o[c]) / d[c];
        double t1 = (hi[c] - o[c]) / d[c];
        if (t0 > t1) {
            double s = t0;
            t0 = t1;
            t1 = s;
        }
        if (t0 > a)
            a = t0;
        if (t1 < z)
            z = t1;
    }
    *tenter = a;
    return a <= z;
}

void or_trace_bvh(const void *h, const float *o_tmin, const float *d_tmax, uint32_t n,
                  float *hits, double *info)
{
    const or_bvh *b = (const or_bvh *)h;
    uint32_t stack[128];
    for (uint32_t i = 0; i < n; ++i) {
        double o[3], d[3];
        for (int c = 0; c < 3; ++c) {
            o[c] = o_tmin[4 * i + c];
            d[c] = d_tmax[4 * i + c];
        }
        double tmin = o_tmin[4 * i + 3];
        double best = d_tmax[4 * i + 3];
        double bu = 0.0, bv = 0.0;
        uint32_t best_tri = OR_MISS;
        int sp = 0;
        if (b->ntris)
            stack[sp++] = 0;
        while (sp > 0) {
            const or_node *nd = &b->nodes[stack[--sp]];
            double te;
            if (!or_ray_box(o, d, nd->lo, nd->hi, tmin, best, &te))
                continue;
            if (nd->count == 0) {
                stack[sp++] = nd->left;
                stack[sp++] = nd->left + 1;
                continue;
            }
            for (uint32_t k = nd->left; k < nd->left + nd->count; ++k) {
                uint32_t id = b->order[k];
                double t, u, v;
                if (!or_ray_triangle(o, d, &b->tris[9 * (size_t)id], &t, &u, &v))
                    continue;
                if (t > tmin && (t < best || (t == best && id < best_tri))) {
                    best = t;
                    bu = u;
                    bv = v;
                    best_tri = id;
                }
            }
        }
        or_write_hit(hits, info, i, best_tri, best, bu, bv);
    }
}

/* Depth of the oracle BVH (for sizing its fixed stack in the tests). */
uint32_t or_bvh_depth(const void *h)
{
    const or_bvh *b = (const or_bvh *)h;
    uint32_t best = 0;
    uint32_t st[256], dp[256];
    int sp = 0;
    if (!b->ntris)
        return 0;
    st[sp] = 0;
    dp[sp++] = 1;
    while (sp > 0) {
        --sp;
        uint32_t nd = st[sp], de = dp[sp];
        if (de > best)
            best = de;
        if (b->nodes[nd].count == 0 && sp + 2 < 256) {
            st[sp] = b->nodes[nd].left;
            dp[sp++] = de + 1;
            st[sp] = b->nodes[nd].left + 1;
            dp[sp++] = de + 1;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Capsule coherence measure (Section 4.3)                                   */
/* ------------------------------------------------------------------------ */

/*
 * Surface area of the capsule fitted to `m` rays: the axis joins the centroid
 * of the origins and the centroid of the termination points; the radii are the
 * mean distances of the origins and of the termination points from that axis
 * (from the centroid itself when the two centroids coincide); the area is two
 * hemispheres plus the lateral area of the cone frustum between them.  A ray's
 * termination point is o + dhat * t with t its hit distance, or 4*E for a miss.
 */
static double or_capsule_area(const float *o_tmin, const float *d_tmax, const float *hits, uint32_t first,
                              uint32_t m, float E)
{
    double co[3] = {0, 0, 0}, ct[3] = {0, 0, 0};
    double po[64][3], pt[64][3];
    for (uint32_t k = 0; k < m; ++k) {
        uint32_t i = first + k;
        double d[3], len = 0.0;
        for (int c = 0; c < 3; ++c) {
            d[c] = d_tmax[4 * i + c];
            len += d[c] * d[c];
        }
        len = sqrt(len);
        double t = hits[4 * i + 0];
        uint32_t tri;
        memcpy(&tri, &hits[4 * i + 3], 4);
        if (tri == OR_MISS || !isfinite(t))
            t = 4.0 * (double)E;
        for (int c = 0; c < 3; ++c) {
            po[k][c] = o_tmin[4 * i + c];
            pt[k][c] = po[k][c] + (len > 0.0 ? d[c] / len : 0.0) * t;
            co[c] += po[k][c] / m;
            ct[c] += pt[k][c] / m;
        }
    }
    double a[3], a2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        a[c] = ct[c] - co[c];
        a2 += a[c] * a[c];
    }
    double ro = 0.0, rt = 0.0;
    for (int which = 0; which < 2; ++which)
        for (uint32_t k = 0; k < m; ++k) {
            const double *x = which == 0 ? po[k] : pt[k];
            double v[3], proj = 0.0, dist2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                v[c] = x[c] - co[c];
                proj += v[c] * a[c];
            }
            proj = a2 > 0.0 ? proj / a2 : 0.0;
            for (int c = 0; c < 3; ++c) {
                double w = v[c] - proj * a[c];
                dist2 += w * w;
            }
            if (which == 0)
                ro += sqrt(dist2) / m;
            else
                rt += sqrt(dist2) / m;
        }
    const double pi = 3.14159265358979323846;
    double h = sqrt(a2);
    return 2.0 * pi * ro * ro + 2.0 * pi * rt * rt + pi * (ro + rt) * sqrt(h * h + (ro - rt) * (ro - rt));
}

/*
 * Capsule areas of the consecutive subsets of `subset` rays (1..64); a tail
 * shorter than `subset` is ignored unless n < subset.  out receives
 * max(1, n / subset) values for n > 0; returns their count.
 */
uint32_t or_capsule_areas(const float *o_tmin, const float *d_tmax, const float *hits, uint32_t n,
                          uint32_t subset, float E, double *out)
{
    if (n == 0 || subset == 0 || subset > 64)
        return 0;
    uint32_t groups = n < subset ? 1 : n / subset;
    for (uint32_t g = 0; g < groups; ++g) {
        uint32_t m = n < subset ? n : subset;
        out[g] = or_capsule_area(o_tmin, d_tmax, hits, g * subset, m, E);
    }
    return groups;
}
