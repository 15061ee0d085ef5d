// rt_common.cuh -- device-side data layout, vector math and BVH traversal
// shared by the kernels of the GB300 radio ray tracer.
//
// Layouts (all in HBM, 16-byte aligned, read with 16- or 32-byte vector loads):
//   BVH node  = 4 x float4 (64 B, 64-byte aligned): the AABBs of both
//               children and their indices (child < 0 means leaf triangle
//               ~child). Nodes are in breadth-first order (root first).
//               After the n_nodes nodes follow 8 copies of them, one per ray
//               octant, with the two children's planes stored in pairs
//               (child 0, child 1) per plane: near x, y, z, far x, y, z for
//               that octant; the traversal reads its ray's copy.
//   8-wide node (selectable) = 15 x float4 (240 B), below; collapsed from
//               the binary hierarchy, breadth-first as well.
//   triangle  = 3 x float4 (48 B), leaf (Morton) order: v0 | id,
//               e1 = v1 - v0 | material, e2 = v2 - v0 | 0.
//   plane     = float4 (n, n . v0) per triangle, original order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RT_PI_F 3.14159265358979f
#define RT_PI_D 3.14159265358979323846
#define RT_C0_D 299792458.0
#define RT_EPS0_D 8.8541878128e-12
#define RT_STACK 64
#define RT_MAX_DEPTH 6

// status bits written by kernels into the context's device status word
#define RT_STAT_STACK 1u
#define RT_STAT_CAPACITY 2u
#define RT_STAT_LOOP 4u
#define RT_STAT_SORT 8u   // a radix-sort tile look-back timed out

struct f3 {
    float x, y, z;
};
__host__ __device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__host__ __device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__host__ __device__ __forceinline__ f3 operator-(f3 a) { return {-a.x, -a.y, -a.z}; }
__host__ __device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 unit(f3 a) { return a * rsqrtf(dot(a, a)); }
__device__ __forceinline__ f3 xyz(float4 v) { return {v.x, v.y, v.z}; }

// 8-wide node (rt_set_bvh_width(8)), 15 x float4 = 240 B:
//   [0..1] lo_x of children 0-3 | 4-7,  [2..3] hi_x,
//   [4..5] lo_y, [6..7] hi_y, [8..9] lo_z, [10..11] hi_z,
//   [12..13] child references (int32: >= 0 a wide node, < 0 leaf triangle
//            ~ref in leaf order; empty slots have the box lo = +1e30,
//            hi = -1e30, which no ray hits, and are in neither mask),
//   [14].x   masks: bits 0-7 internal children, bits 8-15 triangle children.
// Child slot s holds the child lying towards the corner whose axis a is
// positive when bit a of s is set, so a ray visits slots in the order
// j XOR octant (j = 0, 1, ...), near to far.
#define RT_WN_F4 15
#define RT_WN_EMPTY (-2147483647 - 1)

// Scene as seen by kernels.
struct DevScene {
    const float4* __restrict__ nodes;   // [n_nodes*4]
    const float4* __restrict__ wnodes;  // [n_wnodes*RT_WN_F4] 8-wide nodes (layout when wide != 0)
    int n_wnodes, wide;
    const float4* __restrict__ tris;    // [T*3] leaf order
    const float4* __restrict__ big;     // [n_big*3] large triangles, tested by every query
    const float4* __restrict__ tris_o;  // [T*3] original order (same record layout)
    const float4* __restrict__ planes;  // [T] original order: n, n.v0
    const double2* __restrict__ pl64;   // [T*3] original order: (n.x, n.y), (n.z, v0.x), (v0.y, v0.z) in FP64
    const int32_t* __restrict__ mat;    // [T] original order
    const float2* __restrict__ mats;    // [M] eps_r, sigma
    int n_tris, n_nodes, n_mat, n_big;
    float tmin;                         // self-intersection offset (metres)
};

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// float4 words per node of the scene's layout, and the node array
__device__ __forceinline__ int node_f4(const DevScene& s) { return s.wide ? RT_WN_F4 : 4; }
__device__ __forceinline__ const float4* node_base(const DevScene& s) { return s.wide ? s.wnodes : s.nodes; }

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ f3 safe_inv(f3 d) {
    const float big = 1e30f;
    float x = fabsf(d.x) > 1e-30f ? 1.0f / d.x : copysignf(big, d.x);
    float y = fabsf(d.y) > 1e-30f ? 1.0f / d.y : copysignf(big, d.y);
    float z = fabsf(d.z) > 1e-30f ? 1.0f / d.z : copysignf(big, d.z);
    return {x, y, z};
}

// Moller-Trumbore, closed barycentric test. Returns t or +inf. The
// barycentric tests run on the numerators scaled by sign(det) (u det >= 0,
// v det >= 0, (u + v) det <= det^2 written as |.| <= |det|), so the one
// division is taken only for rays that pass inside the triangle.
__device__ __forceinline__ float tri_hit(float4 r0, float4 r1, float4 r2, f3 o, f3 d) {
    f3 v0 = xyz(r0), e1 = xyz(r1), e2 = xyz(r2);
    f3 p = cross(d, e2);
    float det = dot(e1, p);
    f3 s = o - v0;
    f3 q = cross(s, e1);
    const float sg = det < 0.0f ? -1.0f : 1.0f;
    float us = dot(s, p) * sg, vs = dot(d, q) * sg;
    bool in = (det != 0.0f) & (us >= 0.0f) & (vs >= 0.0f) & (us + vs <= fabsf(det));
    if (!in) return __int_as_float(0x7f800000);
    return dot(e2, q) / det;
}

// Entry and exit distances of a box whose planes are already chosen by the
// ray's octant (near planes nx, ny, nz: lo where the direction component is
// positive, hi where it is negative; far planes the others), bounded by
// tlo / thi. These are the values the classic slab test computes for the box
// (its per-axis min/max picks exactly these planes) without its six min/max;
// the box is hit when near <= far.
__device__ __forceinline__ float box_near(float nx, float ny, float nz, f3 oi, f3 inv, float tlo) {
    return fmax3(fmaf(nx, inv.x, -oi.x), fmaf(ny, inv.y, -oi.y), fmaxf(fmaf(nz, inv.z, -oi.z), tlo));
}
__device__ __forceinline__ float box_far(float fx, float fy, float fz, f3 oi, f3 inv, float thi) {
    return fmin3(fmaf(fx, inv.x, -oi.x), fmaf(fy, inv.y, -oi.y), fminf(fmaf(fz, inv.z, -oi.z), thi));
}

// Two FMAs in one instruction: (a0 b.x + c.x, a1 b.y + c.y), each rounded
// once, as fmaf rounds.
__device__ __forceinline__ float2 fma2(float a0, float a1, float2 b, float2 c) {
    unsigned long long x, y, z, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(z) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(y), "l"(z));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// 32 bytes in one load (p 32-byte aligned), through the read-only path.
__device__ __forceinline__ void ldg8(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Ray constants of the binary traversal, each held twice so that one packed
// FMA takes the same plane of both children of a node.
struct PairRay {
    float2 ix, iy, iz;   // reciprocal direction
    float2 mx, my, mz;   // -origin * reciprocal direction
};
__device__ __forceinline__ PairRay pair_ray(f3 inv, f3 oi) {
    return {make_float2(inv.x, inv.x), make_float2(inv.y, inv.y), make_float2(inv.z, inv.z),
            make_float2(-oi.x, -oi.x), make_float2(-oi.y, -oi.y), make_float2(-oi.z, -oi.z)};
}

// Entry and exit distances of both child boxes of an octant-copy node
// record (a, b, c: the planes in pairs, near x, y, z, far x, y, z), bounded
// by tlo and thi. Each value is bit for bit the one box_near / box_far
// computes for that child: the same FMA per plane, the same min/max.
__device__ __forceinline__ void box_pair(float4 a, float4 b, float4 c, const PairRay& r, float tlo, float thi,
                                         float& tn0, float& tf0, float& tn1, float& tf1) {
    const float2 nx = fma2(a.x, a.y, r.ix, r.mx), ny = fma2(a.z, a.w, r.iy, r.my), nz = fma2(b.x, b.y, r.iz, r.mz);
    const float2 fx = fma2(b.z, b.w, r.ix, r.mx), fy = fma2(c.x, c.y, r.iy, r.my), fz = fma2(c.z, c.w, r.iz, r.mz);
    tn0 = fmax3(nx.x, ny.x, fmaxf(nz.x, tlo));
    tn1 = fmax3(nx.y, ny.y, fmaxf(nz.y, tlo));
    tf0 = fmin3(fx.x, fy.x, fminf(fz.x, thi));
    tf1 = fmin3(fx.y, fy.y, fminf(fz.y, thi));
}

// A binary node record: four 16-byte loads, or two 32-byte loads (V8).
// Which is faster depends on the kernel around the traversal (its register
// and L1 pressure), so each kernel picks one.
template <bool V8>
__device__ __forceinline__ void load_node(const float4* p, float4& a, float4& b, float4& c, float4& e) {
    if (V8) {
        ldg8(p, a, b);
        ldg8(p + 2, c, e);
    } else {
        a = ldg4(p);
        b = ldg4(p + 1);
        c = ldg4(p + 2);
        e = ldg4(p + 3);
    }
}

// The binary nodes of the ray's octant (sign bits of the reciprocal
// direction; copy 1 + octant after the n_nodes binary nodes).
__device__ __forceinline__ const float4* octant_nodes(const DevScene& s, f3 inv) {
    const unsigned oct = (__float_as_uint(inv.x) >> 31) | ((__float_as_uint(inv.y) >> 31) << 1) |
                         ((__float_as_uint(inv.z) >> 31) << 2);
    return s.nodes + 4 * (size_t)(1 + oct) * s.n_nodes;
}

// Box test with the planes already chosen by the ray's octant: near planes
// (nx, ny, nz: lo where the direction component is positive, hi where it is
// negative) and far planes (fx, fy, fz). The entry and exit distances are
// the same values the slab test computes for that box (the per-axis min/max
// there picks exactly these planes), without its six min/max. (min and max
// are exact, so the grouping of the three-way min/max does not matter.)
__device__ __forceinline__ bool box_oct(float nx, float ny, float nz, float fx, float fy, float fz, f3 oi, f3 inv,
                                        float tlo, float thi) {
    return box_near(nx, ny, nz, oi, inv, tlo) <= box_far(fx, fy, fz, oi, inv, thi);
}

// Bit j of the result is bit (j XOR oct) of m (8-bit masks): slot order to
// the ray's visiting order, and back.
__device__ __forceinline__ unsigned oct_permute(unsigned m, unsigned oct) {
    if (oct & 1u) m = ((m & 0x55u) << 1) | ((m >> 1) & 0x55u);
    if (oct & 2u) m = ((m & 0x33u) << 2) | ((m >> 2) & 0x33u);
    if (oct & 4u) m = ((m & 0x0fu) << 4) | ((m >> 4) & 0x0fu);
    return m;
}

// Ray constants of the wide traversal: reciprocal direction, origin times
// it, octant (bit a set when the direction's component a is negative, by
// the sign of the reciprocal) and the float4 offsets of the near plane
// words of each axis in a node (the far words are at offset XOR 2).
struct WideRay {
    f3 inv, oi;
    unsigned oct;
    int nx, ny, nz;
};
__device__ __forceinline__ WideRay wide_ray(f3 o, f3 d) {
    WideRay r;
    r.inv = safe_inv(d);
    r.oi = {o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z};
    r.oct = (__float_as_uint(r.inv.x) >> 31) | ((__float_as_uint(r.inv.y) >> 31) << 1) |
            ((__float_as_uint(r.inv.z) >> 31) << 2);
    r.nx = (r.oct & 1u) ? 2 : 0;
    r.ny = (r.oct & 2u) ? 6 : 4;
    r.nz = (r.oct & 4u) ? 10 : 8;
    return r;
}

// Hit mask (slot order) of the 8 children of node np against (tlo, thi):
// per group of 4 children, the entry and exit distances are accumulated one
// axis at a time (the values of box_oct, in its order of operations).
__device__ __forceinline__ unsigned wide_children(const float4* np, const WideRay& r, float tlo, float thi) {
    unsigned hm = 0;
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
        float4 n = np[r.nx + h], f = np[(r.nx ^ 2) + h];
        float n0 = fmaf(n.x, r.inv.x, -r.oi.x), n1 = fmaf(n.y, r.inv.x, -r.oi.x);
        float n2 = fmaf(n.z, r.inv.x, -r.oi.x), n3 = fmaf(n.w, r.inv.x, -r.oi.x);
        float f0 = fmaf(f.x, r.inv.x, -r.oi.x), f1 = fmaf(f.y, r.inv.x, -r.oi.x);
        float f2 = fmaf(f.z, r.inv.x, -r.oi.x), f3v = fmaf(f.w, r.inv.x, -r.oi.x);
        n = np[r.ny + h];
        f = np[(r.ny ^ 2) + h];
        n0 = fmaxf(n0, fmaf(n.x, r.inv.y, -r.oi.y));
        n1 = fmaxf(n1, fmaf(n.y, r.inv.y, -r.oi.y));
        n2 = fmaxf(n2, fmaf(n.z, r.inv.y, -r.oi.y));
        n3 = fmaxf(n3, fmaf(n.w, r.inv.y, -r.oi.y));
        f0 = fminf(f0, fmaf(f.x, r.inv.y, -r.oi.y));
        f1 = fminf(f1, fmaf(f.y, r.inv.y, -r.oi.y));
        f2 = fminf(f2, fmaf(f.z, r.inv.y, -r.oi.y));
        f3v = fminf(f3v, fmaf(f.w, r.inv.y, -r.oi.y));
        n = np[r.nz + h];
        f = np[(r.nz ^ 2) + h];
        n0 = fmax3(n0, fmaf(n.x, r.inv.z, -r.oi.z), tlo);
        n1 = fmax3(n1, fmaf(n.y, r.inv.z, -r.oi.z), tlo);
        n2 = fmax3(n2, fmaf(n.z, r.inv.z, -r.oi.z), tlo);
        n3 = fmax3(n3, fmaf(n.w, r.inv.z, -r.oi.z), tlo);
        f0 = fmin3(f0, fmaf(f.x, r.inv.z, -r.oi.z), thi);
        f1 = fmin3(f1, fmaf(f.y, r.inv.z, -r.oi.z), thi);
        f2 = fmin3(f2, fmaf(f.z, r.inv.z, -r.oi.z), thi);
        f3v = fmin3(f3v, fmaf(f.w, r.inv.z, -r.oi.z), thi);
        if (n0 <= f0) hm |= 1u << (4 * h);
        if (n1 <= f1) hm |= 2u << (4 * h);
        if (n2 <= f2) hm |= 4u << (4 * h);
        if (n3 <= f3v) hm |= 8u << (4 * h);
    }
    return hm;
}

// Node pointer: the staged copy in shared memory for the first n_sm nodes,
// else global memory (a generic pointer, so both take the same loads).
__device__ __forceinline__ const float4* wide_node(const DevScene& s, const float4* sm, int n_sm, int node) {
    return node < n_sm ? sm + RT_WN_F4 * node : s.wnodes + RT_WN_F4 * (size_t)node;
}
__device__ __forceinline__ int wide_ref(const float4* np, int slot) {
    return reinterpret_cast<const int*>(np + 12)[slot];
}

// Per-lane traversal counters (BVH node records and triangle records
// fetched, queries), flushed once per warp at kernel end.
struct TravCount {
    unsigned nodes = 0, tris = 0, queries = 0;
};

// Counter slots of the context's device counter array (uint64 each).
#define RT_CNT_WORK 0
#define RT_CNT_PATHS 1
#define RT_CNT_CLOSEST 2
#define RT_CNT_ANY 3
#define RT_CNT_NODES 4
#define RT_CNT_TRIS 5
#define RT_CNT_KEYS 6
#define RT_CNT_PLANE 7   // last coverage segments tested up to the map plane (any hit)

__device__ __forceinline__ void flush_counts(TravCount& c, unsigned long long* counters, int query_slot) {
    unsigned long long n = c.nodes, t = c.tris, q = c.queries;
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0 && counters) {
        atomicAdd(counters + RT_CNT_NODES, n);
        atomicAdd(counters + RT_CNT_TRIS, t);
        atomicAdd(counters + query_slot, q);
    }
}

// Closest hit along o + t d (d unit), t > tmin, triangle `exclude` (original
// id) skipped; equal t resolves to the lowest original id. Returns the
// original triangle id or -1; t_out receives the distance.
//
// The hierarchy is checked at build time to be a tree whose children have
// larger indices than their parent (level order), with depth below
// RT_STACK, so the loop visits each node at most once and the stack cannot
// overflow. C: count node / triangle records and queries in cnt.
template <bool C, bool V8>
__device__ __forceinline__ int closest_hit_b(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
                                             int exclude, float& t_out, TravCount& cnt) {
    t_out = __int_as_float(0x7f800000);
    if (C) cnt.queries++;
    if (s.n_tris == 0) return -1;
    f3 inv = safe_inv(d);
    f3 oi = {o.x * inv.x, o.y * inv.y, o.z * inv.z};
    int stack[RT_STACK];
    int sp = 0;
    int node = 0;
    float tb = __int_as_float(0x7f800000);
    int best = -1;
    const float tmin = s.tmin;
    // large triangles first: a hit there also bounds the traversal below
    for (int k = 0; k < s.n_big; k++) {
        const float4* tp = s.big + 3 * k;
        float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
        if (C) cnt.tris++;
        int id = __float_as_int(r0.w);
        if (id != exclude) {
            float t = tri_hit(r0, r1, r2, o, d);
            if (t > tmin && (t < tb || (t == tb && id < best))) { tb = t; best = id; }
        }
    }
    const float4* onodes = octant_nodes(s, inv);
    const PairRay pr = pair_ray(inv, oi);
    // the most recently deferred child stays in a register (top); the
    // stack in memory holds the ones below it
    const int no_top = 0x7fffffff;
    int top = no_top;
    while (s.n_nodes > 0) {
        float4 a, b, c, e;
        load_node<V8>(onodes + 4 * (size_t)node, a, b, c, e);
        if (C) cnt.nodes++;
        float tn0, tf0, tn1, tf1;
        box_pair(a, b, c, pr, tmin, tb, tn0, tf0, tn1, tf1);
        int c0 = __float_as_int(e.x), c1 = __float_as_int(e.y);
        bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
        if (h0 && c0 < 0) {
            int k = ~c0;
            const float4* tp = s.tris + 3 * (size_t)k;
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != exclude) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && (t < tb || (t == tb && id < best))) { tb = t; best = id; }
            }
            h0 = false;
        }
        if (h1 && c1 < 0) {
            int k = ~c1;
            const float4* tp = s.tris + 3 * (size_t)k;
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != exclude) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && (t < tb || (t == tb && id < best))) { tb = t; best = id; }
            }
            h1 = false;
        }
        if (h0 && h1) {
            int nearc = tn0 <= tn1 ? c0 : c1;
            int farc = tn0 <= tn1 ? c1 : c0;
            if (top != no_top) stack[sp++] = top;
            top = farc;
            node = nearc;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else if (top != no_top) {
            node = top;
            top = no_top;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    t_out = tb;
    return best;
}

// Any occluder on the open segment (tmin, tmax) along o + t d (d unit),
// skipping original ids ex0 / ex1.
template <bool C, bool V8>
__device__ __forceinline__ bool any_hit_b(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
                                          float tmax, int ex0, int ex1, TravCount& cnt) {
    if (C) cnt.queries++;
    if (s.n_tris == 0) return false;
    f3 inv = safe_inv(d);
    f3 oi = {o.x * inv.x, o.y * inv.y, o.z * inv.z};
    int stack[RT_STACK];
    int sp = 0;
    int node = 0;
    const float tmin = s.tmin;
    for (int k = 0; k < s.n_big; k++) {
        const float4* tp = s.big + 3 * k;
        float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
        if (C) cnt.tris++;
        int id = __float_as_int(r0.w);
        if (id != ex0 && id != ex1) {
            float t = tri_hit(r0, r1, r2, o, d);
            if (t > tmin && t < tmax) return true;
        }
    }
    const float4* onodes = octant_nodes(s, inv);
    const PairRay pr = pair_ray(inv, oi);
    while (s.n_nodes > 0) {
        float4 a, b, c, e;
        load_node<V8>(onodes + 4 * (size_t)node, a, b, c, e);
        if (C) cnt.nodes++;
        float tn0, tf0, tn1, tf1;
        box_pair(a, b, c, pr, tmin, tmax, tn0, tf0, tn1, tf1);
        int c0 = __float_as_int(e.x), c1 = __float_as_int(e.y);
        bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
        if (h0 && c0 < 0) {
            const float4* tp = s.tris + 3 * (size_t)(~c0);
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != ex0 && id != ex1) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && t < tmax) return true;
            }
            h0 = false;
        }
        if (h1 && c1 < 0) {
            const float4* tp = s.tris + 3 * (size_t)(~c1);
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != ex0 && id != ex1) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && t < tmax) return true;
            }
            h1 = false;
        }
        if (h0 && h1) {
            stack[sp++] = c1;
            node = c0;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return false;
}

// Closest hit on the 8-wide layout; same contract as closest_hit_b.
//
// Each step intersects the 8 children of one node (octant-selected planes),
// tests the node's hit triangle children at once, then descends into its
// nearest hit internal child; the other hit internal children stay on the
// stack as one entry (node << 8 | their visiting-order mask), taken in
// order when popped. The hierarchy is checked at build time (children after
// parents, every node and triangle referenced once, depth below RT_STACK),
// so each node is entered at most once and the stack cannot overflow.
template <bool C>
__device__ __forceinline__ int closest_hit_w(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
                                             int exclude, float& t_out, TravCount& cnt) {
    t_out = __int_as_float(0x7f800000);
    if (C) cnt.queries++;
    if (s.n_tris == 0) return -1;
    const WideRay r = wide_ray(o, d);
    float tb = __int_as_float(0x7f800000);
    int best = -1;
    const float tmin = s.tmin;
    for (int k = 0; k < s.n_big; k++) {
        const float4* tp = s.big + 3 * k;
        float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
        if (C) cnt.tris++;
        int id = __float_as_int(r0.w);
        if (id != exclude) {
            float t = tri_hit(r0, r1, r2, o, d);
            if (t > tmin && (t < tb || (t == tb && id < best))) { tb = t; best = id; }
        }
    }
    unsigned stack[RT_STACK];
    int sp = 0;
    int node = 0;
    while (s.n_wnodes > 0) {
        const float4* np = wide_node(s, sm, n_sm, node);
        if (C) cnt.nodes++;
        const unsigned hm = wide_children(np, r, tmin, tb);
        const unsigned meta = __float_as_uint(np[14].x);
        unsigned th = hm & (meta >> 8);
        while (th) {
            const int slot = __ffs(th) - 1;
            th &= th - 1;
            const float4* tp = s.tris + 3 * (size_t)(~wide_ref(np, slot));
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != exclude) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && (t < tb || (t == tb && id < best))) { tb = t; best = id; }
            }
        }
        unsigned v = oct_permute(hm & meta & 0xffu, r.oct);
        if (v) {
            const int j = __ffs(v) - 1;
            v &= v - 1;
            if (v) stack[sp++] = ((unsigned)node << 8) | v;
            node = wide_ref(np, j ^ (int)r.oct);
            continue;
        }
        if (sp == 0) break;
        const unsigned e = stack[sp - 1];
        unsigned pv = e & 0xffu;
        const int j = __ffs(pv) - 1;
        pv &= pv - 1;
        if (pv) stack[sp - 1] = (e & ~0xffu) | pv;
        else sp--;
        node = wide_ref(wide_node(s, sm, n_sm, (int)(e >> 8)), j ^ (int)r.oct);
    }
    t_out = tb;
    return best;
}

// Any occluder on the 8-wide layout; same contract as any_hit_b.
template <bool C>
__device__ __forceinline__ bool any_hit_w(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
                                          float tmax, int ex0, int ex1, TravCount& cnt) {
    if (C) cnt.queries++;
    if (s.n_tris == 0) return false;
    const WideRay r = wide_ray(o, d);
    const float tmin = s.tmin;
    for (int k = 0; k < s.n_big; k++) {
        const float4* tp = s.big + 3 * k;
        float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
        if (C) cnt.tris++;
        int id = __float_as_int(r0.w);
        if (id != ex0 && id != ex1) {
            float t = tri_hit(r0, r1, r2, o, d);
            if (t > tmin && t < tmax) return true;
        }
    }
    unsigned stack[RT_STACK];
    int sp = 0;
    int node = 0;
    while (s.n_wnodes > 0) {
        const float4* np = wide_node(s, sm, n_sm, node);
        if (C) cnt.nodes++;
        const unsigned hm = wide_children(np, r, tmin, tmax);
        const unsigned meta = __float_as_uint(np[14].x);
        unsigned th = hm & (meta >> 8);
        while (th) {
            const int slot = __ffs(th) - 1;
            th &= th - 1;
            const float4* tp = s.tris + 3 * (size_t)(~wide_ref(np, slot));
            float4 r0 = ldg4(tp), r1 = ldg4(tp + 1), r2 = ldg4(tp + 2);
            if (C) cnt.tris++;
            int id = __float_as_int(r0.w);
            if (id != ex0 && id != ex1) {
                float t = tri_hit(r0, r1, r2, o, d);
                if (t > tmin && t < tmax) return true;
            }
        }
        unsigned v = oct_permute(hm & meta & 0xffu, r.oct);
        if (v) {
            const int j = __ffs(v) - 1;
            v &= v - 1;
            if (v) stack[sp++] = ((unsigned)node << 8) | v;
            node = wide_ref(np, j ^ (int)r.oct);
            continue;
        }
        if (sp == 0) break;
        const unsigned e = stack[sp - 1];
        unsigned pv = e & 0xffu;
        const int j = __ffs(pv) - 1;
        pv &= pv - 1;
        if (pv) stack[sp - 1] = (e & ~0xffu) | pv;
        else sp--;
        node = wide_ref(wide_node(s, sm, n_sm, (int)(e >> 8)), j ^ (int)r.oct);
    }
    return false;
}

// Closest hit / any hit on a layout: L = 8 the 8-wide nodes, L = 2 the
// binary nodes, L = 0 the scene's own (a branch, uniform across a launch).
// The hot kernels are compiled per layout (L = 2 or 8), so each carries one
// traversal's registers.
// V8: binary node records read by two 32-byte loads instead of four
// 16-byte loads (the 8-wide layout ignores it).
#define RT_LAYOUT_ANY 0
template <bool C, int L = RT_LAYOUT_ANY, bool V8 = true>
__device__ __forceinline__ int closest_hit(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d, int exclude,
                                           float& t_out, TravCount& cnt) {
    if (L == 8 || (L == RT_LAYOUT_ANY && s.wide)) return closest_hit_w<C>(s, sm, n_sm, o, d, exclude, t_out, cnt);
    return closest_hit_b<C, V8>(s, sm, n_sm, o, d, exclude, t_out, cnt);
}
template <bool C, int L = RT_LAYOUT_ANY, bool V8 = true>
__device__ __forceinline__ bool any_hit(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d, float tmax,
                                        int ex0, int ex1, TravCount& cnt) {
    if (L == 8 || (L == RT_LAYOUT_ANY && s.wide)) return any_hit_w<C>(s, sm, n_sm, o, d, tmax, ex0, ex1, cnt);
    return any_hit_b<C, V8>(s, sm, n_sm, o, d, tmax, ex0, ex1, cnt);
}

// Spherical Fibonacci lattice direction of ray i of N (global frame):
// z = 1 - (2i+1)/N, phi = 2 pi frac(i (sqrt5 - 1)/2), computed in FP64 and
// rounded to FP32 once (Sec. II-B: directions on a Fibonacci lattice).
__device__ __forceinline__ f3 fib_dir(long long N, long long i) {
    const double g = (sqrt(5.0) - 1.0) / 2.0;
    double z = 1.0 - (2.0 * (double)i + 1.0) / (double)N;
    double x = (double)i * g;
    double phi = 2.0 * RT_PI_D * (x - floor(x));
    double rho = sqrt(1.0 - z * z);
    double sp, cp;
    sincos(phi, &sp, &cp);
    return {(float)(rho * cp), (float)(rho * sp), (float)z};
}

// Length of the specular path tx -> triangles ids[0..K-1] -> rx, in FP64:
// for a specular path it equals |rx - I_K|, I_K the last image of tx, with
// the planes' normals taken in FP64 from the stored FP32 triangle edges.
// FP64 unit normal of a triangle from its FP32 edge vectors (computed once
// per triangle at scene load; path lengths reuse it).
__device__ __forceinline__ void plane64(float4 r1, float4 r2, double n[3]) {
    double e1[3] = {r1.x, r1.y, r1.z}, e2[3] = {r2.x, r2.y, r2.z};
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double inl = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] *= inl;
    n[1] *= inl;
    n[2] *= inl;
}

// Length of the specular path tx -> triangles ids[0..K) -> rx in FP64: the
// distance from rx to the last image of tx (images through the triangles'
// FP64 planes).
__device__ __forceinline__ double path_length64(const DevScene& s, const int32_t* ids, int K, f3 tx, f3 rx) {
    double I[3] = {(double)tx.x, (double)tx.y, (double)tx.z};
    for (int k = 0; k < K; k++) {
        const double2* pp = s.pl64 + 3 * (size_t)ids[k];
        const double2 p0 = pp[0], p1 = pp[1], p2 = pp[2];
        const double n[3] = {p0.x, p0.y, p1.x}, v0[3] = {p1.y, p2.x, p2.y};
        double sd = (I[0] - v0[0]) * n[0] + (I[1] - v0[1]) * n[1] + (I[2] - v0[2]) * n[2];
        for (int q = 0; q < 3; q++) I[q] -= 2.0 * sd * n[q];
    }
    double dx = (double)rx.x - I[0], dy = (double)rx.y - I[1], dz = (double)rx.z - I[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

// Specular reflection of d about the plane with unit normal n.
__device__ __forceinline__ f3 reflect(f3 d, f3 n) { return d - n * (2.0f * dot(d, n)); }

// Warp helpers
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
