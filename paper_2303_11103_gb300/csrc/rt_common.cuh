// rt_common.cuh -- device-side data layout, vector math and BVH traversal
// shared by the kernels of the GB300 radio ray tracer.
//
// Layouts (all in HBM, 16-byte aligned, read with 16-byte vector loads):
//   BVH node  = 4 x float4 (64 B): the AABBs of both children and their
//               indices (child < 0 means leaf triangle ~child). Nodes are in
//               breadth-first order, so the top levels are a prefix that a
//               block can stage in shared memory.
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

// Scene as seen by kernels.
struct DevScene {
    const float4* __restrict__ nodes;   // [n_nodes*4]
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

// Fetch one BVH node: from shared memory if staged, else from global.
__device__ __forceinline__ void fetch_node(const DevScene& s, const float4* sm, int n_sm, int node,
                                           float4& a, float4& b, float4& c, float4& d) {
    if (node < n_sm) {
        const float4* p = sm + 4 * node;
        a = p[0]; b = p[1]; c = p[2]; d = p[3];
    } else {
        const float4* p = s.nodes + 4 * (size_t)node;
        a = ldg4(p); b = ldg4(p + 1); c = ldg4(p + 2); d = ldg4(p + 3);
    }
}

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

// Slab test of one AABB; returns the entry distance, or NaN when missed (so
// that every `tn <= bound` test fails, also against an infinite bound).
// Three-input min/max: near = max(tlo, per-axis near planes), far =
// min(thi, per-axis far planes).
__device__ __forceinline__ float slab(float lox, float loy, float loz, float hix, float hiy, float hiz,
                                      f3 oi, f3 inv, float tlo, float thi) {
    float t0x = fmaf(lox, inv.x, -oi.x), t1x = fmaf(hix, inv.x, -oi.x);
    float t0y = fmaf(loy, inv.y, -oi.y), t1y = fmaf(hiy, inv.y, -oi.y);
    float t0z = fmaf(loz, inv.z, -oi.z), t1z = fmaf(hiz, inv.z, -oi.z);
    float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), tlo));
    float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), thi));
    return tn <= tf ? tn : __int_as_float(0x7fc00000);
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
template <bool C>
__device__ __forceinline__ int closest_hit(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
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
    while (s.n_nodes > 0) {
        float4 a, b, c, e;
        fetch_node(s, sm, n_sm, node, a, b, c, e);
        if (C) cnt.nodes++;
        float tn0 = slab(a.x, a.y, a.z, a.w, b.x, b.y, oi, inv, tmin, tb);
        float tn1 = slab(b.z, b.w, c.x, c.y, c.z, c.w, oi, inv, tmin, tb);
        int c0 = __float_as_int(e.x), c1 = __float_as_int(e.y);
        bool h0 = tn0 <= tb, h1 = tn1 <= tb;
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
            stack[sp++] = farc;
            node = nearc;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
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
template <bool C>
__device__ __forceinline__ bool any_hit(const DevScene& s, const float4* sm, int n_sm, f3 o, f3 d,
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
    while (s.n_nodes > 0) {
        float4 a, b, c, e;
        fetch_node(s, sm, n_sm, node, a, b, c, e);
        if (C) cnt.nodes++;
        float tn0 = slab(a.x, a.y, a.z, a.w, b.x, b.y, oi, inv, tmin, tmax);
        float tn1 = slab(b.z, b.w, c.x, c.y, c.z, c.w, oi, inv, tmin, tmax);
        int c0 = __float_as_int(e.x), c1 = __float_as_int(e.y);
        bool h0 = tn0 <= tmax, h1 = tn1 <= tmax;
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
