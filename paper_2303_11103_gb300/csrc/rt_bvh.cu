// rt_bvh.cu -- GPU BVH builders over Morton-ordered triangles (Karras radix
// tree with bottom-up AABB refit, or PLOC clustering), the 64-byte-node
// traversal layout with its 8 ray-octant copies, and the optional 8-wide
// collapse.
//
// The paper delegates ray/triangle intersection to Mitsuba 3 (Sec. II); the
// acceleration structure here is a linear BVH built in parallel on the GPU:
//   1. per triangle: records, plane, padded AABB, centroid;
//   2. scene bounds; 30-bit Morton code of each centroid (large triangles
//      are set aside and tested directly by every query);
//   3. stable radix sort of the codes (ties keep triangle order, which is
//      Karras' index-augmented key);
//   4. either one thread per internal node finds its key range and split
//      from the longest common prefix of neighbouring keys (Karras 2012),
//      and leaves walk to the root, the second child to arrive at a node
//      computing its box (atomic arrival counters); or
//   5. (default) mutual nearest neighbours of the Morton order merge by
//      smallest merged surface area, round by round, in levels of chunks
//      that stop early (PLOC, below);
//   6. the radix tree's nodes are re-numbered by depth (level order); the
//      clustering's merges are numbered in merge order from the top, so
//      parents come before children and the top of the tree first. Either
//      way the top levels form a prefix that traversal blocks can stage in
//      shared memory;
//   7. a device check that the result is a tree with children after their
//      parents (the traversal loop relies on it instead of an iteration cap).
#include <algorithm>
#include <cstring>

#include "rt_internal.h"

namespace {

// Triangles with an AABB side above this fraction of the scene extent are
// kept out of the hierarchy and tested by every query.
constexpr float BIG_FRAC = 0.25f;

__device__ __forceinline__ unsigned ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// FP64 planes of the triangles (for path lengths): one warp per block, so
// that the few FP64 units of many SMs share the work.
__global__ void k_planes64(const float4* __restrict__ tris_o, int T, double2* __restrict__ pl64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    const float4 r0 = tris_o[3 * (size_t)i], r1 = tris_o[3 * (size_t)i + 1], r2 = tris_o[3 * (size_t)i + 2];
    double n[3];
    plane64(r1, r2, n);
    pl64[3 * (size_t)i] = make_double2(n[0], n[1]);
    pl64[3 * (size_t)i + 1] = make_double2(n[2], (double)r0.x);
    pl64[3 * (size_t)i + 2] = make_double2((double)r0.y, (double)r0.z);
}

// bounds layout (ordered uints): [0..2] vmin, [3..5] vmax, [6..8] cmin, [9..11] cmax
__global__ void k_prep(const float* __restrict__ v, const int32_t* __restrict__ mat, int T,
                       float4* __restrict__ tris_o, float4* __restrict__ planes,
                       float* __restrict__ lbox, float* __restrict__ cent,
                       unsigned* __restrict__ bounds) {
    __shared__ unsigned sb[12];
    if (threadIdx.x < 12) sb[threadIdx.x] = (threadIdx.x % 6) < 3 ? 0xffffffffu : 0u;
    __syncthreads();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T) {
        const float* t = v + 9 * (size_t)i;
        f3 a = mk(t[0], t[1], t[2]), b = mk(t[3], t[4], t[5]), c = mk(t[6], t[7], t[8]);
        f3 e1 = b - a, e2 = c - a;
        tris_o[3 * i] = make_float4(a.x, a.y, a.z, __int_as_float(i));
        tris_o[3 * i + 1] = make_float4(e1.x, e1.y, e1.z, __int_as_float(mat[i]));
        tris_o[3 * i + 2] = make_float4(e2.x, e2.y, e2.z, 0.0f);
        f3 n = cross(e1, e2);
        float nl = sqrtf(dot(n, n));
        n = nl > 0.0f ? n * (1.0f / nl) : mk(0.0f, 0.0f, 1.0f);
        planes[i] = make_float4(n.x, n.y, n.z, dot(n, a));
        float lo[3] = {fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z))};
        float hi[3] = {fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z))};
        float ce[3] = {(a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f),
                       (a.z + b.z + c.z) * (1.0f / 3.0f)};
        for (int k = 0; k < 3; k++) {
            lbox[6 * (size_t)i + k] = lo[k];
            lbox[6 * (size_t)i + 3 + k] = hi[k];
            cent[3 * (size_t)i + k] = ce[k];
            atomicMin(&sb[k], ord(lo[k]));
            atomicMax(&sb[3 + k], ord(hi[k]));
            atomicMin(&sb[6 + k], ord(ce[k]));
            atomicMax(&sb[9 + k], ord(ce[k]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        if ((threadIdx.x % 6) < 3)
            atomicMin(&bounds[threadIdx.x], sb[threadIdx.x]);
        else
            atomicMax(&bounds[threadIdx.x], sb[threadIdx.x]);
    }
}

// Largest side of the vertex bounds (1 for a degenerate scene); the host
// computes the same value from the same words.
__device__ __forceinline__ float bounds_extent(const unsigned* __restrict__ b) {
    float e = 0.0f;
    for (int k = 0; k < 3; k++) e = fmaxf(e, unord(b[3 + k]) - unord(b[k]));
    return e > 0.0f ? e : 1.0f;
}

// Build info words: [0..11] bounds (min words all ones, max words zero),
// [12] large-triangle count, [13] tree depth, [14] clustering status,
// [15] tree check, [16] 8-wide node count, [17] 8-wide depth, [18] 8-wide
// tree check.
constexpr int INFO_WORDS = 20;
__global__ void k_info_init(unsigned* __restrict__ info) {
    int k = threadIdx.x;
    if (k < INFO_WORDS) info[k] = (k < 12 && (k % 6) < 3) ? 0xffffffffu : 0u;
}

__device__ __forceinline__ unsigned expand10(unsigned x) {
    x &= 1023u;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Morton key of each triangle's centroid; a "large" triangle (an AABB side
// above big_side, e.g. a ground quad half) gets the key 2^31 instead, so the
// stable sort moves large triangles behind all others: they are tested
// directly by every query rather than inflating the boxes of the BVH.
__global__ void k_morton(const float* __restrict__ cent, const float* __restrict__ lbox, int T,
                         const unsigned* __restrict__ bounds, uint64_t* __restrict__ keys,
                         uint32_t* __restrict__ vals, unsigned* __restrict__ n_big) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T) return;
    vals[i] = (uint32_t)i;
    const float big_side = BIG_FRAC * bounds_extent(bounds);
    const float* b = lbox + 6 * (size_t)i;
    float side = fmaxf(fmaxf(b[3] - b[0], b[4] - b[1]), b[5] - b[2]);
    if (side > big_side) {
        keys[i] = 1ull << 31;
        atomicAdd(n_big, 1u);
        return;
    }
    // one scale for all axes (the centroid bounds' largest side): a flat
    // city keeps its few height bits low in the code instead of splitting
    // buildings horizontally near the root
    float span = 0.0f;
    for (int k = 0; k < 3; k++) span = fmaxf(span, unord(bounds[9 + k]) - unord(bounds[6 + k]));
    unsigned q[3];
    for (int k = 0; k < 3; k++) {
        float lo = unord(bounds[6 + k]);
        float f = span > 0.0f ? (cent[3 * (size_t)i + k] - lo) / span : 0.5f;
        q[k] = (unsigned)fminf(fmaxf(f * 1024.0f, 0.0f), 1023.0f);
    }
    keys[i] = (uint64_t)((expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]));
}

__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned a = (unsigned)k[i], b = (unsigned)k[j];
    if (a == b) return 32 + __clz((unsigned)i ^ (unsigned)j);
    return __clz(a ^ b);
}

// Karras 2012: internal node i of n-1; children: >= 0 internal, < 0 leaf ~k.
__global__ void k_karras(const uint64_t* __restrict__ k, int n, int2* __restrict__ child,
                         int* __restrict__ par_int, int* __restrict__ par_leaf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int g = i + s * d + min(d, 0);
    int left = (min(i, j) == g) ? ~g : g;
    int right = (max(i, j) == g + 1) ? ~(g + 1) : g + 1;
    child[i] = make_int2(left, right);
    if (left < 0) par_leaf[~left] = i; else par_int[left] = i;
    if (right < 0) par_leaf[~right] = i; else par_int[right] = i;
    if (i == 0) par_int[0] = -1;
}

// ------------------------------------------------------------------ PLOC
// Locally-ordered agglomerative clustering (Meister & Bittner 2018) over the
// Morton-sorted leaves: each round, every cluster picks the neighbour within
// +-PLOC_R positions whose merged box has the smallest surface area; mutual
// nearest neighbours merge into a new internal node that takes the lower
// position; the cluster list is compacted in order. Ties resolve to the
// lower index, so the pair that is smallest in the order (area, lower index,
// higher index) is always mutual and every round merges at least one pair.
//
// The list is clustered in levels. At every level but the last, each block
// takes a chunk of PLOC_C1 consecutive clusters in shared memory (one
// cluster per PLOC_C / PLOC_C1 threads in the first rounds) and merges until
// at most PLOC_T1 remain; the survivors of all chunks, in order, form the
// next level's list, so the merges across chunk borders wait only until
// then. The last level takes the whole remaining list (at most PLOC_C
// clusters) in one block down to the root. Merges are first written to
// provisional slots (level, chunk, merge index within the chunk); the
// emission numbers them m-1-c for the c-th merge in (level, chunk, round,
// position) order, so the root is node 0 and every parent precedes its
// children, the layout the Karras builder produces. Boxes come out of the
// merges (leaf boxes padded as in the refit), so no refit pass is needed.
constexpr int PLOC_C = 1024;   // threads of a level block; clusters of the last level
constexpr int PLOC_C1 = 256;   // clusters of a chunk at the other levels
constexpr int PLOC_T1 = 16;    // a chunk there merges until at most this many remain
constexpr int PLOC_R = 16;
constexpr int PLOC_W = PLOC_C / 32;   // warps of a level block (at most 32)
constexpr int PLOC_MAX_LEVELS = 8;
constexpr int PLOC_MAX_SEG = 4096;    // chunks of a level whose survivors the next level reads

// One level of the clustering: K chunks of C clusters, each merging down to
// `target` clusters (1 at the last level); provisional node slots from
// prov_base, C - 1 per chunk; merge counts of its chunks at group_base.
struct PlocLevel {
    int C, target, K, prov_base, group_base;
};
struct PlocPlan {
    int n_levels, n_groups, n_prov;
    PlocLevel lv[PLOC_MAX_LEVELS];
};

__device__ __forceinline__ float half_area(float lx, float ly, float lz, float hx, float hy, float hz) {
    float dx = hx - lx, dy = hy - ly, dz = hz - lz;
    return fmaf(dx, dy, fmaf(dy, dz, dz * dx));
}

// Padded leaf boxes as six planes of n floats (lo x, y, z, hi x, y, z) and
// leaf ids ~k, in Morton order.
__global__ void k_ploc_leaves(int n, const uint32_t* __restrict__ leaf_tri, const float* __restrict__ lbox,
                              float pad, float* __restrict__ box, int* __restrict__ id) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* b = lbox + 6 * (size_t)leaf_tri[i];
    for (int q = 0; q < 3; q++) {
        box[q * (size_t)n + i] = b[q] - pad;
        box[(3 + q) * (size_t)n + i] = b[3 + q] + pad;
    }
    id[i] = ~i;
}

// Exclusive prefix of n ints (read past L1: written by other blocks) into
// out[0..n] (out[n] = the total), by one whole block.
__device__ void block_prefix(const int* in, int n, int* out) {
    __shared__ int wsum[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {
        int v = j0 + t < n ? __ldcg(in + j0 + t) : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        if (w == 0) {
            int u = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            if (lane < nw) wsum[lane] = u;   // inclusive over warps
        }
        __syncthreads();
        const int base = carry + (w > 0 ? wsum[w - 1] : 0);
        if (j0 + t < n) out[j0 + t + 1] = base + v;
        __syncthreads();
        if (t == 0) carry += wsum[nw - 1];
        __syncthreads();
    }
    if (t == 0) out[0] = 0;
}

// One level: block b clusters positions [b C, (b + 1) C) of the level's
// list. The list is the concatenation, in order, of the previous level's
// chunk outputs (segment j: in_pre[j+1] - in_pre[j] clusters at slot
// j * in_seg of the input arrays), or, when in_pre is null, the first n_in
// clusters. Survivors go to slot b * target of the output arrays, their
// count to out_cnt[b] and the chunk's merge count to mcnt[group_base + b].
// The last block to finish (ticket in *done) writes the exclusive prefix of
// out_cnt to out_pre[0..K] for the next level and, at the last level, the
// prefix of all merge counts to gpre[0..n_groups] for the emission.
__global__ void __launch_bounds__(PLOC_C) k_ploc_level(PlocLevel lv, const float* __restrict__ in_box,
                                                     const int* __restrict__ in_id, const int* __restrict__ in_pre,
                                                     int n_seg, int in_seg, int n_in, float* __restrict__ out_box,
                                                     int* __restrict__ out_id, int* __restrict__ out_cnt,
                                                     int* __restrict__ out_pre, int* __restrict__ mcnt,
                                                     int* __restrict__ gpre, int n_groups, unsigned* __restrict__ done,
                                                     int stride, int2* __restrict__ child, int* __restrict__ par_int,
                                                     float* __restrict__ ibox, unsigned* __restrict__ status) {
    extern __shared__ float ploc_sm[];
    float* sb = ploc_sm;                                          // [2][6][PLOC_C]
    int* sid = reinterpret_cast<int*>(ploc_sm + 12 * PLOC_C);    // [2][PLOC_C]
    int* snn = sid + 2 * PLOC_C;                                  // [PLOC_C]
    __shared__ unsigned wk[PLOC_W], wm[PLOC_W];
    __shared__ bool last_block;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int total = in_pre ? in_pre[n_seg] : n_in;
    const int c0 = blockIdx.x * lv.C;
    const int L = max(0, min(lv.C, total - c0));
    if (t < L) {
        const int p = c0 + t;
        int src = p;
        if (in_pre) {
            int lo = 0, hi = n_seg - 1;   // the last segment j with in_pre[j] <= p
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (in_pre[mid] <= p) lo = mid; else hi = mid - 1;
            }
            src = lo * in_seg + (p - in_pre[lo]);
        }
        for (int q = 0; q < 6; q++) sb[q * PLOC_C + t] = in_box[q * (size_t)stride + src];
        sid[t] = in_id[src];
    }
    __syncthreads();
    const int slot_base = lv.prov_base + blockIdx.x * (lv.C - 1);
    int cur = L, created = 0, buf = 0;
    for (int round = 0; cur > lv.target; round++) {
        if (round >= PLOC_C) {   // unreachable for finite boxes
            if (t == 0) atomicOr(status, 1u);
            cur = 0;   // no survivors: the later levels stay consistent, the build fails
            break;
        }
        const float* rb = sb + buf * 6 * PLOC_C;
        const int* ri = sid + buf * PLOC_C;
        float* wb = sb + (buf ^ 1) * 6 * PLOC_C;
        int* wi = sid + (buf ^ 1) * PLOC_C;
        float lx = 0, ly = 0, lz = 0, hx = 0, hy = 0, hz = 0;
        if (t < cur) {
            lx = rb[t]; ly = rb[PLOC_C + t]; lz = rb[2 * PLOC_C + t];
            hx = rb[3 * PLOC_C + t]; hy = rb[4 * PLOC_C + t]; hz = rb[5 * PLOC_C + t];
        }
        {
            // nearest neighbour of every cluster: G lanes per cluster (as many
            // as the block has to spare, at most 32), each scanning an equal
            // share of the +-PLOC_R window in increasing position order; the
            // shares are combined by (area, position), which keeps the
            // sequential scan's choice (the lowest position of the smallest
            // area), so the tree does not depend on G
            int lg = 0;   // G = 2^lg lanes per cluster
            while (lg < 5 && (cur << (lg + 1)) <= PLOC_C) lg++;
            const int G = 1 << lg;
            const int ci = t >> lg, part = t & (G - 1);
            float best = __int_as_float(0x7f800000);
            int bj = 0x7fffffff;
            // warps without a cluster skip the search (warp-uniform)
            if ((w << 5) < (cur << lg)) {
                if (ci < cur) {
                    const float bx0 = rb[ci], by0 = rb[PLOC_C + ci], bz0 = rb[2 * PLOC_C + ci];
                    const float bx1 = rb[3 * PLOC_C + ci], by1 = rb[4 * PLOC_C + ci], bz1 = rb[5 * PLOC_C + ci];
                    const int per = (2 * PLOC_R) >> lg;   // window offsets -R..-1, 1..R in order, `per` per lane
                    for (int q = part * per; q < (part + 1) * per; q++) {
                        const int j = ci + (q < PLOC_R ? q - PLOC_R : q - PLOC_R + 1);
                        if (j < 0 || j >= cur) continue;
                        float c = half_area(fminf(bx0, rb[j]), fminf(by0, rb[PLOC_C + j]), fminf(bz0, rb[2 * PLOC_C + j]),
                                            fmaxf(bx1, rb[3 * PLOC_C + j]), fmaxf(by1, rb[4 * PLOC_C + j]),
                                            fmaxf(bz1, rb[5 * PLOC_C + j]));
                        if (c < best) { best = c; bj = j; }
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1) {   // G is the same for the whole block
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
                }
                if (ci < cur && part == 0) snn[ci] = bj != 0x7fffffff ? bj : (ci > 0 ? ci - 1 : 1);
            }
        }
        __syncthreads();
        int j = -1;
        bool keep = false, merge = false;
        if (t < cur) {
            j = snn[t];
            const bool mutual = snn[j] == t;
            keep = !(mutual && j < t);
            merge = mutual && t < j;
        }
        // block-wide exclusive ranks of keep and merge (warps past the
        // clusters count zero)
        unsigned bk = 0u, bm = 0u;
        if ((w << 5) < cur) {
            bk = __ballot_sync(0xffffffffu, keep);
            bm = __ballot_sync(0xffffffffu, merge);
        }
        if (lane == 0) { wk[w] = __popc(bk); wm[w] = __popc(bm); }
        __syncthreads();
        if (w == 0) {
            unsigned a = lane < PLOC_W ? wk[lane] : 0u, b = lane < PLOC_W ? wm[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned ya = __shfl_up_sync(0xffffffffu, a, o), yb = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) { a += ya; b += yb; }
            }
            if (lane < PLOC_W) {
                wk[lane] = a;   // inclusive
                wm[lane] = b;
            }
        }
        __syncthreads();
        const unsigned lt = lanemask_lt();
        const int K = (int)wk[PLOC_W - 1], M = (int)wm[PLOC_W - 1];
        if (keep) {
            const int kpos = (w > 0 ? (int)wk[w - 1] : 0) + __popc(bk & lt);
            if (merge) {
                const int mpos = (w > 0 ? (int)wm[w - 1] : 0) + __popc(bm & lt);
                const int node = slot_base + created + mpos;   // provisional slot
                float u[6] = {fminf(lx, rb[j]), fminf(ly, rb[PLOC_C + j]), fminf(lz, rb[2 * PLOC_C + j]),
                              fmaxf(hx, rb[3 * PLOC_C + j]), fmaxf(hy, rb[4 * PLOC_C + j]),
                              fmaxf(hz, rb[5 * PLOC_C + j])};
                const int ca = ri[t], cb = ri[j];
                child[node] = make_int2(ca, cb);
                if (ca >= 0) par_int[ca] = node;
                if (cb >= 0) par_int[cb] = node;
                for (int q = 0; q < 6; q++) { ibox[6 * (size_t)node + q] = u[q]; wb[q * PLOC_C + kpos] = u[q]; }
                wi[kpos] = node;
            } else {
                wb[kpos] = lx; wb[PLOC_C + kpos] = ly; wb[2 * PLOC_C + kpos] = lz;
                wb[3 * PLOC_C + kpos] = hx; wb[4 * PLOC_C + kpos] = hy; wb[5 * PLOC_C + kpos] = hz;
                wi[kpos] = ri[t];
            }
        }
        __syncthreads();
        if (M == 0) {   // unreachable for finite boxes
            if (t == 0) atomicOr(status, 1u);
            cur = 0;
            break;
        }
        created += M;
        cur = K;
        buf ^= 1;
    }
    // survivors, in order, to this chunk's output segment
    if (t < cur) {
        const size_t o = (size_t)blockIdx.x * lv.target + t;
        for (int q = 0; q < 6; q++) out_box[q * (size_t)stride + o] = sb[(buf * 6 + q) * PLOC_C + t];
        out_id[o] = sid[buf * PLOC_C + t];
    }
    if (t == 0) {
        out_cnt[blockIdx.x] = cur;
        mcnt[lv.group_base + blockIdx.x] = created;
        // the last level leaves one cluster: the root (an internal node
        // whenever the list had two or more clusters)
        if (lv.target == 1 && cur == 1 && sid[buf * PLOC_C] >= 0) par_int[sid[buf * PLOC_C]] = -1;
        __threadfence();
        last_block = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last_block) {
        __threadfence();
        block_prefix(out_cnt, gridDim.x, out_pre);
        if (lv.target == 1) block_prefix(mcnt, n_groups, gpre);
    }
}

__device__ __forceinline__ void load_box(const float* b, float* o) {
    for (int k = 0; k < 6; k++) o[k] = __ldcg(b + k);
}

// Bottom-up AABBs; leaf boxes padded by `pad`.
__global__ void k_refit(int n, const uint32_t* __restrict__ leaf_tri, const float* __restrict__ lbox,
                        const int2* __restrict__ child, const int* __restrict__ par_int,
                        const int* __restrict__ par_leaf, float* __restrict__ ibox,
                        int* __restrict__ flag, float pad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int p = par_leaf[k];
    for (int steps = 0; p >= 0 && steps < n; steps++) {
        __threadfence();
        if (atomicAdd(&flag[p], 1) == 0) return;
        int2 c = child[p];
        float a[6], b[6];
        if (c.x < 0) { load_box(lbox + 6 * (size_t)leaf_tri[~c.x], a); for (int q = 0; q < 3; q++) { a[q] -= pad; a[3 + q] += pad; } }
        else load_box(ibox + 6 * (size_t)c.x, a);
        if (c.y < 0) { load_box(lbox + 6 * (size_t)leaf_tri[~c.y], b); for (int q = 0; q < 3; q++) { b[q] -= pad; b[3 + q] += pad; } }
        else load_box(ibox + 6 * (size_t)c.y, b);
        for (int q = 0; q < 3; q++) {
            __stcg(ibox + 6 * (size_t)p + q, fminf(a[q], b[q]));
            __stcg(ibox + 6 * (size_t)p + 3 + q, fmaxf(a[3 + q], b[3 + q]));
        }
        p = par_int[p];
    }
}

// Level-order key (depth << shift) | node, depth clamped to 255 in the key
// (a deeper tree is rejected by the stack check anyway); keys may be null
// (depth only). Slots whose parent is negative count as roots.
__global__ void k_depth(int m, int shift, const int* __restrict__ par_int, uint64_t* __restrict__ keys,
                        int* __restrict__ maxdepth) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int d = 0;
    for (int p = par_int[i]; p >= 0 && d < m; p = par_int[p]) d++;
    if (keys) keys[i] = ((uint64_t)min(d, 255) << shift) | (uint32_t)i;
    atomicMax(maxdepth, d);
}

__global__ void k_rank(int m, uint32_t mask, const uint64_t* __restrict__ keys, int* __restrict__ rank) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) rank[(uint32_t)keys[k] & mask] = k;
}

__global__ void k_emit(int m, const uint64_t* __restrict__ order, const int* __restrict__ rank,
                       const int2* __restrict__ child, const float* __restrict__ ibox,
                       const float* __restrict__ lbox, const uint32_t* __restrict__ leaf_tri,
                       float pad, uint32_t mask, float4* __restrict__ nodes) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    int o = (int)((uint32_t)order[k] & mask);
    int2 c = child[o];
    float a[6], b[6];
    int na, nb;
    if (c.x < 0) { for (int q = 0; q < 6; q++) a[q] = lbox[6 * (size_t)leaf_tri[~c.x] + q]; for (int q = 0; q < 3; q++) { a[q] -= pad; a[3 + q] += pad; } na = c.x; }
    else { for (int q = 0; q < 6; q++) a[q] = ibox[6 * (size_t)c.x + q]; na = rank[c.x]; }
    if (c.y < 0) { for (int q = 0; q < 6; q++) b[q] = lbox[6 * (size_t)leaf_tri[~c.y] + q]; for (int q = 0; q < 3; q++) { b[q] -= pad; b[3 + q] += pad; } nb = c.y; }
    else { for (int q = 0; q < 6; q++) b[q] = ibox[6 * (size_t)c.y + q]; nb = rank[c.y]; }
    float4* p = nodes + 4 * (size_t)k;
    p[0] = make_float4(a[0], a[1], a[2], a[3]);
    p[1] = make_float4(a[4], a[5], b[0], b[1]);
    p[2] = make_float4(b[2], b[3], b[4], b[5]);
    p[3] = make_float4(__int_as_float(na), __int_as_float(nb), 0.0f, 0.0f);
}

// Tree check of the emitted hierarchy (level order): every child index is
// larger than its parent's and in range, and every node but the root and
// every leaf has exactly one parent. Traversal relies on it: each node is
// then visited at most once per query, with no iteration cap.
__global__ void k_check_tree(int m, int n_leaves, const float4* __restrict__ nodes, int* __restrict__ indeg,
                             unsigned* __restrict__ bad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const float4 e = nodes[4 * (size_t)k + 3];
    const int cs[2] = {__float_as_int(e.x), __float_as_int(e.y)};
    for (int j = 0; j < 2; j++) {
        const int c = cs[j];
        if (c >= 0) {
            if (c <= k || c >= m) atomicOr(bad, 1u);
            else atomicAdd(&indeg[c], 1);
        } else {
            if (~c >= n_leaves) atomicOr(bad, 1u);
            else atomicAdd(&indeg[m + ~c], 1);
        }
    }
}

__global__ void k_check_degree(int m, int n_leaves, const int* __restrict__ indeg, unsigned* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m + n_leaves) return;
    if (indeg[i] != (i == 0 ? 0 : 1)) atomicOr(bad, 1u);
}

// Final number of provisional slot s (-1: a slot no merge used): node
// m-1-c for the c-th merge in (level, chunk, merge) order. gpre[g] = merges
// of the groups (level chunks) before group g.
__device__ __forceinline__ int ploc_final(const PlocPlan& pl, const int* gpre, const int* mcnt, int m, int s) {
    for (int l = 0; l < pl.n_levels; l++) {
        const PlocLevel& lv = pl.lv[l];
        if (s < lv.prov_base + lv.K * (lv.C - 1)) {
            const int b = (s - lv.prov_base) / (lv.C - 1), loc = (s - lv.prov_base) - b * (lv.C - 1);
            const int g = lv.group_base + b;
            return loc < mcnt[g] ? m - 1 - (gpre[g] + loc) : -1;
        }
    }
    return -1;
}

// Nodes from the clustering's provisional slots, in the final numbering
// (ploc_final): parents before children, root 0. One thread per slot.
__global__ void k_emit_ploc(PlocPlan pl, const int* __restrict__ mcnt, const int* __restrict__ gpre, int m,
                            const int2* __restrict__ child, const float* __restrict__ ibox,
                            const float* __restrict__ lbox, const uint32_t* __restrict__ leaf_tri, float pad,
                            float4* __restrict__ nodes, unsigned* __restrict__ bad) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0 && gpre[pl.n_groups] != m) atomicOr(bad, 1u);   // every internal node made exactly once
    if (s >= pl.n_prov) return;
    const int k = ploc_final(pl, gpre, mcnt, m, s);
    if (k < 0 || k >= m) return;
    const int2 c = child[s];
    float a[6], b[6];
    int ca = c.x, cb = c.y;
    if (ca < 0) { for (int q = 0; q < 6; q++) a[q] = lbox[6 * (size_t)leaf_tri[~ca] + q]; for (int q = 0; q < 3; q++) { a[q] -= pad; a[3 + q] += pad; } }
    else { for (int q = 0; q < 6; q++) a[q] = ibox[6 * (size_t)ca + q]; ca = ploc_final(pl, gpre, mcnt, m, ca); }
    if (cb < 0) { for (int q = 0; q < 6; q++) b[q] = lbox[6 * (size_t)leaf_tri[~cb] + q]; for (int q = 0; q < 3; q++) { b[q] -= pad; b[3 + q] += pad; } }
    else { for (int q = 0; q < 6; q++) b[q] = ibox[6 * (size_t)cb + q]; cb = ploc_final(pl, gpre, mcnt, m, cb); }
    float4* p = nodes + 4 * (size_t)k;
    p[0] = make_float4(a[0], a[1], a[2], a[3]);
    p[1] = make_float4(a[4], a[5], b[0], b[1]);
    p[2] = make_float4(b[2], b[3], b[4], b[5]);
    p[3] = make_float4(__int_as_float(ca), __int_as_float(cb), 0.0f, 0.0f);
}

__global__ void k_leaf_tris(int n, const uint32_t* __restrict__ leaf_tri, const float4* __restrict__ tris_o,
                            float4* __restrict__ tris) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t t = leaf_tri[k];
    tris[3 * (size_t)k] = tris_o[3 * (size_t)t];
    tris[3 * (size_t)k + 1] = tris_o[3 * (size_t)t + 1];
    tris[3 * (size_t)k + 2] = tris_o[3 * (size_t)t + 2];
}

__global__ void k_single_leaf(const float* __restrict__ lbox, const uint32_t* __restrict__ leaf_tri, float pad,
                              float4* __restrict__ nodes) {
    // one triangle in the hierarchy: both children are leaf 0
    float a[6];
    for (int q = 0; q < 6; q++) a[q] = lbox[6 * (size_t)leaf_tri[0] + q];
    for (int q = 0; q < 3; q++) { a[q] -= pad; a[3 + q] += pad; }
    nodes[0] = make_float4(a[0], a[1], a[2], a[3]);
    nodes[1] = make_float4(a[4], a[5], a[0], a[1]);
    nodes[2] = make_float4(a[2], a[3], a[4], a[5]);
    nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), 0.0f, 0.0f);
}

// ------------------------------------------------------ 8-wide collapse
// The binary hierarchy is collapsed top-down into nodes of up to 8
// children, breadth-first, by one block (a few hundred nodes per level):
//   - a wide node starts from the two children of its binary node and
//     repeatedly opens its internal child of largest surface area, until it
//     has 8 children or only triangles;
//   - each child goes to the slot of the corner it lies towards from the
//     children's common centre (bit a of the slot set for the positive side
//     of axis a), greedily by the largest projection onto the corner's
//     diagonal, so that slot order XOR a ray's octant runs near to far;
//   - the new wide nodes of a level are numbered by a block-wide prefix sum
//     in (parent, child) order, so the layout is deterministic and each
//     level follows the previous one (the top levels form a prefix, staged
//     in shared memory by the traversal kernels).
// The loop is bounded by the binary node count and RT_STACK levels; a
// malformed input sets info[18] instead of running on.
constexpr int WC_THREADS = 256;

__device__ __forceinline__ float half_area(const float* b) {
    const float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return dx * dy + dy * dz + dz * dx;
}

// child c (0, 1) of binary node r: box (lo xyz, hi xyz) and reference
__device__ __forceinline__ void binary_child(const float4* __restrict__ nodes, int r, int c, float* box, int& ref) {
    const float4* p = nodes + 4 * (size_t)r;
    if (c == 0) {
        const float4 a = p[0], b = p[1];
        box[0] = a.x; box[1] = a.y; box[2] = a.z; box[3] = a.w; box[4] = b.x; box[5] = b.y;
    } else {
        const float4 b = p[1], c2 = p[2];
        box[0] = b.z; box[1] = b.w; box[2] = c2.x; box[3] = c2.y; box[4] = c2.z; box[5] = c2.w;
    }
    const float4 e = p[3];
    ref = __float_as_int(c == 0 ? e.x : e.y);
}

__global__ void __launch_bounds__(WC_THREADS) k_collapse(const float4* __restrict__ nodes, int m,
                                                         int* __restrict__ wroot, float4* __restrict__ wnodes,
                                                         unsigned* __restrict__ info) {
    __shared__ int s_count, s_begin, s_end, s_stop;
    __shared__ int s_warp[WC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        wroot[0] = 0;
        s_count = 1;
        s_begin = 0;
        s_end = 1;
        s_stop = 0;
    }
    __syncthreads();
    int depth = 0;
    while (true) {
        const int begin = s_begin, end = s_end;
        if (begin >= end || s_stop) break;
        if (++depth > RT_STACK) {
            if (threadIdx.x == 0) atomicOr(info + 18, 1u);
            break;
        }
        for (int base = begin; base < end; base += WC_THREADS) {
            const int w = base + threadIdx.x;
            const bool act = w < end;
            float box[8][6];
            int ref[8];
            int n = 0;
            bool bad = false;
            if (act) {
                const int r0 = wroot[w];
                if (r0 < 0 || r0 >= m) {
                    bad = true;
                } else {
                    binary_child(nodes, r0, 0, box[0], ref[0]);
                    binary_child(nodes, r0, 1, box[1], ref[1]);
                    n = 2;
                }
                while (!bad && n < 8) {
                    int pick = -1;
                    float best = -1.0f;
                    for (int k = 0; k < n; k++)
                        if (ref[k] >= 0) {
                            const float a = half_area(box[k]);
                            if (a > best) { best = a; pick = k; }
                        }
                    if (pick < 0) break;
                    const int r = ref[pick];
                    if (r >= m) { bad = true; break; }
                    binary_child(nodes, r, 0, box[pick], ref[pick]);
                    binary_child(nodes, r, 1, box[n], ref[n]);
                    n++;
                }
            }
            // corner slots: greedy on the projection onto the corner diagonal
            int slot_of[8];
            if (act && !bad) {
                float c[3] = {0.0f, 0.0f, 0.0f}, lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
                for (int k = 0; k < n; k++)
                    for (int a = 0; a < 3; a++) {
                        lo[a] = fminf(lo[a], box[k][a]);
                        hi[a] = fmaxf(hi[a], box[k][3 + a]);
                    }
                for (int a = 0; a < 3; a++) c[a] = 0.5f * (lo[a] + hi[a]);
                unsigned used = 0, done = 0;
                for (int round = 0; round < n; round++) {
                    float bs = -3e38f;
                    int bk = 0, bslot = 0;
                    for (int k = 0; k < n; k++) {
                        if (done >> k & 1u) continue;
                        float dk[3];
                        for (int a = 0; a < 3; a++) dk[a] = 0.5f * (box[k][a] + box[k][3 + a]) - c[a];
                        for (int sl = 0; sl < 8; sl++) {
                            if (used >> sl & 1u) continue;
                            const float sc = ((sl & 1) ? dk[0] : -dk[0]) + ((sl & 2) ? dk[1] : -dk[1]) +
                                             ((sl & 4) ? dk[2] : -dk[2]);
                            if (sc > bs) { bs = sc; bk = k; bslot = sl; }
                        }
                    }
                    slot_of[bk] = bslot;
                    used |= 1u << bslot;
                    done |= 1u << bk;
                }
            }
            // number the internal children: block-wide exclusive scan
            int ni = 0;
            if (act && !bad)
                for (int k = 0; k < n; k++) ni += ref[k] >= 0;
            int incl = ni;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) s_warp[warp] = incl;
            if (bad) atomicOr(info + 18, 1u);
            __syncthreads();
            int wbase = 0, total = 0;
            for (int q = 0; q < WC_THREADS / 32; q++) {
                if (q < warp) wbase += s_warp[q];
                total += s_warp[q];
            }
            const int count0 = s_count;
            const bool room = count0 + total <= m;
            if (act && !bad && room) {
                int next = count0 + wbase + incl - ni;
                float pl[6][8];
                int rf[8];
                for (int sl = 0; sl < 8; sl++) {
                    for (int a = 0; a < 3; a++) {
                        pl[2 * a][sl] = 1e30f;
                        pl[2 * a + 1][sl] = -1e30f;
                    }
                    rf[sl] = RT_WN_EMPTY;
                }
                unsigned imask = 0, tmask = 0;
                for (int k = 0; k < n; k++) {
                    const int sl = slot_of[k];
                    for (int a = 0; a < 3; a++) {
                        pl[2 * a][sl] = box[k][a];
                        pl[2 * a + 1][sl] = box[k][3 + a];
                    }
                    if (ref[k] >= 0) {
                        wroot[next] = ref[k];
                        rf[sl] = next++;
                        imask |= 1u << sl;
                    } else {
                        rf[sl] = ref[k];
                        tmask |= 1u << sl;
                    }
                }
                float4* wp = wnodes + RT_WN_F4 * (size_t)w;
                for (int q = 0; q < 6; q++) {
                    wp[2 * q] = make_float4(pl[q][0], pl[q][1], pl[q][2], pl[q][3]);
                    wp[2 * q + 1] = make_float4(pl[q][4], pl[q][5], pl[q][6], pl[q][7]);
                }
                wp[12] = make_float4(__int_as_float(rf[0]), __int_as_float(rf[1]), __int_as_float(rf[2]),
                                     __int_as_float(rf[3]));
                wp[13] = make_float4(__int_as_float(rf[4]), __int_as_float(rf[5]), __int_as_float(rf[6]),
                                     __int_as_float(rf[7]));
                wp[14] = make_float4(__uint_as_float(imask | (tmask << 8)), 0.0f, 0.0f, 0.0f);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (room) s_count = count0 + total;
                else s_stop = 1;
            }
            if (!room && threadIdx.x == 0) atomicOr(info + 18, 1u);
            __syncthreads();
            if (s_stop) break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_begin = end;
            s_end = s_count;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        info[16] = (unsigned)s_count;
        info[17] = (unsigned)depth;
    }
}

// Tree check of the 8-wide layout: internal references after their node and
// in range, triangle references in range, masks disjoint; with
// k_check_degree, every node but the root and every triangle referenced once.
__global__ void k_wcheck(const unsigned* __restrict__ info, int n_leaves, const float4* __restrict__ wnodes,
                         int* __restrict__ indeg, unsigned* __restrict__ bad) {
    const int W = (int)info[16];
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const float4* np = wnodes + RT_WN_F4 * (size_t)w;
    const unsigned masks = __float_as_uint(np[14].x);
    const unsigned im = masks & 0xffu, tm = (masks >> 8) & 0xffu;
    if ((im & tm) || (masks >> 16)) atomicOr(bad, 1u);
    const int* rf = reinterpret_cast<const int*>(np + 12);
    for (int sl = 0; sl < 8; sl++) {
        const int r = rf[sl];
        if (im >> sl & 1u) {
            if (r <= w || r >= W) atomicOr(bad, 1u);
            else atomicAdd(&indeg[r], 1);
        } else if (tm >> sl & 1u) {
            if (r >= 0 || ~r >= n_leaves) atomicOr(bad, 1u);
            else atomicAdd(&indeg[W + ~r], 1);
        }
    }
}

__global__ void k_wcheck_degree(const unsigned* __restrict__ info, int n_leaves, const int* __restrict__ indeg,
                                unsigned* __restrict__ bad) {
    const int W = (int)info[16];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W + n_leaves) return;
    if (indeg[i] != (i == 0 ? 0 : 1)) atomicOr(bad, 1u);
}

// Octant copies of the binary nodes: copy 1 + o (after the m binary nodes)
// holds each child box as near x, y, z and far x, y, z planes for rays whose
// direction components are negative exactly on the axes set in o, so that a
// ray's box test needs no per-axis min/max (box_oct). The two children's
// planes are interleaved in pairs (near x of child 0, near x of child 1,
// near y ...), so that one packed FMA takes a plane of both (box_pair); the
// fourth word holds the child references as in the binary nodes.
__global__ void k_octants(int m, float4* __restrict__ nodes) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 8 * m) return;
    const int o = k / m, i = k - o * m;
    const float4* p = nodes + 4 * (size_t)i;
    const float4 a = p[0], b = p[1], c = p[2], e = p[3];
    const float b0[6] = {a.x, a.y, a.z, a.w, b.x, b.y}, b1[6] = {b.z, b.w, c.x, c.y, c.z, c.w};
    float n0[6], n1[6];
    for (int ax = 0; ax < 3; ax++) {
        const bool neg = (o >> ax) & 1;
        n0[ax] = neg ? b0[3 + ax] : b0[ax];
        n0[3 + ax] = neg ? b0[ax] : b0[3 + ax];
        n1[ax] = neg ? b1[3 + ax] : b1[ax];
        n1[3 + ax] = neg ? b1[ax] : b1[3 + ax];
    }
    float4* q = nodes + 4 * ((size_t)(1 + o) * m + i);
    q[0] = make_float4(n0[0], n1[0], n0[1], n1[1]);
    q[1] = make_float4(n0[2], n1[2], n0[3], n1[3]);
    q[2] = make_float4(n0[4], n1[4], n0[5], n1[5]);
    q[3] = e;
}

float host_unord(unsigned u) {
    unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

}  // namespace

int bvh_build(rt_ctx* ctx, const float* verts, int64_t n_tris) {
    const int T = (int)n_tris;
    cudaStream_t st = ctx->stream;
    ctx->n_tris = T;
    if (T == 0) {
        ctx->n_nodes = 0;
        ctx->n_bvh = ctx->n_big = 0;
        ctx->bvh_depth = 0;
        ctx->extent = 1.0f;
        ctx->tmin = 2e-6f;
        return RT_OK;
    }
    const int B = 256;
    const int gT = (T + B - 1) / B;
    RT_TRY(buf_reserve(ctx->tris_o, sizeof(float4) * 3 * (size_t)T));
    RT_TRY(buf_reserve(ctx->tris, sizeof(float4) * 3 * (size_t)T));
    RT_TRY(buf_reserve(ctx->planes, sizeof(float4) * (size_t)T));
    RT_TRY(buf_reserve(ctx->planes64, sizeof(double2) * 3 * (size_t)std::max(T, 1)));
    int m = std::max(T - 1, 1);
    // the binary nodes, then their 8 octant copies (k_octants)
    RT_TRY(buf_reserve(ctx->nodes, sizeof(float4) * 4 * 9 * (size_t)m));
    // build scratch, kept in the context between builds
    RT_TRY(buf_reserve(ctx->b_lbox, sizeof(float) * 6 * (size_t)T));
    RT_TRY(buf_reserve(ctx->b_cent, sizeof(float) * 3 * (size_t)T));
    RT_TRY(buf_reserve(ctx->b_info, sizeof(unsigned) * INFO_WORDS));
    RT_TRY(buf_reserve(ctx->b_keys, sizeof(uint64_t) * T));
    RT_TRY(buf_reserve(ctx->b_keys2, sizeof(uint64_t) * T));
    RT_TRY(buf_reserve(ctx->b_vals, sizeof(uint32_t) * T));
    RT_TRY(buf_reserve(ctx->b_vals2, sizeof(uint32_t) * T));
    float* lbox = bp<float>(ctx->b_lbox);
    unsigned* info = bp<unsigned>(ctx->b_info);
    uint64_t* keys = bp<uint64_t>(ctx->b_keys);
    uint32_t* vals = bp<uint32_t>(ctx->b_vals);
    RT_TRY(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), st));
    prof_begin(ctx, "k_info_init");
    k_info_init<<<1, 32, 0, st>>>(info);
    prof_end(ctx);
    prof_begin(ctx, "k_prep");
    k_prep<<<gT, B, 0, st>>>(verts, bp<int32_t>(ctx->mat), T, bp<float4>(ctx->tris_o), bp<float4>(ctx->planes),
                             lbox, bp<float>(ctx->b_cent), info);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    if (T > 0) {
        prof_begin(ctx, "k_planes64");
        k_planes64<<<(T + 31) / 32, 32, 0, st>>>(bp<float4>(ctx->tris_o), T, bp<double2>(ctx->planes64));
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
    }
    prof_begin(ctx, "k_morton");
    k_morton<<<gT, B, 0, st>>>(bp<float>(ctx->b_cent), lbox, T, info, keys, vals, info + 12);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    RT_TRY(radix_sort64(ctx, keys, bp<uint64_t>(ctx->b_keys2), vals, bp<uint32_t>(ctx->b_vals2), T, 32));
    // bounds and large-triangle count in one read
    unsigned hi[13];
    RT_TRY(cudaMemcpyAsync(ctx->host_rb, info, sizeof(hi), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaMemcpyAsync(ctx->host_rb + 7, ctx->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    memcpy(hi, ctx->host_rb, sizeof(hi));
    if (*reinterpret_cast<unsigned*>(ctx->host_rb + 7) & RT_STAT_SORT)
        return set_err(ctx, RT_ERR_TIMEOUT, "BVH build: radix sort look-back timed out");
    float ext = 0.0f;
    for (int k = 0; k < 3; k++) ext = std::max(ext, host_unord(hi[3 + k]) - host_unord(hi[k]));
    if (!(ext > 0.0f)) ext = 1.0f;
    ctx->extent = ext;
    ctx->tmin = 2e-6f * ext;
    const float pad = 1e-6f * ext;
    // sorted order: triangles of the hierarchy (Morton order), then the large ones (id order)
    const unsigned n_big = hi[12];
    const int n = T - (int)n_big;
    ctx->n_big = (int)n_big;
    ctx->n_bvh = n;
    m = std::max(n - 1, 1);
    const uint32_t* leaf_tri = vals;
    // tree depth, clustering status, tree check, 8-wide node count, depth, check
    int hd[6] = {0, 0, 0, 0, 0, 0};
    if (n == 0) {
        ctx->n_nodes = 0;
        ctx->bvh_depth = 0;
    } else if (n == 1) {
        prof_begin(ctx, "k_single_leaf");
        k_single_leaf<<<1, 1, 0, st>>>(lbox, leaf_tri, pad, bp<float4>(ctx->nodes));
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
        ctx->n_nodes = 1;
        ctx->bvh_depth = 1;
    } else {
        const int T = n;   // the hierarchy's triangles
        const int gT = (T + B - 1) / B;
        // the clustering's levels: chunks of PLOC_C1 merged down to PLOC_T1
        // clusters until at most PLOC_C remain, then one block to the root
        PlocPlan pl{};
        if (ctx->bvh_builder == RT_BVH_PLOC) {
            int U = T;   // clusters entering the level, at most
            while (true) {
                if (pl.n_levels == PLOC_MAX_LEVELS) return set_err(ctx, RT_ERR_CAPACITY, "BVH build: too many levels");
                PlocLevel lv;
                if (U <= PLOC_C) lv = {PLOC_C, 1, 1, pl.n_prov, pl.n_groups};
                else lv = {PLOC_C1, PLOC_T1, (U + PLOC_C1 - 1) / PLOC_C1, pl.n_prov, pl.n_groups};
                pl.lv[pl.n_levels++] = lv;
                pl.n_prov += lv.K * (lv.C - 1);
                pl.n_groups += lv.K;
                if (lv.target == 1) break;
                U = lv.K * lv.target;
            }
        }
        const int slots = std::max(m, pl.n_prov);   // internal nodes, or the clustering's provisional slots
        RT_TRY(buf_reserve(ctx->b_child, sizeof(int2) * slots));
        RT_TRY(buf_reserve(ctx->b_pint, sizeof(int) * slots));
        RT_TRY(buf_reserve(ctx->b_pleaf, sizeof(int) * T));
        RT_TRY(buf_reserve(ctx->b_ibox, sizeof(float) * 6 * (size_t)slots));
        int2* child = bp<int2>(ctx->b_child);
        int* pint = bp<int>(ctx->b_pint);
        int* pleaf = bp<int>(ctx->b_pleaf);
        float* ibox = bp<float>(ctx->b_ibox);
        int gm = (m + B - 1) / B;
        const int* gpre = nullptr;
        const int* mcnt = nullptr;
        if (ctx->bvh_builder == RT_BVH_PLOC) {
            // two cluster lists (six box planes + ids each)
            RT_TRY(buf_reserve(ctx->b_flag, (sizeof(float) * 12 + sizeof(int) * 2) * (size_t)T));
            float* boxA = bp<float>(ctx->b_flag);
            float* boxB = boxA + 6 * (size_t)T;
            int* idA = reinterpret_cast<int*>(boxB + 6 * (size_t)T);
            int* idB = idA + T;
            // counts: per level a ticket, the chunks' survivor counts and their
            // prefix; per chunk its merge count, and their prefix
            size_t n_ints = 2 * (size_t)pl.n_groups + 1;
            for (int l = 0; l < pl.n_levels; l++) n_ints += 1 + 2 * (size_t)pl.lv[l].K + 1;
            RT_TRY(buf_reserve(ctx->b_ploc, sizeof(int) * n_ints));
            RT_TRY(cudaMemsetAsync(ctx->b_ploc.p, 0, sizeof(int) * n_ints, st));
            int* cnt = bp<int>(ctx->b_ploc);
            int* mc = cnt;
            int* gp = mc + pl.n_groups;
            int* next = gp + pl.n_groups + 1;
            mcnt = mc;
            gpre = gp;
            // no parent yet: negative
            RT_TRY(cudaMemsetAsync(pint, 0xFF, sizeof(int) * (size_t)pl.n_prov, st));
            prof_begin(ctx, "k_ploc_leaves");
            k_ploc_leaves<<<gT, B, 0, st>>>(T, leaf_tri, lbox, pad, boxA, idA);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            const size_t smem = (sizeof(float) * 12 + sizeof(int) * 3) * PLOC_C;
            RT_TRY(ensure_smem_attr((const void*)k_ploc_level, smem));
            float *bi = boxA, *bo = boxB;
            int *ii = idA, *io = idB;
            const int* in_pre = nullptr;
            int n_seg = 0, in_seg = 0;
            for (int l = 0; l < pl.n_levels; l++) {
                const PlocLevel& lv = pl.lv[l];
                unsigned* done = reinterpret_cast<unsigned*>(next);
                int* out_cnt = next + 1;
                int* out_pre = out_cnt + lv.K;
                next = out_pre + lv.K + 1;
                prof_begin(ctx, lv.target == 1 ? "k_ploc_level_top" : "k_ploc_level");
                k_ploc_level<<<lv.K, PLOC_C, smem, st>>>(lv, bi, ii, in_pre, n_seg, in_seg, T, bo, io, out_cnt,
                                                         out_pre, mc, gp, pl.n_groups, done, T, child, pint, ibox,
                                                         info + 14);
                prof_end(ctx);
                RT_TRY(cudaGetLastError());
                in_pre = out_pre;
                n_seg = lv.K;
                in_seg = lv.target;
                std::swap(bi, bo);
                std::swap(ii, io);
            }
        } else {
            RT_TRY(buf_reserve(ctx->b_flag, sizeof(int) * m));
            RT_TRY(cudaMemsetAsync(ctx->b_flag.p, 0, sizeof(int) * m, st));
            prof_begin(ctx, "k_karras");
            k_karras<<<gm, B, 0, st>>>(keys, T, child, pint, pleaf);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            prof_begin(ctx, "k_refit");
            k_refit<<<gT, B, 0, st>>>(T, leaf_tri, lbox, child, pint, pleaf, ibox, bp<int>(ctx->b_flag), pad);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
        }
        // depths (the deepest bounds the traversal stack)
        RT_TRY(buf_reserve(ctx->b_dkeys, sizeof(uint64_t) * m));
        RT_TRY(buf_reserve(ctx->b_dkeys2, sizeof(uint64_t) * m));
        RT_TRY(buf_reserve(ctx->b_rank, sizeof(int) * m));
        uint64_t* dkeys = bp<uint64_t>(ctx->b_dkeys);
        int* rank = bp<int>(ctx->b_rank);
        int shift = 1;
        while ((1ll << shift) < m) shift++;
        const uint32_t mask = (uint32_t)((1ull << shift) - 1);
        if (ctx->bvh_builder == RT_BVH_PLOC) {
            // depths over the provisional slots (unused ones have no parent)
            prof_begin(ctx, "k_depth");
            k_depth<<<(pl.n_prov + B - 1) / B, B, 0, st>>>(pl.n_prov, shift, pint, nullptr,
                                                             reinterpret_cast<int*>(info + 13));
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            // the final numbering puts parents before children and the top of
            // the tree first
            prof_begin(ctx, "k_emit");
            k_emit_ploc<<<(pl.n_prov + B - 1) / B, B, 0, st>>>(pl, mcnt, gpre, m, child, ibox, lbox, leaf_tri, pad,
                                                               bp<float4>(ctx->nodes), info + 15);
            prof_end(ctx);
        } else {
            prof_begin(ctx, "k_depth");
            k_depth<<<gm, B, 0, st>>>(m, shift, pint, dkeys, reinterpret_cast<int*>(info + 13));
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            // level order: sort internal nodes by (depth, id)
            RT_TRY(radix_sort64(ctx, dkeys, bp<uint64_t>(ctx->b_dkeys2), nullptr, nullptr, m, shift + 8));
            prof_begin(ctx, "k_rank");
            k_rank<<<gm, B, 0, st>>>(m, mask, dkeys, rank);
            prof_end(ctx);
            prof_begin(ctx, "k_emit");
            k_emit<<<gm, B, 0, st>>>(m, dkeys, rank, child, ibox, lbox, leaf_tri, pad, mask, bp<float4>(ctx->nodes));
            prof_end(ctx);
        }
        RT_TRY(cudaGetLastError());
        // tree check (the cluster lists / refit flags are free again)
        RT_TRY(buf_reserve(ctx->b_flag, sizeof(int) * (size_t)(m + T)));
        int* indeg = bp<int>(ctx->b_flag);
        RT_TRY(cudaMemsetAsync(indeg, 0, sizeof(int) * (size_t)(m + T), st));
        prof_begin(ctx, "k_check_tree");
        k_check_tree<<<gm, B, 0, st>>>(m, T, bp<float4>(ctx->nodes), indeg, info + 15);
        prof_end(ctx);
        prof_begin(ctx, "k_check_degree");
        k_check_degree<<<(m + T + B - 1) / B, B, 0, st>>>(m, T, indeg, info + 15);
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
        ctx->n_nodes = m;
        if (ctx->bvh_width == 8) {
            // wide nodes: at most one per binary node
            RT_TRY(buf_reserve(ctx->wnodes, sizeof(float4) * RT_WN_F4 * (size_t)m));
            RT_TRY(buf_reserve(ctx->b_wroot, sizeof(int) * (size_t)m));
            prof_begin(ctx, "k_collapse");
            k_collapse<<<1, WC_THREADS, 0, st>>>(bp<float4>(ctx->nodes), m, bp<int>(ctx->b_wroot),
                                                 bp<float4>(ctx->wnodes), info);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            RT_TRY(cudaMemsetAsync(indeg, 0, sizeof(int) * (size_t)(m + T), st));
            prof_begin(ctx, "k_wcheck");
            k_wcheck<<<gm, B, 0, st>>>(info, T, bp<float4>(ctx->wnodes), indeg, info + 18);
            prof_end(ctx);
            prof_begin(ctx, "k_wcheck_degree");
            k_wcheck_degree<<<(m + T + B - 1) / B, B, 0, st>>>(info, T, indeg, info + 18);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
        }
    }
    if (ctx->n_nodes > 0) {
        prof_begin(ctx, "k_octants");
        k_octants<<<(8 * ctx->n_nodes + B - 1) / B, B, 0, st>>>(ctx->n_nodes, bp<float4>(ctx->nodes));
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
    }
    // leaf records in sorted order: the hierarchy's leaves, then the large triangles
    prof_begin(ctx, "k_leaf_tris");
    k_leaf_tris<<<gT, B, 0, st>>>(T, leaf_tri, bp<float4>(ctx->tris_o), bp<float4>(ctx->tris));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    ctx->n_wnodes = 0;
    if (n >= 2) {
        RT_TRY(cudaMemcpyAsync(ctx->host_rb, info + 13, sizeof(hd), cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaStreamSynchronize(st));
        memcpy(hd, ctx->host_rb, sizeof(hd));
        if (hd[1] != 0)   // the clustering found no pair to merge: non-finite geometry
            return set_err(ctx, RT_ERR_INVALID_ARG, "BVH build: non-finite triangle boxes");
        if (hd[2] != 0 || (ctx->bvh_width == 8 && hd[5] != 0)) {
            ctx->n_nodes = 0;
            ctx->n_tris = 0;
            return set_err(ctx, RT_ERR_CUDA, "BVH build: hierarchy failed the tree check");
        }
        ctx->bvh_depth = hd[0] + 1;
        if (ctx->bvh_width == 8) ctx->n_wnodes = hd[3];
    }
    if (ctx->bvh_depth + 1 >= RT_STACK)
        return set_err(ctx, RT_ERR_CAPACITY, "BVH deeper than the traversal stack");
    return RT_OK;
}
