// rt_paths.cu -- from SBR candidates to stored specular paths (Sec. II-B):
// duplicate removal (sorted keys + warp compare), candidate images, the
// image-method validator with visibility tests, canonical path order, the
// path finalisation (reflection points in FP32, path length in FP64).
#include "rt_field.cuh"
#include "rt_internal.h"

namespace {

constexpr int DD_THREADS = 256;
constexpr int DD_IPT = 8;
constexpr int DD_TILE = DD_THREADS * DD_IPT;

// ---------------------------------------------------------- duplicate removal
// A sorted key starts a run if it differs from its predecessor (warp shuffle
// compare, lane 0 reads the previous key from memory) and is not a sentinel.
__device__ __forceinline__ bool run_start(const uint64_t* __restrict__ k, int64_t n, int64_t i,
                                          uint64_t sentinel_from, uint64_t& key) {
    bool in = i < n;
    key = in ? k[i] : ~0ull;
    uint64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    if ((threadIdx.x & 31) == 0) prev = (in && i > 0) ? k[i - 1] : ~0ull;
    return in && key < sentinel_from && (i == 0 || prev != key);
}

__global__ void __launch_bounds__(DD_THREADS) k_dedup_count(const uint64_t* __restrict__ k, int64_t n,
                                                            uint64_t sentinel_from, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t wc[DD_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * DD_TILE;
    uint32_t c = 0;
    for (int j = 0; j < DD_IPT; j++) {
        uint64_t key;
        bool f = run_start(k, n, base + j * DD_THREADS + threadIdx.x, sentinel_from, key);
        c += __popc(__ballot_sync(0xffffffffu, f));
    }
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < DD_THREADS / 32; w++) s += wc[w];
        cnt[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(DD_THREADS) k_dedup_write(const uint64_t* __restrict__ k,
                                                            const uint32_t* __restrict__ v, int64_t n,
                                                            uint64_t sentinel_from,
                                                            const uint32_t* __restrict__ off,
                                                            uint64_t* __restrict__ out_k,
                                                            uint32_t* __restrict__ out_v) {
    __shared__ uint32_t wbase[DD_THREADS / 32];
    __shared__ uint32_t run;
    if (threadIdx.x == 0) run = off[blockIdx.x];
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * DD_TILE;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < DD_IPT; j++) {
        int64_t i = base + j * DD_THREADS + threadIdx.x;
        uint64_t key;
        bool f = run_start(k, n, i, sentinel_from, key);
        unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wbase[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = run;
            for (int q = 0; q < DD_THREADS / 32; q++) {
                uint32_t t = wbase[q];
                wbase[q] = s;
                s += t;
            }
            run = s;
        }
        __syncthreads();
        if (f) {
            uint32_t pos = wbase[w] + __popc(m & lanemask_lt());
            out_k[pos] = key;
            out_v[pos] = v[i];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- candidates
struct KeyFmt {
    int D, id_bits, depth_shift, tx_shift;
    __device__ __forceinline__ int depth(uint64_t k) const { return (int)((k >> depth_shift) & 7ull); }
    __device__ __forceinline__ int tx(uint64_t k) const { return (int)(k >> tx_shift); }
    __device__ __forceinline__ int id(uint64_t k, int b) const {
        return (int)((k >> ((D - 1 - b) * id_bits)) & ((1ull << id_bits) - 1ull));
    }
};

// LOS keys after the shooting keys: at `at`, or at *at_dev when given (the
// shooting pass's key count, still on the device)
__global__ void k_write_los(uint64_t* keys, uint32_t* vals, int64_t at, const unsigned long long* at_dev, int n_tx,
                            KeyFmt f) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (at_dev) at = (int64_t)*at_dev;
    if (t < n_tx) {
        keys[at + t] = (uint64_t)t << f.tx_shift;
        vals[at + t] = 0xFFFFFFFFu;
    }
}

// witness of every distinct key = the smallest position among its copies
// (the sorted runs keep the append order, which the warps' atomics decide)
__global__ void k_dedup_minwit(const uint64_t* __restrict__ k, const uint32_t* __restrict__ v, int64_t n,
                               const uint64_t* __restrict__ ck, const uint32_t* __restrict__ Up,
                               unsigned* __restrict__ cw) {
    const int64_t U = *Up;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = k[i];
        int64_t lo = 0, hi = U;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (ck[mid] < key) lo = mid + 1; else hi = mid;
        }
        if (lo < U) atomicMin(&cw[lo], v[i]);
    }
}

// per-tx candidate ranges: off[t] = first candidate with tx >= t
__global__ void k_cand_off(const uint64_t* __restrict__ ck, const uint32_t* __restrict__ Up, int n_tx, KeyFmt f,
                           int64_t* __restrict__ off) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_tx) return;
    int64_t lo = 0, hi = *Up;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (f.tx(ck[mid]) < t) lo = mid + 1; else hi = mid;
    }
    off[t] = lo;
}

// ---------------------------------------------------- hash duplicate removal
// Candidate keys into an open-addressing table (linear probing, size a
// power of two at least twice the key count, empty slots all ones, which no
// key equals since keys are narrower than 64 bits); a slot's witness is the
// smallest producing position (deterministic). The occupied slots are then
// compacted and sorted, so the candidate order is the key order. The slot
// hash is MurmurHash3's 64-bit finaliser (Appleby).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// n_dev (optional): the key count is *n_dev + n on the device; when it
// exceeds cap (a table sized from an earlier call), nothing is inserted and
// *overflow is set, so that the host repeats the pass with the count read.
__global__ void k_hash_insert(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n,
                              const unsigned long long* __restrict__ n_dev, int64_t cap, unsigned* __restrict__ overflow,
                              unsigned long long* __restrict__ tab, unsigned* __restrict__ wit, uint64_t mask) {
    // rays of one warp are coherent, so equal keys are merged in the warp first
    // (one table access and one atomicMin per distinct key of the warp)
    if (n_dev) {
        n += (int64_t)*n_dev;
        if (n > cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(overflow, 1u);
            return;
        }
    }
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + lane;
        const bool ok = i < n;
        const unsigned long long k = ok ? keys[i] : ~0ull;
        const unsigned v = ok ? vals[i] : 0xFFFFFFFFu;
        const unsigned grp = __match_any_sync(0xffffffffu, k);
        const unsigned vmin = __reduce_min_sync(grp, v);
        if (!ok || lane != __ffs(grp) - 1) continue;
        uint64_t h = mix64(k) & mask;
        for (uint64_t probe = 0; probe <= mask; probe++) {   // the table is at most half full
            unsigned long long cur = tab[h];
            if (cur == ~0ull) cur = atomicCAS(&tab[h], ~0ull, k);
            if (cur == ~0ull || cur == k) {
                atomicMin(&wit[h], vmin);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void k_hash_compact(const unsigned long long* __restrict__ tab, const unsigned* __restrict__ wit,
                               int64_t S, uint64_t* __restrict__ ck, uint32_t* __restrict__ cw,
                               unsigned* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool occ = i < S && tab[i] != ~0ull;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned b0 = 0;
    if (lane == leader) b0 = atomicAdd(count, (unsigned)__popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, leader);
    if (occ) {
        const unsigned pos = b0 + __popc(m & lanemask_lt());
        ck[pos] = tab[i];
        cw[pos] = wit[i];
    }
}

// images I_k of the transmitter through the candidate's planes (FP32)
__device__ __forceinline__ void cand_img_one(const uint64_t* __restrict__ ck, int64_t c, KeyFmt f,
                                             const float* __restrict__ tx_pos, const float4* __restrict__ planes,
                                             float* __restrict__ img) {
    uint64_t key = ck[c];
    int K = f.depth(key), t = f.tx(key);
    f3 I = mk(tx_pos[3 * t], tx_pos[3 * t + 1], tx_pos[3 * t + 2]);
    for (int k = 0; k < K; k++) {
        float4 pl = planes[f.id(key, k)];
        f3 n = xyz(pl);
        I = I - n * (2.0f * (dot(n, I) - pl.w));
        img[(c * f.D + k) * 3] = I.x;
        img[(c * f.D + k) * 3 + 1] = I.y;
        img[(c * f.D + k) * 3 + 2] = I.z;
    }
}


__global__ void k_cand_img(const uint64_t* __restrict__ ck, const uint32_t* __restrict__ Up, KeyFmt f,
                           const float* __restrict__ tx_pos, const float4* __restrict__ planes,
                           float* __restrict__ img) {
    const int64_t U = *Up;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < U; c += (int64_t)gridDim.x * blockDim.x)
        cand_img_one(ck, c, f, tx_pos, planes, img);
}

// Validation work offsets in warp units: work_off[t] = sum over t' < t of
// U_t' ceil(R_t' / 32), a unit being one candidate against 32 receivers (one
// block; n_tx entries scanned in thread-contiguous runs).
__global__ void __launch_bounds__(1024) k_work_off(const int64_t* __restrict__ cand_off,
                                                   const int32_t* __restrict__ rx_off, int n_tx, int n_rx,
                                                   int64_t* __restrict__ work_off) {
    __shared__ long long ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int seg = (n_tx + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min((int)threadIdx.x * seg, n_tx), s1 = min(s0 + seg, n_tx);
    long long sum = 0;
    for (int t = s0; t < s1; t++) {
        long long R = ((rx_off ? (long long)(rx_off[t + 1] - rx_off[t]) : (long long)n_rx) + 31) >> 5;
        sum += (cand_off[t + 1] - cand_off[t]) * R;
    }
    long long x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        ws[lane] = v;
    }
    __syncthreads();
    long long run = x - sum + (w > 0 ? ws[w - 1] : 0);
    for (int t = s0; t < s1; t++) {
        work_off[t] = run;
        long long R = ((rx_off ? (long long)(rx_off[t + 1] - rx_off[t]) : (long long)n_rx) + 31) >> 5;
        run += (cand_off[t + 1] - cand_off[t]) * R;
    }
    if (threadIdx.x == blockDim.x - 1) work_off[n_tx] = run;
}

// ------------------------------------------------------------ image method
struct ValParams {
    DevScene s;
    KeyFmt f;
    const float* tx_pos;
    const float* rx_pos;
    const uint64_t* cand_key;
    const float* cand_img;
    const int64_t* cand_off;   // [n_tx+1]
    const int64_t* work_off;   // [n_tx+1]
    const int32_t* rx_off;     // [n_tx+1] or null
    int n_tx, n_rx;            // total work = work_off[n_tx]
    uint64_t* out;
    unsigned long long* count;
    long long cap;
    int n_sm;
    unsigned* status;
};

// Back-projection from rx through the candidate's images (Sec. II-B image
// method): P[K+1] = rx, P[k] = crossing of P[k+1] -> I_k with plane k, which
// must lie inside triangle k (closed test) at line parameter in (0, 1).
__device__ __forceinline__ bool back_project(const DevScene& s, const KeyFmt& f, uint64_t key, int K,
                                             const float* img, f3 tx, f3 rx, f3* P, int* ids) {
    P[0] = tx;
    P[K + 1] = rx;
    for (int k = 0; k < K; k++) ids[k] = f.id(key, k);
    for (int k = 1; k < K; k++)
        if (ids[k] == ids[k - 1]) return false;
    for (int k = K; k >= 1; k--) {
        f3 I = mk(img[(k - 1) * 3], img[(k - 1) * 3 + 1], img[(k - 1) * 3 + 2]);
        f3 o = P[k + 1];
        f3 dir = I - o;
        const float4* tp = s.tris_o + 3 * (size_t)ids[k - 1];
        float4 r0 = __ldg(tp), r1 = __ldg(tp + 1), r2 = __ldg(tp + 2);
        float t = tri_hit(r0, r1, r2, o, dir);
        if (!(t > 0.0f && t < 1.0f)) return false;
        P[k] = o + dir * t;
    }
    return true;
}

__device__ __forceinline__ bool sides_ok(const DevScene& s, int K, const f3* P, const int* ids) {
    for (int k = 1; k <= K; k++) {
        float4 pl = __ldg(s.planes + ids[k - 1]);
        f3 n = xyz(pl);
        float s1 = dot(n, P[k - 1]) - pl.w, s2 = dot(n, P[k + 1]) - pl.w;
        if (!((s1 > 0.0f && s2 > 0.0f) || (s1 < 0.0f && s2 < 0.0f))) return false;
    }
    return true;
}

// Per-warp scratch of k_validate, sized by the candidates' depth D: the
// queue of work items that passed the last-reflection test [VQ] (candidate,
// receiver, transmitter), the 32 batch items' path points [32][D+2][3], ids
// [32][D], depths [32], and the queue of their segments still to be tested
// for occluders [32 (D+1)] (lane << 3 | segment).
constexpr int VQ = 64;
__host__ __device__ __forceinline__ size_t val_warp_bytes(int D) {
    return ((size_t)VQ * 16 + (size_t)32 * (D + 2) * 3 * 4 + (size_t)32 * D * 4 + 32 * 4 + (size_t)32 * (D + 1) +
            15) & ~(size_t)15;
}

struct ValWarpPtrs {
    uint32_t* qc;      // [VQ] candidate
    uint32_t* qr;      // [VQ] receiver (global index)
    uint32_t* qt;      // [VQ] transmitter
    float* pts;        // [32][D+2][3]
    int* ids;          // [32][D]
    int* K;            // [32]
    unsigned char* sq; // [32 (D+1)]
};

__device__ __forceinline__ ValWarpPtrs val_warp(float4* sm, int staged_f4, int D) {
    uint8_t* b = reinterpret_cast<uint8_t*>(sm + staged_f4) + (threadIdx.x >> 5) * val_warp_bytes(D);
    ValWarpPtrs w;
    w.qc = reinterpret_cast<uint32_t*>(b);
    w.qr = w.qc + VQ;
    w.qt = w.qr + VQ;
    w.pts = reinterpret_cast<float*>(w.qt + 2 * VQ);
    w.ids = reinterpret_cast<int*>(w.pts + 32 * (D + 2) * 3);
    w.K = w.ids + 32 * D;
    w.sq = reinterpret_cast<unsigned char*>(w.K + 32);
    return w;
}

// Full validation of up to 32 queued items (lane < n takes item (head +
// lane) % VQ): back-projection through every image, side tests, then the
// occluder tests of all passing items' segments, queued so that the lanes
// run them side by side, skipping segments of items already occluded;
// valid paths are appended. Called by all 32 lanes.
template <bool C, int L>
__device__ void validate_batch(const ValParams& p, const float4* sm, const ValWarpPtrs& W, int head, int n,
                               TravCount& cnt) {
    const int lane = threadIdx.x & 31, D = p.f.D;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    bool valid = false;
    uint64_t rec = 0;
    int K = 0;
    if (lane < n) {
        const int e = (head + lane) % VQ;
        const long long c = W.qc[e], rxg = W.qr[e];
        const int t = (int)W.qt[e];
        const long long pair = p.rx_off ? rxg : (long long)t * p.n_rx + rxg;
        const uint64_t key = p.cand_key[c];
        K = p.f.depth(key);
        f3 tx = mk(p.tx_pos[3 * t], p.tx_pos[3 * t + 1], p.tx_pos[3 * t + 2]);
        f3 rx = mk(p.rx_pos[3 * rxg], p.rx_pos[3 * rxg + 1], p.rx_pos[3 * rxg + 2]);
        f3 P[RT_MAX_DEPTH + 2];
        int ids[RT_MAX_DEPTH];
        valid = back_project(p.s, p.f, key, K, p.cand_img + (size_t)c * D * 3, tx, rx, P, ids) &&
                sides_ok(p.s, K, P, ids);
        if (valid) {
            float* pl = W.pts + lane * (D + 2) * 3;
            for (int k = 0; k <= K + 1; k++) {
                pl[3 * k] = P[k].x;
                pl[3 * k + 1] = P[k].y;
                pl[3 * k + 2] = P[k].z;
            }
            for (int k = 0; k < K; k++) W.ids[lane * D + k] = ids[k];
            W.K[lane] = K;
        }
        rec = ((uint64_t)pair << 32) | (uint64_t)c;
    }
    // queue the K+1 segments of every item that passed
    int nq_l = valid ? K + 1 : 0, qo = nq_l;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(full, qo, o);
        if (lane >= o) qo += y;
    }
    const int nq = __shfl_sync(full, qo, 31);
    qo -= nq_l;
    for (int j = 0; j < nq_l; j++) W.sq[qo + j] = (unsigned char)((lane << 3) | j);
    __syncwarp();
    unsigned occluded = 0;   // items with an occluded segment (warp-uniform)
    for (int qb = 0; qb < nq; qb += 32) {
        const int qi = qb + lane;
        bool act = qi < nq;
        int il = 0, j = 0;
        if (act) {
            const unsigned code = W.sq[qi];
            il = (int)(code >> 3);
            j = (int)(code & 7u);
            act = !((occluded >> il) & 1u);
        }
        bool hit = false;
        if (act) {
            const int Ki = W.K[il];
            const float* pl = W.pts + (il * (D + 2) + j) * 3;
            f3 a = mk(pl[0], pl[1], pl[2]);
            f3 b = mk(pl[3], pl[4], pl[5]);
            f3 seg = b - a;
            float Ls = sqrtf(dot(seg, seg));
            f3 d = seg * (1.0f / Ls);
            int ex0 = j >= 1 ? W.ids[il * D + j - 1] : -1, ex1 = j < Ki ? W.ids[il * D + j] : -1;
            hit = any_hit<C, L>(p.s, sm, p.n_sm, a, d, Ls - p.s.tmin, ex0, ex1, cnt);
        }
        occluded |= __reduce_or_sync(full, hit ? (1u << il) : 0u);
    }
    valid = valid && !((occluded >> lane) & 1u);
    __syncwarp();
    unsigned m = __ballot_sync(full, valid);
    if (m) {
        int leader = __ffs(m) - 1;
        unsigned long long b0 = 0;
        if (lane == leader) b0 = atomicAdd(p.count, (unsigned long long)__popc(m));
        b0 = __shfl_sync(full, b0, leader);
        if (valid) {
            unsigned long long idx = b0 + __popc(m & lt);
            if ((long long)idx < p.cap) p.out[idx] = rec;
        }
    }
}

// Image method for every (candidate, receiver) pair (Sec. II-B). A warp
// takes one candidate against 32 receivers (warp units) and first applies
// only the last reflection's test: the segment from the receiver towards the
// candidate's last image must cross the last triangle (closed test, line
// parameter in (0, 1)). Most pairs fail it; the ones that pass go to a
// per-warp queue, and whenever 32 are queued they are validated in full
// (validate_batch) with all lanes busy.
template <bool C, int L>
__global__ void __launch_bounds__(256, 4) k_validate(ValParams p) {
    extern __shared__ float4 sm[];
    const float4* src = node_base(p.s);
    const int staged_f4 = p.n_sm * node_f4(p.s);
    for (int i = threadIdx.x; i < staged_f4; i += blockDim.x) sm[i] = src[i];
    const int D = p.f.D;
    const ValWarpPtrs W = val_warp(sm, staged_f4, D);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu, lt = lanemask_lt();
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    const long long total = p.work_off[p.n_tx];   // warp units: (candidate, 32 receivers)
    TravCount cnt;
    int head = 0, count = 0;   // survivor queue (warp-uniform)
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < total; u += wstride) {
        // the unit's transmitter, candidate and first receiver (warp-uniform)
        int lo = 0, hi = p.n_tx;  // largest t with work_off[t] <= u
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (p.work_off[mid] <= u) lo = mid; else hi = mid;
        }
        const int t = lo;
        const long long R = p.rx_off ? (long long)(p.rx_off[t + 1] - p.rx_off[t]) : (long long)p.n_rx;
        const long long chunks = (R + 31) >> 5;
        const long long local = u - p.work_off[t];
        const long long cl = local / chunks;
        const long long r = ((local - cl * chunks) << 5) + lane;
        const long long c = p.cand_off[t] + cl;
        const uint64_t key = p.cand_key[c];
        const int K = p.f.depth(key);
        bool pass = false;
        long long rxg = 0;
        if (r < R) {
            rxg = p.rx_off ? (long long)p.rx_off[t] + r : r;
            f3 rx = mk(p.rx_pos[3 * rxg], p.rx_pos[3 * rxg + 1], p.rx_pos[3 * rxg + 2]);
            if (K == 0) {
                pass = true;
            } else {
                const float* img = p.cand_img + ((size_t)c * D + (K - 1)) * 3;
                f3 dir = mk(img[0], img[1], img[2]) - rx;
                const float4* tp = p.s.tris_o + 3 * (size_t)p.f.id(key, K - 1);
                float th = tri_hit(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2), rx, dir);
                pass = th > 0.0f && th < 1.0f;
            }
        }
        const unsigned m = __ballot_sync(full, pass);
        if (pass) {
            const int e = (head + count + __popc(m & lt)) % VQ;
            W.qc[e] = (uint32_t)c;
            W.qr[e] = (uint32_t)rxg;
            W.qt[e] = (uint32_t)t;
        }
        count += __popc(m);
        __syncwarp();
        if (count >= 32) {
            validate_batch<C, L>(p, sm, W, head, 32, cnt);
            head = (head + 32) % VQ;
            count -= 32;
            __syncwarp();
        }
    }
    if (count > 0) validate_batch<C, L>(p, sm, W, head, count, cnt);
    if (C) flush_counts(cnt, p.count - RT_CNT_PATHS, RT_CNT_ANY);
}

// offsets[p] = first path with pair >= p (paths sorted by pair, candidate)
__global__ void k_path_off(const uint64_t* __restrict__ pk, int64_t P, int64_t n_pairs,
                           int64_t* __restrict__ off) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q > n_pairs) return;
    int64_t lo = 0, hi = P;
    uint64_t want = (uint64_t)q << 32;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (pk[mid] < want) lo = mid + 1; else hi = mid;
    }
    off[q] = lo;
}

struct FinParams {
    DevScene s;
    KeyFmt f;
    const float* tx_pos;
    const float* rx_pos;
    const uint64_t* cand_key;
    const float* cand_img;
    const uint64_t* path_key;
    const int32_t* rx_off;
    int n_tx, n_rx;
    int64_t P;
    int32_t* seq;
    float* pts;
    int32_t* depth;
    double* len;
    int32_t* pair_tx;   // [P*2]: tx, rx
};

// Reflection points (FP32) and path length accumulated in FP64: the length
// of a specular path equals |rx - I_K| with I_K the last image of the
// transmitter, computed here with FP64 planes from the FP32 vertices.
__global__ void k_path_final(FinParams p) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.P) return;
    uint64_t pk = p.path_key[i];
    int64_t pair = (int64_t)(pk >> 32);
    int64_t c = (int64_t)(pk & 0xFFFFFFFFull);
    int t;
    int64_t rxg;
    if (p.rx_off) {
        int lo = 0, hi = p.n_tx;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (p.rx_off[mid] <= pair) lo = mid; else hi = mid;
        }
        t = lo;
        rxg = pair;
    } else {
        t = (int)(pair / p.n_rx);
        rxg = pair - (int64_t)t * p.n_rx;
    }
    uint64_t key = p.cand_key[c];
    int K = p.f.depth(key);
    f3 tx = mk(p.tx_pos[3 * t], p.tx_pos[3 * t + 1], p.tx_pos[3 * t + 2]);
    f3 rx = mk(p.rx_pos[3 * rxg], p.rx_pos[3 * rxg + 1], p.rx_pos[3 * rxg + 2]);
    f3 P[RT_MAX_DEPTH + 2];
    int ids[RT_MAX_DEPTH];
    back_project(p.s, p.f, key, K, p.cand_img + (size_t)c * p.f.D * 3, tx, rx, P, ids);
    for (int k = 0; k < p.f.D; k++) {
        p.seq[i * p.f.D + k] = k < K ? ids[k] : -1;
        f3 q = k < K ? P[k + 1] : mk(0.0f, 0.0f, 0.0f);
        p.pts[(i * p.f.D + k) * 3] = q.x;
        p.pts[(i * p.f.D + k) * 3 + 1] = q.y;
        p.pts[(i * p.f.D + k) * 3 + 2] = q.z;
    }
    p.depth[i] = K;
    p.pair_tx[2 * i] = t;
    p.pair_tx[2 * i + 1] = (int32_t)rxg;
    p.len[i] = path_length64(p.s, ids, K, tx, rx);
}

}  // namespace

// ----------------------------------------------------------------- host side
int launch_sbr(rt_ctx* ctx, int64_t N, int D, uint64_t* keys, uint32_t* vals, int32_t* hits);

static int key_format(rt_ctx* ctx, int D, KeyFmt& f) {
    int idb = 1;
    while ((1ll << idb) < (long long)std::max(ctx->n_tris, 2)) idb++;
    int txb = 0;
    while ((1ll << txb) < (long long)ctx->n_tx) txb++;
    int bits = txb + 3 + std::max(D, 1) * idb;
    if (bits > 64) return set_err(ctx, RT_ERR_INVALID_ARG, "candidate key wider than 64 bits (max_depth too large for this scene)");
    f.D = std::max(D, 1);
    f.id_bits = idb;
    f.depth_shift = f.D * idb;
    f.tx_shift = f.depth_shift + 3;
    ctx->id_bits = idb;
    ctx->tx_bits = txb;
    ctx->key_bits = bits;
    return RT_OK;
}

int compute_paths_impl(rt_ctx* ctx, int D, int64_t N, uint32_t flags, int64_t* out) {
    cudaStream_t st = ctx->stream;
    KeyFmt f;
    int e = key_format(ctx, D, f);
    if (e) return e;
    const bool los = flags & RT_LOS, refl = (flags & RT_REFLECTION) && D > 0 && N > 0;
    const int64_t nsbr = refl ? (int64_t)ctx->n_tx * N * D : 0;
    const int64_t ncap = nsbr + (los ? ctx->n_tx : 0);
    if (ncap >= 0xFFFFFFFFll) return set_err(ctx, RT_ERR_INVALID_ARG, "n_tx * num_rays * max_depth above 2^32");
    ctx->max_depth = f.D;
    ctx->num_rays = N;
    ctx->recorded_rays = refl && (flags & RT_RECORD_RAYS);
    RT_TRY(buf_reserve(ctx->keys, sizeof(uint64_t) * std::max<int64_t>(ncap, 1)));
    RT_TRY(buf_reserve(ctx->keys_alt, sizeof(uint64_t) * std::max<int64_t>(ncap, 1)));
    RT_TRY(buf_reserve(ctx->vals, sizeof(uint32_t) * std::max<int64_t>(ncap, 1)));
    RT_TRY(buf_reserve(ctx->vals_alt, sizeof(uint32_t) * std::max<int64_t>(ncap, 1)));
    uint64_t* keys = bp<uint64_t>(ctx->keys);
    uint32_t* vals = bp<uint32_t>(ctx->vals);
    RT_TRY(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), st));
    int64_t nhit = 0;  // candidate keys the rays produced (one per hit)
    bool fast = false;  // hash table sized from the previous call's key count
    if (refl) {
        int32_t* hits = nullptr;
        if (ctx->recorded_rays) {
            RT_TRY(buf_reserve(ctx->ray_hits, sizeof(int32_t) * nsbr));
            RT_TRY(cudaMemsetAsync(ctx->ray_hits.p, 0xFF, sizeof(int32_t) * nsbr, st));
            hits = bp<int32_t>(ctx->ray_hits);
        }
        e = launch_sbr(ctx, N, f.D, keys, vals, hits);
        if (e) return e;
        // a coverage map requested with RT_ASYNC_AFTER_TRACE starts here, so
        // that it shares the GPU with the refinement below, not with the trace
        e = side_launch(ctx);
        if (e) return e;
        // the key count is read here only when no earlier call sized the
        // hash table; otherwise it stays on the device until the hash pass
        fast = ctx->dedup == RT_DEDUP_HASH && ctx->key_bits < 64 && ctx->hash_hint > 0;
        if (!fast) {
            RT_TRY(cudaMemcpyAsync(ctx->host_rb, bp<unsigned long long>(ctx->counters) + RT_CNT_KEYS,
                                   sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            RT_TRY(cudaStreamSynchronize(st));
            nhit = (int64_t)ctx->host_rb[0];
        }
    }
    const int64_t extra = los ? ctx->n_tx : 0;
    const unsigned long long* nhit_dev = bp<unsigned long long>(ctx->counters) + RT_CNT_KEYS;
    int64_t nkeys = nhit + extra;   // with fast: known after the hash pass
    if (los) {
        prof_begin(ctx, "k_write_los");
        k_write_los<<<(ctx->n_tx + 255) / 256, 256, 0, st>>>(keys, vals, nhit, fast ? nhit_dev : nullptr, ctx->n_tx,
                                                            f);
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
    }
    RT_TRY(buf_reserve(ctx->cand_off, sizeof(int64_t) * (ctx->n_tx + 1)));
    const uint32_t* Ud = nullptr;   // device candidate count
    // hash table slots: a power of two, at least twice the keys
    auto slots_for = [](int64_t n) {
        int64_t S = 1024;
        while (S < 2 * n) S <<= 1;
        return S;
    };
    // beyond 2^29 slots (6 GB) the table would outgrow the sort's scratch: sort instead
    bool use_hash = ctx->key_bits < 64 && ctx->dedup == RT_DEDUP_HASH && (fast || slots_for(nkeys) <= (1ll << 29));
    if (use_hash) {
        DevBuf& cnt = ctx->htab_cnt;
        RT_TRY(buf_reserve(cnt, sizeof(uint32_t) * 4));
        uint32_t* cntp = bp<uint32_t>(cnt);   // [0] distinct keys, [1] overflow of a table sized beforehand
        int64_t U = 0;
        for (int pass = 0; pass < 2; pass++) {
            const int64_t S = fast ? ctx->hash_hint : slots_for(nkeys);
            const int64_t ucap = std::max<int64_t>(fast ? S / 2 : nkeys, 1);
            RT_TRY(buf_reserve(ctx->cand_key, sizeof(uint64_t) * ucap));
            RT_TRY(buf_reserve(ctx->cand_wit, sizeof(uint32_t) * ucap));
            RT_TRY(buf_reserve(ctx->cand_img, sizeof(float) * 3 * f.D * ucap));
            // duplicate removal by hashing, then a sort of the distinct keys only
            RT_TRY(buf_reserve(ctx->htab_key, sizeof(uint64_t) * S));
            RT_TRY(buf_reserve(ctx->htab_wit, sizeof(uint32_t) * S));
            RT_TRY(cudaMemsetAsync(ctx->htab_key.p, 0xFF, sizeof(uint64_t) * S, st));
            RT_TRY(cudaMemsetAsync(ctx->htab_wit.p, 0xFF, sizeof(uint32_t) * S, st));
            RT_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * 4, st));
            if (fast || nkeys > 0) {
                const int64_t span = fast ? S / 2 : nkeys;   // keys at most
                prof_begin(ctx, "k_hash_insert");
                k_hash_insert<<<(unsigned)std::min<int64_t>((span + 255) / 256, 8 * ctx->num_sms), 256, 0, st>>>(
                    keys, vals, fast ? extra : nkeys, fast ? nhit_dev : nullptr, S / 2, cntp + 1,
                    bp<unsigned long long>(ctx->htab_key), bp<unsigned>(ctx->htab_wit), (uint64_t)(S - 1));
                prof_end(ctx);
                RT_TRY(cudaGetLastError());
                prof_begin(ctx, "k_hash_compact");
                k_hash_compact<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(
                    bp<unsigned long long>(ctx->htab_key), bp<unsigned>(ctx->htab_wit), S,
                    bp<uint64_t>(ctx->cand_key), bp<uint32_t>(ctx->cand_wit), cntp);
                prof_end(ctx);
                RT_TRY(cudaGetLastError());
            }
            // one read: distinct keys and overflow, and the shooting pass's key count
            RT_TRY(cudaMemcpyAsync(ctx->host_rb, cntp, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            if (fast)
                RT_TRY(cudaMemcpyAsync(ctx->host_rb + 1, nhit_dev, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            RT_TRY(cudaStreamSynchronize(st));
            U = reinterpret_cast<uint32_t*>(ctx->host_rb)[0];
            const bool overflow = reinterpret_cast<uint32_t*>(ctx->host_rb)[1] != 0;
            if (fast) {
                nhit = (int64_t)ctx->host_rb[1];
                nkeys = nhit + extra;
                fast = false;
                if (overflow) {
                    // the table was too small: again, sized by the count just
                    // read (or by sorting, for a table beyond 2^29 slots)
                    use_hash = slots_for(nkeys) <= (1ll << 29);
                    if (use_hash) continue;
                }
            }
            break;
        }
        if (use_hash) {
            ctx->hash_hint = slots_for(nkeys);
            RT_TRY(radix_sort64(ctx, bp<uint64_t>(ctx->cand_key), bp<uint64_t>(ctx->keys_alt),
                                bp<uint32_t>(ctx->cand_wit), bp<uint32_t>(ctx->vals_alt), U, ctx->key_bits));
            Ud = cntp;
        }
    }
    if (!use_hash) {
        ctx->hash_hint = 0;
        const int64_t ucap = std::max<int64_t>(nkeys, 1);
        RT_TRY(buf_reserve(ctx->cand_key, sizeof(uint64_t) * ucap));
        RT_TRY(buf_reserve(ctx->cand_wit, sizeof(uint32_t) * ucap));
        RT_TRY(buf_reserve(ctx->cand_img, sizeof(float) * 3 * f.D * ucap));
        RT_TRY(radix_sort64(ctx, keys, bp<uint64_t>(ctx->keys_alt), vals, bp<uint32_t>(ctx->vals_alt), nkeys,
                            ctx->key_bits));
        // duplicate removal of the sorted keys
        DevBuf& cnt = ctx->sort_hist;
        const uint64_t sentinel_from = ~0ull;
        int nb = (int)std::max<int64_t>((nkeys + DD_TILE - 1) / DD_TILE, 1);
        RT_TRY(buf_reserve(cnt, sizeof(uint32_t) * (nb + 1)));
        uint32_t* cntp = bp<uint32_t>(cnt);
        RT_TRY(cudaMemsetAsync(cntp, 0, sizeof(uint32_t) * (nb + 1), st));
        if (nkeys > 0) {
            prof_begin(ctx, "k_dedup_count");
            k_dedup_count<<<nb, DD_THREADS, 0, st>>>(keys, nkeys, sentinel_from, cntp);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
        }
        RT_TRY(exclusive_scan_u32(ctx, cntp, nb + 1));
        Ud = cntp + nb;
        if (nkeys > 0) {
            prof_begin(ctx, "k_dedup_write");
            k_dedup_write<<<nb, DD_THREADS, 0, st>>>(keys, vals, nkeys, sentinel_from, cntp,
                                                     bp<uint64_t>(ctx->cand_key), bp<uint32_t>(ctx->cand_wit));
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
            prof_begin(ctx, "k_dedup_minwit");
            k_dedup_minwit<<<(unsigned)std::min<int64_t>((nkeys + 255) / 256, 8 * ctx->num_sms), 256, 0, st>>>(
                keys, vals, nkeys, bp<uint64_t>(ctx->cand_key), Ud, bp<unsigned>(ctx->cand_wit));
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
        }
    }
    if (nkeys > 0) {
        prof_begin(ctx, "k_cand_img");
        k_cand_img<<<(unsigned)std::min<int64_t>((nkeys + 255) / 256, 8 * ctx->num_sms), 256, 0, st>>>(
            bp<uint64_t>(ctx->cand_key), Ud, f, bp<float>(ctx->tx_pos), bp<float4>(ctx->planes),
            bp<float>(ctx->cand_img));
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
    }
    prof_begin(ctx, "k_cand_off");
    k_cand_off<<<(ctx->n_tx + 256) / 256, 256, 0, st>>>(bp<uint64_t>(ctx->cand_key), Ud, ctx->n_tx, f,
                                                         bp<int64_t>(ctx->cand_off));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    // validation work (sum over tx of U_t * R_t), offsets on the device
    int64_t n_pairs = ctx->rx_sets ? (int64_t)ctx->rx_off[ctx->n_tx] : (int64_t)ctx->n_tx * ctx->n_rx;
    DevBuf& woffd = ctx->path_cap_dummy;
    RT_TRY(buf_reserve(woffd, sizeof(int64_t) * (ctx->n_tx + 1)));
    prof_begin(ctx, "k_work_off");
    k_work_off<<<1, 1024, 0, st>>>(bp<int64_t>(ctx->cand_off), ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr,
                                   ctx->n_tx, ctx->n_rx, bp<int64_t>(woffd));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    if (ctx->path_cap == 0) ctx->path_cap = 1 << 16;
    int64_t P = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        RT_TRY(buf_reserve(ctx->path_key, sizeof(uint64_t) * ctx->path_cap));
        RT_TRY(buf_reserve(ctx->path_key_alt, sizeof(uint64_t) * ctx->path_cap));
        RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long) * 2, st));
        if (nkeys > 0 && n_pairs > 0) {
            ValParams vp;
            vp.s = dev_scene(ctx);
            vp.f = f;
            vp.tx_pos = bp<float>(ctx->tx_pos);
            vp.rx_pos = bp<float>(ctx->rx_pos);
            vp.cand_key = bp<uint64_t>(ctx->cand_key);
            vp.cand_img = bp<float>(ctx->cand_img);
            vp.cand_off = bp<int64_t>(ctx->cand_off);
            vp.work_off = bp<int64_t>(woffd);
            vp.rx_off = ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr;
            vp.n_tx = ctx->n_tx;
            vp.n_rx = ctx->n_rx;
            vp.out = bp<uint64_t>(ctx->path_key);
            vp.count = bp<unsigned long long>(ctx->counters) + 1;
            vp.cap = ctx->path_cap;
            vp.n_sm = staged_nodes(ctx);
            vp.status = bp<unsigned>(ctx->status);
            size_t smem = staged_bytes(ctx) + val_warp_bytes(f.D) * 8;
            auto kern = wide_layout(ctx) ? (ctx->count_work ? k_validate<true, 8> : k_validate<false, 8>)
                                         : (ctx->count_work ? k_validate<true, 2> : k_validate<false, 2>);
            RT_TRY(ensure_smem_attr((const void*)kern, smem));
            const int per_sm = blocks_per_sm((const void*)kern, 256, smem);
            // persistent grid: the work total is read on the device
            const int64_t units = nkeys * std::max<int64_t>((n_pairs / std::max(ctx->n_tx, 1) + 31) / 32, 1);
            const int64_t need = (units + 7) / 8;   // 8 warps per block
            const int64_t grid = std::max<int64_t>(std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * ctx->num_sms), 1);
            prof_begin(ctx, "k_validate");
            kern<<<(unsigned)grid, 256, smem, st>>>(vp);
            prof_end(ctx);
            RT_TRY(cudaGetLastError());
        }
        // one read: path count, candidate count, status
        RT_TRY(cudaMemcpyAsync(ctx->host_rb, bp<unsigned long long>(ctx->counters) + 1, sizeof(uint64_t),
                               cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaMemcpyAsync(reinterpret_cast<uint32_t*>(ctx->host_rb + 1), Ud, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaMemcpyAsync(reinterpret_cast<uint32_t*>(ctx->host_rb + 2), ctx->status.p, sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaStreamSynchronize(st));
        P = (int64_t)ctx->host_rb[0];
        ctx->n_cand = *reinterpret_cast<uint32_t*>(ctx->host_rb + 1);
        const unsigned hs = *reinterpret_cast<uint32_t*>(ctx->host_rb + 2);
        if (hs & RT_STAT_STACK) return set_err(ctx, RT_ERR_CAPACITY, "traversal stack overflow");
        if (hs & RT_STAT_LOOP) return set_err(ctx, RT_ERR_CUDA, "malformed BVH (traversal budget exceeded)");
        if (hs & RT_STAT_SORT) return set_err(ctx, RT_ERR_TIMEOUT, "radix sort: tile look-back timed out");
        if (P <= ctx->path_cap) break;
        ctx->path_cap = P + P / 4 + 1024;  // retry with room for every path
    }
    ctx->n_paths = P;
    int pair_bits = 1;
    while ((1ll << pair_bits) < std::max<int64_t>(n_pairs, 2)) pair_bits++;
    RT_TRY(radix_sort64(ctx, bp<uint64_t>(ctx->path_key), bp<uint64_t>(ctx->path_key_alt), nullptr, nullptr, P,
                        32 + pair_bits));
    RT_TRY(buf_reserve(ctx->path_off, sizeof(int64_t) * (n_pairs + 1)));
    prof_begin(ctx, "k_path_off");
    k_path_off<<<(unsigned)((n_pairs + 256) / 256), 256, 0, st>>>(bp<uint64_t>(ctx->path_key), P, n_pairs,
                                                                  bp<int64_t>(ctx->path_off));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    int64_t Pm = std::max<int64_t>(P, 1);
    RT_TRY(buf_reserve(ctx->path_seq, sizeof(int32_t) * Pm * f.D));
    RT_TRY(buf_reserve(ctx->path_pts, sizeof(float) * 3 * Pm * f.D));
    RT_TRY(buf_reserve(ctx->path_depth, sizeof(int32_t) * Pm));
    RT_TRY(buf_reserve(ctx->path_len, sizeof(double) * Pm));
    RT_TRY(buf_reserve(ctx->path_pair, sizeof(int32_t) * 2 * Pm));
    if (P > 0) {
        FinParams fp;
        fp.s = dev_scene(ctx);
        fp.f = f;
        fp.tx_pos = bp<float>(ctx->tx_pos);
        fp.rx_pos = bp<float>(ctx->rx_pos);
        fp.cand_key = bp<uint64_t>(ctx->cand_key);
        fp.cand_img = bp<float>(ctx->cand_img);
        fp.path_key = bp<uint64_t>(ctx->path_key);
        fp.rx_off = ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr;
        fp.n_tx = ctx->n_tx;
        fp.n_rx = ctx->n_rx;
        fp.P = P;
        fp.seq = bp<int32_t>(ctx->path_seq);
        fp.pts = bp<float>(ctx->path_pts);
        fp.depth = bp<int32_t>(ctx->path_depth);
        fp.len = bp<double>(ctx->path_len);
        fp.pair_tx = bp<int32_t>(ctx->path_pair);
        prof_begin(ctx, "k_path_final");
        k_path_final<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(fp);
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
    }
    *out = P;
    return RT_OK;
}

__global__ void k_cand_export(const uint64_t* __restrict__ ck, const uint32_t* __restrict__ wit, int64_t U,
                              KeyFmt f, int64_t N, int32_t* tx, int32_t* depth, int32_t* seq, int64_t* w) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= U) return;
    uint64_t k = ck[c];
    int K = f.depth(k);
    if (tx) tx[c] = f.tx(k);
    if (depth) depth[c] = K;
    if (seq)
        for (int b = 0; b < f.D; b++) seq[c * f.D + b] = b < K ? f.id(k, b) : -1;
    if (w) {
        uint32_t pos = wit[c];
        w[c] = pos == 0xFFFFFFFFu ? -1 : (int64_t)((pos / f.D) % N);
    }
}

int export_candidates(rt_ctx* ctx, int32_t* tx, int32_t* depth, int32_t* seq, int64_t* wit) {
    if (ctx->n_cand == 0) return RT_OK;
    KeyFmt f;
    f.D = ctx->max_depth;
    f.id_bits = ctx->id_bits;
    f.depth_shift = f.D * f.id_bits;
    f.tx_shift = f.depth_shift + 3;
    prof_begin(ctx, "k_cand_export");
    k_cand_export<<<(unsigned)((ctx->n_cand + 255) / 256), 256, 0, ctx->stream>>>(
        bp<uint64_t>(ctx->cand_key), bp<uint32_t>(ctx->cand_wit), ctx->n_cand, f, std::max<int64_t>(ctx->num_rays, 1),
        tx, depth, seq, wit);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}
