// rt_sort.cu -- stable sort of 64-bit keys (optional 32-bit payload) by
// their low end_bit bits (rounded up to whole bytes). Used for Morton codes,
// BVH level order, candidate keys (duplicate removal) and path keys. Three
// forms:
//   - up to 8192 keys: a stable rank sort (each key's position is the count
//     of smaller keys, ties by index), one launch, no digit passes;
//   - up to 2^30 keys: one histogram kernel for every digit position, then
//     one kernel per pass whose tiles find their global offsets by
//     decoupled look-back over the preceding tiles (Merrill & Garland's
//     single-pass prefix scan, as used by Adinets & Merrill's Onesweep);
//   - larger: per pass a histogram kernel, a multi-block scan over
//     (digit, tile) and a scatter kernel.
// The digit passes (LSD radix, 8-bit digits) rank keys stably with warp
// match/ballot.
#include <algorithm>

#include "rt_internal.h"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                      int shift, uint32_t* __restrict__ hist, int nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = lanemask_lt();
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * RS_THREADS + threadIdx.x;
        bool ok = i < n;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            // one shared atomic per distinct digit in the warp (keys are
            // often heavily repeated)
            unsigned dg = (unsigned)(keys[i] >> shift) & 255u;
            unsigned peers = __match_any_sync(act, dg);
            if ((peers & lt) == 0) atomicAdd(&h[dg], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const uint64_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint64_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout, int64_t n,
                                                         int shift, const uint32_t* __restrict__ off,
                                                         int nb) {
    __shared__ uint32_t cnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * 32 * RS_IPT;
    uint64_t k[RS_IPT];
    uint32_t v[RS_IPT];
    uint32_t rank[RS_IPT];
    const unsigned lt = lanemask_lt();
    // all loads first (independent), then the ranking
#pragma unroll
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        k[j] = i < n ? kin[i] : 0ull;
        if (VALS) v[j] = i < n ? vin[i] : 0u;
    }
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        bool ok = i < n;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            unsigned dg = (unsigned)(k[j] >> shift) & 255u;
            unsigned peers = __match_any_sync(act, dg);
            uint32_t before = cnt[w][dg];
            rank[j] = before + __popc(peers & lt);
            __syncwarp(act);
            if ((peers & lt) == 0) cnt[w][dg] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix across warps
    {
        int dg = threadIdx.x;
        uint32_t run = 0;
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t t = cnt[ww][dg];
            cnt[ww][dg] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        if (i < n) {
            unsigned dg = (unsigned)(k[j] >> shift) & 255u;
            uint32_t pos = off[(size_t)dg * nb + blockIdx.x] + cnt[w][dg] + rank[j];
            kout[pos] = k[j];
            if (VALS) vout[pos] = v[j];
        }
    }
}

// Multi-block exclusive scan: each block scans a tile of SC_TILE entries in
// place and writes the tile total; the totals are scanned recursively and
// added back.
constexpr int SC_THREADS = 1024, SC_IPT = 4, SC_TILE = SC_THREADS * SC_IPT;

__global__ void __launch_bounds__(SC_THREADS) k_scan_tile(uint32_t* __restrict__ a, int64_t m,
                                                          uint32_t* __restrict__ sums) {
    __shared__ uint32_t ws[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_IPT;
    uint32_t v[SC_IPT], s = 0;
#pragma unroll
    for (int i = 0; i < SC_IPT; i++) {
        v[i] = base + i < m ? a[base + i] : 0u;
        s += v[i];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    uint32_t run = x - s + (w > 0 ? ws[w - 1] : 0u);
#pragma unroll
    for (int i = 0; i < SC_IPT; i++) {
        if (base + i < m) a[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SC_THREADS - 1 && sums) sums[blockIdx.x] = ws[31];
}

__global__ void k_scan_add(uint32_t* __restrict__ a, int64_t m, const uint32_t* __restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] += offs[i / SC_TILE];
}

cudaError_t scan_level(rt_ctx* ctx, uint32_t* a, int64_t m, uint32_t* scratch) {
    int64_t nb = (m + SC_TILE - 1) / SC_TILE;
    prof_begin(ctx, "k_scan_tile");
    k_scan_tile<<<(unsigned)nb, SC_THREADS, 0, ctx->stream>>>(a, m, nb > 1 ? scratch : nullptr);
    prof_end(ctx);
    if (nb == 1) return cudaGetLastError();
    cudaError_t e = scan_level(ctx, scratch, nb, scratch + nb);
    if (e != cudaSuccess) return e;
    prof_begin(ctx, "k_scan_add");
    k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(a, m, scratch);
    prof_end(ctx);
    return cudaGetLastError();
}

// ------------------------------------------------------------- one sweep
// Digit histograms of every pass in one read of the keys: hist [passes x 256].
__global__ void __launch_bounds__(RS_THREADS) os_hist(const uint64_t* __restrict__ keys, int64_t n, int passes,
                                                      uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = lanemask_lt();
    for (int64_t i0 = (int64_t)blockIdx.x * RS_TILE; i0 < n; i0 += (int64_t)gridDim.x * RS_TILE) {
        for (int j = 0; j < RS_IPT; j++) {
            int64_t i = i0 + j * RS_THREADS + threadIdx.x;
            bool ok = i < n;
            unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const uint64_t k = keys[i];
                for (int p = 0; p < passes; p++) {
                    unsigned dg = (unsigned)(k >> (8 * p)) & 255u;
                    unsigned peers = __match_any_sync(act, dg);
                    if ((peers & lt) == 0) atomicAdd(&h[p][dg], (uint32_t)__popc(peers));
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += RS_THREADS) {
        uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(hist + i, v);
    }
}

// Tile status word: bits 31..30 = 0 not yet published, 1 tile count only,
// 2 inclusive prefix through this tile; bits 29..0 = the count.
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_VAL = (1u << 30) - 1u;
constexpr int OS_SPIN_MAX = 1 << 22;   // polls per predecessor before giving up

template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS) os_scatter(const uint64_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         int64_t n, int shift, const uint32_t* __restrict__ hist,
                                                         uint32_t* status, unsigned* tile_ctr, unsigned* err) {
    __shared__ uint32_t cnt[RS_WARPS][256];
    __shared__ uint32_t s_off[256];
    __shared__ unsigned s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, d = threadIdx.x;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);   // tiles in start order: no deadlock
    __syncthreads();
    const unsigned tile = s_tile;
    const int64_t base = (int64_t)tile * RS_TILE + (int64_t)w * 32 * RS_IPT;
    uint64_t k[RS_IPT];
    uint32_t v[RS_IPT];
    uint32_t rank[RS_IPT];
    const unsigned lt = lanemask_lt();
    // all loads first (independent), then the ranking
#pragma unroll
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        k[j] = i < n ? kin[i] : 0ull;
        if (VALS) v[j] = i < n ? vin[i] : 0u;
    }
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        bool ok = i < n;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            unsigned dg = (unsigned)(k[j] >> shift) & 255u;
            unsigned peers = __match_any_sync(act, dg);
            uint32_t before = cnt[w][dg];
            rank[j] = before + __popc(peers & lt);
            __syncwarp(act);
            if ((peers & lt) == 0) cnt[w][dg] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix across this tile's warps, tile total
    uint32_t run = 0;
    for (int ww = 0; ww < RS_WARPS; ww++) {
        uint32_t t = cnt[ww][d];
        cnt[ww][d] = run;
        run += t;
    }
    // exclusive digit base of this pass (scan of the 256 totals)
    uint32_t tot = hist[d], x = tot;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    s_off[d] = x;   // inclusive within the warp
    __syncthreads();
    uint32_t wsum = 0;
    for (int ww = 0; ww < w; ww++) wsum += s_off[ww * 32 + 31];
    const uint32_t digit_base = wsum + x - tot;
    // publish this tile's count, look back over the preceding tiles, publish the prefix
    volatile uint32_t* st = status;
    uint32_t excl = 0;
    if (tile == 0) {
        st[d] = OS_INC | run;
    } else {
        st[(size_t)tile * 256 + d] = OS_AGG | run;
        int64_t p = (int64_t)tile - 1;
        int spins = 0;
        while (p >= 0) {
            uint32_t s = st[(size_t)p * 256 + d];
            if ((s & ~OS_VAL) == 0) {
                if (++spins > OS_SPIN_MAX) {   // a predecessor never published: give up, flag it
                    atomicOr(err, RT_STAT_SORT);
                    break;
                }
                __nanosleep(64);
                continue;
            }
            spins = 0;
            excl += s & OS_VAL;
            if (s & OS_INC) break;
            p--;
        }
        st[(size_t)tile * 256 + d] = OS_INC | ((excl + run) & OS_VAL);
    }
    __syncthreads();   // s_off reads above are done
    s_off[d] = digit_base + excl;
    __syncthreads();
    for (int j = 0; j < RS_IPT; j++) {
        int64_t i = base + j * 32 + lane;
        if (i < n) {
            unsigned dg = (unsigned)(k[j] >> shift) & 255u;
            uint32_t pos = s_off[dg] + cnt[w][dg] + rank[j];
            kout[pos] = k[j];
            if (VALS) vout[pos] = v[j];
        }
    }
}

constexpr int RK_MAX = 256;   // up to this many keys: one-block rank sort

// Tiny inputs (<= RK_MAX keys, one per thread): every key's output position
// is the number of keys that are smaller, or equal with a smaller index
// (stable); one shared-memory pass, no digit passes. Only the low end_bit
// bits of the keys take part, as in the radix passes.
template <bool VALS>
__global__ void __launch_bounds__(RK_MAX) k_sort_rank(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, int n,
                                                     uint64_t mask) {
    __shared__ uint64_t sk[RK_MAX];
    const int i = threadIdx.x;
    uint64_t k = 0;
    uint32_t v = 0;
    if (i < n) {
        k = keys[i];
        if (VALS) v = vals[i];
        sk[i] = k & mask;
    }
    __syncthreads();
    int r = 0;
    if (i < n) {
        const uint64_t km = k & mask;
        for (int j = 0; j < n; j++) {
            const uint64_t o = sk[j];
            r += (o < km) | ((o == km) & (j < i));
        }
    }
    __syncthreads();   // every key has been read before the in-place writes
    if (i < n) {
        keys[r] = k;
        if (VALS) vals[r] = v;
    }
}

// Small inputs (RK_MAX < n <= RK_MULTI_MAX): the same stable rank sort
// spread over the GPU. Every block stages all n (masked) keys in shared
// memory and ranks 32 of them (one per lane); its 32 warps count the smaller
// keys in 32 segments of the input (all lanes read the same key at a time:
// broadcast), and the segment counts are summed in shared memory. When the
// masked keys leave 13 bits free, a key's index is appended below it, which
// makes all keys distinct and the stable rank one comparison per pair.
// O(n^2) comparisons, but one launch and no digit passes.
constexpr int RK_MULTI_MAX = 8192;   // index fits in 13 bits
constexpr int RK_IDX_BITS = 13;

template <bool VALS, bool COMP>
__global__ void __launch_bounds__(1024) k_sort_rank_multi(const uint64_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ vals,
                                                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                          int n, uint64_t mask) {
    extern __shared__ uint64_t sk[];   // [n]
    __shared__ int part[32][33];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const uint64_t o = __ldg(keys + j) & mask;
        sk[j] = COMP ? ((o << RK_IDX_BITS) | (uint64_t)j) : o;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const uint64_t km = sk[min(i, n - 1)];
    const int seg = (n + 31) / 32;
    const int j0 = min(w * seg, n), j1 = min(j0 + seg, n);
    int r = 0;
    if (COMP) {
#pragma unroll 8
        for (int j = j0; j < j1; j++) r += sk[j] < km;
    } else {
#pragma unroll 4
        for (int j = j0; j < j1; j++) {
            const uint64_t o = sk[j];
            r += (o < km) | ((o == km) & (j < i));
        }
    }
    part[w][lane] = r;
    __syncthreads();
    if (w == 0 && i < n) {
        int rr = 0;
#pragma unroll
        for (int q = 0; q < 32; q++) rr += part[q][lane];
        kout[rr] = keys[i];
        if (VALS) vout[rr] = vals[i];
    }
}

}  // namespace

cudaError_t radix_sort64(rt_ctx* ctx, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                         uint32_t* vals_alt, int64_t n, int end_bit) {
    if (n <= 1 || end_bit <= 0) return cudaSuccess;
    if (n > (int64_t)0xFFFFFFFFll) return cudaErrorInvalidValue;
    if (n <= RK_MAX) {
        const int bits = 8 * ((end_bit + 7) / 8);   // the bits the digit passes would order by
        const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
        const int threads = 32 * (int)((n + 31) / 32);
        prof_begin(ctx, "k_sort_rank");
        if (vals)
            k_sort_rank<true><<<1, threads, 0, ctx->stream>>>(keys, vals, (int)n, mask);
        else
            k_sort_rank<false><<<1, threads, 0, ctx->stream>>>(keys, nullptr, (int)n, mask);
        prof_end(ctx);
        return cudaGetLastError();
    }
    if (n <= RK_MULTI_MAX) {
        const int bits = 8 * ((end_bit + 7) / 8);
        const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
        const bool comp = bits + RK_IDX_BITS <= 64;
        const unsigned blocks = (unsigned)((n + 31) / 32);
        const size_t smem = sizeof(uint64_t) * (size_t)n;
        const void* fn = comp ? (vals ? (const void*)k_sort_rank_multi<true, true> : (const void*)k_sort_rank_multi<false, true>)
                              : (vals ? (const void*)k_sort_rank_multi<true, false> : (const void*)k_sort_rank_multi<false, false>);
        cudaError_t e = ensure_smem_attr(fn, smem);
        if (e != cudaSuccess) return e;
        prof_begin(ctx, "k_sort_rank_multi");
        if (comp && vals)
            k_sort_rank_multi<true, true><<<blocks, 1024, smem, ctx->stream>>>(keys, vals, keys_alt, vals_alt, (int)n, mask);
        else if (comp)
            k_sort_rank_multi<false, true><<<blocks, 1024, smem, ctx->stream>>>(keys, nullptr, keys_alt, nullptr, (int)n, mask);
        else if (vals)
            k_sort_rank_multi<true, false><<<blocks, 1024, smem, ctx->stream>>>(keys, vals, keys_alt, vals_alt, (int)n, mask);
        else
            k_sort_rank_multi<false, false><<<blocks, 1024, smem, ctx->stream>>>(keys, nullptr, keys_alt, nullptr, (int)n, mask);
        prof_end(ctx);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(keys, keys_alt, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess && vals)
            e = cudaMemcpyAsync(vals, vals_alt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
        return e;
    }
    int nb = (int)((n + RS_TILE - 1) / RS_TILE);
    const int passes_all = (end_bit + 7) / 8;
    if (n < (int64_t)OS_VAL && passes_all <= 8) {
        // scratch: [passes x 256] histograms, [passes] tile counters, error word,
        // [passes x nb x 256] tile status words; zeroed with one memset
        const size_t words = (size_t)passes_all * 256 + 16 + (size_t)passes_all * nb * 256;
        cudaError_t e = buf_reserve(ctx->sort_hist, sizeof(uint32_t) * words);
        if (e != cudaSuccess) return e;
        uint32_t* hist = bp<uint32_t>(ctx->sort_hist);
        unsigned* ctr = hist + passes_all * 256;
        unsigned* err = bp<unsigned>(ctx->status);   // RT_STAT_SORT if a look-back gave up
        uint32_t* status = ctr + 16;
        e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * words, ctx->stream);
        if (e != cudaSuccess) return e;
        prof_begin(ctx, "os_hist");
        os_hist<<<std::min(nb, 4 * ctx->num_sms), RS_THREADS, 0, ctx->stream>>>(keys, n, passes_all, hist);
        prof_end(ctx);
        uint64_t *kin = keys, *kout = keys_alt;
        uint32_t *vin = vals, *vout = vals_alt;
        for (int p = 0; p < passes_all; p++) {
            prof_begin(ctx, "os_scatter");
            uint32_t* stp = status + (size_t)p * nb * 256;
            if (vals)
                os_scatter<true><<<nb, RS_THREADS, 0, ctx->stream>>>(kin, vin, kout, vout, n, 8 * p, hist + 256 * p,
                                                                      stp, ctr + p, err);
            else
                os_scatter<false><<<nb, RS_THREADS, 0, ctx->stream>>>(kin, nullptr, kout, nullptr, n, 8 * p,
                                                                       hist + 256 * p, stp, ctr + p, err);
            prof_end(ctx);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        if (kin != keys) {
            e = cudaMemcpyAsync(keys, kin, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) return e;
            if (vals) e = cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
        }
        return e;
    }
    cudaError_t e = buf_reserve(ctx->sort_hist, sizeof(uint32_t) * 256 * (size_t)nb);
    if (e != cudaSuccess) return e;
    uint32_t* hist = bp<uint32_t>(ctx->sort_hist);
    uint64_t *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    int passes = (end_bit + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        prof_begin(ctx, "rs_hist");
        rs_hist<<<nb, RS_THREADS, 0, ctx->stream>>>(kin, n, shift, hist, nb);
        prof_end(ctx);
        e = exclusive_scan_u32(ctx, hist, (int64_t)256 * nb);
        if (e != cudaSuccess) return e;
        prof_begin(ctx, "rs_scatter");
        if (vals)
            rs_scatter<true><<<nb, RS_THREADS, 0, ctx->stream>>>(kin, vin, kout, vout, n, shift, hist, nb);
        else
            rs_scatter<false><<<nb, RS_THREADS, 0, ctx->stream>>>(kin, nullptr, kout, nullptr, n, shift, hist, nb);
        prof_end(ctx);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {
        e = cudaMemcpyAsync(keys, kin, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) return e;
        if (vals) e = cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    return e;
}

// Exclusive scan of m uint32 entries in place.
cudaError_t exclusive_scan_u32(rt_ctx* ctx, uint32_t* a, int64_t m) {
    if (m <= 0) return cudaSuccess;
    size_t need = 0;
    for (int64_t k = (m + SC_TILE - 1) / SC_TILE; k > 1; k = (k + SC_TILE - 1) / SC_TILE) need += k;
    cudaError_t e = buf_reserve(ctx->scan_buf, sizeof(uint32_t) * (need + 16));
    if (e != cudaSuccess) return e;
    return scan_level(ctx, a, m, bp<uint32_t>(ctx->scan_buf));
}
