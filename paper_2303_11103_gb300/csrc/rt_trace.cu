// rt_trace.cu -- ray shooting: direction-coherent ray order, shooting and
// bouncing of candidate paths (Sec. II-B), coverage-map ray tracing with
// field transport and binning (Sec. II-A, Fig. 2).
//
// Both tracing kernels are persistent: a grid of (SMs x resident blocks)
// warps pulls chunks of rays from one global counter that spans every
// transmitter, so all transmitters run in one launch. Each lane holds one
// ray in registers; when lanes' rays terminate, the warp refills exactly
// those lanes (ballot over dead lanes, popc ranks) from its chunk, so the
// warp keeps tracing with all lanes live between bounces. The top BVH
// levels are staged in shared memory once per block.
#include "rt_field.cuh"
#include "rt_internal.h"

namespace {

// -------------------------------------------------------------- ray ordering
// Key = 2D Morton code of (z, phi) of the lattice direction quantised to
// 2^12 x 2^12 cells: rays whose order is close point in close directions.
__global__ void k_perm_keys(long long N, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    f3 d = fib_dir(N, i);
    float u = fminf(fmaxf((d.z + 1.0f) * 0.5f, 0.0f), 0.99999f);
    float v = (atan2f(d.y, d.x) + RT_PI_F) * (0.5f / RT_PI_F);
    v = fminf(fmaxf(v, 0.0f), 0.99999f);
    unsigned a = (unsigned)(u * 4096.0f), b = (unsigned)(v * 4096.0f);
    unsigned long long code = 0;
    for (int k = 0; k < 12; k++) code |= (unsigned long long)(((a >> k) & 1u) << (2 * k + 1)) |
                                        (unsigned long long)(((b >> k) & 1u) << (2 * k));
    keys[i] = code;
    vals[i] = (uint32_t)i;
}

// Direction table in trace order: (fib_dir(N, perm[k]), perm[k]).
__global__ void k_dir_table(long long N, const uint32_t* __restrict__ perm, float4* __restrict__ dirs) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const uint32_t i = perm[k];
    f3 d = fib_dir(N, (long long)i);
    dirs[k] = make_float4(d.x, d.y, d.z, __uint_as_float(i));
}

struct TraceCommon {
    DevScene s;
    const float* tx_pos;  // [n_tx*3]
    const float* tx_ypr;  // [n_tx*3]
    long long N;          // lattice size (rays per transmitter)
    long long first;      // first lattice index traced
    long long count;      // lattice indices traced per transmitter
    long long total;      // n_tx * count
    const uint32_t* perm; // [N] direction-coherent order (full range only) or null
    const float4* dirs;   // [N] with perm: (direction of lattice ray perm[k], perm[k] as bits), or null
    unsigned long long* counter;
    int chunk;            // rays per warp refill
    int quota;            // refills per warp before it stops (0: until the rays run out)
    int n_sm;             // staged BVH nodes
    unsigned* status;
};

__device__ __forceinline__ void stage_nodes(const TraceCommon& c, float4* sm) {
    const float4* src = node_base(c.s);
    for (int i = threadIdx.x; i < c.n_sm * node_f4(c.s); i += blockDim.x) sm[i] = src[i];
    __syncthreads();
}

// Warp-level ray fetch: refill dead lanes from the warp's chunk. Returns the
// global ray slot (tx * N + lattice index) for a refilled lane, -1 otherwise.
struct WarpFeed {
    long long next = 0, end = 0;
    int fetched = 0;
    bool exhausted = false;
    // k_out receives the ray's index in the trace order (its slot in c.dirs).
    __device__ __forceinline__ long long refill(const TraceCommon& c, bool alive, long long& k_out) {
        const unsigned full = 0xffffffffu;
        unsigned dead = __ballot_sync(full, !alive);
        long long slot = -1;
        if (dead == 0 || exhausted) return slot;
        if (next >= end) {
            // a warp with a refill quota stops after it (its block then ends
            // and frees its SM slot for other work)
            if (c.quota > 0 && fetched >= c.quota) {
                exhausted = true;
                return slot;
            }
            fetched++;
            unsigned long long base = 0;
            if ((threadIdx.x & 31) == 0) base = atomicAdd(c.counter, (unsigned long long)c.chunk);
            base = __shfl_sync(full, base, 0);
            if ((long long)base >= c.total) {
                exhausted = true;
                return slot;
            }
            next = (long long)base;
            end = min((long long)base + c.chunk, c.total);
        }
        int need = __popc(dead);
        int take = (int)min((long long)need, end - next);
        int r = __popc(dead & lanemask_lt());
        if (!alive && r < take) {
            long long q = next + r;
            long long tx = q / c.count, k = q - tx * c.count;
            long long i = c.perm ? (long long)c.perm[k] : c.first + k;
            slot = tx * c.N + i;
            k_out = k;
        }
        next += take;
        return slot;
    }
};

// Direction of lattice ray i (trace-order index k): from the context's table
// when it has one (the FP64 lattice rounded to FP32 once, when the ray order
// was built), else computed here.
__device__ __forceinline__ f3 ray_dir(const TraceCommon& c, long long k, long long i) {
    return c.dirs ? xyz(__ldg(c.dirs + k)) : fib_dir(c.N, i);
}

// ------------------------------------------------------------ SBR candidates
struct SbrParams {
    TraceCommon c;
    int D;
    int id_bits, depth_shift, tx_shift;
    uint64_t* keys;                // compacted candidate keys (capacity total*D)
    uint32_t* vals;                // their (ray slot * D + depth) positions
    unsigned long long* n_keys;    // append counter
    int32_t* hits;                 // [total*D] or null
};

template <bool C, int L>
__global__ void __launch_bounds__(256) k_sbr(SbrParams p) {
    extern __shared__ float4 sm[];
    stage_nodes(p.c, sm);
    WarpFeed feed;
    bool alive = false;
    f3 o = mk(0, 0, 0), d = mk(0, 0, 1);
    int last = -1, depth = 0;
    long long slot = 0;
    uint64_t key = 0;
    TravCount cnt;
    while (true) {
        long long kd = 0;
        long long s = feed.refill(p.c, alive, kd);
        if (s >= 0) {
            slot = s;
            long long tx = s / p.c.N, i = s - tx * p.c.N;
            o = mk(p.c.tx_pos[3 * tx], p.c.tx_pos[3 * tx + 1], p.c.tx_pos[3 * tx + 2]);
            d = ray_dir(p.c, kd, i);
            last = -1;
            depth = 0;
            key = (uint64_t)tx << p.tx_shift;
            alive = true;
        }
        if (!__any_sync(0xffffffffu, alive)) {
            if (feed.exhausted) break;
            continue;
        }
        bool emit = false;
        uint64_t ekey = 0;
        uint32_t epos = 0;
        if (alive) {
            float t;
            int id = closest_hit<C, L, false>(p.c.s, sm, p.c.n_sm, o, d, last, t, cnt);
            if (id < 0) {
                alive = false;
            } else {
                key |= (uint64_t)id << ((p.D - 1 - depth) * p.id_bits);
                size_t pos = (size_t)slot * p.D + depth;
                ekey = key | ((uint64_t)(depth + 1) << p.depth_shift);
                epos = (uint32_t)pos;
                emit = true;
                if (p.hits) p.hits[pos] = id;
                float4 pl = __ldg(p.c.s.planes + id);
                o = o + d * t;
                d = reflect(d, xyz(pl));
                last = id;
                if (++depth >= p.D) alive = false;
            }
        }
        // append this bounce's candidate keys: equal keys within the warp
        // are appended once, by the lowest lane, with the smallest position
        // of the group (so the smallest over all appends is the smallest
        // producing ray, whichever rays the warps held together); one atomic
        // per warp, ballot ranks
        const unsigned em = __ballot_sync(0xffffffffu, emit);
        if (em) {
            const int lane = threadIdx.x & 31;
            bool keep = false;
            if (emit) {
                const unsigned grp = __match_any_sync(em, (unsigned long long)ekey);
                epos = __reduce_min_sync(grp, epos);
                keep = (grp & lanemask_lt()) == 0;
            }
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            const int leader = __ffs(km) - 1;
            unsigned long long b0 = 0;
            if (lane == leader) b0 = atomicAdd(p.n_keys, (unsigned long long)__popc(km));
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (keep) {
                unsigned long long k = b0 + __popc(km & lanemask_lt());
                p.keys[k] = ekey;
                p.vals[k] = epos;
            }
        }
    }
    if (C) flush_counts(cnt, p.c.counter, RT_CNT_CLOSEST);
}

// ------------------------------------------------------------- coverage map
struct CovParams {
    TraceCommon c;
    int D;
    DevAntenna txa, rxa;
    int tx_port;
    float inv_we0;
    float x0, y0, inv_cell, h;
    int nx, ny;
    float wscale;          // lambda^2 / (4 pi cell^2 N)
    float* gain;           // [n_tx*ny*nx]
    uint32_t* hits;        // [n_tx*ny*nx]
};

// The map cell where the ray o + t d (t > 0) crosses the plane z = h, or -1
// when it does not cross it inside the grid; sc receives the distance.
__device__ __forceinline__ long long plane_cell(const CovParams& p, int tx, f3 o, f3 d, float& sc) {
    sc = 0.0f;
    if (d.z == 0.0f) return -1;
    sc = (p.h - o.z) / d.z;
    if (!(sc > 0.0f)) return -1;
    const float fx = (o.x + sc * d.x - p.x0) * p.inv_cell;
    const float fy = (o.y + sc * d.y - p.y0) * p.inv_cell;
    const int ix = (int)floorf(fx), iy = (int)floorf(fy);
    if (!(fx >= 0.0f && fy >= 0.0f && ix < p.nx && iy < p.ny)) return -1;
    return ((long long)tx * p.ny + iy) * p.nx + ix;
}

// One segment of a coverage ray from o along d, leaving triangle `last`.
// Returns the map cell the segment adds to (-1: none). While the ray
// reflects again (more), the closest hit gives the next triangle (id, t)
// and the crossing counts when it comes before that hit. The last segment
// reflects no further, so its closest hit is not needed: an any-hit test of
// the segment up to the crossing decides, and it is taken only when the
// crossing lies in the grid. Both forms count the crossing exactly when no
// triangle other than `last` is hit at a distance in (tmin, sc] (tri_hit
// gives both the same distances). Last-segment tests are counted in cnt_pl.
template <bool C, int L>
__device__ __forceinline__ long long cov_segment(const CovParams& p, const float4* sm, int tx, f3 o, f3 d,
                                                 int last, bool more, int& id, float& t, TravCount& cnt,
                                                 TravCount& cnt_pl) {
    float sc;
    id = -1;
    t = __int_as_float(0x7f800000);
    if (more) {
        id = closest_hit<C, L>(p.c.s, sm, p.c.n_sm, o, d, last, t, cnt);
        const long long cell = plane_cell(p, tx, o, d, sc);
        return (cell >= 0 && (id < 0 || sc < t)) ? cell : -1;
    }
    const long long cell = plane_cell(p, tx, o, d, sc);
    if (cell < 0) return -1;
    // t <= sc  <=>  t < the next float above sc (sc is finite here)
    const float up = nextafterf(sc, __int_as_float(0x7f800000));
    return any_hit<C, L>(p.c.s, sm, p.c.n_sm, o, d, up, last, last, cnt_pl) ? -1 : cell;
}

// Transmitter rotations a coverage block keeps in shared memory (more
// transmitters: computed per ray).
#define RT_ROT_CACHE 64

template <bool C, int L>
__global__ void __launch_bounds__(256) k_coverage(CovParams p) {
    extern __shared__ float4 sm[];
    // each transmitter's rotation once per block instead of once per ray
    // (the same function, so the same values)
    __shared__ float s_rot[RT_ROT_CACHE * 9];
    const long long n_tx = p.c.total / (p.c.count > 0 ? p.c.count : 1);
    const bool rot_cached = n_tx <= RT_ROT_CACHE;
    if (rot_cached) {
        for (int k = threadIdx.x; k < (int)n_tx; k += blockDim.x) {
            const Rot<float> R = rot_ypr(p.c.tx_ypr[3 * k], p.c.tx_ypr[3 * k + 1], p.c.tx_ypr[3 * k + 2]);
            for (int q = 0; q < 9; q++) s_rot[9 * k + q] = R.m[q / 3][q % 3];
        }
    }
    stage_nodes(p.c, sm);   // ends with a block barrier
    WarpFeed feed;
    bool alive = false;
    f3 o = mk(0, 0, 0), d = mk(0, 0, 1);
    int last = -1, depth = 0, tx = 0;
    Cx<float> E[3];
    const float zeta_t = p.txa.slant[p.tx_port], zeta_r = p.rxa.slant[0];
    Rot<float> Rr = rot_ypr(0.0f, 0.0f, 0.0f);
    TravCount cnt, cnt_pl;
    while (true) {
        long long kd = 0;
        long long s = feed.refill(p.c, alive, kd);
        if (s >= 0) {
            long long t64 = s / p.c.N, i = s - t64 * p.c.N;
            tx = (int)t64;
            o = mk(p.c.tx_pos[3 * tx], p.c.tx_pos[3 * tx + 1], p.c.tx_pos[3 * tx + 2]);
            d = ray_dir(p.c, kd, i);
            Rot<float> Rt;
            if (rot_cached) {
                for (int q = 0; q < 9; q++) Rt.m[q / 3][q % 3] = s_rot[9 * tx + q];
            } else {
                Rt = rot_ypr(p.c.tx_ypr[3 * tx], p.c.tx_ypr[3 * tx + 1], p.c.tx_ypr[3 * tx + 2]);
            }
            V3<float> f = antenna_vec<float>(p.txa.kind, zeta_t, Rt, V3<float>{d.x, d.y, d.z});
            E[0] = {f.x, 0.0f};
            E[1] = {f.y, 0.0f};
            E[2] = {f.z, 0.0f};
            last = -1;
            depth = 0;
            alive = true;
        }
        if (!__any_sync(0xffffffffu, alive)) {
            if (feed.exhausted) break;
            continue;
        }
        if (alive) {
            float t;
            int id;
            const bool more = depth < p.D;
            const long long cell = cov_segment<C, L>(p, sm, tx, o, d, last, more, id, t, cnt, cnt_pl);
            if (cell >= 0) {
                V3<float> F = antenna_vec<float>(p.rxa.kind, zeta_r, Rr, V3<float>{-d.x, -d.y, -d.z});
                float re = F.x * E[0].re + F.y * E[1].re + F.z * E[2].re;
                float im = F.x * E[0].im + F.y * E[1].im + F.z * E[2].im;
                float w = (re * re + im * im) * p.wscale / fabsf(d.z);
                atomicAdd(p.gain + cell, w);
                atomicAdd(p.hits + cell, 1u);
            }
            if (id < 0 || !more) {
                alive = false;
            } else {
                float4 pl = __ldg(p.c.s.planes + id);
                int m = __ldg(p.c.s.mat + id);
                float2 mp = __ldg(p.c.s.mats + m);
                f3 n = xyz(pl);
                f3 r = reflect(d, n);
                reflect_field<float>(E, V3<float>{d.x, d.y, d.z}, V3<float>{r.x, r.y, r.z}, n, mp.x, mp.y,
                                     p.inv_we0);
                o = o + d * t;
                d = r;
                last = id;
                depth++;
            }
        }
    }
    if (C) {
        flush_counts(cnt, p.c.counter, RT_CNT_CLOSEST);
        flush_counts(cnt_pl, p.c.counter, RT_CNT_PLANE);
    }
}

// VJP of the coverage map with respect to the transmitters' orientation
// (yaw, pitch, roll): the rays are traced again exactly as in k_coverage
// (the geometry does not depend on the orientation), the field is carried
// as Dual<3> seeded by the transmit pattern at R(yaw, pitch, roll), and every
// crossing of the plane adds g[cell] * d w / d(yaw, pitch, roll) to the
// lane's accumulators, flushed per transmitter (warp-reduced when the warp
// shares one). Sec. III-B optimises an orientation with this gradient.
struct CovVjpParams {
    CovParams p;
    const float* grad_gain;   // [n_tx*ny*nx] upstream gradient of the gain map
    float* grad_ypr;          // [n_tx*3], accumulated
};

__device__ __forceinline__ void flush_ypr(float* g, int tx, float (&acc)[3]) {
    const unsigned full = 0xffffffffu;
    const int t0 = __shfl_sync(full, tx, 0);
    if (__all_sync(full, tx == t0)) {
        for (int k = 0; k < 3; k++) {
            float v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
            if ((threadIdx.x & 31) == 0 && t0 >= 0 && v != 0.0f) atomicAdd(g + 3 * t0 + k, v);
        }
    } else if (tx >= 0) {
        for (int k = 0; k < 3; k++)
            if (acc[k] != 0.0f) atomicAdd(g + 3 * tx + k, acc[k]);
    }
    acc[0] = acc[1] = acc[2] = 0.0f;
}

template <int L>
__global__ void __launch_bounds__(256) k_coverage_vjp(CovVjpParams q) {
    extern __shared__ float4 sm[];
    const CovParams& p = q.p;
    stage_nodes(p.c, sm);
    typedef Dual<3> D3;
    WarpFeed feed;
    bool alive = false;
    f3 o = mk(0, 0, 0), d = mk(0, 0, 1);
    int last = -1, depth = 0, tx = -1;
    Cx<D3> E[3];
    float acc[3] = {0.0f, 0.0f, 0.0f};
    const float zeta_t = p.txa.slant[p.tx_port], zeta_r = p.rxa.slant[0];
    Rot<float> Rr = rot_ypr(0.0f, 0.0f, 0.0f);
    TravCount cnt;
    while (true) {
        long long kd = 0;
        long long s = feed.refill(p.c, alive, kd);
        // a lane moving to another transmitter flushes its accumulators first
        const int next_tx = s >= 0 ? (int)(s / p.c.N) : tx;
        if (__any_sync(0xffffffffu, next_tx != tx && tx >= 0)) {
            int ftx = (next_tx != tx) ? tx : -1;
            float keep[3] = {acc[0], acc[1], acc[2]};
            if (ftx < 0) acc[0] = acc[1] = acc[2] = 0.0f;
            flush_ypr(q.grad_ypr, ftx, acc);
            if (ftx < 0) { acc[0] = keep[0]; acc[1] = keep[1]; acc[2] = keep[2]; }
        }
        if (s >= 0) {
            long long i = s - (long long)next_tx * p.c.N;
            tx = next_tx;
            o = mk(p.c.tx_pos[3 * tx], p.c.tx_pos[3 * tx + 1], p.c.tx_pos[3 * tx + 2]);
            d = ray_dir(p.c, kd, i);
            D3 yaw = dconst<3>(p.c.tx_ypr[3 * tx]), pitch = dconst<3>(p.c.tx_ypr[3 * tx + 1]),
               roll = dconst<3>(p.c.tx_ypr[3 * tx + 2]);
            yaw.d[0] = 1.0f;
            pitch.d[1] = 1.0f;
            roll.d[2] = 1.0f;
            Rot<D3> Rt = rot_ypr(yaw, pitch, roll);
            V3<D3> f = antenna_vec<D3>(p.txa.kind, zeta_t, Rt, v_const<D3>(d));
            E[0] = {f.x, dconst<3>(0.0f)};
            E[1] = {f.y, dconst<3>(0.0f)};
            E[2] = {f.z, dconst<3>(0.0f)};
            last = -1;
            depth = 0;
            alive = true;
        }
        if (!__any_sync(0xffffffffu, alive)) {
            if (feed.exhausted) break;
            continue;
        }
        if (alive) {
            float t;
            int id;
            const bool more = depth < p.D;
            const long long cell = cov_segment<false, L>(p, sm, tx, o, d, last, more, id, t, cnt, cnt);
            if (cell >= 0) {
                const float g = q.grad_gain[cell];
                if (g != 0.0f) {
                    V3<float> F = antenna_vec<float>(p.rxa.kind, zeta_r, Rr, V3<float>{-d.x, -d.y, -d.z});
                    D3 re = E[0].re * F.x + E[1].re * F.y + E[2].re * F.z;
                    D3 im = E[0].im * F.x + E[1].im * F.y + E[2].im * F.z;
                    const float sw = g * p.wscale / fabsf(d.z);
                    for (int k = 0; k < 3; k++)
                        acc[k] += sw * 2.0f * (re.v * re.d[k] + im.v * im.d[k]);
                }
            }
            if (id < 0 || !more) {
                alive = false;
            } else {
                float4 pl = __ldg(p.c.s.planes + id);
                int m = __ldg(p.c.s.mat + id);
                float2 mp = __ldg(p.c.s.mats + m);
                f3 n = xyz(pl);
                f3 r = reflect(d, n);
                reflect_field<D3>(E, v_const<D3>(d), v_const<D3>(r), n, dconst<3>(mp.x), dconst<3>(mp.y), p.inv_we0);
                o = o + d * t;
                d = r;
                last = id;
                depth++;
            }
        }
    }
    flush_ypr(q.grad_ypr, tx, acc);
}

__global__ void k_dirs(long long N, long long first, long long n, float* __restrict__ out) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    f3 d = fib_dir(N, first + k);
    out[3 * k] = d.x;
    out[3 * k + 1] = d.y;
    out[3 * k + 2] = d.z;
}

int trace_grid(rt_ctx* ctx, const void* kernel, size_t smem) {
    int per_sm = blocks_per_sm(kernel, ctx->trace_block, smem);
    if (ctx->grid_cap > 0) per_sm = std::min(per_sm, ctx->grid_cap);
    if (per_sm < 1) per_sm = 1;
    return per_sm * ctx->num_sms;
}

// Rays per warp refill: the tuned value, else 32 (one ray per lane). Larger
// refills cut the counter atomics but lengthen the launch's tail and keep a
// warp on one patch of directions; on the 64-transmitter coverage map (6.4e8
// rays) 32 ran 2.1x faster than 1024.
int pick_chunk(rt_ctx* ctx, long long total, int grid) {
    (void)total;
    (void)grid;
    return ctx->warp_chunk > 0 ? ctx->warp_chunk : 32;
}

}  // namespace

int launch_dirs(rt_ctx* ctx, int64_t N, int64_t first, int64_t n, float* out) {
    if (n <= 0) return RT_OK;
    prof_begin(ctx, "k_dirs");
    k_dirs<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(N, first, n, out);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int ensure_perm(rt_ctx* ctx, int64_t N) {
    if (ctx->perm_n == N) return RT_OK;
    int ej = side_join(ctx);   // a map on the second stream may still read the old order
    if (ej) return ej;
    if (ctx->capturing) return set_err(ctx, RT_ERR_NOT_READY, "first trace at a new num_rays while capturing a graph");
    if (N > 0xFFFFFFFFll) return set_err(ctx, RT_ERR_INVALID_ARG, "num_rays above 2^32");
    DevBuf k1, k2, v2;
    RT_TRY(buf_reserve(ctx->perm, sizeof(uint32_t) * (size_t)N));
    cudaError_t e = buf_reserve(k1, sizeof(uint64_t) * (size_t)N);
    if (e == cudaSuccess) e = buf_reserve(k2, sizeof(uint64_t) * (size_t)N);
    if (e == cudaSuccess) e = buf_reserve(v2, sizeof(uint32_t) * (size_t)N);
    if (e == cudaSuccess) {
        prof_begin(ctx, "k_perm_keys");
        k_perm_keys<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(N, bp<uint64_t>(k1),
                                                                         bp<uint32_t>(ctx->perm));
        prof_end(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = radix_sort64(ctx, bp<uint64_t>(k1), bp<uint64_t>(k2), bp<uint32_t>(ctx->perm), bp<uint32_t>(v2), N, 24);
    // the directions in that order, computed once per ray count: the tracing
    // kernels then read them instead of evaluating the FP64 lattice per ray
    // (GB300's FP64 units are few). Without room for the table they compute
    // the directions themselves.
    ctx->dirs_ok = false;
    if (e == cudaSuccess && buf_reserve(ctx->dirs, sizeof(float4) * (size_t)N) == cudaSuccess) {
        prof_begin(ctx, "k_dir_table");
        k_dir_table<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(N, bp<uint32_t>(ctx->perm),
                                                                        bp<float4>(ctx->dirs));
        prof_end(ctx);
        e = cudaGetLastError();
        ctx->dirs_ok = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    buf_free(k1);
    buf_free(k2);
    buf_free(v2);
    if (e != cudaSuccess) return set_cuda(ctx, e, "ray order");
    ctx->perm_n = N;
    return RT_OK;
}

static TraceCommon make_common(rt_ctx* ctx, int64_t N, int64_t first, int64_t count) {
    TraceCommon c;
    c.s = dev_scene(ctx);
    c.tx_pos = bp<float>(ctx->tx_pos);
    c.tx_ypr = bp<float>(ctx->tx_ypr);
    c.N = N;
    c.first = first;
    c.count = count;
    c.total = (long long)count * ctx->n_tx;
    c.perm = (first == 0 && count == N && ctx->perm_n == N) ? bp<uint32_t>(ctx->perm) : nullptr;
    c.dirs = (c.perm && ctx->dirs_ok) ? bp<float4>(ctx->dirs) : nullptr;
    c.counter = bp<unsigned long long>(ctx->counters);
    c.chunk = ctx->warp_chunk;
    c.quota = 0;
    c.n_sm = staged_nodes(ctx);
    c.status = bp<unsigned>(ctx->status);
    return c;
}

// Shoot and bounce: appends every hit's candidate key with its position
// (tx*N + i)*D + depth; the key count goes to counter slot RT_CNT_KEYS.
int launch_sbr(rt_ctx* ctx, int64_t N, int D, uint64_t* keys, uint32_t* vals, int32_t* hits) {
    int e = ensure_perm(ctx, N);
    if (e) return e;
    SbrParams p;
    p.c = make_common(ctx, N, 0, N);
    p.D = D;
    p.id_bits = ctx->id_bits;
    p.depth_shift = D * ctx->id_bits;
    p.tx_shift = p.depth_shift + 3;
    p.keys = keys;
    p.vals = vals;
    p.n_keys = bp<unsigned long long>(ctx->counters) + RT_CNT_KEYS;
    p.hits = hits;
    size_t smem = staged_bytes(ctx);
    auto kern = wide_layout(ctx) ? (ctx->count_work ? k_sbr<true, 8> : k_sbr<false, 8>)
                                 : (ctx->count_work ? k_sbr<true, 2> : k_sbr<false, 2>);
    RT_TRY(ensure_smem_attr((const void*)kern, smem));
    RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), ctx->stream));
    RT_TRY(cudaMemsetAsync(p.n_keys, 0, sizeof(unsigned long long), ctx->stream));
    int grid = trace_grid(ctx, (const void*)kern, smem);
    p.c.chunk = pick_chunk(ctx, p.c.total, grid);
    prof_begin(ctx, "k_sbr");
    kern<<<grid, ctx->trace_block, smem, ctx->stream>>>(p);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int launch_coverage(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int64_t first, int64_t count, bool zero,
                    int tx_port, float* gain, uint32_t* hits) {
    if (first == 0 && count == N) {
        int e = ensure_perm(ctx, N);
        if (e) return e;
    }
    CovParams p;
    p.c = make_common(ctx, N, first, count);
    p.D = D;
    p.txa = ctx->tx_ant;
    p.rxa = ctx->rx_ant;
    p.tx_port = tx_port;
    p.inv_we0 = (float)(1.0 / (2.0 * RT_PI_D * ctx->fc * RT_EPS0_D));
    p.x0 = g->x0;
    p.y0 = g->y0;
    p.inv_cell = 1.0f / g->cell;
    p.h = g->height;
    p.nx = g->nx;
    p.ny = g->ny;
    double lam = RT_C0_D / ctx->fc;
    p.wscale = (float)(lam * lam / (4.0 * RT_PI_D * (double)g->cell * g->cell * (double)N));
    p.gain = gain;
    p.hits = hits;
    size_t cells = (size_t)ctx->n_tx * g->nx * g->ny;
    if (zero) {
        RT_TRY(cudaMemsetAsync(gain, 0, sizeof(float) * cells, ctx->stream));
        RT_TRY(cudaMemsetAsync(hits, 0, sizeof(uint32_t) * cells, ctx->stream));
    }
    if (count == 0) return RT_OK;
    size_t smem = staged_bytes(ctx);
    auto kern = wide_layout(ctx) ? (ctx->count_work ? k_coverage<true, 8> : k_coverage<false, 8>)
                                 : (ctx->count_work ? k_coverage<true, 2> : k_coverage<false, 2>);
    RT_TRY(ensure_smem_attr((const void*)kern, smem));
    RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), ctx->stream));
    int grid = trace_grid(ctx, (const void*)kern, smem);
    p.c.chunk = pick_chunk(ctx, p.c.total, grid);
    if (ctx->side_yield) {
        // a map beside other work: short-lived blocks, one refill of 32 rays
        // per warp, so that kernels of the context's stream (given a higher
        // priority) take the SM slots these blocks free as they end
        p.c.quota = 1;
        p.c.chunk = 32;
        const long long warps = (p.c.total + 31) / 32;
        const int wpb = ctx->trace_block / 32;
        grid = (int)std::max<long long>(1, (warps + wpb - 1) / wpb);
    }
    prof_begin(ctx, "k_coverage");
    kern<<<grid, ctx->trace_block, smem, ctx->stream>>>(p);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

// VJP of the coverage map w.r.t. the transmitters' (yaw, pitch, roll):
// grad_ypr [n_tx*3] is overwritten.
int launch_coverage_vjp(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int tx_port, const float* grad_gain,
                        float* grad_ypr) {
    int e = ensure_perm(ctx, N);
    if (e) return e;
    CovVjpParams q;
    CovParams& p = q.p;
    p.c = make_common(ctx, N, 0, N);
    p.D = D;
    p.txa = ctx->tx_ant;
    p.rxa = ctx->rx_ant;
    p.tx_port = tx_port;
    p.inv_we0 = (float)(1.0 / (2.0 * RT_PI_D * ctx->fc * RT_EPS0_D));
    p.x0 = g->x0;
    p.y0 = g->y0;
    p.inv_cell = 1.0f / g->cell;
    p.h = g->height;
    p.nx = g->nx;
    p.ny = g->ny;
    double lam = RT_C0_D / ctx->fc;
    p.wscale = (float)(lam * lam / (4.0 * RT_PI_D * (double)g->cell * g->cell * (double)N));
    p.gain = nullptr;
    p.hits = nullptr;
    q.grad_gain = grad_gain;
    q.grad_ypr = grad_ypr;
    RT_TRY(cudaMemsetAsync(grad_ypr, 0, sizeof(float) * 3 * (size_t)ctx->n_tx, ctx->stream));
    size_t smem = staged_bytes(ctx);
    auto kern = wide_layout(ctx) ? k_coverage_vjp<8> : k_coverage_vjp<2>;
    RT_TRY(ensure_smem_attr((const void*)kern, smem));
    RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), ctx->stream));
    int grid = trace_grid(ctx, (const void*)kern, smem);
    p.c.chunk = pick_chunk(ctx, p.c.total, grid);
    prof_begin(ctx, "k_coverage_vjp");
    kern<<<grid, ctx->trace_block, smem, ctx->stream>>>(q);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

// The coverage kernel on scratch the caller provides: the work counter and
// traversal counter slots at `counters` (8 x uint64, zeroed here), the status
// word at `status`, the ray order at `perm` (null = lattice order). Allocates
// no device memory.
int launch_coverage_scratch(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int tx_port, float* gain,
                            uint32_t* hits, unsigned long long* counters, unsigned* status, const uint32_t* perm) {
    CovParams p;
    p.c = make_common(ctx, N, 0, N);
    p.c.counter = counters;
    p.c.status = status;
    p.c.perm = perm;
    p.c.dirs = nullptr;
    p.D = D;
    p.txa = ctx->tx_ant;
    p.rxa = ctx->rx_ant;
    p.tx_port = tx_port;
    p.inv_we0 = (float)(1.0 / (2.0 * RT_PI_D * ctx->fc * RT_EPS0_D));
    p.x0 = g->x0;
    p.y0 = g->y0;
    p.inv_cell = 1.0f / g->cell;
    p.h = g->height;
    p.nx = g->nx;
    p.ny = g->ny;
    double lam = RT_C0_D / ctx->fc;
    p.wscale = (float)(lam * lam / (4.0 * RT_PI_D * (double)g->cell * g->cell * (double)N));
    p.gain = gain;
    p.hits = hits;
    size_t cells = (size_t)ctx->n_tx * g->nx * g->ny;
    RT_TRY(cudaMemsetAsync(gain, 0, sizeof(float) * cells, ctx->stream));
    RT_TRY(cudaMemsetAsync(hits, 0, sizeof(uint32_t) * cells, ctx->stream));
    RT_TRY(cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned long long), ctx->stream));
    size_t smem = staged_bytes(ctx);
    auto kern = wide_layout(ctx) ? k_coverage<false, 8> : k_coverage<false, 2>;
    RT_TRY(ensure_smem_attr((const void*)kern, smem));
    int grid = trace_grid(ctx, (const void*)kern, smem);
    p.c.chunk = pick_chunk(ctx, p.c.total, grid);
    ctx->launches++;
    kern<<<grid, ctx->trace_block, smem, ctx->stream>>>(p);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}
