// rt_scatter.cu -- first-order diffuse scattering (Sec. II-B lists diffuse
// reflections, i.e. scattering, among the features and leaves the model to
// the documentation). Reading used here: the effective-roughness model with
// a Lambertian pattern, the scattered wave depolarised.
//
// Each of the N Fibonacci-lattice rays of a transmitter carries the fraction
// |F_tx,q(d)|^2 / N of the transmitted power. Where it first hits a surface
// of scattering coefficient S, the fraction S^2 is re-radiated with the
// intensity pattern cos(theta_s)/pi on the side the ray came from; a
// receiver there, with the segment to it unoccluded, collects with the
// effective aperture lambda^2/(4 pi) |F_rx,p|^2, half of the depolarised
// wave per port:
//   g[pair][p][q] += S^2 (|F_tx,q(d)|^2/N) (cos theta_s/pi) (lambda^2/(4 pi r^2)) |F_rx,p(-k_s)|^2 / 2.
// The result is the incoherent scattered gain of every pair and port pair.
// A material with a directive pattern (exponent alpha >= 0) replaces
// cos(theta_s)/pi by ((1 + k_r . k_s)/2)^alpha / F_alpha, k_r the specular
// direction and F_alpha the lobe's integral over the hemisphere.
//
// The gain is quadratic in S, so its vector-Jacobian product with respect to
// the coefficients (Sec. II: gradients with respect to the parameters of the
// scattering functions) is, for material m,
//   dL/dS_m = 2 S_m sum over rays hitting m, receivers and ports of dL/dg * g / S_m^2,
// accumulated by the same kernel in its VJP mode.
#include "rt_field.cuh"
#include "rt_internal.h"

namespace {

struct ScatParams {
    DevScene s;
    const float* tx_pos;
    const float* tx_ypr;
    const float* rx_pos;
    const float* rx_ypr;
    const int32_t* rx_off;   // [n_tx+1] or null
    const float* scat;       // [n_mat] scattering coefficients
    const float4* dirs;      // [N] directions in the direction-coherent ray order, or null
    const int32_t* alpha;    // [n_mat] pattern exponent, -1 Lambertian; null: all Lambertian
    const float* up;         // VJP: upstream dL/dgain [n_pairs][nrp][ntp]
    float* grad;             // VJP: dL/dS [n_mat]
    int n_mat;
    bool grad_smem;          // VJP: per-block partial sums in shared memory
    int n_tx, n_rx;
    int n_chunks;            // receiver chunks per ray (each (ray, chunk) is one thread)
    long long N;
    DevAntenna txa, rxa;
    float w0;                // lambda^2 / (4 pi) / (2 pi N)
    float* gain;             // [n_pairs][nrp][ntp]
};

// F_alpha: the integral of ((1 + k_r . k_s)/2)^alpha over the hemisphere
// k_s . n > 0, with cos(theta_i) = k_r . n = ci. Binomial expansion in
// x = k_r . k_s; the hemisphere integral of x^j is 2 pi/(j+1) for even j
// (half the sphere's) and, for odd j = 2w+1,
//   2 pi/(j+1) ci sum_{u=0..w} C(2u, u) (sin^2(theta_i)/4)^u.
__device__ float directive_norm(int alpha, float ci) {
    const float q = 0.25f * fmaxf(0.0f, 1.0f - ci * ci);
    float tot = 0.0f, binom = 1.0f, part = 0.0f, term = 1.0f;
    int u = 0;
    for (int j = 0; j <= alpha; j++) {
        float I;
        if ((j & 1) == 0) {
            I = 2.0f * RT_PI_F / (float)(j + 1);
        } else {
            part += term;                                   // adds C(2u, u) q^u
            term *= q * 2.0f * (float)(2 * u + 1) / (float)(u + 1);
            u++;
            I = 2.0f * RT_PI_F / (float)(j + 1) * ci * part;
        }
        tot += binom * I;
        binom *= (float)(alpha - j) / (float)(j + 1);
    }
    return ldexpf(tot, -alpha);
}

// One thread per (transmitter, lattice ray): first hit, then every receiver
// of that transmitter in order (the warp's lanes visit the same receiver
// together and add their contributions with one atomic when they share the
// transmitter). The rays are taken in the direction-coherent order of the
// tracing kernels (directions from the context's table), so the lanes of a
// warp hit nearby points and their segment tests to a receiver follow
// similar paths through the hierarchy: 2.2x faster than the lattice order,
// whose neighbours are a golden angle apart in azimuth. VJP: each ray's sum of dL/dg * g / S^2 is added, times
// 2 S, to its material's gradient (per block in shared memory first).
template <bool VJP, int L>
__global__ void __launch_bounds__(128) k_scatter(ScatParams p) {
    extern __shared__ float sgrad[];
    const unsigned full = 0xffffffffu;
    if (VJP && p.grad_smem) {
        for (int i = threadIdx.x; i < p.n_mat; i += blockDim.x) sgrad[i] = 0.0f;
        __syncthreads();
    }
    const long long n_slots = (long long)p.n_tx * p.N;
    const long long total = n_slots * p.n_chunks;
    const long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long b = base; b < total; b += (long long)gridDim.x * blockDim.x) {
        const long long vs = b + (threadIdx.x & 31);
        const bool has = vs < total;
        const int c = has ? (int)(vs / n_slots) : p.n_chunks - 1;      // receiver chunk
        const long long slot = has ? vs - (long long)c * n_slots : n_slots - 1;
        const int t = has ? (int)(slot / p.N) : p.n_tx - 1;
        const long long i = has ? slot - (long long)t * p.N : 0;
        const int t0 = __shfl_sync(full, t, 0), c0 = __shfl_sync(full, c, 0);
        const bool uniform = __all_sync(full, t == t0 && c == c0);
        float s2 = 0.0f, sc = 0.0f, acc = 0.0f;
        f3 P = mk(0, 0, 0), n = mk(0, 0, 1);
        int hit = -1, m = 0, am = -1;
        f3 kr = mk(0, 0, 1);
        float fa = 1.0f;
        float ptx[2] = {0.0f, 0.0f};
        if (has) {
            const f3 o = mk(p.tx_pos[3 * t], p.tx_pos[3 * t + 1], p.tx_pos[3 * t + 2]);
            const f3 d = p.dirs ? xyz(__ldg(p.dirs + i)) : fib_dir(p.N, i);
            TravCount cnt;
            float th;
            hit = closest_hit<false, L, false>(p.s, nullptr, 0, o, d, -1, th, cnt);
            if (hit >= 0) {
                m = __ldg(p.s.mat + hit);
                sc = __ldg(p.scat + m);
                s2 = sc > 0.0f ? sc * sc : 0.0f;   // S <= 0: no scattering
                n = xyz(__ldg(p.s.planes + hit));
                if (dot(d, n) > 0.0f) n = n * -1.0f;   // the side the ray came from
                P = o + d * th;
                am = p.alpha ? __ldg(p.alpha + m) : -1;
                if (am >= 0) {
                    const float dn = dot(d, n);                 // < 0: n faces the incoming ray
                    kr = d - n * (2.0f * dn);
                    fa = directive_norm(am, -dn) / RT_PI_F;     // pi / F_alpha replaces 1/pi in w0
                }
                const Rot<float> Rt = rot_ypr(p.tx_ypr[3 * t], p.tx_ypr[3 * t + 1], p.tx_ypr[3 * t + 2]);
                for (int q = 0; q < p.txa.n_ports; q++) {
                    const V3<float> f = antenna_vec<float>(p.txa.kind, p.txa.slant[q], Rt, V3<float>{d.x, d.y, d.z});
                    ptx[q] = f.x * f.x + f.y * f.y + f.z * f.z;
                }
            }
        }
        const bool live = __any_sync(full, s2 > 0.0f);
        if (!live) continue;
        // this lane's chunk of the receivers of its transmitter
        const int rb0 = p.rx_off ? p.rx_off[t] : 0, re0 = p.rx_off ? p.rx_off[t + 1] : p.n_rx;
        const int len = (re0 - rb0 + p.n_chunks - 1) / p.n_chunks;
        const int rb = min(re0, rb0 + c * len), re = min(re0, rb + len);
        const int nr = re - rb;
        const int nr_max = __reduce_max_sync(full, (unsigned)nr);
        for (int k = 0; k < nr_max; k++) {
            float w = 0.0f, prx[2] = {0.0f, 0.0f};
            const int r = rb + k;
            if (s2 > 0.0f && k < nr) {
                const f3 rx = mk(p.rx_pos[3 * r], p.rx_pos[3 * r + 1], p.rx_pos[3 * r + 2]);
                const f3 v = rx - P;
                const float dist = sqrtf(dot(v, v));
                const float cs = dot(v, n) / dist;
                if (cs > 0.0f) {
                    const f3 ks = v * (1.0f / dist);
                    TravCount cnt;
                    if (!any_hit<false, L, false>(p.s, nullptr, 0, P, ks, dist - p.s.tmin, hit, -1, cnt)) {
                        const float pat = am < 0 ? cs : powf(0.5f * (1.0f + dot(kr, ks)), (float)am) / fa;
                        w = (VJP ? 1.0f : s2) * pat * p.w0 / (dist * dist);
                        const Rot<float> Rr = rot_ypr(p.rx_ypr[3 * r], p.rx_ypr[3 * r + 1], p.rx_ypr[3 * r + 2]);
                        for (int pp = 0; pp < p.rxa.n_ports; pp++) {
                            const V3<float> f = antenna_vec<float>(p.rxa.kind, p.rxa.slant[pp], Rr,
                                                                   V3<float>{-ks.x, -ks.y, -ks.z});
                            prx[pp] = f.x * f.x + f.y * f.y + f.z * f.z;
                        }
                    }
                }
            }
            const long long pair = p.rx_off ? (long long)r : (long long)t * p.n_rx + r;
            if (VJP) {   // w is g / S^2 here
                if (w != 0.0f)
                    for (int pp = 0; pp < p.rxa.n_ports; pp++)
                        for (int q = 0; q < p.txa.n_ports; q++)
                            acc += __ldg(p.up + (pair * p.rxa.n_ports + pp) * p.txa.n_ports + q) * w * prx[pp] * ptx[q];
                continue;
            }
            for (int pp = 0; pp < p.rxa.n_ports; pp++)
                for (int q = 0; q < p.txa.n_ports; q++) {
                    float c = w * prx[pp] * ptx[q];
                    if (uniform) {   // same transmitter and receiver in every lane: one atomic per warp
                        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(full, c, o);
                        if ((threadIdx.x & 31) == 0 && c != 0.0f && k < nr)
                            atomicAdd(p.gain + (pair * p.rxa.n_ports + pp) * p.txa.n_ports + q, c);
                    } else if (c != 0.0f) {
                        atomicAdd(p.gain + (pair * p.rxa.n_ports + pp) * p.txa.n_ports + q, c);
                    }
                }
        }
        if (VJP && acc != 0.0f) atomicAdd((p.grad_smem ? sgrad : p.grad) + m, 2.0f * sc * acc);
    }
    if (VJP && p.grad_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < p.n_mat; i += blockDim.x)
            if (sgrad[i] != 0.0f) atomicAdd(p.grad + i, sgrad[i]);
    }
}

}  // namespace

// gain != null: forward; else up / grad: the VJP with respect to S.
int scattering_impl(rt_ctx* ctx, int64_t N, float* gain, const float* up, float* grad) {
    const int64_t n_pairs = ctx->rx_sets ? (int64_t)ctx->rx_off[ctx->n_tx] : (int64_t)ctx->n_tx * ctx->n_rx;
    const int np = ctx->tx_ant.n_ports * ctx->rx_ant.n_ports;
    const bool vjp = gain == nullptr;
    if (vjp) RT_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)ctx->n_mat, ctx->stream));
    else RT_TRY(cudaMemsetAsync(gain, 0, sizeof(float) * (size_t)n_pairs * np, ctx->stream));
    if (N == 0 || ctx->n_tris == 0 || !ctx->scat_set) return RT_OK;
    ScatParams p;
    p.s = dev_scene(ctx);
    p.tx_pos = bp<float>(ctx->tx_pos);
    p.tx_ypr = bp<float>(ctx->tx_ypr);
    p.rx_pos = bp<float>(ctx->rx_pos);
    p.rx_ypr = bp<float>(ctx->rx_ypr);
    p.rx_off = ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr;
    p.scat = bp<float>(ctx->scat);
    {
        int e = ensure_perm(ctx, N);
        if (e) return e;
    }
    p.dirs = ctx->dirs_ok ? bp<float4>(ctx->dirs) : nullptr;
    p.alpha = ctx->scat_alpha_set ? bp<int32_t>(ctx->scat_alpha) : nullptr;
    p.up = up;
    p.grad = grad;
    p.n_mat = ctx->n_mat;
    p.grad_smem = vjp && ctx->n_mat <= 4096;
    p.n_tx = ctx->n_tx;
    p.n_rx = ctx->n_rx;
    p.N = N;
    p.txa = ctx->tx_ant;
    p.rxa = ctx->rx_ant;
    const double lam = RT_C0_D / ctx->fc;
    p.w0 = (float)(lam * lam / (4.0 * RT_PI_D) / (2.0 * RT_PI_D * (double)N));
    p.gain = gain;
    // few rays: split every ray's receivers into chunks, one thread each, so
    // that about 4 x 2048 threads per SM are in flight (the first hit is
    // traced once per chunk, against hundreds of segment tests per chunk)
    int nr_max = ctx->n_rx;
    if (ctx->rx_sets) {
        nr_max = 0;
        for (int t = 0; t < ctx->n_tx; t++) nr_max = std::max(nr_max, ctx->rx_off[t + 1] - ctx->rx_off[t]);
    }
    const long long slots = (long long)ctx->n_tx * N;
    const long long want = 4ll * 2048 * ctx->num_sms;
    const long long by_rx = std::min<long long>(8, (long long)nr_max / 64);
    p.n_chunks = (int)std::max<long long>(1, std::min<long long>(by_rx, (want + slots - 1) / slots));
    const long long total = slots * p.n_chunks;
    const long long blocks = std::min<long long>((total + 127) / 128, 16ll * ctx->num_sms);
    if (vjp) {
        prof_begin(ctx, "k_scatter_vjp");
        auto kern = wide_layout(ctx) ? k_scatter<true, 8> : k_scatter<true, 2>;
        kern<<<(unsigned)blocks, 128, p.grad_smem ? sizeof(float) * ctx->n_mat : 0, ctx->stream>>>(p);
    } else {
        prof_begin(ctx, "k_scatter");
        auto kern = wide_layout(ctx) ? k_scatter<false, 8> : k_scatter<false, 2>;
        kern<<<(unsigned)blocks, 128, 0, ctx->stream>>>(p);
    }
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}
