// rt_cir.cu -- channel impulse response (Listing 3: a_i, tau_i), OFDM
// frequency response (Sec. III-A) and their vector-Jacobian products
// (Sec. I/II: gradients w.r.t. materials and transmitter pose).
//
// The field of one path is written once over a scalar type (rt_field.cuh).
// The VJP kernel replays the stored path (no re-trace): for each group of
// two of the path's local parameters (one group per grid row, so a path's
// groups run in parallel) it runs the field with Dual<2> tangents and
// contracts the Jacobian with the upstream gradient. A path
// depends on at most 6 + 2*depth parameters (tx xyz, yaw/pitch/roll, eps_r
// and sigma of the materials it reflects on), so per-path forward tangents
// are cheaper than a taped reverse pass.
#include "rt_field.cuh"
#include "rt_internal.h"

namespace {

struct CirParams {
    DevScene s;
    const float* tx_pos;
    const float* tx_ypr;
    const float* rx_pos;
    const float* rx_ypr;
    DevAntenna txa, rxa;
    const int32_t* seq;      // [P*D]
    const int32_t* depth;    // [P]
    const double* len;       // [P]
    const int32_t* pair_tx;  // [P*2]
    int D;
    int64_t P;
    double lambda;
    float inv_we0;
    uint32_t flags;
};

template <class S>
struct PathIn {
    V3<S> tx;
    S yaw, pitch, roll;
    S eps[RT_MAX_DEPTH], sig[RT_MAX_DEPTH];
};

// a[p][q] (rx port p, tx port q) and the path length (as S) of path i;
// len64 = the same length accumulated in FP64 (carrier phase).
template <class S>
__device__ __forceinline__ void path_field(const CirParams& c, int64_t i, const PathIn<S>& in, f3 rx,
                                           f3 rx_ypr, double len64, Cx<S> a[4], S& L) {
    const int K = c.depth[i];
    const int32_t* ids = c.seq + i * c.D;
    V3<S> I[RT_MAX_DEPTH + 1];
    I[0] = in.tx;
    for (int k = 1; k <= K; k++) {
        float4 pl = __ldg(c.s.planes + ids[k - 1]);
        V3<S> n = v_const<S>(xyz(pl));
        S sd = v_dot(I[k - 1], n) - pl.w;
        I[k] = v_sub(I[k - 1], v_scale(n, sd * 2.0f));
    }
    V3<S> P[RT_MAX_DEPTH + 2];
    P[0] = in.tx;
    P[K + 1] = v_const<S>(rx);
    for (int k = K; k >= 1; k--) {
        float4 pl = __ldg(c.s.planes + ids[k - 1]);
        V3<S> n = v_const<S>(xyz(pl));
        V3<S> dir = v_sub(I[k], P[k + 1]);
        S sp = (pl.w - v_dot(P[k + 1], n)) / v_dot(dir, n);
        P[k] = v_add(P[k + 1], v_scale(dir, sp));
    }
    V3<S> kd[RT_MAX_DEPTH + 1];
    L = SConst<S>::make(0.0f);
    for (int j = 0; j <= K; j++) {
        V3<S> sg = v_sub(P[j + 1], P[j]);
        S l = s_sqrt(v_dot(sg, sg));
        L = L + l;
        kd[j] = v_scale(sg, SConst<S>::make(1.0f) / l);
    }
    Rot<S> Rt = rot_ypr(in.yaw, in.pitch, in.roll);
    Rot<S> Rr = rot_ypr(SConst<S>::make(rx_ypr.x), SConst<S>::make(rx_ypr.y), SConst<S>::make(rx_ypr.z));
    Cx<S> E[2][3];
    for (int q = 0; q < c.txa.n_ports; q++) {
        V3<S> f = antenna_vec<S>(c.txa.kind, c.txa.slant[q], Rt, kd[0]);
        E[q][0] = {f.x, SConst<S>::make(0.0f)};
        E[q][1] = {f.y, SConst<S>::make(0.0f)};
        E[q][2] = {f.z, SConst<S>::make(0.0f)};
    }
    for (int k = 1; k <= K; k++) {
        f3 n = xyz(__ldg(c.s.planes + ids[k - 1]));
        for (int q = 0; q < c.txa.n_ports; q++)
            reflect_field<S>(E[q], kd[k - 1], kd[k], n, in.eps[k - 1], in.sig[k - 1], c.inv_we0);
    }
    V3<S> u = v_scale(kd[K], -1.0f);
    // phase: value from the FP64 length reduced modulo 2 pi, tangents from L
    double x = len64 / c.lambda;
    float ph0 = (float)(-2.0 * RT_PI_D * (x - floor(x)));
    S ph = L * (float)(-2.0 * RT_PI_D / c.lambda);
    S amp = SConst<S>::make((float)(c.lambda / (4.0 * RT_PI_D))) / L;
    Cx<S> e;
    {
        S phv = with_value(ph, ph0);  // reduced phase value, tangents of -2 pi L / lambda
        e.re = amp * s_cos(phv);
        e.im = amp * s_sin(phv);
    }
    for (int p = 0; p < c.rxa.n_ports; p++) {
        V3<S> F = antenna_vec<S>(c.rxa.kind, c.rxa.slant[p], Rr, u);
        for (int q = 0; q < c.txa.n_ports; q++) {
            Cx<S> fe = {F.x * E[q][0].re + F.y * E[q][1].re + F.z * E[q][2].re,
                        F.x * E[q][0].im + F.y * E[q][1].im + F.z * E[q][2].im};
            a[p * c.txa.n_ports + q] = c_mul(e, fe);
        }
    }
}

__device__ __forceinline__ bool path_enabled(uint32_t flags, int K) {
    return K == 0 ? (flags & RT_LOS) != 0 : (flags & RT_REFLECTION) != 0;
}

__global__ void k_cir(CirParams c, float2* __restrict__ a_out, float* __restrict__ tau) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.P) return;
    int t = c.pair_tx[2 * i], r = c.pair_tx[2 * i + 1];
    PathIn<float> in;
    in.tx = {c.tx_pos[3 * t], c.tx_pos[3 * t + 1], c.tx_pos[3 * t + 2]};
    in.yaw = c.tx_ypr[3 * t];
    in.pitch = c.tx_ypr[3 * t + 1];
    in.roll = c.tx_ypr[3 * t + 2];
    const int K = c.depth[i];
    for (int k = 0; k < K; k++) {
        int m = __ldg(c.s.mat + c.seq[i * c.D + k]);
        float2 mp = __ldg(c.s.mats + m);
        in.eps[k] = mp.x;
        in.sig[k] = mp.y;
    }
    f3 rx = mk(c.rx_pos[3 * r], c.rx_pos[3 * r + 1], c.rx_pos[3 * r + 2]);
    f3 ry = mk(c.rx_ypr[3 * r], c.rx_ypr[3 * r + 1], c.rx_ypr[3 * r + 2]);
    Cx<float> a[4];
    float L;
    const double len64 = path_length64(c.s, c.seq + i * c.D, K, mk(in.tx.x, in.tx.y, in.tx.z), rx);
    path_field<float>(c, i, in, rx, ry, len64, a, L);
    const int np = c.txa.n_ports * c.rxa.n_ports;
    const bool on = path_enabled(c.flags, K);
    for (int k = 0; k < np; k++) a_out[i * np + k] = on ? make_float2(a[k].re, a[k].im) : make_float2(0.0f, 0.0f);
    tau[i] = (float)(len64 / RT_C0_D);
}

// ----------------------------------------------------------------- VJP of cir
constexpr int NT = 2;

__global__ void k_cir_vjp(CirParams c, const float2* __restrict__ ga, const float* __restrict__ gtau,
                          float* g_eps, float* g_sig, float* g_pos, float* g_ypr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.P) return;
    const int K = c.depth[i];
    if (!path_enabled(c.flags, K) && !gtau) return;
    int t = c.pair_tx[2 * i], r = c.pair_tx[2 * i + 1];
    // local parameter list: 0..2 tx xyz, 3..5 yaw pitch roll, then (eps, sigma)
    // of each distinct material along the path
    int mats[RT_MAX_DEPTH], nm = 0, slot[RT_MAX_DEPTH];
    for (int k = 0; k < K; k++) {
        int m = __ldg(c.s.mat + c.seq[i * c.D + k]);
        int j = 0;
        while (j < nm && mats[j] != m) j++;
        if (j == nm) mats[nm++] = m;
        slot[k] = j;
    }
    const int nloc = 6 + 2 * nm;
    const int np = c.txa.n_ports * c.rxa.n_ports;
    const bool on = path_enabled(c.flags, K);
    f3 rx = mk(c.rx_pos[3 * r], c.rx_pos[3 * r + 1], c.rx_pos[3 * r + 2]);
    f3 ry = mk(c.rx_ypr[3 * r], c.rx_ypr[3 * r + 1], c.rx_ypr[3 * r + 2]);
    float2 g[4];
    for (int k = 0; k < np; k++) g[k] = on ? ga[i * np + k] : make_float2(0.0f, 0.0f);
    const float gt = gtau ? gtau[i] : 0.0f;
    // one group of NT local parameters per grid row (blockIdx.y)
    const int base = blockIdx.y * NT;
    if (base >= nloc) return;
    const double len64 = path_length64(c.s, c.seq + i * c.D, K,
                                       mk(c.tx_pos[3 * t], c.tx_pos[3 * t + 1], c.tx_pos[3 * t + 2]), rx);
    {
        auto var = [&](float v, int idx) {
            Dual<NT> d = dconst<NT>(v);
            if (idx >= base && idx < base + NT) d.d[idx - base] = 1.0f;
            return d;
        };
        PathIn<Dual<NT>> in;
        in.tx = {var(c.tx_pos[3 * t], 0), var(c.tx_pos[3 * t + 1], 1), var(c.tx_pos[3 * t + 2], 2)};
        in.yaw = var(c.tx_ypr[3 * t], 3);
        in.pitch = var(c.tx_ypr[3 * t + 1], 4);
        in.roll = var(c.tx_ypr[3 * t + 2], 5);
        for (int k = 0; k < K; k++) {
            float2 mp = __ldg(c.s.mats + mats[slot[k]]);
            in.eps[k] = var(mp.x, 6 + 2 * slot[k]);
            in.sig[k] = var(mp.y, 7 + 2 * slot[k]);
        }
        Cx<Dual<NT>> a[4];
        Dual<NT> L;
        path_field<Dual<NT>>(c, i, in, rx, ry, len64, a, L);
        for (int j = 0; j < NT && base + j < nloc; j++) {
            float acc = gt * L.d[j] * (float)(1.0 / RT_C0_D);
            for (int k = 0; k < np; k++) acc += g[k].x * a[k].re.d[j] + g[k].y * a[k].im.d[j];
            int idx = base + j;
            if (idx < 3) {
                if (g_pos) atomicAdd(g_pos + 3 * t + idx, acc);
            } else if (idx < 6) {
                if (g_ypr) atomicAdd(g_ypr + 3 * t + idx - 3, acc);
            } else {
                int mi = mats[(idx - 6) >> 1];
                if ((idx - 6) & 1) { if (g_sig) atomicAdd(g_sig + mi, acc); }
                else if (g_eps) atomicAdd(g_eps + mi, acc);
            }
        }
    }
}

// ---------------------------------------------------------------- H(f)
// One block column per pair; block y covers 128 * HF_RUN subcarriers, thread t
// the subcarriers kb + t + 128 s (s < HF_RUN), so every store instruction
// writes 128 consecutive values. Accumulators for every port pair stay in
// registers; the pair's paths are staged in shared memory in tiles.
// Twiddles: with uniform spacing one range-reduced sincos for the first
// subcarrier and one for the 128-subcarrier step per (path, thread), then a
// complex-rotation recurrence; otherwise a sincos per (path, subcarrier).
// With uniform spacing two paths are taken per step (their twiddle chains
// interleave; each accumulator still sums the paths in order). Four
// subcarriers per thread keep the registers at about 70 for 2 x 2 port
// pairs, so more warps hide the sincos and recurrence latencies.
// H is cleared by a memset first, so the blocks of pairs without paths
// return at once.
constexpr int HF_RUN = 4;
constexpr int HF_TILE = 64;
constexpr int HF_THREADS = 128;

template <int NP>
__global__ void __launch_bounds__(HF_THREADS) k_freq(const int64_t* __restrict__ off, const float2* __restrict__ a,
                                                     const float* __restrict__ tau, const double* __restrict__ freqs,
                                                     int K, float2* __restrict__ H) {
    __shared__ float2 sa[HF_TILE][NP];
    __shared__ float st[HF_TILE];
    const int64_t pair = blockIdx.x;
    const int64_t b = off[pair], e = off[pair + 1];
    const int kb = blockIdx.y * HF_THREADS * HF_RUN + threadIdx.x;
    if (b == e) return;   // H was cleared before the launch
    float2 acc[HF_RUN][NP];
#pragma unroll
    for (int s = 0; s < HF_RUN; s++)
#pragma unroll
        for (int q = 0; q < NP; q++) acc[s][q] = make_float2(0.0f, 0.0f);
    // this thread's subcarriers; the recurrence needs them evenly spaced
    double f0 = 0.0, df = 0.0;
    if (kb < K) {
        f0 = freqs[kb];
        df = kb + HF_THREADS < K ? freqs[kb + HF_THREADS] - f0 : 0.0;
    }
    bool uniform = true;
#pragma unroll
    for (int s = 0; s < HF_RUN; s++) {
        const int k = kb + s * HF_THREADS;
        double fs = k < K ? freqs[k] : f0 + s * df;
        if (fabs(fs - (f0 + s * df)) > 1e-9 * (fabs(fs) + 1.0)) uniform = false;
    }
    const float fk0 = (float)f0, dff = (float)df;
    for (int64_t tb = b; tb < e; tb += HF_TILE) {
        int n = (int)min((int64_t)HF_TILE, e - tb);
        __syncthreads();
        for (int j = threadIdx.x; j < n * NP; j += blockDim.x) sa[j / NP][j % NP] = a[(tb + j / NP) * NP + j % NP];
        for (int j = threadIdx.x; j < n; j += blockDim.x) st[j] = tau[tb + j];
        __syncthreads();
        if (kb >= K) continue;
        if (uniform) {
            int j = 0;
            for (; j + 1 < n; j += 2) {
                float wr[2], wi[2], cdd[2], sd[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const float t = st[j + u];
                    float cyc = fk0 * t;
                    cyc -= rintf(cyc);
                    __sincosf(-2.0f * RT_PI_F * cyc, &wi[u], &wr[u]);
                    float cd = dff * t;
                    cd -= rintf(cd);
                    __sincosf(-2.0f * RT_PI_F * cd, &sd[u], &cdd[u]);
                }
#pragma unroll
                for (int s = 0; s < HF_RUN; s++) {
#pragma unroll
                    for (int u = 0; u < 2; u++) {
#pragma unroll
                        for (int q = 0; q < NP; q++) {
                            float2 av = sa[j + u][q];
                            acc[s][q].x = fmaf(av.x, wr[u], fmaf(-av.y, wi[u], acc[s][q].x));
                            acc[s][q].y = fmaf(av.x, wi[u], fmaf(av.y, wr[u], acc[s][q].y));
                        }
                        float nr = wr[u] * cdd[u] - wi[u] * sd[u];
                        wi[u] = wr[u] * sd[u] + wi[u] * cdd[u];
                        wr[u] = nr;
                    }
                }
            }
            for (; j < n; j++) {
                const float t = st[j];
                float cyc = fk0 * t;
                cyc -= rintf(cyc);
                float s0, c0;
                __sincosf(-2.0f * RT_PI_F * cyc, &s0, &c0);
                float cd = dff * t;
                cd -= rintf(cd);
                float sdv, cddv;
                __sincosf(-2.0f * RT_PI_F * cd, &sdv, &cddv);
                float wrv = c0, wiv = s0;
#pragma unroll
                for (int s = 0; s < HF_RUN; s++) {
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        float2 av = sa[j][q];
                        acc[s][q].x = fmaf(av.x, wrv, fmaf(-av.y, wiv, acc[s][q].x));
                        acc[s][q].y = fmaf(av.x, wiv, fmaf(av.y, wrv, acc[s][q].y));
                    }
                    float nr = wrv * cddv - wiv * sdv;
                    wiv = wrv * sdv + wiv * cddv;
                    wrv = nr;
                }
            }
        } else {
            float fl[HF_RUN];
#pragma unroll
            for (int s = 0; s < HF_RUN; s++) {
                const int k = kb + s * HF_THREADS;
                fl[s] = k < K ? (float)freqs[k] : 0.0f;
            }
            for (int j = 0; j < n; j++) {
                const float t = st[j];
#pragma unroll
                for (int s = 0; s < HF_RUN; s++) {
                    float cyc = fl[s] * t;
                    cyc -= rintf(cyc);
                    float wi, wr;
                    __sincosf(-2.0f * RT_PI_F * cyc, &wi, &wr);
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        float2 av = sa[j][q];
                        acc[s][q].x = fmaf(av.x, wr, fmaf(-av.y, wi, acc[s][q].x));
                        acc[s][q].y = fmaf(av.x, wi, fmaf(av.y, wr, acc[s][q].y));
                    }
                }
            }
        }
    }
    if (kb >= K) return;
#pragma unroll
    for (int q = 0; q < NP; q++)
#pragma unroll
        for (int s = 0; s < HF_RUN; s++) {
            const int k = kb + s * HF_THREADS;
            if (k < K) H[(pair * NP + q) * K + k] = acc[s][q];
        }
}

// VJP of H: grad_a_i = sum_k gH_k conj(w_ik); grad_tau_i = sum_k Re(conj(gH_k) a_i (-j 2 pi f_k) w_ik).
// One warp per path (all paths in parallel, whatever their pairs), lanes
// over the subcarriers, warp-shuffle reductions; the path's pair is the high
// half of its sorted path key.
template <int NP>
__global__ void __launch_bounds__(128) k_freq_vjp(const uint64_t* __restrict__ pkey, int64_t P,
                                                  const float2* __restrict__ a, const float* __restrict__ tau,
                                                  const double* __restrict__ freqs, int K,
                                                  const float2* __restrict__ gH, float2* __restrict__ ga,
                                                  float* __restrict__ gt) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i < P) {
        const int64_t pair = (int64_t)(pkey[i] >> 32);
        const float t = tau[i];
        float2 av[NP];
        for (int q = 0; q < NP; q++) av[q] = a[i * NP + q];
        float sr[NP], si[NP], sg = 0.0f;
        for (int q = 0; q < NP; q++) { sr[q] = 0.0f; si[q] = 0.0f; }
        // FV subcarriers per lane and step, their loads issued together
        constexpr int FV = 4;
        for (int k0 = lane; k0 < K; k0 += 32 * FV) {
            float fv[FV];
            float2 gv[FV][NP];
#pragma unroll
            for (int u = 0; u < FV; u++) {
                const int k = k0 + 32 * u;
                fv[u] = k < K ? (float)freqs[k] : 0.0f;
#pragma unroll
                for (int q = 0; q < NP; q++) gv[u][q] = k < K ? gH[(pair * NP + q) * K + k] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < FV; u++) {
                const float f = fv[u];
                float cyc = f * t;
                cyc -= rintf(cyc);
                float wi, wr;
                __sincosf(-2.0f * RT_PI_F * cyc, &wi, &wr);
                const float c = 2.0f * RT_PI_F * f;
                for (int q = 0; q < NP; q++) {
                    float2 g = gv[u][q];
                    // g * conj(w)
                    sr[q] += g.x * wr + g.y * wi;
                    si[q] += g.y * wr - g.x * wi;
                    // Re(conj(g) * a * (-j 2 pi f) * w): (-j c)(awr + j awi) = c awi - j c awr
                    float awr = av[q].x * wr - av[q].y * wi, awi = av[q].x * wi + av[q].y * wr;
                    sg += g.x * (c * awi) + g.y * (-c * awr);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            for (int q = 0; q < NP; q++) {
                sr[q] += __shfl_xor_sync(0xffffffffu, sr[q], o);
                si[q] += __shfl_xor_sync(0xffffffffu, si[q], o);
            }
            sg += __shfl_xor_sync(0xffffffffu, sg, o);
        }
        if (lane == 0) {
            for (int q = 0; q < NP; q++) ga[i * NP + q] = make_float2(sr[q], si[q]);
            gt[i] = sg;
        }
    }
}

// Sec. II-A (Listing 3, apply_doppler): time evolution from the devices'
// motion. Per path, the unit direction k_t in which it leaves the
// transmitter and k_r in which it reaches the receiver, from the image
// method at the current positions (the same construction as path_field);
// f_D = (v_tx . k_t - v_rx . k_r) / lambda (the rate of change of -length /
// lambda), stored as cycles per time step f_D / fs.
// Unit directions in which path i leaves its transmitter (kt) and reaches
// its receiver (kr), from the image method at the current positions (the
// same construction as path_field); t, r: the path's devices.
__device__ __forceinline__ void path_end_dirs(const CirParams& c, int64_t i, f3& kt, f3& kr, int& t, int& r) {
    t = c.pair_tx[2 * i];
    r = c.pair_tx[2 * i + 1];
    const f3 tx = mk(c.tx_pos[3 * t], c.tx_pos[3 * t + 1], c.tx_pos[3 * t + 2]);
    const f3 rx = mk(c.rx_pos[3 * r], c.rx_pos[3 * r + 1], c.rx_pos[3 * r + 2]);
    const int K = c.depth[i];
    const int32_t* ids = c.seq + i * c.D;
    f3 first = rx, last = tx;   // neighbours of the transmitter and the receiver along the path
    if (K > 0) {
        f3 I[RT_MAX_DEPTH + 1];
        I[0] = tx;
        for (int k = 1; k <= K; k++) {
            const float4 pl = __ldg(c.s.planes + ids[k - 1]);
            const f3 n = xyz(pl);
            I[k] = I[k - 1] - n * (2.0f * (dot(I[k - 1], n) - pl.w));
        }
        f3 q = rx;   // reflection points from the last one back
        for (int k = K; k >= 1; k--) {
            const float4 pl = __ldg(c.s.planes + ids[k - 1]);
            const f3 n = xyz(pl);
            const f3 dir = I[k] - q;
            q = q + dir * ((pl.w - dot(q, n)) / dot(dir, n));
            if (k == K) last = q;
            if (k == 1) first = q;
        }
    }
    kt = first - tx;
    kr = rx - last;
    kt = kt * (1.0f / sqrtf(dot(kt, kt)));
    kr = kr * (1.0f / sqrtf(dot(kr, kr)));
}

__global__ void k_doppler_shift(CirParams c, const float* __restrict__ vtx, const float* __restrict__ vrx,
                                double inv_lambda_fs, float* __restrict__ cyc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.P) return;
    f3 kt, kr;
    int t, r;
    path_end_dirs(c, i, kt, kr, t, r);
    double fd = (double)vtx[3 * t] * kt.x + (double)vtx[3 * t + 1] * kt.y + (double)vtx[3 * t + 2] * kt.z;
    if (vrx) fd -= (double)vrx[3 * r] * kr.x + (double)vrx[3 * r + 1] * kr.y + (double)vrx[3 * r + 2] * kr.z;
    cyc[i] = (float)(fd * inv_lambda_fs);
}

// Sec. II (synthetic arrays): the path directions in the devices' own frames,
// kt_l = R_tx^T kt and kr_l = R_rx^T kr, scaled by 1/lambda, so that an
// element at r (device frame) adds kt_l . r cycles (transmitter) or
// -kr_l . s cycles (receiver).
__global__ void k_array_dirs(CirParams c, float inv_lambda, float* __restrict__ dirs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.P) return;
    f3 kt, kr;
    int t, r;
    path_end_dirs(c, i, kt, kr, t, r);
    const Rot<float> Rt = rot_ypr(c.tx_ypr[3 * t], c.tx_ypr[3 * t + 1], c.tx_ypr[3 * t + 2]);
    const Rot<float> Rr = rot_ypr(c.rx_ypr[3 * r], c.rx_ypr[3 * r + 1], c.rx_ypr[3 * r + 2]);
    float* o = dirs + 6 * i;
    for (int k = 0; k < 3; k++) {
        o[k] = (Rt.m[0][k] * kt.x + Rt.m[1][k] * kt.y + Rt.m[2][k] * kt.z) * inv_lambda;
        o[3 + k] = (Rr.m[0][k] * kr.x + Rr.m[1][k] * kr.y + Rr.m[2][k] * kr.z) * inv_lambda;
    }
}

// a_el[i][n*nrp + p][m*ntp + q] = a[i][p][q] exp(j 2 pi (kt_l . r_m - kr_l . s_n)):
// one thread per output value, the transmit element and port fastest
__global__ void k_array_apply(const float2* __restrict__ a, const float* __restrict__ dirs, int64_t P, int nrp,
                              int ntp, const float* __restrict__ tel, int Mt, const float* __restrict__ rel, int Mr,
                              float2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cols = (int64_t)Mt * ntp, rows = (int64_t)Mr * nrp;
    if (e >= P * rows * cols) return;
    const int64_t i = e / (rows * cols);
    const int64_t rc = e - i * rows * cols;
    const int row = (int)(rc / cols), col = (int)(rc - (int64_t)row * cols);
    const int n = row / nrp, p = row - n * nrp, m = col / ntp, q = col - m * ntp;
    const float* d = dirs + 6 * i;
    float x = 0.0f;
    if (tel) x += d[0] * __ldg(tel + 3 * m) + d[1] * __ldg(tel + 3 * m + 1) + d[2] * __ldg(tel + 3 * m + 2);
    if (rel) x -= d[3] * __ldg(rel + 3 * n) + d[4] * __ldg(rel + 3 * n + 1) + d[5] * __ldg(rel + 3 * n + 2);
    x -= rintf(x);   // whole cycles dropped
    float sn, cs;
    sincospif(2.0f * x, &sn, &cs);
    const float2 v = a[(i * nrp + p) * ntp + q];
    out[e] = make_float2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

// a_t[i][q][n] = a[i][q] exp(j 2 pi n cyc_i): one thread per output value,
// consecutive threads on consecutive time steps (coalesced stores)
__global__ void k_doppler_apply(const float2* __restrict__ a, const float* __restrict__ cyc, int64_t P, int np,
                                int T, float2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = P * np * (int64_t)T;
    if (e >= total) return;
    const int64_t iq = e / T;
    const int n = (int)(e - iq * T);
    const int64_t i = iq / np;
    float x = cyc[i] * (float)n;
    x -= rintf(x);   // whole cycles dropped
    float sn, cs;
    sincospif(2.0f * x, &sn, &cs);
    const float2 v = a[iq];
    out[e] = make_float2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

CirParams make_cir(rt_ctx* ctx, uint32_t flags) {
    CirParams c;
    c.s = dev_scene(ctx);
    c.tx_pos = bp<float>(ctx->tx_pos);
    c.tx_ypr = bp<float>(ctx->tx_ypr);
    c.rx_pos = bp<float>(ctx->rx_pos);
    c.rx_ypr = bp<float>(ctx->rx_ypr);
    c.txa = ctx->tx_ant;
    c.rxa = ctx->rx_ant;
    c.seq = bp<int32_t>(ctx->path_seq);
    c.depth = bp<int32_t>(ctx->path_depth);
    c.len = bp<double>(ctx->path_len);
    c.pair_tx = bp<int32_t>(ctx->path_pair);
    c.D = ctx->max_depth;
    c.P = ctx->n_paths;
    c.lambda = RT_C0_D / ctx->fc;
    c.inv_we0 = (float)(1.0 / (2.0 * RT_PI_D * ctx->fc * RT_EPS0_D));
    c.flags = flags;
    return c;
}

template <int NP>
cudaError_t launch_freq(rt_ctx* ctx, const int64_t* off, const float* a, const float* tau, const double* freqs,
                        int K, float* H, int64_t n_pairs) {
    dim3 grid((unsigned)n_pairs, (unsigned)((K + HF_THREADS * HF_RUN - 1) / (HF_THREADS * HF_RUN)));
    cudaError_t e = cudaMemsetAsync(H, 0, sizeof(float2) * NP * (size_t)K * (size_t)n_pairs, ctx->stream);
    if (e != cudaSuccess) return e;
    prof_begin(ctx, "k_freq");
    k_freq<NP><<<grid, HF_THREADS, 0, ctx->stream>>>(off, (const float2*)a, tau, freqs, K, (float2*)H);
    prof_end(ctx);
    return cudaGetLastError();
}

template <int NP>
void launch_freq_vjp(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int K,
                     const float* gH, float* ga, float* gt, int64_t n_pairs) {
    (void)n_pairs;
    const int64_t P = ctx->n_paths;
    if (P <= 0) return;
    prof_begin(ctx, "k_freq_vjp");
    k_freq_vjp<NP><<<(unsigned)((P + 3) / 4), 128, 0, ctx->stream>>>(bp<uint64_t>(ctx->path_key), P, (const float2*)a,
                                                                     tau, freqs, K, (const float2*)gH, (float2*)ga,
                                                                     gt);
    prof_end(ctx);
}

}  // namespace

int cir_impl(rt_ctx* ctx, uint32_t flags, float* a, float* tau) {
    if (ctx->n_paths == 0) return RT_OK;
    CirParams c = make_cir(ctx, flags);
    prof_begin(ctx, "k_cir");
    k_cir<<<(unsigned)((c.P + 127) / 128), 128, 0, ctx->stream>>>(c, (float2*)a, tau);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int doppler_impl(rt_ctx* ctx, const float* a, const float* vtx, const float* vrx, double fs, int T, float* a_t) {
    const int64_t P = ctx->n_paths;
    if (P == 0) return RT_OK;
    CirParams c = make_cir(ctx, RT_LOS | RT_REFLECTION);
    const int np = ctx->tx_ant.n_ports * ctx->rx_ant.n_ports;
    RT_TRY(buf_reserve(ctx->dop_cyc, sizeof(float) * (size_t)P));
    prof_begin(ctx, "k_doppler_shift");
    k_doppler_shift<<<(unsigned)((P + 127) / 128), 128, 0, ctx->stream>>>(c, vtx, vrx, 1.0 / (c.lambda * fs),
                                                                          bp<float>(ctx->dop_cyc));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    const int64_t total = P * np * (int64_t)T;
    prof_begin(ctx, "k_doppler_apply");
    k_doppler_apply<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(
        (const float2*)a, bp<float>(ctx->dop_cyc), P, np, T, (float2*)a_t);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int array_impl(rt_ctx* ctx, const float* a, const float* tel, int Mt, const float* rel, int Mr, float* a_el) {
    const int64_t P = ctx->n_paths;
    if (P == 0) return RT_OK;
    CirParams c = make_cir(ctx, RT_LOS | RT_REFLECTION);
    RT_TRY(buf_reserve(ctx->arr_dirs, sizeof(float) * 6 * (size_t)P));
    prof_begin(ctx, "k_array_dirs");
    k_array_dirs<<<(unsigned)((P + 127) / 128), 128, 0, ctx->stream>>>(c, (float)(1.0 / c.lambda),
                                                                       bp<float>(ctx->arr_dirs));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    const int nrp = ctx->rx_ant.n_ports, ntp = ctx->tx_ant.n_ports;
    const int64_t total = P * (int64_t)Mr * nrp * (int64_t)Mt * ntp;
    prof_begin(ctx, "k_array_apply");
    k_array_apply<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(
        (const float2*)a, bp<float>(ctx->arr_dirs), P, nrp, ntp, tel, Mt, rel, Mr, (float2*)a_el);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int cir_vjp_impl(rt_ctx* ctx, uint32_t flags, const float* ga, const float* gtau, float* g_eps, float* g_sig,
                 float* g_pos, float* g_ypr) {
    if (ctx->n_paths == 0) return RT_OK;
    CirParams c = make_cir(ctx, flags);
    prof_begin(ctx, "k_cir_vjp");
    dim3 grid((unsigned)((c.P + 63) / 64), (unsigned)((6 + 2 * c.D + NT - 1) / NT));
    k_cir_vjp<<<grid, 64, 0, ctx->stream>>>(c, (const float2*)ga, gtau, g_eps, g_sig, g_pos, g_ypr);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

// H(f) over the CSR path list off [n_pairs+1] with np port pairs per path
// (1, 2 or 4): the context's own paths, or a caller's list.
int freq_csr_impl(rt_ctx* ctx, const int64_t* off, int64_t n_pairs, int np, const float* a, const float* tau,
                  const double* freqs, int K, float* H) {
    if (K <= 0 || n_pairs <= 0) return RT_OK;
    switch (np) {
        case 1: RT_TRY(launch_freq<1>(ctx, off, a, tau, freqs, K, H, n_pairs)); break;
        case 2: RT_TRY(launch_freq<2>(ctx, off, a, tau, freqs, K, H, n_pairs)); break;
        default: RT_TRY(launch_freq<4>(ctx, off, a, tau, freqs, K, H, n_pairs)); break;
    }
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int freq_impl(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int K, float* H,
              int64_t n_pairs) {
    return freq_csr_impl(ctx, bp<int64_t>(ctx->path_off), n_pairs, ctx->tx_ant.n_ports * ctx->rx_ant.n_ports, a,
                         tau, freqs, K, H);
}

// Per pair: incoherent path gain sum_paths sum_ports |a|^2 in dB, and whether
// the pair has any path (out [pair*2] = (has_path, gain dB or floor_db)).
__global__ void k_pair_gain(const int64_t* __restrict__ off, const float2* __restrict__ a, int np, int64_t n_pairs,
                            float floor_db, float* __restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pairs) return;
    double s = 0.0;
    for (int64_t i = off[q] * np; i < off[q + 1] * np; i++) {
        float2 v = a[i];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    out[2 * q] = s > 0.0 ? 1.0f : 0.0f;
    out[2 * q + 1] = s > 0.0 ? (float)(10.0 * log10(s)) : floor_db;
}

int pair_gain_impl(rt_ctx* ctx, const float* a, float floor_db, float* out, int64_t n_pairs) {
    if (n_pairs <= 0) return RT_OK;
    const int np = ctx->tx_ant.n_ports * ctx->rx_ant.n_ports;
    prof_begin(ctx, "k_pair_gain");
    k_pair_gain<<<(unsigned)((n_pairs + 255) / 256), 256, 0, ctx->stream>>>(bp<int64_t>(ctx->path_off),
                                                                            (const float2*)a, np, n_pairs, floor_db, out);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int freq_vjp_impl(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int K, const float* gH,
                  float* ga, float* gt, int64_t n_pairs) {
    if (K <= 0 || n_pairs <= 0) return RT_OK;
    const int np = ctx->tx_ant.n_ports * ctx->rx_ant.n_ports;
    switch (np) {
        case 1: launch_freq_vjp<1>(ctx, a, tau, freqs, K, gH, ga, gt, n_pairs); break;
        case 2: launch_freq_vjp<2>(ctx, a, tau, freqs, K, gH, ga, gt, n_pairs); break;
        default: launch_freq_vjp<4>(ctx, a, tau, freqs, K, gH, ga, gt, n_pairs); break;
    }
    RT_TRY(cudaGetLastError());
    return RT_OK;
}
