// rt_diff.cu -- first-order edge diffraction (Sec. II-B lists first-order
// diffraction among the features and leaves its equations to the
// documentation). Reading used here: the uniform geometrical theory of
// diffraction of Kouyoumjian and Pathak for perfectly conducting wedges.
//
// Wedges: scene edges shared by exactly two triangles whose planes differ
// (matched on the exact FP32 end points of the input vertices). The solid is
// the smaller of the two sectors the faces bound (convex edges), so the open
// exterior angle is n pi, n = 2 - alpha/pi. Face 0 is the triangle with the
// lower id; angles around the edge run from face 0 through the exterior.
//
// A diffracted path tx -> D -> rx touches the edge where the incidence and
// diffraction angles with the edge agree (Keller's law; on the edge line the
// point of shortest tx -> D -> rx). It is valid when D is strictly inside the
// edge, both devices lie in the exterior (0 < phi < n pi) and both segments
// are free of occluders (the wedge's own faces excepted).
//
// Coefficients (spherical incidence, ray-fixed bases):
//   a = lambda/(4 pi) exp(-j k (s' + s)) / sqrt(s s' (s' + s))
//       F_rx(-k_d) . [-D_s b0 b0'^T - D_h p p'^T] . F_tx(k_i),
//   p' = -(e x k_i)/|.|, b0' = p' x k_i, p = (e x k_d)/|.|, b0 = p x k_d,
//   D_{s,h} = -exp(-j pi/4) / (2 n sqrt(2 pi k) sin b) *
//     { cot((pi + b-)/2n) F(k L a+(b-)) + cot((pi - b-)/2n) F(k L a-(b-))
//       -/+ [cot((pi + b+)/2n) F(k L a+(b+)) + cot((pi - b+)/2n) F(k L a-(b+))] },
//   b-+ = phi -+ phi', L = s s' sin^2 b / (s + s'), a+-(x) = 2 cos^2((2 pi n N+- - x)/2)
//   with N+- the integers nearest (x +- pi)/(2 pi n), and the transition function
//   F(x) = 2 j sqrt(x) exp(j x) int_sqrt(x)^inf exp(-j t^2) dt.
// The coefficients run in FP64 (a few thousand paths); the path length and
// carrier phase in FP64 as for the specular paths.
#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "rt_field.cuh"
#include "rt_internal.h"

namespace {

// 64 B per wedge: (A, length), (e, n), (t0, face 0), (n0, face 1)
struct WedgeDev {
    float4 a, e, t0, n0;
};

// Receivers at the centres of a coverage-map grid (nx = 0: the context's receivers)
struct CellGrid {
    float x0, y0, cell, h;
    int nx, ny;
};

__device__ __forceinline__ f3 cell_centre(const CellGrid& g, int64_t r) {
    const int64_t iy = r / g.nx, ix = r - iy * g.nx;
    return mk(g.x0 + ((float)ix + 0.5f) * g.cell, g.y0 + ((float)iy + 0.5f) * g.cell, g.h);
}

struct DiffFind {
    DevScene s;
    const WedgeDev* w;
    int n_w;
    const float* tx_pos;
    const float* rx_pos;
    const int32_t* rx_off;   // [n_tx+1] or null
    int n_tx, n_rx;
    int64_t total;           // pairs * wedges
    CellGrid grid;           // receivers at cell centres when grid.nx > 0
    unsigned long long* count;
    unsigned long long cap;
    uint64_t* keys;          // pair << 32 | wedge
    float4* pts;             // diffraction points
};

__device__ __forceinline__ void pair_devices(const int32_t* rx_off, int n_tx, int n_rx, int64_t pair, int& t,
                                             int64_t& r) {
    if (rx_off) {
        int lo = 0, hi = n_tx;   // largest t with rx_off[t] <= pair
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rx_off[mid] <= pair) lo = mid; else hi = mid;
        }
        t = lo;
        r = pair;
    } else {
        t = (int)(pair / n_rx);
        r = pair - (int64_t)t * n_rx;
    }
}

// One thread per (pair, wedge): Keller point, exterior test, two segment
// occlusion tests; valid paths are appended (order fixed afterwards by a sort).
template <int LY>
__global__ void __launch_bounds__(256) k_diff_find(DiffFind p) {
    TravCount cnt;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.total;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pair = u / p.n_w;
        const int wi = (int)(u - pair * p.n_w);
        int t;
        int64_t r;
        pair_devices(p.rx_off, p.n_tx, p.n_rx, pair, t, r);
        const WedgeDev w = p.w[wi];
        const f3 A = xyz(w.a), e = xyz(w.e);
        const f3 tx = mk(p.tx_pos[3 * t], p.tx_pos[3 * t + 1], p.tx_pos[3 * t + 2]);
        const f3 rx = p.grid.nx > 0 ? cell_centre(p.grid, r)
                                    : mk(p.rx_pos[3 * r], p.rx_pos[3 * r + 1], p.rx_pos[3 * r + 2]);
        const float ts = dot(tx - A, e), tr = dot(rx - A, e);
        const f3 ps = tx - A - e * ts, pr = rx - A - e * tr;
        const float rs = sqrtf(dot(ps, ps)), rr = sqrtf(dot(pr, pr));
        if (!(rs + rr > 0.0f)) continue;
        const float tpar = ts + (tr - ts) * (rs / (rs + rr));
        if (!(tpar > 0.0f && tpar < w.a.w)) continue;
        const f3 D = A + e * tpar;
        // outside the solid: on the exterior side of face 0 (v . n0 > 0) or of
        // face 1, whose exterior normal is sin(n pi) t0 - cos(n pi) n0
        float sn, cn;
        sincospif(w.e.w, &sn, &cn);
        const f3 vt = tx - D, vr = rx - D;
        const float yt = dot(vt, xyz(w.n0)), yr = dot(vr, xyz(w.n0));
        const bool out_t = yt > 0.0f || sn * dot(vt, xyz(w.t0)) - cn * yt > 0.0f;
        const bool out_r = yr > 0.0f || sn * dot(vr, xyz(w.t0)) - cn * yr > 0.0f;
        if (!(out_t && out_r)) continue;
        const int f0 = __float_as_int(w.t0.w), f1 = __float_as_int(w.n0.w);
        f3 d = D - tx;
        float L = sqrtf(dot(d, d));
        if (any_hit<false, LY>(p.s, nullptr, 0, tx, d * (1.0f / L), L - p.s.tmin, f0, f1, cnt)) continue;
        d = rx - D;
        L = sqrtf(dot(d, d));
        if (any_hit<false, LY>(p.s, nullptr, 0, D, d * (1.0f / L), L - p.s.tmin, f0, f1, cnt)) continue;
        const unsigned long long k = atomicAdd(p.count, 1ull);
        if (k < p.cap) {
            p.keys[k] = ((uint64_t)pair << 32) | (uint64_t)wi;
            p.pts[k] = make_float4(D.x, D.y, D.z, 0.0f);
        }
    }
}

__global__ void k_diff_gather(const uint32_t* __restrict__ idx, const float4* __restrict__ in, int64_t n,
                              float4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}

__global__ void k_diff_off(const uint64_t* __restrict__ k, int64_t P, int64_t n_pairs, int64_t* __restrict__ off) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q > n_pairs) return;
    int64_t lo = 0, hi = P;
    const uint64_t want = (uint64_t)q << 32;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (k[mid] < want) lo = mid + 1; else hi = mid;
    }
    off[q] = lo;
}

// ---------------------------------------------------------------- coefficients
struct C64 {
    double re, im;
};
__device__ __forceinline__ C64 cmul(C64 a, C64 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C64 cscale(C64 a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ C64 cadd(C64 a, C64 b) { return {a.re + b.re, a.im + b.im}; }

// F(x) = 2 j sqrt(x) exp(j x) int_sqrt(x)^inf exp(-j t^2) dt for x >= 0.
// x < 16: the normalised Fresnel integrals from their power series in x
// (with z^2 = 2x/pi: C = z sum_{k even} (-1)^{k/2} x^k / (k! (2k+1)),
// S = z sum_{k odd} (-1)^{(k-1)/2} x^k / (k! (2k+1))), then
// int = sqrt(pi/2) ((1/2 - C) - j (1/2 - S)). x >= 16: the asymptotic series
// from repeated integration by parts, F = sum_k (2k-1)!! / (-2 j x)^k,
// summed while its terms decrease.
__device__ C64 transition_fn(double x) {
    if (!(x > 0.0)) return {0.0, 0.0};
    if (x < 16.0) {
        const double z = sqrt(2.0 * x / RT_PI_D);
        double pk = 1.0, C = 0.0, S = 0.0;   // pk = x^k / k!
        for (int k = 0; k < 80; k++) {
            const double term = pk / (2.0 * k + 1.0);
            switch (k & 3) {
                case 0: C += term; break;
                case 1: S += term; break;
                case 2: C -= term; break;
                default: S -= term; break;
            }
            pk *= x / (double)(k + 1);
            if (pk < 1e-18 * (fabs(C) + fabs(S) + 1e-300) && k > 4) break;
        }
        C *= z;
        S *= z;
        const double g = sqrt(RT_PI_D / 2.0);
        const C64 tail = {g * (0.5 - C), -g * (0.5 - S)};
        double sx, cx;
        sincos(x, &sx, &cx);
        const double u = sqrt(x);
        const C64 pre = {-2.0 * u * sx, 2.0 * u * cx};   // 2 j sqrt(x) exp(j x)
        return cmul(pre, tail);
    }
    C64 sum = {1.0, 0.0}, term = {1.0, 0.0};
    double last = 1.0;
    for (int k = 1; k < 40; k++) {
        // term *= (2k-1) / (-2 j x) = j (2k-1) / (2x)
        const double f = (2.0 * k - 1.0) / (2.0 * x);
        term = {-term.im * f, term.re * f};
        const double mag = fabs(term.re) + fabs(term.im);
        if (mag >= last) break;
        sum = cadd(sum, term);
        last = mag;
        if (mag < 1e-17) break;
    }
    return sum;
}

__device__ __forceinline__ double a_pm(double x, double n, int sign) {
    const double N = rint((x + sign * RT_PI_D) / (2.0 * RT_PI_D * n));
    const double c = cos((2.0 * RT_PI_D * n * N - x) / 2.0);
    return 2.0 * c * c;
}

// cot((pi + sign x) / (2n)) F(k L a(x)); 0 on a shadow or reflection
// boundary itself (a set of measure zero)
__device__ __forceinline__ C64 utd_term(double x, double n, int sign, double kL) {
    const double arg = (RT_PI_D + sign * x) / (2.0 * n);
    double sa, ca;
    sincos(arg, &sa, &ca);
    if (fabs(sa) < 1e-12) return {0.0, 0.0};
    return cscale(transition_fn(kL * a_pm(x, n, sign)), ca / sa);
}

struct DiffField {
    const WedgeDev* w;
    const uint64_t* keys;
    const float4* pts;
    int64_t P;
    const float* tx_pos;
    const float* tx_ypr;
    const float* rx_pos;
    const float* rx_ypr;
    const int32_t* rx_off;
    int n_tx, n_rx;
    DevAntenna txa, rxa;
    double lambda;
    CellGrid grid;   // map mode when grid.nx > 0: receiver port 0, unrotated, at the cell centres
    int tx_port;     // map mode: the transmit port
    float* map;      // map mode: [n_tx][ny][nx] sum of |a|^2
};

// Four lanes per path: lane j evaluates one of the four cot * F terms (the
// FP64 transition function is the long part), a shuffle sums them, lane 0
// finishes the path.
__global__ void __launch_bounds__(64) k_diff_field(DiffField c, float2* __restrict__ a_out, float* __restrict__ tau) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
    const int sub = threadIdx.x & 3;
    const bool live = i0 < c.P;
    const int64_t i = live ? i0 : c.P - 1;   // lanes past the end repeat the last path and write nothing
    const uint64_t key = c.keys[i];
    const int64_t pair = (int64_t)(key >> 32);
    const WedgeDev w = c.w[key & 0xFFFFFFFFull];
    int t;
    int64_t r;
    pair_devices(c.rx_off, c.n_tx, c.n_rx, pair, t, r);
    const float4 Dp = c.pts[i];
    const double D[3] = {Dp.x, Dp.y, Dp.z};
    const double tx[3] = {c.tx_pos[3 * t], c.tx_pos[3 * t + 1], c.tx_pos[3 * t + 2]};
    const bool map = c.grid.nx > 0;
    f3 rxf = map ? cell_centre(c.grid, r) : mk(c.rx_pos[3 * r], c.rx_pos[3 * r + 1], c.rx_pos[3 * r + 2]);
    const double rx[3] = {rxf.x, rxf.y, rxf.z};
    double ki[3], kd[3];
    for (int q = 0; q < 3; q++) { ki[q] = D[q] - tx[q]; kd[q] = rx[q] - D[q]; }
    const double sp = sqrt(ki[0] * ki[0] + ki[1] * ki[1] + ki[2] * ki[2]);
    const double s = sqrt(kd[0] * kd[0] + kd[1] * kd[1] + kd[2] * kd[2]);
    for (int q = 0; q < 3; q++) { ki[q] /= sp; kd[q] /= s; }
    const double e[3] = {w.e.x, w.e.y, w.e.z};
    auto cross = [](const double* a, const double* b, double* o) {
        o[0] = a[1] * b[2] - a[2] * b[1];
        o[1] = a[2] * b[0] - a[0] * b[2];
        o[2] = a[0] * b[1] - a[1] * b[0];
    };
    double pp[3], bp[3], ph[3], bd[3];
    cross(e, ki, pp);
    const double sin_b = sqrt(pp[0] * pp[0] + pp[1] * pp[1] + pp[2] * pp[2]);
    for (int q = 0; q < 3; q++) pp[q] = -pp[q] / sin_b;
    cross(pp, ki, bp);
    cross(e, kd, ph);
    const double nph = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
    for (int q = 0; q < 3; q++) ph[q] /= nph;
    cross(ph, kd, bd);
    // angles around the edge from face 0 through the exterior
    auto angle = [&](const double* X) {
        const double v[3] = {X[0] - D[0], X[1] - D[1], X[2] - D[2]};
        double a = atan2(v[0] * w.n0.x + v[1] * w.n0.y + v[2] * w.n0.z, v[0] * w.t0.x + v[1] * w.t0.y + v[2] * w.t0.z);
        return a < 0.0 ? a + 2.0 * RT_PI_D : a;
    };
    const double phi = angle(rx), phip = angle(tx), n = w.e.w;
    const double k = 2.0 * RT_PI_D / c.lambda;
    const double kL = k * s * sp * sin_b * sin_b / (s + sp);
    // terms: 0: (phi - phi', +), 1: (phi - phi', -), 2: (phi + phi', +), 3: (phi + phi', -)
    const C64 term = utd_term(sub < 2 ? phi - phip : phi + phip, n, (sub & 1) ? -1 : +1, kL);
    const unsigned full = 0xffffffffu;
    C64 pair_sum = {term.re + __shfl_xor_sync(full, term.re, 1), term.im + __shfl_xor_sync(full, term.im, 1)};
    const C64 other = {__shfl_xor_sync(full, pair_sum.re, 2), __shfl_xor_sync(full, pair_sum.im, 2)};
    if (!live || sub != 0) return;
    const C64 d1 = pair_sum, d2 = other;   // lane 0 holds terms 0 + 1, lane 2 terms 2 + 3
    // pre = -exp(-j pi/4) / (2 n sqrt(2 pi k) sin b)
    const double m = 1.0 / (2.0 * n * sqrt(2.0 * RT_PI_D * k) * sin_b);
    const C64 pre = {-m * 0.70710678118654752, m * 0.70710678118654752};
    const C64 Ds = cmul(pre, {d1.re - d2.re, d1.im - d2.im});
    const C64 Dh = cmul(pre, cadd(d1, d2));
    // amplitude and carrier phase (path length in FP64, phase reduced modulo 2 pi)
    const double len = s + sp;
    const double cyc = len / c.lambda;
    double sph, cph;
    sincos(-2.0 * RT_PI_D * (cyc - floor(cyc)), &sph, &cph);
    const double amp = c.lambda / (4.0 * RT_PI_D) / sqrt(s * sp * len);
    const C64 ea = {amp * cph, amp * sph};
    const Rot<float> Rt = rot_ypr(c.tx_ypr[3 * t], c.tx_ypr[3 * t + 1], c.tx_ypr[3 * t + 2]);
    const Rot<float> Rr = map ? rot_ypr(0.0f, 0.0f, 0.0f) : rot_ypr(c.rx_ypr[3 * r], c.rx_ypr[3 * r + 1], c.rx_ypr[3 * r + 2]);
    const V3<float> ui = {(float)ki[0], (float)ki[1], (float)ki[2]};
    const V3<float> ud = {(float)-kd[0], (float)-kd[1], (float)-kd[2]};
    const int ntp = c.txa.n_ports, nrp = map ? 1 : c.rxa.n_ports;
    for (int q = map ? c.tx_port : 0; q < (map ? c.tx_port + 1 : ntp); q++) {
        const V3<float> ft = antenna_vec<float>(c.txa.kind, c.txa.slant[q], Rt, ui);
        // projections of the transmit pattern on the incident basis
        const double fbp = ft.x * bp[0] + ft.y * bp[1] + ft.z * bp[2];
        const double fpp = ft.x * pp[0] + ft.y * pp[1] + ft.z * pp[2];
        for (int pq = 0; pq < nrp; pq++) {
            const V3<float> fr = antenna_vec<float>(c.rxa.kind, c.rxa.slant[pq], Rr, ud);
            const double rbd = fr.x * bd[0] + fr.y * bd[1] + fr.z * bd[2];
            const double rph = fr.x * ph[0] + fr.y * ph[1] + fr.z * ph[2];
            // F_rx . (-Ds bd bp^T - Dh ph pp^T) . F_tx
            const C64 v = cadd(cscale(Ds, -rbd * fbp), cscale(Dh, -rph * fpp));
            const C64 av = cmul(ea, v);
            if (map)
                atomicAdd(c.map + (size_t)t * c.grid.nx * c.grid.ny + r, (float)(av.re * av.re + av.im * av.im));
            else
                a_out[(i * nrp + pq) * ntp + q] = make_float2((float)av.re, (float)av.im);
        }
    }
    if (!map) tau[i] = (float)(len / RT_C0_D);
}

}  // namespace

// Wedges of the current scene, built on the host from the input vertices the
// first time diffraction is asked for after a scene load.
static int build_wedges(rt_ctx* ctx) {
    if (ctx->wedge_gen == ctx->scene_gen) return RT_OK;
    const int T = ctx->n_tris;
    std::vector<float> v(9 * (size_t)std::max(T, 1));
    if (T > 0) {
        RT_TRY(cudaMemcpyAsync(v.data(), ctx->verts_in.p, sizeof(float) * 9 * (size_t)T, cudaMemcpyDeviceToHost,
                               ctx->stream));
        RT_TRY(cudaStreamSynchronize(ctx->stream));
    }
    std::map<std::array<float, 6>, std::vector<std::pair<int, int>>> table;   // edge -> (triangle, opposite vertex)
    for (int t = 0; t < T; t++)
        for (int k = 0; k < 3; k++) {
            const float* p = &v[9 * (size_t)t + 3 * k];
            const float* q = &v[9 * (size_t)t + 3 * ((k + 1) % 3)];
            std::array<float, 3> a = {p[0], p[1], p[2]}, b = {q[0], q[1], q[2]};
            if (b < a) std::swap(a, b);
            table[{a[0], a[1], a[2], b[0], b[1], b[2]}].push_back({t, (k + 2) % 3});
        }
    struct Rec {
        int f0, f1;
        WedgeDev w;
    };
    std::vector<Rec> recs;
    for (auto& kv : table) {
        if (kv.second.size() != 2) continue;
        auto f = kv.second;
        std::sort(f.begin(), f.end());
        const double A[3] = {kv.first[0], kv.first[1], kv.first[2]};
        const double B[3] = {kv.first[3], kv.first[4], kv.first[5]};
        double e[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double L = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        if (!(L > 0.0)) continue;
        for (double& x : e) x /= L;
        auto inward = [&](int t, int k, double* o) {
            const float* c = &v[9 * (size_t)t + 3 * k];
            double d[3] = {c[0] - A[0], c[1] - A[1], c[2] - A[2]};
            const double de = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
            for (int q = 0; q < 3; q++) d[q] -= de * e[q];
            const double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int q = 0; q < 3; q++) o[q] = d[q] / nd;
        };
        double t0[3], t1[3];
        inward(f[0].first, f[0].second, t0);
        inward(f[1].first, f[1].second, t1);
        const double c01 = std::max(-1.0, std::min(1.0, t0[0] * t1[0] + t0[1] * t1[1] + t0[2] * t1[2]));
        const double alpha = std::acos(c01);
        if (alpha > RT_PI_D - 1e-6) continue;   // coplanar faces
        double n0[3] = {e[1] * t0[2] - e[2] * t0[1], e[2] * t0[0] - e[0] * t0[2], e[0] * t0[1] - e[1] * t0[0]};
        if (n0[0] * t1[0] + n0[1] * t1[1] + n0[2] * t1[2] > 0.0)
            for (double& x : n0) x = -x;
        Rec r;
        r.f0 = f[0].first;
        r.f1 = f[1].first;
        r.w.a = make_float4((float)A[0], (float)A[1], (float)A[2], (float)L);
        r.w.e = make_float4((float)e[0], (float)e[1], (float)e[2], (float)(2.0 - alpha / RT_PI_D));
        float i0, i1;
        memcpy(&i0, &r.f0, 4);
        memcpy(&i1, &r.f1, 4);
        r.w.t0 = make_float4((float)t0[0], (float)t0[1], (float)t0[2], i0);
        r.w.n0 = make_float4((float)n0[0], (float)n0[1], (float)n0[2], i1);
        recs.push_back(r);
    }
    std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
        return a.f0 != b.f0 ? a.f0 < b.f0 : a.f1 < b.f1;
    });
    std::vector<WedgeDev> wd(recs.size());
    for (size_t i = 0; i < recs.size(); i++) wd[i] = recs[i].w;
    RT_TRY(buf_reserve(ctx->wedges, sizeof(WedgeDev) * std::max<size_t>(wd.size(), 1)));
    if (!wd.empty())
        RT_TRY(cudaMemcpy(ctx->wedges.p, wd.data(), sizeof(WedgeDev) * wd.size(), cudaMemcpyHostToDevice));
    ctx->n_wedges = (int)wd.size();
    ctx->wedge_gen = ctx->scene_gen;
    return RT_OK;
}

int diffraction_impl(rt_ctx* ctx, int64_t* n_out) {
    {
        const int eb = build_wedges(ctx);
        if (eb) return eb;
    }
    cudaStream_t st = ctx->stream;
    const int64_t n_pairs = ctx->rx_sets ? (int64_t)ctx->rx_off[ctx->n_tx] : (int64_t)ctx->n_tx * ctx->n_rx;
    const int64_t total = n_pairs * ctx->n_wedges;
    ctx->n_dpaths = 0;
    *n_out = 0;
    RT_TRY(buf_reserve(ctx->dpath_off, sizeof(int64_t) * (n_pairs + 1)));
    RT_TRY(cudaMemsetAsync(ctx->dpath_off.p, 0, sizeof(int64_t) * (n_pairs + 1), st));
    if (total == 0) return RT_OK;
    DiffFind p;
    p.s = dev_scene(ctx);
    p.w = bp<WedgeDev>(ctx->wedges);
    p.n_w = ctx->n_wedges;
    p.tx_pos = bp<float>(ctx->tx_pos);
    p.rx_pos = bp<float>(ctx->rx_pos);
    p.rx_off = ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr;
    p.n_tx = ctx->n_tx;
    p.n_rx = ctx->n_rx;
    p.total = total;
    p.grid = CellGrid{0.0f, 0.0f, 0.0f, 0.0f, 0, 0};
    unsigned long long cap = std::max<unsigned long long>(1ull << 14, (unsigned long long)ctx->dpath_cap);
    unsigned long long found = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        RT_TRY(buf_reserve(ctx->dpath_raw_key, sizeof(uint64_t) * cap));
        RT_TRY(buf_reserve(ctx->dpath_raw_pt, sizeof(float4) * cap));
        RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), st));
        p.count = bp<unsigned long long>(ctx->counters);
        p.cap = cap;
        p.keys = bp<uint64_t>(ctx->dpath_raw_key);
        p.pts = bp<float4>(ctx->dpath_raw_pt);
        const int64_t grid = std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->num_sms);
        prof_begin(ctx, "k_diff_find");
        (wide_layout(ctx) ? k_diff_find<8> : k_diff_find<2>)<<<(unsigned)grid, 256, 0, st>>>(p);
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
        RT_TRY(cudaMemcpyAsync(ctx->host_rb, ctx->counters.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaStreamSynchronize(st));
        found = ctx->host_rb[0];
        if (found <= cap) break;
        cap = found;   // grow and trace again
    }
    ctx->dpath_cap = (int64_t)cap;
    if (found > cap) return set_err(ctx, RT_ERR_CUDA, "compute_diffraction: path count changed between passes");
    const int64_t P = (int64_t)found;
    if (P == 0) return RT_OK;
    // order: (pair, wedge); positions carried along and gathered
    RT_TRY(buf_reserve(ctx->dpath_key, sizeof(uint64_t) * P));
    RT_TRY(buf_reserve(ctx->dpath_key_alt, sizeof(uint64_t) * P));
    RT_TRY(buf_reserve(ctx->dpath_idx, sizeof(uint32_t) * P));
    RT_TRY(buf_reserve(ctx->dpath_idx_alt, sizeof(uint32_t) * P));
    RT_TRY(buf_reserve(ctx->dpath_pt, sizeof(float4) * P));
    RT_TRY(cudaMemcpyAsync(ctx->dpath_key.p, ctx->dpath_raw_key.p, sizeof(uint64_t) * P, cudaMemcpyDeviceToDevice, st));
    std::vector<uint32_t> iota(P);
    for (int64_t i = 0; i < P; i++) iota[i] = (uint32_t)i;
    RT_TRY(cudaMemcpyAsync(ctx->dpath_idx.p, iota.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, st));
    int pair_bits = 1;
    while ((1ll << pair_bits) < std::max<int64_t>(n_pairs, 2)) pair_bits++;
    RT_TRY(radix_sort64(ctx, bp<uint64_t>(ctx->dpath_key), bp<uint64_t>(ctx->dpath_key_alt), bp<uint32_t>(ctx->dpath_idx),
                        bp<uint32_t>(ctx->dpath_idx_alt), P, 32 + pair_bits));
    prof_begin(ctx, "k_diff_gather");
    k_diff_gather<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(bp<uint32_t>(ctx->dpath_idx),
                                                                bp<float4>(ctx->dpath_raw_pt), P,
                                                                bp<float4>(ctx->dpath_pt));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    prof_begin(ctx, "k_diff_off");
    k_diff_off<<<(unsigned)((n_pairs + 256) / 256), 256, 0, st>>>(bp<uint64_t>(ctx->dpath_key), P, n_pairs,
                                                                  bp<int64_t>(ctx->dpath_off));
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    RT_TRY(cudaStreamSynchronize(st));   // the host copy of the initial order is released here
    ctx->n_dpaths = P;
    *n_out = P;
    return RT_OK;
}

int diffraction_cir_impl(rt_ctx* ctx, float* a, float* tau) {
    const int64_t P = ctx->n_dpaths;
    if (P == 0) return RT_OK;
    DiffField c;
    c.w = bp<WedgeDev>(ctx->wedges);
    c.keys = bp<uint64_t>(ctx->dpath_key);
    c.pts = bp<float4>(ctx->dpath_pt);
    c.P = P;
    c.tx_pos = bp<float>(ctx->tx_pos);
    c.tx_ypr = bp<float>(ctx->tx_ypr);
    c.rx_pos = bp<float>(ctx->rx_pos);
    c.rx_ypr = bp<float>(ctx->rx_ypr);
    c.rx_off = ctx->rx_sets ? bp<int32_t>(ctx->rx_off_d) : nullptr;
    c.n_tx = ctx->n_tx;
    c.n_rx = ctx->n_rx;
    c.txa = ctx->tx_ant;
    c.rxa = ctx->rx_ant;
    c.lambda = RT_C0_D / ctx->fc;
    c.grid = CellGrid{0.0f, 0.0f, 0.0f, 0.0f, 0, 0};
    c.tx_port = 0;
    c.map = nullptr;
    prof_begin(ctx, "k_diff_field");
    k_diff_field<<<(unsigned)((4 * P + 63) / 64), 64, 0, ctx->stream>>>(c, (float2*)a, tau);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}

int diffraction_get_impl(rt_ctx* ctx, int64_t* offsets, int32_t* wedge, float* points) {
    const int64_t P = ctx->n_dpaths;
    const int64_t n_pairs = ctx->rx_sets ? (int64_t)ctx->rx_off[ctx->n_tx] : (int64_t)ctx->n_tx * ctx->n_rx;
    cudaStream_t st = ctx->stream;
    if (offsets)
        RT_TRY(cudaMemcpyAsync(offsets, ctx->dpath_off.p, sizeof(int64_t) * (n_pairs + 1), cudaMemcpyDeviceToDevice, st));
    if (P == 0) return RT_OK;
    if (wedge)   // low halves of the keys
        RT_TRY(cudaMemcpy2DAsync(wedge, sizeof(int32_t), ctx->dpath_key.p, sizeof(uint64_t), sizeof(int32_t), P,
                                 cudaMemcpyDeviceToDevice, st));
    if (points)
        RT_TRY(cudaMemcpy2DAsync(points, 3 * sizeof(float), ctx->dpath_pt.p, sizeof(float4), 3 * sizeof(float), P,
                                 cudaMemcpyDeviceToDevice, st));
    return RT_OK;
}

int wedges_impl(rt_ctx* ctx, int64_t* n_out, int32_t* faces, float* n_ext) {
    {
        const int eb = build_wedges(ctx);
        if (eb) return eb;
    }
    *n_out = ctx->n_wedges;
    if (ctx->n_wedges == 0) return RT_OK;
    std::vector<WedgeDev> wd(ctx->n_wedges);
    RT_TRY(cudaMemcpyAsync(wd.data(), ctx->wedges.p, sizeof(WedgeDev) * wd.size(), cudaMemcpyDeviceToHost,
                           ctx->stream));
    RT_TRY(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> f(2 * wd.size());
    std::vector<float> n(wd.size());
    for (size_t i = 0; i < wd.size(); i++) {
        memcpy(&f[2 * i], &wd[i].t0.w, 4);
        memcpy(&f[2 * i + 1], &wd[i].n0.w, 4);
        n[i] = wd[i].e.w;
    }
    if (faces)
        RT_TRY(cudaMemcpyAsync(faces, f.data(), sizeof(int32_t) * f.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (n_ext)
        RT_TRY(cudaMemcpyAsync(n_ext, n.data(), sizeof(float) * n.size(), cudaMemcpyHostToDevice, ctx->stream));
    RT_TRY(cudaStreamSynchronize(ctx->stream));
    return RT_OK;
}

// Diffracted coverage map: every transmitter against every cell centre
// (receiver port 0, unrotated, as the specular map), the incoherent sum of
// |a|^2 of its first-order diffracted paths; gain [n_tx*ny*nx] overwritten.
int diffraction_map_impl(rt_ctx* ctx, const rt_grid* g, int tx_port, float* gain) {
    {
        const int eb = build_wedges(ctx);
        if (eb) return eb;
    }
    cudaStream_t st = ctx->stream;
    const int64_t cells = (int64_t)g->nx * g->ny;
    RT_TRY(cudaMemsetAsync(gain, 0, sizeof(float) * cells * ctx->n_tx, st));
    const int64_t n_pairs = cells * ctx->n_tx;
    const int64_t total = n_pairs * ctx->n_wedges;
    if (total == 0) return RT_OK;
    const CellGrid grid{g->x0, g->y0, g->cell, g->height, g->nx, g->ny};
    DiffFind p;
    p.s = dev_scene(ctx);
    p.w = bp<WedgeDev>(ctx->wedges);
    p.n_w = ctx->n_wedges;
    p.tx_pos = bp<float>(ctx->tx_pos);
    p.rx_pos = nullptr;
    p.rx_off = nullptr;
    p.n_tx = ctx->n_tx;
    p.n_rx = (int)cells;
    p.total = total;
    p.grid = grid;
    unsigned long long cap = std::max<unsigned long long>(1ull << 16, (unsigned long long)ctx->dmap_cap);
    unsigned long long found = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        RT_TRY(buf_reserve(ctx->dmap_key, sizeof(uint64_t) * cap));
        RT_TRY(buf_reserve(ctx->dmap_pt, sizeof(float4) * cap));
        RT_TRY(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), st));
        p.count = bp<unsigned long long>(ctx->counters);
        p.cap = cap;
        p.keys = bp<uint64_t>(ctx->dmap_key);
        p.pts = bp<float4>(ctx->dmap_pt);
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->num_sms);
        prof_begin(ctx, "k_diff_find");
        (wide_layout(ctx) ? k_diff_find<8> : k_diff_find<2>)<<<(unsigned)blocks, 256, 0, st>>>(p);
        prof_end(ctx);
        RT_TRY(cudaGetLastError());
        RT_TRY(cudaMemcpyAsync(ctx->host_rb, ctx->counters.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaStreamSynchronize(st));
        found = ctx->host_rb[0];
        if (found <= cap) break;
        cap = found;
    }
    ctx->dmap_cap = (int64_t)cap;
    if (found > cap) return set_err(ctx, RT_ERR_CUDA, "coverage_map_diffraction: path count changed between passes");
    if (found == 0) return RT_OK;
    DiffField c;
    c.w = bp<WedgeDev>(ctx->wedges);
    c.keys = bp<uint64_t>(ctx->dmap_key);
    c.pts = bp<float4>(ctx->dmap_pt);
    c.P = (int64_t)found;
    c.tx_pos = bp<float>(ctx->tx_pos);
    c.tx_ypr = bp<float>(ctx->tx_ypr);
    c.rx_pos = nullptr;
    c.rx_ypr = nullptr;
    c.rx_off = nullptr;
    c.n_tx = ctx->n_tx;
    c.n_rx = (int)cells;
    c.txa = ctx->tx_ant;
    c.rxa = ctx->rx_ant;
    c.lambda = RT_C0_D / ctx->fc;
    c.grid = grid;
    c.tx_port = tx_port;
    c.map = gain;
    prof_begin(ctx, "k_diff_field");
    k_diff_field<<<(unsigned)((4 * c.P + 63) / 64), 64, 0, st>>>(c, nullptr, nullptr);
    prof_end(ctx);
    RT_TRY(cudaGetLastError());
    return RT_OK;
}
