// rt_field.cuh -- polarized field along a specular path in FP32, written
// once over a scalar type S: `float` for the forward kernels and Dual<N>
// (value + N tangents) for the replayed vector-Jacobian products.
//
// Sec. II of the paper: the polarized field components are transformed at
// every interaction (reflection) and combined with the antenna patterns into
// channel coefficients; the formulas are the textbook ones:
//   device rotation  R = Rz(yaw) Ry(pitch) Rx(roll) (3GPP TR 38.901 Sec. 7.1)
//   pattern vector   F = R (C_theta theta_hat + C_phi phi_hat) at the local
//                    direction R^T u; C = g (cos zeta, sin zeta) for slant zeta
//   gains            iso g = 1; short dipole g = sqrt(1.5) sin theta;
//                    TR 38.901 Table 7.3-1: A_V = -min(12((theta-90)/65)^2, 30),
//                    A_H = -min(12(phi/65)^2, 30), A = -min(-(A_V + A_H), 30),
//                    g = 10^((8 + A)/20)
//   reflection       eta = eps_r - j sigma/(omega eps0), c = cos(theta_i),
//                    r_perp = (c - sqrt(eta - s^2))/(c + sqrt(eta - s^2)),
//                    r_par = (eta c - sqrt(eta - s^2))/(eta c + sqrt(eta - s^2)),
//                    E' = r_perp (E.e_perp) e_perp + r_par (E.e_par_i) e_par_r,
//                    e_perp = ki x n / |ki x n|, e_par = e_perp x k.
#pragma once
#include "../../include/rt.h"
#include "rt_common.cuh"

// ---------------------------------------------------------------- dual numbers
template <int N>
struct Dual {
    float v;
    float d[N];
};
template <int N>
__device__ __forceinline__ Dual<N> dconst(float v) {
    Dual<N> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = 0.0f;
    return r;
}
#define DUAL_BIN(OP, VEXPR, DEXPR)                                                   \
    template <int N>                                                                 \
    __device__ __forceinline__ Dual<N> operator OP(const Dual<N>& a, const Dual<N>& b) { \
        Dual<N> r;                                                                   \
        r.v = VEXPR;                                                                 \
        _Pragma("unroll") for (int i = 0; i < N; i++) r.d[i] = DEXPR;               \
        return r;                                                                    \
    }
DUAL_BIN(+, a.v + b.v, a.d[i] + b.d[i])
DUAL_BIN(-, a.v - b.v, a.d[i] - b.d[i])
DUAL_BIN(*, a.v * b.v, a.d[i] * b.v + a.v * b.d[i])
#undef DUAL_BIN
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    float ib = 1.0f / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, float s) {
    Dual<N> r;
    r.v = a.v * s;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * s;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(float s, const Dual<N>& a) { return a * s; }
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, float s) { Dual<N> r = a; r.v += s; return r; }
template <int N>
__device__ __forceinline__ Dual<N> operator+(float s, const Dual<N>& a) { return a + s; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, float s) { Dual<N> r = a; r.v -= s; return r; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(float s, const Dual<N>& a) {
    Dual<N> r;
    r.v = s - a.v;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = -a.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) { return 0.0f - a; }

// scalar functions on float and Dual
__device__ __forceinline__ float val(float a) { return a; }
template <int N>
__device__ __forceinline__ float val(const Dual<N>& a) { return a.v; }
__device__ __forceinline__ float s_sqrt(float a) { return sqrtf(a); }
template <int N>
__device__ __forceinline__ Dual<N> s_sqrt(const Dual<N>& a) {
    Dual<N> r;
    r.v = sqrtf(a.v);
    float h = r.v > 0.0f ? 0.5f / r.v : 0.0f;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = a.d[i] * h;
    return r;
}
__device__ __forceinline__ float s_sin(float a) { return sinf(a); }
__device__ __forceinline__ float s_cos(float a) { return cosf(a); }
template <int N>
__device__ __forceinline__ Dual<N> s_sin(const Dual<N>& a) {
    Dual<N> r;
    float s, c;
    sincosf(a.v, &s, &c);
    r.v = s;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = c * a.d[i];
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> s_cos(const Dual<N>& a) {
    Dual<N> r;
    float s, c;
    sincosf(a.v, &s, &c);
    r.v = c;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = -s * a.d[i];
    return r;
}
__device__ __forceinline__ float s_atan2(float y, float x) { return atan2f(y, x); }
template <int N>
__device__ __forceinline__ Dual<N> s_atan2(const Dual<N>& y, const Dual<N>& x) {
    Dual<N> r;
    r.v = atan2f(y.v, x.v);
    float q = x.v * x.v + y.v * y.v;
    float iq = q > 0.0f ? 1.0f / q : 0.0f;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * iq;
    return r;
}
__device__ __forceinline__ float s_exp10(float a) { return exp10f(a); }
template <int N>
__device__ __forceinline__ Dual<N> s_exp10(const Dual<N>& a) {
    Dual<N> r;
    r.v = exp10f(a.v);
    float k = r.v * 2.302585093f;
#pragma unroll
    for (int i = 0; i < N; i++) r.d[i] = k * a.d[i];
    return r;
}
template <class S>
__device__ __forceinline__ S s_min(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }
// x with its value replaced by v (tangents kept)
__device__ __forceinline__ float with_value(float, float v) { return v; }
template <int N>
__device__ __forceinline__ Dual<N> with_value(Dual<N> x, float v) {
    x.v = v;
    return x;
}
template <class S>
struct SConst {
    __device__ static S make(float v);
};
template <>
struct SConst<float> {
    __device__ __forceinline__ static float make(float v) { return v; }
};
template <int N>
struct SConst<Dual<N>> {
    __device__ __forceinline__ static Dual<N> make(float v) { return dconst<N>(v); }
};

// ------------------------------------------------------------- vectors, complex
template <class S>
struct V3 {
    S x, y, z;
};
template <class S>
__device__ __forceinline__ V3<S> v_add(const V3<S>& a, const V3<S>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S>
__device__ __forceinline__ V3<S> v_sub(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S, class T>
__device__ __forceinline__ V3<S> v_scale(const V3<S>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class S>
__device__ __forceinline__ S v_dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S>
__device__ __forceinline__ V3<S> v_cross(const V3<S>& a, const V3<S>& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S>
__device__ __forceinline__ V3<S> v_const(f3 a) {
    return {SConst<S>::make(a.x), SConst<S>::make(a.y), SConst<S>::make(a.z)};
}
template <class S>
__device__ __forceinline__ f3 v_val(const V3<S>& a) { return {val(a.x), val(a.y), val(a.z)}; }
template <class S>
__device__ __forceinline__ V3<S> v_unit(const V3<S>& a) {
    S n = s_sqrt(v_dot(a, a));
    S inv = SConst<S>::make(1.0f) / n;
    return v_scale(a, inv);
}

template <class S>
struct Cx {
    S re, im;
};
template <class S>
__device__ __forceinline__ Cx<S> c_add(const Cx<S>& a, const Cx<S>& b) { return {a.re + b.re, a.im + b.im}; }
template <class S>
__device__ __forceinline__ Cx<S> c_sub(const Cx<S>& a, const Cx<S>& b) { return {a.re - b.re, a.im - b.im}; }
template <class S>
__device__ __forceinline__ Cx<S> c_mul(const Cx<S>& a, const Cx<S>& b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class S>
__device__ __forceinline__ Cx<S> c_scale(const Cx<S>& a, const S& s) { return {a.re * s, a.im * s}; }
template <class S>
__device__ __forceinline__ Cx<S> c_div(const Cx<S>& a, const Cx<S>& b) {
    S den = b.re * b.re + b.im * b.im;
    S inv = SConst<S>::make(1.0f) / den;
    return {(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}
// principal square root for Re(z) > 0 (eta - sin^2 with eps_r >= 1)
template <class S>
__device__ __forceinline__ Cx<S> c_sqrt(const Cx<S>& z) {
    S r = s_sqrt(z.re * z.re + z.im * z.im);
    S re = s_sqrt((r + z.re) * 0.5f);
    S im = z.im / (re * 2.0f);
    return {re, im};
}

// --------------------------------------------------------------------- antennas
template <class S>
struct Rot {
    S m[3][3];
};
template <class S>
__device__ __forceinline__ Rot<S> rot_ypr(const S& yaw, const S& pitch, const S& roll) {
    S ca = s_cos(yaw), sa = s_sin(yaw), cb = s_cos(pitch), sb = s_sin(pitch);
    S cg = s_cos(roll), sg = s_sin(roll);
    Rot<S> R;
    R.m[0][0] = ca * cb;
    R.m[0][1] = ca * sb * sg - sa * cg;
    R.m[0][2] = ca * sb * cg + sa * sg;
    R.m[1][0] = sa * cb;
    R.m[1][1] = sa * sb * sg + ca * cg;
    R.m[1][2] = sa * sb * cg - ca * sg;
    R.m[2][0] = -sb;
    R.m[2][1] = cb * sg;
    R.m[2][2] = cb * cg;
    return R;
}

// Pattern vector (global frame) of port slant `zeta` along unit direction u.
template <class S>
__device__ __forceinline__ V3<S> antenna_vec(int kind, float zeta, const Rot<S>& R, const V3<S>& u) {
    S lx = R.m[0][0] * u.x + R.m[1][0] * u.y + R.m[2][0] * u.z;
    S ly = R.m[0][1] * u.x + R.m[1][1] * u.y + R.m[2][1] * u.z;
    S lz = R.m[0][2] * u.x + R.m[1][2] * u.y + R.m[2][2] * u.z;
    S rho = s_sqrt(lx * lx + ly * ly);
    S cp, sp, phi;
    bool pole = !(val(rho) > 1e-7f);
    if (!pole) {
        S ir = SConst<S>::make(1.0f) / rho;
        cp = lx * ir;
        sp = ly * ir;
    } else {
        cp = SConst<S>::make(1.0f);
        sp = SConst<S>::make(0.0f);
    }
    S ct = lz, st = rho;
    S g;
    if (kind == RT_ANT_ISO) {
        g = SConst<S>::make(1.0f);
    } else if (kind == RT_ANT_DIPOLE) {
        g = st * 1.224744871f;
    } else {
        const float r2d = 57.29577951f;
        S theta = s_atan2(rho, lz);
        phi = pole ? SConst<S>::make(0.0f) : s_atan2(ly, lx);
        S td = theta * (r2d / 65.0f) - (90.0f / 65.0f);
        S av = 0.0f - s_min(td * td * 12.0f, SConst<S>::make(30.0f));
        S pd = phi * (r2d / 65.0f);
        S ah = 0.0f - s_min(pd * pd * 12.0f, SConst<S>::make(30.0f));
        S a = 0.0f - s_min(0.0f - (av + ah), SConst<S>::make(30.0f));
        g = s_exp10((a + 8.0f) * 0.05f);
    }
    float cz, sz;
    sincosf(zeta, &sz, &cz);
    S cth = g * cz, cph = g * sz;
    // local f = cth * theta_hat + cph * phi_hat
    S fx = cth * ct * cp - cph * sp;
    S fy = cth * ct * sp + cph * cp;
    S fz = 0.0f - cth * st;
    V3<S> out;
    out.x = R.m[0][0] * fx + R.m[0][1] * fy + R.m[0][2] * fz;
    out.y = R.m[1][0] * fx + R.m[1][1] * fy + R.m[1][2] * fz;
    out.z = R.m[2][0] * fx + R.m[2][1] * fy + R.m[2][2] * fz;
    return out;
}

// ------------------------------------------------------------------- reflection
// eta = eps_r - j sigma / (omega eps0); returns the reflected complex field.
template <class S>
__device__ __forceinline__ void reflect_field(Cx<S> E[3], const V3<S>& ki, const V3<S>& kr, f3 n0,
                                              const S& eps_r, const S& sigma, float inv_we0) {
    f3 kv = v_val(ki);
    if (dot(kv, n0) > 0.0f) n0 = -n0;
    V3<S> n = v_const<S>(n0);
    S c1 = 0.0f - v_dot(ki, n);
    S s2 = 1.0f - c1 * c1;
    Cx<S> eta = {eps_r, 0.0f - sigma * inv_we0};
    Cx<S> root = c_sqrt(Cx<S>{eta.re - s2, eta.im});
    Cx<S> cc = {c1, SConst<S>::make(0.0f)};
    Cx<S> rperp = c_div(c_sub(cc, root), c_add(cc, root));
    Cx<S> ec = c_scale(eta, c1);
    Cx<S> rpar = c_div(c_sub(ec, root), c_add(ec, root));
    V3<S> c = v_cross(ki, n);
    f3 cv = v_val(c);
    V3<S> ep;
    if (dot(cv, cv) > 1e-12f) {
        ep = v_unit(c);
    } else {
        f3 a = fabsf(n0.x) > 0.9f ? mk(0.0f, 1.0f, 0.0f) : mk(1.0f, 0.0f, 0.0f);
        f3 p = cross(n0, a);
        p = p * rsqrtf(dot(p, p));
        ep = v_const<S>(p);
    }
    V3<S> epi = v_cross(ep, ki), epr = v_cross(ep, kr);
    Cx<S> dperp = {E[0].re * ep.x + E[1].re * ep.y + E[2].re * ep.z,
                   E[0].im * ep.x + E[1].im * ep.y + E[2].im * ep.z};
    Cx<S> dpar = {E[0].re * epi.x + E[1].re * epi.y + E[2].re * epi.z,
                  E[0].im * epi.x + E[1].im * epi.y + E[2].im * epi.z};
    Cx<S> a = c_mul(rperp, dperp), b = c_mul(rpar, dpar);
    E[0] = {a.re * ep.x + b.re * epr.x, a.im * ep.x + b.im * epr.x};
    E[1] = {a.re * ep.y + b.re * epr.y, a.im * ep.y + b.im * epr.y};
    E[2] = {a.re * ep.z + b.re * epr.z, a.im * ep.z + b.im * epr.z};
}

__device__ __forceinline__ float inv_omega_eps0(double fc) {
    return (float)(1.0 / (2.0 * RT_PI_D * fc * RT_EPS0_D));
}
