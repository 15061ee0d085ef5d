/*
 * oracle.c -- plain, slow FP64 CPU oracle of specular shooting-and-bouncing
 * ray tracing with image-method refinement and the polarized field along each
 * path (paper Sec. II "Current Features & Planned Extensions", Sec. II intro).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code, header, table or constant with the CUDA path; it does brute-force
 * all-triangle intersection and follows the method's steps in the paper's
 * order:
 *   1. rays leave the transmitter along a Fibonacci lattice on the sphere;
 *   2. each ray is traced by closest hit and specular reflection until the
 *      maximum number of reflections; every prefix of its list of hit
 *      triangles is a candidate path;
 *   3. the image method turns each candidate into the specular path through
 *      the same triangles that ends exactly at the receiver, or rejects it;
 *   4. duplicates are removed (done by the Python wrapper with a set) and a
 *      line-of-sight path is added when the direct segment is unoccluded;
 *   5. the polarized field is carried along each path: transmit pattern,
 *      Fresnel reflection of the two polarization components at each
 *      interaction, receive pattern, free-space spreading and phase.
 * The paper states no formulas (it defers them to an external primer); the
 * textbook readings used here are listed with each function.
 *
 * Parity-margin outputs: wherever a decision (hit or miss, inside or outside
 * a triangle, which of two surfaces is closer, which coverage cell) depends on
 * a continuous quantity, the oracle also returns the distance in metres to
 * the decision boundary. Decisions closer than a stated tolerance to their
 * boundary are "near-degenerate": an FP32 implementation may take either side.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_C0 299792458.0
#define ORA_EPS0 8.8541878128e-12
#define ORA_PI 3.14159265358979323846

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Plain FP64 vector helpers                                                 */
/* ------------------------------------------------------------------------ */
static void v_sub(const double* a, const double* b, double* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double* a, const double* b, double* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double v_norm(const double* a) { return sqrt(v_dot(a, a)); }

/* Unit normal (v1-v0)x(v2-v0) of triangle j, and twice its area. */
static void tri_normal(const double* V, int j, double* n, double* area2) {
    const double* t = V + 9 * (size_t)j;
    double e1[3], e2[3];
    v_sub(t + 3, t, e1);
    v_sub(t + 6, t, e2);
    v_cross(e1, e2, n);
    double a = v_norm(n);
    *area2 = a;
    n[0] /= a; n[1] /= a; n[2] /= a;
}

/*
 * Ray/triangle intersection (Moller-Trumbore, FP64). Returns 0 if the ray is
 * parallel to the plane. On success gives the ray parameter t of the plane
 * crossing, the barycentrics (u, v) of v1 and v2, and the signed distance in
 * metres from the crossing point to the nearest edge line (positive inside).
 */
static int ray_tri(const double* V, int j, const double* o, const double* d,
                   double* t, double* sdist, double* sin_el) {
    const double* tri = V + 9 * (size_t)j;
    double e1[3], e2[3], p[3], s[3], q[3];
    v_sub(tri + 3, tri, e1);
    v_sub(tri + 6, tri, e2);
    v_cross(d, e2, p);
    double det = v_dot(e1, p);
    double nn[3];
    v_cross(e1, e2, nn);
    double a2 = v_norm(nn);
    if (a2 <= 0.0) return 0;
    double sn = fabs(v_dot(d, nn)) / a2;  /* |sin| of the ray's elevation over the plane */
    if (sn < 1e-12) return 0;
    double inv = 1.0 / det;
    v_sub(o, tri, s);
    double u = v_dot(s, p) * inv;
    v_cross(s, e1, q);
    double v = v_dot(d, q) * inv;
    *t = v_dot(e2, q) * inv;
    /* heights of the triangle over its three edges */
    double l01 = v_norm(e1), l02 = v_norm(e2), e12[3];
    v_sub(tri + 6, tri + 3, e12);
    double l12 = v_norm(e12);
    double w = 1.0 - u - v;
    double d0 = w * (a2 / l12);   /* to edge v1-v2 */
    double d1 = u * (a2 / l02);   /* to edge v0-v2 */
    double d2 = v * (a2 / l01);   /* to edge v0-v1 */
    double m = d0 < d1 ? d0 : d1;
    *sdist = m < d2 ? m : d2;
    *sin_el = sn;
    return 1;
}

/*
 * Closest hit by brute force over all triangles (paper Sec. II: Mitsuba's
 * ray/primitive intersection; here the plain definition). Rules: closed
 * barycentric test, t > tmin, the triangle the ray leaves is excluded, equal
 * t resolves to the lowest triangle id. margin = distance in metres by which
 * the ray would have to move to change the answer (see file header), computed
 * over the triangles whose crossing lies in (tmin - eps, t_hit + eps).
 */
static int closest_hit(const double* V, int T, const double* o, const double* d,
                       int exclude, double tmin, double eps, double* t_out, double* margin) {
    int best = -1;
    double tb = INFINITY;
    for (int j = 0; j < T; j++) {
        if (j == exclude) continue;
        double t, sd, se;
        if (!ray_tri(V, j, o, d, &t, &sd, &se)) continue;
        if (sd >= 0.0 && t > tmin && t < tb) { best = j; tb = t; }
    }
    double m = INFINITY;
    for (int j = 0; j < T; j++) {
        if (j == exclude) continue;
        double t, sd, se;
        if (!ray_tri(V, j, o, d, &t, &sd, &se)) continue;
        if (!(t > tmin - eps && t < tb + eps)) continue;
        double edge = fabs(sd) * se;
        if (edge < m) m = edge;
        if (sd >= 0.0 && j != best) {
            double g = (t <= tmin) ? (tmin - t) : fabs(t - tb);
            if (g < m) m = g;
        }
        if (j == best && t - tmin < m) m = t - tmin;
    }
    *t_out = tb;
    *margin = m;
    return best;
}

/* Specular reflection of direction d about the plane of triangle j. */
static void reflect_dir(const double* V, int j, const double* d, double* r) {
    double n[3], a2;
    tri_normal(V, j, n, &a2);
    double dn = v_dot(d, n);
    for (int c = 0; c < 3; c++) r[c] = d[c] - 2.0 * dn * n[c];
}

/* ------------------------------------------------------------------------ */
/* Fibonacci lattice (Sec. II: ray directions on a Fibonacci lattice)        */
/* ------------------------------------------------------------------------ */
/*
 * Spherical Fibonacci lattice of N points, global frame:
 *   z_i = 1 - (2i+1)/N,  phi_i = 2*pi*frac(i*(sqrt(5)-1)/2),
 *   d_i = (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z).
 */
static void fib_dir(long long N, long long i, double* d) {
    const double g = (sqrt(5.0) - 1.0) / 2.0;
    double z = 1.0 - (2.0 * (double)i + 1.0) / (double)N;
    double x = (double)i * g;
    double phi = 2.0 * ORA_PI * (x - floor(x));
    double rho = sqrt(1.0 - z * z);
    d[0] = rho * cos(phi);
    d[1] = rho * sin(phi);
    d[2] = z;
}

void ora_fibonacci(long long N, long long i0, long long n, double* dirs) {
    for (long long k = 0; k < n; k++) fib_dir(N, i0 + k, dirs + 3 * k);
}

/* ------------------------------------------------------------------------ */
/* Shooting and bouncing (candidate generation)                              */
/* ------------------------------------------------------------------------ */
/*
 * For each ray id in ray_ids: closest hit, specular reflection, repeated up
 * to D hits; hits[k*D + b] = triangle id of hit b (or -1 after a miss) and
 * margins[k*D + b] = min of the closest-hit margins of hits 0..b.
 * A closest-hit query whose answer is a miss ends the ray.
 */
void ora_trace_sbr(int T, const double* V, const double* tx, long long N,
                   const long long* ray_ids, long long n, int D, double tmin, double eps,
                   int* hits, double* margins, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long long k = 0; k < n; k++) {
        double o[3] = {tx[0], tx[1], tx[2]}, d[3];
        fib_dir(N, ray_ids[k], d);
        int last = -1;
        double macc = INFINITY;
        int b = 0;
        for (; b < D; b++) {
            double t, m;
            int id = closest_hit(V, T, o, d, last, tmin, eps, &t, &m);
            if (m < macc) macc = m;
            if (id < 0) break;
            hits[k * D + b] = id;
            margins[k * D + b] = macc;
            double r[3];
            reflect_dir(V, id, d, r);
            for (int c = 0; c < 3; c++) { o[c] += t * d[c]; d[c] = r[c]; }
            last = id;
        }
        for (; b < D; b++) { hits[k * D + b] = -1; margins[k * D + b] = macc; }
    }
}

/* ------------------------------------------------------------------------ */
/* Image method (Sec. II: candidates refined by the image method)            */
/* ------------------------------------------------------------------------ */
/*
 * Is the segment p -> q free of occluders? Occluder = any triangle other than
 * ex0/ex1 crossed (closed test) at distance in (tmin, L - tmin). margin as in
 * closest_hit, for the window (tmin - eps, L - tmin + eps).
 */
static int segment_clear(const double* V, int T, const double* p, const double* q,
                         int ex0, int ex1, double tmin, double eps, double* margin) {
    double d[3];
    v_sub(q, p, d);
    double L = v_norm(d);
    d[0] /= L; d[1] /= L; d[2] /= L;
    int clear = 1;
    double m = INFINITY;
    for (int j = 0; j < T; j++) {
        if (j == ex0 || j == ex1) continue;
        double t, sd, se;
        if (!ray_tri(V, j, p, d, &t, &sd, &se)) continue;
        if (!(t > tmin - eps && t < L - tmin + eps)) continue;
        double edge = fabs(sd) * se;
        if (edge < m) m = edge;
        if (sd >= 0.0) {
            if (t > tmin && t < L - tmin) clear = 0;
            double g1 = fabs(t - tmin), g2 = fabs(t - (L - tmin));
            if (g1 < m) m = g1;
            if (g2 < m) m = g2;
        }
    }
    *margin = m;
    return clear;
}

/*
 * Image method for the ordered triangle list seq[0..K-1] from tx to rx.
 *   images:   I_0 = tx, I_k = mirror of I_{k-1} in the plane of triangle k;
 *   backward: x_{K+1} = rx, x_k = the point where the line x_{k+1} -> I_k
 *             crosses plane k (line parameter strictly inside (0, 1)).
 * Valid iff: consecutive triangles differ; each x_k lies in its triangle
 * (closed test); x_{k-1} and x_{k+1} lie strictly on the same side of plane
 * k; every segment x_j -> x_{j+1} is unoccluded (its end triangles excluded).
 * K = 0 is the line-of-sight test. Outputs the K reflection points, the path
 * length (sum of segment lengths) and the margin.
 */
int ora_image_path(int T, const double* V, const double* tx, const double* rx,
                   const int* seq, int K, double tmin, double eps,
                   double* points, double* length, double* margin) {
    double P[8][3], Img[8][3];
    double m = INFINITY;
    int ok = 1;
    if (K > 6) return 0;
    for (int k = 1; k < K; k++)
        if (seq[k] == seq[k - 1]) return 0;
    for (int c = 0; c < 3; c++) { Img[0][c] = tx[c]; P[0][c] = tx[c]; P[K + 1][c] = rx[c]; }
    for (int k = 1; k <= K; k++) {
        double n[3], a2, w[3];
        tri_normal(V, seq[k - 1], n, &a2);
        v_sub(Img[k - 1], V + 9 * (size_t)seq[k - 1], w);
        double s = v_dot(w, n);
        for (int c = 0; c < 3; c++) Img[k][c] = Img[k - 1][c] - 2.0 * s * n[c];
    }
    for (int k = K; k >= 1; k--) {
        double n[3], a2, dir[3], w[3];
        const double* v0 = V + 9 * (size_t)seq[k - 1];
        tri_normal(V, seq[k - 1], n, &a2);
        v_sub(Img[k], P[k + 1], dir);
        double den = v_dot(dir, n);
        v_sub(v0, P[k + 1], w);
        if (fabs(den) < 1e-300) return 0;
        double s = v_dot(w, n) / den;
        double L = v_norm(dir);
        double ms = fabs(s < 1.0 - s ? s : 1.0 - s) * L;
        if (ms < m) m = ms;
        if (!(s > 0.0 && s < 1.0)) ok = 0;
        for (int c = 0; c < 3; c++) P[k][c] = P[k + 1][c] + s * dir[c];
        /* closed in-triangle test of P[k], distance to the nearest edge line */
        double t, sd, se;
        double dn[3] = {dir[0] / L, dir[1] / L, dir[2] / L};
        if (!ray_tri(V, seq[k - 1], P[k + 1], dn, &t, &sd, &se)) return 0;
        if (sd < 0.0) ok = 0;
        if (fabs(sd) * se < m) m = fabs(sd) * se;
    }
    if (ok) {
        for (int k = 1; k <= K; k++) {
            double n[3], a2, w1[3], w2[3];
            const double* v0 = V + 9 * (size_t)seq[k - 1];
            tri_normal(V, seq[k - 1], n, &a2);
            v_sub(P[k - 1], v0, w1);
            v_sub(P[k + 1], v0, w2);
            double s1 = v_dot(w1, n), s2 = v_dot(w2, n);
            if (!((s1 > 0.0 && s2 > 0.0) || (s1 < 0.0 && s2 < 0.0))) ok = 0;
            if (fabs(s1) < m) m = fabs(s1);
            if (fabs(s2) < m) m = fabs(s2);
        }
    }
    double len = 0.0;
    if (ok) {
        for (int j = 0; j <= K; j++) {
            int ex0 = j >= 1 ? seq[j - 1] : -1;
            int ex1 = j < K ? seq[j] : -1;
            double mm;
            if (!segment_clear(V, T, P[j], P[j + 1], ex0, ex1, tmin, eps, &mm)) ok = 0;
            if (mm < m) m = mm;
            double d[3];
            v_sub(P[j + 1], P[j], d);
            len += v_norm(d);
        }
    }
    for (int k = 0; k < K; k++)
        for (int c = 0; c < 3; c++) points[3 * k + c] = P[k + 1][c];
    *length = len;
    *margin = m;
    return ok;
}

/*
 * Batched image method: every candidate (depth[c], seqs[c*D ...]) against
 * every receiver. Writes only pairs that are valid or near-degenerate
 * (margin < eps): out_cand, out_rx, out_valid, out_margin, up to cap entries.
 * Returns the number of such pairs (may exceed cap; then call again).
 */
long long ora_validate(int T, const double* V, const double* tx, int n_rx, const double* rxs,
                       long long n_cand, const int* seqs, const int* depths, int D,
                       double tmin, double eps, long long cap, long long* out_cand,
                       int* out_rx, int* out_valid, double* out_margin, int nthreads) {
    long long count = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long long c = 0; c < n_cand; c++) {
        for (int r = 0; r < n_rx; r++) {
            double pts[24], len, m;
            int ok = ora_image_path(T, V, tx, rxs + 3 * r, seqs + c * D, depths[c], tmin, eps,
                                    pts, &len, &m);
            if (ok || m < eps) {
                long long slot;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
                slot = count++;
                if (slot < cap) {
                    out_cand[slot] = c;
                    out_rx[slot] = r;
                    out_valid[slot] = ok;
                    out_margin[slot] = m;
                }
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers (value + tangents w.r.t. real parameters)       */
/* ------------------------------------------------------------------------ */
#define NGMAX 24
typedef struct { cplx v; cplx d[NGMAX]; } dc;
typedef struct { dc x, y, z; } dv;
static int NGA = 0; /* active tangent count; set before any parallel region */

static dc dc_const(cplx v) { dc r; r.v = v; for (int i = 0; i < NGA; i++) r.d[i] = 0; return r; }
static dc dc_var(double v, int idx) { dc r = dc_const(v); if (idx >= 0 && idx < NGA) r.d[idx] = 1.0; return r; }
static dc dc_add(dc a, dc b) { dc r; r.v = a.v + b.v; for (int i = 0; i < NGA; i++) r.d[i] = a.d[i] + b.d[i]; return r; }
static dc dc_sub(dc a, dc b) { dc r; r.v = a.v - b.v; for (int i = 0; i < NGA; i++) r.d[i] = a.d[i] - b.d[i]; return r; }
static dc dc_mul(dc a, dc b) { dc r; r.v = a.v * b.v; for (int i = 0; i < NGA; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
static dc dc_scale(dc a, cplx s) { dc r; r.v = a.v * s; for (int i = 0; i < NGA; i++) r.d[i] = a.d[i] * s; return r; }
static dc dc_div(dc a, dc b) {
    dc r; r.v = a.v / b.v;
    cplx b2 = b.v * b.v;
    for (int i = 0; i < NGA; i++) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / b2;
    return r;
}
static dc dc_csqrt(dc a) { /* principal branch */
    dc r; r.v = csqrt(a.v);
    for (int i = 0; i < NGA; i++) r.d[i] = a.d[i] / (2.0 * r.v);
    return r;
}
static dc dc_rsqrt_real(dc a) { /* sqrt of a real-valued dual */
    dc r; double s = sqrt(creal(a.v)); r.v = s;
    for (int i = 0; i < NGA; i++) r.d[i] = creal(a.d[i]) / (2.0 * s);
    return r;
}
static dc dc_sin(dc a) { dc r; double x = creal(a.v); r.v = sin(x); for (int i = 0; i < NGA; i++) r.d[i] = cos(x) * creal(a.d[i]); return r; }
static dc dc_cos(dc a) { dc r; double x = creal(a.v); r.v = cos(x); for (int i = 0; i < NGA; i++) r.d[i] = -sin(x) * creal(a.d[i]); return r; }
static dc dc_atan2(dc y, dc x) {
    dc r; double yy = creal(y.v), xx = creal(x.v), q = xx * xx + yy * yy;
    r.v = atan2(yy, xx);
    for (int i = 0; i < NGA; i++) r.d[i] = (xx * creal(y.d[i]) - yy * creal(x.d[i])) / q;
    return r;
}
static dc dc_pow10(dc a) {
    dc r; double v = pow(10.0, creal(a.v)); r.v = v;
    for (int i = 0; i < NGA; i++) r.d[i] = v * log(10.0) * creal(a.d[i]);
    return r;
}
static dc dc_expj(dc ph) { /* exp(j*ph), ph real */
    dc r; r.v = cexp(I * creal(ph.v));
    for (int i = 0; i < NGA; i++) r.d[i] = I * r.v * creal(ph.d[i]);
    return r;
}
static dc dc_min(dc a, dc b) { return creal(a.v) <= creal(b.v) ? a : b; }
static double dc_re(dc a) { return creal(a.v); }

static dv dv_const(const double* p) { dv r = {dc_const(p[0]), dc_const(p[1]), dc_const(p[2])}; return r; }
static dv dv_add(dv a, dv b) { dv r = {dc_add(a.x, b.x), dc_add(a.y, b.y), dc_add(a.z, b.z)}; return r; }
static dv dv_sub(dv a, dv b) { dv r = {dc_sub(a.x, b.x), dc_sub(a.y, b.y), dc_sub(a.z, b.z)}; return r; }
static dv dv_scale(dv a, dc s) { dv r = {dc_mul(a.x, s), dc_mul(a.y, s), dc_mul(a.z, s)}; return r; }
static dc dv_dot(dv a, dv b) { return dc_add(dc_add(dc_mul(a.x, b.x), dc_mul(a.y, b.y)), dc_mul(a.z, b.z)); }
static dv dv_cross(dv a, dv b) {
    dv r = {dc_sub(dc_mul(a.y, b.z), dc_mul(a.z, b.y)),
            dc_sub(dc_mul(a.z, b.x), dc_mul(a.x, b.z)),
            dc_sub(dc_mul(a.x, b.y), dc_mul(a.y, b.x))};
    return r;
}
static dc dv_norm(dv a) { return dc_rsqrt_real(dv_dot(a, a)); }
static dv dv_unit(dv a) { dc n = dv_norm(a); dv r = {dc_div(a.x, n), dc_div(a.y, n), dc_div(a.z, n)}; return r; }

/* ------------------------------------------------------------------------ */
/* Antennas and rotations                                                    */
/* ------------------------------------------------------------------------ */
/*
 * Device orientation (Sec. II: yaw, pitch, roll), 3GPP TR 38.901 Sec. 7.1
 * convention: R = Rz(yaw) Ry(pitch) Rx(roll); a positive pitch tilts the
 * boresight (local x) downwards.
 */
static void rot_matrix(dc yaw, dc pitch, dc roll, dc R[3][3]) {
    dc ca = dc_cos(yaw), sa = dc_sin(yaw), cb = dc_cos(pitch), sb = dc_sin(pitch);
    dc cg = dc_cos(roll), sg = dc_sin(roll);
    dc zero = dc_const(0.0);
    /* Rz(a) Ry(b) Rx(g) */
    R[0][0] = dc_mul(ca, cb);
    R[0][1] = dc_sub(dc_mul(dc_mul(ca, sb), sg), dc_mul(sa, cg));
    R[0][2] = dc_add(dc_mul(dc_mul(ca, sb), cg), dc_mul(sa, sg));
    R[1][0] = dc_mul(sa, cb);
    R[1][1] = dc_add(dc_mul(dc_mul(sa, sb), sg), dc_mul(ca, cg));
    R[1][2] = dc_sub(dc_mul(dc_mul(sa, sb), cg), dc_mul(ca, sg));
    R[2][0] = dc_sub(zero, sb);
    R[2][1] = dc_mul(cb, sg);
    R[2][2] = dc_mul(cb, cg);
}

/*
 * Field pattern vector of port `port` of an antenna seen along the global
 * unit direction u (pointing away from the antenna), as a global 3-vector.
 *   kind 0 isotropic: amplitude 1;
 *   kind 1 short dipole: amplitude sqrt(1.5) sin(theta);
 *   kind 2 3GPP TR 38.901 Table 7.3-1 element: A_V = -min(12((theta-90)/65)^2, 30),
 *          A_H = -min(12(phi/65)^2, 30), A = -min(-(A_V+A_H), 30) dB,
 *          power gain 10^((8 + A)/10) (angles in degrees, local frame).
 * Polarization by slant angle zeta (TR 38.901 model 2): C_theta = g cos zeta,
 * C_phi = g sin zeta; zeta = 0 is vertical, pi/2 horizontal, +-pi/4 cross.
 * Local spherical basis: theta_hat = (cos t cos p, cos t sin p, -sin t),
 * phi_hat = (-sin p, cos p, 0); at the poles phi is taken as 0.
 */
static dv antenna_field(int kind, double slant, dc R[3][3], dv u) {
    dc l[3];
    dc ug[3] = {u.x, u.y, u.z};
    for (int i = 0; i < 3; i++)
        l[i] = dc_add(dc_add(dc_mul(R[0][i], ug[0]), dc_mul(R[1][i], ug[1])), dc_mul(R[2][i], ug[2]));
    dc rho = dc_rsqrt_real(dc_add(dc_mul(l[0], l[0]), dc_mul(l[1], l[1])));
    dc ct = l[2], st = rho, cp, sp, theta, phi;
    theta = dc_atan2(rho, l[2]);
    if (dc_re(rho) > 1e-12) {
        cp = dc_div(l[0], rho);
        sp = dc_div(l[1], rho);
        phi = dc_atan2(l[1], l[0]);
    } else {
        cp = dc_const(1.0); sp = dc_const(0.0); phi = dc_const(0.0);
    }
    dc g;
    if (kind == 0) {
        g = dc_const(1.0);
    } else if (kind == 1) {
        g = dc_scale(st, sqrt(1.5));
    } else {
        double rad2deg = 180.0 / ORA_PI;
        dc td = dc_sub(dc_scale(theta, rad2deg / 65.0), dc_const(90.0 / 65.0));
        dc av = dc_sub(dc_const(0.0), dc_min(dc_scale(dc_mul(td, td), 12.0), dc_const(30.0)));
        dc pd = dc_scale(phi, rad2deg / 65.0);
        dc ah = dc_sub(dc_const(0.0), dc_min(dc_scale(dc_mul(pd, pd), 12.0), dc_const(30.0)));
        dc a = dc_sub(dc_const(0.0), dc_min(dc_sub(dc_const(0.0), dc_add(av, ah)), dc_const(30.0)));
        g = dc_pow10(dc_scale(dc_add(a, dc_const(8.0)), 1.0 / 20.0));
    }
    dc cth = dc_scale(g, cos(slant)), cph = dc_scale(g, sin(slant));
    dc th[3] = {dc_mul(ct, cp), dc_mul(ct, sp), dc_sub(dc_const(0.0), st)};
    dc ph[3] = {dc_sub(dc_const(0.0), sp), cp, dc_const(0.0)};
    dc f[3];
    for (int i = 0; i < 3; i++) f[i] = dc_add(dc_mul(cth, th[i]), dc_mul(cph, ph[i]));
    dc gl[3];
    for (int i = 0; i < 3; i++)
        gl[i] = dc_add(dc_add(dc_mul(R[i][0], f[0]), dc_mul(R[i][1], f[1])), dc_mul(R[i][2], f[2]));
    dv r = {gl[0], gl[1], gl[2]};
    return r;
}

/*
 * Specular reflection of the complex field vector E (Fresnel, Sec. II:
 * materials given by eps_r and sigma, mu_r = 1). Incident unit direction ki,
 * reflected kr, plane normal n (any orientation; it is turned to face the
 * incoming wave). eta = eps_r - j sigma/(omega eps0);
 *   r_perp = (cos1 - sqrt(eta - sin1^2)) / (cos1 + sqrt(eta - sin1^2)),
 *   r_par  = (eta cos1 - sqrt(eta - sin1^2)) / (eta cos1 + sqrt(eta - sin1^2));
 * e_perp = ki x n / |ki x n|, e_par_i = e_perp x ki, e_par_r = e_perp x kr,
 * E_r = r_perp (E.e_perp) e_perp + r_par (E.e_par_i) e_par_r.
 */
static dv reflect_field(dv E, dv ki, dv kr, const double* n0, dc eps_r, dc sigma, double omega) {
    double nd[3] = {n0[0], n0[1], n0[2]};
    double kiv[3] = {dc_re(ki.x), dc_re(ki.y), dc_re(ki.z)};
    if (v_dot(kiv, nd) > 0.0) { nd[0] = -nd[0]; nd[1] = -nd[1]; nd[2] = -nd[2]; }
    dv n = dv_const(nd);
    dc cos1 = dc_sub(dc_const(0.0), dv_dot(ki, n));
    dc sin2 = dc_sub(dc_const(1.0), dc_mul(cos1, cos1));
    dc eta = dc_sub(eps_r, dc_scale(sigma, I / (omega * ORA_EPS0)));
    dc root = dc_csqrt(dc_sub(eta, sin2));
    dc rperp = dc_div(dc_sub(cos1, root), dc_add(cos1, root));
    dc ec = dc_mul(eta, cos1);
    dc rpar = dc_div(dc_sub(ec, root), dc_add(ec, root));
    dv c = dv_cross(ki, n);
    double cn = sqrt(dc_re(c.x) * dc_re(c.x) + dc_re(c.y) * dc_re(c.y) + dc_re(c.z) * dc_re(c.z));
    dv eperp;
    if (cn > 1e-12) {
        eperp = dv_unit(c);
    } else { /* normal incidence: any unit vector orthogonal to n */
        double a[3] = {1.0, 0.0, 0.0}, p[3];
        if (fabs(nd[0]) > 0.9) { a[0] = 0.0; a[1] = 1.0; }
        v_cross(nd, a, p);
        double pn = v_norm(p);
        p[0] /= pn; p[1] /= pn; p[2] /= pn;
        eperp = dv_const(p);
    }
    dv epi = dv_cross(eperp, ki), epr = dv_cross(eperp, kr);
    dc cperp = dc_mul(rperp, dv_dot(E, eperp));
    dc cpar = dc_mul(rpar, dv_dot(E, epi));
    return dv_add(dv_scale(eperp, cperp), dv_scale(epr, cpar));
}

/* ------------------------------------------------------------------------ */
/* Path field (CIR coefficient) with optional tangents                      */
/* ------------------------------------------------------------------------ */
/*
 * Channel coefficient of one specular path, for every (rx port, tx port):
 *   a = lambda/(4 pi r) exp(-j 2 pi frac(r/lambda)) F_rx(-k_last) . E,
 * with E the transmit pattern vector along the first segment carried through
 * the reflections, r the path length (sum of segment lengths) and tau = r/c0.
 * The dot product has no conjugation (reciprocal).
 * Parameters whose tangents are tracked (when NGA > 0):
 *   0..2 tx position, 3..5 tx yaw/pitch/roll, 6..6+M-1 eps_r, 6+M.. sigma.
 * The reflection points are recomputed from the image method as functions of
 * the tx position, so geometry tangents flow through them.
 */
static void path_field_one(int T, const double* V, const int* mat, int M, const double* mats,
                           double fc, const double* tx, const double* txypr, int tkind,
                           int ntp, const double* tslant, const double* rx, const double* rxypr,
                           int rkind, int nrp, const double* rslant, const int* seq, int K,
                           cplx* a, cplx* da, double* tau, double* dtau) {
    (void)T;
    double lam = ORA_C0 / fc, omega = 2.0 * ORA_PI * fc;
    dv txv = {dc_var(tx[0], 0), dc_var(tx[1], 1), dc_var(tx[2], 2)};
    dv rxv = dv_const(rx);
    dv Iv[8], Pv[8];
    Iv[0] = txv;
    for (int k = 1; k <= K; k++) {
        double n[3], a2;
        tri_normal(V, seq[k - 1], n, &a2);
        dv nv = dv_const(n), v0 = dv_const(V + 9 * (size_t)seq[k - 1]);
        dc s = dv_dot(dv_sub(Iv[k - 1], v0), nv);
        Iv[k] = dv_sub(Iv[k - 1], dv_scale(nv, dc_scale(s, 2.0)));
    }
    Pv[0] = txv;
    Pv[K + 1] = rxv;
    for (int k = K; k >= 1; k--) {
        double n[3], a2;
        tri_normal(V, seq[k - 1], n, &a2);
        dv nv = dv_const(n), v0 = dv_const(V + 9 * (size_t)seq[k - 1]);
        dv dir = dv_sub(Iv[k], Pv[k + 1]);
        dc s = dc_div(dv_dot(dv_sub(v0, Pv[k + 1]), nv), dv_dot(dir, nv));
        Pv[k] = dv_add(Pv[k + 1], dv_scale(dir, s));
    }
    dv kd[8];
    dc r = dc_const(0.0);
    for (int j = 0; j <= K; j++) {
        dv sg = dv_sub(Pv[j + 1], Pv[j]);
        dc L = dv_norm(sg);
        r = dc_add(r, L);
        kd[j] = dv_scale(sg, dc_div(dc_const(1.0), L));
    }
    /* transmit pattern vectors */
    dc Rt[3][3], Rr[3][3];
    rot_matrix(dc_var(txypr[0], 3), dc_var(txypr[1], 4), dc_var(txypr[2], 5), Rt);
    rot_matrix(dc_const(rxypr[0]), dc_const(rxypr[1]), dc_const(rxypr[2]), Rr);
    dv E[2];
    for (int q = 0; q < ntp; q++) E[q] = antenna_field(tkind, tslant[q], Rt, kd[0]);
    for (int k = 1; k <= K; k++) {
        double n[3], a2;
        tri_normal(V, seq[k - 1], n, &a2);
        int m = mat[seq[k - 1]];
        dc er = dc_var(mats[2 * m], 6 + m), sg = dc_var(mats[2 * m + 1], 6 + M + m);
        for (int q = 0; q < ntp; q++) E[q] = reflect_field(E[q], kd[k - 1], kd[k], n, er, sg, omega);
    }
    dv u = dv_scale(kd[K], dc_const(-1.0));
    dv F[2];
    for (int p = 0; p < nrp; p++) F[p] = antenna_field(rkind, rslant[p], Rr, u);
    /* spreading and phase; the phase is reduced modulo 2 pi in FP64 */
    dc amp = dc_div(dc_const(lam / (4.0 * ORA_PI)), r);
    double x = creal(r.v) / lam;
    dc ph = dc_scale(r, -2.0 * ORA_PI / lam);
    ph.v = -2.0 * ORA_PI * (x - floor(x));
    dc e = dc_mul(amp, dc_expj(ph));
    for (int p = 0; p < nrp; p++)
        for (int q = 0; q < ntp; q++) {
            dc v = dc_mul(e, dv_dot(F[p], E[q]));
            a[p * ntp + q] = v.v;
            if (da)
                for (int i = 0; i < NGA; i++) da[(p * ntp + q) * NGA + i] = v.d[i];
        }
    *tau = creal(r.v) / ORA_C0;
    if (dtau)
        for (int i = 0; i < NGA; i++) dtau[i] = creal(r.d[i]) / ORA_C0;
}

/*
 * Batched path field. Path i runs from tx to rxs[rx_of[i]] through
 * seqs[i*D .. i*D + depth[i] - 1]. Outputs interleaved complex a
 * [n, nrp, ntp] (re, im), tau [n]; with ng > 0 also da [n, nrp, ntp, ng]
 * (re, im) and dtau [n, ng] (ng = 6 + 2M <= 24).
 */
void ora_path_field(int T, const double* V, const int* mat, int M, const double* mats, double fc,
                    const double* tx, const double* txypr, int tkind, int ntp, const double* tslant,
                    const double* rxs, const double* rxyprs, int rkind, int nrp, const double* rslant,
                    long long n, const int* rx_of, const int* seqs, const int* depth, int D,
                    int ng, double* a_out, double* da_out, double* tau_out, double* dtau_out,
                    int nthreads) {
    NGA = ng;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (long long i = 0; i < n; i++) {
        cplx a[4], da[4 * NGMAX];
        double tau, dtau[NGMAX];
        int r = rx_of[i];
        path_field_one(T, V, mat, M, mats, fc, tx, txypr, tkind, ntp, tslant, rxs + 3 * r,
                       rxyprs + 3 * r, rkind, nrp, rslant, seqs + i * D, depth[i], a,
                       ng ? da : NULL, &tau, ng ? dtau : NULL);
        int np = nrp * ntp;
        for (int k = 0; k < np; k++) {
            a_out[2 * (i * np + k)] = creal(a[k]);
            a_out[2 * (i * np + k) + 1] = cimag(a[k]);
            for (int g = 0; g < ng; g++) {
                da_out[2 * ((i * np + k) * ng + g)] = creal(da[k * ng + g]);
                da_out[2 * ((i * np + k) * ng + g) + 1] = cimag(da[k * ng + g]);
            }
        }
        tau_out[i] = tau;
        for (int g = 0; g < ng; g++) dtau_out[i * ng + g] = dtau[g];
    }
    NGA = 0;
}

/* ------------------------------------------------------------------------ */
/* Coverage map (Sec. II, Listing 2: coverage_map; Fig. 2: path gain in dB)   */
/* ------------------------------------------------------------------------ */
/*
 * Ray-density estimator of the path gain on the horizontal plane z = h.
 * Each ray carries the transmit pattern vector E of port tport (no 1/r) and
 * the Fresnel reflections along its bounces (up to D reflections). Each ray
 * segment (Tx -> hit 1, hit k -> hit k+1, and the last segment to the next
 * hit or to infinity) that crosses z = h at x with direction d adds
 *   w = |F_rx(-d) . E|^2 / (N |d_z|)
 * to cell floor((x - x0)/cell) and 1 to its hit count. Cell gain =
 * lambda^2/(4 pi) * sum w / cell^2, which reproduces Friis in free space.
 * marg[c] collects the w of contributions that an FP32 trace may put in a
 * different cell or drop (ray margin < eps, or the crossing closer than eps
 * to a cell edge or to the segment's end); they are added to the cell and to
 * its 8 neighbours.
 */
void ora_coverage(int T, const double* V, const int* mat, int M, const double* mats, double fc,
                  const double* tx, const double* txypr, int tkind, double tslant,
                  int rkind, double rslant, long long N, long long i0, long long i1, int D,
                  double x0, double y0, double cell, int nx, int ny, double h,
                  double tmin, double eps, double* gain, double* hits, double* marg,
                  int nthreads) {
    (void)M;
    NGA = 0;
    double lam = ORA_C0 / fc, omega = 2.0 * ORA_PI * fc;
    size_t nc = (size_t)nx * ny;
    memset(gain, 0, nc * sizeof(double));
    memset(hits, 0, nc * sizeof(double));
    memset(marg, 0, nc * sizeof(double));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double* g = calloc(nc, sizeof(double));
        double* hc = calloc(nc, sizeof(double));
        double* mg = calloc(nc, sizeof(double));
        dc Rt[3][3], Rr[3][3];
        rot_matrix(dc_const(txypr[0]), dc_const(txypr[1]), dc_const(txypr[2]), Rt);
        rot_matrix(dc_const(0.0), dc_const(0.0), dc_const(0.0), Rr);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (long long i = i0; i < i1; i++) {
            double o[3] = {tx[0], tx[1], tx[2]}, d[3];
            fib_dir(N, i, d);
            dv E = antenna_field(tkind, tslant, Rt, dv_const(d));
            int last = -1;
            double macc = INFINITY;
            for (int depth = 0; depth <= D; depth++) {
                double t, m;
                int id = closest_hit(V, T, o, d, last, tmin, eps, &t, &m);
                if (m < macc) macc = m;
                if (d[2] != 0.0) {
                    double s = (h - o[2]) / d[2];
                    if (s > 0.0 && (id < 0 || s < t)) {
                        double x = o[0] + s * d[0], y = o[1] + s * d[1];
                        double fx = (x - x0) / cell, fy = (y - y0) / cell;
                        long ix = (long)floor(fx), iy = (long)floor(fy);
                        if (ix >= 0 && iy >= 0 && ix < nx && iy < ny) {
                            double md[3] = {-d[0], -d[1], -d[2]};
                            dv F = antenna_field(rkind, rslant, Rr, dv_const(md));
                            dc fe = dv_dot(F, E);
                            double w = creal(fe.v * conj(fe.v)) / ((double)N * fabs(d[2]));
                            size_t c = (size_t)iy * nx + ix;
                            g[c] += w;
                            hc[c] += 1.0;
                            /* distance (along the ray-normal scale) to the cell's x and y edges */
                            double ex = fx - ix, ey = fy - iy;
                            double sc = cell * fabs(d[2]);
                            int nxd = ex * sc < eps ? -1 : ((1 - ex) * sc < eps ? 1 : 0);
                            int nyd = ey * sc < eps ? -1 : ((1 - ey) * sc < eps ? 1 : 0);
                            int whole = macc < eps || s < eps || (id >= 0 && t - s < eps);
                            if (whole) {
                                for (long yy = iy - 1; yy <= iy + 1; yy++)
                                    for (long xx = ix - 1; xx <= ix + 1; xx++)
                                        if (xx >= 0 && yy >= 0 && xx < nx && yy < ny)
                                            mg[(size_t)yy * nx + xx] += w;
                            } else if (nxd || nyd) {
                                /* the crossing may land in the cell across the near edge(s) */
                                long cx[2] = {ix, ix + nxd}, cy[2] = {iy, iy + nyd};
                                for (int a = 0; a < (nyd ? 2 : 1); a++)
                                    for (int b = 0; b < (nxd ? 2 : 1); b++) {
                                        long xx = cx[b], yy = cy[a];
                                        if (xx >= 0 && yy >= 0 && xx < nx && yy < ny)
                                            mg[(size_t)yy * nx + xx] += w;
                                    }
                            }
                        }
                    }
                }
                if (id < 0 || depth == D) break;
                double n[3], a2, r[3];
                tri_normal(V, id, n, &a2);
                reflect_dir(V, id, d, r);
                int mm = mat[id];
                dv ki = dv_const(d), kr = dv_const(r);
                E = reflect_field(E, ki, kr, n, dc_const(mats[2 * mm]), dc_const(mats[2 * mm + 1]), omega);
                for (int c = 0; c < 3; c++) { o[c] += t * d[c]; d[c] = r[c]; }
                last = id;
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            for (size_t c = 0; c < nc; c++) { gain[c] += g[c]; hits[c] += hc[c]; marg[c] += mg[c]; }
        }
        free(g); free(hc); free(mg);
    }
    double scale = lam * lam / (4.0 * ORA_PI * cell * cell);
    for (size_t c = 0; c < nc; c++) { gain[c] *= scale; marg[c] *= scale; }
}

/* Closest hit of one ray (exposed for tests). */
int ora_closest_hit(int T, const double* V, const double* o, const double* d, int exclude,
                    double tmin, double eps, double* t, double* margin) {
    return closest_hit(V, T, o, d, exclude, tmin, eps, t, margin);
}

/* Segment occlusion test (exposed for the diffraction oracle). */
int ora_segment_clear(int T, const double* V, const double* p, const double* q, int ex0, int ex1, double tmin,
                      double eps, double* margin) {
    return segment_clear(V, T, p, q, ex0, ex1, tmin, eps, margin);
}

/* Fresnel coefficients (exposed for the closed-form pins). */
void ora_fresnel(double eps_r, double sigma, double fc, double cos1, double* rperp, double* rpar) {
    double omega = 2.0 * ORA_PI * fc;
    cplx eta = eps_r - I * sigma / (omega * ORA_EPS0);
    cplx root = csqrt(eta - (1.0 - cos1 * cos1));
    cplx a = (cos1 - root) / (cos1 + root);
    cplx b = (eta * cos1 - root) / (eta * cos1 + root);
    rperp[0] = creal(a); rperp[1] = cimag(a);
    rpar[0] = creal(b); rpar[1] = cimag(b);
}

/* Antenna pattern vector (exposed for tests): global 3-vector, complex. */
void ora_antenna(int kind, double slant, const double* ypr, const double* u, double* out) {
    NGA = 0;
    dc R[3][3];
    rot_matrix(dc_const(ypr[0]), dc_const(ypr[1]), dc_const(ypr[2]), R);
    dv f = antenna_field(kind, slant, R, dv_const(u));
    out[0] = creal(f.x.v); out[1] = creal(f.y.v); out[2] = creal(f.z.v);
}
