// rt_probe.cu -- measured issue peaks for the roofline of the tracer's
// kernels (rt_probe_peak). The paper has no counterpart.
//
// The traversal kernels keep the scene in L1/L2 and are bound by instruction
// issue, not by HBM. Their algorithmic work is the box tests of BVH child
// boxes and the Moller-Trumbore triangle tests; the rate at which an SM can
// execute exactly that arithmetic depends on how it splits over the FMA and
// ALU pipes (min/max and compares are ALU work). This probe runs the
// tracer's own device functions (box_pair, tri_hit from rt_common.cuh) on
// register-resident data, in the proportions the caller measured, with no
// loads, stack or branching around them, so its rate is the ceiling of that
// arithmetic on this GPU at the clock it runs at.
//
// Every test's result feeds the next test of the same node or triangle (the
// far bound of a node's box tests, the origin of a triangle test), and the
// ray's constants and direction are advanced by a run-time zero before every
// group of eight box tests and every triangle test, so that every operation
// of every test depends on values the compiler cannot know: nothing is
// hoisted out of the loop, merged or dropped as dead. The added operations
// (3 packed FMAs per 8 box tests, an add and a min per triangle test, about
// 2 % of the work) are not counted, so the measured rate slightly
// understates the peak.
#include <algorithm>

#include "rt_internal.h"

namespace {

// Traversal arithmetic: n_box8 x 8 octant-selected box tests and n_tri
// triangle tests per iteration. The box tests run in one of the two forms
// the traversal code has: PAIRED, box_pair (both children of a binary node,
// with packed FMAs, as the binary traversal runs them), or box_oct (one box
// at a time, scalar FMAs). Which form an SM executes faster depends on its
// pipes, so the caller times both and keeps the faster as the peak. Every
// lane holds its own ray (a positive direction: the near planes are the
// boxes' lo planes), eight boxes (four nodes of two) and two triangles,
// arranged so that about half of the box tests and a quarter of the
// triangle tests are hits (the triangle division is then taken as in a
// traversal). Each box test's outcome is recorded by one select, as the
// traversal records it by one bit operation or compare.
template <bool PAIRED>
__global__ void __launch_bounds__(256) k_probe_traversal(int iters, int n_box8, int n_tri, float zero, float* out) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    const float jx = 0.01f * (float)(t & 15), jy = 0.01f * (float)((t >> 4) & 15);
    f3 o = mk(-20.0f + jx, -3.0f + jy, 1.5f);
    f3 d = unit(mk(1.0f, 0.05f + jy, 0.02f + jx));
    const f3 inv = safe_inv(d);
    f3 oi = {o.x * inv.x, o.y * inv.y, o.z * inv.z};
    PairRay pr = pair_ray(inv, oi);
    float bx[8][6], r[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const float y0 = ((k & 1) ? -2.0f : 4.0f) + 0.1f * k;
        bx[k][0] = -10.0f + 2.5f * k; bx[k][1] = y0 - 3.0f; bx[k][2] = 0.05f * k;
        bx[k][3] = -8.0f + 2.5f * k;  bx[k][4] = y0 + 3.0f; bx[k][5] = 3.0f + 0.07f * k;
        r[k] = 1e30f;
    }
    // boxes 2j and 2j + 1 as the two children of node j, planes in pairs
    float4 nd[4][3];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float* u = bx[2 * j];
        const float* v = bx[2 * j + 1];
        nd[j][0] = make_float4(u[0], v[0], u[1], v[1]);
        nd[j][1] = make_float4(u[2], v[2], u[3], v[3]);
        nd[j][2] = make_float4(u[4], v[4], u[5], v[5]);
    }
    const float2 one2 = make_float2(1.0f, 1.0f), zero2 = make_float2(zero, zero);
    float4 tr[2][3];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float yc = ((t >> k) & 1u) ? -2.0f : 9.0f;
        tr[k][0] = make_float4(5.0f + k, yc - 4.0f, -4.0f, __int_as_float(k));
        tr[k][1] = make_float4(0.0f, 8.0f, 0.0f, 0.0f);
        tr[k][2] = make_float4(0.0f, 0.0f, 12.0f, 0.0f);
    }
    const float tmin = 1e-4f;
    for (int it = 0; it < iters; it++) {
        for (int s = 0; s < n_box8; s++) {
            if (PAIRED) {
                pr.mx = fma2(pr.mx.x, pr.mx.y, one2, zero2);
                pr.my = fma2(pr.my.x, pr.my.y, one2, zero2);
                pr.mz = fma2(pr.mz.x, pr.mz.y, one2, zero2);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    float tn0, tf0, tn1, tf1;
                    box_pair(nd[j][0], nd[j][1], nd[j][2], pr, tmin, r[2 * j], tn0, tf0, tn1, tf1);
                    r[2 * j] = tn0 <= tf0 ? pr.my.x : r[2 * j];
                    r[2 * j + 1] = tn1 <= tf1 ? pr.my.y : r[2 * j + 1];
                }
            } else {
                oi.x += zero;
                oi.y += zero;
                oi.z += zero;
#pragma unroll
                for (int k = 0; k < 8; k++)
                    r[k] = box_oct(bx[k][0], bx[k][1], bx[k][2], bx[k][3], bx[k][4], bx[k][5], oi, inv, tmin,
                                   r[k])
                               ? oi.y
                               : r[k];
            }
        }
        for (int q = 0; q < n_tri; q++) {
            d.x += zero;
            const float th = (q & 1) ? tri_hit(tr[1][0], tr[1][1], tr[1][2], o, d)
                                     : tri_hit(tr[0][0], tr[0][1], tr[0][2], o, d);
            o.x = fminf(o.x, th);
        }
    }
    float sum = o.x + d.x + oi.x + oi.y + oi.z + pr.mx.x + pr.my.y + pr.mz.x;
#pragma unroll
    for (int k = 0; k < 8; k++) sum += r[k];
    if (sum == 12345.678f) out[0] = sum;
}

// FP32 FMA: 8 independent chains of 16 FMAs per iteration.
__global__ void __launch_bounds__(256) k_probe_ffma(int iters, float seed, float* out) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = seed + (float)(threadIdx.x + k);
    const float m = 0.999f, c = 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    if (s == 12345.678f) out[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int rt_probe_peak(rt_ctx* ctx, int32_t kind, int32_t n_slab, int32_t n_tri, double* ops_per_s) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    cudaError_t de = cudaSetDevice(ctx->device);
    if (de != cudaSuccess) return set_cuda(ctx, de, "cudaSetDevice");
    if (!ops_per_s || (kind != RT_PROBE_TRAVERSAL && kind != RT_PROBE_FFMA))
        return set_err(ctx, RT_ERR_INVALID_ARG, "probe_peak: bad arguments");
    if (kind == RT_PROBE_TRAVERSAL && (n_slab < 8 || n_slab % 8 || n_tri < 0 || n_slab > 4096 || n_tri > 4096))
        return set_err(ctx, RT_ERR_INVALID_ARG, "probe_peak: n_slab a positive multiple of 8, n_tri >= 0");
    if (ctx->capturing) return set_err(ctx, RT_ERR_NOT_READY, "probe_peak while capturing a graph");
    const int block = 256;
    // algorithmic operations per iteration and thread: 11 per
    // octant-selected box test (6 FMA, 4 min/max, 1 compare), 35 per
    // triangle test; 2 flops per FMA
    const double per_iter = kind == RT_PROBE_TRAVERSAL ? 11.0 * n_slab + 35.0 * n_tri : 2.0 * 16 * 8;
    float* sink = bp<float>(ctx->counters);   // never written (see the kernels' last lines)
    cudaEvent_t e0, e1;
    RT_TRY(cudaEventCreate(&e0));
    RT_TRY(cudaEventCreate(&e1));
    cudaError_t err = cudaSuccess;
    double rate = 0.0;
    // the traversal's box test in both of its forms (packed pairs, scalar);
    // the faster is the peak
    const int n_forms = kind == RT_PROBE_TRAVERSAL ? 2 : 1;
    for (int form = 0; form < n_forms && err == cudaSuccess; form++) {
        const void* kern = kind != RT_PROBE_TRAVERSAL ? (const void*)k_probe_ffma
                           : form == 0                 ? (const void*)k_probe_traversal<true>
                                                       : (const void*)k_probe_traversal<false>;
        const int grid = blocks_per_sm(kern, block, 0) * ctx->num_sms;
        const double threads = (double)grid * block;
        // about 2 ms of work at 40e12 operations/s
        const int iters = (int)std::max(8.0, 8e10 / (threads * per_iter));
        float best = 1e30f;
        for (int rep = 0; rep < 6 && err == cudaSuccess; rep++) {
            cudaEventRecord(e0, ctx->stream);
            if (kind != RT_PROBE_TRAVERSAL)
                k_probe_ffma<<<grid, block, 0, ctx->stream>>>(iters, 1.0f, sink);
            else if (form == 0)
                k_probe_traversal<true><<<grid, block, 0, ctx->stream>>>(iters, n_slab / 8, n_tri, 0.0f, sink);
            else
                k_probe_traversal<false><<<grid, block, 0, ctx->stream>>>(iters, n_slab / 8, n_tri, 0.0f, sink);
            ctx->launches++;
            cudaEventRecord(e1, ctx->stream);
            err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && rep > 0) best = std::min(best, ms);   // the first launch is a warm-up
        }
        if (err == cudaSuccess) rate = std::max(rate, threads * iters * per_iter / (best * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return set_cuda(ctx, err, "probe_peak");
    *ops_per_s = rate;
    return RT_OK;
}
