// rt_api.cu -- the C ABI (include/rt.h): context, argument checks, buffer
// ownership and error reporting around the kernels.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <utility>

#include "rt_internal.h"

int compute_paths_impl(rt_ctx* ctx, int D, int64_t N, uint32_t flags, int64_t* out);
int export_candidates(rt_ctx* ctx, int32_t* tx, int32_t* depth, int32_t* seq, int64_t* wit);
int cir_impl(rt_ctx* ctx, uint32_t flags, float* a, float* tau);
int doppler_impl(rt_ctx* ctx, const float* a, const float* vtx, const float* vrx, double fs, int T, float* a_t);
int array_impl(rt_ctx* ctx, const float* a, const float* tel, int Mt, const float* rel, int Mr, float* a_el);
int diffraction_impl(rt_ctx* ctx, int64_t* n_out);
int diffraction_cir_impl(rt_ctx* ctx, float* a, float* tau);
int diffraction_get_impl(rt_ctx* ctx, int64_t* offsets, int32_t* wedge, float* points);
int wedges_impl(rt_ctx* ctx, int64_t* n_out, int32_t* faces, float* n_ext);
int diffraction_map_impl(rt_ctx* ctx, const rt_grid* g, int tx_port, float* gain);
int scattering_impl(rt_ctx* ctx, int64_t N, float* gain, const float* up, float* grad);
int cir_vjp_impl(rt_ctx* ctx, uint32_t flags, const float* ga, const float* gtau, float* g_eps, float* g_sig,
                 float* g_pos, float* g_ypr);
int freq_impl(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int K, float* H,
              int64_t n_pairs);
int freq_csr_impl(rt_ctx* ctx, const int64_t* off, int64_t n_pairs, int np, const float* a, const float* tau,
                  const double* freqs, int K, float* H);
int freq_vjp_impl(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int K, const float* gH,
                  float* ga, float* gt, int64_t n_pairs);
int launch_coverage_vjp(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int tx_port, const float* grad_gain,
                        float* grad_ypr);
int launch_coverage(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int64_t first, int64_t count, bool zero,
                    int tx_port, float* gain, uint32_t* hits);
int launch_dirs(rt_ctx* ctx, int64_t N, int64_t first, int64_t n, float* out);
int pair_gain_impl(rt_ctx* ctx, const float* a, float floor_db, float* out, int64_t n_pairs);

cudaError_t buf_reserve(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return e;
    }
    b.bytes = want;
    return cudaSuccess;
}

void buf_free(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int set_err(rt_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int set_cuda(rt_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return set_err(ctx, e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, m);
}

DevScene dev_scene(rt_ctx* ctx) {
    DevScene s;
    s.nodes = bp<float4>(ctx->nodes);
    s.wnodes = bp<float4>(ctx->wnodes);
    s.n_wnodes = ctx->n_wnodes;
    s.wide = wide_layout(ctx) ? 1 : 0;
    s.tris = bp<float4>(ctx->tris);
    s.tris_o = bp<float4>(ctx->tris_o);
    s.planes = bp<float4>(ctx->planes);
    s.pl64 = bp<double2>(ctx->planes64);
    s.mat = bp<int32_t>(ctx->mat);
    s.mats = bp<float2>(ctx->mats);
    s.big = bp<float4>(ctx->tris) + 3 * (size_t)ctx->n_bvh;
    s.n_big = ctx->n_big;
    s.n_tris = ctx->n_tris;
    s.n_nodes = ctx->n_nodes;
    s.n_mat = ctx->n_mat;
    s.tmin = ctx->tmin;
    return s;
}

static const size_t PROF_MAX = 1 << 16;

cudaError_t ensure_smem_attr(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = done[{dev, kernel}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

int blocks_per_sm(const void* kernel, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(dev, kernel, block, smem);
    auto it = done.find(key);
    if (it != done.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    done[key] = n;
    return n;
}

void prof_begin(rt_ctx* ctx, const char* name) {
    ctx->launches++;
    if (!ctx->prof || ctx->capturing || ctx->prof_name.size() >= PROF_MAX) return;
    if (!ctx->prof_only.empty() &&
        std::find(ctx->prof_only.begin(), ctx->prof_only.end(), name) == ctx->prof_only.end())
        return;
    size_t k = ctx->prof_name.size();
    while (ctx->prof_ev.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        ctx->prof_ev.push_back(e);
    }
    cudaEventRecord(ctx->prof_ev[2 * k], ctx->stream);
    ctx->prof_name.push_back(name);
    ctx->prof_open = true;
}

void prof_end(rt_ctx* ctx) {
    if (!ctx->prof_open) return;
    ctx->prof_open = false;
    size_t k = ctx->prof_name.size() - 1;
    cudaEventRecord(ctx->prof_ev[2 * k + 1], ctx->stream);
}

static int use_device(rt_ctx* ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_cuda(ctx, e, "cudaSetDevice");
    return RT_OK;
}

#define CHECK_CTX(c)                       \
    do {                                   \
        if (!(c)) return RT_ERR_INVALID_ARG; \
        int e__ = use_device(c);           \
        if (e__) return e__;               \
    } while (0)

#define NO_CAPTURE(c, what)                                                        \
    do {                                                                           \
        if ((c)->capturing)                                                        \
            return set_err(c, RT_ERR_NOT_READY, what ": reads results back, not allowed while capturing"); \
    } while (0)

static bool valid_antenna(const rt_antenna* a) {
    return a && a->kind >= RT_ANT_ISO && a->kind <= RT_ANT_TR38901 && (a->n_ports == 1 || a->n_ports == 2);
}

int side_launch(rt_ctx* ctx) {
    if (!ctx->side_deferred) return RT_OK;
    ctx->side_deferred = false;
    const rt_ctx::SideReq r = ctx->side_req;
    RT_TRY(cudaEventRecord(ctx->ev_fork, ctx->stream));
    RT_TRY(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    // the launch code uses the context's stream, counter and status word:
    // point them at the second stream's for this one launch
    std::swap(ctx->stream, ctx->side);
    std::swap(ctx->counters, ctx->side_counters);
    std::swap(ctx->status, ctx->side_status);
    const int cap = ctx->grid_cap;
    ctx->grid_cap = r.blocks_per_sm;
    ctx->side_yield = r.blocks_per_sm == 0;
    cudaError_t me = cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), ctx->stream);
    int e = me != cudaSuccess ? set_cuda(ctx, me, "cudaMemsetAsync")
                              : launch_coverage(ctx, &r.g, r.D, r.N, 0, r.N, true, r.tx_port, r.gain, r.hits);
    ctx->grid_cap = cap;
    ctx->side_yield = false;
    std::swap(ctx->stream, ctx->side);
    std::swap(ctx->counters, ctx->side_counters);
    std::swap(ctx->status, ctx->side_status);
    // whatever was queued, later calls that need it wait for its end
    RT_TRY(cudaEventRecord(ctx->ev_side, ctx->side));
    ctx->side_pending = true;
    return e;
}

int side_join(rt_ctx* ctx) {
    int e = side_launch(ctx);
    if (!ctx->side_pending) return e;
    ctx->side_pending = false;
    RT_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_side, 0));
    return e;
}

extern "C" {

int rt_create(rt_ctx** out, int device, void* stream) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return RT_ERR_INVALID_ARG;
    }
    rt_ctx* ctx = new (std::nothrow) rt_ctx();
    if (!ctx) return RT_ERR_OOM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return RT_ERR_CUDA;
    }
    if (buf_reserve(ctx->counters, 64) != cudaSuccess || buf_reserve(ctx->status, 64) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->host_rb, sizeof(uint64_t) * RB_WORDS) != cudaSuccess) {
        cudaGetLastError();
        buf_free(ctx->counters);
        buf_free(ctx->status);
        delete ctx;
        return RT_ERR_OOM;
    }
    *out = ctx;
    return RT_OK;
}

int rt_destroy(rt_ctx* ctx) {
    if (!ctx) return RT_OK;
    cudaSetDevice(ctx->device);
    ctx->side_deferred = false;   // a map still waiting for a path trace is dropped, not started
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
        cudaEventDestroy(ctx->ev_fork);
        cudaEventDestroy(ctx->ev_side);
        buf_free(ctx->side_counters);
        buf_free(ctx->side_status);
    }
    for (DevBuf* b : {&ctx->nodes, &ctx->tris, &ctx->tris_o, &ctx->planes, &ctx->planes64, &ctx->mat, &ctx->mats, &ctx->tx_pos,
                      &ctx->tx_ypr, &ctx->rx_pos, &ctx->rx_ypr, &ctx->rx_off_d, &ctx->keys, &ctx->keys_alt,
                      &ctx->vals, &ctx->vals_alt, &ctx->ray_hits, &ctx->cand_key, &ctx->cand_wit, &ctx->cand_off,
                      &ctx->cand_img, &ctx->htab_key, &ctx->htab_wit, &ctx->htab_cnt, &ctx->dop_cyc, &ctx->arr_dirs,
                      &ctx->verts_in, &ctx->wedges, &ctx->dpath_raw_key, &ctx->dpath_raw_pt, &ctx->dpath_key,
                      &ctx->dpath_key_alt, &ctx->dpath_idx, &ctx->dpath_idx_alt, &ctx->dpath_pt, &ctx->dpath_off,
                      &ctx->dmap_key, &ctx->dmap_pt, &ctx->scat, &ctx->scat_alpha, &ctx->path_key,
                      &ctx->path_key_alt, &ctx->path_cap_dummy, &ctx->path_off,
                      &ctx->path_seq, &ctx->path_pts, &ctx->path_depth, &ctx->path_len, &ctx->path_pair,
                      &ctx->sort_hist, &ctx->scan_buf, &ctx->counters, &ctx->status, &ctx->perm, &ctx->dirs,
                      &ctx->b_lbox, &ctx->b_cent, &ctx->b_info, &ctx->b_keys, &ctx->b_keys2, &ctx->b_vals,
                      &ctx->b_vals2, &ctx->b_child, &ctx->b_pint, &ctx->b_pleaf, &ctx->b_ibox, &ctx->b_flag, &ctx->b_ploc,
                      &ctx->b_dkeys, &ctx->b_dkeys2, &ctx->b_rank, &ctx->b_wroot, &ctx->wnodes})
        buf_free(*b);
    if (ctx->host_rb) cudaFreeHost(ctx->host_rb);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return RT_OK;
}

int rt_set_stream(rt_ctx* ctx, void* stream) {
    CHECK_CTX(ctx);
    if ((cudaStream_t)stream == ctx->stream) return RT_OK;
    ctx->stream = (cudaStream_t)stream;
    return side_join(ctx);   // a map still running on the second stream comes before the new stream's work
}

int rt_join(rt_ctx* ctx) {
    CHECK_CTX(ctx);
    return side_join(ctx);
}

int rt_last_error(const rt_ctx* ctx, char* buf, size_t len) {
    if (!ctx || !buf || len == 0) return RT_ERR_INVALID_ARG;
    size_t n = std::min(len - 1, ctx->err.size());
    memcpy(buf, ctx->err.data(), n);
    buf[n] = 0;
    return RT_OK;
}

int rt_set_frequency(rt_ctx* ctx, double fc) {
    CHECK_CTX(ctx);
    if (!(fc > 0.0)) return set_err(ctx, RT_ERR_INVALID_ARG, "frequency must be positive");
    {
        int ej = side_join(ctx);   // a deferred map is traced at the frequency it was requested at
        if (ej) return ej;
    }
    ctx->fc = fc;
    return RT_OK;
}

int rt_load_scene(rt_ctx* ctx, const float* verts, int64_t n_tris, const int32_t* mat_id, const float* mat_params,
                  int32_t n_mat) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "load_scene");
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (n_tris < 0 || n_tris >= (1ll << 30) || n_mat <= 0 || !mat_params || (n_tris > 0 && (!verts || !mat_id)))
        return set_err(ctx, RT_ERR_INVALID_ARG, "load_scene: bad arguments");
    ctx->has_scene = false;
    ctx->n_paths = 0;
    ctx->n_cand = 0;
    ctx->n_dpaths = 0;
    ctx->scat_set = false;
    ctx->scat_alpha_set = false;
    ctx->scene_gen++;
    ctx->n_mat = n_mat;
    RT_TRY(buf_reserve(ctx->verts_in, sizeof(float) * 9 * std::max<int64_t>(n_tris, 1)));
    if (n_tris > 0)
        RT_TRY(cudaMemcpyAsync(ctx->verts_in.p, verts, sizeof(float) * 9 * n_tris, cudaMemcpyDeviceToDevice,
                               ctx->stream));
    RT_TRY(buf_reserve(ctx->mats, sizeof(float) * 2 * n_mat));
    RT_TRY(cudaMemcpyAsync(ctx->mats.p, mat_params, sizeof(float) * 2 * n_mat, cudaMemcpyDeviceToDevice, ctx->stream));
    RT_TRY(buf_reserve(ctx->mat, sizeof(int32_t) * std::max<int64_t>(n_tris, 1)));
    if (n_tris > 0)
        RT_TRY(cudaMemcpyAsync(ctx->mat.p, mat_id, sizeof(int32_t) * n_tris, cudaMemcpyDeviceToDevice, ctx->stream));
    int e = bvh_build(ctx, verts, n_tris);
    if (e) return e;
    ctx->has_scene = true;
    return RT_OK;
}

int rt_set_bvh_builder(rt_ctx* ctx, int32_t builder) {
    CHECK_CTX(ctx);
    if (builder != RT_BVH_KARRAS && builder != RT_BVH_PLOC)
        return set_err(ctx, RT_ERR_INVALID_ARG, "unknown BVH builder");
    ctx->bvh_builder = builder;
    return RT_OK;
}

int rt_set_bvh_width(rt_ctx* ctx, int32_t width) {
    CHECK_CTX(ctx);
    if (width != 2 && width != 8) return set_err(ctx, RT_ERR_INVALID_ARG, "BVH width must be 2 or 8");
    ctx->bvh_width = width;
    return RT_OK;
}

int rt_get_bvh(rt_ctx* ctx, float* nodes, int64_t cap, int64_t* n_nodes) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "get_bvh");
    if (!n_nodes || cap < 0) return set_err(ctx, RT_ERR_INVALID_ARG, "get_bvh: bad arguments");
    const int64_t n = ctx->has_scene ? ctx->n_nodes : 0;
    *n_nodes = n;
    if (!nodes || cap < n || n == 0) return RT_OK;
    RT_TRY(cudaMemcpyAsync(nodes, ctx->nodes.p, sizeof(float4) * 4 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    RT_TRY(cudaStreamSynchronize(ctx->stream));
    return RT_OK;
}

int rt_set_dedup(rt_ctx* ctx, int32_t mode) {
    CHECK_CTX(ctx);
    if (mode != RT_DEDUP_HASH && mode != RT_DEDUP_SORT) return set_err(ctx, RT_ERR_INVALID_ARG, "unknown dedup mode");
    ctx->dedup = mode;
    return RT_OK;
}

int rt_set_materials(rt_ctx* ctx, const float* mat_params, int32_t n_mat) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (!ctx->has_scene || n_mat != ctx->n_mat || !mat_params)
        return set_err(ctx, RT_ERR_INVALID_ARG, "set_materials: material count differs from the scene's");
    RT_TRY(cudaMemcpyAsync(ctx->mats.p, mat_params, sizeof(float) * 2 * n_mat, cudaMemcpyDeviceToDevice, ctx->stream));
    return RT_OK;
}

static int set_devices(rt_ctx* ctx, DevBuf& pos, DevBuf& ypr, const float* p, const float* y, int32_t n) {
    RT_TRY(buf_reserve(pos, sizeof(float) * 3 * std::max(n, 1)));
    RT_TRY(buf_reserve(ypr, sizeof(float) * 3 * std::max(n, 1)));
    if (n > 0) {
        RT_TRY(cudaMemcpyAsync(pos.p, p, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, ctx->stream));
        if (y)
            RT_TRY(cudaMemcpyAsync(ypr.p, y, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, ctx->stream));
        else
            RT_TRY(cudaMemsetAsync(ypr.p, 0, sizeof(float) * 3 * n, ctx->stream));
    }
    return RT_OK;
}

int rt_set_tx(rt_ctx* ctx, const float* pos, const float* ypr, int32_t n, const rt_antenna* pat) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (n < 1 || !pos || !valid_antenna(pat)) return set_err(ctx, RT_ERR_INVALID_ARG, "set_tx: bad arguments");
    // Same count and ports: a pose update. The stored paths (triangle
    // sequences) and receiver sets stay; rt_cir re-evaluates the paths at
    // the new pose (replay for gradients). Otherwise both are dropped.
    bool pose_only = n == ctx->n_tx && pat->n_ports == ctx->tx_ant.n_ports;
    int e = set_devices(ctx, ctx->tx_pos, ctx->tx_ypr, pos, ypr, n);
    if (e) return e;
    ctx->n_tx = n;
    ctx->tx_ant = {pat->kind, pat->n_ports, {pat->slant[0], pat->slant[1]}};
    if (!pose_only) {
        ctx->rx_sets = false;
        ctx->n_paths = 0;
    }
    return RT_OK;
}

int rt_set_rx(rt_ctx* ctx, const float* pos, const float* ypr, int32_t m, const rt_antenna* pat,
              const int32_t* off_host) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (m < 1 || !pos || !valid_antenna(pat)) return set_err(ctx, RT_ERR_INVALID_ARG, "set_rx: bad arguments");
    if (off_host) {
        NO_CAPTURE(ctx, "set_rx with receiver sets");
        if (ctx->n_tx < 1) return set_err(ctx, RT_ERR_INVALID_ARG, "set_rx: receiver sets need set_tx first");
        if (off_host[0] != 0 || off_host[ctx->n_tx] != m)
            return set_err(ctx, RT_ERR_INVALID_ARG, "set_rx: offsets must start at 0 and end at m");
        for (int t = 0; t < ctx->n_tx; t++)
            if (off_host[t + 1] < off_host[t]) return set_err(ctx, RT_ERR_INVALID_ARG, "set_rx: decreasing offsets");
    }
    int e = set_devices(ctx, ctx->rx_pos, ctx->rx_ypr, pos, ypr, m);
    if (e) return e;
    ctx->n_rx = m;
    ctx->rx_ant = {pat->kind, pat->n_ports, {pat->slant[0], pat->slant[1]}};
    ctx->rx_sets = off_host != nullptr;
    ctx->rx_off.assign(off_host ? off_host : nullptr, off_host ? off_host + ctx->n_tx + 1 : nullptr);
    if (ctx->rx_sets) {
        RT_TRY(buf_reserve(ctx->rx_off_d, sizeof(int32_t) * (ctx->n_tx + 1)));
        RT_TRY(cudaMemcpyAsync(ctx->rx_off_d.p, ctx->rx_off.data(), sizeof(int32_t) * (ctx->n_tx + 1),
                               cudaMemcpyHostToDevice, ctx->stream));
        RT_TRY(cudaStreamSynchronize(ctx->stream));
    }
    ctx->n_paths = 0;
    return RT_OK;
}

int rt_ray_directions(rt_ctx* ctx, int64_t num_rays, int64_t first, int64_t n, float* dirs) {
    CHECK_CTX(ctx);
    if (num_rays < 1 || first < 0 || n < 0 || first + n > num_rays || (n > 0 && !dirs))
        return set_err(ctx, RT_ERR_INVALID_ARG, "ray_directions: bad range");
    return launch_dirs(ctx, num_rays, first, n, dirs);
}

int rt_num_pairs(const rt_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return RT_ERR_INVALID_ARG;
    *n = ctx->rx_sets ? (int64_t)ctx->rx_off[ctx->n_tx] : (int64_t)ctx->n_tx * ctx->n_rx;
    return RT_OK;
}

int rt_compute_paths(rt_ctx* ctx, int32_t max_depth, int64_t num_rays, uint32_t flags, int64_t* num_paths) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "compute_paths");
    if (!num_paths || max_depth < 0 || max_depth > RT_MAX_DEPTH || num_rays < 0)
        return set_err(ctx, RT_ERR_INVALID_ARG, "compute_paths: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "compute_paths: scene, transmitters and receivers must be set");
    *num_paths = 0;
    ctx->n_paths = 0;
    return compute_paths_impl(ctx, max_depth, num_rays, flags, num_paths);
}

int rt_get_paths(rt_ctx* ctx, int64_t* offsets, int32_t* seq, float* points, int32_t* depth, double* length) {
    CHECK_CTX(ctx);
    int64_t np = 0;
    rt_num_pairs(ctx, &np);
    const int64_t P = ctx->n_paths;
    const int D = ctx->max_depth;
    cudaStream_t st = ctx->stream;
    if (offsets) RT_TRY(cudaMemcpyAsync(offsets, ctx->path_off.p, sizeof(int64_t) * (np + 1), cudaMemcpyDeviceToDevice, st));
    if (P > 0) {
        if (seq) RT_TRY(cudaMemcpyAsync(seq, ctx->path_seq.p, sizeof(int32_t) * P * D, cudaMemcpyDeviceToDevice, st));
        if (points) RT_TRY(cudaMemcpyAsync(points, ctx->path_pts.p, sizeof(float) * 3 * P * D, cudaMemcpyDeviceToDevice, st));
        if (depth) RT_TRY(cudaMemcpyAsync(depth, ctx->path_depth.p, sizeof(int32_t) * P, cudaMemcpyDeviceToDevice, st));
        if (length) RT_TRY(cudaMemcpyAsync(length, ctx->path_len.p, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
    }
    return RT_OK;
}

int rt_get_candidates(rt_ctx* ctx, int64_t* n_out, int32_t* tx, int32_t* depth, int32_t* seq, int64_t* wit) {
    CHECK_CTX(ctx);
    if (!n_out) return RT_ERR_INVALID_ARG;
    *n_out = ctx->n_cand;
    return export_candidates(ctx, tx, depth, seq, wit);
}

int rt_get_ray_hits(rt_ctx* ctx, int32_t* hits) {
    CHECK_CTX(ctx);
    if (!ctx->recorded_rays || !hits)
        return set_err(ctx, RT_ERR_NOT_READY, "get_ray_hits: compute_paths ran without RT_RECORD_RAYS");
    size_t n = (size_t)ctx->n_tx * ctx->num_rays * ctx->max_depth;
    RT_TRY(cudaMemcpyAsync(hits, ctx->ray_hits.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    return RT_OK;
}

int rt_cir(rt_ctx* ctx, uint32_t flags, float* a, float* tau) {
    CHECK_CTX(ctx);
    if ((!a || !tau) && ctx->n_paths > 0) return set_err(ctx, RT_ERR_INVALID_ARG, "cir: null output");
    return cir_impl(ctx, flags, a, tau);
}

int rt_apply_doppler(rt_ctx* ctx, const float* a, const float* tx_vel, const float* rx_vel, double fs,
                     int32_t n_steps, float* a_t) {
    CHECK_CTX(ctx);
    if (n_steps < 1 || !(fs > 0.0) || !tx_vel || ((!a || !a_t) && ctx->n_paths > 0))
        return set_err(ctx, RT_ERR_INVALID_ARG, "apply_doppler: bad arguments");
    return doppler_impl(ctx, a, tx_vel, rx_vel, fs, n_steps, a_t);
}

int rt_apply_array(rt_ctx* ctx, const float* a, const float* tx_elements, int32_t n_tx_el, const float* rx_elements,
                   int32_t n_rx_el, float* a_el) {
    CHECK_CTX(ctx);
    if (n_tx_el < 0 || n_rx_el < 0 || (n_tx_el > 0 && !tx_elements) || (n_rx_el > 0 && !rx_elements) ||
        ((!a || !a_el) && ctx->n_paths > 0))
        return set_err(ctx, RT_ERR_INVALID_ARG, "apply_array: bad arguments");
    // no element list: one element at the centre
    return array_impl(ctx, a, n_tx_el > 0 ? tx_elements : nullptr, std::max(n_tx_el, 1),
                      n_rx_el > 0 ? rx_elements : nullptr, std::max(n_rx_el, 1), a_el);
}

int rt_compute_diffraction(rt_ctx* ctx, int64_t* num_paths) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "compute_diffraction");
    if (!num_paths) return set_err(ctx, RT_ERR_INVALID_ARG, "compute_diffraction: null count");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "compute_diffraction: scene, transmitters and receivers must be set");
    return diffraction_impl(ctx, num_paths);
}

int rt_get_diffraction(rt_ctx* ctx, int64_t* offsets, int32_t* wedge, float* points) {
    CHECK_CTX(ctx);
    return diffraction_get_impl(ctx, offsets, wedge, points);
}

int rt_diffraction_cir(rt_ctx* ctx, float* a, float* tau) {
    CHECK_CTX(ctx);
    if ((!a || !tau) && ctx->n_dpaths > 0) return set_err(ctx, RT_ERR_INVALID_ARG, "diffraction_cir: null output");
    return diffraction_cir_impl(ctx, a, tau);
}

int rt_coverage_map_diffraction(rt_ctx* ctx, const rt_grid* g, int32_t tx_port, float* gain) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "coverage_map_diffraction");
    if (!g || !gain || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || tx_port < 0 || tx_port >= ctx->tx_ant.n_ports ||
        (int64_t)g->nx * g->ny * ctx->n_tx >= (1ll << 32))
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_diffraction: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_diffraction: scene, transmitters and receivers must be set");
    return diffraction_map_impl(ctx, g, tx_port, gain);
}

int rt_set_scattering(rt_ctx* ctx, const float* coeff, int32_t n_mat) {
    CHECK_CTX(ctx);
    if (!ctx->has_scene || n_mat != ctx->n_mat || !coeff)
        return set_err(ctx, RT_ERR_INVALID_ARG, "set_scattering: material count differs from the scene's");
    RT_TRY(buf_reserve(ctx->scat, sizeof(float) * n_mat));
    RT_TRY(cudaMemcpyAsync(ctx->scat.p, coeff, sizeof(float) * n_mat, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->scat_set = true;
    return RT_OK;
}

int rt_set_scattering_pattern(rt_ctx* ctx, const int32_t* alpha_r, int32_t n_mat) {
    CHECK_CTX(ctx);
    if (!ctx->has_scene || n_mat != ctx->n_mat || !alpha_r)
        return set_err(ctx, RT_ERR_INVALID_ARG, "set_scattering_pattern: material count differs from the scene's");
    for (int i = 0; i < n_mat; i++)
        if (alpha_r[i] < -1 || alpha_r[i] > RT_MAX_ALPHA_R)
            return set_err(ctx, RT_ERR_INVALID_ARG, "set_scattering_pattern: alpha_r must be -1 or 0..64");
    RT_TRY(buf_reserve(ctx->scat_alpha, sizeof(int32_t) * n_mat));
    RT_TRY(cudaMemcpyAsync(ctx->scat_alpha.p, alpha_r, sizeof(int32_t) * n_mat, cudaMemcpyHostToDevice, ctx->stream));
    RT_TRY(cudaStreamSynchronize(ctx->stream));   // the host array may go away after the call
    ctx->scat_alpha_set = true;
    return RT_OK;
}

int rt_scattering_gain(rt_ctx* ctx, int64_t num_rays, float* gain) {
    CHECK_CTX(ctx);
    if (num_rays < 0 || num_rays >= (1ll << 40) || !gain)
        return set_err(ctx, RT_ERR_INVALID_ARG, "scattering_gain: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "scattering_gain: scene, transmitters and receivers must be set");
    return scattering_impl(ctx, num_rays, gain, nullptr, nullptr);
}

int rt_scattering_gain_vjp(rt_ctx* ctx, int64_t num_rays, const float* grad_gain, float* grad_coeff) {
    CHECK_CTX(ctx);
    if (num_rays < 0 || num_rays >= (1ll << 40) || !grad_gain || !grad_coeff)
        return set_err(ctx, RT_ERR_INVALID_ARG, "scattering_gain_vjp: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "scattering_gain_vjp: scene, transmitters and receivers must be set");
    return scattering_impl(ctx, num_rays, nullptr, grad_gain, grad_coeff);
}

int rt_get_wedges(rt_ctx* ctx, int64_t* n_out, int32_t* faces, float* n_ext) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "get_wedges");
    if (!n_out) return set_err(ctx, RT_ERR_INVALID_ARG, "get_wedges: null count");
    if (!ctx->has_scene) return set_err(ctx, RT_ERR_INVALID_ARG, "get_wedges: no scene");
    return wedges_impl(ctx, n_out, faces, n_ext);
}

int rt_freq_response(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int32_t K, float* H) {
    CHECK_CTX(ctx);
    if (K < 0 || (K > 0 && (!freqs || !H)) || ((!a || !tau) && ctx->n_paths > 0))
        return set_err(ctx, RT_ERR_INVALID_ARG, "freq_response: bad arguments");
    int64_t np = 0;
    rt_num_pairs(ctx, &np);
    return freq_impl(ctx, a, tau, freqs, K, H, np);
}

int rt_freq_response_paths(rt_ctx* ctx, const int64_t* offsets, int64_t n_pairs, int32_t n_port_pairs,
                           const float* a, const float* tau, const double* freqs, int32_t K, float* H) {
    CHECK_CTX(ctx);
    if (n_pairs < 0 || K < 0 || (n_port_pairs != 1 && n_port_pairs != 2 && n_port_pairs != 4) ||
        (n_pairs > 0 && K > 0 && (!offsets || !a || !tau || !freqs || !H)))
        return set_err(ctx, RT_ERR_INVALID_ARG, "freq_response_paths: bad arguments");
    if (n_pairs > 0x7fffffffll) return set_err(ctx, RT_ERR_INVALID_ARG, "freq_response_paths: n_pairs above 2^31-1");
    return freq_csr_impl(ctx, offsets, n_pairs, n_port_pairs, a, tau, freqs, K, H);
}

int rt_coverage_map(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, int32_t tx_port,
                    float* gain, uint32_t* hits) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (!g || !gain || !hits || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || max_depth < 0 || num_rays < 1 ||
        tx_port < 0 || tx_port >= ctx->tx_ant.n_ports)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map: scene, transmitters and receivers must be set");
    RT_TRY(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), ctx->stream));
    return launch_coverage(ctx, g, max_depth, num_rays, 0, num_rays, true, tx_port, gain, hits);
}

int rt_coverage_map_accumulate(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays,
                               int64_t first_ray, int64_t ray_count, int32_t tx_port, float* gain, uint32_t* hits) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (!g || !gain || !hits || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || max_depth < 0 || num_rays < 1 ||
        first_ray < 0 || ray_count < 0 || first_ray + ray_count > num_rays || tx_port < 0 ||
        tx_port >= ctx->tx_ant.n_ports)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_accumulate: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_accumulate: scene, transmitters and receivers must be set");
    return launch_coverage(ctx, g, max_depth, num_rays, first_ray, ray_count, false, tx_port, gain, hits);
}

int rt_coverage_map_async(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, int32_t tx_port,
                          uint32_t flags, int32_t blocks_per_sm, float* gain, uint32_t* hits) {
    CHECK_CTX(ctx);
    if (ctx->capturing) return set_err(ctx, RT_ERR_NOT_READY, "coverage_map_async while capturing a graph");
    if (!g || !gain || !hits || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || max_depth < 0 || num_rays < 1 ||
        tx_port < 0 || tx_port >= ctx->tx_ant.n_ports || blocks_per_sm < 0 || (flags & ~RT_ASYNC_AFTER_TRACE))
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_async: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_async: scene, transmitters and receivers must be set");
    int e = side_join(ctx);   // one map at a time
    if (e) return e;
    if (!ctx->side) {
        int least = 0, greatest = 0;
        RT_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        RT_TRY(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, least));
        RT_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        RT_TRY(cudaEventCreateWithFlags(&ctx->ev_side, cudaEventDisableTiming));
    }
    RT_TRY(buf_reserve(ctx->side_counters, 64));
    RT_TRY(buf_reserve(ctx->side_status, 64));
    e = ensure_perm(ctx, num_rays);   // the ray order is built on the context stream
    if (e) return e;
    ctx->side_req = {*g, max_depth, tx_port, blocks_per_sm, num_rays, gain, hits};
    ctx->side_deferred = true;
    return (flags & RT_ASYNC_AFTER_TRACE) ? RT_OK : side_launch(ctx);
}

int rt_coverage_map_backward(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, int32_t tx_port,
                             const float* grad_gain, float* grad_ypr) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    NO_CAPTURE(ctx, "coverage_map_backward");
    if (!g || !grad_gain || !grad_ypr || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || max_depth < 0 ||
        num_rays < 1 || tx_port < 0 || tx_port >= ctx->tx_ant.n_ports)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_backward: bad arguments");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_backward: scene, transmitters and receivers must be set");
    return launch_coverage_vjp(ctx, g, max_depth, num_rays, tx_port, grad_gain, grad_ypr);
}

int rt_cir_backward(rt_ctx* ctx, uint32_t flags, const float* grad_a, const float* grad_tau, float* g_eps,
                    float* g_sigma, float* g_txpos, float* g_txypr) {
    CHECK_CTX(ctx);
    if (!grad_a && ctx->n_paths > 0) return set_err(ctx, RT_ERR_INVALID_ARG, "cir_backward: null grad_a");
    return cir_vjp_impl(ctx, flags, grad_a, grad_tau, g_eps, g_sigma, g_txpos, g_txypr);
}

int rt_freq_response_backward(rt_ctx* ctx, const float* a, const float* tau, const double* freqs, int32_t K,
                              const float* grad_H, float* grad_a, float* grad_tau) {
    CHECK_CTX(ctx);
    if (K < 1 || !freqs || !grad_H || ((!a || !tau || !grad_a || !grad_tau) && ctx->n_paths > 0))
        return set_err(ctx, RT_ERR_INVALID_ARG, "freq_response_backward: bad arguments");
    int64_t np = 0;
    rt_num_pairs(ctx, &np);
    return freq_vjp_impl(ctx, a, tau, freqs, K, grad_H, grad_a, grad_tau, np);
}

int rt_pair_gain(rt_ctx* ctx, const float* a, float floor_db, float* out) {
    CHECK_CTX(ctx);
    if (!out || (!a && ctx->n_paths > 0)) return set_err(ctx, RT_ERR_INVALID_ARG, "pair_gain: null pointer");
    int64_t np = 0;
    rt_num_pairs(ctx, &np);
    return pair_gain_impl(ctx, a, floor_db, out, np);
}

// Addresses of the context buffers a captured graph may read or write. A
// later call may reallocate one of them (a larger scene, a new ray count);
// the graph would then use freed memory, so its replay is refused.
static std::vector<void*> graph_buffers(rt_ctx* ctx) {
    std::vector<void*> v;
    for (DevBuf* b : {&ctx->nodes, &ctx->wnodes, &ctx->tris, &ctx->tris_o, &ctx->planes, &ctx->planes64, &ctx->mat,
                      &ctx->mats, &ctx->tx_pos, &ctx->tx_ypr, &ctx->rx_pos, &ctx->rx_ypr, &ctx->rx_off_d, &ctx->perm,
                      &ctx->dirs, &ctx->counters, &ctx->status, &ctx->scat, &ctx->scat_alpha})
        v.push_back(b->p);
    return v;
}

int rt_graph_begin(rt_ctx* ctx) {
    CHECK_CTX(ctx);
    if (ctx->capturing) return set_err(ctx, RT_ERR_INVALID_ARG, "graph_begin: already capturing");
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    if (!ctx->cap_stream) RT_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    // the capture starts after everything already queued on the user's stream
    RT_TRY(cudaStreamSynchronize(ctx->stream));
    {
        int ej = side_launch(ctx);
        if (ej) return ej;
    }
    if (ctx->side_pending) {
        RT_TRY(cudaStreamSynchronize(ctx->side));
        ctx->side_pending = false;
    }
    ctx->user_stream = ctx->stream;
    ctx->stream = ctx->cap_stream;
    RT_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
    ctx->capturing = true;
    ctx->launches_at_begin = ctx->launches;
    return RT_OK;
}

int rt_graph_end(rt_ctx* ctx) {
    CHECK_CTX(ctx);
    if (!ctx->capturing) return set_err(ctx, RT_ERR_INVALID_ARG, "graph_end: not capturing");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    ctx->capturing = false;
    ctx->stream = ctx->user_stream;
    ctx->graph_kernels = ctx->launches - ctx->launches_at_begin;
    ctx->launches = ctx->launches_at_begin;
    if (e != cudaSuccess) return set_cuda(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    cudaGraphDestroy(g);
    ctx->graph_bufs = graph_buffers(ctx);
    if (e != cudaSuccess) {
        ctx->graph_exec = nullptr;
        return set_cuda(ctx, e, "cudaGraphInstantiate");
    }
    return RT_OK;
}

int rt_graph_launch(rt_ctx* ctx) {
    CHECK_CTX(ctx);
    if (!ctx->graph_exec) return set_err(ctx, RT_ERR_NOT_READY, "graph_launch: no graph");
    if (graph_buffers(ctx) != ctx->graph_bufs)
        return set_err(ctx, RT_ERR_NOT_READY,
                       "graph_launch: a buffer the graph uses was reallocated since capture (larger scene, "
                       "devices or ray count); capture the graph again");
    RT_TRY(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->launches += ctx->graph_kernels;
    return RT_OK;
}

int rt_get_tuning(const rt_ctx* ctx, int32_t* block, int32_t* chunk, int32_t* smem_nodes) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (block) *block = ctx->trace_block;
    if (chunk) *chunk = ctx->warp_chunk;
    if (smem_nodes) *smem_nodes = ctx->n_smem_nodes;
    return RT_OK;
}

int rt_set_tuning(rt_ctx* ctx, int32_t block, int32_t chunk, int32_t smem_nodes) {
    CHECK_CTX(ctx);
    if ((block != 128 && block != 256) || (chunk != 0 && chunk < 32) || chunk > (1 << 20) || smem_nodes < 0 ||
        (size_t)smem_nodes * 64 > 200 * 1024)
        return set_err(ctx, RT_ERR_INVALID_ARG,
                       "set_tuning: block 128|256, chunk 0 (auto) or >= 32, staged nodes <= 3200");
    {
        int ej = side_join(ctx);   // a deferred map is launched with the tuning it was requested with
        if (ej) return ej;
    }
    ctx->trace_block = block;
    ctx->warp_chunk = chunk;
    ctx->n_smem_nodes = smem_nodes;
    return RT_OK;
}

int rt_autotune(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays, float* gain, uint32_t* hits,
                const char* cache_path) {
    CHECK_CTX(ctx);
    {
        int ej = side_join(ctx);   // the map on the second stream reads what this call changes
        if (ej) return ej;
    }
    if (ctx->capturing) return set_err(ctx, RT_ERR_NOT_READY, "autotune while capturing a graph");
    char key[160];
    snprintf(key, sizeof(key), "tris=%d tx=%d rays=%lld depth=%d cells=%dx%d", ctx->n_tris, ctx->n_tx,
             (long long)num_rays, max_depth, g ? g->nx : 0, g ? g->ny : 0);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[256];
            while (fgets(line, sizeof(line), f)) {
                int b, c, s;
                char k[160];
                if (sscanf(line, "%d %d %d %159[^\n]", &b, &c, &s, k) == 4 && strcmp(k, key) == 0) {
                    fclose(f);
                    return rt_set_tuning(ctx, b, c, s);
                }
            }
            fclose(f);
        }
    }
    const int blocks[] = {128, 256};
    const int chunks[] = {0, 64, 256};   // 0 = automatic (32 rays per refill)
    // staging in shared memory applies to the 8-wide layout only (the binary
    // layout's octant copies are read through L1)
    const std::vector<int> smems = wide_layout(ctx) ? std::vector<int>{0, 256, 1024, 3072} : std::vector<int>{0};
    cudaEvent_t e0, e1;
    RT_TRY(cudaEventCreate(&e0));
    RT_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bb = ctx->trace_block, bc = ctx->warp_chunk, bs = ctx->n_smem_nodes;
    int rc = RT_OK;
    for (int b : blocks)
        for (int c : chunks)
            for (int s : smems) {
                ctx->trace_block = b;
                ctx->warp_chunk = c;
                ctx->n_smem_nodes = s;
                rc = rt_coverage_map(ctx, g, max_depth, num_rays, 0, gain, hits);  // warm (and ray order)
                if (rc) break;
                cudaEventRecord(e0, ctx->stream);
                rc = rt_coverage_map(ctx, g, max_depth, num_rays, 0, gain, hits);
                cudaEventRecord(e1, ctx->stream);
                if (rc) break;
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; bb = b; bc = c; bs = s; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->trace_block = bb;
    ctx->warp_chunk = bc;
    ctx->n_smem_nodes = bs;
    if (rc) return rc;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%d %d %d %s\n", bb, bc, bs, key);
            fclose(f);
        }
    }
    return RT_OK;
}

int rt_profile(rt_ctx* ctx, int enable) {
    CHECK_CTX(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->prof = (enable & 1) != 0;
    ctx->count_work = (enable & 2) != 0;
    ctx->prof_open = false;
    ctx->prof_name.clear();
    return RT_OK;
}

int rt_profile_select(rt_ctx* ctx, const char* names) {
    CHECK_CTX(ctx);
    ctx->prof_only.clear();
    if (!names) return RT_OK;
    std::string cur;
    for (const char* c = names;; c++) {
        if (*c == ',' || *c == 0) {
            if (!cur.empty()) ctx->prof_only.push_back(cur);
            cur.clear();
            if (*c == 0) break;
        } else if (*c != ' ') {
            cur.push_back(*c);
        }
    }
    return RT_OK;
}

int rt_profile_report(rt_ctx* ctx, char* buf, size_t len, int reset) {
    CHECK_CTX(ctx);
    NO_CAPTURE(ctx, "profile_report");
    if (!buf || len == 0) return set_err(ctx, RT_ERR_INVALID_ARG, "profile_report: null buffer");
    RT_TRY(cudaStreamSynchronize(ctx->stream));
    std::vector<std::string> names;
    std::vector<int64_t> counts;
    std::vector<double> ms;
    for (size_t k = 0; k < ctx->prof_name.size(); k++) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]) != cudaSuccess) {
            cudaGetLastError();
            t = 0.0f;
        }
        size_t j = 0;
        while (j < names.size() && names[j] != ctx->prof_name[k]) j++;
        if (j == names.size()) {
            names.push_back(ctx->prof_name[k]);
            counts.push_back(0);
            ms.push_back(0.0);
        }
        counts[j]++;
        ms[j] += t;
    }
    unsigned long long c[8] = {0};
    RT_TRY(cudaMemcpy(c, ctx->counters.p, sizeof(c), cudaMemcpyDeviceToHost));
    std::string s = "{\"launches\": " + std::to_string(ctx->launches) + ", \"kernels\": {";
    for (size_t j = 0; j < names.size(); j++) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f]", j ? ", " : "", names[j].c_str(), (long long)counts[j],
                 ms[j]);
        s += tmp;
    }
    s += "}, \"closest_hit\": " + std::to_string(c[RT_CNT_CLOSEST]) + ", \"any_hit\": " +
         std::to_string(c[RT_CNT_ANY]) + ", \"nodes\": " + std::to_string(c[RT_CNT_NODES]) +
         ", \"tris\": " + std::to_string(c[RT_CNT_TRIS]) + ", \"sbr_keys\": " + std::to_string(c[RT_CNT_KEYS]) +
         ", \"plane_segments\": " + std::to_string(c[RT_CNT_PLANE]) +
         ", \"candidates\": " + std::to_string(ctx->n_cand) + ", \"paths\": " + std::to_string(ctx->n_paths) + "}";
    size_t n = std::min(len - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
    if (reset) {
        ctx->launches = 0;
        ctx->prof_name.clear();
        ctx->prof_open = false;
        RT_TRY(cudaMemset(ctx->counters.p, 0, sizeof(c)));
    }
    return s.size() < len ? RT_OK : set_err(ctx, RT_ERR_CAPACITY, "profile_report: buffer too small");
}

}  // extern "C"
