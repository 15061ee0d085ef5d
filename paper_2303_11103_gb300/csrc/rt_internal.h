// rt_internal.h -- host-side context and launcher declarations shared by the
// translation units of the library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rt.h"
#include "rt_common.cuh"

// Device buffer owned by the context; grows, never shrinks.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};
cudaError_t buf_reserve(DevBuf& b, size_t bytes);
void buf_free(DevBuf& b);
template <class T>
T* bp(DevBuf& b) {
    return reinterpret_cast<T*>(b.p);
}

struct DevAntenna {
    int kind;
    int n_ports;
    float slant[2];
};

constexpr int RB_WORDS = 16;

struct rt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    double fc = 3.5e9;
    int num_sms = 152;

    // scene
    bool has_scene = false;
    int n_tris = 0, n_mat = 0, n_nodes = 0, bvh_depth = 0;
    int n_bvh = 0, n_big = 0;  // triangles in the hierarchy / tested directly (large)
    float tmin = 0.0f, extent = 1.0f;
    DevBuf nodes, tris, tris_o, planes, mat, mats;
    DevBuf wnodes;        // 8-wide layout [n_wnodes * RT_WN_F4] (when bvh_width == 8)
    int n_wnodes = 0;
    DevBuf planes64;   // [T*3] double2: FP64 unit normal and first vertex per triangle (original order)

    // devices
    int n_tx = 0, n_rx = 0;
    DevBuf tx_pos, tx_ypr, rx_pos, rx_ypr;
    DevAntenna tx_ant{0, 1, {0, 0}}, rx_ant{0, 1, {0, 0}};
    bool rx_sets = false;
    std::vector<int32_t> rx_off;  // host CSR [n_tx+1] when rx_sets
    DevBuf rx_off_d;              // device copy

    // path store
    int max_depth = 0;
    int64_t num_rays = 0;
    int64_t n_cand = 0, n_paths = 0;
    int id_bits = 1, tx_bits = 0, key_bits = 0;
    bool recorded_rays = false;
    DevBuf keys, keys_alt, vals, vals_alt;       // SBR keys + positions
    DevBuf ray_hits;
    DevBuf cand_key, cand_wit, cand_off, cand_img; // candidates
    DevBuf htab_key, htab_wit, htab_cnt;           // duplicate-removal hash table
    DevBuf dop_cyc;                                // Doppler cycles per time step, per path
    DevBuf arr_dirs;                               // per path: R_tx^T kt / lambda, R_rx^T kr / lambda
    // first-order diffraction: input vertices (kept for the edge search),
    // wedges of the scene, diffracted paths sorted by (pair, wedge)
    DevBuf verts_in, wedges;
    int64_t scene_gen = 0, wedge_gen = -1;
    int n_wedges = 0;
    int64_t n_dpaths = 0, dpath_cap = 0;
    DevBuf dpath_raw_key, dpath_raw_pt, dpath_key, dpath_key_alt, dpath_idx, dpath_idx_alt, dpath_pt, dpath_off;
    DevBuf dmap_key, dmap_pt;   // diffracted coverage map: found (tx, cell, wedge) entries
    DevBuf scat;                // [n_mat] scattering coefficients (rt_set_scattering)
    bool scat_set = false;
    DevBuf scat_alpha;          // [n_mat] int32 pattern exponent, -1 Lambertian (rt_set_scattering_pattern)
    bool scat_alpha_set = false;
    int64_t dmap_cap = 0;
    DevBuf path_key, path_key_alt, path_cap_dummy;
    DevBuf path_off, path_seq, path_pts, path_depth, path_len, path_pair;
    int64_t path_cap = 0;
    int64_t hash_hint = 0;   // hash slots the last compute_paths needed (0: read the key count first)

    // BVH build scratch (kept between builds: no allocation per rt_load_scene)
    DevBuf b_lbox, b_cent, b_info, b_keys, b_keys2, b_vals, b_vals2, b_child, b_pint, b_pleaf, b_ibox, b_flag, b_ploc,
        b_dkeys, b_dkeys2, b_rank, b_wroot;

    // scratch
    DevBuf sort_hist, scan_buf, counters, status;
    // second stream for rt_coverage_map_async: its own work counter and
    // status word; ev_side marks the end of the last map queued there
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_side = nullptr;
    bool side_pending = false;
    DevBuf side_counters, side_status;
    // a map requested with RT_ASYNC_AFTER_TRACE, not launched yet
    bool side_deferred = false;
    bool side_yield = false;   // the second stream's map is being launched as short-lived blocks
    struct SideReq {
        rt_grid g;
        int32_t D, tx_port, blocks_per_sm;
        int64_t N;
        float* gain;
        uint32_t* hits;
    } side_req{};
    int grid_cap = 0;     // resident blocks per SM of a traversal launch (0 = occupancy limit)
    uint64_t* host_rb = nullptr;  // pinned host words for device -> host reads (RB_WORDS)
    DevBuf perm;          // direction-coherent ray order
    int64_t perm_n = -1;
    DevBuf dirs;          // float4 [perm_n]: FP32 lattice direction of ray perm[k], perm[k]
    bool dirs_ok = false;

    // tuning
    int n_smem_nodes = 256;   // BVH node bytes / 64 staged in shared memory (8-wide layout)
    int bvh_builder = RT_BVH_PLOC;  // hierarchy over the Morton order: RT_BVH_KARRAS or RT_BVH_PLOC
    int bvh_width = 2;              // traversal layout: 2 (binary nodes) or 8 (wide nodes)
    int dedup = RT_DEDUP_HASH;      // candidate duplicate removal: RT_DEDUP_HASH or RT_DEDUP_SORT
    int trace_block = 256;
    int warp_chunk = 0;       // rays a warp takes per refill (0 = automatic: 32)

    // instrumentation: host count of kernel launches; optional CUDA-event
    // timing of every launch on the context's stream
    int64_t launches = 0;
    bool prof = false, prof_open = false;
    bool count_work = false;  // traversal kernels count node / triangle records and queries
    std::vector<const char*> prof_name;
    std::vector<cudaEvent_t> prof_ev;  // 2 per record
    std::vector<std::string> prof_only;  // kernels timed (empty = all)

    // CUDA graph capture
    bool capturing = false;
    cudaStream_t user_stream = nullptr, cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t launches_at_begin = 0, graph_kernels = 0;
    std::vector<void*> graph_bufs;   // addresses of the buffers a graph may use, at capture
};

// Bracket one kernel launch: counts it and, when profiling, records CUDA
// events on the context's stream right before and after it.
// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` (the attribute call is made once per kernel, device and size
// increase; thread-safe).
cudaError_t ensure_smem_attr(const void* kernel, size_t bytes);
// resident blocks per SM of kernel at (block, dynamic shared memory), cached per device
int blocks_per_sm(const void* kernel, int block, size_t smem);

void prof_begin(rt_ctx* ctx, const char* name);
void prof_end(rt_ctx* ctx);

#define RT_TRY(expr)                                       \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return set_cuda(ctx, e_, #expr); \
    } while (0)

int set_err(rt_ctx* ctx, int code, const std::string& msg);
int set_cuda(rt_ctx* ctx, cudaError_t e, const char* what);
DevScene dev_scene(rt_ctx* ctx);

// The traversal layout of the context's scene, and the nodes the traversal
// kernels stage in shared memory: the 8-wide layout stages the top of its
// tree (n_smem_nodes counts 64-byte binary nodes' worth of bytes); the
// binary layout stages nothing (each ray reads its octant's copy of the
// nodes through L1).
inline bool wide_layout(const rt_ctx* c) { return c->bvh_width == 8 && c->n_wnodes > 0; }
inline int staged_nodes(const rt_ctx* c) {
    if (!wide_layout(c)) return 0;
    const int n = c->n_smem_nodes * 4 / RT_WN_F4;
    return n < c->n_wnodes ? n : c->n_wnodes;
}
inline size_t staged_bytes(const rt_ctx* c) {
    return sizeof(float4) * (wide_layout(c) ? RT_WN_F4 : 4) * (size_t)staged_nodes(c);
}

// radix sort of 64-bit keys with an optional 32-bit payload, bits [0, end_bit)
// result in keys/vals (alt buffers used as ping-pong), n may be 0
cudaError_t radix_sort64(rt_ctx* ctx, uint64_t* keys, uint64_t* keys_alt, uint32_t* vals,
                         uint32_t* vals_alt, int64_t n, int end_bit);

cudaError_t exclusive_scan_u32(rt_ctx* ctx, uint32_t* a, int64_t m);

// BVH build from the context's original-order triangle buffers
int bvh_build(rt_ctx* ctx, const float* verts, int64_t n_tris);

// ray order (direction-coherent permutation of [0, N))
int ensure_perm(rt_ctx* ctx, int64_t N);
// orders the context stream after the map of rt_coverage_map_async
// (launching it first if it was deferred)
int side_join(rt_ctx* ctx);
// launches a deferred map on the second stream, after the work queued so far
int side_launch(rt_ctx* ctx);
