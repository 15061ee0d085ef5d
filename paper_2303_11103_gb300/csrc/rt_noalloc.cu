// rt_noalloc.cu -- rt_coverage_map_noalloc: the coverage map without any
// device allocation. Its scratch (work counter, status word, the
// direction-coherent ray order and the counting-sort cells that build it)
// lives in one file-scope static __device__ array, sized for at most
// RT_NOALLOC_MAX_RAYS rays per transmitter.
#include "rt_field.cuh"
#include "rt_internal.h"

int launch_coverage_scratch(rt_ctx* ctx, const rt_grid* g, int D, int64_t N, int tx_port, float* gain,
                            uint32_t* hits, unsigned long long* counters, unsigned* status, const uint32_t* perm);

namespace {

constexpr int64_t NA_MAX_RAYS = 1 << 20;      // RT_NOALLOC_MAX_RAYS in include/rt.h
constexpr int NA_ZB = 64, NA_PB = 128;         // direction cells: z bands x azimuth bins
constexpr int NA_CELLS = NA_ZB * NA_PB;
constexpr size_t NA_OFF_CELLS = 256;           // after 8 counters + status
constexpr size_t NA_OFF_PERM = NA_OFF_CELLS + sizeof(uint32_t) * NA_CELLS;
constexpr size_t NA_BYTES = NA_OFF_PERM + sizeof(uint32_t) * NA_MAX_RAYS;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

__device__ __forceinline__ int na_cell(f3 d) {
    int zb = (int)((d.z + 1.0f) * 0.5f * NA_ZB);
    int pb = (int)((atan2f(d.y, d.x) + RT_PI_F) * (0.5f / RT_PI_F) * NA_PB);
    zb = min(max(zb, 0), NA_ZB - 1);
    pb = min(max(pb, 0), NA_PB - 1);
    return zb * NA_PB + pb;
}

__global__ void k_na_count(long long N, uint32_t* __restrict__ cells) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) atomicAdd(cells + na_cell(fib_dir(N, i)), 1u);
}

// exclusive scan of the NA_CELLS cell counts, one block
__global__ void __launch_bounds__(1024) k_na_scan(uint32_t* __restrict__ cells) {
    __shared__ uint32_t part[1024];
    constexpr int PER = NA_CELLS / 1024;
    uint32_t v[PER], s = 0;
    for (int k = 0; k < PER; k++) {
        v[k] = cells[threadIdx.x * PER + k];
        s += v[k];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        uint32_t x = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int k = 0; k < PER; k++) {
        cells[threadIdx.x * PER + k] = run;
        run += v[k];
    }
}

// rays of the same direction cell become neighbours in the trace order
__global__ void k_na_scatter(long long N, uint32_t* __restrict__ cells, uint32_t* __restrict__ perm) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) perm[atomicAdd(cells + na_cell(fib_dir(N, i)), 1u)] = (uint32_t)i;
}

// Device address of the scratch array in the current context, looked up on
// every call with the context's device current: a cached address would
// dangle after cudaDeviceReset or under another context of the same device.
// The lookup allocates nothing; the first one on a device may load the
// library's module, which is why the first call belongs before any capture.
int na_scratch(rt_ctx* ctx, unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_cuda(ctx, e, "cudaGetSymbolAddress(noalloc scratch)");
    *out = (unsigned char*)p;
    return RT_OK;
}

}  // namespace

extern "C" int rt_coverage_map_noalloc(rt_ctx* ctx, const rt_grid* g, int32_t max_depth, int64_t num_rays,
                                       int32_t tx_port, float* gain, uint32_t* hits) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    cudaError_t de = cudaSetDevice(ctx->device);
    if (de != cudaSuccess) return set_cuda(ctx, de, "cudaSetDevice");
    if (!g || !gain || !hits || g->nx < 1 || g->ny < 1 || !(g->cell > 0.0f) || max_depth < 0 || num_rays < 1 ||
        tx_port < 0 || tx_port >= ctx->tx_ant.n_ports)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_noalloc: bad arguments");
    if (num_rays > NA_MAX_RAYS)
        return set_err(ctx, RT_ERR_INVALID_ARG,
                       "coverage_map_noalloc: num_rays above RT_NOALLOC_MAX_RAYS (1048576), the size of its "
                       "static scratch; use rt_coverage_map");
    if (!ctx->has_scene || ctx->n_tx < 1 || ctx->n_rx < 1)
        return set_err(ctx, RT_ERR_INVALID_ARG, "coverage_map_noalloc: scene, transmitters and receivers must be set");
    unsigned char* base = nullptr;
    int e = na_scratch(ctx, &base);
    if (e) return e;
    unsigned long long* counters = (unsigned long long*)base;
    unsigned* status = (unsigned*)(base + 8 * sizeof(unsigned long long));
    uint32_t* cells = (uint32_t*)(base + NA_OFF_CELLS);
    uint32_t* perm = (uint32_t*)(base + NA_OFF_PERM);
    cudaStream_t st = ctx->stream;
    // the array keeps the previous call's contents: clear what must start at zero
    RT_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    RT_TRY(cudaMemsetAsync(cells, 0, sizeof(uint32_t) * NA_CELLS, st));
    unsigned blocks = (unsigned)((num_rays + 255) / 256);
    ctx->launches += 3;
    k_na_count<<<blocks, 256, 0, st>>>(num_rays, cells);
    k_na_scan<<<1, 1024, 0, st>>>(cells);
    k_na_scatter<<<blocks, 256, 0, st>>>(num_rays, cells, perm);
    RT_TRY(cudaGetLastError());
    return launch_coverage_scratch(ctx, g, max_depth, num_rays, tx_port, gain, hits, counters, status, perm);
}
