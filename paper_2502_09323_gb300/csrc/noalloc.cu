// pb_apply_dot_noalloc: y = A x and x.(A x) in FP64 without allocating any
// device memory.
//
// Some callers cannot allocate device memory while they work: an application
// whose device memory is owned entirely by its own pool or by another
// framework, or a latency-critical loop that cannot accept cudaMalloc's
// implicit device synchronisation.  This entry point serves them: besides
// the caller's inputs and outputs it uses only the fixed scratch array below,
// which lives in the library image and is held by every GPU that loads the
// library until the process exits.
//
// Scratch: one FP64 partial sum per block plus a block counter, at most
// NOALLOC_MAX_BLOCKS blocks of NOALLOC_NODES_PER_BLOCK nodes, i.e. grids of up
// to NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK nodes; larger grids are
// rejected.  All calls share the array: calls that overlap on the GPU (on
// different streams, or from different threads) race on it and must be
// serialised by the caller.
#include <mutex>

#include "pb_internal.h"

namespace pbg {
namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr long long NOALLOC_NODES_PER_BLOCK = 2048;
constexpr int NOALLOC_MAX_BLOCKS = 16384;
constexpr size_t NOALLOC_BYTES = sizeof(double) * NOALLOC_MAX_BLOCKS + 256;

// [0, NOALLOC_MAX_BLOCKS) doubles: block partials; then one unsigned counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_addr[MAX_DEVICES] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// y = A x on interior nodes (boundary entries of x read as zero, y = 0 on
// boundary nodes) in the canonical node layout, FP64 edge weights; the last
// block sums the per-block partials of x.y in block order.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_apply_dot_static(const double *__restrict__ Wx, const double *__restrict__ Wy,
                   const double *__restrict__ Wz, const double *__restrict__ diag, GridGeo g,
                   const double *__restrict__ x, double *__restrict__ y, double *__restrict__ dot,
                   unsigned char *scratch) {
    double *partials = reinterpret_cast<double *>(scratch);
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + sizeof(double) * NOALLOC_MAX_BLOCKS);
    __shared__ double sred[NOALLOC_THREADS / 32];
    __shared__ int s_last;
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    double acc = 0.0;
    const long long a0 = (long long)blockIdx.x * NOALLOC_NODES_PER_BLOCK;
    const long long a1 = min(a0 + NOALLOC_NODES_PER_BLOCK, g.N);
    for (long long a = a0 + threadIdx.x; a < a1; a += NOALLOC_THREADS) {
        const long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / sz;
        const bool interior =
            i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
        double v = 0.0;
        if (interior) {
            double s = 0.0;
            if (i > 1) s += Wx[a - 1] * x[a - 1];
            if (i < g.nx - 2) s += Wx[a] * x[a + 1];
            if (j > 1) s += Wy[a - sy] * x[a - sy];
            if (j < g.ny - 2) s += Wy[a] * x[a + sy];
            if (k > 1) s += Wz[a - sz] * x[a - sz];
            if (k < g.nz - 2) s += Wz[a] * x[a + sz];
            v = diag[a] * x[a] - s;
            acc += x[a] * v;
        }
        y[a] = v;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) b += sred[w];
        partials[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += NOALLOC_THREADS) t += __ldcg(partials + q);
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) tot += sred[w];
        *dot = tot;
        *counter = 0u;
    }
}

// Device address of the scratch array for the current device, looked up once
// per device (the first call on a device does this set-up).
pb_status scratch_for_current_device(unsigned char **out) {
    int dev = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("device ordinal %d beyond the static scratch table", dev);
        return PB_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return PB_ERR_CUDA;
        }
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return PB_OK;
}

}  // namespace
}  // namespace pbg

extern "C" pb_status pb_apply_dot_noalloc(const pb_system *s, const double *x, double *y,
                                          double *xAx, void *stream) {
    using namespace pbg;
    set_error("");
    if (!s || !x || !y || !xAx) {
        set_error("pb_apply_dot_noalloc: NULL argument");
        return PB_ERR_ARG;
    }
    if (s->g->is_oct) {
        set_error("pb_apply_dot_noalloc: octree systems are not supported");
        return PB_ERR_UNIMPL;
    }
    const GridGeo &g = s->g->geo;
    const long long blocks = (g.N + NOALLOC_NODES_PER_BLOCK - 1) / NOALLOC_NODES_PER_BLOCK;
    if (blocks > NOALLOC_MAX_BLOCKS) {
        set_error("pb_apply_dot_noalloc: grid of %lld nodes exceeds the static scratch limit of "
                  "%lld nodes", g.N, (long long)NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK);
        return PB_ERR_ARG;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != s->g->device) {
        cudaGetLastError();
        set_error("pb_apply_dot_noalloc: the system's device must be the current device");
        return PB_ERR_ARG;
    }
    unsigned char *scratch = nullptr;
    pb_status rc = scratch_for_current_device(&scratch);
    if (rc != PB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // the block counter must start at zero (each call's last block also resets it)
    PB_CUDA_TRY(cudaMemsetAsync(scratch + sizeof(double) * NOALLOC_MAX_BLOCKS, 0, sizeof(unsigned), st));
    k_apply_dot_static<<<(unsigned)blocks, NOALLOC_THREADS, 0, st>>>(
        s->W[0], s->W[1], s->W[2], s->diag, g, x, y, xAx, scratch);
    PB_LAUNCH_CHECK();
    return PB_OK;
}
