// Allocation-free float64 stencil apply with its fused x^T A x reduction.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- for instance a host code that hands this library a fixed memory
// budget at start-up, or one running under an allocator that forbids
// cudaMalloc/cudaFree on its hot path (a frozen memory pool, or a process
// that has to keep its device footprint fixed after initialisation).  The
// grid-based entry points allocate at lm_grid_create; this one allocates
// nothing: the caller passes the coefficients (as lm_get_coefficients
// returns them), x and y, and the device scalar that receives x^T A x.
//
// The per-block partial sums of the reduction live in the file-scope static
// device array below, LM_NOALLOC_MAX_BLOCKS doubles (512 KiB).  Every GPU
// that loads this library holds that array until the process exits.  Each
// block covers LM_NOALLOC_CELLS_PER_BLOCK cells, so a call handles at most
// LM_NOALLOC_MAX_BLOCKS * LM_NOALLOC_CELLS_PER_BLOCK cells; larger grids are
// rejected before any device work.  Every call shares the array: a call
// writes the partials of all its blocks before reading them, so nothing has
// to start at zero, but two calls whose kernels overlap on the GPU (on
// different streams, or from different threads) race on it.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in).  The device address is looked up once per
// device, with that device current, by cudaGetSymbolAddress; the first call
// on a device does this set-up, so make that first call before any stream
// capture.
#include <cstdio>
#include <mutex>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"
#include "lm_tiles.cuh"

constexpr int LM_NOALLOC_ITEMS = 16;                                        // cells per thread
constexpr int LM_NOALLOC_CELLS_PER_BLOCK = lm::NT * LM_NOALLOC_ITEMS;       // 4096
constexpr int LM_NOALLOC_MAX_BLOCKS = 65536;                                // 512 KiB of partials
constexpr long long LM_NOALLOC_MAX_CELLS = (long long)LM_NOALLOC_MAX_BLOCKS * LM_NOALLOC_CELLS_PER_BLOCK;
constexpr int LM_NOALLOC_MAX_DEVICES = 64;

// The scratch: one partial sum per block, shared by every call on a device.
static __device__ __align__(256) double lm_noalloc_partials[LM_NOALLOC_MAX_BLOCKS];

namespace {

std::mutex g_setup_mutex;
double* g_partials_addr[LM_NOALLOC_MAX_DEVICES] = {};

// Device address of the static partials on the current device (set-up once per device).
int partials_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LM_ERR_CUDA;
    if (dev < 0 || dev >= LM_NOALLOC_MAX_DEVICES) return LM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, lm_noalloc_partials);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "lowmach: lm_apply_dot_noalloc: cudaGetSymbolAddress failed: %s\n",
                    cudaGetErrorString(e));
            return LM_ERR_CUDA;
        }
        g_partials_addr[dev] = (double*)p;
    }
    *out = g_partials_addr[dev];
    return LM_OK;
}

// Block b applies A to its LM_NOALLOC_CELLS_PER_BLOCK cells and writes its
// partial sum of x_i (A x)_i to partials[b].
__global__ void __launch_bounds__(lm::NT) k_apply_dot_noalloc(lm::Geo g, const double* __restrict__ ct,
                                                              const double* __restrict__ gx,
                                                              const double* __restrict__ gy,
                                                              const double* __restrict__ gz,
                                                              const double* __restrict__ x, double* __restrict__ y,
                                                              double* __restrict__ partials) {
    __shared__ double sm[32];
    double acc[1] = {0.0};
    const int base = blockIdx.x * LM_NOALLOC_CELLS_PER_BLOCK;
    for (int s = 0; s < LM_NOALLOC_ITEMS; ++s) {
        const int idx = base + s * lm::NT + threadIdx.x;
        if (idx < g.N) {
            // the grid-based apply's stencil on the caller's coefficients
            const double v = lm::apply64_at(idx, g, lm::Op64{ct, gx, gy, gz, nullptr}, x);
            y[idx] = v;
            acc[0] += x[idx] * v;
        }
    }
    lm::block_sum<1>(acc, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// One block: *dot_out = sum of the G partials, in a fixed order.
__global__ void __launch_bounds__(lm::NT) k_sum_partials_noalloc(const double* __restrict__ partials, int G,
                                                                 double* __restrict__ dot_out) {
    __shared__ double sm[32];
    const double v = lm::reduce_partials(partials, G, sm);
    if (threadIdx.x == 0) *dot_out = v;
}

}  // namespace

extern "C" int lm_apply_dot_noalloc(int ndim, const int64_t n[3], const int bc[3], const double* ctilde,
                                    const double* gx, const double* gy, const double* gz, const double* x,
                                    double* y, double* dot_out, void* stream) {
    if (!n || !bc || !ctilde || !gx || !gy || !gz || !x || !y || !dot_out) return LM_ERR_INVALID_ARG;
    if (ndim != 2 && ndim != 3) return LM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return LM_ERR_INVALID_ARG;
        if (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN) return LM_ERR_INVALID_ARG;
    }
    if (ndim == 2 && n[1] != 1) return LM_ERR_INVALID_ARG;
    const long long N = (long long)n[0] * n[1] * n[2];
    if (N > LM_NOALLOC_MAX_CELLS) {
        fprintf(stderr,
                "lowmach: lm_apply_dot_noalloc: %lld cells exceed the static scratch limit of %lld cells "
                "(%d blocks of %d cells)\n",
                N, LM_NOALLOC_MAX_CELLS, LM_NOALLOC_MAX_BLOCKS, LM_NOALLOC_CELLS_PER_BLOCK);
        return LM_ERR_INVALID_ARG;
    }
    double* partials = nullptr;
    int rc = partials_address(&partials);
    if (rc != LM_OK) return rc;
    lm::Geo g{};
    g.nx = (int)n[0];
    g.ny = (int)n[1];
    g.nz = (int)n[2];
    g.N = (int)N;
    g.bcx = bc[0];
    g.bcy = bc[1];
    g.bcz = bc[2];
    const int G = (int)((N + LM_NOALLOC_CELLS_PER_BLOCK - 1) / LM_NOALLOC_CELLS_PER_BLOCK);
    cudaStream_t s = (cudaStream_t)stream;
    lm::count_launches(2);
    k_apply_dot_noalloc<<<G, lm::NT, 0, s>>>(g, ctilde, gx, gy, gz, x, y, partials);
    k_sum_partials_noalloc<<<1, lm::NT, 0, s>>>(partials, G, dot_out);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}
