// Shared device-side definitions of the generalized-Poisson solver library.
//
// Grid layout: cell (i, j, k) of an nx x ny x nz grid lives at flat index
// i + nx*(j + ny*k) (x fastest).  2D grids have ny = 1.  Flat indices are
// 32-bit: grids hold fewer than 2^31 cells.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lowmach.h"

namespace lm {

constexpr int NT = 256;             // threads per block of the streaming kernels
constexpr int MAX_PARTIALS = 65536; // upper bound on blocks of a reducing kernel
constexpr int NSLOT = 8;            // partial-sum slots per reduction buffer

struct Geo {
    int nx, ny, nz;
    int N;
    int bcx, bcy, bcz;          // LM_BC_PERIODIC / LM_BC_NEUMANN
    double ih2x, ih2y, ih2z;    // 1/h^2 per axis
};

// Per-solve state shared by the Krylov kernels (device memory).
struct SolveState {
    int done;        // 1: every later kernel of the solve returns at once
    int status;      // LM_OK or LM_ERR_*
    int iters;       // iterations completed
    int converged;   // recursive residual met the tolerance
    double fnorm;    // ||f||_2
    double rtol;
    double rel;      // last relative residual
    double scale;    // free slot (IR: norm of the current residual)
};

// Neighbour indices along one axis, with periodic wrap.  On a Neumann axis
// the wrapped index is only ever paired with a zero face coefficient.
struct Nbr {
    int im, ip;
};

__device__ __forceinline__ void cell_coords(int idx, const Geo& g, int& i, int& j, int& k) {
    i = idx % g.nx;
    int t = idx / g.nx;
    j = t % g.ny;
    k = t / g.ny;
}

__device__ __forceinline__ Nbr nbr_x(int idx, int i, const Geo& g) {
    return {i > 0 ? idx - 1 : idx + g.nx - 1, i < g.nx - 1 ? idx + 1 : idx - (g.nx - 1)};
}
__device__ __forceinline__ Nbr nbr_y(int idx, int j, const Geo& g) {
    int s = g.nx;
    return {j > 0 ? idx - s : idx + (g.ny - 1) * s, j < g.ny - 1 ? idx + s : idx - (g.ny - 1) * s};
}
__device__ __forceinline__ Nbr nbr_z(int idx, int k, const Geo& g) {
    int s = g.nx * g.ny;
    return {k > 0 ? idx - s : idx + (g.nz - 1) * s, k < g.nz - 1 ? idx + s : idx - (g.nz - 1) * s};
}

// Does the face of a cell at position c (of n) on its minus/plus side carry
// flux?  Wall faces of a Neumann axis and the self-face of a 1-cell axis do not.
__device__ __forceinline__ bool face_minus(int c, int n, int bc) {
    return n > 1 && (c > 0 || bc == LM_BC_PERIODIC);
}
__device__ __forceinline__ bool face_plus(int c, int n, int bc) {
    return n > 1 && (c < n - 1 || bc == LM_BC_PERIODIC);
}

// ---- L2 prefetch ---------------------------------------------------------------

// Planes ahead of their first use that the whole-row z-march kernels ask the
// copy engine to bring into L2 (see prefetch_l2).
#ifndef LM_PF_PLANES
#define LM_PF_PLANES 1
#endif
constexpr int PF_PLANES = LM_PF_PLANES;

// One bulk asynchronous prefetch of `bytes` (a multiple of 16) of global
// memory into L2 (PTX cp.async.bulk.prefetch.L2, sm_90 and later): it holds
// no register or shared memory, so a z-march can run it several planes ahead
// of its staged loads, which then hit L2 instead of waiting on HBM.  Skipped
// when the address is not 16-byte aligned, which the instruction requires.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    if (((uintptr_t)p & 15) == 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The power of two nearest 1/v for v > 0 finite (1 otherwise), clamped to
// 2^-100 .. 2^100: an exact scaling factor.
__host__ __device__ __forceinline__ double pow2_near_inv(double v) {
    if (!(v > 0.0) || !(v < 1e300)) return 1.0;
    int e = -(int)rint(log2(v));
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    return ldexp(1.0, e);
}

// ---- reductions ------------------------------------------------------------

__device__ __forceinline__ int lin_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int lin_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }
__device__ __forceinline__ unsigned lin_block() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Sum of v over the block (any shape, whole warps); result valid in linear
// thread 0 only.  Fixed order.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* K*32 */) {
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int t = lin_tid();
    const int w = t >> 5, l = t & 31, nw = lin_nthreads() >> 5;
    if (l == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[q * 32 + w] = v[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double s = l < nw ? smem[q * 32 + l] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            v[q] = s;
        }
    }
    __syncthreads();
}

// Write the block's K partial sums to part[q*MAX_PARTIALS + block].
template <int K>
__device__ __forceinline__ void write_partials(double (&v)[K], double* part, double* smem) {
    block_sum<K>(v, smem);
    if (lin_tid() == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) part[q * MAX_PARTIALS + lin_block()] = v[q];
}

// Deterministic sum of G block partials, computed identically by every block
// that calls it (same data, same order); the value is returned to all threads.
__device__ __forceinline__ double reduce_partials(const double* part, int G, double* smem) {
    double v[1] = {0.0};
    for (int t = lin_tid(); t < G; t += lin_nthreads()) v[0] += __ldcg(part + t);
    block_sum<1>(v, smem);
    __shared__ double bcast;
    if (lin_tid() == 0) bcast = v[0];
    __syncthreads();
    double r = bcast;
    __syncthreads();
    return r;
}

// Grid-wide reduction by the last block to finish (no waiting): every block
// stores its partial sums, counts itself in, and the block that arrives last
// sums all partials in block order -- the same order every run -- into
// scal[slot[q]] and re-arms the counter.  Returns true in that block.
struct Red {
    double* part;        // K * MAX_PARTIALS
    double* scal;        // result slots
    unsigned int* ctr;   // arrival counter, 0 between launches
};

template <int K>
__device__ __forceinline__ bool grid_reduce_n(double (&v)[K], const Red& red, const int (&slot)[K], double* smem,
                                              unsigned blk, unsigned nb) {
    block_sum<K>(v, smem);
    __shared__ unsigned int s_last;
    if (lin_tid() == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) red.part[q * MAX_PARTIALS + blk] = v[q];
        __threadfence();
        s_last = (atomicAdd(red.ctr, 1u) == nb - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const double tot = reduce_partials(red.part + q * MAX_PARTIALS, (int)nb, smem);
        if (lin_tid() == 0) red.scal[slot[q]] = tot;
    }
    if (lin_tid() == 0) *red.ctr = 0u;
    return true;
}

template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], const Red& red, const int (&slot)[K], double* smem) {
    return grid_reduce_n<K>(v, red, slot, smem, lin_block(), gridDim.x * gridDim.y * gridDim.z);
}

// Float-float accumulator: products formed exactly (TwoProduct by FMA) and
// summed with Knuth's TwoSum, so a float32 kernel reduces to about 44-bit
// accuracy; it is converted to float64 before the block/grid reduction.
// (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2.)  The _rn intrinsics keep the
// compiler from contracting or reassociating these steps.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add_prod(FF& s, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s.hi, p);
    const float bp = __fsub_rn(t, s.hi);
    const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ double ff_value(const FF& s) { return (double)s.hi + (double)s.lo; }

}  // namespace lm
