// The dissipative fourth-order second derivative of the viscous terms
// (Sec. 4, Eqs. fv-approach2 and dissipativestencil4), summed over the grid
// axes (directional splitting): out = beta u + alpha sum_a (U_aa).
//
// The paper builds (U_xx)_i as the difference of two face derivatives
// p_{i+1/2} = (U_{i-1} - 15 U_i + 15 U_{i+1} - U_{i+2}) / (12 h), which
// telescopes to the centred five-point stencil (-1, 16, -30, 16, -1) / (12 h^2).
// A periodic axis wraps; a wall axis takes mirror ghosts U_{-1-k} = U_k, with
// which the face derivative at the wall vanishes by symmetry, so the
// five-point stencil on the mirrored values is the flux form with no flux
// through the wall (the scheme stays conservative).
//
// One thread per (x, y) column marches up z with the five z-values of its
// column in registers (one new load a plane); the x- and y-neighbours come
// through L1/L2.  Float32: HBM-bound (8 bytes a cell); float64: GB300's
// float64 pipe bounds it (about 17 float64 operations a 3D cell).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace {

// index of cell c + k on an axis of n cells: wrapped, or mirrored about the walls
__device__ __forceinline__ int ax_index(int c, int k, int n, bool per) {
    int j = c + k;
    if (per) {
        j = j < 0 ? j + n : (j >= n ? j - n : j);
    } else {
        j = j < 0 ? -1 - j : (j >= n ? 2 * n - 1 - j : j);
    }
    return j;
}

template <typename T>
__device__ __forceinline__ T five_point(T um2, T um1, T u0, T up1, T up2) {
    return ((T)16 * (um1 + up1) - (um2 + up2)) - (T)30 * u0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_diffusion4(lm::Geo g, T wx, T wy, T wz, T alpha, T beta,
                                                    const T* __restrict__ u, T* __restrict__ out, int KZ) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * KZ, k1 = min(k0 + KZ, g.nz);
    if (i >= g.nx || j >= g.ny) return;
    const bool px = g.bcx == LM_BC_PERIODIC, py = g.bcy == LM_BC_PERIODIC, pz = g.bcz == LM_BC_PERIODIC;
    const int sz = g.nx * g.ny;
    int xi[4], yj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = q < 2 ? q - 2 : q - 1;       // -2, -1, +1, +2
        xi[q] = ax_index(i, k, g.nx, px);
        yj[q] = ax_index(j, k, g.ny, py);
    }
    const int col = i + g.nx * j;
    // the column's z-values of planes k - 2 .. k + 2 (k = k0)
    T z[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) z[q] = g.nz > 1 ? u[col + sz * ax_index(k0, q - 2, g.nz, pz)] : (T)0;
    for (int k = k0; k < k1; ++k) {
        if (g.nz == 1) z[2] = u[col];
        const T* pl = u + sz * k;
        const T c = z[2];
        T acc = (T)0;
        if (g.nx > 1) {
            const int r = g.nx * j;
            acc += wx * five_point(pl[r + xi[0]], pl[r + xi[1]], c, pl[r + xi[2]], pl[r + xi[3]]);
        }
        if (g.ny > 1)
            acc += wy * five_point(pl[i + g.nx * yj[0]], pl[i + g.nx * yj[1]], c, pl[i + g.nx * yj[2]],
                                   pl[i + g.nx * yj[3]]);
        if (g.nz > 1) acc += wz * five_point(z[0], z[1], c, z[3], z[4]);
        out[col + sz * k] = beta * c + alpha * acc;
        if (g.nz > 1 && k + 1 < k1) {                // shift the column window up one plane
#pragma unroll
            for (int q = 0; q < 4; ++q) z[q] = z[q + 1];
            z[4] = u[col + sz * ax_index(k + 1, 2, g.nz, pz)];
        }
    }
}

}  // namespace

extern "C" int lm_diffusion4(int ndim, const int64_t n[3], const double h[3], const int bc[3], int prec,
                             double alpha, const void* u, double beta, void* out, void* stream) {
    if (!n || !h || !bc || !u || !out || u == out || (ndim != 2 && ndim != 3) ||
        (prec != LM_PREC_FP64 && prec != LM_PREC_FP32))
        return LM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || !(h[a] > 0.0) || (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN)) return LM_ERR_INVALID_ARG;
    }
    if (ndim == 2 && n[1] != 1) return LM_ERR_INVALID_ARG;
    if ((long long)n[0] * n[1] * n[2] >= (1LL << 31)) return LM_ERR_INVALID_ARG;
    lm::Geo g{};
    g.nx = (int)n[0];
    g.ny = (int)n[1];
    g.nz = (int)n[2];
    g.N = g.nx * g.ny * g.nz;
    g.bcx = bc[0];
    g.bcy = bc[1];
    g.bcz = bc[2];
    // z chunks of KZ planes: enough blocks for eight per SM
    const long long cols = (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8);
    int chunks = (int)std::max(1LL, std::min<long long>(g.nz, (8LL * 152 + cols - 1) / cols));
    const int KZ = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + KZ - 1) / KZ;
    const dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8, chunks);
    cudaStream_t s = (cudaStream_t)stream;
    lm::count_launches(1);
    const double w[3] = {1.0 / (12.0 * h[0] * h[0]), 1.0 / (12.0 * h[1] * h[1]), 1.0 / (12.0 * h[2] * h[2])};
    if (prec == LM_PREC_FP64)
        k_diffusion4<double><<<grd, blk, 0, s>>>(g, w[0], w[1], w[2], alpha, beta, (const double*)u, (double*)out, KZ);
    else
        k_diffusion4<float><<<grd, blk, 0, s>>>(g, (float)w[0], (float)w[1], (float)w[2], (float)alpha, (float)beta,
                                                (const float*)u, (float*)out, KZ);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lowmach: lm_diffusion4: %s\n", cudaGetErrorString(e));
        return LM_ERR_CUDA;
    }
    return LM_OK;
}
