// Building blocks of a solve decomposed into z slabs, one per GPU.
//
// A rank owns the planes [z0, z1) of the global grid and keeps them in an
// extended local grid with ghost planes below and above (an lm_grid with
// a wall in z: the ghost planes supply the neighbours' values, so the wall
// faces past them are never used for an owned cell).  Cell-centred arrays
// are plane-contiguous in z (x fastest), so the halo of a slab is a run of
// whole planes: the pack/unpack kernels copy the boundary planes of an
// array into one message buffer and back, both sides in one launch.
//
// The rest are the vector and multigrid steps the host driver sequences
// between its exchanges: float64 axpby, dot products over a range of
// planes (deterministic, float64 accumulation), the inverse Jacobi
// diagonal, and the level-0 <-> level-1 transfers of the V-cycle (residual
// + restriction, prolongation) that frame the coarse solve gathered on one
// rank.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_internal.h"
#include "lm_kernels.h"

using namespace lm;

namespace {

constexpr int DOT_BLOCKS = 1024;    // partial sums of lm_vec_dot (its scratch: DOT_BLOCKS doubles)

// buf = [planes lo_first .. lo_first + np) | [planes hi_first .. + np), in
// 16-byte words when every offset allows it, else 4-byte words (one
// side is skipped when its first plane is negative).
template <typename W>
__global__ void __launch_bounds__(NT) k_halo_copy(W* __restrict__ a, W* __restrict__ buf, long long plane_w,
                                                  long long lo_first, long long hi_first, int np, int unpack) {
    const long long side_w = plane_w * np;
    const long long total = 2 * side_w;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const bool hi = t >= side_w;
        const long long first = hi ? hi_first : lo_first;
        if (first < 0) continue;
        const long long ai = first * plane_w + (hi ? t - side_w : t);
        if (unpack) a[ai] = buf[t];
        else buf[t] = a[ai];
    }
}

template <typename TX, typename TY, typename TO>
__global__ void __launch_bounds__(NT) k_axpby(long long n, double alpha, const TX* x, double beta,
                                              const TY* y, TO* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = alpha * (double)x[i] + (y ? beta * (double)y[i] : 0.0);
        out[i] = (TO)v;
    }
}

// Block partials of sum a_i b_i in float64 (fixed order: block b sums the
// grid-stride set of b in thread order, then a fixed tree), then one block
// adds the partials in block order.
template <typename TA, typename TB>
__global__ void __launch_bounds__(NT) k_dot_part(long long n, const TA* __restrict__ a, const TB* __restrict__ b,
                                                 double* __restrict__ part) {
    __shared__ double sm[32];
    double v[1] = {0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[0] += (double)a[i] * (double)b[i];
    block_sum<1>(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void __launch_bounds__(NT) k_dot_final(const double* __restrict__ part, int G, double* __restrict__ out) {
    __shared__ double sm[32];
    const double v = reduce_partials(part, G, sm);
    if (threadIdx.x == 0) *out = v;
}

__global__ void __launch_bounds__(NT) k_mul64(long long n, const double* __restrict__ d, const double* __restrict__ r,
                                              double* __restrict__ z) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = d[i] * r[i];
}

// x += P ec: piecewise-constant prolongation from the next level (children
// of a coarse cell take its value), over every cell of the fine level.
__global__ void __launch_bounds__(NT) k_prolong_add(Geo F, Geo C, int hx, int hy, int hz, const float* __restrict__ ec,
                                                    float* __restrict__ x) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < F.N; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(idx, F, i, j, k);
        x[idx] += ec[(i >> hx) + C.nx * ((j >> hy) + C.ny * (k >> hz))];
    }
}

int blocks_for(long long n) {
    const long long b = (n + NT - 1) / NT;
    return (int)(b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b));
}

bool prec_ok(int p) { return p == LM_PREC_FP64 || p == LM_PREC_FP32; }

#define CKR(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            fprintf(stderr, "lowmach: %s failed: %s\n", #call, cudaGetErrorString(e_));             \
            return LM_ERR_CUDA;                                                                     \
        }                                                                                           \
    } while (0)

}  // namespace

extern "C" {

int lm_halo_pack(const void* a, int elem_bytes, int64_t plane_elems, int64_t lo_first, int64_t hi_first, int nplanes,
                 void* buf, int unpack, void* stream) {
    if (!a || !buf || (elem_bytes != 4 && elem_bytes != 8) || plane_elems < 1 || nplanes < 1 ||
        (lo_first < 0 && hi_first < 0))
        return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long plane_bytes = plane_elems * elem_bytes;
    const bool wide = plane_bytes % 16 == 0 && ((uintptr_t)a & 15) == 0 && ((uintptr_t)buf & 15) == 0;
    const long long plane_w = wide ? plane_bytes / 16 : plane_bytes / 4;
    count_launches(1);
    const int G = blocks_for(2 * plane_w * nplanes);
    if (wide)
        k_halo_copy<float4><<<G, NT, 0, s>>>((float4*)a, (float4*)buf, plane_w, lo_first, hi_first, nplanes, unpack);
    else
        k_halo_copy<float><<<G, NT, 0, s>>>((float*)a, (float*)buf, plane_w, lo_first, hi_first, nplanes, unpack);
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_vec_axpby(int64_t n, double alpha, const void* x, int x_prec, double beta, const void* y, int y_prec, void* out,
                 int out_prec, void* stream) {
    if (n < 0 || !x || !out || !prec_ok(x_prec) || !prec_ok(out_prec) || (y && !prec_ok(y_prec)))
        return LM_ERR_INVALID_ARG;
    if (n == 0) return LM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = blocks_for(n);
    count_launches(1);
    const bool x64 = x_prec == LM_PREC_FP64, y64 = !y || y_prec == LM_PREC_FP64, o64 = out_prec == LM_PREC_FP64;
#define LM_AXPBY(TX, TY, TO) \
    k_axpby<TX, TY, TO><<<G, NT, 0, s>>>(n, alpha, (const TX*)x, beta, (const TY*)y, (TO*)out)
    if (x64 && y64 && o64) LM_AXPBY(double, double, double);
    else if (x64 && y64) LM_AXPBY(double, double, float);
    else if (x64 && o64) LM_AXPBY(double, float, double);
    else if (x64) LM_AXPBY(double, float, float);
    else if (y64 && o64) LM_AXPBY(float, double, double);
    else if (y64) LM_AXPBY(float, double, float);
    else if (o64) LM_AXPBY(float, float, double);
    else LM_AXPBY(float, float, float);
#undef LM_AXPBY
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_vec_dot(int64_t n, const void* a, int a_prec, const void* b, int b_prec, double* scratch, double* out,
               void* stream) {
    if (n < 0 || !a || !b || !scratch || !out || !prec_ok(a_prec) || !prec_ok(b_prec)) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = (int)std::min<long long>(DOT_BLOCKS, std::max<long long>(1, (n + NT - 1) / NT));
    count_launches(2);
    const bool a64 = a_prec == LM_PREC_FP64, b64 = b_prec == LM_PREC_FP64;
    if (a64 && b64) k_dot_part<double, double><<<G, NT, 0, s>>>(n, (const double*)a, (const double*)b, scratch);
    else if (a64) k_dot_part<double, float><<<G, NT, 0, s>>>(n, (const double*)a, (const float*)b, scratch);
    else if (b64) k_dot_part<float, double><<<G, NT, 0, s>>>(n, (const float*)a, (const double*)b, scratch);
    else k_dot_part<float, float><<<G, NT, 0, s>>>(n, (const float*)a, (const float*)b, scratch);
    k_dot_final<<<1, NT, 0, s>>>(scratch, G, scratch + DOT_BLOCKS);
    CKR(cudaGetLastError());
    CKR(cudaMemcpyAsync(out, scratch + DOT_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaStreamSynchronize(s));
    return LM_OK;
}

int lm_vec_mul(int64_t n, const double* d, const double* r, double* z, void* stream) {
    if (n < 0 || !d || !r || !z) return LM_ERR_INVALID_ARG;
    if (n == 0) return LM_OK;
    count_launches(1);
    k_mul64<<<blocks_for(n), NT, 0, (cudaStream_t)stream>>>(n, d, r, z);
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_jacobi_inverse_diagonal(lm_grid* g, double* dinv, void* stream) {
    if (!g || !dinv) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    launch_jacobi_diag(g->geo, g->G, (cudaStream_t)stream, Op64{g->ct, g->gx, g->gy, g->gz, nullptr}, dinv);
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_mg_restrict_residual(lm_grid* g, const float* x, const float* f, float* fc, void* stream) {
    if (!g || !x || !f || !fc) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!g->fp32_ok) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = grid_build_mg(g, s);
    if (rc) return rc;
    if (g->mg.size() < 2) return LM_ERR_INVALID_ARG;
    const MgLevel& F = g->mg[0];
    const MgLevel& C = g->mg[1];
    launch_resid_restrict(F.L, C.L, F.halved[0], F.halved[1], F.halved[2], s, x, f, fc);
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_mg_prolong_add(lm_grid* g, const float* ec, float* x, void* stream) {
    if (!g || !ec || !x) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!g->fp32_ok) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = grid_build_mg(g, s);
    if (rc) return rc;
    if (g->mg.size() < 2) return LM_ERR_INVALID_ARG;
    const MgLevel& F = g->mg[0];
    const MgLevel& C = g->mg[1];
    count_launches(1);
    k_prolong_add<<<blocks_for(F.L.g.N), NT, 0, s>>>(F.L.g, C.L.g, F.halved[0], F.halved[1], F.halved[2], ec, x);
    CKR(cudaGetLastError());
    return LM_OK;
}

int lm_mg_level_coefficients(lm_grid* g, int level, float* ct, float* rho, double* rho_scale, void* stream) {
    if (!g || level < 0) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!g->fp32_ok) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = grid_build_mg(g, s);
    if (rc) return rc;
    if (level >= (int)g->mg.size()) return LM_ERR_INVALID_ARG;
    const Lev32& L = g->mg[level].L;
    const size_t B = sizeof(float) * (size_t)L.g.N;
    if (ct) CKR(cudaMemcpyAsync(ct, L.ct, B, cudaMemcpyDeviceToDevice, s));
    if (rho) CKR(cudaMemcpyAsync(rho, L.rho, B, cudaMemcpyDeviceToDevice, s));
    if (rho_scale) *rho_scale = g->rho_scale;
    return LM_OK;
}

}  // extern "C"
