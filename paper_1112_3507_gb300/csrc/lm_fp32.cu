// Float32 kernels: the operator with faces formed on the fly from rho, the
// flexible-CG vector steps with float64-accurate dot products, and the
// geometric-multigrid V-cycle (coefficient coarsening, a fused red-black
// Gauss-Seidel sweep, fused residual + restriction, exact coarsest solve).
// The bodies live in lm_tiles.cuh; these are the single-grid launches.
//
// These kernels are HBM-bound.  They stream each array once: face
// conductances are recomputed from rho instead of stored; cells are mapped
// to threads with 2D/3D launches (no integer division per cell); the
// stencils march along z keeping the z-neighbours in registers; and a whole
// red-black sweep is one pass over memory (see rbgs_tile).
#include "lm_common.cuh"
#include "lm_kernels.h"
#include "lm_tiles.cuh"

namespace lm {

template <bool HAS_Y, bool DOT_XY, bool DOT_XR>
__global__ void __launch_bounds__(256) k_apply32z(Lev32 L, const float* __restrict__ x, float* __restrict__ y,
                                                  const float* __restrict__ r, Red red, int slot_xy, int slot_xr,
                                                  int kz) {
    __shared__ double sm[64];
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
    apply32z_tile<HAS_Y, DOT_XY, DOT_XR>(L, x, y, r, kz, blockIdx.x, blockIdx.y, blockIdx.z, axy, axr);
    if (DOT_XY && DOT_XR) {
        double v[2] = {ff_value(axy), ff_value(axr)};
        const int sl[2] = {slot_xy, slot_xr};
        grid_reduce<2>(v, red, sl, sm);
    } else if (DOT_XY) {
        double v[1] = {ff_value(axy)};
        const int sl[1] = {slot_xy};
        grid_reduce<1>(v, red, sl, sm);
    }
}

// scal[slot] = a.b; if fnorm_st: also fnorm_st->fnorm = sqrt(a.b), rel = 1.
__global__ void __launch_bounds__(NT) k_dot32(int N, const float* __restrict__ a, const float* __restrict__ b,
                                              Red red, int slot, SolveState* fnorm_st) {
    __shared__ double sm[32];
    const FF acc = dot32_range(N, a, b, blockIdx.x, gridDim.x);
    double v[1] = {ff_value(acc)};
    const int sl[1] = {slot};
    if (grid_reduce<1>(v, red, sl, sm) && fnorm_st && lin_tid() == 0) {
        fnorm_st->fnorm = sqrt(red.scal[slot]);
        fnorm_st->rel = 1.0;
    }
}

__global__ void __launch_bounds__(NT) k_fcg_beta_p(int N, const float* __restrict__ z, float* __restrict__ p,
                                                   const double* __restrict__ scal, int first) {
    fcg_beta_p_range(N, z, p, scal, first, blockIdx.x, gridDim.x);
}

// e, r update; scal[1] = r.r; the last block sets st->rel = ||r|| / st->fnorm
__global__ void __launch_bounds__(NT) k_fcg_update(int N, float* __restrict__ e, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   Red red, SolveState* st) {
    __shared__ double sm[32];
    bool bad;
    const FF rr = fcg_update_range(N, e, r, p, q, red.scal, bad, blockIdx.x, gridDim.x);
    double v[1] = {ff_value(rr)};
    const int sl[1] = {1};
    if (grid_reduce<1>(v, red, sl, sm) && lin_tid() == 0) {
        if (bad) st->status = LM_ERR_BREAKDOWN;
        st->rel = sqrt(red.scal[1]) / st->fnorm;
    }
}

// out = y + alpha x (out may alias y)
__global__ void __launch_bounds__(NT) k_axpy32(int N, float alpha, const float* __restrict__ x, const float* y,
                                               float* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        out[i] = __fmaf_rn(alpha, x[i], y[i]);
}

// out = y + alpha x with alpha = scal[num] / scal[den] when both are positive
// and finite, else alpha = 0 (the energy-optimal step along x, dropped when
// x is not a descent direction)
__global__ void __launch_bounds__(NT) k_axpy_ratio32(int N, const double* __restrict__ scal, int num, int den,
                                                     const float* __restrict__ x, const float* y, float* out) {
    const double a = scal[num], b = scal[den];
    const float alpha = (a > 0.0 && b > 0.0 && isfinite(a) && isfinite(b)) ? (float)(a / b) : 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        out[i] = __fmaf_rn(alpha, x[i], y[i]);
}

// Mean of the children's c~ and rho (coarse coefficients); one thread per coarse cell.
__global__ void __launch_bounds__(256) k_coarsen(Lev32 F, Geo C, int hx, int hy, int hz, float* __restrict__ ct_c,
                                                 float* __restrict__ rho_c) {
    int I, J, K;
    if (!map_cell(C, blockIdx.x, blockIdx.y, blockIdx.z, I, J, K)) return;
    float sc = 0.f, sr = 0.f;
    for (int c = 0; c <= hz; ++c)
        for (int b = 0; b <= hy; ++b)
            for (int a = 0; a <= hx; ++a) {
                const int idx = ((I << hx) + a) + F.g.nx * (((J << hy) + b) + F.g.ny * ((K << hz) + c));
                sc += F.ct[idx];
                sr += F.rho[idx];
            }
    const float inv = 1.f / (float)((1 << hx) << hy << hz);
    const int t = I + C.nx * (J + C.ny * K);
    ct_c[t] = sc * inv;
    rho_c[t] = sr * inv;
}

__global__ void __launch_bounds__(256) k_resid_restrict(Lev32 F, Geo C, int hx, int hy, int hz,
                                                        const float* __restrict__ x, const float* __restrict__ f,
                                                        float* __restrict__ fc) {
    resid_restrict_tile(F, C, hx, hy, hz, x, f, fc, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int BX, int TY, bool HAS_Y, int FIRST, bool ZERO, bool PROLONG>
__global__ void __launch_bounds__(BX * TY, 1024 / (BX * TY)) k_rbgs(Lev32 L, const float* __restrict__ xin,
                                                                   const float* __restrict__ ec, Geo C, int hx,
                                                                   int hy, int hz, const float* __restrict__ f,
                                                                   float* __restrict__ xout, int KZ) {
    rbgs_tile<BX, TY, HAS_Y, FIRST, ZERO, PROLONG>(L, xin, ec, C, hx, hy, hz, f, xout, KZ, blockIdx.x, blockIdx.y,
                                                   blockIdx.z);
}

// Inverse of the coarsest level's matrix (n <= 64) by in-place Gauss-Jordan
// elimination in float64 (SPD: no pivoting needed); one block.
__global__ void __launch_bounds__(NT) k_coarse_inverse(Lev32 L, float* __restrict__ ainv) {
    __shared__ double A[64 * 64];
    __shared__ double colk[64], rowk[64];
    const Geo& g = L.g;
    const int n = g.N;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = 0.0;
    __syncthreads();
    if (threadIdx.x < n) {
        const int idx = threadIdx.x;
        const int i = idx % g.nx, j = (idx / g.nx) % g.ny, k = idx / (g.nx * g.ny);
        const double rc = L.rho[idx];
        double d = L.ct[idx];
        auto add = [&](bool has, int nb, float c2) {
            if (!has) return;
            const double w = (double)c2 / (rc + (double)L.rho[nb]);
            d += w;
            A[idx * n + nb] -= w;
        };
        Nbr nb = nbr_x(idx, i, g);
        add(face_minus(i, g.nx, g.bcx), nb.im, L.c2x);
        add(face_plus(i, g.nx, g.bcx), nb.ip, L.c2x);
        nb = nbr_y(idx, j, g);
        add(face_minus(j, g.ny, g.bcy), nb.im, L.c2y);
        add(face_plus(j, g.ny, g.bcy), nb.ip, L.c2y);
        nb = nbr_z(idx, k, g);
        add(face_minus(k, g.nz, g.bcz), nb.im, L.c2z);
        add(face_plus(k, g.nz, g.bcz), nb.ip, L.c2z);
        A[idx * n + idx] += d;
    }
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        if (threadIdx.x < n) {
            colk[threadIdx.x] = A[threadIdx.x * n + kk];
            rowk[threadIdx.x] = A[kk * n + threadIdx.x];
        }
        __syncthreads();
        const double ipiv = 1.0 / rowk[kk];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double v;
            if (i == kk && j == kk) v = ipiv;
            else if (i == kk) v = rowk[j] * ipiv;
            else if (j == kk) v = -colk[i] * ipiv;
            else v = A[e] - colk[i] * (rowk[j] * ipiv);
            A[e] = v;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) ainv[e] = (float)A[e];
}

__global__ void k_coarse_solve(int n, const float* __restrict__ ainv, const float* __restrict__ f,
                               float* __restrict__ x) {
    coarse_solve_block(n, ainv, f, x);
}

// ---- host launchers -----------------------------------------------------------

static inline int hdiv(int a, int b) { return (a + b - 1) / b; }

static dim3 cell_grid(const Geo& g) {
    return g.ny > 1 ? dim3(hdiv(g.nx, 32), hdiv(g.ny, 8), g.nz) : dim3(hdiv(g.nx, 32), hdiv(g.nz, 8), 1);
}

void launch_apply32(const Lev32& L, cudaStream_t s, const float* x, float* y, const float* r, const Red& red,
                    int slot_xy, int slot_xr) {
    const Geo& g = L.g;
    const dim3 blk(32, 8);
    const bool y3 = g.ny > 1;
    int kz = 1;
    auto grid_for = [&](int k) {
        return y3 ? dim3(hdiv(g.nx, 32), hdiv(g.ny, 8), hdiv(g.nz, k))
                  : dim3(hdiv(g.nx, 32), hdiv(hdiv(g.nz, k), 8), 1);
    };
    while ((long long)grid_for(kz).x * grid_for(kz).y * grid_for(kz).z > 4096) kz *= 2;
    const dim3 grd = grid_for(kz);
    count_launches(1);
    const bool dxy = slot_xy >= 0, dxr = slot_xr >= 0;
#define LM_APPLY(Y, A, B) k_apply32z<Y, A, B><<<grd, blk, 0, s>>>(L, x, y, r, red, slot_xy, slot_xr, kz)
    if (y3) {
        if (dxy && dxr) LM_APPLY(true, true, true);
        else if (dxy) LM_APPLY(true, true, false);
        else LM_APPLY(true, false, false);
    } else {
        if (dxy && dxr) LM_APPLY(false, true, true);
        else if (dxy) LM_APPLY(false, true, false);
        else LM_APPLY(false, false, false);
    }
#undef LM_APPLY
}
void launch_dot32(int N, int G, cudaStream_t s, const float* a, const float* b, const Red& red, int slot,
                  SolveState* fnorm_st) {
    count_launches(1);
    k_dot32<<<G, NT, 0, s>>>(N, a, b, red, slot, fnorm_st);
}
void launch_axpy32(int N, int G, cudaStream_t s, float alpha, const float* x, const float* y, float* out) {
    count_launches(1);
    k_axpy32<<<G, NT, 0, s>>>(N, alpha, x, y, out);
}
void launch_axpy_ratio32(int N, int G, cudaStream_t s, const double* scal, int num, int den, const float* x,
                         const float* y, float* out) {
    count_launches(1);
    k_axpy_ratio32<<<G, NT, 0, s>>>(N, scal, num, den, x, y, out);
}
void launch_fcg_beta_p(int N, int G, cudaStream_t s, const float* z, float* p, const double* scal, int first) {
    count_launches(1);
    k_fcg_beta_p<<<G, NT, 0, s>>>(N, z, p, scal, first);
}
void launch_fcg_update(int N, int G, cudaStream_t s, float* e, float* r, const float* p, const float* q,
                       const Red& red, SolveState* st) {
    count_launches(1);
    k_fcg_update<<<G, NT, 0, s>>>(N, e, r, p, q, red, st);
}
void launch_coarsen(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s, float* ct_c,
                    float* rho_c) {
    count_launches(1);
    k_coarsen<<<cell_grid(C.g), dim3(32, 8), 0, s>>>(F, C.g, hx, hy, hz, ct_c, rho_c);
}
void launch_resid_restrict(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s,
                           const float* x, const float* f, float* fc) {
    count_launches(1);
    k_resid_restrict<<<cell_grid(C.g), dim3(32, 8), 0, s>>>(F, C.g, hx, hy, hz, x, f, fc);
}

// One red-black sweep xout = S(xin [+ P ec]); first = colour updated first;
// kz = planes per block (<= 0: enough blocks to fill the GPU).
void launch_rbgs_kz(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx,
                    int hy, int hz, const float* f, float* xout, int first, int zero, int prolong, int kz) {
    const Geo& g = L.g;
    const Geo Cg = C ? C->g : g;
    count_launches(1);
    if (g.ny > 1) {
        constexpr int BX = 32, TY = 8;
        const int tiles = hdiv(g.nx, 2 * BX) * hdiv(g.ny, TY);
        int KZ = kz;
        if (KZ <= 0) {
            KZ = 16;
            while (KZ > 4 && (long long)tiles * hdiv(g.nz, KZ) < 1216) KZ /= 2;
        }
        const dim3 grd(hdiv(g.nx, 2 * BX), hdiv(g.ny, TY), hdiv(g.nz, KZ)), blk(BX, TY);
#define LM_RB(F, Z, P) k_rbgs<BX, TY, true, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
        if (zero) { if (first) LM_RB(1, true, false); else LM_RB(0, true, false); }
        else if (prolong) { if (first) LM_RB(1, false, true); else LM_RB(0, false, true); }
        else { if (first) LM_RB(1, false, false); else LM_RB(0, false, false); }
#undef LM_RB
    } else {
        constexpr int BX = 128, TY = 1;
        const int tiles = hdiv(g.nx, 2 * BX);
        int KZ = kz;
        if (KZ <= 0) {
            KZ = 32;
            while (KZ > 4 && (long long)tiles * hdiv(g.nz, KZ) < 1216) KZ /= 2;
        }
        const dim3 grd(hdiv(g.nx, 2 * BX), hdiv(g.nz, KZ), 1), blk(BX, TY);
#define LM_RB(F, Z, P) k_rbgs<BX, TY, false, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
        if (zero) { if (first) LM_RB(1, true, false); else LM_RB(0, true, false); }
        else if (prolong) { if (first) LM_RB(1, false, true); else LM_RB(0, false, true); }
        else { if (first) LM_RB(1, false, false); else LM_RB(0, false, false); }
#undef LM_RB
    }
}
void launch_rbgs(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx, int hy,
                 int hz, const float* f, float* xout, int first, int zero, int prolong) {
    launch_rbgs_kz(L, s, xin, ec, C, hx, hy, hz, f, xout, first, zero, prolong, 0);
}
void launch_coarse_inverse(const Lev32& L, cudaStream_t s, float* ainv) {
    count_launches(1);
    k_coarse_inverse<<<1, NT, 0, s>>>(L, ainv);
}
void launch_coarse_solve(int n, cudaStream_t s, const float* ainv, const float* f, float* x) {
    count_launches(1);
    k_coarse_solve<<<1, 64, 0, s>>>(n, ainv, f, x);
}

}  // namespace lm
