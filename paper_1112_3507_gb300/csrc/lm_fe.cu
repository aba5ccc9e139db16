// The generalized Poisson operator of Eq. GeneralizedPoisson in Q1 finite
// elements (Sec. 2.5: the paper discretizes with finite elements, which give
// a symmetric positive-definite system), and its solvers.
//
// Unknowns sit at the points x_i = i h of every axis, stored like the cell
// grids (x fastest; 2D grids are (x, z) with one point along y).  A periodic
// axis of n points closes into a ring of n elements; a walled (Neumann)
// axis has n - 1 elements with its end points on the walls, where the
// homogeneous Neumann condition is the weak form's natural one.  Per element
// e, kappa_e is the harmonic mean of kappa = 1/rho over its corners and the
// element matrix is kappa_e K_ref, K_ref the tensor-product Q1 stiffness;
// the c~ term is mass-lumped (V_i c~_i, V_i the point's share of its
// elements).  So
//
//     B = diag(V c~) + sum_e kappa_e K_ref,    B x = b (b = V f + boundary data).
//
// Matrix-free form used by every kernel: a neighbour i + o of point i
// (o in {-1,0,1}^d, o != 0) couples with weight c(o) K_o(i), where K_o(i) is
// the sum of kappa_e over the elements holding both points and c(o) the
// entry of K_ref between two corners that differ along the axes where o is
// nonzero: c = sum_a S(d_a) prod_{b != a} M(d_b) with the 1D element
// stiffness S(0) = 1/h, S(1) = -1/h and mass M(0) = h/3, M(1) = h/6.  Each
// element matrix annihilates constants, hence
//
//     (B x)_i = V_i c~_i x_i + sum_{o != 0} c(o) K_o(i) (x_{i+o} - x_i).
//
// Elements are stored by their lowest corner with kappa_e = 0 at the
// positions past a wall, so every neighbour index simply wraps and the walls
// need no test.  On cubic elements the face-neighbour weight c is zero and
// those six neighbours are skipped.
//
// Solvers (lm_fe_solve): float64 Jacobi-PCG, and float64 iterative
// refinement around float32 flexible CG whose preconditioner is a two-level
// cycle: a damped Jacobi step on B, the finite-volume multigrid V-cycle of
// the same coefficients on the residual divided by V (B is close to V times
// the cell-centred operator on the same points), and a second Jacobi step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_internal.h"
#include "lm_kernels.h"

#define FECK(call)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            fprintf(stderr, "lowmach fe: %s: %s\n", #call, cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? LM_ERR_OUT_OF_MEMORY : LM_ERR_CUDA;   \
        }                                                                                  \
    } while (0)

namespace {

using lm::FF;
using lm::NT;
using lm::Red;
using lm::SolveState;

constexpr double FE_OMEGA = 0.8;     // Jacobi damping of the two-level preconditioner
constexpr int SLOT_RR = 8, SLOT_FF = 9;   // scalar slots of the refinement residual

struct FeGeo {
    int nx, ny, nz, N;
    int wx, wy, wz;          // 1: walled (Neumann) axis
    int dim;                 // 2: (x, z); 3
    double hx, hy, hz;
};

template <typename T>
struct FeOp {
    FeGeo g;
    T c[8];                  // c(o) by class: bit 0 x, bit 1 y, bit 2 z nonzero
    int faces;               // c of the single-axis classes nonzero
    const T* ke;             // element kappa by lowest corner
    const T* vc;             // V c~
    const T* dinv;           // 1 / diag(B)
};

// the point's share of its elements along one axis
__host__ __device__ __forceinline__ double vol1(int c, int n, int wall, double h) {
    return n == 1 ? 1.0 : ((wall && (c == 0 || c == n - 1)) ? 0.5 * h : h);
}

__device__ __forceinline__ void coords(int idx, const FeGeo& g, int& i, int& j, int& k) {
    i = idx % g.nx;
    const int t = idx / g.nx;
    j = t % g.ny;
    k = t / g.ny;
}

__device__ __forceinline__ int wrap_m(int c, int n) { return c > 0 ? c - 1 : n - 1; }
__device__ __forceinline__ int wrap_p(int c, int n) { return c < n - 1 ? c + 1 : 0; }

// Stiffness part of (B x)_i in 2D from X[oz+1][ox+1] and E[dz][dx] = kappa
// of the element with lowest corner (i - dx, k - dz).  Classes 1 (x), 4 (z), 5.
template <typename T>
__device__ __forceinline__ T stencil2(const T (&X)[3][3], const T (&E)[2][2], const T* c) {
    const T xc = X[1][1];
    const T ax = (E[0][0] + E[1][0]) * (X[1][2] - xc) + (E[0][1] + E[1][1]) * (X[1][0] - xc);
    const T az = (E[0][0] + E[0][1]) * (X[2][1] - xc) + (E[1][0] + E[1][1]) * (X[0][1] - xc);
    const T ac = E[0][0] * (X[2][2] - xc) + E[0][1] * (X[2][0] - xc) + E[1][0] * (X[0][2] - xc) +
                 E[1][1] * (X[0][0] - xc);
    return c[1] * ax + c[4] * az + c[5] * ac;
}

// Stiffness part of (B x)_i in 3D from X[oz+1][oy+1][ox+1] and E[dz][dy][dx]
// = kappa of the element with lowest corner (i - dx, j - dy, k - dz).  The
// elements holding both i and i + o have d_a = 0 where o_a = +1, d_a = 1
// where o_a = -1, and either where o_a = 0.
template <typename T>
__device__ __forceinline__ T stencil3(const T (&X)[3][3][3], const T (&E)[2][2][2], const T* c, int faces) {
    const T xc = X[1][1][1];
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = T(0);
#pragma unroll
    for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int cls = (ox != 0) | ((oy != 0) << 1) | ((oz != 0) << 2);
                if (cls == 0) continue;
                if ((cls == 1 || cls == 2 || cls == 4) && !faces) continue;
                T K = T(0);
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    if ((oz == 1 && dz == 1) || (oz == -1 && dz == 0)) continue;
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        if ((oy == 1 && dy == 1) || (oy == -1 && dy == 0)) continue;
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            if ((ox == 1 && dx == 1) || (ox == -1 && dx == 0)) continue;
                            K += E[dz][dy][dx];
                        }
                    }
                }
                acc[cls] += K * (X[oz + 1][oy + 1][ox + 1] - xc);
            }
    T y = T(0);
#pragma unroll
    for (int q = 1; q < 8; ++q) y += c[q] * acc[q];
    return y;
}

// (B x)_i at one point, every value loaded (ld(j) = x_j); xc returns x_i.
template <typename T, typename LD>
__device__ __forceinline__ T bx_point(int idx, const FeOp<T>& op, LD ld, T& xc) {
    const FeGeo& g = op.g;
    int i, j, k;
    coords(idx, g, i, j, k);
    const int sz = g.nx * g.ny;
    const int cx[3] = {wrap_m(i, g.nx), i, wrap_p(i, g.nx)};
    const int pz[3] = {wrap_m(k, g.nz) * sz, k * sz, wrap_p(k, g.nz) * sz};
    T st;
    if (g.dim == 2) {
        T X[3][3], E[2][2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) X[a][b] = ld(pz[a] + cx[b]);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) E[dz][dx] = op.ke[pz[1 - dz] + cx[1 - dx]];
        xc = X[1][1];
        st = stencil2(X, E, op.c);
    } else {
        const int ry[3] = {wrap_m(j, g.ny) * g.nx, j * g.nx, wrap_p(j, g.ny) * g.nx};
        T X[3][3][3], E[2][2][2];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) X[a][b][d] = ld(pz[a] + ry[b] + cx[d]);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) E[dz][dy][dx] = op.ke[pz[1 - dz] + ry[1 - dy] + cx[1 - dx]];
        xc = X[1][1][1];
        st = stencil3(X, E, op.c, op.faces);
    }
    return op.vc[idx] * xc + st;
}

// ---- set-up -----------------------------------------------------------------

struct FeFlags {
    int bad;       // rho or c~ not strictly positive and finite
    int bad32;     // a float32 coefficient outside the normal float32 range
};

__device__ __forceinline__ bool pos_finite(double v) { return v > 0.0 && v < INFINITY; }
__device__ __forceinline__ bool normal32(double v) { return v == 0.0 || (fabs(v) < 0x1p126 && fabs(v) > 0x1p-125); }

// kappa_e of the element with lowest corner idx (0 past a wall) and V c~.
__global__ void __launch_bounds__(NT) k_fe_setup(FeGeo g, const double* __restrict__ ct,
                                                 const double* __restrict__ rho, double* __restrict__ ke,
                                                 double* __restrict__ vc, FeFlags* fl) {
    bool bad = false;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        coords(idx, g, i, j, k);
        const double cti = ct[idx], ri = rho[idx];
        bad |= !pos_finite(cti) || !pos_finite(ri);
        const bool none = (g.wx && g.nx > 1 && i == g.nx - 1) || (g.wy && g.ny > 1 && j == g.ny - 1) ||
                          (g.wz && g.nz > 1 && k == g.nz - 1);
        double e = 0.0;
        if (!none) {
            const int sz = g.nx * g.ny;
            const int xs[2] = {i, wrap_p(i, g.nx)};
            const int ys[2] = {j * g.nx, wrap_p(j, g.ny) * g.nx};
            const int zs[2] = {k * sz, wrap_p(k, g.nz) * sz};
            const int ny2 = g.ny > 1 ? 2 : 1;
            double s = 0.0;
            int cnt = 0;
            for (int c = 0; c < 2; ++c)
                for (int b = 0; b < ny2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        s += rho[zs[c] + ys[b] + xs[a]];
                        ++cnt;
                    }
            e = cnt / s;
        }
        ke[idx] = e;
        vc[idx] = vol1(i, g.nx, g.wx, g.hx) * vol1(j, g.ny, g.wy, g.hy) * vol1(k, g.nz, g.wz, g.hz) * cti;
    }
    if (bad) atomicOr(&fl->bad, 1);
}

// 1/diag(B) = 1 / (V c~ + kd sum_{e ni i} kappa_e), and the float32 copies.
__global__ void __launch_bounds__(NT) k_fe_diag(FeGeo g, double kd, const double* __restrict__ ke,
                                                const double* __restrict__ vc, double* __restrict__ dinv,
                                                float* __restrict__ ke32, float* __restrict__ vc32,
                                                float* __restrict__ dinv32, FeFlags* fl) {
    bool bad32 = false;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        coords(idx, g, i, j, k);
        const int sz = g.nx * g.ny;
        const int xs[2] = {i, wrap_m(i, g.nx)};
        const int ys[2] = {j * g.nx, wrap_m(j, g.ny) * g.nx};
        const int zs[2] = {k * sz, wrap_m(k, g.nz) * sz};
        const int ny2 = g.ny > 1 ? 2 : 1;
        double s = 0.0;
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < ny2; ++b)
                for (int a = 0; a < 2; ++a) s += ke[zs[c] + ys[b] + xs[a]];
        const double d = vc[idx] + kd * s;
        const double di = 1.0 / d;
        dinv[idx] = di;
        const double kei = ke[idx], vci = vc[idx];
        bad32 |= !normal32(kei) || !normal32(vci) || !normal32(di);
        ke32[idx] = (float)kei;
        vc32[idx] = (float)vci;
        dinv32[idx] = (float)di;
    }
    if (bad32) atomicOr(&fl->bad32, 1);
}

// c~ = 1 / (dt^2 rho^n c_s^2) (Eq. cpoiss), evaluated as 1/(((dt*dt)*rho)*cs2); out may alias rho_old
__global__ void __launch_bounds__(NT) k_fe_ctilde(int N, double dt, const double* rho_old, const double* cs2,
                                                  double* out) {
    const double dt2 = dt * dt;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        out[idx] = 1.0 / ((dt2 * rho_old[idx]) * cs2[idx]);
}

// b = V f (f may alias b)
__global__ void __launch_bounds__(NT) k_fe_mass_times(FeGeo g, const double* f, double* b) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        coords(idx, g, i, j, k);
        b[idx] = vol1(i, g.nx, g.wx, g.hx) * vol1(j, g.ny, g.wy, g.hy) * vol1(k, g.nz, g.wz, g.hz) * f[idx];
    }
}

__global__ void __launch_bounds__(NT) k_fe_volume(FeGeo g, double* __restrict__ v) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        int i, j, k;
        coords(idx, g, i, j, k);
        v[idx] = vol1(i, g.nx, g.wx, g.hx) * vol1(j, g.ny, g.wy, g.hy) * vol1(k, g.nz, g.wz, g.hz);
    }
}

// ---- float64 kernels (one thread a point; the float64 pipe bounds them) ------

// y = B x; partial x.y (slot 0) when part; nothing once st->done
__global__ void __launch_bounds__(NT) k_fe_apply64(FeOp<double> op, const double* __restrict__ x,
                                                   double* __restrict__ y, double* part, const SolveState* st) {
    if (st && st->done) return;
    __shared__ double sm[32];
    double acc[1] = {0.0};
    auto ld = [&](int j) { return x[j]; };
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < op.g.N; idx += gridDim.x * blockDim.x) {
        double xc;
        const double v = bx_point(idx, op, ld, xc);
        y[idx] = v;
        acc[0] += xc * v;
    }
    if (part) lm::write_partials<1>(acc, part, sm);
}

// r = f - B x (zero_x: r = f and x = 0); partials r.r (slot 1) and f.f (slot 4)
__global__ void __launch_bounds__(NT) k_fe_resid64(FeOp<double> op, const double* __restrict__ f, double* x,
                                                   double* __restrict__ r, double* part, int zero_x) {
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    auto ld = [&](int j) { return x[j]; };
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < op.g.N; idx += gridDim.x * blockDim.x) {
        const double fi = f[idx];
        double xc;
        const double ri = zero_x ? fi : fi - bx_point(idx, op, ld, xc);
        r[idx] = ri;
        acc[0] += ri * ri;
        acc[1] += fi * fi;
    }
    if (zero_x)
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < op.g.N; idx += gridDim.x * blockDim.x) x[idx] = 0.0;
    lm::block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        part[1 * lm::MAX_PARTIALS + blockIdx.x] = acc[0];
        part[4 * lm::MAX_PARTIALS + blockIdx.x] = acc[1];
    }
}

// Refinement residual: r = f - B x, r32 = r * rscale (a power of two);
// the last block sets st->rel = ||r|| / ||f|| (and st->fnorm when SET_FNORM).
template <bool SET_FNORM>
__global__ void __launch_bounds__(NT) k_fe_ir_res64(FeOp<double> op, const double* __restrict__ f, double* x,
                                                    float* __restrict__ r32, int zero_x, double rscale, Red red,
                                                    SolveState* st) {
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    auto ld = [&](int j) { return x[j]; };
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < op.g.N; idx += gridDim.x * blockDim.x) {
        const double fi = f[idx];
        double xc;
        const double ri = zero_x ? fi : fi - bx_point(idx, op, ld, xc);
        if (zero_x) x[idx] = 0.0;
        r32[idx] = (float)(ri * rscale);
        acc[0] += ri * ri;
        acc[1] += fi * fi;
    }
    const int sl[2] = {SLOT_RR, SLOT_FF};
    if (lm::grid_reduce<2>(acc, red, sl, sm) && threadIdx.x == 0) {
        if (SET_FNORM) st->fnorm = sqrt(red.scal[SLOT_FF]);
        const double fn = st->fnorm;
        st->rel = fn > 0.0 ? sqrt(red.scal[SLOT_RR]) / fn : 0.0;
    }
}

// ---- float32 kernels -----------------------------------------------------------

enum { M_APPLY = 0, M_PRE = 1, M_POST = 2 };

// What a float32 operator kernel reads and writes:
//   M_APPLY  y = B a; x.y into scal slot 0 and r.x into slot 2 (r may be null)
//   M_PRE    y = (r - B a) / V
//   M_POST   y = (a + b) + omega D^-1 (r - B (a + b))
struct FeIO32 {
    const float* a;
    const float* b;
    const float* r;
    float* y;
    float omega;
};

// DOTS: 0 none, 1 x.y into scal slot 0, 2 also r.x into slot 2 (M_APPLY only)
template <int MODE, int DOTS>
__device__ __forceinline__ float fe_out(const FeIO32& io, const FeOp<float>& op, int idx, float xc, float bx,
                                        float iv, FF& axy, FF& arx) {
    if (MODE == M_APPLY) {
        if (DOTS >= 1) lm::ff_add_prod(axy, xc, bx);
        if (DOTS == 2) lm::ff_add_prod(arx, io.r[idx], xc);
        return bx;
    } else if (MODE == M_PRE) {
        return (io.r[idx] - bx) * iv;
    } else {
        return xc + io.omega * op.dinv[idx] * (io.r[idx] - bx);
    }
}

template <int MODE, int DOTS>
__device__ __forceinline__ void fe_reduce(FF axy, FF arx, const Red& red) {
    if (MODE != M_APPLY || DOTS == 0) return;
    __shared__ double sm[64];
    if (DOTS == 2) {
        double v[2] = {lm::ff_value(axy), lm::ff_value(arx)};
        const int sl[2] = {0, 2};
        lm::grid_reduce<2>(v, red, sl, sm);
    } else {
        double v[1] = {lm::ff_value(axy)};
        const int sl[1] = {0};
        lm::grid_reduce<1>(v, red, sl, sm);
    }
}

// 1/V along one axis in float32: interior and wall-end values
struct InvVol {
    float in, wall;
};
__host__ __device__ __forceinline__ InvVol inv_vol(int n, int wall, double h) {
    if (n == 1) return {1.f, 1.f};
    return {(float)(1.0 / h), (float)(wall ? 2.0 / h : 1.0 / h)};
}
__device__ __forceinline__ float inv_vol_at(const InvVol& v, int c, int n) {
    return (c == 0 || c == n - 1) ? v.wall : v.in;
}

// 2D, or any shape: one thread a point, grid-stride.
template <int MODE, int DOTS>
__global__ void __launch_bounds__(NT) k_fe_pt32(FeOp<float> op, FeIO32 io, Red red) {
    const FeGeo& g = op.g;
    const InvVol vx = inv_vol(g.nx, g.wx, g.hx), vy = inv_vol(g.ny, g.wy, g.hy), vz = inv_vol(g.nz, g.wz, g.hz);
    FF axy{0.f, 0.f}, arx{0.f, 0.f};
    auto ld = [&](int j) { return MODE == M_POST ? io.a[j] + io.b[j] : io.a[j]; };
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += gridDim.x * blockDim.x) {
        float xc;
        const float bx = bx_point(idx, op, ld, xc);
        float iv = 1.f;
        if (MODE == M_PRE) {
            int i, j, k;
            coords(idx, g, i, j, k);
            iv = inv_vol_at(vx, i, g.nx) * inv_vol_at(vy, j, g.ny) * inv_vol_at(vz, k, g.nz);
        }
        io.y[idx] = fe_out<MODE, DOTS>(io, op, idx, xc, bx, iv, axy, arx);
    }
    fe_reduce<MODE, DOTS>(axy, arx, red);
}

// Stiffness part of (B x)_i in 3D from the three planes of the x window
// (Xm: k - 1, Xc: k, Xp: k + 1, each [y offset + 1][x offset + 1]) and
// E[dz][dy][dx]; the same sums as stencil3 with the face classes fixed at
// compile time.
template <bool FACES>
__device__ __forceinline__ float stencil3p(const float (&Xm)[3][3], const float (&Xc)[3][3], const float (&Xp)[3][3],
                                           const float (&E)[2][2][2], const float* c) {
    const float xc = Xc[1][1];
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
#pragma unroll
    for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int cls = (ox != 0) | ((oy != 0) << 1) | ((oz != 0) << 2);
                if (cls == 0) continue;
                if (!FACES && (cls == 1 || cls == 2 || cls == 4)) continue;
                float K = 0.f;
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    if ((oz == 1 && dz == 1) || (oz == -1 && dz == 0)) continue;
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        if ((oy == 1 && dy == 1) || (oy == -1 && dy == 0)) continue;
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            if ((ox == 1 && dx == 1) || (ox == -1 && dx == 0)) continue;
                            K += E[dz][dy][dx];
                        }
                    }
                }
                const float xo = oz < 0 ? Xm[oy + 1][ox + 1] : (oz == 0 ? Xc[oy + 1][ox + 1] : Xp[oy + 1][ox + 1]);
                acc[cls] += K * (xo - xc);
            }
    float y = 0.f;
#pragma unroll
    for (int q = 1; q < 8; ++q)
        if (FACES || !(q == 1 || q == 2 || q == 4)) y += c[q] * acc[q];
    return y;
}

// 3D: a (32, 8) block of (x, y) columns marches up a chunk of KZ planes with
// the 3 x 3 x 3 window of x values and the 2 x 2 x 2 window of element
// kappas in registers: 9 new x values and 4 new kappas a point, through L1.
// Three plane arrays rotate roles (the loop unrolled three times, so no
// value moves).  (Issuing the next plane's loads before the point's
// arithmetic, with a fourth array, measured slower: 148 against 140 us.)
// (Four blocks per SM, 64 registers, for the solver's variants: measured
// 24.2 against 25.8 ms per 256^3 solve; the plain apply is faster at three
// blocks, 135 against 154 us, and keeps its 80 registers.)
template <int MODE, int DOTS, bool FACES>
__global__ void __launch_bounds__(256, (MODE == M_APPLY && DOTS == 0) ? 1 : 4)
    k_fe3_32(FeOp<float> op, FeIO32 io, Red red, int KZ) {
    const FeGeo& g = op.g;
    const int ti = blockIdx.x * 32 + threadIdx.x, tj = blockIdx.y * 8 + threadIdx.y;
    const bool live = ti < g.nx && tj < g.ny;
    const int i = live ? ti : 0, j = live ? tj : 0;
    const int k0 = blockIdx.z * KZ, k1 = min(k0 + KZ, g.nz);
    const int sz = g.nx * g.ny;
    const int cx[3] = {wrap_m(i, g.nx), i, wrap_p(i, g.nx)};
    const int ry[3] = {wrap_m(j, g.ny) * g.nx, j * g.nx, wrap_p(j, g.ny) * g.nx};
    int off[3][3];                      // in-plane offsets of the 3 x 3 neighbourhood
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int d = 0; d < 3; ++d) off[b][d] = ry[b] + cx[d];
    auto plane = [&](int k) { return (k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k)) * sz; };
    const InvVol vz = inv_vol(g.nz, g.wz, g.hz);
    const float ivxy = inv_vol_at(inv_vol(g.nx, g.wx, g.hx), i, g.nx) * inv_vol_at(inv_vol(g.ny, g.wy, g.hy), j, g.ny);
    const float* __restrict__ xa = io.a;
    const float* __restrict__ xb = io.b;
    const float* __restrict__ ke = op.ke;
    FF axy{0.f, 0.f}, arx{0.f, 0.f};
    float XA[3][3], XB[3][3], XC[3][3], E[2][2][2];
    auto load_plane = [&](float (&X)[3][3], int k) {
        const int p = plane(k);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int d = 0; d < 3; ++d) X[b][d] = MODE == M_POST ? xa[p + off[b][d]] + xb[p + off[b][d]] : xa[p + off[b][d]];
    };
    auto load_kappa = [&](float (&Ek)[2][2], int k) {
        const int p = plane(k);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) Ek[dy][dx] = ke[p + off[1 - dy][1 - dx]];
    };
    // point k from (Xm, Xc, Xp) = planes k - 1, k, k + 1; then plane k + 2
    // into Xm and the kappas of plane k + 1 into E[0] (E[1] <- E[0])
    auto step = [&](int k, float (&Xm)[3][3], float (&Xc)[3][3], float (&Xp)[3][3]) {
        const int idx = plane(k) + off[1][1];
        const float xc = Xc[1][1];
        const float bx = op.vc[idx] * xc + stencil3p<FACES>(Xm, Xc, Xp, E, op.c);
        const float iv = MODE == M_PRE ? ivxy * inv_vol_at(vz, k, g.nz) : 1.f;
        io.y[idx] = fe_out<MODE, DOTS>(io, op, idx, xc, bx, iv, axy, arx);
        if (k + 1 < k1) {
            load_plane(Xm, k + 2);
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) E[1][dy][dx] = E[0][dy][dx];
            load_kappa(E[0], k + 1);
        }
    };
    if (live && k0 < k1) {
        load_plane(XA, k0 - 1);
        load_plane(XB, k0);
        load_plane(XC, k0 + 1);
        load_kappa(E[1], k0 - 1);
        load_kappa(E[0], k0);
        for (int k = k0; k < k1; k += 3) {
            step(k, XA, XB, XC);
            if (k + 1 < k1) step(k + 1, XB, XC, XA);
            if (k + 2 < k1) step(k + 2, XC, XA, XB);
        }
    }
    fe_reduce<MODE, DOTS>(axy, arx, red);
}

__global__ void __launch_bounds__(NT) k_fe_jacobi32(int N, float omega, const float* __restrict__ dinv,
                                                    const float* __restrict__ r, float* __restrict__ t) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
        t[idx] = omega * dinv[idx] * r[idx];
}

}  // namespace

// ---- host side -------------------------------------------------------------------

struct lm_fe {
    int ndim = 0;
    int n[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    int bc[3] = {0, 0, 0};
    int N = 0;
    int G = 1;
    FeGeo geo{};
    double c[8] = {0};
    double kd = 0.0;           // K_ref's diagonal entry
    int faces = 1;
    lm_grid* fv = nullptr;     // cell-centred grid on the same points (the preconditioner's hierarchy)
    double *ke = nullptr, *vc = nullptr, *dinv = nullptr;
    double *f = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    float *ke32 = nullptr, *vc32 = nullptr, *dinv32 = nullptr;
    float *r32 = nullptr, *e32 = nullptr, *t32 = nullptr, *w32 = nullptr, *v32 = nullptr, *z32 = nullptr,
          *p32 = nullptr, *q32 = nullptr;
    double* part = nullptr;
    double* scal = nullptr;
    unsigned* ctr = nullptr;
    double* dscal = nullptr;
    double* hist_dev = nullptr;
    int hist_cap = 0;
    SolveState *st = nullptr, *st_in = nullptr, *st_host = nullptr;
    FeFlags *fl = nullptr, *fl_host = nullptr;
    bool have_coefs = false, fp32_ok = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

template <typename T>
int fe_alloc(T** p, size_t count) {
    return cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1)) == cudaSuccess ? LM_OK
                                                                                     : LM_ERR_OUT_OF_MEMORY;
}

template <typename T>
FeOp<T> fe_op(const lm_fe* fe) {
    FeOp<T> op;
    op.g = fe->geo;
    for (int q = 0; q < 8; ++q) op.c[q] = (T)fe->c[q];
    op.faces = fe->faces;
    if (sizeof(T) == sizeof(double)) {
        op.ke = (const T*)fe->ke;
        op.vc = (const T*)fe->vc;
        op.dinv = (const T*)fe->dinv;
    } else {
        op.ke = (const T*)fe->ke32;
        op.vc = (const T*)fe->vc32;
        op.dinv = (const T*)fe->dinv32;
    }
    return op;
}

Red fe_red(const lm_fe* fe) { return Red{fe->part, fe->scal, fe->ctr}; }

int fe_sync(lm_fe* fe, SolveState* dev, cudaStream_t s) {
    FECK(cudaMemcpyAsync(fe->st_host, dev, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    FECK(cudaStreamSynchronize(s));
    return LM_OK;
}

int fe_init_state(lm_fe* fe, SolveState* st, double rtol, cudaStream_t s) {
    SolveState h{};
    h.rtol = rtol;
    FECK(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, s));
    FECK(cudaStreamSynchronize(s));
    return LM_OK;
}

// float32 operator kernel of the given mode; dots as in fe_out
template <int MODE, int DOTS>
void launch_fe32_d(const lm_fe* fe, cudaStream_t s, const FeIO32& io) {
    const FeOp<float> op = fe_op<float>(fe);
    lm::count_launches(1);
    const int bx = (fe->geo.nx + 31) / 32, by = (fe->geo.ny + 7) / 8;
    const long long cols = (long long)bx * by;
    int chunks = (int)std::max(1LL, std::min<long long>(fe->geo.nz, (8LL * 152 + cols - 1) / cols));
    const int KZ = (fe->geo.nz + chunks - 1) / chunks;
    chunks = (fe->geo.nz + KZ - 1) / KZ;
    // one reduction partial a block: the column kernel when its blocks fit
    if (fe->geo.dim == 3 && cols * chunks <= lm::MAX_PARTIALS) {
        const dim3 grid(bx, by, chunks), block(32, 8);
        if (fe->faces)
            k_fe3_32<MODE, DOTS, true><<<grid, block, 0, s>>>(op, io, fe_red(fe), KZ);
        else
            k_fe3_32<MODE, DOTS, false><<<grid, block, 0, s>>>(op, io, fe_red(fe), KZ);
    } else {
        k_fe_pt32<MODE, DOTS><<<fe->G, NT, 0, s>>>(op, io, fe_red(fe));
    }
}

template <int MODE>
void launch_fe32(const lm_fe* fe, cudaStream_t s, const FeIO32& io, int dots = 0) {
    if (dots == 2)
        launch_fe32_d<MODE, 2>(fe, s, io);
    else if (dots == 1)
        launch_fe32_d<MODE, 1>(fe, s, io);
    else
        launch_fe32_d<MODE, 0>(fe, s, io);
}

void launch_fe_ir_res(const lm_fe* fe, cudaStream_t s, int zero_x, int set_fnorm, double rscale) {
    lm::count_launches(1);
    const FeOp<double> op = fe_op<double>(fe);
    if (set_fnorm)
        k_fe_ir_res64<true><<<fe->G, NT, 0, s>>>(op, fe->f, fe->x, fe->r32, zero_x, rscale, fe_red(fe), fe->st);
    else
        k_fe_ir_res64<false><<<fe->G, NT, 0, s>>>(op, fe->f, fe->x, fe->r32, zero_x, rscale, fe_red(fe), fe->st);
}

lm::PcgArgs fe_pcg_args(lm_fe* fe, int max_iter) {
    lm::PcgArgs a{};
    a.g.N = fe->N;
    a.op = lm::Op64{nullptr, nullptr, nullptr, nullptr, fe->dinv};
    a.f = fe->f;
    a.x = fe->x;
    a.r = fe->r;
    a.p = fe->p;
    a.q = fe->q;
    a.part = fe->part;
    a.st = fe->st;
    a.hist = fe->hist_dev;
    a.max_iter = max_iter;
    return a;
}

int fe_true_residual(lm_fe* fe, cudaStream_t s) {
    lm::count_launches(1);
    k_fe_resid64<<<fe->G, NT, 0, s>>>(fe_op<double>(fe), fe->f, fe->x, fe->r, fe->part, 0);
    lm::launch_reduce_rel(fe->part, fe->G, s, fe->st, nullptr);
    FECK(cudaGetLastError());
    return fe_sync(fe, fe->st, s);
}

// float64 Jacobi-PCG on B x = b
int fe_solve_pcg(lm_fe* fe, const lm_solve_opts* o, lm_solve_result* res, bool x0) {
    cudaStream_t s = S(o->cuda_stream);
    int rc;
    if (fe->hist_cap < o->max_iter + 2) {
        cudaFree(fe->hist_dev);
        fe->hist_dev = nullptr;
        fe->hist_cap = 0;
        if ((rc = fe_alloc(&fe->hist_dev, (size_t)o->max_iter + 2))) return rc;
        fe->hist_cap = o->max_iter + 2;
    }
    if ((rc = fe_init_state(fe, fe->st, o->rtol, s))) return rc;
    const lm::PcgArgs a = fe_pcg_args(fe, o->max_iter);
    const FeOp<double> op = fe_op<double>(fe);
    lm::count_launches(1);
    k_fe_resid64<<<fe->G, NT, 0, s>>>(op, fe->f, fe->x, fe->r, fe->part, x0 ? 0 : 1);
    lm::launch_pcg_init_p(a, fe->G, s, 2, 0);
    FECK(cudaGetLastError());
    if ((rc = fe_sync(fe, fe->st, s))) return rc;
    int k = 0, restarts = 0;
    const int chunk = std::max(1, o->check_every);
    while (!fe->st_host->done) {
        for (int c = 0; c < chunk && k < o->max_iter; ++c, ++k) {
            lm::count_launches(1);
            k_fe_apply64<<<fe->G, NT, 0, s>>>(op, fe->p, fe->q, fe->part, fe->st);
            lm::launch_pcg_xr(a, fe->G, s, k);
            lm::launch_pcg_p(a, fe->G, s, k);
        }
        FECK(cudaGetLastError());
        if ((rc = fe_sync(fe, fe->st, s))) return rc;
        if (fe->st_host->status) break;
        if (fe->st_host->converged) {
            // confirm on the true residual; restart from it when the recursion drifted
            if ((rc = fe_true_residual(fe, s))) return rc;
            if (fe->st_host->rel <= o->rtol || restarts >= 3 || k >= o->max_iter) break;
            ++restarts;
            k = fe->st_host->iters;
            lm::launch_pcg_restart(a, fe->G, s, k);
            if ((rc = fe_sync(fe, fe->st, s))) return rc;
            continue;
        }
        if (k >= o->max_iter) break;
    }
    const SolveState h = *fe->st_host;
    if ((rc = fe_true_residual(fe, s))) return rc;
    res->iters = h.iters;
    res->rel_residual = fe->st_host->rel;
    if (h.status) return h.status;
    return fe->st_host->rel <= o->rtol ? LM_OK : LM_ERR_NO_CONVERGENCE;
}

// z = M r: Jacobi step, V-cycle of the cell-centred operator on (r - B t) / V, Jacobi step
int fe_precond(lm_fe* fe, const lm_solve_opts* o, cudaStream_t s) {
    const float om = (float)FE_OMEGA;
    lm::count_launches(1);
    k_fe_jacobi32<<<fe->G, NT, 0, s>>>(fe->N, om, fe->dinv32, fe->r32, fe->t32);
    launch_fe32<M_PRE>(fe, s, FeIO32{fe->t32, nullptr, fe->r32, fe->w32, om});
    const int rc = lm_mg_vcycle(fe->fv, fe->w32, fe->v32, o->nu1, o->nu2, s);
    if (rc) return rc;
    launch_fe32<M_POST>(fe, s, FeIO32{fe->t32, fe->v32, fe->r32, fe->z32, om});
    return LM_OK;
}

// inner float32 flexible CG on B e = r (r overwritten)
int fe_inner(lm_fe* fe, const lm_solve_opts* o, cudaStream_t s, int* iters, int* vcycles) {
    int rc;
    const Red red = fe_red(fe);
    FECK(cudaMemsetAsync(fe->e32, 0, sizeof(float) * fe->N, s));
    if ((rc = fe_init_state(fe, fe->st_in, o->inner_rtol, s))) return rc;
    lm::launch_dot32(fe->N, fe->G, s, fe->r32, fe->r32, red, 4, fe->st_in);
    for (int it = 0; it < o->inner_max_iter; ++it) {
        if ((rc = fe_precond(fe, o, s))) return rc;
        ++*vcycles;
        if (it > 0) lm::launch_dot32(fe->N, fe->G, s, fe->z32, fe->q32, red, 3, nullptr);
        lm::launch_fcg_beta_p(fe->N, fe->G, s, fe->z32, fe->p32, fe->scal, it == 0);
        launch_fe32<M_APPLY>(fe, s, FeIO32{fe->p32, nullptr, fe->r32, fe->q32, 0.f}, 2);
        lm::launch_fcg_update(fe->N, fe->G, s, fe->e32, fe->r32, fe->p32, fe->q32, red, fe->st_in);
        FECK(cudaGetLastError());
        ++*iters;
        if ((rc = fe_sync(fe, fe->st_in, s))) return rc;
        if (fe->st_host->status) return LM_OK;
        if (fe->st_host->rel <= o->inner_rtol) break;
    }
    return LM_OK;
}

// float64 iterative refinement around the float32 inner solve
int fe_solve_mixed(lm_fe* fe, const lm_solve_opts* o, lm_solve_result* res, bool x0) {
    cudaStream_t s = S(o->cuda_stream);
    int rc;
    if (!fe->fp32_ok) return LM_ERR_INVALID_ARG;
    if ((rc = fe_init_state(fe, fe->st, o->rtol, s))) return rc;
    launch_fe_ir_res(fe, s, x0 ? 0 : 1, 1, 1.0);
    FECK(cudaGetLastError());
    if ((rc = fe_sync(fe, fe->st, s))) return rc;
    if (!(fe->st_host->fnorm > 0.0)) {
        res->rel_residual = 0.0;
        return LM_OK;
    }
    double rel = fe->st_host->rel;
    const double fnorm = fe->st_host->fnorm, sqN = std::sqrt((double)fe->N);
    // inner right-hand sides of about unit size (power-of-two scaling, exact)
    double rs = lm::pow2_near_inv(rel * fnorm / sqN);
    if (rs > 0x1p20 || rs < 0x1p-20) lm::launch_scale32(fe->N, fe->G, s, fe->r32, (float)rs);
    else rs = 1.0;
    int outer = 0, iters = 0, vc = 0, status = LM_OK;
    while (rel > o->rtol && outer < o->max_outer && iters < o->max_iter) {
        if ((rc = fe_inner(fe, o, s, &iters, &vc))) return rc;
        if (fe->st_host->status) status = fe->st_host->status;
        lm::launch_ir_correct(fe->N, fe->G, s, fe->x, fe->e32, 1.0 / rs);
        const double rs_next = lm::pow2_near_inv(rel * fnorm * std::max(o->inner_rtol, 1e-12) / sqN);
        launch_fe_ir_res(fe, s, 0, 0, rs_next);
        FECK(cudaGetLastError());
        if ((rc = fe_sync(fe, fe->st, s))) return rc;
        const double nrel = fe->st_host->rel;
        ++outer;
        rs = rs_next;
        if (!(nrel < rel) && status) break;
        rel = nrel;
        status = LM_OK;
    }
    res->iters = iters;
    res->outer_iters = outer;
    res->vcycles = vc;
    res->rel_residual = rel;
    if (status) return status;
    return rel <= o->rtol ? LM_OK : LM_ERR_NO_CONVERGENCE;
}

void fe_free(lm_fe* fe) {
    if (fe->fv) lm_grid_destroy(fe->fv);
    void* bufs[] = {fe->ke, fe->vc, fe->dinv, fe->f, fe->x, fe->r, fe->p, fe->q, fe->ke32, fe->vc32, fe->dinv32,
                    fe->r32, fe->e32, fe->t32, fe->w32, fe->v32, fe->z32, fe->p32, fe->q32, fe->part, fe->scal,
                    fe->ctr, fe->dscal, fe->hist_dev, fe->st, fe->st_in, fe->fl};
    for (void* b : bufs) cudaFree(b);
    cudaFreeHost(fe->st_host);
    cudaFreeHost(fe->fl_host);
    if (fe->ev0) cudaEventDestroy(fe->ev0);
    if (fe->ev1) cudaEventDestroy(fe->ev1);
}

// element kappa, V c~, the inverse diagonal, the float32 copies and the
// preconditioner's cell-centred coefficients from device c~ and rho
int fe_setup(lm_fe* fe, const double* ct, const double* rh, cudaStream_t s) {
    FECK(cudaMemsetAsync(fe->fl, 0, sizeof(FeFlags), s));
    lm::count_launches(2);
    k_fe_setup<<<fe->G, NT, 0, s>>>(fe->geo, ct, rh, fe->ke, fe->vc, fe->fl);
    k_fe_diag<<<fe->G, NT, 0, s>>>(fe->geo, fe->kd, fe->ke, fe->vc, fe->dinv, fe->ke32, fe->vc32, fe->dinv32, fe->fl);
    FECK(cudaGetLastError());
    FECK(cudaMemcpyAsync(fe->fl_host, fe->fl, sizeof(FeFlags), cudaMemcpyDeviceToHost, s));
    FECK(cudaStreamSynchronize(s));
    if (fe->fl_host->bad) return LM_ERR_NOT_POSITIVE;
    const int rc = lm_set_coefficients_raw(fe->fv, ct, rh, 1, s);
    fe->fp32_ok = rc == LM_OK && !fe->fl_host->bad32;
    if (rc && rc != LM_ERR_INVALID_ARG) return rc;
    fe->have_coefs = true;
    return LM_OK;
}

}  // namespace

extern "C" {

int lm_fe_create(int ndim, const int64_t n[3], const double h[3], const int bc[3], lm_fe** out) {
    if (!out || !n || !h || !bc || (ndim != 2 && ndim != 3)) return LM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || !(h[a] > 0.0) || !(h[a] < 1e300) || (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN))
            return LM_ERR_INVALID_ARG;
    if ((ndim == 2 && n[1] != 1) || (ndim == 3 && n[1] < 2) || n[0] < 2 || n[2] < 2) return LM_ERR_INVALID_ARG;
    if ((long long)n[0] * n[1] * n[2] >= (1LL << 31)) return LM_ERR_INVALID_ARG;
    lm_fe* fe = new lm_fe;
    fe->ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        fe->n[a] = (int)n[a];
        fe->h[a] = h[a];
        fe->bc[a] = bc[a];
    }
    fe->N = fe->n[0] * fe->n[1] * fe->n[2];
    fe->G = std::max(1, std::min(8 * 152, (fe->N + NT - 1) / NT));
    FeGeo& g = fe->geo;
    g.nx = fe->n[0];
    g.ny = fe->n[1];
    g.nz = fe->n[2];
    g.N = fe->N;
    g.wx = bc[0] == LM_BC_NEUMANN;
    g.wy = bc[1] == LM_BC_NEUMANN;
    g.wz = bc[2] == LM_BC_NEUMANN;
    g.dim = ndim;
    g.hx = h[0];
    g.hy = h[1];
    g.hz = h[2];
    // K_ref entries by class (bit a: the two corners differ along axis a),
    // over the axes that carry elements
    const int live[3] = {1, ndim == 3 ? 1 : 0, 1};
    for (int cls = 0; cls < 8; ++cls) {
        double v = 0.0;
        bool any = false;
        for (int a = 0; a < 3; ++a) {
            if (!live[a]) continue;
            const int da = (cls >> a) & 1;
            double t = (da ? -1.0 : 1.0) / h[a];
            for (int b = 0; b < 3; ++b) {
                if (b == a || !live[b]) continue;
                const int db = (cls >> b) & 1;
                t *= h[b] * (db ? 1.0 / 6.0 : 2.0 / 6.0);
            }
            v += t;
            any = true;
        }
        bool valid = true;
        for (int a = 0; a < 3; ++a)
            if (!live[a] && ((cls >> a) & 1)) valid = false;
        fe->c[cls] = (any && valid) ? v : 0.0;
    }
    fe->kd = fe->c[0];
    fe->c[0] = 0.0;
    const double tiny = 1e-14 * std::fabs(fe->kd);
    fe->faces = (std::fabs(fe->c[1]) > tiny || std::fabs(fe->c[2]) > tiny || std::fabs(fe->c[4]) > tiny) ? 1 : 0;
    if (!fe->faces) fe->c[1] = fe->c[2] = fe->c[4] = 0.0;
    const size_t N = fe->N;
    int rc = lm_grid_create(ndim, n, h, bc, &fe->fv);
    double** d64[] = {&fe->ke, &fe->vc, &fe->dinv, &fe->f, &fe->x, &fe->r, &fe->p, &fe->q};
    float** d32[] = {&fe->ke32, &fe->vc32, &fe->dinv32, &fe->r32, &fe->e32, &fe->t32,
                     &fe->w32,  &fe->v32,  &fe->z32,    &fe->p32, &fe->q32};
    for (double** b : d64)
        if (!rc) rc = fe_alloc(b, N);
    for (float** b : d32)
        if (!rc) rc = fe_alloc(b, N);
    if (!rc) rc = fe_alloc(&fe->part, (size_t)lm::NSLOT * lm::MAX_PARTIALS);
    if (!rc) rc = fe_alloc(&fe->scal, 16);
    if (!rc) rc = fe_alloc(&fe->ctr, 1);
    if (!rc) rc = fe_alloc(&fe->dscal, 4);
    if (!rc) rc = fe_alloc(&fe->st, 1);
    if (!rc) rc = fe_alloc(&fe->st_in, 1);
    if (!rc) rc = fe_alloc(&fe->fl, 1);
    if (!rc && (cudaMallocHost((void**)&fe->st_host, sizeof(SolveState)) != cudaSuccess ||
                cudaMallocHost((void**)&fe->fl_host, sizeof(FeFlags)) != cudaSuccess ||
                cudaMemset(fe->ctr, 0, sizeof(unsigned)) != cudaSuccess ||
                cudaEventCreate(&fe->ev0) != cudaSuccess || cudaEventCreate(&fe->ev1) != cudaSuccess))
        rc = LM_ERR_OUT_OF_MEMORY;
    if (rc) {
        fe_free(fe);
        delete fe;
        return rc;
    }
    *out = fe;
    return LM_OK;
}

void lm_fe_destroy(lm_fe* fe) {
    if (!fe) return;
    cudaDeviceSynchronize();
    fe_free(fe);
    delete fe;
}

int lm_fe_set_coefficients(lm_fe* fe, const double* ctilde, const double* rho, int on_device, void* stream) {
    if (!fe || !ctilde || !rho) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    fe->have_coefs = false;
    const double* ct = ctilde;
    const double* rh = rho;
    if (!on_device) {      // stage through the solver's own buffers
        FECK(cudaMemcpyAsync(fe->r, ctilde, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
        FECK(cudaMemcpyAsync(fe->p, rho, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
        ct = fe->r;
        rh = fe->p;
    }
    return fe_setup(fe, ct, rh, s);
}

int lm_fe_set_state(lm_fe* fe, const double* rho_old, const double* rho_new, const double* cs2, double dt,
                    int on_device, void* stream) {
    if (!fe || !rho_old || !rho_new || !cs2) return LM_ERR_INVALID_ARG;
    if (!(dt > 0.0 && dt < 1e300)) return LM_ERR_NOT_POSITIVE;
    cudaStream_t s = S(stream);
    fe->have_coefs = false;
    const double* ro = rho_old;
    const double* rn = rho_new;
    const double* c2 = cs2;
    if (!on_device) {
        FECK(cudaMemcpyAsync(fe->r, rho_old, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
        FECK(cudaMemcpyAsync(fe->p, rho_new, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
        FECK(cudaMemcpyAsync(fe->q, cs2, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
        ro = fe->r;
        rn = fe->p;
        c2 = fe->q;
    }
    lm::count_launches(1);
    k_fe_ctilde<<<fe->G, NT, 0, s>>>(fe->N, dt, ro, c2, fe->r);
    FECK(cudaGetLastError());
    return fe_setup(fe, fe->r, rn, s);
}

int lm_fe_mass_times(lm_fe* fe, const double* f, double* b, int on_device, void* stream) {
    if (!fe || !f || !b) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    if (on_device) {
        lm::count_launches(1);
        k_fe_mass_times<<<fe->G, NT, 0, s>>>(fe->geo, f, b);
        FECK(cudaGetLastError());
        return LM_OK;
    }
    FECK(cudaMemcpyAsync(fe->q, f, sizeof(double) * fe->N, cudaMemcpyHostToDevice, s));
    lm::count_launches(1);
    k_fe_mass_times<<<fe->G, NT, 0, s>>>(fe->geo, fe->q, fe->q);
    FECK(cudaGetLastError());
    FECK(cudaMemcpyAsync(b, fe->q, sizeof(double) * fe->N, cudaMemcpyDeviceToHost, s));
    FECK(cudaStreamSynchronize(s));
    return LM_OK;
}

int lm_fe_lumped_mass(lm_fe* fe, double* v, int on_device, void* stream) {
    if (!fe || !v) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    lm::count_launches(1);
    k_fe_volume<<<fe->G, NT, 0, s>>>(fe->geo, on_device ? v : fe->q);
    FECK(cudaGetLastError());
    if (!on_device) {
        FECK(cudaMemcpyAsync(v, fe->q, sizeof(double) * fe->N, cudaMemcpyDeviceToHost, s));
        FECK(cudaStreamSynchronize(s));
    }
    return LM_OK;
}

int lm_fe_apply(lm_fe* fe, int prec, const void* x, void* y, double* dot_out, void* stream) {
    if (!fe || !x || !y || x == y || (prec != LM_PREC_FP64 && prec != LM_PREC_FP32)) return LM_ERR_INVALID_ARG;
    if (!fe->have_coefs) return LM_ERR_STATE;
    cudaStream_t s = S(stream);
    const double* dot_dev = fe->dscal;
    if (prec == LM_PREC_FP64) {
        lm::count_launches(1);
        k_fe_apply64<<<fe->G, NT, 0, s>>>(fe_op<double>(fe), (const double*)x, (double*)y,
                                          dot_out ? fe->part : nullptr, nullptr);
        if (dot_out) lm::launch_reduce_slot(fe->part, 0, fe->G, s, fe->dscal);
    } else {
        if (!fe->fp32_ok) return LM_ERR_INVALID_ARG;
        launch_fe32<M_APPLY>(fe, s, FeIO32{(const float*)x, nullptr, nullptr, (float*)y, 0.f}, dot_out ? 1 : 0);
        dot_dev = fe->scal;
    }
    FECK(cudaGetLastError());
    if (dot_out) {
        double hv;
        FECK(cudaMemcpyAsync(&hv, dot_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        FECK(cudaStreamSynchronize(s));
        *dot_out = hv;
    }
    return LM_OK;
}

int lm_fe_solve(lm_fe* fe, const double* b, double* x, int on_device, const lm_solve_opts* opts,
                lm_solve_result* res) {
    if (!fe || !b || !x || !opts || !res) return LM_ERR_INVALID_ARG;
    if (!fe->have_coefs) return LM_ERR_STATE;
    const lm_solve_opts& o = *opts;
    if (!(o.rtol > 0.0) || o.max_iter < 1 || o.max_outer < 1 || o.inner_max_iter < 1 || o.nu1 < 1 || o.nu2 < 1 ||
        o.nu1 > 8 || o.nu2 > 8 || !(o.inner_rtol > 0.0 && o.inner_rtol < 1.0))
        return LM_ERR_INVALID_ARG;
    if (o.mode != LM_FP64_JACOBI_PCG && o.mode != LM_MIXED_MG_IR) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(o.cuda_stream);
    *res = lm_solve_result{};
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    FECK(cudaMemcpyAsync(fe->f, b, sizeof(double) * fe->N, in, s));
    if (o.use_x0) FECK(cudaMemcpyAsync(fe->x, x, sizeof(double) * fe->N, in, s));
    FECK(cudaEventRecord(fe->ev0, s));
    int rc = o.mode == LM_FP64_JACOBI_PCG ? fe_solve_pcg(fe, &o, res, o.use_x0 != 0)
                                           : fe_solve_mixed(fe, &o, res, o.use_x0 != 0);
    FECK(cudaEventRecord(fe->ev1, s));
    if (rc == LM_OK || rc == LM_ERR_NO_CONVERGENCE || rc == LM_ERR_BREAKDOWN) {
        FECK(cudaMemcpyAsync(x, fe->x, sizeof(double) * fe->N,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    FECK(cudaStreamSynchronize(s));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, fe->ev0, fe->ev1) == cudaSuccess) res->seconds = 1e-3 * ms;
    res->status = rc;
    return rc;
}

}  // extern "C"
