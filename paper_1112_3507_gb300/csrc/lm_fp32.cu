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

// ---- 3D red-black sweep on whole tiles: a staged, recomputed halo box -----
//
// For 3D levels whose extents are multiples of the 32 x 8 x KZ tile.  The
// block owning the tile stages x_old and rho on the tile plus two cells in
// every direction in shared memory (periodic axes wrapped; past a Neumann
// wall x = 0 and rho = +inf, so that face's weight c2 / (rho_c + inf) is 0
// and no wall test is needed later).  Phase 1 updates the FIRST colour on the
// tile plus a one-cell halo in place -- a first-colour update reads only
// second-colour neighbours, so in-place is the red-black sweep -- and the
// halo values equal those the neighbouring blocks compute for their own
// cells; phase 2 updates the second colour of the tile from them; phase 3
// writes the tile in whole rows.  Work items enumerate only cells of the
// colour being updated, so no lane idles on a colour test.  Wrapped global
// offsets come from small per-block tables, so the staging and the f, c~
// loads need no per-cell wrap logic.  Same operations in the same order as
// rbgs_tile, so both kernels produce the same bits.
template <int KZ, int FIRST, bool ZERO, bool PROLONG>
__global__ void __launch_bounds__(256) k_rbgs_box(Lev32 L, const float* __restrict__ xin,
                                                 const float* __restrict__ ec, Geo C, int hx, int hy, int hz,
                                                 const float* __restrict__ f, float* __restrict__ xout) {
    constexpr int TX = 32, TY = 8, SX = TX + 4, SY = TY + 4, SZ = KZ + 4, PL = SX * SY;
    __shared__ float X[SZ * PL];
    __shared__ float R[SZ * PL];
    __shared__ int ox[SX], oy[SY], oz[SZ];       // wrapped offsets of staged coordinates, -1 past a wall
    __shared__ int px[SX], py[SY], pz[SZ];       // parent offsets (PROLONG)
    const Geo& g = L.g;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int k0 = blockIdx.x * KZ, i0 = blockIdx.y * TX, j0 = blockIdx.z * TY;
    const int sy = g.nx, sz = g.nx * g.ny;
    auto wrap = [](int c, int n, int bc) -> int {     // c within two cells of [0, n), n >= 2
        if (c < 0) return bc == LM_BC_PERIODIC ? c + n : -1;
        if (c >= n) return bc == LM_BC_PERIODIC ? c - n : -1;
        return c;
    };
    if (tid < SX) {
        const int c = wrap(i0 - 2 + tid, g.nx, g.bcx);
        ox[tid] = c;
        px[tid] = c >> hx;
    } else if (tid < SX + SY) {
        const int c = wrap(j0 - 2 + tid - SX, g.ny, g.bcy);
        oy[tid - SX] = c < 0 ? -1 : sy * c;
        py[tid - SX] = C.nx * (c >> hy);
    } else if (tid < SX + SY + SZ) {
        const int c = wrap(k0 - 2 + tid - SX - SY, g.nz, g.bcz);
        oz[tid - SX - SY] = c < 0 ? -1 : sz * c;
        pz[tid - SX - SY] = C.nx * C.ny * (c >> hz);
    }
    __syncthreads();
    // staging: each thread owns in-plane positions tid and tid + 256 of every
    // staged plane, so its wrapped (i, j) offsets are computed once
    {
        int pos[2], base[2], pbase[2];
        bool ok[2], use[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            pos[q] = tid + q * TX * TY;
            use[q] = pos[q] < PL;
            const int sj = use[q] ? pos[q] / SX : 0, si = use[q] ? pos[q] - sj * SX : 0;
            const int a = ox[si], b = oy[sj];
            ok[q] = use[q] && (a | b) >= 0;
            base[q] = a + b;
            pbase[q] = px[si] + py[sj];
        }
#pragma unroll 4
        for (int sk = 0; sk < SZ; ++sk) {
            const int c = oz[sk], pc = pz[sk];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!use[q]) continue;
                float xv = 0.f, rv = __int_as_float(0x7f800000);      // +inf
                if (ok[q] && c >= 0) {
                    const int idx = base[q] + c;
                    rv = L.rho[idx];
                    if (!ZERO) {
                        xv = xin[idx];
                        if (PROLONG) xv += ec[pbase[q] + pc];
                    }
                }
                X[sk * PL + pos[q]] = xv;
                R[sk * PL + pos[q]] = rv;
            }
        }
    }
    __syncthreads();

    // Gauss-Seidel value at staged position s of the in-domain cell with global index idx
    auto gs = [&](int s, int idx) -> float {
        const float rc = R[s];
        const float wxm = face32(rc, R[s - 1], L.c2x);
        const float wxp = face32(rc, R[s + 1], L.c2x);
        const float wym = face32(rc, R[s - SX], L.c2y);
        const float wyp = face32(rc, R[s + SX], L.c2y);
        const float wzm = face32(rc, R[s - PL], L.c2z);
        const float wzp = face32(rc, R[s + PL], L.c2z);
        const float d = L.ct[idx] + ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
        float num = f[idx];
        num = fmaf(wxm, X[s - 1], num);
        num = fmaf(wxp, X[s + 1], num);
        num = fmaf(wym, X[s - SX], num);
        num = fmaf(wyp, X[s + SX], num);
        num = fmaf(wzm, X[s - PL], num);
        num = fmaf(wzp, X[s + PL], num);
        return __fdividef(num, d);
    };

    // phase 1: first colour on the tile + one-cell halo (staged coordinates
    // 1 .. S - 2); thread t < 17 * 10 owns the t-th first-colour cell of
    // every halo-box plane
    constexpr int BXH = (TX + 2) / 2, BY = TY + 2, BZ = KZ + 2;
    const int par0 = (i0 + j0 + k0 + 1) & 1;                      // parity of staged cell (1, 1, 1)
    if (tid < BXH * BY) {
        const int m = tid % BXH, bj = tid / BXH;
        const int b = oy[bj + 1];
        const int ae = ox[2 * m + 1], ao = ox[2 * m + 2];          // the two x positions of the pair
#pragma unroll 2
        for (int bk = 0; bk < BZ; ++bk) {
            const int odd = (FIRST + par0 + bj + bk) & 1;
            const int s = ((bk + 1) * SY + bj + 1) * SX + 2 * m + odd + 1;
            const int a = odd ? ao : ae, c = oz[bk + 1];
            if ((a | b | c) >= 0) X[s] = gs(s, a + b + c);
        }
    }
    __syncthreads();
    // phase 2: second colour on the tile (staged coordinates 2 .. S - 3);
    // the two halves of the block take alternate planes
    {
        const int half = tid >> 7, t = tid & 127;
        const int m = t % (TX / 2), tj = t / (TX / 2);
        const int part = (i0 + j0 + k0) & 1;
        const int gbase = i0 + 2 * m + sy * (j0 + tj);
#pragma unroll 2
        for (int tk = half; tk < KZ; tk += 2) {
            const int odd = (1 - FIRST + part + tj + tk) & 1;
            const int s = ((tk + 2) * SY + tj + 2) * SX + 2 * m + odd + 2;
            X[s] = gs(s, gbase + odd + sz * (k0 + tk));
        }
    }
    __syncthreads();
    // phase 3: the tile, row by row
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll 4
    for (int tk = 0; tk < KZ; ++tk)
        xout[(i0 + tx) + sy * (j0 + ty) + sz * (k0 + tk)] = X[((tk + 2) * SY + ty + 2) * SX + tx + 2];
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
__global__ void __launch_bounds__(1024) k_coarse_inverse(Lev32 L, float* __restrict__ ainv) {
    // Gauss-Jordan inversion of the dense coarsest operator (n <= 64) in
    // float64; block (64, 16): thread (j, r) owns column j of rows r, r+16, ...
    __shared__ double A[64 * 64];
    __shared__ double colk[64], rowk[64];
    const Geo& g = L.g;
    const int n = g.N;
    const int lin = threadIdx.x + 64 * threadIdx.y;
    for (int e = lin; e < n * n; e += 1024) A[e] = 0.0;
    __syncthreads();
    if (lin < n) {
        const int idx = lin;
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
    const int jc = threadIdx.x;
    for (int kk = 0; kk < n; ++kk) {
        // pivot row scaled by the pivot's inverse, and the pivot column
        if (lin < n) {
            const double ipiv = 1.0 / A[kk * n + kk];
            colk[lin] = A[lin * n + kk];
            rowk[lin] = lin == kk ? ipiv : A[kk * n + lin] * ipiv;
        }
        __syncthreads();
        if (jc < n) {
            const double rj = rowk[jc];
            for (int i = threadIdx.y; i < n; i += 16) {
                double v;
                if (i == kk) v = rj;
                else if (jc == kk) v = -colk[i] * rj;
                else v = A[i * n + jc] - colk[i] * rj;
                A[i * n + jc] = v;
            }
        }
        __syncthreads();
    }
    for (int e = lin; e < n * n; e += 1024) ainv[e] = (float)A[e];
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
    if (g.ny > 1 && g.nx % 32 == 0 && g.ny % 8 == 0 && g.nz % 2 == 0) {
        // whole 32 x 8 x KZ tiles: the halo-box sweep; KZ the largest of
        // 8, 4, 2 that divides nz and still gives two blocks per SM (KZ = 8
        // keeps the staged box within 48 KB of static shared memory)
        const long long tiles = (long long)(g.nx / 32) * (g.ny / 8);
        int KZ = (kz == 2 || kz == 4 || kz == 8) && g.nz % kz == 0 ? kz : 0;
        if (!KZ) {
            KZ = 8;
            while (KZ > 2 && (g.nz % KZ || tiles * (g.nz / KZ) < 2 * 152)) KZ /= 2;
        }
        const dim3 grd(g.nz / KZ, g.nx / 32, g.ny / 8), blk(32, 8);
#define LM_RBB(K, F, Z, P) k_rbgs_box<K, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout)
#define LM_RBK(K)                                                              \
    if (zero) { if (first) LM_RBB(K, 1, true, false); else LM_RBB(K, 0, true, false); }          \
    else if (prolong) { if (first) LM_RBB(K, 1, false, true); else LM_RBB(K, 0, false, true); }  \
    else { if (first) LM_RBB(K, 1, false, false); else LM_RBB(K, 0, false, false); }
        if (KZ == 8) { LM_RBK(8) } else if (KZ == 4) { LM_RBK(4) } else { LM_RBK(2) }
#undef LM_RBK
#undef LM_RBB
    } else if (g.ny > 1) {
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
    k_coarse_inverse<<<1, dim3(64, 16), 0, s>>>(L, ainv);
}
void launch_coarse_solve(int n, cudaStream_t s, const float* ainv, const float* f, float* x) {
    count_launches(1);
    k_coarse_solve<<<1, 64, 0, s>>>(n, ainv, f, x);
}

}  // namespace lm
