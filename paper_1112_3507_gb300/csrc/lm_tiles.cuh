// Device bodies of the float32 kernels, written against explicit block
// coordinates so that one launch can serve a single grid (block = its
// blockIdx) or a batch of grids (block = an entry of a task table).
#pragma once

#include "lm_common.cuh"
#include "lm_kernels.h"

namespace lm {

// ---- float64 operator -------------------------------------------------------
// (A x)_i = c~_i x_i + sum over the faces g_f (x_i - x_nb), with the assembled
// minus-face conductances (0 on walls): 13 float64 operations per 3D cell.
__device__ __forceinline__ double apply64_at(int idx, const Geo& g, const Op64& op,
                                             const double* __restrict__ x) {
    int i, j, k;
    cell_coords(idx, g, i, j, k);
    const double xc = x[idx];
    double y = op.ct[idx] * xc;
    Nbr n = nbr_x(idx, i, g);
    y += op.gx[idx] * (xc - x[n.im]);
    y += op.gx[n.ip] * (xc - x[n.ip]);
    if (g.ny > 1) {
        n = nbr_y(idx, j, g);
        y += op.gy[idx] * (xc - x[n.im]);
        y += op.gy[n.ip] * (xc - x[n.ip]);
    }
    n = nbr_z(idx, k, g);
    y += op.gz[idx] * (xc - x[n.im]);
    y += op.gz[n.ip] * (xc - x[n.ip]);
    return y;
}

// Coefficient assembly (step (v); Eqs. cpoiss, kappapoiss) of the cells
// start, start + stride, ... of one grid, with the range of rho^{n+1} and
// the failure flags reduced per warp into a.fl (every lane of a warp must
// call this; the launches use whole warps).
__device__ __forceinline__ void assemble_range(const AsmArgs& a, int start, int stride) {
    const Geo& g = a.g;
    const double *a_in = a.a_in, *rho_new = a.rho_new, *cs2 = a.cs2;
    const double dt = a.dt, c2x = a.c2x, c2y = a.c2y, c2z = a.c2z;
    const int raw = a.raw;
    const Op64Out& out = a.out;
    AsmFlags* fl = a.fl;
    unsigned long long rmax = 0ull, rmin = ~0ull;        // range of the valid rho^{n+1}
    bool bad32 = false;
    for (int idx = start; idx < g.N; idx += stride) {
        const double rn = rho_new[idx];
        double c;
        bool ok = rn > 0.0 && isfinite(rn);
        if (raw) {
            c = a_in[idx];
        } else {
            const double ro = a_in[idx], c2 = cs2[idx];
            ok = ok && ro > 0.0 && isfinite(ro) && c2 > 0.0 && isfinite(c2);
            c = __drcp_rn((dt * dt) * ro * c2);                // Eq. cpoiss: 1/(...) rounded to nearest
        }
        ok = ok && c > 0.0 && isfinite(c);
        if (!ok) atomicOr(&fl->bad, 1);
        if (rn > 0.0 && isfinite(rn)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(rn);
            rmax = b > rmax ? b : rmax;
            rmin = b < rmin ? b : rmin;
        }
        int i, j, k;
        cell_coords(idx, g, i, j, k);
        // g_f = kappa_f / h^2 with kappa_f = 2/(rho_L + rho_R) (Eq. kappapoiss, harmonic
        // mean), evaluated as (2/h^2) * RN(1/(rho_L + rho_R)): a correctly rounded
        // float64 reciprocal per face (cheaper than a division on GB300's float64
        // pipe); exact scaling, so bit-identical to 2/(rho_L + rho_R)/h^2 when h is
        // a power of two, within 2 ulp otherwise
        const double gxm = face_minus(i, g.nx, g.bcx) ? c2x * __drcp_rn(rn + rho_new[nbr_x(idx, i, g).im]) : 0.0;
        const double gym = face_minus(j, g.ny, g.bcy) ? c2y * __drcp_rn(rn + rho_new[nbr_y(idx, j, g).im]) : 0.0;
        const double gzm = face_minus(k, g.nz, g.bcz) ? c2z * __drcp_rn(rn + rho_new[nbr_z(idx, k, g).im]) : 0.0;
        out.ct[idx] = c;
        out.gx[idx] = gxm;
        out.gy[idx] = gym;
        out.gz[idx] = gzm;
        const float c32 = (float)c;
        bad32 = bad32 || !(c32 > 0.f) || isinf(c32);
        out.ct32[idx] = c32;
        out.rho32[idx] = (float)rn;
    }
    // the block's range and float32 flag: one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, rmax, o), b = __shfl_xor_sync(0xffffffffu, rmin, o);
        rmax = a > rmax ? a : rmax;
        rmin = b < rmin ? b : rmin;
    }
    bad32 = __any_sync(0xffffffffu, bad32);
    if ((threadIdx.x & 31) == 0) {
        if (rmax) atomicMax(&fl->rho_max, rmax);
        if (rmin != ~0ull) atomicMin(&fl->rho_min, rmin);
        if (bad32) atomicOr(&fl->bad32, 1);
    }
}

// ---- float32 operator -------------------------------------------------------
// g = (2/h^2) / (rho_a + rho_b); the sum is commutative, so both cells of a
// face compute the same bits and the operator stays exactly symmetric.
__device__ __forceinline__ float face32(float ra, float rb, float c2) { return __fdividef(c2, ra + rb); }

// y = A x on the tile (bx, by, bz) of a block (32, 8): 3D, an x-y tile and
// the z chunk bz of KZ_APPLY planes; 2D, 32 columns and 8 chunks of rows.
// Accumulates x.y and x.r of this thread into axy, axr.
template <bool HAS_Y, bool DOT_XY, bool DOT_XR>
__device__ __forceinline__ void apply32z_tile(const Lev32& L, const float* __restrict__ x, float* __restrict__ y,
                                              const float* __restrict__ r, int KZ_APPLY, int bx, int by, int bz,
                                              FF& axy, FF& axr) {
    const Geo& g = L.g;
    const int i = bx * 32 + threadIdx.x;
    int j, kb;
    if (HAS_Y) {
        j = by * 8 + threadIdx.y;
        kb = bz * KZ_APPLY;
    } else {
        j = 0;
        kb = (by * 8 + threadIdx.y) * KZ_APPLY;
    }
    if (i < g.nx && j < g.ny && kb < g.nz) {
        const int ke = min(kb + KZ_APPLY, g.nz);
        const int sz = g.nx * g.ny;
        const int col = i + g.nx * j;
        const int cxm = i > 0 ? col - 1 : col + g.nx - 1;
        const int cxp = i < g.nx - 1 ? col + 1 : col - (g.nx - 1);
        const bool fxm = face_minus(i, g.nx, g.bcx), fxp = face_plus(i, g.nx, g.bcx);
        int cym = col, cyp = col;
        bool fym = false, fyp = false;
        if (HAS_Y) {
            cym = j > 0 ? col - g.nx : col + (g.ny - 1) * g.nx;
            cyp = j < g.ny - 1 ? col + g.nx : col - (g.ny - 1) * g.nx;
            fym = face_minus(j, g.ny, g.bcy);
            fyp = face_plus(j, g.ny, g.bcy);
        }
        const int kd0 = kb > 0 ? kb - 1 : g.nz - 1;
        float xd = x[col + sz * kd0], rd = L.rho[col + sz * kd0];
        float xc = x[col + sz * kb], rc = L.rho[col + sz * kb];
        float ctc = L.ct[col + sz * kb], rrc = DOT_XR ? r[col + sz * kb] : 0.f;
        for (int k = kb; k < ke; ++k) {
            const int ku = k < g.nz - 1 ? k + 1 : 0;
            // next plane's streams are requested before this plane's arithmetic
            const float xu = x[col + sz * ku], ru = L.rho[col + sz * ku];
            const float ctn = L.ct[col + sz * ku], rrn = DOT_XR ? r[col + sz * ku] : 0.f;
            const int o = sz * k;
            float v = ctc * xc;
            if (fxm) v += face32(rc, L.rho[cxm + o], L.c2x) * (xc - x[cxm + o]);
            if (fxp) v += face32(rc, L.rho[cxp + o], L.c2x) * (xc - x[cxp + o]);
            if (HAS_Y) {
                if (fym) v += face32(rc, L.rho[cym + o], L.c2y) * (xc - x[cym + o]);
                if (fyp) v += face32(rc, L.rho[cyp + o], L.c2y) * (xc - x[cyp + o]);
            }
            if (face_minus(k, g.nz, g.bcz)) v += face32(rc, rd, L.c2z) * (xc - xd);
            if (face_plus(k, g.nz, g.bcz)) v += face32(rc, ru, L.c2z) * (xc - xu);
            y[col + o] = v;
            if (DOT_XY) ff_add_prod(axy, xc, v);
            if (DOT_XR) ff_add_prod(axr, xc, rrc);
            xd = xc;
            rd = rc;
            xc = xu;
            rc = ru;
            ctc = ctn;
            rrc = rrn;
        }
    }
}

// ---- 1D vector steps over a block range (block blk of nblk, NT threads) --

__device__ __forceinline__ FF dot32_range(int N, const float* __restrict__ a, const float* __restrict__ b, int blk,
                                          int nblk) {
    FF acc{0.f, 0.f};
    const int stride = nblk * NT;
#pragma unroll 4
    for (int idx = blk * NT + threadIdx.x; idx < N; idx += stride) ff_add_prod(acc, a[idx], b[idx]);
    return acc;
}

// Flexible CG, truncation 1 (Notay 2000): p = z - (z.q_old / p_old.q_old) p_old.
__device__ __forceinline__ void fcg_beta_p_range(int N, const float* __restrict__ z, float* __restrict__ p,
                                                 const double* __restrict__ scal, int first, int blk, int nblk) {
    float beta = 0.f;
    if (!first) {
        const double pq = scal[0];
        beta = pq > 0.0 ? (float)(-scal[3] / pq) : 0.f;
    }
    const int stride = nblk * NT;
#pragma unroll 4
    for (int idx = blk * NT + threadIdx.x; idx < N; idx += stride) p[idx] = first ? z[idx] : fmaf(beta, p[idx], z[idx]);
}

// alpha = p.r / p.q (scal 2, 0); e += alpha p; r -= alpha q; returns r.r of this thread
__device__ __forceinline__ FF fcg_update_range(int N, float* __restrict__ e, float* __restrict__ r,
                                               const float* __restrict__ p, const float* __restrict__ q,
                                               const double* scal, bool& bad, int blk, int nblk) {
    const double pq = scal[0], pr = scal[2];
    bad = !(pq > 0.0) || !isfinite(pq) || !isfinite(pr);
    const float alpha = bad ? 0.f : (float)(pr / pq);
    FF rr{0.f, 0.f};
    const int stride = nblk * NT;
#pragma unroll 4
    for (int idx = blk * NT + threadIdx.x; idx < N; idx += stride) {
        const float pi = p[idx];
        e[idx] = fmaf(alpha, pi, e[idx]);
        const float ri = fmaf(-alpha, q[idx], r[idx]);
        r[idx] = ri;
        ff_add_prod(rr, ri, ri);
    }
    return rr;
}

// Cell of a 2D/3D-mapped launch: block (32, 8); 3D grid (nx/32, ny/8, nz),
// 2D grid (nx/32, nz/8, 1).
__device__ __forceinline__ bool map_cell(const Geo& g, int bx, int by, int bz, int& i, int& j, int& k) {
    i = bx * 32 + threadIdx.x;
    if (g.ny > 1) {
        j = by * 8 + threadIdx.y;
        k = bz;
    } else {
        j = 0;
        k = by * 8 + threadIdx.y;
    }
    return i < g.nx && j < g.ny && k < g.nz;
}

// Coarse c~ and rho of the coarse cell a thread of block (bx, by, bz) of a
// (32, 8) block maps to (map_cell): the means over its children.
__device__ __forceinline__ void coarsen_cell(const Lev32& F, const Geo& C, int hx, int hy, int hz,
                                             float* __restrict__ ct_c, float* __restrict__ rho_c, int bx, int by,
                                             int bz) {
    int I, J, K;
    if (!map_cell(C, bx, by, bz, I, J, K)) return;
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

__device__ __forceinline__ float apply32_at(int idx, int i, int j, int k, const Lev32& L,
                                            const float* __restrict__ x) {
    const Geo& g = L.g;
    const float xc = x[idx], rc = L.rho[idx];
    float y = L.ct[idx] * xc;
    Nbr n = nbr_x(idx, i, g);
    if (face_minus(i, g.nx, g.bcx)) y += face32(rc, L.rho[n.im], L.c2x) * (xc - x[n.im]);
    if (face_plus(i, g.nx, g.bcx)) y += face32(rc, L.rho[n.ip], L.c2x) * (xc - x[n.ip]);
    if (g.ny > 1) {
        n = nbr_y(idx, j, g);
        if (face_minus(j, g.ny, g.bcy)) y += face32(rc, L.rho[n.im], L.c2y) * (xc - x[n.im]);
        if (face_plus(j, g.ny, g.bcy)) y += face32(rc, L.rho[n.ip], L.c2y) * (xc - x[n.ip]);
    }
    n = nbr_z(idx, k, g);
    if (face_minus(k, g.nz, g.bcz)) y += face32(rc, L.rho[n.im], L.c2z) * (xc - x[n.im]);
    if (face_plus(k, g.nz, g.bcz)) y += face32(rc, L.rho[n.ip], L.c2z) * (xc - x[n.ip]);
    return y;
}

// fc = mean over the children of (f - A x): residual and restriction fused;
// one thread per coarse cell of the mapped block (bx, by, bz).
__device__ __forceinline__ void resid_restrict_tile(const Lev32& F, const Geo& C, int hx, int hy, int hz,
                                                    const float* __restrict__ x, const float* __restrict__ f,
                                                    float* __restrict__ fc, int bx, int by, int bz) {
    int I, J, K;
    if (!map_cell(C, bx, by, bz, I, J, K)) return;
    float s = 0.f;
    for (int c = 0; c <= hz; ++c)
        for (int b = 0; b <= hy; ++b)
            for (int a = 0; a <= hx; ++a) {
                const int i = (I << hx) + a, j = (J << hy) + b, k = (K << hz) + c;
                const int idx = i + F.g.nx * (j + F.g.ny * k);
                s += f[idx] - apply32_at(idx, i, j, k, F, x);
            }
    fc[I + C.nx * (J + C.ny * K)] = s * (1.f / (float)((1 << hx) << hy << hz));
}

// ---- fused red-black Gauss-Seidel sweep ------------------------------------
//
// xout = one red-black Gauss-Seidel sweep applied to xold, the FIRST colour
// ((i + j + k) mod 2 == FIRST) updated first, then the other colour.  The
// sweep is out of place (xold is read-only), so a block can recompute the
// first-colour values it needs on a one-cell halo around its tile from xold
// exactly as the neighbouring block computes them: every block sees the same
// values, the result equals the in-place sequential sweep, and the whole
// sweep is a single pass over memory.
//
// A block owns a tile of 2*BX x TY cells and marches along z.  Each thread
// owns an x-pair of cells, which always holds one cell of each colour, so
// no lane idles on a colour test; the cell that is first-coloured on plane p
// is second-coloured on plane p - 1, so each thread updates one of its cells
// per plane and phase.  Shared memory holds rings of planes of xold and rho
// on the tile + 2-cell halo and of the new first-colour values on the tile +
// 1-cell halo; f and c~ of a thread's own cells stay in registers.  A few
// threads also compute the first colour on the halo ring.  Loads for the
// next plane are issued before the current plane's arithmetic.
// ZERO:    xold = 0 (first sweep of a V-cycle level: zero initial guess).
// PROLONG: xold = xin + P ec (piecewise-constant prolongation of the coarse
//          correction, fused into the post-smoothing sweep).
template <int BX, int TY, bool HAS_Y, int FIRST, bool ZERO, bool PROLONG>
__device__ __forceinline__ void rbgs_tile(const Lev32& L, const float* __restrict__ xin,
                                          const float* __restrict__ ec, const Geo& C, int hx, int hy, int hz,
                                          const float* __restrict__ f, float* __restrict__ xout, int KZ, int bx,
                                          int by, int bz) {
    constexpr int TXC = 2 * BX;
    constexpr int HY = HAS_Y ? 1 : 0;
    constexpr int EX2 = TXC + 4, EY2 = TY + 4 * HY;    // tile + 2-cell halo (R2)
    constexpr int EX1 = TXC + 2, EY1 = TY + 2 * HY;    // tile + 1-cell halo (R1)
    constexpr int NTH = BX * TY;
    constexpr int N2 = (EX2 * EY2 + NTH - 1) / NTH;
    constexpr int NHP = HAS_Y ? EX1 : 0;               // halo pairs: EX1/2 on the top and on the bottom R1 row
    constexpr int NH = NHP + 2 * TY;                   // + single cells of the left and right R1 columns
    static_assert(NH <= NTH, "halo tasks exceed the block");
    __shared__ float XO[3][EY2 * EX2];
    __shared__ float RH[5][EY2 * EX2];
    __shared__ float F1[3][EY1 * EX1];
    __syncthreads();               // shared tiles may be reused by the next task of a block
    const Geo& g = L.g;
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int i0 = bx * TXC;
    const int j0 = HAS_Y ? by * TY : 0;
    const int k0 = (HAS_Y ? bz : by) * KZ;
    const int k1 = min(k0 + KZ, g.nz);
    const int sz = g.nx * g.ny;

    // coordinates reach at most 2 cells past either end: wrap by adding or
    // subtracting n (twice for n = 1), no division
    auto wrap = [](int c, int n, int bc, bool& ok) -> int {
        ok = (c >= 0 && c < n) || bc == LM_BC_PERIODIC;
        while (c < 0) c += n;
        while (c >= n) c -= n;
        return c;
    };
    auto ring = [](int p, int m) { return (p + 6) % m; };   // plane p >= -4 -> slot
    auto flags = [&](int gi, int gj) {
        return (face_minus(gi, g.nx, g.bcx) ? 1 : 0) | (face_plus(gi, g.nx, g.bcx) ? 2 : 0) |
               (HAS_Y && face_minus(gj, g.ny, g.bcy) ? 4 : 0) | (HAS_Y && face_plus(gj, g.ny, g.bcy) ? 8 : 0);
    };

    // staged R2 elements of this thread: in-plane offset (-1: outside a wall), parent offset
    int off2[N2], poff2[N2];
#pragma unroll
    for (int u = 0; u < N2; ++u) {
        const int e = tid + u * NTH;
        off2[u] = -1;
        poff2[u] = 0;
        if (e < EX2 * EY2) {
            bool oki, okj = true;
            const int gi = wrap(i0 - 2 + e % EX2, g.nx, g.bcx, oki);
            const int gj = HAS_Y ? wrap(j0 - 2 + e / EX2, g.ny, g.bcy, okj) : 0;
            if (oki && okj) {
                off2[u] = gi + g.nx * gj;
                poff2[u] = (gi >> hx) + C.nx * (gj >> hy);
            }
        }
    }
    // Update cells: c = 0, 1 the thread's own x-pair (a tile wider than a
    // small grid holds wrapped copies of periodic cells: computed, not
    // written); c = 2, 3 its halo task (a pair of the top/bottom R1 row or one
    // cell of the left/right R1 column), spread round-robin over the warps.
    // Per cell: R1 index, R2 index, in-plane offset (-1: outside a wall),
    // parity, face flags.
    int i1c[4], i2c[4], offc[4], parc[4], flc[4];
    bool outc[2];
    {
        const int ti = threadIdx.x, tj = HAS_Y ? threadIdx.y : 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            bool oki, okj = true;
            const int ui = i0 + 2 * ti + c, uj = j0 + tj;
            const int gi = wrap(ui, g.nx, g.bcx, oki);
            const int gj = HAS_Y ? wrap(uj, g.ny, g.bcy, okj) : 0;
            const int ex1 = 2 * ti + 1 + c, ey1 = tj + HY;
            i1c[c] = ey1 * EX1 + ex1;
            i2c[c] = (ey1 + HY) * EX2 + ex1 + 1;
            const bool ok = oki && okj;
            offc[c] = ok ? gi + g.nx * gj : -1;
            parc[c] = (gi + gj) & 1;
            flc[c] = ok ? flags(gi, gj) : 0;
            outc[c] = ok && ui < g.nx && uj < g.ny;
        }
        // task number: warps take turns, so every warp carries a share
        const int lane = tid & 31, warp = tid >> 5, nwarp = NTH / 32;
        const int t = lane * nwarp + warp;
        int hxp[2] = {0, 0}, hyp = 0, nh = 0;
        if (t < NHP) {
            const int m = t % (EX1 / 2);
            hyp = t < EX1 / 2 ? 0 : EY1 - 1;
            hxp[0] = 2 * m;
            hxp[1] = 2 * m + 1;
            nh = 2;
        } else if (t < NH) {
            const int sidx = t - NHP;
            hxp[0] = sidx < TY ? 0 : EX1 - 1;
            hyp = (sidx % TY) + HY;
            nh = 1;
        }
#pragma unroll
        for (int c = 2; c < 4; ++c) {
            const int ex1 = hxp[c - 2];
            i1c[c] = hyp * EX1 + ex1;
            i2c[c] = (hyp + HY) * EX2 + ex1 + 1;
            offc[c] = -1;
            parc[c] = 0;
            flc[c] = 0;
            if (c - 2 < nh) {
                bool oki, okj = true;
                const int gi = wrap(i0 - 1 + ex1, g.nx, g.bcx, oki);
                const int gj = HAS_Y ? wrap(j0 - 1 + hyp, g.ny, g.bcy, okj) : 0;
                if (oki && okj) {
                    offc[c] = gi + g.nx * gj;
                    parc[c] = (gi + gj) & 1;
                    flc[c] = flags(gi, gj);
                }
            }
        }
    }

    // Gauss-Seidel value x = (f + sum g v) / (c~ + sum g) of an update cell;
    // neighbour values v from the plane rows Vm/V0/Vp (row width exv) at vi,
    // rho from the R2 planes Rm/R0/Rp at ri.  Face weights first, then the
    // sums, so the reciprocals of the six faces are independent.
    auto gs = [&](int fl, bool zm, bool zp, float fv, float cv, const float* Vm, const float* V0, const float* Vp,
                  int exv, int vi, const float* Rm, const float* R0, const float* Rp, int ri) -> float {
        const float rc = R0[ri];
        const float wxm = (fl & 1) ? face32(rc, R0[ri - 1], L.c2x) : 0.f;
        const float wxp = (fl & 2) ? face32(rc, R0[ri + 1], L.c2x) : 0.f;
        const float wym = (HAS_Y && (fl & 4)) ? face32(rc, R0[ri - EX2], L.c2y) : 0.f;
        const float wyp = (HAS_Y && (fl & 8)) ? face32(rc, R0[ri + EX2], L.c2y) : 0.f;
        const float wzm = zm ? face32(rc, Rm[ri], L.c2z) : 0.f;
        const float wzp = zp ? face32(rc, Rp[ri], L.c2z) : 0.f;
        const float d = cv + ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
        float num = fv;
        num = fmaf(wxm, V0[vi - 1], num);
        num = fmaf(wxp, V0[vi + 1], num);
        if (HAS_Y) {
            num = fmaf(wym, V0[vi - exv], num);
            num = fmaf(wyp, V0[vi + exv], num);
        }
        num = fmaf(wzm, Vm[vi], num);
        num = fmaf(wzp, Vp[vi], num);
        return __fdividef(num, d);
    };

    // register staging: x, rho of plane p + 1 on R2 and f, c~ of the update
    // cells on plane p (own pair; halo task: the cell first-coloured on p)
    float px[N2], pr[N2], pf[3], pc[3];
    auto fetch = [&](int p) {
        bool okp, okq;
        const int gp = wrap(p + 1, g.nz, g.bcz, okp);
        const int gq = wrap(p, g.nz, g.bcz, okq);
#pragma unroll
        for (int u = 0; u < N2; ++u) {
            float xv = 0.f, rv = 1.f;
            if (okp && off2[u] >= 0) {
                const int idx = off2[u] + sz * gp;
                rv = L.rho[idx];
                if (!ZERO) {
                    xv = xin[idx];
                    if (PROLONG) xv += ec[poff2[u] + C.nx * C.ny * (gp >> hz)];
                }
            }
            px[u] = xv;
            pr[u] = rv;
        }
        // colour parity from the unwrapped plane index (a wrapped periodic
        // axis has an even count; a plane past a Neumann wall computes nothing)
        const int hsel = ((parc[2] + p) & 1) == FIRST ? 2 : 3;
        const int hoff = hsel == 2 ? offc[2] : offc[3];
        const int offs[3] = {offc[0], offc[1], hoff};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float fv = 0.f, cv = 1.f;
            if (okq && offs[c] >= 0) {
                const int idx = offs[c] + sz * gq;
                fv = f[idx];
                cv = L.ct[idx];
            }
            pf[c] = fv;
            pc[c] = cv;
        }
    };
    auto store_xr = [&](int sx, int sr) {
        float* xo = XO[sx];
        float* rh = RH[sr];
#pragma unroll
        for (int u = 0; u < N2; ++u) {
            const int e = tid + u * NTH;
            if (e < EX2 * EY2) {
                xo[e] = px[u];
                rh[e] = pr[u];
            }
        }
    };

    // gs() reads neighbour values even where a face weight is 0 (a wall):
    // first-colour slots that are never written must hold finite values
    for (int e = tid; e < 3 * EY1 * EX1; e += NTH) (&F1[0][0])[e] = 0.f;
    float fcur[3], ccur[3], fprev[2], cprev[2];
    fetch(k0 - 3);
    store_xr(ring(k0 - 2, 3), ring(k0 - 2, 5));
    fetch(k0 - 2);
    store_xr(ring(k0 - 1, 3), ring(k0 - 1, 5));
    fetch(k0 - 1);                 // x, rho of plane k0; f, c~ of plane k0 - 1
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        fcur[c] = 0.f;
        ccur[c] = 1.f;
    }
    // slots for p = k0 - 1: XO/F1 of planes p-2 .. p+1 (3-ring: p-2 and p+1
    // share a slot), RH of planes p-3 .. p+1
    int x2 = ring(k0 - 3, 3), x1 = ring(k0 - 2, 3), x0 = ring(k0 - 1, 3), xp = ring(k0, 3);
    int r3 = ring(k0 - 4, 5), r2 = ring(k0 - 3, 5), r1 = ring(k0 - 2, 5), r0 = ring(k0 - 1, 5),
        rp = ring(k0, 5);
    bool okp;
    int gp = wrap(k0 - 1, g.nz, g.bcz, okp);
    for (int p = k0 - 1; p <= k1; ++p) {
        store_xr(xp, rp);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            fprev[c] = fcur[c];
            cprev[c] = ccur[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fcur[c] = pf[c];
            ccur[c] = pc[c];
        }
        if (p < k1) fetch(p + 1);
        __syncthreads();
        // first colour on plane p: own cell A (first-coloured on p) and the halo task's cell
        const int a = ((parc[0] + p) & 1) == FIRST ? 0 : 1;
        const int i1a = a ? i1c[1] : i1c[0], i2a = a ? i2c[1] : i2c[0];
        const int fla = a ? flc[1] : flc[0];
        const int ha = ((parc[2] + p) & 1) == FIRST ? 2 : 3;
        const int i1h = ha == 2 ? i1c[2] : i1c[3], i2h = ha == 2 ? i2c[2] : i2c[3];
        const int flh = ha == 2 ? flc[2] : flc[3];
        const bool hval = (ha == 2 ? offc[2] : offc[3]) >= 0 && (((ha == 2 ? parc[2] : parc[3]) + p) & 1) == FIRST;
        {
            const float* Xm = XO[x1];
            const float* X0 = XO[x0];
            const float* Xp = XO[xp];
            const float* Rm = RH[r1];
            const float* R0 = RH[r0];
            const float* Rp = RH[rp];
            float* f1 = F1[x0];
            const bool zm = face_minus(gp, g.nz, g.bcz), zp = face_plus(gp, g.nz, g.bcz);
            const float va = gs(fla, zm, zp, a ? fcur[1] : fcur[0], a ? ccur[1] : ccur[0], Xm, X0, Xp, EX2, i2a,
                                Rm, R0, Rp, i2a);
            const float vh = gs(flh, zm, zp, fcur[2], ccur[2], Xm, X0, Xp, EX2, i2h, Rm, R0, Rp, i2h);
            if ((a ? offc[1] : offc[0]) >= 0) f1[i1a] = okp ? va : 0.f;
            if (hval) f1[i1h] = okp ? vh : 0.f;
        }
        __syncthreads();
        // second colour on plane q = p - 1: own cell A (second-coloured on q);
        // own cell B is first-coloured on q and was computed last plane
        const int q = p - 1;
        if (q >= k0) {
            const float* Fm = F1[x2];
            const float* F0 = F1[x1];
            const float* Fp = F1[x0];
            const bool zm = face_minus(q, g.nz, g.bcz), zp = face_plus(q, g.nz, g.bcz);
            const int b = 1 - a;
            const int i1b = b ? i1c[1] : i1c[0];
            const float va = gs(fla, zm, zp, a ? fprev[1] : fprev[0], a ? cprev[1] : cprev[0], Fm, F0, Fp, EX1, i1a,
                                RH[r2], RH[r1], RH[r0], i2a);
            const float vb = F0[i1b];
            if (outc[0]) xout[offc[0] + sz * q] = a ? vb : va;
            if (outc[1]) xout[offc[1] + sz * q] = a ? va : vb;
        }
        // rotate to plane p + 1 (in the 3-ring, p + 2 takes the slot of p - 1)
        x2 = x1;
        x1 = x0;
        x0 = xp;
        xp = x2;
        {
            const int t5 = r3;
            r3 = r2;
            r2 = r1;
            r1 = r0;
            r0 = rp;
            rp = t5;
        }
        ++gp;
        if (gp == g.nz) gp = 0;
        okp = (p + 1 >= 0 && p + 1 < g.nz) || g.bcz == LM_BC_PERIODIC;
    }
}

__device__ __forceinline__ void coarse_solve_block(int n, const float* __restrict__ ainv, const float* __restrict__ f,
                                                   float* __restrict__ x) {
    const int i = threadIdx.x;
    if (i >= n || threadIdx.y > 0) return;
    float s = 0.f;
    for (int j = 0; j < n; ++j) s = fmaf(ainv[i * n + j], f[j], s);
    x[i] = s;
}

// ---- 2D red-black sweep on whole 256-cell rows: in-place z-march -----------
//
// The 2D counterpart of the 3D z-march sweep, for levels (ny = 1) whose nx is
// a multiple of 256, on blocks of 128 threads: the block owns 256 columns
// over a chunk of KZ rows and marches up z with a five-row ring of (x, rho)
// staged on the row plus two cells (periodic x wrapped; past a wall x = 0
// and rho = +inf, so that face's weight is 0).  At step p it stores row
// p + 1 and issues the loads of row p + 2, updates the FIRST colour of row p
// on the tile plus one cell each side in place (a first-colour update reads
// only second-colour neighbours), the second colour of row p - 1, and
// writes row p - 2.  Used by the single-grid sweep and the batched solver
// (the same 256-wide tiles and row chunks as rbgs_tile).
__device__ __forceinline__ float rcp_hw(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int FIRST, bool ZERO, bool PROLONG>
__device__ __forceinline__ void zm2d_tile(const Lev32& L, const float* __restrict__ xin,
                                          const float* __restrict__ ec, const Geo& C, int hx, int hz,
                                          const float* __restrict__ f, float* __restrict__ xout, int KZ, int bx,
                                          int bz) {
    constexpr int NT2 = 128, TX = 256, SX = TX + 4, NR = 5;
    constexpr int NA = (TX + 2) / 2, NB = TX / 2;
    constexpr int QS = (SX + NT2 - 1) / NT2, QA = (NA + NT2 - 1) / NT2, QW = TX / NT2;
    __shared__ float2 XR[NR * SX];
    __shared__ int ox[SX], px[SX];
    __syncthreads();                                     // shared tiles may be reused by the next task
    const Geo& g = L.g;
    const int tid = threadIdx.x;
    const int i0 = bx * TX;
    const int k0 = bz * KZ, k1 = min(k0 + KZ, g.nz);
    for (int t = tid; t < SX; t += NT2) {
        int c = i0 - 2 + t;
        if (c < 0) c = g.bcx == LM_BC_PERIODIC ? c + g.nx : -1;
        else if (c >= g.nx) c = g.bcx == LM_BC_PERIODIC ? c - g.nx : -1;
        ox[t] = c;
        px[t] = c >> hx;
    }
    __syncthreads();
    auto zwrap = [&](int p) -> int { return ((p % g.nz) + g.nz) % g.nz; };
    auto zoff = [&](int p) -> int {
        if (p >= 0 && p < g.nz) return g.nx * p;
        return g.bcz == LM_BC_PERIODIC ? g.nx * zwrap(p) : -1;
    };
    auto zpar = [&](int p) -> int { return C.nx * (zwrap(p) >> hz); };
    int spos[QS], sbase[QS], spar[QS];
    bool sok[QS];
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        spos[q] = tid + q * NT2;
        const bool use = spos[q] < SX;
        sok[q] = use && ox[use ? spos[q] : 0] >= 0;
        sbase[q] = use ? ox[spos[q]] : 0;
        spar[q] = use ? px[spos[q]] : 0;
        if (!use) spos[q] = -1;
    }
    float vx[QS], vr[QS], ve[QS];
    auto fetch = [&](int zo, int zp) {
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            vx[q] = 0.f;
            ve[q] = 0.f;
            vr[q] = __int_as_float(0x7f800000);          // +inf
            if (sok[q] && zo >= 0) {
                const int idx = sbase[q] + zo;
                vr[q] = L.rho[idx];
                if (!ZERO) {
                    vx[q] = xin[idx];
                    if (PROLONG) ve[q] = ec[spar[q] + zp];
                }
            }
        }
    };
    auto store = [&](int o) {
#pragma unroll
        for (int q = 0; q < QS; ++q)
            if (spos[q] >= 0) XR[o + spos[q]] = make_float2(PROLONG ? vx[q] + ve[q] : vx[q], vr[q]);
    };
    auto gs = [&](int e, int sm, int s0, int sp, float fv, float cv) -> float {
        const int c = s0 + e;
        const float rc = XR[c].y;
        const float2 nxm = XR[c - 1], nxp = XR[c + 1], nzm = XR[sm + e], nzp = XR[sp + e];
        const float wxm = L.c2x * rcp_hw(rc + nxm.y);
        const float wxp = L.c2x * rcp_hw(rc + nxp.y);
        const float wzm = L.c2z * rcp_hw(rc + nzm.y);
        const float wzp = L.c2z * rcp_hw(rc + nzp.y);
        const float d = cv + (wxm + wxp) + (wzm + wzp);
        float num = fv;
        num = fmaf(wxm, nxm.x, num);
        num = fmaf(wxp, nxp.x, num);
        num = fmaf(wzm, nzm.x, num);
        num = fmaf(wzp, nzp.x, num);
        return num * rcp_hw(d);
    };
    // first-colour tasks: pair am of the halo row (x positions 2am and 2am + 1
    // of the staged row shifted by one); second-colour task: pair bm of the tile
    bool hasA[QA];
    int aeE[QA], aoE[QA], aoO[QA];
#pragma unroll
    for (int u = 0; u < QA; ++u) {
        const int am = tid + u * NT2;
        hasA[u] = am < NA;
        aeE[u] = 2 * (hasA[u] ? am : 0) + 1;
        aoE[u] = ox[aeE[u]];
        aoO[u] = ox[aeE[u] + 1];
    }
    const int apar = (FIRST + i0) & 1;
    const int bpar = (1 - FIRST + i0) & 1;
    const int beE = 2 * tid + 2;
    const int bidxE = i0 + 2 * tid;
    int wpos[QW], wbase[QW];
#pragma unroll
    for (int v = 0; v < QW; ++v) {
        wpos[v] = tid + v * NT2 + 2;
        wbase[v] = i0 + tid + v * NT2;
    }
    int om2 = 0 * SX, om1 = 1 * SX, o0 = 2 * SX, op1 = 3 * SX, op2 = 4 * SX;
    int z0 = zoff(k0 - 1), z1 = zoff(k0), z2 = zoff(k0 + 1);
    int zp2 = PROLONG ? zpar(k0 + 1) : 0;
    fetch(zoff(k0 - 2), PROLONG ? zpar(k0 - 2) : 0);
    store(om1);
    fetch(z0, PROLONG ? zpar(k0 - 1) : 0);
    store(o0);
    fetch(z1, PROLONG ? zpar(k0) : 0);
    float fa[QA], ca[QA];
    bool okA[QA];
    int eA[QA];
    auto load_a = [&](int p, int zo, bool in_chunk) {
#pragma unroll
        for (int u = 0; u < QA; ++u) {
            // staged position aeE + odd is global x = i0 - 1 + 2 am + odd, of
            // colour (x + p) & 1 = FIRST when odd = (FIRST + i0 + p + 1) & 1
            const int odd = (apar + p + 1) & 1;
            const int a = odd ? aoO[u] : aoE[u];
            okA[u] = hasA[u] && in_chunk && (a | zo) >= 0;
            eA[u] = aeE[u] + odd;
            fa[u] = 0.f;
            ca[u] = 1.f;
            if (okA[u]) {
                fa[u] = f[a + zo];
                ca[u] = L.ct[a + zo];
            }
        }
    };
    // L2 prefetch of the tile's row segments (256 cells, contiguous) PF_PLANES
    // steps ahead: x and rho of row P are fetched at step P - 2, f and c~ of
    // row P first read at step P - 1; array a = 0..3 by thread a
    auto prefetch = [&](int a, int P) {
        if (P > (a < 2 ? k1 + 1 : k1) || (ZERO && a == 0)) return;
        const int zo = zoff(P);
        if (zo < 0) return;
        const float* base = a == 0 ? xin : a == 1 ? L.rho : a == 2 ? f : L.ct;
        prefetch_l2(base + zo + i0, TX * sizeof(float));
    };
    if (tid < 4)
        for (int d = 1; d <= PF_PLANES; ++d) prefetch(tid, (tid < 2 ? k0 : k0 - 1) + d);
    load_a(k0 - 1, z0, true);
    float fb = 0.f, cb = 1.f;
    bool okB = false;
    int eB = 0;
    for (int p = k0 - 1; p <= k1 + 1; ++p) {
        if (tid < 4) prefetch(tid, (tid < 2 ? p + 2 : p + 1) + PF_PLANES);
        if (p <= k1) store(op1);
        if (p + 1 <= k1) fetch(z2, zp2);
        float fA[QA], cA[QA];
        bool doA[QA];
        int eAc[QA];
#pragma unroll
        for (int u = 0; u < QA; ++u) {
            fA[u] = fa[u];
            cA[u] = ca[u];
            doA[u] = okA[u] && p <= k1;
            eAc[u] = eA[u];
        }
        const float fB = fb, cB = cb;
        const bool doB = okB;
        const int eBc = eB;
        {
            const int odd = (bpar + p) & 1;
            okB = p >= k0 && p < k1;
            eB = beE + odd;
            if (okB) {
                const int idx = bidxE + odd + g.nx * p;
                fb = f[idx];
                cb = L.ct[idx];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < QA; ++u)
            if (doA[u]) XR[o0 + eAc[u]].x = gs(eAc[u], om1, o0, op1, fA[u], cA[u]);
        load_a(p + 1, z1, p + 1 <= k1);
        __syncthreads();
        if (doB) XR[om1 + eBc].x = gs(eBc, om2, om1, o0, fB, cB);
        if (p - 2 >= k0) {
#pragma unroll
            for (int v = 0; v < QW; ++v) xout[wbase[v] + g.nx * (p - 2)] = XR[om2 + wpos[v]].x;
        }
        const int t = om2;
        om2 = om1;
        om1 = o0;
        o0 = op1;
        op1 = op2;
        op2 = t;
        z0 = z1;
        z1 = z2;
        {
            int c = p + 3;
            if (c >= g.nz) c -= g.nz;
            if (c >= g.nz) c -= g.nz;
            const bool ok = (p + 3 < g.nz || g.bcz == LM_BC_PERIODIC) && c >= 0 && c < g.nz;
            z2 = ok ? g.nx * c : -1;
            if (PROLONG) zp2 = C.nx * ((ok ? c : 0) >> hz);
        }
    }
}

// ---- the coarse V-cycle in one block (see k_coarse_cycle) ------------------
//
// The block keeps the whole chain in shared memory: per level x, f, the three
// minus-face conductances (plus faces are the neighbours' minus faces), c~ and
// the inverse diagonal, seven floats per cell (cc_smem_bytes), and the dense
// inverse of the coarsest level.  Face weights and diagonals are formed once
// per cycle; every later phase reads shared memory only.  Each thread owns
// cells tid + CC_THREADS q of a level and keeps their (i, j, k) in registers.

__device__ __forceinline__ void coarse_cycle_block(const CoarseCycle& cc) {
    extern __shared__ float cc_sm[];
    const int tid = threadIdx.x;
    const int nl = cc.nl;
    struct CS {
        float *x, *f, *wx, *wy, *wz, *ct, *di;
    };
    auto cs = [&](int l) -> CS {                        // level l's arrays, laid out level after level
        float* b = cc_sm;
        for (int m = 0; m < l; ++m) b += 7 * cc.L[m].g.N;
        const int N = cc.L[l].g.N;
        return CS{b, b + N, b + 2 * N, b + 3 * N, b + 4 * N, b + 5 * N, b + 6 * N};
    };
    // setup: x = 0, f (level 0: the caller's rhs), c~ and minus-face weights
    for (int l = 0; l < nl; ++l) {
        const Lev32& L = cc.L[l];
        const Geo& g = L.g;
        const CS s = cs(l);
        for (int idx = tid; idx < g.N; idx += CC_THREADS) {
            int i, j, k;
            cell_coords(idx, g, i, j, k);
            const float rc = L.rho[idx];
            s.wx[idx] = face_minus(i, g.nx, g.bcx) ? face32(rc, L.rho[nbr_x(idx, i, g).im], L.c2x) : 0.f;
            s.wy[idx] = face_minus(j, g.ny, g.bcy) ? face32(rc, L.rho[nbr_y(idx, j, g).im], L.c2y) : 0.f;
            s.wz[idx] = face_minus(k, g.nz, g.bcz) ? face32(rc, L.rho[nbr_z(idx, k, g).im], L.c2z) : 0.f;
            s.ct[idx] = L.ct[idx];
            s.f[idx] = l == 0 ? cc.f[0][idx] : 0.f;
            s.x[idx] = 0.f;
        }
    }
    const int nc = cc.L[nl - 1].g.N;
    float* const Ai = cs(nl - 1).x + 7 * nc;            // after the last level's arrays
    for (int e = tid; e < nc * nc; e += CC_THREADS) Ai[e] = cc.ainv[e];
    __syncthreads();
    // plus-face weight of cell idx along an axis: the minus face of its plus
    // neighbour, 0 past a wall
    auto wplus = [&](const float* w, bool has, int ip) -> float { return has ? w[ip] : 0.f; };
    for (int l = 0; l < nl; ++l) {
        const Geo& g = cc.L[l].g;
        const CS s = cs(l);
        for (int idx = tid; idx < g.N; idx += CC_THREADS) {
            int i, j, k;
            cell_coords(idx, g, i, j, k);
            const float d = s.ct[idx] + ((s.wx[idx] + wplus(s.wx, face_plus(i, g.nx, g.bcx), nbr_x(idx, i, g).ip)) +
                                         (s.wy[idx] + wplus(s.wy, face_plus(j, g.ny, g.bcy), nbr_y(idx, j, g).ip))) +
                            (s.wz[idx] + wplus(s.wz, face_plus(k, g.nz, g.bcz), nbr_z(idx, k, g).ip));
            s.di[idx] = 1.f / d;
        }
    }
    __syncthreads();

    int ci[CC_PER], cj[CC_PER], ck[CC_PER];
    auto coords = [&](int l) {
        const Geo& g = cc.L[l].g;
#pragma unroll
        for (int q = 0; q < CC_PER; ++q) {
            const int idx = tid + q * CC_THREADS;
            ci[q] = cj[q] = ck[q] = 0;
            if (idx < g.N) cell_coords(idx, g, ci[q], cj[q], ck[q]);
        }
    };
    // (A x) at cell idx of a level from its shared arrays
    auto apply_at = [&](const Geo& g, const CS& s, int idx, int i, int j, int k) -> float {
        const float xc = s.x[idx];
        float y = s.ct[idx] * xc;
        Nbr n = nbr_x(idx, i, g);
        if (face_minus(i, g.nx, g.bcx)) y += s.wx[idx] * (xc - s.x[n.im]);
        if (face_plus(i, g.nx, g.bcx)) y += s.wx[n.ip] * (xc - s.x[n.ip]);
        n = nbr_y(idx, j, g);
        if (face_minus(j, g.ny, g.bcy)) y += s.wy[idx] * (xc - s.x[n.im]);
        if (face_plus(j, g.ny, g.bcy)) y += s.wy[n.ip] * (xc - s.x[n.ip]);
        n = nbr_z(idx, k, g);
        if (face_minus(k, g.nz, g.bcz)) y += s.wz[idx] * (xc - s.x[n.im]);
        if (face_plus(k, g.nz, g.bcz)) y += s.wz[n.ip] * (xc - s.x[n.ip]);
        return y;
    };
    // one colour of a red-black sweep on level l, in place
    auto colour = [&](int l, int col) {
        const Geo& g = cc.L[l].g;
        const CS s = cs(l);
#pragma unroll
        for (int q = 0; q < CC_PER; ++q) {
            const int idx = tid + q * CC_THREADS;
            const int i = ci[q], j = cj[q], k = ck[q];
            if (idx < g.N && ((i + j + k) & 1) == col) {
                float num = s.f[idx];
                Nbr n = nbr_x(idx, i, g);
                if (face_minus(i, g.nx, g.bcx)) num = fmaf(s.wx[idx], s.x[n.im], num);
                if (face_plus(i, g.nx, g.bcx)) num = fmaf(s.wx[n.ip], s.x[n.ip], num);
                n = nbr_y(idx, j, g);
                if (face_minus(j, g.ny, g.bcy)) num = fmaf(s.wy[idx], s.x[n.im], num);
                if (face_plus(j, g.ny, g.bcy)) num = fmaf(s.wy[n.ip], s.x[n.ip], num);
                n = nbr_z(idx, k, g);
                if (face_minus(k, g.nz, g.bcz)) num = fmaf(s.wz[idx], s.x[n.im], num);
                if (face_plus(k, g.nz, g.bcz)) num = fmaf(s.wz[n.ip], s.x[n.ip], num);
                s.x[idx] = num * s.di[idx];
            }
        }
        __syncthreads();
    };

    for (int l = 0; l + 1 < nl; ++l) {
        coords(l);
        for (int it = 0; it < cc.nu1; ++it) {
            colour(l, 0);
            colour(l, 1);
        }
        const Geo& F = cc.L[l].g;
        const Geo& C = cc.L[l + 1].g;
        const CS s = cs(l), c = cs(l + 1);
        const int hx = cc.hx[l], hy = cc.hy[l], hz = cc.hz[l];
        const float inv = 1.f / (float)((1 << hx) << hy << hz);
        for (int e = tid; e < C.N; e += CC_THREADS) {
            int I, J, K;
            cell_coords(e, C, I, J, K);
            float sum = 0.f;
            for (int cz = 0; cz <= hz; ++cz)
                for (int by = 0; by <= hy; ++by)
                    for (int ax = 0; ax <= hx; ++ax) {
                        const int i = (I << hx) + ax, j = (J << hy) + by, k = (K << hz) + cz;
                        const int idx = i + F.nx * (j + F.ny * k);
                        sum += s.f[idx] - apply_at(F, s, idx, i, j, k);
                    }
            c.f[e] = sum * inv;
        }
        __syncthreads();
    }
    {   // coarsest level: x = A^-1 f, 16 threads per row
        const CS s = cs(nl - 1);
        const int r = tid >> 4, part = tid & 15;
        float v = 0.f;
        if (r < nc)
            for (int c = part; c < nc; c += 16) v = fmaf(Ai[r * nc + c], s.f[c], v);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (r < nc && part == 0) s.x[r] = v;
        __syncthreads();
    }
    for (int l = nl - 2; l >= 0; --l) {
        coords(l);
        const Geo& g = cc.L[l].g;
        const Geo& C = cc.L[l + 1].g;
        const CS s = cs(l), c = cs(l + 1);
        const int hx = cc.hx[l], hy = cc.hy[l], hz = cc.hz[l];
#pragma unroll
        for (int q = 0; q < CC_PER; ++q) {
            const int idx = tid + q * CC_THREADS;
            if (idx < g.N) s.x[idx] += c.x[(ci[q] >> hx) + C.nx * ((cj[q] >> hy) + C.ny * (ck[q] >> hz))];
        }
        __syncthreads();
        for (int it = 0; it < cc.nu2; ++it) {
            colour(l, 1);
            colour(l, 0);
        }
    }
    {
        const CS s = cs(0);
        for (int idx = tid; idx < cc.L[0].g.N; idx += CC_THREADS) cc.x[0][idx] = s.x[idx];
    }
}

}  // namespace lm
