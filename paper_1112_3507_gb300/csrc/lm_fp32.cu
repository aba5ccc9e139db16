// Float32 kernels: the operator with faces formed on the fly from rho, the
// flexible-CG vector steps with float64-accurate dot products, and the
// geometric-multigrid V-cycle (coefficient coarsening, a fused red-black
// Gauss-Seidel sweep, fused residual + restriction, exact coarsest solve).
//
// These kernels are HBM-bound.  They stream each array once: face
// conductances are recomputed from rho instead of stored; cells are mapped
// to threads with 2D/3D launches (no integer division per cell); the
// stencils march along z keeping the z-neighbours in registers; and a whole
// red-black sweep is one pass over memory (see k_rbgs).
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace lm {

// g = (2/h^2) / (rho_a + rho_b); the sum is commutative, so both cells of a
// face compute the same bits and the operator stays exactly symmetric.
__device__ __forceinline__ float face32(float ra, float rb, float c2) { return __fdividef(c2, ra + rb); }

// ---- y = A x, marching along z --------------------------------------------
// 3D: block (32, 8) covers an x-y tile, blockIdx.z a chunk of kz planes.
// 2D (ny = 1): block (32, 8) covers 32 columns x 8 chunks of kz rows.
// kz is the smallest that keeps the launch within 4096 blocks (the
// last-block reduction sums one partial per block).

template <bool HAS_Y, bool DOT_XY, bool DOT_XR>
__global__ void __launch_bounds__(256) k_apply32z(Lev32 L, const float* __restrict__ x, float* __restrict__ y,
                                                  const float* __restrict__ r, Red red, int slot_xy, int slot_xr,
                                                  int KZ_APPLY) {
    __shared__ double sm[64];
    const Geo& g = L.g;
    const int i = blockIdx.x * 32 + threadIdx.x;
    int j, kb;
    if (HAS_Y) {
        j = blockIdx.y * 8 + threadIdx.y;
        kb = blockIdx.z * KZ_APPLY;
    } else {
        j = 0;
        kb = (blockIdx.y * 8 + threadIdx.y) * KZ_APPLY;
    }
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
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

// ---- flexible-CG vector steps (1D, grid-stride) ---------------------------
// scal slots: 0 p.q, 1 r.r, 2 p.r, 3 z.q_old, 4 r0.r0

// scal[slot] = a.b; if fnorm_st: also fnorm_st->fnorm = sqrt(a.b), rel = 1.
__global__ void __launch_bounds__(NT) k_dot32(int N, const float* __restrict__ a, const float* __restrict__ b,
                                              Red red, int slot, SolveState* fnorm_st) {
    __shared__ double sm[32];
    FF acc{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
#pragma unroll 4
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) ff_add_prod(acc, a[idx], b[idx]);
    double v[1] = {ff_value(acc)};
    const int sl[1] = {slot};
    if (grid_reduce<1>(v, red, sl, sm) && fnorm_st && lin_tid() == 0) {
        fnorm_st->fnorm = sqrt(red.scal[slot]);
        fnorm_st->rel = 1.0;
    }
}

// Flexible CG, truncation 1 (Notay 2000): p = z - (z.q_old / p_old.q_old) p_old.
__global__ void __launch_bounds__(NT) k_fcg_beta_p(int N, const float* __restrict__ z, float* __restrict__ p,
                                                   const double* __restrict__ scal, int first) {
    float beta = 0.f;
    if (!first) {
        const double pq = scal[0];
        beta = pq > 0.0 ? (float)(-scal[3] / pq) : 0.f;
    }
    const int stride = gridDim.x * blockDim.x;
#pragma unroll 4
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
        p[idx] = first ? z[idx] : fmaf(beta, p[idx], z[idx]);
}

// alpha = p.r / p.q; e += alpha p; r -= alpha q; scal[1] = r.r; the last
// block sets st->rel = ||r|| / st->fnorm (and the breakdown status).
__global__ void __launch_bounds__(NT) k_fcg_update(int N, float* __restrict__ e, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   Red red, SolveState* st) {
    __shared__ double sm[32];
    const double pq = red.scal[0], pr = red.scal[2];
    const bool bad = !(pq > 0.0) || !isfinite(pq) || !isfinite(pr);
    const float alpha = bad ? 0.f : (float)(pr / pq);
    FF rr{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
#pragma unroll 4
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
        const float pi = p[idx];
        e[idx] = fmaf(alpha, pi, e[idx]);
        const float ri = fmaf(-alpha, q[idx], r[idx]);
        r[idx] = ri;
        ff_add_prod(rr, ri, ri);
    }
    double v[1] = {ff_value(rr)};
    const int sl[1] = {1};
    if (grid_reduce<1>(v, red, sl, sm) && lin_tid() == 0) {
        if (bad) st->status = LM_ERR_BREAKDOWN;
        st->rel = sqrt(red.scal[1]) / st->fnorm;
    }
}

// ---- multigrid --------------------------------------------------------------

// Cell of a 2D/3D-mapped launch: block (32, 8); 3D grid (nx/32, ny/8, nz),
// 2D grid (nx/32, nz/8, 1).
__device__ __forceinline__ bool map_cell(const Geo& g, int& i, int& j, int& k) {
    i = blockIdx.x * 32 + threadIdx.x;
    if (g.ny > 1) {
        j = blockIdx.y * 8 + threadIdx.y;
        k = blockIdx.z;
    } else {
        j = 0;
        k = blockIdx.y * 8 + threadIdx.y;
    }
    return i < g.nx && j < g.ny && k < g.nz;
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

// Mean of the children's c~ and rho (coarse coefficients); one thread per coarse cell.
__global__ void __launch_bounds__(256) k_coarsen(Lev32 F, Geo C, int hx, int hy, int hz, float* __restrict__ ct_c,
                                                 float* __restrict__ rho_c) {
    int I, J, K;
    if (!map_cell(C, I, J, K)) return;
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

// fc = mean over the children of (f - A x): residual and restriction fused.
__global__ void __launch_bounds__(256) k_resid_restrict(Lev32 F, Geo C, int hx, int hy, int hz,
                                                        const float* __restrict__ x, const float* __restrict__ f,
                                                        float* __restrict__ fc) {
    int I, J, K;
    if (!map_cell(C, I, J, K)) return;
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
__global__ void __launch_bounds__(BX * TY, 1024 / (BX * TY)) k_rbgs(Lev32 L, const float* __restrict__ xin,
                                                                   const float* __restrict__ ec, Geo C, int hx,
                                                                   int hy, int hz, const float* __restrict__ f,
                                                                   float* __restrict__ xout, int KZ) {
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
    const Geo& g = L.g;
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int i0 = blockIdx.x * TXC;
    const int j0 = HAS_Y ? blockIdx.y * TY : 0;
    const int k0 = (HAS_Y ? blockIdx.z : blockIdx.y) * KZ;
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
    const int i = threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int j = 0; j < n; ++j) s = fmaf(ainv[i * n + j], f[j], s);
    x[i] = s;
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

// One red-black sweep xout = S(xin [+ P ec]); first = colour updated first.
void launch_rbgs(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx, int hy,
                 int hz, const float* f, float* xout, int first, int zero, int prolong) {
    const Geo& g = L.g;
    const Geo Cg = C ? C->g : g;
    count_launches(1);
    if (g.ny > 1) {
        constexpr int BX = 32, TY = 8;
        const int tiles = hdiv(g.nx, 2 * BX) * hdiv(g.ny, TY);
        int KZ = 16;
        while (KZ > 4 && (long long)tiles * hdiv(g.nz, KZ) < 1216) KZ /= 2;
        const dim3 grd(hdiv(g.nx, 2 * BX), hdiv(g.ny, TY), hdiv(g.nz, KZ)), blk(BX, TY);
#define LM_RB(F, Z, P) k_rbgs<BX, TY, true, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
        if (zero) { if (first) LM_RB(1, true, false); else LM_RB(0, true, false); }
        else if (prolong) { if (first) LM_RB(1, false, true); else LM_RB(0, false, true); }
        else { if (first) LM_RB(1, false, false); else LM_RB(0, false, false); }
#undef LM_RB
    } else {
        constexpr int BX = 128, TY = 1;
        const int tiles = hdiv(g.nx, 2 * BX);
        int KZ = 32;
        while (KZ > 4 && (long long)tiles * hdiv(g.nz, KZ) < 1216) KZ /= 2;
        const dim3 grd(hdiv(g.nx, 2 * BX), hdiv(g.nz, KZ), 1), blk(BX, TY);
#define LM_RB(F, Z, P) k_rbgs<BX, TY, false, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
        if (zero) { if (first) LM_RB(1, true, false); else LM_RB(0, true, false); }
        else if (prolong) { if (first) LM_RB(1, false, true); else LM_RB(0, false, true); }
        else { if (first) LM_RB(1, false, false); else LM_RB(0, false, false); }
#undef LM_RB
    }
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
