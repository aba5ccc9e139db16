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
__device__ __forceinline__ void assemble_range(const AsmArgs& a, int start, int stride, int end = -1) {
    const Geo& g = a.g;
    const double *a_in = a.a_in, *rho_new = a.rho_new, *cs2 = a.cs2;
    const double dt = a.dt, c2x = a.c2x, c2y = a.c2y, c2z = a.c2z;
    const int raw = a.raw;
    const Op64Out& out = a.out;
    AsmFlags* fl = a.fl;
    unsigned long long rmax = 0ull, rmin = ~0ull;        // range of the valid rho^{n+1}
    bool bad32 = false;
    const int stop = end < 0 ? g.N : end;
    for (int idx = start; idx < stop; idx += stride) {
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
//
// With N a multiple of 4 and 16-byte aligned vectors (every vector the
// library allocates; the test is uniform over a launch) a thread takes four
// consecutive elements per float4 access, otherwise one.

__device__ __forceinline__ bool vec4_ok(int N, const void* a, const void* b, const void* c = nullptr,
                                        const void* d = nullptr) {
    return (N & 3) == 0 && (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) & 15) == 0;
}
__device__ __forceinline__ float4 ld4v(const float* p, int i4) { return reinterpret_cast<const float4*>(p)[i4]; }
__device__ __forceinline__ void st4v(float* p, int i4, float4 v) { reinterpret_cast<float4*>(p)[i4] = v; }

__device__ __forceinline__ FF dot32_range(int N, const float* __restrict__ a, const float* __restrict__ b, int blk,
                                          int nblk) {
    FF acc{0.f, 0.f};
    const int stride = nblk * NT;
    if (vec4_ok(N, a, b)) {
#pragma unroll 2
        for (int i4 = blk * NT + threadIdx.x; i4 < (N >> 2); i4 += stride) {
            const float4 x = ld4v(a, i4), y = ld4v(b, i4);
            ff_add_prod(acc, x.x, y.x);
            ff_add_prod(acc, x.y, y.y);
            ff_add_prod(acc, x.z, y.z);
            ff_add_prod(acc, x.w, y.w);
        }
        return acc;
    }
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
    if (vec4_ok(N, z, p)) {
#pragma unroll 2
        for (int i4 = blk * NT + threadIdx.x; i4 < (N >> 2); i4 += stride) {
            const float4 zv = ld4v(z, i4);
            if (first) {
                st4v(p, i4, zv);
            } else {
                const float4 pv = ld4v(p, i4);
                st4v(p, i4, make_float4(fmaf(beta, pv.x, zv.x), fmaf(beta, pv.y, zv.y), fmaf(beta, pv.z, zv.z),
                                        fmaf(beta, pv.w, zv.w)));
            }
        }
        return;
    }
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
    if (vec4_ok(N, e, r, p, q)) {
#pragma unroll 2
        for (int i4 = blk * NT + threadIdx.x; i4 < (N >> 2); i4 += stride) {
            const float4 pv = ld4v(p, i4), qv = ld4v(q, i4), ev = ld4v(e, i4), rv = ld4v(r, i4);
            st4v(e, i4, make_float4(fmaf(alpha, pv.x, ev.x), fmaf(alpha, pv.y, ev.y), fmaf(alpha, pv.z, ev.z),
                                    fmaf(alpha, pv.w, ev.w)));
            const float4 rn = make_float4(fmaf(-alpha, qv.x, rv.x), fmaf(-alpha, qv.y, rv.y),
                                          fmaf(-alpha, qv.z, rv.z), fmaf(-alpha, qv.w, rv.w));
            st4v(r, i4, rn);
            ff_add_prod(rr, rn.x, rn.x);
            ff_add_prod(rr, rn.y, rn.y);
            ff_add_prod(rr, rn.z, rn.z);
            ff_add_prod(rr, rn.w, rn.w);
        }
        return rr;
    }
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

// ---- 2D operator on 128-column segments: residual-restriction and apply -----
//
// For 2D levels (ny = 1) whose nx is a multiple of 128.  A warp takes the 128
// fine columns c0 .. c0 + 127 over a run of rows and walks up them: lane l
// holds cells c0 + 4l .. c0 + 4l + 3 of a row (one float4 of each array), gets
// its x-neighbours from the next lanes by shuffles (the two cells outside the
// segment come from lanes 0 and 31), and keeps x and rho of the rows below and
// above in registers, so every value is loaded once, plus two rows of x and
// rho per warp.  The operator's arithmetic is that of apply32_at, term by
// term.  seg2d_ok: the shape, and 16-byte aligned arrays (float4 accesses).
__host__ __device__ inline bool seg2d_ok(const Geo& g, const void* a, const void* b, const void* c, const void* d,
                                         const void* e) {
    const uintptr_t u = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)e;
    return g.ny == 1 && g.nx % 128 == 0 && g.nz >= 2 && (u & 15) == 0;
}
// the residual-restriction's case: halved in x and z (fc is written as float2)
__host__ __device__ inline bool rr2d_ok(const Lev32& F, int hx, int hy, int hz, const float* x, const float* f,
                                        const float* fc) {
    return hx == 1 && hy == 0 && hz == 1 && seg2d_ok(F.g, x, f, F.rho, F.ct, nullptr) && ((uintptr_t)fc & 7) == 0;
}

struct Row4 {
    float4 x, rho;     // the lane's four cells
    float gx, grho;    // lane 0: the cell left of the segment; lane 31: right
};

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

struct Seg2D {
    const Lev32& L;
    int lane, cl, cg;  // cl: the lane's first column; cg: its outside cell (-1: a wall or none)
    bool fl, fr;       // x faces at the lane's two ends
    __device__ __forceinline__ Seg2D(const Lev32& L_, int c0) : L(L_) {
        const Geo& g = L.g;
        lane = threadIdx.x & 31;
        cl = c0 + 4 * lane;
        cg = -1;
        if (lane == 0) cg = c0 > 0 ? c0 - 1 : (g.bcx == LM_BC_PERIODIC ? g.nx - 1 : -1);
        if (lane == 31) cg = c0 + 128 < g.nx ? c0 + 128 : (g.bcx == LM_BC_PERIODIC ? 0 : -1);
        fl = lane > 0 || cg >= 0;
        fr = lane < 31 || cg >= 0;
    }
    // x and rho of row r (wrapped on a periodic z axis; zeros past a wall, where no face reads them)
    __device__ __forceinline__ Row4 load(const float* __restrict__ x, int r) const {
        const Geo& g = L.g;
        Row4 v;
        if (r < 0) r = g.bcz == LM_BC_PERIODIC ? r + g.nz : -1;
        else if (r >= g.nz) r = g.bcz == LM_BC_PERIODIC ? r - g.nz : -1;
        if (r < 0) {
            v.x = v.rho = make_float4(0.f, 0.f, 0.f, 0.f);
            v.gx = v.grho = 0.f;
            return v;
        }
        const size_t o = (size_t)r * g.nx;
        v.x = ld4(x + o + cl);
        v.rho = ld4(L.rho + o + cl);
        v.gx = cg >= 0 ? __ldg(x + o + cg) : 0.f;
        v.grho = cg >= 0 ? __ldg(L.rho + o + cg) : 0.f;
        return v;
    }
    // (A x) on the lane's four cells of row r (B, M, A: rows r - 1, r, r + 1; every lane calls it)
    __device__ __forceinline__ void apply(int r, const Row4& B, const Row4& M, const Row4& A, float y[4]) const {
        const Geo& g = L.g;
        const unsigned FULL = 0xffffffffu;
        float xl = __shfl_up_sync(FULL, M.x.w, 1), rl = __shfl_up_sync(FULL, M.rho.w, 1);
        float xr = __shfl_down_sync(FULL, M.x.x, 1), rr = __shfl_down_sync(FULL, M.rho.x, 1);
        if (lane == 0) xl = M.gx, rl = M.grho;
        if (lane == 31) xr = M.gx, rr = M.grho;
        const float4 cv = ld4(L.ct + (size_t)r * g.nx + cl);
        const bool zm = face_minus(r, g.nz, g.bcz), zp = face_plus(r, g.nz, g.bcz);
        const float xc[4] = {M.x.x, M.x.y, M.x.z, M.x.w}, rc[4] = {M.rho.x, M.rho.y, M.rho.z, M.rho.w};
        const float xb[4] = {B.x.x, B.x.y, B.x.z, B.x.w}, rb[4] = {B.rho.x, B.rho.y, B.rho.z, B.rho.w};
        const float xa[4] = {A.x.x, A.x.y, A.x.z, A.x.w}, ra[4] = {A.rho.x, A.rho.y, A.rho.z, A.rho.w};
        const float ct[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float xm = e ? xc[e - 1] : xl, rm = e ? rc[e - 1] : rl;
            const float xp = e < 3 ? xc[e + 1] : xr, rp = e < 3 ? rc[e + 1] : rr;
            float v = ct[e] * xc[e];
            if (e > 0 || fl) v += face32(rc[e], rm, L.c2x) * (xc[e] - xm);
            if (e < 3 || fr) v += face32(rc[e], rp, L.c2x) * (xc[e] - xp);
            if (zm) v += face32(rc[e], rb[e], L.c2z) * (xc[e] - xb[e]);
            if (zp) v += face32(rc[e], ra[e], L.c2z) * (xc[e] - xa[e]);
            y[e] = v;
        }
    }
};

// fc = mean over the four children of (f - A x) on the coarse rows K0 .. K1 - 1
// of a warp's segment: per coarse row it loads x and rho of fine rows 2K + 1,
// 2K + 2 and f, c~ of rows 2K, 2K + 1, and writes the lane's two coarse cells
// as one float2.  Sums in resid_restrict_tile's order.
__device__ __forceinline__ void rr2d_rows(const Lev32& F, const Geo& C, const float* __restrict__ x,
                                          const float* __restrict__ f, float* __restrict__ fc, int c0, int K0,
                                          int K1) {
    const Seg2D S(F, c0);
    const int nx = F.g.nx;
    Row4 rB = S.load(x, 2 * K0 - 1), rM = S.load(x, 2 * K0);
    for (int K = K0; K < K1; ++K) {
        const Row4 r1 = S.load(x, 2 * K + 1), r2 = S.load(x, 2 * K + 2);
        const float4 f0 = ld4(f + (size_t)(2 * K) * nx + S.cl), f1 = ld4(f + (size_t)(2 * K + 1) * nx + S.cl);
        float y0[4], y1[4];
        S.apply(2 * K, rB, rM, r1, y0);
        S.apply(2 * K + 1, rM, r1, r2, y1);
        float2 v;
        v.x = ((((0.f + (f0.x - y0[0])) + (f0.y - y0[1])) + (f1.x - y1[0])) + (f1.y - y1[1])) * 0.25f;
        v.y = ((((0.f + (f0.z - y0[2])) + (f0.w - y0[3])) + (f1.z - y1[2])) + (f1.w - y1[3])) * 0.25f;
        *reinterpret_cast<float2*>(fc + (size_t)K * C.nx + (c0 >> 1) + 2 * S.lane) = v;
        rB = r1;
        rM = r2;
    }
}

// y = A x on the rows k0 .. k1 - 1 of a warp's segment (float4 stores), with
// the lane's x.y and x.r accumulated into axy, axr (DOT_XR: r read too).
template <bool DOT_XY, bool DOT_XR>
__device__ __forceinline__ void apply2d_rows(const Lev32& L, const float* __restrict__ x, float* __restrict__ y,
                                             const float* __restrict__ r, int c0, int k0, int k1, FF& axy, FF& axr) {
    const Seg2D S(L, c0);
    const int nx = L.g.nx;
    Row4 rB = S.load(x, k0 - 1), rM = S.load(x, k0);
    for (int k = k0; k < k1; ++k) {
        const Row4 rA = S.load(x, k + 1);
        const size_t o = (size_t)k * nx + S.cl;
        const float4 rv = DOT_XR ? ld4(r + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        float v[4];
        S.apply(k, rB, rM, rA, v);
        *reinterpret_cast<float4*>(y + o) = make_float4(v[0], v[1], v[2], v[3]);
        const float xc[4] = {rM.x.x, rM.x.y, rM.x.z, rM.x.w}, rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (DOT_XY) ff_add_prod(axy, xc[e], v[e]);
            if (DOT_XR) ff_add_prod(axr, xc[e], rr[e]);
        }
        rB = rM;
        rM = rA;
    }
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

// float32 reciprocal by the hardware approximation (flushes denormals)
__device__ __forceinline__ float rcp_hw(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- 2D red-black sweep: a warp per row segment and z-chunk ------------------
//
// For 2D levels whose nx is a multiple of 128.  The four warps of a 128-thread
// block take a task (tile bx of TW = 256 or 128 columns, chunk of KZ rows bz)
// as two 128-cell segments times two halves of the chunk, or (TW = 128) one
// segment times four quarters, and each warp marches up its rows on its own:
// no block barrier, only warp synchronisation.  A warp keeps a
// five-row ring of (x, rho) in shared memory, each staged row an even-cell
// run and an odd-cell run (conflict-free accesses) between run-end slots that
// hold the neighbouring cells outside the segment (two each side; wrapped on
// a periodic x axis, x = 0 and rho = Z2_WALL past a wall).  At step p the warp
// updates the first colour of row p -- and, in lane 0, the segment's
// first-colour neighbour outside it, the value the neighbouring segment
// computes for its own cell -- and the second colour of row p - 2, whose
// first-colour neighbours (rows p - 3 .. p - 1) are final; neither update
// reads a cell the other writes.  Row p - 3 is then final and written, and
// row p + 2, loaded at the start of the step, is staged into its slot.  The
// two faces of an axis share one reciprocal.  f and c~ are loaded a step
// ahead, and x, rho, f, c~ of later rows are prefetched into L2.
// columns of a task of zrow2d_tile on a level of nx (a multiple of 128) cells
__host__ __device__ inline int zrow2d_width(int nx) { return nx % 256 == 0 ? 256 : 128; }
constexpr float Z2_WALL = 1e30f;                    // rho past a wall: face weight negligible, products finite
__device__ __forceinline__ int z2_e(int m) { return 1 + m; }             // even cell 2m of the segment
__device__ __forceinline__ int z2_o(int m) { return 3 + 64 + m; }        // odd cell 2m + 1 (64 pairs)

// Gauss-Seidel value of cell 2m + A of the staged row at b (dzm, dzp: ring
// offsets of the rows below and above)
template <int A>
__device__ __forceinline__ float z2_gs(const float2* __restrict__ XR, int b, int m, int dzm, int dzp, float fv,
                                       float cv, float c2x, float c2z) {
    const int cc = b + (A ? z2_o(m) : z2_e(m));
    const int im = b + (A ? z2_e(m) : z2_o(m - 1));
    const int ip = b + (A ? z2_e(m + 1) : z2_o(m));
    const float2 me = XR[cc], xm = XR[im], xp = XR[ip], zm = XR[cc + dzm], zp = XR[cc + dzp];
    const float axm = me.y + xm.y, axp = me.y + xp.y, tx = rcp_hw(axm * axp);
    const float azm = me.y + zm.y, azp = me.y + zp.y, tz = rcp_hw(azm * azp);
    const float rxm = axp * tx, rxp = axm * tx, rzm = azp * tz, rzp = azm * tz;
    const float sx = fmaf(rxp, xp.x, rxm * xm.x);
    const float sz = fmaf(rzp, zp.x, rzm * zm.x);
    const float num = fmaf(c2z, sz, fmaf(c2x, sx, fv));
    const float d = fmaf(c2z, rzm + rzp, fmaf(c2x, rxm + rxp, cv));
    return num * rcp_hw(d);
}

template <int FIRST, bool ZERO, bool PROLONG>
__device__ __forceinline__ void zrow2d_tile(const Lev32& L, const float* __restrict__ xin,
                                            const float* __restrict__ ec, const Geo& C, int hx, int hz,
                                            const float* __restrict__ f, float* __restrict__ xout, int KZ, int bx,
                                            int bz, int TW) {
    constexpr int NX = 128, M = 64, RS = NX + 4, NR = 5, H = 2;
    __shared__ float2 z2_ring[4][NR * RS];
    const Geo& g = L.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2* XR = z2_ring[w];
    // a task of TW = 256 columns: two segments times two halves of the chunk;
    // of TW = 128 columns: one segment times four quarters
    const int nseg = TW >> 7, parts = 4 / nseg, part = w / nseg;
    const int c0 = bx * TW + (w % nseg) * NX;
    const int t0 = bz * KZ, t1 = min(t0 + KZ, g.nz), len = t1 - t0;
    const int k0 = t0 + len * part / parts, k1 = t0 + len * (part + 1) / parts;
    if (k0 >= k1) return;                                // warp-uniform: no block barrier follows
    const int W = g.nx, i2 = 2 * lane;
    auto plane = [&](int p, int& pw) -> bool {           // row p wrapped; false past a wall
        if (p < 0 || p >= g.nz) {
            if (g.bcz != LM_BC_PERIODIC) return false;
            p = p < 0 ? p + g.nz : p - g.nz;
        }
        pw = p;
        return true;
    };
    // lanes 0..3 stage the outside cells: columns c0 - 2, c0 - 1, c0 + NX, c0 + NX + 1
    int gCol = c0 + (lane == 0 ? -2 : lane == 1 ? -1 : lane == 2 ? NX : NX + 1);
    bool gOK = lane < 4;
    if (gCol < 0 || gCol >= W) {
        if (g.bcx == LM_BC_PERIODIC) gCol = gCol < 0 ? gCol + W : gCol - W;
        else gOK = false;
    }
    const int gSlot = lane == 0 ? z2_e(-1) : lane == 1 ? z2_o(-1) : lane == 2 ? z2_e(M) : z2_o(M);
    float vx[2 * H], vr[2 * H], ve[2 * H], gx = 0.f, gr = Z2_WALL, ge = 0.f;
    auto fetch = [&](int p) {
        int pw = 0;
        const bool okp = plane(p, pw);
#pragma unroll
        for (int u = 0; u < H; ++u) {
            if (okp) {
                const int o = W * pw + c0 + 64 * u + i2;
                const float2 r2 = *reinterpret_cast<const float2*>(L.rho + o);
                vr[2 * u] = r2.x;
                vr[2 * u + 1] = r2.y;
                if (!ZERO) {
                    const float2 x2 = *reinterpret_cast<const float2*>(xin + o);
                    vx[2 * u] = x2.x;
                    vx[2 * u + 1] = x2.y;
                } else {
                    vx[2 * u] = vx[2 * u + 1] = 0.f;
                }
                if (PROLONG) {
                    const int po = C.nx * (pw >> hz);
                    ve[2 * u] = ec[po + ((c0 + 64 * u + i2) >> hx)];
                    ve[2 * u + 1] = ec[po + ((c0 + 64 * u + i2 + 1) >> hx)];
                }
            } else {
                vx[2 * u] = vx[2 * u + 1] = 0.f;
                vr[2 * u] = vr[2 * u + 1] = Z2_WALL;
                ve[2 * u] = ve[2 * u + 1] = 0.f;
            }
        }
        if (lane < 4) {
            if (okp && gOK) {
                const int o = W * pw + gCol;
                gx = ZERO ? 0.f : xin[o];
                gr = L.rho[o];
                ge = PROLONG ? ec[C.nx * (pw >> hz) + (gCol >> hx)] : 0.f;
            } else {
                gx = 0.f;
                gr = Z2_WALL;
                ge = 0.f;
            }
        }
    };
    auto store = [&](int s) {
        float2* R = XR + s * RS;
#pragma unroll
        for (int u = 0; u < H; ++u) {
            const int m = lane + 32 * u;
            R[z2_e(m)] = make_float2(PROLONG ? vx[2 * u] + ve[2 * u] : vx[2 * u], vr[2 * u]);
            R[z2_o(m)] = make_float2(PROLONG ? vx[2 * u + 1] + ve[2 * u + 1] : vx[2 * u + 1], vr[2 * u + 1]);
        }
        if (lane < 4) R[gSlot] = make_float2(PROLONG ? gx + ge : gx, gr);
    };
    // f and c~ of the updated cell of each of the lane's pairs in row p (a: 0 even, 1 odd)
    auto load_fc = [&](int p, bool ok, int a, float* F, float* Cv) {
        int pw = 0;
        if (ok && plane(p, pw)) {
            const int o = W * pw + c0 + i2 + a;
#pragma unroll
            for (int u = 0; u < H; ++u) {
                F[u] = f[o + 64 * u];
                Cv[u] = L.ct[o + 64 * u];
            }
        } else {
#pragma unroll
            for (int u = 0; u < H; ++u) {
                F[u] = 0.f;
                Cv[u] = 1.f;
            }
        }
    };
    auto par = [&](int p, int col) -> int { return (col + p) & 1; };   // updated cell of each pair
    // the first-colour outside cell of row p (lane 0): column c0 - 1 when the
    // row's first colour is odd, c0 + NX when even; its f and c~ a step ahead
    float fX = 0.f, cX = 1.f;
    bool xOK = false;
    auto load_fcx = [&](int p) {
        if (lane != 0) return;
        int pw = 0;
        xOK = false;
        if (p > k1 || !plane(p, pw)) return;
        int col = par(p, FIRST) ? c0 - 1 : c0 + NX;
        if (col < 0 || col >= W) {
            if (g.bcx != LM_BC_PERIODIC) return;
            col = col < 0 ? col + W : col - W;
        }
        xOK = true;
        fX = f[W * pw + col];
        cX = L.ct[W * pw + col];
    };
    auto prefetch = [&](int P) {                          // lane a < 4: x, rho, f, c~ of row P
        int pw = 0;
        if (lane >= 4 || P > (lane < 2 ? k1 + 1 : k1) || (ZERO && lane == 0) || !plane(P, pw)) return;
        const float* base = lane == 0 ? xin : lane == 1 ? L.rho : lane == 2 ? f : L.ct;
        prefetch_l2(base + W * pw + c0, NX * sizeof(float));
    };
    auto run_row = [&](int a, int b, int dzm, int dzp, const float* F, const float* Cv) {
        float nv[H];
#pragma unroll
        for (int u = 0; u < H; ++u)
            nv[u] = a ? z2_gs<1>(XR, b, lane + 32 * u, dzm, dzp, F[u], Cv[u], L.c2x, L.c2z)
                      : z2_gs<0>(XR, b, lane + 32 * u, dzm, dzp, F[u], Cv[u], L.c2x, L.c2z);
#pragma unroll
        for (int u = 0; u < H; ++u) XR[b + (a ? z2_o(lane + 32 * u) : z2_e(lane + 32 * u))].x = nv[u];
    };
    for (int d = 1; d <= PF_PLANES; ++d) prefetch((lane < 2 ? k0 : k0 - 1) + d);
    // prologue: rows k0 - 2 .. k0 staged; f, c~ of the first step's cells
    for (int q = 0; q < 3; ++q) {
        fetch(k0 - 2 + q);
        store(q);
    }
    int s_m3 = 3, s_m2 = 4, s_m1 = 0, s_0 = 1, s_p1 = 2;    // slots of rows p - 3 .. p + 1 at p = k0 - 1
    float fT[H], cT[H], fS[H], cS[H];
    load_fc(k0 - 1, true, par(k0 - 1, FIRST), fT, cT);
#pragma unroll
    for (int u = 0; u < H; ++u) {
        fS[u] = 0.f;
        cS[u] = 1.f;
    }
    load_fcx(k0 - 1);
    __syncwarp();
    for (int p = k0 - 1; p <= k1 + 2; ++p) {
        const bool stage = p + 2 <= k1 + 1;
        prefetch((lane < 2 ? p + 2 : p + 1) + PF_PLANES);
        if (stage) fetch(p + 2);
        int pw = 0;
        if (p <= k1 && plane(p, pw)) {                    // first colour on row p
            const int dzm = (s_m1 - s_0) * RS, dzp = (s_p1 - s_0) * RS, b = s_0 * RS;
            run_row(par(p, FIRST), b, dzm, dzp, fT, cT);
            if (lane == 0 && xOK) {
                if (par(p, FIRST)) XR[b + z2_o(-1)].x = z2_gs<1>(XR, b, -1, dzm, dzp, fX, cX, L.c2x, L.c2z);
                else XR[b + z2_e(M)].x = z2_gs<0>(XR, b, M, dzm, dzp, fX, cX, L.c2x, L.c2z);
            }
        }
        load_fc(p + 1, p + 1 <= k1, par(p + 1, FIRST), fT, cT);
        load_fcx(p + 1);
        const int q = p - 2;
        if (q >= k0 && q < k1)                           // second colour on row p - 2
            run_row(par(q, 1 - FIRST), s_m2 * RS, (s_m3 - s_m2) * RS, (s_m1 - s_m2) * RS, fS, cS);
        load_fc(q + 1, q + 1 >= k0 && q + 1 < k1, par(q + 1, 1 - FIRST), fS, cS);
        __syncwarp();
        if (p - 3 >= k0 && p - 3 < k1) {                 // row p - 3 is final
            const float2* R = XR + s_m3 * RS;
            float* dst = xout + W * (p - 3) + c0 + i2;
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int m = lane + 32 * u;
                *reinterpret_cast<float2*>(dst + 64 * u) = make_float2(R[z2_e(m)].x, R[z2_o(m)].x);
            }
        }
        __syncwarp();
        if (stage) store(s_m3);                           // row p + 2 takes row p - 3's slot
        __syncwarp();
        const int t = s_m3;
        s_m3 = s_m2;
        s_m2 = s_m1;
        s_m1 = s_0;
        s_0 = s_p1;
        s_p1 = t;
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
