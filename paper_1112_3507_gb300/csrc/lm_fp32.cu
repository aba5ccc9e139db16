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

// 2D levels passing seg2d_ok: warp w of block (bx, by) takes columns
// 128 bx .. 128 bx + 127 and rows (8 by + w) KR .. + KR - 1.
template <bool DOT_XY, bool DOT_XR>
__global__ void __launch_bounds__(256) k_apply32_2d(Lev32 L, const float* __restrict__ x, float* __restrict__ y,
                                                    const float* __restrict__ r, Red red, int slot_xy, int slot_xr,
                                                    int KR) {
    __shared__ double sm[64];
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
    const int k0 = (blockIdx.y * 8 + threadIdx.y) * KR;
    if (k0 < L.g.nz) apply2d_rows<DOT_XY, DOT_XR>(L, x, y, r, blockIdx.x * 128, k0, min(k0 + KR, L.g.nz), axy, axr);
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

// ---- 3D apply on whole tiles: a z-march over staged planes ----------------
// y = A x with x.y and x.r accumulated to float64 accuracy, for 3D levels
// whose nx, ny are multiples of the TX x 8 tile.  A block owns a tile's
// columns over a chunk of KZ planes and marches up z with a four-plane ring
// of x and rho staged on the tile plus one cell (periodic axes wrapped; past
// a Neumann wall x = 0 and rho = +inf, so that face's weight is 0): at step
// p it stores plane p + 1, issues the loads of plane p + 2 and, after one
// barrier, forms y on plane p from shared memory.  c~ and r of the next
// plane are loaded a step ahead.
__device__ __forceinline__ float rcp_approx(float x) {
    float q;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(x));
    return q;
}

template <int TX, bool DOT_XY, bool DOT_XR>
__global__ void __launch_bounds__(256) k_apply32_zm(Lev32 L, const float* __restrict__ x, float* __restrict__ y,
                                                   const float* __restrict__ r, Red red, int slot_xy, int slot_xr,
                                                   int KZ) {
    constexpr int NT2 = 256, TY = 8, SX = TX + 2, SY = TY + 2, PL = SX * SY, NR = 4;
    constexpr int QS = (PL + NT2 - 1) / NT2, QW = TX * TY / NT2;
    static_assert(SX + SY <= NT2 && QW * NT2 == TX * TY, "tile does not fit the block");
    __shared__ float X[NR * PL];
    __shared__ float R[NR * PL];
    __shared__ int ox[SX], oy[SY];
    __shared__ double sm[64];
    const Geo& g = L.g;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int k0 = blockIdx.z * KZ, k1 = min(k0 + KZ, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    if (tid < SX) {
        int c = i0 - 1 + tid;
        if (c < 0) c = g.bcx == LM_BC_PERIODIC ? c + g.nx : -1;
        else if (c >= g.nx) c = g.bcx == LM_BC_PERIODIC ? c - g.nx : -1;
        ox[tid] = c;
    } else if (tid < SX + SY) {
        int c = j0 - 1 + tid - SX;
        if (c < 0) c = g.bcy == LM_BC_PERIODIC ? c + g.ny : -1;
        else if (c >= g.ny) c = g.bcy == LM_BC_PERIODIC ? c - g.ny : -1;
        oy[tid - SX] = c < 0 ? -1 : sy * c;
    }
    __syncthreads();
    auto zoff = [&](int p) -> int {                      // p within one plane of [0, nz)
        if (p >= 0 && p < g.nz) return sz * p;
        if (g.bcz != LM_BC_PERIODIC) return -1;
        return sz * (p < 0 ? p + g.nz : p - g.nz);
    };
    int spos[QS], sbase[QS];
    bool sok[QS];
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        spos[q] = tid + q * NT2;
        const bool use = spos[q] < PL;
        const int sj = use ? spos[q] / SX : 0, si = use ? spos[q] - sj * SX : 0;
        sok[q] = use && (ox[si] | oy[sj]) >= 0;
        sbase[q] = ox[si] + oy[sj];
        if (!use) spos[q] = -1;
    }
    float vx[QS], vr[QS];
    auto fetch = [&](int zo) {
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            vx[q] = 0.f;
            vr[q] = __int_as_float(0x7f800000);          // +inf
            if (sok[q] && zo >= 0) {
                vx[q] = x[sbase[q] + zo];
                vr[q] = L.rho[sbase[q] + zo];
            }
        }
    };
    auto store = [&](int o) {
#pragma unroll
        for (int q = 0; q < QS; ++q)
            if (spos[q] >= 0) {
                X[o + spos[q]] = vx[q];
                R[o + spos[q]] = vr[q];
            }
    };
    int we[QW], wg[QW];
#pragma unroll
    for (int v = 0; v < QW; ++v) {
        const int w = tid + v * NT2, wx = w % TX, wy = w / TX;
        we[v] = (wy + 1) * SX + wx + 1;
        wg[v] = (i0 + wx) + sy * (j0 + wy);
    }
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
    float ctn[QW], rrn[QW];
    auto load_c = [&](int p) {
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            ctn[v] = L.ct[wg[v] + sz * p];
            rrn[v] = DOT_XR ? r[wg[v] + sz * p] : 0.f;
        }
    };
    fetch(zoff(k0 - 1));
    store(((k0 - 1) & 3) * PL);
    fetch(zoff(k0));
    store((k0 & 3) * PL);
    fetch(zoff(k0 + 1));
    load_c(k0);
    for (int p = k0; p < k1; ++p) {
        store(((p + 1) & 3) * PL);
        if (p + 2 <= k1) fetch(zoff(p + 2));
        float ctc[QW], rrc[QW];
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            ctc[v] = ctn[v];
            rrc[v] = rrn[v];
        }
        if (p + 1 < k1) load_c(p + 1);
        __syncthreads();
        const int om = ((p - 1) & 3) * PL, o0 = (p & 3) * PL, op = ((p + 1) & 3) * PL;
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            const int c = o0 + we[v];
            const float xc = X[c], rc = R[c];
            float val = ctc[v] * xc;
            val += L.c2x * rcp_approx(rc + R[c - 1]) * (xc - X[c - 1]);
            val += L.c2x * rcp_approx(rc + R[c + 1]) * (xc - X[c + 1]);
            val += L.c2y * rcp_approx(rc + R[c - SX]) * (xc - X[c - SX]);
            val += L.c2y * rcp_approx(rc + R[c + SX]) * (xc - X[c + SX]);
            val += L.c2z * rcp_approx(rc + R[om + we[v]]) * (xc - X[om + we[v]]);
            val += L.c2z * rcp_approx(rc + R[op + we[v]]) * (xc - X[op + we[v]]);
            y[wg[v] + sz * p] = val;
            if (DOT_XY) ff_add_prod(axy, xc, val);
            if (DOT_XR) ff_add_prod(axr, xc, rrc[v]);
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

// ---- float32 apply on whole rows: a warp per row, all lanes contiguous -------
//
// For 3D levels with nx = 32 CPT, ny a multiple of TY and nz >= 2 (the
// levels the whole-row sweep takes).  A block owns all nx columns of TY rows
// over a chunk of KZ planes and marches up z with a four-plane ring of
// (x, rho) staged on its rows plus one row each side (periodic axes wrapped;
// past a Neumann wall x = 0 and rho = +inf, so that face's weight is 0).
// Lane t of warp w computes the cells t + 32 v of row j0 + w, so every
// shared-memory and global access of a warp is contiguous.  A step computes
// plane p from the slots of planes p - 1 .. p + 1 and stages plane p + 2,
// loaded at the start of the step, into the fourth slot: one barrier per
// step.  Fused dot products as in k_apply32_zm.
template <int CPT, int TY>
constexpr size_t apply_row_smem() {
    return sizeof(float2) * 4 * (TY + 2) * (32 * CPT + 4);
}

template <int CPT, int TY, bool DOT_XY, bool DOT_XR, int SEG = 1>
__global__ void __launch_bounds__(32 * TY, 1) k_apply32_row(Lev32 L, const float* __restrict__ x,
                                                           float* __restrict__ y, const float* __restrict__ r,
                                                           Red red, int slot_xy, int slot_xr, int KZ) {
    constexpr int NX = 32 * CPT, RS = NX + 4, NRW = TY + 2, PL = NRW * RS, H = CPT / 2;
    constexpr int W = NX * SEG;                           // cells in a grid row
    static_assert(SEG == 1 || (SEG == 2 && 2 * NRW <= 32 * TY && 4 * TY <= 32 * TY), "x-halo threads");
    static_assert(CPT % 2 == 0 && TY >= 2 * H, "a warp per halo pair group");
    extern __shared__ float4 ap_smem[];
    float2* XR = reinterpret_cast<float2*>(ap_smem);
    __shared__ double sm[64];
    const Geo& g = L.g;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = lane + 32 * wy;
    const int j0 = (blockIdx.x / SEG) * TY, c0 = (blockIdx.x % SEG) * NX, k0 = blockIdx.y * KZ,
              k1 = min(k0 + KZ, g.nz);
    const int sz = W * g.ny, i2 = 2 * lane;
    const float INF = __int_as_float(0x7f800000);
    for (int t = tid; t < 4 * NRW; t += 32 * TY) {       // row-end ghosts: x = 0, rho = +inf
        XR[t * RS + 1] = make_float2(0.f, INF);
        XR[t * RS + NX + 2] = make_float2(0.f, INF);
    }
    if (SEG > 1) __syncthreads();                         // segments stage those slots: after the walls
    auto rowj = [&](int r_, int& jw) -> bool {           // staged row -> grid row; false past a wall
        int j = j0 - 1 + r_;
        if (j < 0 || j >= g.ny) {
            if (g.bcy != LM_BC_PERIODIC) return false;
            j = j < 0 ? j + g.ny : j - g.ny;
        }
        jw = j;
        return true;
    };
    auto plane = [&](int p, int& pw) -> bool {
        if (p < 0 || p >= g.nz) {
            if (g.bcz != LM_BC_PERIODIC) return false;
            p = p < 0 ? p + g.nz : p - g.nz;
        }
        pw = p;
        return true;
    };
    const int rT = wy + 1;
    const int uS = wy >> 1, rS = (wy & 1) ? TY + 1 : 0;   // this warp's pair group of a halo row
    int jT = 0, jS = 0;
    rowj(rT, jT);
    const bool hasS = uS < H, okS = hasS && rowj(rS, jS);
    // whole rows wrap around the staged row; a segment's x-neighbours outside
    // it are staged into the row-end slots each plane (SEG > 1): thread
    // 2 r + e stages staged row r's cell c0 - 1 (e = 0) or c0 + NX (e = 1);
    // past a wall x = 0, rho = +inf
    const bool perx = SEG == 1 && g.bcx == LM_BC_PERIODIC;
    const bool hasG = SEG > 1 && tid < 2 * NRW;
    const int rG = tid >> 1, gG = tid & 1;
    int gCol = gG ? c0 + NX : c0 - 1;
    bool gOK = true;
    if (gCol < 0 || gCol >= W) {
        if (g.bcx == LM_BC_PERIODIC) gCol = gCol < 0 ? gCol + W : gCol - W;
        else gOK = false;
    }
    float gxv = 0.f, grv = INF;
    float vx[CPT], vr[CPT], hx2[2], hr2[2];
    auto fetch = [&](int p) {
        int pw = 0;
        const bool okp = plane(p, pw);
#pragma unroll
        for (int u = 0; u < H; ++u) {
            if (okp) {
                const int o = sz * pw + W * jT + c0 + 64 * u + i2;
                const float2 a = *reinterpret_cast<const float2*>(x + o), b = *reinterpret_cast<const float2*>(L.rho + o);
                vx[2 * u] = a.x; vx[2 * u + 1] = a.y; vr[2 * u] = b.x; vr[2 * u + 1] = b.y;
            } else {
                vx[2 * u] = vx[2 * u + 1] = 0.f;
                vr[2 * u] = vr[2 * u + 1] = INF;
            }
        }
        if (hasS) {
            if (okp && okS) {
                const int o = sz * pw + W * jS + c0 + 64 * uS + i2;
                const float2 a = *reinterpret_cast<const float2*>(x + o), b = *reinterpret_cast<const float2*>(L.rho + o);
                hx2[0] = a.x; hx2[1] = a.y; hr2[0] = b.x; hr2[1] = b.y;
            } else {
                hx2[0] = hx2[1] = 0.f;
                hr2[0] = hr2[1] = INF;
            }
        }
        if (SEG > 1 && hasG) {                            // x-halo cell of staged row rG
            int jw = 0;
            if (okp && rowj(rG, jw) && gOK) {
                const int o = sz * pw + W * jw + gCol;
                gxv = x[o];
                grv = L.rho[o];
            } else {
                gxv = 0.f;
                grv = INF;
            }
        }
    };
    auto store = [&](int s) {
#pragma unroll
        for (int u = 0; u < H; ++u)
            *reinterpret_cast<float4*>(XR + (s * NRW + rT) * RS + 2 + 64 * u + i2) =
                make_float4(vx[2 * u], vr[2 * u], vx[2 * u + 1], vr[2 * u + 1]);
        if (hasS)
            *reinterpret_cast<float4*>(XR + (s * NRW + rS) * RS + 2 + 64 * uS + i2) =
                make_float4(hx2[0], hr2[0], hx2[1], hr2[1]);
        if (SEG > 1 && hasG) XR[(s * NRW + rG) * RS + (gG ? NX + 2 : 1)] = make_float2(gxv, grv);
    };
    float ctv[CPT], rrv[CPT];
    auto load_c = [&](int p) {                            // c~ (and r) of the warp's row on plane p
        const int o = sz * p + W * jT + c0 + lane;
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
            ctv[v] = L.ct[o + 32 * v];
            rrv[v] = DOT_XR ? r[o + 32 * v] : 0.f;
        }
    };
    const int lrel = (lane == 0 && perx) ? NX - 1 : -1;         // left of cell 0, right of cell nx - 1
    const int rrel = (lane == 31 && perx) ? 1 - NX : 1;
    // L2 prefetch of the block's own rows, PF_PLANES steps ahead: x and rho of
    // plane P are staged at step P - 2, c~ and r read at step P - 1; array
    // a = 0..3 (x, rho, c~, r) is requested by thread a (a segment's rows are
    // not contiguous: one request per row, thread a TY + r for row r)
    constexpr int NPF = SEG == 1 ? 4 : 4 * TY;
    const int pfa = SEG == 1 ? tid : tid / TY, pfr = SEG == 1 ? 0 : tid % TY;
    auto prefetch = [&](int a, int P) {
        int pw = 0;
        if (P > (a < 2 ? k1 : k1 - 1) || (!DOT_XR && a == 3) || !plane(P, pw)) return;
        const float* base = a == 0 ? x : a == 1 ? L.rho : a == 2 ? L.ct : r;
        if (SEG == 1) prefetch_l2(base + sz * pw + NX * j0, NX * TY * sizeof(float));
        else prefetch_l2(base + sz * pw + W * (j0 + pfr) + c0, NX * sizeof(float));
    };
    if (tid < NPF)
        for (int d = 1; d <= PF_PLANES; ++d) prefetch(pfa, (pfa < 2 ? k0 + 1 : k0) + d);
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
    int sm1 = 0, s0 = 1, sp1 = 2, sp2 = 3;                // slots of planes p - 1 .. p + 2
    fetch(k0 - 1);
    store(sm1);
    fetch(k0);
    store(s0);
    fetch(k0 + 1);
    store(sp1);
    load_c(k0);
    __syncthreads();
    for (int p = k0; p < k1; ++p) {
        const bool stage = p + 2 <= k1;
        if (tid < NPF) prefetch(pfa, (pfa < 2 ? p + 2 : p + 1) + PF_PLANES);
        if (stage) fetch(p + 2);
        const int b0 = (s0 * NRW + rT) * RS + 2 + lane, dzm = (sm1 - s0) * PL, dzp = (sp1 - s0) * PL;
        float* yrow = y + sz * p + W * jT + c0 + lane;
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
            const int c = b0 + 32 * v;
            const float2 me = XR[c];
            const float2 xm = XR[c + (v == 0 ? lrel : -1)], xp = XR[c + (v == CPT - 1 ? rrel : 1)];
            const float2 ym = XR[c - RS], yp = XR[c + RS], zm = XR[c + dzm], zp = XR[c + dzp];
            float val = ctv[v] * me.x;
            val += L.c2x * rcp_approx(me.y + xm.y) * (me.x - xm.x);
            val += L.c2x * rcp_approx(me.y + xp.y) * (me.x - xp.x);
            val += L.c2y * rcp_approx(me.y + ym.y) * (me.x - ym.x);
            val += L.c2y * rcp_approx(me.y + yp.y) * (me.x - yp.x);
            val += L.c2z * rcp_approx(me.y + zm.y) * (me.x - zm.x);
            val += L.c2z * rcp_approx(me.y + zp.y) * (me.x - zp.x);
            yrow[32 * v] = val;
            if (DOT_XY) ff_add_prod(axy, me.x, val);
            if (DOT_XR) ff_add_prod(axr, me.x, rrv[v]);
        }
        if (p + 1 < k1) load_c(p + 1);
        if (stage) store(sp2);                            // no one reads that slot in this step
        __syncthreads();
        const int t = sm1;
        sm1 = s0;
        s0 = sp1;
        sp1 = sp2;
        sp2 = t;
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

// ---- 3D residual + restriction on whole tiles: a z-march -------------------
// fc = mean over the children of (f - A x), for 3D fine levels whose nx, ny
// are multiples of the TX x 8 tile: the same staged four-plane ring as
// k_apply32_zm; each step forms the residual of one fine plane of the tile
// in shared memory, the threads of the coarse cells add their children in
// x and y, and the sum over the (1 << hz) fine planes of a coarse plane
// is carried in a register until the coarse plane is written.
template <int TX>
__global__ void __launch_bounds__(256) k_resid_restrict_zm(Lev32 L, Geo C, int hx, int hy, int hz,
                                                          const float* __restrict__ x, const float* __restrict__ f,
                                                          float* __restrict__ fc, int KZ) {
    constexpr int NT2 = 256, TY = 8, SX = TX + 2, SY = TY + 2, PL = SX * SY, NR = 4;
    constexpr int QS = (PL + NT2 - 1) / NT2, QW = TX * TY / NT2;
    __shared__ float X[NR * PL];
    __shared__ float R[NR * PL];
    __shared__ float RS[TX * TY];
    __shared__ int ox[SX], oy[SY];
    const Geo& g = L.g;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int k0 = blockIdx.z * KZ, k1 = min(k0 + KZ, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    if (tid < SX) {
        int c = i0 - 1 + tid;
        if (c < 0) c = g.bcx == LM_BC_PERIODIC ? c + g.nx : -1;
        else if (c >= g.nx) c = g.bcx == LM_BC_PERIODIC ? c - g.nx : -1;
        ox[tid] = c;
    } else if (tid < SX + SY) {
        int c = j0 - 1 + tid - SX;
        if (c < 0) c = g.bcy == LM_BC_PERIODIC ? c + g.ny : -1;
        else if (c >= g.ny) c = g.bcy == LM_BC_PERIODIC ? c - g.ny : -1;
        oy[tid - SX] = c < 0 ? -1 : sy * c;
    }
    __syncthreads();
    auto zoff = [&](int p) -> int {
        if (p >= 0 && p < g.nz) return sz * p;
        if (g.bcz != LM_BC_PERIODIC) return -1;
        return sz * (p < 0 ? p + g.nz : p - g.nz);
    };
    int spos[QS], sbase[QS];
    bool sok[QS];
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        spos[q] = tid + q * NT2;
        const bool use = spos[q] < PL;
        const int sj = use ? spos[q] / SX : 0, si = use ? spos[q] - sj * SX : 0;
        sok[q] = use && (ox[si] | oy[sj]) >= 0;
        sbase[q] = ox[si] + oy[sj];
        if (!use) spos[q] = -1;
    }
    float vx[QS], vr[QS];
    auto fetch = [&](int zo) {
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            vx[q] = 0.f;
            vr[q] = __int_as_float(0x7f800000);          // +inf
            if (sok[q] && zo >= 0) {
                vx[q] = x[sbase[q] + zo];
                vr[q] = L.rho[sbase[q] + zo];
            }
        }
    };
    auto store = [&](int o) {
#pragma unroll
        for (int q = 0; q < QS; ++q)
            if (spos[q] >= 0) {
                X[o + spos[q]] = vx[q];
                R[o + spos[q]] = vr[q];
            }
    };
    int we[QW], wg[QW], wl[QW];
#pragma unroll
    for (int v = 0; v < QW; ++v) {
        const int w = tid + v * NT2, wx = w % TX, wy = w / TX;
        we[v] = (wy + 1) * SX + wx + 1;
        wg[v] = (i0 + wx) + sy * (j0 + wy);
        wl[v] = w;
    }
    // coarse cell of this thread: (ci, cj) of the (TX >> hx) x (TY >> hy) coarse tile
    const int CX = TX >> hx, CY = TY >> hy;
    const bool hasC = tid < CX * CY;
    const int cci = hasC ? tid % CX : 0, ccj = hasC ? tid / CX : 0;
    const int cbase = ((i0 >> hx) + cci) + C.nx * ((j0 >> hy) + ccj);
    const float inv = 1.f / (float)((1 << hx) << hy << hz);
    float csum = 0.f;
    float ctn[QW], fn[QW];
    auto load_c = [&](int p) {
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            ctn[v] = L.ct[wg[v] + sz * p];
            fn[v] = f[wg[v] + sz * p];
        }
    };
    fetch(zoff(k0 - 1));
    store(((k0 - 1) & 3) * PL);
    fetch(zoff(k0));
    store((k0 & 3) * PL);
    fetch(zoff(k0 + 1));
    load_c(k0);
    for (int p = k0; p < k1; ++p) {
        store(((p + 1) & 3) * PL);
        if (p + 2 <= k1) fetch(zoff(p + 2));
        float ctc[QW], fcur[QW];
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            ctc[v] = ctn[v];
            fcur[v] = fn[v];
        }
        if (p + 1 < k1) load_c(p + 1);
        __syncthreads();
        const int om = ((p - 1) & 3) * PL, o0 = (p & 3) * PL, op = ((p + 1) & 3) * PL;
#pragma unroll
        for (int v = 0; v < QW; ++v) {
            const int c = o0 + we[v];
            const float xc = X[c], rc = R[c];
            float val = ctc[v] * xc;
            val += L.c2x * rcp_approx(rc + R[c - 1]) * (xc - X[c - 1]);
            val += L.c2x * rcp_approx(rc + R[c + 1]) * (xc - X[c + 1]);
            val += L.c2y * rcp_approx(rc + R[c - SX]) * (xc - X[c - SX]);
            val += L.c2y * rcp_approx(rc + R[c + SX]) * (xc - X[c + SX]);
            val += L.c2z * rcp_approx(rc + R[om + we[v]]) * (xc - X[om + we[v]]);
            val += L.c2z * rcp_approx(rc + R[op + we[v]]) * (xc - X[op + we[v]]);
            RS[wl[v]] = fcur[v] - val;
        }
        __syncthreads();
        if (hasC) {
            for (int b = 0; b <= hy; ++b)
                for (int a = 0; a <= hx; ++a) csum += RS[((ccj << hy) + b) * TX + (cci << hx) + a];
            if (hz == 0 || (p & 1)) {
                fc[cbase + C.nx * C.ny * (p >> hz)] = csum * inv;
                csum = 0.f;
            }
        }
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
    coarsen_cell(F, C, hx, hy, hz, ct_c, rho_c, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(256) k_resid_restrict(Lev32 F, Geo C, int hx, int hy, int hz,
                                                        const float* __restrict__ x, const float* __restrict__ f,
                                                        float* __restrict__ fc) {
    resid_restrict_tile(F, C, hx, hy, hz, x, f, fc, blockIdx.x, blockIdx.y, blockIdx.z);
}

// 2D levels passing rr2d_ok: warp w of block (bx, by) takes fine columns
// 128 bx .. 128 bx + 127 and coarse rows (8 by + w) KR .. + KR - 1.
__global__ void __launch_bounds__(256, 3) k_resid_restrict_2d(Lev32 F, Geo C, const float* __restrict__ x,
                                                           const float* __restrict__ f, float* __restrict__ fc,
                                                           int KR) {
    const int K0 = (blockIdx.y * 8 + threadIdx.y) * KR;
    if (K0 >= C.nz) return;
    rr2d_rows(F, C, x, f, fc, blockIdx.x * 128, K0, min(K0 + KR, C.nz));
}

// ---- 3D red-black sweep on whole tiles: in-place z-march ------------------
//
// For 3D levels whose nx, ny are multiples of the 32 x 8 tile.  A block owns
// the columns of one tile over a chunk of KZ planes and marches up z with a
// five-plane ring of x and rho staged on the tile plus two cells in x and y
// (periodic axes wrapped; past a Neumann wall x = 0 and rho = +inf, so that
// face's weight c2 / (rho_c + inf) is 0 and no wall test is needed).  At
// step s the block (1) stores the staged plane s + 1 and issues the loads of
// plane s + 2, (2) updates the FIRST colour of plane s on the tile plus a
// one-cell halo in place -- a first-colour update reads only second-colour
// neighbours, and the halo values equal those the neighbouring blocks
// compute for their own cells -- (3) updates the second colour of plane
// s - 1 on the tile, whose first-colour neighbours (planes s - 2 .. s) are
// final, and (4) writes plane s - 2, final since step s - 1.  One sweep is
// thus one pass over memory with no grid-wide barrier.  Work items
// enumerate only cells of the colour being updated; wrapped in-plane
// offsets are per-thread constants from small tables; f and c~ of the next
// step's cells are loaded a step ahead.  Face weights and the final
// division use the hardware reciprocal approximation (rcp_fast), so the
// result can differ from rbgs_tile's in the last bits.
// Reciprocal by the hardware approximation (rcp.approx.ftz: relative error
// below 2^-22; +inf -> 0), the z-march's face weights and GS division.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int TX, int FIRST, bool ZERO, bool PROLONG>
__global__ void __launch_bounds__(256) k_rbgs_zm(Lev32 L, const float* __restrict__ xin,
                                                const float* __restrict__ ec, Geo C, int hx, int hy, int hz,
                                                const float* __restrict__ f, float* __restrict__ xout, int KZ) {
    constexpr int NT2 = 256, TY = 8, SX = TX + 4, SY = TY + 4, PL = SX * SY, NR = 5;
    constexpr int AW = (TX + 2) / 2;                     // first-colour cells per halo-box row
    constexpr int NA = AW * (TY + 2);                    // ... per halo-box plane (170 / 330)
    constexpr int NB = TX / 2 * TY;                      // second-colour cells per tile plane (128 / 256)
    constexpr int QS = (PL + NT2 - 1) / NT2;             // staged positions per thread
    constexpr int QA = (NA + NT2 - 1) / NT2;             // first-colour tasks per thread
    constexpr int QW = TX * TY / NT2;                    // written cells per thread
    static_assert(NB <= NT2 && SX + SY <= NT2 && QW * NT2 == TX * TY, "tile does not fit the block");
    __shared__ float2 XR[NR * PL];                       // (x, rho) per staged cell: one 64-bit access
    __shared__ int ox[SX], oy[SY], pxy[SX + SY];
    const Geo& g = L.g;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int k0 = blockIdx.z * KZ, k1 = min(k0 + KZ, g.nz);
    const int sy = g.nx, sz = g.nx * g.ny;
    if (tid < SX) {
        int c = i0 - 2 + tid;
        if (c < 0) c = g.bcx == LM_BC_PERIODIC ? c + g.nx : -1;
        else if (c >= g.nx) c = g.bcx == LM_BC_PERIODIC ? c - g.nx : -1;
        ox[tid] = c;
        pxy[tid] = c >> hx;
    } else if (tid < SX + SY) {
        int c = j0 - 2 + tid - SX;
        if (c < 0) c = g.bcy == LM_BC_PERIODIC ? c + g.ny : -1;
        else if (c >= g.ny) c = g.bcy == LM_BC_PERIODIC ? c - g.ny : -1;
        oy[tid - SX] = c < 0 ? -1 : sy * c;
        pxy[tid] = C.nx * (c >> hy);
    }
    __syncthreads();
    // plane p (unwrapped) -> wrapped plane offset, -1 past a wall; and the
    // parent plane offset (PROLONG)
    auto zwrap = [&](int p) -> int { return ((p % g.nz) + g.nz) % g.nz; };
    auto zoff = [&](int p) -> int {
        if (p >= 0 && p < g.nz) return sz * p;
        return g.bcz == LM_BC_PERIODIC ? sz * zwrap(p) : -1;
    };
    auto zpar = [&](int p) -> int { return C.nx * C.ny * (zwrap(p) >> hz); };

    // staging positions of this thread: tid + 256 q of the in-plane positions
    int spos[QS], sbase[QS], spar[QS];
    bool sok[QS];
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        spos[q] = tid + q * NT2;
        const bool use = spos[q] < PL;
        const int sj = use ? spos[q] / SX : 0, si = use ? spos[q] - sj * SX : 0;
        sok[q] = use && (ox[si] | oy[sj]) >= 0;
        sbase[q] = ox[si] + oy[sj];
        spar[q] = pxy[si] + pxy[SX + sj];
        if (!use) spos[q] = -1;
    }
    // x, rho and (PROLONG) the coarse correction of a staged plane, held in
    // registers from their loads until the plane is stored a step later, so
    // nothing waits on the loads within the step that issues them
    float vx[QS], vr[QS], ve[QS];
    auto fetch = [&](int zo, int zp) {                   // plane with offset zo -> registers
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
    auto store = [&](int o) {                            // registers -> ring slot at offset o
#pragma unroll
        for (int q = 0; q < QS; ++q)
            if (spos[q] >= 0) {
                XR[o + spos[q]] = make_float2(PROLONG ? vx[q] + ve[q] : vx[q], vr[q]);
            }
    };

    // Gauss-Seidel value at in-plane staged position e of the plane in ring
    // slot s0 (slots sm, sp: the planes below and above)
    auto gs = [&](int e, int sm, int s0, int sp, float fv, float cv) -> float {
        const int c = s0 + e;
        const float rc = XR[c].y;
        const float2 nxm = XR[c - 1], nxp = XR[c + 1], nym = XR[c - SX], nyp = XR[c + SX];
        const float2 nzm = XR[sm + e], nzp = XR[sp + e];
        const float wxm = L.c2x * rcp_fast(rc + nxm.y);
        const float wxp = L.c2x * rcp_fast(rc + nxp.y);
        const float wym = L.c2y * rcp_fast(rc + nym.y);
        const float wyp = L.c2y * rcp_fast(rc + nyp.y);
        const float wzm = L.c2z * rcp_fast(rc + nzm.y);
        const float wzp = L.c2z * rcp_fast(rc + nzp.y);
        const float d = cv + ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
        float num = fv;
        num = fmaf(wxm, nxm.x, num);
        num = fmaf(wxp, nxp.x, num);
        num = fmaf(wym, nym.x, num);
        num = fmaf(wyp, nyp.x, num);
        num = fmaf(wzm, nzm.x, num);
        num = fmaf(wzp, nzp.x, num);
        return num * rcp_fast(d);
    };

    // first-colour tasks of this thread: task tid + 256 u is pair am of
    // halo-box row abj; its cell alternates between the pair's two x positions
    bool hasA[QA];
    int aeE[QA], aoy[QA], aoE[QA], aoO[QA], apar[QA];
#pragma unroll
    for (int u = 0; u < QA; ++u) {
        const int ta = tid + u * NT2;
        hasA[u] = ta < NA;
        const int am = hasA[u] ? ta % AW : 0, abj = hasA[u] ? ta / AW : 0;
        aeE[u] = (abj + 1) * SX + 2 * am + 1;
        aoy[u] = oy[abj + 1];
        aoE[u] = ox[2 * am + 1];
        aoO[u] = ox[2 * am + 2];
        apar[u] = (FIRST + i0 + j0 + abj) & 1;           // odd-x on plane p iff (apar + p) & 1
    }
    // second-colour task (tid < NB): pair bm of tile row btj
    const bool hasB = tid < NB;
    const int bm = tid % (TX / 2), btj = (tid / (TX / 2)) % TY;
    const int beE = (btj + 2) * SX + 2 * bm + 2;
    const int bidxE = i0 + 2 * bm + sy * (j0 + btj);
    const int bpar = (1 - FIRST + i0 + j0 + btj) & 1;
    // written cells: tid + 256 v of the tile plane
    int wpos[QW], wbase[QW];
#pragma unroll
    for (int v = 0; v < QW; ++v) {
        const int w = tid + v * NT2, wx = w % TX, wy = w / TX;
        wpos[v] = (wy + 2) * SX + wx + 2;
        wbase[v] = (i0 + wx) + sy * (j0 + wy);
    }

    // ring slot offsets of planes p - 2 .. p + 2 at step p (rotated each step)
    int om2 = 0 * PL, om1 = 1 * PL, o0 = 2 * PL, op1 = 3 * PL, op2 = 4 * PL;
    // wrapped offsets of planes p, p + 1, p + 2 (shift register)
    int z0 = zoff(k0 - 1), z1 = zoff(k0), z2 = zoff(k0 + 1);
    // parent plane offset of plane p + 2 (PROLONG), carried like z2
    int zp2 = PROLONG ? zpar(k0 + 1) : 0;
    // prologue: planes k0 - 2, k0 - 1 staged; plane k0 in registers
    fetch(zoff(k0 - 2), PROLONG ? zpar(k0 - 2) : 0);
    store(om1);
    fetch(z0, PROLONG ? zpar(k0 - 1) : 0);
    store(o0);
    fetch(z1, PROLONG ? zpar(k0) : 0);
    // f, c~ of the first-colour cells of plane p (loaded a step ahead)
    float fa[QA], ca[QA];
    bool okA[QA];
    int eA[QA];
    auto load_a = [&](int p, int zo, bool in_chunk) {
#pragma unroll
        for (int u = 0; u < QA; ++u) {
            const int odd = (apar[u] + p) & 1;
            const int a = odd ? aoO[u] : aoE[u];
            okA[u] = hasA[u] && in_chunk && (a | aoy[u] | zo) >= 0;
            eA[u] = aeE[u] + odd;
            fa[u] = 0.f;
            ca[u] = 1.f;
            if (okA[u]) {
                fa[u] = f[a + aoy[u] + zo];
                ca[u] = L.ct[a + aoy[u] + zo];
            }
        }
    };
    load_a(k0 - 1, z0, true);
    float fb = 0.f, cb = 1.f;
    bool okB = false;
    int eB = 0;
    for (int p = k0 - 1; p <= k1 + 1; ++p) {
        // (1) stage plane p + 1, fetch plane p + 2
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
        // f, c~ of the second-colour cell of plane p (used at step p + 1)
        {
            const int odd = (bpar + p) & 1;
            okB = hasB && p >= k0 && p < k1;
            eB = beE + odd;
            if (okB) {
                const int idx = bidxE + odd + sz * p;
                fb = f[idx];
                cb = L.ct[idx];
            }
        }
        __syncthreads();
        // (2) first colour on plane p (tile + halo)
#pragma unroll
        for (int u = 0; u < QA; ++u)
            if (doA[u]) XR[o0 + eAc[u]].x = gs(eAc[u], om1, o0, op1, fA[u], cA[u]);
        load_a(p + 1, z1, p + 1 <= k1);                  // for the next step
        __syncthreads();
        // (3) second colour on plane p - 1 (tile)
        if (doB) XR[om1 + eBc].x = gs(eBc, om2, om1, o0, fB, cB);
        // (4) write plane p - 2
        if (p - 2 >= k0) {
#pragma unroll
            for (int v = 0; v < QW; ++v) xout[wbase[v] + sz * (p - 2)] = XR[om2 + wpos[v]].x;
        }
        // rotate to step p + 1
        const int t = om2;
        om2 = om1;
        om1 = o0;
        o0 = op1;
        op1 = op2;
        op2 = t;
        z0 = z1;
        z1 = z2;
        {   // offset of plane p + 3 (p + 3 <= nz + 4: at most two wraps)
            int c = p + 3;
            if (c >= g.nz) c -= g.nz;
            if (c >= g.nz) c -= g.nz;
            z2 = (p + 3 < g.nz || g.bcz == LM_BC_PERIODIC) && c >= 0 && c < g.nz ? sz * c : -1;
            if (PROLONG) zp2 = C.nx * C.ny * ((c >= 0 && c < g.nz ? c : 0) >> hz);
        }
    }
}

// ---- 3D red-black sweep on whole rows: a warp per row, one barrier a plane --
//
// For 3D levels with nx = 32 CPT, ny a multiple of TY and nz >= 2.  A block
// owns all nx columns of TY rows over a chunk of KZ planes; warp w owns row
// j0 + w.  The block marches up z with a five-plane ring of (x, rho) staged
// on its rows plus two rows each side (periodic axes wrapped; past a Neumann
// wall x = 0 and rho = ROW_WALL, so that face's weight is negligible and no
// wall test is needed).  A staged row keeps its even cells, then its
// odd cells, each run between two ghost cells: the cells of one colour in a
// row are then contiguous, and so are their x-neighbours (the other run), so
// a warp updating 32 cells of one colour reads every neighbour with one
// conflict-free access (lane t: cells 2 (t + 32 u) + a, u < CPT / 2).  At
// step p the block updates in place
//   - the first colour of plane p on its rows and one halo row each side
//     (a first-colour update reads only second-colour cells, which nobody
//     has updated yet, so the halo values equal the neighbours' own), and
//   - the second colour of plane p - 2 on its rows, whose first-colour
//     neighbours (planes p - 3 .. p - 1, rows and halo rows) are final.
// Neither update reads a cell the other writes, so one barrier per step
// suffices.  Plane p - 3 is then final and written out, and plane p + 2,
// loaded at the start of the step, is staged into its ring slot.  A row's
// colour parity is uniform over its warp, so each warp takes the branch for
// its parity.  f and c~ of the next step's cells are loaded a step ahead.
// The halo rows' staging and updates are spread one pair group per warp.

// rho of the cells past a wall: large but finite, so that a face weight
// c2 / (rho_c + ROW_WALL) is negligible (x there is 0) and the product of an
// axis's two face sums stays finite (for rho within [2^-60, 2^26], the band
// the assembly keeps the float32 copy of rho in)
constexpr float ROW_WALL = 1e30f;

// Ring index of even cell m (run E) and odd cell m (run O) of a staged row
// of M = nx / 2 pairs; E(-1), E(M), O(-1), O(M) are the ghosts.
__device__ __forceinline__ int run_e(int M, int m) { return 1 + m; }
__device__ __forceinline__ int run_o(int M, int m) { return 3 + M + m; }

// Gauss-Seidel value of cell 2 m + A of the row at ring index b (plane),
// with dzm, dzp the ring offsets of the planes below and above; wrap: the
// cell's outer x-neighbour (left of cell 0, right of cell nx - 1) wraps
// around the row (periodic x) instead of reading the ghost.
template <int A>
__device__ __forceinline__ float gs_run(const float2* __restrict__ XR, int b, int M, int m, bool wrap, int RS,
                                        int dzm, int dzp, float fv, float cv, float c2x, float c2y, float c2z) {
    const int cc = b + (A ? run_o(M, m) : run_e(M, m));
    const int im = A ? run_e(M, m) : (wrap ? run_o(M, M - 1) : run_o(M, m - 1));
    const int ip = A ? (wrap ? run_e(M, 0) : run_e(M, m + 1)) : run_o(M, m);
    const float2 me = XR[cc];
    const float2 xm = XR[b + im], xp = XR[b + ip];
    const float2 ym = XR[cc - RS], yp = XR[cc + RS];
    const float2 zm = XR[cc + dzm], zp = XR[cc + dzp];
    // the two faces of an axis share one reciprocal: 1/a = b/(ab), 1/b = a/(ab)
    // (at most one face of an axis is a wall, rho = ROW_WALL, so ab stays finite)
    const float axm = me.y + xm.y, axp = me.y + xp.y, tx = rcp_fast(axm * axp);
    const float aym = me.y + ym.y, ayp = me.y + yp.y, ty = rcp_fast(aym * ayp);
    const float azm = me.y + zm.y, azp = me.y + zp.y, tz = rcp_fast(azm * azp);
    const float rxm = axp * tx, rxp = axm * tx, rym = ayp * ty, ryp = aym * ty, rzm = azp * tz, rzp = azm * tz;
    const float sx = fmaf(rxp, xp.x, rxm * xm.x);
    const float sy = fmaf(ryp, yp.x, rym * ym.x);
    const float sz = fmaf(rzp, zp.x, rzm * zm.x);
    const float num = fmaf(c2z, sz, fmaf(c2y, sy, fmaf(c2x, sx, fv)));
    const float d = fmaf(c2z, rzm + rzp, fmaf(c2y, rym + ryp, fmaf(c2x, rxm + rxp, cv)));
    return num * rcp_fast(d);
}

// The colour-A cells of a warp's row at ring index b: all values formed
// before any is stored, so their loads can be in flight together.
template <int CPT, int A>
__device__ __forceinline__ void gs_row_runs(float2* __restrict__ XR, int b, int lane, bool perx, int RS, int dzm,
                                            int dzp, const float* fv, const float* cv, float c2x, float c2y,
                                            float c2z) {
    constexpr int H = CPT / 2, M = 16 * CPT;
    float nv[H];
#pragma unroll
    for (int u = 0; u < H; ++u) {
        const int m = lane + 32 * u;
        const bool wrap = perx && (A ? (u == H - 1 && lane == 31) : (u == 0 && lane == 0));
        nv[u] = gs_run<A>(XR, b, M, m, wrap, RS, dzm, dzp, fv[u], cv[u], c2x, c2y, c2z);
    }
#pragma unroll
    for (int u = 0; u < H; ++u) XR[b + (A ? run_o(M, lane + 32 * u) : run_e(M, lane + 32 * u))].x = nv[u];
}

template <int CPT, int TY>
constexpr size_t rbgs_row_smem() {
    return sizeof(float2) * 5 * (TY + 4) * (32 * CPT + 4);
}

template <int CPT, int TY, int FIRST, bool ZERO, bool PROLONG, int SEG>
__global__ void __launch_bounds__(32 * TY, 1) k_rbgs_row(Lev32 L, const float* __restrict__ xin,
                                                        const float* __restrict__ ec, Geo C, int hx, int hy,
                                                        int hz, const float* __restrict__ f,
                                                        float* __restrict__ xout, int KZ) {
    constexpr int NX = 32 * CPT, M = NX / 2, RS = NX + 4, NRW = TY + 4, PL = NRW * RS, NR = 5, H = CPT / 2;
    constexpr int W = NX * SEG;                           // cells in a grid row
    static_assert(CPT % 2 == 0 && TY >= 4 * H / 2 && TY >= 2 * H, "a warp per halo pair group");
    static_assert(SEG == 1 || (SEG == 2 && 4 * NRW <= 32 * TY && 4 * TY <= 32 * TY), "x-halo threads");
    extern __shared__ float4 row_smem[];
    float2* XR = reinterpret_cast<float2*>(row_smem);
    const Geo& g = L.g;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = lane + 32 * wy;
    const int j0 = (blockIdx.x / SEG) * TY, c0 = (blockIdx.x % SEG) * NX;
    const int k0 = blockIdx.y * KZ, k1 = min(k0 + KZ, g.nz);
    const int sz = W * g.ny, i2 = 2 * lane;
    for (int t = tid; t < NR * NRW; t += 32 * TY) {      // the run-end ghosts: x = 0, rho = ROW_WALL
        const float2 gh = make_float2(0.f, ROW_WALL);
        XR[t * RS + run_e(M, -1)] = gh;
        XR[t * RS + run_e(M, M)] = gh;
        XR[t * RS + run_o(M, -1)] = gh;
        XR[t * RS + run_o(M, M)] = gh;
    }
    if (SEG > 1) __syncthreads();                         // segments stage those slots: after the walls
    // staged row r <-> grid row j0 - 2 + r, wrapped; false past a wall
    auto rowj = [&](int r, int& jw) -> bool {
        int j = j0 - 2 + r;
        if (j < 0 || j >= g.ny) {
            if (g.bcy != LM_BC_PERIODIC) return false;
            j = j < 0 ? j + g.ny : j - g.ny;
        }
        jw = j;
        return true;
    };
    // plane p (k0 - 2 <= p <= k1 + 1) -> wrapped plane; false past a wall
    auto plane = [&](int p, int& pw) -> bool {
        if (p < 0 || p >= g.nz) {
            if (g.bcz != LM_BC_PERIODIC) return false;
            p = p < 0 ? p + g.nz : p - g.nz;
        }
        pw = p;
        return true;
    };
    // the warp's own row; one pair group of a staged halo row (rows 0, 1,
    // TY + 2, TY + 3) and of a first-colour halo row (rows 1, TY + 2) per warp
    const int rT = wy + 2;
    const int hs = wy & 3, uS = wy >> 2, rS = hs < 2 ? hs : TY + hs;
    const int uF = wy >> 1, rF = (wy & 1) ? TY + 2 : 1;
    int jT = 0, jS = 0, jF = 0;
    rowj(rT, jT);
    const bool hasS = uS < H, okS = hasS && rowj(rS, jS);
    const bool okF = uF < H && rowj(rF, jF);
    // whole rows wrap around the staged row; a segment's x-neighbours outside
    // it are the staged x-halo cells in the run-end slots
    const bool perx = SEG == 1 && g.bcx == LM_BC_PERIODIC;

    // x-halo of a segment (SEG > 1): threads 0 .. 4 NRW - 1 stage cell gG of
    // staged row rG (gG = 0..3: columns c0 - 2, c0 - 1, c0 + NX, c0 + NX + 1,
    // run slots E(-1), O(-1), E(M), O(M)); past a wall x = 0, rho = ROW_WALL
    const bool hasG = SEG > 1 && tid < 4 * NRW;
    const int rG = tid >> 2, gG = tid & 3;
    int gCol = c0 + (gG == 0 ? -2 : gG == 1 ? -1 : gG == 2 ? NX : NX + 1);
    bool gOK = true;
    if (gCol < 0 || gCol >= W) {
        if (g.bcx == LM_BC_PERIODIC) gCol = gCol < 0 ? gCol + W : gCol - W;
        else gOK = false;
    }
    const int gSlot = gG == 0 ? run_e(M, -1) : gG == 1 ? run_o(M, -1) : gG == 2 ? run_e(M, M) : run_o(M, M);
    float gxv = 0.f, grv = ROW_WALL, gev = 0.f;

    // staged plane: the own row (H pairs) and the halo pair, in registers
    float vx[CPT], vr[CPT], ve[CPT], sxh[2], srh[2], seh[2];
    auto fetch_pair = [&](int o, int pw, int jw, int u, float* X, float* R, float* E) {
        const float2 r2 = *reinterpret_cast<const float2*>(L.rho + o);
        R[0] = r2.x;
        R[1] = r2.y;
        if (!ZERO) {
            const float2 x2 = *reinterpret_cast<const float2*>(xin + o);
            X[0] = x2.x;
            X[1] = x2.y;
        } else {
            X[0] = X[1] = 0.f;
        }
        if (PROLONG) {
            const int po = C.nx * (jw >> hy) + C.nx * C.ny * (pw >> hz);
            E[0] = ec[po + ((c0 + 64 * u + i2) >> hx)];
            E[1] = ec[po + ((c0 + 64 * u + i2 + 1) >> hx)];
        }
    };
    auto wall_pair = [&](float* X, float* R, float* E) {
        X[0] = X[1] = 0.f;
        R[0] = R[1] = ROW_WALL;
        if (PROLONG) E[0] = E[1] = 0.f;
    };
    auto fetch = [&](int p) {
        int pw = 0;
        const bool okp = plane(p, pw);
#pragma unroll
        for (int u = 0; u < H; ++u) {
            if (okp) fetch_pair(sz * pw + W * jT + c0 + 64 * u + i2, pw, jT, u, vx + 2 * u, vr + 2 * u, ve + 2 * u);
            else wall_pair(vx + 2 * u, vr + 2 * u, ve + 2 * u);
        }
        if (hasS) {
            if (okp && okS) fetch_pair(sz * pw + W * jS + c0 + 64 * uS + i2, pw, jS, uS, sxh, srh, seh);
            else wall_pair(sxh, srh, seh);
        }
        if (SEG > 1 && hasG) {                            // x-halo cell gG of staged row rG
            int jw = 0;
            if (okp && rowj(rG, jw) && gOK) {
                const int o = sz * pw + W * jw + gCol;
                gxv = ZERO ? 0.f : xin[o];
                grv = L.rho[o];
                if (PROLONG) gev = ec[C.nx * (jw >> hy) + C.nx * C.ny * (pw >> hz) + (gCol >> hx)];
            } else {
                gxv = 0.f;
                grv = ROW_WALL;
                gev = 0.f;
            }
        }
    };
    // pair m = lane + 32 u of row r: cell 2 m to run E, cell 2 m + 1 to run O
    auto store_pair = [&](int b, int m, const float* X, const float* R, const float* E) {
        XR[b + run_e(M, m)] = make_float2(PROLONG ? X[0] + E[0] : X[0], R[0]);
        XR[b + run_o(M, m)] = make_float2(PROLONG ? X[1] + E[1] : X[1], R[1]);
    };
    auto store = [&](int s) {
#pragma unroll
        for (int u = 0; u < H; ++u) store_pair((s * NRW + rT) * RS, lane + 32 * u, vx + 2 * u, vr + 2 * u, ve + 2 * u);
        if (hasS) store_pair((s * NRW + rS) * RS, lane + 32 * uS, sxh, srh, seh);
        if (SEG > 1 && hasG) XR[(s * NRW + rG) * RS + gSlot] = make_float2(PROLONG ? gxv + gev : gxv, grv);
    };
    // f and c~ of cells 2 (lane + 32 u) + a, u < n, of a row at offset rowoff of plane p
    auto load_fc = [&](int p, bool ok, int rowoff, int a, float* F, float* Cv, int n) {
        int pw = 0;
        if (ok && plane(p, pw)) {
            const int o = sz * pw + rowoff + i2 + a;
#pragma unroll
            for (int u = 0; u < H; ++u)
                if (u < n) {
                    F[u] = f[o + 64 * u];
                    Cv[u] = L.ct[o + 64 * u];
                }
        } else {
#pragma unroll
            for (int u = 0; u < H; ++u)
                if (u < n) {
                    F[u] = 0.f;
                    Cv[u] = 1.f;
                }
        }
    };
    auto parity = [&](int j, int p, int col) -> int { return (col + j + p) & 1; };   // updated cell of each pair
    const int jTu = j0 + wy, jFu = (wy & 1) ? j0 + TY : j0 - 1;   // unwrapped rows (even periodic sizes)
    // L2 prefetch of the block's own TY rows (contiguous: one bulk request per
    // array and plane), PF_PLANES steps before their first use: x and rho of
    // plane P are staged at step P - 2, f and c~ first read at step P - 1.
    // Array a = 0..3 (x, rho, f, c~) is requested by thread a.
    // (a segment's rows are not contiguous: one request per row, thread
    // a * TY + r for array a and row r)
    constexpr int NPF = SEG == 1 ? 4 : 4 * TY;
    const int pfa = SEG == 1 ? tid : tid / TY, pfr = SEG == 1 ? 0 : tid % TY;
    auto prefetch = [&](int a, int P) {
        int pw = 0;
        if (P > (a < 2 ? k1 + 1 : k1) || (ZERO && a == 0) || !plane(P, pw)) return;
        const float* base = a == 0 ? xin : a == 1 ? L.rho : a == 2 ? f : L.ct;
        if (SEG == 1) prefetch_l2(base + sz * pw + NX * j0, NX * TY * sizeof(float));
        else prefetch_l2(base + sz * pw + W * (j0 + pfr) + c0, NX * sizeof(float));
    };
    if (tid < NPF)
        for (int d = 1; d <= PF_PLANES; ++d) prefetch(pfa, (pfa < 2 ? k0 : k0 - 1) + d);
    auto gs_row = [&](int a, int b, int dzm, int dzp, const float* F, const float* Cv) {
        if (a) gs_row_runs<CPT, 1>(XR, b, lane, perx, RS, dzm, dzp, F, Cv, L.c2x, L.c2y, L.c2z);
        else gs_row_runs<CPT, 0>(XR, b, lane, perx, RS, dzm, dzp, F, Cv, L.c2x, L.c2y, L.c2z);
    };
    // The first-colour x-halo cell of the warp's own row (SEG > 1): column
    // c0 - 1 when the row's first colour is odd, c0 + NX when even; lane 0
    // updates it with the first colour of its plane (the second-colour cells
    // at the segment's ends read it), f and c~ loaded a step ahead.
    float fX = 0.f, cX = 1.f;
    int xCol = 0;
    bool xOK = false;
    auto load_fcx = [&](int p) {
        if (SEG == 1 || lane != 0) return;
        int pw = 0;
        xOK = false;
        if (p > k1 || !plane(p, pw)) return;
        const int aT = parity(jTu, p, FIRST);
        int col = aT ? c0 - 1 : c0 + NX;
        if (col < 0 || col >= W) {
            if (g.bcx != LM_BC_PERIODIC) return;
            col = col < 0 ? col + W : col - W;
        }
        xCol = col;
        xOK = true;
        const int o = sz * pw + W * jT + col;
        fX = f[o];
        cX = L.ct[o];
    };
    float fT[H], cT[H], fS[H], cS[H], fF[1], cF[1];
#pragma unroll
    for (int u = 0; u < H; ++u) {
        fS[u] = 0.f;
        cS[u] = 1.f;
    }
    // prologue: planes k0 - 2 .. k0 staged; f, c~ of the first step's cells
    int sl = (k0 + 8) % NR;                               // ring slot of plane k0 - 2
    for (int p = k0 - 2; p <= k0; ++p) {
        fetch(p);
        store(sl);
        sl = sl + 1 == NR ? 0 : sl + 1;
    }
    // slots of planes p - 3 .. p + 1 at step p = k0 - 1 (rotated each step)
    int s_m3 = (k0 + 6) % NR, s_m2 = (k0 + 7) % NR, s_m1 = (k0 + 8) % NR, s_0 = (k0 + 9) % NR, s_p1 = (k0 + 10) % NR;
    load_fc(k0 - 1, true, W * jT + c0, parity(jTu, k0 - 1, FIRST), fT, cT, H);
    load_fc(k0 - 1, okF, W * jF + c0 + 64 * uF, parity(jFu, k0 - 1, FIRST), fF, cF, 1);
    load_fcx(k0 - 1);
    __syncthreads();
    for (int p = k0 - 1; p <= k1 + 2; ++p) {
        const bool stage = p + 2 <= k1 + 1;
        if (tid < NPF) prefetch(pfa, (pfa < 2 ? p + 2 : p + 1) + PF_PLANES);
        if (stage) fetch(p + 2);
        int pw = 0;
        if (p <= k1 && plane(p, pw)) {                    // first colour on plane p
            const int dzm = (s_m1 - s_0) * PL, dzp = (s_p1 - s_0) * PL;
            gs_row(parity(jTu, p, FIRST), (s_0 * NRW + rT) * RS, dzm, dzp, fT, cT);
            if (SEG > 1 && lane == 0 && xOK) {            // the own row's first-colour x-halo cell
                const int b = (s_0 * NRW + rT) * RS;
                if (parity(jTu, p, FIRST)) {
                    XR[b + run_o(M, -1)].x = gs_run<1>(XR, b, M, -1, false, RS, dzm, dzp, fX, cX, L.c2x, L.c2y, L.c2z);
                } else {
                    XR[b + run_e(M, M)].x = gs_run<0>(XR, b, M, M, false, RS, dzm, dzp, fX, cX, L.c2x, L.c2y, L.c2z);
                }
            }
            if (okF) {                                    // this warp's pair group of a halo row
                const int aF = parity(jFu, p, FIRST), b = (s_0 * NRW + rF) * RS, m = lane + 32 * uF;
                const bool wrapF = perx && (aF ? (uF == H - 1 && lane == 31) : (uF == 0 && lane == 0));
                const float v = aF ? gs_run<1>(XR, b, M, m, wrapF, RS, dzm, dzp, fF[0], cF[0], L.c2x, L.c2y, L.c2z)
                                   : gs_run<0>(XR, b, M, m, wrapF, RS, dzm, dzp, fF[0], cF[0], L.c2x, L.c2y, L.c2z);
                XR[b + (aF ? run_o(M, m) : run_e(M, m))].x = v;
            }
        }
        load_fc(p + 1, p + 1 <= k1, W * jT + c0, parity(jTu, p + 1, FIRST), fT, cT, H);
        load_fc(p + 1, okF && p + 1 <= k1, W * jF + c0 + 64 * uF, parity(jFu, p + 1, FIRST), fF, cF, 1);
        load_fcx(p + 1);
        const int q = p - 2;
        if (q >= k0 && q < k1)                            // second colour on plane p - 2
            gs_row(parity(jTu, q, 1 - FIRST), (s_m2 * NRW + rT) * RS, (s_m3 - s_m2) * PL, (s_m1 - s_m2) * PL, fS,
                   cS);
        load_fc(q + 1, q + 1 >= k0 && q + 1 < k1, W * jT + c0, parity(jTu, q + 1, 1 - FIRST), fS, cS, H);
        if (p - 3 >= k0 && p - 3 < k1) {                  // plane p - 3 is final
            const int b = (s_m3 * NRW + rT) * RS;
            float* dst = xout + sz * (p - 3) + W * jT + c0 + i2;
#pragma unroll
            for (int u = 0; u < H; ++u) {
                const int m = lane + 32 * u;
                *reinterpret_cast<float2*>(dst + 64 * u) = make_float2(XR[b + run_e(M, m)].x, XR[b + run_o(M, m)].x);
            }
        }
        if (stage) store(s_m3);                           // plane p + 2 takes plane p - 3's slot
        __syncthreads();
        const int t = s_m3;
        s_m3 = s_m2;
        s_m2 = s_m1;
        s_m1 = s_0;
        s_0 = s_p1;
        s_p1 = t;
    }
}

template <int FIRST, bool ZERO, bool PROLONG>
__global__ void __launch_bounds__(128, 8) k_rbgs_zm2d(Lev32 L, const float* __restrict__ xin,
                                                  const float* __restrict__ ec, Geo C, int hx, int hz,
                                                  const float* __restrict__ f, float* __restrict__ xout, int KZ,
                                                  int TW) {
    zrow2d_tile<FIRST, ZERO, PROLONG>(L, xin, ec, C, hx, hz, f, xout, KZ, blockIdx.x, blockIdx.y, TW);
}

template <int BX, int TY, bool HAS_Y, int FIRST, bool ZERO, bool PROLONG>
__global__ void __launch_bounds__(BX * TY, 1024 / (BX * TY)) k_rbgs(Lev32 L, const float* __restrict__ xin,
                                                                   const float* __restrict__ ec, Geo C, int hx,
                                                                   int hy, int hz, const float* __restrict__ f,
                                                                   float* __restrict__ xout, int KZ) {
    rbgs_tile<BX, TY, HAS_Y, FIRST, ZERO, PROLONG>(L, xin, ec, C, hx, hy, hz, f, xout, KZ, blockIdx.x, blockIdx.y,
                                                   blockIdx.z);
}

// Row b = blockIdx.x of the inverse of the dense coarsest operator (n <= 64),
// in float64.  Every block factors A = L L^T (right-looking Cholesky) and
// carries the forward solve of L y = e_b along; one warp then solves
// L^T z = y.  A^-1 is symmetric, so z is row b as well as column b.  GB300
// issues float64 at 1/64 of the float32 rate, so the factorisation is spread
// over n SMs (one block each) instead of one Gauss-Jordan block, and every
// trailing update runs with all lanes busy: the lower triangle of the
// trailing block is enumerated through a packed (i, j) table ordered so that
// the step-k triangle is a prefix of it.
__device__ __forceinline__ void coarse_inverse_row(const Lev32& L, float* __restrict__ ainv, int b) {
    __shared__ double A[64 * 64];
    __shared__ double y[64], yf[64], rinv[64];      // y: forward-solve updates; yf: final values
    __shared__ int tri[64 * 65 / 2];
    const Geo& g = L.g;
    const int n = g.N, tid = threadIdx.x;
    for (int e = tid; e < n * n; e += 256) {
        A[e] = 0.0;
        const int i = e / n, j = e - i * n;
        // column j from the last: (n - 1 - j)(n - j) / 2 entries come before it
        if (i >= j) tri[(n - 1 - j) * (n - j) / 2 + (i - j)] = (i << 8) | j;
    }
    if (tid < n) y[tid] = tid == b ? 1.0 : 0.0;
    __syncthreads();
    if (tid < n) {
        const int idx = tid;
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
    for (int k = 0; k < n; ++k) {
        // 1/sqrt(pivot), formed by each thread of rows k.. (float seed, one
        // Newton step in float64: relative error ~1e-13, far below the float32
        // the inverse is stored in); column k of L and the forward-solve step
        const int i = k + tid;
        if (i < n) {
            const double p = A[k * n + k];
            const float pf = (float)p;
            double r;
            if (pf > 1e-30f && pf < 1e30f) {
                const double r0 = (double)rsqrtf(pf);
                r = r0 * fma(-0.5 * p * r0, r0, 1.5);
            } else {
                r = 1.0 / sqrt(p);
            }
            const double yk = y[k] * r;                 // y[k] itself is not written in this phase
            if (i == k) {
                rinv[k] = r;
                yf[k] = yk;
            } else {
                const double l = A[i * n + k] * r;
                A[i * n + k] = l;
                y[i] -= l * yk;
            }
        }
        __syncthreads();
        const int m = n - 1 - k;
#pragma unroll 4
        for (int e = tid; e < m * (m + 1) / 2; e += 256) {
            const int t = tri[e], ti = t >> 8, tj = t & 255;
            A[ti * n + tj] -= A[ti * n + k] * A[tj * n + k];
        }
        __syncthreads();
    }
    if (tid < 32) {                                      // L^T z = y; lane owns rows tid, tid + 32
        double z0 = tid < n ? yf[tid] : 0.0, z1 = tid + 32 < n ? yf[tid + 32] : 0.0;
        for (int m = n - 1; m >= 0; --m) {
            const double zm = __shfl_sync(0xffffffffu, m < 32 ? z0 : z1, m & 31) * rinv[m];
            if ((m & 31) == tid) {
                if (m < 32) z0 = zm;
                else z1 = zm;
            }
            if (tid < m) z0 -= A[m * n + tid] * zm;
            if (tid + 32 < m) z1 -= A[m * n + tid + 32] * zm;
        }
        if (tid < n) ainv[b * n + tid] = (float)z0;
        if (tid + 32 < n) ainv[b * n + tid + 32] = (float)z1;
    }
}

__global__ void __launch_bounds__(256) k_coarse_inverse(Lev32 L, float* __restrict__ ainv) {
    coarse_inverse_row(L, ainv, blockIdx.x);
}

// The inverses of several grids' coarsest levels in one launch: block t
// computes row (task[t] & 255) of item (task[t] >> 8).
__global__ void __launch_bounds__(256) k_coarse_inverse_many(const CoarseInv* __restrict__ items,
                                                             const int* __restrict__ task) {
    const int t = task[blockIdx.x];
    const CoarseInv& it = items[t >> 8];
    coarse_inverse_row(it.L, it.ainv, t & 255);
}

// The whole inverse of one grid's dense coarsest operator (n <= 64) in one
// block: the factorisation of coarse_inverse_row done once, then thread t
// solves L y = e_t (y_i = 0 above row t) and L^T z = y for column t of A^-1
// (= row t, A^-1 being symmetric).  For many grids at once this does 1/n of
// the per-row kernel's float64 factorisation work.
constexpr size_t COARSE_INV_SMEM = sizeof(double) * (2 * 64 * 64 + 64) + sizeof(int) * (64 * 65 / 2);
__device__ __forceinline__ void coarse_inverse_block(const Lev32& L, float* __restrict__ ainv) {
    extern __shared__ double cinv_smem[];           // COARSE_INV_SMEM bytes
    double* A = cinv_smem;
    double* Y = A + 64 * 64;                        // Y[i * 64 + t]: entry i of thread t's column
    double* rinv = Y + 64 * 64;
    int* tri = reinterpret_cast<int*>(rinv + 64);
    const Geo& g = L.g;
    const int n = g.N, tid = threadIdx.x;
    for (int e = tid; e < n * n; e += blockDim.x) {
        A[e] = 0.0;
        const int i = e / n, j = e - i * n;
        if (i >= j) tri[(n - 1 - j) * (n - j) / 2 + (i - j)] = (i << 8) | j;
    }
    __syncthreads();
    if (tid < n) {
        const int idx = tid;
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
    for (int k = 0; k < n; ++k) {                   // right-looking Cholesky, as in coarse_inverse_row
        const int i = k + tid;
        if (i < n) {
            const double p = A[k * n + k];
            const float pf = (float)p;
            double r;
            if (pf > 1e-30f && pf < 1e30f) {
                const double r0 = (double)rsqrtf(pf);
                r = r0 * fma(-0.5 * p * r0, r0, 1.5);
            } else {
                r = 1.0 / sqrt(p);
            }
            if (i == k) rinv[k] = r;
            else A[i * n + k] *= r;
        }
        __syncthreads();
        const int m = n - 1 - k;
        for (int e = tid; e < m * (m + 1) / 2; e += blockDim.x) {
            const int t = tri[e], ti = t >> 8, tj = t & 255;
            A[ti * n + tj] -= A[ti * n + k] * A[tj * n + k];
        }
        __syncthreads();
    }
    if (tid < n) {
        const int t = tid;
        for (int i = t; i < n; ++i) {               // L y = e_t
            double sum = i == t ? 1.0 : 0.0;
            for (int j = t; j < i; ++j) sum -= A[i * n + j] * Y[j * 64 + t];
            Y[i * 64 + t] = sum * rinv[i];
        }
        for (int i = n - 1; i >= 0; --i) {          // L^T z = y (z over y, in place)
            double sum = i >= t ? Y[i * 64 + t] : 0.0;
            for (int j = i + 1; j < n; ++j) sum -= A[j * n + i] * Y[j * 64 + t];
            Y[i * 64 + t] = sum * rinv[i];
        }
        for (int i = 0; i < n; ++i) ainv[t * n + i] = (float)Y[i * 64 + t];
    }
}

// One block per grid: the inverses of many grids' coarsest levels.
__global__ void __launch_bounds__(256) k_coarse_inverse_grids(const CoarseInv* __restrict__ items) {
    const CoarseInv& it = items[blockIdx.x];
    coarse_inverse_block(it.L, it.ainv);
}

__global__ void k_coarse_solve(int n, const float* __restrict__ ainv, const float* __restrict__ f,
                               float* __restrict__ x) {
    coarse_solve_block(n, ainv, f, x);
}

// ---- the coarse V-cycle in one block ------------------------------------------
// The V-cycle below a level of at most CC_MAX_CELLS cells, run by one block of
// 1024 threads: per level, nu1 red-black sweeps from zero (in place, the two
// colours separated by a barrier, so the result equals the fused sweeps'),
// the residual restricted to the next level's rhs, recursion, then the
// prolonged correction and nu2 black-red sweeps; the coarsest level is
// solved with its dense inverse.  Replaces ~3 launches per level and sweep
// that are all latency-bound at these sizes; the chain lives in shared memory
// (cc_smem_bytes), so only the setup and the final store touch global memory.
__global__ void __launch_bounds__(CC_THREADS, 1) k_coarse_cycle(CoarseCycle cc) { coarse_cycle_block(cc); }

// ---- host launchers -----------------------------------------------------------

static inline int hdiv(int a, int b) { return (a + b - 1) / b; }

static dim3 cell_grid(const Geo& g) {
    return g.ny > 1 ? dim3(hdiv(g.nx, 32), hdiv(g.ny, 8), g.nz) : dim3(hdiv(g.nx, 32), hdiv(g.nz, 8), 1);
}

// fc = mean over the 2 x 2 x 2 children of (f - A x), on whole rows: the
// staging and stencil of k_apply32_row; a thread adds the residuals of its
// cells over a plane pair, lanes 2 i and 2 i + 1 combine the x pair by a
// shuffle, and the odd row of each row pair stores its sums in fc, which the
// even row adds to its own and scales at the next step (after the step's
// barrier).  For levels halved along all three axes.
template <int CPT, int TY, int SEG = 1>
__global__ void __launch_bounds__(32 * TY, 1) k_resid_restrict_row(Lev32 L, Geo C, const float* __restrict__ x,
                                                                  const float* __restrict__ f,
                                                                  float* __restrict__ fc, int KZ) {
    constexpr int NX = 32 * CPT, RS = NX + 4, NRW = TY + 2, PL = NRW * RS, H = CPT / 2;
    static_assert(CPT % 2 == 0 && TY % 2 == 0 && TY >= 2 * H, "row pairs; a warp per halo pair group");
    constexpr int W = NX * SEG;                           // cells in a grid row
    static_assert(SEG == 1 || (SEG == 2 && 2 * NRW <= 32 * TY && 4 * TY <= 32 * TY), "x-halo threads");
    extern __shared__ float4 ap_smem[];
    float2* XR = reinterpret_cast<float2*>(ap_smem);
    const Geo& g = L.g;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = lane + 32 * wy;
    const int j0 = (blockIdx.x / SEG) * TY, c0 = (blockIdx.x % SEG) * NX, k0 = blockIdx.y * KZ,
              k1 = min(k0 + KZ, g.nz);
    const int sz = W * g.ny, i2 = 2 * lane;
    const float INF = __int_as_float(0x7f800000);
    for (int t = tid; t < 4 * NRW; t += 32 * TY) {
        XR[t * RS + 1] = make_float2(0.f, INF);
        XR[t * RS + NX + 2] = make_float2(0.f, INF);
    }
    if (SEG > 1) __syncthreads();                         // segments stage those slots: after the walls
    auto rowj = [&](int r_, int& jw) -> bool {
        int j = j0 - 1 + r_;
        if (j < 0 || j >= g.ny) {
            if (g.bcy != LM_BC_PERIODIC) return false;
            j = j < 0 ? j + g.ny : j - g.ny;
        }
        jw = j;
        return true;
    };
    auto plane = [&](int p, int& pw) -> bool {
        if (p < 0 || p >= g.nz) {
            if (g.bcz != LM_BC_PERIODIC) return false;
            p = p < 0 ? p + g.nz : p - g.nz;
        }
        pw = p;
        return true;
    };
    const int rT = wy + 1;
    const int uS = wy >> 1, rS = (wy & 1) ? TY + 1 : 0;
    int jT = 0, jS = 0;
    rowj(rT, jT);
    const bool hasS = uS < H, okS = hasS && rowj(rS, jS);
    // a segment's x-neighbours outside it: staged into the row-end slots (as in k_apply32_row)
    const bool perx = SEG == 1 && g.bcx == LM_BC_PERIODIC;
    const bool hasG = SEG > 1 && tid < 2 * NRW;
    const int rG = tid >> 1, gG = tid & 1;
    int gCol = gG ? c0 + NX : c0 - 1;
    bool gOK = true;
    if (gCol < 0 || gCol >= W) {
        if (g.bcx == LM_BC_PERIODIC) gCol = gCol < 0 ? gCol + W : gCol - W;
        else gOK = false;
    }
    float gxv = 0.f, grv = INF;
    float vx[CPT], vr[CPT], hx2[2], hr2[2];
    auto fetch = [&](int p) {
        int pw = 0;
        const bool okp = plane(p, pw);
#pragma unroll
        for (int u = 0; u < H; ++u) {
            if (okp) {
                const int o = sz * pw + W * jT + c0 + 64 * u + i2;
                const float2 a = *reinterpret_cast<const float2*>(x + o), b = *reinterpret_cast<const float2*>(L.rho + o);
                vx[2 * u] = a.x; vx[2 * u + 1] = a.y; vr[2 * u] = b.x; vr[2 * u + 1] = b.y;
            } else {
                vx[2 * u] = vx[2 * u + 1] = 0.f;
                vr[2 * u] = vr[2 * u + 1] = INF;
            }
        }
        if (hasS) {
            if (okp && okS) {
                const int o = sz * pw + W * jS + c0 + 64 * uS + i2;
                const float2 a = *reinterpret_cast<const float2*>(x + o), b = *reinterpret_cast<const float2*>(L.rho + o);
                hx2[0] = a.x; hx2[1] = a.y; hr2[0] = b.x; hr2[1] = b.y;
            } else {
                hx2[0] = hx2[1] = 0.f;
                hr2[0] = hr2[1] = INF;
            }
        }
        if (SEG > 1 && hasG) {
            int jw = 0;
            if (okp && rowj(rG, jw) && gOK) {
                const int o = sz * pw + W * jw + gCol;
                gxv = x[o];
                grv = L.rho[o];
            } else {
                gxv = 0.f;
                grv = INF;
            }
        }
    };
    auto store = [&](int s) {
#pragma unroll
        for (int u = 0; u < H; ++u)
            *reinterpret_cast<float4*>(XR + (s * NRW + rT) * RS + 2 + 64 * u + i2) =
                make_float4(vx[2 * u], vr[2 * u], vx[2 * u + 1], vr[2 * u + 1]);
        if (hasS)
            *reinterpret_cast<float4*>(XR + (s * NRW + rS) * RS + 2 + 64 * uS + i2) =
                make_float4(hx2[0], hr2[0], hx2[1], hr2[1]);
        if (SEG > 1 && hasG) XR[(s * NRW + rG) * RS + (gG ? NX + 2 : 1)] = make_float2(gxv, grv);
    };
    float ctv[CPT], fv[CPT], acc[CPT];
    auto load_c = [&](int p) {
        const int o = sz * p + W * jT + c0 + lane;
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
            ctv[v] = L.ct[o + 32 * v];
            fv[v] = f[o + 32 * v];
        }
    };
    const int lrel = (lane == 0 && perx) ? NX - 1 : -1;
    const int rrel = (lane == 31 && perx) ? 1 - NX : 1;
    // L2 prefetch as in k_apply32_row; arrays x, rho, c~, f
    constexpr int NPF = SEG == 1 ? 4 : 4 * TY;
    const int pfa = SEG == 1 ? tid : tid / TY, pfr = SEG == 1 ? 0 : tid % TY;
    auto prefetch = [&](int a, int P) {
        int pw = 0;
        if (P > (a < 2 ? k1 : k1 - 1) || !plane(P, pw)) return;
        const float* base = a == 0 ? x : a == 1 ? L.rho : a == 2 ? L.ct : f;
        if (SEG == 1) prefetch_l2(base + sz * pw + NX * j0, NX * TY * sizeof(float));
        else prefetch_l2(base + sz * pw + W * (j0 + pfr) + c0, NX * sizeof(float));
    };
    if (tid < NPF)
        for (int d = 1; d <= PF_PLANES; ++d) prefetch(pfa, (pfa < 2 ? k0 + 1 : k0) + d);
    int sm1 = 0, s0 = 1, sp1 = 2, sp2 = 3;
    // an even row's pair sums wait one step (one barrier) for the odd row's
    float accP[CPT];
    float* dstP = nullptr;
    fetch(k0 - 1);
    store(sm1);
    fetch(k0);
    store(s0);
    fetch(k0 + 1);
    store(sp1);
    load_c(k0);
    __syncthreads();
    auto finish_pairs = [&]() {                           // even row: add the odd row's sums, scale
        if (dstP) {
#pragma unroll
            for (int v = 0; v < CPT; ++v) dstP[16 * v] = (accP[v] + dstP[16 * v]) * 0.125f;
            dstP = nullptr;
        }
    };
    for (int p = k0; p < k1; ++p) {
        const bool stage = p + 2 <= k1;
        if (tid < NPF) prefetch(pfa, (pfa < 2 ? p + 2 : p + 1) + PF_PLANES);
        if (stage) fetch(p + 2);
        finish_pairs();
        const int b0 = (s0 * NRW + rT) * RS + 2 + lane, dzm = (sm1 - s0) * PL, dzp = (sp1 - s0) * PL;
        const bool odd = (p - k0) & 1;                    // second plane of a pair (k0 is even)
#pragma unroll
        for (int v = 0; v < CPT; ++v) {
            const int c = b0 + 32 * v;
            const float2 me = XR[c];
            const float2 xm = XR[c + (v == 0 ? lrel : -1)], xp = XR[c + (v == CPT - 1 ? rrel : 1)];
            const float2 ym = XR[c - RS], yp = XR[c + RS], zm = XR[c + dzm], zp = XR[c + dzp];
            float val = ctv[v] * me.x;
            val += L.c2x * rcp_approx(me.y + xm.y) * (me.x - xm.x);
            val += L.c2x * rcp_approx(me.y + xp.y) * (me.x - xp.x);
            val += L.c2y * rcp_approx(me.y + ym.y) * (me.x - ym.x);
            val += L.c2y * rcp_approx(me.y + yp.y) * (me.x - yp.x);
            val += L.c2z * rcp_approx(me.y + zm.y) * (me.x - zm.x);
            val += L.c2z * rcp_approx(me.y + zp.y) * (me.x - zp.x);
            const float rv = fv[v] - val;
            acc[v] = odd ? acc[v] + rv : rv;
        }
        float* const dst = fc + C.nx * (((j0 + wy) >> 1) + C.ny * (p >> 1)) + (c0 >> 1) + (lane >> 1);
        if (odd) {                                        // x pairs; the odd row's sums to fc
#pragma unroll
            for (int v = 0; v < CPT; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], 1);
            if (!(lane & 1)) {
                if (wy & 1) {
#pragma unroll
                    for (int v = 0; v < CPT; ++v) dst[16 * v] = acc[v];
                } else {
#pragma unroll
                    for (int v = 0; v < CPT; ++v) accP[v] = acc[v];
                    dstP = dst;
                }
            }
        }
        if (p + 1 < k1) load_c(p + 1);
        if (stage) store(sp2);
        __syncthreads();
        const int t = sm1;
        sm1 = s0;
        s0 = sp1;
        sp1 = sp2;
        sp2 = t;
    }
    finish_pairs();                                       // the last step ended with a barrier
}

template <int CPT, int SEG = 1>
static void launch_resid_restrict_row(const Lev32& F, const Geo& C, cudaStream_t s, const float* x, const float* f,
                                      float* fc) {
    constexpr int TY = 16;
    const Geo& g = F.g;
    const int ntile = g.ny / TY * SEG;
    int chunks = std::max(1, std::min(g.nz / 2, 152 / ntile));
    int KZ = hdiv(g.nz, chunks);
    KZ += KZ & 1;                                         // chunks start on even planes
    const dim3 grd(ntile, hdiv(g.nz, KZ)), blk(32, TY);
    const size_t sm = apply_row_smem<CPT, TY>();
    count_launches(1);
    k_resid_restrict_row<CPT, TY, SEG><<<grd, blk, sm, s>>>(F, C, x, f, fc, KZ);
}

template <int CPT, int SEG = 1>
static void launch_apply32_row(const Lev32& L, cudaStream_t s, const float* x, float* y, const float* r,
                               const Red& red, int slot_xy, int slot_xr) {
    constexpr int TY = 16;
    const Geo& g = L.g;
    const int ntile = g.ny / TY * SEG;
    const int chunks = std::max(1, std::min(g.nz / 2, 152 / ntile));
    const int KZ = hdiv(g.nz, chunks);
    const dim3 grd(ntile, hdiv(g.nz, KZ)), blk(32, TY);
    const size_t sm = apply_row_smem<CPT, TY>();
    const bool dxy = slot_xy >= 0, dxr = slot_xr >= 0;
    count_launches(1);
#define LM_AR(A, B) k_apply32_row<CPT, TY, A, B, SEG><<<grd, blk, sm, s>>>(L, x, y, r, red, slot_xy, slot_xr, KZ)
    if (dxy && dxr) LM_AR(true, true);
    else if (dxy) LM_AR(true, false);
    else LM_AR(false, false);
#undef LM_AR
}

void launch_apply32(const Lev32& L, cudaStream_t s, const float* x, float* y, const float* r, const Red& red,
                    int slot_xy, int slot_xr) {
    const Geo& g = L.g;
    if (g.ny > 1 && g.ny % 16 == 0 && g.nz >= 2 && (g.nx == 512 || g.nx == 256 || g.nx == 128) &&
        ((uintptr_t)x & 7) == 0) {
        // whole rows of 256 or 128 cells, or 512-cell rows as two 256-cell
        // segments with an x-halo: a warp per row, 16 rows per block
        if (g.nx == 512) launch_apply32_row<8, 2>(L, s, x, y, r, red, slot_xy, slot_xr);
        else if (g.nx == 256) launch_apply32_row<8>(L, s, x, y, r, red, slot_xy, slot_xr);
        else launch_apply32_row<4>(L, s, x, y, r, red, slot_xy, slot_xr);
        return;
    }
    if (g.ny > 1 && g.nx % 32 == 0 && g.ny % 8 == 0 && g.nz >= 2) {
        // whole TX x 8 tiles: the staged z-march; KZ planes per block, the
        // largest of 64, 32, ..., 2 that still gives eight blocks per SM
        const int TXc = g.nx % 64 == 0 ? 64 : 32;
        const long long tiles = (long long)(g.nx / TXc) * (g.ny / 8);
        int KZ = 64;
        while (KZ > 2 && tiles * hdiv(g.nz, KZ) < 8 * 152) KZ /= 2;
        const dim3 grd(g.nx / TXc, g.ny / 8, hdiv(g.nz, KZ)), blk(32, 8);
        count_launches(1);
        const bool dxy = slot_xy >= 0, dxr = slot_xr >= 0;
#define LM_AZ(T, A, B) k_apply32_zm<T, A, B><<<grd, blk, 0, s>>>(L, x, y, r, red, slot_xy, slot_xr, KZ)
#define LM_AZT(T)                              \
    if (dxy && dxr) LM_AZ(T, true, true);      \
    else if (dxy) LM_AZ(T, true, false);       \
    else LM_AZ(T, false, false);
        if (TXc == 64) { LM_AZT(64) } else { LM_AZT(32) }
#undef LM_AZT
#undef LM_AZ
        return;
    }
    if (seg2d_ok(g, x, y, L.rho, L.ct, slot_xr >= 0 ? r : nullptr) && (long long)(g.nx / 128) * g.nz >= 16 * 152) {
        // 2D rows of 128-column segments: a warp per segment and KR rows, KR
        // as large as still gives about 32 warps per SM (grids too small for
        // 16 warps per SM at one row a warp take the thread-per-column walk
        // below, whose 32-column warps give more parallelism)
        const int segs = g.nx / 128;
        int KR = 16;
        while (KR > 1 && (long long)segs * hdiv(g.nz, KR) < 32 * 152) KR /= 2;
        const dim3 grd(segs, hdiv(g.nz, 8 * KR)), blk(32, 8);
        count_launches(1);
        if (slot_xy >= 0 && slot_xr >= 0) k_apply32_2d<true, true><<<grd, blk, 0, s>>>(L, x, y, r, red, slot_xy, slot_xr, KR);
        else if (slot_xy >= 0) k_apply32_2d<true, false><<<grd, blk, 0, s>>>(L, x, y, r, red, slot_xy, slot_xr, KR);
        else k_apply32_2d<false, false><<<grd, blk, 0, s>>>(L, x, y, r, red, slot_xy, slot_xr, KR);
        return;
    }
    const dim3 blk(32, 8);
    const bool y3 = g.ny > 1;
    int kz = 1;
    auto grid_for = [&](int k) {
        return y3 ? dim3(hdiv(g.nx, 32), hdiv(g.ny, 8), hdiv(g.nz, k))
                  : dim3(hdiv(g.nx, 32), hdiv(hdiv(g.nz, k), 8), 1);
    };
    auto nblocks = [&](int k) { return (long long)grid_for(k).x * grid_for(k).y * grid_for(k).z; };
    if (!y3)            // 2D: up to 8 rows per thread while two blocks per SM remain
        for (int k = 8; k > 1; k /= 2)
            if (nblocks(k) >= 2 * 152) {
                kz = k;
                break;
            }
    while (nblocks(kz) > 4096) kz *= 2;
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
    const Geo& g = F.g;
    if (hx && hy && hz && g.ny % 16 == 0 && g.nz % 2 == 0 && (g.nx == 512 || g.nx == 256 || g.nx == 128) &&
        ((uintptr_t)x & 7) == 0) {
        // whole rows of 256 or 128 cells, or 512-cell rows as two 256-cell
        // segments with an x-halo: a warp per row, 16 rows per block
        if (g.nx == 512) launch_resid_restrict_row<8, 2>(F, C.g, s, x, f, fc);
        else if (g.nx == 256) launch_resid_restrict_row<8>(F, C.g, s, x, f, fc);
        else launch_resid_restrict_row<4>(F, C.g, s, x, f, fc);
        return;
    }
    count_launches(1);
    if (rr2d_ok(F, hx, hy, hz, x, f, fc) && (long long)(g.nx / 128) * C.g.nz >= 16 * 152) {
        // 2D rows: a warp per 128-column segment and KR coarse rows, KR as
        // large as still gives about 32 warps per SM (smaller grids: the
        // thread-per-coarse-cell kernel below)
        const int segs = g.nx / 128;
        int KR = 8;
        while (KR > 1 && (long long)segs * hdiv(C.g.nz, KR) < 32 * 152) KR /= 2;
        k_resid_restrict_2d<<<dim3(segs, hdiv(C.g.nz, 8 * KR)), dim3(32, 8), 0, s>>>(F, C.g, x, f, fc, KR);
        return;
    }
    if (g.ny > 1 && g.nx % 32 == 0 && g.ny % 8 == 0 && g.nz >= 2 && (!hz || g.nz % 2 == 0)) {
        // whole TX x 8 tiles: the staged z-march; KZ (even) planes per block
        const int TXc = g.nx % 64 == 0 ? 64 : 32;
        const long long tiles = (long long)(g.nx / TXc) * (g.ny / 8);
        int KZ = 64;
        while (KZ > 2 && tiles * hdiv(g.nz, KZ) < 8 * 152) KZ /= 2;
        const dim3 grd(g.nx / TXc, g.ny / 8, hdiv(g.nz, KZ)), blk(32, 8);
        if (TXc == 64) k_resid_restrict_zm<64><<<grd, blk, 0, s>>>(F, C.g, hx, hy, hz, x, f, fc, KZ);
        else k_resid_restrict_zm<32><<<grd, blk, 0, s>>>(F, C.g, hx, hy, hz, x, f, fc, KZ);
        return;
    }
    k_resid_restrict<<<cell_grid(C.g), dim3(32, 8), 0, s>>>(F, C.g, hx, hy, hz, x, f, fc);
}

// The whole-row sweep's shared memory exceeds the default 48 KB: raise the
// limit of every instantiation (host, once per hierarchy build).
template <int CPT, int TY, int SEG = 1>
static void rbgs_row_allow() {
    const int sm = (int)rbgs_row_smem<CPT, TY>();
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 0, false, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 1, false, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 0, true, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 1, true, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 0, false, true, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_rbgs_row<CPT, TY, 1, false, true, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}
template <int CPT, int TY, int SEG = 1>
static void apply_row_allow() {
    const int sm = (int)apply_row_smem<CPT, TY>();
    cudaFuncSetAttribute(k_apply32_row<CPT, TY, true, true, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_apply32_row<CPT, TY, true, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_apply32_row<CPT, TY, false, false, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}
void rbgs_row_allow_smem() {
    rbgs_row_allow<8, 16>();
    rbgs_row_allow<4, 16>();
    rbgs_row_allow<8, 16, 2>();
    apply_row_allow<8, 16>();
    apply_row_allow<4, 16>();
    apply_row_allow<8, 16, 2>();
    cudaFuncSetAttribute(k_resid_restrict_row<8, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)apply_row_smem<8, 16>());
    cudaFuncSetAttribute(k_resid_restrict_row<4, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)apply_row_smem<4, 16>());
    cudaFuncSetAttribute(k_resid_restrict_row<8, 16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)apply_row_smem<8, 16>());
}

static bool aligned8(const void* p) { return ((uintptr_t)p & 7) == 0; }

template <int CPT, int SEG = 1>
static void launch_rbgs_row(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Geo& Cg,
                            int hx, int hy, int hz, const float* f, float* xout, int first, int zero, int prolong) {
    constexpr int TY = 16;
    const Geo& g = L.g;
    const int ntile = g.ny / TY * SEG;
    // z chunks (one block per SM fits): the count that maximises the busy
    // fraction of the last wave times the share of planes a chunk does not
    // stage twice (KZ / (KZ + 4))
    int KZ = g.nz;
    double best = -1.0;
    for (int c = 1; c <= std::max(1, g.nz / 2); ++c) {
        const int kz = hdiv(g.nz, c), blocks = ntile * hdiv(g.nz, kz);
        const double eff = (double)blocks / (hdiv(blocks, 152) * 152.0) * kz / (kz + 4.0);
        if (eff > best + 1e-9) {
            best = eff;
            KZ = kz;
        }
    }
    const dim3 grd(ntile, hdiv(g.nz, KZ)), blk(32, TY);
    const size_t sm = rbgs_row_smem<CPT, TY>();
#define LM_ROW(F, Z, P) k_rbgs_row<CPT, TY, F, Z, P, SEG><<<grd, blk, sm, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
    if (zero) { if (first) LM_ROW(1, true, false); else LM_ROW(0, true, false); }
    else if (prolong) { if (first) LM_ROW(1, false, true); else LM_ROW(0, false, true); }
    else { if (first) LM_ROW(1, false, false); else LM_ROW(0, false, false); }
#undef LM_ROW
}

// One red-black sweep xout = S(xin [+ P ec]); first = colour updated first;
// kz = planes per block (<= 0: enough blocks to fill the GPU).
void launch_rbgs_kz(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx,
                    int hy, int hz, const float* f, float* xout, int first, int zero, int prolong, int kz) {
    const Geo& g = L.g;
    const Geo Cg = C ? C->g : g;
    count_launches(1);
    if (kz <= 0 && g.ny > 1 && g.ny % 16 == 0 && g.nz >= 2 && (g.nx == 512 || g.nx == 256 || g.nx == 128) &&
        aligned8(xin) && aligned8(xout) && aligned8(ec)) {
        // whole rows of 256 or 128 cells, or 512-cell rows as two 256-cell
        // segments with an x-halo: a warp per row, 16 rows per block
        if (g.nx == 512) launch_rbgs_row<8, 2>(L, s, xin, ec, Cg, hx, hy, hz, f, xout, first, zero, prolong);
        else if (g.nx == 256) launch_rbgs_row<8>(L, s, xin, ec, Cg, hx, hy, hz, f, xout, first, zero, prolong);
        else launch_rbgs_row<4>(L, s, xin, ec, Cg, hx, hy, hz, f, xout, first, zero, prolong);
        return;
    }
    if (g.ny > 1 && g.nx % 32 == 0 && g.ny % 8 == 0 && g.nz >= 2) {
        // whole TX x 8 tiles (TX = 64 when nx allows, else 32): the in-place
        // z-march; KZ planes per block, the largest of 64, 32, ..., 2 that
        // still gives eight blocks per SM (small levels are latency-bound:
        // short chunks, more blocks)
        const int TXc = g.nx % 64 == 0 ? 64 : 32;
        const long long tiles = (long long)(g.nx / TXc) * (g.ny / 8);
        int KZ = kz > 0 ? kz : 64;
        if (kz <= 0)
            while (KZ > 2 && tiles * hdiv(g.nz, KZ) < 8 * 152) KZ /= 2;
        const dim3 grd(g.nx / TXc, g.ny / 8, hdiv(g.nz, KZ)), blk(32, 8);
#define LM_RBZ(T, F, Z, P) k_rbgs_zm<T, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
#define LM_RBZT(T)                                                                                   \
    if (zero) { if (first) LM_RBZ(T, 1, true, false); else LM_RBZ(T, 0, true, false); }            \
    else if (prolong) { if (first) LM_RBZ(T, 1, false, true); else LM_RBZ(T, 0, false, true); }    \
    else { if (first) LM_RBZ(T, 1, false, false); else LM_RBZ(T, 0, false, false); }
        if (TXc == 64) { LM_RBZT(64) } else { LM_RBZT(32) }
#undef LM_RBZT
#undef LM_RBZ
    } else if (g.ny > 1) {
        constexpr int BX = 32, TY = 8;
        const int tiles = hdiv(g.nx, 2 * BX) * hdiv(g.ny, TY);
        int KZ = kz;
        if (KZ <= 0) {
            KZ = 16;
            while (KZ > 1 && (long long)tiles * hdiv(g.nz, KZ) < 1216) KZ /= 2;
        }
        const dim3 grd(hdiv(g.nx, 2 * BX), hdiv(g.ny, TY), hdiv(g.nz, KZ)), blk(BX, TY);
#define LM_RB(F, Z, P) k_rbgs<BX, TY, true, F, Z, P><<<grd, blk, 0, s>>>(L, xin, ec, Cg, hx, hy, hz, f, xout, KZ)
        if (zero) { if (first) LM_RB(1, true, false); else LM_RB(0, true, false); }
        else if (prolong) { if (first) LM_RB(1, false, true); else LM_RB(0, false, true); }
        else { if (first) LM_RB(1, false, false); else LM_RB(0, false, false); }
#undef LM_RB
    } else if (g.ny == 1 && g.nx % 128 == 0 && g.nz >= 2) {
        // 2D rows of 256- (or 128-) cell tiles: a warp per 128-cell segment
        // and half (quarter) chunk; KZ rows per block, about eight blocks (32
        // warps) per SM in all -- four blocks per SM left the loads too few
        // to cover the HBM latency (0.43 against 0.58 of the copy bandwidth
        // at 4096^2) -- and at least 2 rows a warp (small grids, which cannot
        // fill the GPU, get as many warps as that allows: their time is the
        // length of one warp's march)
        const int TW = zrow2d_width(g.nx), tiles = g.nx / TW, parts = 512 / TW;
        int KZ = kz;
        if (kz <= 0) {
            const int chunks = std::max(1, std::min(hdiv(1216, tiles), g.nz / (2 * parts)));
            KZ = hdiv(g.nz, chunks);
        }
        const dim3 grd(tiles, hdiv(g.nz, KZ));
#define LM_RB2(F, Z, P) k_rbgs_zm2d<F, Z, P><<<grd, 128, 0, s>>>(L, xin, ec, Cg, hx, hz, f, xout, KZ, TW)
        if (zero) { if (first) LM_RB2(1, true, false); else LM_RB2(0, true, false); }
        else if (prolong) { if (first) LM_RB2(1, false, true); else LM_RB2(0, false, true); }
        else { if (first) LM_RB2(1, false, false); else LM_RB2(0, false, false); }
#undef LM_RB2
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
void coarse_cycle_allow_smem() {
    cudaFuncSetAttribute(k_coarse_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM_MAX);
}
void launch_coarse_cycle(const CoarseCycle& cc, cudaStream_t s) {
    count_launches(1);
    k_coarse_cycle<<<1, CC_THREADS, cc_smem_bytes(cc), s>>>(cc);
}
void launch_coarse_inverse_many(const CoarseInv* items, const int* task, int ntask, cudaStream_t s) {
    if (ntask <= 0) return;
    count_launches(1);
    k_coarse_inverse_many<<<ntask, 256, 0, s>>>(items, task);
}
void launch_coarse_inverse_grids(const CoarseInv* items, int count, cudaStream_t s) {
    if (count <= 0) return;
    cudaFuncSetAttribute(k_coarse_inverse_grids, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COARSE_INV_SMEM);
    count_launches(1);
    k_coarse_inverse_grids<<<count, 256, COARSE_INV_SMEM, s>>>(items);
}
void launch_coarse_inverse(const Lev32& L, cudaStream_t s, float* ainv) {
    count_launches(1);
    k_coarse_inverse<<<L.g.N, 256, 0, s>>>(L, ainv);
}
void launch_coarse_solve(int n, cudaStream_t s, const float* ainv, const float* f, float* x) {
    count_launches(1);
    k_coarse_solve<<<1, 64, 0, s>>>(n, ainv, f, x);
}

}  // namespace lm
