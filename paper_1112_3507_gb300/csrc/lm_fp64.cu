// Float64 kernels: coefficient assembly, the float64 operator, the Jacobi-
// preconditioned conjugate-gradient iteration and the iterative-refinement
// residual/correction.
//
// GB300 executes float64 at 1/64 of the float32 rate, so these kernels are
// bound by float64 issue, not by HBM: they keep the float64 operation count
// per cell minimal (face conductances and the inverse Jacobi diagonal are
// computed once, at assembly; the stencil uses 13 float64 operations per 3D
// cell) and stream each vector once per kernel.
#include "lm_common.cuh"
#include "lm_kernels.h"
#include "lm_tiles.cuh"

namespace lm {

// ---- coefficient assembly (step (v); Eqs. cpoiss, kappapoiss) -------------

// cells i0 .. i1 - 1 (one launch per chunk of planes when the inputs arrive in chunks)
__global__ void __launch_bounds__(NT) k_assemble(AsmArgs a, int i0, int i1) {
    assemble_range(a, i0 + blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, i1);
}

__global__ void __launch_bounds__(NT) k_scale32(int N, float* __restrict__ x, float scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) x[i] *= scale;
}

// Inverse Jacobi diagonal 1/(c~ + sum of the cell's face conductances), from
// the assembled faces (the plus face of a cell is its plus-neighbour's minus face).
__global__ void __launch_bounds__(NT) k_jacobi_diag(Geo g, const double* __restrict__ ct,
                                                    const double* __restrict__ gx, const double* __restrict__ gy,
                                                    const double* __restrict__ gz, double* __restrict__ dinv) {
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        int i, j, k;
        cell_coords(idx, g, i, j, k);
        const double d = ct[idx] + gx[idx] + gx[nbr_x(idx, i, g).ip] + gy[idx] + gy[nbr_y(idx, j, g).ip] +
                         gz[idx] + gz[nbr_z(idx, k, g).ip];
        dinv[idx] = 1.0 / d;
    }
}

// ---- the float64 operator --------------------------------------------------

// y = A x; optional partial sums of x^T A x into part slot 0.
__global__ void __launch_bounds__(NT) k_apply64(Geo g, Op64 op, const double* __restrict__ x,
                                                double* __restrict__ y, double* __restrict__ part) {
    __shared__ double sm[32];
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const double v = apply64_at(idx, g, op, x);
        y[idx] = v;
        acc[0] += x[idx] * v;
    }
    if (part) write_partials<1>(acc, part, sm);
}

// ---- Jacobi-preconditioned CG (float64) ------------------------------------
// Partial-sum slots: 0 p.q, 1 r.r, 2/3 r.z (even/odd iteration), 4 f.f

__global__ void __launch_bounds__(NT) k_pcg_init_res(PcgArgs a, int use_x0) {
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        const double fi = a.f[idx];
        const double ri = use_x0 ? fi - apply64_at(idx, a.g, a.op, a.x) : fi;
        a.r[idx] = ri;
        acc[0] += ri * ri;
        acc[1] += fi * fi;
    }
    if (!use_x0) {
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) a.x[idx] = 0.0;
    }
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        a.part[1 * MAX_PARTIALS + blockIdx.x] = acc[0];
        a.part[4 * MAX_PARTIALS + blockIdx.x] = acc[1];
    }
}

// p = D^-1 r, partial r.z into slot rz_slot.  restart = 0: first call of a
// solve (sets ||f|| and the initial history entry); restart = 1: after a
// failed true-residual check.
__global__ void __launch_bounds__(NT) k_pcg_init_p(PcgArgs a, int rz_slot, int restart) {
    __shared__ double sm[32];
    const double rr = reduce_partials(a.part + 1 * MAX_PARTIALS, gridDim.x, sm);
    double fnorm;
    if (!restart) {
        const double ff = reduce_partials(a.part + 4 * MAX_PARTIALS, gridDim.x, sm);
        fnorm = sqrt(ff);
    } else {
        fnorm = a.st->fnorm;
    }
    const double rel = fnorm > 0.0 ? sqrt(rr) / fnorm : 0.0;
    const bool stop = !(fnorm > 0.0) || rel <= a.st->rtol;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!restart) {
            a.st->fnorm = fnorm;
            a.hist[0] = rel;
        }
        a.st->rel = rel;
        a.st->converged = stop ? 1 : 0;
        a.st->done = stop ? 1 : 0;
    }
    if (stop) return;
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        const double ri = a.r[idx];
        const double zi = a.op.dinv[idx] * ri;
        a.p[idx] = zi;
        acc[0] += ri * zi;
    }
    write_partials<1>(acc, a.part + rz_slot * MAX_PARTIALS, sm);
}

// q = A p, partial p.q (slot 0)
__global__ void __launch_bounds__(NT) k_pcg_apply(PcgArgs a) {
    if (a.st->done) return;
    __shared__ double sm[32];
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        const double v = apply64_at(idx, a.g, a.op, a.p);
        a.q[idx] = v;
        acc[0] += a.p[idx] * v;
    }
    write_partials<1>(acc, a.part, sm);
}

// alpha = r.z / p.q; x += alpha p; r -= alpha q; partial r.r and r.z (z = D^-1 r)
__global__ void __launch_bounds__(NT) k_pcg_xr(PcgArgs a, int k) {
    if (a.st->done) return;
    __shared__ double sm[64];
    const double pq = reduce_partials(a.part, gridDim.x, sm);
    const double rz = reduce_partials(a.part + (2 + (k & 1)) * MAX_PARTIALS, gridDim.x, sm);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.st->status = LM_ERR_BREAKDOWN;
            a.st->done = 1;
        }
        return;
    }
    const double alpha = rz / pq;
    double acc[2] = {0.0, 0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        const double pi = a.p[idx];
        a.x[idx] += alpha * pi;
        const double ri = a.r[idx] - alpha * a.q[idx];
        a.r[idx] = ri;
        acc[0] += ri * ri;
        acc[1] += ri * (a.op.dinv[idx] * ri);
    }
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        a.part[1 * MAX_PARTIALS + blockIdx.x] = acc[0];
        a.part[(2 + ((k + 1) & 1)) * MAX_PARTIALS + blockIdx.x] = acc[1];
    }
}

// convergence test; beta = r.z_new / r.z_old; p = D^-1 r + beta p
__global__ void __launch_bounds__(NT) k_pcg_p(PcgArgs a, int k) {
    if (a.st->done) return;
    __shared__ double sm[32];
    const double rr = reduce_partials(a.part + 1 * MAX_PARTIALS, gridDim.x, sm);
    const double rz_new = reduce_partials(a.part + (2 + ((k + 1) & 1)) * MAX_PARTIALS, gridDim.x, sm);
    const double rz_old = reduce_partials(a.part + (2 + (k & 1)) * MAX_PARTIALS, gridDim.x, sm);
    const double rel = sqrt(rr) / a.st->fnorm;
    const bool conv = rel <= a.st->rtol;
    const bool bad = !isfinite(rel) || !isfinite(rz_new) || !(rz_old != 0.0);
    const bool last = k + 1 >= a.max_iter;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.hist[k + 1] = rel;
        a.st->iters = k + 1;
        a.st->rel = rel;
        if (conv) a.st->converged = 1;
        if (bad) a.st->status = LM_ERR_BREAKDOWN;
        if (conv || bad || last) a.st->done = 1;
    }
    if (conv || bad || last) return;
    const double beta = rz_new / rz_old;
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride)
        a.p[idx] = a.op.dinv[idx] * a.r[idx] + beta * a.p[idx];
}

// r = f - A x, partial r.r (slot 1): the true residual
__global__ void __launch_bounds__(NT) k_true_residual(PcgArgs a) {
    __shared__ double sm[32];
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.g.N; idx += stride) {
        const double ri = a.f[idx] - apply64_at(idx, a.g, a.op, a.x);
        a.r[idx] = ri;
        acc[0] += ri * ri;
    }
    write_partials<1>(acc, a.part + 1 * MAX_PARTIALS, sm);
}

// Single block: st->rel = sqrt(sum of slot) / st->fnorm (or sets fnorm from slot 4)
__global__ void __launch_bounds__(NT) k_finish_rel(double* part, int G, SolveState* st, int set_fnorm,
                                                   double* hist_entry) {
    __shared__ double sm[32];
    const double rr = reduce_partials(part + 1 * MAX_PARTIALS, G, sm);
    if (set_fnorm) {
        const double ff = reduce_partials(part + 4 * MAX_PARTIALS, G, sm);
        if (threadIdx.x == 0) st->fnorm = sqrt(ff);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double fn = st->fnorm;
        st->rel = fn > 0.0 ? sqrt(rr) / fn : 0.0;
        if (hist_entry) *hist_entry = st->rel;
    }
}

// ---- iterative refinement (float64 residual and correction) ---------------

// r = f - A x in float64, stored as float32 times rscale (a power of two
// that keeps the inner problem's float32 values near unit size, so that the
// products of its dot products neither underflow nor overflow) for the
// inner solve; partial r.r (slot 1) and, with FNORM, f.f (slot 4).
// zero_x: x := 0 first (r = f).
// SC: 0 no scaling; 1 the float32 value scaled (a float multiply by a power
// of two, exact while the unscaled residual is a normal float32 -- the
// launcher asks for it when the residual's expected size is well inside
// float32 range; it saves a float64 multiply a cell on GB300's slow float64
// pipe); 2 scaled in float64 before rounding.
template <bool FNORM, int SC>
__global__ void __launch_bounds__(NT) k_ir_residual(Geo g, Op64 op, const double* __restrict__ f,
                                                    double* __restrict__ x, float* __restrict__ r32,
                                                    double* __restrict__ part, int zero_x, double rscale) {
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    const float rs32 = (float)rscale;
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const double fi = f[idx];
        const double ri = zero_x ? fi : fi - apply64_at(idx, g, op, x);
        r32[idx] = SC == 2 ? (float)(ri * rscale) : (SC == 1 ? (float)ri * rs32 : (float)ri);
        acc[0] += ri * ri;
        if (FNORM) acc[1] += fi * fi;
    }
    if (zero_x)
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) x[idx] = 0.0;
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        part[1 * MAX_PARTIALS + blockIdx.x] = acc[0];
        if (FNORM) part[4 * MAX_PARTIALS + blockIdx.x] = acc[1];
    }
}

// Warm-start scaling.  Along a direction x the A-norm error of alpha x is
// least at alpha = f.x / x^T A x (then J(alpha x) = -(f.x)^2 / (2 x^T A x) <= J(0)
// for the energy J(x) = x^T A x / 2 - f.x of the SPD system).  Pass 1: partial
// x^T A x (slot 0) and f.x (slot 1).
__global__ void __launch_bounds__(NT) k_warm_dots(Geo g, Op64 op, const double* __restrict__ f,
                                                  const double* __restrict__ x, double* __restrict__ part) {
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const double xi = x[idx];
        acc[0] += xi * apply64_at(idx, g, op, x);
        acc[1] += f[idx] * xi;
    }
    write_partials<2>(acc, part, sm);
}

// Pass 2: x *= alpha, with alpha = 0 (drop the warm start) unless f.x > 0
// and x^T A x > 0 are finite.  Every block forms alpha from the partials in
// the same order.
__global__ void __launch_bounds__(NT) k_warm_scale(int N, double* __restrict__ x, const double* part, int G) {
    __shared__ double sm[32];
    const double xax = reduce_partials(part, G, sm);
    const double fx = reduce_partials(part + MAX_PARTIALS, G, sm);
    const double alpha = (fx > 0.0 && xax > 0.0 && isfinite(fx) && isfinite(xax)) ? fx / xax : 0.0;
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
        x[idx] = alpha > 0.0 ? alpha * x[idx] : 0.0;
}

// x += e * escale (float32 correction accumulated in float64; escale undoes
// the power-of-two scaling of the inner right-hand side, exactly)
__global__ void __launch_bounds__(NT) k_ir_correct(int N, double* __restrict__ x, const float* __restrict__ e,
                                                   double escale) {
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
        x[idx] += (double)e[idx] * escale;
}


// Single block: *out = sum of the G partials of slot `slot`.
__global__ void __launch_bounds__(NT) k_reduce_slot(const double* part, int slot, int G, double* out) {
    __shared__ double sm[32];
    const double v = reduce_partials(part + slot * MAX_PARTIALS, G, sm);
    if (threadIdx.x == 0) *out = v;
}

// ---- float64 flexible CG with the float32 multigrid preconditioner --------
// Slots: 0 p.q, 1 r.r, 5 z.q_old, 6 p.r

// partial z.q_old with z the float32 V-cycle output
__global__ void __launch_bounds__(NT) k_fcg64_zq(int N, const float* __restrict__ z, const double* __restrict__ q,
                                                 double* __restrict__ part, const SolveState* st) {
    if (st->done) return;
    __shared__ double sm[32];
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) acc[0] += (double)z[idx] * q[idx];
    write_partials<1>(acc, part + 5 * MAX_PARTIALS, sm);
}

// p = z - (z.q_old / p_old.q_old) p_old
__global__ void __launch_bounds__(NT) k_fcg64_p(int N, const float* __restrict__ z, double* __restrict__ p,
                                                const double* __restrict__ part, int first, const SolveState* st) {
    if (st->done) return;
    __shared__ double sm[32];
    double beta = 0.0;
    if (!first) {
        const double zq = reduce_partials(part + 5 * MAX_PARTIALS, gridDim.x, sm);
        const double pq = reduce_partials(part + 0 * MAX_PARTIALS, gridDim.x, sm);
        beta = -zq / pq;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
        p[idx] = (double)z[idx] + beta * (first ? 0.0 : p[idx]);
}

// q = A p; partials p.q (slot 0), p.r (slot 6)
__global__ void __launch_bounds__(NT) k_fcg64_apply(Geo g, Op64 op, const double* __restrict__ p,
                                                    double* __restrict__ q, const double* __restrict__ r,
                                                    double* __restrict__ part, const SolveState* st) {
    if (st->done) return;
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.N; idx += stride) {
        const double v = apply64_at(idx, g, op, p);
        q[idx] = v;
        const double pi = p[idx];
        acc[0] += pi * v;
        acc[1] += pi * r[idx];
    }
    block_sum<2>(acc, sm);
    if (threadIdx.x == 0) {
        part[0 * MAX_PARTIALS + blockIdx.x] = acc[0];
        part[6 * MAX_PARTIALS + blockIdx.x] = acc[1];
    }
}

// alpha = p.r / p.q; x += alpha p; r -= alpha q; r32 = r; partial r.r (slot 1)
__global__ void __launch_bounds__(NT) k_fcg64_update(int N, double* __restrict__ x, double* __restrict__ r,
                                                     float* __restrict__ r32, const double* __restrict__ p,
                                                     const double* __restrict__ q, double* __restrict__ part,
                                                     SolveState* st) {
    if (st->done) return;
    __shared__ double sm[32];
    const double pq = reduce_partials(part + 0 * MAX_PARTIALS, gridDim.x, sm);
    const double pr = reduce_partials(part + 6 * MAX_PARTIALS, gridDim.x, sm);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(pr)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = LM_ERR_BREAKDOWN;
            st->done = 1;
        }
        return;
    }
    const double alpha = pr / pq;
    // the preconditioner's input in float32, scaled by a power of two near
    // 1/rms of the previous residual: flexible CG is invariant under a
    // positive scaling of z, and the scaling keeps the float32 V-cycle's
    // values away from underflow as the residual shrinks
    const double rs = pow2_near_inv(st->rel * st->fnorm * rsqrt((double)N));
    double acc[1] = {0.0};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
        x[idx] += alpha * p[idx];
        const double ri = r[idx] - alpha * q[idx];
        r[idx] = ri;
        r32[idx] = (float)(ri * rs);
        acc[0] += ri * ri;
    }
    write_partials<1>(acc, part + 1 * MAX_PARTIALS, sm);
}

// r32 = r (float32 copy for the preconditioner)
__global__ void __launch_bounds__(NT) k_to32(int N, const double* __restrict__ r, float* __restrict__ r32) {
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) r32[idx] = (float)r[idx];
}

// Single block: st->fnorm = sqrt(sum of slot), st->rel = 1 (start of a solve
// whose reference norm is that of its initial residual).
__global__ void __launch_bounds__(NT) k_set_fnorm(const double* part, int slot, int G, SolveState* st) {
    __shared__ double sm[32];
    const double v = reduce_partials(part + slot * MAX_PARTIALS, G, sm);
    if (threadIdx.x == 0) {
        st->fnorm = sqrt(v);
        st->rel = 1.0;
    }
}

// ---- host launchers ---------------------------------------------------------

void launch_assemble(const Geo& g, int G, cudaStream_t s, const double* a_in, const double* rho_new,
                     const double* cs2, double dt, int raw, const double h[3], const Op64Out& out, AsmFlags* fl,
                     int i0, int i1) {
    count_launches(1);
    k_assemble<<<G, NT, 0, s>>>(asm_args(g, a_in, rho_new, cs2, dt, raw, h, out, fl), i0, i1 < 0 ? g.N : i1);
}
void launch_scale32(int N, int G, cudaStream_t s, float* x, float scale) {
    count_launches(1);
    k_scale32<<<G, NT, 0, s>>>(N, x, scale);
}
void launch_jacobi_diag(const Geo& g, int G, cudaStream_t s, const Op64& op, double* dinv) {
    count_launches(1);
    k_jacobi_diag<<<G, NT, 0, s>>>(g, op.ct, op.gx, op.gy, op.gz, dinv);
}
void launch_apply64(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* x, double* y,
                    double* part) {
    count_launches(1);
    k_apply64<<<G, NT, 0, s>>>(g, op, x, y, part);
}
void launch_pcg_init(const PcgArgs& a, int G, cudaStream_t s, int use_x0) {
    count_launches(1);
    k_pcg_init_res<<<G, NT, 0, s>>>(a, use_x0);
    count_launches(1);
    k_pcg_init_p<<<G, NT, 0, s>>>(a, 2, 0);
}
void launch_pcg_init_p(const PcgArgs& a, int G, cudaStream_t s, int rz_slot, int restart) {
    count_launches(1);
    k_pcg_init_p<<<G, NT, 0, s>>>(a, rz_slot, restart);
}
void launch_pcg_xr(const PcgArgs& a, int G, cudaStream_t s, int k) {
    count_launches(1);
    k_pcg_xr<<<G, NT, 0, s>>>(a, k);
}
void launch_pcg_p(const PcgArgs& a, int G, cudaStream_t s, int k) {
    count_launches(1);
    k_pcg_p<<<G, NT, 0, s>>>(a, k);
}
void launch_pcg_restart(const PcgArgs& a, int G, cudaStream_t s, int k) {
    count_launches(1);
    k_pcg_init_p<<<G, NT, 0, s>>>(a, 2 + (k & 1), 1);
}
void launch_pcg_iter(const PcgArgs& a, int G, cudaStream_t s, int k) {
    count_launches(1);
    k_pcg_apply<<<G, NT, 0, s>>>(a);
    count_launches(1);
    k_pcg_xr<<<G, NT, 0, s>>>(a, k);
    count_launches(1);
    k_pcg_p<<<G, NT, 0, s>>>(a, k);
}
void launch_true_residual(const PcgArgs& a, int G, cudaStream_t s) {
    count_launches(1);
    k_true_residual<<<G, NT, 0, s>>>(a);
    count_launches(1);
    k_finish_rel<<<1, NT, 0, s>>>(a.part, G, a.st, 0, nullptr);
}
void launch_ir_residual(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* f, double* x,
                        float* r32, double* part, int zero_x, SolveState* st, int set_fnorm, double* hist_entry,
                        double rscale) {
    count_launches(1);
    // rscale near 1/rms(r): the residual's size is about 1/rscale, a normal
    // float32 (with room for small entries) when rscale is within 2^+-90
    const int sc = rscale == 1.0 ? 0 : (rscale >= 0x1p-90 && rscale <= 0x1p90 ? 1 : 2);
#define LM_IRR(F, SC) k_ir_residual<F, SC><<<G, NT, 0, s>>>(g, op, f, x, r32, part, zero_x, rscale)
    if (set_fnorm) {
        if (sc == 0) LM_IRR(true, 0); else if (sc == 1) LM_IRR(true, 1); else LM_IRR(true, 2);
    } else {
        if (sc == 0) LM_IRR(false, 0); else if (sc == 1) LM_IRR(false, 1); else LM_IRR(false, 2);
    }
#undef LM_IRR
    count_launches(1);
    k_finish_rel<<<1, NT, 0, s>>>(part, G, st, set_fnorm, hist_entry);
}
void launch_warm_scale(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* f, double* x,
                       double* part) {
    count_launches(2);
    k_warm_dots<<<G, NT, 0, s>>>(g, op, f, x, part);
    k_warm_scale<<<G, NT, 0, s>>>(g.N, x, part, G);
}
void launch_ir_correct(int N, int G, cudaStream_t s, double* x, const float* e, double escale) {
    count_launches(1);
    k_ir_correct<<<G, NT, 0, s>>>(N, x, e, escale);
}
void launch_reduce_rel(double* part, int G, cudaStream_t s, SolveState* st, double* hist_entry) {
    count_launches(1);
    k_finish_rel<<<1, NT, 0, s>>>(part, G, st, 0, hist_entry);
}

void launch_reduce_slot(const double* part, int slot, int G, cudaStream_t s, double* out) {
    count_launches(1);
    k_reduce_slot<<<1, NT, 0, s>>>(part, slot, G, out);
}
void launch_fcg64_iter_a(int N, int G, cudaStream_t s, const float* z, const double* q, double* part, int first,
                         double* p, const SolveState* st) {
    if (!first) {
        count_launches(1);
        k_fcg64_zq<<<G, NT, 0, s>>>(N, z, q, part, st);
    }
    count_launches(1);
    k_fcg64_p<<<G, NT, 0, s>>>(N, z, p, part, first, st);
}
void launch_fcg64_iter_b(const Geo& g, int G, cudaStream_t s, const Op64& op, double* x, double* r, float* r32,
                         const double* p, double* q, double* part, SolveState* st) {
    count_launches(1);
    k_fcg64_apply<<<G, NT, 0, s>>>(g, op, p, q, r, part, st);
    count_launches(1);
    k_fcg64_update<<<G, NT, 0, s>>>(g.N, x, r, r32, p, q, part, st);
    count_launches(1);
    k_finish_rel<<<1, NT, 0, s>>>(part, G, st, 0, nullptr);
}
void launch_set_fnorm(const double* part, int slot, int G, cudaStream_t s, SolveState* st) {
    count_launches(1);
    k_set_fnorm<<<1, NT, 0, s>>>(part, slot, G, st);
}
void launch_to32(int N, int G, cudaStream_t s, const double* r, float* r32) {
    count_launches(1);
    k_to32<<<G, NT, 0, s>>>(N, r, r32);
}

}  // namespace lm
