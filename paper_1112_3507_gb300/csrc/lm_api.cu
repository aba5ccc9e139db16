// C ABI of the generalized-Poisson solver: grid object, inputs, solve
// drivers (float64 Jacobi-PCG, float64 flexible CG with the float32
// multigrid preconditioner, mixed-precision iterative refinement) and the
// row-level entry points.  Host code here only sequences kernels on the
// caller's stream and reads back a few scalars; all arithmetic on grid data
// runs in the kernels of lm_fp64.cu / lm_fp32.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"
#include "lm_internal.h"

using namespace lm;

static std::atomic<long long> g_launches{0};
void lm::count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            fprintf(stderr, "lowmach: %s failed: %s (%s:%d)\n", #call,  \
                    cudaGetErrorString(e_), __FILE__, __LINE__);        \
            return e_ == cudaErrorMemoryAllocation ? LM_ERR_OUT_OF_MEMORY : LM_ERR_CUDA; \
        }                                                               \
    } while (0)

namespace {

template <class T>
int dalloc(T** p, size_t count) {
    CK(cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)));
    return LM_OK;
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

Op64 op64(const lm_grid* g) { return Op64{g->ct, g->gx, g->gy, g->gz, g->dinv}; }

bool halvable(int n, int bc) {
    if (n < 2 || (n % 2)) return false;
    if (bc == LM_BC_PERIODIC) return ((n / 2) % 2 == 0) || n / 2 == 1;
    return true;
}

// A float32 level view; its rho array holds rho / rho_scale, so its face
// factors 2/h^2 are divided by rho_scale too (exactly: a power of two).
Lev32 make_lev(const int n[3], const int bc[3], const double h[3], const float* ct, const float* rho,
               double rho_scale = 1.0) {
    Lev32 L{};
    L.g.nx = n[0];
    L.g.ny = n[1];
    L.g.nz = n[2];
    L.g.N = n[0] * n[1] * n[2];
    L.g.bcx = bc[0];
    L.g.bcy = bc[1];
    L.g.bcz = bc[2];
    L.g.ih2x = 1.0 / (h[0] * h[0]);
    L.g.ih2y = 1.0 / (h[1] * h[1]);
    L.g.ih2z = 1.0 / (h[2] * h[2]);
    L.c2x = (float)(2.0 / (h[0] * h[0]) / rho_scale);
    L.c2y = (float)(2.0 / (h[1] * h[1]) / rho_scale);
    L.c2z = (float)(2.0 / (h[2] * h[2]) / rho_scale);
    L.ct = ct;
    L.rho = rho;
    return L;
}

int sync_state(lm_grid* g, SolveState* dev, cudaStream_t s) {
    CK(cudaMemcpyAsync(g->st_host, dev, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return LM_OK;
}

void free_mg(lm_grid* g) {
    for (size_t l = 0; l < g->mg.size(); ++l) {
        MgLevel& M = g->mg[l];
        if (l > 0) {
            cudaFree(M.ct);
            cudaFree(M.rho);
            cudaFree(M.xa);
            cudaFree(M.xb);
            cudaFree(M.xo);
            cudaFree(M.f);
        }
        cudaFree(M.ainv);
    }
    g->mg.clear();
    g->mg_built = false;
}

bool mg_supported(const lm_grid* g) {
    if (!g->fp32_ok) return false;          // rho or c~ beyond what the float32 levels can hold
    for (int a = 0; a < 3; ++a)
        if (g->bc[a] == LM_BC_PERIODIC && g->n[a] > 1 && (g->n[a] % 2)) return false;
    return true;
}

// Multigrid hierarchy from the float32 coefficients (coarse c~, rho = child means).
int build_mg(lm_grid* g, cudaStream_t s, bool defer_inverse = false) {
    // the coarsest level's dense inverse, now or left to the caller
    auto inverse = [&](MgLevel& Lc) {
        g->inv_pending = defer_inverse;
        if (!defer_inverse) launch_coarse_inverse(Lc.L, s, Lc.ainv);
    };
    if (g->mg_built) {
        if (g->inv_pending && !defer_inverse) inverse(g->mg.back());
        CK(cudaGetLastError());
        return LM_OK;
    }
    if (!g->mg.empty()) {
        // the grid's shape never changes: keep the buffers, recompute the
        // coarse coefficients and the coarsest inverse from the new values
        for (size_t l = 1; l < g->mg.size(); ++l) {
            const MgLevel& F = g->mg[l - 1];
            MgLevel& C = g->mg[l];
            launch_coarsen(F.L, C.L, F.halved[0], F.halved[1], F.halved[2], s, C.ct, C.rho);
        }
        MgLevel& Lc = g->mg.back();
        if (Lc.ainv) inverse(Lc);
        CK(cudaGetLastError());
        g->mg_built = true;
        return LM_OK;
    }
    ++g->version;       // new buffers: cached batch plans of this grid are stale
    rbgs_row_allow_smem();
    MgLevel L0;
    L0.L = make_lev(g->n, g->bc, g->h, g->ct32, g->rho32, g->rho_scale);
    std::memcpy(L0.h, g->h, sizeof L0.h);
    L0.xa = g->tmp_a;
    L0.xb = g->tmp_b;
    g->mg.push_back(L0);
    while (g->mg.back().L.g.N > COARSE_MAX) {
        MgLevel& F = g->mg.back();
        int nf[3] = {F.L.g.nx, F.L.g.ny, F.L.g.nz};
        int hv[3];
        bool any = false;
        for (int a = 0; a < 3; ++a) {
            hv[a] = halvable(nf[a], g->bc[a]) ? 1 : 0;
            any = any || hv[a];
        }
        if (!any) break;
        MgLevel C;
        int nc[3];
        for (int a = 0; a < 3; ++a) {
            nc[a] = hv[a] ? nf[a] / 2 : nf[a];
            C.h[a] = F.h[a] * (hv[a] ? 2.0 : 1.0);
            F.halved[a] = hv[a];
        }
        const int Nc = nc[0] * nc[1] * nc[2];
        int rc;
        if ((rc = dalloc(&C.ct, Nc)) || (rc = dalloc(&C.rho, Nc)) || (rc = dalloc(&C.xa, Nc)) ||
            (rc = dalloc(&C.xb, Nc)) || (rc = dalloc(&C.xo, Nc)) || (rc = dalloc(&C.f, Nc)))
            return rc;
        C.L = make_lev(nc, g->bc, C.h, C.ct, C.rho, g->rho_scale);
        launch_coarsen(F.L, C.L, hv[0], hv[1], hv[2], s, C.ct, C.rho);
        g->mg.push_back(C);
    }
    MgLevel& Lc = g->mg.back();
    if (Lc.L.g.N <= COARSE_EXACT) {
        int rc = dalloc(&Lc.ainv, (size_t)Lc.L.g.N * Lc.L.g.N);
        if (rc) return rc;
        inverse(Lc);
    }
    // the one-block coarse V-cycle takes over from the first level small
    // enough, when the chain ends in a directly solved level
    g->cc_level = -1;
    if (g->mg.back().ainv)
        for (size_t l = 0; l < g->mg.size(); ++l)
            if (g->mg[l].L.g.N <= CC_MAX_CELLS && g->mg.size() - l <= (size_t)CC_MAXL && g->mg.size() - l >= 2) {
                int N[CC_MAXL];
                const int nl = (int)(g->mg.size() - l);
                for (int i = 0; i < nl; ++i) N[i] = g->mg[l + i].L.g.N;
                if (cc_smem_bytes(N, nl) <= CC_SMEM_MAX) {
                    coarse_cycle_allow_smem();
                    g->cc_level = (int)l;
                }
                break;
            }
    CK(cudaGetLastError());
    g->mg_built = true;
    return LM_OK;
}

// A chain of fused red-black sweeps on one level: sweep 0 reads `src`
// (or zero, or src + P ec), each later sweep reads the previous result; the
// last sweep writes `dst`, the others ping-pong through the level's xa/xb
// without writing the buffer they read.  Returns the buffer holding the result.
float* sweep_chain(MgLevel& M, cudaStream_t s, int count, const int* first, const float* src, bool zero,
                   const float* ec, const MgLevel* C, const float* f, float* dst) {
    const float* cur = src;
    float* out = dst;
    for (int it = 0; it < count; ++it) {
        if (it == count - 1 && dst) {
            out = dst;
        } else {
            out = (cur == M.xa) ? M.xb : M.xa;
        }
        const bool z0 = zero && it == 0;
        const bool pr = ec && it == 0;
        launch_rbgs(M.L, s, z0 ? nullptr : cur, pr ? ec : nullptr, pr ? &C->L : nullptr,
                    pr ? M.halved[0] : 0, pr ? M.halved[1] : 0, pr ? M.halved[2] : 0, f, out, first[it], z0, pr);
        cur = out;
    }
    return out;
}

// One V-cycle on level l: xout = M_l f from a zero initial guess.  Pre-
// smoothing sweeps red then black, post-smoothing black then red (the
// adjoint order), so the cycle is symmetric for nu1 == nu2.
void vcycle(lm_grid* g, int l, float* xout, const float* f, int nu1, int nu2, cudaStream_t s) {
    MgLevel& M = g->mg[l];
    if (l == g->cc_level) {          // the rest of the cycle in one block
        CoarseCycle cc{};
        cc.nl = (int)g->mg.size() - l;
        for (int i = 0; i < cc.nl; ++i) {
            const MgLevel& Li = g->mg[l + i];
            cc.L[i] = Li.L;
            cc.hx[i] = Li.halved[0];
            cc.hy[i] = Li.halved[1];
            cc.hz[i] = Li.halved[2];
            cc.x[i] = i == 0 ? xout : Li.xo;
            cc.f[i] = i == 0 ? const_cast<float*>(f) : Li.f;
        }
        cc.ainv = g->mg.back().ainv;
        cc.nu1 = nu1;
        cc.nu2 = nu2;
        launch_coarse_cycle(cc, s);
        return;
    }
    const bool last = (size_t)l + 1 == g->mg.size();
    int order[2 * COARSE_SWEEPS + 8];
    if (last) {
        if (M.ainv) {
            launch_coarse_solve(M.L.g.N, s, M.ainv, f, xout);
        } else {
            for (int it = 0; it < 2 * COARSE_SWEEPS; ++it) order[it] = it & 1;   // (RB, BR) pairs
            sweep_chain(M, s, 2 * COARSE_SWEEPS, order, nullptr, true, nullptr, nullptr, f, xout);
        }
        return;
    }
    for (int it = 0; it < nu1; ++it) order[it] = 0;
    float* pre = sweep_chain(M, s, nu1, order, nullptr, true, nullptr, nullptr, f, nullptr);
    MgLevel& C = g->mg[l + 1];
    launch_resid_restrict(M.L, C.L, M.halved[0], M.halved[1], M.halved[2], s, pre, f, C.f);
    vcycle(g, l + 1, C.xo, C.f, nu1, nu2, s);
    for (int it = 0; it < nu2; ++it) order[it] = 1;
    sweep_chain(M, s, nu2, order, pre, false, C.xo, &C, f, xout);
}

PcgArgs pcg_args(lm_grid* g, int max_iter) {
    PcgArgs a;
    a.g = g->geo;
    a.op = op64(g);
    a.f = g->f;
    a.x = g->x;
    a.r = g->r;
    a.p = g->p;
    a.q = g->q;
    a.part = g->part;
    a.st = g->st;
    a.hist = g->hist_dev;
    a.max_iter = max_iter;
    return a;
}

int ensure_hist(lm_grid* g, int n) {
    if (g->hist_cap >= n) return LM_OK;
    cudaFree(g->hist_dev);
    g->hist_dev = nullptr;
    g->hist_cap = 0;
    int rc = dalloc(&g->hist_dev, n);
    if (rc) return rc;
    g->hist_cap = n;
    return LM_OK;
}

int init_state(lm_grid* g, SolveState* st, double rtol, cudaStream_t s) {
    SolveState h{};
    h.rtol = rtol;
    CK(cudaMemcpyAsync(st, &h, sizeof h, cudaMemcpyHostToDevice, s));
    // the copy reads a stack object: wait for it before returning
    CK(cudaStreamSynchronize(s));
    return LM_OK;
}

// ---- float64 Jacobi-PCG ------------------------------------------------------
int solve_jacobi_pcg(lm_grid* g, const lm_solve_opts* o, lm_solve_result* res) {
    cudaStream_t s = S(o->cuda_stream);
    int rc;
    if ((rc = ensure_hist(g, o->max_iter + 2))) return rc;
    if ((rc = init_state(g, g->st, o->rtol, s))) return rc;
    PcgArgs a = pcg_args(g, o->max_iter);
    if (!g->have_dinv) {
        launch_jacobi_diag(g->geo, g->G, s, op64(g), g->dinv);
        g->have_dinv = true;
    }
    if (o->use_x0 && g->have_x0) CK(cudaMemcpyAsync(g->x, g->x0, sizeof(double) * g->N, cudaMemcpyDeviceToDevice, s));
    launch_pcg_init(a, g->G, s, o->use_x0 && g->have_x0);
    CK(cudaGetLastError());
    int k = 0, restarts = 0;
    const int chunk = std::max(1, o->check_every);
    if ((rc = sync_state(g, g->st, s))) return rc;
    while (!g->st_host->done) {
        for (int c = 0; c < chunk && k < o->max_iter; ++c, ++k) launch_pcg_iter(a, g->G, s, k);
        CK(cudaGetLastError());
        if ((rc = sync_state(g, g->st, s))) return rc;
        SolveState* h = g->st_host;
        if (h->status) break;
        if (h->converged) {
            launch_true_residual(a, g->G, s);
            if ((rc = sync_state(g, g->st, s))) return rc;
            if (g->st_host->rel <= o->rtol || restarts >= 3 || k >= o->max_iter) break;
            ++restarts;
            k = g->st_host->iters;
            launch_pcg_restart(a, g->G, s, k);
            if ((rc = sync_state(g, g->st, s))) return rc;
            continue;
        }
        if (k >= o->max_iter) break;
    }
    SolveState h = *g->st_host;
    const int iters = h.iters;
    g->history.assign(iters + 1, 0.0);
    CK(cudaMemcpy(g->history.data(), g->hist_dev, sizeof(double) * (iters + 1), cudaMemcpyDeviceToHost));
    // final true residual
    launch_true_residual(a, g->G, s);
    if ((rc = sync_state(g, g->st, s))) return rc;
    res->iters = iters;
    res->rel_residual = g->st_host->rel;
    if (h.status) return h.status;
    return g->st_host->rel <= o->rtol ? LM_OK : LM_ERR_NO_CONVERGENCE;
}

// ---- float64 flexible CG with the float32 V-cycle ---------------------------
int solve_mg_pcg(lm_grid* g, const lm_solve_opts* o, lm_solve_result* res) {
    cudaStream_t s = S(o->cuda_stream);
    int rc;
    if ((rc = build_mg(g, s))) return rc;
    if ((rc = init_state(g, g->st, o->rtol, s))) return rc;
    PcgArgs a = pcg_args(g, o->max_iter);
    const bool x0 = o->use_x0 && g->have_x0;
    if (x0) CK(cudaMemcpyAsync(g->x, g->x0, sizeof(double) * g->N, cudaMemcpyDeviceToDevice, s));
    // r = f - A x (or f), ||f||, ||r||
    launch_ir_residual(g->geo, g->G, s, op64(g), g->f, g->x, g->r32, g->part, !x0, g->st, 1, nullptr);
    launch_true_residual(a, g->G, s);     // float64 r
    if ((rc = sync_state(g, g->st, s))) return rc;
    g->history.assign(1, g->st_host->rel);
    if (!(g->st_host->fnorm > 0.0)) {
        res->rel_residual = 0.0;
        return LM_OK;
    }
    int k = 0;
    while (g->st_host->rel > o->rtol && k < o->max_iter) {
        vcycle(g, 0, g->z32, g->r32, o->nu1, o->nu2, s);
        res->vcycles++;
        launch_fcg64_iter_a(g->N, g->G, s, g->z32, g->q, g->part, k == 0, g->p, g->st);
        launch_fcg64_iter_b(g->geo, g->G, s, op64(g), g->x, g->r, g->r32, g->p, g->q, g->part, g->st);
        CK(cudaGetLastError());
        ++k;
        if ((rc = sync_state(g, g->st, s))) return rc;
        g->history.push_back(g->st_host->rel);
        if (g->st_host->status) break;
    }
    launch_true_residual(a, g->G, s);
    if ((rc = sync_state(g, g->st, s))) return rc;
    res->iters = k;
    res->rel_residual = g->st_host->rel;
    if (g->st_host->status) return g->st_host->status;
    return g->st_host->rel <= o->rtol ? LM_OK : LM_ERR_NO_CONVERGENCE;
}

// Learned two-level preconditioner z = M_net r: a two-grid cycle whose
// coarse-grid correction is replaced by the network,
//   x1 = one red-black sweep on A x = r from x = 0,
//   n  = s NN(features(r1)),  r1 = r - A x1,
//   x2 = x1 + alpha n,  alpha = n.r1 / n^T A n  (0 unless both are positive),
//   z  = one black-red sweep from x2.
// alpha is the step along n that minimises the A-norm error of x2, so the
// network correction never makes x2 worse than x1 in that norm; the sweeps
// remove the oscillatory error the network leaves.  Buffers: the level-0
// sweep buffers and the network's own output buffer (q32 holds A p of the
// flexible CG between iterations).
int learned_precond(lm_grid* g, float* z, const float* r, cudaStream_t s) {
    MgLevel& M = g->mg[0];
    const Red red{g->part, g->scal, g->ctr};
    const int rb = 0, br = 1;
    constexpr int S_NAN = 5, S_NR = 6;              // scal slots: n^T A n, n.r1
    float* x1 = sweep_chain(M, s, 1, &rb, nullptr, true, nullptr, nullptr, r, nullptr);
    float* r1 = (x1 == M.xa) ? M.xb : M.xa;
    launch_apply32(M.L, s, x1, r1, nullptr, red, -1, -1);
    launch_axpy32(g->N, g->G, s, -1.f, r1, r, r1);                 // r1 = r - A x1
    int rc = lm::net_apply<float, float>(g, r1, z, s);              // n (into z)
    if (rc) return rc;
    launch_apply32(M.L, s, z, g->nny, r1, red, S_NAN, S_NR);        // n^T A n, n.r1
    launch_axpy_ratio32(g->N, g->G, s, g->scal, S_NR, S_NAN, z, x1, r1);   // x2 (into r1's buffer)
    sweep_chain(M, s, 1, &br, r1, false, nullptr, nullptr, r, z);
    CK(cudaGetLastError());
    return LM_OK;
}

// One inner flexible-CG iteration with the V-cycle preconditioner:
// z = M r, p = z (first) or z + beta p, q = A p with p.q and p.r, then the
// e, r update and r.r (the last block sets the inner state's rel).
void inner_iteration(lm_grid* g, const lm_solve_opts* o, cudaStream_t s, bool first) {
    MgLevel& M = g->mg[0];
    const Red red{g->part, g->scal, g->ctr};
    vcycle(g, 0, g->z32, g->r32, o->nu1, o->nu2, s);
    if (!first) launch_dot32(g->N, g->G, s, g->z32, g->q32, red, 3, nullptr);
    launch_fcg_beta_p(g->N, g->G, s, g->z32, g->p32, g->scal, first);
    launch_apply32(M.L, s, g->p32, g->q32, g->r32, red, 0, 2);
    launch_fcg_update(g->N, g->G, s, g->e32, g->r32, g->p32, g->q32, red, g->st_in);
}

// The two inner iterations as CUDA graphs, captured on the grid's own stream
// (graphs launch on any stream) once per hierarchy version and smoothing
// counts: an iteration is ~40 dependent launches, most of them tiny on the
// coarse levels.  Returns false when capture is unavailable (the caller then
// launches directly).
bool ensure_inner_graphs(lm_grid* g, const lm_solve_opts* o) {
    if (g->ig_exec[0] && g->ig_version == g->version && g->ig_nu1 == o->nu1 && g->ig_nu2 == o->nu2) return true;
    for (cudaGraphExec_t& e : g->ig_exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    if (!g->cap_stream && cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (int k = 0; k < 2; ++k) {
        const long long before = lm_kernel_launches();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
        inner_iteration(g, o, g->cap_stream, k == 0);
        const cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        g->ig_nk[k] = lm_kernel_launches() - before;
        count_launches(-g->ig_nk[k]);                  // captured, not launched
        if (e != cudaSuccess || !graph) {
            cudaGetLastError();
            return false;
        }
        const cudaError_t ei = cudaGraphInstantiate(&g->ig_exec[k], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g->ig_exec[k] = nullptr;
            cudaGetLastError();
            return false;
        }
    }
    g->ig_version = g->version;
    g->ig_nu1 = o->nu1;
    g->ig_nu2 = o->nu2;
    return true;
}

// Set-up of a device-side inner solve: the inner state (tolerance rtol,
// nothing done) and the iteration counter.
__global__ void k_inner_init(SolveState* st, double rtol, int* it) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        SolveState h{};
        h.rtol = rtol;
        *st = h;
        *it = 0;
    }
}

// End of an inner iteration of the device-side loop: count it and keep
// looping while the inner solve has neither broken down nor reached its
// tolerance, below the iteration limit.
__global__ void k_inner_cond(SolveState* st, int* it, int max_it, cudaGraphConditionalHandle loop) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int n = *it + 1;
        *it = n;
        st->iters = n;
        const bool more = !st->status && st->rel > st->rtol && n < max_it;
        cudaGraphSetConditional(loop, more ? 1u : 0u);
    }
}

// The inner solve with the V-cycle as one graph: e = 0, the inner state,
// ||r||, the first iteration, then a while node (condition set by
// k_inner_cond) repeating the later iteration.  Captured once per
// hierarchy version, smoothing counts, tolerance and iteration limit;
// returns false when capture is unavailable.
bool ensure_loop_graph(lm_grid* g, const lm_solve_opts* o) {
    if (g->loop_exec && g->loop_version == g->version && g->loop_nu1 == o->nu1 && g->loop_nu2 == o->nu2 &&
        g->loop_max == o->inner_max_iter && g->loop_rtol == o->inner_rtol)
        return true;
    if (g->loop_exec) {
        cudaGraphExecDestroy(g->loop_exec);
        g->loop_exec = nullptr;
    }
    if (!g->cap_stream && cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (!g->cap_body && cudaStreamCreateWithFlags(&g->cap_body, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (!g->d_inner_it && cudaMalloc(&g->d_inner_it, sizeof(int)) != cudaSuccess) return false;
    const Red red{g->part, g->scal, g->ctr};
    cudaStream_t cs = g->cap_stream;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const long long before = lm_kernel_launches();
    bool ok = cudaMemsetAsync(g->e32, 0, sizeof(float) * g->N, cs) == cudaSuccess;
    k_inner_init<<<1, 32, 0, cs>>>(g->st_in, o->inner_rtol, g->d_inner_it);
    count_launches(1);
    launch_dot32(g->N, g->G, cs, g->r32, g->r32, red, 4, g->st_in);
    inner_iteration(g, o, cs, true);
    cudaGraphConditionalHandle loop{};
    cudaGraph_t cg = nullptr;
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    ok = ok && cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps) == cudaSuccess &&
         cudaGraphConditionalHandleCreate(&loop, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        k_inner_cond<<<1, 32, 0, cs>>>(g->st_in, g->d_inner_it, o->inner_max_iter, loop);
        count_launches(1);
        ok = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps) == cudaSuccess;
    }
    const long long n_pro = lm_kernel_launches() - before;
    long long n_body = 0;
    cudaGraphNode_t cnode{};
    if (ok) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp) == cudaSuccess;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (ok && cudaStreamBeginCaptureToGraph(g->cap_body, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const long long b0 = lm_kernel_launches();
            inner_iteration(g, o, g->cap_body, false);
            k_inner_cond<<<1, 32, 0, g->cap_body>>>(g->st_in, g->d_inner_it, o->inner_max_iter, loop);
            count_launches(1);
            n_body = lm_kernel_launches() - b0;
            ok = cudaStreamEndCapture(g->cap_body, &body) == cudaSuccess;
        } else {
            ok = false;
        }
        ok = ok && cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                       cudaSuccess;
    }
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    count_launches(-(n_pro + n_body));                 // captured, not launched
    if (!ok || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->loop_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        g->loop_exec = nullptr;
        cudaGetLastError();
        return false;
    }
    g->loop_nk[0] = n_pro;
    g->loop_nk[1] = n_body;
    g->loop_version = g->version;
    g->loop_nu1 = o->nu1;
    g->loop_nu2 = o->nu2;
    g->loop_max = o->inner_max_iter;
    g->loop_rtol = o->inner_rtol;
    return true;
}

// Inner float32 flexible CG on A32 e = r (r overwritten).  Preconditioner:
// the V-cycle, or (*use_net) the learned two-level cycle above; a network
// preconditioner that leaves the inner residual above 1/2 after 4
// iterations, or returns a non-finite value, switches the rest of the solve
// to the V-cycle (*use_net = false).
// Inner iterations and launches of a device-side inner solve whose state
// the caller copied into st_host[1] and has waited for.
void account_device_inner(lm_grid* g, int* iters, int* vcycles) {
    const int n = std::max(1, g->st_host[1].iters);
    count_launches(g->loop_nk[0] + (long long)(n - 1) * g->loop_nk[1]);
    *iters += n;
    *vcycles += n;
}

// *deferred (when given) lets the device-side inner solve return without a
// host wait: its state is queued for copy into st_host[1], and the caller
// waits once for it and the next refinement residual together, then calls
// account_device_inner.
int inner_fcg(lm_grid* g, const lm_solve_opts* o, cudaStream_t s, int* iters, int* vcycles, bool* use_net,
              bool* deferred = nullptr) {
    int rc;
    MgLevel& M = g->mg[0];
    const Red red{g->part, g->scal, g->ctr};
    if (deferred) *deferred = false;
    if (!(use_net && *use_net) && o->check_every != 1 && ensure_loop_graph(g, o)) {
        // the whole inner solve on the device: one launch, one host check
        // (check_every == 1 asks for a host check after every iteration: the
        // loop below, one graph launch per iteration)
        CK(cudaGraphLaunch(g->loop_exec, s));
        CK(cudaMemcpyAsync(g->st_host + 1, g->st_in, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        if (deferred) {
            *deferred = true;
            return LM_OK;
        }
        CK(cudaStreamSynchronize(s));
        account_device_inner(g, iters, vcycles);
        g->st_host[0] = g->st_host[1];
        return LM_OK;
    }
    CK(cudaMemsetAsync(g->e32, 0, sizeof(float) * g->N, s));
    if ((rc = init_state(g, g->st_in, o->inner_rtol, s))) return rc;
    // the inner problem's reference norm: ||r|| of its right-hand side
    launch_dot32(g->N, g->G, s, g->r32, g->r32, red, 4, g->st_in);
    bool graphs = false;
    for (int it = 0; it < o->inner_max_iter; ++it) {
        if (use_net && *use_net) {
            if ((rc = learned_precond(g, g->z32, g->r32, s))) return rc;
            if (it > 0) launch_dot32(g->N, g->G, s, g->z32, g->q32, red, 3, nullptr);
            launch_fcg_beta_p(g->N, g->G, s, g->z32, g->p32, g->scal, it == 0);
            launch_apply32(M.L, s, g->p32, g->q32, g->r32, red, 0, 2);
            launch_fcg_update(g->N, g->G, s, g->e32, g->r32, g->p32, g->q32, red, g->st_in);
        } else {
            if (!graphs) graphs = ensure_inner_graphs(g, o);
            const int k = it == 0 ? 0 : 1;
            if (graphs) {
                CK(cudaGraphLaunch(g->ig_exec[k], s));
                count_launches(g->ig_nk[k]);
            } else {
                inner_iteration(g, o, s, it == 0);
            }
            ++*vcycles;
        }
        CK(cudaGetLastError());
        ++*iters;
        if ((rc = sync_state(g, g->st_in, s))) return rc;
        const double rel = g->st_host->rel;
        if (use_net && *use_net && (!std::isfinite(rel) || g->st_host->status ||
                                    (o->net_precond == 1 && it >= 3 && rel > 0.5))) {
            *use_net = false;                     // the network does not help here: V-cycle from now on
            if (!std::isfinite(rel) || g->st_host->status) return LM_OK;   // restart from the outer residual
        }
        if (g->st_host->status) return LM_OK;     // breakdown: keep e so far
        if (rel <= o->inner_rtol) break;
    }
    return LM_OK;
}

// ---- mixed precision: float64 iterative refinement around float32 FCG+MG ----
// learned = true: warm start x0 = alpha s NN(features(f)) with the
// energy-optimal alpha (x0 = 0 when alpha <= 0), smoothed by one symmetric
// sweep pair; the inner preconditioner is the V-cycle, or (net_precond 1/2)
// the learned two-level cycle.
int solve_mixed_ir(lm_grid* g, const lm_solve_opts* o, lm_solve_result* res, bool learned) {
    cudaStream_t s = S(o->cuda_stream);
    int rc;
    if ((rc = build_mg(g, s))) return rc;
    if ((rc = init_state(g, g->st, o->rtol, s))) return rc;
    const bool have_net = learned && lm::net_usable(g);
    bool use_net = have_net && o->net_precond != 0;     // network as the inner preconditioner
    const bool x0 = o->use_x0 && g->have_x0;
    if (x0) CK(cudaMemcpyAsync(g->x, g->x0, sizeof(double) * g->N, cudaMemcpyDeviceToDevice, s));
    bool warm = false;
    if (have_net && !x0) {
        // warm start: the scaled network guess, then one symmetric sweep pair
        // on its residual, x += S(f - A x), which removes the oscillatory
        // error a network leaves (large in the residual, small in the energy)
        if ((rc = lm::net_apply<double, double>(g, g->f, g->x, s))) return rc;
        launch_warm_scale(g->geo, g->G, s, op64(g), g->f, g->x, g->part);
        launch_ir_residual(g->geo, g->G, s, op64(g), g->f, g->x, g->r32, g->part, 0, g->st, 1, nullptr);
        const int order[2] = {0, 1};
        sweep_chain(g->mg[0], s, 2, order, nullptr, true, nullptr, nullptr, g->r32, g->e32);
        launch_ir_correct(g->N, g->G, s, g->x, g->e32);
        warm = true;
    }
    launch_ir_residual(g->geo, g->G, s, op64(g), g->f, g->x, g->r32, g->part, !(x0 || warm), g->st, 1, nullptr);
    CK(cudaGetLastError());
    if ((rc = sync_state(g, g->st, s))) return rc;
    if (warm && !std::isfinite(g->st_host->rel)) {   // a non-finite warm start: start from zero
        launch_ir_residual(g->geo, g->G, s, op64(g), g->f, g->x, g->r32, g->part, 1, g->st, 1, nullptr);
        if ((rc = sync_state(g, g->st, s))) return rc;
    }
    g->history.assign(1, g->st_host->rel);
    if (!(g->st_host->fnorm > 0.0)) {
        res->rel_residual = 0.0;
        return LM_OK;
    }
    double rel = g->st_host->rel;
    const double fnorm = g->st_host->fnorm, sqN = std::sqrt((double)g->N);
    // The inner right-hand side is r32 = r * rs, rs a power of two near
    // 1/rms(r): the float32 inner solve is linear, and a right-hand side of
    // about unit size keeps the products in its dot products clear of
    // float32 underflow as the refinement drives r down.  The first residual
    // is written unscaled and rescaled only when far from unit size; later
    // ones are scaled as they are written, from the previous norm times the
    // inner reduction.  The correction is scaled back exactly.
    double rs = pow2_near_inv(rel * fnorm / sqN);
    if (rs > 0x1p20 || rs < 0x1p-20) launch_scale32(g->N, g->G, s, g->r32, (float)rs);
    else rs = 1.0;
    int outer = 0, iters = 0, vc = 0;
    int status = LM_OK;
    while (rel > o->rtol && outer < o->max_outer && iters < o->max_iter) {
        bool deferred = false;
        if ((rc = inner_fcg(g, o, s, &iters, &vc, &use_net, &deferred))) return rc;
        if (!deferred && g->st_host->status) status = g->st_host->status;
        launch_ir_correct(g->N, g->G, s, g->x, g->e32, 1.0 / rs);
        const double rs_next = pow2_near_inv(rel * fnorm * std::max(o->inner_rtol, 1e-12) / sqN);
        launch_ir_residual(g->geo, g->G, s, op64(g), g->f, g->x, g->r32, g->part, 0, g->st, 0, nullptr, rs_next);
        CK(cudaGetLastError());
        if ((rc = sync_state(g, g->st, s))) return rc;     // also the inner state queued before
        if (deferred) {
            account_device_inner(g, &iters, &vc);
            if (g->st_host[1].status) status = g->st_host[1].status;
        }
        const double nrel = g->st_host->rel;
        g->history.push_back(nrel);
        ++outer;
        rs = rs_next;
        if (!(nrel < rel) && status) break;       // inner breakdown and no progress
        rel = nrel;
        status = LM_OK;
    }
    res->iters = iters;
    res->outer_iters = outer;
    res->vcycles += vc;
    res->rel_residual = rel;
    if (status) return status;
    return rel <= o->rtol ? LM_OK : LM_ERR_NO_CONVERGENCE;
}

int copy_in(lm_grid* g, double* dst, const double* src, int on_device, cudaStream_t s, bool sync = true) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * g->N,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (!on_device && sync) CK(cudaStreamSynchronize(s));   // the caller may reuse its host buffer
    return LM_OK;
}

int assemble(lm_grid* g, const double* a_in, const double* rho_new, const double* cs2, double dt, int raw,
             int on_device, cudaStream_t s) {
    if (!g || !a_in || !rho_new || (!raw && !cs2)) return LM_ERR_INVALID_ARG;
    if (!raw && !(dt > 0.0 && std::isfinite(dt))) return LM_ERR_NOT_POSITIVE;
    const double* A = a_in;
    const double* R = rho_new;
    const double* C = cs2;
    int rc;
    // flags: max 0, min all ones, no failures
    CK(cudaMemsetAsync(g->asm_fl, 0, sizeof(AsmFlags), s));
    CK(cudaMemsetAsync(&g->asm_fl->rho_min, 0xff, sizeof(unsigned long long), s));
    Op64Out dst{g->ct, g->gx, g->gy, g->gz, g->dinv, g->ct32, g->rho32};
    if (!on_device) {
        // Host inputs: copied in chunks of planes on the grid's copy stream,
        // each chunk assembled on s as soon as it has arrived, so the copies
        // (bound by the host link) and the assembly (bound by the float64
        // pipe) overlap.  A cell reads rho^{n+1} of its own plane and the one
        // below (minus faces only); on a periodic z axis plane 0 reads the
        // last plane, which is copied first.  The host buffers are free again
        // once the stream is waited for, before this call returns.
        if (!g->stage && (rc = dalloc(&g->stage, (size_t)3 * g->N))) return rc;
        if (!g->copy_stream) {
            CK(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
            for (cudaEvent_t& e : g->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        A = g->stage;
        R = g->stage + g->N;
        C = raw ? nullptr : g->stage + 2 * (size_t)g->N;
        const double* src[3] = {a_in, rho_new, cs2};
        double* dstp[3] = {g->stage, g->stage + g->N, g->stage + 2 * (size_t)g->N};
        const int narr = raw ? 2 : 3, nz = g->n[2];
        const size_t plane = (size_t)g->n[0] * g->n[1];
        // one chunk for small grids: the copies and launches of several cost more than they hide
        const int nch = g->N >= (1 << 20) ? std::min(8, nz) : 1;
        const bool wrap_z = nch > 1 && g->bc[2] == LM_BC_PERIODIC;
        CK(cudaEventRecord(g->ev_in, s));                    // an earlier assembly may still read the stage
        CK(cudaStreamWaitEvent(g->copy_stream, g->ev_in, 0));
        auto copy = [&](int a, int k0, int k1) -> cudaError_t {
            const size_t o = (size_t)k0 * plane;
            return cudaMemcpyAsync(dstp[a] + o, src[a] + o, sizeof(double) * plane * (k1 - k0), cudaMemcpyHostToDevice,
                                   g->copy_stream);
        };
        if (wrap_z) CK(copy(1, nz - 1, nz));
        for (int c = 0; c < nch; ++c) {
            const int k0 = (int)((long long)nz * c / nch), k1 = (int)((long long)nz * (c + 1) / nch);
            for (int a = 0; a < narr; ++a) {
                const int e1 = (a == 1 && wrap_z && c == nch - 1) ? k1 - 1 : k1;   // the last plane is there already
                if (e1 > k0) CK(copy(a, k0, e1));
            }
            CK(cudaEventRecord(g->ev_chunk[c], g->copy_stream));
            CK(cudaStreamWaitEvent(s, g->ev_chunk[c], 0));
            launch_assemble(g->geo, g->G, s, A, R, C, dt, raw, g->h, dst, g->asm_fl, (int)(k0 * plane),
                            (int)(k1 * plane));
        }
    } else {
        launch_assemble(g->geo, g->G, s, A, R, C, dt, raw, g->h, dst, g->asm_fl);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(g->asm_fl_host, g->asm_fl, sizeof(AsmFlags), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    g->mg_built = false;
    g->have_dinv = false;
    return lm::grid_finish_assembly(g, *g->asm_fl_host, s);
}

}  // namespace

// After an assembly: the positivity verdict and the float32 range handling.
int lm::grid_finish_assembly(lm_grid* g, const AsmFlags& fl, cudaStream_t s) {
    g->mg_built = false;
    g->have_dinv = false;
    if (fl.bad) {
        g->have_coefs = false;
        return LM_ERR_NOT_POSITIVE;
    }
    // Range of the float32 copy of rho.  The whole-row sweep forms both faces
    // of an axis from one reciprocal of the product (rho_c + rho_m)(rho_c +
    // rho_p), with rho = 1e30 (about 2^99.7) past a wall: that stays a normal
    // float32 while rho <= 2^26 and rho >= 2^-60.  Outside that band the copy
    // is divided by a power of two centred on the geometric mean of the
    // extremes (an exact scaling; the level face factors are divided by the
    // same power); a range that no scaling fits (max/min >= 2^86), or a c~
    // outside float32, leaves only the float64 Jacobi-PCG mode available.
    double rmax = 0.0, rmin = 0.0;
    std::memcpy(&rmax, &fl.rho_max, sizeof rmax);
    std::memcpy(&rmin, &fl.rho_min, sizeof rmin);
    constexpr double HI = 0x1p26, LO = 0x1p-60;
    double scale = 1.0;
    if (rmax > HI || rmin < LO) scale = std::ldexp(1.0, (int)std::lround(0.5 * (std::log2(rmax) + std::log2(rmin))));
    g->fp32_ok = !fl.bad32 && rmax / scale <= HI && rmin / scale >= LO;
    if (scale != 1.0 && g->fp32_ok) launch_scale32(g->N, g->G, s, g->rho32, (float)(1.0 / scale));
    if (scale != g->rho_scale) {
        // the level views carry the old face factors (and captured graphs and
        // batch plans hold them): rebuild the hierarchy from scratch
        free_mg(g);
        lm::batch_forget_grid(g);
        ++g->version;
        g->rho_scale = scale;
    }
    CK(cudaGetLastError());
    g->have_coefs = true;
    return LM_OK;
}

int lm::grid_build_mg(lm_grid* g, cudaStream_t s, bool defer_inverse) { return build_mg(g, s, defer_inverse); }
lm::Lev32 lm::make_level(const int n[3], const int bc[3], const double h[3], const float* ct, const float* rho,
                         double rho_scale) {
    return make_lev(n, bc, h, ct, rho, rho_scale);
}

// ============================ C ABI =========================================

extern "C" {

void lm_default_opts(lm_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->mode = LM_MIXED_MG_IR;
    o->rtol = 1e-8;
    o->max_iter = 10000;
    o->use_x0 = 0;
    o->max_outer = 12;
    o->nu1 = 2;
    o->nu2 = 3;
    o->inner_rtol = 1e-4;
    o->inner_max_iter = 30;
    o->check_every = 8;
    o->net_precond = 0;
    o->cuda_stream = nullptr;
}

const char* lm_status_string(int s) {
    switch (s) {
        case LM_OK: return "ok";
        case LM_ERR_INVALID_ARG: return "invalid argument";
        case LM_ERR_NOT_POSITIVE: return "coefficients not strictly positive and finite (rho, c_s^2, dt, c~)";
        case LM_ERR_NO_CONVERGENCE: return "no convergence within the iteration limit";
        case LM_ERR_BREAKDOWN: return "Krylov breakdown (p^T A p <= 0 or non-finite)";
        case LM_ERR_TIMEOUT: return "bounded device wait expired";
        case LM_ERR_CUDA: return "CUDA runtime error";
        case LM_ERR_NETWORK: return "network weights missing or malformed";
        case LM_ERR_OUT_OF_MEMORY: return "out of device memory";
        case LM_ERR_STATE: return "coefficients or right-hand side not set";
        default: return "unknown status";
    }
}

int lm_grid_create(int ndim, const int64_t n[3], const double h[3], const int bc[3], lm_grid** out) {
    if (!out || !n || !h || !bc || (ndim != 2 && ndim != 3)) return LM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || !(h[a] > 0.0) || !std::isfinite(h[a])) return LM_ERR_INVALID_ARG;
        if (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN) return LM_ERR_INVALID_ARG;
    }
    if (ndim == 2 && n[1] != 1) return LM_ERR_INVALID_ARG;
    const long long N = (long long)n[0] * n[1] * n[2];
    if (N >= (1LL << 31)) return LM_ERR_INVALID_ARG;
    lm_grid* g = new (std::nothrow) lm_grid();
    if (!g) return LM_ERR_OUT_OF_MEMORY;
    g->ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        g->n[a] = (int)n[a];
        g->h[a] = h[a];
        g->bc[a] = bc[a];
    }
    g->N = (int)N;
    int rc = LM_OK;
    auto fail = [&](int code) {
        lm_grid_destroy(g);
        return code;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess) return fail(LM_ERR_CUDA);
    // the whole-row and one-block coarse-cycle kernels need more than the
    // default 48 KB of shared memory: allow it before any entry point launches them
    rbgs_row_allow_smem();
    coarse_cycle_allow_smem();
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, g->device);
    const long long want = (N + NT - 1) / NT;
    g->G = (int)std::max(1LL, std::min<long long>(want, std::min<long long>(MAX_PARTIALS, (long long)nsm * 8)));
    g->geo = make_lev(g->n, g->bc, g->h, nullptr, nullptr).g;
    double** d64[] = {&g->ct, &g->gx, &g->gy, &g->gz, &g->dinv, &g->f, &g->x, &g->r, &g->p, &g->q};
    for (double** p : d64)
        if ((rc = dalloc(p, N))) return fail(rc);
    float** d32[] = {&g->ct32, &g->rho32, &g->r32, &g->e32, &g->z32, &g->p32, &g->q32, &g->tmp_a, &g->tmp_b};
    for (float** p : d32)
        if ((rc = dalloc(p, N))) return fail(rc);
    if ((rc = dalloc(&g->part, (size_t)NSLOT * MAX_PARTIALS))) return fail(rc);
    if ((rc = dalloc(&g->dscal, 8))) return fail(rc);
    if ((rc = dalloc(&g->scal, 16))) return fail(rc);
    if ((rc = dalloc(&g->ctr, 1))) return fail(rc);
    if (cudaMemset(g->ctr, 0, sizeof(unsigned int)) != cudaSuccess) return fail(LM_ERR_CUDA);
    if ((rc = dalloc(&g->st, 1))) return fail(rc);
    if ((rc = dalloc(&g->st_in, 1))) return fail(rc);
    if ((rc = dalloc(&g->asm_fl, 1))) return fail(rc);
    // st_host[0]: the state last waited for; st_host[1]: a device-side inner solve's
    if (cudaMallocHost((void**)&g->st_host, 2 * sizeof(SolveState)) != cudaSuccess) return fail(LM_ERR_OUT_OF_MEMORY);
    if (cudaMallocHost((void**)&g->asm_fl_host, sizeof(AsmFlags)) != cudaSuccess) return fail(LM_ERR_OUT_OF_MEMORY);
    if (cudaMallocHost((void**)&g->dscal_host, 8 * sizeof(double)) != cudaSuccess) return fail(LM_ERR_OUT_OF_MEMORY);
    if (cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess) return fail(LM_ERR_CUDA);
    if (cudaMemset(g->part, 0, sizeof(double) * NSLOT * MAX_PARTIALS) != cudaSuccess) return fail(LM_ERR_CUDA);
    *out = g;
    return LM_OK;
}

void lm_grid_destroy(lm_grid* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    lm::batch_forget_grid(g);
    if (g->net) lm_net_destroy(g->net);
    cudaFree(g->feat);
    cudaFree(g->nny);
    free_mg(g);
    void* bufs[] = {g->ct, g->gx, g->gy, g->gz, g->dinv, g->f, g->x, g->x0, g->r, g->p, g->q,
                    g->ct32, g->rho32, g->r32, g->e32, g->z32, g->p32, g->q32, g->tmp_a, g->tmp_b,
                    g->scal, g->ctr, g->stage, g->part,
                    g->dscal, g->st, g->st_in, g->hist_dev, g->asm_fl};
    for (void* b : bufs) cudaFree(b);
    cudaFreeHost(g->st_host);
    cudaFreeHost(g->asm_fl_host);
    cudaFreeHost(g->dscal_host);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    for (cudaGraphExec_t& e : g->ig_exec)
        if (e) cudaGraphExecDestroy(e);
    if (g->loop_exec) cudaGraphExecDestroy(g->loop_exec);
    cudaFree(g->d_inner_it);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->cap_body) cudaStreamDestroy(g->cap_body);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    for (cudaEvent_t e : g->ev_chunk)
        if (e) cudaEventDestroy(e);
    delete g;
}

int64_t lm_grid_size(const lm_grid* g) { return g ? (int64_t)g->N : 0; }

int64_t lm_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int lm_set_coefficients(lm_grid* g, const double* rho_old, const double* rho_new, const double* cs2, double dt,
                        int on_device, void* stream) {
    return assemble(g, rho_old, rho_new, cs2, dt, 0, on_device, S(stream));
}

int lm_set_coefficients_raw(lm_grid* g, const double* ctilde, const double* rho_face_src, int on_device,
                            void* stream) {
    return assemble(g, ctilde, rho_face_src, nullptr, 1.0, 1, on_device, S(stream));
}

int lm_set_rhs(lm_grid* g, const double* f, int on_device, void* stream) {
    if (!g || !f) return LM_ERR_INVALID_ARG;
    int rc = copy_in(g, g->f, f, on_device, S(stream));
    if (rc) return rc;
    g->have_rhs = true;
    return LM_OK;
}

int lm_set_initial_guess(lm_grid* g, const double* x0, int on_device, void* stream) {
    if (!g || !x0) return LM_ERR_INVALID_ARG;
    int rc;
    if (!g->x0 && (rc = dalloc(&g->x0, g->N))) return rc;
    if ((rc = copy_in(g, g->x0, x0, on_device, S(stream)))) return rc;
    g->have_x0 = true;
    return LM_OK;
}

int lm_load_network(lm_grid* g, const char* path) {
    if (!g || !path) return LM_ERR_INVALID_ARG;
    lm_net* N = nullptr;
    int rc = lm_net_load(path, &N);
    if (rc) return rc;
    if (g->net) lm_net_destroy(g->net);
    g->net = N;
    if (!g->feat && (rc = dalloc(&g->feat, (size_t)3 * g->N))) return rc;
    if (!g->nny && (rc = dalloc(&g->nny, g->N))) return rc;
    return LM_OK;
}

int lm_solve(lm_grid* g, const lm_solve_opts* o, lm_solve_result* res) {
    if (!g || !o) return LM_ERR_INVALID_ARG;
    lm_solve_result dummy;
    if (!res) res = &dummy;
    std::memset(res, 0, sizeof *res);
    if (!g->have_coefs || !g->have_rhs) return res->status = LM_ERR_STATE;
    if (!(o->rtol > 0.0) || o->max_iter < 1) return res->status = LM_ERR_INVALID_ARG;
    const bool mg = o->mode != LM_FP64_JACOBI_PCG;
    if (mg && (!mg_supported(g) || o->nu1 < 1 || o->nu2 < 1 || o->nu1 > 8 || o->nu2 > 8))
        return res->status = LM_ERR_INVALID_ARG;
    if (o->mode < 0 || o->mode > LM_MIXED_LEARNED_FCG_IR) return res->status = LM_ERR_INVALID_ARG;
    cudaStream_t s = S(o->cuda_stream);
    CK(cudaEventRecord(g->ev0, s));
    int rc;
    switch (o->mode) {
        case LM_FP64_JACOBI_PCG: rc = solve_jacobi_pcg(g, o, res); break;
        case LM_FP64_MG_PCG: rc = solve_mg_pcg(g, o, res); break;
        case LM_MIXED_MG_IR: rc = solve_mixed_ir(g, o, res, false); break;
        default: rc = solve_mixed_ir(g, o, res, true); break;
    }
    cudaEventRecord(g->ev1, s);
    cudaEventSynchronize(g->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    res->seconds = ms * 1e-3;
    res->status = rc;
    return rc;
}

int lm_get_solution(lm_grid* g, double* out, int on_device, void* stream) {
    if (!g || !out) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    CK(cudaMemcpyAsync(out, g->x, sizeof(double) * g->N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       s));
    if (!on_device) CK(cudaStreamSynchronize(s));
    return LM_OK;
}

int lm_get_residual_history(lm_grid* g, double* out, int cap, int* n_written) {
    if (!g || (!out && cap > 0)) return LM_ERR_INVALID_ARG;
    const int n = std::min<int>(cap, (int)g->history.size());
    if (n > 0) std::memcpy(out, g->history.data(), sizeof(double) * n);
    if (n_written) *n_written = (int)g->history.size();
    return LM_OK;
}

int lm_get_coefficients(lm_grid* g, double* ctilde, double* gx, double* gy, double* gz, void* stream) {
    if (!g) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    cudaStream_t s = S(stream);
    const size_t B = sizeof(double) * g->N;
    if (ctilde) CK(cudaMemcpyAsync(ctilde, g->ct, B, cudaMemcpyDeviceToDevice, s));
    if (gx) CK(cudaMemcpyAsync(gx, g->gx, B, cudaMemcpyDeviceToDevice, s));
    if (gy) CK(cudaMemcpyAsync(gy, g->gy, B, cudaMemcpyDeviceToDevice, s));
    if (gz) CK(cudaMemcpyAsync(gz, g->gz, B, cudaMemcpyDeviceToDevice, s));
    return LM_OK;
}

int lm_apply(lm_grid* g, int prec, const void* x, void* y, double* dot_out, void* stream) {
    if (!g || !x || !y || (prec != LM_PREC_FP64 && prec != LM_PREC_FP32)) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    cudaStream_t s = S(stream);
    const double* dot_dev = g->dscal;
    if (prec == LM_PREC_FP64) {
        launch_apply64(g->geo, g->G, s, op64(g), (const double*)x, (double*)y, dot_out ? g->part : nullptr);
        if (dot_out) launch_reduce_slot(g->part, 0, g->G, s, g->dscal);
    } else {
        if (!g->fp32_ok) return LM_ERR_INVALID_ARG;
        Lev32 L = make_lev(g->n, g->bc, g->h, g->ct32, g->rho32, g->rho_scale);
        const Red red{g->part, g->scal, g->ctr};
        launch_apply32(L, s, (const float*)x, (float*)y, nullptr, red, dot_out ? 0 : -1, -1);
        dot_dev = g->scal;
    }
    CK(cudaGetLastError());
    if (dot_out) {
        CK(cudaMemcpyAsync(g->dscal_host, dot_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *dot_out = g->dscal_host[0];
    }
    return LM_OK;
}

int lm_mg_vcycle(lm_grid* g, const float* r, float* z, int nu1, int nu2, void* stream) {
    if (!g || !r || !z || nu1 < 1 || nu2 < 1 || nu1 > 8 || nu2 > 8) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!mg_supported(g)) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    int rc = build_mg(g, s);
    if (rc) return rc;
    vcycle(g, 0, z, r, nu1, nu2, s);
    CK(cudaGetLastError());
    return LM_OK;
}

int lm_mg_sweep(lm_grid* g, const float* x_in, const float* f, float* x_out, int order, void* stream) {
    if (!g || !f || !x_out || (order != 0 && order != 1) || x_out == x_in || x_out == f) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!mg_supported(g)) return LM_ERR_INVALID_ARG;
    cudaStream_t s = S(stream);
    int rc = build_mg(g, s);
    if (rc) return rc;
    launch_rbgs(g->mg[0].L, s, x_in, nullptr, nullptr, 0, 0, 0, f, x_out, order, x_in == nullptr, false);
    CK(cudaGetLastError());
    return LM_OK;
}

int lm_mg_level_shape(lm_grid* g, int level, int64_t n_out[3], int* num_levels) {
    if (!g || !n_out) return LM_ERR_INVALID_ARG;
    if (!g->have_coefs) return LM_ERR_STATE;
    if (!mg_supported(g)) return LM_ERR_INVALID_ARG;
    int rc = build_mg(g, 0);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    if (num_levels) *num_levels = (int)g->mg.size();
    if (level < 0 || level >= (int)g->mg.size()) return LM_ERR_INVALID_ARG;
    n_out[0] = g->mg[level].L.g.nx;
    n_out[1] = g->mg[level].L.g.ny;
    n_out[2] = g->mg[level].L.g.nz;
    return LM_OK;
}

}  // extern "C"
