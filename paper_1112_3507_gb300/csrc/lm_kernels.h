// Host-visible kernel interfaces of the solver library (internal).
#pragma once

#include <cuda_runtime.h>

#include "lm_common.cuh"

namespace lm {

// Number of kernels this library has launched (all grids, all streams).
void count_launches(long long n);

// Float64 operator: c~, minus-face conductances per axis, inverse diagonal.
struct Op64 {
    const double* ct;
    const double* gx;
    const double* gy;
    const double* gz;
    const double* dinv;
};
struct Op64Out {
    double* ct;
    double* gx;
    double* gy;
    double* gz;
    double* dinv;
    float* ct32;
    float* rho32;
};

struct PcgArgs {
    Geo g;
    Op64 op;
    const double* f;
    double* x;
    double* r;
    double* p;
    double* q;
    double* part;     // NSLOT * MAX_PARTIALS
    SolveState* st;
    double* hist;     // max_iter + 1
    int max_iter;
};

// One float32 multigrid level (device view).  Faces are formed on the fly
// from rho: g = 2 (1/h^2) / (rho_L + rho_R).
struct Lev32 {
    Geo g;
    float c2x, c2y, c2z;     // 2/h^2 per axis
    const float* ct;
    const float* rho;
};

// What the assembly reports besides the coefficients: the range of rho^{n+1}
// (float64 bit patterns, monotone in the value for positive numbers), a
// positivity/finiteness failure, and a c~ outside float32 range.
struct AsmFlags {
    unsigned long long rho_max;
    unsigned long long rho_min;
    int bad;        // rho, c_s^2, dt or c~ not strictly positive and finite
    int bad32;      // c~ overflows or underflows float32
};

// Everything the assembly of one grid reads and writes.
struct AsmArgs {
    Geo g;
    const double* a_in;      // rho^n (or c~ when raw)
    const double* rho_new;
    const double* cs2;
    double dt;
    int raw;
    double c2x, c2y, c2z;    // 2 / h^2 per axis
    Op64Out out;
    AsmFlags* fl;
};
inline AsmArgs asm_args(const Geo& g, const double* a_in, const double* rho_new, const double* cs2, double dt,
                        int raw, const double h[3], const Op64Out& out, AsmFlags* fl) {
    return AsmArgs{g, a_in, rho_new, cs2, dt, raw, 2.0 / (h[0] * h[0]), 2.0 / (h[1] * h[1]), 2.0 / (h[2] * h[2]),
                   out, fl};
}

// fp64
void launch_assemble(const Geo& g, int G, cudaStream_t s, const double* a_in, const double* rho_new,
                     const double* cs2, double dt, int raw, const double h[3], const Op64Out& out, AsmFlags* fl,
                     int i0 = 0, int i1 = -1);
// x *= scale (float32; scale a power of two, so the scaling is exact)
void launch_scale32(int N, int G, cudaStream_t s, float* x, float scale);
void launch_jacobi_diag(const Geo& g, int G, cudaStream_t s, const Op64& op, double* dinv);
void launch_apply64(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* x, double* y,
                    double* part);
void launch_pcg_init(const PcgArgs& a, int G, cudaStream_t s, int use_x0);
void launch_pcg_restart(const PcgArgs& a, int G, cudaStream_t s, int k);
// the operator-free steps of one Jacobi-PCG iteration, for operators applied
// elsewhere: p = D^-1 r with r.z (after the residual), the x, r update after
// q = A p with its p.q partials (slot 0), and the convergence test with the p update
void launch_pcg_init_p(const PcgArgs& a, int G, cudaStream_t s, int rz_slot, int restart);
void launch_pcg_xr(const PcgArgs& a, int G, cudaStream_t s, int k);
void launch_pcg_p(const PcgArgs& a, int G, cudaStream_t s, int k);
void launch_pcg_iter(const PcgArgs& a, int G, cudaStream_t s, int k);
void launch_true_residual(const PcgArgs& a, int G, cudaStream_t s);
void launch_ir_residual(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* f, double* x,
                        float* r32, double* part, int zero_x, SolveState* st, int set_fnorm, double* hist_entry,
                        double rscale = 1.0);
void launch_warm_scale(const Geo& g, int G, cudaStream_t s, const Op64& op, const double* f, double* x,
                       double* part);
void launch_ir_correct(int N, int G, cudaStream_t s, double* x, const float* e, double escale = 1.0);
void launch_reduce_rel(double* part, int G, cudaStream_t s, SolveState* st, double* hist_entry);
void launch_reduce_slot(const double* part, int slot, int G, cudaStream_t s, double* out);
void launch_fcg64_iter_a(int N, int G, cudaStream_t s, const float* z, const double* q, double* part, int first,
                         double* p, const SolveState* st);
void launch_fcg64_iter_b(const Geo& g, int G, cudaStream_t s, const Op64& op, double* x, double* r, float* r32,
                         const double* p, double* q, double* part, SolveState* st);
void launch_to32(int N, int G, cudaStream_t s, const double* r, float* r32);
void launch_set_fnorm(const double* part, int slot, int G, cudaStream_t s, SolveState* st);

// fp32 operator and flexible CG (reductions land in red.scal[slot]; slot < 0: none)
void launch_apply32(const Lev32& L, cudaStream_t s, const float* x, float* y, const float* r, const Red& red,
                    int slot_xy, int slot_xr);
void launch_dot32(int N, int G, cudaStream_t s, const float* a, const float* b, const Red& red, int slot,
                  SolveState* fnorm_st);
void launch_axpy32(int N, int G, cudaStream_t s, float alpha, const float* x, const float* y, float* out);
void launch_axpy_ratio32(int N, int G, cudaStream_t s, const double* scal, int num, int den, const float* x,
                         const float* y, float* out);
void launch_fcg_beta_p(int N, int G, cudaStream_t s, const float* z, float* p, const double* scal, int first);
void launch_fcg_update(int N, int G, cudaStream_t s, float* e, float* r, const float* p, const float* q,
                       const Red& red, SolveState* st);

// multigrid
void launch_coarsen(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s, float* ct_c,
                    float* rho_c);
void launch_rbgs(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx, int hy,
                 int hz, const float* f, float* xout, int first, int zero, int prolong);
void launch_rbgs_kz(const Lev32& L, cudaStream_t s, const float* xin, const float* ec, const Lev32* C, int hx,
                    int hy, int hz, const float* f, float* xout, int first, int zero, int prolong, int kz);
void launch_resid_restrict(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s,
                           const float* x, const float* f, float* fc);
// A whole coarse V-cycle (levels with at most CC_MAX_CELLS cells down to a
// directly solved coarsest level) run by one block.
constexpr int CC_MAXL = 5;
constexpr int CC_MAX_CELLS = 4096;
struct CoarseCycle {
    int nl;                        // levels in the chain; the last is solved with ainv
    Lev32 L[CC_MAXL];
    int hx[CC_MAXL], hy[CC_MAXL], hz[CC_MAXL];   // halvings from chain level i to i + 1
    float* x[CC_MAXL];             // level solutions (chain level 0: the caller's output)
    float* f[CC_MAXL];             // level right-hand sides (chain level 0: the caller's rhs)
    const float* ainv;
    int nu1, nu2;
};
constexpr int CC_THREADS = 1024;                 // threads of the block that runs a cycle
constexpr int CC_PER = CC_MAX_CELLS / CC_THREADS;  // cells a thread owns on a chain level
constexpr size_t CC_SMEM_MAX = 200 * 1024;       // shared-memory limit of the one-block cycle
// Shared memory of the one-block cycle over levels of N_0 .. N_{nl-1} cells:
// seven floats per cell and the dense inverse of the coarsest level.
inline size_t cc_smem_bytes(const int* N, int nl) {
    size_t b = 0;
    for (int l = 0; l < nl; ++l) b += 7 * sizeof(float) * (size_t)N[l];
    return b + sizeof(float) * (size_t)N[nl - 1] * (size_t)N[nl - 1];
}
inline size_t cc_smem_bytes(const CoarseCycle& cc) {
    int N[CC_MAXL];
    for (int l = 0; l < cc.nl; ++l) N[l] = cc.L[l].g.N;
    return cc_smem_bytes(N, cc.nl);
}
void launch_coarse_cycle(const CoarseCycle& cc, cudaStream_t s);
void coarse_cycle_allow_smem();
void rbgs_row_allow_smem();                      // raises the whole-row sweep's dynamic shared-memory limit                  // raises k_coarse_cycle's dynamic shared-memory limit
void launch_coarse_inverse(const Lev32& L, cudaStream_t s, float* ainv);
// one grid's coarsest level and where its dense inverse goes
struct CoarseInv {
    Lev32 L;
    float* ainv;
};
// rows (task & 255) of items[task >> 8] for every task: many grids' inverses in one launch
void launch_coarse_inverse_many(const CoarseInv* items, const int* task, int ntask, cudaStream_t s);
// one block per item: each grid's whole inverse (the factorisation done once per grid)
void launch_coarse_inverse_grids(const CoarseInv* items, int count, cudaStream_t s);
void launch_coarse_solve(int n, cudaStream_t s, const float* ainv, const float* f, float* x);

}  // namespace lm
