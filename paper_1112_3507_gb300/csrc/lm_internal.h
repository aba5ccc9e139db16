// Internal definitions shared by the solver's host translation units
// (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace lm {

constexpr int COARSE_MAX = 16;      // coarsen while a level has more cells than this and an axis halves
constexpr int COARSE_EXACT = 64;    // a coarsest level of at most this many cells is solved exactly
constexpr int COARSE_SWEEPS = 32;   // (RB, BR) sweep pairs when it cannot be

struct MgLevel {
    Lev32 L;
    double h[3];
    int halved[3] = {0, 0, 0};      // axes halved to reach the next level
    float* ct = nullptr;            // coefficients (owned on levels >= 1)
    float* rho = nullptr;
    float* xa = nullptr;            // sweep buffers (level 0: the grid's tmp_a/tmp_b)
    float* xb = nullptr;
    float* xo = nullptr;            // V-cycle output (levels >= 1; level 0 writes the caller's z)
    float* f = nullptr;             // right-hand side (levels >= 1)
    float* ainv = nullptr;          // dense inverse on a direct coarsest level
};

}  // namespace lm

struct lm_net;
using lm::Geo;
using lm::Op64;
using lm::SolveState;

struct lm_grid {
    int ndim = 0;
    int n[3] = {1, 1, 1};
    double h[3] = {1, 1, 1};
    int bc[3] = {0, 0, 0};
    int N = 0;
    int device = 0;
    int G = 1;          // blocks of the grid-stride streaming kernels
    Geo geo{};

    double *ct = nullptr, *gx = nullptr, *gy = nullptr, *gz = nullptr, *dinv = nullptr;
    double *f = nullptr, *x = nullptr, *x0 = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    float *ct32 = nullptr, *rho32 = nullptr;
    float *r32 = nullptr, *e32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *tmp_a = nullptr, *tmp_b = nullptr;   // level-0 sweep buffers
    double* scal = nullptr;         // reduction results (float32 kernels)
    unsigned int* ctr = nullptr;    // last-block arrival counter
    double* stage = nullptr;        // 3N host-input staging (allocated on first use)
    // host inputs of an assembly arrive in chunks of planes on copy_stream
    // (one event per chunk) while the assembly of the chunks before runs
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_in = nullptr;
    cudaEvent_t ev_chunk[8] = {};
    double* part = nullptr;         // NSLOT * MAX_PARTIALS
    double* dscal = nullptr;        // device scalars for lm_apply dots
    SolveState* st = nullptr;       // outer solve state
    SolveState* st_in = nullptr;    // inner (float32) solve state
    SolveState* st_host = nullptr;  // pinned mirror
    double* hist_dev = nullptr;
    int hist_cap = 0;
    lm::AsmFlags* asm_fl = nullptr;         // assembly report (device) and its pinned mirror
    lm::AsmFlags* asm_fl_host = nullptr;
    // The float32 copy of rho^{n+1} holds rho / rho_scale (a power of two,
    // 1 unless rho leaves the band the float32 face formulas are safe in);
    // the float32 levels carry 2 / (h^2 rho_scale) so their faces are
    // unchanged.  fp32_ok: the float32 operator is representable at all.
    double rho_scale = 1.0;
    bool fp32_ok = true;
    double* dscal_host = nullptr;

    bool have_coefs = false, have_rhs = false, have_x0 = false;
    bool have_dinv = false;         // inverse Jacobi diagonal (formed on the first Jacobi solve)
    bool mg_built = false;
    bool inv_pending = false;       // hierarchy built, its coarsest inverse not yet computed
    unsigned version = 0;           // bumped when the hierarchy buffers are (re)allocated
    lm_net* net = nullptr;          // learned warm start / preconditioner (2D grids)
    float* feat = nullptr;          // network input (N x 3)
    float* nny = nullptr;           // network output (N)
    std::vector<lm::MgLevel> mg;
    int cc_level = -1;              // first level of the one-block coarse V-cycle (-1: none)
    std::vector<double> history;
    // CUDA graphs of one inner flexible-CG iteration with the V-cycle (the
    // first and the later ones), captured on cap_stream for hierarchy
    // version ig_version and smoothing (ig_nu1, ig_nu2); ig_nk kernels each
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_body = nullptr;     // captures the body of the device-side loop
    // The whole inner solve as one graph: its set-up, the first iteration,
    // then a conditional while node repeating the later iteration until the
    // inner tolerance or the iteration limit (loop_nk: kernels before the
    // loop and in one loop pass); keyed like ig_exec plus the limit
    cudaGraphExec_t loop_exec = nullptr;
    long long loop_nk[2] = {0, 0};
    unsigned loop_version = ~0u;
    int loop_nu1 = -1, loop_nu2 = -1, loop_max = -1;
    double loop_rtol = -1.0;
    int* d_inner_it = nullptr;           // iterations of the current inner solve (device)
    cudaGraphExec_t ig_exec[2] = {nullptr, nullptr};
    long long ig_nk[2] = {0, 0};
    unsigned ig_version = ~0u;
    int ig_nu1 = -1, ig_nu2 = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};


namespace lm {
// multigrid hierarchy (idempotent); defer_inverse leaves the coarsest inverse
// to the caller (inv_pending), which computes many grids' in one launch
int grid_build_mg(lm_grid* g, cudaStream_t s, bool defer_inverse = false);
// the end of an assembly (host): positivity verdict, float32 range of rho,
// hierarchy invalidation; fl = the assembly's report, already on the host
int grid_finish_assembly(lm_grid* g, const AsmFlags& fl, cudaStream_t s);
void batch_forget_grid(const lm_grid* g);            // drop cached batch plans that use g
int net_forward(lm_net* N, const float* x, float* y, int B, int H, int W, cudaStream_t s);
int net_backward(lm_net* N, const float* gy, cudaStream_t s);
int net_create(const int ch[4], lm_net** out);
void net_destroy(lm_net* N);
int net_set_params(lm_net* N, const float* host, int n);
bool net_usable(const lm_grid* g);
template <typename TV, typename TO>
int net_apply(lm_grid* g, const TV* v, TO* dst, cudaStream_t s);
Lev32 make_level(const int n[3], const int bc[3], const double h[3], const float* ct, const float* rho,
                 double rho_scale = 1.0);
}  // namespace lm
