// Batched mixed-precision solve of many independent 2D grids of uneven size
// (lm_batch_solve).
//
// Every phase of the solve -- the float64 residual, each level's fused
// red-black sweeps, the fused residual + restriction, the exact coarsest
// solves, the flexible-CG vector steps and the float64 correction -- is one
// launch covering the tiles of every grid, through a task table (block b
// works on task[b] = grid, level, tile).  Per-grid device flags make the
// tiles of converged grids no-ops, so a fixed launch sequence serves grids
// that converge at different iterations; that sequence is captured once as
// a CUDA graph (one graph for the first residual, one per refinement step)
// and replayed.  No block ever waits for another: ordering comes from the
// kernel boundaries inside the graph.
//
// The sweep's z-chunk per level size is chosen by an autotuner that times
// the candidates on the first grid of each size class and keeps the result
// in a JSON cache file keyed by GPU name, level shape and boundary conditions.
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_internal.h"
#include "lm_kernels.h"
#include "lm_tiles.cuh"

namespace lm {

// ---- device tables ------------------------------------------------------------

struct BTask {
    int g, l, bx, by, bz, lblk, nblk;
};

struct BLev {
    Lev32 L;            // this level
    Geo C;              // the next (coarser) level
    int hx, hy, hz;     // halving to the next level
    int kz;             // sweep z-chunk (autotuned)
    int kr;             // coarse rows per warp of the 2D residual-restriction (0: the generic tile)
    float* xa;          // pre-smoothed iterate
    float* xb;          // sweep scratch (sweeps beyond the first of a pre- or post-smoothing chain)
    float* xo;          // V-cycle output (level 0: the grid's z)
    const float* f;     // right-hand side (level 0: the grid's r32)
    float* fc;          // the next level's right-hand side
    const float* ec;    // the next level's output (the coarse correction)
    const float* ainv;  // dense inverse on the coarsest level
};

struct BGrid {
    Geo geo;
    Op64 op;
    const double* f;
    double* x;
    float *r32, *e32, *z32, *p32, *q32;
    SolveState* st;     // outer (refinement) state: done = converged or failed
    SolveState* st_in;  // inner state: done = inner tolerance met
    Red red;
    int N;
    int kz_apply;       // rows per thread of the apply (seg_apply: rows per warp)
    int seg_apply;      // 1: the level-0 apply runs as apply2d_rows (seg2d_ok)
};

// scal slots per grid: 0 p.q, 1 r.r, 2 p.r, 3 z.q_old, 4 r0.r0, 5 float64 r.r, 6 f.f

__device__ __forceinline__ bool inner_off(const BGrid& G) { return G.st->done || G.st_in->done; }

__global__ void __launch_bounds__(NT) kb_init_states(const BGrid* __restrict__ Gs, int count, double rtol,
                                                     double inner_rtol) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    SolveState s{};
    s.rtol = rtol;
    *Gs[g].st = s;
    s.rtol = inner_rtol;
    s.done = 1;
    *Gs[g].st_in = s;
}

// r = f - A x in float64 (zero_x: x := 0, r = f), r32 = r; the grid's last
// block sets ||f|| (first residual of a solve), rel = ||r||/||f||, counts a
// refinement step (later residuals), and done when rel <= rtol.
__global__ void __launch_bounds__(NT) kb_ir_residual(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                     int zero_x, int first) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (G.st->done) return;
    __shared__ double sm[64];
    double acc[2] = {0.0, 0.0};
    const int stride = t.nblk * NT;
    for (int idx = t.lblk * NT + threadIdx.x; idx < G.N; idx += stride) {
        const double fi = G.f[idx];
        const double ri = zero_x ? fi : fi - apply64_at(idx, G.geo, G.op, G.x);
        G.r32[idx] = (float)ri;
        acc[0] += ri * ri;
        if (first) acc[1] += fi * fi;                 // ||f|| is kept from the first residual
    }
    if (zero_x)
        for (int idx = t.lblk * NT + threadIdx.x; idx < G.N; idx += stride) G.x[idx] = 0.0;
    const int sl[2] = {5, 6};
    if (grid_reduce_n<2>(acc, G.red, sl, sm, t.lblk, t.nblk) && lin_tid() == 0) {
        if (first) G.st->fnorm = sqrt(G.red.scal[6]);
        const double fn = G.st->fnorm;
        const double rel = fn > 0.0 ? sqrt(G.red.scal[5]) / fn : 0.0;
        G.st->rel = rel;
        if (!first) G.st->iters += 1;
        if (!isfinite(rel)) {
            G.st->status = LM_ERR_BREAKDOWN;
            G.st->done = 1;
        } else if (rel <= G.st->rtol) {
            G.st->converged = 1;
            G.st->done = 1;
        }
    }
}

// e = 0; ||r32|| of the inner problem; re-arm the inner state; block 0
// zeroes the inner-iteration counter of the refinement step
__global__ void __launch_bounds__(NT) kb_inner_init(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                    int* __restrict__ inner_it) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *inner_it = 0;
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (G.st->done) return;
    __shared__ double sm[32];
    const int stride = t.nblk * NT;
    for (int idx = t.lblk * NT + threadIdx.x; idx < G.N; idx += stride) G.e32[idx] = 0.f;
    const FF a = dot32_range(G.N, G.r32, G.r32, t.lblk, t.nblk);
    double v[1] = {ff_value(a)};
    const int sl[1] = {4};
    if (grid_reduce_n<1>(v, G.red, sl, sm, t.lblk, t.nblk) && lin_tid() == 0) {
        const double fn = sqrt(G.red.scal[4]);
        G.st_in->fnorm = fn;
        G.st_in->rel = 1.0;
        G.st_in->status = 0;
        G.st_in->done = fn > 0.0 ? 0 : 1;
    }
}

// The level buffer a batched sweep reads or writes: 1 xa, 2 xb, 3 xo.
__device__ __forceinline__ float* lev_buf(const BLev& V, int sel) {
    return sel == 1 ? V.xa : sel == 2 ? V.xb : V.xo;
}

// One red-black sweep of every grid's level (task t.l) from buffer `src`
// into buffer `dst`: ZERO, the first pre-smoothing sweep (from zero, red
// first); PROLONG, the first post-smoothing sweep (from xa plus the coarse
// correction, black first); otherwise a plain sweep in the chain's order.
// (CHECK false: every grid's tiles run, whatever the solve states -- the
// autotuner's timing launches.)
template <int FIRST, bool ZERO, bool PROLONG, bool CHECK = true>
__global__ void __launch_bounds__(128, 8) kb_rbgs(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                  const BLev* __restrict__ Ls, int src, int dst) {
    const BTask t = T[blockIdx.x];
    if (CHECK && inner_off(Gs[t.g])) return;
    const BLev& V = Ls[t.l];
    const float* xin = ZERO ? nullptr : lev_buf(V, src);
    float* xout = lev_buf(V, dst);
    if (V.L.g.nx % 128 == 0 && V.L.g.nz >= 2)        // rows of 128-cell segments: the warp z-march
        zrow2d_tile<FIRST, ZERO, PROLONG>(V.L, xin, PROLONG ? V.ec : nullptr, V.C, PROLONG ? V.hx : 0,
                                        PROLONG ? V.hz : 0, V.f, xout, V.kz, t.bx, t.by, zrow2d_width(V.L.g.nx));
    else
        rbgs_tile<128, 1, false, FIRST, ZERO, PROLONG>(V.L, xin, PROLONG ? V.ec : nullptr, V.C, PROLONG ? V.hx : 0,
                                                        PROLONG ? V.hy : 0, PROLONG ? V.hz : 0, V.f, xout, V.kz,
                                                        t.bx, t.by, 0);
}

__global__ void __launch_bounds__(256) kb_resid_restrict(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                         const BLev* __restrict__ Ls) {
    const BTask t = T[blockIdx.x];
    if (inner_off(Gs[t.g])) return;
    const BLev& V = Ls[t.l];
    if (V.kr) {                                    // rr2d_ok levels: a warp per segment and V.kr coarse rows
        const int K0 = (t.by * 8 + threadIdx.y) * V.kr;
        if (K0 < V.C.nz) rr2d_rows(V.L, V.C, V.xa, V.f, V.fc, t.bx * 128, K0, min(K0 + V.kr, V.C.nz));
        return;
    }
    resid_restrict_tile(V.L, V.C, V.hx, V.hy, V.hz, V.xa, V.f, V.fc, t.bx, t.by, t.bz);
}

// one block per grid: the grid's coarse V-cycle (its levels from the one-block
// cycle's first level down), in place of the per-level launches there
__global__ void __launch_bounds__(CC_THREADS, 1) kb_coarse_cycle(const CoarseCycle* __restrict__ ccs,
                                                        const BGrid* __restrict__ Gs) {
    if (inner_off(Gs[blockIdx.x])) return;
    coarse_cycle_block(ccs[blockIdx.x]);
}

__global__ void kb_coarse(const BTask* __restrict__ T, const BGrid* __restrict__ Gs, const BLev* __restrict__ Ls) {
    const BTask t = T[blockIdx.x];
    if (inner_off(Gs[t.g])) return;
    const BLev& V = Ls[t.l];
    coarse_solve_block(V.L.g.N, V.ainv, V.f, V.xo);
}

// z.q_old (not on the first inner iteration of a refinement step, *inner_it == 0)
__global__ void __launch_bounds__(NT) kb_dot_zq(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                const int* __restrict__ inner_it) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (inner_off(G) || *inner_it == 0) return;
    __shared__ double sm[32];
    const FF a = dot32_range(G.N, G.z32, G.q32, t.lblk, t.nblk);
    double v[1] = {ff_value(a)};
    const int sl[1] = {3};
    grid_reduce_n<1>(v, G.red, sl, sm, t.lblk, t.nblk);
}

__global__ void __launch_bounds__(NT) kb_beta_p(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                const int* __restrict__ inner_it) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (inner_off(G)) return;
    fcg_beta_p_range(G.N, G.z32, G.p32, G.red.scal, *inner_it == 0, t.lblk, t.nblk);
}

// End of one inner iteration of the device-side loop: count it, and keep
// looping while some grid is still iterating (neither converged overall nor
// at its inner tolerance) and the step's iteration limit is not reached.
__global__ void __launch_bounds__(256) kb_inner_cond(const BGrid* __restrict__ Gs, int count,
                                                     int* __restrict__ inner_it, int inner_max,
                                                     cudaGraphConditionalHandle loop) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int g = threadIdx.x; g < count; g += blockDim.x)
        if (!inner_off(Gs[g])) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int it = *inner_it + 1;
        *inner_it = it;
        cudaGraphSetConditional(loop, (any && it < inner_max) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(256) kb_apply(const BTask* __restrict__ T, const BGrid* __restrict__ Gs,
                                                const BLev* __restrict__ Ls, const int* __restrict__ lev0) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (inner_off(G)) return;
    __shared__ double sm[64];
    FF axy{0.f, 0.f}, axr{0.f, 0.f};
    const Lev32& L = Ls[lev0[t.g]].L;
    if (G.seg_apply) {
        const int k0 = (t.by * 8 + threadIdx.y) * G.kz_apply;
        if (k0 < L.g.nz)
            apply2d_rows<true, true>(L, G.p32, G.q32, G.r32, t.bx * 128, k0, min(k0 + G.kz_apply, L.g.nz), axy, axr);
    } else {
        apply32z_tile<false, true, true>(L, G.p32, G.q32, G.r32, G.kz_apply, t.bx, t.by, 0, axy, axr);
    }
    double v[2] = {ff_value(axy), ff_value(axr)};
    const int sl[2] = {0, 2};
    grid_reduce_n<2>(v, G.red, sl, sm, t.lblk, t.nblk);
}

__global__ void __launch_bounds__(NT, 4) kb_update(const BTask* __restrict__ T, const BGrid* __restrict__ Gs) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (inner_off(G)) return;
    __shared__ double sm[32];
    bool bad;
    const FF rr = fcg_update_range(G.N, G.e32, G.r32, G.p32, G.q32, G.red.scal, bad, t.lblk, t.nblk);
    double v[1] = {ff_value(rr)};
    const int sl[1] = {1};
    if (grid_reduce_n<1>(v, G.red, sl, sm, t.lblk, t.nblk) && lin_tid() == 0) {
        const double rel = sqrt(G.red.scal[1]) / G.st_in->fnorm;
        G.st_in->rel = rel;
        G.st_in->iters += 1;
        if (bad || !isfinite(rel)) {
            G.st_in->status = LM_ERR_BREAKDOWN;
            G.st_in->done = 1;
        } else if (rel <= G.st_in->rtol) {
            G.st_in->done = 1;
        }
    }
}

__global__ void __launch_bounds__(NT) kb_ir_correct(const BTask* __restrict__ T, const BGrid* __restrict__ Gs) {
    const BTask t = T[blockIdx.x];
    const BGrid& G = Gs[t.g];
    if (G.st->done) return;
    const int stride = t.nblk * NT;
    for (int idx = t.lblk * NT + threadIdx.x; idx < G.N; idx += stride) G.x[idx] += (double)G.e32[idx];
}

// out[g] = the outer state, out[count + g] = the inner state
__global__ void kb_gather(const BGrid* __restrict__ Gs, int count, SolveState* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    out[g] = *Gs[g].st;
    out[count + g] = *Gs[g].st_in;
}

// ---- batched set-up ------------------------------------------------------------

// Task t of a batched assembly: blocks lblk of nblk over grid g's cells.
__global__ void __launch_bounds__(NT) kb_assemble(const BTask* __restrict__ T, const AsmArgs* __restrict__ A) {
    const BTask t = T[blockIdx.x];
    assemble_range(A[t.g], t.lblk * NT + threadIdx.x, t.nblk * NT);
}

// flags of every grid to "nothing seen yet" (before), and gathered into one buffer (after)
__global__ void kb_asm_flags(const AsmArgs* __restrict__ A, int count, AsmFlags* __restrict__ out, int gather) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    if (gather) {
        out[g] = *A[g].fl;
    } else {
        AsmFlags f{};
        f.rho_max = 0ull;
        f.rho_min = ~0ull;
        *A[g].fl = f;
    }
}

// One coarsening step (level l -> l + 1) of many grids: task t is block
// (bx, by, bz) of the coarse level of item t.g.
struct BCoarsen {
    Lev32 F;
    Geo C;
    int hx, hy, hz;
    float *ct_c, *rho_c;
};
__global__ void __launch_bounds__(256) kb_coarsen(const BTask* __restrict__ T, const BCoarsen* __restrict__ items) {
    const BTask t = T[blockIdx.x];
    const BCoarsen& it = items[t.g];
    coarsen_cell(it.F, it.C, it.hx, it.hy, it.hz, it.ct_c, it.rho_c, t.bx, t.by, t.bz);
}

}  // namespace lm

using namespace lm;

#define BCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            fprintf(stderr, "lowmach: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                                      \
            return e_ == cudaErrorMemoryAllocation ? LM_ERR_OUT_OF_MEMORY : LM_ERR_CUDA;            \
        }                                                                                           \
    } while (0)

namespace {

// ---- autotuner --------------------------------------------------------------

std::mutex g_tune_mu;
std::string g_tune_path;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string default_cache_path() {
    const char* env = getenv("LM_AUTOTUNE_CACHE");
    if (env && *env) return env;
    const char* home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/lowmach_autotune.json";
}

// The cache file is a flat JSON object {"key": value, ...}.
void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    if (g_tune_path.empty()) g_tune_path = default_cache_path();
    FILE* fp = fopen(g_tune_path.c_str(), "r");
    if (!fp) return;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, fp)) > 0) txt.append(buf, n);
    fclose(fp);
    size_t i = 0;
    while ((i = txt.find('"', i)) != std::string::npos) {
        const size_t j = txt.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = txt.substr(i + 1, j - i - 1);
        const size_t c = txt.find(':', j);
        if (c == std::string::npos) break;
        g_tune[key] = atoi(txt.c_str() + c + 1);
        i = txt.find_first_of(",}", c);
        if (i == std::string::npos) break;
    }
}

void tune_save() {
    const size_t slash = g_tune_path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) {
        const std::string dir = g_tune_path.substr(0, slash);
        for (size_t k = 1; k <= dir.size(); ++k)       // create the directory level by level
            if (k == dir.size() || dir[k] == '/') ::mkdir(dir.substr(0, k).c_str(), 0755);
    }
    const std::string tmp = g_tune_path + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "w");
    if (!fp) return;
    fputs("{\n", fp);
    size_t k = 0;
    for (const auto& kv : g_tune) fprintf(fp, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_tune.size() ? "," : "");
    fputs("}\n", fp);
    fclose(fp);
    rename(tmp.c_str(), g_tune_path.c_str());
}

std::string gpu_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    std::string s = prop.name;
    for (char& c : s)
        if (c == ' ' || c == '"') c = '_';
    return s;
}

// z-chunk of the 2D sweep for one level shape: the fastest candidate, timed
// on this level's own data (into its scratch buffer), remembered per shape.
int tune_sweep_kz(const MgLevel& M, const float* fin, float* scratch, cudaStream_t s, bool* changed) {
    char key[256];
    snprintf(key, sizeof key, "%s|rbgs2d-zrow|%dx%d|bc%d%d|f32", gpu_name().c_str(), M.L.g.nx, M.L.g.nz, M.L.g.bcx,
             M.L.g.bcz);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    const int cands[] = {8, 16, 32, 64, 128, 256};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 16;
    float best_ms = 1e30f;
    for (int kz : cands) {
        if (kz > M.L.g.nz && kz != cands[0]) continue;
        launch_rbgs_kz(M.L, s, nullptr, nullptr, nullptr, 0, 0, 0, fin, scratch, 0, 1, 0, kz);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch_rbgs_kz(M.L, s, nullptr, nullptr, nullptr, 0, 0, 0, fin, scratch, 0, 1, 0, kz);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = kz;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tune[key] = best;
    *changed = true;
    return best;
}

int hdiv(int a, int b) { return (a + b - 1) / b; }

// columns of a task of the batched sweep: zrow2d_tile's width on levels of
// 128-cell segments, rbgs_tile's 256 on the others
int sweep_tile_width(const Geo& g) { return g.nx % 128 == 0 && g.nz >= 2 ? zrow2d_width(g.nx) : 256; }

// Batched z-chunk: the chunk of the sweeps at multigrid depth d of a batch,
// timed on the batched sweep itself (every grid's tiles of that depth in one
// launch: the per-grid choice above fills the GPU with one grid's blocks,
// which a batch does not need) over the candidates 8..256, and remembered
// per depth and batch composition (an FNV-1a hash of the level shapes and
// boundary conditions).  Sets the chunk of every level at that depth.
int tune_batch_kz(lm_grid* const* grids, int count, std::vector<BLev>& hl, const std::vector<int>& lev0,
                  const std::vector<int>& lstop, int max_depth, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    bool changed = false;
    BLev* dL = nullptr;
    BTask* dT = nullptr;
    size_t tcap = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LM_OK;
    for (int d = 0; d < max_depth && rc == LM_OK; ++d) {
        unsigned long long h = 1469598103934665603ULL;
        auto mix = [&](long long v) {
            for (int b = 0; b < 8; ++b) {
                h ^= (unsigned long long)((v >> (8 * b)) & 0xff);
                h *= 1099511628211ULL;
            }
        };
        int nlev = 0, maxnz = 0;
        for (int i = 0; i < count; ++i) {
            if (d >= lstop[i]) continue;
            const Geo& g = hl[lev0[i] + d].L.g;
            mix(g.nx), mix(g.nz), mix(g.bcx * 2 + g.bcz);
            ++nlev;
            maxnz = std::max(maxnz, g.nz);
        }
        if (!nlev) continue;
        char key[256];
        snprintf(key, sizeof key, "%s|rbgs2d-batch-zrow|d%d|%016llx", gpu_name().c_str(), d, h);
        int best = -1;
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            best = it->second;
        } else {
            if (!dL) {
                if (cudaMalloc(&dL, sizeof(BLev) * hl.size()) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                    cudaEventCreate(&e1) != cudaSuccess) {
                    rc = LM_ERR_CUDA;
                    break;
                }
            }
            float best_ms = 1e30f;
            for (int kz : {8, 16, 32, 64, 128, 256}) {
                if (kz > maxnz && kz != 8) continue;
                std::vector<BTask> tasks;
                for (int i = 0; i < count; ++i) {
                    if (d >= lstop[i]) continue;
                    BLev& V = hl[lev0[i] + d];
                    V.kz = kz;
                    const int gx = hdiv(V.L.g.nx, sweep_tile_width(V.L.g)), gy = hdiv(V.L.g.nz, kz);
                    for (int by = 0; by < gy; ++by)
                        for (int bx = 0; bx < gx; ++bx) tasks.push_back(BTask{i, lev0[i] + d, bx, by, 0, 0, 0});
                }
                if (tasks.size() > tcap) {
                    cudaFree(dT);
                    dT = nullptr;
                    if (cudaMalloc(&dT, sizeof(BTask) * tasks.size()) != cudaSuccess) {
                        rc = LM_ERR_CUDA;
                        break;
                    }
                    tcap = tasks.size();
                }
                cudaMemcpy(dL, hl.data(), sizeof(BLev) * hl.size(), cudaMemcpyHostToDevice);
                cudaMemcpy(dT, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice);
                const unsigned nb = (unsigned)tasks.size();
                count_launches(4);
                kb_rbgs<0, true, false, false><<<nb, 128, 0, s>>>(dT, nullptr, dL, 0, 1);
                cudaEventRecord(e0, s);
                for (int r = 0; r < 3; ++r) kb_rbgs<0, true, false, false><<<nb, 128, 0, s>>>(dT, nullptr, dL, 0, 1);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = LM_ERR_CUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = kz;
                }
            }
            if (best > 0) {
                g_tune[key] = best;
                changed = true;
            }
        }
        if (best > 0)
            for (int i = 0; i < count; ++i)
                if (d < lstop[i]) hl[lev0[i] + d].kz = best;
    }
    if (changed) tune_save();
    cudaFree(dL);
    cudaFree(dT);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess && rc == LM_OK) rc = LM_ERR_CUDA;
    return rc;
}

// ---- plan -----------------------------------------------------------------------

struct Plan {
    std::vector<lm_grid*> grids;
    std::vector<unsigned> versions;
    int inner_max = 0, first = 0, count = 0, nu1 = 1, nu2 = 1;
    BGrid* dgrids = nullptr;
    BLev* dlevs = nullptr;
    int* dlev0 = nullptr;
    BTask* dtasks = nullptr;
    SolveState* dgather = nullptr;
    SolveState* hgather = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t g_first = nullptr, g_step = nullptr;
    CoarseInv* dinv_items = nullptr;     // the grids' coarsest levels, and the rows of their inverses
    int* dinv_tasks = nullptr;
    int n_inv_tasks = 0;
    CoarseCycle* dcc = nullptr;          // per-grid one-block coarse cycles (null: per-level launches)
    size_t cc_smem = 0;                  // their dynamic shared memory (the largest chain's)
    int max_depth = 0;
    long long n_first = 0, n_step = 0;   // kernels per graph launch (n_step: outside the inner loop)
    long long n_iter = 0;                // kernels per inner iteration of the device-side loop
    int* dinner = nullptr;               // inner iterations run in the last refinement step (device)
    int* hinner = nullptr;

    ~Plan() {
        if (g_first) cudaGraphExecDestroy(g_first);
        if (g_step) cudaGraphExecDestroy(g_step);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(dgrids);
        cudaFree(dlevs);
        cudaFree(dlev0);
        cudaFree(dtasks);
        cudaFree(dcc);
        cudaFree(dinv_items);
        cudaFree(dinv_tasks);
        cudaFree(dgather);
        cudaFreeHost(hgather);
        cudaFree(dinner);
        cudaFreeHost(hinner);
    }
};

std::mutex g_plan_mu;
std::vector<Plan*> g_plans;

struct TaskList {
    int off = 0, n = 0;
};

int build_plan(lm_grid* const* grids, int count, const lm_solve_opts* o, cudaStream_t s, Plan** out) {
    Plan* P = new Plan();
    P->grids.assign(grids, grids + count);
    for (int i = 0; i < count; ++i) P->versions.push_back(grids[i]->version);
    P->inner_max = o->inner_max_iter;
    P->nu1 = o->nu1;
    P->nu2 = o->nu2;
    P->first = !o->use_x0;
    P->count = count;
    {   // every grid's coarsest inverse, one block per row of it
        std::vector<CoarseInv> items(count);
        std::vector<int> task;
        for (int i = 0; i < count; ++i) {
            const MgLevel& Lc = grids[i]->mg.back();
            items[i] = CoarseInv{Lc.L, Lc.ainv};
            for (int b = 0; b < Lc.L.g.N; ++b) task.push_back(i << 8 | b);
        }
        BCK(cudaMalloc(&P->dinv_items, sizeof(CoarseInv) * count));
        BCK(cudaMalloc(&P->dinv_tasks, sizeof(int) * task.size()));
        BCK(cudaMemcpy(P->dinv_items, items.data(), sizeof(CoarseInv) * count, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(P->dinv_tasks, task.data(), sizeof(int) * task.size(), cudaMemcpyHostToDevice));
        P->n_inv_tasks = (int)task.size();
    }

    // autotune the sweep chunks of every level shape in the batch
    bool changed = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        for (int i = 0; i < count; ++i)
            for (size_t l = 0; l < grids[i]->mg.size(); ++l) {
                const MgLevel& M = grids[i]->mg[l];
                (void)tune_sweep_kz(M, l == 0 ? grids[i]->r32 : M.f, M.xa, s, &changed);
            }
        if (changed) tune_save();
    }

    std::vector<BGrid> hg(count);
    std::vector<BLev> hl;
    std::vector<int> lev0(count), nlev(count);
    for (int i = 0; i < count; ++i) {
        lm_grid* g = grids[i];
        BGrid& G = hg[i];
        G.geo = g->geo;
        G.op = Op64{g->ct, g->gx, g->gy, g->gz, g->dinv};
        G.f = g->f;
        G.x = g->x;
        G.r32 = g->r32;
        G.e32 = g->e32;
        G.z32 = g->z32;
        G.p32 = g->p32;
        G.q32 = g->q32;
        G.st = g->st;
        G.st_in = g->st_in;
        G.red = Red{g->part, g->scal, g->ctr};
        G.N = g->N;
        // rows per thread of the batched apply: at least 8 (2048 cells per
        // block, so the per-block dot reduction stays small against the
        // stencil work), more when the grid would exceed 4096 blocks
        int kz = 8;
        while ((long long)hdiv(g->n[0], 32) * hdiv(hdiv(g->n[2], kz), 8) > 4096) kz *= 2;
        G.kz_apply = kz;
        // 2D grids of 128-column segments: a warp per segment and 8 rows
        G.seg_apply = seg2d_ok(g->mg[0].L.g, g->p32, g->q32, g->r32, g->mg[0].L.rho, g->mg[0].L.ct) ? 1 : 0;
        if (G.seg_apply) G.kz_apply = 8;
        lev0[i] = (int)hl.size();
        nlev[i] = (int)g->mg.size();
        P->max_depth = std::max(P->max_depth, nlev[i]);
        for (size_t l = 0; l < g->mg.size(); ++l) {
            const MgLevel& M = g->mg[l];
            BLev V{};
            V.L = M.L;
            const bool last = l + 1 == g->mg.size();
            if (!last) {
                V.C = g->mg[l + 1].L.g;
                V.hx = M.halved[0];
                V.hy = M.halved[1];
                V.hz = M.halved[2];
                V.fc = g->mg[l + 1].f;
                V.ec = g->mg[l + 1].xo;
            } else {
                V.C = M.L.g;
            }
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                V.kz = tune_sweep_kz(M, l == 0 ? g->r32 : M.f, M.xa, s, &changed);
            }
            V.xa = M.xa;
            V.xb = M.xb;
            V.xo = l == 0 ? g->z32 : M.xo;
            V.f = l == 0 ? g->r32 : M.f;
            V.ainv = M.ainv;
            V.kr = !last && rr2d_ok(V.L, V.hx, V.hy, V.hz, V.xa, V.f, V.fc) ? std::max(1, std::min(8, V.C.nz / 16))
                                                                             : 0;
            hl.push_back(V);
        }
    }

    // task tables
    std::vector<BTask> tasks;
    auto one_d = [&]() {
        TaskList L{(int)tasks.size(), 0};
        for (int i = 0; i < count; ++i) {
            const int nb = std::max(1, std::min(1024, hdiv(hg[i].N, NT * 8)));
            for (int b = 0; b < nb; ++b) tasks.push_back(BTask{i, 0, 0, 0, 0, b, nb});
        }
        L.n = (int)tasks.size() - L.off;
        return L;
    };
    const TaskList t1d = one_d();
    TaskList tap{(int)tasks.size(), 0};
    for (int i = 0; i < count; ++i) {
        const Geo& g = hg[i].geo;
        const int gx = hg[i].seg_apply ? g.nx / 128 : hdiv(g.nx, 32);
        const int gy = hg[i].seg_apply ? hdiv(g.nz, 8 * hg[i].kz_apply) : hdiv(hdiv(g.nz, hg[i].kz_apply), 8);
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) tasks.push_back(BTask{i, lev0[i], bx, by, 0, bx + gx * by, gx * gy});
    }
    tap.n = (int)tasks.size() - tap.off;
    // one-block coarse cycles when every grid's hierarchy has one: the
    // per-level task lists then stop at each grid's coarse-cycle level
    bool fused = true;
    std::vector<int> lstop(count);
    for (int i = 0; i < count; ++i) {
        fused = fused && grids[i]->cc_level >= 0;
        lstop[i] = nlev[i] - 1;
    }
    if (fused) {
        std::vector<CoarseCycle> hcc(count);
        for (int i = 0; i < count; ++i) {
            lm_grid* g = grids[i];
            const int lc = g->cc_level;
            lstop[i] = lc;
            CoarseCycle& cc = hcc[i];
            cc = CoarseCycle{};
            cc.nl = (int)g->mg.size() - lc;
            for (int k = 0; k < cc.nl; ++k) {
                const MgLevel& Mk = g->mg[lc + k];
                cc.L[k] = Mk.L;
                cc.hx[k] = Mk.halved[0];
                cc.hy[k] = Mk.halved[1];
                cc.hz[k] = Mk.halved[2];
                cc.x[k] = (lc + k == 0) ? g->z32 : Mk.xo;
                cc.f[k] = (lc + k == 0) ? g->r32 : Mk.f;
            }
            cc.ainv = g->mg.back().ainv;
            cc.nu1 = o->nu1;
            cc.nu2 = o->nu2;
        }
        for (const CoarseCycle& cc : hcc) P->cc_smem = std::max(P->cc_smem, cc_smem_bytes(cc));
        BCK(cudaFuncSetAttribute(kb_coarse_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CC_SMEM_MAX));
        BCK(cudaMalloc(&P->dcc, sizeof(CoarseCycle) * count));
        BCK(cudaMemcpy(P->dcc, hcc.data(), sizeof(CoarseCycle) * count, cudaMemcpyHostToDevice));
    }
    if (int rc = tune_batch_kz(grids, count, hl, lev0, lstop, P->max_depth, s)) return rc;
    std::vector<TaskList> tpre(P->max_depth), trr(P->max_depth);
    for (int d = 0; d < P->max_depth; ++d) {
        tpre[d].off = (int)tasks.size();
        for (int i = 0; i < count; ++i) {
            if (d >= lstop[i]) continue;
            const BLev& V = hl[lev0[i] + d];
            const int gx = hdiv(V.L.g.nx, sweep_tile_width(V.L.g)), gy = hdiv(V.L.g.nz, V.kz);
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) tasks.push_back(BTask{i, lev0[i] + d, bx, by, 0, 0, 0});
        }
        tpre[d].n = (int)tasks.size() - tpre[d].off;
        trr[d].off = (int)tasks.size();
        for (int i = 0; i < count; ++i) {
            if (d >= lstop[i]) continue;
            const BLev& V = hl[lev0[i] + d];
            const int gx = V.kr ? V.L.g.nx / 128 : hdiv(V.C.nx, 32), gy = V.kr ? hdiv(V.C.nz, 8 * V.kr) : hdiv(V.C.nz, 8);
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) tasks.push_back(BTask{i, lev0[i] + d, bx, by, 0, 0, 0});
        }
        trr[d].n = (int)tasks.size() - trr[d].off;
    }
    TaskList tco{(int)tasks.size(), 0};
    for (int i = 0; i < count; ++i) tasks.push_back(BTask{i, lev0[i] + nlev[i] - 1, 0, 0, 0, 0, 1});
    tco.n = count;

    BCK(cudaMalloc(&P->dgrids, sizeof(BGrid) * count));
    BCK(cudaMalloc(&P->dlevs, sizeof(BLev) * hl.size()));
    BCK(cudaMalloc(&P->dlev0, sizeof(int) * count));
    BCK(cudaMalloc(&P->dtasks, sizeof(BTask) * tasks.size()));
    BCK(cudaMalloc(&P->dgather, sizeof(SolveState) * 2 * count));
    BCK(cudaMallocHost(&P->hgather, sizeof(SolveState) * 2 * count));
    BCK(cudaMemcpy(P->dgrids, hg.data(), sizeof(BGrid) * count, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(P->dlevs, hl.data(), sizeof(BLev) * hl.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(P->dlev0, lev0.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(P->dtasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice));
    BCK(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
    BCK(cudaMalloc(&P->dinner, sizeof(int)));
    BCK(cudaMallocHost(&P->hinner, sizeof(int)));
    BCK(cudaMemset(P->dinner, 0, sizeof(int)));
    cudaStream_t body_stream = nullptr;
    BCK(cudaStreamCreateWithFlags(&body_stream, cudaStreamNonBlocking));

    const BTask* T = P->dtasks;
    const BGrid* Gs = P->dgrids;
    const BLev* Ls = P->dlevs;
    long long nk = 0;
    // one inner flexible-CG iteration over all grids (converged grids idle),
    // ending with the loop's condition
    auto launch_iteration = [&](cudaStream_t cs, cudaGraphConditionalHandle loop) {
        // pre-smoothing: nu1 red-black sweeps, the last one into xa (the
        // residual's and the first post-sweep's input); post-smoothing: nu2
        // black-red sweeps from xa + P ec, through xb / xa, the last into xo
        const int nu1 = P->nu1, nu2 = P->nu2;
        for (int d = 0; d < P->max_depth; ++d) {
            if (tpre[d].n) {
                for (int k = 0; k < nu1; ++k) {
                    const int dst = ((nu1 - 1 - k) % 2 == 0) ? 1 : 2, src = dst == 1 ? 2 : 1;
                    if (k == 0) kb_rbgs<0, true, false><<<tpre[d].n, 128, 0, cs>>>(T + tpre[d].off, Gs, Ls, 0, dst);
                    else kb_rbgs<0, false, false><<<tpre[d].n, 128, 0, cs>>>(T + tpre[d].off, Gs, Ls, src, dst);
                }
                nk += nu1;
            }
            if (trr[d].n) {
                kb_resid_restrict<<<trr[d].n, dim3(32, 8), 0, cs>>>(T + trr[d].off, Gs, Ls);
                ++nk;
            }
        }
        if (P->dcc) kb_coarse_cycle<<<count, CC_THREADS, P->cc_smem, cs>>>(P->dcc, Gs);
        else kb_coarse<<<tco.n, 64, 0, cs>>>(T + tco.off, Gs, Ls);
        for (int d = P->max_depth - 1; d >= 0; --d)
            if (tpre[d].n) {
                int src = 1;
                for (int k = 0; k < nu2; ++k) {
                    const int dst = k == nu2 - 1 ? 3 : (k % 2 == 0 ? 2 : 1);
                    if (k == 0) kb_rbgs<1, false, true><<<tpre[d].n, 128, 0, cs>>>(T + tpre[d].off, Gs, Ls, src, dst);
                    else kb_rbgs<1, false, false><<<tpre[d].n, 128, 0, cs>>>(T + tpre[d].off, Gs, Ls, src, dst);
                    src = dst;
                }
                nk += nu2;
            }
        kb_dot_zq<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs, P->dinner);
        kb_beta_p<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs, P->dinner);
        kb_apply<<<tap.n, dim3(32, 8), 0, cs>>>(T + tap.off, Gs, Ls, P->dlev0);
        kb_update<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs);
        kb_inner_cond<<<1, 256, 0, cs>>>(Gs, count, P->dinner, P->inner_max, loop);
        nk += 6;
    };
    // One refinement step: the inner flexible CG as a device-side while loop
    // (a conditional node of the graph: it repeats its body while some grid
    // still iterates, so the step launches only the iterations the slowest
    // grid needs), then the correction and the new float64 residual.
    auto launch_step = [&](cudaStream_t cs) -> cudaError_t {
        kb_inner_init<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs, P->dinner);
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) return e;
        cudaGraphConditionalHandle loop;
        if ((e = cudaGraphConditionalHandleCreate(&loop, cg, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        if ((e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp)) != cudaSuccess) return e;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return e;
        nk = 0;
        launch_iteration(body_stream, loop);
        P->n_iter = nk;
        if ((e = cudaStreamEndCapture(body_stream, &body)) != cudaSuccess) return e;
        if ((e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess)
            return e;
        kb_ir_correct<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs);
        kb_ir_residual<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs, 0, 0);
        kb_gather<<<hdiv(count, 64), 64, 0, cs>>>(Gs, count, P->dgather);
        nk = 4;    // inner init, correction, residual, gather
        return cudaSuccess;
    };
    auto launch_first = [&](cudaStream_t cs) {
        nk += 2;
        kb_ir_residual<<<t1d.n, NT, 0, cs>>>(T + t1d.off, Gs, P->first, 1);
        kb_gather<<<hdiv(count, 64), 64, 0, cs>>>(Gs, count, P->dgather);
    };
    for (int pass = 0; pass < 2; ++pass) {
        cudaGraph_t graph = nullptr;
        BCK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
        nk = 0;
        cudaError_t e = cudaSuccess;
        if (pass == 0) launch_first(P->cap);
        else e = launch_step(P->cap);
        (pass == 0 ? P->n_first : P->n_step) = nk;
        const cudaError_t e2 = cudaStreamEndCapture(P->cap, &graph);
        BCK(e);
        BCK(e2);
        BCK(cudaGraphInstantiate(pass == 0 ? &P->g_first : &P->g_step, graph, 0));
        cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(body_stream);
    *out = P;
    return LM_OK;
}

bool plan_matches(const Plan* P, lm_grid* const* grids, int count, const lm_solve_opts* o) {
    if (P->count != count || P->inner_max != o->inner_max_iter || P->first != !o->use_x0 || P->nu1 != o->nu1 ||
        P->nu2 != o->nu2)
        return false;
    for (int i = 0; i < count; ++i)
        if (P->grids[i] != grids[i] || P->versions[i] != grids[i]->version) return false;
    return true;
}

void drop_plans_of(const lm_grid* g) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (size_t i = 0; i < g_plans.size();) {
        if (std::find(g_plans[i]->grids.begin(), g_plans[i]->grids.end(), g) != g_plans[i]->grids.end()) {
            delete g_plans[i];
            g_plans.erase(g_plans.begin() + i);
        } else {
            ++i;
        }
    }
}

// Device tables of the batched set-up, grown as needed and reused by later
// calls (one set per process; calls are serialised by its mutex).
struct SetupTables {
    std::mutex mu;
    BTask* dtask = nullptr;
    size_t ntask_cap = 0;
    void* ditems = nullptr;
    size_t items_cap = 0;
    AsmFlags* dflags = nullptr;
    AsmFlags* hflags = nullptr;
    int flags_cap = 0;
    void* hitems = nullptr;
    size_t hitems_cap = 0;
};
SetupTables g_setup;

int ensure_tables(size_t ntask, size_t item_bytes, int nflags) {
    SetupTables& S = g_setup;
    if (ntask > S.ntask_cap) {
        cudaFree(S.dtask);
        S.dtask = nullptr;
        S.ntask_cap = 0;
        BCK(cudaMalloc(&S.dtask, sizeof(BTask) * ntask));
        S.ntask_cap = ntask;
    }
    if (item_bytes > S.items_cap) {
        cudaFree(S.ditems);
        cudaFreeHost(S.hitems);
        S.ditems = S.hitems = nullptr;
        S.items_cap = 0;
        BCK(cudaMalloc(&S.ditems, item_bytes));
        BCK(cudaMallocHost(&S.hitems, item_bytes));
        S.items_cap = item_bytes;
    }
    if (nflags > S.flags_cap) {
        cudaFree(S.dflags);
        cudaFreeHost(S.hflags);
        S.dflags = nullptr;
        S.hflags = nullptr;
        S.flags_cap = 0;
        BCK(cudaMalloc(&S.dflags, sizeof(AsmFlags) * nflags));
        BCK(cudaMallocHost(&S.hflags, sizeof(AsmFlags) * nflags));
        S.flags_cap = nflags;
    }
    return LM_OK;
}

// Coarse coefficients of every grid whose hierarchy exists but is stale,
// level by level, one launch per level over all of them.
int batch_refresh(lm_grid* const* grids, int count, cudaStream_t s) {
    std::vector<lm_grid*> todo;
    size_t depth = 0;
    for (int i = 0; i < count; ++i)
        if (!grids[i]->mg_built && grids[i]->mg.size() > 1 && grids[i]->fp32_ok) {
            todo.push_back(grids[i]);
            depth = std::max(depth, grids[i]->mg.size() - 1);
        }
    if (todo.empty()) return LM_OK;
    std::lock_guard<std::mutex> lk(g_setup.mu);
    for (size_t d = 0; d < depth; ++d) {
        std::vector<BCoarsen> items;
        std::vector<BTask> tasks;
        for (lm_grid* g : todo) {
            if (d + 1 >= g->mg.size()) continue;
            const MgLevel& F = g->mg[d];
            const MgLevel& C = g->mg[d + 1];
            const int it = (int)items.size();
            items.push_back(BCoarsen{F.L, C.L.g, F.halved[0], F.halved[1], F.halved[2], C.ct, C.rho});
            const Geo& cg = C.L.g;
            const int gx = hdiv(cg.nx, 32);
            const int gy = cg.ny > 1 ? hdiv(cg.ny, 8) : hdiv(cg.nz, 8);
            const int gz = cg.ny > 1 ? cg.nz : 1;
            for (int bz = 0; bz < gz; ++bz)
                for (int by = 0; by < gy; ++by)
                    for (int bx = 0; bx < gx; ++bx) tasks.push_back(BTask{it, 0, bx, by, bz, 0, 0});
        }
        if (tasks.empty()) continue;
        if (int rc = ensure_tables(tasks.size(), sizeof(BCoarsen) * items.size(), 0)) return rc;
        // the previous level's launch may still read the tables: wait before rewriting them
        BCK(cudaStreamSynchronize(s));
        std::memcpy(g_setup.hitems, items.data(), sizeof(BCoarsen) * items.size());
        BCK(cudaMemcpyAsync(g_setup.ditems, g_setup.hitems, sizeof(BCoarsen) * items.size(), cudaMemcpyHostToDevice,
                            s));
        BCK(cudaMemcpyAsync(g_setup.dtask, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice, s));
        count_launches(1);
        kb_coarsen<<<(unsigned)tasks.size(), dim3(32, 8), 0, s>>>(g_setup.dtask, (const BCoarsen*)g_setup.ditems);
        BCK(cudaGetLastError());
    }
    BCK(cudaStreamSynchronize(s));
    for (lm_grid* g : todo) {
        g->mg_built = true;
        if (g->mg.back().ainv) g->inv_pending = true;
    }
    return LM_OK;
}

}  // namespace

void lm::batch_forget_grid(const lm_grid* g) { drop_plans_of(g); }

extern "C" {

int lm_autotune_set_cache(const char* path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_tune_loaded = false;
    g_tune_path = path && *path ? path : default_cache_path();
    return LM_OK;
}

int lm_batch_set_coefficients(lm_grid* const* grids, int count, const double* const* rho_old,
                              const double* const* rho_new, const double* const* cs2, const double* dt,
                              void* stream) {
    if (!grids || count < 1 || !rho_old || !rho_new || !cs2 || !dt) return LM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (!grids[i] || !rho_old[i] || !rho_new[i] || !cs2[i]) return LM_ERR_INVALID_ARG;
        if (!(dt[i] > 0.0 && std::isfinite(dt[i]))) return LM_ERR_NOT_POSITIVE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_setup.mu);
    std::vector<BTask> tasks;
    for (int i = 0; i < count; ++i) {
        const int nb = std::max(1, std::min(1024, hdiv(grids[i]->N, NT * 8)));
        for (int b = 0; b < nb; ++b) tasks.push_back(BTask{i, 0, 0, 0, 0, b, nb});
    }
    if (int rc = ensure_tables(tasks.size(), sizeof(AsmArgs) * count, count)) return rc;
    BCK(cudaStreamSynchronize(s));                 // an earlier call's launches may still read the tables
    AsmArgs* h = (AsmArgs*)g_setup.hitems;
    for (int i = 0; i < count; ++i) {
        lm_grid* g = grids[i];
        h[i] = asm_args(g->geo, rho_old[i], rho_new[i], cs2[i], dt[i], 0, g->h,
                        Op64Out{g->ct, g->gx, g->gy, g->gz, g->dinv, g->ct32, g->rho32}, g->asm_fl);
    }
    const AsmArgs* dA = (const AsmArgs*)g_setup.ditems;
    BCK(cudaMemcpyAsync(g_setup.ditems, h, sizeof(AsmArgs) * count, cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(g_setup.dtask, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice, s));
    count_launches(3);
    kb_asm_flags<<<hdiv(count, 64), 64, 0, s>>>(dA, count, nullptr, 0);
    kb_assemble<<<(unsigned)tasks.size(), NT, 0, s>>>(g_setup.dtask, dA);
    kb_asm_flags<<<hdiv(count, 64), 64, 0, s>>>(dA, count, g_setup.dflags, 1);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(g_setup.hflags, g_setup.dflags, sizeof(AsmFlags) * count, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    int worst = LM_OK;
    for (int i = 0; i < count; ++i) {
        const int rc = grid_finish_assembly(grids[i], g_setup.hflags[i], s);
        if (rc && !worst) worst = rc;
    }
    return worst;
}

int lm_batch_solve(lm_grid* const* grids, int count, const lm_solve_opts* o, lm_solve_result* results) {
    if (!grids || count < 1 || !o || !results) return LM_ERR_INVALID_ARG;
    if (!(o->rtol > 0.0) || o->inner_max_iter < 1 || o->max_outer < 1 || o->nu1 < 1 || o->nu2 < 1 || o->nu1 > 8 ||
        o->nu2 > 8)
        return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    for (int i = 0; i < count; ++i) {
        lm_grid* g = grids[i];
        if (!g) return LM_ERR_INVALID_ARG;
        std::memset(&results[i], 0, sizeof(lm_solve_result));
        if (!g->have_coefs || !g->have_rhs) return LM_ERR_STATE;
        if (g->ndim != 2 || g->n[1] != 1) return LM_ERR_INVALID_ARG;       // the batch path is 2D
        if (!g->fp32_ok) return LM_ERR_INVALID_ARG;                         // no float32 operator
        for (int a = 0; a < 3; ++a)
            if (g->bc[a] == LM_BC_PERIODIC && g->n[a] > 1 && (g->n[a] % 2)) return LM_ERR_INVALID_ARG;
        if (o->use_x0 && !g->have_x0) return LM_ERR_STATE;
        for (int j = 0; j < i; ++j)
            if (grids[j] == g) return LM_ERR_INVALID_ARG;
    }
    // grids whose coefficients changed since their hierarchy was built: the
    // coarse coefficients of all of them, one launch per level
    if (int rc = batch_refresh(grids, count, s)) return rc;
    for (int i = 0; i < count; ++i) {
        const int rc = grid_build_mg(grids[i], s, true);
        if (rc) return rc;
        if (!grids[i]->mg.back().ainv) return LM_ERR_INVALID_ARG;   // the batch path needs a direct coarsest level
    }
    BCK(cudaStreamSynchronize(s));
    Plan* P = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (Plan* q : g_plans)
            if (plan_matches(q, grids, count, o)) P = q;
    }
    if (!P) {
        for (int i = 0; i < count; ++i) drop_plans_of(grids[i]);
        const int rc = build_plan(grids, count, o, s, &P);
        if (rc) return rc;
        std::lock_guard<std::mutex> lk(g_plan_mu);
        g_plans.push_back(P);
    }
    {   // every grid's coarsest inverse left pending by its refresh, in one launch
        bool pending = false;
        for (int i = 0; i < count; ++i) pending = pending || grids[i]->inv_pending;
        if (pending) {
            launch_coarse_inverse_grids(P->dinv_items, count, s);
            BCK(cudaGetLastError());
            for (int i = 0; i < count; ++i) grids[i]->inv_pending = false;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    BCK(cudaEventRecord(e0, s));
    for (int i = 0; i < count; ++i)
        if (o->use_x0)
            BCK(cudaMemcpyAsync(grids[i]->x, grids[i]->x0, sizeof(double) * grids[i]->N, cudaMemcpyDeviceToDevice, s));
    count_launches(1);
    kb_init_states<<<hdiv(count, NT), NT, 0, s>>>(P->dgrids, count, o->rtol, o->inner_rtol);
    BCK(cudaGraphLaunch(P->g_first, s));
    count_launches(P->n_first);
    int outer = 0;
    for (;;) {
        BCK(cudaMemcpyAsync(P->hgather, P->dgather, sizeof(SolveState) * 2 * count, cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        if (outer > 0) count_launches(P->n_step + P->n_iter * (long long)*P->hinner);
        bool all = true;
        for (int i = 0; i < count; ++i) all = all && P->hgather[i].done;
        if (all || outer >= o->max_outer) break;
        BCK(cudaGraphLaunch(P->g_step, s));
        BCK(cudaMemcpyAsync(P->hinner, P->dinner, sizeof(int), cudaMemcpyDeviceToHost, s));
        ++outer;
    }
    BCK(cudaEventRecord(e1, s));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = LM_OK;
    for (int i = 0; i < count; ++i) {
        const SolveState& so = P->hgather[i];
        const SolveState& si = P->hgather[count + i];
        lm_solve_result& r = results[i];
        r.iters = si.iters;
        r.outer_iters = so.iters;
        r.vcycles = si.iters;
        r.rel_residual = so.rel;
        r.seconds = ms * 1e-3;
        r.status = so.status ? so.status : (so.converged ? LM_OK : LM_ERR_NO_CONVERGENCE);
        grids[i]->history.assign(1, so.rel);
        if (r.status && !worst) worst = r.status;
    }
    return worst;
}

}  // extern "C"
