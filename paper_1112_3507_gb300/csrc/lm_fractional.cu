// The explicit parts of one fractional step around the pressure solve
// (Sec. 2.4), in float64:
//
//   lm_advect      steps (i)-(iii): face velocities of Eq. step1 from the
//                  cell momenta, the modified flux F~ = (rho, rho c, rho u,
//                  e) u_{i+1/2} evaluated with the upwind side's MUSCL state
//                  (minmod-limited slope; the paper's CPM/MENO reconstruction
//                  is not reproduced in its text), and the explicit update
//                  q^{new} = q^n - dt d(F~)/dx summed over the axes;
//   lm_eos_ideal   step (ix): P = (gamma - 1)(e - |rho u|^2 / (2 rho)) and
//                  c_s^2 = gamma P / rho for the next step's c~.
//
// A wall face carries no flux and a cell next to a wall has zero slope (its
// outer neighbour does not exist); periodic axes wrap.  One thread per
// cell computes both faces of each axis it needs (the face fluxes are
// recomputed by the two cells that share them), so the kernel needs no
// synchronisation; the float64 pipe bounds it on GB300.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace {

constexpr int MAXQ = 6;       // rho, rho u (3), e, rho c

struct AdvGeo {
    int n[3];
    int N;
    int wall[3];
    double rh[3];             // 1 / h
    int stride[3];
    int nq;                   // 5, or 6 with rho c
};

struct AdvIO {
    const double* q[MAXQ];    // rho, m_x, m_y, m_z, e, rho c
    double* out[MAXQ];
};

__device__ __forceinline__ double minmod(double a, double b) {
    return a * b > 0.0 ? (fabs(a) < fabs(b) ? a : b) : 0.0;
}

// index of the cell at offset t (|t| <= 2) along an axis from position c:
// wrapped on a periodic axis, clamped on a wall axis (clamped values are
// never used: wall cells have zero slope and the wall face no flux)
__device__ __forceinline__ int along(int idx, int c, int t, int n, int stride, int wall) {
    int d = c + t;
    if (wall) {
        d = d < 0 ? 0 : (d >= n ? n - 1 : d);
    } else {
        d = d < 0 ? d + n : (d >= n ? d - n : d);
    }
    return idx + (d - c) * stride;
}

__global__ void __launch_bounds__(lm::NT) k_advect(AdvGeo G, AdvIO io, double dt) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
        int c[3];
        c[0] = idx % G.n[0];
        const int t = idx / G.n[0];
        c[1] = t % G.n[1];
        c[2] = t / G.n[1];
        double acc[MAXQ];
        for (int q = 0; q < G.nq; ++q) acc[q] = io.q[q][idx];
        for (int a = 0; a < 3; ++a) {
            const int n = G.n[a];
            if (n == 1) continue;
            const int s = G.stride[a], w = G.wall[a];
            int id[5];
#pragma unroll
            for (int o = 0; o < 5; ++o) id[o] = along(idx, c[a], o - 2, n, s, w);
            // slope use: a wall axis' end cells have zero slope
            bool flat[5];
#pragma unroll
            for (int o = 0; o < 5; ++o) {
                const int d = c[a] + o - 2;
                flat[o] = w && (d <= 0 || d >= n - 1);
            }
            const bool wall_m = w && c[a] == 0, wall_p = w && c[a] == n - 1;
            // face velocities (Eq. step1): minus face between cells 1 and 2 of
            // the five, plus face between 2 and 3
            const double* rho = io.q[0];
            const double* m = io.q[1 + a];
            const double um = wall_m ? 0.0 : (m[id[1]] + m[id[2]]) / (rho[id[1]] + rho[id[2]]);
            const double up = wall_p ? 0.0 : (m[id[2]] + m[id[3]]) / (rho[id[2]] + rho[id[3]]);
            for (int q = 0; q < G.nq; ++q) {
                const double* v = io.q[q];
                double x[5];
#pragma unroll
                for (int o = 0; o < 5; ++o) x[o] = v[id[o]];
                double sl[4];        // slopes of cells 1..4 of the five
#pragma unroll
                for (int o = 1; o < 4; ++o) sl[o] = flat[o] ? 0.0 : minmod(x[o] - x[o - 1], x[o + 1] - x[o]);
                // minus face: left state from cell 1, right state from cell 2
                const double fm = um > 0.0 ? (x[1] + 0.5 * sl[1]) * um : (x[2] - 0.5 * sl[2]) * um;
                const double fp = up > 0.0 ? (x[2] + 0.5 * sl[2]) * up : (x[3] - 0.5 * sl[3]) * up;
                acc[q] -= dt * (fp - fm) * G.rh[a];
            }
        }
        for (int q = 0; q < G.nq; ++q) io.out[q][idx] = acc[q];
    }
}

__global__ void __launch_bounds__(lm::NT) k_eos_ideal(int N, double gamma, const double* __restrict__ rho,
                                                      const double* __restrict__ mom,
                                                      const double* __restrict__ e, double* __restrict__ p,
                                                      double* __restrict__ cs2) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        const double r = rho[idx];
        const double mx = mom[idx], my = mom[(size_t)N + idx], mz = mom[2 * (size_t)N + idx];
        const double kin = 0.5 * (mx * mx + my * my + mz * mz) / r;
        const double pi = (gamma - 1.0) * (e[idx] - kin);
        p[idx] = pi;
        if (cs2) cs2[idx] = gamma * pi / r;
    }
}

int blocks_for(long long N) {
    long long b = (N + lm::NT - 1) / lm::NT;
    return (int)(b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b));
}

int finish(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lowmach: %s: %s\n", what, cudaGetErrorString(e));
        return LM_ERR_CUDA;
    }
    return LM_OK;
}

}  // namespace

extern "C" {

int lm_advect(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt, const double* rho,
              const double* mom, const double* e, const double* rho_c, double* rho_new, double* mom_star,
              double* e_star, double* rho_c_new, void* stream) {
    if (!n || !h || !bc || (ndim != 2 && ndim != 3) || !rho || !mom || !e || !rho_new || !mom_star || !e_star ||
        (!rho_c) != (!rho_c_new) || !(dt >= 0.0 && dt < 1e300))
        return LM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || !(h[a] > 0.0) || (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN)) return LM_ERR_INVALID_ARG;
    if ((ndim == 2 && n[1] != 1) || (long long)n[0] * n[1] * n[2] >= (1LL << 31)) return LM_ERR_INVALID_ARG;
    AdvGeo G{};
    G.N = 1;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = (int)n[a];
        G.wall[a] = bc[a] == LM_BC_NEUMANN;
        G.rh[a] = 1.0 / h[a];
    }
    G.N = G.n[0] * G.n[1] * G.n[2];
    G.stride[0] = 1;
    G.stride[1] = G.n[0];
    G.stride[2] = G.n[0] * G.n[1];
    G.nq = rho_c ? 6 : 5;
    const size_t N = (size_t)G.N;
    // the outputs must not overlap the inputs (every thread reads neighbours)
    const double* ins[MAXQ] = {rho, mom, mom + N, mom + 2 * N, e, rho_c};
    double* outs[MAXQ] = {rho_new, mom_star, mom_star + N, mom_star + 2 * N, e_star, rho_c_new};
    for (int q = 0; q < G.nq; ++q)
        for (int r = 0; r < G.nq; ++r)
            if (outs[q] < ins[r] + N && ins[r] < outs[q] + N) return LM_ERR_INVALID_ARG;
    AdvIO io{};
    for (int q = 0; q < G.nq; ++q) {
        io.q[q] = ins[q];
        io.out[q] = outs[q];
    }
    lm::count_launches(1);
    k_advect<<<blocks_for(G.N), lm::NT, 0, (cudaStream_t)stream>>>(G, io, dt);
    return finish("lm_advect");
}

int lm_eos_ideal(int64_t n_cells, double gamma, const double* rho, const double* mom, const double* e, double* p,
                 double* cs2, void* stream) {
    if (n_cells < 1 || n_cells >= (1LL << 31) || !(gamma > 1.0) || !rho || !mom || !e || !p) return LM_ERR_INVALID_ARG;
    lm::count_launches(1);
    k_eos_ideal<<<blocks_for(n_cells), lm::NT, 0, (cudaStream_t)stream>>>((int)n_cells, gamma, rho, mom, e, p, cs2);
    return finish("lm_eos_ideal");
}

}  // extern "C"
