// The steps either side of the pressure solve in one fractional step of the
// paper's method (Sec. 2, steps (iv)-(viii)), in float64:
//
//   lm_projection_rhs     the right-hand side f of Eq. fpoiss from the old
//                         pressure, density, sound speed and momentum and the
//                         advected momentum (rho u)*, with the face velocities
//                         u* it needs (MAC values ((rho u)_L + (rho u)_R) /
//                         (rho_L + rho_R) of rho^{n+1});
//   lm_projection_update  with the predicted pressure: the momentum update
//                         (Eq. momupdate), the separate face-velocity update
//                         of step (vii) and the energy update of step (viii).
//
// Pressures at faces follow the dual-cell interpolation of Eq. pbnd and cell
// gradients its central difference (Eq. nablaP); a wall face carries no
// velocity and the wall cell's pressure (zero normal gradient), a periodic
// axis wraps.  The face update uses the same 2 / (rho_L + rho_R) factor as
// the operator's face conductances, so the divergence of the new face
// velocities is the discrete pressure evolution, exactly up to the solve's
// residual.  Vector fields are three arrays of N values (x, y, z components,
// consecutive); face arrays hold each cell's minus face per axis.  One
// thread per cell; the float64 pipe bounds these kernels on GB300.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/lowmach.h"
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace {

struct AxisNb {
    int m, p;          // minus and plus neighbour (wrapped)
    bool wm, wp;       // the minus / plus face is a wall
    bool live;         // the axis has more than one cell
};

__device__ __forceinline__ AxisNb axis_nb(int idx, int c, int n, int stride, int bc) {
    AxisNb a;
    a.live = n > 1;
    a.m = c > 0 ? idx - stride : idx + (n - 1) * stride;
    a.p = c < n - 1 ? idx + stride : idx - (n - 1) * stride;
    a.wm = bc != LM_BC_PERIODIC && c == 0;
    a.wp = bc != LM_BC_PERIODIC && c == n - 1;
    return a;
}

// Eq. pbnd between cells a and b
__device__ __forceinline__ double pbnd(double Pa, double ra, double Pb, double rb) {
    return (Pb * ra + Pa * rb) / (ra + rb);
}

// the cell gradient of Eq. nablaP along one axis
__device__ __forceinline__ double grad_axis(const AxisNb& a, int idx, const double* __restrict__ P,
                                            const double* __restrict__ rho, double ih) {
    const double Pc = P[idx], rc = rho[idx];
    const double pm = a.wm ? Pc : pbnd(P[a.m], rho[a.m], Pc, rc);
    const double pp = a.wp ? Pc : pbnd(Pc, rc, P[a.p], rho[a.p]);
    return (pp - pm) * ih;
}

__device__ __forceinline__ void cell_axes(int idx, const lm::Geo& g, const int bc[3], AxisNb ax[3]) {
    int i, j, k;
    lm::cell_coords(idx, g, i, j, k);
    ax[0] = axis_nb(idx, i, g.nx, 1, bc[0]);
    ax[1] = axis_nb(idx, j, g.ny, g.nx, bc[1]);
    ax[2] = axis_nb(idx, k, g.nz, g.nx * g.ny, bc[2]);
}

struct ProjGeo {
    lm::Geo g;
    int bc[3];
    double ih[3];      // 1 / h per axis
};

__global__ void __launch_bounds__(lm::NT) k_projection_rhs(ProjGeo G, double dt, const double* __restrict__ P,
                                                           const double* __restrict__ rho_o,
                                                           const double* __restrict__ cs2,
                                                           const double* __restrict__ m_o,
                                                           const double* __restrict__ m_s,
                                                           const double* __restrict__ rho_n,
                                                           const double* __restrict__ S, double* __restrict__ f,
                                                           double* __restrict__ uf) {
    const int N = G.g.N;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        AxisNb ax[3];
        cell_axes(idx, G.g, G.bc, ax);
        const double ro = rho_o[idx], rn = rho_n[idx];
        double adv = 0.0, div = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double* ma = m_s + (size_t)a * N;
            double um = 0.0;
            if (ax[a].live) {
                adv += (m_o[(size_t)a * N + idx] / ro) * grad_axis(ax[a], idx, P, rho_o, G.ih[a]);
                const double mc = ma[idx];
                um = ax[a].wm ? 0.0 : (ma[ax[a].m] + mc) / (rho_n[ax[a].m] + rn);
                const double up = ax[a].wp ? 0.0 : (mc + ma[ax[a].p]) / (rn + rho_n[ax[a].p]);
                div += (up - um) * G.ih[a];
            }
            uf[(size_t)a * N + idx] = um;
        }
        double fi = (P[idx] - dt * adv) / (dt * dt * ro * cs2[idx]) - div / dt;
        if (S) fi -= S[idx];
        f[idx] = fi;
    }
}

__global__ void __launch_bounds__(lm::NT) k_projection_update(ProjGeo G, double dt, const double* __restrict__ P,
                                                              const double* __restrict__ rho_n,
                                                              const double* __restrict__ m_s,
                                                              const double* __restrict__ uf_s,
                                                              const double* __restrict__ e_s,
                                                              double* __restrict__ m_new,
                                                              double* __restrict__ uf_new,
                                                              double* __restrict__ e_new) {
    const int N = G.g.N;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
        AxisNb ax[3];
        cell_axes(idx, G.g, G.bc, ax);
        const double Pc = P[idx], rn = rho_n[idx];
        double div = 0.0, ugp = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double* ua = uf_s + (size_t)a * N;
            double um = 0.0, mnew = m_s[(size_t)a * N + idx];
            if (ax[a].live) {
                const double gp = grad_axis(ax[a], idx, P, rho_n, G.ih[a]);
                mnew -= dt * gp;                                         // Eq. momupdate
                // step (vii) on the minus and plus faces
                um = ax[a].wm ? 0.0 : ua[idx] - dt * (Pc - P[ax[a].m]) * G.ih[a] * 2.0 / (rn + rho_n[ax[a].m]);
                const double up = ax[a].wp ? 0.0
                                           : ua[ax[a].p] - dt * (P[ax[a].p] - Pc) * G.ih[a] * 2.0 /
                                                               (rho_n[ax[a].p] + rn);
                div += (up - um) * G.ih[a];
                ugp += (mnew / rn) * gp;
            }
            m_new[(size_t)a * N + idx] = mnew;
            uf_new[(size_t)a * N + idx] = um;
        }
        e_new[idx] = e_s[idx] - dt * (Pc * div + ugp);                   // step (viii)
    }
}

int proj_geo(int ndim, const int64_t n[3], const double h[3], const int bc[3], ProjGeo* G) {
    if (!n || !h || !bc || (ndim != 2 && ndim != 3)) return LM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || !(h[a] > 0.0) || (bc[a] != LM_BC_PERIODIC && bc[a] != LM_BC_NEUMANN)) return LM_ERR_INVALID_ARG;
    if ((ndim == 2 && n[1] != 1) || (long long)n[0] * n[1] * n[2] >= (1LL << 31)) return LM_ERR_INVALID_ARG;
    *G = ProjGeo{};
    G->g.nx = (int)n[0];
    G->g.ny = (int)n[1];
    G->g.nz = (int)n[2];
    G->g.N = G->g.nx * G->g.ny * G->g.nz;
    for (int a = 0; a < 3; ++a) {
        G->bc[a] = bc[a];
        G->ih[a] = 1.0 / h[a];
    }
    G->g.bcx = bc[0];
    G->g.bcy = bc[1];
    G->g.bcz = bc[2];
    return LM_OK;
}

int blocks(int N) {
    int b = (N + lm::NT - 1) / lm::NT;
    return b < 1 ? 1 : (b > 8 * 152 ? 8 * 152 : b);
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

int lm_projection_rhs(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt, const double* p_old,
                      const double* rho_old, const double* cs2_old, const double* mom_old, const double* mom_star,
                      const double* rho_new, const double* source, double* f, double* uface_star, void* stream) {
    ProjGeo G;
    int rc = proj_geo(ndim, n, h, bc, &G);
    if (rc) return rc;
    if (!p_old || !rho_old || !cs2_old || !mom_old || !mom_star || !rho_new || !f || !uface_star ||
        !(dt > 0.0 && dt < 1e300))
        return LM_ERR_INVALID_ARG;
    lm::count_launches(1);
    k_projection_rhs<<<blocks(G.g.N), lm::NT, 0, (cudaStream_t)stream>>>(G, dt, p_old, rho_old, cs2_old, mom_old,
                                                                          mom_star, rho_new, source, f, uface_star);
    return finish("lm_projection_rhs");
}

int lm_projection_update(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt,
                         const double* p_pred, const double* rho_new, const double* mom_star,
                         const double* uface_star, const double* e_star, double* mom_new, double* uface_new,
                         double* e_new, void* stream) {
    ProjGeo G;
    int rc = proj_geo(ndim, n, h, bc, &G);
    if (rc) return rc;
    if (!p_pred || !rho_new || !mom_star || !uface_star || !e_star || !mom_new || !uface_new || !e_new ||
        uface_new == uface_star || !(dt > 0.0 && dt < 1e300))
        return LM_ERR_INVALID_ARG;
    lm::count_launches(1);
    k_projection_update<<<blocks(G.g.N), lm::NT, 0, (cudaStream_t)stream>>>(G, dt, p_pred, rho_new, mom_star,
                                                                             uface_star, e_star, mom_new, uface_new,
                                                                             e_new);
    return finish("lm_projection_update");
}

}  // extern "C"
