// Float32 kernels: the operator with faces formed on the fly from rho, the
// flexible-CG vector steps with float64-accurate dot products, and the
// geometric-multigrid V-cycle pieces (coefficient coarsening, red-black
// Gauss-Seidel, fused residual + restriction, prolongation, exact coarsest
// solve).  These are HBM-bound: each reads its vectors once and recomputes
// face conductances from rho instead of storing them.
#include "lm_common.cuh"
#include "lm_kernels.h"

namespace lm {

// g = (2/h^2) / (rho_a + rho_b); the sum is commutative, so both cells of a
// face compute the same bits and the operator stays exactly symmetric.
__device__ __forceinline__ float face32(float ra, float rb, float c2) { return __fdividef(c2, ra + rb); }

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

// ---- operator and flexible CG ---------------------------------------------

__global__ void __launch_bounds__(NT) k_apply32(Lev32 L, const float* __restrict__ x, float* __restrict__ y,
                                                double* __restrict__ part) {
    __shared__ double sm[32];
    FF acc{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.g.N; idx += stride) {
        int i, j, k;
        cell_coords(idx, L.g, i, j, k);
        const float v = apply32_at(idx, i, j, k, L, x);
        y[idx] = v;
        ff_add_prod(acc, x[idx], v);
    }
    if (part) {
        double v[1] = {ff_value(acc)};
        write_partials<1>(v, part, sm);
    }
}

__global__ void __launch_bounds__(NT) k_dot32(int N, const float* __restrict__ a, const float* __restrict__ b,
                                              double* __restrict__ part) {
    __shared__ double sm[32];
    FF acc{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) ff_add_prod(acc, a[idx], b[idx]);
    double v[1] = {ff_value(acc)};
    write_partials<1>(v, part, sm);
}

// Flexible CG, truncation 1 (Notay 2000): p = z - (z.q_old / p_old.q_old) p_old.
// Slots: 0 p.q, 1 r.r, 5 z.q_old, 6 p.r
__global__ void __launch_bounds__(NT) k_fcg_beta_p(int N, const float* __restrict__ z, float* __restrict__ p,
                                                   const double* __restrict__ part, int first) {
    __shared__ double sm[32];
    float beta = 0.f;
    if (!first) {
        const double zq = reduce_partials(part + 5 * MAX_PARTIALS, gridDim.x, sm);
        const double pq = reduce_partials(part + 0 * MAX_PARTIALS, gridDim.x, sm);
        beta = pq > 0.0 ? (float)(-zq / pq) : 0.f;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride)
        p[idx] = first ? z[idx] : fmaf(beta, p[idx], z[idx]);
}

__global__ void __launch_bounds__(NT) k_fcg_apply(Lev32 L, const float* __restrict__ p, float* __restrict__ q,
                                                  const float* __restrict__ r, double* __restrict__ part) {
    __shared__ double sm[64];
    FF pq{0.f, 0.f}, pr{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.g.N; idx += stride) {
        int i, j, k;
        cell_coords(idx, L.g, i, j, k);
        const float v = apply32_at(idx, i, j, k, L, p);
        q[idx] = v;
        const float pi = p[idx];
        ff_add_prod(pq, pi, v);
        ff_add_prod(pr, pi, r[idx]);
    }
    double v[2] = {ff_value(pq), ff_value(pr)};
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) {
        part[0 * MAX_PARTIALS + blockIdx.x] = v[0];
        part[6 * MAX_PARTIALS + blockIdx.x] = v[1];
    }
}

// alpha = p.r / p.q; e += alpha p; r -= alpha q; partial r.r (slot 1)
__global__ void __launch_bounds__(NT) k_fcg_update(int N, float* __restrict__ e, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   double* __restrict__ part, SolveState* st) {
    __shared__ double sm[32];
    const double pq = reduce_partials(part + 0 * MAX_PARTIALS, gridDim.x, sm);
    const double pr = reduce_partials(part + 6 * MAX_PARTIALS, gridDim.x, sm);
    const bool bad = !(pq > 0.0) || !isfinite(pq) || !isfinite(pr);
    if (bad) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->status = LM_ERR_BREAKDOWN;
    }
    const float alpha = bad ? 0.f : (float)(pr / pq);
    FF rr{0.f, 0.f};
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += stride) {
        const float pi = p[idx];
        e[idx] = fmaf(alpha, pi, e[idx]);
        const float ri = fmaf(-alpha, q[idx], r[idx]);
        r[idx] = ri;
        ff_add_prod(rr, ri, ri);
    }
    double v[1] = {ff_value(rr)};
    write_partials<1>(v, part + 1 * MAX_PARTIALS, sm);
}

// ---- multigrid ----------------------------------------------------------------

__device__ __forceinline__ void coords3(int t, int nx, int ny, int& i, int& j, int& k) {
    i = t % nx;
    const int u = t / nx;
    j = u % ny;
    k = u / ny;
}

// Mean of the children's c~ and rho (coarse coefficients).
__global__ void k_coarsen(Lev32 F, Geo C, int hx, int hy, int hz, float* __restrict__ ct_c,
                          float* __restrict__ rho_c) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= C.N) return;
    int I, J, K;
    coords3(t, C.nx, C.ny, I, J, K);
    float sc = 0.f, sr = 0.f;
    const int nch = (1 << hx) << hy << hz;
    for (int c = 0; c <= hz; ++c)
        for (int b = 0; b <= hy; ++b)
            for (int a = 0; a <= hx; ++a) {
                const int i = (I << hx) + a, j = (J << hy) + b, k = (K << hz) + c;
                const int idx = i + F.g.nx * (j + F.g.ny * k);
                sc += F.ct[idx];
                sr += F.rho[idx];
            }
    ct_c[t] = sc / (float)nch;
    rho_c[t] = sr / (float)nch;
}

// Red-black Gauss-Seidel: update every cell of colour `colour`
// ((i + j + k) mod 2) from its row: x_i = (f_i + sum g x_nb) / (c~_i + sum g).
// One thread per cell of the colour.  zero_guess: neighbours are taken as 0.
__global__ void __launch_bounds__(NT) k_smooth(Lev32 L, float* __restrict__ x, const float* __restrict__ f,
                                               int colour, int zero_guess) {
    const Geo& g = L.g;
    const int hw = (g.nx + 1) >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= hw * g.ny * g.nz) return;
    const int m = t % hw;
    const int row = t / hw;
    const int j = row % g.ny, k = row / g.ny;
    const int i = 2 * m + ((colour + j + k) & 1);
    if (i >= g.nx) return;
    const int idx = i + g.nx * row;
    const float rc = L.rho[idx];
    float d = L.ct[idx], num = f[idx];
    Nbr n = nbr_x(idx, i, g);
    if (face_minus(i, g.nx, g.bcx)) {
        const float w = face32(rc, L.rho[n.im], L.c2x);
        d += w;
        if (!zero_guess) num += w * x[n.im];
    }
    if (face_plus(i, g.nx, g.bcx)) {
        const float w = face32(rc, L.rho[n.ip], L.c2x);
        d += w;
        if (!zero_guess) num += w * x[n.ip];
    }
    if (g.ny > 1) {
        n = nbr_y(idx, j, g);
        if (face_minus(j, g.ny, g.bcy)) {
            const float w = face32(rc, L.rho[n.im], L.c2y);
            d += w;
            if (!zero_guess) num += w * x[n.im];
        }
        if (face_plus(j, g.ny, g.bcy)) {
            const float w = face32(rc, L.rho[n.ip], L.c2y);
            d += w;
            if (!zero_guess) num += w * x[n.ip];
        }
    }
    n = nbr_z(idx, k, g);
    if (face_minus(k, g.nz, g.bcz)) {
        const float w = face32(rc, L.rho[n.im], L.c2z);
        d += w;
        if (!zero_guess) num += w * x[n.im];
    }
    if (face_plus(k, g.nz, g.bcz)) {
        const float w = face32(rc, L.rho[n.ip], L.c2z);
        d += w;
        if (!zero_guess) num += w * x[n.ip];
    }
    x[idx] = __fdividef(num, d);
}

// fc = mean over children of (f - A x): residual and restriction fused.
__global__ void __launch_bounds__(NT) k_resid_restrict(Lev32 F, Geo C, int hx, int hy, int hz,
                                                       const float* __restrict__ x, const float* __restrict__ f,
                                                       float* __restrict__ fc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= C.N) return;
    int I, J, K;
    coords3(t, C.nx, C.ny, I, J, K);
    float s = 0.f;
    for (int c = 0; c <= hz; ++c)
        for (int b = 0; b <= hy; ++b)
            for (int a = 0; a <= hx; ++a) {
                const int i = (I << hx) + a, j = (J << hy) + b, k = (K << hz) + c;
                const int idx = i + F.g.nx * (j + F.g.ny * k);
                s += f[idx] - apply32_at(idx, i, j, k, F, x);
            }
    fc[t] = s / (float)((1 << hx) << hy << hz);
}

// x += P xc (piecewise-constant prolongation)
__global__ void __launch_bounds__(NT) k_prolong_add(Geo F, Geo C, int hx, int hy, int hz, float* __restrict__ x,
                                                    const float* __restrict__ xc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F.N) return;
    int i, j, k;
    coords3(t, F.nx, F.ny, i, j, k);
    x[t] += xc[(i >> hx) + C.nx * ((j >> hy) + C.ny * (k >> hz))];
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
        int i, j, k;
        coords3(idx, g.nx, g.ny, i, j, k);
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
        const double piv = rowk[kk];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e % n;
            double v;
            if (i == kk && j == kk) v = 1.0 / piv;
            else if (i == kk) v = rowk[j] / piv;
            else if (j == kk) v = -colk[i] / piv;
            else v = A[e] - colk[i] * rowk[j] / piv;
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

static inline int nblk(long long n) { return (int)((n + NT - 1) / NT); }

void launch_apply32(const Lev32& L, int G, cudaStream_t s, const float* x, float* y, double* part) {
    count_launches(1);
    k_apply32<<<G, NT, 0, s>>>(L, x, y, part);
}
void launch_dot32(int N, int G, cudaStream_t s, const float* a, const float* b, double* part, int slot) {
    count_launches(1);
    k_dot32<<<G, NT, 0, s>>>(N, a, b, part + slot * MAX_PARTIALS);
}
void launch_fcg_beta_p(int N, int G, cudaStream_t s, const float* z, float* p, const float* /*q_old*/,
                       double* part, int first) {
    count_launches(1);
    k_fcg_beta_p<<<G, NT, 0, s>>>(N, z, p, part, first);
}
void launch_fcg_apply(const Lev32& L, int G, cudaStream_t s, const float* p, float* q, const float* r,
                      double* part) {
    count_launches(1);
    k_fcg_apply<<<G, NT, 0, s>>>(L, p, q, r, part);
}
void launch_fcg_update(int N, int G, cudaStream_t s, float* e, float* r, const float* p, const float* q,
                       double* part, SolveState* st) {
    count_launches(1);
    k_fcg_update<<<G, NT, 0, s>>>(N, e, r, p, q, part, st);
}
void launch_coarsen(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s, float* ct_c,
                    float* rho_c) {
    count_launches(1);
    k_coarsen<<<nblk(C.g.N), NT, 0, s>>>(F, C.g, hx, hy, hz, ct_c, rho_c);
}
void launch_smooth(const Lev32& L, cudaStream_t s, float* x, const float* f, int colour, int zero_guess) {
    const long long n = (long long)((L.g.nx + 1) >> 1) * L.g.ny * L.g.nz;
    count_launches(1);
    k_smooth<<<nblk(n), NT, 0, s>>>(L, x, f, colour, zero_guess);
}
void launch_resid_restrict(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s,
                           const float* x, const float* f, float* fc) {
    count_launches(1);
    k_resid_restrict<<<nblk(C.g.N), NT, 0, s>>>(F, C.g, hx, hy, hz, x, f, fc);
}
void launch_prolong_add(const Lev32& F, const Lev32& C, int hx, int hy, int hz, cudaStream_t s, float* x,
                        const float* xc) {
    count_launches(1);
    k_prolong_add<<<nblk(F.g.N), NT, 0, s>>>(F.g, C.g, hx, hy, hz, x, xc);
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
