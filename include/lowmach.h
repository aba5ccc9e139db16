/*
 * lowmach.h -- C ABI of the GB300 generalized-Poisson pressure solver.
 *
 * The solver computes the pressure prediction of the semi-implicit low-Mach
 * fractional-step method of Happenhofer et al. (arXiv 1112.3507): every
 * timestep (every Runge-Kutta stage, Sec. 2.6) it solves
 *
 *     c~ P - div(kappa grad P) = f                       (Sec. 2, Eq. Poiss;
 *                                        Sec. 2.5, Eq. GeneralizedPoisson)
 *     c~    = 1 / (dt^2 rho^n c_s^2)                      (Eq. cpoiss)
 *     kappa = 1 / rho^{n+1}                               (Eq. kappapoiss)
 *
 * with homogeneous Neumann walls (Eq. vonNeumannBC) or periodic axes
 * (Sec. 3.2), on a cell-centred structured 2D/3D grid.  Discretization: the
 * cell-centred finite-volume operator
 *
 *     (A x)_i = c~_i x_i + sum_{faces f of i} g_f (x_i - x_nb(f)),
 *     g_f = kappa_f / h_axis^2,  kappa_f = 2 / (rho_L + rho_R),
 *
 * the face kappa being the harmonic mean of 1/rho (the factor of the
 * face-velocity update, step (viii) of Sec. 2.4).  A is symmetric positive
 * definite whenever rho > 0 and c~ > 0 (Sec. 2.5: Lax-Milgram conditions).
 *
 * Layout: every field is a dense array of n[0]*n[1]*n[2] values, x fastest:
 * flat index i + n[0]*(j + n[1]*k).  A 2D grid has ndim = 2, n[1] = 1 (x is
 * horizontal, the second extent n[2] is vertical).  All values are float64
 * unless stated.
 *
 * Pointers: arguments named *_on_device / on_device = 1 are CUDA device
 * pointers on the grid's device (for instance torch.Tensor.data_ptr());
 * on_device = 0 means host memory.  Input pointers are borrowed: the library
 * copies what it needs before returning (device copies are ordered on the
 * given stream).  Output buffers are allocated by the caller.  `stream` is a
 * cudaStream_t (NULL = legacy default stream); every kernel of a call runs
 * on it.
 *
 * Errors: 0 = LM_OK, negative = failure (see lm_status_string).  A failing
 * call leaves the grid usable.  Calls on one grid are not reentrant; distinct
 * grids may be used from distinct threads.
 *
 * Every entry point runs its arithmetic in this library's CUDA kernels; there
 * is no CPU fallback.  A grid's device is the current CUDA device at
 * lm_grid_create.
 */
#ifndef LOWMACH_H
#define LOWMACH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LM_OK                  0
#define LM_ERR_INVALID_ARG    -1   /* bad size, pointer, enum or option           */
#define LM_ERR_NOT_POSITIVE   -2   /* rho <= 0, c_s^2 <= 0, dt <= 0, c~ <= 0 or
                                      non-finite input: the Lax-Milgram
                                      positivity of Sec. 2.5 fails               */
#define LM_ERR_NO_CONVERGENCE -3   /* max_iter reached; solution and history kept */
#define LM_ERR_BREAKDOWN      -4   /* p^T A p <= 0 or non-finite inside a Krylov
                                      iteration                                  */
#define LM_ERR_TIMEOUT        -5   /* a bounded device-side wait expired           */
#define LM_ERR_CUDA           -6   /* a CUDA runtime call failed                   */
#define LM_ERR_NETWORK        -7   /* network weights missing or malformed         */
#define LM_ERR_OUT_OF_MEMORY  -8
#define LM_ERR_STATE          -9   /* a required input (coefficients, rhs) unset  */

/* ---- enums ------------------------------------------------------------- */
#define LM_BC_PERIODIC 0
#define LM_BC_NEUMANN  1

/* Solve modes.
 *  LM_FP64_JACOBI_PCG   conjugate gradients (Sec. 2.5) in float64 with the
 *                       Jacobi preconditioner: the plain GPU baseline.
 *  LM_FP64_MG_PCG       float64 vectors, conjugate gradients preconditioned
 *                       by a float32 geometric-multigrid V-cycle.
 *  LM_MIXED_MG_IR       iterative refinement: float64 residual and
 *                       correction, float32 inner flexible CG with the
 *                       multigrid V-cycle (float64-accurate dot products).
 *  LM_MIXED_LEARNED_FCG_IR  as LM_MIXED_MG_IR, with the learned network's
 *                       warm start and the network as preconditioner inside
 *                       flexible CG (falls back to LM_MIXED_MG_IR when no
 *                       network is loaded or the network output is unusable).
 */
#define LM_FP64_JACOBI_PCG      0
#define LM_FP64_MG_PCG          1
#define LM_MIXED_MG_IR          2
#define LM_MIXED_LEARNED_FCG_IR 3

#define LM_PREC_FP64 0
#define LM_PREC_FP32 1

typedef struct lm_grid lm_grid;

typedef struct {
    int    mode;            /* LM_FP64_JACOBI_PCG ...                              */
    double rtol;            /* stop when ||f - A x||_2 <= rtol ||f||_2 (true
                               float64 residual, unweighted over cells)          */
    int    max_iter;        /* Krylov iterations (all inner iterations in IR)     */
    int    use_x0;          /* 1: start from lm_set_initial_guess, 0: from zero   */
    int    max_outer;       /* iterative-refinement steps (mixed modes)           */
    int    nu1, nu2;        /* red-black Gauss-Seidel sweeps before/after the
                               coarse correction; nu1 == nu2 keeps the V-cycle
                               symmetric                                          */
    double inner_rtol;      /* relative reduction asked of each inner solve      */
    int    inner_max_iter;  /* inner iterations per refinement step               */
    int    check_every;     /* Krylov iterations between host convergence checks
                               (float64 modes).  Mixed modes check the inner
                               solve on the device (one host check per
                               refinement step) unless check_every == 1: then
                               the host checks after every inner iteration,
                               each iteration one CUDA graph launch (slower;
                               every kernel a plain graph node, which profilers
                               that time kernels one by one can see)          */
    int    net_precond;     /* LM_MIXED_LEARNED_FCG_IR, the inner preconditioner:
                               0 = the V-cycle (the network gives the warm
                               start only); 1 = the learned two-level cycle,
                               replaced by the V-cycle when it stalls (inner
                               residual above 1/2 after 4 iterations, or not
                               finite); 2 = the learned two-level cycle
                               throughout                                      */
    void*  cuda_stream;     /* cudaStream_t for every kernel of the solve         */
} lm_solve_opts;

typedef struct {
    int    status;          /* LM_OK or an LM_ERR_* code                          */
    int    iters;           /* Krylov iterations (inner iterations summed)        */
    int    outer_iters;     /* refinement steps (mixed modes), else 0             */
    int    vcycles;         /* multigrid V-cycles applied                         */
    double rel_residual;    /* final true relative residual ||f-Ax||/||f||, fp64 */
    double seconds;         /* device time of the solve (CUDA events)             */
} lm_solve_result;

/* Defaults: mode LM_MIXED_MG_IR, rtol 1e-8, max_iter 10000, nu1 = 2, nu2 = 3,
 * inner_rtol 1e-4, inner_max_iter 30, max_outer 12, check_every 8,
 * net_precond 0. */
void lm_default_opts(lm_solve_opts* opts);

/* ---- grid lifecycle ---------------------------------------------------- */

/* Create a grid of n[0] x n[1] x n[2] cells with spacings h[0..2] and one
 * boundary condition per axis (bc[a] in {LM_BC_PERIODIC, LM_BC_NEUMANN},
 * applied at both ends of axis a).  ndim 2 requires n[1] == 1.  Allocates
 * the grid's device buffers on the current device.  Errors:
 * LM_ERR_INVALID_ARG (non-positive sizes or spacings, bad bc),
 * LM_ERR_OUT_OF_MEMORY. */
int  lm_grid_create(int ndim, const int64_t n[3], const double h[3], const int bc[3], lm_grid** out);
void lm_grid_destroy(lm_grid* g);
int64_t lm_grid_size(const lm_grid* g);

/* ---- inputs ------------------------------------------------------------ */

/* Coefficient assembly (step (v) of Sec. 2.4): from rho^n, rho^{n+1}, c_s^2
 * (N values each) and dt, form c~ (Eq. cpoiss) and the face conductances
 * g_f from kappa = 1/rho^{n+1} (Eq. kappapoiss), the Jacobi diagonal and the
 * float32 copies used by multigrid.  Validates positivity and finiteness:
 * on LM_ERR_NOT_POSITIVE the grid holds no valid coefficients until the next
 * successful call (a solve then returns LM_ERR_STATE). */
int  lm_set_coefficients(lm_grid* g, const double* rho_old, const double* rho_new,
                         const double* cs2, double dt, int on_device, void* stream);

/* As lm_set_coefficients, with c~ given directly (N values) and kappa taken
 * as 1/rho_face_src: for problems stated in c~ and kappa (e.g. the solver
 * test of Sec. 2.5.2, kappa = 1/rho). */
int  lm_set_coefficients_raw(lm_grid* g, const double* ctilde, const double* rho_face_src,
                             int on_device, void* stream);

/* Right-hand side f (Eq. fpoiss / fpoiss2), N values, per unit volume in the
 * units of c~ P.  Inhomogeneous Neumann data g (outward normal derivative)
 * is folded in by the caller: f_i += kappa_wall g / h for wall cells. */
int  lm_set_rhs(lm_grid* g, const double* f, int on_device, void* stream);

/* Initial guess x0 (N values), used when opts.use_x0 = 1. */
int  lm_set_initial_guess(lm_grid* g, const double* x0, int on_device, void* stream);

/* Load the learned warm-start/preconditioner network (file written by
 * lm_unet_save); LM_ERR_NETWORK if missing or malformed. */
int  lm_load_network(lm_grid* g, const char* weights_path);

/* ---- solve --------------------------------------------------------------- */

/* Solve A P = f (step (vi) of Sec. 2.4) to opts->rtol in the chosen mode.
 * Returns LM_OK, LM_ERR_NO_CONVERGENCE (best iterate kept), LM_ERR_BREAKDOWN,
 * LM_ERR_STATE (coefficients or rhs missing), LM_ERR_INVALID_ARG (e.g. a
 * multigrid mode on a periodic axis with an odd cell count > 1).  `res` may
 * be NULL.  Synchronises the stream before returning. */
int  lm_solve(lm_grid* g, const lm_solve_opts* opts, lm_solve_result* res);

/* Copy the solution (N float64 values) out. */
int  lm_get_solution(lm_grid* g, double* out, int on_device, void* stream);

/* Relative residual ||r_k||/||f|| of every Krylov iteration of the last
 * solve (index 0 = initial residual); writes min(cap, count) values. */
int  lm_get_residual_history(lm_grid* g, double* out, int cap, int* n_written);

const char* lm_status_string(int status);

/* Number of CUDA kernels this library has launched in the process so far
 * (all grids, all streams); for launch accounting in benchmarks. */
int64_t lm_kernel_launches(void);

/* ---- row-level entry points (device pointers, caller's stream) -------- */

/* The assembled float64 coefficients: c~ (N), and per axis a the
 * conductance g of each cell's face with its minus-neighbour (N each; 0 on
 * a wall face and on an axis with one cell).  Any pointer may be NULL. */
int  lm_get_coefficients(lm_grid* g, double* ctilde, double* gx, double* gy, double* gz,
                         void* stream);

/* y = A x on device vectors of N values, float64 (prec LM_PREC_FP64, x and y
 * double*) or float32 (LM_PREC_FP32, float*, faces formed from float32
 * rho).  If dot_out != NULL it receives x^T A x accumulated to float64
 * accuracy (host pointer; the call then synchronises the stream). */
int  lm_apply(lm_grid* g, int prec, const void* x, void* y, double* dot_out, void* stream);

/* One float32 multigrid V-cycle z = M r (zero initial guess, nu1/nu2
 * red-black Gauss-Seidel sweeps, exact coarsest solve), the preconditioner
 * of the multigrid modes; r, z float32 device vectors of N values.  Builds
 * the hierarchy from the current coefficients if needed. */
int  lm_mg_vcycle(lm_grid* g, const float* r, float* z, int nu1, int nu2, void* stream);

/* One red-black Gauss-Seidel sweep of the V-cycle's smoother on the finest
 * level, float32: every cell of the first colour takes the value that
 * solves its row of A x = f with its neighbours' values from x_in, then
 * every cell of the second colour does the same with the updated values.
 * order 0: red (i+j+k even) first, 1: black first.  x_in == NULL means
 * x_in = 0.  x_in, f, x_out: float32 device vectors of N values; x_out
 * must not overlap x_in or f.  LM_ERR_INVALID_ARG for an order other than
 * 0/1 or a grid the hierarchy does not support (odd periodic extent). */
int  lm_mg_sweep(lm_grid* g, const float* x_in, const float* f, float* x_out, int order, void* stream);

/* Number of multigrid levels and the cell counts of level `level`
 * (n_out[3]); LM_ERR_INVALID_ARG past the coarsest level. */
int  lm_mg_level_shape(lm_grid* g, int level, int64_t n_out[3], int* num_levels);

/* ---- the learned warm start / preconditioner ----------------------------- */
/* A 4-level U-Net on 2D images (rows = z, columns = x; NHWC, batch B):
 * encoder e_l = relu(conv3(relu(conv3(in_l, A_l)), B_l)), in_0 = the 3-channel
 * input, in_l = 2x2 mean of e_{l-1}; decoder d_l = relu(conv3(relu(conv3(
 * [up2(d_{l+1}), e_l], C_l)), D_l)), d_3 = e_3; output y = conv1(d_0, O).
 * conv3: 3x3, zero padding, weights [3][3][Cin][Cout]; channels ch[0..3]
 * (16, 32, 48, 64 by default).  BF16 weights and activations, FP32
 * accumulation, FP32 master weights trained by Adam.  The paper has no
 * learned component: this serves the learned mode LM_MIXED_LEARNED_FCG_IR.
 * Images need H, W divisible by 8.  Device buffers are float32 and ordered
 * on `stream`; parameter arrays are host float32 in the storage order
 * A0 a0 B0 b0 A1 a1 B1 b1 A2 a2 B2 b2 A3 a3 B3 b3 C2 c2 D2 d2 C1 c1 D1 d1
 * C0 c0 D0 d0 O o. */
typedef struct lm_net lm_net;
int  lm_net_create(const int ch[4], lm_net** out);
void lm_net_destroy(lm_net* net);
int  lm_net_num_params(const lm_net* net);
int  lm_net_set_params(lm_net* net, const float* host, int n);   /* also resets Adam state */
int  lm_net_get_params(lm_net* net, float* host, int n);
int  lm_net_get_grads(lm_net* net, float* host, int n);          /* of the last lm_net_backward */
/* y (B*H*W) = net(x (B*H*W*3)); keeps the activations for lm_net_backward */
int  lm_net_forward(lm_net* net, const float* x, float* y, int B, int H, int W, void* stream);
/* parameter gradients of sum(gy * y) for the last forward (overwritten) */
int  lm_net_backward(lm_net* net, const float* gy, void* stream);
/* loss = mean((y - t)^2) over n values, gy = its gradient (device); *loss on host if non-NULL */
int  lm_net_mse(lm_net* net, const float* y, const float* t, float* gy, long long n, double* loss, void* stream);
/* one Adam step (Kingma & Ba) with bias correction on the last gradients */
int  lm_net_adam(lm_net* net, float lr, float beta1, float beta2, float eps, void* stream);
/* file: "LMUNET01", int32 ch[4], int32 n, float32 params[n], uint64 FNV-1a of the params */
int  lm_net_save(lm_net* net, const char* path);
int  lm_net_load(const char* path, lm_net** out);               /* LM_ERR_NETWORK if bad */
/* Network input of a 2D grid from v (device float64, N): channel 0 = v/rms(v),
 * 1 = log(rho/mean rho), 2 = log(1/(c~ rho h_z^2))/10 (feat: N*3 float, device);
 * *scale = rms(v)/(mean c~ + pi^2 mean(1/rho)), the factor that turns the
 * network output into an approximation of A^-1 v. */
int  lm_net_features(lm_grid* g, const double* v, float* feat, double* scale, void* stream);

/* ---- batched solves ------------------------------------------------------ */

/* Solve `count` independent 2D grids (distinct lm_grid handles, each with
 * coefficients and rhs set) in the mixed-precision mode of LM_MIXED_MG_IR,
 * all at once: every phase of the solve is one launch over the tiles of all
 * grids, grids that have converged skip their tiles, and one refinement
 * step is captured as a CUDA graph whose inner flexible-CG iterations form
 * a device-side while loop (a conditional graph node that repeats while
 * some grid still iterates, at most opts->inner_max_iter times); the graph
 * is replayed up to opts->max_outer times.  The sweep
 * z-chunk of every level shape is chosen by the autotuner (see
 * lm_autotune_set_cache).  The captured plan is cached per (grids,
 * coefficient versions, inner_max_iter, use_x0) and reused by later calls.
 * Grids whose coefficients changed since their last solve get their
 * multigrid hierarchies refreshed first, their coarsest-level inverses all
 * formed in one launch.
 * Requirements: 2D grids (ndim 2), 1 <= nu1, nu2 <= 8, an exactly solved
 * coarsest level (grids whose halvings reach <= 64 cells), even periodic
 * extents.
 * results[i] receives grid i's status, inner iterations (iters = vcycles),
 * refinement steps and final float64 relative residual; `seconds` is the
 * device time of the whole batch.  Returns LM_OK or the first failing
 * grid's status; LM_ERR_INVALID_ARG / LM_ERR_STATE before any work. */
int  lm_batch_solve(lm_grid* const* grids, int count, const lm_solve_opts* opts, lm_solve_result* results);

/* Coefficient assembly of `count` grids at once: lm_set_coefficients of
 * each (step (v) of Sec. 2.4; Eqs. cpoiss, kappapoiss) in one launch over
 * all of them and one wait for their positivity reports.  rho_old[i],
 * rho_new[i], cs2[i]: device pointers to grid i's N_i values (float64);
 * dt[i]: host.  Each grid is left as lm_set_coefficients would leave it;
 * returns LM_OK or the first failing grid's status (LM_ERR_NOT_POSITIVE for
 * a non-positive or non-finite input; that grid then holds no coefficients).
 * The hierarchies of the grids are refreshed by the next lm_batch_solve, one
 * launch per level over all of them. */
int  lm_batch_set_coefficients(lm_grid* const* grids, int count, const double* const* rho_old,
                               const double* const* rho_new, const double* const* cs2, const double* dt,
                               void* stream);

/* Autotuner cache: a JSON object {"<gpu>|rbgs2d-zm|<nx>x<nz>|bc<x><z>|f32": kz,
 * "<gpu>|rbgs2d-batch|d<depth>|<hash>": kz, ...}: the fastest sweep z-chunk
 * (rows per tile) per level shape for one grid, and per multigrid depth of a
 * batch (timed on the batched sweep over every grid's tiles of that depth;
 * <hash> = FNV-1a of the batch's level shapes and boundary conditions),
 * read on first use and rewritten when new entries are timed.  Default path: $LM_AUTOTUNE_CACHE or
 * $HOME/.cache/lowmach_autotune.json.  NULL or "" restores the default.
 * Clears the in-memory table. */
int  lm_autotune_set_cache(const char* path);

/* ---- building blocks of a z-slab decomposed solve ------------------------- */
/* The paper runs its pressure solve domain-decomposed on a CPU cluster
 * (Sec. 2.5, the parallel solver and its strong-scaling table); here a rank
 * (one GPU) owns the planes [z0, z1) of the global grid in an extended
 * local lm_grid whose first and last planes are ghost copies of the
 * neighbours' boundary planes (a wall in z on the local grid; its wall
 * faces touch ghost planes only).  A host driver (the package's shard
 * module) exchanges ghost planes and float64 scalars between ranks and
 * sequences the entry points below; all arithmetic on grid data runs in
 * these kernels.  Device pointers, ordered on `stream`. */

/* Halo pack (unpack = 0) or unpack (unpack = 1) of the z-boundary planes of
 * a cell array `a` (elem_bytes 4 or 8, plane_elems = nx*ny values a plane):
 * buf = [planes lo_first .. lo_first + nplanes) then [planes hi_first ..
 * hi_first + nplanes); a side whose first plane is negative is skipped
 * (its part of buf untouched).  One launch for both sides.
 * LM_ERR_INVALID_ARG for bad sizes or both sides skipped. */
int  lm_halo_pack(const void* a, int elem_bytes, int64_t plane_elems, int64_t lo_first, int64_t hi_first,
                  int nplanes, void* buf, int unpack, void* stream);

/* out = alpha x + beta y (y may be NULL: out = alpha x), n values; x, y,
 * out in float64 (LM_PREC_FP64) or float32 (LM_PREC_FP32) each, arithmetic
 * in float64; out may alias x or y. */
int  lm_vec_axpby(int64_t n, double alpha, const void* x, int x_prec, double beta, const void* y, int y_prec,
                  void* out, int out_prec, void* stream);

/* *out (host) = sum a_i b_i over n values, float64 accumulation in a fixed
 * order (bitwise reproducible); scratch: caller-allocated device buffer of
 * at least 1025 doubles.  Synchronises the stream. */
int  lm_vec_dot(int64_t n, const void* a, int a_prec, const void* b, int b_prec, double* scratch, double* out,
                void* stream);

/* z = d .* r (float64, n values). */
int  lm_vec_mul(int64_t n, const double* d, const double* r, double* z, void* stream);

/* The inverse Jacobi diagonal 1/(c~ + sum of the cell's face conductances)
 * of the grid's float64 operator (N values), the preconditioner of the
 * plain float64 PCG (Sec. 2.5 uses incomplete Cholesky). */
int  lm_jacobi_inverse_diagonal(lm_grid* g, double* dinv, void* stream);

/* The V-cycle's transfers between level 0 and level 1 (lm_mg_level_shape):
 * fc = R (f - A32 x), the restriction (mean over the children) of the
 * float32 residual; x += P ec, the piecewise-constant prolongation of a
 * level-1 vector.  Float32 device vectors. */
int  lm_mg_restrict_residual(lm_grid* g, const float* x, const float* f, float* fc, void* stream);
int  lm_mg_prolong_add(lm_grid* g, const float* ec, float* x, void* stream);

/* The float32 coefficients of multigrid level `level`: c~ and rho /
 * *rho_scale (the float32 copy of rho is kept divided by a power of two,
 * reported in *rho_scale), as the hierarchy holds them (levels >= 1: means
 * over the children).  ct, rho: device arrays of the level's cell count (or
 * NULL). */
int  lm_mg_level_coefficients(lm_grid* g, int level, float* ct, float* rho, double* rho_scale, void* stream);

/* ---- the steps either side of the solve (Sec. 2, steps (iv)-(viii)) ------- */
/* One fractional step's pressure projection around lm_solve, float64.
 * Vector fields (momenta) are three arrays of N values, x then y then z
 * components, consecutive (the y component of a 2D grid is carried along
 * unchanged); face arrays hold, per axis, each cell's minus face (the face
 * with its -1 neighbour), 3N values.  Pressures at faces follow Eq. pbnd,
 * cell gradients Eq. nablaP; on a wall axis (LM_BC_NEUMANN) the wall face
 * has no velocity and the wall cell's pressure; periodic axes wrap.  n, h,
 * bc: host arrays as in lm_grid_create; all fields device pointers. */

/* f (Eq. fpoiss) = (P^n - dt u^n.grad P^n) / (dt^2 rho^n c_s^2) - div u* / dt
 * - source, with u^n = mom_old / rho_old, u* on the faces = ((rho u)*_L +
 * (rho u)*_R) / (rho^{n+1}_L + rho^{n+1}_R) (written to uface_star) and
 * source the viscous and conductive part of Eq. fpoiss (NULL: inviscid).
 * Then lm_set_coefficients(rho_old, rho_new, cs2_old, dt) and lm_set_rhs(f)
 * pose Eq. Poiss for lm_solve. */
int  lm_projection_rhs(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt,
                       const double* p_old, const double* rho_old, const double* cs2_old, const double* mom_old,
                       const double* mom_star, const double* rho_new, const double* source, double* f,
                       double* uface_star, void* stream);

/* With the predicted pressure p_pred (lm_get_solution): mom_new = mom_star -
 * dt grad P (Eq. momupdate, rho^{n+1} in Eq. pbnd); uface_new = uface_star -
 * dt (P_R - P_L)/h * 2/(rho_L + rho_R) (step (vii)); e_new = e_star - dt
 * (P div u^{n+1} + u^{n+1}.grad P) (step (viii)), u^{n+1} = mom_new / rho_new.
 * uface_new must not overlap uface_star; mom_new / e_new may alias mom_star
 * / e_star. */
int  lm_projection_update(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt,
                          const double* p_pred, const double* rho_new, const double* mom_star,
                          const double* uface_star, const double* e_star, double* mom_new, double* uface_new,
                          double* e_new, void* stream);

/* Steps (i)-(iii) of Sec. 2.4, the explicit advection: face velocities
 * u_{i+1/2} = ((rho u)_i + (rho u)_{i+1}) / (rho_i + rho_{i+1}) (Eq. step1),
 * the modified flux F~ = (rho, rho u, e, rho c) u_{i+1/2} with the advected
 * quantity taken from the upwind side's MUSCL state (minmod-limited slope:
 * the paper's CPM/MENO reconstruction is not given in its text), and
 * q^{new} = q^n - dt d(F~)/dx summed over the axes with more than one cell.
 * A wall face (LM_BC_NEUMANN) carries no flux and the cells next to a wall
 * have zero slope; periodic axes wrap.  n, h, bc: host arrays as in
 * lm_grid_create.  Device arrays of N = n[0] n[1] n[2] doubles: rho, e,
 * rho_c (optional, the two-component flow's rho c; NULL with rho_c_new
 * NULL), and mom, mom_star: three consecutive arrays (x, y, z components).
 * Outputs rho_new, mom_star, e_star, rho_c_new must not overlap any input.
 * Inviscid: the viscous flux of step (ii) is the caller's (lm_diffusion4).
 * LM_ERR_INVALID_ARG for bad sizes, dt < 0 or overlapping arrays. */
int  lm_advect(int ndim, const int64_t n[3], const double h[3], const int bc[3], double dt, const double* rho,
               const double* mom, const double* e, const double* rho_c, double* rho_new, double* mom_star,
               double* e_star, double* rho_c_new, void* stream);

/* Step (ix) of Sec. 2.4 for an ideal gas: p = (gamma - 1)(e - |rho u|^2 /
 * (2 rho)) and, when cs2 is not NULL, c_s^2 = gamma p / rho (the next step's
 * c~, Eq. cpoiss).  Device arrays of n_cells doubles (mom: three consecutive
 * arrays).  LM_ERR_INVALID_ARG for gamma <= 1 or a bad size. */
int  lm_eos_ideal(int64_t n_cells, double gamma, const double* rho, const double* mom, const double* e, double* p,
                  double* cs2, void* stream);

/* ---- the viscous terms' dissipative stencil (Sec. 4) --------------------- */

/* out = beta u + alpha sum_a (U_aa): the dissipative fourth-order second
 * derivative of Sec. 4 (face derivatives of Eq. fv-approach2 differenced,
 * i.e. the five-point stencil of Eq. dissipativestencil4,
 * (-U_{i-2} + 16 U_{i-1} - 30 U_i + 16 U_{i+1} - U_{i+2}) / (12 h^2)), summed
 * over the axes with more than one cell (directional splitting).  A
 * periodic axis wraps; a wall axis (LM_BC_NEUMANN) carries no flux through
 * the wall (mirror ghosts U_{-1-k} = U_k).  With beta = 1, alpha = nu dt it
 * is one explicit Euler step of u_t = nu Delta u, monotone while
 * nu dt / h^2 <= 3 / (8 d) in d dimensions.  n, h, bc: host arrays as in
 * lm_grid_create; u, out: device arrays of n[0]*n[1]*n[2] values of
 * precision prec (LM_PREC_FP64 or LM_PREC_FP32), not overlapping.
 * LM_ERR_INVALID_ARG for bad sizes, precision or aliasing. */
int  lm_diffusion4(int ndim, const int64_t n[3], const double h[3], const int bc[3], int prec, double alpha,
                   const void* u, double beta, void* out, void* stream);

/* ---- the operator in Q1 finite elements (Sec. 2.5) ----------------------- */

/* The paper discretizes Eq. GeneralizedPoisson with finite elements (Sec.
 * 2.5: the system matrix is then symmetric positive definite).  Here:
 * multilinear (Q1) elements on the points x_i = i h of every axis, stored
 * like the cell grids (x fastest, 2D grids are (x, z) with n[1] = 1).  A
 * periodic axis of n points is a ring of n elements; a walled axis
 * (LM_BC_NEUMANN) has n - 1 elements and its end points on the walls, where
 * the homogeneous Neumann condition is the natural one of the weak form.
 * Element kappa_e is the harmonic mean of kappa = 1/rho over the element's
 * corners; the c~ term is mass-lumped.  The system is
 *
 *     B x = b,   B = diag(V c~) + sum_e kappa_e K_ref,
 *
 * V_i the point's share of its elements (h per axis, h/2 at a wall end;
 * lm_fe_lumped_mass), K_ref the Q1 element stiffness, b the load vector:
 * V f for a right-hand side f, plus g times the wall share of each wall
 * point for inhomogeneous Neumann data g.  The handle owns every buffer it
 * uses, including a cell-centred grid on the same points whose multigrid
 * V-cycle preconditions the mixed solve. */
typedef struct lm_fe lm_fe;

/* n[0] and n[2] >= 2 points; ndim 2: n[1] == 1; ndim 3: n[1] >= 2.  Errors:
 * LM_ERR_INVALID_ARG, LM_ERR_OUT_OF_MEMORY. */
int  lm_fe_create(int ndim, const int64_t n[3], const double h[3], const int bc[3], lm_fe** out);
void lm_fe_destroy(lm_fe* fe);

/* c~ and rho at the points (N values each; host or device per on_device,
 * read on `stream`; host buffers may be reused on return).  Forms kappa_e,
 * V c~, the inverse diagonal and their float32 copies, and the
 * preconditioner's cell-centred coefficients.  LM_ERR_NOT_POSITIVE when a
 * value is not strictly positive and finite (Sec. 2.5's conditions); the
 * handle then holds no coefficients. */
int  lm_fe_set_coefficients(lm_fe* fe, const double* ctilde, const double* rho, int on_device, void* stream);

/* As lm_fe_set_coefficients, with c~ formed on the device from the state
 * (step (v) of Sec. 2.4, Eq. cpoiss): c~ = 1 / (dt^2 rho^n c_s^2) from
 * rho_old, cs2 and dt, kappa from rho_new.  LM_ERR_NOT_POSITIVE for dt <= 0
 * or a c~ / rho that is not strictly positive and finite. */
int  lm_fe_set_state(lm_fe* fe, const double* rho_old, const double* rho_new, const double* cs2, double dt,
                     int on_device, void* stream);

/* V (N doubles, host or device per on_device). */
int  lm_fe_lumped_mass(lm_fe* fe, double* v, int on_device, void* stream);

/* b = V f, the load vector of a right-hand side f (N doubles each, host or
 * device per on_device; f and b may be the same array). */
int  lm_fe_mass_times(lm_fe* fe, const double* f, double* b, int on_device, void* stream);

/* y = B x on the device in precision prec (float64: double arrays; float32:
 * float arrays, LM_ERR_INVALID_ARG when a coefficient leaves the float32
 * range); with dot_out, also *dot_out = x^T B x (synchronises the stream).
 * x and y must not overlap.  LM_ERR_STATE before lm_fe_set_coefficients. */
int  lm_fe_apply(lm_fe* fe, int prec, const void* x, void* y, double* dot_out, void* stream);

/* Solve B x = b to ||b - B x||_2 <= opts->rtol ||b||_2 (float64 true
 * residual).  opts->mode: LM_FP64_JACOBI_PCG (float64 conjugate gradients,
 * Jacobi preconditioner) or LM_MIXED_MG_IR (float64 iterative refinement;
 * inner float32 flexible CG preconditioned by a damped Jacobi step on B, the
 * cell-centred V-cycle (opts->nu1, nu2) on the residual divided by V, and a
 * second Jacobi step; it needs an even number of points on every periodic
 * axis and float32-representable coefficients, else LM_ERR_INVALID_ARG).
 * b and x: N doubles on host or device per on_device;
 * x is the initial guess when opts->use_x0 and receives the solution (also
 * on LM_ERR_NO_CONVERGENCE / LM_ERR_BREAKDOWN).  Synchronises
 * opts->cuda_stream; res->seconds is the device time of the solve. */
int  lm_fe_solve(lm_fe* fe, const double* b, double* x, int on_device, const lm_solve_opts* opts,
                 lm_solve_result* res);

/* ---- measurement ---------------------------------------------------------- */

/* Arithmetic-rate probe of the current device, the measured roof of the
 * float64 kernels (the paper reports CPU timings only and has no
 * counterpart).  which: 0 = float64 fused multiply-adds per second, 1 =
 * float32 fused multiply-adds per second, 2 = float64 <-> float32
 * conversions per second.  One launch of `steps` steps of 8 independent
 * chains per thread, 8 blocks of 256 threads per SM, timed with CUDA events
 * on `stream` after a short warm-up launch (steps = 20000 runs for tens of
 * milliseconds in float64).  Allocates and frees 64 bytes of device memory;
 * synchronises the stream.  LM_ERR_INVALID_ARG for a bad `which`, `steps`
 * or pointer. */
int  lm_probe_rate(int which, int steps, double* ops_per_s, void* stream);

/* Allocation-free float64 apply: y = A x and *dot_out = x^T A x, like
 * lm_apply(LM_PREC_FP64) with dot_out, but with no grid object and no device
 * allocation at all.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc after start-up (a fixed device-memory budget, a
 * frozen memory pool).  The operator is given by its assembled float64
 * coefficients, laid out as lm_get_coefficients returns them (c~, and each
 * cell's minus-face conductance per axis); n, bc describe the grid as in
 * lm_grid_create (host arrays); ctilde, gx, gy, gz, x, y and dot_out are
 * device pointers (dot_out: one double), ordered on `stream`.
 * Scratch: the reduction's partial sums live in a static device array of
 * 65536 doubles (512 KiB), held by every GPU that loads the library until
 * the process exits; a call covers at most 65536 * 4096 = 268435456 cells
 * and larger grids are rejected with LM_ERR_INVALID_ARG (and a message on
 * stderr) before any device work.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make it before any
 * stream capture.  Calls share the array: calls whose kernels overlap on
 * the GPU (different streams or threads) race on it. */
int  lm_apply_dot_noalloc(int ndim, const int64_t n[3], const int bc[3], const double* ctilde,
                          const double* gx, const double* gy, const double* gz, const double* x,
                          double* y, double* dot_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LOWMACH_H */
