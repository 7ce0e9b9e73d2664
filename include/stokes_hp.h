/*
 * stokes_hp.h - C ABI of a GB300 (sm_103a) library for the hyper-power preconditioned Krylov
 * solve of the 3D Stokes saddle-point system of arXiv 2311.06926 ("Matrix-free polynomial
 * preconditioning of saddle point systems using the hyper-power method").
 *
 * Problem (Sec. 3): Stokes flow on the unit cube, n^3 uniform elements, div-conforming B-spline
 * (isogeometric Raviart-Thomas) spaces (App. B.2). With this library's degree p (the pressure
 * degree; the paper's degree is p + 1):
 *   velocity component c: degree p+1 (C^p) in direction c, degree p (C^(p-1)) in the others;
 *   pressure: degree p (C^(p-1)) in every direction.
 * Normal velocity is zero strongly (the first and last spline in direction c is removed);
 * tangential velocity is imposed weakly by Nitsche's method with alpha = C_pen / h (Sec. 3.2).
 * The discrete system (Eq. 3.3) is K [u; q] = [f; 0] with
 *   K = [[A, B], [B^T, 0]],  A_ij = a(v_j, v_i) + sigma(v_j, v_i),  B_ij = int div(v_i) q_j.
 *
 * Sizes: a = n + p - 1, b = n + p. Vector layout (every vector argument): the three velocity
 * components then the pressure, each a 3D coefficient tensor stored with x1 fastest:
 *   u1 (a, b, b), u2 (b, a, b), u3 (b, b, a), q (b, b, b)   [extents along (x1, x2, x3)]
 * n_vel = 3 a b^2, n_pres = b^3. All values are float64.
 *
 * Memory and streams: unless a name ends in _host, every vector pointer is a DEVICE pointer to
 * caller-owned memory of the stated length; the library never frees or retains it. The context
 * owns its own device workspace (allocated by stokes_setup, freed by stokes_destroy). Every call
 * is ordered on the context's stream (stokes_opts.stream, or a stream the library creates) and
 * returns after its work is enqueued, except stokes_solve / stokes_solve_host, which return when
 * the solve has finished.
 *
 * Errors: every int-returning call returns STOKES_OK (0) or a negative STOKES_ERR_* code and
 * never throws; stokes_last_error(ctx) gives a message. A context whose call failed with
 * STOKES_ERR_CUDA should be destroyed.
 */
#ifndef STOKES_HP_H
#define STOKES_HP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  STOKES_OK = 0,
  STOKES_ERR_ARG = -1,        /* invalid argument (null pointer, size, order < 2, ...) */
  STOKES_ERR_CUDA = -2,       /* a CUDA call failed */
  STOKES_ERR_NONFINITE = -3,  /* NaN or Inf met in the Krylov recurrence */
  STOKES_ERR_NOT_SPD = -4,    /* preconditioner not positive definite (<z, r> < 0) */
  STOKES_ERR_MAXIT = -5,      /* iteration cap reached; x holds the last iterate */
  STOKES_ERR_BREAKDOWN = -6,  /* Krylov breakdown */
  STOKES_ERR_SETUP = -7       /* setup failed (1D matrix not positive definite, ...) */
};

enum { STOKES_SCHUR_INNER = 0, STOKES_SCHUR_NONE = 1 };
enum { STOKES_PREC_FP64 = 0, STOKES_PREC_FP32 = 1, STOKES_PREC_TF32 = 2, STOKES_PREC_BF16 = 3 };
enum { STOKES_SOLVER_MINRES = 0, STOKES_SOLVER_FGMRES = 1 };

enum { STOKES_FORWARD_KRONECKER = 0, STOKES_FORWARD_QUADRATURE = 1 };
enum { STOKES_OUTER_FP64 = 0, STOKES_OUTER_PAIR = 1 };

typedef struct stokes_opts {
  double c_pen;       /* Nitsche penalty constant C_pen (Sec. 3.2); <= 0 selects 14 */
  int schur;          /* Q-block sequence: STOKES_SCHUR_INNER = Eq. 4.5 (with inner updates,
                         the sequence of Table 1), STOKES_SCHUR_NONE = Eq. 4.6 */
  int precision;      /* arithmetic of the preconditioner (base blocks and hyper-power
                         steps): STOKES_PREC_FP64, or FP32 / TF32 / BF16 with FP32 accumulation;
                         the outer Krylov residual, K apply and inner products are always FP64 */
  int solver;         /* STOKES_SOLVER_MINRES (needs an FP64 preconditioner) or
                         STOKES_SOLVER_FGMRES (flexible GMRES, for reduced precision) */
  int max_order;      /* largest hyper-power order used with this context (workspace); >= 2 */
  int max_steps;      /* largest hyper-power step count used with this context; >= 0 */
  int maxit;          /* Krylov iteration cap */
  int restart;        /* FGMRES restart length */
  void* stream;       /* cudaStream_t to run on; NULL: the library creates one */
  int nrhs;           /* right-hand sides held by the context (<= 1: one). With nrhs > 1 every
                         vector argument of stokes_apply_K, stokes_apply_P,
                         stokes_apply_hyperpower and stokes_solve_multi holds nrhs items of
                         n_vel + n_pres entries one after the other, and each kernel of those
                         calls processes all items in one launch (the mode products of the fast
                         diagonalisation become GEMMs with nrhs times the rows). Needs
                         precision TF32 or BF16 and solver FGMRES. */
  int autotune;       /* nonzero (default): time the candidate launch shapes of the FP64 kernels
                         at setup and keep the fastest (stokes_get_tuning); results do not depend
                         on the choice. 0: fixed defaults. */
  int forward;        /* forward operator of stokes_apply_K and of the solvers:
                         STOKES_FORWARD_KRONECKER (default; banded Kronecker products, Sec. 3.3)
                         or STOKES_FORWARD_QUADRATURE (matrix-free formation by global sum
                         factorisation on the Gauss grid of p + 2 points per element and
                         direction, the forward operator of the paper's timings, Sec. 5.3; equal
                         to the Kronecker operator up to rounding; nrhs = 1 only).
                         stokes_apply_A always uses the Kronecker form. */
  int outer;          /* arithmetic of the products w = K z of flexible GMRES when the
                         preconditioner runs in reduced precision (z is then its FP32 output):
                         STOKES_OUTER_FP64 (default) or STOKES_OUTER_PAIR (every value carried as
                         an unevaluated sum of two FP32 numbers, about 48 significant bits, w
                         rounded to FP64; on this GPU's reduced FP64 pipe about twice as fast).
                         Residuals of the iterate (restarts, the final true residual),
                         stokes_apply_K and every FP64-preconditioned solve use the FP64
                         operator either way. Used with the Kronecker forward operator when
                         n_elems + degree_p <= 256 and every band has half width <= 6; the FP64
                         operator otherwise. */
} stokes_opts;

typedef struct stokes_ctx* stokes_t;

/* Fill *o with the defaults: c_pen 14, Schur with inner updates, FP64, MINRES, max_order 3,
 * max_steps 4, maxit 2000, restart 60, stream NULL, nrhs 1, autotune on, Kronecker forward
 * operator, FP64 Arnoldi products. */
void stokes_default_opts(stokes_opts* o);

/* Build the univariate matrices (App. B.3, T-check of Sec. 3.3), the fast-diagonalisation
 * factors (generalised eigenpairs, App. A.4) and the device workspace for n_elems^3 elements,
 * degree_p >= 1 (pressure degree), viscosity nu > 0. opts may be NULL (defaults). On success
 * *out receives a new context. Errors: STOKES_ERR_ARG, STOKES_ERR_SETUP, STOKES_ERR_CUDA. */
int stokes_setup(stokes_t* out, int n_elems, int degree_p, double nu, const stokes_opts* opts);

/* n_vel = 3 a b^2 and n_pres = b^3 (either pointer may be NULL). */
int stokes_sizes(stokes_t ctx, int64_t* n_vel, int64_t* n_pres);

/* Select the preconditioner used by stokes_solve: the order-`order` hyper-power sequence after
 * `steps` steps (Eq. 2.1 for order 2; steps = 0 is the base P_0). Requires 2 <= order <=
 * max_order and 0 <= steps <= max_steps. */
int stokes_set_preconditioner(stokes_t ctx, int order, int steps);

/* y = A x on the velocity block (x, y: n_vel). A = the 15 Kronecker products of Sec. 3.3 with
 * the weak-form scaling (2 nu on the printed diagonal blocks, nu on the off-diagonal ones).
 * One item, also on a context with nrhs > 1 (as stokes_apply_mass, the stokes_rhs_* loads and
 * stokes_dot). */
int stokes_apply_A(stokes_t ctx, const double* x, double* y);

/* y = K x on the full saddle-point system (Eq. 3.3; x, y: n_vel + n_pres). */
int stokes_apply_K(stokes_t ctx, const double* x, double* y);

/* y = P_0^-1 x, the base block preconditioner (Eq. 4.1): fast diagonalisation of the three
 * diagonal blocks of A (Sec. 4, App. A.4) and the pressure mass block M-check^3 / (2 nu)
 * (Sec. 4). Runs in the context's preconditioner precision. x, y: n_vel + n_pres. */
int stokes_apply_P(stokes_t ctx, const double* x, double* y);

/* y = K x for an FP32 vector x (nrhs items), in the arithmetic of the context's Arnoldi products
 * (stokes_opts.outer): pairs of FP32 numbers rounded to FP64, or the FP64 operator applied to x
 * converted exactly to FP64. x: device FP32 (n_vel + n_pres entries per item, the layout of the
 * FP64 vectors); y: device FP64. Needs a reduced-precision context (STOKES_ERR_ARG otherwise).
 * Returns STOKES_OK or a negative code. */
int stokes_apply_K_f32(stokes_t ctx, const float* x, double* y);

/* y = P_s^-1 x for the order-q hyper-power sequence (Eqs. 2.1, 4.4 for the velocity block,
 * 4.5 or 4.6 for the pressure block) with q = order, s = steps; steps = 0 equals
 * stokes_apply_P. One application costs q^s base applications and q^s - 1 applications of the
 * approximation (Eq. 4.8). */
int stokes_apply_hyperpower(stokes_t ctx, int order, int steps, const double* x, double* y);

/* f = load of the lid-driven cavity (Sec. 5, Fig. 2): tangential lid velocity (lid_speed, 0, 0)
 * on the face x2 = 1 through the Nitsche terms, no slip elsewhere, no body force.
 * f: n_vel + n_pres (pressure part zero). */
int stokes_rhs_cavity(stokes_t ctx, double lid_speed, double* f);

/* f = load int b . v of the body force b_c(x) = sum_m coef[c*n_modes+m] prod_d
 * sin(waves[(c*n_modes+m)*3+d] pi x_d) (Sec. 3.1, l(v)). coef and waves are HOST arrays of
 * 3*n_modes and 9*n_modes entries (wave numbers >= 1). If accumulate != 0 the load is added to f. */
int stokes_rhs_body(stokes_t ctx, int n_modes, const double* coef, const int* waves,
                    int accumulate, double* f);

/* f = Nitsche load (Sec. 3.1, sigma with boundary data; the cavity lid of Sec. 5 generalised to
 * a profile) of a lid velocity (g(x1), 0, 0) on the face x2 = 1 with g = sum_k theta[k] S_k, S_k
 * the ncoef >= 4 cubic B-splines of an open uniform knot vector on [0, 1]. theta: HOST array of
 * ncoef entries. theta = (U, ..., U) gives stokes_rhs_cavity(U). If accumulate != 0 the load is
 * added to f. f: device, n_vel + n_pres. */
int stokes_rhs_lid_profile(stokes_t ctx, int ncoef, const double* theta, int accumulate,
                           double* f);

/* y = M_V x, the L2 Gram (mass) matrix of the velocity basis (App. B.3 mass matrices, one
 * Kronecker product per component). x, y: device, n_vel. */
int stokes_apply_mass(stokes_t ctx, const double* x, double* y);

/* *result (HOST) = <x, y> over n float64 entries of device vectors, by the deterministic
 * fixed-order reduction of the solver. Synchronizes the context's stream. */
int stokes_dot(stokes_t ctx, const double* x, const double* y, int64_t n, double* result);

/* Inner products of x with the unit loads of the two load families, without forming them (each
 * is separable: the device contracts x with the outer product of its three 1D factors); they are
 * the gradient of lambda^T f with respect to the load coefficients (adjoint, Sec. 3.1 loads).
 * stokes_body_load_dots: out[c n_modes + m] = x_c . (load of mode (c, m) of stokes_rhs_body with
 * coefficient 1), waves as there; out: host, 3 n_modes.
 * stokes_lid_profile_dots: out[k] = x . (stokes_rhs_lid_profile with theta = e_k), k < ncoef;
 * out: host, ncoef.
 * x: device, n_vel + n_pres (the velocity part is read). Deterministic. One item. */
int stokes_body_load_dots(stokes_t ctx, int n_modes, const int* waves, const double* x,
                          double* out);
int stokes_lid_profile_dots(stokes_t ctx, int ncoef, const double* x, double* out);

/* Solve K x = rhs with the selected preconditioner and solver to relative tolerance tol
 * (MINRES: ||r||_{P^-1} / ||rhs||_{P^-1}; FGMRES: ||r||_2 / ||rhs||_2), starting from x = 0,
 * then shift the pressure to zero mean. iterations and final_rel_res (the true
 * ||rhs - K x||_2 / ||rhs||_2) may be NULL. rhs, x: device, n_vel + n_pres.
 * Returns STOKES_OK, or STOKES_ERR_MAXIT / _NONFINITE / _NOT_SPD / _BREAKDOWN with x holding the
 * last iterate. */
int stokes_solve(stokes_t ctx, const double* rhs, double tol, double* x, int* iterations,
                 double* final_rel_res);

/* Solve all nrhs systems of a context (stokes_opts.nrhs): rhs and x hold nrhs items of
 * n_vel + n_pres entries one after the other (device). Flexible GMRES runs for all items in
 * lockstep: one Arnoldi step applies the preconditioner and K to every item in the same launches,
 * while each item keeps its own Krylov basis, Hessenberg matrix, restarts and stopping test, so its
 * result and iteration count equal those of a context with nrhs = 1 for that item alone.
 * iterations, final_rel_res and status (per-item return codes) are HOST arrays of nrhs entries and
 * may be NULL. Returns STOKES_OK or the first nonzero per-item code. (stokes_solve on such a
 * context solves all items and reports the largest iteration count and residual.) */
int stokes_solve_multi(stokes_t ctx, const double* rhs, double tol, double* x, int* iterations,
                       double* final_rel_res, int* status);

/* As stokes_solve with HOST buffers rhs_host and x_host (pinned memory gives full copy speed):
 * the host-to-device copy, the solve and the device-to-host copy all happen inside the call.
 * Contexts with nrhs = 1 only (STOKES_ERR_ARG otherwise). */
int stokes_solve_host(stokes_t ctx, const double* rhs_host, double tol, double* x_host,
                      int* iterations, double* final_rel_res);

/* Solve `count` independent systems at once: ctxs[i] (distinct contexts, any meshes, degrees,
 * precisions and solvers) with rhs[i] -> x[i] (device pointers of that context's size). Each
 * solve runs on its own context's stream, driven by its own host thread, so the solves execute
 * concurrently on the GPU. A context with nrhs > 1 solves all its items (as stokes_solve, with
 * the largest iteration count and residual reported). iterations, final_rel_res and status
 * (per-context return codes) may be NULL. Returns STOKES_OK or the first nonzero code. */
int stokes_solve_batch(stokes_t* ctxs, int count, const double* const* rhs, double tol,
                       double* const* x, int* iterations, double* final_rel_res, int* status);

/* Per-iteration convergence ratios of the last solve: copies min(capacity, iterations) values
 * into the host array ratios and returns the number copied (or a negative error). */
int stokes_last_ratios(stokes_t ctx, double* ratios, int capacity);

/* ---- instrumentation (no counterpart in the paper) ------------------------------------------
 * Kernel classes: 0 banded Kronecker passes in FP32, 1 dense mode products on CUDA cores,
 * 2 discrete divergence / transpose, 3 Krylov vector kernels, 4 tensor-core mode products,
 * 5 banded Cholesky line solves, 6 banded Kronecker passes in FP64, 7 the saddle-point operator
 * in pair-of-FP32 arithmetic (its banded passes and fused divergence).
 * stokes_profile_begin brackets every later launch of this thread with CUDA events on the
 * launching stream; stokes_profile_end synchronizes, writes per-class totals (launches, summed
 * event intervals in ms, algorithmic flops and bytes: each input read once, each output written
 * once) into out[0 .. capacity) and returns the number of classes written. The events add a
 * little time per launch, so profiled runs are not used as throughput numbers. */
typedef struct stokes_kernel_stat {
  int kernel_class;
  int64_t launches;
  double ms;
  double flops;
  double bytes;
} stokes_kernel_stat;
int stokes_profile_begin(stokes_t ctx);
int stokes_profile_end(stokes_t ctx, stokes_kernel_stat* out, int capacity);
/* Number of kernels this library has launched in this process (all contexts and threads). Kernels
 * of a captured CUDA graph are counted each time the graph is replayed, not when it is captured. */
int64_t stokes_kernel_launches(void);

/* Launch shapes of the FP64 kernels, chosen at setup by timing when stokes_opts.autotune is set,
 * otherwise {512, 256, 0, 1}:
 *   mode_block: threads per block of the fast-diagonalisation mode products (128, 256 or 512);
 *   band_block: threads per block of the banded passes (128, 256 or 512);
 *   fd_fused:   how the fast diagonalisation (App. A.4) is launched: 0 = six single-direction
 *               mode products; 1, 2 or 4 = three fused launches (the x1 and x2 products of each
 *               x1-x2 plane in one cluster of fd_fused blocks sharing the plane through
 *               distributed shared memory, the forward x3 product, eigenvalue scaling and
 *               backward x3 product of each line group in one block, then the x2 and x1
 *               products per plane); fused forms need every plane to fit in shared memory
 *               (2 x n1 x n2 doubles <= 200 KiB, meshes up to about 110 elements per direction).
 *   tc_nsplit:  tile shape of the tensor-core mode products (TF32/BF16 contexts): the N columns
 *               of each 128-row tile computed as one work unit (1) or as two units of at most
 *               half the columns each (2; more units where a launch has few tiles); the tuner
 *               times both on the context's fast diagonalisation; default 1.
 * Every output is computed by one thread in a fixed order whatever the choice (and each output
 * column by the same tensor-core operations), so results do not depend on it. stokes_set_tuning
 * rejects other values, and a fused form on a mesh whose planes do not fit, with STOKES_ERR_ARG
 * (the context keeps its shapes). */
typedef struct stokes_tuning {
  int mode_block;
  int band_block;
  int fd_fused;
  int tc_nsplit;
} stokes_tuning;
int stokes_get_tuning(stokes_t ctx, stokes_tuning* out);
int stokes_set_tuning(stokes_t ctx, const stokes_tuning* tuning);

/* Test hook (no counterpart in the paper): the number of polls each pipeline wait of the
 * tensor-core mode products (mbarrier waits on TMA copies, MMA completion and the epilogue) makes
 * before it gives up; 0 restores the default (2^22 polls, at least 128 ns apart after the first
 * 64: about half a second). A wait that gives up raises the context's error flag, the kernel
 * stops issuing work, waits (with the default limit) for the copies and tensor-core operations it
 * has in flight, frees its tensor memory and returns; the call then fails with STOKES_ERR_CUDA
 * ("tensor-core pipeline wait timed out") and the context should be destroyed. A tiny limit makes
 * the waits run out on purpose, so that this path can be tested without a fault or a hang. Applies
 * to launches made after the call (CUDA graphs the solvers captured earlier keep their limit);
 * contexts without tensor-core mode products ignore it. */
int stokes_set_wait_limit(stokes_t ctx, int64_t polls);

/* ---- allocation-free variant (no counterpart in the paper) --------------------------------
 * For callers that cannot allocate device memory (their allocator is owned by a framework or
 * memory pool, or allocation is forbidden after start-up): the fast-diagonalisation apply of one
 * Kronecker-sum block without a context and without any device allocation,
 *   y = (U3 (x) U2 (x) U1) diag(1 / (scale (lam1[i1] + lam2[i2] + lam3[i3]))) (U3 (x) U2 (x) U1)^T x,
 * on a tensor of extents (n1, n2, n3), x1 fastest. U_k: device, row-major n_k x n_k with the
 * eigenvectors as columns; lam_k: device, n_k entries; x, y: device, n1 n2 n3 entries, not
 * aliased. stream: a cudaStream_t (NULL = legacy default stream). Returns after enqueueing.
 * Its two intermediate tensors live in a static device array of 2 x 2^19 float64 (8 MiB), held
 * by every GPU that loads the library until the process exits; n1 n2 n3 > 2^19 is rejected with
 * STOKES_ERR_ARG. Each of the six mode products stages its contracted lines in shared memory, so
 * an extent must also fit the device's opt-in shared memory per block: with 227 KiB, n1 <= 7264
 * and n2, n3 <= 14528 (7264 when every extent before it is 1); a call beyond that is rejected
 * with STOKES_ERR_ARG before anything is launched. A launch that fails stops the sequence and
 * returns STOKES_ERR_CUDA (y is then incomplete); errors left pending by unrelated earlier work
 * are neither reported nor cleared. The first call on a device (made with that device current) looks up the
 * array's device address; make it before any stream capture. All calls share the array: calls
 * that overlap on the GPU race, so serialise them. No part of the array needs to start at zero. */
int stokes_fd_apply_noalloc(int n1, int n2, int n3, const double* U1, const double* U2,
                            const double* U3, const double* lam1, const double* lam2,
                            const double* lam3, double scale, const double* x, double* y,
                            void* stream);

/* Release the context and its device workspace. NULL is ignored. */
void stokes_destroy(stokes_t ctx);

/* Message of the last error on ctx ("" if none); ctx may be NULL (setup errors). The string
 * stays valid until the next call on ctx. */
const char* stokes_last_error(stokes_t ctx);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_HP_H */
