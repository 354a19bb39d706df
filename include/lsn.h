/*
 * lsn.h - C ABI of the GB300 (sm_103a) neural-subspace reduced-order solver.
 *
 * The library solves, on one GPU, the reduced implicit-Euler problem of
 * Eq. 2 (Sec. 3.1):
 *
 *   z^{k+1} = argmin_z E(z),
 *   E(z)    = 1/(2 dt^2) ||x(z) - qbar||_M^2 + sum_{e in S} w_e P_e(x(z))
 *
 * (quasi-static when dt = 0: the inertia term is dropped and gravity acts as
 * the potential -sum_v m_v g . x_v), where x(z) = X0 + s f_theta(z) is an MLP
 * decoder (the neural subspace map of Sec. 3.1), P_e the Stable Neo-Hookean
 * energy of tet e (Sec. 5.1) and S a cubature set with weights w_e (Eq. 11;
 * S = all tets, w = 1 by default).  Each Newton iteration of the projective
 * Newton solver (Supplement, "Tests with Projective Newton's method") runs
 * hand-written CUDA kernels: decoder + forward-mode Jacobian J = dx/dz, a
 * per-tet energy / gradient / PSD-projected Hessian kernel fused with the
 * J_e^T H_e J_e contraction, an FP64 r x r Cholesky, and an Armijo
 * backtracking line search whose energy comparison is done in FP64.
 *
 * Conventions
 * -----------
 *  - Every call returns an int status.  Negative values are errors and leave
 *    the context unchanged (except that the stream may hold finished work);
 *    positive values from lsn_step mean the solve ended without meeting the
 *    tolerance but produced a usable result.  lsn_last_error() describes the
 *    last error.  No exception crosses the ABI.
 *  - The library owns the context, its device buffers and the simulation
 *    state (q, v, z).  The caller owns every array it passes; the library
 *    copies what it keeps.
 *  - Pointers marked "host or device" may point to host memory (pageable or
 *    pinned) or to device memory of the context's GPU; the library detects
 *    which.  All other pointers are host pointers.
 *  - All work is issued on the context's CUDA stream (given at creation; NULL
 *    means the default stream).  Calls that return data synchronise that
 *    stream before returning.
 *  - Vertex data is xyz-interleaved: entry 3*v + c.  Matrices are row-major.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef LSN_H
#define LSN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsn_ctx lsn_ctx; /* opaque, owned by the library */

enum lsn_status {
  LSN_OK = 0,              /* solve converged: ||g||_inf < tol                */
  LSN_NOT_CONVERGED = 1,   /* Newton iteration cap reached                     */
  LSN_LS_FAILED = 2,       /* line search found no Armijo step in max_ls trials */
  LSN_NOT_SPD = 3,         /* reduced Hessian not positive definite after the
                              diagonal-shift retries                          */
  LSN_PRECISION_FLOOR = 4, /* line search stalled at the rounding level of the
                              chosen precision while ||g||_inf < 100 tol (FP32
                              and tensor-core forms: also after 4 iterations
                              without a 10 % drop of ||g||_inf whose accepted
                              steps were all shorter than 2^-10)              */
  LSN_SADDLE = 5,          /* L-BFGS: no positive curvature along the accepted
                              step (s^T y <= 0; exit II of Sec. 5)             */
  LSN_ERR_ARG = -1,        /* invalid argument or size                         */
  LSN_ERR_CUDA = -2,       /* CUDA runtime error                               */
  LSN_ERR_NONFINITE = -3,  /* NaN / Inf in inputs or in the reduced system     */
  LSN_ERR_STATE = -4,      /* call out of order (e.g. step before set_mesh)    */
  LSN_ERR_OOM = -5         /* device allocation failed                         */
};

/* Arithmetic of the decoder, Jacobian and J_e^T H_e J_e contraction.  The
 * r x r Cholesky and the line-search energy comparison are FP64 in every
 * mode; energies, gradients and partial sums are accumulated in FP64 (or, in
 * the tensor-core kernels, in double-float FP32 pairs summed in FP64).
 *
 * Tensor-core forms (tcgen05, FP32 accumulation in TMEM): the decoder output
 * layer + Jacobian, the inertia Hessian J^T M J / dt^2 and the element
 * contraction sum_e w_e J_e^T Hproj_e J_e.  Hidden layers, per-element
 * energies, stresses, PSD projection and the gradient stay FP32.
 *   TF32: W_L and the hidden activations rounded to TF32; Gram operands TF32.
 *   BF16: W_L stored in BF16 (rounded once, at lsn_set_decoder time), the
 *         activations entered as a two-term BF16 split (so only W_L is
 *         rounded), Gram operands BF16.  The rounding of W_L changes the model
 *         by about 1e-3 relative; the form agrees with the FP64 evaluation of
 *         its own BF16 weights to FP32 accuracy.
 * The tensor-core output layer needs the last hidden width times the element
 * size (2 / 4 bytes) to be a multiple of 16 bytes; otherwise the FP32
 * CUDA-core output layer is used with the FP32 weights. */
enum lsn_precision {
  LSN_PREC_FP64 = 0, /* everything in FP64                                 */
  LSN_PREC_FP32 = 1, /* plain FP32 on CUDA cores                           */
  LSN_PREC_TF32 = 2, /* tensor-core form, TF32 operands (see above)        */
  LSN_PREC_BF16 = 3  /* tensor-core form, BF16 weights (see above)         */
};

typedef struct {
  int newton_iters; /* Newton updates taken                                */
  int ls_trials;    /* energy evaluations in the line searches             */
  int exit;         /* lsn_status of the solve (>= 0)                      */
  double grad_inf;  /* ||g||_inf at exit                                   */
  double energy;    /* E(z) at exit                                        */
  double ms;        /* wall time of the call (host clock)                  */
} lsn_stats;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = default stream). */
int lsn_create(lsn_ctx** out, int device, void* cuda_stream);
void lsn_destroy(lsn_ctx* ctx);
const char* lsn_last_error(const lsn_ctx* ctx);

/* Tet mesh (Sec. 3.1: the DOF vector q in R^n, n = 3 nv, holds vertex
 * positions).  X0: nv x 3 rest positions; tets: ne x 4 vertex indices, each
 * tet with positive rest orientation det[X1-X0, X2-X0, X3-X0] > 0 (rejected
 * with LSN_ERR_ARG otherwise).  Rest-shape inverses, volumes and the lumped
 * mass (m_v = sum rho V_e / 4) are computed on the GPU.  Resets cubature to
 * all tets and clears constraints. */
int lsn_set_mesh(lsn_ctx* ctx, const double* X0, int nv, const int32_t* tets,
                 int ne);

/* Stable Neo-Hookean material (Sec. 5.1): Lame parameters from Young's
 * modulus and Poisson ratio, density rho, gravity vector g (3 doubles).
 * Must follow lsn_set_mesh (the lumped mass depends on both). */
int lsn_set_material(lsn_ctx* ctx, double youngs, double poisson,
                     double density, const double* gravity);

/* Positional constraints (Sec. 5.1 "positional / moving constraints"): the
 * nc vertices vidx are held at targets (nc x 3, host or device).  Their rows
 * of x are overwritten by the targets and their rows of J are zero.  Calling
 * again with the same vidx and new targets is the per-frame update; vidx ==
 * NULL keeps the current vertex set and only uploads targets. */
int lsn_set_constraints(lsn_ctx* ctx, const int32_t* vidx, int nc,
                        const double* targets);

/* Cubature set S with non-negative weights (Eq. 11).  s == 0 selects every
 * tet with weight 1. */
int lsn_set_cubature(lsn_ctx* ctx, const int32_t* tet_idx, const double* w,
                     int s);

/* Ground plane z = height with penalty energy k/2 sum_v min(0, x_v,z - h)^2
 * (the energy-based contact of Sec. 5.2, as a plane).  stiffness 0 = off. */
int lsn_set_ground(lsn_ctx* ctx, double height, double stiffness);

/* MLP decoder (Sec. 3.1): widths[0] = r, widths[nlayers] = n; W[l] is
 * widths[l+1] x widths[l] row-major, b[l] has widths[l+1] entries (host
 * pointers).  Hidden layers use ELU; the last layer is linear; positions are
 * x = X0 + out_scale * out.  1 <= r <= 64.  `precision` is an lsn_precision. */
int lsn_set_decoder(lsn_ctx* ctx, int nlayers, const int* widths,
                    const float* const* W, const float* const* b,
                    double out_scale, int precision);

/* Affine modes (optional; off by default): 12 coordinates appended to z,
 * z = (z_nn, M row-major (9), t (3)), with
 *   x(z) = X0 + out_scale * (f(z_nn) + Phi z_aff),
 *   i.e. u_v += out_scale * (M (X0_v - center) + t),
 * a linear map in parallel with the network (inside the same output scale,
 * so that one gradient tolerance suits both kinds of coordinate), so that a
 * free body can translate and (to first order) rotate.  The columns of J
 * for these coordinates are the constant out_scale * Phi; constrained DOFs
 * still follow their targets.  Every z array of the ABI then has widths[0] + 12 entries (at
 * most 64).  Call after lsn_set_decoder; enable = 0 turns them off; center
 * (3 doubles, host) is ignored then.  Decoder training (lsn_train_*) uses
 * the network alone. */
int lsn_set_affine_modes(lsn_ctx* ctx, int enable, const double* center);

/* Newton controls: exit when ||g||_inf < tol_inf (Supplement, convergence
 * condition), at most max_newton iterations (Sec. 5: 1024) and max_ls line
 * search trials per iteration (Sec. 5: 128), Armijo constant armijo_c.
 * Defaults of a new context: tol_inf = 1e-5, max_newton = 1024,
 * max_ls = 128, armijo_c = 1e-4. */
int lsn_set_solver(lsn_ctx* ctx, double tol_inf, int max_newton, int max_ls,
                   double armijo_c);

/* Optimiser of the solves (Sec. 5 and the Supplement's projective Newton
 * tests).  Both share the evaluation passes, the Armijo backtracking line
 * search, the tolerance and the caps of lsn_set_solver (max_newton caps the
 * iterations of either).
 *   LSN_OPT_NEWTON (default): projective Newton, d = -K^-1 g with the
 *     Gauss-Newton reduced Hessian K (FP64 Cholesky, in its square-root-free
 *     L D L^T form).
 *   LSN_OPT_LBFGS: L-BFGS, d = -H g by the two-loop recursion over the
 *     `history` (1..32) most recent curvature pairs s = alpha d,
 *     y = g(z + s) - g(z), initial matrix (s^T y / y^T y) I of the newest
 *     pair (identity while the history is empty).  Its passes evaluate E and
 *     g only (no per-element Hessian, eigen-decomposition or K).  Exits:
 *     LSN_OK (I), LSN_SADDLE (II: s^T y <= 0 at a gradient above tol),
 *     LSN_LS_FAILED (III), LSN_NOT_CONVERGED (IV), as well as
 *     LSN_PRECISION_FLOOR in the FP32 / tensor-core forms.  A direction
 *     with g.d >= 0 in rounding restarts from -g with an empty history.
 * The history is cleared at the start of every solve.  Takes effect at the
 * next call that evaluates (the device engine is rebuilt). */
enum lsn_optimizer { LSN_OPT_NEWTON = 0, LSN_OPT_LBFGS = 1 };
int lsn_set_optimizer(lsn_ctx* ctx, int kind, int history);

/* Exact-form reduced Hessian for projective Newton (opt-in; off by default).
 * The Gauss-Newton K of Eq. 2's reduced solve drops the decoder's curvature;
 * with enable != 0 every evaluation pass adds it back over the free DOFs,
 *   K_x = K + sum_{k free} dE/dx_k d2x_k/dz2
 *       = K + s sum_j (W_L^T G)_j d2h_j/dz2   (G = dE/dx, 0 on constrained
 *         DOFs; h the last hidden layer; x = X0 + s (W_L h + b_L)),
 * with the second derivatives of h carried forward through the hidden layers
 * (ELU' and ELU''), and then projects the r x r sum: its eigenvalues below
 * clamp * max |eigenvalue| are raised to that value (cyclic Jacobi in FP64).
 * The affine coordinates (lsn_set_affine_modes) add no curvature.  The
 * element Hessians stay PSD-projected; lsn_eval's K is then K_x.  Used by
 * LSN_OPT_NEWTON only.  0 <= clamp < 1 (else LSN_ERR_ARG).  Takes effect at
 * the next call that evaluates (the device engine is rebuilt).  Device
 * memory: 12 S + n values of the element precision and three
 * (max hidden width) x (1 + r + r (r + 1) / 2) buffers. */
int lsn_set_exact_hessian(lsn_ctx* ctx, int enable, double clamp);

/* Failure detection without a GPU fault: every mbarrier wait of the tensor-
 * core kernels gives up after a wall-clock limit (2 s), records an error code
 * in a device flag and lets its CTA stop issuing work; the solve then returns
 * LSN_ERR_CUDA.  This call runs that wait once on an mbarrier that nothing
 * arrives on (no bulk copy or MMA is in flight), with a limit of `seconds`
 * (0 < seconds <= 10, else LSN_ERR_ARG), and writes the recorded code (1) to
 * *code (host).  The context stays usable. */
int lsn_selftest_bounded_wait(lsn_ctx* ctx, double seconds, int* code);

/* Execution of a solve: mode 0 (default) launches the whole Newton loop as
 * one CUDA graph whose conditional WHILE node repeats an evaluation pass
 * until the device-side solver stops it; mode 1 drives the same kernels from
 * the host with one stream synchronisation per pass (used when kernel events
 * are recorded, see lsn_set_profiling, which also selects mode 1 while an
 * event mask is set). */
int lsn_set_execution(lsn_ctx* ctx, int mode);

/* Simulation state.  z (r, host or device) is the subspace coordinate;
 * q, v (n, host or device) the full-space positions and velocities used by
 * the inertial guess.  q == NULL sets q = x(z); v == NULL sets v = 0. */
int lsn_set_state(lsn_ctx* ctx, const double* z, const double* q,
                  const double* v);

/* One time step: with dt > 0 an implicit-Euler step (Eq. 2) with inertial
 * guess qbar = q + dt v + dt^2 g; with dt == 0 a quasi-static solve.  Starts
 * Newton at z_in (r, host or device; NULL = current z), writes the solution
 * to z_out (r, host or device; may be NULL), then updates q = x(z*),
 * v = (x(z*) - q_old) / dt.  Returns the exit status (>= 0) or an error. */
int lsn_step(lsn_ctx* ctx, const double* z_in, double dt, double* z_out,
             lsn_stats* stats);

/* Copy the current state: z (r), q and v (n each) to host or device pointers
 * (any may be NULL).  With lsn_set_state this snapshots and restores a
 * simulation. */
int lsn_get_state(lsn_ctx* ctx, double* z, double* q, double* v);

/* Copy the current positions q (n doubles) to x_out (host or device). */
int lsn_get_positions(lsn_ctx* ctx, double* x_out);

/* Parity hook: evaluate at z (r, host or device; becomes the current z) the
 * reduced energy E, the
 * reduced gradient g (r) and the Gauss-Newton reduced Hessian K (r x r,
 * row-major) for the current dynamics setting (dt, qbar from the last
 * lsn_step or lsn_set_dynamics).  Outputs are host pointers; any may be NULL.
 * With LSN_OPT_LBFGS selected and K == NULL, E and g come from the
 * gradient-only pass that the L-BFGS solve uses. */
int lsn_eval(lsn_ctx* ctx, const double* z, double* E, double* g, double* K);

/* Optimised cubature (Sec. 4.3: the cubature set and weights are fitted on
 * the initial subspace, after von Tycowicz et al. 2013; Sec. 5.3 discusses
 * the cubature count).  At the K subspace points z (K x r, host or device;
 * r includes the affine modes) every tet e of the mesh gives the r reduced
 * elastic forces a_{k,e} = J_e(z_k)^T d(V_e Psi(F_e))/dx_e (unit weight;
 * constrained rows of J are zero).
 *
 * lsn_tet_forces: the matrix A ((K r) x ne, row k r + i, column e,
 * row-major FP64; host or device) of these forces (parity hook).
 *
 * lsn_select_cubature: each snapshot's r rows of A and of the full force
 * b = A 1 are divided by ||b_k||; the non-negative least-squares fit
 * min ||A w - b||, w >= 0, by the Lawson-Hanson active-set method (the
 * column with the largest entry of A^T (b - A w) enters the active set per
 * outer iteration), stopped once S columns are active.  Writes the active
 * tets in ascending order to idx, their weights to w (host, room for S
 * each), their number to *count (<= S) and ||A w - b|| / ||b|| to
 * *rel_residual (may be NULL).  The result feeds lsn_set_cubature or the
 * training cubature of lsn_train_init.  The solver's current z is kept.
 * Device memory: K r ne doubles for A. */
int lsn_tet_forces(lsn_ctx* ctx, const double* z, int K, double* A);
int lsn_select_cubature(lsn_ctx* ctx, const double* z, int K, int S, int32_t* idx, double* w,
                        int* count, double* rel_residual);

/* Full-space solve (the comparison for the reduced solve; Sec. 3.1, Eq. 1
 * minimised over all n DOFs, every tet at unit weight).  The method is
 * projective Newton: per-tet PSD projection of d2Psi/dF2, the same as in the
 * reduced solve.  It uses the same Armijo backtracking, the tolerance and
 * caps of lsn_set_solver, and the same exit codes.  Constrained DOFs are
 * held at their lsn_set_constraints targets.  The ground penalty is not part
 * of this solve: with a ground set, lsn_fullspace_step returns
 * LSN_ERR_STATE.
 *
 * Newton directions solve the projected Hessian (+ M / dt^2) system on the
 * free DOFs by Jacobi-preconditioned conjugate gradients, stopped at
 * |r| <= cg_rtol |r_0| or after max_cg iterations (rounded up to a multiple
 * of 16).  The Hessian is applied matrix-free per tet.  A breakdown
 * (non-positive curvature) ends the solve with LSN_NOT_SPD.  With FP32
 * element math, the line search accepts an energy rise within the rounding
 * of the element sums.  With FP32 element math, LSN_PRECISION_FLOOR is
 * returned in three cases.  (1) ||g||_inf has gone 4 iterations without a
 * 10 % drop while below 100 tol or within 64 u max_i sum |element
 * contributions to g_i|.  (2) ||g||_inf has gone 16 iterations without such
 * a drop.  (3) The line search failed at such a gradient.
 *
 * lsn_fullspace_setup: allocates the solver, discarding any previous one.
 * Requires lsn_set_mesh and lsn_set_material.  precision is LSN_PREC_FP64 or
 * LSN_PREC_FP32 (element math; vectors and sums are FP64); 0 <= cg_rtol < 1;
 * max_cg >= 1.  The solver keeps its own full state, independent of the
 * reduced solve's, starting at q = X0, v = 0.  Device memory: 13 n doubles,
 * n + 43 ne values of the element precision and 16 ne bytes of tet indices.
 * lsn_fullspace_set_state: q, v (n each, host or device; NULL: X0 and 0).
 * lsn_fullspace_step: one implicit-Euler step (dt > 0: q_bar = q + dt v +
 * dt^2 g, then v = (q' - q) / dt) or quasi-static solve (dt == 0, gravity as
 * the potential -sum m g.x).  Writes q' to q_out (n, host or device; may be
 * NULL), stats (may be NULL; energy is the full-space objective at q'), and
 * the total number of CG iterations to cg_iters (may be NULL).  Returns the
 * exit status (>= 0) or an error. */
int lsn_fullspace_setup(lsn_ctx* ctx, int precision, double cg_rtol, int max_cg);
int lsn_fullspace_set_state(lsn_ctx* ctx, const double* q, const double* v);
int lsn_fullspace_step(lsn_ctx* ctx, double dt, double* q_out, lsn_stats* stats,
                       long long* cg_iters);

/* Parity hook for the inertia term: sets dt and qbar (n, host or device)
 * directly, as lsn_step would. dt == 0 selects the quasi-static objective. */
int lsn_set_dynamics(lsn_ctx* ctx, double dt, const double* qbar);

/* Parity hook for the decoder (z becomes the current z): x(z) (n doubles) and
 * J(z) (n x r doubles,
 * row-major), with constraints applied, copied to host pointers x_out and
 * J_out (either may be NULL). */
int lsn_decode(lsn_ctx* ctx, const double* z, double* x_out, double* J_out);

/* History of the last lsn_step: for Newton iteration k < count (at most
 * `max` and at most 128 entries) the entry k of each non-NULL host array
 * receives ||g||_inf, E (without the quasi-static constant), the rounding
 * scale max_i sum |contributions to g_i| and the accepted step length (0 for
 * the final, exiting evaluation). */
int lsn_get_trace(lsn_ctx* ctx, int max, double* grad_inf, double* energy,
                  double* grad_scale, double* alpha, int* count);

/* ---------------------------------------------------------------------------
 * Decoder training with the Lipschitz loss (Sec. 4), on the GPU, with
 * hand-written forward and backward kernels (FP32, FP64 loss sums):
 *   L_C  = 1/B sum_b ||x(g(q_b)) - q_b||_M^2                       (Eq. 3)
 *   L_LS = 1/(B(B-1)) sum_{i != j} ||Ht_i - Ht_j||_F^2 / ||z_i - z_j||^2  (Eq. 9)
 *   L    = L_C + lambda_LS L_LS                                     (Eq. 10)
 * with the linear encoder g(q) = Ew (q - X0) + eb (supervised setting,
 * Sec. 3.2), z_b = g(q_b) held fixed in L_LS (no gradient through the
 * samples), and Ht_b the exact Hessian in z of the cubature elastic
 * potential sum_{e in S} w_e V_e Psi(F_e(x(z))) (Sec. 4.2-4.3: elastic term
 * only, cubature set S with weights w).  The decoder in training is the one
 * set by lsn_set_decoder, without constraint override.  r <= 32.
 *
 * Parameters are one flat vector, exchanged as FP64 arrays: Ew (r x n
 * row-major), eb (r), then W_l (out x in row-major), b_l for each decoder
 * layer.  The trainer computes in FP64 when the decoder precision is
 * LSN_PREC_FP64 and in FP32 otherwise (FP64 loss sums in both).  Its plain
 * matrix products run on the tensor cores in the tensor-core forms: with
 * TF32 operands (LSN_PREC_TF32), or with BF16 operands, the weights and
 * activations of every product rounded to BF16 with FP32 accumulation and the
 * parameters, gradient and Adam moments kept in FP32 as the master copy
 * (LSN_PREC_BF16).
 * --------------------------------------------------------------------------- */

/* Start training: initial encoder (enc_W r x n, enc_b r; host), training
 * cubature set (tet_idx, non-negative w, s >= 1; host).  Uses the current
 * mesh, material and decoder weights; Adam state is reset. */
int lsn_train_init(lsn_ctx* ctx, const float* enc_W, const float* enc_b,
                   const int32_t* tet_idx, const double* w, int s);
int lsn_train_num_params(lsn_ctx* ctx, long long* count);
/* Copy the flat parameter vector out of / into the trainer (host or device). */
int lsn_train_get_params(lsn_ctx* ctx, double* theta);
int lsn_train_set_params(lsn_ctx* ctx, const double* theta);
/* Adam state, for checkpoint / resume of training: the first and second
 * moment estimates m, v (num_params doubles each, host) and the number of
 * Adam steps taken (the bias-correction exponent).  With the parameters
 * (lsn_train_get_params) they resume training exactly where it stopped.
 * set: m, v finite, v >= 0, step >= 0 (else LSN_ERR_ARG / LSN_ERR_NONFINITE,
 * nothing changed). */
int lsn_train_get_adam(lsn_ctx* ctx, double* m, double* v, long long* step);
int lsn_train_set_adam(lsn_ctx* ctx, const double* m, const double* v, long long step);
/* Losses (losses[0..2] = L_C, L_LS, L; host, may be NULL) and the gradient
 * of L w.r.t. the flat parameters (grad: host or device, may be NULL) for the
 * snapshot positions q (B x n doubles, host or device), B >= 1.  L_LS needs
 * B >= 2 and lambda_ls > 0 (otherwise it is 0). */
int lsn_train_eval(lsn_ctx* ctx, const double* q, int B, double lambda_ls,
                   double* losses, double* grad);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the
 * gradient of L for the batch q; losses as in lsn_train_eval. */
int lsn_train_step(lsn_ctx* ctx, const double* q, int B, double lambda_ls,
                   double lr, double* losses);
/* Unsupervised construction (Eq. 4, Sec. 3.2) at the B samples z (B x r,
 * host or device; the caller draws them from N(0, I)), with the Lipschitz
 * loss of Eq. 9 at the same samples (Eq. 10 in the unsupervised setting; the
 * paper estimates the Lipschitz term from Gaussian subspace samples there):
 *   L_P = 1/B sum_b Pt(x(z_b))          (the cubature elastic potential above)
 *   L_R = 1/(B(B-1)) sum_{i != j} log(||x(z_i) - x(z_j)||_M / (sigma ||z_i - z_j||))^2
 *   L_U = L_P + lambda L_R,   L = L_U + lambda_ls L_LS
 * losses[0..4] = L_P, L_R, L_U, L_LS, L (host, may be NULL); grad (of L) as
 * in lsn_train_eval (the encoder's entries are zero).  lambda, lambda_ls >=
 * 0, sigma > 0; the samples must be distinct (L_R is reported for B >= 2;
 * B >= 2 is required when lambda or lambda_ls is positive). */
int lsn_train_eval_unsup(lsn_ctx* ctx, const double* z, int B, double lambda, double sigma,
                         double lambda_ls, double* losses, double* grad);
/* One Adam step (as lsn_train_step) on the gradient of L. */
int lsn_train_step_unsup(lsn_ctx* ctx, const double* z, int B, double lambda, double sigma,
                         double lambda_ls, double lr, double* losses);
/* Order of the Lipschitz loss in lsn_train_eval / lsn_train_step (the
 * Supplement's family L_LS,o of Lipschitz losses of the o-th derivative of
 * the potential in z): 2 (default) is Eq. 9 on the cubature Hessians; 1 is
 * 1/(B(B-1)) sum_{i != j} ||dPt/dz(z_i) - dPt/dz(z_j)||^2 / ||z_i - z_j||^2;
 * 0 is the same with Pt(z_i) - Pt(z_j); all with the same cubature
 * potential and samples (for the ablation of the order).
 * Other orders: LSN_ERR_ARG.  Applies to the current and later trainers;
 * the unsupervised calls always use order 2. */
int lsn_set_lipschitz_order(lsn_ctx* ctx, int order);

/* Cubature Hessians Ht at the B subspace points z (B x r, host) into H
 * (B x r x r, host), with the trainer's current decoder. */
int lsn_train_hessians(lsn_ctx* ctx, const double* z, int B, double* H);
/* Make the trained decoder the solver's decoder (takes effect at the next
 * solve; the precision set by lsn_set_decoder is kept; weights are rounded
 * to FP32 as lsn_set_decoder takes them). */
int lsn_train_apply(lsn_ctx* ctx);

/* Kernel classes for profiling. */
enum lsn_kernel_class {
  LSN_K_DECODER_HIDDEN = 0, /* hidden layers, Jacobian and trial passes       */
  LSN_K_DECODER_LAST = 1,   /* output layer + x, J and inertia partials       */
  LSN_K_ELEMENT = 2,        /* per-tet energy/gradient/projected Hessian with
                               the J_e^T H_e J_e contraction                   */
  LSN_K_DECODER_TRIAL = 3,  /* output layer of the line-search trial pass     */
  LSN_K_ELEMENT_ENERGY = 4, /* per-tet energy of the line-search trials       */
  LSN_K_SOLVE = 5,          /* partial reductions, Cholesky, Armijo, updates  */
  LSN_K_COUNT = 6
};

/* Profiling: launches of every class are always counted.  Classes whose bit
 * (1 << class) is set in `event_mask` are also timed with CUDA events
 * recorded on the context stream around each launch (device time; the
 * events add a few microseconds of host work per launch). */
int lsn_set_profiling(lsn_ctx* ctx, unsigned event_mask);

/* Accumulated launches and device milliseconds (timed classes only) of
 * kernel class `cls` since the last lsn_reset_profile.  Synchronises the
 * stream. */
int lsn_get_profile(lsn_ctx* ctx, int cls, long long* launches,
                    long long* timed_launches, double* ms_total);
int lsn_reset_profile(lsn_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart to this call: it
 * exists for callers that cannot allocate device memory while they run, for
 * example an engine that gives the library a fixed memory budget up front, a
 * caller working inside a memory pool or arena that must not grow, or a
 * real-time loop where cudaMalloc / cudaFree (which can synchronise the
 * device and can fail) is not allowed.
 *
 * lsn_element_system_noalloc evaluates the elastic part of the reduced
 * system for S tets with the solver's own element kernel (Stable Neo-Hookean
 * energy, gradient and PSD-projected Hessian per tet, contracted with the
 * tets' rows of J) and writes
 *     out[0] = sum_e P_e, out[1] = sum_e |P_e|, out[2 + i] = g_i,
 *     out[2 + r + i] = sum of |contributions to g_i|,
 *     out[2 + 2r + k] = K upper triangle, row-major (i <= j), k < r(r+1)/2,
 * i.e. nslots = 2 + 2r + r(r+1)/2 doubles.  It allocates nothing: its
 * partial sums live in a file-scope device array of LSN_NOALLOC_SCRATCH_DOUBLES
 * doubles (4 MiB) that every GPU which loads the library holds until the
 * process exits.  A problem whose partial sums do not fit, that is
 * (CTAs + 1) * (nslots + 6) > LSN_NOALLOC_SCRATCH_DOUBLES with the solver's
 * launch shape (at most two CTAs per SM, one per 64 or 128 tets), is
 * rejected with LSN_ERR_ARG; r is limited to 64 as elsewhere.
 *
 * All inputs are device pointers (FP32 apart from the indices): tets S x 4
 * vertex indices (16-byte aligned, every index < n / 3: the call cannot check
 * device-resident indices, and an index out of range reads out of bounds),
 * dminv the per-tet inverse rest edge matrices stored
 * structure-of-arrays (entry (a, b) of tet e at dminv[(3 a + b) S + e]),
 * wvol the weight times rest volume of each tet, u the n displacements
 * x - X0 (n a multiple of 3), J the n x r Jacobian (row-major; 16-byte
 * aligned when r is a multiple of 4).  A misaligned pointer or n not a
 * multiple of 3 returns LSN_ERR_ARG.  mu, lam are the Lame
 * parameters.  out is device memory or pinned host memory.  Work is issued on
 * cuda_stream (a cudaStream_t, NULL = default stream) and is complete when
 * that stream has synchronised.
 *
 * The first call on a device (the current device when it is made) looks up
 * the device address of the scratch array for that device (under a mutex, so
 * first calls from several host threads are safe); make that first call
 * before any stream capture.  The address is cached for the life of the
 * process: after cudaDeviceReset (or any teardown of the device's primary
 * context) this call must not be used on that device again.  Every call on
 * a device shares the one scratch array, and the array keeps the last call's
 * partial sums: calls that may overlap on the GPU (different streams, or host
 * threads without ordering) race and must be serialised by the caller.  Nothing needs
 * clearing between calls: each call writes every partial it reads. */
#define LSN_NOALLOC_SCRATCH_DOUBLES 524288
int lsn_element_system_noalloc(int S, int r, int n, const int32_t* tets,
                               const float* dminv, const float* wvol,
                               const float* u, const float* J, double mu,
                               double lam, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LSN_H */
