// Internal declarations shared by the CUDA translation units of liblsn.
// Kernels are written for sm_103a (GB300); host code follows the C ABI in
// include/lsn.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace lsn {

constexpr int RMAX = 64;           // largest subspace dimension
constexpr int KTRIAL = 3;          // extra line-search step lengths per pass
constexpr int GEMM_BK = 32;        // k-chunk of the decoder GEMM tiles
constexpr int TRACE = 128;         // Newton iterations kept in the solve trace
constexpr int MHIST = 32;          // largest L-BFGS history (curvature pairs)

// Number of upper-triangle entries of an r x r symmetric matrix.
__host__ __device__ inline int npairs(int r) { return r * (r + 1) / 2; }
// Slots of one reduced-system partial: E, sum |E terms|, g[r], gabs[r]
// (sum of |contributions| per gradient entry: the rounding scale of g), K
// upper triangle (row-major, i <= j); then (E_j, sum|E_j terms|) of the
// KTRIAL trial points.
__host__ __device__ inline int nslots(int r) { return 2 + 2 * r + npairs(r); }
__host__ __device__ inline int nslots_total(int r) { return nslots(r) + 2 * KTRIAL; }
// Column stride of the decoder activations Z[k][c]: C rounded up to a
// multiple of 4 with an odd number of 4-element groups, so that eight
// consecutive rows of Z fall into distinct shared-memory bank groups.
__host__ __device__ inline int zstride(int C) {
  int c = (C + 3) & ~3;
  return ((c / 4) % 2 == 0) ? c + 4 : c;
}
__host__ __device__ inline int slot_g(int i) { return 2 + i; }
__host__ __device__ inline int slot_gabs(int r, int i) { return 2 + r + i; }
__host__ __device__ inline int slot_K(int r) { return 2 + 2 * r; }

// Device-resident Newton / line-search state (one per context).  Scalars
// first so that the host can copy the summary (up to and including z)
// without the trace arrays.
struct DevSolver {
  // controls (set by the host)
  double tol, armijo_c, eta_scale;
  double floor_scale;  // kappa * unit roundoff of the element precision
  int r, max_ls, max_newton, eval_only;
  // dynamics of the current step
  double inv_dt2;      // 1/dt^2, 0 for quasi-static
  // progress
  double E, Eabs;      // energy at z and sum of |terms| (rounding scale)
  double gd;           // g . d
  double grad_inf;     // ||g||_inf at z
  double gabs_max;     // max_i of the rounding scale of g_i
  double g_best;       // reference ||g||_inf for the stall counter
  double alpha_base;   // step length of candidate 0 of the current pass
  double alpha_taken;  // last accepted step length
  int status;          // -1 running, else lsn_status of the solve
  int iters, ls_trials;
  int ls_iter;         // trials spent in the current line search
  int have_dir;        // the current pass evaluated z + alpha d (speculative)
  int final_pass;      // one more pass at z is queued to refresh positions
  int running;         // the solve loop continues
  int stall;           // iterations without a 10 % drop of ||g||_inf
  int passes;          // evaluation passes of this solve
  int kind;            // optimiser: 0 projective Newton, 1 L-BFGS
  int hist_m;          // L-BFGS: history size m
  int hist_n;          // L-BFGS: stored curvature pairs
  int hist_head;       // L-BFGS: ring slot of the oldest pair
  int pair_pending;    // L-BFGS: a step was taken; its pair is formed at the next gradient
  int tiny_steps;      // consecutive accepted steps with alpha < 2^-10
  int pad_;
  double gamma;        // L-BFGS: initial scaling s^T y / y^T y of the newest pair
  double* zd;          // FP64 copy of the pass points [r][zstride(C)] (affine modes) or null
  double z[RMAX];      // current iterate
  double d[RMAX];      // Newton direction
  double g[RMAX];      // reduced gradient at z
  // per-iteration history of the current solve (first TRACE iterations)
  double trace_g[TRACE], trace_E[TRACE], trace_gabs[TRACE], trace_alpha[TRACE];
};

// L-BFGS curvature pairs (s_i, y_i) of the current solve, a ring of
// DevSolver::hist_m slots, and the reduced gradient at z (for y = g' - g).
struct DevHistory {
  double gz[RMAX];
  double S[MHIST][RMAX], Y[MHIST][RMAX];
  double rho[MHIST];   // 1 / s_i^T y_i
};

// ---------------------------------------------------------------- launchers
// mesh.cu
void launch_rest_shape(const double* X0, const int4* tets, int ne,
                       double* dminv, double* vol, int* bad, cudaStream_t s);
void launch_lumped_mass(const int* adj_ptr, const int* adj_tet, const double* vol,
                        int nv, double rho, double* mass, cudaStream_t s);
void launch_constraint_disp(const int* cidx, const double* targets, const double* X0, int nc,
                            double* cu, cudaStream_t s);
template <typename Real>
void launch_gather_cubature(const int4* tets, const double* dminv, const double* vol,
                            const int* idx, const double* w, int s_cnt, int ne,
                            int4* ctets, Real* cdminv, Real* cwv, cudaStream_t s);
template <typename Real>
void launch_convert(const double* src, Real* dst, long long count, cudaStream_t s);

// decoder.cu
struct LastArgs {            // data of the output-layer epilogue
  int n, r;
  double scale;
  const int* cslot;          // per vertex: constraint slot or -1
  const double* cu;          // constrained displacement targets (3 per slot)
  const double* mass;        // per vertex
  const double* ubar;        // qbar - X0 (n), dynamics only
  const double* inv_dt2;     // device scalar: 1/dt^2, 0 for quasi-static
  double grav[3];
  double ground_h, ground_k; // ground plane, k = 0 off
  const double* X0;          // rest positions (n)
  // affine modes (aff0 < 0: none): coordinates aff0 .. aff0 + 11 of z are
  // (M row-major, t) with u_v += M (X0_v - acen) + t; zaff points at row aff0
  // of the FP64 copy of the pass points (column stride zcps)
  int aff0, zcps;
  const double* zaff;
  double acen[3];
};

// Activations are unit-major Z[k][c] with column stride zstride(C).
template <typename Real>
void launch_hidden_layer(const Real* W, const Real* b, int M, int K, const Real* Zin, int C,
                         int nj, Real* Zout, cudaStream_t s, void* Bh = nullptr,
                         void* Bl = nullptr, int bkind = 0);
// tc_gemm.cu: C[m][n] = alpha sum_k A(m,k) B(k,n) + beta C[m][n] with
// A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn] (any strides), FP32
// operands read as TF32 on tcgen05; K split over the grid (deterministic
// fixed-order sum) when the tiles leave SMs idle, using ws (ws_floats of
// tc_gemm_workspace_floats; no split without it).  err: device flag, set
// when a bounded wait ran out.
size_t tc_gemm_workspace_floats(int M, int N, int K, int num_sms);
cudaError_t tc_gemm_tf32(cudaStream_t s, int M, int N, int K, float alpha, const float* A,
                         long long sam, long long sak, const float* B, long long sbk,
                         long long sbn, float beta, float* C, long long ldc, float* ws,
                         size_t ws_floats, int num_sms, int* err, bool bf16_operands = false);
// tc_hidden.cu: hidden layers on the tensor cores (BF16 / TF32 forms; the
// TcHidden handle is in tc_internal.cuh).  tc_hidden_applies: the layer's
// shared-memory plan fits one CTA.
bool tc_hidden_applies(int M, int K, int C);
template <typename Real>
void launch_last_layer(const Real* W, const Real* b, int M, int K, const Real* Zin, int C,
                       int nj, Real* u_out, Real* J_out, Real* u_trial, double* part,
                       int part_stride, const LastArgs& la, int grid, cudaStream_t s);
int decoder_last_grid(int n, int C, int num_sms);

// element.cu
struct ElemArgs {
  int S, r, n;
  const int4* tets;
  const void* dminv;   // Real [9][S]
  const void* wv;      // Real [S]: w_e * V_e
  double mu, lam;
};
// grid = gfull + genergy blocks: the first gfull take the fused
// energy / gradient / projected-Hessian contraction at u, the others the
// energies of the KTRIAL trial fields ut[j * n + .].  Row b of `part` (stride
// nslots_total(r)) receives the JAC slots (b < gfull) or the trial slots.
template <typename Real>
void launch_element(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                    double* part, int gfull, int genergy, cudaStream_t s);
void element_grids(int S, int r, int num_sms, int& gfull, int& genergy);
// Tensor-core element kernel (TF32 / BF16 forms, r <= 64): `grid` CTAs, each
// writing one complete partial row (elastic slots and trial energies) of
// nslots_total(r) doubles; err receives a nonzero code if a bounded wait ran out.
int element_tc_grid(int S, int r, bool bf16, int num_sms);
// Warp-specialised tensor-core element kernel (element_ws.cu) for large tet
// sets: used by launch_element_tc when element_ws_applies (the BF16 form, r a
// multiple of 4 and at most 64, at least 160 tets per SM); same partial-row
// output.
bool element_ws_applies(int S, int r, bool bf16, int num_sms);
int element_ws_grid(int S, int num_sms);
cudaError_t launch_element_ws(const ElemArgs& ea, const float* u, const float* J, const float* ut,
                              double* part, int grid, int* err, cudaStream_t s);
// Gradient-only element kernel of the L-BFGS passes (any precision form):
// `grid` CTAs, each writing the E, g, gabs and trial-energy slots of one
// partial row (stride nslots_total(r)); the K slots are not written.
int element_grad_grid(int S, int num_sms);
// Per-tet reduced elastic forces of every mesh tet (unit weight) for the
// cubature fit: A[i * ne + e] = (J_e^T dP_e/dx_e)_i, i < r (FP64 output).
template <typename Real>
void launch_tet_forces(const int4* tets, const double* dminv, const double* vol, int ne, int r,
                       const Real* u, const Real* J, double mu, double lam, double* A,
                       cudaStream_t s);
template <typename Real>
void launch_element_grad(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                         double* part, int grid, cudaStream_t s);
// Full-space projective Newton (the comparison solve, all tets at unit
// weight).  fs_elem: at u = q - X0 the per-CTA energy sums (part[2 b],
// part[2 b + 1] = sum |terms|), the gradient, its sum of |contributions| and
// the diagonal of the projected Hessian added into g, gabs and diag (zeroed
// by the caller), and the
// per-tet factor data [FS_NF][ne] of Hproj_e = A_e^T A_e.  fs_hv: y +=
// sum_e A_e^T A_e p_e unless *done.  fs_energy: per-CTA elastic energy sums
// at q + alpha d.  ea.dminv / ea.wv hold Dm^-1 [9][ne] and V_e in Real.
constexpr int FS_NF = 33;
int fs_grid(int ne, int threads, int num_sms);
template <typename Real>
void launch_fs_elem(const ElemArgs& ea, const Real* u, Real* fac, double* g, double* gabs,
                    double* diag, double* part, int grid, cudaStream_t s);
template <typename Real>
void launch_fs_hv(const int4* tets, const Real* dminv, int ne, const Real* fac, const double* p,
                  double* y, const int* done, int grid, cudaStream_t s);
template <typename Real>
void launch_fs_energy(const int4* tets, const Real* dminv, const Real* wv, int ne,
                      const double* q, const double* X0, const double* d, double alpha,
                      double mu, double lam, double* part, int grid, cudaStream_t s);
cudaError_t launch_element_tc(const ElemArgs& ea, const float* u, const float* J,
                              const float* ut, double* part, int grid, bool bf16, int* err,
                              int num_sms, cudaStream_t s);

// cubature.cu: optimised cubature fit on the per-tet force matrix A
// ([m][ne] row-major, device, FP64; rows of r per snapshot).  normalise:
// b = A 1, each snapshot's rows of A and b divided by ||b_k||.  nnls:
// Lawson-Hanson active set stopped at S active columns; P the active tets,
// xP their weights, rel = ||A_P xP - b|| / ||b||.
cudaError_t cubature_normalise(double* A, int m, int ne, int r, std::vector<double>& b,
                               cudaStream_t s);
cudaError_t cubature_nnls(const double* A, int m, int ne, const std::vector<double>& b, int S,
                          std::vector<int>& P, std::vector<double>& xP, double& rel,
                          cudaStream_t s);

// fullspace.cu: full-space projective Newton with preconditioned CG (the
// comparison solve).  FsArgs carries the context's mesh, material, current
// constraint targets and solver controls for one step; the solver owns its
// full state q, v (n doubles each, device).
struct FsArgs {
  int nv, n, ne;
  const double* X0;     // rest positions (n)
  const int4* tets;     // (ne)
  const double* dminv;  // Dm^-1 [9][ne]
  const double* vol;    // (ne)
  const double* mass;   // lumped, per vertex (nv)
  const int* cslot;     // per vertex: constraint slot or -1
  const double* cu;     // constrained displacement targets (3 per slot)
  double mu, lam, grav[3];
  double tol, armijo_c, cg_rtol;
  int max_newton, max_ls, max_cg;
};
struct FsResult {
  int status, newton_iters, ls_trials;
  long long cg_iters;
  double grad_inf, energy;
};
struct FullSpaceBase {
  virtual ~FullSpaceBase() {}
  virtual double* positions() = 0;   // q (device, n)
  virtual double* velocities() = 0;  // v (device, n)
  // One implicit-Euler step (dt > 0) or quasi-static solve (dt = 0) from the
  // current q, v; res.status is an lsn_status (LSN_ERR_NONFINITE when E or g
  // is not finite, q then left at the last finite iterate).
  virtual cudaError_t step(const FsArgs& a, double dt, FsResult& res, cudaStream_t s) = 0;
};
// Allocates the solver (FP64 or FP32 element math) with q = X0, v = 0.
cudaError_t make_fullspace(bool fp64, const FsArgs& a, int num_sms, cudaStream_t s,
                           FullSpaceBase** out);

// solve.cu
// out[c] = sum over rows of A (all rows) and of B: rows [0, splitB) for
// c < split, rows [splitB, rowsB) for c >= split (splitB < 0: all rows for
// every column).  Fixed order.  Columns [gap0, gap0 + gapn) are skipped (out
// left unchanged there).
void launch_reduce_partials(const double* A, int rowsA, const double* B, int rowsB,
                            int splitB, int split, int ncols, double* out, cudaStream_t s,
                            int gap0 = 0, int gapn = 0);
// Z0 is the first layer's input [r][zstride(C)]: column 0 the point y0,
// columns 1..r the identity, columns r+1..r+KTRIAL the trial points.
template <typename Real>
void launch_solve_begin(DevSolver* sv, Real* Z0, int C, int eval_only, cudaStream_t s);
template <typename Real>
void launch_select_direction(DevSolver* sv, const double* sys, Real* Z0,
                             unsigned long long cond, int use_cond, cudaStream_t s);
// L-BFGS counterpart of launch_select_direction: the same line search and
// exits, the direction from the two-loop recursion over the history.
template <typename Real>
void launch_select_lbfgs(DevSolver* sv, DevHistory* hist, const double* sys, Real* Z0,
                         unsigned long long cond, int use_cond, cudaStream_t s);
template <typename Real>
void launch_finish_positions(const double* X0, const Real* u, int n, double dt, double* q,
                             double* v, cudaStream_t s);
// ubar = q + dt v + dt^2 g - X0 (dt > 0, q != NULL) and sv->inv_dt2 = 1/dt^2
// (0 if dt == 0)
void launch_begin_step(const double* X0, const double* q, const double* v, int n, double dt,
                       const double* g /* host, 3 */, double* ubar, DevSolver* sv,
                       cudaStream_t s);

// Exact-form reduced Hessian (curvature.cu, lsn_set_exact_hessian): per
// evaluation pass, the decoder-curvature term sum_{k free} dE/dx_k d2x_k/dz2
// added to the K slots of the reduced system row, then the r x r projection.
struct CurvView {
  std::vector<int> widths;   // r_nn, hidden widths..., n
  int n = 0, nv = 0, ne = 0, S = 0, r = 0, num_sms = 1;
  const int4* tets = nullptr;     // every tet of the mesh (device)
  const int* cub_idx = nullptr;   // cubature tets (device; null: every tet, S = ne)
  bool use_tc_gemm = false;       // hidden-layer products on the TF32 tensor-core GEMM
  cudaStream_t s = nullptr;
};
template <typename Real>
struct Curvature {
  CurvView v;
  double clamp = 1e-10;
  int rn = 0, NY = 0, Hl = 0, nb = 0;
  size_t proj_smem = 0, ws_floats = 0;
  Real *F = nullptr, *G = nullptr, *Y[2] = {nullptr, nullptr}, *A = nullptr, *vv = nullptr;
  double* part = nullptr;
  int *vptr = nullptr, *ventry = nullptr;
  float* ws = nullptr;
  int* gerr = nullptr;
  cudaError_t setup(const CurvView& cv);
  void release();
  // u: displacements at the pass point y0; Z0: the pass points (column 0 =
  // y0, column stride zcps); dW, db: the decoder (device, Real); wl_bf16: the
  // BF16 copy of W_L the output layer reads in the BF16 form (else null);
  // sys: the reduced system row after the partial-row reduction
  cudaError_t launch(const ElemArgs& ea, const LastArgs& la, const Real* u, const Real* Z0,
                     int zcps, const std::vector<Real*>& dW, const std::vector<Real*>& db,
                     const void* wl_bf16, double* sys, cudaStream_t s) const;
  int launches() const { return 7 + 2 * ((int)v.widths.size() - 2); }
  int device_error() const;
  ~Curvature() { release(); }
};

// tc_decoder.cu: one bounded mbarrier wait that runs out (nothing arrives):
// *code (host) receives the error flag the wait records (1)
cudaError_t bounded_wait_selftest(double seconds, int* code, cudaStream_t s);

}  // namespace lsn
