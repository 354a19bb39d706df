// Internal declarations shared by the CUDA translation units of liblsn.
// Kernels are written for sm_103a (GB300); host code follows the C ABI in
// include/lsn.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lsn {

constexpr int RMAX = 64;           // largest subspace dimension
constexpr int KTRIAL = 4;          // line-search step lengths evaluated per pass
constexpr int GEMM_BK = 32;        // k-chunk of the decoder GEMM tiles
constexpr int TRACE = 128;         // Newton iterations kept in the solve trace

// Number of upper-triangle entries of an r x r symmetric matrix.
__host__ __device__ inline int npairs(int r) { return r * (r + 1) / 2; }
// Slots of one reduced-system partial: E, sum |E terms|, g[r], gabs[r]
// (sum of |contributions| per gradient entry: the rounding scale of g), K
// upper triangle (row-major, i <= j).
__host__ __device__ inline int nslots(int r) { return 2 + 2 * r + npairs(r); }
__host__ __device__ inline int slot_g(int i) { return 2 + i; }
__host__ __device__ inline int slot_gabs(int r, int i) { return 2 + r + i; }
__host__ __device__ inline int slot_K(int r) { return 2 + 2 * r; }

// Device-resident Newton / line-search state (one per context).
struct DevSolver {
  double z[RMAX];      // current iterate
  double d[RMAX];      // Newton direction
  double g[RMAX];      // reduced gradient at z
  double E, Eabs;      // energy at z and sum of |terms| (rounding scale)
  double gd;           // g . d
  double grad_inf;     // ||g||_inf at z
  double gabs_max;     // max_i of the rounding scale of g_i
  double g_best;       // smallest ||g||_inf of this solve
  int stall;           // iterations since ||g||_inf last halved
  double alpha_base;   // step length of trial 0 of the current batch
  double alpha_taken;  // accepted step length
  double tol, armijo_c, eta_scale;
  double floor_scale;  // kappa * unit roundoff of the element precision
  int r, max_ls;
  int status;          // -1 running, else lsn_status of the solve
  int iters, ls_trials;
  int ls_iter;         // trials spent in the current line search
  int accepted;        // line search of this iteration accepted a step
  int eval_only;       // direction kernel only reduces (parity hook)
  // per-iteration history of the current solve (first TRACE iterations)
  double trace_g[TRACE], trace_E[TRACE], trace_gabs[TRACE], trace_alpha[TRACE];
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
enum class Epi { HiddenJac = 0, HiddenVal = 1, LastJac = 2, LastVal = 3 };

struct LastArgs {            // data of the output-layer epilogue
  int n, r;
  double scale;
  const int* cslot;          // per vertex: constraint slot or -1
  const double* cu;          // constrained displacement targets (3 per slot)
  const double* mass;        // per vertex
  const double* ubar;        // qbar - X0 (n), dynamics only
  double inv_dt2;            // 1/dt^2, 0 for quasi-static
  double grav[3];
  double ground_h, ground_k; // ground plane, k = 0 off
  const double* X0;          // rest positions (n)
};

template <typename Real>
void launch_decoder_layer(Epi epi, const Real* W, const Real* b, int M, int K,
                          const Real* Zin, int C, Real* Zout, int ldo,
                          Real* u_out, Real* J_out, double* part,
                          int part_stride, const LastArgs& la, int grid_cap,
                          cudaStream_t s);
int decoder_last_grid(int n, int C, int num_sms);
int decoder_cpad(int C);

// element.cu
struct ElemArgs {
  int S, r, n;
  const int4* tets;
  const void* dminv;   // Real [9][S]
  const void* wv;      // Real [S]: w_e * V_e
  double mu, lam;
};
template <typename Real>
void launch_element_full(const ElemArgs& ea, const Real* u, const Real* J,
                         double* part, int grid, cudaStream_t s);
template <typename Real>
void launch_element_energy(const ElemArgs& ea, const Real* ut, int k,
                           double* part, int grid, cudaStream_t s);
int element_full_grid(int S, int num_sms);
int element_energy_grid(int S, int num_sms);

// solve.cu
void launch_reduce_cols(const double* A, int rowsA, const double* B, int rowsB,
                        int ncols, double* out, cudaStream_t s);
template <typename Real>
void launch_newton_direction(DevSolver* sv, const double* sys, Real* Z0, int max_newton,
                             cudaStream_t s);
template <typename Real>
void launch_ls_select(DevSolver* sv, const double* sys_t, Real* Z0, cudaStream_t s);
template <typename Real>
void launch_write_jac_columns(const DevSolver* sv, Real* Z0, cudaStream_t s);
template <typename Real>
void launch_finish_positions(const double* X0, const Real* u, int n, double dt, double* q,
                             double* v, cudaStream_t s);
void launch_inertial_guess(const double* X0, const double* q, const double* v, int n,
                           double dt, const double* g /* host, 3 */, double* ubar,
                           cudaStream_t s);

}  // namespace lsn
