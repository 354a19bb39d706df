// Reduced-system kernels of the projective Newton solve (Supplement, "Tests
// with Projective Newton's method"; exits of Sec. 5): fixed-order reduction
// of the per-CTA partials, FP64 r x r Cholesky with diagonal-shift retries,
// Newton direction, and the Armijo acceptance test of the backtracking line
// search (FP64 comparison).  Single-block kernels; r <= 64.
#include "lsn_internal.cuh"

namespace lsn {
namespace {

constexpr int ST = 256;

__device__ __forceinline__ int upper_index(int i, int j, int r) {
  // row-major enumeration of the upper triangle, i <= j
  return i * r - (i * (i - 1)) / 2 + (j - i);
}

__global__ void reduce_cols_kernel(const double* __restrict__ A, int rowsA,
                                   const double* __restrict__ B, int rowsB, int ncols,
                                   double* __restrict__ out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < rowsA; ++b) s += A[(size_t)b * ncols + c];
  for (int b = 0; b < rowsB; ++b) s += B[(size_t)b * ncols + c];
  out[c] = s;
}

template <typename Real>
__device__ void write_trial_columns(DevSolver* sv, Real* Z0) {
  const int r = sv->r;
  for (int e = threadIdx.x; e < KTRIAL * r; e += blockDim.x) {
    const int j = e / r, i = e - j * r;
    const double a = ldexp(sv->alpha_base, -j);
    Z0[j * r + i] = (Real)(sv->z[i] + a * sv->d[i]);
  }
}

template <typename Real>
__global__ void __launch_bounds__(ST) newton_direction_kernel(DevSolver* sv,
                                                              const double* __restrict__ sys,
                                                              Real* Z0, int max_newton) {
  __shared__ double L[RMAX][RMAX + 1];
  __shared__ double g[RMAX], y[RMAX];
  __shared__ double red[ST];
  __shared__ int fail;
  __shared__ double diag_j;
  const int t = threadIdx.x;
  const int r = sv->r;
  if (sv->status != -1) return;
  // g and the symmetric K (upper triangle in sys) from the reduced partial sums
  const double* Ku = sys + slot_K(r);
  for (int i = t; i < r; i += ST) g[i] = sys[slot_g(i)];
  __syncthreads();
  double gm = 0.0, ga = 0.0;
  bool finite = true;
  for (int i = t; i < r; i += ST) {
    gm = fmax(gm, fabs(g[i]));
    ga = fmax(ga, sys[slot_gabs(r, i)]);
    finite = finite && isfinite(g[i]);
  }
  for (int e = t; e < npairs(r); e += ST) finite = finite && isfinite(Ku[e]);
  red[t] = finite ? gm : -1.0;
  __syncthreads();
  for (int s = ST / 2; s > 0; s >>= 1) {
    if (t < s) red[t] = (red[t] < 0.0 || red[t + s] < 0.0) ? -1.0 : fmax(red[t], red[t + s]);
    __syncthreads();
  }
  const double ginf = red[0];
  __syncthreads();
  red[t] = ga;
  __syncthreads();
  for (int s = ST / 2; s > 0; s >>= 1) {
    if (t < s) red[t] = fmax(red[t], red[t + s]);
    __syncthreads();
  }
  const double gabs_max = red[0];
  const double E = sys[0];
  __syncthreads();
  // progress bookkeeping for the precision-floor exit
  __shared__ int stall;
  if (t == 0) {
    sv->E = E;
    sv->Eabs = sys[1];
    sv->grad_inf = ginf;
    sv->gabs_max = gabs_max;
    if (!sv->eval_only) {
      if (sv->iters < TRACE) {
        sv->trace_g[sv->iters] = ginf;
        sv->trace_E[sv->iters] = E;
        sv->trace_gabs[sv->iters] = gabs_max;
        sv->trace_alpha[sv->iters] = 0.0;
      }
      if (ginf <= 0.5 * sv->g_best) {
        sv->g_best = ginf;
        sv->stall = 0;
      } else {
        sv->g_best = fmin(sv->g_best, ginf);
        sv->stall += 1;
      }
    }
    stall = sv->stall;
  }
  for (int i = t; i < r; i += ST) sv->g[i] = g[i];
  __syncthreads();
  if (sv->eval_only) return;
  if (ginf < 0.0 || !isfinite(E)) {
    if (t == 0) sv->status = -3;  // LSN_ERR_NONFINITE
    return;
  }
  if (ginf < sv->tol) {
    if (t == 0) sv->status = 0;  // LSN_OK
    return;
  }
  // ||g|| has stopped decreasing and is within the rounding scale of its own
  // evaluation: further iterations cannot be resolved at this precision
  if (stall >= 4 && ginf <= sv->floor_scale * gabs_max) {
    if (t == 0) sv->status = 4;  // LSN_PRECISION_FLOOR
    return;
  }
  if (sv->iters >= max_newton) {
    if (t == 0) sv->status = 1;  // LSN_NOT_CONVERGED
    return;
  }
  // Cholesky K + shift I = L L^T, shift = 0, then 1e-12 max(1, max|K_ii|) x 10^k
  double dmax = 0.0;
  for (int i = 0; i < r; ++i) dmax = fmax(dmax, fabs(Ku[upper_index(i, i, r)]));
  const double base = 1e-12 * fmax(1.0, dmax);
  double shift = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 21 && !ok; ++attempt) {
    for (int e = t; e < r * r; e += ST) {
      int i = e / r, j = e - i * r;
      L[i][j] = (i <= j ? Ku[upper_index(i, j, r)] : Ku[upper_index(j, i, r)]) +
                (i == j ? shift : 0.0);
    }
    if (t == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
      if (t == 0) {
        double s = L[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0)) fail = 1;
        diag_j = s > 0.0 ? sqrt(s) : 1.0;
        L[j][j] = diag_j;
      }
      __syncthreads();
      if (fail) break;
      for (int i = j + 1 + t; i < r; i += ST) {
        double s = L[i][j];
        for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
        L[i][j] = s / diag_j;
      }
      __syncthreads();
    }
    __syncthreads();
    ok = !fail;
    if (!ok) shift = shift == 0.0 ? base : shift * 10.0;
    __syncthreads();
  }
  if (!ok) {
    if (t == 0) sv->status = 3;  // LSN_NOT_SPD
    return;
  }
  // forward L y = -g, backward L^T d = y (column sweeps)
  for (int i = t; i < r; i += ST) y[i] = -g[i];
  __syncthreads();
  for (int i = 0; i < r; ++i) {
    if (t == 0) y[i] /= L[i][i];
    __syncthreads();
    for (int k = i + 1 + t; k < r; k += ST) y[k] -= L[k][i] * y[i];
    __syncthreads();
  }
  for (int i = r - 1; i >= 0; --i) {
    if (t == 0) y[i] /= L[i][i];
    __syncthreads();
    for (int k = t; k < i; k += ST) y[k] -= L[i][k] * y[i];
    __syncthreads();
  }
  for (int i = t; i < r; i += ST) sv->d[i] = y[i];
  red[t] = 0.0;
  for (int i = t; i < r; i += ST) red[t] += g[i] * y[i];
  __syncthreads();
  for (int s = ST / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) {
    sv->gd = red[0];
    sv->alpha_base = 1.0;
    sv->accepted = 0;
    sv->ls_iter = 0;
  }
  __syncthreads();
  write_trial_columns<Real>(sv, Z0);
}

// Armijo test of the batch of KTRIAL step lengths alpha_base 2^-j, in order;
// the first that passes is taken (same result as one-at-a-time halving).
template <typename Real>
__global__ void ls_select_kernel(DevSolver* sv, const double* __restrict__ sys_t, Real* Z0) {
  __shared__ int acc, go;
  if (threadIdx.x == 0) go = (sv->status == -1 && !sv->accepted);
  __syncthreads();
  if (!go) return;
  if (threadIdx.x == 0) {
    acc = -1;
    for (int j = 0; j < KTRIAL; ++j) {
      if (sv->ls_iter >= sv->max_ls) break;
      sv->ls_iter += 1;
      sv->ls_trials += 1;
      const double a = ldexp(sv->alpha_base, -j);
      const double Et = sys_t[2 * j];
      const double eta = sv->eta_scale * (sys_t[2 * j + 1] + sv->Eabs);
      if (isfinite(Et) && Et <= sv->E + sv->armijo_c * a * sv->gd + eta) {
        acc = j;
        sv->alpha_taken = a;
        break;
      }
    }
    if (acc < 0) {
      if (sv->ls_iter >= sv->max_ls) {
        sv->status = (sv->grad_inf < 100.0 * sv->tol) ? 4 : 2;
      } else {
        sv->alpha_base = ldexp(sv->alpha_base, -KTRIAL);
      }
    } else {
      if (sv->iters < TRACE) sv->trace_alpha[sv->iters] = ldexp(sv->alpha_base, -acc);
      sv->accepted = 1;
      sv->iters += 1;
    }
  }
  __syncthreads();
  if (acc >= 0) {
    const double a = ldexp(sv->alpha_base, -acc);
    for (int i = threadIdx.x; i < sv->r; i += blockDim.x) sv->z[i] += a * sv->d[i];
  } else if (sv->status == -1) {
    write_trial_columns<Real>(sv, Z0);
  }
}

// Z0 = [z | I_r] (Jacobian pass; column-major, leading dimension r).
template <typename Real>
__global__ void write_jac_columns_kernel(const DevSolver* sv, Real* Z0) {
  const int r = sv->r;
  for (int e = threadIdx.x; e < (r + 1) * r; e += blockDim.x) {
    const int c = e / r, i = e - c * r;
    Z0[e] = c == 0 ? (Real)sv->z[i] : (i == c - 1 ? Real(1) : Real(0));
  }
}

template <typename Real>
__global__ void finish_positions_kernel(const double* __restrict__ X0,
                                        const Real* __restrict__ u, int n, double dt,
                                        double* __restrict__ q, double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double qn = X0[i] + (double)u[i];
  if (dt > 0.0) v[i] = (qn - q[i]) / dt;
  q[i] = qn;
}

__global__ void inertial_guess_kernel(const double* __restrict__ X0,
                                      const double* __restrict__ q,
                                      const double* __restrict__ v, int n, double dt,
                                      double gx, double gy, double gz,
                                      double* __restrict__ ubar) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = i % 3;
  const double g = c == 0 ? gx : (c == 1 ? gy : gz);
  ubar[i] = (q[i] - X0[i]) + dt * v[i] + dt * dt * g;
}

}  // namespace

void launch_reduce_cols(const double* A, int rowsA, const double* B, int rowsB, int ncols,
                        double* out, cudaStream_t s) {
  reduce_cols_kernel<<<(ncols + 127) / 128, 128, 0, s>>>(A, rowsA, B, rowsB, ncols, out);
}

template <typename Real>
void launch_newton_direction(DevSolver* sv, const double* sys, Real* Z0, int max_newton,
                             cudaStream_t s) {
  newton_direction_kernel<Real><<<1, ST, 0, s>>>(sv, sys, Z0, max_newton);
}

template <typename Real>
void launch_ls_select(DevSolver* sv, const double* sys_t, Real* Z0, cudaStream_t s) {
  ls_select_kernel<Real><<<1, 64, 0, s>>>(sv, sys_t, Z0);
}

template <typename Real>
void launch_write_jac_columns(const DevSolver* sv, Real* Z0, cudaStream_t s) {
  write_jac_columns_kernel<Real><<<1, 256, 0, s>>>(sv, Z0);
}

template <typename Real>
void launch_finish_positions(const double* X0, const Real* u, int n, double dt, double* q,
                             double* v, cudaStream_t s) {
  finish_positions_kernel<Real><<<(n + 255) / 256, 256, 0, s>>>(X0, u, n, dt, q, v);
}

void launch_inertial_guess(const double* X0, const double* q, const double* v, int n,
                           double dt, const double* g, double* ubar, cudaStream_t s) {
  inertial_guess_kernel<<<(n + 255) / 256, 256, 0, s>>>(X0, q, v, n, dt, g[0], g[1], g[2],
                                                        ubar);
}

#define LSN_INST(R)                                                                   \
  template void launch_newton_direction<R>(DevSolver*, const double*, R*, int,        \
                                           cudaStream_t);                             \
  template void launch_ls_select<R>(DevSolver*, const double*, R*, cudaStream_t);     \
  template void launch_write_jac_columns<R>(const DevSolver*, R*, cudaStream_t);      \
  template void launch_finish_positions<R>(const double*, const R*, int, double,      \
                                           double*, double*, cudaStream_t);
LSN_INST(float)
LSN_INST(double)
#undef LSN_INST

}  // namespace lsn
