// Reduced-system kernels of the projective Newton solve (Supplement, "Tests
// with Projective Newton's method"; exits of Sec. 5): fixed-order reduction
// of the per-CTA partials, the Armijo test of the backtracking line search
// (FP64 comparison), the FP64 r x r factorisation (L D L^T: the Cholesky
// pivots without square roots) with diagonal-shift retries and the Newton
// direction.
//
// Evaluation passes.  Every pass evaluates x, J, E, g, K at one point y0 and
// the energies at KTRIAL more points.  While a line search is open the pass
// points are z + alpha_base 2^-j d, j = 0..KTRIAL, i.e. the next candidates
// of the halving sequence 1, 1/2, 1/4, ...; the first that satisfies Armijo
// is taken, exactly as one-at-a-time backtracking would.  When the full
// candidate y0 is taken, the pass already holds g and K there and the next
// direction follows at once (one pass per Newton iteration); when a shorter
// step is taken, the next pass evaluates at the new z.  select_direction runs
// after every pass, decides, and writes the points of the next pass.
// Single-block kernels; r <= 64.
#include "lsn_internal.cuh"
#include "pdl.cuh"

#include <cstddef>

namespace lsn {
namespace {

constexpr int ST = 256;

__device__ __forceinline__ int upper_index(int i, int j, int r) {
  // row-major enumeration of the upper triangle, i <= j
  return i * r - (i * (i - 1)) / 2 + (j - i);
}

// One warp per output column; lanes stride over the rows, then a fixed
// shuffle tree: the summation order does not depend on scheduling.
__global__ void reduce_partials_kernel(const double* __restrict__ A, int rowsA,
                                       const double* __restrict__ B, int rowsB, int splitB,
                                       int split, int ncols, double* __restrict__ out, int gap0,
                                       int gapn) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  pdl_wait();
  if (warp >= ncols - gapn) return;
  const int c = warp < gap0 ? warp : warp + gapn;  // columns [gap0, gap0 + gapn) skipped
  double s = 0.0;
  for (int b = lane; b < rowsA; b += 32) s += A[(size_t)b * ncols + c];
  // splitB < 0: every B row carries every column
  const int b0 = (splitB < 0 || c < split) ? 0 : splitB;
  const int b1 = splitB < 0 ? rowsB : (c < split ? splitB : rowsB);
  for (int b = b0 + lane; b < b1; b += 32) s += B[(size_t)b * ncols + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

// y0 = z + a0 d, trial j: z + a0 2^-j d (Z0[i][col], column stride CPs).
template <typename Real>
__device__ void write_pass_points(DevSolver* sv, Real* Z0, double a0, bool with_dir) {
  const int r = sv->r, CPs = zstride(r + 1 + KTRIAL);
  for (int e = threadIdx.x & 31; e < (1 + KTRIAL) * r; e += 32) {  // warp 0
    const int j = e / r, i = e - j * r;
    const double a = with_dir ? ldexp(a0, -j) : 0.0;
    const double v = sv->z[i] + a * sv->d[i];
    const int col = j == 0 ? 0 : r + j;
    Z0[i * CPs + col] = (Real)v;
    if (sv->zd) sv->zd[i * CPs + col] = v;
  }
}

template <typename Real>
__global__ void solve_begin_kernel(DevSolver* sv, Real* Z0, int C, int eval_only) {
  const int r = sv->r;
  if (threadIdx.x == 0) {
    sv->status = -1;
    sv->iters = 0;
    sv->ls_trials = 0;
    sv->ls_iter = 0;
    sv->have_dir = 0;
    sv->final_pass = 0;
    sv->running = 1;
    sv->stall = 0;
    sv->passes = 0;
    sv->g_best = 1e300;
    sv->alpha_base = 1.0;
    sv->eval_only = eval_only;
    sv->hist_n = 0;
    sv->hist_head = 0;
    sv->pair_pending = 0;
    sv->gamma = 1.0;
    sv->tiny_steps = 0;
  }
  const int CPs = zstride(C);
  double* zd = sv->zd;
  for (int e = threadIdx.x; e < CPs * r; e += blockDim.x) {
    const int i = e / CPs, c = e - i * CPs;
    const double v = c >= C ? 0.0 : ((c == 0 || c > r) ? sv->z[i] : (i == c - 1 ? 1.0 : 0.0));
    Z0[e] = (Real)v;
    if (zd) zd[e] = v;
  }
}

// Warp-wide helpers (the select kernel is a single warp: no block barriers).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The select kernel works on a shared-memory copy of the solver state: one
// parallel load at entry and one parallel store at exit, so that the serial
// decision logic of lane 0 does not wait on global-memory round trips.
constexpr int SV_SCALAR_WORDS = (int)(offsetof(DevSolver, z) / sizeof(double));

constexpr int SEL_THREADS = 128;  // warp 0: solver state logic; all four warps: L D L^T

// FP64 reciprocal: an FP32 reciprocal estimate refined by two Newton steps
// y <- y (2 - d y) (quadratic convergence: about 2^-23 -> 2^-46 -> FP64
// rounding), a short chain of FP64 instructions on the factorisation's serial
// path (GB300 issues a warp-wide FP64 instruction in about 64 cycles per
// sub-partition).
__device__ __forceinline__ double reciprocal(double d) {
  if (!(fabs(d) > 1e-30 && fabs(d) < 1e30)) return 1.0 / d;
  double y = (double)__frcp_rn((float)d);
  y = y * fma(-d, y, 2.0);
  y = y * fma(-d, y, 2.0);
  return y;
}

// Right-looking L D L^T factorisation (unit lower L, positive diagonal D) of
// the symmetric matrix held in L (lower triangle used), all SEL_THREADS
// threads; the same pivots as Cholesky without its square roots.  Per column
// j: warp 0 takes the pivot d_j (lane 0: one reciprocal), keeps the column's
// unscaled entries in u and scales the column by 1 / d_j; after one block
// barrier every warp updates its rows of the trailing lower triangle
// (a_ik -= l_ij a_kj; row i by warp i mod 4, its columns by the lanes), then
// a second barrier.  On return L holds l_ij below the diagonal, d_j on it,
// and invd[j] = 1 / d_j.  Returns false (uniformly) when a pivot is not
// positive (the matrix is not positive definite).
__device__ bool block_ldlt(double (*L)[RMAX + 1], double* invd, double* u, int r,
                           int* s_fail) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  constexpr int NW = SEL_THREADS / 32;
  for (int j = 0; j < r; ++j) {
    if (warp == 0) {
      double inv = 0.0;
      int bad = 0;
      if (lane == 0) {
        const double djj = L[j][j];
        if (!(djj > 0.0)) {
          bad = 1;
        } else {
          inv = reciprocal(djj);
          invd[j] = inv;
        }
        *s_fail = bad;
      }
      bad = __shfl_sync(0xffffffffu, bad, 0);
      inv = __shfl_sync(0xffffffffu, inv, 0);
      if (!bad)
        for (int i = j + 1 + lane; i < r; i += 32) {
          const double a = L[i][j];
          u[i] = a;
          L[i][j] = a * inv;
        }
    }
    __syncthreads();
    if (*s_fail) return false;
    for (int i = j + 1 + warp; i < r; i += NW) {
      const double lij = L[i][j];
      for (int k = j + 1 + lane; k <= i; k += 32) L[i][k] -= lij * u[k];
    }
    __syncthreads();
  }
  return true;
}

// Line-search decision on the energies of the pass (lane 0 of warp 0):
// at_z = -2: the final re-evaluation at z is done; -1: keep backtracking
// along d (or a final pass at z is queued); 0: a shorter step was taken, the
// next pass evaluates at the new z; 1: the pass point y0 is the current z
// (sys holds E and g there).  stepped = 1 when a step was accepted.
__device__ void line_search_decide(DevSolver* sv, DevSolver* gsv, const double* sE,
                                   const double* sT, int& at_z, int& stepped) {
  at_z = 1;
  stepped = 0;
  sv->passes += 1;
  if (sv->final_pass) {
    sv->final_pass = 0;
    sv->running = 0;
    at_z = -2;
  } else if (sv->have_dir) {
    int acc = -1;
    for (int j = 0; j <= KTRIAL; ++j) {
      if (sv->ls_iter >= sv->max_ls) break;
      sv->ls_iter += 1;
      sv->ls_trials += 1;
      const double a = ldexp(sv->alpha_base, -j);
      const double Et = j == 0 ? sE[0] : sT[2 * (j - 1)];
      const double Ea = j == 0 ? sE[1] : sT[2 * (j - 1) + 1];
      const double eta = sv->eta_scale * (Ea + sv->Eabs);
      if (isfinite(Et) && Et <= sv->E + sv->armijo_c * a * sv->gd + eta) {
        acc = j;
        break;
      }
    }
    if (acc >= 0) {
      const double a = ldexp(sv->alpha_base, -acc);
      sv->alpha_taken = a;
      sv->tiny_steps = a < 0x1p-10 ? sv->tiny_steps + 1 : 0;
      if (sv->iters < TRACE) gsv->trace_alpha[sv->iters] = a;
      sv->iters += 1;
      sv->have_dir = 0;
      at_z = acc == 0 ? 1 : 0;
      stepped = 1;
    } else if (sv->ls_iter >= sv->max_ls) {
      sv->status = (sv->grad_inf < 100.0 * sv->tol) ? 4 : 2;  // PRECISION_FLOOR : LS_FAILED
      sv->have_dir = 0;
      sv->final_pass = 1;  // positions must be re-evaluated at z
      at_z = -1;
    } else {
      sv->alpha_base = ldexp(sv->alpha_base, -(KTRIAL + 1));
      at_z = -1;  // keep backtracking along d
    }
  }
}

// Exit tests at the current z (warp 0; lane 0 writes the state): records E,
// ||g||_inf, the rounding scale of g and the trace entry, updates the stall
// counter, and returns the solve's exit status or -1 to continue.  `finite`
// carries the caller's finiteness check of further data (the reduced
// Hessian); `saddle` is the L-BFGS curvature exit.
__device__ int gradient_exits(DevSolver* sv, DevSolver* gsv, const double* sE, const double* sg,
                              const double* sga, int r, bool finite, bool saddle) {
  const int t = threadIdx.x;
  double gm = 0.0, ga = 0.0;
  for (int i = t; i < r; i += 32) {
    const double gi = sg[i];
    gm = fmax(gm, fabs(gi));
    ga = fmax(ga, sga[i]);
    finite = finite && isfinite(gi);
  }
  const double ginf = __all_sync(0xffffffffu, finite) ? warp_max(gm) : -1.0;
  const double gabs_max = warp_max(ga);
  const double E = sE[0];
  int stall = 0;
  if (t == 0) {
    sv->E = E;
    sv->Eabs = sE[1];
    sv->grad_inf = ginf;
    sv->gabs_max = gabs_max;
    if (!sv->eval_only) {
      if (sv->iters < TRACE) {
        gsv->trace_g[sv->iters] = ginf;
        gsv->trace_E[sv->iters] = E;
        gsv->trace_gabs[sv->iters] = gabs_max;
        gsv->trace_alpha[sv->iters] = 0.0;
      }
      // stall counter: iterations since ||g||_inf last dropped by 10 %
      if (ginf <= 0.9 * sv->g_best) {
        sv->g_best = ginf;
        sv->stall = 0;
      } else {
        sv->stall += 1;
      }
    }
    stall = sv->stall;
  }
  stall = __shfl_sync(0xffffffffu, stall, 0);
  if (sv->eval_only) return 0;
  if (ginf < 0.0 || !isfinite(E)) return -3;                     // LSN_ERR_NONFINITE
  if (ginf < sv->tol) return 0;                                  // LSN_OK
  if (saddle) return 5;                                          // LSN_SADDLE
  if (stall >= 4 && ginf <= sv->floor_scale * gabs_max) return 4;  // PRECISION_FLOOR
  // reduced-precision forms: the line search keeps accepting only tiny steps
  // (the energy or the reduced Hessian is resolved no better than this)
  if (sv->eta_scale > 0.0 && stall >= 4 && sv->tiny_steps >= 4 && ginf < 100.0 * sv->tol)
    return 4;
  if (sv->iters >= sv->max_newton) return 1;                     // LSN_NOT_CONVERGED
  return -1;
}

// Warp-0 state logic around a block-wide FP64 L D L^T (SEL_THREADS threads,
// one CTA): the line-search decision on the trial energies of the pass, the
// exit tests, and (when a new direction is due) d = -K^-1 g with diagonal
// shifts on failure, then the points of the next pass.
template <typename Real>
__global__ void __launch_bounds__(SEL_THREADS) select_direction_kernel(
    DevSolver* gsv, const double* __restrict__ sys, Real* Z0, unsigned long long cond,
    int use_cond) {
  __shared__ double L[RMAX][RMAX + 1];
  __shared__ double y[RMAX];
  __shared__ double invd[RMAX];  // reciprocals of the L D L^T diagonal
  __shared__ double ucol[RMAX];  // unscaled column of the factorisation step
  __shared__ double ssys[4 * RMAX + 2 * KTRIAL + 2];
  __shared__ __align__(16) DevSolver svs;
  __shared__ int s_need, s_fail;
  __shared__ double s_base;
  DevSolver* sv = &svs;
  const int t = threadIdx.x;
  pdl_wait();
  // ---- parallel load of the state (scalars, z, d) and of E, g, gabs, trials
  {
    const double* src = reinterpret_cast<const double*>(gsv);
    double* dst = reinterpret_cast<double*>(&svs);
    for (int e = t; e < SV_SCALAR_WORDS + 2 * RMAX; e += SEL_THREADS) dst[e] = src[e];
  }
  if (t == 0) s_need = 0;
  __syncthreads();
  const int r = sv->r;
  const int tslot = nslots(r);
  const double* Ku = sys + slot_K(r);
  for (int e = t; e < 2 + 2 * r; e += SEL_THREADS) ssys[e] = sys[e];
  for (int e = t; e < 2 * KTRIAL; e += SEL_THREADS) ssys[2 + 2 * r + e] = sys[tslot + e];
  // K into L (needed only when a direction is computed; issued early)
  for (int e = t; e < r * r; e += SEL_THREADS) {
    const int i = e / r, j = e - i * r;
    L[i][j] = i <= j ? Ku[upper_index(i, j, r)] : Ku[upper_index(j, i, r)];
  }
  __syncthreads();
  int status = -1;
  bool want_cond = true;
  int cond_val = 1;
  if (t < 32) {
    const double* sE = ssys;                    // E, Eabs at y0
    const double* sg = ssys + 2;                // g
    const double* sga = ssys + 2 + r;           // gabs
    const double* sT = ssys + 2 + 2 * r;        // trial (E_j, Eabs_j)
    // ------------------------------------------------ line-search decision
    int at_z = 1, stepped = 0;
    if (t == 0) line_search_decide(sv, gsv, sE, sT, at_z, stepped);
    at_z = __shfl_sync(0xffffffffu, at_z, 0);
    stepped = __shfl_sync(0xffffffffu, stepped, 0);
    __syncwarp();
    if (stepped) {  // a step was taken: z += alpha d
      for (int i = t; i < r; i += 32) sv->z[i] += sv->alpha_taken * sv->d[i];
      __syncwarp();
    }
    if (at_z == -2) {  // the final re-evaluation at z is done
      cond_val = 0;
    } else if (at_z == -1) {
      write_pass_points<Real>(sv, Z0, sv->alpha_base, sv->status == -1);
      if (t == 0) sv->running = 1;
    } else if (at_z == 0) {  // a shorter step was taken: evaluate at the new z next
      write_pass_points<Real>(sv, Z0, 0.0, false);
    } else {
      // ------------------------------------------- sys holds E, g, K at z
      bool finite = true;
      for (int i = t; i < r; i += 32) y[i] = -sg[i];
      for (int e = t; e < r * r; e += 32) finite = finite && isfinite(L[e / r][e % r]);
      status = gradient_exits(sv, gsv, sE, sg, sga, r, finite, false);
      if (status != -1) {
        if (t == 0) {
          if (!sv->eval_only) sv->status = status;
          sv->running = 0;
        }
        cond_val = 0;
      } else {
        // a new direction is due: factorised below by all four warps
        double dm = 0.0;
        for (int i = t; i < r; i += 32) dm = fmax(dm, fabs(L[i][i]));
        const double base = 1e-12 * fmax(1.0, warp_max(dm));
        if (t == 0) {
          s_base = base;
          s_need = 1;
        }
      }
    }
    for (int i = t; i < r; i += 32) gsv->g[i] = sg[i];
  }
  __syncthreads();
  if (s_need) {
    // K + shift I = L D L^T, shift = 0, then 1e-12 max(1, max|K_ii|) x 10^k
    double shift = 0.0;
    bool ok = false;
    for (int attempt = 0; attempt < 21 && !ok; ++attempt) {
      if (attempt > 0) {
        for (int e = t; e < r * r; e += SEL_THREADS) {
          const int i = e / r, j = e - i * r;
          L[i][j] = (i <= j ? Ku[upper_index(i, j, r)] : Ku[upper_index(j, i, r)]) +
                    (i == j ? shift : 0.0);
        }
        __syncthreads();
      }
      ok = block_ldlt(L, invd, ucol, r, &s_fail);
      if (!ok) shift = shift == 0.0 ? s_base : shift * 10.0;
      __syncthreads();
    }
    if (t < 32) {
      const double* sg = ssys + 2;
      if (!ok) {
        if (t == 0) {
          sv->status = 3;  // LSN_NOT_SPD
          sv->running = 0;
        }
        cond_val = 0;
      } else {
        // forward L y = -g (unit lower), y <- D^-1 y, backward L^T d = y (unit
        // upper): column sweeps within warp 0
        for (int i = 0; i < r; ++i) {
          const double yi = y[i];
          for (int k = i + 1 + t; k < r; k += 32) y[k] -= L[k][i] * yi;
          __syncwarp();
        }
        for (int i = t; i < r; i += 32) y[i] *= invd[i];
        __syncwarp();
        for (int i = r - 1; i >= 0; --i) {
          const double yi = y[i];
          for (int k = t; k < i; k += 32) y[k] -= L[i][k] * yi;
          __syncwarp();
        }
        double gd = 0.0;
        for (int i = t; i < r; i += 32) {
          sv->d[i] = y[i];
          gd += sg[i] * y[i];
        }
        gd = warp_sum(gd);
        if (t == 0) {
          sv->gd = gd;
          sv->alpha_base = 1.0;
          sv->ls_iter = 0;
          sv->have_dir = 1;
          sv->running = 1;
        }
        __syncwarp();
        write_pass_points<Real>(sv, Z0, 1.0, true);
      }
    }
  }
  // ---- parallel store of the state
  __syncthreads();
  {
    const double* src = reinterpret_cast<const double*>(&svs);
    double* dst = reinterpret_cast<double*>(gsv);
    for (int e = t; e < SV_SCALAR_WORDS + 2 * RMAX; e += SEL_THREADS) dst[e] = src[e];
  }
  if (want_cond && use_cond && t == 0) cudaGraphSetConditional(cond, cond_val);
}

// L-BFGS state logic (Sec. 5: the optimiser of the main results, exits I-IV).
// The same passes, line search and exit tests as the Newton solve; the
// direction is d = -H g by the two-loop recursion (Nocedal & Wright,
// Algorithm 7.4) over the hist_n most recent curvature pairs, H0 = gamma I
// with gamma = s^T y / y^T y of the newest pair (1 while the history is
// empty).  The pair of an accepted step, s = alpha d and y = g(z + s) - g(z),
// is formed at the next gradient at z; s^T y <= 0 (no positive curvature
// along the step) ends the solve with exit II, LSN_SADDLE, unless that
// gradient already meets the tolerance.  A direction that is not a descent
// direction in rounding (g.d >= 0) restarts from d = -g with an empty history.
// The history is staged in shared memory by all SEL_THREADS threads; the
// logic and the recursion run in warp 0 (FP64, lanes own entries i, i + 32).
template <typename Real>
__global__ void __launch_bounds__(SEL_THREADS) select_lbfgs_kernel(
    DevSolver* gsv, DevHistory* gh, const double* __restrict__ sys, Real* Z0,
    unsigned long long cond, int use_cond) {
  __shared__ double hS[MHIST][RMAX], hY[MHIST][RMAX];
  __shared__ double hrho[MHIST], ha[MHIST];
  __shared__ double sgz[RMAX];
  __shared__ double ssys[2 + 2 * RMAX + 2 * KTRIAL];
  __shared__ __align__(16) DevSolver svs;
  DevSolver* sv = &svs;
  const int t = threadIdx.x;
  pdl_wait();
  {
    const double* src = reinterpret_cast<const double*>(gsv);
    double* dst = reinterpret_cast<double*>(&svs);
    for (int e = t; e < SV_SCALAR_WORDS + 2 * RMAX; e += SEL_THREADS) dst[e] = src[e];
  }
  __syncthreads();
  const int r = sv->r, m = sv->hist_m, hn = sv->hist_n, head = sv->hist_head;
  const int tslot = nslots(r);
  for (int e = t; e < 2 + 2 * r; e += SEL_THREADS) ssys[e] = sys[e];
  for (int e = t; e < 2 * KTRIAL; e += SEL_THREADS) ssys[2 + 2 * r + e] = sys[tslot + e];
  for (int e = t; e < hn * r; e += SEL_THREADS) {
    const int k = e / r, i = e - k * r, slot = (head + k) % m;
    hS[slot][i] = gh->S[slot][i];
    hY[slot][i] = gh->Y[slot][i];
  }
  for (int k = t; k < hn; k += SEL_THREADS) hrho[(head + k) % m] = gh->rho[(head + k) % m];
  for (int i = t; i < r; i += SEL_THREADS) sgz[i] = gh->gz[i];
  __syncthreads();
  int cond_val = 1;
  if (t < 32) {
    const double* sE = ssys;
    const double* sg = ssys + 2;
    const double* sga = ssys + 2 + r;
    const double* sT = ssys + 2 + 2 * r;
    int at_z = 1, stepped = 0;
    if (t == 0) line_search_decide(sv, gsv, sE, sT, at_z, stepped);
    at_z = __shfl_sync(0xffffffffu, at_z, 0);
    stepped = __shfl_sync(0xffffffffu, stepped, 0);
    __syncwarp();
    if (stepped) {  // z += alpha d; the pair is formed at the gradient of the new z
      for (int i = t; i < r; i += 32) sv->z[i] += sv->alpha_taken * sv->d[i];
      if (t == 0) sv->pair_pending = 1;
      __syncwarp();
    }
    if (at_z == -2) {
      cond_val = 0;
    } else if (at_z == -1) {
      write_pass_points<Real>(sv, Z0, sv->alpha_base, sv->status == -1);
      if (t == 0) sv->running = 1;
    } else if (at_z == 0) {
      write_pass_points<Real>(sv, Z0, 0.0, false);
    } else {
      // ------------------------------------------- sys holds E, g at z
      bool saddle = false;
      const int i0 = t, i1 = t + 32;
      if (!sv->eval_only) {
        if (sv->pair_pending) {
          const double a = sv->alpha_taken;
          const double s0 = i0 < r ? a * sv->d[i0] : 0.0, s1 = i1 < r ? a * sv->d[i1] : 0.0;
          const double y0 = i0 < r ? sg[i0] - sgz[i0] : 0.0;
          const double y1 = i1 < r ? sg[i1] - sgz[i1] : 0.0;
          const double sy = warp_sum(s0 * y0 + s1 * y1);
          const double yy = warp_sum(y0 * y0 + y1 * y1);
          if (sy > 0.0 && isfinite(sy) && isfinite(yy)) {
            const int slot = hn < m ? (head + hn) % m : head;
            if (i0 < r) {
              hS[slot][i0] = s0; hY[slot][i0] = y0;
              gh->S[slot][i0] = s0; gh->Y[slot][i0] = y0;
            }
            if (i1 < r) {
              hS[slot][i1] = s1; hY[slot][i1] = y1;
              gh->S[slot][i1] = s1; gh->Y[slot][i1] = y1;
            }
            if (t == 0) {
              hrho[slot] = 1.0 / sy;
              gh->rho[slot] = 1.0 / sy;
              if (hn < m) sv->hist_n = hn + 1;
              else sv->hist_head = (head + 1) % m;
              sv->gamma = sy / yy;
            }
          } else {
            saddle = true;
          }
          if (t == 0) sv->pair_pending = 0;
        }
        for (int i = t; i < r; i += 32) gh->gz[i] = sg[i];
      }
      __syncwarp();
      const int status = gradient_exits(sv, gsv, sE, sg, sga, r, true, saddle);
      if (status != -1) {
        if (t == 0) {
          if (!sv->eval_only) sv->status = status;
          sv->running = 0;
        }
        cond_val = 0;
      } else {
        // two-loop recursion: q = g; newest to oldest a_k = rho_k s_k.q,
        // q -= a_k y_k; q *= gamma; oldest to newest b = rho_k y_k.q,
        // q += (a_k - b) s_k; d = -q
        const int n2 = sv->hist_n, h2 = sv->hist_head;
        double q0 = i0 < r ? sg[i0] : 0.0, q1 = i1 < r ? sg[i1] : 0.0;
        for (int k = n2 - 1; k >= 0; --k) {
          const int slot = (h2 + k) % m;
          const double sk0 = i0 < r ? hS[slot][i0] : 0.0, sk1 = i1 < r ? hS[slot][i1] : 0.0;
          const double ak = hrho[slot] * warp_sum(sk0 * q0 + sk1 * q1);
          if (t == 0) ha[k] = ak;
          if (i0 < r) q0 -= ak * hY[slot][i0];
          if (i1 < r) q1 -= ak * hY[slot][i1];
        }
        __syncwarp();
        const double gm = n2 > 0 ? sv->gamma : 1.0;
        q0 *= gm;
        q1 *= gm;
        for (int k = 0; k < n2; ++k) {
          const int slot = (h2 + k) % m;
          const double yk0 = i0 < r ? hY[slot][i0] : 0.0, yk1 = i1 < r ? hY[slot][i1] : 0.0;
          const double b = hrho[slot] * warp_sum(yk0 * q0 + yk1 * q1);
          const double c = ha[k] - b;
          if (i0 < r) q0 += c * hS[slot][i0];
          if (i1 < r) q1 += c * hS[slot][i1];
        }
        const double g0 = i0 < r ? sg[i0] : 0.0, g1 = i1 < r ? sg[i1] : 0.0;
        double gd = -warp_sum(g0 * q0 + g1 * q1);
        if (!(gd < 0.0)) {  // not a descent direction in rounding: restart
          q0 = g0;
          q1 = g1;
          gd = -warp_sum(g0 * g0 + g1 * g1);
          if (t == 0) {
            sv->hist_n = 0;
            sv->hist_head = 0;
          }
        }
        if (i0 < r) sv->d[i0] = -q0;
        if (i1 < r) sv->d[i1] = -q1;
        if (t == 0) {
          sv->gd = gd;
          sv->alpha_base = 1.0;
          sv->ls_iter = 0;
          sv->have_dir = 1;
          sv->running = 1;
        }
        __syncwarp();
        write_pass_points<Real>(sv, Z0, 1.0, true);
      }
    }
    for (int i = t; i < r; i += 32) gsv->g[i] = sg[i];
  }
  __syncthreads();
  {
    const double* src = reinterpret_cast<const double*>(&svs);
    double* dst = reinterpret_cast<double*>(gsv);
    for (int e = t; e < SV_SCALAR_WORDS + 2 * RMAX; e += SEL_THREADS) dst[e] = src[e];
  }
  if (use_cond && t == 0) cudaGraphSetConditional(cond, cond_val);
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

__global__ void begin_step_kernel(const double* __restrict__ X0,
                                  const double* __restrict__ q,
                                  const double* __restrict__ v, int n, double dt,
                                  double gx, double gy, double gz,
                                  double* __restrict__ ubar, DevSolver* sv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) sv->inv_dt2 = dt > 0.0 ? 1.0 / (dt * dt) : 0.0;
  if (i >= n || !(dt > 0.0) || q == nullptr) return;
  const int c = i % 3;
  const double g = c == 0 ? gx : (c == 1 ? gy : gz);
  ubar[i] = (q[i] - X0[i]) + dt * v[i] + dt * dt * g;
}

}  // namespace

void launch_reduce_partials(const double* A, int rowsA, const double* B, int rowsB,
                            int splitB, int split, int ncols, double* out, cudaStream_t s,
                            int gap0, int gapn) {
  const int threads = 256, warps = threads / 32;
  launch_pdl(reduce_partials_kernel, dim3((ncols - gapn + warps - 1) / warps), dim3(threads), 0,
             s, A, rowsA, B, rowsB, splitB, split, ncols, out, gap0, gapn);
}

template <typename Real>
void launch_solve_begin(DevSolver* sv, Real* Z0, int C, int eval_only, cudaStream_t s) {
  solve_begin_kernel<Real><<<1, 256, 0, s>>>(sv, Z0, C, eval_only);
}

template <typename Real>
void launch_select_direction(DevSolver* sv, const double* sys, Real* Z0,
                             unsigned long long cond, int use_cond, cudaStream_t s) {
  launch_pdl(select_direction_kernel<Real>, dim3(1), dim3(SEL_THREADS), 0, s, sv, sys, Z0, cond,
             use_cond);
}

template <typename Real>
void launch_select_lbfgs(DevSolver* sv, DevHistory* hist, const double* sys, Real* Z0,
                         unsigned long long cond, int use_cond, cudaStream_t s) {
  launch_pdl(select_lbfgs_kernel<Real>, dim3(1), dim3(SEL_THREADS), 0, s, sv, hist, sys, Z0,
             cond, use_cond);
}

template <typename Real>
void launch_finish_positions(const double* X0, const Real* u, int n, double dt, double* q,
                             double* v, cudaStream_t s) {
  finish_positions_kernel<Real><<<(n + 255) / 256, 256, 0, s>>>(X0, u, n, dt, q, v);
}

void launch_begin_step(const double* X0, const double* q, const double* v, int n, double dt,
                       const double* g, double* ubar, DevSolver* sv, cudaStream_t s) {
  begin_step_kernel<<<(n + 255) / 256, 256, 0, s>>>(X0, q, v, n, dt, g[0], g[1], g[2], ubar,
                                                    sv);
}

#define LSN_INST(R)                                                                      \
  template void launch_solve_begin<R>(DevSolver*, R*, int, int, cudaStream_t);           \
  template void launch_select_direction<R>(DevSolver*, const double*, R*,                \
                                           unsigned long long, int, cudaStream_t);       \
  template void launch_select_lbfgs<R>(DevSolver*, DevHistory*, const double*, R*,       \
                                       unsigned long long, int, cudaStream_t);           \
  template void launch_finish_positions<R>(const double*, const R*, int, double,         \
                                           double*, double*, cudaStream_t);
LSN_INST(float)
LSN_INST(double)
#undef LSN_INST

}  // namespace lsn
