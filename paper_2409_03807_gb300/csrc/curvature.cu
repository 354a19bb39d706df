// Exact-form reduced Hessian (opt-in, lsn_set_exact_hessian): the term that
// the Gauss-Newton reduced Hessian leaves out, differentiating Eq. 2 twice,
//
//   C(z) = sum_{k free} dE/dx_k d2x_k/dz2 = s sum_j v_j d2h_j/dz2,
//   v = W_L^T G,   G_k = dE/dx_k on the free DOFs (0 on the constrained ones),
//
// with h the last hidden layer of the decoder and x = X0 + s (W_L h + b_L),
// added to K at the pass point, and the projection of the r x r sum: its
// eigenvalues below clamp * max |eigenvalue| raised to that value.
//
// Steps (one chain per evaluation pass, after the partial rows are reduced):
//   1. tet_forces_kernel   per cubature tet, the weighted elastic forces at u
//   2. full_gradient_kernel per vertex, those forces gathered over the
//      cubature slots touching it, in slot order (no atomics), plus the
//      per-DOF terms (inertia or gravity, ground penalty); zero on
//      constrained vertices
//   3. wtv_kernel / wtv_reduce_kernel  v = s W_L^T G, per-CTA partial sums
//      over row chunks added in CTA order
//   4. per hidden layer: A = W_l Y_{l-1} (tensor-core TF32 GEMM in the
//      tensor-core forms, a tiled CUDA-core GEMM otherwise), then
//      act2_kernel: Y_l = [h | T | U] with the forward tangents
//      T = e1 (W T), U_cd = e2 (W T)_c (W T)_d + e1 (W U)_cd
//      (e1, e2 the ELU derivatives at a = W h + b); Y_0 = [z | I | 0]
//   5. contract_kernel  C_cd = sum_j v_j U_j,cd, added to K in the system row
//   6. project_kernel   one CTA, FP64: an L D L^T attempt on K - clamp ||K||_F I
//      first (when it succeeds every eigenvalue is above f = clamp max |lambda|
//      and K is left as it is); otherwise cyclic Jacobi (parallel round-robin
//      pairs) on the r x r K, then K += sum_{lambda_i < f} (f - lambda_i) q_i q_i^T
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "element_math.cuh"
#include "lsn_internal.cuh"

namespace lsn {
namespace {

template <typename Real>
__global__ void tet_forces_kernel(ElemArgs ea, const Real* __restrict__ u, Real* __restrict__ F) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ea.S) return;
  int4 tv;
  Real Dmi[3][3], wv, H[3][3], ge[12];
  load_tet<Real>(ea, e, tv, Dmi, wv);
  disp_grad<Real>(u, tv, Dmi, H);
  snh_tet_forces<Real>(H, Dmi, wv, (Real)ea.mu, (Real)ea.lam, ge);
#pragma unroll
  for (int k = 0; k < 12; ++k) F[(size_t)e * 12 + k] = ge[k];
}

// G[3 v + i] on the free vertices; ventry[vptr[v] ..] = 4 slot + local
// vertex of every cubature slot touching v, in slot order
template <typename Real>
__global__ void full_gradient_kernel(int nv, const int* __restrict__ vptr,
                                     const int* __restrict__ ventry,
                                     const Real* __restrict__ F, const Real* __restrict__ u,
                                     LastArgs la, Real* __restrict__ G) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  if (la.cslot[v] >= 0) {
    G[3 * v] = G[3 * v + 1] = G[3 * v + 2] = Real(0);
    return;
  }
  double acc[3] = {0.0, 0.0, 0.0};
  for (int k = vptr[v]; k < vptr[v + 1]; ++k) {
    const int ent = ventry[k];
    const Real* f = F + (size_t)(ent >> 2) * 12 + 3 * (ent & 3);
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] += (double)f[i];
  }
  const double inv_dt2 = *la.inv_dt2, mv = la.mass[v];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int m = 3 * v + i;
    double gv = inv_dt2 > 0.0 ? inv_dt2 * mv * ((double)u[m] - la.ubar[m]) : -mv * la.grav[i];
    if (la.ground_k > 0.0 && i == 2) {
      const double pen = la.X0[m] + (double)u[m] - la.ground_h;
      if (pen < 0.0) gv += la.ground_k * pen;
    }
    G[m] = (Real)(acc[i] + gv);
  }
}

constexpr int WTV_THREADS = 256;
constexpr int WTV_ROWS = 128;  // rows of W_L per CTA

__device__ __forceinline__ float wval(__nv_bfloat16 w) { return __bfloat162float(w); }
__device__ __forceinline__ float wval(float w) { return w; }
__device__ __forceinline__ double wval(double w) { return w; }

// part[b][j] = sum over rows m of chunk b of W[m][j] G[m] (in the element
// precision within a chunk, FP64 across chunks); W is the output layer's
// weights as the output layer reads them (the BF16 copy in the BF16 form)
template <typename Real, typename WT>
__global__ void wtv_kernel(const WT* __restrict__ W, const Real* __restrict__ G, int n, int H,
                           double* __restrict__ part) {
  const int m0 = blockIdx.x * WTV_ROWS, m1 = min(n, m0 + WTV_ROWS);
  for (int j = threadIdx.x; j < H; j += WTV_THREADS) {
    // four interleaved partial sums (independent FMA chains), added in order
    Real a0 = Real(0), a1 = Real(0), a2 = Real(0), a3 = Real(0);
    int m = m0;
    for (; m + 4 <= m1; m += 4) {
      a0 += (Real)wval(W[(size_t)m * H + j]) * G[m];
      a1 += (Real)wval(W[(size_t)(m + 1) * H + j]) * G[m + 1];
      a2 += (Real)wval(W[(size_t)(m + 2) * H + j]) * G[m + 2];
      a3 += (Real)wval(W[(size_t)(m + 3) * H + j]) * G[m + 3];
    }
    for (; m < m1; ++m) a0 += (Real)wval(W[(size_t)m * H + j]) * G[m];
    part[(size_t)blockIdx.x * H + j] = (double)((a0 + a1) + (a2 + a3));
  }
}

// v[j] = s sum_b part[b][j]: one warp per j, lanes over the chunks, then a
// fixed shuffle tree (the order does not depend on scheduling)
template <typename Real>
__global__ void wtv_reduce_kernel(const double* __restrict__ part, int nb, int H, double s,
                                  Real* __restrict__ v) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= H) return;
  double acc = 0.0;
  for (int b = lane; b < nb; b += 32) acc += part[(size_t)b * H + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) v[j] = (Real)(s * acc);
}

// pair index p (c <= d, row-major upper triangle of an rn x rn matrix) -> (c, d)
__device__ __forceinline__ void pair_of(int p, int rn, int& c, int& d) {
  c = 0;
  while (p >= rn - c) {
    p -= rn - c;
    ++c;
  }
  d = c + p;
}

// Y_0 = [z | I | 0] (rows: the rn network coordinates, NY columns)
template <typename Real>
__global__ void y0_kernel(const Real* __restrict__ Z0, int cps, int rn, int NY,
                          Real* __restrict__ Y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rn * NY) return;
  const int k = e / NY, col = e - k * NY;
  Real v = Real(0);
  if (col == 0) v = Z0[(size_t)k * cps];
  else if (col <= rn) v = (col - 1 == k) ? Real(1) : Real(0);
  Y[e] = v;
}

// C[M][N] = A[M][K] B[K][N], all row-major (CUDA-core forms)
template <typename Real>
__global__ void gemm_rm_kernel(int M, int N, int K, const Real* __restrict__ A,
                               const Real* __restrict__ B, Real* __restrict__ C) {
  __shared__ Real As[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  Real acc = Real(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    As[ty][tx] = (row < M && k0 + tx < K) ? A[(size_t)row * K + k0 + tx] : Real(0);
    Bs[ty][tx] = (k0 + ty < K && col < N) ? B[(size_t)(k0 + ty) * N + col] : Real(0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += As[ty][k] * Bs[k][tx];
    __syncthreads();
  }
  if (row < M && col < N) C[(size_t)row * N + col] = acc;
}

// Y_l from A = W_l Y_{l-1}: ELU and its first and second derivative at a
template <typename Real>
__global__ void act2_kernel(const Real* __restrict__ A, const Real* __restrict__ b, int M,
                            int rn, int NY, Real* __restrict__ Y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * NY) return;
  const int i = e / NY, col = e - i * NY;
  const Real* Ai = A + (size_t)i * NY;
  const Real a = Ai[0] + b[i];
  const bool pos = a > Real(0);
  const Real ex = pos ? Real(1) : exp(a);  // e1 = e2 = exp(a) for a <= 0
  const Real e1 = ex, e2 = pos ? Real(0) : ex;
  Real v;
  if (col == 0) {
    v = pos ? a : expm1(a);
  } else if (col <= rn) {
    v = e1 * Ai[col];
  } else {
    int c, d;
    pair_of(col - 1 - rn, rn, c, d);
    v = e2 * Ai[1 + c] * Ai[1 + d] + e1 * Ai[col];
  }
  Y[e] = v;
}

constexpr int CON_WARPS = 8;

// sys K slots (c <= d < rn, in the r x r upper triangle) += sum_j v_j U_j,cd:
// a CTA takes 32 pairs (one per lane); its warps split j into CON_WARPS
// ranges (element precision within a range), summed in FP64 in warp order
template <typename Real>
__global__ void contract_kernel(const Real* __restrict__ Y, const Real* __restrict__ v, int H,
                                int rn, int NY, int r, double* __restrict__ sys) {
  __shared__ double red[CON_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  const int P = rn * (rn + 1) / 2;
  const int j0 = (H * w) / CON_WARPS, j1 = (H * (w + 1)) / CON_WARPS;
  Real a0 = Real(0), a1 = Real(0);
  if (p < P) {
    const Real* y = Y + 1 + rn + p;
    int j = j0;
    for (; j + 2 <= j1; j += 2) {
      a0 += v[j] * y[(size_t)j * NY];
      a1 += v[j + 1] * y[(size_t)(j + 1) * NY];
    }
    for (; j < j1; ++j) a0 += v[j] * y[(size_t)j * NY];
  }
  red[w][lane] = (double)a0 + (double)a1;
  __syncthreads();
  if (w == 0 && p < P) {
    double acc = 0.0;
    for (int k = 0; k < CON_WARPS; ++k) acc += red[k][lane];
    int c, d;
    pair_of(p, rn, c, d);
    sys[slot_K(r) + c * r - (c * (c - 1)) / 2 + (d - c)] += acc;
  }
}

constexpr int PROJ_THREADS = 256;
constexpr int PROJ_SWEEPS = 30;
// Jacobi stops once the off-diagonal part is below (64 u)^2 of the squared
// Frobenius norm, or stops shrinking (it stalls at the rounding level)
constexpr double PROJ_OFF_REL = 1.9e-25;

// The r x r K of the system row, eigen-decomposed by cyclic Jacobi (parallel
// round-robin ordering, disjoint rotations per round) in FP64; eigenvalues
// below f = clamp * max |lambda| raised to f by adding (f - lambda_i) q_i q_i^T.
__global__ void __launch_bounds__(PROJ_THREADS) project_kernel(double* __restrict__ sys, int r,
                                                               double clamp) {
  extern __shared__ double sm[];
  const int m = r + (r & 1);  // even number of indices (a dummy when r is odd)
  const int ld = m + 1;
  double* A = sm;                  // m x ld
  double* V = A + (size_t)m * ld;  // m x ld
  double* cs = V + (size_t)m * ld; // m / 2 cosines, then m / 2 sines
  double* sn = cs + m / 2;
  int* pp = reinterpret_cast<int*>(sn + m / 2);
  int* qq = pp + m / 2;
  __shared__ double red[PROJ_THREADS / 32];
  __shared__ double s_off, s_tot;
  const int t = threadIdx.x;
  const double* K = sys + slot_K(r);
  for (int e = t; e < m * m; e += PROJ_THREADS) {
    const int i = e / m, j = e - i * m;
    double a = 0.0;
    if (i < r && j < r) {
      const int c = min(i, j), d = max(i, j);
      a = K[c * r - (c * (c - 1)) / 2 + (d - c)];
    }
    A[i * ld + j] = a;
    V[i * ld + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  auto block_sum = [&](double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((t & 31) == 0) red[t >> 5] = x;
    __syncthreads();
    double s = 0.0;
    if (t == 0)
      for (int w = 0; w < PROJ_THREADS / 32; ++w) s += red[w];
    __syncthreads();
    return s;  // valid in thread 0
  };
  // L D L^T attempt on K - f' I with f' = clamp ||K||_F >= f (on a copy in
  // V): when it succeeds every eigenvalue is above f and the projection is
  // the identity, so K stays as it is
  {
    __shared__ int s_bad;
    __shared__ double s_fp;
    double sq = 0.0;
    for (int e = t; e < m * m; e += PROJ_THREADS) {
      const int i = e / m, j = e - i * m;
      const double a = A[i * ld + j];
      V[i * ld + j] = a;
      sq += a * a;
    }
    sq = block_sum(sq);
    if (t == 0) {
      s_bad = 0;
      s_fp = clamp * sqrt(sq);
    }
    __syncthreads();
    for (int j = t; j < r; j += PROJ_THREADS) V[j * ld + j] -= s_fp;
    __syncthreads();
    // L D L^T pivots (positive definite iff every pivot is positive); the
    // unscaled column j is kept in cs (free until the Jacobi rounds)
    __shared__ double s_inv;
    for (int j = 0; j < r; ++j) {
      if (t == 0) {
        const double pv = V[j * ld + j];
        if (!(pv > 0.0)) s_bad = 1;
        else s_inv = 1.0 / pv;
      }
      __syncthreads();
      if (s_bad) break;
      const double inv = s_inv;
      for (int i = j + 1 + t; i < r; i += PROJ_THREADS) {
        const double a = V[i * ld + j];
        cs[i] = a;
        V[i * ld + j] = a * inv;
      }
      __syncthreads();
      const int rem = r - j - 1;
      for (int e = t; e < rem * rem; e += PROJ_THREADS) {
        const int i = j + 1 + e / rem, k = j + 1 + e % rem;
        if (k <= i) V[i * ld + k] -= V[i * ld + j] * cs[k];
      }
      __syncthreads();
    }
    if (!s_bad) return;
    for (int e = t; e < m * m; e += PROJ_THREADS) {
      const int i = e / m, j = e - i * m;
      V[i * ld + j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  double prev_off = -1.0;
  for (int sweep = 0; sweep < PROJ_SWEEPS; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = t; e < m * m; e += PROJ_THREADS) {
      const int i = e / m, j = e - i * m;
      const double a = A[i * ld + j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    off = block_sum(off);
    tot = block_sum(tot);
    if (t == 0) {
      s_off = off;
      s_tot = tot;
    }
    __syncthreads();
    if (!(s_off > PROJ_OFF_REL * s_tot)) break;
    // stalled at the rounding level
    if (prev_off >= 0.0 && s_off < 1e-20 * s_tot && !(s_off < 0.5 * prev_off)) break;
    prev_off = s_off;
    for (int round = 0; round < m - 1; ++round) {
      // round-robin pairs: index 0 fixed, the others rotate by `round`
      if (t < m / 2) {
        const int a0 = t == 0 ? 0 : 1 + (t - 1 + round) % (m - 1);
        const int b0 = 1 + (m - 2 - t + round) % (m - 1);
        const int p = min(a0, b0), q = max(a0, b0);
        pp[t] = p;
        qq[t] = q;
        const double apq = A[p * ld + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double th = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
          const double tn = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          c = 1.0 / sqrt(tn * tn + 1.0);
          s = tn * c;
        }
        cs[t] = c;
        sn[t] = s;
      }
      __syncthreads();
      for (int e = t; e < (m / 2) * m; e += PROJ_THREADS) {  // rows p, q
        const int i = e / m, k = e - i * m;
        const int p = pp[i], q = qq[i];
        const double c = cs[i], s = sn[i], ap = A[p * ld + k], aq = A[q * ld + k];
        A[p * ld + k] = c * ap - s * aq;
        A[q * ld + k] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = t; e < (m / 2) * m; e += PROJ_THREADS) {  // columns p, q; V
        const int i = e / m, k = e - i * m;
        const int p = pp[i], q = qq[i];
        const double c = cs[i], s = sn[i];
        const double ap = A[k * ld + p], aq = A[k * ld + q];
        A[k * ld + p] = c * ap - s * aq;
        A[k * ld + q] = s * ap + c * aq;
        const double vp = V[k * ld + p], vq = V[k * ld + q];
        V[k * ld + p] = c * vp - s * vq;
        V[k * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // floor f = clamp * max |lambda| over the r true eigenvalues
  __shared__ double s_f;
  if (t < 32) {
    double mx = 0.0;
    for (int i = t; i < r; i += 32) mx = fmax(mx, fabs(A[i * ld + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (t == 0) s_f = clamp * mx;
  }
  __syncthreads();
  const double f = s_f;
  double* Kw = sys + slot_K(r);
  for (int e = t; e < r * r; e += PROJ_THREADS) {
    const int c = e / r, d = e - c * r;
    if (d < c) continue;
    double add = 0.0;
    for (int i = 0; i < r; ++i) {
      // the dummy index of an odd r carries eigenvalue 0 on a zero row
      const double lam_i = A[i * ld + i];
      if (lam_i < f) add += (f - lam_i) * V[c * ld + i] * V[d * ld + i];
    }
    Kw[c * r - (c * (c - 1)) / 2 + (d - c)] += add;
  }
}

}  // namespace

template <typename Real>
cudaError_t Curvature<Real>::setup(const CurvView& cv) {
  release();
  v = cv;
  rn = v.widths[0];
  NY = 1 + rn + rn * (rn + 1) / 2;
  int hmax = rn;
  for (int l = 1; l < (int)v.widths.size() - 1; ++l) hmax = std::max(hmax, v.widths[l]);
  Hl = v.widths[v.widths.size() - 2];
  nb = (v.n + WTV_ROWS - 1) / WTV_ROWS;
  cudaError_t e;
  auto get = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  };
  e = cudaSuccess;
  get(reinterpret_cast<void**>(&F), sizeof(Real) * 12 * (size_t)v.S);
  get(reinterpret_cast<void**>(&G), sizeof(Real) * (size_t)v.n);
  get(reinterpret_cast<void**>(&Y[0]), sizeof(Real) * (size_t)hmax * NY);
  get(reinterpret_cast<void**>(&Y[1]), sizeof(Real) * (size_t)hmax * NY);
  get(reinterpret_cast<void**>(&A), sizeof(Real) * (size_t)hmax * NY);
  get(reinterpret_cast<void**>(&vv), sizeof(Real) * (size_t)Hl);
  get(reinterpret_cast<void**>(&part), sizeof(double) * (size_t)nb * Hl);
  get(reinterpret_cast<void**>(&vptr), sizeof(int) * ((size_t)v.nv + 1));
  get(reinterpret_cast<void**>(&ventry), sizeof(int) * 4 * (size_t)v.S);
  if (e != cudaSuccess) return e;
  // vertex -> (slot, local vertex) lists of the cubature set, slots ascending
  {
    std::vector<int4> tets(v.ne);
    std::vector<int> cub(v.S);
    e = cudaMemcpyAsync(tets.data(), v.tets, sizeof(int4) * v.ne, cudaMemcpyDeviceToHost, v.s);
    if (e == cudaSuccess && v.cub_idx)
      e = cudaMemcpyAsync(cub.data(), v.cub_idx, sizeof(int) * v.S, cudaMemcpyDeviceToHost,
                          v.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.s);
    if (e != cudaSuccess) return e;
    std::vector<int> cnt(v.nv + 1, 0), ent(4 * (size_t)v.S);
    for (int sl = 0; sl < v.S; ++sl) {
      const int4 tv = tets[v.cub_idx ? cub[sl] : sl];
      for (int a : {tv.x, tv.y, tv.z, tv.w}) ++cnt[a + 1];
    }
    for (int i = 0; i < v.nv; ++i) cnt[i + 1] += cnt[i];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (int sl = 0; sl < v.S; ++sl) {
      const int4 tv = tets[v.cub_idx ? cub[sl] : sl];
      const int vv4[4] = {tv.x, tv.y, tv.z, tv.w};
      for (int a = 0; a < 4; ++a) ent[pos[vv4[a]]++] = 4 * sl + a;
    }
    e = cudaMemcpyAsync(vptr, cnt.data(), sizeof(int) * (v.nv + 1), cudaMemcpyHostToDevice, v.s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ventry, ent.data(), sizeof(int) * 4 * (size_t)v.S,
                          cudaMemcpyHostToDevice, v.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.s);
    if (e != cudaSuccess) return e;
  }
  const int m = v.r + (v.r & 1);
  proj_smem = sizeof(double) * (2 * (size_t)m * (m + 1) + m) + sizeof(int) * m;
  e = cudaFuncSetAttribute(project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)proj_smem);
  if (e != cudaSuccess) return e;
  if (v.use_tc_gemm) {
    size_t need = 0;
    for (int l = 1; l < (int)v.widths.size() - 1; ++l)
      need = std::max(need, tc_gemm_workspace_floats(v.widths[l], NY, v.widths[l - 1],
                                                     v.num_sms));
    ws_floats = need;
    if (need) get(reinterpret_cast<void**>(&ws), sizeof(float) * need);
    get(reinterpret_cast<void**>(&gerr), sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(gerr, 0, sizeof(int), v.s);
  }
  return e;
}

template <typename Real>
void Curvature<Real>::release() {
  for (void* p : {(void*)F, (void*)G, (void*)Y[0], (void*)Y[1], (void*)A, (void*)vv, (void*)part,
                  (void*)vptr, (void*)ventry, (void*)ws, (void*)gerr})
    if (p) cudaFree(p);
  F = G = A = vv = nullptr;
  Y[0] = Y[1] = nullptr;
  part = nullptr;
  vptr = ventry = nullptr;
  ws = nullptr;
  gerr = nullptr;
}

template <typename Real>
cudaError_t Curvature<Real>::launch(const ElemArgs& ea, const LastArgs& la, const Real* u,
                                    const Real* Z0, int zcps, const std::vector<Real*>& dW,
                                    const std::vector<Real*>& db, const void* wl_bf16,
                                    double* sys, cudaStream_t s) const {
  const int L = (int)v.widths.size() - 1;
  tet_forces_kernel<Real><<<(ea.S + 127) / 128, 128, 0, s>>>(ea, u, F);
  full_gradient_kernel<Real><<<(v.nv + 127) / 128, 128, 0, s>>>(v.nv, vptr, ventry, F, u, la,
                                                                  G);
  if (wl_bf16)
    wtv_kernel<Real, __nv_bfloat16><<<nb, WTV_THREADS, 0, s>>>(
        static_cast<const __nv_bfloat16*>(wl_bf16), G, v.n, Hl, part);
  else
    wtv_kernel<Real, Real><<<nb, WTV_THREADS, 0, s>>>(dW[L - 1], G, v.n, Hl, part);
  wtv_reduce_kernel<Real><<<(Hl + 3) / 4, 128, 0, s>>>(part, nb, Hl, la.scale, vv);
  y0_kernel<Real><<<(rn * NY + 255) / 256, 256, 0, s>>>(Z0, zcps, rn, NY, Y[0]);
  int cur = 0;
  for (int l = 0; l < L - 1; ++l) {
    const int M = v.widths[l + 1], K = v.widths[l];
    if (v.use_tc_gemm && sizeof(Real) == 4) {
      cudaError_t e = tc_gemm_tf32(s, M, NY, K, 1.f, reinterpret_cast<const float*>(dW[l]), K, 1,
                                   reinterpret_cast<const float*>(Y[cur]), NY, 1, 0.f,
                                   reinterpret_cast<float*>(A), NY, ws, ws_floats, v.num_sms,
                                   gerr);
      if (e != cudaSuccess) return e;
    } else {
      gemm_rm_kernel<Real><<<dim3((NY + 15) / 16, (M + 15) / 16), dim3(16, 16), 0, s>>>(
          M, NY, K, dW[l], Y[cur], A);
    }
    act2_kernel<Real><<<(M * NY + 255) / 256, 256, 0, s>>>(A, db[l], M, rn, NY, Y[cur ^ 1]);
    cur ^= 1;
  }
  contract_kernel<Real><<<(rn * (rn + 1) / 2 + 31) / 32, 32 * CON_WARPS, 0, s>>>(
      Y[cur], vv, Hl, rn, NY, v.r, sys);
  project_kernel<<<1, PROJ_THREADS, proj_smem, s>>>(sys, v.r, clamp);
  return cudaGetLastError();
}

template <typename Real>
int Curvature<Real>::device_error() const {
  if (!gerr) return 0;
  int h = 0;
  if (cudaMemcpy(&h, gerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  return h;
}

template struct Curvature<float>;
template struct Curvature<double>;

}  // namespace lsn
