// Lipschitz-loss training of the subspace decoder (Sec. 4) on the GPU:
// forward and backward kernels written out by hand, FP32 arithmetic with
// FP64 loss sums.
//
//   L_C  = 1/B sum_b ||x(g(q_b)) - q_b||_M^2                              (Eq. 3)
//   Ht_b = d2/dz2 sum_{e in S} w_e V_e Psi(F_e(x(z))) at z_b = g(q_b)      (Sec. 4.3)
//   L_LS = 1/(B(B-1)) sum_{i != j} ||Ht_i - Ht_j||_F^2 / ||z_i - z_j||^2  (Eq. 9)
//   L    = L_C + lambda L_LS                                               (Eq. 10)
//
// with the linear encoder g(q) = Ew (q - X0) + eb, the solver's decoder
// x(z) = X0 + s f(z), no gradient through the samples z_b in L_LS, and the
// exact (unprojected) Hessian
//   Ht = sum_e w_e (J_e^T H_e J_e + sum_k g_{e,k} d2x_k/dz2).
//
// Forward-mode second derivatives.  Every sample carries Cs = 1 + r + P
// columns through the decoder (P = r(r+1)/2): its value, the r tangents and
// the upper triangle of the second-order tangents,
//   T' = s'(a) (W T),  U'_cd = s''(a) (W T)_c (W T)_d + s'(a) (W U)_cd,
// and the last layer is evaluated on the decoder rows the cubature tets
// touch.  The backward pass reverses this propagation:
//   da  = s' gh + s'' sum_c gT_c T^_c + s''' sum_cd gU_cd T^_c T^_d + s'' sum_cd gU_cd U^_cd
//   dT^_c = s' gT_c + s'' sum_d gU_{cd} T^_d (both index orders),  dU^ = s' gU,
// where ^ marks the pre-activation products W Z.  The element part of the
// backward pass uses the third derivative of Psi contracted with the adjoint
// of the element Hessian, evaluated with forward-mode dual numbers.
//
// Matrices are row-major; one sample's columns are contiguous.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lsn_internal.cuh"
#include "train_internal.cuh"

namespace lsn {
namespace {

// ------------------------------------------------------------ generic GEMM
// C[m][n] = alpha sum_k A(m,k) B(k,n) + beta C[m][n], A(m,k) = A[m sam + k sak],
// B(k,n) = B[k sbk + n sbn].  64x64 tiles, 256 threads, 4x4 per thread.
constexpr int GT = 64, GK = 16;

template <typename Real>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, Real alpha,
                                                   const Real* __restrict__ A, long long sam,
                                                   long long sak, const Real* __restrict__ B,
                                                   long long sbk, long long sbn, Real beta,
                                                   Real* __restrict__ C, long long ldc) {
  __shared__ Real As[GK][GT + 1], Bs[GK][GT + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  Real acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = t; e < GT * GK; e += 256) {
      const int mm = e / GK, kk = e % GK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : Real(0);
      const int nn = e / GK, kb = e % GK;
      const int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < N && gk2 < K) ? B[gk2 * sbk + gn * sbn] : Real(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      Real a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        Real* c = C + m * ldc + n;
        *c = alpha * acc[i][j] + (beta != Real(0) ? beta * *c : Real(0));
      }
    }
}

template <typename Real>
void gemm(cudaStream_t s, int M, int N, int K, Real alpha, const Real* A, long long sam,
          long long sak, const Real* B, long long sbk, long long sbn, Real beta, Real* C,
          long long ldc) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  gemm_kernel<Real><<<grid, 256, 0, s>>>(M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C,
                                         ldc);
}

template <typename Real> __device__ __forceinline__ Real elu0(Real a) { return a > Real(0) ? a : (Real)expm1(a); }
template <typename Real> __device__ __forceinline__ Real elu1(Real a) { return a > Real(0) ? Real(1) : (Real)exp(a); }
template <typename Real> __device__ __forceinline__ Real elu2(Real a) { return a > Real(0) ? Real(0) : (Real)exp(a); }
template <typename Real> __device__ __forceinline__ Real elu3(Real a) { return a > Real(0) ? Real(0) : (Real)exp(a); }

// ------------------------------------------------------- reconstruction
// D[k][b] = q_b[k] - X0[k]  (q given as B x n doubles)
template <typename Real>
__global__ void snapshots_kernel(const double* __restrict__ q, const double* __restrict__ X0,
                                 int n, int B, Real* __restrict__ D) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * B) return;
  const int k = (int)(i / B), b = (int)(i % B);
  D[i] = (Real)(q[(long long)b * n + k] - X0[k]);
}

// A = Zlin + bias (row), H = ELU(A); in place on A when H == A is not wanted
template <typename Real>
__global__ void bias_elu_kernel(Real* __restrict__ A, const Real* __restrict__ bias, int M,
                                int N, Real* __restrict__ H) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)M * N) return;
  const Real a = A[i] + bias[i / N];
  A[i] = a;
  H[i] = elu0(a);
}

// per row k: R = s (OUT + b) - D;  loss partial sum m R^2; dOUT = (2/B) s m R
template <typename Real>
__global__ void recon_kernel(const Real* __restrict__ OUT, const Real* __restrict__ bias,
                             const Real* __restrict__ D, const double* __restrict__ mass,
                             int n, int B, Real scale, Real* __restrict__ dOUT,
                             double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n * B;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / B);
    const Real R = scale * (OUT[i] + bias[k]) - D[i];
    const double m = mass[k / 3];
    acc += m * (double)R * (double)R;
    dOUT[i] = (Real)(2.0 / B * scale * m * (double)R);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out[m] (+)= sum_j M[m][j stride + off], j < cnt   (fixed order)
template <typename Real>
__global__ void rowsum_kernel(const Real* __restrict__ Mx, int rows, int cols_total, int cnt,
                              int stride, int off, Real alpha, Real* __restrict__ out,
                              int accumulate) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= rows) return;
  Real s = Real(0);
  const Real* row = Mx + (long long)m * cols_total;
  for (int j = 0; j < cnt; ++j) s += row[j * stride + off];
  out[m] = (accumulate ? out[m] : Real(0)) + alpha * s;
}

template <typename Real>
__global__ void elu_back_kernel(const Real* __restrict__ A, Real* __restrict__ dH, long long N) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) dH[i] *= elu1(A[i]);
}

// ------------------------------------------------- second-order propagation
// Y0[i][b Cs + c]: value z_b, tangents e_i, second-order tangents 0
template <typename Real>
__global__ void so_init_kernel(const Real* __restrict__ Z, int r, int B, int Cs,
                               Real* __restrict__ Y0) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long NC = (long long)B * Cs;
  if (e >= r * NC) return;
  const int i = (int)(e / NC);
  const long long col = e % NC;
  const int b = (int)(col / Cs), c = (int)(col % Cs);
  Real v = Real(0);
  if (c == 0) v = Z[i * B + b];
  else if (c <= r) v = (c - 1 == i) ? Real(1) : Real(0);
  Y0[e] = v;
}

__device__ __forceinline__ int pidx(int c, int d, int r) {  // c <= d, upper row-major
  return c * r - (c * (c - 1)) / 2 + (d - c);
}

// One thread per (unit i, sample b): Y = activation of the linear products Zh
// (Zh[i][b Cs + .] = W Y_prev) with bias on the value column.
template <typename Real>
__global__ void so_act_kernel(const Real* __restrict__ Zh, const Real* __restrict__ bias,
                              int H, int B, int r, int Cs, Real* __restrict__ Y) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)H * B) return;
  const int i = (int)(e / B), b = (int)(e % B);
  const long long o = (long long)i * B * Cs + (long long)b * Cs;
  const Real a = Zh[o] + bias[i];
  const Real s1 = elu1(a), s2 = elu2(a);
  Y[o] = elu0(a);
  for (int c = 0; c < r; ++c) Y[o + 1 + c] = s1 * Zh[o + 1 + c];
  int p = 0;
  for (int c = 0; c < r; ++c)
    for (int d = c; d < r; ++d, ++p)
      Y[o + 1 + r + p] = s2 * Zh[o + 1 + c] * Zh[o + 1 + d] + s1 * Zh[o + 1 + r + p];
}

// Reverse of so_act_kernel: dY (adjoints of the outputs) -> dZh.
template <typename Real>
__global__ void so_act_back_kernel(const Real* __restrict__ Zh, const Real* __restrict__ bias,
                                   const Real* __restrict__ dY, int H, int B, int r, int Cs,
                                   Real* __restrict__ dZh) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)H * B) return;
  const int i = (int)(e / B), b = (int)(e % B);
  const long long o = (long long)i * B * Cs + (long long)b * Cs;
  const Real a = Zh[o] + bias[i];
  const Real s1 = elu1(a), s2 = elu2(a), s3 = elu3(a);
  Real da = s1 * dY[o];
  for (int c = 0; c < r; ++c) {
    da += s2 * dY[o + 1 + c] * Zh[o + 1 + c];
    dZh[o + 1 + c] = s1 * dY[o + 1 + c];
  }
  int p = 0;
  for (int c = 0; c < r; ++c)
    for (int d = c; d < r; ++d, ++p) {
      const Real g = dY[o + 1 + r + p];
      const Real tc = Zh[o + 1 + c], td = Zh[o + 1 + d];
      da += g * (s3 * tc * td + s2 * Zh[o + 1 + r + p]);
      dZh[o + 1 + c] += g * s2 * td;
      dZh[o + 1 + d] += g * s2 * tc;
      dZh[o + 1 + r + p] = s1 * g;
    }
  dZh[o] = da;
}

// W_S[k][:] = W_L[rows[k]][:], b_S[k] = b_L[rows[k]]
template <typename Real>
__global__ void gather_rows_kernel(const Real* __restrict__ WL, const Real* __restrict__ bL,
                                   const int* __restrict__ rows, int RS, int Hc,
                                   Real* __restrict__ WS, Real* __restrict__ bS) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)RS * Hc) return;
  const int k = (int)(e / Hc), j = (int)(e % Hc);
  WS[e] = WL[(long long)rows[k] * Hc + j];
  if (j == 0) bS[k] = bL[rows[k]];
}

// dW_L[rows[k]][:] += dW_S[k][:], db_L[rows[k]] += db_S[k]
template <typename Real>
__global__ void scatter_rows_kernel(const Real* __restrict__ dWS, const Real* __restrict__ dbS,
                                    const int* __restrict__ rows, int RS, int Hc, Real alpha,
                                    Real* __restrict__ dWL, Real* __restrict__ dbL) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)RS * Hc) return;
  const int k = (int)(e / Hc), j = (int)(e % Hc);
  dWL[(long long)rows[k] * Hc + j] += alpha * dWS[e];
  if (j == 0) dbL[rows[k]] += alpha * dbS[k];
}

// ------------------------------------------------------- element physics
template <typename Real>
struct DualT {
  Real v, d;
};
template <typename R>
__device__ __forceinline__ DualT<R> operator+(DualT<R> a, DualT<R> b) { return {a.v + b.v, a.d + b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator-(DualT<R> a, DualT<R> b) { return {a.v - b.v, a.d - b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator*(DualT<R> a, DualT<R> b) {
  return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <typename R>
__device__ __forceinline__ DualT<R> operator*(R a, DualT<R> b) { return {a * b.v, a * b.d}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator*(DualT<R> a, R b) { return {a.v * b, a.d * b}; }
template <typename R>
__device__ __forceinline__ DualT<R> operator/(DualT<R> a, DualT<R> b) {
  const R iv = R(1) / b.v;
  return {a.v * iv, (a.d * b.v - a.v * b.d) * iv * iv};
}

__host__ __device__ constexpr int lc_sign(int i, int k) { return (k == (i + 1) % 3) ? 1 : -1; }

// <G, d2Psi/dF2(F)> for a 9x9 weight matrix G (row-major vec), in type T
template <typename T, typename Real>
__device__ __forceinline__ T hess_contract(const T (&F)[9], const Real* Gm, Real mu, Real lam,
                                           Real alpha) {
  T Ic = F[0] * F[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) Ic = Ic + F[k] * F[k];
  T cof[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof[3 * i + j] = F[3 * i1 + j1] * F[3 * i2 + j2] - F[3 * i1 + j2] * F[3 * i2 + j1];
    }
  const T J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
  T one = F[0] * Real(0);
  one.v = Real(1);
  const T Ic1 = Ic + one;
  const T c1 = mu * (Ic / Ic1);
  const T c2 = (Real(2) * mu) * (one / (Ic1 * Ic1));
  T Jm = J;
  Jm.v -= alpha;
  const T c3 = lam * Jm;
  // sum_ab G_ab [c1 d_ab + c2 F_a F_b + lam cof_a cof_b + c3 H_J(F)_ab]
  T trG = one * Real(0), fGf = one * Real(0), cGc = one * Real(0), hj = one * Real(0);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    trG.v += Gm[10 * a];
    T ga = one * Real(0), gc = one * Real(0);
#pragma unroll
    for (int b = 0; b < 9; ++b) {
      ga = ga + Gm[9 * a + b] * F[b];
      gc = gc + Gm[9 * a + b] * cof[b];
    }
    fGf = fGf + F[a] * ga;
    cGc = cGc + cof[a] * gc;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
          if (i != k && j != l) {
            const Real g = Gm[9 * (3 * i + j) + 3 * k + l];
            const Real sg = (Real)(lc_sign(i, k) * lc_sign(j, l));
            hj = hj + (g * sg) * F[3 * (3 - i - k) + (3 - j - l)];
          }
  return c1 * trG + c2 * fGf + lam * cGc + c3 * hj;
}

// value-only version of the element derivatives at F (full-F formulation)
template <typename Real>
struct ElemD {
  Real P[9];    // dPsi/dF
  Real A[81];   // d2Psi/dF2
};

template <typename Real>
__device__ __forceinline__ void elem_derivs(const Real (&F)[9], Real mu, Real lam, Real alpha,
                                            ElemD<Real>& ed) {
  Real Ic = Real(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) Ic += F[k] * F[k];
  Real cof[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof[3 * i + j] = F[3 * i1 + j1] * F[3 * i2 + j2] - F[3 * i1 + j2] * F[3 * i2 + j1];
    }
  const Real J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
  const Real c1 = mu * Ic / (Ic + Real(1)), c2 = Real(2) * mu / ((Ic + Real(1)) * (Ic + Real(1)));
  const Real c3 = lam * (J - alpha);
#pragma unroll
  for (int a = 0; a < 9; ++a) ed.P[a] = c1 * F[a] + c3 * cof[a];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          const int a = 3 * i + j, b = 3 * k + l;
          Real v = c2 * F[a] * F[b] + lam * cof[a] * cof[b];
          if (a == b) v += c1;
          if (i != k && j != l)
            v += c3 * (Real)(lc_sign(i, k) * lc_sign(j, l)) * F[3 * (3 - i - k) + (3 - j - l)];
          ed.A[9 * a + b] = v;
        }
}

// Warp per (tet, sample): contribution to Ht_b (upper triangle) and, in the
// backward pass, the adjoints of the tet's rows.  Lane c < r owns column c.
template <typename Real>
struct ElemCtx {
  int S, r, P, B, Cs, RS;
  const int4* tets;     // local vertex indices (into the cubature rows / 3)
  const Real* dminv;    // [9][S]
  const Real* wv;       // [S]
  const Real* XS;       // [RS][B Cs] last-layer linear outputs on cubature rows
  const Real* bS;       // [RS]
  const Real* X0S;      // [RS]
  Real scale, mu, lam, alpha;
};

template <typename Real>
__device__ __forceinline__ void load_elem(const ElemCtx<Real>& ec, int e, int b, int lane, Real (&F)[9],
                                          Real (&Dc)[12], Real (&Gc)[9], int (&rowi)[12],
                                          Real& wv) {
  const int4 tv = ec.tets[e];
  const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
  Real Dm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dm[k] = ec.dminv[k * ec.S + e];
  wv = ec.wv[e];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Dc[j] = -(Dm[j] + Dm[3 + j] + Dm[6 + j]);
#pragma unroll
    for (int a = 1; a < 4; ++a) Dc[3 * a + j] = Dm[3 * (a - 1) + j];
  }
  const long long NC = (long long)ec.B * ec.Cs;
  Real x[12], jc[12];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int row = 3 * vv[a] + i;
      rowi[3 * a + i] = row;
      const long long o = row * NC + (long long)b * ec.Cs;
      x[3 * a + i] = ec.X0S[row] + ec.scale * (ec.XS[o] + ec.bS[row]);
      jc[3 * a + i] = lane < ec.r ? ec.scale * ec.XS[o + 1 + lane] : Real(0);
    }
  // F = I + sum_a (x_a - x_0) Dm^-1 rows
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Real f = Real(0), g = Real(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        f += Dc[3 * a + j] * x[3 * a + i];
        g += Dc[3 * a + j] * jc[3 * a + i];
      }
      F[3 * i + j] = f;
      Gc[3 * i + j] = g;
    }
}

template <typename Real>
__global__ void __launch_bounds__(128) elem_hess_kernel(ElemCtx<Real> ec, Real* __restrict__ contrib) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ec.S * ec.B) return;
  const int b = warp / ec.S, e = warp % ec.S;
  Real F[9], Dc[12], Gc[9], wv;
  int rowi[12];
  load_elem(ec, e, b, lane, F, Dc, Gc, rowi, wv);
  ElemD<Real> ed;
  elem_derivs(F, ec.mu, ec.lam, ec.alpha, ed);
  // AG[:,c] = wV A G[:,c]
  Real AG[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Real s = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += ed.A[9 * a + k] * Gc[k];
    AG[a] = wv * s;
  }
  // element gradient rows g_k = wV (B^T vec P)_k
  Real gk[12];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Real s = Real(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) s += Dc[3 * a + j] * ed.P[3 * i + j];
      gk[3 * a + i] = wv * s;
    }
  const long long NC = (long long)ec.B * ec.Cs;
  Real* out = contrib + (long long)warp * ec.P;
  // Ht entries (c, d >= c) for c = lane: G[:,c]^T AG[:,d] + sum_k g_k D_k[c][d]
  for (int d = 0; d < ec.r; ++d) {
    Real Gd[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Gd[k] = __shfl_sync(0xffffffffu, Gc[k], d);
    if (lane < ec.r && d >= lane) {
      Real s = Real(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) s += AG[k] * Gd[k];
      const int p = pidx(lane, d, ec.r);
      Real sd = Real(0);
#pragma unroll
      for (int k = 0; k < 12; ++k)
        sd += gk[k] * ec.scale * ec.XS[rowi[k] * NC + (long long)b * ec.Cs + 1 + ec.r + p];
      out[p] = s + sd;
    }
  }
}

// Hs[b][p] = sum_e contrib[(b S + e) P + p]  (fixed order)
// First-order Lipschitz loss (the Supplement's order-o family, o = 1).
// Forward: per (tet, sample) the contribution w V P : G_e[:, c] of the tet to
// the reduced gradient dPt/dz_c (lane c), contrib[(b S + e) r + c].
template <typename Real>
__global__ void __launch_bounds__(128) grad1_kernel(ElemCtx<Real> ec, Real* __restrict__ contrib) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ec.S * ec.B) return;
  const int b = warp / ec.S, e = warp % ec.S;
  Real F[9], Dc[12], Gc[9], wv;
  int rowi[12];
  load_elem(ec, e, b, lane, F, Dc, Gc, rowi, wv);
  ElemD<Real> ed;
  elem_derivs(F, ec.mu, ec.lam, ec.alpha, ed);
  if (lane < ec.r) {
    Real s = Real(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) s += ed.P[a] * Gc[a];
    contrib[((long long)b * ec.S + e) * ec.r + lane] = wv * s;
  }
}

// Backward: with gbar_b = dL/d(dPt/dz)(z_b) (B x r), the adjoints of the
// tet's rows: value rows gx = w V B^T A dF with dF = sum_c gbar_c G_e[:, c],
// tangent rows gJ[k][c] = gbar_c g_k (g_k the element gradient rows).
template <typename Real>
__global__ void __launch_bounds__(128) elem_back1_kernel(ElemCtx<Real> ec,
                                                         const Real* __restrict__ gbar,
                                                         Real* __restrict__ gx,
                                                         Real* __restrict__ gJ) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ec.S * ec.B) return;
  const int b = warp / ec.S, e = warp % ec.S;
  Real F[9], Dc[12], Gc[9], wv;
  int rowi[12];
  load_elem(ec, e, b, lane, F, Dc, Gc, rowi, wv);
  ElemD<Real> ed;
  elem_derivs(F, ec.mu, ec.lam, ec.alpha, ed);
  const Real gb = lane < ec.r ? gbar[b * ec.r + lane] : Real(0);
  Real dF[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Real v = gb * Gc[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    dF[a] = v;
  }
  Real AdF[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Real v = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) v += ed.A[9 * a + k] * dF[k];
    AdF[a] = v;
  }
  const long long w = (long long)b * ec.S + e;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Real gk = Real(0), gxv = Real(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        gk += ed.P[3 * i + j] * Dc[3 * a + j];
        gxv += AdF[3 * i + j] * Dc[3 * a + j];
      }
      const int k = 3 * a + i;
      if (lane == 0) gx[w * 12 + k] = wv * gxv;
      if (lane < ec.r) gJ[(w * 12 + k) * ec.r + lane] = gb * wv * gk;
    }
}

template <typename Real>
__global__ void sum_hess_kernel(const Real* __restrict__ contrib, int S, int B, int P,
                                double* __restrict__ Hs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P, p = i % P;
  double s = 0.0;
  for (int e = 0; e < S; ++e) s += (double)contrib[((long long)b * S + e) * P + p];
  Hs[i] = s;
}

// L_LS and its adjoint Gbar_b (full-matrix adjoint, stored upper) per sample.
template <typename Real>
__global__ void lls_kernel(const double* __restrict__ Hs, const Real* __restrict__ Z, int B,
                           int r, int P, Real* __restrict__ Gbar, double* __restrict__ lpart) {
  const int b = blockIdx.x, t = threadIdx.x;
  __shared__ double red[256];
  double lsum = 0.0;
  const double norm = 1.0 / ((double)B * (B - 1));
  for (int p = t; p < P; p += blockDim.x) {
    int c = 0, q = p;
    while (q >= r - c) {
      q -= r - c;
      ++c;
    }
    const double mult = (q == 0) ? 1.0 : 2.0;  // off-diagonal entries appear twice
    double g = 0.0;
    for (int j = 0; j < B; ++j) {
      if (j == b) continue;
      double dz = 0.0;
      for (int i = 0; i < r; ++i) {
        const double v = (double)Z[i * B + b] - (double)Z[i * B + j];
        dz += v * v;
      }
      const double diff = Hs[b * P + p] - Hs[j * P + p];
      g += diff / dz;
      lsum += mult * diff * diff / dz;
    }
    Gbar[b * P + p] = (Real)(4.0 * norm * g);
  }
  red[t] = lsum * norm;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) lpart[b] = red[0];
}

// Backward per (tet, sample) warp: adjoints of the tet's 12 rows
//   gx (12), gJ (12 x r), and the element gradient rows g_k (12), which
// multiply the sample's Gbar in the second-order adjoint of each row.
template <typename Real>
__global__ void __launch_bounds__(128) elem_back_kernel(ElemCtx<Real> ec, const Real* __restrict__ Gbar,
                                                        Real* __restrict__ gx,
                                                        Real* __restrict__ gJ,
                                                        Real* __restrict__ gkout) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ec.S * ec.B) return;
  const int b = warp / ec.S, e = warp % ec.S;
  const int r = ec.r;
  Real F[9], Dc[12], Gc[9], wv;
  int rowi[12];
  load_elem(ec, e, b, lane, F, Dc, Gc, rowi, wv);
  ElemD<Real> ed;
  elem_derivs(F, ec.mu, ec.lam, ec.alpha, ed);
  const Real* Gb = Gbar + (long long)b * ec.P;
  auto gbar = [&](int c, int d) { return c <= d ? Gb[pidx(c, d, r)] : Gb[pidx(d, c, r)]; };
  // V[:,c] = sum_d G[:,d] Gbar[d][c]
  Real V[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = 0; d < r; ++d) {
    const Real gdc = lane < r ? gbar(d, lane) : Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) V[k] += __shfl_sync(0xffffffffu, Gc[k], d) * gdc;
  }
  // dG[:,c] = 2 wV A V[:,c];  gJ rows = B^T dG
  Real dG[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    Real s = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += ed.A[9 * a + k] * V[k];
    dG[a] = Real(2) * wv * s;
  }
  Real* gJo = gJ + (long long)warp * 12 * r;
  if (lane < r) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Real s = Real(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) s += Dc[3 * a + j] * dG[3 * i + j];
        gJo[(3 * a + i) * r + lane] = s;
      }
  }
  // adjoint of wV A:  Abar = G Gbar G^T = sum_c G[:,c] V[:,c]^T  (9 x 9)
  __shared__ Real Abar_s[4][81];
  __shared__ Real gt_s[4][12];
  Real* Abar = Abar_s[(threadIdx.x >> 5)];
  for (int ab = 0; ab < 81; ++ab) {
    Real v = lane < r ? Gc[ab / 9] * V[ab % 9] : Real(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) Abar[ab] = wv * v;
  }
  // gamma_k = <Gbar, D_k> over the full matrix (rows of the tet)
  const long long NC = (long long)ec.B * ec.Cs;
  Real* gt = gt_s[(threadIdx.x >> 5)];
  for (int k = 0; k < 12; ++k) {
    Real v = Real(0);
    for (int p = lane; p < ec.P; p += 32) {
      int c = 0, q = p;
      while (q >= r - c) {
        q -= r - c;
        ++c;
      }
      const Real mult = q == 0 ? Real(1) : Real(2);
      v += mult * Gb[p] * ec.scale * ec.XS[rowi[k] * NC + (long long)b * ec.Cs + 1 + r + p];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) gt[k] = v;
  }
  __syncwarp();
  // dF = d/dF <Abar, A(F)> (third derivative, dual numbers; lane m < 9 takes
  //      direction m) + wV A (B gamma)
  Real dF = Real(0);
  if (lane < 9) {
    DualT<Real> Fd[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fd[k] = {F[k], k == lane ? Real(1) : Real(0)};
    const DualT<Real> cval = hess_contract<DualT<Real>, Real>(Fd, Abar, ec.mu, ec.lam, ec.alpha);
    dF = cval.d;
    // (B gamma)_m and A row m
    Real bg[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Real s = Real(0);
#pragma unroll
        for (int a = 0; a < 4; ++a) s += Dc[3 * a + j] * gt[3 * a + i];
        bg[3 * i + j] = s;
      }
    Real s = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += ed.A[9 * lane + k] * bg[k];
    dF += wv * s;
  }
  // gx = B^T dF
  Real dFa[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) dFa[k] = __shfl_sync(0xffffffffu, dF, k);
  if (lane < 12) {
    const int a = lane / 3, i = lane % 3;
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) s += Dc[3 * a + j] * dFa[3 * i + j];
    gx[(long long)warp * 12 + lane] = s;
    // element gradient row g_k = wV (B^T vec P)_k
    Real g = Real(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) g += Dc[3 * a + j] * ed.P[3 * i + j];
    gkout[(long long)warp * 12 + lane] = wv * g;
  }
}

// Adjoint of the cubature-row outputs XS (linear outputs, before the scale):
// gather over the (tet, slot) incidences of each row (fixed CSR order).
template <typename Real>
__global__ void row_adjoint_kernel(const int* __restrict__ inc_ptr, const int* __restrict__ inc,
                                   int RS, int S, int B, int r, int P, int Cs, Real scale,
                                   const Real* __restrict__ gx, const Real* __restrict__ gJ,
                                   const Real* __restrict__ gk, const Real* __restrict__ Gbar,
                                   Real* __restrict__ dXS) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)RS * B) return;
  const int row = (int)(e / B), b = (int)(e % B);
  const int vtx = row / 3, comp = row % 3;
  Real sx = Real(0), sg = Real(0);
  Real* out = dXS + (long long)row * B * Cs + (long long)b * Cs;
  for (int c = 0; c < r; ++c) out[1 + c] = Real(0);
  for (int q = inc_ptr[vtx]; q < inc_ptr[vtx + 1]; ++q) {
    const int tet = inc[q] >> 2, slot = inc[q] & 3;
    const long long w = (long long)b * S + tet;
    const int k = 3 * slot + comp;
    sx += gx[w * 12 + k];
    sg += gk[w * 12 + k];
    for (int c = 0; c < r; ++c) out[1 + c] += gJ[(w * 12 + k) * r + c];
  }
  out[0] = scale * sx;
  for (int c = 0; c < r; ++c) out[1 + c] *= scale;
  // second-order columns: d/dD_k[c][d] of sum_k g_k <Gbar, D_k> over the full
  // matrix, for the stored upper entry (both (c,d) and (d,c) for c < d)
  int p = 0;
  for (int c = 0; c < r; ++c)
    for (int d = c; d < r; ++d, ++p)
      out[1 + r + p] = scale * sg * (c == d ? Real(1) : Real(2)) * Gbar[b * P + p];
}

// ------------------------------------------------ unsupervised loss (Eq. 4)
// Potential term: per (cubature tet, sample) the weighted energy w V Psi(F)
// and its 12 position derivatives, from the decoder output OUT (n x B, raw,
// before bias and scale) on the cubature rows.  Psi and dPsi/dF are written
// in Hd = F - I (as in the solver's element kernels).
template <typename Real>
__global__ void unsup_elem_kernel(const int4* __restrict__ tets, const Real* __restrict__ dminv,
                                  const Real* __restrict__ wv, const int* __restrict__ rows,
                                  const Real* __restrict__ X0S, const Real* __restrict__ OUT,
                                  const Real* __restrict__ bias, int S, int B, Real scale,
                                  Real mu, Real lam, Real alpha, double* __restrict__ epart,
                                  Real* __restrict__ gx) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)S * B) return;
  const int b = (int)(id / S), e = (int)(id % S);
  const int4 tv = tets[e];
  const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
  Real xv[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int lr = 3 * vv[a] + i, gr = rows[lr];
      xv[a][i] = X0S[lr] + scale * (OUT[(long long)gr * B + b] + bias[gr]);
    }
  Real Dm[3][3], H[3][3];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dm[k / 3][k % 3] = dminv[k * S + e];
  // Hd = Ds Dm^-1 - I, Ds the edge matrix of the deformed tet
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Real v = Real(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) v += (xv[a + 1][i] - xv[0][i]) * Dm[a][j];
      H[i][j] = v - (i == j ? Real(1) : Real(0));
    }
  Real trH = H[0][0] + H[1][1] + H[2][2], nrm = Real(0), cofH[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      nrm += H[i][j] * H[i][j];
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cofH[i][j] = H[i1][j1] * H[i2][j2] - H[i1][j2] * H[i2][j1];
    }
  const Real Ic3 = Real(2) * trH + nrm;
  const Real m2 = cofH[0][0] + cofH[1][1] + cofH[2][2];
  const Real detH = H[0][0] * cofH[0][0] + H[0][1] * cofH[0][1] + H[0][2] * cofH[0][2];
  const Real Jm1 = trH + m2 + detH;
  const Real oma = Real(1) - alpha;
  const Real w = wv[e];
  const Real psi = Real(0.5) * mu * Ic3 - Real(0.5) * mu * log1p(Ic3 * Real(0.25)) +
                   Real(0.5) * lam * Jm1 * (Jm1 + Real(2) * oma);
  epart[id] = (double)(w * psi);
  const Real dl = Ic3 / (Real(4) * (Ic3 + Real(4)));
  Real* g = gx + id * 12;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Real P[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Real Fij = H[i][j] + (i == j ? Real(1) : Real(0));
      const Real cofF = (i == j ? Real(1) + trH : Real(0)) - H[j][i] + cofH[i][j];
      P[j] = w * (mu * dl * Fij + lam * Jm1 * cofF +
                  Real(0.75) * mu * (H[i][j] + H[j][i] - (i == j ? trH : Real(0)) - cofH[i][j]));
    }
    Real s0 = Real(0);
#pragma unroll
    for (int a = 1; a < 4; ++a) {
      const Real v = P[0] * Dm[a - 1][0] + P[1] * Dm[a - 1][1] + P[2] * Dm[a - 1][2];
      g[3 * a + i] = v;
      s0 += v;
    }
    g[i] = -s0;
  }
}

// dOUT[row][b] += coef * sum over the tets at the row's vertex of their
// derivative (fixed order along the incidence list)
template <typename Real>
__global__ void unsup_row_kernel(const int* __restrict__ inc_ptr, const int* __restrict__ inc,
                                 const int* __restrict__ rows, int RS, int S, int B,
                                 const Real* __restrict__ gx, Real coef,
                                 const Real* __restrict__ coefb, Real* __restrict__ dOUT) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)RS * B) return;
  const int lr = (int)(id / B), b = (int)(id % B);
  const int vtx = lr / 3, comp = lr % 3;
  Real sx = Real(0);
  for (int q = inc_ptr[vtx]; q < inc_ptr[vtx + 1]; ++q) {
    const int tet = inc[q] >> 2, slot = inc[q] & 3;
    sx += gx[((long long)b * S + tet) * 12 + 3 * slot + comp];
  }
  dOUT[(long long)rows[lr] * B + b] += coef * (coefb ? coefb[b] : Real(1)) * sx;
}

// Y[row][b] = c m_{row / 3} X[row][b]
template <typename Real>
__global__ void mass_rows_kernel(const Real* __restrict__ X, const double* __restrict__ mass,
                                 int n, int B, Real c, Real* __restrict__ Yo) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * B) return;
  Yo[i] = c * (Real)mass[(i / B) / 3] * X[i];
}

template <typename Real>
__global__ void adam_kernel(Real* __restrict__ th, const Real* __restrict__ g,
                            Real* __restrict__ m, Real* __restrict__ v, long long N, Real lr,
                            Real b1, Real b2, Real eps, Real c1, Real c2) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const Real gi = g[i];
  const Real mi = b1 * m[i] + (Real(1) - b1) * gi;
  const Real vi = b2 * v[i] + (Real(1) - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
}

inline int blocks(long long n, int t = 256) { return (int)((n + t - 1) / t); }

}  // namespace

// =====================================================================
namespace {
struct CudaFail {
  cudaError_t e;
};
inline void tck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaFail{e};
}
template <typename Real>
__global__ void bias_add_kernel(Real* __restrict__ M, const Real* __restrict__ bias, int rows,
                                int cols) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (long long)rows * cols) M[i] += bias[i / cols];
}
template <typename Real>
__global__ void x0_rows_kernel(const double* __restrict__ X0, const int* __restrict__ rows,
                               int RS, Real* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < RS) out[k] = (Real)X0[rows[k]];
}

template <typename Real>
struct Trainer : TrainerBase {
  TrainSetup ts;
  // TF32 tensor-core GEMMs (tc_gemm.cu) for the plain matrix products of the
  // forward and backward passes; otherwise the CUDA-core kernel above
  bool tf32 = false;
  // BF16 form: the GEMMs round both operands to BF16 (the weights and the
  // activations of every product); theta, the gradient and Adam stay FP32
  bool bf16ops = false;
  float* gws = nullptr;   // split-K workspace of the tensor-core GEMM (grown on demand)
  size_t gws_cap = 0;
  int* gerr = nullptr;    // device flag: a bounded wait of the GEMM ran out
  int num_sms = 1;

  // C[m][n] = alpha sum_k A(m,k) B(k,n) + beta C[m][n] with the strides of
  // gemm(); as column-major, C^T (N x M, ld ldc) = op(B) op(A)
  void mm(cudaStream_t s, int M, int N, int K, Real alpha, const Real* A, long long sam,
          long long sak, const Real* B, long long sbk, long long sbn, Real beta, Real* C,
          long long ldc) {
    if (!tf32 || M <= 0 || N <= 0 || K <= 0 || sizeof(Real) != 4) {
      gemm<Real>(s, M, N, K, alpha, A, sam, sak, B, sbk, sbn, beta, C, ldc);
      return;
    }
    const size_t need = tc_gemm_workspace_floats(M, N, K, num_sms);
    if (need > gws_cap) {
      if (gws) cudaFree(gws);
      gws = nullptr;
      gws_cap = 0;
      tck(cudaMalloc(&gws, need * sizeof(float)));
      gws_cap = need;
    }
    tck(tc_gemm_tf32(s, M, N, K, (float)alpha, reinterpret_cast<const float*>(A), sam, sak,
                     reinterpret_cast<const float*>(B), sbk, sbn, (float)beta,
                     reinterpret_cast<float*>(C), ldc, gws, gws_cap, num_sms, gerr, bf16ops));
  }
  int device_error() override {
    if (!gerr) return 0;
    int h = 0;
    tck(cudaMemcpy(&h, gerr, sizeof(int), cudaMemcpyDeviceToHost));
    return h;
  }
  std::vector<void*> sbufs, bbufs;   // static / per-batch allocations
  Real *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  long long step = 0;
  int4* ctl = nullptr;
  Real *cdminv = nullptr, *cwv = nullptr, *X0S = nullptr;
  int *rows = nullptr, *inc_ptr = nullptr, *inc = nullptr;
  int Bcap = 0;
  Real *D = nullptr, *Z = nullptr, *OUT = nullptr, *dOUT = nullptr, *dH = nullptr,
       *dH2 = nullptr;
  std::vector<Real*> A, Hh, Y, Zh;
  Real *WS = nullptr, *bS = nullptr, *dWS = nullptr, *dbS = nullptr, *XS = nullptr,
       *dXS = nullptr, *dY = nullptr, *dZh = nullptr, *contrib = nullptr, *gx = nullptr,
       *gJ = nullptr, *gk = nullptr, *Gbar = nullptr;
  double *Hs = nullptr, *lpart = nullptr, *rpart = nullptr, *epart = nullptr;
  Real *Gm = nullptr, *Cm = nullptr;  // B x B Gram and repulsion coefficients (Eq. 4)
  Real* G1 = nullptr;                 // B x r adjoint of the reduced gradients (order 1)

  template <typename T>
  T* alloc(std::vector<void*>& keep, size_t count) {
    void* p = nullptr;
    tck(cudaMalloc(&p, (count ? count : 1) * sizeof(T)));
    keep.push_back(p);
    return static_cast<T*>(p);
  }

  explicit Trainer(const TrainSetup& s) : ts(s) {
    const int r = ts.widths[0], n = ts.n;
    L = (int)ts.widths.size() - 1;
    P = r * (r + 1) / 2;
    Cs = 1 + r + P;
    long long o = 0;
    off.push_back(o);
    o += (long long)r * n;
    off.push_back(o);
    o += r;
    for (int l = 0; l < L; ++l) {
      off.push_back(o);
      o += (long long)ts.widths[l + 1] * ts.widths[l];
      off.push_back(o);
      o += ts.widths[l + 1];
    }
    nparams = o;
  }
  ~Trainer() override {
    for (void* p : bbufs) cudaFree(p);
    for (void* p : sbufs) cudaFree(p);
    if (gws) cudaFree(gws);
    if (gerr) cudaFree(gerr);
  }

  void init_device(const double* theta_host) override {
    if (tf32) {
      int dev = 0;
      tck(cudaGetDevice(&dev));
      tck(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
      tck(cudaMalloc(&gerr, sizeof(int)));
      tck(cudaMemset(gerr, 0, sizeof(int)));
    }
    theta = alloc<Real>(sbufs, nparams);
    grad = alloc<Real>(sbufs, nparams);
    am = alloc<Real>(sbufs, nparams);
    av = alloc<Real>(sbufs, nparams);
    set_params(theta_host);
    tck(cudaMemset(am, 0, sizeof(Real) * nparams));
    tck(cudaMemset(av, 0, sizeof(Real) * nparams));
    step = 0;
    ctl = alloc<int4>(sbufs, ts.S);
    tck(cudaMemcpy(ctl, ts.tets_local.data(), sizeof(int) * 4 * ts.S, cudaMemcpyHostToDevice));
    int4* gtets = alloc<int4>(sbufs, ts.S);
    cdminv = alloc<Real>(sbufs, 9 * (size_t)ts.S);
    cwv = alloc<Real>(sbufs, ts.S);
    launch_gather_cubature<Real>(ts.tets, ts.dminv, ts.vol, ts.cub_idx, ts.cub_w, ts.S, ts.ne,
                                 gtets, cdminv, cwv, 0);
    rows = alloc<int>(sbufs, ts.RS);
    tck(cudaMemcpy(rows, ts.rows.data(), sizeof(int) * ts.RS, cudaMemcpyHostToDevice));
    inc_ptr = alloc<int>(sbufs, ts.inc_ptr.size());
    tck(cudaMemcpy(inc_ptr, ts.inc_ptr.data(), sizeof(int) * ts.inc_ptr.size(),
                   cudaMemcpyHostToDevice));
    inc = alloc<int>(sbufs, ts.inc.size());
    tck(cudaMemcpy(inc, ts.inc.data(), sizeof(int) * ts.inc.size(), cudaMemcpyHostToDevice));
    X0S = alloc<Real>(sbufs, ts.RS);
    x0_rows_kernel<Real><<<blocks(ts.RS), 256>>>(ts.X0, rows, ts.RS, X0S);
    tck(cudaDeviceSynchronize());
    tck(cudaGetLastError());
  }

  void set_params(const double* in) override {
    std::vector<Real> h(nparams);
    for (long long i = 0; i < nparams; ++i) h[i] = (Real)in[i];
    tck(cudaMemcpy(theta, h.data(), sizeof(Real) * nparams, cudaMemcpyHostToDevice));
  }
  void get_params(double* out) override {
    std::vector<Real> h(nparams);
    tck(cudaMemcpy(h.data(), theta, sizeof(Real) * nparams, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < nparams; ++i) out[i] = (double)h[i];
  }
  void get_grad(double* out) override {
    std::vector<Real> h(nparams);
    tck(cudaMemcpy(h.data(), grad, sizeof(Real) * nparams, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < nparams; ++i) out[i] = (double)h[i];
  }
  void get_adam(double* m, double* v, long long* st) override {
    std::vector<Real> h(nparams);
    tck(cudaMemcpy(h.data(), am, sizeof(Real) * nparams, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < nparams; ++i) m[i] = (double)h[i];
    tck(cudaMemcpy(h.data(), av, sizeof(Real) * nparams, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < nparams; ++i) v[i] = (double)h[i];
    *st = step;
  }
  void set_adam(const double* m, const double* v, long long st) override {
    std::vector<Real> h(nparams);
    for (long long i = 0; i < nparams; ++i) h[i] = (Real)m[i];
    tck(cudaMemcpy(am, h.data(), sizeof(Real) * nparams, cudaMemcpyHostToDevice));
    for (long long i = 0; i < nparams; ++i) h[i] = (Real)v[i];
    tck(cudaMemcpy(av, h.data(), sizeof(Real) * nparams, cudaMemcpyHostToDevice));
    step = st;
  }

  void ensure_batch(int B) {
    if (B <= Bcap) return;
    for (void* p : bbufs) cudaFree(p);
    bbufs.clear();
    const int r = ts.widths[0], n = ts.n;
    int hmax = r, hid = r;
    for (int w : ts.widths) hmax = std::max(hmax, w);
    for (int l = 1; l < L; ++l) hid = std::max(hid, ts.widths[l]);
    const long long NC = (long long)B * Cs;
    D = alloc<Real>(bbufs, (size_t)n * B);
    Z = alloc<Real>(bbufs, (size_t)r * B);
    OUT = alloc<Real>(bbufs, (size_t)n * B);
    dOUT = alloc<Real>(bbufs, (size_t)n * B);
    dH = alloc<Real>(bbufs, (size_t)hmax * B);
    dH2 = alloc<Real>(bbufs, (size_t)hmax * B);
    A.assign(L, nullptr);
    Hh.assign(L, nullptr);
    Y.assign(L, nullptr);
    Zh.assign(L, nullptr);
    for (int l = 0; l + 1 < L; ++l) {
      A[l] = alloc<Real>(bbufs, (size_t)ts.widths[l + 1] * B);
      Hh[l] = alloc<Real>(bbufs, (size_t)ts.widths[l + 1] * B);
      Zh[l] = alloc<Real>(bbufs, (size_t)ts.widths[l + 1] * NC);
    }
    for (int l = 0; l < L; ++l) Y[l] = alloc<Real>(bbufs, (size_t)ts.widths[l] * NC);
    const int Hc = ts.widths[L - 1];
    WS = alloc<Real>(bbufs, (size_t)ts.RS * Hc);
    bS = alloc<Real>(bbufs, ts.RS);
    dWS = alloc<Real>(bbufs, (size_t)ts.RS * Hc);
    dbS = alloc<Real>(bbufs, ts.RS);
    XS = alloc<Real>(bbufs, (size_t)ts.RS * NC);
    dXS = alloc<Real>(bbufs, (size_t)ts.RS * NC);
    dY = alloc<Real>(bbufs, (size_t)hid * NC);
    dZh = alloc<Real>(bbufs, (size_t)hid * NC);
    contrib = alloc<Real>(bbufs, (size_t)B * ts.S * P);
    gx = alloc<Real>(bbufs, (size_t)B * ts.S * 12);
    gJ = alloc<Real>(bbufs, (size_t)B * ts.S * 12 * r);
    gk = alloc<Real>(bbufs, (size_t)B * ts.S * 12);
    Gbar = alloc<Real>(bbufs, (size_t)B * P);
    Hs = alloc<double>(bbufs, (size_t)B * P);
    lpart = alloc<double>(bbufs, B);
    rpart = alloc<double>(bbufs, 1024);
    Gm = alloc<Real>(bbufs, (size_t)B * B);
    G1 = alloc<Real>(bbufs, (size_t)B * r);
    Cm = alloc<Real>(bbufs, (size_t)B * B);
    epart = alloc<double>(bbufs, (size_t)B * ts.S);
    Bcap = B;
  }

  ElemCtx<Real> elem_ctx(int B) {
    ElemCtx<Real> ec;
    ec.S = ts.S;
    ec.r = ts.widths[0];
    ec.P = P;
    ec.B = B;
    ec.Cs = Cs;
    ec.RS = ts.RS;
    ec.tets = ctl;
    ec.dminv = cdminv;
    ec.wv = cwv;
    ec.XS = XS;
    ec.bS = bS;
    ec.X0S = X0S;
    ec.scale = (Real)ts.scale;
    ec.mu = (Real)ts.mu;
    ec.lam = (Real)ts.lam;
    ec.alpha = (Real)ts.alpha;
    return ec;
  }

  // forward second-order pass from Z to XS and the per-sample Hessians Hs
  void hessians(int B, cudaStream_t s) {
    const int r = ts.widths[0];
    const long long NC = (long long)B * Cs;
    so_init_kernel<Real><<<blocks(r * NC), 256, 0, s>>>(Z, r, B, Cs, Y[0]);
    for (int l = 0; l + 1 < L; ++l) {
      const int M = ts.widths[l + 1], K = ts.widths[l];
      mm(s, M, (int)NC, K, Real(1), theta + off[2 + 2 * l], K, 1, Y[l], NC, 1, Real(0),
                 Zh[l], NC);
      so_act_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(Zh[l], theta + off[3 + 2 * l],
                                                                   M, B, r, Cs, Y[l + 1]);
    }
    const int Hc = ts.widths[L - 1];
    gather_rows_kernel<Real><<<blocks((long long)ts.RS * Hc), 256, 0, s>>>(
        theta + off[2 + 2 * (L - 1)], theta + off[3 + 2 * (L - 1)], rows, ts.RS, Hc, WS, bS);
    mm(s, ts.RS, (int)NC, Hc, Real(1), WS, Hc, 1, Y[L - 1], NC, 1, Real(0), XS, NC);
    const long long warps = (long long)ts.S * B;
    elem_hess_kernel<Real><<<blocks(warps * 32, 128), 128, 0, s>>>(elem_ctx(B), contrib);
    sum_hess_kernel<Real><<<blocks((long long)B * P), 256, 0, s>>>(contrib, ts.S, B, P, Hs);
  }

  void hessians_host(const double* z, int B, double* Hout, cudaStream_t s) override {
    ensure_batch(B);
    const int r = ts.widths[0];
    std::vector<Real> zt((size_t)r * B);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < r; ++i) zt[(size_t)i * B + b] = (Real)z[(size_t)b * r + i];
    tck(cudaMemcpyAsync(Z, zt.data(), sizeof(Real) * zt.size(), cudaMemcpyHostToDevice, s));
    hessians(B, s);
    tck(cudaMemcpyAsync(Hout, Hs, sizeof(double) * (size_t)B * P, cudaMemcpyDeviceToHost, s));
    tck(cudaStreamSynchronize(s));
    tck(cudaGetLastError());
  }

  void evaluate(const double* q, int B, double lambda_ls, double* losses,
                cudaStream_t s) override {
    ensure_batch(B);
    const int r = ts.widths[0], n = ts.n;
    const Real one = Real(1), zero = Real(0);
    tck(cudaMemsetAsync(grad, 0, sizeof(Real) * nparams, s));
    // ---- reconstruction loss (Eq. 3) and its gradient
    snapshots_kernel<Real><<<blocks((long long)n * B), 256, 0, s>>>(q, ts.X0, n, B, D);
    mm(s, r, B, n, one, theta + off[0], n, 1, D, B, 1, zero, Z, B);
    bias_add_kernel<Real><<<blocks((long long)r * B), 256, 0, s>>>(Z, theta + off[1], r, B);
    const Real* hin = Z;
    for (int l = 0; l + 1 < L; ++l) {
      const int M = ts.widths[l + 1], K = ts.widths[l];
      mm(s, M, B, K, one, theta + off[2 + 2 * l], K, 1, hin, B, 1, zero, A[l], B);
      bias_elu_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(
          A[l], theta + off[3 + 2 * l], M, B, Hh[l]);
      hin = Hh[l];
    }
    const int Hc = ts.widths[L - 1];
    mm(s, n, B, Hc, one, theta + off[2 + 2 * (L - 1)], Hc, 1, hin, B, 1, zero, OUT, B);
    const int rb = 256;
    recon_kernel<Real><<<rb, 256, 0, s>>>(OUT, theta + off[3 + 2 * (L - 1)], D, ts.mass, n, B,
                                          (Real)ts.scale, dOUT, rpart);
    mm(s, n, Hc, B, one, dOUT, B, 1, hin, 1, B, zero, grad + off[2 + 2 * (L - 1)], Hc);
    rowsum_kernel<Real><<<blocks(n), 256, 0, s>>>(dOUT, n, B, B, 1, 0, one,
                                                  grad + off[3 + 2 * (L - 1)], 0);
    mm(s, Hc, B, n, one, theta + off[2 + 2 * (L - 1)], 1, Hc, dOUT, B, 1, zero, dH, B);
    Real* dcur = dH;
    Real* dnext = dH2;
    for (int l = L - 2; l >= 0; --l) {
      const int M = ts.widths[l + 1], K = ts.widths[l];
      elu_back_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(A[l], dcur,
                                                                     (long long)M * B);
      const Real* hprev = l == 0 ? Z : Hh[l - 1];
      mm(s, M, K, B, one, dcur, B, 1, hprev, 1, B, zero, grad + off[2 + 2 * l], K);
      rowsum_kernel<Real><<<blocks(M), 256, 0, s>>>(dcur, M, B, B, 1, 0, one,
                                                    grad + off[3 + 2 * l], 0);
      mm(s, K, B, M, one, theta + off[2 + 2 * l], 1, K, dcur, B, 1, zero, dnext, B);
      std::swap(dcur, dnext);
    }
    mm(s, r, n, B, one, dcur, B, 1, D, 1, B, zero, grad + off[0], n);
    rowsum_kernel<Real><<<blocks(r), 256, 0, s>>>(dcur, r, B, B, 1, 0, one, grad + off[1], 0);
    // ---- Lipschitz loss on the cubature Hessians (Eq. 9), or of the
    // potential itself (order 0)
    const double lls = lip_order == 0 ? lipschitz0_part(B, lambda_ls, hin, s)
                                      : lipschitz_part(B, lambda_ls, s, lip_order);
    std::vector<double> rp(rb);
    tck(cudaMemcpyAsync(rp.data(), rpart, sizeof(double) * rb, cudaMemcpyDeviceToHost, s));
    tck(cudaStreamSynchronize(s));
    tck(cudaGetLastError());
    double lc = 0.0;
    for (double v : rp) lc += v;
    lc /= B;
    losses[0] = lc;
    losses[1] = lls;
    losses[2] = lc + lambda_ls * lls;
  }

  // Eq. 9 at the samples held in Z (r x B): returns L_LS and adds
  // lambda_ls dL_LS/dtheta to the gradient (the samples held fixed)
  // order 2: Eq. 9 on the cubature Hessians; order 1: the same family on
  // the reduced gradients (the second-order columns of the pass carry zero
  // adjoints then)
  double lipschitz_part(int B, double lambda_ls, cudaStream_t s, int order = 2) {
    const int r = ts.widths[0], Hc = ts.widths[L - 1];
    const Real one = Real(1), zero = Real(0);
    double lls = 0.0;
    if (lambda_ls != 0.0 && B >= 2) {
      const Real lam = (Real)lambda_ls;
      const long long NC = (long long)B * Cs;
      hessians(B, s);
      const long long warps = (long long)ts.S * B;
      double l1 = 0.0;
      if (order == 1) {
        grad1_kernel<Real><<<blocks(warps * 32, 128), 128, 0, s>>>(elem_ctx(B), contrib);
        sum_hess_kernel<Real><<<blocks((long long)B * r), 256, 0, s>>>(contrib, ts.S, B, r, Hs);
        std::vector<double> gh((size_t)B * r);
        std::vector<Real> zt((size_t)r * B);
        tck(cudaMemcpyAsync(gh.data(), Hs, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost,
                            s));
        tck(cudaMemcpyAsync(zt.data(), Z, sizeof(Real) * zt.size(), cudaMemcpyDeviceToHost, s));
        tck(cudaStreamSynchronize(s));
        const double np = (double)B * (B - 1);
        std::vector<Real> gbar((size_t)B * r, Real(0));
        std::vector<double> acc((size_t)B * r, 0.0);
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j) {
            if (i == j) continue;
            double dz = 0.0, dg = 0.0;
            for (int k = 0; k < r; ++k) {
              const double d = (double)zt[(size_t)k * B + i] - (double)zt[(size_t)k * B + j];
              dz += d * d;
              const double q = gh[(size_t)i * r + k] - gh[(size_t)j * r + k];
              dg += q * q;
            }
            l1 += dg / dz;
            for (int k = 0; k < r; ++k)  // both orders of the pair (i, j)
              acc[(size_t)i * r + k] +=
                  4.0 * (gh[(size_t)i * r + k] - gh[(size_t)j * r + k]) / (np * dz);
          }
        l1 /= np;
        for (size_t q = 0; q < acc.size(); ++q) gbar[q] = (Real)acc[q];
        tck(cudaMemcpyAsync(G1, gbar.data(), sizeof(Real) * gbar.size(), cudaMemcpyHostToDevice,
                            s));
        tck(cudaMemsetAsync(gk, 0, sizeof(Real) * (size_t)B * ts.S * 12, s));
        tck(cudaMemsetAsync(Gbar, 0, sizeof(Real) * (size_t)B * P, s));
        elem_back1_kernel<Real><<<blocks(warps * 32, 128), 128, 0, s>>>(elem_ctx(B), G1, gx, gJ);
      } else {
        lls_kernel<Real><<<B, 128, 0, s>>>(Hs, Z, B, r, P, Gbar, lpart);
        elem_back_kernel<Real><<<blocks(warps * 32, 128), 128, 0, s>>>(elem_ctx(B), Gbar, gx,
                                                                        gJ, gk);
      }
      row_adjoint_kernel<Real><<<blocks((long long)ts.RS * B, 128), 128, 0, s>>>(
          inc_ptr, inc, ts.RS, ts.S, B, r, P, Cs, (Real)ts.scale, gx, gJ, gk, Gbar, dXS);
      mm(s, ts.RS, Hc, (int)NC, one, dXS, NC, 1, Y[L - 1], 1, NC, zero, dWS, Hc);
      rowsum_kernel<Real><<<blocks(ts.RS), 256, 0, s>>>(dXS, ts.RS, (int)NC, B, Cs, 0, one, dbS,
                                                        0);
      scatter_rows_kernel<Real><<<blocks((long long)ts.RS * Hc), 256, 0, s>>>(
          dWS, dbS, rows, ts.RS, Hc, lam, grad + off[2 + 2 * (L - 1)],
          grad + off[3 + 2 * (L - 1)]);
      mm(s, Hc, (int)NC, ts.RS, one, WS, 1, Hc, dXS, NC, 1, zero, dY, NC);
      for (int l = L - 2; l >= 0; --l) {
        const int M = ts.widths[l + 1], K = ts.widths[l];
        so_act_back_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(
            Zh[l], theta + off[3 + 2 * l], dY, M, B, r, Cs, dZh);
        mm(s, M, K, (int)NC, lam, dZh, NC, 1, Y[l], 1, NC, one, grad + off[2 + 2 * l], K);
        rowsum_kernel<Real><<<blocks(M), 256, 0, s>>>(dZh, M, (int)NC, B, Cs, 0, lam,
                                                      grad + off[3 + 2 * l], 1);
        if (l > 0)
          mm(s, K, (int)NC, M, one, theta + off[2 + 2 * l], 1, K, dZh, NC, 1, zero, dY,
                     NC);
      }
      if (order == 1) {
        lls = l1;
      } else {
        std::vector<double> lp(B);
        tck(cudaMemcpyAsync(lp.data(), lpart, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
        tck(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) lls += lp[b];
      }
    }
    return lls;
  }

  // The zeroth-order Lipschitz loss at the samples held in Z, with OUT (and
  // the activations) of the decoder forward at them: returns L_LS,0 and adds
  // lambda_ls dL_LS,0/dtheta to the decoder blocks of the gradient (the
  // samples held fixed: nothing flows into the encoder).
  double lipschitz0_part(int B, double lambda_ls, const Real* hin, cudaStream_t s) {
    if (lambda_ls == 0.0 || B < 2) return 0.0;
    const int r = ts.widths[0], S = ts.S;
    const double sc = ts.scale;
    unsup_elem_kernel<Real><<<blocks((long long)S * B, 128), 128, 0, s>>>(
        ctl, cdminv, cwv, rows, X0S, OUT, theta + off[3 + 2 * (L - 1)], S, B, (Real)sc,
        (Real)ts.mu, (Real)ts.lam, (Real)ts.alpha, epart, gx);
    std::vector<double> ep((size_t)S * B);
    std::vector<Real> zt((size_t)r * B);
    tck(cudaMemcpyAsync(ep.data(), epart, sizeof(double) * ep.size(), cudaMemcpyDeviceToHost, s));
    tck(cudaMemcpyAsync(zt.data(), Z, sizeof(Real) * zt.size(), cudaMemcpyDeviceToHost, s));
    tck(cudaStreamSynchronize(s));
    std::vector<double> Pb(B, 0.0), cb(B, 0.0);
    for (int b = 0; b < B; ++b)
      for (int e = 0; e < S; ++e) Pb[b] += ep[(size_t)b * S + e];
    const double np = (double)B * (B - 1);
    double l0 = 0.0;
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) {
        if (i == j) continue;
        double dz = 0.0;
        for (int k = 0; k < r; ++k) {
          const double d = (double)zt[(size_t)k * B + i] - (double)zt[(size_t)k * B + j];
          dz += d * d;
        }
        const double dp = Pb[i] - Pb[j];
        l0 += dp * dp / dz;
        cb[i] += 4.0 * dp / (np * dz);  // both orders of the pair (i, j)
      }
    l0 /= np;
    std::vector<Real> cr(cb.begin(), cb.end());
    tck(cudaMemcpyAsync(Cm, cr.data(), sizeof(Real) * B, cudaMemcpyHostToDevice, s));
    tck(cudaMemsetAsync(dOUT, 0, sizeof(Real) * (size_t)ts.n * B, s));
    unsup_row_kernel<Real><<<blocks((long long)ts.RS * B, 128), 128, 0, s>>>(
        inc_ptr, inc, rows, ts.RS, S, B, gx, (Real)(lambda_ls * sc), Cm, dOUT);
    backward_from_out(B, hin, s, true);
    return l0;
  }

  // decoder forward of the samples held in Z (r x B) to OUT (n x B)
  const Real* forward_out(int B, cudaStream_t s) {
    const Real one = Real(1), zero = Real(0);
    const Real* hin = Z;
    for (int l = 0; l + 1 < L; ++l) {
      const int M = ts.widths[l + 1], K = ts.widths[l];
      mm(s, M, B, K, one, theta + off[2 + 2 * l], K, 1, hin, B, 1, zero, A[l], B);
      bias_elu_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(
          A[l], theta + off[3 + 2 * l], M, B, Hh[l]);
      hin = Hh[l];
    }
    const int Hc = ts.widths[L - 1];
    mm(s, ts.n, B, Hc, one, theta + off[2 + 2 * (L - 1)], Hc, 1, hin, B, 1, zero, OUT, B);
    return hin;
  }

  // gradient of the decoder parameters from the adjoint dOUT (n x B) of OUT
  // (accumulate: add to the gradient instead of overwriting the decoder blocks)
  void backward_from_out(int B, const Real* hin, cudaStream_t s, bool accumulate = false) {
    const Real one = Real(1), zero = Real(0), beta = accumulate ? one : zero;
    const int n = ts.n, Hc = ts.widths[L - 1];
    mm(s, n, Hc, B, one, dOUT, B, 1, hin, 1, B, beta, grad + off[2 + 2 * (L - 1)], Hc);
    rowsum_kernel<Real><<<blocks(n), 256, 0, s>>>(dOUT, n, B, B, 1, 0, one,
                                                  grad + off[3 + 2 * (L - 1)], accumulate);
    mm(s, Hc, B, n, one, theta + off[2 + 2 * (L - 1)], 1, Hc, dOUT, B, 1, zero, dH, B);
    Real* dcur = dH;
    Real* dnext = dH2;
    for (int l = L - 2; l >= 0; --l) {
      const int M = ts.widths[l + 1], K = ts.widths[l];
      elu_back_kernel<Real><<<blocks((long long)M * B), 256, 0, s>>>(A[l], dcur,
                                                                     (long long)M * B);
      const Real* hprev = l == 0 ? Z : Hh[l - 1];
      mm(s, M, K, B, one, dcur, B, 1, hprev, 1, B, beta, grad + off[2 + 2 * l], K);
      rowsum_kernel<Real><<<blocks(M), 256, 0, s>>>(dcur, M, B, B, 1, 0, one,
                                                    grad + off[3 + 2 * l], accumulate);
      if (l > 0)
        mm(s, K, B, M, one, theta + off[2 + 2 * l], 1, K, dcur, B, 1, zero, dnext, B);
      std::swap(dcur, dnext);
    }
  }

  void evaluate_unsup(const double* z, int B, double lambda, double sigma, double lambda_ls,
                      double* losses, cudaStream_t s) override {
    ensure_batch(B);
    const int r = ts.widths[0], n = ts.n, S = ts.S;
    const Real one = Real(1), zero = Real(0);
    const double sc = ts.scale;
    tck(cudaMemsetAsync(grad, 0, sizeof(Real) * nparams, s));
    std::vector<Real> zt((size_t)r * B);
    for (int b = 0; b < B; ++b)
      for (int i = 0; i < r; ++i) zt[(size_t)i * B + b] = (Real)z[(size_t)b * r + i];
    tck(cudaMemcpyAsync(Z, zt.data(), sizeof(Real) * zt.size(), cudaMemcpyHostToDevice, s));
    const Real* hin = forward_out(B, s);
    // repulsion: Gram G = OUT^T M OUT, ||x_i - x_j||_M^2 = s^2 (G_ii + G_jj - 2 G_ij)
    double lr_sum = 0.0;
    std::vector<double> cmat((size_t)B * B, 0.0);
    if (B >= 2) {
      mass_rows_kernel<Real><<<blocks((long long)n * B), 256, 0, s>>>(OUT, ts.mass, n, B, one, D);
      mm(s, B, B, n, one, OUT, 1, B, D, B, 1, zero, Gm, B);
      std::vector<Real> G((size_t)B * B);
      tck(cudaMemcpyAsync(G.data(), Gm, sizeof(Real) * G.size(), cudaMemcpyDeviceToHost, s));
      tck(cudaStreamSynchronize(s));
      const double np = (double)B * (B - 1);
      std::vector<double> c((size_t)B * B, 0.0);
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
          if (i == j) continue;
          const double dm = sc * sc * ((double)G[i * B + i] + (double)G[j * B + j] -
                                       2.0 * (double)G[i * B + j]);
          double dz = 0.0;
          for (int k = 0; k < r; ++k) {
            const double d = z[(size_t)i * r + k] - z[(size_t)j * r + k];
            dz += d * d;
          }
          const double ell = 0.5 * std::log(dm) - std::log(sigma) - 0.5 * std::log(dz);
          lr_sum += ell * ell;
          c[(size_t)i * B + j] = ell / (np * dm);  // dL_R / d(dm_ij)
        }
      // dL_R/dOUT_i = sum_j (c_ij + c_ji) 2 s^2 M (OUT_i - OUT_j): OUT times
      // (diag(row sums of C + C^T) - (C + C^T))
      for (int i = 0; i < B; ++i) {
        double d = 0.0;
        for (int j = 0; j < B; ++j) {
          if (i == j) continue;
          const double cs = c[(size_t)i * B + j] + c[(size_t)j * B + i];
          cmat[(size_t)j * B + i] = -cs;  // column i: sample i's adjoint
          d += cs;
        }
        cmat[(size_t)i * B + i] = d;
      }
      lr_sum /= np;
      std::vector<Real> cr(cmat.begin(), cmat.end());
      tck(cudaMemcpyAsync(Cm, cr.data(), sizeof(Real) * cr.size(), cudaMemcpyHostToDevice, s));
      mm(s, n, B, B, one, OUT, B, 1, Cm, B, 1, zero, D, B);
      mass_rows_kernel<Real><<<blocks((long long)n * B), 256, 0, s>>>(
          D, ts.mass, n, B, (Real)(2.0 * lambda * sc * sc), dOUT);
    } else {
      tck(cudaMemsetAsync(dOUT, 0, sizeof(Real) * (size_t)n * B, s));
    }
    // potential: per (tet, sample) energies and derivatives on the cubature rows
    unsup_elem_kernel<Real><<<blocks((long long)S * B, 128), 128, 0, s>>>(
        ctl, cdminv, cwv, rows, X0S, OUT, theta + off[3 + 2 * (L - 1)], S, B, (Real)sc,
        (Real)ts.mu, (Real)ts.lam, (Real)ts.alpha, epart, gx);
    unsup_row_kernel<Real><<<blocks((long long)ts.RS * B, 128), 128, 0, s>>>(
        inc_ptr, inc, rows, ts.RS, S, B, gx, (Real)(sc / B), nullptr, dOUT);
    backward_from_out(B, hin, s);
    const double lls = lipschitz_part(B, lambda_ls, s);
    std::vector<double> ep((size_t)S * B);
    tck(cudaMemcpyAsync(ep.data(), epart, sizeof(double) * ep.size(), cudaMemcpyDeviceToHost, s));
    tck(cudaStreamSynchronize(s));
    tck(cudaGetLastError());
    double lp = 0.0;
    for (double v : ep) lp += v;
    lp /= B;
    losses[0] = lp;
    losses[1] = lr_sum;
    losses[2] = lp + lambda * lr_sum;
    losses[3] = lls;
    losses[4] = losses[2] + lambda_ls * lls;
  }

  void adam(double lr, cudaStream_t s) override {
    step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const double c1 = 1.0 - std::pow(b1, (double)step), c2 = 1.0 - std::pow(b2, (double)step);
    adam_kernel<Real><<<blocks(nparams), 256, 0, s>>>(theta, grad, am, av, nparams, (Real)lr,
                                                      (Real)b1, (Real)b2, (Real)1e-8, (Real)c1,
                                                      (Real)c2);
    tck(cudaGetLastError());
  }
};

}  // namespace

TrainerBase* TrainerBase::create(int mode, const TrainSetup& ts) {
  if (mode == 1) return new Trainer<double>(ts);
  Trainer<float>* t = new Trainer<float>(ts);
  t->tf32 = mode == 2 || mode == 3;
  t->bf16ops = mode == 3;
  return t;
}

}  // namespace lsn
