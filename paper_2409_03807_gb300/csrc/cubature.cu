// Optimised cubature selection (Sec. 4.3: the cubature set and its weights
// are fitted on the initial subspace, after von Tycowicz et al. 2013;
// cubature-count trade-off, Sec. 5.3).
//
// Input: the per-tet reduced elastic forces A (m = K r rows: snapshot k,
// subspace column i; one column per tet, row-major [m][ne], device, FP64)
// from launch_tet_forces at K subspace points.  The target is the full
// force b = A 1.  Each snapshot's r rows of A and b are divided by ||b_k||
// so every snapshot counts alike.  The fit is the non-negative least-squares
// problem min ||A w - b||, w >= 0, solved by the Lawson-Hanson active-set
// method, which moves one column (the largest entry of A^T (b - A w)) into
// the active set per outer iteration; it stops once S columns are active.
// The active columns are the cubature tets, their values the weights.
//
// The scores A^T res (one pass over A per outer iteration) run on the GPU;
// the least-squares solves on the active set (at most S columns) run on the
// host in FP64 with an incrementally extended Cholesky factor of the active
// columns' Gram matrix (rebuilt when a column leaves the set).
#include <cmath>
#include <vector>

#include "lsn_internal.cuh"

namespace lsn {
namespace {

constexpr int CT = 256;

// b[row] = sum_e A[row][e] (fixed order: thread strides, then a tree)
__global__ void __launch_bounds__(CT) row_sum_kernel(const double* __restrict__ A, int ne,
                                                     double* __restrict__ b) {
  __shared__ double red[CT];
  const int row = blockIdx.x, t = threadIdx.x;
  double s = 0.0;
  for (int e = t; e < ne; e += CT) s += A[(size_t)row * ne + e];
  red[t] = s;
  __syncthreads();
  for (int h = CT / 2; h > 0; h >>= 1) {
    if (t < h) red[t] += red[t + h];
    __syncthreads();
  }
  if (t == 0) b[row] = red[0];
}

__global__ void scale_rows_kernel(double* __restrict__ A, int m, int ne,
                                  const double* __restrict__ scale) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)m * ne) return;
  A[i] *= scale[i / ne];
}

// w[e] = sum_row A[row][e] res[row]; res staged in shared memory in chunks
__global__ void __launch_bounds__(CT) scores_kernel(const double* __restrict__ A, int m, int ne,
                                                    const double* __restrict__ res,
                                                    double* __restrict__ w) {
  __shared__ double rs[1024];
  const int e = blockIdx.x * CT + threadIdx.x;
  double s = 0.0;
  for (int r0 = 0; r0 < m; r0 += 1024) {
    const int rn = min(1024, m - r0);
    __syncthreads();
    for (int i = threadIdx.x; i < rn; i += CT) rs[i] = res[r0 + i];
    __syncthreads();
    if (e < ne)
      for (int i = 0; i < rn; ++i) s += A[(size_t)(r0 + i) * ne + e] * rs[i];
  }
  if (e < ne) w[e] = s;
}

// Cholesky factor L (row-major, n x n, lower) of the Gram matrix G; false if
// a pivot is not positive.
bool cholesky(const std::vector<double>& G, int n, std::vector<double>& L) {
  L.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = G[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = G[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  return true;
}

// solve L L^T s = c
void chol_solve(const std::vector<double>& L, int n, const std::vector<double>& c,
                std::vector<double>& s) {
  s = c;
  for (int i = 0; i < n; ++i) {
    double v = s[i];
    for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * s[k];
    s[i] = v / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = s[i];
    for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * s[k];
    s[i] = v / L[(size_t)i * n + i];
  }
}

struct CubFail {
  cudaError_t e;
};
inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CubFail{e};
}
// device scratch freed on every exit path
struct DevBuf {
  double* p = nullptr;
  explicit DevBuf(size_t count) { ck(cudaMalloc(&p, sizeof(double) * (count ? count : 1))); }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

}  // namespace

cudaError_t cubature_normalise(double* A, int m, int ne, int r, std::vector<double>& b,
                               cudaStream_t s) try {
  DevBuf bdb(m), scb(m);
  double* bd = bdb.p;
  double* sc = scb.p;
  row_sum_kernel<<<m, CT, 0, s>>>(A, ne, bd);
  b.resize(m);
  ck(cudaMemcpyAsync(b.data(), bd, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  std::vector<double> scale(m, 1.0);
  for (int k = 0; k < m / r; ++k) {
    double nb = 0.0;
    for (int i = 0; i < r; ++i) nb += b[k * r + i] * b[k * r + i];
    nb = std::sqrt(nb);
    if (nb > 0.0)
      for (int i = 0; i < r; ++i) {
        scale[k * r + i] = 1.0 / nb;
        b[k * r + i] /= nb;
      }
  }
  ck(cudaMemcpyAsync(sc, scale.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
  const size_t cnt = (size_t)m * ne;
  scale_rows_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(A, m, ne, sc);
  ck(cudaGetLastError());
  ck(cudaStreamSynchronize(s));
  return cudaSuccess;
} catch (const CubFail& f) {
  return f.e;
}

cudaError_t cubature_nnls(const double* A, int m, int ne, const std::vector<double>& b, int S,
                          std::vector<int>& P, std::vector<double>& xP, double& rel,
                          cudaStream_t s) try {
  DevBuf resb(m), wb(ne);
  double* resd = resb.p;
  double* wd = wb.p;
  std::vector<double> res(b), w(ne), col(m);
  std::vector<char> excluded(ne, 0);  // active, or dependent on the active set
  std::vector<std::vector<double>> cols;
  std::vector<double> G, L, c, sol;
  P.clear();
  xP.clear();
  auto scores = [&]() {
    ck(cudaMemcpyAsync(resd, res.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    scores_kernel<<<(ne + CT - 1) / CT, CT, 0, s>>>(A, m, ne, resd, wd);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(w.data(), wd, sizeof(double) * ne, cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
  };
  scores();
  double wmax = 0.0;
  for (int e = 0; e < ne; ++e) wmax = std::fmax(wmax, std::fabs(w[e]));
  const double tol = 1e-12 * std::fmax(1.0, wmax);
  const int max_inner = 3 * ne;
  while ((int)P.size() < S) {
    int j = -1;
    for (int e = 0; e < ne; ++e)
      if (!excluded[e] && (j < 0 || w[e] > w[j])) j = e;
    if (j < 0 || !(w[j] > tol)) break;
    // column j (strided copy out of the row-major matrix)
    ck(cudaMemcpy2DAsync(col.data(), sizeof(double), A + j, sizeof(double) * ne,
                         sizeof(double), m, cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    excluded[j] = 1;
    // extend the Gram matrix and its factor; a column dependent on the
    // active ones (non-positive pivot) is left out
    const int n = (int)P.size();
    std::vector<double> g(n);
    for (int i = 0; i < n; ++i) g[i] = dot(cols[i], col);
    const double gjj = dot(col, col);
    std::vector<double> l(g);
    for (int i = 0; i < n; ++i) {
      double v = l[i];
      for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * l[k];
      l[i] = v / L[(size_t)i * n + i];
    }
    const double d2 = gjj - dot(l, l);
    if (!(d2 > 1e-14 * gjj)) continue;
    std::vector<double> G2((size_t)(n + 1) * (n + 1)), L2((size_t)(n + 1) * (n + 1), 0.0);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) {
        G2[(size_t)i * (n + 1) + k] = G[(size_t)i * n + k];
        L2[(size_t)i * (n + 1) + k] = L[(size_t)i * n + k];
      }
    for (int i = 0; i < n; ++i) {
      G2[(size_t)i * (n + 1) + n] = G2[(size_t)n * (n + 1) + i] = g[i];
      L2[(size_t)n * (n + 1) + i] = l[i];
    }
    G2[(size_t)n * (n + 1) + n] = gjj;
    L2[(size_t)n * (n + 1) + n] = std::sqrt(d2);
    G.swap(G2);
    L.swap(L2);
    P.push_back(j);
    cols.push_back(col);
    c.push_back(dot(col, b));
    xP.push_back(0.0);
    // inner loop: least squares on the active set; step back into the
    // feasible region and drop columns that reach zero
    for (int it = 0; it < max_inner && !P.empty(); ++it) {
      const int na = (int)P.size();
      chol_solve(L, na, c, sol);
      bool pos = true;
      for (int i = 0; i < na; ++i) pos = pos && sol[i] > 0.0;
      if (pos) {
        xP = sol;
        break;
      }
      double alpha = 1e300;
      for (int i = 0; i < na; ++i)
        if (sol[i] <= 0.0) alpha = std::fmin(alpha, xP[i] / (xP[i] - sol[i]));
      std::vector<int> keep;
      for (int i = 0; i < na; ++i) {
        xP[i] += alpha * (sol[i] - xP[i]);
        if (xP[i] > 1e-15) keep.push_back(i);
        else excluded[P[i]] = 0;  // back among the candidates
      }
      const int nk = (int)keep.size();
      std::vector<int> P2(nk);
      std::vector<double> x2(nk), c2(nk), G3((size_t)nk * nk);
      std::vector<std::vector<double>> cols2(nk);
      for (int a = 0; a < nk; ++a) {
        P2[a] = P[keep[a]];
        x2[a] = xP[keep[a]];
        c2[a] = c[keep[a]];
        cols2[a].swap(cols[keep[a]]);
        for (int bb = 0; bb < nk; ++bb) G3[(size_t)a * nk + bb] = G[(size_t)keep[a] * na + keep[bb]];
      }
      P.swap(P2);
      xP.swap(x2);
      c.swap(c2);
      cols.swap(cols2);
      G.swap(G3);
      if (nk > 0 && !cholesky(G, nk, L)) break;
    }
    // residual b - A_P x_P
    res = b;
    for (size_t a = 0; a < P.size(); ++a)
      for (int i = 0; i < m; ++i) res[i] -= cols[a][i] * xP[a];
    scores();
  }
  double nr = 0.0, nb = 0.0;
  for (int i = 0; i < m; ++i) {
    nr += res[i] * res[i];
    nb += b[i] * b[i];
  }
  rel = nb > 0.0 ? std::sqrt(nr / nb) : std::sqrt(nr);
  return cudaSuccess;
} catch (const CubFail& f) {
  return f.e;
}

}  // namespace lsn
