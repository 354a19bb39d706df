// Decoder MLP with forward-mode Jacobian (the subspace map f_theta of
// Sec. 3.1, differentiated as the paper's autodiff does, Sec. 5), FP32/FP64
// CUDA-core form.
//
// Every layer is one GEMM  out[c][m] = sum_k W[m][k] Z[c][k]  whose columns
// c carry either the value and the r tangent directions (Jacobian pass,
// C = r + 1 columns: Z_0 = [z | I_r]) or k independent values (line-search
// pass, C = k columns: z + alpha_j d).  Column-major activations Z[c][k]
// (leading dimension = layer width) keep both operands of the k-loop
// contiguous.  Epilogues:
//   HiddenJac  a = acc_0 + b,  h = ELU(a),  T_c = ELU'(a) acc_c
//   HiddenVal  h_c = ELU(acc_c + b)
//   LastJac    u = s (acc_0 + b), J_c = s acc_c, constrained rows replaced by
//              target displacement / zero, then the per-row inertia, gravity
//              and ground terms are folded into per-CTA partials of
//              (E, sum|E|, g = J^T gv, K = J^T diag(kv) J)  (fixed order)
//   LastVal    u_j = s (acc_j + b), constraints, per-trial energy partials.
// Positions are handled as displacements u = x - X0, and the inertia term as
// u - (qbar - X0), so that FP32 arithmetic works on small numbers.
#include "lsn_internal.cuh"

#include <algorithm>

namespace lsn {

namespace {

template <typename Real>
__device__ __forceinline__ Real elu_f(Real a) {
  return a > Real(0) ? a : (Real)expm1(a);
}
template <>
__device__ __forceinline__ float elu_f<float>(float a) {
  return a > 0.f ? a : expm1f(a);
}
template <typename Real>
__device__ __forceinline__ Real elu_d(Real a) {
  return a > Real(0) ? Real(1) : (Real)exp(a);
}
template <>
__device__ __forceinline__ float elu_d<float>(float a) {
  return a > 0.f ? 1.f : expf(a);
}

__device__ __forceinline__ void pair_of(int p, int r, int& i, int& j) {
  i = 0;
  while (p >= r - i) {
    p -= r - i;
    ++i;
  }
  j = i + p;
}

constexpr int NT = 256;  // threads per CTA

template <typename Real, int TN, int TM>
struct Tile {
  static constexpr int CP = 16 * TN;
  static constexpr int BM = 16 * TM;
  static constexpr int BK = GEMM_BK;
  static constexpr int WS = BK * (BM + 1);
  static constexpr int ZS = BK * CP;
};

// Accumulate the BM x CP tile at rows m0.. for all k.
template <typename Real, int TN, int TM>
__device__ __forceinline__ void gemm_tile(const Real* __restrict__ W, int M, int K,
                                          const Real* __restrict__ Zin, int C, int m0,
                                          Real* Ws, Real* Zs, Real (&acc)[TM][TN]) {
  using T = Tile<Real, TN, TM>;
  const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Real(0);
  for (int k0 = 0; k0 < K; k0 += T::BK) {
    for (int e = t; e < T::BM * T::BK; e += NT) {
      int row = e / T::BK, kk = e % T::BK, gr = m0 + row, gk = k0 + kk;
      Ws[kk * (T::BM + 1) + row] = (gr < M && gk < K) ? W[(size_t)gr * K + gk] : Real(0);
    }
    for (int e = t; e < T::CP * T::BK; e += NT) {
      int c = e / T::BK, kk = e % T::BK, gk = k0 + kk;
      Zs[kk * T::CP + c] = (c < C && gk < K) ? Zin[(size_t)c * K + gk] : Real(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < T::BK; ++kk) {
      Real wv[TM], zv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) wv[i] = Ws[kk * (T::BM + 1) + rg + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) zv[j] = Zs[kk * T::CP + cg + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += wv[i] * zv[j];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ hidden layers
template <typename Real, int TN, bool JAC>
__global__ void __launch_bounds__(NT) hidden_kernel(const Real* __restrict__ W,
                                                    const Real* __restrict__ b, int M,
                                                    int K, const Real* __restrict__ Zin,
                                                    int C, Real* __restrict__ Zout,
                                                    int ldo) {
  using T = Tile<Real, TN, 1>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Ws = reinterpret_cast<Real*>(smem_raw);
  Real* Zs = Ws + T::WS;
  Real* e1s = Zs + T::ZS;
  const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
  const int m0 = blockIdx.x * T::BM;
  Real acc[1][TN];
  gemm_tile<Real, TN, 1>(W, M, K, Zin, C, m0, Ws, Zs, acc);
  const int m = m0 + rg;
  if (JAC) {
    if (cg == 0 && m < M) {
      Real a = acc[0][0] + b[m];
      e1s[rg] = elu_d<Real>(a);
      Zout[m] = elu_f<Real>(a);
    }
    __syncthreads();
    if (m < M) {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int c = cg + 16 * j;
        if (c >= 1 && c < C) Zout[(size_t)c * ldo + m] = e1s[rg] * acc[0][j];
      }
    }
  } else if (m < M) {
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int c = cg + 16 * j;
      if (c < C) Zout[(size_t)c * ldo + m] = elu_f<Real>(acc[0][j] + b[m]);
    }
  }
}

// Per-row energy, force and stiffness scalars of the terms that act on each
// DOF separately: inertia (dynamics) or gravity (quasi-static), and ground.
__device__ __forceinline__ void row_terms(const LastArgs& la, int m, double u, double& e,
                                          double& gv, double& kv) {
  const int v = m / 3, comp = m - 3 * v;
  const double mv = la.mass[v];
  if (la.inv_dt2 > 0.0) {
    double diff = u - la.ubar[m];
    e = 0.5 * la.inv_dt2 * mv * diff * diff;
    gv = la.inv_dt2 * mv * diff;
    kv = la.inv_dt2 * mv;
  } else {
    e = -mv * la.grav[comp] * u;
    gv = -mv * la.grav[comp];
    kv = 0.0;
  }
  if (la.ground_k > 0.0 && comp == 2) {
    double pen = la.X0[m] + u - la.ground_h;
    if (pen < 0.0) {
      e += 0.5 * la.ground_k * pen * pen;
      gv += la.ground_k * pen;
      kv += la.ground_k;
    }
  }
}

// ------------------------------------------------------------ output layer
template <typename Real, int TN>
__global__ void __launch_bounds__(NT) last_jac_kernel(const Real* __restrict__ W,
                                                      const Real* __restrict__ b, int M,
                                                      int K, const Real* __restrict__ Zin,
                                                      int C, Real* __restrict__ u_out,
                                                      Real* __restrict__ J_out,
                                                      double* __restrict__ part,
                                                      int part_stride, LastArgs la) {
  constexpr int TM = 4;
  using T = Tile<Real, TN, TM>;
  constexpr int BM = T::BM, CP = T::CP, OS = CP + 1;
  constexpr int PQ = (16 * TN * (16 * TN + 1) / 2 + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Ws = reinterpret_cast<Real*>(smem_raw);
  Real* Zs = Ws + T::WS;
  Real* Os = Zs + T::ZS;                                   // BM x OS
  double* gvs = reinterpret_cast<double*>(Os + BM * OS + (BM * OS) % 2);
  double* kvs = gvs + BM;
  double* red = kvs + BM;                                  // NT * 2
  const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
  const int r = la.r;
  const int np = npairs(r);
  int pi[PQ], pj[PQ];
  double kacc[PQ];
#pragma unroll
  for (int q = 0; q < PQ; ++q) {
    int p = t + NT * q;
    if (p < np) pair_of(p, r, pi[q], pj[q]);
    else pi[q] = pj[q] = -1;
    kacc[q] = 0.0;
  }
  double gacc = 0.0, gabs = 0.0, eacc = 0.0, eabs = 0.0;
  const int ntiles = (M + BM - 1) / BM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int m0 = tile * BM;
    Real acc[TM][TN];
    gemm_tile<Real, TN, TM>(W, M, K, Zin, C, m0, Ws, Zs, acc);
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int row = rg + 16 * i, c = cg + 16 * j, m = m0 + row;
        Real val = acc[i][j];
        if (c == 0 && m < M) val += b[m];
        Os[row * OS + c] = (Real)(la.scale * (double)val);
      }
    __syncthreads();
    if (t < BM) {
      const int m = m0 + t;
      double gv = 0.0, kv = 0.0;
      if (m < M) {
        const int v = m / 3, comp = m - 3 * v;
        const int slot = la.cslot[v];
        if (slot >= 0) {
          Os[t * OS] = (Real)la.cu[3 * slot + comp];
          for (int c = 1; c < C; ++c) Os[t * OS + c] = Real(0);
        }
        double e;
        row_terms(la, m, (double)Os[t * OS], e, gv, kv);
        eacc += e;
        eabs += fabs(e);
      }
      gvs[t] = gv;
      kvs[t] = kv;
    }
    __syncthreads();
    const int rows = min(BM, M - m0);
    for (int e = t; e < rows; e += NT) u_out[m0 + e] = Os[e * OS];
    for (int e = t; e < rows * r; e += NT) {
      int row = e / r, c = e - row * r;
      J_out[(size_t)(m0 + row) * r + c] = Os[row * OS + 1 + c];
    }
    if (t < r) {
      double s = 0.0, a = 0.0;
      for (int row = 0; row < rows; ++row) {
        const double term = gvs[row] * (double)Os[row * OS + 1 + t];
        s += term;
        a += fabs(term);
      }
      gacc += s;
      gabs += a;
    }
#pragma unroll
    for (int q = 0; q < PQ; ++q) {
      if (pi[q] >= 0) {
        double s = 0.0;
        const int i = 1 + pi[q], j = 1 + pj[q];
        for (int row = 0; row < rows; ++row)
          s += kvs[row] * (double)Os[row * OS + i] * (double)Os[row * OS + j];
        kacc[q] += s;
      }
    }
    __syncthreads();
  }
  // block reduction of the energy scalars, then one partial row per CTA
  red[t] = eacc;
  red[NT + t] = eabs;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (t < s) {
      red[t] += red[t + s];
      red[NT + t] += red[NT + t + s];
    }
    __syncthreads();
  }
  double* prow = part + (size_t)blockIdx.x * part_stride;
  if (t == 0) {
    prow[0] = red[0];
    prow[1] = red[NT];
  }
  if (t < r) {
    prow[slot_g(t)] = gacc;
    prow[slot_gabs(r, t)] = gabs;
  }
#pragma unroll
  for (int q = 0; q < PQ; ++q)
    if (pi[q] >= 0) prow[slot_K(r) + t + NT * q] = kacc[q];
}

template <typename Real>
__global__ void __launch_bounds__(NT) last_val_kernel(const Real* __restrict__ W,
                                                      const Real* __restrict__ b, int M,
                                                      int K, const Real* __restrict__ Zin,
                                                      int C, Real* __restrict__ u_trial,
                                                      double* __restrict__ part,
                                                      int part_stride, LastArgs la) {
  constexpr int TM = 4, TN = 1;
  using T = Tile<Real, TN, TM>;
  constexpr int BM = T::BM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Ws = reinterpret_cast<Real*>(smem_raw);
  Real* Zs = Ws + T::WS;
  double* red = reinterpret_cast<double*>(Zs + T::ZS + (T::ZS % 2));  // 2 * NT
  const int t = threadIdx.x, cg = t & 15, rg = t >> 4;
  double eacc = 0.0, eabs = 0.0;
  const int ntiles = (M + BM - 1) / BM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int m0 = tile * BM;
    Real acc[TM][TN];
    gemm_tile<Real, TN, TM>(W, M, K, Zin, C, m0, Ws, Zs, acc);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + rg + 16 * i;
      if (m < M && cg < C) {
        const int v = m / 3, comp = m - 3 * v;
        const int slot = la.cslot[v];
        double u = slot >= 0 ? la.cu[3 * slot + comp]
                             : (double)(Real)(la.scale * (double)(acc[i][0] + b[m]));
        Real ur = (Real)u;
        u_trial[(size_t)cg * M + m] = ur;
        double e, gv, kv;
        row_terms(la, m, (double)ur, e, gv, kv);
        eacc += e;
        eabs += fabs(e);
      }
    }
  }
  red[t] = eacc;
  red[NT + t] = eabs;
  __syncthreads();
  if (t < 16) {  // column t: sum over the 16 row groups
    double s = 0.0, a = 0.0;
    for (int g = 0; g < 16; ++g) {
      s += red[g * 16 + t];
      a += red[NT + g * 16 + t];
    }
    if (t < C) {
      part[(size_t)blockIdx.x * part_stride + 2 * t] = s;
      part[(size_t)blockIdx.x * part_stride + 2 * t + 1] = a;
    }
  }
}

template <typename Real, int TN>
size_t hidden_smem() {
  using T = Tile<Real, TN, 1>;
  return (T::WS + T::ZS + T::BM) * sizeof(Real);
}
template <typename Real, int TN>
size_t last_jac_smem() {
  using T = Tile<Real, TN, 4>;
  size_t reals = T::WS + T::ZS + T::BM * (T::CP + 1);
  reals += reals % 2;
  return reals * sizeof(Real) + (2 * T::BM + 2 * NT) * sizeof(double);
}
template <typename Real>
size_t last_val_smem() {
  using T = Tile<Real, 1, 4>;
  size_t reals = T::WS + T::ZS;
  reals += reals % 2;
  return reals * sizeof(Real) + 2 * NT * sizeof(double);
}

template <typename Real, int TN>
void run_hidden(bool jac, const Real* W, const Real* b, int M, int K, const Real* Zin,
                int C, Real* Zout, int ldo, cudaStream_t s) {
  size_t sm = hidden_smem<Real, TN>();
  int grid = (M + 15) / 16;
  if (jac) {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(hidden_kernel<Real, TN, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set = true;
    }
    hidden_kernel<Real, TN, true><<<grid, NT, sm, s>>>(W, b, M, K, Zin, C, Zout, ldo);
  } else {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(hidden_kernel<Real, TN, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set = true;
    }
    hidden_kernel<Real, TN, false><<<grid, NT, sm, s>>>(W, b, M, K, Zin, C, Zout, ldo);
  }
}

template <typename Real, int TN>
void run_last_jac(const Real* W, const Real* b, int M, int K, const Real* Zin, int C,
                  Real* u_out, Real* J_out, double* part, int stride, const LastArgs& la,
                  int grid, cudaStream_t s) {
  size_t sm = last_jac_smem<Real, TN>();
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(last_jac_kernel<Real, TN>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = true;
  }
  last_jac_kernel<Real, TN><<<grid, NT, sm, s>>>(W, b, M, K, Zin, C, u_out, J_out, part,
                                                 stride, la);
}

}  // namespace

int decoder_cpad(int C) { return 16 * ((C + 15) / 16); }

int decoder_last_grid(int n, int C, int num_sms) {
  int tiles = (n + 63) / 64;
  int cap = num_sms * (C > 48 ? 1 : 2);
  return std::max(1, std::min(tiles, cap));
}

template <typename Real>
void launch_decoder_layer(Epi epi, const Real* W, const Real* b, int M, int K,
                          const Real* Zin, int C, Real* Zout, int ldo, Real* u_out,
                          Real* J_out, double* part, int part_stride,
                          const LastArgs& la, int grid, cudaStream_t s) {
  const int tn = (C + 15) / 16;
  switch (epi) {
    case Epi::HiddenJac:
    case Epi::HiddenVal: {
      bool jac = epi == Epi::HiddenJac;
      switch (tn) {
        case 1: run_hidden<Real, 1>(jac, W, b, M, K, Zin, C, Zout, ldo, s); break;
        case 2: run_hidden<Real, 2>(jac, W, b, M, K, Zin, C, Zout, ldo, s); break;
        case 3: run_hidden<Real, 3>(jac, W, b, M, K, Zin, C, Zout, ldo, s); break;
        case 4: run_hidden<Real, 4>(jac, W, b, M, K, Zin, C, Zout, ldo, s); break;
        default: run_hidden<Real, 5>(jac, W, b, M, K, Zin, C, Zout, ldo, s); break;
      }
      break;
    }
    case Epi::LastJac:
      switch (tn) {
        case 1: run_last_jac<Real, 1>(W, b, M, K, Zin, C, u_out, J_out, part, part_stride, la, grid, s); break;
        case 2: run_last_jac<Real, 2>(W, b, M, K, Zin, C, u_out, J_out, part, part_stride, la, grid, s); break;
        case 3: run_last_jac<Real, 3>(W, b, M, K, Zin, C, u_out, J_out, part, part_stride, la, grid, s); break;
        case 4: run_last_jac<Real, 4>(W, b, M, K, Zin, C, u_out, J_out, part, part_stride, la, grid, s); break;
        default: run_last_jac<Real, 5>(W, b, M, K, Zin, C, u_out, J_out, part, part_stride, la, grid, s); break;
      }
      break;
    case Epi::LastVal: {
      size_t sm = last_val_smem<Real>();
      last_val_kernel<Real><<<grid, NT, sm, s>>>(W, b, M, K, Zin, C, Zout, part,
                                                 part_stride, la);
      break;
    }
  }
}

template void launch_decoder_layer<float>(Epi, const float*, const float*, int, int,
                                          const float*, int, float*, int, float*, float*,
                                          double*, int, const LastArgs&, int,
                                          cudaStream_t);
template void launch_decoder_layer<double>(Epi, const double*, const double*, int, int,
                                           const double*, int, double*, int, double*,
                                           double*, double*, int, const LastArgs&, int,
                                           cudaStream_t);

}  // namespace lsn
