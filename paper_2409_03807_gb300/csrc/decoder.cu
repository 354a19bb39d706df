// Decoder MLP with forward-mode Jacobian (the subspace map f_theta of
// Sec. 3.1, differentiated forward as the paper's autodiff does, Sec. 5),
// FP32/FP64 CUDA-core form.
//
// Every layer is one skinny GEMM  out[m][c] = sum_k W[m][k] Z[k][c]  over C
// columns (C <= 2 r + 4).  Columns c < nj carry the Jacobian pass: column 0
// the value at the point y0 and columns 1..r the tangent directions
// (Z_0 = [y0 | I_r]); columns c >= nj carry the line-search trial points y_j
// (values only).  Activations are stored unit-major, Z[k][c] with a padded
// column stride CPs (zstride(C)), so a layer's input tile is one contiguous
// block.  Epilogues:
//   hidden   value columns  h = ELU(acc + b);  tangent columns  ELU'(a0) acc
//            with a0 = acc_0 + b of the same row
//   output   u = s (acc_0 + b), J_c = s acc_c (constrained rows replaced by
//            the target displacement and a zero row), folded into per-CTA
//            partials of (E, sum|E|, g = J^T gv, sum|J gv|, K = J^T diag(kv) J)
//            for the terms that act on each DOF alone (inertia, gravity,
//            ground); trial columns give u_j and per-trial energy partials.
// Positions are handled as displacements u = x - X0, and the inertia term as
// u - (qbar - X0), so that FP32 arithmetic works on small numbers.
//
// Mapping: a CTA owns BM rows; KP = 8 consecutive lanes share a row and
// take every eighth k, so a warp reads eight consecutive k of Z (one 16-byte
// vector per lane, conflict-free for the padded stride) and four rows of W.
// Tiles are staged with 16-byte cp.async (one load phase for k <= 256), and
// the eight partial sums of a row are combined with three shuffles.
#include <cuda_bf16.h>

#include "lsn_internal.cuh"
#include "pdl.cuh"

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

template <typename Real>
struct KChunk {
  static constexpr int BK = 256;  // k staged per phase
};
template <>
struct KChunk<double> {
  static constexpr int BK = 128;
};

// 16-byte asynchronous copy global -> shared (zero-filled when !valid).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n)
               : "memory");
}
template <typename Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(Real) : 0;
  if (sizeof(Real) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr int KP = 8;  // lanes (k-phases) per row

// Shared-memory strides: W rows padded so that 4 rows x 8 k-phases hit 32
// distinct banks; Z rows have the padded column stride CPs.
template <typename Real>
__host__ __device__ constexpr int w_stride() {
  return KChunk<Real>::BK + (sizeof(Real) == 4 ? 8 : 4);
}

// acc[c] += sum over this lane's k (k = KP i + q) of W[row][k] Z[k][c] for
// the CTA's BM rows; returns with the KP phases of a row NOT yet combined.
template <typename Real, int CQ, int BM>
__device__ __forceinline__ void skinny_gemm(const Real* __restrict__ W, int M, int K,
                                            const Real* __restrict__ Zin, int CPs, int m0,
                                            Real* Ws, Real* Zs, Real (&acc)[4 * CQ]) {
  constexpr int NT = KP * BM, BK = KChunk<Real>::BK, WSs = w_stride<Real>();
  constexpr int EV = 16 / sizeof(Real);  // elements per 16-byte chunk
  const int t = threadIdx.x, q = t % KP, row = t / KP;
#pragma unroll
  for (int c = 0; c < 4 * CQ; ++c) acc[c] = Real(0);
  const bool vecW = (K % EV) == 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const int kw = min(BK, K - k0);
    // W tile: BM rows x kw
    if (vecW) {
      const int nch = kw / EV;
      for (int e = t; e < BM * nch; e += NT) {
        const int rr = e / nch, ch = e - rr * nch, gr = m0 + rr;
        const bool ok = gr < M;
        cp_async16(&Ws[rr * WSs + ch * EV], W + (ok ? (size_t)gr * K + k0 + ch * EV : 0), ok);
      }
    } else {
      for (int e = t; e < BM * kw; e += NT) {
        const int rr = e / kw, kk = e - rr * kw, gr = m0 + rr;
        const bool ok = gr < M;
        cp_async_elem<Real>(&Ws[rr * WSs + kk], W + (ok ? (size_t)gr * K + k0 + kk : 0), ok);
      }
    }
    // Z tile: kw rows x CPs, contiguous in global memory
    {
      const int nel = kw * CPs, nch = nel / EV;
      const Real* src = Zin + (size_t)k0 * CPs;
      for (int e = t; e < nch; e += NT) cp_async16(&Zs[e * EV], src + e * EV, true);
    }
    cp_async_wait_all();
    __syncthreads();
    const int ksteps = (kw - q + KP - 1) / KP;
#pragma unroll 2
    for (int i = 0; i < ksteps; ++i) {
      const int kk = KP * i + q;
      const Real w = Ws[row * WSs + kk];
      const Real* zr = Zs + kk * CPs;
      if (sizeof(Real) == 4) {
#pragma unroll
        for (int g = 0; g < CQ; ++g) {
          const float4 z4 = *reinterpret_cast<const float4*>(zr + 4 * g);
          acc[4 * g + 0] += w * (Real)z4.x;
          acc[4 * g + 1] += w * (Real)z4.y;
          acc[4 * g + 2] += w * (Real)z4.z;
          acc[4 * g + 3] += w * (Real)z4.w;
        }
      } else {
#pragma unroll
        for (int g = 0; g < 2 * CQ; ++g) {
          const double2 z2 = *reinterpret_cast<const double2*>(zr + 2 * g);
          acc[2 * g + 0] += w * (Real)z2.x;
          acc[2 * g + 1] += w * (Real)z2.y;
        }
      }
    }
    __syncthreads();
  }
}

// combine the KP k-phases of a row (KP consecutive lanes); every lane gets
// the sum
template <typename Real, int N>
__device__ __forceinline__ void combine_phases(Real (&acc)[N]) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
#pragma unroll
    for (int o = 1; o < KP; o <<= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
  }
}

template <typename Real>
__host__ __device__ constexpr size_t gemm_smem(int BM, int CPs) {
  return (size_t)(BM * w_stride<Real>() + KChunk<Real>::BK * CPs) * sizeof(Real);
}

// ------------------------------------------------------------ hidden layers
constexpr int HBM = 8;  // rows per CTA of a hidden layer (more CTAs: the layers are short)

// When the next layer is the tensor-core output layer, the layer's columns
// are also written as its K-major B operand: bkind 1 = BF16 two-term split
// (Bh = bf16(v), Bl = bf16(v - Bh)), 2 = FP32 (B[c][m], c < C).
template <typename Real, int CQ>
__global__ void __launch_bounds__(KP * HBM) hidden_kernel(const Real* __restrict__ W,
                                                         const Real* __restrict__ b, int M,
                                                         int K, const Real* __restrict__ Zin,
                                                         int C, int CPs, int nj,
                                                         Real* __restrict__ Zout, void* Bh,
                                                         void* Bl, int bkind) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Ws = reinterpret_cast<Real*>(smem_raw);
  Real* Zs = Ws + HBM * w_stride<Real>();
  const int t = threadIdx.x, q = t % KP, row = t / KP;
  const int m0 = blockIdx.x * HBM, m = m0 + row;
  pdl_wait();
  const Real bm = m < M ? b[m] : Real(0);
  Real acc[4 * CQ];
  skinny_gemm<Real, CQ, HBM>(W, M, K, Zin, CPs, m0, Ws, Zs, acc);
  combine_phases<Real, 4 * CQ>(acc);
  const Real a0 = acc[0] + bm;
  const Real e1 = elu_d<Real>(a0);
  if (m < M) {
    // lane q writes columns q, q + KP, ... of the row
#pragma unroll
    for (int c = 0; c < 4 * CQ; ++c) {
      if ((c % KP) != q || c >= C) continue;
      const Real v = (c == 0 || c >= nj) ? elu_f<Real>(acc[c] + bm) : e1 * acc[c];
      Zout[(size_t)m * CPs + c] = v;
      if (bkind == 1) {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
        static_cast<__nv_bfloat16*>(Bh)[(size_t)c * M + m] = hi;
        static_cast<__nv_bfloat16*>(Bl)[(size_t)c * M + m] =
            __float2bfloat16_rn((float)v - __bfloat162float(hi));
      } else if (bkind == 2) {
        static_cast<float*>(Bh)[(size_t)c * M + m] = (float)v;
      }
    }
  }
}

// Per-row energy, force and stiffness scalars of the terms that act on each
// DOF separately: inertia (dynamics) or gravity (quasi-static), and ground.
__device__ __forceinline__ void row_terms(const LastArgs& la, double inv_dt2, int comp,
                                          double mv, double ubar, double x0, double u,
                                          double& e, double& gv, double& kv) {
  if (inv_dt2 > 0.0) {
    const double diff = u - ubar;
    e = 0.5 * inv_dt2 * mv * diff * diff;
    gv = inv_dt2 * mv * diff;
    kv = inv_dt2 * mv;
  } else {
    e = -mv * la.grav[comp] * u;
    gv = -mv * la.grav[comp];
    kv = 0.0;
  }
  if (la.ground_k > 0.0 && comp == 2) {
    const double pen = x0 + u - la.ground_h;
    if (pen < 0.0) {
      e += 0.5 * la.ground_k * pen * pen;
      gv += la.ground_k * pen;
      kv += la.ground_k;
    }
  }
}

// Affine modes (scaled by the output scale, like the network): the unscaled
// displacement M (X0_v - c) + t of DOF (v, comp) at the pass point of column
// `col` (FP64 copy of the point), and the unscaled constant Jacobian entry of
// affine coordinate k (0..8: M row-major, 9..11: t).
__device__ __forceinline__ double affine_disp(const LastArgs& la, int comp, const double (&dX)[3],
                                              int col) {
  const double* Za = la.zaff;
  const int s = la.zcps;
  return Za[(3 * comp) * s + col] * dX[0] + Za[(3 * comp + 1) * s + col] * dX[1] +
         Za[(3 * comp + 2) * s + col] * dX[2] + Za[(9 + comp) * s + col];
}
__device__ __forceinline__ double affine_jac(int comp, const double (&dX)[3], int k) {
  if (k < 9) return (k / 3 == comp) ? dX[k - 3 * comp] : 0.0;
  return (k - 9 == comp) ? 1.0 : 0.0;
}

// ------------------------------------------------------------ output layer
constexpr int LBM = 64;        // rows per tile of the output layer
constexpr int LNT = KP * LBM;  // threads per CTA

// AFF: the body has affine modes (a separate instantiation)
template <typename Real, int CQ, bool AFF>
__global__ void __launch_bounds__(LNT) last_kernel(const Real* __restrict__ W,
                                                   const Real* __restrict__ b, int M, int K,
                                                   const Real* __restrict__ Zin, int C,
                                                   int CPs, int nj, Real* __restrict__ u_out,
                                                   Real* __restrict__ J_out,
                                                   Real* __restrict__ u_trial,
                                                   double* __restrict__ part, int part_stride,
                                                   LastArgs la) {
  constexpr int RQ = 4 * CQ;  // padded columns held per lane
  constexpr int PQ = (RQ * (RQ + 1) / 2 + LNT - 1) / LNT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Ws = reinterpret_cast<Real*>(smem_raw);
  Real* Zs = Ws + LBM * w_stride<Real>();
  size_t off = gemm_smem<Real>(LBM, CPs);
  off = (off + 15) & ~size_t(15);
  const int r = la.r, OS = r + 1;
  double* gvs = reinterpret_cast<double*>(smem_raw + off);  // LBM (row forces)
  double* red = gvs + LBM;                                  // (LNT/32 + 1) x 8
  Real* Js = reinterpret_cast<Real*>(red + (LNT / 32 + 1) * (2 + 2 * KTRIAL));  // LBM x OS
  Real* kvs = Js + LBM * OS;                                                    // LBM
  const int t = threadIdx.x, q = t % KP, row = t / KP;
  const int np = npairs(r);
  const int ntr = C - nj;
  const double inv_dt2 = *la.inv_dt2;
  const int tslot = nslots(r);
  int pi[PQ], pj[PQ];
  double kacc[PQ];
#pragma unroll
  for (int p = 0; p < PQ; ++p) {
    const int e = t + LNT * p;
    if (e < np) pair_of(e, r, pi[p], pj[p]);
    else pi[p] = pj[p] = -1;
    kacc[p] = 0.0;
  }
  double gacc = 0.0, gabs = 0.0, eacc = 0.0, eabs = 0.0;
  double etr = 0.0, atr = 0.0;  // trial column q - 1 of this lane (q = 1..KTRIAL)
  const int ntiles = (M + LBM - 1) / LBM;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int m0 = tile * LBM, m = m0 + row;
    const bool live = m < M;
    const int v = m / 3, comp = m - 3 * v;
    // per-row constants, fetched before the GEMM
    double mv = 0.0, ub = 0.0, x0 = 0.0, bm = 0.0;
    double dX[3] = {0.0, 0.0, 0.0};  // X0_v - c of the affine modes
    int slot = -1;
    if (live) {
      mv = la.mass[v];
      ub = la.ubar[m];
      x0 = la.X0[m];
      slot = la.cslot[v];
      bm = (double)b[m];
      if (AFF)
        for (int k = 0; k < 3; ++k) dX[k] = la.X0[3 * v + k] - la.acen[k];
    }
    Real acc[RQ];
    skinny_gemm<Real, CQ, LBM>(W, M, K, Zin, CPs, m0, Ws, Zs, acc);
    combine_phases<Real, RQ>(acc);
    const double cu = (live && slot >= 0) ? la.cu[3 * slot + comp] : 0.0;
    // value at y0 and the row terms
    double u0 = la.scale * ((double)acc[0] + bm);
    if (AFF && live) u0 += la.scale * affine_disp(la, comp, dX, 0);
    if (slot >= 0) u0 = cu;
    const Real u0r = (Real)u0;
    double e = 0.0, gv = 0.0, kv = 0.0;
    // (with affine modes the row terms take the unrounded displacement: a free
    // body's u is large, and its rounding would swamp the inertia force)
    if (live)
      row_terms(la, inv_dt2, comp, mv, ub, x0, AFF ? u0 : (double)u0r, e, gv, kv);
    if (q == 0) {
      if (live) {
        u_out[m] = u0r;
        eacc += e;
        eabs += fabs(e);
      }
      kvs[row] = live ? (Real)kv : Real(0);
      gvs[row] = live ? gv : 0.0;
    }
    // J row: lane q stores the columns c = q (mod KP) (zero if constrained)
#pragma unroll
    for (int c = 1; c < RQ; ++c) {
      if ((c % KP) != q || c >= nj) continue;
      const bool aff = AFF && c - 1 >= la.aff0;
      const Real jv = (live && slot < 0)
                          ? (Real)(la.scale * (aff ? affine_jac(comp, dX, c - 1 - la.aff0)
                                                   : (double)acc[c]))
                          : Real(0);
      if (live) J_out[(size_t)m * r + (c - 1)] = jv;
      Js[row * OS + (c - 1)] = jv;
    }
    // trial columns: lane q = 1..KTRIAL handles trial q - 1
    if (q >= 1 && q <= ntr && live) {
      double ut = 0.0;
#pragma unroll
      for (int c = 0; c < RQ; ++c)
        if (c == nj + q - 1) ut = la.scale * ((double)acc[c] + bm);
      if (AFF) ut += la.scale * affine_disp(la, comp, dX, nj + q - 1);
      if (slot >= 0) ut = cu;
      const Real utr = (Real)ut;
      u_trial[(size_t)(q - 1) * M + m] = utr;
      double et, g2, k2;
      row_terms(la, inv_dt2, comp, mv, ub, x0, AFF ? ut : (double)utr, et, g2, k2);
      etr += et;
      atr += fabs(et);
    }
    __syncthreads();
    const int rows = min(LBM, M - m0);
    if (t < r) {
      double s = 0.0, a = 0.0;
#pragma unroll 4
      for (int rr = 0; rr < rows; ++rr) {
        const double term = gvs[rr] * (double)Js[rr * OS + t];
        s += term;
        a += fabs(term);
      }
      gacc += s;
      gabs += a;
    }
#pragma unroll
    for (int p = 0; p < PQ; ++p) {
      if (pi[p] >= 0) {
        // the Hessian partial of a tile is summed in the element precision
        Real s0 = Real(0), s1 = Real(0);
        int rr = 0;
        for (; rr + 2 <= rows; rr += 2) {
          s0 += kvs[rr] * Js[rr * OS + pi[p]] * Js[rr * OS + pj[p]];
          s1 += kvs[rr + 1] * Js[(rr + 1) * OS + pi[p]] * Js[(rr + 1) * OS + pj[p]];
        }
        if (rr < rows) s0 += kvs[rr] * Js[rr * OS + pi[p]] * Js[rr * OS + pj[p]];
        kacc[p] += (double)(s0 + s1);
      }
    }
    __syncthreads();
  }
  // block reduction of the energy scalars: warp shuffles, then one value per
  // warp in shared memory (fixed order), then one partial row per CTA
  {
    double vals[2 + 2 * KTRIAL];
    vals[0] = eacc;
    vals[1] = eabs;
#pragma unroll
    for (int j = 0; j < KTRIAL; ++j) {
      vals[2 + 2 * j] = (q == j + 1) ? etr : 0.0;
      vals[3 + 2 * j] = (q == j + 1) ? atr : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 2 + 2 * KTRIAL; ++j) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vals[j] += __shfl_down_sync(0xffffffffu, vals[j], o);
    }
    if ((t & 31) == 0)
#pragma unroll
      for (int j = 0; j < 2 + 2 * KTRIAL; ++j) red[(t >> 5) * (2 + 2 * KTRIAL) + j] = vals[j];
    __syncthreads();
    if (t < 2 + 2 * KTRIAL) {
      double sum = 0.0;
      for (int w = 0; w < LNT / 32; ++w) sum += red[w * (2 + 2 * KTRIAL) + t];
      red[LNT / 32 * (2 + 2 * KTRIAL) + t] = sum;
    }
    __syncthreads();
  }
  const double* tot = red + LNT / 32 * (2 + 2 * KTRIAL);
  double* prow = part + (size_t)blockIdx.x * part_stride;
  if (t == 0) {
    prow[0] = tot[0];
    prow[1] = tot[1];
  }
  if (t < 2 * KTRIAL) prow[tslot + t] = (t / 2 < ntr) ? tot[2 + t] : 0.0;
  if (t < r) {
    prow[slot_g(t)] = gacc;
    prow[slot_gabs(r, t)] = gabs;
  }
#pragma unroll
  for (int p = 0; p < PQ; ++p) {
    const int e = t + LNT * p;
    if (e < np) prow[slot_K(r) + e] = kacc[p];
  }
}

template <typename Real>
size_t last_smem(int r, int CPs) {
  size_t off = gemm_smem<Real>(LBM, CPs);
  off = (off + 15) & ~size_t(15);
  return off + ((size_t)LBM + (LNT / 32 + 1) * (2 + 2 * KTRIAL)) * sizeof(double) +
         ((size_t)LBM * (r + 1) + LBM) * sizeof(Real);
}

template <typename Real, int CQ>
void run_hidden(const Real* W, const Real* b, int M, int K, const Real* Zin, int C, int CPs,
                int nj, Real* Zout, void* Bh, void* Bl, int bkind, cudaStream_t s) {
  const size_t sm = gemm_smem<Real>(HBM, CPs);
  static size_t set = 0;
  if (sm > set) {
    cudaFuncSetAttribute(hidden_kernel<Real, CQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    set = sm;
  }
  launch_pdl(hidden_kernel<Real, CQ>, dim3((M + HBM - 1) / HBM), dim3(KP * HBM), sm, s, W, b,
             M, K, Zin, C, CPs, nj, Zout, Bh, Bl, bkind);
}

template <typename Real, int CQ>
void run_last(const Real* W, const Real* b, int M, int K, const Real* Zin, int C, int CPs,
              int nj, Real* u_out, Real* J_out, Real* u_trial, double* part, int stride,
              const LastArgs& la, int grid, cudaStream_t s) {
  const size_t sm = last_smem<Real>(la.r, CPs);
  static size_t set = 0;
  if (sm > set) {
    cudaFuncSetAttribute(last_kernel<Real, CQ, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(last_kernel<Real, CQ, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = sm;
  }
  if (la.aff0 >= 0)
    last_kernel<Real, CQ, true><<<grid, LNT, sm, s>>>(W, b, M, K, Zin, C, CPs, nj, u_out, J_out,
                                                      u_trial, part, stride, la);
  else
    last_kernel<Real, CQ, false><<<grid, LNT, sm, s>>>(W, b, M, K, Zin, C, CPs, nj, u_out,
                                                       J_out, u_trial, part, stride, la);
}

}  // namespace

int decoder_last_grid(int n, int C, int num_sms) {
  const int tiles = (n + LBM - 1) / LBM;
  const int per_sm = C > 48 ? 1 : 2;
  return std::max(1, std::min(tiles, num_sms * per_sm));
}

#define LSN_CQ_SWITCH(CPs, CALL)                 \
  switch ((CPs) / 4) {                           \
    case 1: { constexpr int CQ = 1; CALL; } break; \
    case 3: { constexpr int CQ = 3; CALL; } break; \
    case 5: { constexpr int CQ = 5; CALL; } break; \
    case 7: { constexpr int CQ = 7; CALL; } break; \
    case 9: { constexpr int CQ = 9; CALL; } break; \
    case 11: { constexpr int CQ = 11; CALL; } break; \
    case 13: { constexpr int CQ = 13; CALL; } break; \
    case 15: { constexpr int CQ = 15; CALL; } break; \
    case 17: { constexpr int CQ = 17; CALL; } break; \
    default: break;                              \
  }

template <typename Real>
void launch_hidden_layer(const Real* W, const Real* b, int M, int K, const Real* Zin, int C,
                         int nj, Real* Zout, cudaStream_t s, void* Bh, void* Bl, int bkind) {
  const int CPs = zstride(C);
  LSN_CQ_SWITCH(CPs,
                (run_hidden<Real, CQ>(W, b, M, K, Zin, C, CPs, nj, Zout, Bh, Bl, bkind, s)))
}

template <typename Real>
void launch_last_layer(const Real* W, const Real* b, int M, int K, const Real* Zin, int C,
                       int nj, Real* u_out, Real* J_out, Real* u_trial, double* part,
                       int part_stride, const LastArgs& la, int grid, cudaStream_t s) {
  const int CPs = zstride(C);
  LSN_CQ_SWITCH(CPs, (run_last<Real, CQ>(W, b, M, K, Zin, C, CPs, nj, u_out, J_out, u_trial,
                                          part, part_stride, la, grid, s)))
}

#define LSN_INST(R)                                                                        \
  template void launch_hidden_layer<R>(const R*, const R*, int, int, const R*, int, int,  \
                                       R*, cudaStream_t, void*, void*, int);               \
  template void launch_last_layer<R>(const R*, const R*, int, int, const R*, int, int, R*, \
                                     R*, R*, double*, int, const LastArgs&, int,           \
                                     cudaStream_t);
LSN_INST(float)
LSN_INST(double)
#undef LSN_INST

}  // namespace lsn
