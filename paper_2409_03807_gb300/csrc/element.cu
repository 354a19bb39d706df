// Per-tet Stable Neo-Hookean element kernel fused with the reduced
// contraction (Sec. 3.1 Eq. 2 and Eq. 11; stable neo-Hookean energy of
// Sec. 5.1; PSD-projected Hessian of projective Newton, Supplement).
//
// For tet e with displacement gradient Hd = F - I = [u1-u0, u2-u0, u3-u0] Dm^-1
// the kernel evaluates (w_e V_e times) the energy density, its first
// derivative P and the eigen-decomposition of the 9x9 second derivative
// A = d2Psi/dF2, clamps negative eigenvalues (PSD projection), and
// accumulates
//     g += G_e^T p_e,            p_e = w_e V_e vec(P)
//     K += C_e^T C_e,            C_e = diag(sqrt(w_e V_e lambda_+)) Q^T G_e
// where G_e = dvec(F)/dz = B_e J_e (9 x r) is formed from the tet's four
// vertex rows of J, so that C_e^T C_e = w_e J_e^T Hproj_e J_e.
//
// Eigen-decomposition.  Psi depends on F only through I2 = |F|^2 and
// I3 = det F, so with the rotation-signed SVD F = U diag(s) V^T the 9
// eigenvectors of A are U M V^T for
//   twist  M = (e_j e_k^T - e_k e_j^T)/sqrt2:  lambda = 2 Psi_2 + Psi_3 s_i
//   flip   M = (e_j e_k^T + e_k e_j^T)/sqrt2:  lambda = 2 Psi_2 - Psi_3 s_i
// ((i, j, k) a permutation of (0, 1, 2)) and M = diag(a) for the three
// eigenvectors a of the 3x3 matrix
//   A_s = 2 Psi_2 I + 4 Psi_22 s s^T + Psi_33 pi pi^T + Psi_3 S,
// pi_i = s_j s_k, S_jk = s_i (j != k), S_ii = 0, where Psi_2, Psi_3, Psi_22,
// Psi_33 are the partial derivatives in (I2, I3) (Psi_23 = 0 here).  This
// follows from d2/dt2 det(diag(s) + t M) and the invariance of Psi; the SVD
// comes from a Jacobi eigen-decomposition of F^T F.  The coordinates of a
// perturbation dF along these eigenvectors are read from R = U^T dF V.
//
// The density is written in terms of Hd (no cancellation near rest):
//   Psi = mu/2 (Ic-3) - mu/2 log1p((Ic-3)/4) + lam/2 (J-1)(J-1 + 2(1-a))
//   P   = mu d F + lam (J-1) cof(F) + (3 mu/4)(Hd + Hd^T - tr(Hd) I - cof(Hd))
// with Ic-3 = 2 tr Hd + |Hd|^2, J-1 = tr Hd + (sum of principal 2x2 minors)
// + det Hd, d = (Ic-3)/(4 (Ic+1)), a = 1 + 3 mu/(4 lam): algebraically the
// same function as mu/2 (Ic-3) + lam/2 (J-a)^2 - mu/2 log(Ic+1) - Psi(I).
//
// Work split: a CTA takes tiles of 128 tets.  Phase 1 is one thread per tet
// (element math, eigen-decomposition); phase 2 spreads (tet, column) pairs
// over the threads to form G_e and C_e in shared memory; phase 3 is the
// symmetric rank-9T update of the CTA's register-resident K partial, each
// thread owning a fixed set of upper-triangle entries.  Each CTA writes one
// partial row (E, sum|E|, g, K upper) that a fixed-order reduction sums.
#include <cuda_bf16.h>

#include "element_math.cuh"
#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace lsn {
namespace {

// tets per contraction batch (FP64 halves it to fit the shared memory)
template <typename Real>
struct Batch {
  static constexpr int CB = 16;
};
template <>
struct Batch<double> {
  static constexpr int CB = 8;
};

// Asynchronous copies of the tets' J rows into shared memory.
template <typename Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(Real) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename Real, int ET>
struct ElemTile {  // shared memory of one tile (ET tets)
  Real U[ET][9];    // U of the signed SVD (row-major)
  Real V[ET][9];    // V of the signed SVD (row-major)
  Real As[ET][9];   // row m: sqrt(w V lambda_s,m+) a_m (scaling modes)
  Real tf[ET][6];   // sqrt(w V lambda+ / 2) of the 3 twist, then 3 flip modes
  Real D[ET][12];
  Real p[ET][9];
  int4 v[ET];
};

__device__ __forceinline__ void pair_of(int p, int r, int& i, int& j) {
  i = 0;
  while (p >= r - i) {
    p -= r - i;
    ++i;
  }
  j = i + p;
}

// Phase 1 of a tile: element math of tet e by thread t (energy, P, the
// signed SVD and the clamped eigen-decomposition of d2Psi/dF2), stored in the
// tile's shared memory; a slot past the last tet is zeroed.
template <typename Real, int ET>
__device__ __forceinline__ void element_phase1(const ElemArgs& ea, const Real* __restrict__ u,
                                               int e, int t, ElemTile<Real, ET>& tl, Real mu,
                                               Real lam, Real oma, Real& pe_out) {
  if (e < ea.S) {
    int4 tv;
    Real Dmi[3][3], wv, H[3][3];
    load_tet<Real>(ea, e, tv, Dmi, wv);
    disp_grad<Real>(u, tv, Dmi, H);
    Invariants<Real> iv;
    invariants<Real>(H, iv);
    const Real psi = snh_psi<Real>(iv, mu, lam, oma);
    pe_out = wv * psi;
    const Real Ic = iv.Ic3 + Real(3);
    const Real dl = iv.Ic3 / (Real(4) * (Ic + Real(1)));
    const Real lJ = lam * iv.Jm1;
    // first derivative P, stored as p = w V vec(P)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const Real Fij = H[i][j] + (i == j ? Real(1) : Real(0));
        const Real P = mu * dl * Fij + lJ * iv.cof[i][j] +
                       Real(0.75) * mu *
                           (H[i][j] + H[j][i] - (i == j ? iv.trH : Real(0)) - iv.cofH[i][j]);
        tl.p[t][3 * i + j] = wv * P;
      }
    // eigen-decomposition of the second derivative (see header)
    const Real c1 = mu * Ic / (Ic + Real(1));                   // 2 Psi_2
    const Real c2 = Real(2) * mu / ((Ic + Real(1)) * (Ic + Real(1)));  // 4 Psi_22
    const Real c3 = lam * (iv.Jm1 + oma);                       // Psi_3 = lam (J - a)
    Real F[3][3], U[3][3], V[3][3], sg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? Real(1) : Real(0));
    svd3<Real>(F, U, sg, V);
    Real As[3][3], Aq[3][3];
    const Real pi3[3] = {sg[1] * sg[2], sg[0] * sg[2], sg[0] * sg[1]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        As[i][j] = c2 * sg[i] * sg[j] + lam * pi3[i] * pi3[j] +
                   (i == j ? c1 : c3 * sg[3 - i - j]);
    jacobi3<Real>(As, Aq);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const Real sc = sqrt_r<Real>(wv * (As[m][m] > Real(0) ? As[m][m] : Real(0)));
#pragma unroll
      for (int i = 0; i < 3; ++i) tl.As[t][3 * m + i] = sc * Aq[i][m];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const Real lt = c1 + c3 * sg[i], lf = c1 - c3 * sg[i];
      tl.tf[t][i] = sqrt_r<Real>(Real(0.5) * wv * (lt > Real(0) ? lt : Real(0)));
      tl.tf[t][3 + i] = sqrt_r<Real>(Real(0.5) * wv * (lf > Real(0) ? lf : Real(0)));
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      tl.U[t][k] = U[k / 3][k % 3];
      tl.V[t][k] = V[k / 3][k % 3];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      tl.D[t][j] = -(Dmi[0][j] + Dmi[1][j] + Dmi[2][j]);
#pragma unroll
      for (int a = 1; a < 4; ++a) tl.D[t][3 * a + j] = Dmi[a - 1][j];
    }
  } else {
    pe_out = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) tl.U[t][k] = tl.V[t][k] = tl.As[t][k] = Real(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) tl.tf[t][k] = Real(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) tl.D[t][k] = Real(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) tl.p[t][k] = Real(0);
  }
}

// Per-tet data of phase 2 held in registers.
template <typename Real>
struct TetData {
  Real D[12], p[9], U[9], V[9], As[9], tf[6];
};

template <typename Real, int ET>
__device__ __forceinline__ void load_tet_data(const ElemTile<Real, ET>& tl, int q,
                                              TetData<Real>& td) {
#pragma unroll
  for (int k = 0; k < 12; ++k) td.D[k] = tl.D[q][k];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    td.p[k] = tl.p[q][k];
    td.U[k] = tl.U[q][k];
    td.V[k] = tl.V[q][k];
    td.As[k] = tl.As[q][k];
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) td.tf[k] = tl.tf[q][k];
}

// C_e rows (9) and p_e . G for one (tet, subspace column) pair: G = dvec(F)
// along the column from the tet's four J rows jv, R = U^T G V, then the
// projected eigen-coordinates scaled by sqrt(w V lambda+).
template <typename Real>
__device__ __forceinline__ void element_item_td(const TetData<Real>& td, const Real (&jv)[4][3],
                                                Real (&Cv)[9], Real& gp) {
  Real G[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Real s = Real(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) s += td.D[3 * a + j] * jv[a][i];
      G[3 * i + j] = s;
    }
#pragma unroll
  for (int k = 0; k < 9; ++k) gp += td.p[k] * G[k];
  // R = U^T dF V with dF = G as a 3x3 matrix
  Real T3[3][3], R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      T3[i][b] = G[3 * i] * td.V[b] + G[3 * i + 1] * td.V[3 + b] + G[3 * i + 2] * td.V[6 + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      R[a][b] = td.U[a] * T3[0][b] + td.U[3 + a] * T3[1][b] + td.U[6 + a] * T3[2][b];
#pragma unroll
  for (int m = 0; m < 3; ++m)
    Cv[m] = td.As[3 * m] * R[0][0] + td.As[3 * m + 1] * R[1][1] + td.As[3 * m + 2] * R[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    Cv[3 + i] = td.tf[i] * (R[j][k] - R[k][j]);
    Cv[6 + i] = td.tf[3 + i] * (R[j][k] + R[k][j]);
  }
}

// The same as element_item_td, reading the tet's data from shared memory as
// it goes (fewer live registers in the CUDA-core kernel).
template <typename Real, int ET>
__device__ __forceinline__ void element_item(const ElemTile<Real, ET>& tl, int q,
                                             const Real (&jv)[4][3], Real (&Cv)[9], Real& gp) {
  Real G[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Real s = Real(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) s += tl.D[q][3 * a + j] * jv[a][i];
      G[3 * i + j] = s;
    }
#pragma unroll
  for (int k = 0; k < 9; ++k) gp += tl.p[q][k] * G[k];
  Real T3[3][3], R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      T3[i][b] = G[3 * i] * tl.V[q][b] + G[3 * i + 1] * tl.V[q][3 + b] +
                 G[3 * i + 2] * tl.V[q][6 + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      R[a][b] = tl.U[q][a] * T3[0][b] + tl.U[q][3 + a] * T3[1][b] + tl.U[q][6 + a] * T3[2][b];
#pragma unroll
  for (int m = 0; m < 3; ++m)
    Cv[m] = tl.As[q][3 * m] * R[0][0] + tl.As[q][3 * m + 1] * R[1][1] +
            tl.As[q][3 * m + 2] * R[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    Cv[3 + i] = tl.tf[q][i] * (R[j][k] - R[k][j]);
    Cv[6 + i] = tl.tf[q][3 + i] * (R[j][k] + R[k][j]);
  }
}

// Energy of the KTRIAL trial displacement fields ut[j * n + .] for the tets
// e = first, first + stride, ...; block-reduced into prow[2 j], prow[2 j + 1].
template <typename Real, int ET>
__device__ __forceinline__ void element_energy_block(const ElemArgs& ea,
                                                     const Real* __restrict__ ut, int first,
                                                     int stride, double* prow,
                                                     double (*red)[ET]) {
  const int t = threadIdx.x;
  const Real mu = (Real)ea.mu, lam = (Real)ea.lam;
  const Real oma = (Real)(-0.75 * ea.mu / ea.lam);
  double ea_[KTRIAL], ab_[KTRIAL];
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) ea_[j] = ab_[j] = 0.0;
  for (int e = first + t; e < ea.S; e += stride) {
    int4 tv;
    Real Dmi[3][3], wv;
    load_tet<Real>(ea, e, tv, Dmi, wv);
#pragma unroll
    for (int j = 0; j < KTRIAL; ++j) {
      Real H[3][3];
      disp_grad<Real>(ut + (size_t)j * ea.n, tv, Dmi, H);
      Invariants<Real> iv;
      invariants<Real>(H, iv);
      const double pe = (double)(wv * snh_psi<Real>(iv, mu, lam, oma));
      ea_[j] += pe;
      ab_[j] += fabs(pe);
    }
  }
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) {
    red[2 * j][t] = ea_[j];
    red[2 * j + 1][t] = ab_[j];
  }
  __syncthreads();
  for (int s = ET / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int j = 0; j < 2 * KTRIAL; ++j) red[j][t] += red[j][t + s];
    }
    __syncthreads();
  }
  if (t < 2 * KTRIAL) prow[t] = red[t][0];
}

template <typename Real, int RT, int ET>
__global__ void __launch_bounds__(ET) element_kernel(ElemArgs ea, const Real* __restrict__ u,
                                                     const Real* __restrict__ J,
                                                     const Real* __restrict__ ut,
                                                     double* __restrict__ part,
                                                     int part_stride, int gfull) {
  __shared__ double red[2 * KTRIAL][ET];
  if ((int)blockIdx.x >= gfull) {
    const int b = blockIdx.x - gfull, nb = gridDim.x - gfull;
    element_energy_block<Real, ET>(ea, ut, b * ET, nb * ET,
                                   part + (size_t)blockIdx.x * part_stride + nslots(ea.r), red);
    return;
  }
  constexpr int PQ = (RT * (RT + 1) / 2 + ET - 1) / ET;
  constexpr int CB = Batch<Real>::CB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ElemTile<Real, ET>& tl = *reinterpret_cast<ElemTile<Real, ET>*>(smem_raw);
  Real* Cs = reinterpret_cast<Real*>(smem_raw + sizeof(ElemTile<Real, ET>));  // CB*9 x r
  Real* Gp = Cs + CB * 9 * ea.r;                                               // CB x r
  Real* Jb = Gp + CB * ea.r;  // 2 buffers of CB tets x 12 rows x r (J rows of a batch)
  const int t = threadIdx.x;
  const int r = ea.r, np = npairs(r);
  const Real mu = (Real)ea.mu, lam = (Real)ea.lam;
  const Real oma = (Real)(-0.75 * ea.mu / ea.lam);  // 1 - a
  int pi[PQ], pj[PQ];
  double kacc[PQ];
#pragma unroll
  for (int q = 0; q < PQ; ++q) {
    int p = t + ET * q;
    if (p < np) pair_of(p, r, pi[q], pj[q]);
    else pi[q] = pj[q] = -1;
    kacc[q] = 0.0;
  }
  double gacc = 0.0, gabs = 0.0, eacc = 0.0, eabs = 0.0;
  const int ntiles = (ea.S + ET - 1) / ET;
  const int jbs = CB * 12 * r;  // elements per J buffer
  // issue the copies of the 12 J rows of tets b0 .. b0 + CB - 1 into buffer buf
  auto prefetch = [&](int b0, int nb, int buf) {
    Real* dst = Jb + buf * jbs;
    if ((r * (int)sizeof(Real)) % 16 == 0) {
      const int per_row = r * (int)sizeof(Real) / 16, ev = 16 / (int)sizeof(Real);
      for (int e2 = t; e2 < nb * 12 * per_row; e2 += ET) {
        const int rowi = e2 / per_row, ch = e2 - rowi * per_row;
        const int lt = rowi / 12, k = rowi - lt * 12, a = k / 3, i = k - 3 * a;
        const int4 tv = tl.v[b0 + lt];
        const int v = a == 0 ? tv.x : (a == 1 ? tv.y : (a == 2 ? tv.z : tv.w));
        cp_async_16(dst + rowi * r + ch * ev, J + (size_t)(3 * v + i) * r + ch * ev);
      }
    } else {
      for (int e2 = t; e2 < nb * 12 * r; e2 += ET) {
        const int rowi = e2 / r, c = e2 - rowi * r;
        const int lt = rowi / 12, k = rowi - lt * 12, a = k / 3, i = k - 3 * a;
        const int4 tv = tl.v[b0 + lt];
        const int v = a == 0 ? tv.x : (a == 1 ? tv.y : (a == 2 ? tv.z : tv.w));
        cp_async_elem<Real>(dst + rowi * r + c, J + (size_t)(3 * v + i) * r + c);
      }
    }
    cp_async_commit();
  };
  for (int tile = blockIdx.x; tile < ntiles; tile += gfull) {
    const int e = tile * ET + t;
    const int tile_tets = min(ET, ea.S - tile * ET);
    // tet indices first, so that the J rows of the first batch load during
    // the element math
    tl.v[t] = e < ea.S ? ea.tets[e] : make_int4(0, 0, 0, 0);
    __syncthreads();
    prefetch(0, min(CB, tile_tets), 0);
    // ---------------- phase 1: element math, one tet per thread
    {
      Real pe;
      element_phase1<Real, ET>(ea, u, e, t, tl, mu, lam, oma, pe);
      eacc += (double)pe;
      eabs += fabs((double)pe);
    }
    // ---------------- phases 2 + 3 in batches of CB tets
    int buf = 0;
    for (int b0 = 0; b0 < tile_tets; b0 += CB, buf ^= 1) {
      const int nb = min(CB, tile_tets - b0);
      if (b0 + CB < tile_tets) {
        prefetch(b0 + CB, min(CB, tile_tets - b0 - CB), buf ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const Real* Jt = Jb + buf * jbs;
      for (int item = t; item < CB * r; item += ET) {
        const int lt = item / r, c = item - lt * r;
        Real Cv[9];
        Real gp = Real(0);
        if (lt < nb) {
          const int q = b0 + lt;
          Real jv[4][3];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) jv[a][i] = Jt[(lt * 12 + 3 * a + i) * r + c];
          element_item<Real, ET>(tl, q, jv, Cv, gp);
        } else {
#pragma unroll
          for (int m = 0; m < 9; ++m) Cv[m] = Real(0);
        }
#pragma unroll
        for (int m = 0; m < 9; ++m) Cs[(lt * 9 + m) * r + c] = Cv[m];
        Gp[lt * r + c] = gp;
      }
      __syncthreads();
      if (t < r) {
        double s = 0.0, a = 0.0;
        for (int lt = 0; lt < nb; ++lt) {
          s += (double)Gp[lt * r + t];
          a += fabs((double)Gp[lt * r + t]);
        }
        gacc += s;
        gabs += a;
      }
      const int rows = nb * 9;
#pragma unroll
      for (int q = 0; q < PQ; ++q) {
        if (pi[q] >= 0) {
          Real s0 = Real(0), s1 = Real(0), s2 = Real(0), s3 = Real(0);
          int row = 0;
          for (; row + 4 <= rows; row += 4) {
            s0 += Cs[row * r + pi[q]] * Cs[row * r + pj[q]];
            s1 += Cs[(row + 1) * r + pi[q]] * Cs[(row + 1) * r + pj[q]];
            s2 += Cs[(row + 2) * r + pi[q]] * Cs[(row + 2) * r + pj[q]];
            s3 += Cs[(row + 3) * r + pi[q]] * Cs[(row + 3) * r + pj[q]];
          }
          for (; row < rows; ++row) s0 += Cs[row * r + pi[q]] * Cs[row * r + pj[q]];
          kacc[q] += (double)((s0 + s1) + (s2 + s3));
        }
      }
      __syncthreads();
    }
  }
  red[0][t] = eacc;
  red[1][t] = eabs;
  __syncthreads();
  for (int s = ET / 2; s > 0; s >>= 1) {
    if (t < s) {
      red[0][t] += red[0][t + s];
      red[1][t] += red[1][t + s];
    }
    __syncthreads();
  }
  double* prow = part + (size_t)blockIdx.x * part_stride;
  if (t == 0) {
    prow[0] = red[0][0];
    prow[1] = red[1][0];
  }
  if (t < r) {
    prow[slot_g(t)] = gacc;
    prow[slot_gabs(r, t)] = gabs;
  }
#pragma unroll
  for (int q = 0; q < PQ; ++q)
    if (pi[q] >= 0) prow[slot_K(r) + t + ET * q] = kacc[q];
}

template <typename Real, int RT, int ET>
void run_element(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                 double* part, int gfull, int genergy, cudaStream_t s) {
  constexpr int CB = Batch<Real>::CB;
  const size_t sm = sizeof(ElemTile<Real, ET>) +
                    (size_t)(CB * 9 * ea.r + CB * ea.r + 2 * CB * 12 * ea.r) * sizeof(Real);
  static size_t set = 0;
  if (sm > set) {
    cudaFuncSetAttribute(element_kernel<Real, RT, ET>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set = sm;
  }
  element_kernel<Real, RT, ET><<<gfull + genergy, ET, sm, s>>>(ea, u, J, ut, part,
                                                               nslots_total(ea.r), gfull);
}

template <typename Real, int ET>
void run_element_r(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                   double* part, int gfull, int genergy, cudaStream_t s) {
  if (ea.r <= 16) run_element<Real, 16, ET>(ea, u, J, ut, part, gfull, genergy, s);
  else if (ea.r <= 32) run_element<Real, 32, ET>(ea, u, J, ut, part, gfull, genergy, s);
  else run_element<Real, 64, ET>(ea, u, J, ut, part, gfull, genergy, s);
}


// ------------------------------------------------------------------------
// Tensor-core form of the element kernel (TF32 / BF16 forms): the same
// element math (phase 1, element_item), with the rank-9 updates
// K += C_e^T C_e of phase 3 replaced by tcgen05 MMAs.  The C_e rows of a
// chunk of tets are written, rounded to BF16 or TF32, into a K-major
// 128-byte-swizzled operand whose rows are the subspace columns c and whose
// K index is (tet, eigen-row); one MMA chain D += Op * Op^T (M = 64, N =
// r rounded up to 16) accumulates into TMEM across all of the CTA's chunks,
// while the threads build the next chunk in the other buffer.  The per-tet
// Hessians and the gradient stay FP32 (FP64 partial sums).  The trial
// energies of the line search are computed in phase 1 as well, so every CTA
// writes one complete partial row.
namespace tcel {

using namespace tc;

constexpr int ET = 256;        // tets per tile
constexpr int NT = 512;        // threads: phase 1 element math by the first ET, the
                               // trial energies by the others; phase 2 by all
constexpr int GROWS = 64;      // operand rows (subspace columns, r <= 64)
constexpr uint32_t KBB = GROWS * 128;  // bytes per 128-byte K block
constexpr unsigned long long WAIT_NS = 2000000000ull;

template <bool BF>
struct Cfg {
  static constexpr int CH = BF ? 64 : 32;     // tets per chunk
  static constexpr int EPB = BF ? 64 : 32;    // K values per 128-byte block
  static constexpr int NKB = 9 * CH / EPB;    // K blocks per chunk (9)
  static constexpr uint32_t BUF = NKB * KBB;  // operand bytes per chunk
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > WAIT_NS) {
      atomicOr(err, code);
      return false;
    }
  }
}

template <bool BF>
__host__ __device__ inline size_t smem_bytes(int r) {
  return 2 * (size_t)Cfg<BF>::BUF + sizeof(ElemTile<float, ET>) +
         (size_t)Cfg<BF>::CH * r * sizeof(float) + 1024;
}

template <bool BF>
__global__ void __launch_bounds__(NT, 1)
    element_tc_kernel(ElemArgs ea, const float* __restrict__ u, const float* __restrict__ J,
                      const float* __restrict__ ut, double* __restrict__ part, int part_stride,
                      int TT, int* __restrict__ err) {
  using C = Cfg<BF>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t done[2], fin;
  __shared__ uint32_t tbase_s;
  __shared__ FAcc red[NT / 32][2 + 2 * KTRIAL];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  ElemTile<float, ET>& tl = *reinterpret_cast<ElemTile<float, ET>*>(sb + 2 * C::BUF);
  float* Gp = reinterpret_cast<float*>(sb + 2 * C::BUF + sizeof(ElemTile<float, ET>));
  const int r = ea.r, S = ea.S;
  const int Ng = (r + 15) / 16 * 16;
  const uint32_t idesc = BF ? idesc_bf16(GROWS, Ng) : idesc_tf32(GROWS, Ng);
  const float mu = (float)ea.mu, lam = (float)ea.lam;
  const float oma = (float)(-0.75 * ea.mu / ea.lam);
  if (warp == 0) {
    tmem_alloc(&tbase_s, 64);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(&done[0], 1);
    mbar_init(&done[1], 1);
    mbar_init(&fin, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  pdl_wait();  // u, J and the trial displacements come from the output layer
  // energies and gradient partials in double-float (FP32 TwoSum) accumulators
  FAcc eacc, eabs, etr[KTRIAL], atr[KTRIAL], gacc, gabs;
  // TT <= ET tets per tile (small cubature sets use small tiles, more CTAs)
  const int ntiles = (S + TT - 1) / TT;
  int qc = 0;  // chunks issued by this CTA
  bool alive = true;
  for (int tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
    const int e = t < TT ? tile * TT + t : S;  // (threads < ET)
    const int tile_tets = min(TT, S - tile * TT);
    // ---------------- phase 1: element math (threads < ET) and the trial
    // energies of the line search (threads >= ET), one tet per thread
    if (t < ET) {
      tl.v[t] = e < S ? ea.tets[e] : make_int4(0, 0, 0, 0);
      float pe;
      element_phase1<float, ET>(ea, u, e, t, tl, mu, lam, oma, pe);
      facc_add(eacc, pe);
      facc_add(eabs, fabsf(pe));
    } else {
      const int e2 = tile * TT + (t - ET);
      if (t - ET < TT && e2 < S) {
        int4 tv;
        float Dmi[3][3], wv;
        load_tet<float>(ea, e2, tv, Dmi, wv);
#pragma unroll
        for (int j = 0; j < KTRIAL; ++j) {
          float H[3][3];
          disp_grad<float>(ut + (size_t)j * ea.n, tv, Dmi, H);
          Invariants<float> iv;
          invariants<float>(H, iv);
          const float pe = wv * snh_psi<float>(iv, mu, lam, oma);
          facc_add(etr[j], pe);
          facc_add(atr[j], fabsf(pe));
        }
      }
    }
    __syncthreads();
    // ---------------- phases 2 + 3 in chunks of CH tets
    for (int c0 = 0; c0 < tile_tets; c0 += C::CH, ++qc) {
      const int nb = min(C::CH, tile_tets - c0);
      const int buf = qc & 1;
      // the buffer was last read by the MMAs of chunk qc - 2
      const bool ok = qc < 2 || wait_bar(&done[buf], ((qc >> 1) & 1) ^ 1, err, 1);
      if (!__syncthreads_and(ok)) {
        alive = false;
        break;
      }
      uint8_t* op = sb + buf * C::BUF;
      // a warp takes 8 consecutive columns of 4 tets: the J reads stay in
      // 32-byte segments and the operand stores spread over the banks.  A
      // thread keeps one tet (lt) for all of its column blocks, so the tet's
      // data is read from shared memory once per chunk.
      {
        static_assert((NT / 8) % C::CH == 0, "column groups must tile the chunk");
        constexpr int CBSTEP = (NT / 8) / C::CH;        // column blocks in parallel per tet
        const int slot = t >> 3, c8 = t & 7;
        const int lt = slot % C::CH, cb0 = slot / C::CH;
        const bool live_t = lt < nb;
        // byte offsets of the tet's nine operand entries (K = 9 lt + m) within
        // a column row: the swizzle XOR uses c & 7 = c8, fixed for the thread
        uint32_t koff[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
          const int k = lt * 9 + m, kb = k / C::EPB, kin = k - kb * C::EPB;
          koff[m] = BF ? kb * KBB + ((((uint32_t)kin >> 3) ^ (uint32_t)c8) << 4) + (kin & 7) * 2
                       : kb * KBB + ((((uint32_t)kin >> 2) ^ (uint32_t)c8) << 4) + (kin & 3) * 4;
        }
        TetData<float> td;
        int vv[4] = {0, 0, 0, 0};
        if (live_t) {
          load_tet_data<float, ET>(tl, c0 + lt, td);
          const int4 tv = tl.v[c0 + lt];
          vv[0] = tv.x;
          vv[1] = tv.y;
          vv[2] = tv.z;
          vv[3] = tv.w;
        }
        for (int cb = cb0; cb * 8 < r; cb += CBSTEP) {
          const int c = cb * 8 + c8;
          if (c >= r) continue;
          float Cv[9];
          float gp = 0.f;
          if (live_t) {
            float jv[4][3];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int i = 0; i < 3; ++i) jv[a][i] = J[(size_t)(3 * vv[a] + i) * r + c];
            element_item_td<float>(td, jv, Cv, gp);
          } else {
#pragma unroll
            for (int m = 0; m < 9; ++m) Cv[m] = 0.f;
          }
          uint8_t* orow = op + (uint32_t)c * 128u;  // operand row c (128-byte rows)
#pragma unroll
          for (int m = 0; m < 9; ++m) {
            if (BF)
              *reinterpret_cast<__nv_bfloat16*>(orow + koff[m]) = __float2bfloat16_rn(Cv[m]);
            else
              *reinterpret_cast<float*>(orow + koff[m]) = Cv[m];
          }
          Gp[lt * r + c] = gp;
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        const uint32_t ob = base + buf * C::BUF;
        for (int kb = 0; kb < C::NKB; ++kb)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t d = sdesc_sw128(ob + kb * KBB + ks * 32);
            const uint32_t acc = (qc > 0 || kb > 0 || ks > 0) ? 1u : 0u;
            if (BF) mma_bf16(tbase, d, d, idesc, acc);
            else mma_tf32(tbase, d, d, idesc, acc);
          }
        mma_commit(&done[buf]);
      }
      if (t < r) {  // gradient: FP32 over the chunk, FP64 across chunks
        float s0 = 0.f, s1 = 0.f, a0 = 0.f, a1 = 0.f;
        int lt = 0;
        for (; lt + 2 <= nb; lt += 2) {
          const float x0 = Gp[lt * r + t], x1 = Gp[(lt + 1) * r + t];
          s0 += x0;
          s1 += x1;
          a0 += fabsf(x0);
          a1 += fabsf(x1);
        }
        if (lt < nb) {
          s0 += Gp[lt * r + t];
          a0 += fabsf(Gp[lt * r + t]);
        }
        facc_add(gacc, s0 + s1);
        facc_add(gabs, a0 + a1);
      }
      __syncthreads();
    }
  }
  if (t == 0) mma_commit(&fin);
  const bool fok = __syncthreads_and(alive && wait_bar(&fin, 0, err, 2));
  tc_fence_after();
  // energies: warp shuffles, then the warps in fixed order (double-float)
  FAcc vals[2 + 2 * KTRIAL];
  vals[0] = eacc;
  vals[1] = eabs;
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) {
    vals[2 + 2 * j] = etr[j];
    vals[3 + 2 * j] = atr[j];
  }
#pragma unroll
  for (int j = 0; j < 2 + 2 * KTRIAL; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) facc_merge(vals[j], facc_shfl_down(vals[j], o));
    if (lane == 0) red[warp][j] = vals[j];
  }
  __syncthreads();
  double* prow = part + (size_t)blockIdx.x * part_stride;
  if (t < 2 + 2 * KTRIAL) {
    FAcc sum;
    for (int w = 0; w < NT / 32; ++w) facc_merge(sum, red[w][t]);
    if (t < 2) prow[t] = facc_value(sum);
    else prow[nslots(r) + t - 2] = facc_value(sum);
  }
  if (t < r) {
    prow[slot_g(t)] = facc_value(gacc);
    prow[slot_gabs(r, t)] = facc_value(gabs);
  }
  // Gram rows: row c of the M = 64 accumulator is TMEM lane 32 (c / 16) + c % 16
  if (warp < 4) {
    const int c = 16 * warp + lane;
    const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16);
    for (int d0 = 0; d0 < Ng; d0 += 16) {
      uint32_t vv[16];
      tmem_ld16(ta + d0, vv);
      tmem_ld_wait();
      if (lane < 16 && c < r)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int d = d0 + j;
          if (d >= c && d < r)
            prow[slot_K(r) + c * r - (c * (c - 1)) / 2 + (d - c)] =
                fok ? (double)__uint_as_float(vv[j]) : 0.0;
        }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 64);
  }
}

}  // namespace tcel

// ------------------------------------------------------------------------
// Gradient-only form (the passes of the L-BFGS solve, Sec. 5): per tet the
// energy, its first derivative P and the KTRIAL trial energies (one tet per
// thread), then g += sum_e J_e^T ge_e with ge_e = w_e V_e dPsi/dx_e, the 12
// values (vertex a >= 1, component i) sum_j P_ij Dm^-1_{a-1,j} and their
// negated sum for vertex 0, held in shared memory while groups of r threads
// (one subspace column each) stream the tets' J rows, coalesced along the
// columns.  No Hessian, eigen-decomposition or K contraction.  Each CTA
// writes one complete partial row: E, sum |E terms|, g, gabs and the trial
// energies (the K slots are not written).
namespace gradel {
constexpr int ET = 128;

// VEC (FP32, r a multiple of 4): each thread of a group takes four adjacent
// columns and loads them as one float4 per J row (a quarter of the load
// instructions of the one-column mapping).
template <typename Real, bool VEC>
__global__ void __launch_bounds__(ET) element_grad_kernel(ElemArgs ea, const Real* __restrict__ u,
                                                          const Real* __restrict__ J,
                                                          const Real* __restrict__ ut,
                                                          double* __restrict__ part,
                                                          int part_stride) {
  __shared__ Real ge[ET][13];
  __shared__ int4 tvs[ET];
  __shared__ double red[2 + 2 * KTRIAL][ET];
  __shared__ double redv[VEC ? 2 : 1][VEC ? 4 * ET : 1];
  const int t = threadIdx.x, r = ea.r;
  const int G = ET / r;  // column groups
  const int grp = t / r, c = t - grp * r;
  const bool active = grp < G;
  const int Q = VEC ? r / 4 : 1;  // column quads (VEC)
  const int G4 = ET / Q;
  const int grp4 = t / Q, cq = t - grp4 * Q;
  const bool active4 = VEC && grp4 < G4;
  double gacc4[4] = {0.0, 0.0, 0.0, 0.0}, gabs4[4] = {0.0, 0.0, 0.0, 0.0};
  const Real mu = (Real)ea.mu, lam = (Real)ea.lam;
  const Real oma = (Real)(-0.75 * ea.mu / ea.lam);  // 1 - a
  double eacc = 0.0, eabs = 0.0, gacc = 0.0, gabs = 0.0;
  double tacc[KTRIAL], tabs[KTRIAL];
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) tacc[j] = tabs[j] = 0.0;
  const int ntiles = (ea.S + ET - 1) / ET;
  pdl_wait();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e = tile * ET + t;
    const int nt = min(ET, ea.S - tile * ET);
    if (e < ea.S) {
      int4 tv;
      Real Dmi[3][3], wv, H[3][3];
      load_tet<Real>(ea, e, tv, Dmi, wv);
      disp_grad<Real>(u, tv, Dmi, H);
      Invariants<Real> iv;
      invariants<Real>(H, iv);
      const double pe = (double)(wv * snh_psi<Real>(iv, mu, lam, oma));
      eacc += pe;
      eabs += fabs(pe);
      const Real Ic = iv.Ic3 + Real(3);
      const Real dl = iv.Ic3 / (Real(4) * (Ic + Real(1)));
      const Real lJ = lam * iv.Jm1;
      Real P[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const Real Fij = H[i][j] + (i == j ? Real(1) : Real(0));
          P[i][j] = wv * (mu * dl * Fij + lJ * iv.cof[i][j] +
                          Real(0.75) * mu *
                              (H[i][j] + H[j][i] - (i == j ? iv.trH : Real(0)) - iv.cofH[i][j]));
        }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Real s0 = Real(0);
#pragma unroll
        for (int a = 1; a < 4; ++a) {
          const Real v = P[i][0] * Dmi[a - 1][0] + P[i][1] * Dmi[a - 1][1] +
                         P[i][2] * Dmi[a - 1][2];
          ge[t][3 * a + i] = v;
          s0 += v;
        }
        ge[t][i] = -s0;
      }
      tvs[t] = tv;
#pragma unroll
      for (int j = 0; j < KTRIAL; ++j) {
        Real Ht[3][3];
        disp_grad<Real>(ut + (size_t)j * ea.n, tv, Dmi, Ht);
        Invariants<Real> ivt;
        invariants<Real>(Ht, ivt);
        const double pt = (double)(wv * snh_psi<Real>(ivt, mu, lam, oma));
        tacc[j] += pt;
        tabs[j] += fabs(pt);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) ge[t][k] = Real(0);
      tvs[t] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    if (VEC) {
      // four columns per thread: one 16-byte load per J row
      if (active4) {
        float sg[4] = {0.f, 0.f, 0.f, 0.f}, sa[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int lt = grp4; lt < nt; lt += G4) {
          const int4 tv = tvs[lt];
          const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
          float gp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const float4 jv = __ldg(reinterpret_cast<const float4*>(
                  J + (size_t)(3 * vv[a] + i) * r + 4 * cq));
              const float w = (float)ge[lt][3 * a + i];
              gp[0] += w * jv.x;
              gp[1] += w * jv.y;
              gp[2] += w * jv.z;
              gp[3] += w * jv.w;
            }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            sg[k] += gp[k];
            sa[k] += fabsf(gp[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          gacc4[k] += (double)sg[k];
          gabs4[k] += (double)sa[k];
        }
      }
    } else if (active) {
      Real sg = Real(0), sa = Real(0);
#pragma unroll 4
      for (int lt = grp; lt < nt; lt += G) {
        const int4 tv = tvs[lt];
        const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
        Real gp = Real(0);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i)
            gp += ge[lt][3 * a + i] * __ldg(J + (size_t)(3 * vv[a] + i) * r + c);
        sg += gp;
        sa += fabs(gp);
      }
      gacc += (double)sg;
      gabs += (double)sa;
    }
    __syncthreads();
  }
  red[0][t] = eacc;
  red[1][t] = eabs;
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) {
    red[2 + 2 * j][t] = tacc[j];
    red[3 + 2 * j][t] = tabs[j];
  }
  __syncthreads();
  for (int h = ET / 2; h > 0; h >>= 1) {
    if (t < h) {
#pragma unroll
      for (int k = 0; k < 2 + 2 * KTRIAL; ++k) red[k][t] += red[k][t + h];
    }
    __syncthreads();
  }
  double* prow = part + (size_t)blockIdx.x * part_stride;
  if (t == 0) {
    prow[0] = red[0][0];
    prow[1] = red[1][0];
  }
  if (t < 2 * KTRIAL) prow[nslots(r) + t] = red[2 + t][0];
  __syncthreads();
  if (VEC) {
    // thread (grp4, cq) holds columns 4 cq .. 4 cq + 3 of group grp4
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      redv[0][4 * t + k] = active4 ? gacc4[k] : 0.0;
      redv[1][4 * t + k] = active4 ? gabs4[k] : 0.0;
    }
    __syncthreads();
    if (t < r) {  // column t = 4 cq + k: entry 4 (q Q + cq) + k of group q
      double s0 = 0.0, a0 = 0.0;
      for (int q = 0; q < G4; ++q) {
        s0 += redv[0][4 * q * Q + t];
        a0 += redv[1][4 * q * Q + t];
      }
      prow[slot_g(t)] = s0;
      prow[slot_gabs(r, t)] = a0;
    }
    return;
  }
  red[0][t] = active ? gacc : 0.0;
  red[1][t] = active ? gabs : 0.0;
  __syncthreads();
  if (t < r) {  // the column groups in fixed order
    double s0 = 0.0, a0 = 0.0;
    for (int q = 0; q < G; ++q) {
      s0 += red[0][q * r + t];
      a0 += red[1][q * r + t];
    }
    prow[slot_g(t)] = s0;
    prow[slot_gabs(r, t)] = a0;
  }
}
}  // namespace gradel

// ------------------------------------------------------------------------
// Per-tet reduced elastic forces for the cubature fit (Sec. 4.3): for every
// tet e of the mesh (unit weight) the r values J_e^T dP_e/dx_e, P_e = V_e
// Psi(F_e), written to A[i * ne + e] (one row per subspace column, coalesced
// along the tets).  One thread per tet.
template <typename Real>
__global__ void __launch_bounds__(128) tet_force_kernel(const int4* __restrict__ tets,
                                                        const double* __restrict__ dminv,
                                                        const double* __restrict__ vol, int ne,
                                                        int r, const Real* __restrict__ u,
                                                        const Real* __restrict__ J, Real mu,
                                                        Real lam, double* __restrict__ A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int4 tv = tets[e];
  Real Dmi[3][3], H[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Dmi[a][b] = (Real)dminv[(3 * a + b) * ne + e];
  const Real wv = (Real)vol[e];
  disp_grad<Real>(u, tv, Dmi, H);
  Real ge[12];
  snh_tet_forces<Real>(H, Dmi, wv, mu, lam, ge);
  const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
  for (int c = 0; c < r; ++c) {
    Real acc = Real(0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) acc += ge[3 * a + i] * J[(size_t)(3 * vv[a] + i) * r + c];
    A[(size_t)c * ne + e] = (double)acc;
  }
}

// ------------------------------------------------------------- full space
// Full-space projective Newton (Eq. 1 over all n DOFs, every tet at unit
// weight): the comparison solve of the reduced method.  The projected element
// Hessian is kept in factored form, Hproj_e = A_e^T A_e, with A_e the map of
// element_item_td applied to the tet's four vertex displacements (in place of
// four rows of J), so a Hessian-vector product is A_e^T (A_e v_e) per tet,
// scattered with FP64 atomics.  The per-tet factor data (U, V, the scaled
// scaling modes and the twist / flip scales: FS_NF values) are stored
// structure-of-arrays [FS_NF][ne] at each Newton iterate.
namespace fullsp {
constexpr int NT = 64;   // tets per CTA of the evaluation kernel
constexpr int HT = 128;  // threads of the Hessian-vector and energy kernels

// Sums a and b over the CTA (NTH threads) and stores them at out[0], out[1].
template <int NTH>
__device__ __forceinline__ void block_sum2(double a, double b, double* out) {
  __shared__ double sh[2][NTH / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < NTH / 32; ++k) {
      s0 += sh[0][k];
      s1 += sh[1][k];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

// Adjoint of element_item_td: f = A_e^T Cv as forces on the tet's four
// vertices.  The eigen coordinates Cv give S in the (U, V) frame, the
// perturbation of F is U S V^T, and its vertex forces follow from D.
template <typename Real>
__device__ __forceinline__ void item_adjoint(const TetData<Real>& td, const Real (&Cv)[9],
                                             Real (&f)[4][3]) {
  Real S[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) S[a][b] = Real(0);
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int a = 0; a < 3; ++a) S[a][a] += td.As[3 * m + a] * Cv[m];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    const Real tw = td.tf[i] * Cv[3 + i], fl = td.tf[3 + i] * Cv[6 + i];
    S[j][k] += tw + fl;
    S[k][j] += fl - tw;
  }
  Real US[3][3], Gb[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      US[i][b] = td.U[3 * i] * S[0][b] + td.U[3 * i + 1] * S[1][b] + td.U[3 * i + 2] * S[2][b];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Gb[i][c] = US[i][0] * td.V[3 * c] + US[i][1] * td.V[3 * c + 1] + US[i][2] * td.V[3 * c + 2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      f[a][i] = td.D[3 * a] * Gb[i][0] + td.D[3 * a + 1] * Gb[i][1] + td.D[3 * a + 2] * Gb[i][2];
}

// Evaluation at the Newton iterate u = q - X0: per tet the energy (summed
// per CTA into part[2 b], part[2 b + 1] = sum |terms|), the gradient
// scattered into g (and |contributions| into gabs: the rounding scale of
// each g_i), the factor data into fac and the diagonal of A_e^T A_e (the
// Jacobi preconditioner) scattered into diag.  g, gabs and diag are zeroed
// by the caller.  ea.S = ne, ea.dminv / ea.wv the tets' Dm^-1 and volumes.
template <typename Real>
__global__ void __launch_bounds__(NT) fs_elem_kernel(ElemArgs ea, const Real* __restrict__ u,
                                                     Real* __restrict__ fac,
                                                     double* __restrict__ g,
                                                     double* __restrict__ gabs,
                                                     double* __restrict__ diag,
                                                     double* __restrict__ part) {
  __shared__ ElemTile<Real, NT> tl;
  const int t = threadIdx.x;
  const int ne = ea.S;
  const Real mu = (Real)ea.mu, lam = (Real)ea.lam;
  const Real oma = (Real)(-0.75 * ea.mu / ea.lam);  // 1 - a
  double eacc = 0.0, eabs = 0.0;
  for (int e0 = blockIdx.x * NT; e0 < ne; e0 += gridDim.x * NT) {
    const int e = e0 + t;
    Real pe;
    // each thread writes and reads back only its own slot of the tile
    element_phase1<Real, NT>(ea, u, e, t, tl, mu, lam, oma, pe);
    if (e >= ne) continue;
    eacc += (double)pe;
    eabs += fabs((double)pe);
    TetData<Real> td;
    load_tet_data<Real, NT>(tl, t, td);
    const int4 tv = ea.tets[e];
    const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const Real fa = td.D[3 * a] * td.p[3 * i] + td.D[3 * a + 1] * td.p[3 * i + 1] +
                        td.D[3 * a + 2] * td.p[3 * i + 2];
        atomicAdd(&g[3 * vv[a] + i], (double)fa);
        atomicAdd(&gabs[3 * vv[a] + i], fabs((double)fa));
      }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      fac[(size_t)k * ne + e] = td.U[k];
      fac[(size_t)(9 + k) * ne + e] = td.V[k];
      fac[(size_t)(18 + k) * ne + e] = td.As[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) fac[(size_t)(27 + k) * ne + e] = td.tf[k];
    // diagonal entries |A_e e_(a,i)|^2
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        Real jv[4][3];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int k = 0; k < 3; ++k) jv[b][k] = (b == a && k == i) ? Real(1) : Real(0);
        Real Cv[9], gp = Real(0);
        element_item_td<Real>(td, jv, Cv, gp);
        Real s = Real(0);
#pragma unroll
        for (int m = 0; m < 9; ++m) s += Cv[m] * Cv[m];
        atomicAdd(&diag[3 * vv[a] + i], (double)s);
      }
  }
  block_sum2<NT>(eacc, eabs, part + 2 * blockIdx.x);
}

// y += sum_e A_e^T A_e p_e (skipped once *done is set).
template <typename Real>
__global__ void __launch_bounds__(HT) fs_hv_kernel(const int4* __restrict__ tets,
                                                   const Real* __restrict__ dminv, int ne,
                                                   const Real* __restrict__ fac,
                                                   const double* __restrict__ p,
                                                   double* __restrict__ y,
                                                   const int* __restrict__ done) {
  if (*done) return;
  for (int e = blockIdx.x * HT + threadIdx.x; e < ne; e += gridDim.x * HT) {
    const int4 tv = tets[e];
    const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
    TetData<Real> td;
    Real Dmi[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Dmi[a][b] = dminv[(size_t)(3 * a + b) * ne + e];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      td.D[j] = -(Dmi[0][j] + Dmi[1][j] + Dmi[2][j]);
#pragma unroll
      for (int a = 1; a < 4; ++a) td.D[3 * a + j] = Dmi[a - 1][j];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      td.p[k] = Real(0);
      td.U[k] = fac[(size_t)k * ne + e];
      td.V[k] = fac[(size_t)(9 + k) * ne + e];
      td.As[k] = fac[(size_t)(18 + k) * ne + e];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) td.tf[k] = fac[(size_t)(27 + k) * ne + e];
    Real jv[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) jv[a][i] = (Real)p[3 * vv[a] + i];
    Real Cv[9], gp = Real(0), f[4][3];
    element_item_td<Real>(td, jv, Cv, gp);
    item_adjoint<Real>(td, Cv, f);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(&y[3 * vv[a] + i], (double)f[a][i]);
  }
}

// Elastic energy at q + alpha d (line-search trials), summed per CTA into
// part[2 b] and part[2 b + 1] = sum |terms|.
template <typename Real>
__global__ void __launch_bounds__(HT) fs_energy_kernel(
    const int4* __restrict__ tets, const Real* __restrict__ dminv, const Real* __restrict__ wv,
    int ne, const double* __restrict__ q, const double* __restrict__ X0,
    const double* __restrict__ d, double alpha, double mu_d, double lam_d,
    double* __restrict__ part) {
  const Real mu = (Real)mu_d, lam = (Real)lam_d;
  const Real oma = (Real)(-0.75 * mu_d / lam_d);
  double eacc = 0.0, eabs = 0.0;
  for (int e = blockIdx.x * HT + threadIdx.x; e < ne; e += gridDim.x * HT) {
    const int4 tv = tets[e];
    const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
    Real uu[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int k = 3 * vv[a] + i;
        uu[a][i] = (Real)(q[k] - X0[k] + alpha * d[k]);
      }
    Real Dmi[3][3], H[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Dmi[a][b] = dminv[(size_t)(3 * a + b) * ne + e];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Real s = Real(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) s += (uu[a + 1][i] - uu[0][i]) * Dmi[a][j];
        H[i][j] = s;
      }
    Invariants<Real> iv;
    invariants<Real>(H, iv);
    const double pe = (double)(wv[e] * snh_psi<Real>(iv, mu, lam, oma));
    eacc += pe;
    eabs += fabs(pe);
  }
  block_sum2<HT>(eacc, eabs, part + 2 * blockIdx.x);
}
}  // namespace fullsp

}  // namespace

// Small cubature sets use 64-tet tiles so that more CTAs share the work.
static int element_tile(int S, int num_sms) { return S <= 64 * 2 * num_sms ? 64 : 128; }

void element_grids(int S, int r, int num_sms, int& gfull, int& genergy) {
  const int et = element_tile(S, num_sms);
  const int tiles = (S + et - 1) / et;
  gfull = std::max(1, std::min(tiles, num_sms * 2));
  genergy = std::max(1, std::min(tiles, num_sms * 2));
  (void)r;
}

template <typename Real>
void launch_element(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                    double* part, int gfull, int genergy, cudaStream_t s) {
  // the tile size must match element_grids
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (element_tile(ea.S, sms) == 64)
    run_element_r<Real, 64>(ea, u, J, ut, part, gfull, genergy, s);
  else
    run_element_r<Real, 128>(ea, u, J, ut, part, gfull, genergy, s);
}

static int num_sms_cached() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

// tets per tile: 256, or fewer (down to 16) when that leaves SMs idle
int element_tc_tile(int S, int num_sms) {
  int tt = tcel::ET;
  while (tt > 16 && (long long)(tt / 2) * num_sms >= S) tt /= 2;
  return tt;
}

int element_tc_grid(int S, int r, bool bf16, int num_sms) {
  if (element_ws_applies(S, r, bf16, num_sms)) return element_ws_grid(S, num_sms);
  const int tt = element_tc_tile(S, num_sms);
  return std::max(1, std::min((S + tt - 1) / tt, num_sms));
}

cudaError_t launch_element_tc(const ElemArgs& ea, const float* u, const float* J,
                              const float* ut, double* part, int grid, bool bf16, int* err,
                              int num_sms, cudaStream_t s) {
  if (ea.r > tcel::GROWS) return cudaErrorInvalidValue;
  // large tet sets: the warp-specialised kernel (element_ws.cu)
  if (element_ws_applies(ea.S, ea.r, bf16, num_sms))
    return launch_element_ws(ea, u, J, ut, part, grid, err, s);
  static size_t set_bf = 0, set_tf = 0;
  if (bf16) {
    const size_t sm = tcel::smem_bytes<true>(ea.r);
    if (sm > set_bf) {
      cudaError_t e = cudaFuncSetAttribute(tcel::element_tc_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      set_bf = sm;
    }
    return launch_pdl(tcel::element_tc_kernel<true>, dim3(grid), dim3(tcel::NT), sm, s, ea, u, J,
                      ut, part, nslots_total(ea.r), element_tc_tile(ea.S, num_sms_cached()), err);
  } else {
    const size_t sm = tcel::smem_bytes<false>(ea.r);
    if (sm > set_tf) {
      cudaError_t e = cudaFuncSetAttribute(tcel::element_tc_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      set_tf = sm;
    }
    return launch_pdl(tcel::element_tc_kernel<false>, dim3(grid), dim3(tcel::NT), sm, s, ea, u,
                      J, ut, part, nslots_total(ea.r), element_tc_tile(ea.S, num_sms_cached()),
                      err);
  }
  return cudaGetLastError();
}

template <typename Real>
void launch_tet_forces(const int4* tets, const double* dminv, const double* vol, int ne, int r,
                       const Real* u, const Real* J, double mu, double lam, double* A,
                       cudaStream_t s) {
  tet_force_kernel<Real><<<(ne + 127) / 128, 128, 0, s>>>(tets, dminv, vol, ne, r, u, J,
                                                          (Real)mu, (Real)lam, A);
}
template void launch_tet_forces<float>(const int4*, const double*, const double*, int, int,
                                       const float*, const float*, double, double, double*,
                                       cudaStream_t);
template void launch_tet_forces<double>(const int4*, const double*, const double*, int, int,
                                        const double*, const double*, double, double, double*,
                                        cudaStream_t);

int fs_grid(int ne, int threads, int num_sms) {
  return std::max(1, std::min((ne + threads - 1) / threads, 8 * num_sms));
}

template <typename Real>
void launch_fs_elem(const ElemArgs& ea, const Real* u, Real* fac, double* g, double* gabs,
                    double* diag, double* part, int grid, cudaStream_t s) {
  fullsp::fs_elem_kernel<Real><<<grid, fullsp::NT, 0, s>>>(ea, u, fac, g, gabs, diag, part);
}

template <typename Real>
void launch_fs_hv(const int4* tets, const Real* dminv, int ne, const Real* fac, const double* p,
                  double* y, const int* done, int grid, cudaStream_t s) {
  fullsp::fs_hv_kernel<Real><<<grid, fullsp::HT, 0, s>>>(tets, dminv, ne, fac, p, y, done);
}

template <typename Real>
void launch_fs_energy(const int4* tets, const Real* dminv, const Real* wv, int ne,
                      const double* q, const double* X0, const double* d, double alpha,
                      double mu, double lam, double* part, int grid, cudaStream_t s) {
  fullsp::fs_energy_kernel<Real><<<grid, fullsp::HT, 0, s>>>(tets, dminv, wv, ne, q, X0, d,
                                                             alpha, mu, lam, part);
}

template void launch_fs_elem<float>(const ElemArgs&, const float*, float*, double*, double*,
                                    double*, double*, int, cudaStream_t);
template void launch_fs_elem<double>(const ElemArgs&, const double*, double*, double*,
                                     double*, double*, double*, int, cudaStream_t);
template void launch_fs_hv<float>(const int4*, const float*, int, const float*, const double*,
                                  double*, const int*, int, cudaStream_t);
template void launch_fs_hv<double>(const int4*, const double*, int, const double*,
                                   const double*, double*, const int*, int, cudaStream_t);
template void launch_fs_energy<float>(const int4*, const float*, const float*, int,
                                      const double*, const double*, const double*, double,
                                      double, double, double*, int, cudaStream_t);
template void launch_fs_energy<double>(const int4*, const double*, const double*, int,
                                       const double*, const double*, const double*, double,
                                       double, double, double*, int, cudaStream_t);

int element_grad_grid(int S, int num_sms) {
  const int tiles = (S + gradel::ET - 1) / gradel::ET;
  return std::max(1, std::min(tiles, 8 * num_sms));
}

template <typename Real>
void launch_element_grad(const ElemArgs& ea, const Real* u, const Real* J, const Real* ut,
                         double* part, int grid, cudaStream_t s) {
  if (sizeof(Real) == 4 && ea.r % 4 == 0)
    launch_pdl(gradel::element_grad_kernel<Real, sizeof(Real) == 4>, dim3(grid),
               dim3(gradel::ET), 0, s, ea, u, J, ut, part, nslots_total(ea.r));
  else
    launch_pdl(gradel::element_grad_kernel<Real, false>, dim3(grid), dim3(gradel::ET), 0, s, ea,
               u, J, ut, part, nslots_total(ea.r));
}

template void launch_element_grad<float>(const ElemArgs&, const float*, const float*,
                                         const float*, double*, int, cudaStream_t);
template void launch_element_grad<double>(const ElemArgs&, const double*, const double*,
                                          const double*, double*, int, cudaStream_t);
template void launch_element<float>(const ElemArgs&, const float*, const float*, const float*,
                                    double*, int, int, cudaStream_t);
template void launch_element<double>(const ElemArgs&, const double*, const double*,
                                     const double*, double*, int, int, cudaStream_t);

}  // namespace lsn
