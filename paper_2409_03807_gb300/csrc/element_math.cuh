// Per-tet element math shared by the element kernels (Sec. 5.1 stable
// neo-Hookean energy; projective Newton's per-element eigensystem,
// Supplement): invariants of the displacement gradient Hd = F - I, the
// energy density, a cyclic Jacobi eigen-decomposition of symmetric 3x3
// matrices and the rotation-signed SVD built on it, the loads of a tet's
// indices, inverse rest edges and weight, and a tet's elastic forces.
// Included by element.cu, element_ws.cu and curvature.cu.
#pragma once
#include "lsn_internal.cuh"

namespace lsn {
namespace {

template <typename Real>
struct Consts {
  static constexpr int sweeps = 10;
};
template <>
struct Consts<double> {
  static constexpr int sweeps = 16;
};

template <typename Real>
__device__ __forceinline__ Real sqrt_r(Real x) { return sqrt(x); }
template <>
__device__ __forceinline__ float sqrt_r<float>(float x) { return sqrtf(x); }
template <typename Real>
__device__ __forceinline__ Real log1p_r(Real x) { return log1p(x); }
template <>
__device__ __forceinline__ float log1p_r<float>(float x) { return log1pf(x); }

template <typename Real>
struct Invariants {
  Real Ic3, Jm1, cof[3][3], cofH[3][3], trH;
};

template <typename Real>
__device__ __forceinline__ void invariants(const Real (&H)[3][3], Invariants<Real>& iv) {
  iv.trH = H[0][0] + H[1][1] + H[2][2];
  Real nrm2 = Real(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) nrm2 += H[i][j] * H[i][j];
  iv.Ic3 = Real(2) * iv.trH + nrm2;
  // cofactor of Hd: cofH_ij = Hd_{i+1,j+1} Hd_{i+2,j+2} - Hd_{i+1,j+2} Hd_{i+2,j+1}
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      iv.cofH[i][j] = H[i1][j1] * H[i2][j2] - H[i1][j2] * H[i2][j1];
    }
  const Real m2 = iv.cofH[0][0] + iv.cofH[1][1] + iv.cofH[2][2];
  const Real detH = H[0][0] * iv.cofH[0][0] + H[0][1] * iv.cofH[0][1] + H[0][2] * iv.cofH[0][2];
  iv.Jm1 = iv.trH + m2 + detH;
  // cof(I + Hd) = (1 + tr Hd) I - Hd^T + cof(Hd)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      iv.cof[i][j] = (i == j ? Real(1) + iv.trH : Real(0)) - H[j][i] + iv.cofH[i][j];
}

template <typename Real>
__device__ __forceinline__ Real snh_psi(const Invariants<Real>& iv, Real mu, Real lam,
                                        Real oma /* 1 - a */) {
  return Real(0.5) * mu * iv.Ic3 - Real(0.5) * mu * log1p_r<Real>(iv.Ic3 * Real(0.25)) +
         Real(0.5) * lam * iv.Jm1 * (iv.Jm1 + Real(2) * oma);
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix A (in place:
// A becomes diagonal), accumulating the rotations in Q (A_in = Q diag Q^T).
// FAST (FP32 only): the rotation's tangent from an approximate quotient and
// reciprocal, and c = rsqrt(1 + t^2), s = t c.  The tangent only steers how
// fast the sweep converges; c^2 + s^2 = 1 holds to the rsqrt rounding, so the
// accumulated Q stays orthogonal and the stopping test is the same.
template <bool FAST, typename Real>
__device__ __forceinline__ Real quot(Real a, Real b) {
  if (FAST && sizeof(Real) == 4) return (Real)__fdividef((float)a, (float)b);
  return a / b;
}
template <bool FAST, typename Real>
__device__ __forceinline__ Real inv_sqrt(Real x) {
  if (FAST && sizeof(Real) == 4) return (Real)rsqrtf((float)x);
  return Real(1) / sqrt_r<Real>(x);
}

template <typename Real, bool FAST = false>
__device__ __forceinline__ void jacobi3(Real (&A)[3][3], Real (&Q)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = (i == j) ? Real(1) : Real(0);
  const Real tiny = sizeof(Real) == 4 ? Real(1e-30) : Real(1e-300);
  // off-diagonal mass below (unit roundoff)^2 of the diagonal: converged
  const Real rel = sizeof(Real) == 4 ? Real(1e-13) : Real(1e-29);
#pragma unroll 1
  for (int sweep = 0; sweep < Consts<Real>::sweeps; ++sweep) {
    const Real off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const Real dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= rel * dia + tiny) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const Real apq = A[p][q];
      if (fabs(apq) > tiny) {
        const Real theta = quot<FAST>(A[q][q] - A[p][p], Real(2) * apq);
        const Real at = fabs(theta);
        Real t = (at > Real(1e15)) ? quot<FAST>(Real(0.5), at)
                                   : quot<FAST>(Real(1), at + sqrt_r<Real>(theta * theta + Real(1)));
        if (theta < Real(0)) t = -t;
        const Real c = inv_sqrt<FAST>(t * t + Real(1));
        const Real s = t * c;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const Real akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const Real apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        A[p][q] = Real(0);
        A[q][p] = Real(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const Real qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = c * qkp - s * qkq;
          Q[k][q] = s * qkp + c * qkq;
        }
      }
    }
  }
}

// Rotation-signed SVD F = U diag(sig) V^T with det U = det V = +1 (sig[i]
// may be negative for an inverted element).
template <typename Real, bool FAST = false>
__device__ __forceinline__ void svd3(const Real (&F)[3][3], Real (&U)[3][3], Real (&sig)[3],
                                     Real (&V)[3][3]) {
  Real S[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) S[a][b] = F[0][a] * F[0][b] + F[1][a] * F[1][b] + F[2][a] * F[2][b];
  jacobi3<Real, FAST>(S, V);
  const Real detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                    V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                    V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < Real(0)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
  }
  // largest, middle, smallest of the squared singular values
  const Real d0 = S[0][0], d1 = S[1][1], d2 = S[2][2];
  int i0 = 0, i1 = 1, i2 = 2;
  if (d1 > d0) { i0 = 1; i1 = 0; }
  if (d2 > (i0 == 0 ? d0 : d1)) { i2 = i1; i1 = i0; i0 = 2; }
  else if (d2 > (i1 == 0 ? d0 : (i1 == 1 ? d1 : d2))) { i2 = i1; i1 = 2; }
  Real FV[3][3];  // columns F v_i
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) FV[a][i] = F[a][0] * V[0][i] + F[a][1] * V[1][i] + F[a][2] * V[2][i];
  Real u0[3], u1[3], u2[3];
  const Real tiny = sizeof(Real) == 4 ? Real(1e-30) : Real(1e-300);
  Real n0 = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u0[a] = FV[a][i0];
    n0 += u0[a] * u0[a];
  }
  if (n0 > tiny) {
    n0 = inv_sqrt<FAST>(n0);
#pragma unroll
    for (int a = 0; a < 3; ++a) u0[a] *= n0;
  } else {
    u0[0] = Real(1); u0[1] = Real(0); u0[2] = Real(0);
  }
  Real dp = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) dp += u0[a] * FV[a][i1];
  Real n1 = Real(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u1[a] = FV[a][i1] - dp * u0[a];
    n1 += u1[a] * u1[a];
  }
  if (n1 > tiny * Real(1e6)) {
    n1 = inv_sqrt<FAST>(n1);
#pragma unroll
    for (int a = 0; a < 3; ++a) u1[a] *= n1;
  } else {  // any unit vector orthogonal to u0
    const int k = fabs(u0[0]) < Real(0.6) ? 0 : (fabs(u0[1]) < Real(0.6) ? 1 : 2);
    Real e[3] = {Real(0), Real(0), Real(0)};
    e[k] = Real(1);
    const Real ue = u0[k];
    Real nn = Real(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      u1[a] = e[a] - ue * u0[a];
      nn += u1[a] * u1[a];
    }
    nn = inv_sqrt<FAST>(nn);
#pragma unroll
    for (int a = 0; a < 3; ++a) u1[a] *= nn;
  }
  // u2 = +-(u0 x u1) so that det[U] = +1 with columns placed at i0, i1, i2
  const bool even = (i0 == 0 && i1 == 1) || (i0 == 1 && i1 == 2) || (i0 == 2 && i1 == 0);
  const Real sg = even ? Real(1) : Real(-1);
  u2[0] = sg * (u0[1] * u1[2] - u0[2] * u1[1]);
  u2[1] = sg * (u0[2] * u1[0] - u0[0] * u1[2]);
  u2[2] = sg * (u0[0] * u1[1] - u0[1] * u1[0]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    U[a][i0] = u0[a];
    U[a][i1] = u1[a];
    U[a][i2] = u2[a];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    sig[i] = U[0][i] * FV[0][i] + U[1][i] * FV[1][i] + U[2][i] * FV[2][i];
}

template <typename Real>
__device__ __forceinline__ void load_tet(const ElemArgs& ea, int e, int4& tv, Real (&Dmi)[3][3],
                                         Real& wv) {
  const Real* dm = static_cast<const Real*>(ea.dminv);
  tv = ea.tets[e];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Dmi[a][b] = dm[(3 * a + b) * ea.S + e];
  wv = static_cast<const Real*>(ea.wv)[e];
}

template <typename Real>
__device__ __forceinline__ void disp_grad(const Real* __restrict__ u, const int4& tv,
                                          const Real (&Dmi)[3][3], Real (&H)[3][3]) {
  const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
  Real Du[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const Real u0 = u[3 * vv[0] + i];
#pragma unroll
    for (int a = 0; a < 3; ++a) Du[i][a] = u[3 * vv[a + 1] + i] - u0;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[i][j] = Du[i][0] * Dmi[0][j] + Du[i][1] * Dmi[1][j] + Du[i][2] * Dmi[2][j];
}

// Elastic forces of one tet, d(wv Psi(F))/dx for its four vertices
// (ge[3 a + i]: vertex a, component i), from the displacement gradient H =
// F - I, the inverse rest edge matrix and the weighted volume wv.
template <typename Real>
__device__ __forceinline__ void snh_tet_forces(const Real (&H)[3][3], const Real (&Dmi)[3][3],
                                               Real wv, Real mu, Real lam, Real (&ge)[12]) {
  Invariants<Real> iv;
  invariants<Real>(H, iv);
  const Real Ic = iv.Ic3 + Real(3);
  const Real dl = iv.Ic3 / (Real(4) * (Ic + Real(1)));
  const Real lJ = lam * iv.Jm1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Real P[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Real Fij = H[i][j] + (i == j ? Real(1) : Real(0));
      P[j] = wv * (mu * dl * Fij + lJ * iv.cof[i][j] +
                   Real(0.75) * mu *
                       (H[i][j] + H[j][i] - (i == j ? iv.trH : Real(0)) - iv.cofH[i][j]));
    }
    Real s0 = Real(0);
#pragma unroll
    for (int a = 1; a < 4; ++a) {
      const Real v = P[0] * Dmi[a - 1][0] + P[1] * Dmi[a - 1][1] + P[2] * Dmi[a - 1][2];
      ge[3 * a + i] = v;
      s0 += v;
    }
    ge[i] = -s0;
  }
}

}  // namespace
}  // namespace lsn
