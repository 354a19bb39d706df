// Warp-specialised tensor-core element kernel for large tet sets (the BF16
// form when every tet of a large mesh, or a large cubature set, is
// evaluated; the TF32 form keeps element_tc_kernel, whose K-major operand
// tcgen05 needs for TF32).  It computes what element_tc_kernel computes
// (Sec. 3.1 Eq. 2 and Eq. 11: per-tet stable neo-Hookean energy, gradient and the
// PSD-projected Hessian of projective Newton, contracted with the tets' rows
// of J into g and K; the line-search trial energies), with the three kinds of
// work running concurrently on different warps of a persistent CTA:
//
//   warps 0-4  (element math)  one tet per thread: energy, P, the signed SVD
//              and the clamped eigensystem of d2Psi/dF2, and the KTRIAL
//              trial energies; each tet's result is a 60-word record in
//              shared memory (double-buffered units of 160 tets); five
//              warps of this long per-tet dependency chain (two 3x3 Jacobi
//              decompositions) keep ten column-build warps supplied;
//   warps 5-14 (column build)  for a tet and four adjacent subspace columns
//              (one float4 per J row, staged in shared memory by
//              asynchronous copies one tet ahead, bypassing L1): dJ_a = J_a - J_0 (a = 1..3),
//              w_a = U^T dJ_a, R = sum_a w_a y_a^T (= U^T G V with
//              y_a = V^T Dm^-1 row a), the nine eigen-coordinates C_e (scaled
//              by sqrt(w V lambda+)) and the gradient term sum_a ge_a . dJ_a;
//              C_e goes, rounded, into an MN-major operand (K row = (tet,
//              eigen-row), the 64 subspace columns contiguous, 128-byte
//              swizzle), one 8-byte store of four BF16 values per row;
//   warp 15    issues the MMA chain D += Op Op^T (M = 64, N = r rounded up to
//              16) into TMEM per operand chunk and commits it.
//
// Hand-offs are mbarriers (records full / free, operand chunk full / free);
// every wait is bounded by %globaltimer and reports through the error flag.
// The gradient stays FP32 per chunk and double-float across chunks; energies
// are double-float.  Each CTA writes one complete partial row (E, sum|E|, g,
// sum|g terms|, K upper triangle, trial energies).
#include <cuda_bf16.h>

#include "element_math.cuh"
#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace lsn {
namespace tcws {

using namespace tc;

constexpr int NPW = 5;                    // element-math warps
constexpr int NBW = 10;                   // column-build warps
constexpr int MMAW = NPW + NBW;           // the MMA-issuing warp
constexpr int NT = 32 * (NPW + NBW + 1);  // 512 threads
constexpr int UNIT = 32 * NPW;            // tets per record unit
constexpr int NBT = 32 * NBW;             // column-build threads
constexpr int RW = 60;                    // words per tet record (conflict-free float4 rows)
constexpr int GROWS = 64;                 // operand columns (r <= 64)
constexpr unsigned long long WAIT_NS = 2000000000ull;

// record layout (words; each group starts on a float4)
constexpr int R_V = 0;    // int4 vertex ids
constexpr int R_UT = 4;   // U^T, row-major: UT[p][i] = U[i][p]
constexpr int R_Y = 16;   // y_a[q] = sum_j Dm^-1[a][j] V[j][q], a = 0..2 (vertices 1..3)
constexpr int R_AS = 28;  // scaling modes: sqrt(w V lambda_m+) a_m[i]
constexpr int R_TF = 40;  // sqrt(w V lambda+ / 2): 3 twist, then 3 flip modes
constexpr int R_GE = 48;  // ge_a[i] = sum_j (w V P)[i][j] Dm^-1[a][j]

constexpr int CH = NBT / 16;              // tets per operand chunk: one per column-build
                                          // thread group of r / 4 <= 16 threads
constexpr int NCH = UNIT / CH;            // chunks per unit
constexpr int KSTEP = 16;                 // K rows (BF16 values) per MMA
constexpr int KR = (9 * CH + KSTEP - 1) / KSTEP * KSTEP;  // K rows per chunk (zero-padded)
constexpr int NSTEP = KR / KSTEP;         // MMAs per chunk
constexpr uint32_t BUF = KR * 128u;       // operand bytes per chunk (128 bytes per K row)
constexpr uint32_t STG = 12 * 16;         // staged J rows per column-build thread
constexpr int NOB = 3;                    // operand buffers (chunks in flight)
static_assert(UNIT % CH == 0, "chunks tile a unit");

constexpr size_t smem_bytes() {
  return NOB * (size_t)BUF + 2 * (size_t)UNIT * RW * 4 + (size_t)NBT * STG + 1024;
}
// the dynamic shared memory plus the kernel's static barriers and reduction
// buffer (about 1.1 KB) must fit the 227 KB a block may use
static_assert(smem_bytes() + 2048 <= 232448, "shared memory of the element kernel");

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase of `bar` with the given parity; on time-out the
// error code is recorded and false returned
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

// MN-major, 128-byte-swizzled operand descriptor: 8 K rows of 128 bytes (64
// BF16 columns each) form a 1024-byte atom; `sbo` is the distance between
// the atoms of successive 8-row groups along K, `lbo` the distance between
// the atoms of successive 64-column blocks (unused with 64 columns).
__device__ __forceinline__ uint64_t sdesc_mn128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}

// byte offset of (K row kr, column c) in a chunk's operand (c a multiple of
// 4): one 128-byte row per K row, 8 BF16 columns per 16-byte chunk, chunk j
// of row kr at position j ^ (kr & 7)
__device__ __forceinline__ uint32_t op_offset(uint32_t kr, uint32_t c) {
  return kr * 128u + (((c >> 3) ^ (kr & 7u)) << 4) + (c & 7u) * 2u;
}

// displacement gradient Hd = [x1 - x0, x2 - x0, x3 - x0] Dm^-1 from the four
// vertex rows x[a][i] of a displacement field
__device__ __forceinline__ void grad_of(const float (&x)[4][3], const float (&Dmi)[3][3],
                                        float (&H)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[i][j] = (x[1][i] - x[0][i]) * Dmi[0][j] + (x[2][i] - x[0][i]) * Dmi[1][j] +
                (x[3][i] - x[0][i]) * Dmi[2][j];
}

// Element math of tet e into its record (zeros past the last tet) and the
// energies at u and at the KTRIAL trial fields.  tv: the tet's vertex
// indices (loaded a unit ahead); every other load of the
// tet (inverse rest edges, weight, the vertex rows of u and of the trial
// fields) is issued together, and the trial energies come first so that
// their registers are free before the eigen-decompositions
__device__ __forceinline__ void tet_record(const ElemArgs& ea, const float* __restrict__ u,
                                           const float* __restrict__ ut, int e, int4 tv,
                                           float* rec, float mu, float lam, float oma,
                                           FAcc& eacc, FAcc& eabs, FAcc (&etr)[KTRIAL],
                                           FAcc (&atr)[KTRIAL]) {
  float4* r4 = reinterpret_cast<float4*>(rec);
  if (e >= ea.S) {
#pragma unroll
    for (int k = 0; k < RW / 4; ++k) r4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
  float Dmi[3][3], wv, H[3][3];
  float xu[4][3], xt[KTRIAL][4][3];
  {
    const float* dm = static_cast<const float*>(ea.dminv);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) Dmi[a][c] = dm[(3 * a + c) * ea.S + e];
    wv = static_cast<const float*>(ea.wv)[e];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xu[a][i] = u[3 * vv[a] + i];
#pragma unroll
        for (int j = 0; j < KTRIAL; ++j) xt[j][a][i] = ut[(size_t)j * ea.n + 3 * vv[a] + i];
      }
  }
  // trial energies of the line search at this tet
#pragma unroll
  for (int j = 0; j < KTRIAL; ++j) {
    float Ht[3][3];
    grad_of(xt[j], Dmi, Ht);
    Invariants<float> it;
    invariants<float>(Ht, it);
    const float pt = wv * snh_psi<float>(it, mu, lam, oma);
    facc_add(etr[j], pt);
    facc_add(atr[j], fabsf(pt));
  }
  grad_of(xu, Dmi, H);
  Invariants<float> iv;
  invariants<float>(H, iv);
  const float pe = wv * snh_psi<float>(iv, mu, lam, oma);
  facc_add(eacc, pe);
  facc_add(eabs, fabsf(pe));
  float w[RW];
  w[R_V + 0] = __int_as_float(tv.x);
  w[R_V + 1] = __int_as_float(tv.y);
  w[R_V + 2] = __int_as_float(tv.z);
  w[R_V + 3] = __int_as_float(tv.w);
#pragma unroll
  for (int k = 0; k < RW; ++k)
    if (k >= 4) w[k] = 0.f;  // pads (the groups below overwrite their words)
  {
    const float Ic = iv.Ic3 + 3.f;
    const float dl = iv.Ic3 / (4.f * (Ic + 1.f));
    const float lJ = lam * iv.Jm1;
    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float Fij = H[i][j] + (i == j ? 1.f : 0.f);
        P[i][j] = wv * (mu * dl * Fij + lJ * iv.cof[i][j] +
                        0.75f * mu * (H[i][j] + H[j][i] - (i == j ? iv.trH : 0.f) - iv.cofH[i][j]));
      }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        w[R_GE + 3 * a + i] = P[i][0] * Dmi[a][0] + P[i][1] * Dmi[a][1] + P[i][2] * Dmi[a][2];
  }
  // eigensystem of the second derivative (the header of element.cu derives it)
  {
    const float Ic = iv.Ic3 + 3.f;
    const float c1 = mu * Ic / (Ic + 1.f);                  // 2 Psi_2
    const float c2 = 2.f * mu / ((Ic + 1.f) * (Ic + 1.f));  // 4 Psi_22
    const float c3 = lam * (iv.Jm1 + oma);                  // Psi_3 = lam (J - a)
    float F[3][3], U[3][3], V[3][3], sg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? 1.f : 0.f);
    svd3<float, true>(F, U, sg, V);
    float As[3][3], Aq[3][3];
    const float pi3[3] = {sg[1] * sg[2], sg[0] * sg[2], sg[0] * sg[1]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        As[i][j] = c2 * sg[i] * sg[j] + lam * pi3[i] * pi3[j] + (i == j ? c1 : c3 * sg[3 - i - j]);
    jacobi3<float, true>(As, Aq);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float sc = sqrtf(wv * (As[m][m] > 0.f ? As[m][m] : 0.f));
#pragma unroll
      for (int i = 0; i < 3; ++i) w[R_AS + 3 * m + i] = sc * Aq[i][m];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float lt = c1 + c3 * sg[i], lf = c1 - c3 * sg[i];
      w[R_TF + i] = sqrtf(0.5f * wv * (lt > 0.f ? lt : 0.f));
      w[R_TF + 3 + i] = sqrtf(0.5f * wv * (lf > 0.f ? lf : 0.f));
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int i = 0; i < 3; ++i) w[R_UT + 3 * p + i] = U[i][p];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        w[R_Y + 3 * a + q] = Dmi[a][0] * V[0][q] + Dmi[a][1] * V[1][q] + Dmi[a][2] * V[2][q];
  }
#pragma unroll
  for (int k = 0; k < RW / 4; ++k) r4[k] = make_float4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

// Column build of one tet (record rec) for the four columns c0 .. c0 + 3:
// C_e rows into the operand (K rows 9 lt .. 9 lt + 8), gradient terms into gp.
// The twelve J rows of a tet for a thread's four columns, staged in shared
// memory by asynchronous copies issued one tet ahead.  Component-major: slot
// k = 3 a + i (row 3 v_a + i) of thread tb is stg[k * NBT + tb], so the 16-byte
// accesses of a warp fall on consecutive addresses (no bank conflicts).
__device__ __forceinline__ void stage_rows(float4* stg, const float* __restrict__ J, int r, int c0,
                                           int4 vv) {
  const int v[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const uint32_t dst = smem_u32(stg + (3 * a + i) * NBT);
      const float* src = J + (size_t)(3 * v[a] + i) * r + c0;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void staged_wait() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// The column build works on column pairs: Blackwell's paired FP32
// instructions (__ffma2_rn, __fmul2_rn, __fadd2_rn: two independent IEEE
// operations per instruction) halve the instruction count of the
// per-(tet, column) arithmetic, which together with the element math fills
// the issue slots of the SM.
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }

// dJ_a = J_{a+1} - J_0 (a = 0..2) for the four columns from the staged rows,
// as two column pairs: d[a][i][0] = columns c0, c0 + 1; d[a][i][1] = c0 + 2, c0 + 3
__device__ __forceinline__ void staged_diffs(const float4* stg, float2 (&d)[3][3][2]) {
  float4 x[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) x[k] = stg[k * NBT];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float4 p = x[3 * (a + 1) + i], q = x[i];
      d[a][i][0] = __fadd2_rn(make_float2(p.x, p.y), make_float2(-q.x, -q.y));
      d[a][i][1] = __fadd2_rn(make_float2(p.z, p.w), make_float2(-q.z, -q.w));
    }
}

// Column build of one tet (record rec) from dJ (staged_diffs) for the four
// columns c0 .. c0 + 3: C_e rows into the operand (K rows 9 lt .. 9 lt + 8),
// gradient terms into gp (two column pairs).
__device__ __forceinline__ void build_tet(const float* rec, const float2 (&d)[3][3][2], int c0,
                                          uint8_t* op, int lt, float2 (&gp)[2],
                                          float2 (&ga)[2]) {
  const float4* r4 = reinterpret_cast<const float4*>(rec);
  // gradient: sum_a ge_a . dJ_a
  {
    float ge[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 x = r4[R_GE / 4 + k];
      ge[4 * k] = x.x; ge[4 * k + 1] = x.y; ge[4 * k + 2] = x.z; ge[4 * k + 3] = x.w;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 g2 = __fmul2_rn(bc2(ge[0]), d[0][0][h]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (a > 0 || i > 0) g2 = __ffma2_rn(bc2(ge[3 * a + i]), d[a][i][h], g2);
      gp[h] = __fadd2_rn(gp[h], g2);
      ga[h] = __fadd2_rn(ga[h], make_float2(fabsf(g2.x), fabsf(g2.y)));
    }
  }
  // R = sum_a (U^T dJ_a) y_a^T
  float2 R[3][3][2];
  {
    float ut[12], y[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 x = r4[R_UT / 4 + k], z = r4[R_Y / 4 + k];
      ut[4 * k] = x.x; ut[4 * k + 1] = x.y; ut[4 * k + 2] = x.z; ut[4 * k + 3] = x.w;
      y[4 * k] = z.x; y[4 * k + 1] = z.y; y[4 * k + 2] = z.z; y[4 * k + 3] = z.w;
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      float2 wa[3][2];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 w = __fmul2_rn(bc2(ut[3 * p]), d[a][0][h]);
          w = __ffma2_rn(bc2(ut[3 * p + 1]), d[a][1][h], w);
          wa[a][h] = __ffma2_rn(bc2(ut[3 * p + 2]), d[a][2][h], w);
        }
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float2 v = __fmul2_rn(wa[0][h], bc2(y[q]));
          v = __ffma2_rn(wa[1][h], bc2(y[3 + q]), v);
          R[p][q][h] = __ffma2_rn(wa[2][h], bc2(y[6 + q]), v);
        }
    }
  }
  float as[12], tf[8];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 x = r4[R_AS / 4 + k];
    as[4 * k] = x.x; as[4 * k + 1] = x.y; as[4 * k + 2] = x.z; as[4 * k + 3] = x.w;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 x = r4[R_TF / 4 + k];
    tf[4 * k] = x.x; tf[4 * k + 1] = x.y; tf[4 * k + 2] = x.z; tf[4 * k + 3] = x.w;
  }
  // the nine eigen-coordinates, stored as K rows 9 lt + m
  const uint32_t kr0 = 9u * (uint32_t)lt;
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    float2 cv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (m < 3) {
        float2 v = __fmul2_rn(bc2(as[3 * m]), R[0][0][h]);
        v = __ffma2_rn(bc2(as[3 * m + 1]), R[1][1][h], v);
        cv[h] = __ffma2_rn(bc2(as[3 * m + 2]), R[2][2][h], v);
      } else {
        const int i = (m - 3) % 3, j = (i + 1) % 3, l = (i + 2) % 3;
        const float2 o = R[l][j][h];
        const float2 sum = m < 6 ? __fadd2_rn(R[j][l][h], make_float2(-o.x, -o.y))
                                 : __fadd2_rn(R[j][l][h], o);
        cv[h] = __fmul2_rn(bc2(tf[m - 3]), sum);
      }
    }
    const __nv_bfloat162 lo = __floats2bfloat162_rn(cv[0].x, cv[0].y);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(cv[1].x, cv[1].y);
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t*>(&lo);
    v.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(op + op_offset(kr0 + m, (uint32_t)c0)) = v;
  }
}

__global__ void __launch_bounds__(NT, 1)
    element_ws_kernel(ElemArgs ea, const float* __restrict__ u, const float* __restrict__ J,
                      const float* __restrict__ ut, double* __restrict__ part, int part_stride,
                      int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t cfull[2], cempty[2], ofull[NOB], oempty[NOB], fin;
  __shared__ uint32_t tbase_s;
  __shared__ FAcc red[NT / 32][2 + 2 * KTRIAL];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  float* recs = reinterpret_cast<float*>(sb + NOB * BUF);  // [2][UNIT][RW]
  const int r = ea.r, S = ea.S;
  const int Ng = (r + 15) / 16 * 16;
  const uint32_t idesc = idesc_bf16(GROWS, Ng) | (1u << 15) | (1u << 16);  // both MN-major
  const float mu = (float)ea.mu, lam = (float)ea.lam;
  const float oma = (float)(-0.75 * ea.mu / ea.lam);
  const int nunits = (S + UNIT - 1) / UNIT;
  // columns >= r of the operands are never written: zero both buffers once
  for (int i = t; i < (int)(NOB * BUF / 16); i += NT)
    reinterpret_cast<uint4*>(sb)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tmem_alloc(&tbase_s, 64);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(&cfull[0], 32 * NPW);
    mbar_init(&cfull[1], 32 * NPW);
    mbar_init(&cempty[0], NBT);
    mbar_init(&cempty[1], NBT);
    for (int i = 0; i < NOB; ++i) {
      mbar_init(&ofull[i], NBT);
      mbar_init(&oempty[i], 1);
    }
    mbar_init(&fin, 1);
    fence_barrier_init();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  pdl_wait();  // u, J and the trial displacements come from the output layer

  FAcc eacc, eabs, etr[KTRIAL], atr[KTRIAL];
  FAcc gacc[4];
  float2 gabs[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  bool alive = true;
  const int tb = t - 32 * NPW;  // column-build thread index
  const int Q = r >> 2;         // column quads (r is a multiple of 4)
  const int slots = min(NBT / Q, CH);  // tets of a chunk in parallel (== CH for r <= 64)
  const int slot = tb / Q, quad = tb - slot * Q;

  if (warp < NPW) {
    // ---------------- element math: one tet per thread per unit
    int li = 0;
    const int4 z4 = make_int4(0, 0, 0, 0);
    int4 tv = blockIdx.x * UNIT + t < S ? ea.tets[blockIdx.x * UNIT + t] : z4;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x, ++li) {
      const int b = li & 1;
      // the next unit's tet indices, a unit ahead
      const int en = (unit + gridDim.x) * UNIT + t;
      const int4 tv_next = (unit + (int)gridDim.x < nunits && en < S) ? ea.tets[en] : z4;
      if (li >= 2) {
        const bool ok = wait_bar(&cempty[b], ((li >> 1) - 1) & 1, err, 4);
        if (!__all_sync(0xffffffffu, ok)) {
          alive = false;
          break;
        }
      }
      tet_record(ea, u, ut, unit * UNIT + t, tv, recs + ((size_t)b * UNIT + t) * RW, mu, lam,
                 oma, eacc, eabs, etr, atr);
      mbar_arrive(&cfull[b]);
      tv = tv_next;
    }
  } else if (warp < MMAW) {
    // ---------------- column build: chunks of CH tets, four columns per thread;
    // a thread takes tet `slot` of every chunk (slots == CH) and stages the J
    // rows of its next tet while it builds the current one
    const int c0 = 4 * quad;
    const bool act = slot < slots && c0 < r;
    float4* stg = reinterpret_cast<float4*>(sb + NOB * BUF + 2 * UNIT * RW * 4) + tb;
    const int my_units = (nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int ntet = my_units * NCH;  // this thread's tets, one per chunk
    const int4 z4 = make_int4(0, 0, 0, 0);
    auto vids = [&](int idx) {  // vertex ids of the thread's idx-th tet (0 past the end)
      if (idx >= ntet) return z4;
      const int e = (blockIdx.x + (idx / NCH) * (int)gridDim.x) * UNIT + (idx % NCH) * CH + slot;
      return e < S ? ea.tets[e] : z4;
    };
    int4 vnext = z4;
    if (act) {
      stage_rows(stg, J, r, c0, vids(0));
      vnext = vids(1);
    }
    int li = 0, q = 0;
    for (int unit = blockIdx.x; unit < nunits && alive; unit += gridDim.x, ++li) {
      const int b = li & 1;
      const bool okc = wait_bar(&cfull[b], (li >> 1) & 1, err, 8);
      if (!__all_sync(0xffffffffu, okc)) {
        alive = false;
        break;
      }
      const float* urec = recs + (size_t)b * UNIT * RW;
      for (int h = 0; h < NCH; ++h, ++q) {
        const int ob = q % NOB;
        if (q >= NOB) {  // the MMAs of chunk q - NOB have read the buffer
          const bool oko = wait_bar(&oempty[ob], ((q / NOB) - 1) & 1, err, 16);
          if (!__all_sync(0xffffffffu, oko)) {
            alive = false;
            break;
          }
        }
        if (act) {
          staged_wait();
          float2 d[3][3][2];
          staged_diffs(stg, d);  // consumes every staged row before it is refilled
          if (q + 1 < ntet) stage_rows(stg, J, r, c0, vnext);
          vnext = vids(q + 2);
          float2 gp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
          build_tet(urec + (size_t)(h * CH + slot) * RW, d, c0, sb + ob * BUF, slot, gp, gabs);
          facc_add(gacc[0], gp[0].x);
          facc_add(gacc[1], gp[0].y);
          facc_add(gacc[2], gp[1].x);
          facc_add(gacc[3], gp[1].y);
        }
        fence_proxy_async_smem();  // operand writes -> the MMAs (async proxy)
        mbar_arrive(&ofull[ob]);
      }
      if (!alive) break;
      mbar_arrive(&cempty[b]);
    }
    if (act) staged_wait();  // no copy is left in flight
  } else if (lane == 0) {
    // ---------------- MMA issue, one chain per operand chunk
    const int nchunks = ((nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x) * NCH;
    for (int q = 0; q < nchunks; ++q) {
      const int ob = q % NOB;
      if (!wait_bar(&ofull[ob], (q / NOB) & 1, err, 32)) {
        alive = false;
        break;
      }
      tc_fence_after();
      const uint32_t opa = base + ob * BUF;
#pragma unroll 1
      for (int k = 0; k < NSTEP; ++k) {
        // K step k: 16 K rows = two 8-row atoms = 2048 bytes
        const uint64_t d = sdesc_mn128(opa + k * 2048u, 8192u, 1024u);
        mma_bf16(tbase, d, d, idesc, (q > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&oempty[ob]);
    }
    mma_commit(&fin);  // every MMA issued so far has completed
  }
  __syncwarp();
  const bool all_alive = __syncthreads_and(alive);
  // the last MMAs must finish before TMEM is read or the operands are reused
  const bool fok = wait_bar(&fin, 0, err, 2);
  const bool good = __syncthreads_and(fok) && all_alive;
  tc_fence_after();

  double* prow = part + (size_t)blockIdx.x * part_stride;
  // energies: warp shuffles, then the warps in a fixed order (double-float)
  {
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
  }
  // gradient partials of the column-build threads, then a fixed-order sum
  // over the slots (the operand buffers are free once `fin` has completed)
  FAcc* gred = reinterpret_cast<FAcc*>(sb);                 // [slots <= CH][64]
  float* ared = reinterpret_cast<float*>(sb + CH * 64 * 8);  // [slots <= CH][64]
  if (warp >= NPW && warp < MMAW && slot < slots && 4 * quad < r) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gred[slot * 64 + 4 * quad + k] = gacc[k];
      ared[slot * 64 + 4 * quad + k] = k < 2 ? (k == 0 ? gabs[0].x : gabs[0].y)
                                             : (k == 2 ? gabs[1].x : gabs[1].y);
    }
  }
  __syncthreads();
  if (t < 2 + 2 * KTRIAL) {
    FAcc sum;
    for (int w = 0; w < NT / 32; ++w) facc_merge(sum, red[w][t]);
    if (t < 2) prow[t] = facc_value(sum);
    else prow[nslots(r) + t - 2] = facc_value(sum);
  }
  if (t < r) {
    FAcc gs;
    double as = 0.0;
    for (int s2 = 0; s2 < slots; ++s2) {
      facc_merge(gs, gred[s2 * 64 + t]);
      as += (double)ared[s2 * 64 + t];
    }
    prow[slot_g(t)] = facc_value(gs);
    prow[slot_gabs(r, t)] = as;
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
          const int dd = d0 + j;
          if (dd >= c && dd < r)
            prow[slot_K(r) + c * r - (c * (c - 1)) / 2 + (dd - c)] =
                good ? (double)__uint_as_float(vv[j]) : 0.0;
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

}  // namespace tcws

bool element_ws_applies(int S, int r, bool bf16, int num_sms) {
  return bf16 && r >= 4 && r <= tcws::GROWS && r % 4 == 0 &&
         (long long)S >= (long long)tcws::UNIT * num_sms;
}

int element_ws_grid(int S, int num_sms) {
  const int units = (S + tcws::UNIT - 1) / tcws::UNIT;
  return std::max(1, std::min(units, num_sms));
}

cudaError_t launch_element_ws(const ElemArgs& ea, const float* u, const float* J, const float* ut,
                              double* part, int grid, int* err, cudaStream_t s) {
  if (ea.r > tcws::GROWS || ea.r % 4 != 0) return cudaErrorInvalidValue;
  constexpr size_t sm = tcws::smem_bytes();
  static bool set = false;
  if (!set) {
    cudaError_t e = cudaFuncSetAttribute(tcws::element_ws_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    set = true;
  }
  return launch_pdl(tcws::element_ws_kernel, dim3(grid), dim3(tcws::NT), sm, s, ea, u, J, ut,
                    part, nslots_total(ea.r), err);
}

}  // namespace lsn
