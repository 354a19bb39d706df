// Decoder hidden layers on the 5th-generation tensor cores (tcgen05), for
// the BF16 and TF32 forms: the layer h_l = ELU(W_l h_{l-1} + b_l) of the MLP
// subspace map (Sec. 3.1) together with its forward-mode tangents
// T_l = ELU'(a_l) (W_l T_{l-1}) and the line-search trial points, i.e. for
// the column block Y = [h, T, trial points] (C columns, unit-major Zin[k][c]):
//
//   acc = W_l Y,   out[m][0] = ELU(acc_0 + b),  out[m][c] = ELU'(acc_0 + b) acc_c
//   (tangent columns 1 <= c < nj),  out[m][c] = ELU(acc_c + b) (trial columns)
//
// The products keep FP32-grade accuracy: both operands are split into two
// TF32 parts, v = hi + lo (hi = tf32(v), lo = tf32(v - hi), 22 significant
// bits together), and hi*hi + hi*lo + lo*hi accumulate in FP32 in TMEM (the
// dropped lo*lo term is below 2^-22 relative), so the hidden layers of the
// tensor-core forms compute what the FP32 CUDA-core kernels compute.
//
// Work split.  A CTA owns a tile of 128 output rows and a slice of K (at
// most 128 values); the KS CTAs of one row tile form a thread-block cluster.
// Each CTA stages its slice of W (FP32 from global, split to hi / lo in a
// K-major 128-byte-swizzled layout) before waiting on the previous kernel,
// then its slice of Y, issues the MMA chain (M = 128, N = C rounded up to
// 16) and reads its partial accumulator from TMEM into shared memory.  CTA
// rank j of the cluster then sums rows [j 128/KS, (j+1) 128/KS) over the KS
// partials through distributed shared memory in rank order (deterministic)
// and applies the ELU / tangent epilogue, writing the layer's columns and,
// for the last hidden layer, the tensor-core output layer's packed B
// operand (BF16 hi / lo split, or FP32).  The one mbarrier wait (MMA
// completion) is bounded by %globaltimer and reports through `err`.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"

namespace lsn {
namespace tch {

namespace cg = cooperative_groups;
using namespace tc;

constexpr int TM = 128;          // rows per tile
constexpr int NT = 256;          // threads (two per TMEM lane)
constexpr int KB = 32;           // TF32 values per 128-byte K block
constexpr unsigned long long WAIT_NS = 2000000000ull;

struct Plan {
  int ks;      // CTAs per cluster (K slices)
  int kslice;  // K values per slice (multiple of KB)
  int cp;      // N: columns rounded up to 16
};

__host__ __device__ inline Plan plan(int K, int C) {
  Plan p;
  p.ks = K <= 128 ? 1 : std::min(8, (K + 127) / 128);
  const int per = (K + p.ks - 1) / p.ks;
  p.kslice = (per + KB - 1) / KB * KB;
  p.cp = (C + 15) / 16 * 16;
  return p;
}

struct Layout {  // byte offsets from the 1024-aligned base
  uint32_t a_hi, a_lo, b_hi, b_lo, part, red, total;
};

__host__ __device__ inline Layout layout(const Plan& p) {
  Layout L;
  const uint32_t ablk = TM * 128u, bblk = (uint32_t)p.cp * 128u;
  const uint32_t nkb = (uint32_t)(p.kslice / KB);
  L.a_hi = 0;
  L.a_lo = nkb * ablk;
  L.b_hi = 2 * nkb * ablk;
  L.b_lo = L.b_hi + nkb * bblk;
  const uint32_t ops = L.b_lo + nkb * bblk;
  // once the MMAs are done the partial accumulator (read by the other CTAs
  // of the cluster) reuses the W space and the reduced rows the Y space
  const uint32_t pbytes = TM * (uint32_t)(p.cp + 1) * 4u;
  L.part = 0;
  L.red = (std::max(L.b_hi, pbytes) + 15u) & ~15u;
  L.total = std::max(ops, L.red + (uint32_t)(TM / p.ks) * (uint32_t)(p.cp + 1) * 4u);
  return L;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// (row, k) of a K-major operand with R rows: block k / 32, 16-byte chunk
// (k % 32) / 4 swizzled by the row, word k % 4
__device__ __forceinline__ uint32_t kmaj_offset(uint32_t row, uint32_t k, uint32_t R) {
  return (k >> 5) * R * 128u + sw128_offset(row, (k & 31u) >> 2) + (k & 3u) * 4u;
}

__device__ __forceinline__ void put_split(uint8_t* hi, uint8_t* lo, uint32_t off, float v) {
  const float h = to_tf32(v);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = to_tf32(v - h);
}

}  // namespace tch
}  // namespace lsn
