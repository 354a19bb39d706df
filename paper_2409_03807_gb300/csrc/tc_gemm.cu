// Strided TF32 GEMM on the 5th-generation tensor cores (tcgen05), for the
// plain matrix products of the decoder trainer's forward and backward passes
// (Eq. 3, 9, 10 and their gradients) in the tensor-core forms:
//
//   C[m][n] = alpha sum_k A(m, k) B(k, n) + beta C[m][n],
//   A(m, k) = A[m sam + k sak],  B(k, n) = B[k sbk + n sbn],  C row-major (ldc),
//
// with FP32 inputs rounded to TF32 (to nearest) and FP32 accumulation (the
// products the trainer's TF32 form specifies), or rounded to BF16 (to nearest
// even; the trainer's BF16 form: BF16 weights and activations in every
// product, FP32 master weights).  A product of two BF16 values is exact in
// FP32, so the TF32 MMA gives on BF16-valued operands the products of a BF16
// MMA.  Any strides: both transposes occur in the backward pass.
//
// A CTA computes a 128 x BN tile of C (BN = 32, 64 or 128 from N) over a
// range of K.  Operand tiles of one 128-byte K block (32 values) are copied
// by all threads with 4-byte cp.async (zero-filled past the matrix edge) into
// a K-major 128-byte-swizzled layout, four stages deep; one thread issues the
// MMAs (M = 128, N = BN, four K steps of 8 per stage) into a TMEM accumulator
// and commits each stage to that stage's mbarrier, which the loaders wait on
// before refilling it.  When the output has few tiles and K is long (the
// n-row reductions of the backward pass), K is split over the grid's z
// dimension: every split writes its partial tile to a workspace and a second
// kernel sums the splits in a fixed order (no atomics: results do not depend
// on scheduling) and applies alpha and beta.  Every mbarrier wait is bounded
// by %globaltimer; a wait that runs out records an error flag the caller
// reads.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"

namespace lsn {
namespace tcg {

using namespace tc;

constexpr int BM = 128;      // rows of a C tile (MMA M)
constexpr int NT = 256;      // threads
constexpr int KB = 32;       // TF32 values per 128-byte K block (one stage)
constexpr int STAGES = 4;
constexpr unsigned long long WAIT_NS = 2000000000ull;

__host__ __device__ inline int tile_n(int N) { return N <= 32 ? 32 : (N <= 64 ? 64 : 128); }

__host__ __device__ inline size_t smem_bytes(int BN) {
  return (size_t)STAGES * (BM + BN) * 128 + 1024;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > WAIT_NS) return false;
  return true;
}

// 4-byte asynchronous copy; ok = false fills the destination with zero
__device__ __forceinline__ void cp4(uint32_t dst, const float* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
               "r"(ok ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
__device__ __forceinline__ float to_bf16(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// (row, k) of one 128-byte K block of a K-major operand: chunk k / 4 of the
// row, swizzled by the row, word k % 4
__device__ __forceinline__ uint32_t blk_offset(int row, int k) {
  return sw128_offset((uint32_t)row, (uint32_t)k >> 2) + ((uint32_t)k & 3u) * 4u;
}

// One C tile (blockIdx.y: 128 rows, blockIdx.x: BN columns) over the K range
// [blockIdx.z klen, (blockIdx.z + 1) klen).  ws == nullptr: C = alpha acc +
// beta C; otherwise the raw partial goes to ws[z][m][n].
__global__ void __launch_bounds__(NT, 1)
    gemm_kernel(int M, int N, int K, int klen, const float* __restrict__ A, long long sam,
                long long sak, const float* __restrict__ B, long long sbk, long long sbn,
                float alpha, float beta, float* __restrict__ C, long long ldc,
                float* __restrict__ ws, int* __restrict__ err, int opbf16) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t done[STAGES], fin;
  __shared__ uint32_t tbase_s;
  const int BN = tile_n(N);
  const uint32_t ncols = BN;  // TMEM columns (32, 64 or 128)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t stage_bytes = (uint32_t)(BM + BN) * 128u;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * klen, kend = min(K, kbeg + klen);
  const int nk = max(0, (kend - kbeg + KB - 1) / KB);
  if (warp == 0) {
    tmem_alloc(&tbase_s, ncols);
    tmem_relinquish();
  }
  if (t == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&done[i], 1);
    mbar_init(&fin, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  pdl_wait();
  // copies of K block kb into stage st: A rows m0.., B rows (columns of C) n0..
  auto load = [&](int kb, int st) {
    const uint32_t sa = base + st * stage_bytes, sbb = sa + BM * 128u;
    const int k0 = kbeg + kb * KB;
#pragma unroll 4
    for (int i = t; i < BM * KB; i += NT) {
      int row, k;
      if (sak == 1) { row = i >> 5; k = i & 31; }
      else { row = i & (BM - 1); k = i >> 7; }
      const int m = m0 + row, kk = k0 + k;
      const bool ok = m < M && kk < kend;
      cp4(sa + blk_offset(row, k), ok ? A + (size_t)m * sam + (size_t)kk * sak : A, ok);
    }
    for (int i = t; i < BN * KB; i += NT) {
      int nn, k;
      if (sbk == 1) { nn = i >> 5; k = i & 31; }
      else { nn = i % BN; k = i / BN; }
      const int n = n0 + nn, kk = k0 + k;
      const bool ok = n < N && kk < kend;
      cp4(sbb + blk_offset(nn, k), ok ? B + (size_t)kk * sbk + (size_t)n * sbn : B, ok);
    }
  };
  // the copies hand the MMA raw FP32 bits, which it would truncate to TF32:
  // each thread rounds the values it copied (to nearest: TF32, or BF16 in
  // the BF16 form) once they have landed
  auto round_stage = [&](int st) {
    uint8_t* sa = smem_raw + (base - raw) + st * stage_bytes;
    uint8_t* sbb = sa + BM * 128u;
#pragma unroll 4
    for (int i = t; i < BM * KB; i += NT) {
      int row, k;
      if (sak == 1) { row = i >> 5; k = i & 31; }
      else { row = i & (BM - 1); k = i >> 7; }
      float* x = reinterpret_cast<float*>(sa + blk_offset(row, k));
      *x = opbf16 ? to_bf16(*x) : to_tf32(*x);
    }
    for (int i = t; i < BN * KB; i += NT) {
      int nn, k;
      if (sbk == 1) { nn = i >> 5; k = i & 31; }
      else { nn = i % BN; k = i / BN; }
      float* x = reinterpret_cast<float*>(sbb + blk_offset(nn, k));
      *x = opbf16 ? to_bf16(*x) : to_tf32(*x);
    }
  };
  bool ok = true;
  for (int p = 0; p < STAGES - 1; ++p) {
    if (p < nk) load(p, p);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  const uint32_t idesc = idesc_tf32(BM, BN);
  for (int kb = 0; kb < nk; ++kb) {
    const int st = kb % STAGES;
    const int nxt = kb + STAGES - 1;
    if (nxt < nk) {
      // stage nxt % STAGES was last read by the MMAs of block kb - 1
      if (kb >= 1 && !bounded_wait(&done[(kb - 1) % STAGES], ((kb - 1) / STAGES) & 1)) ok = false;
      if (__syncthreads_and(ok)) load(nxt, nxt % STAGES);
      else ok = false;
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group %0;\n" ::"n"(STAGES - 1) : "memory");
    round_stage(st);
    fence_proxy_async_smem();
    __syncthreads();
    if (!ok) break;
    if (t == 0) {
      tc_fence_after();
      const uint32_t sa = base + st * stage_bytes, sbb = sa + BM * 128u;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_tf32(tbase, sdesc_sw128(sa + ks * 32), sdesc_sw128(sbb + ks * 32), idesc,
                 (kb > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&done[st]);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (t == 0) mma_commit(&fin);
  ok = __syncthreads_and(ok) && bounded_wait(&fin, 0);
  if (!ok && t == 0) atomicOr(err, 1);
  tc_fence_after();
  // ---- epilogue: warp w reads TMEM lanes 32 (w % 4).. and half of the columns
  const int q = warp & 3, h = warp >> 2;
  const int m = m0 + 32 * q + lane;
  const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16);
  for (int c0 = h * (BN / 2); c0 < (h + 1) * (BN / 2); c0 += 16) {
    uint32_t v[16];
    tmem_ld16(ta + c0, v);
    tmem_ld_wait();
    if (m < M && ok) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = n0 + c0 + j;
        if (n >= N) continue;
        const float acc = nk > 0 ? __uint_as_float(v[j]) : 0.f;
        if (ws) {
          ws[((size_t)blockIdx.z * M + m) * N + n] = acc;
        } else {
          float* c = C + (size_t)m * ldc + n;
          *c = alpha * acc + (beta != 0.f ? beta * *c : 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, ncols);
  }
}

// C[m][n] = alpha sum_z ws[z][m][n] + beta C[m][n], splits summed in order
__global__ void splitk_reduce_kernel(int M, int N, int S, const float* __restrict__ ws,
                                     float alpha, float beta, float* __restrict__ C,
                                     long long ldc) {
  pdl_wait();
  const size_t MN = (size_t)M * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < MN;
       i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int z = 0; z < S; ++z) acc += ws[z * MN + i];
    const int m = (int)(i / N), n = (int)(i - (size_t)m * N);
    float* c = C + (size_t)m * ldc + n;
    *c = alpha * acc + (beta != 0.f ? beta * *c : 0.f);
  }
}

}  // namespace tcg
}  // namespace lsn

namespace lsn {

size_t tc_gemm_workspace_floats(int M, int N, int K, int num_sms) {
  const int BN = tcg::tile_n(N);
  const long long tiles = (long long)((M + tcg::BM - 1) / tcg::BM) * ((N + BN - 1) / BN);
  const int kblocks = (K + tcg::KB - 1) / tcg::KB;
  // split K when the tiles leave most SMs idle and each split keeps >= 8 K blocks
  int splits = 1;
  if (tiles < num_sms) splits = (int)std::min<long long>(num_sms / tiles, kblocks / 8);
  splits = std::max(1, std::min(splits, 64));
  return splits > 1 ? (size_t)splits * M * N : 0;
}

cudaError_t tc_gemm_tf32(cudaStream_t s, int M, int N, int K, float alpha, const float* A,
                         long long sam, long long sak, const float* B, long long sbk,
                         long long sbn, float beta, float* C, long long ldc, float* ws,
                         size_t ws_floats, int num_sms, int* err, bool bf16_operands) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int BN = tcg::tile_n(N);
  const int tm = (M + tcg::BM - 1) / tcg::BM, tn = (N + BN - 1) / BN;
  const int kblocks = std::max(1, (K + tcg::KB - 1) / tcg::KB);
  int splits = 1;
  const size_t need = tc_gemm_workspace_floats(M, N, K, num_sms);
  if (need > 0 && ws && ws_floats >= need) splits = (int)(need / ((size_t)M * N));
  const int klen = ((kblocks + splits - 1) / splits) * tcg::KB;
  splits = std::max(1, (std::max(K, 1) + klen - 1) / klen);
  static size_t set = 0;
  const size_t smem = tcg::smem_bytes(128);
  if (set < smem) {
    cudaError_t e = cudaFuncSetAttribute(tcg::gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set = smem;
  }
  cudaError_t e = launch_pdl(tcg::gemm_kernel, dim3(tn, tm, splits), dim3(tcg::NT),
                             tcg::smem_bytes(BN), s, M, N, K, klen, A, sam, sak, B, sbk, sbn,
                             alpha, beta, C, ldc, splits > 1 ? ws : nullptr, err,
                             bf16_operands ? 1 : 0);
  if (e != cudaSuccess || splits == 1) return e;
  const size_t MN = (size_t)M * N;
  const int grid = (int)std::min<size_t>((MN + 255) / 256, 4 * (size_t)num_sms);
  return launch_pdl(tcg::splitk_reduce_kernel, dim3(grid), dim3(256), 0, s, M, N, splits,
                    (const float*)ws, alpha, beta, C, ldc);
}

}  // namespace lsn
