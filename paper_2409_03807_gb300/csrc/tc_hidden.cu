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
// The weights are static: at set-up every CTA's slice of W is split to hi /
// lo and laid out exactly as the MMA reads it (K-major, 128-byte swizzle), so
// a CTA loads its slice with one bulk copy, issued before it waits on the
// previous kernel.  The layer input arrives the same way: each layer's
// epilogue writes the next layer's input slices in that layout; the first
// layer reads the pass points (unit-major FP32) and splits them itself.  One
// thread issues the MMA chain (M = 128, N = C rounded up to 16) and the CTA
// reads its partial accumulator from TMEM into shared memory.  CTA rank j of
// the cluster then sums rows [j 128/KS, (j+1) 128/KS) over the KS partials
// through distributed shared memory in rank order (deterministic) and
// applies the ELU / tangent epilogue, writing the next layer's input, the
// unit-major columns when a CUDA-core kernel reads them, and, for the last
// hidden layer, the tensor-core output layer's packed B operand (BF16 hi /
// lo split, or FP32).  Every mbarrier wait is bounded by %globaltimer and
// reports through `err`.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"
#include "tc_internal.cuh"

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
  // slices of at most 128 (K blocks of 32): at least two CTAs per row tile
  // once K > 32, so that the epilogue of a tile is shared
  p.ks = K <= 32 ? 1 : std::max(2, std::min(8, (K + 127) / 128));
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

__device__ __forceinline__ float elu_f(float a) { return a > 0.f ? a : expm1f(a); }
__device__ __forceinline__ float elu_d(float a) { return a > 0.f ? 1.f : expf(a); }

// bytes of one CTA's W image (hi blocks, then lo blocks) and of one K slice
// of a layer's input image (hi, then lo)
__host__ __device__ inline uint32_t wimg_bytes(const Plan& p) {
  return 2u * (uint32_t)(p.kslice / KB) * TM * 128u;
}
__host__ __device__ inline uint32_t bimg_bytes(const Plan& p) {
  return 2u * (uint32_t)(p.kslice / KB) * (uint32_t)p.cp * 128u;
}

// Set-up: every CTA's slice of W (M x K, row-major FP32) as its hi / lo image.
__global__ void wimage_kernel(const float* __restrict__ W, int M, int K, int C,
                              uint8_t* __restrict__ img) {
  const Plan P = plan(K, C);
  const int tiles = (M + TM - 1) / TM;
  const long long total = (long long)tiles * P.ks * TM * P.kslice;
  const uint32_t half = (uint32_t)(P.kslice / KB) * TM * 128u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % P.kslice);
    const int row = (int)((i / P.kslice) % TM);
    const int cta = (int)(i / ((long long)P.kslice * TM));
    const int tile = cta / P.ks, rank = cta - tile * P.ks;
    const int m = tile * TM + row, kk = rank * P.kslice + k;
    const float v = (m < M && kk < K && k < P.kslice) ? W[(size_t)m * K + kk] : 0.f;
    uint8_t* base = img + (size_t)cta * wimg_bytes(P);
    put_split(base, base + half, kmaj_offset(row, k, TM), v);
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool bounded_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gtimer() - t0 > WAIT_NS) return false;
  return true;
}

// Bin: this layer's input image (nullptr: split Zin here, the first layer);
// Bnext: the next hidden layer's input image (or nullptr); Zout (or nullptr):
// the unit-major columns.
__global__ void __launch_bounds__(NT, 1)
    tc_hidden_kernel(const uint8_t* __restrict__ Wimg, const float* __restrict__ b, int M, int K,
                     const float* __restrict__ Zin, const uint8_t* __restrict__ Bin, int C,
                     int CPs, int nj, float* __restrict__ Zout, uint8_t* __restrict__ Bnext,
                     void* Bh, void* Bl, int bkind, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t wbar, bbar, mdone;
  __shared__ uint32_t tbase_s;
  const Plan P = plan(K, C);
  const Layout L = layout(P);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();      // K slice
  const int tile = blockIdx.x / P.ks;         // row tile
  const int m0 = tile * TM, k0 = rank * P.kslice;
  const int kn = max(0, min(P.kslice, K - k0));
  const int nkb = P.kslice / KB;
  if (warp == 0) {
    tmem_alloc(&tbase_s, 128);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(&wbar, 1);
    mbar_init(&bbar, 1);
    mbar_init(&mdone, 1);
    fence_barrier_init();
  }
  __syncthreads();
  // ---- the W slice: static, so loaded before the dependency wait
  if (t == 0) {
    const uint32_t wb = wimg_bytes(P);
    mbar_expect_tx(&wbar, wb);
    bulk_load(sb + L.a_hi, Wimg + (size_t)blockIdx.x * wb, wb, &wbar);
  }
  pdl_wait();  // the layer input comes from the previous kernel
  if (Bin) {
    if (t == 0) {
      const uint32_t bb = bimg_bytes(P);
      mbar_expect_tx(&bbar, bb);
      bulk_load(sb + L.b_hi, Bin + (size_t)rank * bb, bb, &bbar);
    }
  } else {
    // first layer: Zin rows k0 .. k0 + kn - 1, columns c < C, split here
    for (int k = warp; k < P.kslice; k += NT / 32)
      for (int c = lane; c < P.cp; c += 32) {
        const float v = (c < C && k < kn) ? Zin[(size_t)(k0 + k) * CPs + c] : 0.f;
        put_split(sb + L.b_hi, sb + L.b_lo, kmaj_offset(c, k, P.cp), v);
      }
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  bool ok = true;
  if (t == 0) {
    ok = bounded_wait(&wbar, 0) && (!Bin || bounded_wait(&bbar, 0));
    if (ok) {
      tc_fence_after();
      const uint32_t idesc = idesc_tf32(TM, P.cp);
      for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ao = kb * TM * 128u + ks * 32u, bo = kb * P.cp * 128u + ks * 32u;
          const uint64_t ah = sdesc_sw128(base + L.a_hi + ao), al = sdesc_sw128(base + L.a_lo + ao);
          const uint64_t bh = sdesc_sw128(base + L.b_hi + bo), bl = sdesc_sw128(base + L.b_lo + bo);
          mma_tf32(tbase, ah, bh, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tbase, ah, bl, idesc, 1u);
          mma_tf32(tbase, al, bh, idesc, 1u);
        }
    }
    mma_commit(&mdone);
  }
  // ---- wait for the MMAs (bounded), partial accumulator TMEM -> shared
  ok = __syncthreads_and(ok) && bounded_wait(&mdone, 0);
  if (!ok && lane == 0) atomicOr(err, 64);
  tc_fence_after();
  const int PS = P.cp + 1;
  float* part = reinterpret_cast<float*>(sb + L.part);  // [TM][PS]
  {
    const int q = warp & 3, h = warp >> 2;  // TMEM lane quadrant, column half
    const int row = 32 * q + lane;
    const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16);
    for (int c0 = 16 * h; c0 < P.cp; c0 += 32) {
      uint32_t v[16];
      tmem_ld16(ta + c0, v);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) part[row * PS + c0 + j] = ok ? __uint_as_float(v[j]) : 0.f;
    }
  }
  tc_fence_before();
  cl.sync();  // every partial of the cluster is in its CTA's shared memory
  // ---- rows [rank rpr, (rank + 1) rpr): sum of the KS partials in rank order
  const int rpr = TM / P.ks;
  float* red = reinterpret_cast<float*>(sb + L.red);  // [rpr][PS]
  for (int lr = warp; lr < rpr; lr += NT / 32)
    for (int c = lane; c < P.cp; c += 32) {
    const int off = (rank * rpr + lr) * PS + c;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = j < P.ks ? cl.map_shared_rank(part, j)[off] : 0.f;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < P.ks) acc += v[j];
    red[lr * PS + c] = acc;
  }
  __syncthreads();
  // ---- epilogue (rows fastest): ELU of the value and trial columns, ELU'
  // times the tangents
  const Plan PN = plan(M, C);  // the next layer's input slices (K = M)
  const uint32_t nb = bimg_bytes(PN), nhalf = nb / 2;
  for (int c = warp; c < C; c += NT / 32)
    for (int lr = lane; lr < rpr; lr += 32) {
    const int m = m0 + rank * rpr + lr;
    if (m >= M) continue;
    const float bm = b[m];
    const float a = red[lr * PS + c];
    const float v = (c == 0 || c >= nj) ? elu_f(a + bm) : elu_d(red[lr * PS] + bm) * a;
    if (Zout) Zout[(size_t)m * CPs + c] = v;
    if (Bnext) {
      const int rn = m / PN.kslice, kk = m - rn * PN.kslice;
      uint8_t* nbase = Bnext + (size_t)rn * nb;
      put_split(nbase, nbase + nhalf, kmaj_offset(c, kk, PN.cp), v);
    }
    if (bkind == 1) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(Bh)[(size_t)c * M + m] = hi;
      static_cast<__nv_bfloat16*>(Bl)[(size_t)c * M + m] = __float2bfloat16_rn(v - __bfloat162float(hi));
    } else if (bkind == 2) {
      static_cast<float*>(Bh)[(size_t)c * M + m] = v;
    }
  }
  cl.sync();  // the other CTAs have finished reading this CTA's partial
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, 128);
  }
}

}  // namespace tch
}  // namespace lsn

namespace lsn {

bool tc_hidden_applies(int M, int K, int C) {
  const tch::Plan P = tch::plan(K, C);
  return M >= 1 && K >= 1 && P.cp <= 256 && tch::layout(P).total + 1024 <= 227u * 1024u;
}

void TcHidden::release() {
  for (auto& L : layers) {
    if (L.wimg) cudaFree(L.wimg);
    if (L.bimg) cudaFree(L.bimg);
  }
  layers.clear();
}

cudaError_t TcHidden::setup(const std::vector<const float*>& W, const std::vector<int>& widths,
                            int C_, int nj_, cudaStream_t s) {
  release();
  C = C_;
  nj = nj_;
  const int nh = (int)widths.size() - 2;  // widths = r, H_1, ..., H_{L-1}, n
  for (int l = 0; l < nh; ++l)
    if (!tc_hidden_applies(widths[l + 1], widths[l], C)) return cudaErrorInvalidValue;
  layers.resize(nh);
  size_t smem = 0;
  for (int l = 0; l < nh; ++l) {
    Layer& Ly = layers[l];
    Ly.M = widths[l + 1];
    Ly.K = widths[l];
    const tch::Plan P = tch::plan(Ly.K, C);
    const size_t tiles = (size_t)(Ly.M + tch::TM - 1) / tch::TM;
    const size_t wbytes = tiles * P.ks * tch::wimg_bytes(P);
    cudaError_t e = cudaMalloc(&Ly.wimg, wbytes);
    if (e != cudaSuccess) return e;
    const long long items = (long long)tiles * P.ks * tch::TM * P.kslice;
    const int grid = (int)std::min<long long>((items + 255) / 256, 4096);
    tch::wimage_kernel<<<grid, 256, 0, s>>>(W[l], Ly.M, Ly.K, C, static_cast<uint8_t*>(Ly.wimg));
    if (l >= 1) {  // the input slices written by layer l - 1 (padding stays zero)
      const size_t bbytes = (size_t)P.ks * tch::bimg_bytes(P);
      e = cudaMalloc(&Ly.bimg, bbytes);
      if (e != cudaSuccess) return e;
      e = cudaMemsetAsync(Ly.bimg, 0, bbytes, s);
      if (e != cudaSuccess) return e;
    }
    smem = std::max(smem, (size_t)tch::layout(P).total + 1024);
  }
  cudaError_t e = cudaFuncSetAttribute(tch::tc_hidden_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t TcHidden::launch(int l, const float* b, const float* Zin, float* Zout, void* Bh,
                             void* Bl, int bkind, int* err, cudaStream_t s) const {
  const Layer& Ly = layers[l];
  const tch::Plan P = tch::plan(Ly.K, C);
  const size_t smem = tch::layout(P).total + 1024;
  const int tiles = (Ly.M + tch::TM - 1) / tch::TM;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles * P.ks);
  cfg.blockDim = dim3(tch::NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P.ks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  uint8_t* next = l + 1 < (int)layers.size() ? static_cast<uint8_t*>(layers[l + 1].bimg) : nullptr;
  return cudaLaunchKernelEx(&cfg, tch::tc_hidden_kernel, static_cast<const uint8_t*>(Ly.wimg), b,
                            Ly.M, Ly.K, Zin, static_cast<const uint8_t*>(Ly.bimg), C, zstride(C),
                            nj, Zout, next, Bh, Bl, bkind, err);
}

}  // namespace lsn
