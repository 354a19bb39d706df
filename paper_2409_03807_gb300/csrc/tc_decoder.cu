// Decoder output layer on the 5th-generation tensor cores (tcgen05): the
// BF16 and TF32 forms of the decoder + forward-mode Jacobian (Sec. 3.1 Eq. 2,
// evaluated forward as the paper's autodiff does, Sec. 5), with the terms
// that act on each DOF alone (inertia / gravity / ground) fused into the
// epilogue, as in the CUDA-core form (decoder.cu).
//
//   acc[m][c] = sum_k W_L[m][k] Y[k][c],  c < C = 1 + r + trials
//   u = s (acc_0 + b),  J_c = s acc_c   (constrained rows: target, zero row)
//   g += J^T gv,  K += (sqrt(kv) J)^T (sqrt(kv) J),  E += e(u)
//
// Operands.  A = W_L tiles of 128 rows, read by TMA with the 128-byte
// swizzle (BF16 copy of the weights, or the FP32 weights as TF32).  B = the
// last hidden layer's columns, packed K-major ([C][H]) by pack_kernel.  In
// the BF16 form the activations are split y = y_hi + y_lo into two BF16
// parts and both products accumulate into the same FP32 accumulator, so
// only the weights are rounded to BF16; the TF32 form rounds both to TF32.
//
// Pipeline (one CTA per SM, persistent over row tiles):
//   warp 0  TMA producer: W_L tile + B block per 128-byte K block, 4 stages
//   warp 1  MMA issuer: M = 128, N = Cp; TMEM accumulator double-buffered so
//           the epilogue of tile i overlaps the main loop of tile i + 1; it
//           also issues the inertia Gram MMA (M = 64) of the previous tile
//   warps 2-9 epilogue: one thread per row and column half, two warps per
//           TMEM lane quadrant (= warp % 4): warps 2-5 take the column chunks
//           below 32 (the value column and the first Jacobian columns),
//           warps 6-9 the rest (further Jacobian columns, trial points)
// Every mbarrier wait is bounded by wall time (globaltimer); a wait that
// runs out records an error code and the CTA stops issuing work.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "lsn_internal.cuh"
#include "pdl.cuh"
#include "tc_ptx.cuh"
#include "tc_internal.cuh"

namespace lsn {
namespace {

using namespace tc;

constexpr int TBM = 128;      // rows per tile
constexpr int TST = 4;        // pipeline stages
constexpr int TNT = 320;      // threads: producer, MMA, 8 epilogue warps
constexpr int NEW = 8;        // epilogue warps
constexpr int GM = 64;        // Gram accumulator rows (M = 64 layout)
constexpr uint32_t COL_ACC1 = 128, COL_GRAM = 256, TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// bounded wait; on time-out records `code` and returns false
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int* err, int code,
                                         unsigned long long limit_ns = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > limit_ns) {
      atomicOr(err, code);
      return false;
    }
  }
}

// The time-out path of wait_bar on an mbarrier that nothing arrives on (no
// bulk copy or MMA is issued, so nothing is left in flight when it returns).
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_bar(&bar, 0, err, 1, limit_ns);
}

__device__ __forceinline__ void epi_sync() {  // the 8 epilogue warps
  asm volatile("bar.sync 1, 256;\n" ::: "memory");
}
// barrier of the 8 epilogue warps that also returns the AND of `v` over them
__device__ __forceinline__ bool epi_sync_and(bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.and.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v)
      : "memory");
  return out != 0;
}

// Per-row energy, force and stiffness of the terms that act on each DOF
// alone, in FP32 (GB300's FP64 rate is a small fraction of FP32; the row
// values are summed in FP64 across rows)
__device__ __forceinline__ void row_terms_tc(const LastArgs& la, float inv_dt2, int comp,
                                             float mv, float ubar, float x0, float u, float& e,
                                             float& gv, float& kv) {
  if (inv_dt2 > 0.f) {
    const float diff = u - ubar;
    e = 0.5f * inv_dt2 * mv * diff * diff;
    gv = inv_dt2 * mv * diff;
    kv = inv_dt2 * mv;
  } else {
    e = -mv * (float)la.grav[comp] * u;
    gv = -mv * (float)la.grav[comp];
    kv = 0.f;
  }
  if (la.ground_k > 0.0 && comp == 2) {
    const float gk = (float)la.ground_k;
    const float pen = x0 + u - (float)la.ground_h;
    if (pen < 0.f) {
      e += 0.5f * gk * pen * pen;
      gv += gk * pen;
      kv += gk;
    }
  }
}

// Affine modes, in FP64 (a free body's displacement is large: its FP32
// rounding times the body's m / dt^2 would swamp the inertia force): the
// unscaled displacement M (X0_v - c) + t of DOF (v, comp) at the pass point
// of column `col`, and the unscaled constant Jacobian entry of affine
// coordinate k (0..8: M row-major, 9..11: t); both enter times the output
// scale.
__device__ __forceinline__ double affine_disp_tc(const LastArgs& la, int comp,
                                                 const double (&dX)[3], int col) {
  const double* Za = la.zaff;
  const int s = la.zcps;
  return Za[(3 * comp) * s + col] * dX[0] + Za[(3 * comp + 1) * s + col] * dX[1] +
         Za[(3 * comp + 2) * s + col] * dX[2] + Za[(9 + comp) * s + col];
}
// The row terms of row_terms_tc with the displacement difference taken in
// FP64 (rows of a body with affine modes)
__device__ __forceinline__ void row_terms_tc_aff(const LastArgs& la, float inv_dt2, int comp,
                                                 float mv, double ubar, double x0, double u,
                                                 float& e, float& gv, float& kv) {
  if (inv_dt2 > 0.f) {
    const float diff = (float)(u - ubar);
    e = 0.5f * inv_dt2 * mv * diff * diff;
    gv = inv_dt2 * mv * diff;
    kv = inv_dt2 * mv;
  } else {
    e = (float)(-(double)mv * la.grav[comp] * u);
    gv = -mv * (float)la.grav[comp];
    kv = 0.f;
  }
  if (la.ground_k > 0.0 && comp == 2) {
    const float gk = (float)la.ground_k;
    const float pen = (float)(x0 + u - la.ground_h);
    if (pen < 0.f) {
      e += 0.5f * gk * pen * pen;
      gv += gk * pen;
      kv += gk;
    }
  }
}
__device__ __forceinline__ double affine_jac(int comp, const double (&dX)[3], int k) {
  if (k < 9) return (k / 3 == comp) ? dX[k - 3 * comp] : 0.0;
  return (k - 9 == comp) ? 1.0 : 0.0;
}

// Z[k][c] (unit-major, column stride CPs) -> B operand rows c < Cp, K-major
template <bool BF>
__global__ void pack_kernel(const float* __restrict__ Z, int H, int C, int CPs, int Cp,
                            void* __restrict__ Bh, void* __restrict__ Bl) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Cp * H) return;
  const int c = e / H, k = e - c * H;
  const float v = c < C ? Z[(size_t)k * CPs + c] : 0.f;
  if (BF) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    static_cast<__nv_bfloat16*>(Bh)[e] = hi;
    static_cast<__nv_bfloat16*>(Bl)[e] = lo;
  } else {
    static_cast<float*>(Bh)[e] = v;
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, size_t count,
                               __nv_bfloat16* __restrict__ dst) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

struct TcSmem {  // byte offsets from the 1024-aligned base
  uint32_t stage_bytes, a_bytes, bh_off, bl_off, jt_off, jt_bytes, js_off, gv_off, gp_off,
      red_off, total;
};

// split: the Gram operand buffers hold a BF16 hi and lo part each
__host__ __device__ inline TcSmem tc_smem_layout(bool bf, int Cp, int r, bool split) {
  TcSmem L;
  L.a_bytes = TBM * 128;
  L.bh_off = L.a_bytes;
  L.bl_off = L.bh_off + Cp * 128;
  L.stage_bytes = L.a_bytes + Cp * 128 * (bf ? 2 : 1);
  L.jt_off = TST * L.stage_bytes;
  L.jt_bytes = GM * TBM * (bf ? 2 : 4) * (split ? 2 : 1);
  L.js_off = L.jt_off + 2 * L.jt_bytes;
  const uint32_t js_bytes = TBM * (r + 4) * 4;
  L.gv_off = (L.js_off + js_bytes + 15) & ~15u;
  L.gp_off = L.gv_off + TBM * 8;  // (gv stored as float; 8 bytes kept)
  L.red_off = L.gp_off + 2 * 4 * 64 * 4;  // g partials of 4 row groups (value, |term|)
  L.total = L.red_off + NEW * (2 + 2 * KTRIAL) * 8;
  return L;
}

// AFF: the body has affine modes (a separate instantiation, so the rows of
// the other workloads carry none of their FP64 registers)
template <bool BF, bool AFF>
__global__ void __launch_bounds__(TNT, 1)
    tc_last_kernel(const __grid_constant__ CUtensorMap mapW,
                   const __grid_constant__ CUtensorMap mapBh,
                   const __grid_constant__ CUtensorMap mapBl, const float* __restrict__ b, int M,
                   int H, int C, int Cp, int nj, float* __restrict__ u_out,
                   float* __restrict__ J_out, float* __restrict__ u_trial,
                   double* __restrict__ part, int part_stride, LastArgs la,
                   int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[TST], empty[TST], tfull[2], tempty[2], jfull[2], jempty[2], gdone;
  __shared__ uint32_t tbase_s;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const int r = la.r;
  // bodies with affine modes take the inertia Gram from a two-term BF16 split
  // of sqrt(kv) J (hi hi^T + hi lo^T + lo hi^T): the reduced Hessian of a free
  // body spans its whole m / dt^2 and the network curvatures, and one BF16
  // rounding of the operand leaves too little of the small ones
  constexpr bool SPLIT = BF && AFF;
  const TcSmem SL = tc_smem_layout(BF, Cp, r, SPLIT);
  constexpr int EPB = BF ? 64 : 32;  // K values per 128-byte block
  const int nkb = (H + EPB - 1) / EPB;
  const int ntiles = (M + TBM - 1) / TBM;
  const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int Ng = (r + 15) / 16 * 16;
  if (warp == 1) {
    tmem_alloc(&tbase_s, TMEM_COLS);
    tmem_relinquish();
  }
  if (t == 0) {
    for (int i = 0; i < TST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], NEW);
      mbar_init(&jfull[i], 1);
      mbar_init(&jempty[i], 1);
    }
    mbar_init(&gdone, 1);
    fence_barrier_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  pdl_wait();  // the packed columns and the row data come from earlier kernels

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&mapW);
      tma_prefetch_desc(&mapBh);
      if (BF) tma_prefetch_desc(&mapBl);
      int kc = 0;
      bool alive = true;
      for (int i = 0; i < my_tiles && alive; ++i) {
        const int m0 = (blockIdx.x + i * gridDim.x) * TBM;
        for (int kb = 0; kb < nkb; ++kb, ++kc) {
          const int st = kc % TST;
          const uint32_t ph = (kc / TST) & 1;
          if (!wait_bar(&empty[st], ph ^ 1, err, 1)) {
            alive = false;
            break;
          }
          uint8_t* stage = sb + st * SL.stage_bytes;
          mbar_expect_tx(&full[st], SL.stage_bytes);
          tma_load_2d(stage, &mapW, &full[st], kb * EPB, m0);
          tma_load_2d(stage + SL.bh_off, &mapBh, &full[st], kb * EPB, 0);
          if (BF) tma_load_2d(stage + SL.bl_off, &mapBl, &full[st], kb * EPB, 0);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idm = BF ? idesc_bf16(TBM, Cp) : idesc_tf32(TBM, Cp);
      const uint32_t idg = BF ? idesc_bf16(GM, Ng) : idesc_tf32(GM, Ng);
      const int nkbj = (TBM * (BF ? 2 : 4)) / 128;
      bool alive = true;
      auto gram = [&](int j) {
        const int jb = j & 1;
        if (!wait_bar(&jfull[jb], (j >> 1) & 1, err, 2)) {
          alive = false;
          return;
        }
        tc_fence_after();
        const uint32_t jt = base + SL.jt_off + jb * SL.jt_bytes;
        for (int kb = 0; kb < nkbj; ++kb)
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t d = sdesc_sw128(jt + kb * GM * 128 + ks * 32);
            const uint32_t acc = (j > 0 || kb > 0 || ks > 0) ? 1u : 0u;
            if (BF) {
              mma_bf16(tbase + COL_GRAM, d, d, idg, acc);
              if (SPLIT) {
                const uint64_t dl = sdesc_sw128(jt + SL.jt_bytes / 2 + kb * GM * 128 + ks * 32);
                mma_bf16(tbase + COL_GRAM, d, dl, idg, 1u);
                mma_bf16(tbase + COL_GRAM, dl, d, idg, 1u);
              }
            } else {
              mma_tf32(tbase + COL_GRAM, d, d, idg, acc);
            }
          }
        mma_commit(&jempty[jb]);
      };
      // the Gram MMA of tile i is issued once its epilogue has written the
      // operand: polled between the K blocks of tile i + 1, forced at the
      // end of that tile (the operand buffer is reused two tiles later)
      int pending = -1;
      auto poll_gram = [&](bool force) {
        if (pending < 0) return;
        const int jb = pending & 1;
        const uint32_t par = (pending >> 1) & 1;
        if (!force && !mbar_try_wait(&jfull[jb], par)) return;
        gram(pending);
        pending = -1;
      };
      int kc = 0;
      for (int i = 0; i < my_tiles && alive; ++i) {
        const int ab = i & 1;
        if (!wait_bar(&tempty[ab], ((i >> 1) & 1) ^ 1, err, 4)) {
          alive = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tbase + (ab ? COL_ACC1 : 0u);
        for (int kb = 0; kb < nkb; ++kb, ++kc) {
          const int st = kc % TST;
          const uint32_t ph = (kc / TST) & 1;
          if (!wait_bar(&full[st], ph, err, 8)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base + st * SL.stage_bytes;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t ad = sdesc_sw128(sa + ks * 32);
            const uint64_t bh = sdesc_sw128(sa + SL.bh_off + ks * 32);
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            if (BF) {
              mma_bf16(d, ad, bh, idm, acc);
              mma_bf16(d, ad, sdesc_sw128(sa + SL.bl_off + ks * 32), idm, 1u);
            } else {
              mma_tf32(d, ad, bh, idm, acc);
            }
          }
          mma_commit(&empty[st]);
          poll_gram(false);
        }
        if (!alive) break;
        mma_commit(&tfull[ab]);
        poll_gram(true);
        if (!alive) break;
        pending = i;
      }
      if (alive) poll_gram(true);
      mma_commit(&gdone);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue
    const int q = warp & 3;          // TMEM lane quadrant
    const int et = t - 64;           // 0..255 within the epilogue warps
    const int ew = et >> 5;          // epilogue warp 0..7
    const int h = ew >> 2;           // column half
    const int row = 32 * q + lane;   // row of the tile
    float* Js = reinterpret_cast<float*>(sb + SL.js_off);
    float* gvs = reinterpret_cast<float*>(sb + SL.gv_off);
    float* gp = reinterpret_cast<float*>(sb + SL.gp_off);
    const int JS = r + 1 - (r & 1);  // odd row pitch: the per-row stores hit 32 banks
    // column chunks of this warp: [0, 32) or [32, Cp)
    const int cbeg = h ? 32 : 0, cend = h ? Cp : min(Cp, 32);
    const float inv_dt2 = (float)*la.inv_dt2;
    const float scale = (float)la.scale;
    const int ntr = C - nj;
    // double-float (FP32 TwoSum) accumulators: no FP64 instructions per row
    FAcc eacc, eabs, etr[KTRIAL], atr[KTRIAL];
    FAcc gacc, gabs;  // column et of g (et < r)
    bool alive = true;
    for (int i = 0; i < my_tiles; ++i) {
      const int m0 = (blockIdx.x + i * gridDim.x) * TBM, m = m0 + row;
      const bool live = m < M;
      const int v = m / 3, comp = m - 3 * v;
      float mv = 0.f, ub = 0.f, x0 = 0.f, bm = 0.f;
      double dX[3] = {0.0, 0.0, 0.0};  // X0_v - c of the affine modes
      int slot = -1;
      if (live) {
        mv = (float)la.mass[v];
        ub = (float)la.ubar[m];
        x0 = (float)la.X0[m];
        slot = la.cslot[v];
        bm = b[m];
        if (AFF)
          for (int k = 0; k < 3; ++k) dX[k] = la.X0[3 * v + k] - la.acen[k];
      }
      const int ab = i & 1;
      // every decision to stop is taken by all 256 epilogue threads together
      alive = epi_sync_and(wait_bar(&tfull[ab], (i >> 1) & 1, err, 16));
      if (!alive) break;
      tc_fence_after();
      // columns in chunks of 16 straight from TMEM: column 0 (value) first,
      // then the Jacobian columns 1..r, then the trial columns
      const uint32_t ta = tbase + (ab ? COL_ACC1 : 0u) + ((uint32_t)(32 * q) << 16);
      const float cu = (live && slot >= 0) ? (float)la.cu[3 * slot + comp] : 0.f;
      const bool jlive = live && slot < 0;
      const int jb = i & 1;
      // the Gram operand buffer jb was last read by the Gram MMA of tile i - 2
      const bool jok = (i < 2) || wait_bar(&jempty[jb], ((i >> 1) & 1) ^ 1, err, 32);
      uint8_t* jt = sb + SL.jt_off + jb * SL.jt_bytes;
      float gv = 0.f, wk = 0.f;
      // the value column: row terms, and u and the energies (owner); sqrt(kv)
      // scales the Gram operand
      auto value_col = [&](float a, bool owner) {
        const bool aff = AFF && live && slot < 0;
        const double u0d =
            aff ? (double)(scale * (a + bm)) + la.scale * affine_disp_tc(la, comp, dX, 0)
                : 0.0;
        const float u0r = slot >= 0 ? cu : (aff ? (float)u0d : scale * (a + bm));
        float e = 0.f, kv = 0.f;
        if (live) {
          if (aff)
            row_terms_tc_aff(la, inv_dt2, comp, mv, la.ubar[m], la.X0[m], u0d, e, gv, kv);
          else
            row_terms_tc(la, inv_dt2, comp, mv, ub, x0, u0r, e, gv, kv);
          if (owner) {
            u_out[m] = u0r;
            facc_add(eacc, e);
            facc_add(eabs, fabsf(e));
          }
        }
        wk = sqrtf(kv);
      };
      if (cbeg > 0 && cbeg < cend) {  // the second half needs sqrt(kv) too
        uint32_t vv[16];
        tmem_ld16(ta, vv);
        tmem_ld_wait();
        value_col(__uint_as_float(vv[0]), false);
      }
      for (int c0 = cbeg; c0 < cend; c0 += 16) {
        uint32_t vv[16];
        tmem_ld16(ta + c0, vv);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          const float a = __uint_as_float(vv[j]);
          if (c == 0) {
            value_col(a, true);
          } else if (c <= r) {
            // Jacobian row into the staging tile; sqrt(kv) J row into the
            // Gram operand (K-major: operand row = column, K = tile row)
            const int cc = c - 1;
            const float jv = !jlive ? 0.f
                             : (AFF && cc >= la.aff0)
                                 ? (float)(la.scale * affine_jac(comp, dX, cc - la.aff0))
                                 : scale * a;
            Js[row * JS + cc] = jv;
            if (jok) {
              const float gval = wk * jv;
              if (BF) {
                const int kb = row >> 6, kin = row & 63;
                const uint32_t off = kb * GM * 128 + sw128_offset(cc, kin >> 3) + (kin & 7) * 2;
                const __nv_bfloat16 hi = __float2bfloat16_rn(gval);
                *reinterpret_cast<__nv_bfloat16*>(jt + off) = hi;
                if (SPLIT)
                  *reinterpret_cast<__nv_bfloat16*>(jt + SL.jt_bytes / 2 + off) =
                      __float2bfloat16_rn(gval - __bfloat162float(hi));
              } else {
                const int kb = row >> 5, kin = row & 31;
                *reinterpret_cast<float*>(jt + kb * GM * 128 + sw128_offset(cc, kin >> 2) +
                                          (kin & 3) * 4) = gval;
              }
            }
          } else if (c >= nj && c < C && live) {
            const int tj = c - nj;
            const bool aff = AFF && slot < 0;
            const double utd =
                aff ? (double)(scale * (a + bm)) + la.scale * affine_disp_tc(la, comp, dX, c)
                    : 0.0;
            const float utr = slot >= 0 ? cu : (aff ? (float)utd : scale * (a + bm));
            u_trial[(size_t)tj * M + m] = utr;
            float et2, g2, k2;
            if (aff)
              row_terms_tc_aff(la, inv_dt2, comp, mv, la.ubar[m], la.X0[m], utd, et2, g2, k2);
            else
              row_terms_tc(la, inv_dt2, comp, mv, ub, x0, utr, et2, g2, k2);
#pragma unroll
            for (int x = 0; x < KTRIAL; ++x)
              if (x == tj) {
                facc_add(etr[x], et2);
                facc_add(atr[x], fabsf(et2));
              }
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(&tempty[ab]);
      if (h == 0) gvs[row] = live ? gv : 0.f;
      fence_proxy_async_smem();
      alive = epi_sync_and(jok);
      if (et == 0 && alive) mbar_arrive(&jfull[jb]);
      // g partial (double) and the coalesced copy of the J tile
      const int rows = min(TBM, M - m0);
      {
        // FP32 within a group of 32 rows (four interleaved partial sums), the
        // four groups in fixed order, FP64 (double-float) across tiles
        const int c = et & 63, rg = et >> 6;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (c < r) {
          const int rend = min(rows, 32 * rg + 32);
          int rr = 32 * rg;
          for (; rr + 4 <= rend; rr += 4) {
            const float t0 = gvs[rr] * Js[rr * JS + c];
            const float t1 = gvs[rr + 1] * Js[(rr + 1) * JS + c];
            const float t2 = gvs[rr + 2] * Js[(rr + 2) * JS + c];
            const float t3 = gvs[rr + 3] * Js[(rr + 3) * JS + c];
            s0 += t0;
            s1 += t1;
            s2 += t2;
            s3 += t3;
            a0 += fabsf(t0);
            a1 += fabsf(t1);
            a2 += fabsf(t2);
            a3 += fabsf(t3);
          }
          for (; rr < rend; ++rr) {
            const float t0 = gvs[rr] * Js[rr * JS + c];
            s0 += t0;
            a0 += fabsf(t0);
          }
        }
        gp[rg * 64 + c] = (s0 + s1) + (s2 + s3);
        gp[256 + rg * 64 + c] = (a0 + a1) + (a2 + a3);
      }
      float* Jdst = J_out + (size_t)m0 * r;
      for (int rr = ew; rr < rows; rr += NEW)
        for (int c = lane; c < r; c += 32) Jdst[(size_t)rr * r + c] = Js[rr * JS + c];
      epi_sync();
      if (et < r) {
        facc_add(gacc, (gp[et] + gp[64 + et]) + (gp[128 + et] + gp[192 + et]));
        facc_add(gabs, (gp[256 + et] + gp[320 + et]) + (gp[384 + et] + gp[448 + et]));
      }
      if (!alive) break;
    }
    // energy sums: warp shuffles, then the 8 warps in fixed order
    FAcc vals[2 + 2 * KTRIAL];
    vals[0] = eacc;
    vals[1] = eabs;
#pragma unroll
    for (int j = 0; j < KTRIAL; ++j) {
      vals[2 + 2 * j] = etr[j];
      vals[3 + 2 * j] = atr[j];
    }
#pragma unroll
    for (int j = 0; j < 2 + 2 * KTRIAL; ++j)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) facc_merge(vals[j], facc_shfl_down(vals[j], o));
    FAcc* red = reinterpret_cast<FAcc*>(sb + SL.red_off);
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < 2 + 2 * KTRIAL; ++j) red[ew * (2 + 2 * KTRIAL) + j] = vals[j];
    epi_sync();
    double* prow = part + (size_t)blockIdx.x * part_stride;
    if (et < 2 + 2 * KTRIAL) {
      FAcc sum;
      for (int w = 0; w < NEW; ++w) facc_merge(sum, red[w * (2 + 2 * KTRIAL) + et]);
      const double v = facc_value(sum);
      const int tslot = nslots(r);
      if (et < 2) prow[et] = v;
      else prow[tslot + et - 2] = ((et - 2) / 2 < ntr) ? v : 0.0;
    }
    if (et < r) {
      prow[slot_g(et)] = facc_value(gacc);
      prow[slot_gabs(r, et)] = facc_value(gabs);
    }
    // inertia Gram (read by the first four epilogue warps): row c of the
    // M = 64 accumulator is TMEM lane 32 (c / 16) + c % 16, i.e. lanes 0-15
    // of quadrant c / 16
    const bool gok =
        h == 0 && __all_sync(0xffffffffu, alive && wait_bar(&gdone, 0, err, 64));
    tc_fence_after();
    if (gok) {
      const int c = 16 * q + lane;
      const uint32_t tg = tbase + COL_GRAM + ((uint32_t)(32 * q) << 16);
      for (int d0 = 0; d0 < Ng; d0 += 16) {
        uint32_t vv[16];
        tmem_ld16(tg + d0, vv);
        tmem_ld_wait();
        if (lane < 16 && c < r)
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int d = d0 + j;
            if (d >= c && d < r)
              prow[slot_K(r) + c * r - (c * (c - 1)) / 2 + (d - c)] =
                  (double)__uint_as_float(vv[j]);
          }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, TMEM_COLS);
  }
}

}  // namespace

cudaError_t bounded_wait_selftest(double seconds, int* code, cudaStream_t s) {
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)(seconds * 1e9), err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(code, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  return e;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* ptr, bool bf, int inner, int outer, int box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = bf ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)inner * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_outer};
  cuuint32_t es[2] = {1, 1};
  std::memset(map, 0, sizeof(*map));
  return fn(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t TcLast::setup(const float* W_fp32, int M_, int H_, int C_, int r_, bool bf16_,
                          int num_sms, cudaStream_t s, bool aff_) {
  release();
  aff = aff_;
  M = M_;
  H = H_;
  C = C_;
  r = r_;
  bf16 = bf16_;
  Cp = bf16 ? (C + 7) / 8 * 8 : (C + 15) / 16 * 16;
  if (bf16 && Cp % 16) Cp += 8;  // N multiple of 16 for M = 128
  // TMA: the row pitch H x element size must be a multiple of 16 bytes; K
  // blocks past H are zero-filled by the copy
  if (Cp > 96 || r > 64 || (H * (bf16 ? 2 : 4)) % 16 != 0) return cudaErrorInvalidValue;
  const int ntiles = (M + TBM - 1) / TBM;
  grid = std::max(1, std::min(ntiles, num_sms));
  const TcSmem L = tc_smem_layout(bf16, Cp, r, bf16 && aff);
  smem = L.total + 1024;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  const size_t wcount = (size_t)M * H;
  if (bf16) {
    e = cudaMalloc(&Wlow, wcount * 2);
    if (e != cudaSuccess) return e;
    to_bf16_kernel<<<1024, 256, 0, s>>>(W_fp32, wcount, static_cast<__nv_bfloat16*>(Wlow));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t bbytes = (size_t)Cp * H * (bf16 ? 2 : 4);
  e = cudaMalloc(&Bh, bbytes);
  if (e != cudaSuccess) return e;
  if (bf16) {
    e = cudaMalloc(&Bl, bbytes);
    if (e != cudaSuccess) return e;
  }
  // rows c >= C of the B operand stay zero (the hidden layer writes c < C)
  e = cudaMemsetAsync(Bh, 0, bbytes, s);
  if (e == cudaSuccess && bf16) e = cudaMemsetAsync(Bl, 0, bbytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&err, sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const void* wsrc = bf16 ? Wlow : static_cast<const void*>(W_fp32);
  if (!make_map(&mapW, wsrc, bf16, H, M, TBM) || !make_map(&mapBh, Bh, bf16, H, Cp, Cp) ||
      !make_map(&mapBl, bf16 ? Bl : Bh, bf16, H, Cp, Cp))
    return cudaErrorInvalidValue;
  const int sm_i = (int)smem;
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (bf16) {
    e = cudaFuncSetAttribute(tc_last_kernel<true, false>, at, sm_i);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_last_kernel<true, true>, at, sm_i);
  } else {
    e = cudaFuncSetAttribute(tc_last_kernel<false, false>, at, sm_i);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_last_kernel<false, true>, at, sm_i);
  }
  return e;
}

void TcLast::release() {
  if (Wlow) cudaFree(Wlow);
  if (Bh) cudaFree(Bh);
  if (Bl) cudaFree(Bl);
  if (err) cudaFree(err);
  Wlow = Bh = Bl = nullptr;
  err = nullptr;
}

void TcLast::launch(const float* Z, int CPs, const float* bias, int nj, float* u, float* J,
                    float* ut, double* part, int part_stride, const LastArgs& la,
                    cudaStream_t s, bool packed) const {
  const int n = Cp * H;
  // the instantiation (and its shared-memory layout) follows the setup flag
  if (bf16) {
    if (!packed) pack_kernel<true><<<(n + 255) / 256, 256, 0, s>>>(Z, H, C, CPs, Cp, Bh, Bl);
    launch_pdl(aff ? tc_last_kernel<true, true> : tc_last_kernel<true, false>, dim3(grid),
               dim3(TNT), smem, s, mapW, mapBh, mapBl, bias, M, H, C, Cp, nj, u, J, ut, part,
               part_stride, la, err);
  } else {
    if (!packed) pack_kernel<false><<<(n + 255) / 256, 256, 0, s>>>(Z, H, C, CPs, Cp, Bh, nullptr);
    launch_pdl(aff ? tc_last_kernel<false, true> : tc_last_kernel<false, false>, dim3(grid),
               dim3(TNT), smem, s, mapW, mapBh, mapBl, bias, M, H, C, Cp, nj, u, J, ut, part,
               part_stride, la, err);
  }
}

}  // namespace lsn
