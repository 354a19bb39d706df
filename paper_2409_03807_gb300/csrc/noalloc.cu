// Allocation-free evaluation of the reduced elastic system.
//
// Some callers cannot allocate device memory while they run: an engine that
// hands the solver a fixed memory budget up front, code running inside a
// memory pool or arena that must not grow, or a real-time loop in which a
// cudaMalloc / cudaFree (which may synchronise the device and can fail) is
// not acceptable.  For them this file offers lsn_element_system_noalloc, the
// per-tet energy / gradient / PSD-projected Hessian kernel fused with the
// J_e^T H_e J_e contraction (the same kernel and launch shape as the solver
// uses), whose per-CTA partial sums live in a fixed file-scope device array
// instead of a buffer from cudaMalloc.  The caller supplies every input and
// the output buffer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/lsn.h"
#include "lsn_internal.cuh"

namespace lsn {
namespace {

// 4 MiB of partial sums (LSN_NOALLOC_SCRATCH_DOUBLES doubles) on every GPU
// that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[LSN_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};  // device address, per device
int g_num_sms[kMaxDevices] = {0};
std::mutex g_scratch_mutex;  // guards the two tables above

// Host code must not use g_noalloc_scratch itself (on the host it names a
// stand-in, not device memory): resolve its device address once per device,
// with that device current.  Concurrent first calls from several host
// threads serialise on the mutex.
cudaError_t scratch_for_device(int dev, double** out, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  *sms = g_num_sms[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lsn

using namespace lsn;

extern "C" int lsn_element_system_noalloc(int S, int r, int n, const int32_t* tets,
                                          const float* dminv, const float* wvol,
                                          const float* u, const float* J, double mu,
                                          double lam, double* out, void* cuda_stream) {
  if (S < 1 || r < 1 || r > RMAX || n < 12 || n % 3 != 0 || !tets || !dminv || !wvol || !u ||
      !J || !out || !(mu > 0.0) || !(lam > 0.0))
    return LSN_ERR_ARG;
  // the kernel reads a tet's four indices as one 16-byte load and, when a J
  // row is a whole number of 16-byte chunks, copies J rows 16 bytes at a time
  auto misaligned = [](const void* p, uintptr_t a) {
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0;
  };
  if (misaligned(tets, 16) || misaligned(J, (r * sizeof(float)) % 16 == 0 ? 16 : 4) ||
      misaligned(dminv, 4) || misaligned(wvol, 4) || misaligned(u, 4) || misaligned(out, 8))
    return LSN_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LSN_ERR_CUDA;
  }
  double* scratch = nullptr;
  int sms = 1;
  if (scratch_for_device(dev, &scratch, &sms) != cudaSuccess) {
    cudaGetLastError();
    return LSN_ERR_CUDA;
  }
  // the same launch shape as the solver: gfull CTAs write one partial row
  // each, then a fixed-order reduction writes the sums after the rows
  int gfull = 0, genergy = 0;
  element_grids(S, r, sms, gfull, genergy);
  const int nst = nslots_total(r);
  if ((long long)(gfull + 1) * nst > LSN_NOALLOC_SCRATCH_DOUBLES) return LSN_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  ElemArgs ea;
  ea.S = S;
  ea.r = r;
  ea.n = n;
  ea.tets = reinterpret_cast<const int4*>(tets);
  ea.dminv = dminv;
  ea.wv = wvol;
  ea.mu = mu;
  ea.lam = lam;
  // every partial slot the reduction reads is written by this call's
  // element kernel first (the trial-energy slots are summed over no rows),
  // so nothing needs clearing between calls
  launch_element<float>(ea, u, J, nullptr, scratch, gfull, 0, s);
  double* sums = scratch + (size_t)gfull * nst;
  launch_reduce_partials(scratch, 0, scratch, gfull, gfull, nslots(r), nst, sums, s);
  cudaError_t e = cudaMemcpyAsync(out, sums, sizeof(double) * nslots(r), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSN_ERR_CUDA;
  }
  return LSN_OK;
}
