// Full-space implicit Euler / quasi-static solve of Eq. 1 over all n DOFs by
// projective Newton with Armijo backtracking (Sec. 3.1; the same PSD
// projection, line search and exit codes as the reduced solve): the
// comparison solve of the reduced method on the GPU.
//
// Newton directions come from Jacobi-preconditioned conjugate gradients on
// the projected Hessian sum_e A_e^T A_e (+ M / dt^2 in dynamics), applied
// matrix-free per tet (element.cu, fullsp::fs_hv_kernel); constrained DOFs
// are held at their targets and masked out of the system.  One CG iteration
// is four kernels (Hessian-vector product; mass term and p.y; the d / r / z
// update; the p update).  A batch of CG_BATCH iterations is one CUDA-graph
// launch; once CG has converged the remaining kernels of the batch return at
// once, and the host reads the convergence flag between batches, so the
// number of iterations is bounded by the host loop.  Scalar reductions are
// summed in a fixed order by every CTA that needs them (same data, same
// order, same value), so no grid-wide barrier is needed.  Element math runs
// in Real (FP64 or FP32); every vector and reduction is FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/lsn.h"
#include "lsn_internal.cuh"

namespace lsn {
namespace {

constexpr int VT = 256;       // threads of the vector kernels
constexpr int CG_BATCH = 16;  // CG iterations per graph launch

// CG scalars on the device.  rz and it are committed from rz_next / it_next
// by the first CUDA-core kernel of the next iteration, so that no kernel
// writes a value that its own CTAs read.
struct FsScal {
  double rz, rz_next;  // r . z of the current and of the next iteration
  double rr0, tol2;    // |r_0|^2 and rtol^2 |r_0|^2
  double inv_dt2;      // 1 / dt^2 of the current step (0: quasi-static)
  int it, it_next;     // completed CG iterations
  int done, bad;       // stopped; non-positive curvature or non-finite values
  int max_it, pad_;
};

struct FsFail {
  cudaError_t e;
};
inline void fck(cudaError_t e) {
  if (e != cudaSuccess) throw FsFail{e};
}
template <typename T>
T* fs_alloc(size_t count) {
  void* p = nullptr;
  fck(cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1)));
  return static_cast<T*>(p);
}

// NaN-propagating maximum.
__device__ __forceinline__ double nmax(double a, double b) { return (b > a || b != b) ? b : a; }

// CTA reduction of NV values (the first NSUM summed, the others maxima),
// stored at out[0 .. NV-1] by thread 0.  blockDim.x == VT.
template <int NV, int NSUM>
__device__ __forceinline__ void cta_store(double (&v)[NV], double* out) {
  __shared__ double sh[NV][VT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      const double w = __shfl_down_sync(0xffffffffu, v[j], o);
      v[j] = j >= NSUM ? nmax(v[j], w) : v[j] + w;
    }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sh[j][w] = v[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = sh[j][0];
      for (int k = 1; k < VT / 32; ++k)
        s = j >= NSUM ? nmax(s, sh[j][k]) : s + sh[j][k];
      out[j] = s;
    }
}

// Sum of part[k * stride + off] over k < count in a fixed order (lane 0 of
// warp 0), returned to every thread of the CTA: CTAs that call it on the
// same data get the same value.  blockDim.x >= 32.
__device__ double cta_sum(const double* __restrict__ part, int count, int stride, int off) {
  __shared__ double res;
  __syncthreads();  // res may still be read from a previous call
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int k = threadIdx.x; k < count; k += 32) s += part[(size_t)k * stride + off];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) res = s;
  }
  __syncthreads();
  return res;
}

// CTA-uniform read of the stop flag.
__device__ __forceinline__ bool cta_done(const FsScal* sc) {
  __shared__ int dn;
  if (threadIdx.x == 0) dn = *reinterpret_cast<const volatile int*>(&sc->done);
  __syncthreads();
  return dn != 0;
}

__device__ __forceinline__ double grav_k(int k, double g0, double g1, double g2) {
  return k == 0 ? g0 : (k == 1 ? g1 : g2);
}

// Start of a step: qold = q; dynamics: qbar = q + dt v + dt^2 g; the
// constrained DOFs of q are set to their targets X0 + cu.
__global__ void fs_begin_kernel(int n, double* __restrict__ q, const double* __restrict__ v,
                                const double* __restrict__ X0, const int* __restrict__ cslot,
                                const double* __restrict__ cu, double dt, double g0, double g1,
                                double g2, double* __restrict__ qbar,
                                double* __restrict__ qold) {
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    const int k = i % 3, s = cslot[i / 3];
    const double qi = q[i];
    qold[i] = qi;
    if (dt > 0.0) qbar[i] = qi + dt * v[i] + dt * dt * grav_k(k, g0, g1, g2);
    if (s >= 0) q[i] = X0[i] + cu[3 * s + k];
  }
}

template <typename Real>
__global__ void fs_prep_kernel(int n, const double* __restrict__ q,
                               const double* __restrict__ X0, Real* __restrict__ u,
                               double* __restrict__ g, double* __restrict__ gabs,
                               double* __restrict__ diag) {
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    u[i] = (Real)(q[i] - X0[i]);
    g[i] = 0.0;
    gabs[i] = 0.0;
    diag[i] = 0.0;
  }
}

// Vertex terms at q: inertia (dynamics) or gravity (quasi-static) energy and
// gradient, the mass part of the Jacobi diagonal, the constrained rows
// masked out.  Per CTA: sum of the terms, sum of |terms|, and over the free
// DOFs max |g_i| and max gabs_i (the element contributions' rounding scale).
__global__ void __launch_bounds__(VT) fs_vertex_kernel(
    int n, const double* __restrict__ q, const double* __restrict__ qbar,
    const double* __restrict__ mass, const int* __restrict__ cslot, double inv_dt2, double g0,
    double g1, double g2, double* __restrict__ g, const double* __restrict__ gabs,
    const double* __restrict__ diag, double* __restrict__ dinv, double* __restrict__ part) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    const int vtx = i / 3;
    const double m = mass[vtx];
    double e, gi = g[i], di = diag[i];
    if (inv_dt2 > 0.0) {
      const double dq = q[i] - qbar[i];
      e = 0.5 * m * inv_dt2 * dq * dq;
      gi += m * inv_dt2 * dq;
      di += m * inv_dt2;
    } else {
      const double gk = grav_k(i % 3, g0, g1, g2);
      e = -m * gk * q[i];
      gi -= m * gk;
    }
    const bool fr = cslot[vtx] < 0;
    g[i] = fr ? gi : 0.0;
    dinv[i] = fr ? (di > 0.0 ? 1.0 / di : 1.0) : 0.0;
    acc[0] += e;
    acc[1] += fabs(e);
    if (fr) {
      acc[2] = nmax(acc[2], fabs(gi));
      acc[3] = nmax(acc[3], gabs[i]);
    }
  }
  cta_store<4, 2>(acc, part + 4 * blockIdx.x);
}

// Vertex-term energy at q + alpha d (line-search trials).
__global__ void __launch_bounds__(VT) fs_vertex_energy_kernel(
    int n, const double* __restrict__ q, const double* __restrict__ d, double alpha,
    const double* __restrict__ qbar, const double* __restrict__ mass, double inv_dt2, double g0,
    double g1, double g2, double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    const double m = mass[i / 3], qt = q[i] + alpha * d[i];
    double e;
    if (inv_dt2 > 0.0) {
      const double dq = qt - qbar[i];
      e = 0.5 * m * inv_dt2 * dq * dq;
    } else {
      e = -m * grav_k(i % 3, g0, g1, g2) * qt;
    }
    acc[0] += e;
    acc[1] += fabs(e);
  }
  cta_store<2, 2>(acc, part + 2 * blockIdx.x);
}

// r = -g, z = r / diag, p = z, d = y = 0; per CTA r.z and r.r.
__global__ void __launch_bounds__(VT) fs_cg_init_kernel(
    int n, const double* __restrict__ g, const double* __restrict__ dinv, double* __restrict__ r,
    double* __restrict__ z, double* __restrict__ p, double* __restrict__ d,
    double* __restrict__ y, double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    const double ri = -g[i], zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    d[i] = 0.0;
    y[i] = 0.0;
    acc[0] += ri * zi;
    acc[1] += ri * ri;
  }
  cta_store<2, 2>(acc, part + 2 * blockIdx.x);
}

// One CTA of 32 threads: the CG start scalars.
__global__ void fs_cg_start_kernel(FsScal* sc, const double* __restrict__ part, int nb,
                                   double rtol, int max_it, double inv_dt2) {
  const double rz = cta_sum(part, nb, 2, 0);
  const double rr = cta_sum(part, nb, 2, 1);
  if (threadIdx.x == 0) {
    sc->rz = sc->rz_next = rz;
    sc->rr0 = rr;
    sc->tol2 = rtol * rtol * rr;
    sc->inv_dt2 = inv_dt2;
    sc->it = sc->it_next = 0;
    sc->max_it = max_it;
    const bool fin = isfinite(rr) && isfinite(rz);
    sc->bad = fin ? 0 : 1;
    sc->done = (fin && rr > 0.0 && max_it > 0) ? 0 : 1;
  }
}

// y = (Hproj p + M p / dt^2) on the free DOFs, 0 on the constrained ones;
// per CTA p.y.  Commits rz and it of the iteration.
__global__ void __launch_bounds__(VT) fs_cg_py_kernel(int n, FsScal* sc,
                                                      const double* __restrict__ p,
                                                      double* __restrict__ y,
                                                      const double* __restrict__ mass,
                                                      const int* __restrict__ cslot,
                                                      double* __restrict__ part) {
  if (cta_done(sc)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz = sc->rz_next;
    sc->it = sc->it_next;
  }
  const double f = sc->inv_dt2;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    const int vtx = i / 3;
    const double yi = cslot[vtx] < 0 ? y[i] + mass[vtx] * f * p[i] : 0.0;
    y[i] = yi;
    acc[0] += p[i] * yi;
  }
  cta_store<1, 1>(acc, part + blockIdx.x);
}

// alpha = r.z / p.y; d += alpha p, r -= alpha y, z = r / diag, y = 0 (for
// the next product); per CTA the new r.z and r.r.
__global__ void __launch_bounds__(VT) fs_cg_upd_kernel(
    int n, FsScal* sc, const double* __restrict__ ppart, int nb, const double* __restrict__ p,
    double* __restrict__ y, const double* __restrict__ dinv, double* __restrict__ d,
    double* __restrict__ r, double* __restrict__ z, double* __restrict__ part) {
  if (cta_done(sc)) return;
  const double pkp = cta_sum(ppart, nb, 1, 0);
  if (!(pkp > 0.0) || !isfinite(pkp)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->bad = 1;
      sc->done = 1;
    }
    return;
  }
  const double alpha = sc->rz / pkp;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) {
    d[i] += alpha * p[i];
    const double ri = r[i] - alpha * y[i];
    const double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    y[i] = 0.0;
    acc[0] += ri * zi;
    acc[1] += ri * ri;
  }
  cta_store<2, 2>(acc, part + 2 * blockIdx.x);
}

// Convergence test |r|^2 <= rtol^2 |r_0|^2 or the iteration cap; otherwise
// p = z + beta p with beta = (new r.z) / (r.z).
__global__ void __launch_bounds__(VT) fs_cg_p_kernel(int n, FsScal* sc,
                                                     const double* __restrict__ upart, int nb,
                                                     const double* __restrict__ z,
                                                     double* __restrict__ p) {
  if (cta_done(sc)) return;
  const double rzn = cta_sum(upart, nb, 2, 0);
  const double rr = cta_sum(upart, nb, 2, 1);
  const int itn = sc->it + 1;
  const bool fin = isfinite(rzn) && isfinite(rr);
  const bool stop = !fin || !(rr > sc->tol2) || itn >= sc->max_it;
  if (!stop) {
    const double beta = rzn / sc->rz;
    for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT)
      p[i] = z[i] + beta * p[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc->rz_next = rzn;
    sc->it_next = itn;
    if (!fin) sc->bad = 1;
    if (stop) sc->done = 1;
  }
}

__global__ void __launch_bounds__(VT) fs_dot_kernel(int n, const double* __restrict__ a,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ part) {
  double acc[1] = {0.0};
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) acc[0] += a[i] * b[i];
  cta_store<1, 1>(acc, part + blockIdx.x);
}

__global__ void fs_axpy_kernel(int n, double* __restrict__ q, const double* __restrict__ d,
                               double alpha) {
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT) q[i] += alpha * d[i];
}

__global__ void fs_velocity_kernel(int n, const double* __restrict__ q,
                                   const double* __restrict__ qold, double inv_dt,
                                   double* __restrict__ v) {
  for (int i = blockIdx.x * VT + threadIdx.x; i < n; i += gridDim.x * VT)
    v[i] = (q[i] - qold[i]) * inv_dt;
}

template <typename Real>
struct FullSpace : FullSpaceBase {
  int nv = 0, n = 0, ne = 0;
  int gv = 1, ge = 1, gh = 1;  // grids: vector kernels, evaluation kernel, per-tet kernels
  double *q = nullptr, *v = nullptr, *qold = nullptr, *qbar = nullptr, *g = nullptr,
         *gabs = nullptr, *diag = nullptr, *dinv = nullptr, *d = nullptr, *r = nullptr, *z = nullptr,
         *p = nullptr, *y = nullptr;
  double *pe = nullptr, *pv = nullptr, *pc = nullptr, *ppy = nullptr, *pen = nullptr,
         *pve = nullptr;
  Real *u = nullptr, *fac = nullptr, *rdminv = nullptr, *rwv = nullptr;
  int4* ctets = nullptr;
  FsScal* sc = nullptr;
  FsScal* hsc = nullptr;   // pinned mirror of sc
  double* hpart = nullptr; // pinned staging of the partial sums
  size_t hpart_n = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* cap_key[3] = {nullptr, nullptr, nullptr};  // pointers baked into the graph

  ~FullSpace() override {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    for (void* ptr : {(void*)q, (void*)v, (void*)qold, (void*)qbar, (void*)g, (void*)gabs,
                      (void*)diag,
                      (void*)dinv, (void*)d, (void*)r, (void*)z, (void*)p, (void*)y, (void*)pe,
                      (void*)pv, (void*)pc, (void*)ppy, (void*)pen, (void*)pve, (void*)u,
                      (void*)fac, (void*)rdminv, (void*)rwv, (void*)ctets, (void*)sc})
      if (ptr) cudaFree(ptr);
    if (hsc) cudaFreeHost(hsc);
    if (hpart) cudaFreeHost(hpart);
  }

  void init(const FsArgs& a, int num_sms, cudaStream_t s) {
    nv = a.nv;
    n = a.n;
    ne = a.ne;
    gv = std::max(1, std::min((n + VT - 1) / VT, 2 * num_sms));
    ge = fs_grid(ne, 64, num_sms);
    gh = fs_grid(ne, 128, num_sms);
    for (double** b : {&q, &v, &qold, &qbar, &g, &gabs, &diag, &dinv, &d, &r, &z, &p, &y})
      *b = fs_alloc<double>(n);
    pe = fs_alloc<double>(2 * ge);
    pv = fs_alloc<double>(4 * gv);
    pc = fs_alloc<double>(2 * gv);
    ppy = fs_alloc<double>(gv);
    pen = fs_alloc<double>(2 * gh);
    pve = fs_alloc<double>(2 * gv);
    u = fs_alloc<Real>(n);
    fac = fs_alloc<Real>((size_t)FS_NF * ne);
    rdminv = fs_alloc<Real>((size_t)9 * ne);
    rwv = fs_alloc<Real>(ne);
    ctets = fs_alloc<int4>(ne);
    sc = fs_alloc<FsScal>(1);
    fck(cudaMallocHost(&hsc, sizeof(FsScal)));
    hpart_n = (size_t)std::max(2 * ge, 2 * gh) + 4 * gv;
    fck(cudaMallocHost(&hpart, sizeof(double) * hpart_n));
    fck(cudaMemsetAsync(sc, 0, sizeof(FsScal), s));
    launch_gather_cubature<Real>(a.tets, a.dminv, a.vol, nullptr, nullptr, ne, ne, ctets,
                                 rdminv, rwv, s);
    fck(cudaMemcpyAsync(q, a.X0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    fck(cudaMemsetAsync(v, 0, sizeof(double) * n, s));
    fck(cudaStreamSynchronize(s));
    fck(cudaGetLastError());
  }

  double* positions() override { return q; }
  double* velocities() override { return v; }

  // One batch of CG_BATCH iterations captured once; rebuilt if a baked-in
  // pointer of the context (mass, constraint slots) changed.
  void ensure_graph(const FsArgs& a) {
    const void* key[3] = {a.mass, a.cslot, a.tets};
    if (exec && std::equal(key, key + 3, cap_key)) return;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    if (!cap) fck(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    fck(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < CG_BATCH; ++k) {
      launch_fs_hv<Real>(ctets, rdminv, ne, fac, p, y, &sc->done, gh, cap);
      fs_cg_py_kernel<<<gv, VT, 0, cap>>>(n, sc, p, y, a.mass, a.cslot, ppy);
      fs_cg_upd_kernel<<<gv, VT, 0, cap>>>(n, sc, ppy, gv, p, y, dinv, d, r, z, pc);
      fs_cg_p_kernel<<<gv, VT, 0, cap>>>(n, sc, pc, gv, z, p);
    }
    const cudaError_t launch_err = cudaGetLastError();
    cudaGraph_t gr = nullptr;
    cudaError_t err = cudaStreamEndCapture(cap, &gr);
    if (err == cudaSuccess) err = launch_err;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, gr, 0);
    if (err != cudaSuccess) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      if (gr) cudaGraphDestroy(gr);
      exec = nullptr;
      throw FsFail{err};
    }
    graph = gr;
    std::copy(key, key + 3, cap_key);
  }

  // Partial sums of the last evaluation kernels, copied to the host.
  void fetch(const double* src, size_t count, size_t at, cudaStream_t s) {
    fck(cudaMemcpyAsync(hpart + at, src, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  }

  cudaError_t step(const FsArgs& a, double dt, FsResult& res, cudaStream_t s) override {
    try {
      run(a, dt, res, s);
    } catch (const FsFail& f) {
      cudaGetLastError();
      return f.e;
    }
    return cudaSuccess;
  }

  void run(const FsArgs& a, double dt, FsResult& res, cudaStream_t s) {
    const bool fp32 = sizeof(Real) == 4;
    const double inv_dt2 = dt > 0.0 ? 1.0 / (dt * dt) : 0.0;
    const double g0 = a.grav[0], g1 = a.grav[1], g2 = a.grav[2];
    ElemArgs ea;
    ea.S = ne;
    ea.r = 0;
    ea.n = n;
    ea.tets = ctets;
    ea.dminv = rdminv;
    ea.wv = rwv;
    ea.mu = a.mu;
    ea.lam = a.lam;
    fs_begin_kernel<<<gv, VT, 0, s>>>(n, q, v, a.X0, a.cslot, a.cu, dt, g0, g1, g2, qbar, qold);
    fck(cudaGetLastError());
    int status = LSN_NOT_CONVERGED, it = 0, ls_total = 0, stall = 0;
    long long cg_total = 0;
    double E = 0.0, gi = 0.0, g_best = INFINITY;
    for (it = 0; it <= a.max_newton; ++it) {
      fs_prep_kernel<Real><<<gv, VT, 0, s>>>(n, q, a.X0, u, g, gabs, diag);
      launch_fs_elem<Real>(ea, u, fac, g, gabs, diag, pe, ge, s);
      fs_vertex_kernel<<<gv, VT, 0, s>>>(n, q, qbar, a.mass, a.cslot, inv_dt2, g0, g1, g2, g,
                                         gabs, diag, dinv, pv);
      fck(cudaGetLastError());
      fetch(pe, 2 * ge, 0, s);
      fetch(pv, 4 * gv, 2 * ge, s);
      fck(cudaStreamSynchronize(s));
      double Eabs = 0.0;  // sum of |element terms|: the rounding scale of the Real sums
      E = 0.0;
      gi = 0.0;
      double gabs_max = 0.0;
      for (int b = 0; b < ge; ++b) {
        E += hpart[2 * b];
        Eabs += hpart[2 * b + 1];
      }
      for (int b = 0; b < gv; ++b) {  // vertex terms (FP64)
        const double* pb = hpart + 2 * ge + 4 * b;
        E += pb[0];
        gi = (pb[2] > gi || pb[2] != pb[2]) ? pb[2] : gi;
        gabs_max = std::max(gabs_max, pb[3]);
      }
      if (!std::isfinite(E) || !std::isfinite(gi)) {
        status = LSN_ERR_NONFINITE;
        break;
      }
      if (gi < a.tol) {
        status = LSN_OK;
        break;
      }
      if (it == a.max_newton) {
        status = LSN_NOT_CONVERGED;
        break;
      }
      // FP32: ||g||_inf at the rounding level of the element sums (64 u
      // max_i sum |contributions to g_i|, as in the reduced solve) or near
      // tol, without a 10 % drop for 4 iterations, ends at the precision
      // floor; so do 16 iterations without that drop (the rounding of the
      // FP32 displacements also bounds how far g can fall)
      const bool at_floor =
          fp32 && (gi < 100.0 * a.tol || gi <= 64.0 * std::ldexp(1.0, -24) * gabs_max);
      if (fp32) {
        if (gi < 0.9 * g_best) {
          g_best = gi;
          stall = 0;
        } else if ((++stall >= 4 && at_floor) || stall >= 16) {
          status = LSN_PRECISION_FLOOR;
          break;
        }
      }
      // Newton direction by preconditioned CG
      fs_cg_init_kernel<<<gv, VT, 0, s>>>(n, g, dinv, r, z, p, d, y, pc);
      fs_cg_start_kernel<<<1, 32, 0, s>>>(sc, pc, gv, a.cg_rtol, a.max_cg, inv_dt2);
      fck(cudaGetLastError());
      ensure_graph(a);
      for (int b = 0; b * CG_BATCH < a.max_cg; ++b) {
        fck(cudaGraphLaunch(exec, s));
        fck(cudaMemcpyAsync(hsc, sc, sizeof(FsScal), cudaMemcpyDeviceToHost, s));
        fck(cudaStreamSynchronize(s));
        if (hsc->done) break;
      }
      cg_total += hsc->it_next;
      if (hsc->bad) {
        status = LSN_NOT_SPD;
        break;
      }
      fs_dot_kernel<<<gv, VT, 0, s>>>(n, g, d, pc);
      fetch(pc, gv, 0, s);
      fck(cudaStreamSynchronize(s));
      double gd = 0.0;
      for (int b = 0; b < gv; ++b) gd += hpart[b];
      // Armijo backtracking (halving)
      const double slack = fp32 ? 8.0 * std::ldexp(1.0, -24) * Eabs : 0.0;
      double alpha = 1.0;
      bool accepted = false;
      for (int t = 0; t < a.max_ls; ++t) {
        ++ls_total;
        launch_fs_energy<Real>(ctets, rdminv, rwv, ne, q, a.X0, d, alpha, a.mu, a.lam, pen, gh,
                               s);
        fs_vertex_energy_kernel<<<gv, VT, 0, s>>>(n, q, d, alpha, qbar, a.mass, inv_dt2, g0,
                                                  g1, g2, pve);
        fck(cudaGetLastError());
        fetch(pen, 2 * gh, 0, s);
        fetch(pve, 2 * gv, 2 * gh, s);
        fck(cudaStreamSynchronize(s));
        double Et = 0.0;
        for (int b = 0; b < gh; ++b) Et += hpart[2 * b];
        for (int b = 0; b < gv; ++b) Et += hpart[2 * gh + 2 * b];
        if (Et <= E + a.armijo_c * alpha * gd + slack) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!accepted) {
        status = at_floor ? LSN_PRECISION_FLOOR : LSN_LS_FAILED;
        break;
      }
      fs_axpy_kernel<<<gv, VT, 0, s>>>(n, q, d, alpha);
    }
    if (dt > 0.0 && status != LSN_ERR_NONFINITE)
      fs_velocity_kernel<<<gv, VT, 0, s>>>(n, q, qold, 1.0 / dt, v);
    fck(cudaGetLastError());
    fck(cudaStreamSynchronize(s));
    res.status = status;
    res.newton_iters = it;
    res.ls_trials = ls_total;
    res.cg_iters = cg_total;
    res.grad_inf = gi;
    res.energy = E;
  }
};

}  // namespace

cudaError_t make_fullspace(bool fp64, const FsArgs& a, int num_sms, cudaStream_t s,
                           FullSpaceBase** out) {
  *out = nullptr;
  FullSpaceBase* f = nullptr;
  try {
    if (fp64) {
      auto* x = new FullSpace<double>();
      f = x;
      x->init(a, num_sms, s);
    } else {
      auto* x = new FullSpace<float>();
      f = x;
      x->init(a, num_sms, s);
    }
  } catch (const FsFail& e) {
    cudaGetLastError();
    delete f;
    return e.e;
  }
  *out = f;
  return cudaSuccess;
}

}  // namespace lsn
