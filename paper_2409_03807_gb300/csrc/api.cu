// C ABI of liblsn (declared in include/lsn.h): context, set-up calls, and the
// host side of the Newton loop.  Every step of the computation runs in the
// kernels of mesh.cu, decoder.cu, element.cu and solve.cu; this file only
// owns buffers, uploads inputs and sequences launches on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/lsn.h"
#include "lsn_internal.cuh"
#include "tc_internal.cuh"
#include "train_internal.cuh"

using namespace lsn;

namespace {

struct CudaError {
  cudaError_t e;
};

inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaError{e};
}

template <typename T>
T* dalloc(size_t count) {
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw CudaError{e};
  }
  return static_cast<T*>(p);
}

inline void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy `bytes` from a host-or-device pointer into device memory
void upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  ck(cudaMemcpyAsync(dst, src, bytes,
                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}
void download(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  ck(cudaMemcpyAsync(dst, src, bytes,
                     is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

// CUDA-event timing of kernel classes (see lsn_set_profiling).
struct Profiler {
  cudaStream_t stream = nullptr;
  unsigned mask = 0;
  long long launches[LSN_K_COUNT] = {0};
  long long timed[LSN_K_COUNT] = {0};
  double ms[LSN_K_COUNT] = {0};
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int open_cls = -1;
  cudaEvent_t open_a = nullptr;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    ck(cudaEventCreate(&e));
    return e;
  }
  void begin(int cls, int count = 1) {
    launches[cls] += count;
    if (mask & (1u << cls)) {
      open_cls = cls;
      open_a = get();
      ck(cudaEventRecord(open_a, stream));
    }
  }
  void end(int cls) {
    if (open_cls == cls && open_a) {
      cudaEvent_t b = get();
      ck(cudaEventRecord(b, stream));
      pending.push_back({cls, open_a, b});
      open_cls = -1;
      open_a = nullptr;
    }
  }
  void resolve() {
    if (pending.empty()) return;
    ck(cudaStreamSynchronize(stream));
    for (auto& p : pending) {
      float t = 0.f;
      ck(cudaEventElapsedTime(&t, p.a, p.b));
      ms[p.cls] += t;
      timed[p.cls] += 1;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    resolve();
    for (int k = 0; k < LSN_K_COUNT; ++k) launches[k] = timed[k] = 0, ms[k] = 0.0;
  }
  ~Profiler() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct EngineBase {
  virtual ~EngineBase() {}
  // one evaluation pass (decoder, element, reduction, select_direction)
  virtual void pass(cudaStream_t s, unsigned long long cond, int use_cond) = 0;
  virtual void begin(int eval_only) = 0;   // reset the device solve state
  virtual void finish(double dt) = 0;      // q, v from the positions at z
  virtual void decode_to_host(double* x, double* J) = 0;
  // per-tet reduced elastic forces of every mesh tet at the point of the
  // last pass into A (r rows of ne, device)
  virtual void tet_forces(double* A) = 0;
  virtual int kernels_per_pass() const = 0;
  // nonzero when a bounded wait inside a tensor-core kernel ran out (reads a
  // device flag; call after the stream's work is queued)
  virtual int device_error(cudaStream_t) { return 0; }
  DevSolver* sv = nullptr;
  double* sys = nullptr;
  int kind = 0;       // optimiser of the solves: 0 projective Newton, 1 L-BFGS
  int pass_kind = 0;  // passes issued by pass(): 0 full (E, g, K), 1 gradient-only
  // CUDA graph of the whole solve loop (conditional WHILE node)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
};

}  // namespace

struct lsn_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  std::string err;
  // mesh (FP64)
  int nv = 0, n = 0, ne = 0;
  double* X0 = nullptr;
  int4* tets = nullptr;
  double* dminv = nullptr;
  double* vol = nullptr;
  double* mass = nullptr;
  int* adj_ptr = nullptr;
  int* adj_tet = nullptr;
  // material
  bool have_material = false;
  double youngs = 0, poisson = 0, rho = 0, grav[3] = {0, 0, 0};
  // constraints
  int nc = 0;
  std::vector<int> cidx;
  int* cslot = nullptr;   // nv
  double* cu = nullptr;   // 3 nc target displacements
  double* ctmp = nullptr; // 3 nc targets (positions) before X0 is subtracted
  // cubature
  int S = 0;
  int* cub_idx = nullptr;
  double* cub_w = nullptr;
  // ground
  double ground_h = 0.0, ground_k = 0.0;
  // affine modes in parallel with the network (12 extra coordinates of z)
  bool affine = false;
  double acen[3] = {0.0, 0.0, 0.0};
  // decoder (host copy)
  bool have_decoder = false;
  std::vector<int> widths;
  std::vector<std::vector<float>> W, b;
  double scale = 1.0;
  int precision = LSN_PREC_FP32;
  // solver controls
  double tol = 1e-5, armijo_c = 1e-4;
  int max_newton = 1024, max_ls = 128;
  int opt_kind = LSN_OPT_NEWTON, hist_m = 10;  // optimiser and L-BFGS history size
  bool exact_hessian = false;  // decoder-curvature term in K (curvature.cu)
  double exact_clamp = 1e-10;
  // state
  double* q = nullptr;
  double* v = nullptr;
  double* ubar = nullptr;
  double dt = 0.0;
  bool q_valid = false;
  std::vector<double> z0;   // host copy of the initial z (set_state)
  bool z_pending = false;
  // engine
  std::unique_ptr<EngineBase> eng;
  bool dirty = true;
  int* pinned_status = nullptr;
  double E_const = 0.0;  // -sum m g . X0 in quasi-static solves
  int* cidx_dev = nullptr;  // constrained vertex indices
  Profiler prof;
  bool use_graph = true;
  long long passes_total = 0;
  // decoder training (lsn_train_*)
  std::unique_ptr<TrainerBase> trainer;
  int lip_order = 2;  // order of the Lipschitz loss in training (0 or 2)
  int* tr_cub_idx = nullptr;
  double* tr_cub_w = nullptr;
  double* tr_q = nullptr;
  long long tr_qcap = 0;
  // full-space comparison solve (lsn_fullspace_*): its own q, v
  std::unique_ptr<FullSpaceBase> fs;
  double fs_rtol = 1e-4;
  int fs_max_cg = 4096;
};

namespace {

// dimension of z: the network's input width, plus 12 with affine modes
int subspace_r(const lsn_ctx* c) { return c->widths[0] + (c->affine ? 12 : 0); }

// ----------------------------------------------------------------- engine
template <typename Real>
struct Engine : EngineBase {
  lsn_ctx* c;
  int r, L, n, S, C, nj;
  std::vector<Real*> dW, db;
  Real *Z[2] = {nullptr, nullptr}, *Z0 = nullptr, *u = nullptr, *J = nullptr,
       *ut = nullptr;
  int4* ctets = nullptr;
  Real *cdminv = nullptr, *cwv = nullptr;
  double *part_dec = nullptr, *part_el = nullptr;
  int grid_dec, gfull, genergy, nst;
  LastArgs la;
  ElemArgs ea;
  TcLast tcl;          // tensor-core output layer (TF32 / BF16 forms)
  bool use_tc = false;       // TF32 / BF16 form: tensor-core element contraction
  bool use_tc_last = false;  // ... and tensor-core output layer (hidden width allows TMA)
  bool use_tc_hidden = false;  // ... and tensor-core hidden layers
  TcHidden tch;
  int* tc_err = nullptr;     // device flag: a bounded wait of a tensor-core kernel ran out
  DevHistory* hist = nullptr;  // L-BFGS curvature pairs
  double* Zd = nullptr;        // FP64 copy of the pass points (affine modes)
  int ggrid = 0;               // CTAs of the gradient-only element kernel
  Curvature<Real> curv;        // exact-form reduced Hessian (opt-in)
  bool use_exact = false;

  explicit Engine(lsn_ctx* ctx) : c(ctx) {
    cudaStream_t s = c->stream;
    r = subspace_r(c);
    L = (int)c->widths.size() - 1;
    n = c->n;
    S = c->S > 0 ? c->S : c->ne;
    nj = r + 1;
    C = nj + KTRIAL;
    nst = nslots_total(r);
    int hmax = r;
    for (int w : c->widths) hmax = std::max(hmax, w);
    for (int l = 0; l < L; ++l) {
      size_t cnt = (size_t)c->widths[l + 1] * c->widths[l];
      std::vector<Real> tmp(cnt);
      for (size_t i = 0; i < cnt; ++i) tmp[i] = (Real)c->W[l][i];
      dW.push_back(dalloc<Real>(cnt));
      ck(cudaMemcpyAsync(dW.back(), tmp.data(), cnt * sizeof(Real), cudaMemcpyHostToDevice, s));
      std::vector<Real> tb(c->widths[l + 1]);
      for (int i = 0; i < c->widths[l + 1]; ++i) tb[i] = (Real)c->b[l][i];
      db.push_back(dalloc<Real>(tb.size()));
      ck(cudaMemcpyAsync(db.back(), tb.data(), tb.size() * sizeof(Real), cudaMemcpyHostToDevice,
                         s));
      ck(cudaStreamSynchronize(s));
    }
    const int CPs = zstride(C);
    Z[0] = dalloc<Real>((size_t)CPs * hmax);
    Z[1] = dalloc<Real>((size_t)CPs * hmax);
    Z0 = dalloc<Real>((size_t)CPs * r);
    ck(cudaMemsetAsync(Z[0], 0, sizeof(Real) * CPs * hmax, s));
    ck(cudaMemsetAsync(Z[1], 0, sizeof(Real) * CPs * hmax, s));
    u = dalloc<Real>(n);
    J = dalloc<Real>((size_t)n * r);
    ut = dalloc<Real>((size_t)KTRIAL * n);
    ctets = dalloc<int4>(S);
    cdminv = dalloc<Real>((size_t)9 * S);
    cwv = dalloc<Real>(S);
    launch_gather_cubature<Real>(c->tets, c->dminv, c->vol, c->S > 0 ? c->cub_idx : nullptr,
                                 c->S > 0 ? c->cub_w : nullptr, S, c->ne, ctets, cdminv, cwv,
                                 s);
    grid_dec = decoder_last_grid(n, C, c->num_sms);
    use_tc = sizeof(Real) == 4 &&
             (c->precision == LSN_PREC_TF32 || c->precision == LSN_PREC_BF16);
    if (use_tc) {
      tc_err = dalloc<int>(1);
      ck(cudaMemsetAsync(tc_err, 0, sizeof(int), s));
      // the TMA row pitch (hidden width x element size) must be a multiple of
      // 16 bytes; otherwise the FP32 CUDA-core output layer serves this form
      const cudaError_t te = tcl.setup(reinterpret_cast<const float*>(dW[L - 1]), n,
                                       c->widths[L - 1], C, r,
                                       c->precision == LSN_PREC_BF16, c->num_sms, s,
                                       c->affine);
      if (te == cudaSuccess) {
        use_tc_last = true;
        grid_dec = tcl.grid;
      } else if (te == cudaErrorInvalidValue) {
        cudaGetLastError();
        tcl.release();
      } else {
        ck(te);
      }
      if (L >= 2) {  // hidden layers on the tensor cores when every layer's plan fits
        std::vector<const float*> wl;
        for (int l = 0; l < L - 1; ++l) wl.push_back(reinterpret_cast<const float*>(dW[l]));
        const cudaError_t he = tch.setup(wl, c->widths, C, nj, s);
        if (he == cudaSuccess) {
          use_tc_hidden = true;
        } else if (he == cudaErrorInvalidValue) {
          cudaGetLastError();
          tch.release();
        } else {
          ck(he);
        }
      }
    }
    element_grids(S, r, c->num_sms, gfull, genergy);
    if (use_tc) {  // one complete partial row per CTA (trial energies included)
      gfull = element_tc_grid(S, r, c->precision == LSN_PREC_BF16, c->num_sms);
      genergy = 0;
    }
    part_dec = dalloc<double>((size_t)grid_dec * nst);
    kind = pass_kind = c->opt_kind;
    ggrid = element_grad_grid(S, c->num_sms);
    hist = dalloc<DevHistory>(1);
    part_el = dalloc<double>((size_t)std::max(gfull + genergy, ggrid) * nst);
    sys = dalloc<double>(nst);
    sv = dalloc<DevSolver>(1);
    ck(cudaMemsetAsync(sv, 0, sizeof(DevSolver), s));
    ck(cudaMemsetAsync(Z0, 0, sizeof(Real) * CPs * r, s));
    la.n = n;
    la.r = r;
    la.scale = c->scale;
    la.cslot = c->cslot;
    la.cu = c->cu;
    la.mass = c->mass;
    la.ubar = c->ubar;
    la.inv_dt2 = &sv->inv_dt2;
    for (int i = 0; i < 3; ++i) la.grav[i] = c->grav[i];
    la.ground_h = c->ground_h;
    la.ground_k = c->ground_k;
    la.X0 = c->X0;
    la.aff0 = c->affine ? c->widths[0] : -1;
    la.zcps = zstride(C);
    if (c->affine) {
      Zd = dalloc<double>((size_t)zstride(C) * r);
      ck(cudaMemsetAsync(Zd, 0, sizeof(double) * zstride(C) * r, s));
    }
    la.zaff = c->affine ? Zd + (size_t)c->widths[0] * zstride(C) : nullptr;
    for (int i = 0; i < 3; ++i) la.acen[i] = c->acen[i];
    ea.S = S;
    ea.r = r;
    ea.n = n;
    ea.tets = ctets;
    ea.dminv = cdminv;
    ea.wv = cwv;
    ea.mu = c->youngs / (2.0 * (1.0 + c->poisson));
    ea.lam = c->youngs * c->poisson / ((1.0 + c->poisson) * (1.0 - 2.0 * c->poisson));
    // solver controls
    DevSolver h;
    std::memset(&h, 0, sizeof(h));
    h.tol = c->tol;
    h.armijo_c = c->armijo_c;
    // rounding unit of the energy and gradient evaluation: FP64, FP32 (also
    // the BF16 form, whose activations enter as a two-term split), TF32
    // (10 stored mantissa bits; the tensor core may truncate)
    const double unit = c->precision == LSN_PREC_FP64   ? 1.1102230246251565e-16
                        : c->precision == LSN_PREC_TF32 ? 9.765625e-04
                                                        : 5.960464477539063e-08;
    // FP64: the plain Armijo test of the paper's line search.  Lower
    // precisions accept a step whose energy rise stays within the rounding
    // scale of the energy evaluation, so the solve can reach their floor.
    // (TF32: the unit itself is coarse, so the slack and the floor stay within
    // two units of the energy / gradient scale)
    const bool tf32 = c->precision == LSN_PREC_TF32;
    h.eta_scale = c->precision == LSN_PREC_FP64 ? 0.0 : (tf32 ? 2.0 : 8.0) * unit;
    h.floor_scale = (tf32 ? 2.0 : 64.0) * unit;
    h.r = r;
    h.max_ls = c->max_ls;
    h.max_newton = c->max_newton;
    h.kind = kind;
    h.hist_m = c->hist_m;
    h.zd = Zd;
    h.gamma = 1.0;
    h.status = -1;
    ck(cudaMemcpyAsync(sv, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    ck(cudaStreamSynchronize(s));
    ck(cudaGetLastError());
    if (c->exact_hessian && kind == LSN_OPT_NEWTON) {
      CurvView cv;
      cv.widths = c->widths;
      cv.n = n;
      cv.nv = c->nv;
      cv.ne = c->ne;
      cv.S = S;
      cv.r = r;
      cv.num_sms = c->num_sms;
      cv.tets = c->tets;
      cv.cub_idx = c->S > 0 ? c->cub_idx : nullptr;
      cv.use_tc_gemm = use_tc;
      cv.s = s;
      curv.clamp = c->exact_clamp;
      ck(curv.setup(cv));
      use_exact = true;
    }
  }

  ~Engine() override {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto p : dW) dfree(p);
    for (auto p : db) dfree(p);
    dfree(Z[0]);
    dfree(Z[1]);
    dfree(Z0);
    dfree(u);
    dfree(J);
    dfree(ut);
    dfree(ctets);
    dfree(cdminv);
    dfree(cwv);
    dfree(part_dec);
    dfree(part_el);
    dfree(tc_err);
    dfree(hist);
    dfree(Zd);
    dfree(sys);
    dfree(sv);
  }

  int kernels_per_pass() const override {
    return (L - 1) + 4 + (use_exact ? curv.launches() : 0);
  }

  void begin(int eval_only) override {
    Profiler& P = c->prof;
    P.begin(LSN_K_SOLVE);
    launch_solve_begin<Real>(sv, Z0, C, eval_only, c->stream);
    P.end(LSN_K_SOLVE);
  }

  // Layers 1..L-1 of the pass; returns the buffer with the last hidden layer.
  const Real* hidden(cudaStream_t s, bool prof) {
    const Real* in = Z0;
    int cur = 0;
    if (prof) c->prof.begin(LSN_K_DECODER_HIDDEN, L - 1);
    for (int l = 0; l < L - 1; ++l) {
      const int M = c->widths[l + 1], K = c->widths[l];
      // the last hidden layer also writes the tensor-core output layer's operand
      const bool pack = use_tc_last && l == L - 2;
      if (use_tc_hidden)  // tensor-core forms: tcgen05 layers; the unit-major columns
                          // only when the CUDA-core output layer reads them
        ck(tch.launch(l, reinterpret_cast<const float*>(db[l]),
                      reinterpret_cast<const float*>(in),
                      use_tc_last ? nullptr : reinterpret_cast<float*>(Z[cur]),
                      pack ? tcl.Bh : nullptr, pack ? tcl.Bl : nullptr, pack ? tcl.bkind() : 0,
                      tc_err, s));
      else
        launch_hidden_layer<Real>(dW[l], db[l], M, K, in, C, nj, Z[cur], s,
                                  pack ? tcl.Bh : nullptr, pack ? tcl.Bl : nullptr,
                                  pack ? tcl.bkind() : 0);
      in = Z[cur];
      cur ^= 1;
    }
    if (prof) c->prof.end(LSN_K_DECODER_HIDDEN);
    return in;
  }

  void pass(cudaStream_t s, unsigned long long cond, int use_cond) override {
    const bool prof = !use_cond;  // no event timing inside a captured graph
    Profiler& P = c->prof;
    const Real* h = hidden(s, prof);
    if (prof) P.begin(LSN_K_DECODER_LAST);
    if (use_tc_last)
      tcl.launch(reinterpret_cast<const float*>(h), zstride(C),
                 reinterpret_cast<const float*>(db[L - 1]), nj, reinterpret_cast<float*>(u),
                 reinterpret_cast<float*>(J), reinterpret_cast<float*>(ut), part_dec, nst, la,
                 s, /*packed=*/L >= 2);
    else
      launch_last_layer<Real>(dW[L - 1], db[L - 1], n, c->widths[L - 1], h, C, nj, u, J, ut,
                              part_dec, nst, la, grid_dec, s);
    if (prof) P.end(LSN_K_DECODER_LAST);
    if (pass_kind == 1) {  // L-BFGS: energies and gradient only
      if (prof) P.begin(LSN_K_ELEMENT);
      launch_element_grad<Real>(ea, u, J, ut, part_el, ggrid, s);
      if (prof) P.end(LSN_K_ELEMENT);
      if (prof) P.begin(LSN_K_SOLVE, 2);
      launch_reduce_partials(part_dec, grid_dec, part_el, ggrid, -1, nslots(r), nst, sys, s,
                             slot_K(r), npairs(r));
      launch_select_lbfgs<Real>(sv, hist, sys, Z0, cond, use_cond, s);
      if (prof) P.end(LSN_K_SOLVE);
      return;
    }
    if (prof) P.begin(LSN_K_ELEMENT);
    if (use_tc)
      ck(launch_element_tc(ea, reinterpret_cast<const float*>(u),
                           reinterpret_cast<const float*>(J), reinterpret_cast<const float*>(ut),
                           part_el, gfull, c->precision == LSN_PREC_BF16, tc_err, c->num_sms,
                           s));
    else
      launch_element<Real>(ea, u, J, ut, part_el, gfull, genergy, s);
    if (prof) P.end(LSN_K_ELEMENT);
    if (prof) P.begin(LSN_K_SOLVE, 2 + (use_exact ? curv.launches() : 0));
    launch_reduce_partials(part_dec, grid_dec, part_el, gfull + genergy, use_tc ? -1 : gfull,
                           nslots(r), nst, sys, s);
    if (use_exact)
      ck(curv.launch(ea, la, u, Z0, zstride(C), dW, db,
                     (use_tc_last && tcl.bf16) ? tcl.Wlow : nullptr, sys, s));
    launch_select_direction<Real>(sv, sys, Z0, cond, use_cond, s);
    if (prof) P.end(LSN_K_SOLVE);
  }

  int device_error(cudaStream_t s) override {
    if (!use_tc) return 0;
    int h[2] = {0, 0};
    ck(cudaMemcpyAsync(&h[0], tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (use_tc_last) ck(cudaMemcpyAsync(&h[1], tcl.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    return h[0] | h[1] | (use_exact ? curv.device_error() : 0);
  }

  void finish(double dt) override {
    c->prof.begin(LSN_K_SOLVE);
    launch_finish_positions<Real>(c->X0, u, n, dt, c->q, c->v, c->stream);
    c->prof.end(LSN_K_SOLVE);
  }

  void tet_forces(double* A) override {
    launch_tet_forces<Real>(c->tets, c->dminv, c->vol, c->ne, r, u, J, ea.mu, ea.lam, A,
                            c->stream);
    ck(cudaGetLastError());
  }

  void decode_to_host(double* x, double* Jh) override {
    cudaStream_t s = c->stream;
    begin(1);
    pass(s, 0, 0);
    std::vector<Real> hu(n), hJ;
    ck(cudaMemcpyAsync(hu.data(), u, n * sizeof(Real), cudaMemcpyDeviceToHost, s));
    if (Jh) {
      hJ.resize((size_t)n * r);
      ck(cudaMemcpyAsync(hJ.data(), J, hJ.size() * sizeof(Real), cudaMemcpyDeviceToHost, s));
    }
    std::vector<double> X0h(n);
    ck(cudaMemcpyAsync(X0h.data(), c->X0, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    if (x)
      for (int i = 0; i < n; ++i) x[i] = X0h[i] + (double)hu[i];
    if (Jh)
      for (size_t i = 0; i < hJ.size(); ++i) Jh[i] = (double)hJ[i];
  }
};

int fail(lsn_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(lsn_ctx* c, cudaError_t e) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? LSN_ERR_OOM : LSN_ERR_CUDA,
              std::string("CUDA error: ") + cudaGetErrorString(e));
}

#define LSN_GUARD_BEGIN try {
#define LSN_GUARD_END                                                   \
  }                                                                     \
  catch (const CudaError& ce) {                                         \
    return cuda_fail(c, ce.e);                                          \
  }                                                                     \
  catch (const std::exception& ex) {                                    \
    return fail(c, LSN_ERR_STATE, std::string("internal error: ") + ex.what()); \
  }

int ensure_engine(lsn_ctx* c) {
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "lsn_set_mesh has not been called");
  if (!c->have_material) return fail(c, LSN_ERR_STATE, "lsn_set_material has not been called");
  if (!c->have_decoder) return fail(c, LSN_ERR_STATE, "lsn_set_decoder has not been called");
  if (!c->dirty && c->eng) return LSN_OK;
  c->eng.reset();
  if (c->precision == LSN_PREC_FP64)
    c->eng.reset(new Engine<double>(c));
  else
    c->eng.reset(new Engine<float>(c));
  c->dirty = false;
  return LSN_OK;
}

// Build (once per engine) the CUDA graph of the solve loop: a conditional
// WHILE node whose body is one evaluation pass; select_direction sets the
// loop condition on the device, so a whole solve is one graph launch.
void ensure_graph(lsn_ctx* c) {
  EngineBase* e = c->eng.get();
  if (e->exec) return;
  if (!e->cap_stream) ck(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
  ck(cudaGraphCreate(&e->graph, 0));
  cudaGraphConditionalHandle h;
  ck(cudaGraphConditionalHandleCreate(&h, e->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  ck(cudaGraphAddNode(&node, e->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  ck(cudaStreamBeginCaptureToGraph(e->cap_stream, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  // a launch that fails inside the capture must not leave the stream
  // capturing: end the capture first, then report the error
  cudaError_t launch_err = cudaSuccess;
  try {
    e->pass(e->cap_stream, (unsigned long long)h, 1);
    launch_err = cudaGetLastError();
  } catch (const CudaError& ce) {
    launch_err = ce.e;
  }
  cudaGraph_t captured = nullptr;
  cudaError_t err = cudaStreamEndCapture(e->cap_stream, &captured);
  if (err == cudaSuccess) err = launch_err;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->exec, e->graph, 0);
  if (err != cudaSuccess) {  // leave no half-built graph behind
    cudaGetLastError();
    if (e->exec) cudaGraphExecDestroy(e->exec);
    cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    throw CudaError{err};
  }
}

// One solve from the current device z: graph launch (default) or host loop
// (when kernel-event profiling is on).
// eval_pass: for eval_only, the pass kind to evaluate with (0 full, 1
// gradient-only); solves use the engine's optimiser.
void run_solve(lsn_ctx* c, int eval_only, int eval_pass = -1) {
  EngineBase* e = c->eng.get();
  cudaStream_t s = c->stream;
  const int want = (eval_only && eval_pass >= 0) ? eval_pass : e->kind;
  e->begin(eval_only);
  if (c->prof.mask == 0 && c->use_graph && want == e->kind) {
    ensure_graph(c);
    ck(cudaGraphLaunch(e->exec, s));
  } else {
    e->pass_kind = want;
    for (int guard = 0; guard < 4 * (c->max_newton + 2) * (c->max_ls + 2); ++guard) {
      e->pass(s, 0, 0);
      ck(cudaMemcpyAsync(c->pinned_status, &e->sv->running, sizeof(int),
                         cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      if (!c->pinned_status[0]) break;
    }
    e->pass_kind = e->kind;
  }
}

double quasi_static_constant(lsn_ctx* c) {
  // -sum_v m_v g . X0_v (the part of the gravity potential that does not
  // depend on z); evaluated once per mesh/material on the host from device
  // copies of the lumped mass and rest positions.
  std::vector<double> m(c->nv), X(c->n);
  ck(cudaMemcpyAsync(m.data(), c->mass, c->nv * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  ck(cudaMemcpyAsync(X.data(), c->X0, c->n * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  ck(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int v = 0; v < c->nv; ++v)
    for (int k = 0; k < 3; ++k) s -= m[v] * c->grav[k] * X[3 * v + k];
  return s;
}

}  // namespace

// ===================================================================== ABI
extern "C" {

int lsn_create(lsn_ctx** out, int device, void* cuda_stream) {
  if (!out) return LSN_ERR_ARG;
  *out = nullptr;
  lsn_ctx* c = new lsn_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMallocHost(&c->pinned_status, 8 * sizeof(int));
  c->prof.stream = c->stream;
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return LSN_ERR_CUDA;
  }
  *out = c;
  return LSN_OK;
}

static void free_mesh(lsn_ctx* c) {
  dfree(c->X0);
  dfree(c->tets);
  dfree(c->dminv);
  dfree(c->vol);
  dfree(c->mass);
  dfree(c->adj_ptr);
  dfree(c->adj_tet);
  dfree(c->cslot);
  dfree(c->cu);
  dfree(c->ctmp);
  dfree(c->cub_idx);
  dfree(c->cub_w);
  dfree(c->cidx_dev);
  c->cidx_dev = nullptr;
  dfree(c->q);
  dfree(c->v);
  dfree(c->ubar);
  c->X0 = c->dminv = c->vol = c->mass = c->cu = c->ctmp = c->cub_w = c->q = c->v = c->ubar = nullptr;
  c->tets = nullptr;
  c->adj_ptr = c->adj_tet = c->cslot = c->cub_idx = nullptr;
}

void lsn_destroy(lsn_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->eng.reset();
  c->fs.reset();
  c->trainer.reset();
  dfree(c->tr_cub_idx);
  dfree(c->tr_cub_w);
  dfree(c->tr_q);
  free_mesh(c);
  if (c->pinned_status) cudaFreeHost(c->pinned_status);
  delete c;  // the profiler releases its events
}

const char* lsn_last_error(const lsn_ctx* c) { return c ? c->err.c_str() : "null context"; }

int lsn_set_mesh(lsn_ctx* c, const double* X0, int nv, const int32_t* tets, int ne) {
  if (!c) return LSN_ERR_ARG;
  if (!X0 || !tets || nv < 4 || ne < 1) return fail(c, LSN_ERR_ARG, "set_mesh: empty mesh");
  for (long long i = 0; i < 4LL * ne; ++i)
    if (tets[i] < 0 || tets[i] >= nv)
      return fail(c, LSN_ERR_ARG, "set_mesh: tet vertex index out of range");
  for (long long i = 0; i < 3LL * nv; ++i)
    if (!std::isfinite(X0[i])) return fail(c, LSN_ERR_NONFINITE, "set_mesh: non-finite X0");
  LSN_GUARD_BEGIN
  ck(cudaSetDevice(c->device));
  c->eng.reset();
  c->fs.reset();
  free_mesh(c);
  cudaStream_t s = c->stream;
  c->nv = nv;
  c->n = 3 * nv;
  c->ne = ne;
  c->X0 = dalloc<double>(c->n);
  c->tets = dalloc<int4>(ne);
  c->dminv = dalloc<double>((size_t)9 * ne);
  c->vol = dalloc<double>(ne);
  c->mass = dalloc<double>(nv);
  c->q = dalloc<double>(c->n);
  c->v = dalloc<double>(c->n);
  c->ubar = dalloc<double>(c->n);
  c->cslot = dalloc<int>(nv);
  c->cu = dalloc<double>(3);
  c->ctmp = dalloc<double>(3);
  ck(cudaMemcpyAsync(c->X0, X0, sizeof(double) * c->n, cudaMemcpyHostToDevice, s));
  ck(cudaMemcpyAsync(c->tets, tets, sizeof(int4) * ne, cudaMemcpyHostToDevice, s));
  ck(cudaMemsetAsync(c->cslot, 0xff, sizeof(int) * nv, s));
  ck(cudaMemcpyAsync(c->q, X0, sizeof(double) * c->n, cudaMemcpyHostToDevice, s));
  ck(cudaMemsetAsync(c->v, 0, sizeof(double) * c->n, s));
  ck(cudaMemsetAsync(c->ubar, 0, sizeof(double) * c->n, s));
  // vertex -> incident tet lists (CSR) for the fixed-order lumped mass
  std::vector<int> cnt(nv + 1, 0), adj(4LL * ne);
  for (long long i = 0; i < 4LL * ne; ++i) cnt[tets[i] + 1]++;
  for (int v = 0; v < nv; ++v) cnt[v + 1] += cnt[v];
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 4; ++a) adj[fill[tets[4 * e + a]]++] = e;
  c->adj_ptr = dalloc<int>(nv + 1);
  c->adj_tet = dalloc<int>(adj.size());
  ck(cudaMemcpyAsync(c->adj_ptr, cnt.data(), sizeof(int) * (nv + 1), cudaMemcpyHostToDevice, s));
  ck(cudaMemcpyAsync(c->adj_tet, adj.data(), sizeof(int) * adj.size(), cudaMemcpyHostToDevice, s));
  int* bad = dalloc<int>(1);
  ck(cudaMemsetAsync(bad, 0, sizeof(int), s));
  launch_rest_shape(c->X0, c->tets, ne, c->dminv, c->vol, bad, s);
  int hbad = 0;
  ck(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  dfree(bad);
  ck(cudaGetLastError());
  c->nc = 0;
  c->cidx.clear();
  c->S = 0;
  c->q_valid = false;
  c->dirty = true;
  c->have_material = false;
  if (hbad) {
    free_mesh(c);
    c->nv = c->n = c->ne = 0;
    return fail(c, LSN_ERR_ARG, "set_mesh: a tet has non-positive rest volume");
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_material(lsn_ctx* c, double youngs, double poisson, double density,
                     const double* gravity) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "set_material: call lsn_set_mesh first");
  if (!(youngs > 0) || !(poisson > -1.0 && poisson < 0.5) || !(density > 0) || !gravity)
    return fail(c, LSN_ERR_ARG, "set_material: invalid material parameters");
  LSN_GUARD_BEGIN
  c->youngs = youngs;
  c->poisson = poisson;
  c->rho = density;
  for (int k = 0; k < 3; ++k) c->grav[k] = gravity[k];
  launch_lumped_mass(c->adj_ptr, c->adj_tet, c->vol, c->nv, density, c->mass, c->stream);
  ck(cudaStreamSynchronize(c->stream));
  ck(cudaGetLastError());
  c->E_const = quasi_static_constant(c);
  c->have_material = true;
  c->dirty = true;
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_constraints(lsn_ctx* c, const int32_t* vidx, int nc, const double* targets) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "set_constraints: call lsn_set_mesh first");
  LSN_GUARD_BEGIN
  cudaStream_t s = c->stream;
  if (vidx) {
    if (nc < 0 || nc > c->nv) return fail(c, LSN_ERR_ARG, "set_constraints: bad count");
    std::vector<int> slot(c->nv, -1);
    for (int i = 0; i < nc; ++i) {
      if (vidx[i] < 0 || vidx[i] >= c->nv)
        return fail(c, LSN_ERR_ARG, "set_constraints: vertex index out of range");
      if (slot[vidx[i]] >= 0) return fail(c, LSN_ERR_ARG, "set_constraints: duplicate vertex");
      slot[vidx[i]] = i;
    }
    if (nc != c->nc) {
      dfree(c->cu);
      dfree(c->ctmp);
      c->cu = dalloc<double>(3 * std::max(nc, 1));
      c->ctmp = dalloc<double>(3 * std::max(nc, 1));
      c->dirty = true;  // engine holds the pointer
    }
    c->nc = nc;
    c->cidx.assign(vidx, vidx + nc);
    dfree(c->cidx_dev);
    c->cidx_dev = dalloc<int>(std::max(nc, 1));
    if (nc > 0)
      ck(cudaMemcpyAsync(c->cidx_dev, vidx, sizeof(int) * nc, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(c->cslot, slot.data(), sizeof(int) * c->nv, cudaMemcpyHostToDevice, s));
    ck(cudaStreamSynchronize(s));
  } else if (nc != c->nc) {
    return fail(c, LSN_ERR_ARG, "set_constraints: count differs from the current set");
  }
  if (c->nc > 0) {
    if (!targets) return fail(c, LSN_ERR_ARG, "set_constraints: targets missing");
    upload(c->ctmp, targets, sizeof(double) * 3 * c->nc, s);
    c->prof.begin(LSN_K_SOLVE);
    launch_constraint_disp(c->cidx_dev, c->ctmp, c->X0, c->nc, c->cu, s);
    c->prof.end(LSN_K_SOLVE);
    ck(cudaGetLastError());
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_cubature(lsn_ctx* c, const int32_t* tet_idx, const double* w, int s_cnt) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "set_cubature: call lsn_set_mesh first");
  if (s_cnt < 0 || s_cnt > c->ne) return fail(c, LSN_ERR_ARG, "set_cubature: bad size");
  LSN_GUARD_BEGIN
  dfree(c->cub_idx);
  dfree(c->cub_w);
  c->cub_idx = nullptr;
  c->cub_w = nullptr;
  c->S = s_cnt;
  if (s_cnt > 0) {
    if (!tet_idx || !w) return fail(c, LSN_ERR_ARG, "set_cubature: null arrays");
    for (int i = 0; i < s_cnt; ++i) {
      if (tet_idx[i] < 0 || tet_idx[i] >= c->ne)
        return fail(c, LSN_ERR_ARG, "set_cubature: tet index out of range");
      if (!(w[i] >= 0.0) || !std::isfinite(w[i]))
        return fail(c, LSN_ERR_ARG, "set_cubature: weights must be finite and >= 0");
    }
    c->cub_idx = dalloc<int>(s_cnt);
    c->cub_w = dalloc<double>(s_cnt);
    ck(cudaMemcpyAsync(c->cub_idx, tet_idx, sizeof(int) * s_cnt, cudaMemcpyHostToDevice,
                       c->stream));
    ck(cudaMemcpyAsync(c->cub_w, w, sizeof(double) * s_cnt, cudaMemcpyHostToDevice, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  }
  c->dirty = true;
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_ground(lsn_ctx* c, double height, double stiffness) {
  if (!c) return LSN_ERR_ARG;
  if (!(stiffness >= 0.0) || !std::isfinite(height))
    return fail(c, LSN_ERR_ARG, "set_ground: invalid parameters");
  c->ground_h = height;
  c->ground_k = stiffness;
  c->dirty = true;
  return LSN_OK;
}

int lsn_set_decoder(lsn_ctx* c, int nlayers, const int* widths, const float* const* W,
                    const float* const* b, double out_scale, int precision) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "set_decoder: call lsn_set_mesh first");
  if (nlayers < 1 || !widths || !W || !b) return fail(c, LSN_ERR_ARG, "set_decoder: bad layers");
  if (widths[0] < 1 || widths[0] + (c->affine ? 12 : 0) > RMAX)
    return fail(c, LSN_ERR_ARG,
                "set_decoder: subspace dimension (with affine modes) must be in [1, 64]");
  if (widths[nlayers] != c->n)
    return fail(c, LSN_ERR_ARG, "set_decoder: last width must equal 3 * nv");
  if (precision < LSN_PREC_FP64 || precision > LSN_PREC_BF16)
    return fail(c, LSN_ERR_ARG, "set_decoder: unknown precision");
  if (!std::isfinite(out_scale)) return fail(c, LSN_ERR_ARG, "set_decoder: bad scale");
  for (int l = 0; l <= nlayers; ++l)
    if (widths[l] < 1) return fail(c, LSN_ERR_ARG, "set_decoder: zero width");
  std::vector<std::vector<float>> Wc, bc;
  for (int l = 0; l < nlayers; ++l) {
    size_t cnt = (size_t)widths[l + 1] * widths[l];
    if (!W[l] || !b[l]) return fail(c, LSN_ERR_ARG, "set_decoder: null layer");
    Wc.emplace_back(W[l], W[l] + cnt);
    bc.emplace_back(b[l], b[l] + widths[l + 1]);
    for (float x : Wc.back())
      if (!std::isfinite(x)) return fail(c, LSN_ERR_NONFINITE, "set_decoder: non-finite weight");
    for (float x : bc.back())
      if (!std::isfinite(x)) return fail(c, LSN_ERR_NONFINITE, "set_decoder: non-finite bias");
  }
  c->widths.assign(widths, widths + nlayers + 1);
  c->W.swap(Wc);
  c->b.swap(bc);
  c->scale = out_scale;
  c->precision = precision;
  c->have_decoder = true;
  c->dirty = true;
  c->z0.assign(subspace_r(c), 0.0);
  c->z_pending = true;
  return LSN_OK;
}

int lsn_set_affine_modes(lsn_ctx* c, int enable, const double* center) {
  if (!c) return LSN_ERR_ARG;
  if (!c->have_decoder) return fail(c, LSN_ERR_STATE, "set_affine_modes: set the decoder first");
  if (enable && (!center || !std::isfinite(center[0]) || !std::isfinite(center[1]) ||
                 !std::isfinite(center[2])))
    return fail(c, LSN_ERR_ARG, "set_affine_modes: bad centre");
  if (enable && c->widths[0] + 12 > RMAX)
    return fail(c, LSN_ERR_ARG, "set_affine_modes: network input width + 12 exceeds 64");
  c->affine = enable != 0;
  for (int i = 0; i < 3; ++i) c->acen[i] = enable ? center[i] : 0.0;
  c->dirty = true;
  c->z0.assign(subspace_r(c), 0.0);
  c->z_pending = true;
  return LSN_OK;
}

int lsn_set_solver(lsn_ctx* c, double tol_inf, int max_newton, int max_ls, double armijo_c) {
  if (!c) return LSN_ERR_ARG;
  if (!(tol_inf > 0) || max_newton < 0 || max_ls < 1 || !(armijo_c > 0 && armijo_c < 1))
    return fail(c, LSN_ERR_ARG, "set_solver: invalid controls");
  c->tol = tol_inf;
  c->max_newton = max_newton;
  c->max_ls = max_ls;
  c->armijo_c = armijo_c;
  if (c->eng && !c->dirty) {  // update the controls of the live engine
    try {
      DevSolver* sv = c->eng->sv;
      ck(cudaMemcpyAsync(&sv->tol, &c->tol, sizeof(double), cudaMemcpyHostToDevice, c->stream));
      ck(cudaMemcpyAsync(&sv->armijo_c, &c->armijo_c, sizeof(double), cudaMemcpyHostToDevice,
                         c->stream));
      ck(cudaMemcpyAsync(&sv->max_ls, &c->max_ls, sizeof(int), cudaMemcpyHostToDevice,
                         c->stream));
      ck(cudaMemcpyAsync(&sv->max_newton, &c->max_newton, sizeof(int), cudaMemcpyHostToDevice,
                         c->stream));
      ck(cudaStreamSynchronize(c->stream));
    } catch (const CudaError& ce) {
      return cuda_fail(c, ce.e);
    }
  }
  return LSN_OK;
}

int lsn_set_optimizer(lsn_ctx* c, int kind, int history) {
  if (!c) return LSN_ERR_ARG;
  if ((kind != LSN_OPT_NEWTON && kind != LSN_OPT_LBFGS) || history < 1 || history > MHIST)
    return fail(c, LSN_ERR_ARG, "set_optimizer: invalid optimiser or history size");
  if (kind != c->opt_kind || history != c->hist_m) c->dirty = true;
  c->opt_kind = kind;
  c->hist_m = history;
  return LSN_OK;
}

int lsn_set_exact_hessian(lsn_ctx* c, int enable, double clamp) {
  if (!c) return LSN_ERR_ARG;
  if (!(clamp >= 0.0 && clamp < 1.0))
    return fail(c, LSN_ERR_ARG, "set_exact_hessian: clamp must be in [0, 1)");
  if ((enable != 0) != c->exact_hessian || clamp != c->exact_clamp) c->dirty = true;
  c->exact_hessian = enable != 0;
  c->exact_clamp = clamp;
  return LSN_OK;
}

int lsn_selftest_bounded_wait(lsn_ctx* c, double seconds, int* code) {
  if (!c || !code || !(seconds > 0.0 && seconds <= 10.0)) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  ck(bounded_wait_selftest(seconds, code, c->stream));
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_execution(lsn_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 1) return LSN_ERR_ARG;
  c->use_graph = mode == 0;
  return LSN_OK;
}

}  // extern "C"

namespace {
// apply a pending z to the device solver state
int sync_z(lsn_ctx* c) {
  if (c->z_pending) {
    ck(cudaMemcpyAsync(&c->eng->sv->z[0], c->z0.data(), sizeof(double) * c->z0.size(),
                       cudaMemcpyHostToDevice, c->stream));
    c->z_pending = false;
  }
  return LSN_OK;
}
int prepare(lsn_ctx* c) {
  bool rebuilt = c->dirty || !c->eng;
  int rc = ensure_engine(c);
  if (rc != LSN_OK) return rc;
  if (rebuilt) c->z_pending = true;  // new engine: z from the host copy
  return sync_z(c);
}
}  // namespace

extern "C" {

int lsn_set_state(lsn_ctx* c, const double* z, const double* q, const double* v) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  const int r = subspace_r(c);
  cudaStream_t s = c->stream;
  if (z) {
    upload(&c->eng->sv->z[0], z, sizeof(double) * r, s);
    ck(cudaMemcpyAsync(c->z0.data(), &c->eng->sv->z[0], sizeof(double) * r,
                       cudaMemcpyDeviceToHost, s));
  }
  if (q) {
    upload(c->q, q, sizeof(double) * c->n, s);
  } else {  // q = x(z): one evaluation pass at z
    run_solve(c, 1);
    c->eng->finish(0.0);
  }
  if (v) upload(c->v, v, sizeof(double) * c->n, s);
  else ck(cudaMemsetAsync(c->v, 0, sizeof(double) * c->n, s));
  ck(cudaStreamSynchronize(s));
  ck(cudaGetLastError());
  c->q_valid = true;
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_dynamics(lsn_ctx* c, double dt, const double* qbar) {
  if (!c) return LSN_ERR_ARG;
  if (!(dt >= 0.0)) return fail(c, LSN_ERR_ARG, "set_dynamics: dt must be >= 0");
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  c->dt = dt;
  if (dt > 0.0) {
    if (!qbar) return fail(c, LSN_ERR_ARG, "set_dynamics: qbar missing");
    // ubar = qbar - X0: the inertial-guess kernel with q = qbar, v = 0, g = 0
    const double zero3[3] = {0.0, 0.0, 0.0};
    upload(c->ubar, qbar, sizeof(double) * c->n, c->stream);
    launch_begin_step(c->X0, c->ubar, c->ubar, c->n, 1e-300, zero3, c->ubar, c->eng->sv,
                      c->stream);
  }
  launch_begin_step(c->X0, nullptr, nullptr, c->n, dt, c->grav, c->ubar, c->eng->sv,
                    c->stream);
  ck(cudaStreamSynchronize(c->stream));
  ck(cudaGetLastError());
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_eval(lsn_ctx* c, const double* z, double* E, double* g, double* K) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  const int r = subspace_r(c);
  if (z) {
    upload(&c->eng->sv->z[0], z, sizeof(double) * r, c->stream);
    ck(cudaMemcpyAsync(c->z0.data(), &c->eng->sv->z[0], sizeof(double) * r,
                       cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  }
  // the L-BFGS passes carry no reduced Hessian: K comes from a full pass
  run_solve(c, 1, (c->opt_kind == LSN_OPT_LBFGS && !K) ? 1 : 0);
  std::vector<double> sys(nslots(r));
  ck(cudaMemcpyAsync(sys.data(), c->eng->sys, sizeof(double) * sys.size(),
                     cudaMemcpyDeviceToHost, c->stream));
  ck(cudaStreamSynchronize(c->stream));
  ck(cudaGetLastError());
  if (E) *E = sys[0] + (c->dt > 0.0 ? 0.0 : c->E_const);
  if (g)
    for (int i = 0; i < r; ++i) g[i] = sys[slot_g(i)];
  if (K)
    for (int i = 0; i < r; ++i)
      for (int j = i; j < r; ++j) {
        double val = sys[slot_K(r) + i * r - (i * (i - 1)) / 2 + (j - i)];
        K[i * r + j] = val;
        K[j * r + i] = val;
      }
  return LSN_OK;
  LSN_GUARD_END
}

}  // extern "C"

namespace {
// A (K r x ne, device) of the per-tet reduced elastic forces at the K points
// z (host or device); the solver's current z is restored afterwards
void tet_force_matrix(lsn_ctx* c, const double* z, int K, double* Ad) {
  const int r = subspace_r(c);
  cudaStream_t s = c->stream;
  std::vector<double> zsave(r);
  ck(cudaMemcpyAsync(zsave.data(), &c->eng->sv->z[0], sizeof(double) * r,
                     cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  const bool zdev = is_device_ptr(z);
  for (int k = 0; k < K; ++k) {
    ck(cudaMemcpyAsync(&c->eng->sv->z[0], z + (size_t)k * r, sizeof(double) * r,
                       zdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    run_solve(c, 1, 0);
    c->eng->tet_forces(Ad + (size_t)k * r * c->ne);
  }
  ck(cudaMemcpyAsync(&c->eng->sv->z[0], zsave.data(), sizeof(double) * r,
                     cudaMemcpyHostToDevice, s));
  ck(cudaStreamSynchronize(s));
}
}  // namespace

extern "C" {

int lsn_tet_forces(lsn_ctx* c, const double* z, int K, double* A) {
  if (!c) return LSN_ERR_ARG;
  if (!z || !A || K < 1) return fail(c, LSN_ERR_ARG, "tet_forces: bad arguments");
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  const size_t cnt = (size_t)K * subspace_r(c) * c->ne;
  const bool adev = is_device_ptr(A);
  double* Ad = adev ? A : dalloc<double>(cnt);
  try {
    tet_force_matrix(c, z, K, Ad);
    if (!adev) {
      ck(cudaMemcpyAsync(A, Ad, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
      ck(cudaStreamSynchronize(c->stream));
    }
  } catch (...) {
    if (!adev) dfree(Ad);
    throw;
  }
  if (!adev) dfree(Ad);
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_select_cubature(lsn_ctx* c, const double* z, int K, int S, int32_t* idx, double* w,
                        int* count, double* rel_residual) {
  if (!c) return LSN_ERR_ARG;
  if (!z || !idx || !w || !count || K < 1 || S < 1)
    return fail(c, LSN_ERR_ARG, "select_cubature: bad arguments");
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  if (S > c->ne) return fail(c, LSN_ERR_ARG, "select_cubature: S exceeds the tet count");
  const int r = subspace_r(c), m = K * r;
  double* Ad = dalloc<double>((size_t)m * c->ne);
  std::vector<int> P;
  std::vector<double> xP, b;
  double rel = 0.0;
  cudaError_t e = cudaSuccess;
  try {
    tet_force_matrix(c, z, K, Ad);
    e = cubature_normalise(Ad, m, c->ne, r, b, c->stream);
    if (e == cudaSuccess) e = cubature_nnls(Ad, m, c->ne, b, S, P, xP, rel, c->stream);
  } catch (...) {
    dfree(Ad);
    throw;
  }
  dfree(Ad);
  ck(e);
  // ascending tet order (the cubature gather reads the mesh in that order)
  std::vector<int> ord(P.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
  std::sort(ord.begin(), ord.end(), [&](int a, int bb) { return P[a] < P[bb]; });
  for (size_t i = 0; i < ord.size(); ++i) {
    idx[i] = P[ord[i]];
    w[i] = xP[ord[i]];
  }
  *count = (int)P.size();
  if (rel_residual) *rel_residual = rel;
  return LSN_OK;
  LSN_GUARD_END
}

}  // extern "C"

namespace {
FsArgs fullspace_args(const lsn_ctx* c) {
  FsArgs a;
  a.nv = c->nv;
  a.n = c->n;
  a.ne = c->ne;
  a.X0 = c->X0;
  a.tets = c->tets;
  a.dminv = c->dminv;
  a.vol = c->vol;
  a.mass = c->mass;
  a.cslot = c->cslot;
  a.cu = c->cu;
  a.mu = c->youngs / (2.0 * (1.0 + c->poisson));
  a.lam = c->youngs * c->poisson / ((1.0 + c->poisson) * (1.0 - 2.0 * c->poisson));
  for (int k = 0; k < 3; ++k) a.grav[k] = c->grav[k];
  a.tol = c->tol;
  a.armijo_c = c->armijo_c;
  a.cg_rtol = c->fs_rtol;
  a.max_newton = c->max_newton;
  a.max_ls = c->max_ls;
  a.max_cg = c->fs_max_cg;
  return a;
}
}  // namespace

extern "C" {

int lsn_fullspace_setup(lsn_ctx* c, int precision, double cg_rtol, int max_cg) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "fullspace_setup: call lsn_set_mesh first");
  if (!c->have_material)
    return fail(c, LSN_ERR_STATE, "fullspace_setup: call lsn_set_material first");
  if (precision != LSN_PREC_FP64 && precision != LSN_PREC_FP32)
    return fail(c, LSN_ERR_ARG, "fullspace_setup: precision must be LSN_PREC_FP64 or FP32");
  if (!(cg_rtol >= 0.0 && cg_rtol < 1.0) || max_cg < 1)
    return fail(c, LSN_ERR_ARG, "fullspace_setup: need 0 <= cg_rtol < 1 and max_cg >= 1");
  LSN_GUARD_BEGIN
  c->fs.reset();
  c->fs_rtol = cg_rtol;
  c->fs_max_cg = max_cg;
  FullSpaceBase* f = nullptr;
  cudaError_t e = make_fullspace(precision == LSN_PREC_FP64, fullspace_args(c), c->num_sms,
                                 c->stream, &f);
  if (e != cudaSuccess) return cuda_fail(c, e);
  c->fs.reset(f);
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_fullspace_set_state(lsn_ctx* c, const double* q, const double* v) {
  if (!c) return LSN_ERR_ARG;
  if (!c->fs) return fail(c, LSN_ERR_STATE, "fullspace_set_state: call lsn_fullspace_setup first");
  LSN_GUARD_BEGIN
  cudaStream_t s = c->stream;
  if (q) upload(c->fs->positions(), q, sizeof(double) * c->n, s);
  else ck(cudaMemcpyAsync(c->fs->positions(), c->X0, sizeof(double) * c->n,
                          cudaMemcpyDeviceToDevice, s));
  if (v) upload(c->fs->velocities(), v, sizeof(double) * c->n, s);
  else ck(cudaMemsetAsync(c->fs->velocities(), 0, sizeof(double) * c->n, s));
  ck(cudaStreamSynchronize(s));
  ck(cudaGetLastError());
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_fullspace_step(lsn_ctx* c, double dt, double* q_out, lsn_stats* stats,
                       long long* cg_iters) {
  if (!c) return LSN_ERR_ARG;
  if (!(dt >= 0.0) || !std::isfinite(dt))
    return fail(c, LSN_ERR_ARG, "fullspace_step: dt must be >= 0");
  if (!c->fs) return fail(c, LSN_ERR_STATE, "fullspace_step: call lsn_fullspace_setup first");
  if (c->ground_k > 0.0)
    return fail(c, LSN_ERR_STATE, "fullspace_step: the ground penalty is not part of this solve");
  auto t0 = std::chrono::steady_clock::now();
  LSN_GUARD_BEGIN
  FsResult res;
  cudaError_t e = c->fs->step(fullspace_args(c), dt, res, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e);
  if (res.status == LSN_ERR_NONFINITE)
    return fail(c, LSN_ERR_NONFINITE, "fullspace_step: non-finite energy or gradient");
  if (q_out) {
    if (is_device_ptr(q_out))
      ck(cudaMemcpyAsync(q_out, c->fs->positions(), sizeof(double) * c->n,
                         cudaMemcpyDeviceToDevice, c->stream));
    else
      ck(cudaMemcpyAsync(q_out, c->fs->positions(), sizeof(double) * c->n,
                         cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  }
  auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->newton_iters = res.newton_iters;
    stats->ls_trials = res.ls_trials;
    stats->exit = res.status;
    stats->grad_inf = res.grad_inf;
    stats->energy = res.energy;
    stats->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  if (cg_iters) *cg_iters = res.cg_iters;
  return res.status;
  LSN_GUARD_END
}


int lsn_decode(lsn_ctx* c, const double* z, double* x_out, double* J_out) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  if (z) {
    upload(&c->eng->sv->z[0], z, sizeof(double) * subspace_r(c), c->stream);
    ck(cudaMemcpyAsync(c->z0.data(), &c->eng->sv->z[0], sizeof(double) * subspace_r(c),
                       cudaMemcpyDeviceToHost, c->stream));
    ck(cudaStreamSynchronize(c->stream));
  }
  c->eng->decode_to_host(x_out, J_out);
  ck(cudaGetLastError());
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_step(lsn_ctx* c, const double* z_in, double dt, double* z_out, lsn_stats* stats) {
  if (!c) return LSN_ERR_ARG;
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(c, LSN_ERR_ARG, "step: dt must be >= 0");
  auto t0 = std::chrono::steady_clock::now();
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  cudaStream_t s = c->stream;
  const int r = subspace_r(c);
  if (!c->q_valid) {  // q = x(current z), v = 0
    rc = lsn_set_state(c, nullptr, nullptr, nullptr);
    if (rc != LSN_OK) return rc;
  }
  if (z_in) upload(&c->eng->sv->z[0], z_in, sizeof(double) * r, s);
  c->dt = dt;
  c->prof.begin(LSN_K_SOLVE);
  launch_begin_step(c->X0, c->q, c->v, c->n, dt, c->grav, c->ubar, c->eng->sv, s);
  c->prof.end(LSN_K_SOLVE);
  run_solve(c, 0);
  // the last pass evaluated the positions at the final z
  c->eng->finish(dt);
  DevSolver h;  // summary: scalars and z (not the trace arrays)
  const size_t summary = offsetof(DevSolver, z) + sizeof(h.z);
  ck(cudaMemcpyAsync(&h, c->eng->sv, summary, cudaMemcpyDeviceToHost, s));
  if (z_out && is_device_ptr(z_out))
    ck(cudaMemcpyAsync(z_out, &c->eng->sv->z[0], sizeof(double) * r, cudaMemcpyDeviceToDevice,
                       s));
  ck(cudaStreamSynchronize(s));
  ck(cudaGetLastError());
  if (c->prof.mask == 0 && c->use_graph)  // launches inside the graph, counted per pass
    for (int k = 0; k < LSN_K_COUNT; ++k) {
      const long long per = k == LSN_K_DECODER_HIDDEN ? c->eng->kernels_per_pass() - 4
                            : k == LSN_K_SOLVE        ? 2
                            : (k == LSN_K_DECODER_LAST || k == LSN_K_ELEMENT) ? 1
                                                                              : 0;
      c->prof.launches[k] += per * h.passes;
    }
  c->passes_total += h.passes;
  if (c->eng->device_error(s))
    return fail(c, LSN_ERR_CUDA, "step: a tensor-core pipeline wait timed out");
  if (h.status < -1) return fail(c, h.status, "step: non-finite values in the reduced system");
  if (z_out && !is_device_ptr(z_out)) std::memcpy(z_out, h.z, sizeof(double) * r);
  std::copy(h.z, h.z + r, c->z0.begin());
  auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->newton_iters = h.iters;
    stats->ls_trials = h.ls_trials;
    stats->exit = h.status;
    stats->grad_inf = h.grad_inf;
    stats->energy = h.E + (dt > 0.0 ? 0.0 : c->E_const);
    stats->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  return h.status;
  LSN_GUARD_END
}

int lsn_get_trace(lsn_ctx* c, int max, double* grad_inf, double* energy,
                  double* grad_scale, double* alpha, int* count) {
  if (!c || max < 0) return LSN_ERR_ARG;
  if (!c->eng) return fail(c, LSN_ERR_STATE, "get_trace: no solve yet");
  LSN_GUARD_BEGIN
  DevSolver h;
  ck(cudaMemcpyAsync(&h, c->eng->sv, sizeof(DevSolver), cudaMemcpyDeviceToHost, c->stream));
  ck(cudaStreamSynchronize(c->stream));
  int n = std::min(std::min(h.iters + 1, TRACE), max);
  for (int k = 0; k < n; ++k) {
    if (grad_inf) grad_inf[k] = h.trace_g[k];
    if (energy) energy[k] = h.trace_E[k];
    if (grad_scale) grad_scale[k] = h.trace_gabs[k];
    if (alpha) alpha[k] = h.trace_alpha[k];
  }
  if (count) *count = n;
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_profiling(lsn_ctx* c, unsigned event_mask) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  c->prof.resolve();
  c->prof.mask = event_mask & ((1u << LSN_K_COUNT) - 1);
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_get_profile(lsn_ctx* c, int cls, long long* launches, long long* timed_launches,
                    double* ms_total) {
  if (!c || cls < 0 || cls >= LSN_K_COUNT) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  c->prof.resolve();
  if (launches) *launches = c->prof.launches[cls];
  if (timed_launches) *timed_launches = c->prof.timed[cls];
  if (ms_total) *ms_total = c->prof.ms[cls];
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_reset_profile(lsn_ctx* c) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  c->prof.reset();
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_get_state(lsn_ctx* c, double* z, double* q, double* v) {
  if (!c) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  int rc = prepare(c);
  if (rc != LSN_OK) return rc;
  if (z) download(z, &c->eng->sv->z[0], sizeof(double) * subspace_r(c), c->stream);
  if (q) download(q, c->q, sizeof(double) * c->n, c->stream);
  if (v) download(v, c->v, sizeof(double) * c->n, c->stream);
  ck(cudaStreamSynchronize(c->stream));
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_get_positions(lsn_ctx* c, double* x_out) {
  if (!c || !x_out) return LSN_ERR_ARG;
  if (c->n == 0) return fail(c, LSN_ERR_STATE, "get_positions: no mesh");
  LSN_GUARD_BEGIN
  download(x_out, c->q, sizeof(double) * c->n, c->stream);
  ck(cudaStreamSynchronize(c->stream));
  return LSN_OK;
  LSN_GUARD_END
}

}  // extern "C"

// ========================================================== decoder training
namespace {
int train_ready(lsn_ctx* c) {
  if (!c) return LSN_ERR_ARG;
  if (!c->trainer) return fail(c, LSN_ERR_STATE, "lsn_train_init has not been called");
  return LSN_OK;
}
const double* train_upload_q(lsn_ctx* c, const double* q, int B) {
  const long long cnt = (long long)B * c->n;
  if (is_device_ptr(q)) return q;
  if (cnt > c->tr_qcap) {
    dfree(c->tr_q);
    c->tr_q = dalloc<double>(cnt);
    c->tr_qcap = cnt;
  }
  ck(cudaMemcpyAsync(c->tr_q, q, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream));
  return c->tr_q;
}
}  // namespace

extern "C" {

int lsn_train_init(lsn_ctx* c, const float* enc_W, const float* enc_b, const int32_t* tet_idx,
                   const double* w, int s) {
  if (!c) return LSN_ERR_ARG;
  if (c->n == 0 || !c->have_material || !c->have_decoder)
    return fail(c, LSN_ERR_STATE, "train_init: set mesh, material and decoder first");
  if (!enc_W || !enc_b || !tet_idx || !w || s < 1 || s > c->ne)
    return fail(c, LSN_ERR_ARG, "train_init: bad arguments");
  const int r = c->widths[0];
  if (r > 32) return fail(c, LSN_ERR_ARG, "train_init: training supports r <= 32");
  for (int i = 0; i < s; ++i) {
    if (tet_idx[i] < 0 || tet_idx[i] >= c->ne)
      return fail(c, LSN_ERR_ARG, "train_init: tet index out of range");
    if (!(w[i] >= 0.0) || !std::isfinite(w[i]))
      return fail(c, LSN_ERR_ARG, "train_init: weights must be finite and >= 0");
  }
  LSN_GUARD_BEGIN
  cudaStream_t st = c->stream;
  c->trainer.reset();
  dfree(c->tr_cub_idx);
  dfree(c->tr_cub_w);
  c->tr_cub_idx = dalloc<int>(s);
  c->tr_cub_w = dalloc<double>(s);
  ck(cudaMemcpyAsync(c->tr_cub_idx, tet_idx, sizeof(int) * s, cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(c->tr_cub_w, w, sizeof(double) * s, cudaMemcpyHostToDevice, st));
  std::vector<int> all(4 * (size_t)c->ne);
  ck(cudaMemcpyAsync(all.data(), c->tets, sizeof(int) * all.size(), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  TrainSetup ts;
  ts.n = c->n;
  ts.nv = c->nv;
  ts.widths = c->widths;
  ts.scale = c->scale;
  ts.mu = c->youngs / (2.0 * (1.0 + c->poisson));
  ts.lam = c->youngs * c->poisson / ((1.0 + c->poisson) * (1.0 - 2.0 * c->poisson));
  ts.alpha = 1.0 + 0.75 * ts.mu / ts.lam;
  ts.X0 = c->X0;
  ts.mass = c->mass;
  ts.S = s;
  ts.cub_idx = c->tr_cub_idx;
  ts.cub_w = c->tr_cub_w;
  ts.tets = c->tets;
  ts.dminv = c->dminv;
  ts.vol = c->vol;
  ts.ne = c->ne;
  // local numbering of the vertices the cubature tets touch (sorted)
  std::vector<int> verts;
  for (int i = 0; i < s; ++i)
    for (int a = 0; a < 4; ++a) verts.push_back(all[4 * (size_t)tet_idx[i] + a]);
  std::sort(verts.begin(), verts.end());
  verts.erase(std::unique(verts.begin(), verts.end()), verts.end());
  const int nvl = (int)verts.size();
  ts.RS = 3 * nvl;
  for (int v : verts)
    for (int k = 0; k < 3; ++k) ts.rows.push_back(3 * v + k);
  ts.tets_local.resize(4 * (size_t)s);
  std::vector<std::vector<int>> lists(nvl);
  for (int i = 0; i < s; ++i)
    for (int a = 0; a < 4; ++a) {
      const int v = all[4 * (size_t)tet_idx[i] + a];
      const int lv = (int)(std::lower_bound(verts.begin(), verts.end(), v) - verts.begin());
      ts.tets_local[4 * (size_t)i + a] = lv;
      lists[lv].push_back((i << 2) | a);
    }
  ts.inc_ptr.assign(nvl + 1, 0);
  for (int v = 0; v < nvl; ++v) {
    ts.inc_ptr[v + 1] = ts.inc_ptr[v] + (int)lists[v].size();
    ts.inc.insert(ts.inc.end(), lists[v].begin(), lists[v].end());
  }
  // initial parameters: encoder, then the context's decoder
  // the tensor-core forms train with tensor-core matrix products: TF32
  // operands, or BF16 operands (FP32 master weights) in the BF16 form
  const int tmode = c->precision == LSN_PREC_FP64   ? 1
                    : c->precision == LSN_PREC_TF32 ? 2
                    : c->precision == LSN_PREC_BF16 ? 3
                                                    : 0;
  std::unique_ptr<TrainerBase> tr(TrainerBase::create(tmode, ts));
  tr->lip_order = c->lip_order;
  std::vector<double> theta(tr->nparams);
  std::copy(enc_W, enc_W + (size_t)r * c->n, theta.begin() + tr->off[0]);
  std::copy(enc_b, enc_b + r, theta.begin() + tr->off[1]);
  for (int l = 0; l + 1 < (int)c->widths.size(); ++l) {
    std::copy(c->W[l].begin(), c->W[l].end(), theta.begin() + tr->off[2 + 2 * l]);
    std::copy(c->b[l].begin(), c->b[l].end(), theta.begin() + tr->off[3 + 2 * l]);
  }
  try {
    tr->init_device(theta.data());
  } catch (...) {
    cudaGetLastError();
    return fail(c, LSN_ERR_CUDA, "train_init: CUDA error while setting up the trainer");
  }
  c->trainer = std::move(tr);
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_num_params(lsn_ctx* c, long long* count) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!count) return LSN_ERR_ARG;
  *count = c->trainer->nparams;
  return LSN_OK;
}

// parameters and gradients cross the ABI as FP64 arrays (host or device)
static void host_to_user(const std::vector<double>& h, double* dst, cudaStream_t s) {
  download(dst, h.data(), sizeof(double) * h.size(), s);  // direction by dst
  ck(cudaStreamSynchronize(s));
}

int lsn_train_get_params(lsn_ctx* c, double* theta) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!theta) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  std::vector<double> h(c->trainer->nparams);
  try {
    c->trainer->get_params(h.data());
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_get_params: CUDA error");
  }
  if (is_device_ptr(theta)) host_to_user(h, theta, c->stream);
  else std::copy(h.begin(), h.end(), theta);
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_get_adam(lsn_ctx* c, double* m, double* v, long long* step) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!m || !v || !step) return fail(c, LSN_ERR_ARG, "train_get_adam: null output");
  if (is_device_ptr(m) || is_device_ptr(v))
    return fail(c, LSN_ERR_ARG, "train_get_adam: m and v are host arrays");
  LSN_GUARD_BEGIN
  try {
    c->trainer->get_adam(m, v, step);
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_get_adam: CUDA error");
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_set_adam(lsn_ctx* c, const double* m, const double* v, long long step) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!m || !v || step < 0) return fail(c, LSN_ERR_ARG, "train_set_adam: bad arguments");
  if (is_device_ptr(m) || is_device_ptr(v))
    return fail(c, LSN_ERR_ARG, "train_set_adam: m and v are host arrays");
  const long long np = c->trainer->nparams;
  for (long long i = 0; i < np; ++i) {
    if (!std::isfinite(m[i]) || !std::isfinite(v[i]))
      return fail(c, LSN_ERR_NONFINITE, "train_set_adam: non-finite moments");
    if (v[i] < 0.0) return fail(c, LSN_ERR_ARG, "train_set_adam: negative second moment");
  }
  LSN_GUARD_BEGIN
  try {
    c->trainer->set_adam(m, v, step);
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_set_adam: CUDA error");
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_set_params(lsn_ctx* c, const double* theta) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!theta) return LSN_ERR_ARG;
  LSN_GUARD_BEGIN
  std::vector<double> h(c->trainer->nparams);
  if (is_device_ptr(theta)) {
    ck(cudaMemcpyAsync(h.data(), theta, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    ck(cudaStreamSynchronize(c->stream));
  } else {
    std::copy(theta, theta + h.size(), h.begin());
  }
  for (double v : h)
    if (!std::isfinite(v)) return fail(c, LSN_ERR_NONFINITE, "train_set_params: non-finite");
  try {
    c->trainer->set_params(h.data());
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_set_params: CUDA error");
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_eval(lsn_ctx* c, const double* q, int B, double lambda_ls, double* losses,
                   double* grad) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!q || B < 1 || !(lambda_ls >= 0.0)) return fail(c, LSN_ERR_ARG, "train_eval: bad arguments");
  LSN_GUARD_BEGIN
  double l[3];
  const double* qd = train_upload_q(c, q, B);
  try {
    c->trainer->evaluate(qd, B, lambda_ls, l, c->stream);
    if (c->trainer->device_error())
      return fail(c, LSN_ERR_CUDA, "train_eval: a tensor-core GEMM wait ran out");
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_eval: CUDA error in the training kernels");
  }
  if (losses) std::copy(l, l + 3, losses);
  if (grad) {
    std::vector<double> h(c->trainer->nparams);
    try {
      c->trainer->get_grad(h.data());
    } catch (...) {
      return fail(c, LSN_ERR_CUDA, "train_eval: CUDA error reading the gradient");
    }
    if (is_device_ptr(grad)) host_to_user(h, grad, c->stream);
    else std::copy(h.begin(), h.end(), grad);
  }
  return std::isfinite(l[2]) ? LSN_OK : fail(c, LSN_ERR_NONFINITE, "train_eval: non-finite loss");
  LSN_GUARD_END
}

int lsn_train_step(lsn_ctx* c, const double* q, int B, double lambda_ls, double lr,
                   double* losses) {
  if (!(lr > 0.0)) return fail(c, LSN_ERR_ARG, "train_step: lr must be > 0");
  int rc = lsn_train_eval(c, q, B, lambda_ls, losses, nullptr);
  if (rc != LSN_OK) return rc;
  LSN_GUARD_BEGIN
  try {
    c->trainer->adam(lr, c->stream);
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_step: CUDA error in the Adam update");
  }
  ck(cudaStreamSynchronize(c->stream));
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_eval_unsup(lsn_ctx* c, const double* z, int B, double lambda, double sigma,
                         double lambda_ls, double* losses, double* grad) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!z || B < 1 || !(lambda >= 0.0) || !(sigma > 0.0) || !(lambda_ls >= 0.0) ||
      ((lambda > 0.0 || lambda_ls > 0.0) && B < 2))
    return fail(c, LSN_ERR_ARG, "train_eval_unsup: bad arguments");
  LSN_GUARD_BEGIN
  const int r = c->widths[0];
  std::vector<double> zh((size_t)B * r);
  if (is_device_ptr(z)) {
    ck(cudaMemcpyAsync(zh.data(), z, sizeof(double) * zh.size(), cudaMemcpyDeviceToHost,
                       c->stream));
    ck(cudaStreamSynchronize(c->stream));
  } else {
    std::copy(z, z + zh.size(), zh.begin());
  }
  for (int b = 0; b < B; ++b)
    for (int a = 0; a < b; ++a) {
      bool same = true;
      for (int k = 0; k < r && same; ++k) same = zh[(size_t)a * r + k] == zh[(size_t)b * r + k];
      if (same) return fail(c, LSN_ERR_ARG, "train_eval_unsup: repeated sample");
    }
  double l[5];
  try {
    c->trainer->evaluate_unsup(zh.data(), B, lambda, sigma, lambda_ls, l, c->stream);
    if (c->trainer->device_error())
      return fail(c, LSN_ERR_CUDA, "train_eval_unsup: a tensor-core GEMM wait ran out");
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_eval_unsup: CUDA error in the training kernels");
  }
  if (losses) std::copy(l, l + 5, losses);
  if (grad) {
    std::vector<double> h(c->trainer->nparams);
    try {
      c->trainer->get_grad(h.data());
    } catch (...) {
      return fail(c, LSN_ERR_CUDA, "train_eval_unsup: CUDA error reading the gradient");
    }
    if (is_device_ptr(grad)) host_to_user(h, grad, c->stream);
    else std::copy(h.begin(), h.end(), grad);
  }
  return std::isfinite(l[4]) ? LSN_OK
                             : fail(c, LSN_ERR_NONFINITE, "train_eval_unsup: non-finite loss");
  LSN_GUARD_END
}

int lsn_train_step_unsup(lsn_ctx* c, const double* z, int B, double lambda, double sigma,
                         double lambda_ls, double lr, double* losses) {
  if (!(lr > 0.0)) return fail(c, LSN_ERR_ARG, "train_step_unsup: lr must be > 0");
  int rc = lsn_train_eval_unsup(c, z, B, lambda, sigma, lambda_ls, losses, nullptr);
  if (rc != LSN_OK) return rc;
  LSN_GUARD_BEGIN
  try {
    c->trainer->adam(lr, c->stream);
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_step_unsup: CUDA error in the Adam update");
  }
  ck(cudaStreamSynchronize(c->stream));
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_set_lipschitz_order(lsn_ctx* c, int order) {
  if (!c) return LSN_ERR_ARG;
  if (order < 0 || order > 2)
    return fail(c, LSN_ERR_ARG, "set_lipschitz_order: orders 0, 1 and 2 are supported");
  c->lip_order = order;
  if (c->trainer) c->trainer->lip_order = order;
  return LSN_OK;
}

int lsn_train_hessians(lsn_ctx* c, const double* z, int B, double* H) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  if (!z || !H || B < 1) return fail(c, LSN_ERR_ARG, "train_hessians: bad arguments");
  LSN_GUARD_BEGIN
  TrainerBase& tr = *c->trainer;
  const int r = c->widths[0], P = tr.P;
  std::vector<double> hs((size_t)B * P);
  try {
    tr.hessians_host(z, B, hs.data(), c->stream);
    if (tr.device_error()) return fail(c, LSN_ERR_CUDA, "train_hessians: a tensor-core GEMM wait ran out");
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_hessians: CUDA error");
  }
  for (int b = 0; b < B; ++b) {
    int p = 0;
    for (int i = 0; i < r; ++i)
      for (int j = i; j < r; ++j, ++p) {
        H[(size_t)b * r * r + i * r + j] = hs[(size_t)b * P + p];
        H[(size_t)b * r * r + j * r + i] = hs[(size_t)b * P + p];
      }
  }
  return LSN_OK;
  LSN_GUARD_END
}

int lsn_train_apply(lsn_ctx* c) {
  int rc = train_ready(c);
  if (rc != LSN_OK) return rc;
  LSN_GUARD_BEGIN
  TrainerBase& tr = *c->trainer;
  std::vector<double> theta(tr.nparams);
  try {
    tr.get_params(theta.data());
  } catch (...) {
    return fail(c, LSN_ERR_CUDA, "train_apply: CUDA error");
  }
  for (int l = 0; l + 1 < (int)c->widths.size(); ++l) {
    const double* W = theta.data() + tr.off[2 + 2 * l];
    const double* b = theta.data() + tr.off[3 + 2 * l];
    for (size_t i = 0; i < c->W[l].size(); ++i) c->W[l][i] = (float)W[i];
    for (size_t i = 0; i < c->b[l].size(); ++i) c->b[l][i] = (float)b[i];
  }
  c->dirty = true;
  return LSN_OK;
  LSN_GUARD_END
}

}  // extern "C"
