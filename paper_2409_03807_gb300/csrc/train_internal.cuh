// Host-side training engine (csrc/train.cu): parameters, Adam state and the
// per-batch buffers of the forward / backward passes.  The engine computes
// in FP32 or FP64 (TrainerBase::create); parameters and gradients cross the
// interface as FP64 host arrays.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <vector>

namespace lsn {

struct TrainSetup {
  int n = 0, nv = 0;
  std::vector<int> widths;       // r, hidden..., n
  double scale = 1.0;
  double mu = 0, lam = 0, alpha = 0;
  const double* X0 = nullptr;    // device, n
  const double* mass = nullptr;  // device, nv
  // training cubature set
  int S = 0, RS = 0;             // tets, decoder rows touched (3 x vertices)
  std::vector<int> tets_local;   // S x 4 local vertex numbers (host)
  std::vector<int> rows;         // RS global decoder rows (host)
  std::vector<int> inc_ptr, inc; // local vertex -> (tet << 2 | slot) (host)
  const int* cub_idx = nullptr;  // device, S (global tet ids)
  const double* cub_w = nullptr; // device, S
  const int4* tets = nullptr;    // device, all tets (global)
  const double* dminv = nullptr; // device, [9][ne]
  const double* vol = nullptr;   // device, ne
  int ne = 0;
};

struct TrainerBase {
  long long nparams = 0;
  std::vector<long long> off;    // offsets of Ew, eb, W_1, b_1, ...
  int L = 0, P = 0, Cs = 0;
  int lip_order = 2;  // Lipschitz loss of the potential's Hessian (2) or of the potential (0)
  virtual ~TrainerBase() {}
  // mode 0: FP32 (CUDA cores), 1: FP64, 2: FP32 with TF32 tensor-core GEMMs (tc_gemm.cu)
  static TrainerBase* create(int mode, const TrainSetup& ts);
  virtual void init_device(const double* theta_host) = 0;
  // losses[3] = L_C, L_LS, L; gradient kept on the device
  virtual void evaluate(const double* q_dev, int B, double lambda_ls, double* losses,
                        cudaStream_t s) = 0;
  // unsupervised loss of Eq. 4 at the samples z (B x r, host), with the
  // Lipschitz loss of Eq. 9 at the same samples: losses[5] = L_P, L_R,
  // L_U = L_P + lambda L_R, L_LS, L_U + lambda_ls L_LS; gradient of the last
  // kept on the device
  virtual void evaluate_unsup(const double* z, int B, double lambda, double sigma,
                              double lambda_ls, double* losses, cudaStream_t s) = 0;
  // Ht (B x P upper, row-major) at the subspace points z (B x r), host arrays
  virtual void hessians_host(const double* z, int B, double* Hs, cudaStream_t s) = 0;
  virtual void adam(double lr, cudaStream_t s) = 0;
  virtual void get_params(double* out) = 0;
  virtual void set_params(const double* in) = 0;
  virtual void get_grad(double* out) = 0;
  // Adam moments (nparams each, host FP64) and step count
  virtual void get_adam(double* m, double* v, long long* step) = 0;
  virtual void set_adam(const double* m, const double* v, long long step) = 0;
  // nonzero when a bounded wait of a tensor-core GEMM ran out (reads a device flag)
  virtual int device_error() { return 0; }
};

}  // namespace lsn
