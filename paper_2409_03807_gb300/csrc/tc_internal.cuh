// Host-side handles of the tensor-core (tcgen05) kernels: the decoder output
// layer in the BF16 and TF32 forms (tc_decoder.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "lsn_internal.cuh"

namespace lsn {

struct TcLast {
  CUtensorMap mapW, mapBh, mapBl;  // W_L tiles, packed hidden columns (hi / lo)
  void* Wlow = nullptr;            // BF16 copy of W_L (BF16 form)
  void* Bh = nullptr;              // [Cp][H] packed B operand (BF16 hi or FP32)
  void* Bl = nullptr;              // [Cp][H] BF16 low part (BF16 form)
  int* err = nullptr;              // device: nonzero when a pipeline wait timed out
  int M = 0, H = 0, C = 0, Cp = 0, r = 0, grid = 0;
  size_t smem = 0;
  bool bf16 = false;
  bool aff = false;  // affine modes: the epilogue adds them (and, in the BF16
                     // form, the inertia Gram operand is a hi + lo BF16 split)
  // W_fp32: the output layer's FP32 weights (M x H, row-major, device)
  cudaError_t setup(const float* W_fp32, int M, int H, int C, int r, bool bf16, int num_sms,
                    cudaStream_t s, bool aff = false);
  void release();
  // Z: last hidden layer, unit-major [H][CPs] (FP32); same outputs and
  // partial-row layout as launch_last_layer
  // packed: the B operand was already written by the last hidden layer
  // (launch_hidden_layer with bkind()), so the packing kernel is skipped
  void launch(const float* Z, int CPs, const float* bias, int nj, float* u, float* J, float* ut,
              double* part, int part_stride, const LastArgs& la, cudaStream_t s,
              bool packed = false) const;
  int bkind() const { return bf16 ? 1 : 2; }
  ~TcLast() { release(); }
};

// The hidden layers in the BF16 / TF32 forms (tc_hidden.cu): every layer's
// weights as per-CTA hi / lo TF32 images (built once), each layer writing the
// next layer's input image.  setup: W[l] the FP32 weights of hidden layer l
// (device), widths = r, H_1, ..., H_{L-1}, n; fails with cudaErrorInvalidValue
// when a layer's plan does not fit one CTA.  launch(l): layer l from Zin (the
// pass points, layer 0) or its input image; Zout (nullable) the unit-major
// columns; Bh / Bl / bkind the output layer's packed operand (last layer).
struct TcHidden {
  struct Layer {
    void* wimg = nullptr;
    void* bimg = nullptr;  // input image (layers >= 1)
    int M = 0, K = 0;
  };
  std::vector<Layer> layers;
  int C = 0, nj = 0;
  cudaError_t setup(const std::vector<const float*>& W, const std::vector<int>& widths, int C,
                    int nj, cudaStream_t s);
  cudaError_t launch(int l, const float* b, const float* Zin, float* Zout, void* Bh, void* Bl,
                     int bkind, int* err, cudaStream_t s) const;
  void release();
  ~TcHidden() { release(); }
};

}  // namespace lsn
