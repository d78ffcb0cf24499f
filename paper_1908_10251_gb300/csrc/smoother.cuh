// Learned post-smoother: launchers (smoother.cu) and its buffers.
#pragma once
#include "kernels.cuh"

namespace pasm {

constexpr int kNNWeights = 144 + 2304 + 144;

// Grid view of one level: nx * ny interior nodes (x fastest), ldk columns of
// which the first k are pairs.
struct NNGrid {
  int nx = 0, ny = 0, ldk = 0, k = 0;
};

// Device scratch for one grid size (capacity in pixel-pairs x 16 floats).
struct NNBuf {
  static constexpr int kWgradBlocks = 1024;
  int64_t cap = 0;  // pixel-pairs
  float *z1 = nullptr, *z2p = nullptr, *z2m = nullptr, *h = nullptr;   // forward activations (x16)
  float *gh = nullptr, *gzp = nullptr, *gzm = nullptr, *gap = nullptr, *gam = nullptr, *gz1 = nullptr;  // backward
  float* wpart = nullptr;   // kWgradBlocks x 2304
  float* wflip2 = nullptr;  // 2304
  float* wflip3 = nullptr;  // 144
};

// D = N(R) on grid g (R, D: n x ldk float32)
void nn_forward(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, const float* R, float* D);
// gW = dL/dW given gD = dL/dD, after nn_forward on the same R (activations kept in b)
void nn_backward(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, const float* R, const float* gD,
                 float* gW);
// norms[c] = |a_c|^2, norms[ldk + c] = |b_c|^2 (float64 sums); partial >= ceil(n/64) x 2 x ldk doubles
void nn_column_norms(const Launch& L, int n, int ldk, const float* a, const float* b, double* partial,
                     double* norms);
// Es = -2 E / (k |r_c|^2) and loss = mean_c |E_c|^2 / |r_c|^2 from norms (|r|^2, |E|^2)
void nn_loss_seed(const Launch& L, int64_t total, int ldk, int k, const float* E, const double* norms, float* Es,
                  double* loss);
void nn_adam(const Launch& L, int nw, float* w, const float* g, float* m, float* v, float lr, int t);
void nn_add(const Launch& L, int64_t total, const float* a, const float* b, float* o);
// out = (|R_try_c| <= |R_c|) ? E + D : E + omega dinv R   (norms from nn_column_norms(R, R_try))
void nn_select(const Launch& L, int n, int ldk, const float* E, const float* D, const float* R, const float* dinv,
               float omega, const double* norms, float* out, int* accepted);

// Fused tensor-core forward (smoother_tc.cu): D = N(R) with layer 2 on tcgen05
// (bf16 operands, float32 accumulation); needs ldk % 8 == 0.  A timed-out wait
// increments *err and leaves D unwritten for that tile.
// The CUDA-core weights of layers 1 (1 -> 16) and 3 (16 -> 1), passed by value
// so that the kernel reads them from its parameter space; layer 2 comes from a
// device copy already in the tensor-core operand layout (nn_tc_layer2_layout,
// 4608 bytes).  Both host-side forms must track every change of W.
struct NNOuterWeights {
  float w1[144];  // [tap][out]
  float w3[144];  // [tap][in]
};
cudaError_t nn_tc_prepare();
bool nn_tc_supported(int ldk);
void nn_tc_layer2_layout(const float* W2, uint16_t* out);  // 2304 floats -> 2304 bf16 (4608 bytes)
void nn_forward_tc(const Launch& L, const NNGrid& g, const NNOuterWeights& w13, const void* w2, const float* R,
                   float* D, int* err);

// Tensor-core training of layer 2 (smoother_tc_train.cu): bf16 operands,
// float32 accumulation.  Needs ldk % 8 == 0.
cudaError_t nn_tc_train_prepare();
// persistent CTAs of the weight-gradient kernel (rows of its partial sums) on grid g
int nn_tc_wgrad_ctas(const NNGrid& g);
// W2 (2304 floats, device) -> bf16 operand layout; flip: the input-gradient kernel
void nn_tc_w2_layout(const Launch& L, const float* W2, bool flip, uint16_t* out);
// out = W (*) tf(in), 16 -> 16 channels; mode 0 identity, 1 relu, 2 relu of the negation
void nn_tc_conv16(const Launch& L, const NNGrid& g, int mode, const uint16_t* w2, const float* in, float* out,
                  int* err);
// per-CTA partial sums (nn_tc_wgrad_ctas rows of 2304) of layer 2's weight gradient, both branches
void nn_tc_wgrad16(const Launch& L, const NNGrid& g, const float* z1, const float* gp, const float* gm,
                   float* partial, int* err);
// The training forward and backward with layer 2 on the tensor cores (the CUDA-core
// layers 1 and 3 unchanged); w2f / w2t: device scratch for the forward and flipped
// layouts of W2 (2304 bf16 each), rebuilt from W on every call.
void nn_forward_train_tc(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, uint16_t* w2f,
                         const float* R, float* D, int* err);
void nn_backward_tc(const Launch& L, const NNGrid& g, const NNBuf& b, const float* W, uint16_t* w2t, const float* R,
                    const float* gD, float* gW, int* err);

}  // namespace pasm
