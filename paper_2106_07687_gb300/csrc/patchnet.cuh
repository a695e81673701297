// Patch network of DNN-MG (Sec. 2.2, Sec. 3.1): n stacked GRU cells with
// hidden size m (m x n in {32, 64} x {1, 2, 3}, the sizes of Table 1) and a
// dense head, either Linear(m -> 128) + ReLU + Linear(128 -> C_out) (mlp =
// 128) or the single dense layer Linear(m -> C_out) of Table 1's networks
// (mlp = 0), with or without biases, evaluated for every patch with tcgen05
// tensor-core GEMMs.
//
// Flat FP32 parameter order (PyTorch's GRU order, gate rows r, z, n):
//   per layer l: W_ih (3m x C_l), W_hh (3m x m), [b_ih (3m), b_hh (3m)]
//   then [W1 (128 x m), [b1 (128)]], W2 (C_out x K2), [b2 (C_out)]
// with C_0 = C_in (40 for one replaced level), C_l = m above, K2 = 128 with
// the hidden dense layer and m without it; the bracketed biases exist only
// with bias = 1.  Table 1's networks (bias-free, one dense layer, 51 inputs,
// 18 outputs) have 171 m + 3 m^2 + 6 m^2 (n - 1) parameters.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace dnnmg {

constexpr int kMaxLayers = 3;

constexpr size_t kNoParam = ~(size_t)0;  // offset of a parameter block that does not exist

// Offsets of the parameter blocks in the flat vector (kNoParam if absent).
struct NetOffsets {
  size_t wih[kMaxLayers], whh[kMaxLayers], bih[kMaxLayers], bhh[kMaxLayers], w1, b1, w2, b2, total;
};

struct NetDims {
  int c_in = 40, hidden = 64, layers = 2, mlp = 128, c_out = 18, bias = 1;
  __host__ __device__ int kx0() const { return (c_in + 15) / 16 * 16; }  // padded K of layer 0
  __host__ __device__ int nout() const {
    return (c_out + 15) / 16 * 16 < 32 ? 32 : (c_out + 15) / 16 * 16;
  }
  // K of the output layer: the hidden dense layer's width, or m without it
  __host__ __device__ int k2() const { return mlp ? mlp : hidden; }
  __host__ __device__ NetOffsets offsets() const {
    NetOffsets o{};
    size_t n = 0;
    const size_t H = hidden;
    for (int l = 0; l < layers; ++l) {
      const size_t c = l == 0 ? c_in : hidden;
      o.wih[l] = n;  n += 3 * H * c;
      o.whh[l] = n;  n += 3 * H * H;
      o.bih[l] = bias ? n : kNoParam;  n += bias ? 3 * H : 0;
      o.bhh[l] = bias ? n : kNoParam;  n += bias ? 3 * H : 0;
    }
    o.w1 = mlp ? n : kNoParam;          n += mlp ? (size_t)mlp * H : 0;
    o.b1 = mlp && bias ? n : kNoParam;  n += mlp && bias ? mlp : 0;
    o.w2 = n;                           n += (size_t)c_out * k2();
    o.b2 = bias ? n : kNoParam;         n += bias ? c_out : 0;
    o.total = n;
    return o;
  }
  __host__ __device__ size_t num_params() const { return offsets().total; }
};

// Packed BF16 operand image of the weights (the shared-memory layout of the
// forward kernel, copied verbatim) and FP32 biases.
struct PackedNet {
  uint16_t* w = nullptr;     // BF16 operand image
  float* bias = nullptr;     // [layers][4][m] (r: b_ir+b_hr, z: b_iz+b_hz, b_in, b_hn), b1, b2
  size_t w_elems = 0;
  size_t bias_elems = 0;
};

// element offsets of the packed operand blocks: per layer the gate rows r, z
// of W_ih (2m x kx) and W_hh (2m x m), the n rows of W_ih (m x kx) and W_hh
// (m x m); then W1 (128 x m, only with the hidden dense layer) and W2
// (nout x K2)
struct PackLayout {
  size_t rz[kMaxLayers], in[kMaxLayers], hrz[kMaxLayers], hn[kMaxLayers], w1, w2, total;
  int kx[kMaxLayers];
  __host__ __device__ static PackLayout of(const NetDims& d) {
    PackLayout p{};
    const size_t H = d.hidden;
    size_t o = 0;
    for (int l = 0; l < d.layers; ++l) {
      p.kx[l] = l == 0 ? d.kx0() : d.hidden;
      p.rz[l] = o;  o += 2 * H * p.kx[l];
      p.in[l] = o;  o += H * p.kx[l];
      p.hrz[l] = o; o += 2 * H * H;
      p.hn[l] = o;  o += H * H;
    }
    p.w1 = o; o += d.mlp ? (size_t)128 * H : 0;
    p.w2 = o; o += (size_t)d.nout() * d.k2();
    p.total = o;
    return p;
  }
};

// Per (step, patch) activations saved by the training forward pass (FP32):
// the new hidden state of every layer, the gates (r, z, n and the hidden
// part of n incl. bias, m each) of every layer and the pre-activation of the
// hidden dense layer.
__host__ __device__ constexpr int act_h(int H, int l) { return l * H; }
__host__ __device__ constexpr int act_g(int H, int NL, int l) { return NL * H + 4 * H * l; }
__host__ __device__ constexpr int act_a1(int H, int NL) { return 5 * NL * H; }
__host__ __device__ constexpr int act_size(int H, int NL) { return 5 * NL * H + 128; }

// Buffers of one training step for B sequences of T steps.  Columns of the
// transposed BF16 streams are indexed t * B + b; every hT[l] holds a leading
// block of B zero columns so that the previous step's state of column
// t * B + b is at the same column of the unshifted view.  Row C_in of xT,
// row m of every hT[l] and row 128 of y1T hold ones (bias gradients).
struct TrainBufs {
  float* act = nullptr;                   // [T][B][act_size]
  uint16_t* xT = nullptr;                 // [kx0 + 16][T B]
  uint16_t* hT[kMaxLayers] = {};          // [m + 16][(T+1) B]
  uint16_t* y1T = nullptr;                // [144][T B]
};

// Shared-memory bytes of the forward and backward kernels (0 if the shape
// has no kernel).
size_t patchnet_forward_smem(const NetDims& d);
size_t patchnet_backward_smem(const NetDims& d);
bool net_supported(const NetDims& d);
// master FP32 flat weights -> packed BF16 operands + fused biases
void launch_pack_weights(const NetDims& d, const float* w, PackedNet& pk, cudaStream_t st);
// one recurrent step for P patches: x [P][C_in] BF16, h [layers][P][m] FP32
// in, h_out [layers][P][m] (may alias h), out [P][C_out] FP32
void launch_patchnet_forward(const NetDims& d, const PackedNet& pk, const uint16_t* x,
                             const float* h, float* h_out, float* out, int P, int* status,
                             cudaStream_t st);
// training forward over T steps from a zero hidden state, saving activations
void launch_patchnet_train_forward(const NetDims& d, const PackedNet& pk, const uint16_t* x, int B,
                                   int T, float* ypred, const TrainBufs& tb, int* status,
                                   cudaStream_t st);
// C[M x N] = A[M x K] * B[N x K]^T (BF16 row-major inputs, FP32 row-major out)
int launch_umma_gemm(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                     int* status, cudaStream_t st);

}  // namespace dnnmg
