// Training kernels of the patch network (internal to libdnnmg).
#pragma once
#include <cstddef>
#include <cstdint>

#include "patchnet.cuh"

namespace dnnmg {

// Element offsets of the transposed BF16 weight operands used by the
// backward pass (B operands of dY W2, dA1 W1 (with the hidden dense layer),
// dG_h W_hh of every layer and dG_i W_ih of the layers above the first; m =
// hidden size).
struct BwdPack {
  size_t w2t, w1t, whh[kMaxLayers], wih[kMaxLayers], total;
  __host__ __device__ static BwdPack of(const NetDims& d) {
    BwdPack p{};
    const size_t H = d.hidden;
    size_t o = 0;
    p.w2t = o; o += (size_t)d.k2() * d.nout();      // [K2][nout]   W2^T
    p.w1t = o; o += d.mlp ? H * 128 : 0;             // [m][128]     W1^T (hidden dense layer)
    for (int l = 0; l < d.layers; ++l) {     // [m][3m]      W_hh^T
      p.whh[l] = o;
      o += H * 3 * H;
    }
    for (int l = 1; l < d.layers; ++l) {     // [m][3m]      W_ih^T (layers >= 1)
      p.wih[l] = o;
      o += H * 3 * H;
    }
    p.total = o;
    return p;
  }
};

// rows of the transposed gate-gradient streams: 3m rounded up to the 128-row
// tiles of the weight-gradient GEMM (the rows above 3m stay zero)
inline int gate_rows(const NetDims& d) { return (3 * d.hidden + 127) / 128 * 128; }

struct BwdArgs {
  const float* act;      // [T][B][act_size] from the training forward
  const float* ypred;    // [B][T][C_out]
  const float* Y;        // [B][T][C_out] targets
  int B, T;
  float scale;           // 2 / (B T C_out)
  uint16_t* dyT;         // [128][T B]   rows >= C_out stay zero
  uint16_t* da1T;        // [128][T B]
  uint16_t* giT[kMaxLayers];  // [gate_rows][T B]  dG_i of layer l (r, z, n)
  uint16_t* ghT[kMaxLayers];  // [gate_rows][T B]  dG_h of layer l (r, z, r * dn)
  double* loss_partial;  // [gridDim]
  int* status;
};

void launch_pack_backward(const NetDims& d, const float* w, uint16_t* wT, cudaStream_t st);
void launch_patchnet_backward(const NetDims& d, const uint16_t* wT, const BwdArgs& a, int nblocks,
                              cudaStream_t st);
// One weight-gradient product dW = A B^T over the K = steps x patches
// columns (A [M][lda], B [N][ldb], BF16, row-major); rows >= m_valid and
// columns >= n_valid of the product are padding, column bias_col of B holds
// ones so that column gives the bias gradient.
struct WGradJob {
  const uint16_t* A;
  const uint16_t* B;
  size_t lda, ldb;
  int M, N;  // M a multiple of 128, N a multiple of 16, <= 144
  int m_valid, n_valid, bias_col;
  float* gw;  // [m_valid][n_valid]
  float* gb;  // [m_valid]
};
constexpr int kMaxWGradJobs = 8;
struct WGradArgs {
  WGradJob job[kMaxWGradJobs];
  long long coff[kMaxWGradJobs];  // offset of each job's partial sums
  int first[kMaxWGradJobs + 1];   // first block of each job
  int eoff[kMaxWGradJobs + 1];    // first reduced element of each job
  int njobs, K, Ks, splits;
};
// All jobs' products, the K range split `splits` ways into partial sums
// (Cpart: wgrad_partials() floats), then reduced in a fixed order.  Returns
// nonzero on an unsupported shape.
int launch_wgrad(const WGradJob* jobs, int njobs, int K, int splits, float* Cpart, int* status,
                 cudaStream_t st);
size_t wgrad_partials(const WGradJob* jobs, int njobs, int K, int splits);
void launch_loss(const double* part, int n, double inv, float* out, cudaStream_t st);
void launch_adam(float* w, const float* g, float* m, float* v, size_t n, float lr, int step,
                 cudaStream_t st);

}  // namespace dnnmg
