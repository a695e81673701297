// Kernels of the DNN-MG correction (the network correction of Algorithm 1, Sec. 2.2):
// network input gathering per patch, scatter-averaging of the predicted
// corrections to the fine nodes, and boundary values of prolongated states.
//
// A patch is one fluid cell (I, J) of the finest solved level L; with one
// replaced level it covers the 3x3 nodes (2I+s, 2J+t), s, t in 0..2, of
// level L+1 (local index m = s + 3t).  Input features per patch (C_in = 40):
//   [0,9)  prolongated u at the 9 nodes      [9,18)  prolongated v
//   [18,27) fine residual of the u rows       [27,36) fine residual of v rows
//   36: h_L / 0.25   37: aspect ratio h_x/h_y = 1   38: Peclet number
//   |mean prolongated velocity over the patch| * h_L / nu   39: k / h_L
// each standardised as (value - mean) / std and rounded to bfloat16.
#include <cuda_bf16.h>

#include "dnnmg_body.cuh"
#include "dnnmg_step.h"

namespace dnnmg {

namespace {

constexpr int kBX = 32, kBY = 4;

__global__ void impose_dirichlet_kernel(Grid g, double* __restrict__ x) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  impose_dirichlet_node(g, x, i, j);
}

template <bool RAW, int K>
__global__ void gather_kernel(Grid gL, Grid gF, const int* __restrict__ patch_cell, int P,
                              const double* __restrict__ xt, const double* __restrict__ r,
                              const float* __restrict__ mean, const float* __restrict__ stdv,
                              FeatConsts fc, uint16_t* __restrict__ X,
                              float* __restrict__ Xraw) {
  constexpr int C = 4 * K * K + 4;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  gather_patch<RAW, K>(gL, gF, patch_cell[p], xt, r, mean, stdv, fc,
                       RAW ? nullptr : X + (size_t)p * C, RAW ? Xraw + (size_t)p * C : nullptr);
}

template <int K>
__global__ void target_kernel(Grid gL, Grid gF, const int* __restrict__ patch_cell, int P,
                              const double* __restrict__ xnext, const double* __restrict__ xt,
                              float* __restrict__ Y) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  target_patch<K>(gL, gF, patch_cell[p], xnext, xt, Y + (size_t)p * 2 * K * K);
}

// Per-feature sums (x, x^2) over row chunks: partial[block][C][2] (FP64).
__global__ void feature_sums_kernel(const float* __restrict__ X, long long rows, int C,
                                    double* __restrict__ partial) {
  extern __shared__ double sh[];  // [C][2] per warp: blockDim/32 * C * 2
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long chunk = (rows + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk, hi = min(rows, lo + chunk);
  for (int c = lane; c < C; c += 32) {
    double s = 0, q = 0;
    for (long long r = lo + warp; r < hi; r += nw) {
      const double v = X[r * C + c];
      s += v;
      q += v * v;
    }
    sh[(warp * C + c) * 2] = s;
    sh[(warp * C + c) * 2 + 1] = q;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double s = 0, q = 0;
    for (int w = 0; w < nw; ++w) s += sh[(w * C + c) * 2], q += sh[(w * C + c) * 2 + 1];
    partial[((size_t)blockIdx.x * C + c) * 2] = s;
    partial[((size_t)blockIdx.x * C + c) * 2 + 1] = q;
  }
}

__global__ void feature_stats_kernel(const double* __restrict__ partial, int nb, int C,
                                     long long rows, float* __restrict__ mean,
                                     float* __restrict__ stdv) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double s = 0, q = 0;
    for (int b = 0; b < nb; ++b) s += partial[((size_t)b * C + c) * 2], q += partial[((size_t)b * C + c) * 2 + 1];
    const double m = s / (double)rows;
    const double var = fmax(q / (double)rows - m * m, 0.0);
    const double sd = sqrt(var);
    mean[c] = (float)m;
    stdv[c] = sd > 1e-6 * fmax(1.0, fabs(m)) ? (float)sd : 1.0f;  // constant features
  }
}

// Batch b = rows idx[b][0] + t * stride + idx[b][1] (t = 0..T-1) of the raw
// corpus, standardised and rounded to bfloat16; targets copied.
__global__ void gather_batch_kernel(const float* __restrict__ Xraw, const float* __restrict__ Yc,
                                    const int* __restrict__ idx, int B, int T, long long stride,
                                    int Ci, int Co, const float* __restrict__ mean,
                                    const float* __restrict__ stdv, uint16_t* __restrict__ Xb,
                                    float* __restrict__ Yb) {
  const long long total = (long long)B * T * (Ci + Co);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % (Ci + Co));
    const long long bt = e / (Ci + Co);
    const int t = (int)(bt % T), b = (int)(bt / T);
    const long long row = (long long)idx[2 * b] * stride + (long long)t * stride + idx[2 * b + 1];
    if (k < Ci)
      Xb[bt * Ci + k] = __bfloat16_as_ushort(
          __float2bfloat16_rn((Xraw[row * Ci + k] - mean[k]) / stdv[k]));
    else
      Yb[bt * Co + (k - Ci)] = Yc[row * Co + (k - Ci)];
  }
}

template <int K>
__global__ void scatter_kernel(Grid gL, Grid gF, const int* __restrict__ cell_patch,
                               const float* __restrict__ out, int c_out,
                               const double* __restrict__ xt, double* __restrict__ vcorr) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= gF.nnx || j >= gF.nny) return;
  scatter_node<K>(gL, gF, cell_patch, out, c_out, xt, vcorr, i, j);
}

inline dim3 grid_of(const Grid& g) { return dim3(cdiv(g.nnx, kBX), cdiv(g.nny, kBY)); }

}  // namespace

void launch_impose_dirichlet64(const Grid& g, double* x, cudaStream_t st) {
  note_launch();
  impose_dirichlet_kernel<<<grid_of(g), dim3(kBX, kBY), 0, st>>>(g, x);
}

void launch_gather(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                   const double* xt, const double* r, const float* mean, const float* stdv,
                   double nu, double dt, uint16_t* X, cudaStream_t st) {
  if (P <= 0) return;
  note_launch();
  const FeatConsts fc = feat_consts(gL.h, nu, dt, K);
  if (K == 5)
    gather_kernel<false, 5><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xt, r, mean,
                                                          stdv, fc, X, nullptr);
  else
    gather_kernel<false, 3><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xt, r, mean,
                                                          stdv, fc, X, nullptr);
}

void launch_gather_raw(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                       const double* xt, const double* r, double nu, double dt, float* Xraw,
                       cudaStream_t st) {
  if (P <= 0) return;
  note_launch();
  const FeatConsts fc = feat_consts(gL.h, nu, dt, K);
  if (K == 5)
    gather_kernel<true, 5><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xt, r, nullptr,
                                                         nullptr, fc, nullptr, Xraw);
  else
    gather_kernel<true, 3><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xt, r, nullptr,
                                                         nullptr, fc, nullptr, Xraw);
}

void launch_targets(const Grid& gL, const Grid& gF, int K, const int* patch_cell, int P,
                    const double* xnext, const double* xt, float* Y, cudaStream_t st) {
  if (P <= 0) return;
  note_launch();
  if (K == 5)
    target_kernel<5><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xnext, xt, Y);
  else
    target_kernel<3><<<cdiv(P, 128), 128, 0, st>>>(gL, gF, patch_cell, P, xnext, xt, Y);
}

void launch_feature_stats(const float* X, long long rows, int C, double* partial, int nb,
                          float* mean, float* stdv, cudaStream_t st) {
  note_launch();
  feature_sums_kernel<<<nb, 256, sizeof(double) * 8 * C * 2, st>>>(X, rows, C, partial);
  note_launch();
  feature_stats_kernel<<<1, 64, 0, st>>>(partial, nb, C, rows, mean, stdv);
}

void launch_gather_batch(const float* Xraw, const float* Yc, const int* idx, int B, int T,
                         long long stride, int Ci, int Co, const float* mean, const float* stdv,
                         uint16_t* Xb, float* Yb, cudaStream_t st) {
  note_launch();
  gather_batch_kernel<<<1024, 256, 0, st>>>(Xraw, Yc, idx, B, T, stride, Ci, Co, mean, stdv, Xb, Yb);
}

void launch_scatter(const Grid& gL, const Grid& gF, int K, const int* cell_patch, const float* out,
                    int c_out, const double* xt, double* vcorr, cudaStream_t st) {
  note_launch();
  if (K == 5)
    scatter_kernel<5><<<grid_of(gF), dim3(kBX, kBY), 0, st>>>(gL, gF, cell_patch, out, c_out, xt,
                                                              vcorr);
  else
    scatter_kernel<3><<<grid_of(gF), dim3(kBX, kBY), 0, st>>>(gL, gF, cell_patch, out, c_out, xt,
                                                              vcorr);
}

}  // namespace dnnmg
