// Device bodies of the DNN-MG correction (the network correction of Algorithm 1), shared by
// the single-problem kernels (dnnmg_step.cu) and the batched kernels
// (batch.cu).
//
// A patch is one fluid cell (I, J) of the finest solved level L; with r
// replaced levels it covers the K x K nodes (S I + s, S J + t), s, t in
// 0..S, of level L + r, with S = 2^r and K = S + 1 (local index
// m = s + K t): 3x3 nodes for one replaced level, 5x5 for two.  Input
// features per patch (C_in = 4 K^2 + 4: 40 or 104):
//   prolongated u at the K^2 nodes, prolongated v, fine residual of the u
//   rows, of the v rows, then h_L / 0.25, aspect ratio h_x/h_y = 1, Peclet
//   number |mean prolongated velocity over the patch| * h_L / nu, k / h_L,
// each standardised as (value - mean) / std and rounded to bfloat16.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace dnnmg {

// constrained DOFs of node (i, j) of a level state get their Dirichlet values
__device__ __forceinline__ void impose_dirichlet_node(const Grid& g, double* __restrict__ x, int i,
                                                      int j) {
  const int n = j * g.nnx + i;
  const uint8_t f = g.flags[n];
  if (f & kVDir) {
    const double y = j * g.h;
    x[n] = (i == 0) ? 6.0 * y * (1.0 - y) : 0.0;
    x[g.nn + n] = 0.0;
  }
  if (f & kPFix) x[2 * g.nn + n] = 0.0;
}

// Per-launch constants of the patch features: h_L / 0.25, k / h_L and the
// factor h_L / (K^2 nu) of the Peclet number |sum of the patch's velocities|
// h_L / (K^2 nu) (formed once on the host: no FP64 division per patch).
struct FeatConsts {
  float h_rel, k_rel, pe;
};
inline FeatConsts feat_consts(double hL, double nu, double dt, int K) {
  return FeatConsts{(float)(hL / 0.25), (float)(dt / hL), (float)(hL / ((double)(K * K) * nu))};
}

// The network inputs of the patch on level-L cell `cell` whose K x K nodes
// (K = 2^r + 1 for r replaced levels: 3 or 5) lie on level L + r, in the
// order [u at the K^2 nodes, v, residual u, residual v, h_L / 0.25,
// aspect ratio 1, Peclet number, k / h_L] (4 K^2 + 4 values): standardised
// BF16 into X or, if RAW, unstandardised FP32 into Xraw.
template <bool RAW, int K>
__device__ __forceinline__ void gather_patch(const Grid& gL, const Grid& gF, int cell,
                                             const double* __restrict__ xt,
                                             const double* __restrict__ r,
                                             const float* __restrict__ mean,
                                             const float* __restrict__ stdv, const FeatConsts& fc,
                                             uint16_t* __restrict__ X, float* __restrict__ Xraw) {
  constexpr int K2 = K * K, C = 4 * K2 + 4, S = K - 1;
  const int I = cell % gL.nx, J = cell / gL.nx;
  float f[C];
  // the Peclet feature from the FP32 velocities (the features are rounded to
  // BF16; FP64 sums and square roots per patch would cost far more here)
  float su = 0.0f, sv = 0.0f;
#pragma unroll
  for (int m = 0; m < K2; ++m) {
    const int n = (S * J + m / K) * gF.nnx + S * I + m % K;
    const float u = (float)xt[n], v = (float)xt[gF.nn + n];
    su += u;
    sv += v;
    f[m] = u;
    f[K2 + m] = v;
    f[2 * K2 + m] = (float)r[n];
    f[3 * K2 + m] = (float)r[gF.nn + n];
  }
  f[4 * K2] = fc.h_rel;
  f[4 * K2 + 1] = 1.0f;
  f[4 * K2 + 2] = sqrtf(su * su + sv * sv) * fc.pe;
  f[4 * K2 + 3] = fc.k_rel;
  if (RAW) {
#pragma unroll
    for (int k = 0; k < C; ++k) Xraw[k] = f[k];
    return;
  }
  // C = 40 or 104 BF16 values, a multiple of 8: 16-byte stores
  static_assert(C % 8 == 0, "patch row of whole 16-byte chunks");
#pragma unroll
  for (int q = 0; q < C / 8; ++q) {
    uint32_t wv[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int k = 8 * q + 2 * h;
      const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn((f[k] - mean[k]) / stdv[k]));
      const uint32_t hi =
          __bfloat16_as_ushort(__float2bfloat16_rn((f[k + 1] - mean[k + 1]) / stdv[k + 1]));
      wv[h] = lo | (hi << 16);
    }
    reinterpret_cast<uint4*>(X)[q] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// v_corr = xt + d at fine node (i, j), d = mean of the predictions of the
// patches containing the node (K x K-node patches, K = 3 or 5), zero on
// velocity Dirichlet nodes; pressure 0.
template <int K>
__device__ __forceinline__ void scatter_node(const Grid& gL, const Grid& gF,
                                             const int* __restrict__ cell_patch,
                                             const float* __restrict__ out, int c_out,
                                             const double* __restrict__ xt,
                                             double* __restrict__ vcorr, int i, int j) {
  constexpr int S = K - 1, K2 = K * K;
  const int n = j * gF.nnx + i;
  // the mean of the (FP32) predictions in FP32; only the sum with the
  // prolongated state in FP64 (FP64 work per node is costly on this GPU)
  float du = 0.0f, dv = 0.0f;
  int cnt = 0;
  for (int dJ = 0; dJ < 2; ++dJ) {
    const int J = j / S - dJ;
    if (J < 0 || J >= gL.ny || j - S * J > S) continue;
    for (int dI = 0; dI < 2; ++dI) {
      const int I = i / S - dI;
      if (I < 0 || I >= gL.nx || i - S * I > S) continue;
      const int p = cell_patch[J * gL.nx + I];
      if (p < 0) continue;
      const int m = (i - S * I) + K * (j - S * J);
      du += out[(size_t)p * c_out + m];
      dv += out[(size_t)p * c_out + K2 + m];
      ++cnt;
    }
  }
  // the mean; counts 1, 2 and 4 scale by exact powers of two (the same
  // result as the division)
  if (cnt == 0 || (gF.flags[n] & kVDir)) {
    du = dv = 0.0f;
  } else if (cnt == 3) {
    du /= 3.0f, dv /= 3.0f;
  } else {
    const float sc = cnt == 4 ? 0.25f : (cnt == 2 ? 0.5f : 1.0f);
    du *= sc, dv *= sc;
  }
  vcorr[n] = xt[n] + (double)du;
  vcorr[gF.nn + n] = xt[gF.nn + n] + (double)dv;
  vcorr[2 * gF.nn + n] = 0.0;
}

// Training target of a patch: (next fine velocity - prolongated velocity)
// at its K x K nodes, zero on velocity Dirichlet nodes.
template <int K>
__device__ __forceinline__ void target_patch(const Grid& gL, const Grid& gF, int cell,
                                             const double* __restrict__ xnext,
                                             const double* __restrict__ xt,
                                             float* __restrict__ Y) {
  constexpr int S = K - 1, K2 = K * K;
  const int I = cell % gL.nx, J = cell / gL.nx;
#pragma unroll
  for (int m = 0; m < K2; ++m) {
    const int n = (S * J + m / K) * gF.nnx + S * I + m % K;
    const bool dir = gF.flags[n] & kVDir;
    Y[m] = dir ? 0.0f : (float)(xnext[n] - xt[n]);
    Y[K2 + m] = dir ? 0.0f : (float)(xnext[gF.nn + n] - xt[gF.nn + n]);
  }
}

}  // namespace dnnmg
