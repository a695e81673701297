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
  float h_rel, k_rel;
  double pe;
};
inline FeatConsts feat_consts(double hL, double nu, double dt, int K) {
  return FeatConsts{(float)(hL / 0.25), (float)(dt / hL), hL / ((double)(K * K) * nu)};
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
  double su = 0, sv = 0;
#pragma unroll
  for (int m = 0; m < K2; ++m) {
    const int n = (S * J + m / K) * gF.nnx + S * I + m % K;
    const double u = xt[n], v = xt[gF.nn + n];
    su += u;
    sv += v;
    f[m] = (float)u;
    f[K2 + m] = (float)v;
    f[2 * K2 + m] = (float)r[n];
    f[3 * K2 + m] = (float)r[gF.nn + n];
  }
  f[4 * K2] = fc.h_rel;
  f[4 * K2 + 1] = 1.0f;
  f[4 * K2 + 2] = (float)(sqrt(su * su + sv * sv) * fc.pe);
  f[4 * K2 + 3] = fc.k_rel;
  if (RAW) {
#pragma unroll
    for (int k = 0; k < C; ++k) Xraw[k] = f[k];
    return;
  }
#pragma unroll
  for (int k = 0; k < C; ++k)
    X[k] = __bfloat16_as_ushort(__float2bfloat16_rn((f[k] - mean[k]) / stdv[k]));
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
  double du = 0, dv = 0;
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
  // result as the division, without an FP64 division per node)
  if (cnt == 0 || (gF.flags[n] & kVDir)) {
    du = dv = 0.0;
  } else if (cnt == 3) {
    du /= 3.0, dv /= 3.0;
  } else {
    const double sc = cnt == 4 ? 0.25 : (cnt == 2 ? 0.5 : 1.0);
    du *= sc, dv *= sc;
  }
  vcorr[n] = xt[n] + du;
  vcorr[gF.nn + n] = xt[gF.nn + n] + dv;
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
