// Device bodies of the DNN-MG correction (Algorithm 1 lines 6-9), shared by
// the single-problem kernels (dnnmg_step.cu) and the batched kernels
// (batch.cu).
//
// A patch is one fluid cell (I, J) of the finest solved level L; with one
// replaced level it covers the 3x3 nodes (2I+s, 2J+t), s, t in 0..2, of
// level L+1 (local index m = s + 3t).  Input features per patch (C_in = 40):
//   [0,9)  prolongated u at the 9 nodes      [9,18)  prolongated v
//   [18,27) fine residual of the u rows       [27,36) fine residual of v rows
//   36: h_L / 0.25   37: aspect ratio h_x/h_y = 1   38: Peclet number
//   |mean prolongated velocity over the patch| * h_L / nu   39: k / h_L
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

// the 40 network inputs of the patch on level-L cell `cell`: standardised
// BF16 into X[0..40) or, if RAW, unstandardised FP32 into Xraw[0..40)
template <bool RAW>
__device__ __forceinline__ void gather_patch(const Grid& gL, const Grid& gF, int cell,
                                             const double* __restrict__ xt,
                                             const double* __restrict__ r,
                                             const float* __restrict__ mean,
                                             const float* __restrict__ stdv, double nu, double dt,
                                             uint16_t* __restrict__ X, float* __restrict__ Xraw) {
  const int I = cell % gL.nx, J = cell / gL.nx;
  float f[40];
  double su = 0, sv = 0;
#pragma unroll
  for (int m = 0; m < 9; ++m) {
    const int n = (2 * J + m / 3) * gF.nnx + 2 * I + m % 3;
    const double u = xt[n], v = xt[gF.nn + n];
    su += u;
    sv += v;
    f[m] = (float)u;
    f[9 + m] = (float)v;
    f[18 + m] = (float)r[n];
    f[27 + m] = (float)r[gF.nn + n];
  }
  const double hL = gL.h;
  f[36] = (float)(hL / 0.25);
  f[37] = 1.0f;
  f[38] = (float)(sqrt(su * su + sv * sv) / 9.0 * hL / nu);
  f[39] = (float)(dt / hL);
  if (RAW) {
#pragma unroll
    for (int k = 0; k < 40; ++k) Xraw[k] = f[k];
    return;
  }
#pragma unroll
  for (int k = 0; k < 40; ++k)
    X[k] = __bfloat16_as_ushort(__float2bfloat16_rn((f[k] - mean[k]) / stdv[k]));
}

// v_corr = xt + d at fine node (i, j), d = mean of the predictions of the
// patches containing the node, zero on velocity Dirichlet nodes; pressure 0.
__device__ __forceinline__ void scatter_node(const Grid& gL, const Grid& gF,
                                             const int* __restrict__ cell_patch,
                                             const float* __restrict__ out, int c_out,
                                             const double* __restrict__ xt,
                                             double* __restrict__ vcorr, int i, int j) {
  const int n = j * gF.nnx + i;
  double du = 0, dv = 0;
  int cnt = 0;
  for (int dJ = 0; dJ < 2; ++dJ) {
    const int J = (j >> 1) - dJ;
    if (J < 0 || J >= gL.ny || j - 2 * J > 2) continue;
    for (int dI = 0; dI < 2; ++dI) {
      const int I = (i >> 1) - dI;
      if (I < 0 || I >= gL.nx || i - 2 * I > 2) continue;
      const int p = cell_patch[J * gL.nx + I];
      if (p < 0) continue;
      const int m = (i - 2 * I) + 3 * (j - 2 * J);
      du += out[(size_t)p * c_out + m];
      dv += out[(size_t)p * c_out + 9 + m];
      ++cnt;
    }
  }
  if (cnt == 0 || (gF.flags[n] & kVDir)) du = dv = 0.0;
  else du /= cnt, dv /= cnt;
  vcorr[n] = xt[n] + du;
  vcorr[gF.nn + n] = xt[gF.nn + n] + dv;
  vcorr[2 * gF.nn + n] = 0.0;
}

}  // namespace dnnmg
