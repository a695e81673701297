// Small-matrix steps of flexible GMRES (Sec. 2.2), shared by the
// single-problem kernels (vec.cu) and the batched kernels (batch.cu).
#pragma once
#include <cuda_runtime.h>

namespace dnnmg {

// Sum of v over the block in a fixed order (warp shuffles, then warp 0);
// the result is valid in thread 0.  sh holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Hessenberg column j (H column-major, ldh rows) from hcol = [h_0..h_j (first
// CGS pass), h_0..h_j (second pass), ||w||^2]; the previous Givens rotations
// are applied, the new one is stored in (cs[j], sn[j]) and g is rotated.
// Returns the residual estimate |g[j+1]|.
__device__ __forceinline__ double givens_column(double* H, int ldh, double* cs, double* sn,
                                                double* g, const double* hcol, int j) {
  double* col = H + (size_t)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = hcol[i] + hcol[j + 1 + i];
  col[j + 1] = sqrt(fmax(hcol[2 * j + 2], 0.0));
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  const double c = den > 0 ? col[j] / den : 1.0, s = den > 0 ? col[j + 1] / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  return fabs(g[j + 1]);
}

// y = H[0:k, 0:k]^{-1} g[0:k] by back substitution (upper triangular H)
__device__ __forceinline__ void backsolve_small(const double* H, int ldh, const double* g, int k,
                                                double* y) {
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int c = i + 1; c < k; ++c) acc -= H[(size_t)c * ldh + i] * y[c];
    const double d = H[(size_t)i * ldh + i];
    y[i] = d != 0.0 ? acc / d : 0.0;
  }
}

}  // namespace dnnmg
