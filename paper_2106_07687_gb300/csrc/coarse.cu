// Direct solve on the coarsest multigrid level: launchers of the assembly,
// banded LU, explicit inverse and the dense solve (bodies in coarse_body.cuh).
#include <cstdio>

#include "coarse_body.cuh"
#include "kernels.h"

namespace dnnmg {

namespace {

// One thread per row of the coarse Jacobian.
__global__ void assemble_kernel(Grid g, Sten<double> s, const double* __restrict__ vb,
                                double* __restrict__ ab) {
  assemble_row(g, s, vb, ab, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(kLUThreads)
    band_lu_kernel(Grid g, double* __restrict__ ab, int* __restrict__ piv, int* status) {
  extern __shared__ double win[];  // kWin * W
  band_lu_block(g, ab, piv, status, win);
}

__global__ void diag_recip_kernel(Grid g, const double* __restrict__ ab, double* __restrict__ rd) {
  band_diag_recip(g, ab, rd, blockIdx.x * blockDim.x + threadIdx.x);
}

// Columns [kInvWarps * block, +kInvWarps) of the inverse.
__global__ void __launch_bounds__(32 * kInvWarps)
    band_inverse_kernel(Grid g, const double* __restrict__ ab, const int* __restrict__ piv,
                        const double* __restrict__ rd, double* __restrict__ Ainv) {
  extern __shared__ __align__(16) double sm[];
  band_inverse_block(g, ab, piv, rd, Ainv, blockIdx.x * kInvWarps, sm);
}

// x = Ainv b with the band numbering on both sides; one warp per row.
template <typename T>
__global__ void __launch_bounds__(32 * kSolveWarps)
    coarse_solve_kernel(Grid g, const double* __restrict__ Ainv, const T* __restrict__ b,
                        T* __restrict__ x) {
  extern __shared__ double sb[];
  coarse_solve_rows<T>(g, Ainv, b, x, blockIdx.x, sb);
}

// x = (LU)^{-1} b with the factors and pivots of band_lu_kernel; one block,
// b and x in the [3][nn] layout of the level, work in shared memory.
__global__ void __launch_bounds__(1024)
    band_solve_kernel(Grid g, const double* __restrict__ ab, const int* __restrict__ piv,
                      const double* __restrict__ b, double* __restrict__ x) {
  const Band bd = band_of(g);
  extern __shared__ double sx[];
  const int tid = threadIdx.x;
  for (int p = tid; p < bd.n; p += blockDim.x) sx[p] = b[lidx(g, p)];
  __syncthreads();
  for (int k = 0; k < bd.n; ++k) {
    const int p = piv[k];
    if (tid == 0 && p != k) {
      const double t = sx[k];
      sx[k] = sx[p];
      sx[p] = t;
    }
    __syncthreads();
    const double xk = sx[k];
    const int rmax = min(bd.n - 1, k + bd.kl);
    for (int r = k + 1 + tid; r <= rmax; r += blockDim.x)
      sx[r] -= ab[(size_t)r * bd.W + (k - r + bd.kl)] * xk;
    __syncthreads();
  }
  __shared__ double red[32];
  for (int k = bd.n - 1; k >= 0; --k) {
    const int cmax = min(bd.n - 1, k + bd.ku + bd.kl);
    double acc = 0.0;
    for (int c2 = k + 1 + tid; c2 <= cmax; c2 += blockDim.x)
      acc += ab[(size_t)k * bd.W + (c2 - k + bd.kl)] * sx[c2];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      sx[k] = (sx[k] - t) / ab[(size_t)k * bd.W + bd.kl];
    }
    __syncthreads();
  }
  for (int p = tid; p < bd.n; p += blockDim.x) x[lidx(g, p)] = sx[p];
}

}  // namespace

size_t coarse_band_doubles(const Grid& g) {
  const Band bd = band_of(g);
  return (size_t)bd.n * bd.W;
}

void launch_coarse_lu(const Grid& g, const Sten<double>& s, const double* vb, double* band,
                      int* piv, int* status, cudaStream_t st) {
  const Band bd = band_of(g);
  note_launch();
  assemble_kernel<<<cdiv(bd.n, 128), 128, 0, st>>>(g, s, vb, band);
  const size_t win_bytes = sizeof(double) * kWin * bd.W;
  cudaFuncSetAttribute(band_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)win_bytes);
  note_launch();
  band_lu_kernel<<<1, kLUThreads, win_bytes, st>>>(g, band, piv, status);
}

void launch_coarse_lu_solve(const Grid& g, const double* band, const int* piv, const double* b,
                            double* x, cudaStream_t st) {
  const Band bd = band_of(g);
  note_launch();
  band_solve_kernel<<<1, 1024, sizeof(double) * bd.n, st>>>(g, band, piv, b, x);
}

bool coarse_supported(const Grid& g) {
  const Band bd = band_of(g);
  return bd.kl + 2 <= kWin && bd.W <= kLUThreads && sizeof(double) * kWin * bd.W <= 200 * 1024 &&
         bd.kl <= kInvLW && bd.ku + bd.kl + 1 <= kInvUW &&
         sizeof(double) * inv_block_smem_doubles(bd.n) <= 200 * 1024;
}

size_t coarse_work_doubles(const Grid& g) {
  const Band bd = band_of(g);
  // band + pivots (as ints, over-allocated) + reciprocals of the U diagonal
  return (size_t)bd.n * bd.W + (size_t)bd.n + (size_t)bd.n;
}

void launch_coarse_factor(const Grid& g, const Sten<double>& s, const double* vb, double* work,
                          double* Ainv, int* status, cudaStream_t st) {
  const Band bd = band_of(g);
  double* ab = work;
  int* piv = reinterpret_cast<int*>(work + (size_t)bd.n * bd.W);
  note_launch();
  assemble_kernel<<<cdiv(bd.n, 128), 128, 0, st>>>(g, s, vb, ab);
  const size_t win_bytes = sizeof(double) * kWin * bd.W;
  cudaFuncSetAttribute(band_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)win_bytes);
  note_launch();
  band_lu_kernel<<<1, kLUThreads, win_bytes, st>>>(g, ab, piv, status);
  double* rd = work + (size_t)bd.n * bd.W + bd.n;
  note_launch();
  diag_recip_kernel<<<cdiv(bd.n, 128), 128, 0, st>>>(g, ab, rd);
  const size_t smem = sizeof(double) * inv_block_smem_doubles(bd.n);
  static const bool inv_attr =
      cudaFuncSetAttribute(band_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) == cudaSuccess;
  (void)inv_attr;
  note_launch();
  band_inverse_kernel<<<cdiv(bd.n, kInvWarps), 32 * kInvWarps, smem, st>>>(g, ab, piv, rd, Ainv);
}

template <typename T>
void launch_coarse_solve(const Grid& g, const double* Ainv, const T* b, T* x, cudaStream_t st) {
  const Band bd = band_of(g);
  note_launch();
  coarse_solve_kernel<T><<<cdiv(bd.n, kSolveWarps), 32 * kSolveWarps, sizeof(double) * bd.n, st>>>(
      g, Ainv, b, x);
}

template void launch_coarse_solve<float>(const Grid&, const double*, const float*, float*,
                                         cudaStream_t);
template void launch_coarse_solve<double>(const Grid&, const double*, const double*, double*,
                                          cudaStream_t);

}  // namespace dnnmg
