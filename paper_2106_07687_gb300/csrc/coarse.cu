// Direct solve on the coarsest multigrid level: launchers of the assembly,
// banded LU, explicit inverse and the dense solve (bodies in coarse_body.cuh).
#include <cooperative_groups.h>
#include <cstdio>

#include "coarse_body.cuh"
#include "kernels.h"

namespace dnnmg {

namespace {

// One thread per row of the coarse Jacobian.
__global__ void assemble_kernel(Grid g, Sten<double> s, const double* __restrict__ vb,
                                double* __restrict__ ab, const __grid_constant__ PatchPieces pp,
                                int use_pieces) {
  assemble_row(g, s, vb, ab, blockIdx.x * blockDim.x + threadIdx.x, use_pieces ? &pp : nullptr);
}

void launch_assemble(const Grid& g, const Sten<double>& s, const double* vb, double* ab,
                     const PatchPieces* pp, cudaStream_t st) {
  static const PatchPieces none{};
  note_launch();
  assemble_kernel<<<cdiv(band_of(g).n, 128), 128, 0, st>>>(g, s, vb, ab, pp ? *pp : none,
                                                            pp ? 1 : 0);
}

__global__ void __launch_bounds__(kLUThreads)
    band_lu_kernel(Grid g, double* __restrict__ ab, int* __restrict__ piv, int* status) {
  extern __shared__ double win[];  // kWin * W
  band_lu_block(g, ab, piv, status, win);
}

// The same banded LU (dgbtf2 ordering, partial pivoting, lowest row on
// ties, multipliers in place) by a cluster of kLUCluster CTAs.  The columns
// are dealt to the CTAs in panels of two (panel j = columns 2j, 2j + 1 in
// CTA j % kLUCluster) and stay in its shared memory for the whole
// factorisation, entry (r, c) at position r - c + ku + kl of the column (the
// kl subdiagonals, the diagonal and the ku + kl superdiagonals of U with
// fill-in).  Warp 0 of a panel's owner factors it: pivot of the first
// column, its step applied to the second column, pivot of the second; it
// writes both pivots and multiplier columns into every CTA's shared memory
// (double-buffered by panel parity).  After one cluster barrier per panel,
// every CTA applies the panel's two steps (row interchange, rank-1 update) to
// its columns right of the panel, one warp per column; the next panel's
// owner does its own panel columns first (warp 0) and factors them while its
// other warps finish.  Every entry sees the same floating-point operations
// in the same order as in band_lu_block, so the factors are the same.
namespace cg = cooperative_groups;
constexpr int kLUCluster = 8;
constexpr int kLUCThreads = 256;

__host__ __device__ inline int lu_cluster_cols(const Band& b) {
  const int panels = (b.n + 1) / 2;
  return 2 * ((panels + kLUCluster - 1) / kLUCluster);
}
__host__ __device__ inline size_t lu_cluster_smem(const Band& b) {
  return sizeof(double) * ((size_t)lu_cluster_cols(b) * b.W + 4 * (b.kl + 1)) + 4 * sizeof(int);
}

__device__ __forceinline__ void cl_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__global__ void __launch_bounds__(kLUCThreads)
    band_lu_cluster_kernel(Grid g, double* __restrict__ ab, int* __restrict__ piv, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const Band bd = band_of(g);
  const int q = (int)cl.block_rank();
  const int n = bd.n, kl = bd.kl, KU2 = bd.ku + bd.kl, W = bd.W;
  const int ncl = lu_cluster_cols(bd);
  const int NP = (n + 1) / 2;  // panels
  extern __shared__ __align__(16) double lsm[];
  double* cols = lsm;                                  // [ncl][W]
  double* mult = lsm + (size_t)ncl * W;                // [2 parity][2 step][kl + 1]
  int* pv = reinterpret_cast<int*>(mult + 4 * (kl + 1));  // [2 parity][2 step]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kLUCThreads / 32;
  // local slot of (owned) column c: panel c / 2 is the (c / 2 / kLUCluster)-th of this CTA
  auto slot = [&](int c) { return ((c >> 1) / kLUCluster) * 2 + (c & 1); };
  auto A = [&](int r, int c) -> double& { return cols[(size_t)slot(c) * W + (r - c + KU2)]; };
  auto col_of = [&](int lc) { return ((lc >> 1) * kLUCluster + q) * 2 + (lc & 1); };
  // this CTA's columns from the row-major band: (r, c) at ab[r W + c - r + kl]
  for (int e = tid; e < ncl * W; e += kLUCThreads) {
    const int lc = e / W, t = e % W;
    const int c = col_of(lc), r = c - KU2 + t;
    cols[e] = (c < n && r >= 0 && r < n) ? ab[(size_t)r * W + (W - 1 - t)] : 0.0;
  }
  __syncthreads();
  // step k applied to column c (one warp): rows k and p interchanged, then
  // rows k+1 .. k+kl minus multiplier times the new row-k entry
  auto apply = [&](int k, int p, const double* m, int c) {
    const double a = A(k, c), b = A(p, c);
    __syncwarp();
    if (lane == 0 && p != k) {
      A(k, c) = b;
      A(p, c) = a;
    }
    __syncwarp();
    const int rmax = min(n - 1, k + kl);
    for (int r = k + 1 + lane; r <= rmax; r += 32) A(r, c) -= m[r - k - 1] * b;
    __syncwarp();
  };
  // pivot of column k (owned here, up to date): |entries| compared as the
  // bit patterns of non-negative doubles (the same order), lowest row on
  // ties; multipliers in place and into slot `sl` of every CTA.  One warp.
  auto pivot = [&](int k, double* mloc, int sl) {
    const int rmax = min(n - 1, k + kl);
    long long best = -1;
    int bi = k;
    for (int r = k + lane; r <= rmax; r += 32) {
      const long long v = __double_as_longlong(A(r, k)) & 0x7FFFFFFFFFFFFFFFLL;
      if (v > best) best = v, bi = r;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
    }
    const int p = __shfl_sync(0xffffffffu, bi, 0);
    best = __shfl_sync(0xffffffffu, best, 0);
    const double d = A(p, k), akk = A(k, k);
    const double id = d != 0.0 ? 1.0 / d : 0.0;
    __syncwarp();
    for (int r = k + 1 + lane; r <= rmax; r += 32) {
      const double m = (r == p ? akk : A(r, k)) * id;
      A(r, k) = m;
      mloc[r - k - 1] = m;
      for (int dst = 0; dst < kLUCluster; ++dst)
        if (dst != q) cl.map_shared_rank(mloc, dst)[r - k - 1] = m;
    }
    if (lane == 0) {
      A(k, k) = d;
      piv[k] = p;
      pv[sl] = p;
      for (int dst = 0; dst < kLUCluster; ++dst)
        if (dst != q) cl.map_shared_rank(pv, dst)[sl] = p;
      if (!(best > 0)) atomicOr(status, 2);
    }
    __syncwarp();
    return p;
  };
  // panel j by warp 0 of its owner: columns 2j (and 2j + 1)
  auto factor_panel = [&](int j) {
    const int k = 2 * j, par = j & 1;
    double* m0 = mult + (size_t)(2 * par) * (kl + 1);
    const int p0 = pivot(k, m0, 2 * par);
    if (k + 1 < n) {
      apply(k, p0, m0, k + 1);
      pivot(k + 1, m0 + (kl + 1), 2 * par + 1);
    }
  };
  if (q == 0 && warp == 0) factor_panel(0);
  cl_arrive();
  for (int J = 0; J < NP; ++J) {
    cl_wait();  // pivots and multipliers of panel J are in buffer J & 1
    const int k0 = 2 * J, par = J & 1;
    const double* m0 = mult + (size_t)(2 * par) * (kl + 1);
    const double* m1 = m0 + (kl + 1);
    const int p0 = pv[2 * par], p1 = pv[2 * par + 1];
    const bool two = k0 + 1 < n;
    // columns right of the panel that its steps reach: (k0 + 1, cmax]
    const int cmax = min(n - 1, (two ? k0 + 1 : k0) + KU2);
    auto both = [&](int c) {
      if (c <= k0 + KU2) apply(k0, p0, m0, c);
      if (two) apply(k0 + 1, p1, m1, c);
    };
    // this CTA's panels j in [J + 1, cmax / 2]
    const int j0 = J + 1, j1 = cmax >> 1;
    const int jf = j0 + ((q - j0 % kLUCluster) + kLUCluster) % kLUCluster;  // first owned
    const bool next_owner = J + 1 < NP && jf == J + 1;
    if (next_owner && warp == 0) {  // the next panel first, then factor it
      both(k0 + 2);
      if (k0 + 3 <= cmax) both(k0 + 3);
      factor_panel(J + 1);
    }
    // the other owned columns, one warp each
    const int w0 = next_owner ? 1 : 0;
    int idx = 0;  // running index over the owned columns (next panel excluded)
    for (int j = next_owner ? jf + kLUCluster : jf; j <= j1; j += kLUCluster)
      for (int h = 0; h < 2; ++h, ++idx) {
        const int c = 2 * j + h;
        if (c > cmax) break;
        if (warp >= w0 && idx % (kWarps - w0) == warp - w0) both(c);
      }
    cl_arrive();
  }
  cl_wait();
  // the factored columns back into the row-major band
  for (int e = tid; e < ncl * W; e += kLUCThreads) {
    const int lc = e / W, t = e % W;
    const int c = col_of(lc), r = c - KU2 + t;
    if (c < n && r >= 0 && r < n) ab[(size_t)r * W + (W - 1 - t)] = cols[e];
  }
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

// Banded LU of the assembled coarse Jacobian: the cluster kernel when a
// cluster of kLUCluster CTAs with its shared memory can be placed, else the
// single-block kernel.
void launch_band_lu(const Grid& g, double* ab, int* piv, int* status, cudaStream_t st) {
  const Band bd = band_of(g);
  const size_t csm = lu_cluster_smem(bd);
  // whether the cluster can be placed, checked once per process (thread-safe
  // initialisation of a function-local static)
  static const int cluster_ok = [&] {
    int ok = 0;
    if (csm <= 227 * 1024 &&
        cudaFuncSetAttribute(band_lu_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = kLUCluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(kLUCluster);
      cfg.blockDim = dim3(kLUCThreads);
      cfg.dynamicSmemBytes = csm;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, (void*)band_lu_cluster_kernel, &cfg) == cudaSuccess &&
          n > 0)
        ok = 1;
    }
    cudaGetLastError();
    return ok;
  }();
  if (cluster_ok == 1 && csm <= 227 * 1024) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLUCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kLUCluster);
    cfg.blockDim = dim3(kLUCThreads);
    cfg.dynamicSmemBytes = csm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch();
    if (cudaLaunchKernelEx(&cfg, band_lu_cluster_kernel, g, ab, piv, status) == cudaSuccess) return;
    cudaGetLastError();
  }
  const size_t win_bytes = sizeof(double) * kWin * bd.W;
  cudaFuncSetAttribute(band_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)win_bytes);
  note_launch();
  band_lu_kernel<<<1, kLUThreads, win_bytes, st>>>(g, ab, piv, status);
}

}  // namespace

size_t coarse_band_doubles(const Grid& g) {
  const Band bd = band_of(g);
  return (size_t)bd.n * bd.W;
}

void launch_coarse_lu(const Grid& g, const Sten<double>& s, const double* vb, double* band,
                      int* piv, int* status, cudaStream_t st) {
  launch_assemble(g, s, vb, band, nullptr, st);
  launch_band_lu(g, band, piv, status, st);
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
         bd.kl <= 64 && bd.ku + bd.kl <= 128 &&  // L and U entries of a step per lane
         sizeof(double) * inv_block_smem_doubles(bd.n) <= 200 * 1024;
}

size_t coarse_work_doubles(const Grid& g) {
  const Band bd = band_of(g);
  // band + pivots (as ints, over-allocated) + reciprocals of the U diagonal
  return (size_t)bd.n * bd.W + (size_t)bd.n + (size_t)bd.n;
}

void launch_coarse_factor(const Grid& g, const Sten<double>& s, const double* vb, double* work,
                          double* Ainv, int* status, cudaStream_t st, const PatchPieces* pp) {
  const Band bd = band_of(g);
  double* ab = work;
  int* piv = reinterpret_cast<int*>(work + (size_t)bd.n * bd.W);
  launch_assemble(g, s, vb, ab, pp, st);
  launch_band_lu(g, ab, piv, status, st);
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
