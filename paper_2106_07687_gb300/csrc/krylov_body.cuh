// Small-matrix steps of flexible GMRES (Sec. 2.2), shared by the
// single-problem kernels (vec.cu) and the batched kernels (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

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

// the values of a post are stored before the sequence number, with a
// system-scope fence between them (the host reads seq first)
__device__ __forceinline__ void mail_post(HostMail* m, unsigned long long seq) {
  __threadfence_system();
  m->seq = seq;
}

// One Arnoldi step of FGMRES for the new vector w against V[0..j]
// (Algorithm 1's Krylov solver: CGS with one re-orthogonalisation, then
// normalisation and the Givens update of Hessenberg column j).
template <typename T>
struct ArnoldiArgs {
  const T* V;
  size_t ld;
  int j;
  T* w;
  size_t n;
  double* partials;  // (2 j + 3) x gridDim.x doubles
  double* hcol;      // 2 j + 3
  double* H;
  int ldh;
  double *cs, *sn, *g, *resid;
  HostMail* mail;  // may be null
  unsigned long long seq;
  int slot;        // resid goes to mail->v[slot]
  // Device-side stop flag of a speculatively enqueued iteration (may be
  // null): the step does nothing if *skip is set when it starts, and sets
  // *skip itself when the cycle stops here, that is when resid <= *target,
  // its >= maxit (its counts this iteration) or resid is not finite: the
  // test the host applies to the posted value.
  int* skip;
  const double* target;
  int its, maxit;
};

// The step over all blocks of a cooperative grid with two grid barriers
// (sync): the second pass's products include <w, w>, and the norm of the
// re-orthogonalised vector follows from it as ||w||^2 - |h2|^2 (the columns
// of V are orthonormal).  Block b owns the b-th chunk of the elements: it
// updates only that chunk, so the second pass's and the norm's partial sums
// follow its own updates without a barrier, and every block finishes the
// sums over all partials itself in one fixed order (one warp per
// coefficient), so all blocks hold the same coefficients.  Products,
// updates and the sums within a warp (about a hundred products) are taken in
// the vectors' precision T, the sums over warps and blocks in FP64: on this
// GPU (FP64 at 1/64 of the FP32 rate) FP64 work per element, or per thread,
// would make the step FP64-bound.  NT threads
// per block; block 0 then rotates column j (resid = |g[j+1]|) and posts
// resid into mail->v[0] when mail is set.
template <typename T, int NT, class Sync>
__device__ __forceinline__ void arnoldi_body(const ArnoldiArgs<T>& a, Sync sync) {
  __shared__ double h[2][64];
  __shared__ double nrm2;
  __shared__ T hT[64];
  constexpr int kG = 8;  // dot products reduced together
  constexpr int kW = NT / 32;
  __shared__ double sg[kW][kG];
  if (a.skip && *reinterpret_cast<volatile int*>(a.skip)) return;  // the same in every block
  const T* __restrict__ V = a.V;
  T* __restrict__ w = a.w;
  const size_t ld = a.ld;
  const int j = a.j, k = j + 1, nb = (int)gridDim.x;
  const size_t chunk = (a.n + nb - 1) / nb;
  const size_t lo = blockIdx.x * chunk, hi = min(a.n, lo + chunk);
  double* p1 = a.partials;                    // [k][nb]
  double* p2 = a.partials + (size_t)k * nb;   // [k + 1][nb]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // per value of a group of gk <= kG dot products (this thread's sums in
  // acc): a shuffle tree in each warp in T, then a second tree over the
  // warps' sums in FP64 (the order of block_sum); the block's partial of
  // value i0 + u goes to part[(i0 + u) nb + block]
  auto reduce_group = [&](const T* acc, int gk, int i0, double* part) {
#pragma unroll
    for (int u = 0; u < kG; ++u) {
      if (u >= gk) break;
      T v = acc[u];  // the warp's sum in T, then FP64 from the block level on
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sg[warp][u] = (double)v;
    }
    __syncthreads();
    if (warp < gk) {  // warp u finishes value u
      double t = lane < kW ? sg[lane][warp] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) part[(size_t)(i0 + warp) * nb + blockIdx.x] = t;
    }
    __syncthreads();  // sg is rewritten by the next group
  };
  // the nk partial dot products <V[i], w> for i < nv and <w, w> for i >= nv
  // of this block's chunk, kG at a time in one pass over the elements
  // (products and per-thread sums in T)
  auto dots = [&](int nv, int nk, double* part) {
    for (int i0 = 0; i0 < nk; i0 += kG) {
      const int gk = min(kG, nk - i0);
      T acc[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) acc[u] = T(0);
      for (size_t e = lo + threadIdx.x; e < hi; e += NT) {
        const T we = w[e];
#pragma unroll
        for (int u = 0; u < kG; ++u)
          if (u < gk) acc[u] += (i0 + u < nv ? V[(size_t)(i0 + u) * ld + e] : we) * we;
      }
      reduce_group(acc, gk, i0, part);
    }
  };
  // out[i] = sum over the blocks' partials of row i, i < nk: one warp per
  // row, lane l adding partials l, l + 32, ... in order, then a shuffle
  // tree; the same fixed order in every block.  The loads of eight partials
  // are issued before they are added (one round trip to L2 per eight).
  auto finish = [&](const double* part, int nk, double* out) {
    for (int i = warp; i < nk; i += kW) {
      double t = 0.0;
      for (int b0 = lane; b0 < nb; b0 += 32 * 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int bb = b0 + 32 * u;
          v[u] = bb < nb ? part[(size_t)i * nb + bb] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) t += v[u];
      }
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) out[i] = t;
    }
    __syncthreads();
  };
  auto axpy = [&](const double* hh) {
    if (threadIdx.x < k) hT[threadIdx.x] = (T)hh[threadIdx.x];
    __syncthreads();
    for (size_t e = lo + threadIdx.x; e < hi; e += NT) {
      T acc = w[e];
      for (int i = 0; i < k; ++i) acc -= hT[i] * V[(size_t)i * ld + e];
      w[e] = acc;
    }
    __syncthreads();  // hT is rewritten by the next pass
  };
  auto norm_scale = [&]() -> T {
    if (threadIdx.x == 0) {
      double q = h[1][k];
      for (int i = 0; i < k; ++i) q -= h[1][i] * h[1][i];
      nrm2 = q;
    }
    __syncthreads();
    const double s = block_scalar([&] {
      const double v = sqrt(fmax(nrm2, 0.0));
      return v != 0.0 ? 1.0 / v : 0.0;
    });
    return (T)s;
  };
  // With few basis vectors, the thread's elements of w and of V[0..j] stay
  // in registers through both passes (one load of each, one store of w):
  // the same operations in the same order as the general path below, which
  // reloads them from L2 for every pass.
  // (the second pass's k + 1 products form one group of at most kG)
  constexpr int kRK = sizeof(T) == 4 ? kG - 1 : 4;  // basis vectors held in registers
  constexpr int kRE = 4;                       // elements per thread
  if (k <= kRK && hi - lo <= (size_t)kRE * NT) {
    T wr[kRE], vr[kRK][kRE];
    bool in[kRE];
#pragma unroll
    for (int q = 0; q < kRE; ++q) {
      const size_t e = lo + threadIdx.x + (size_t)q * NT;
      in[q] = e < hi;
      wr[q] = in[q] ? w[e] : T(0);
#pragma unroll
      for (int i = 0; i < kRK; ++i) vr[i][q] = (in[q] && i < k) ? V[(size_t)i * ld + e] : T(0);
    }
    auto rdots = [&](int nk, double* part) {  // <V[i], w> for i < k, then <w, w>
      T acc[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) acc[u] = T(0);
#pragma unroll
      for (int q = 0; q < kRE; ++q) {
        if (!in[q]) continue;
#pragma unroll
        for (int u = 0; u < kG; ++u)
          if (u < nk) acc[u] += (u < k && u < kRK ? vr[u < kRK ? u : 0][q] : wr[q]) * wr[q];
      }
      reduce_group(acc, nk, 0, part);
    };
    auto raxpy = [&](const double* hh) {
      if (threadIdx.x < k) hT[threadIdx.x] = (T)hh[threadIdx.x];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kRE; ++q) {
        T acc = wr[q];
#pragma unroll
        for (int i = 0; i < kRK; ++i)
          if (i < k) acc -= hT[i] * vr[i][q];
        wr[q] = acc;
      }
      __syncthreads();  // hT is rewritten by the next pass
    };
    rdots(k, p1);
    sync();
    finish(p1, k, h[0]);
    raxpy(h[0]);
    rdots(k + 1, p2);
    sync();
    finish(p2, k + 1, h[1]);  // h[1][k] = <w, w> before the second update
    raxpy(h[1]);
    const T sT = norm_scale();
#pragma unroll
    for (int q = 0; q < kRE; ++q)
      if (in[q]) w[lo + threadIdx.x + (size_t)q * NT] = wr[q] * sT;
  } else {
    dots(k, k, p1);
    sync();
    finish(p1, k, h[0]);
    axpy(h[0]);
    dots(k, k + 1, p2);
    sync();
    finish(p2, k + 1, h[1]);  // h[1][k] = <w, w> before the second update
    axpy(h[1]);
    const T sT = norm_scale();
    for (size_t e = lo + threadIdx.x; e < hi; e += NT) w[e] *= sT;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < k; ++i) a.hcol[i] = h[0][i], a.hcol[k + i] = h[1][i];
    a.hcol[2 * k] = nrm2;
    const double res = givens_column(a.H, a.ldh, a.cs, a.sn, a.g, a.hcol, j);
    *a.resid = res;
    // every block read *skip before the first grid barrier: setting it now
    // only affects the launches after this one
    if (a.skip) *a.skip = (res <= *a.target || a.its >= a.maxit || !isfinite(res)) ? 1 : 0;
    if (a.mail) {
      a.mail->v[a.slot] = res;
      mail_post(a.mail, a.seq);
    }
  }
}

}  // namespace dnnmg
