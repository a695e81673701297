// Device bodies of the coarsest-level direct solve (level 1, 32x8 cells),
// shared by the single-problem kernels (coarse.cu) and the batched kernels
// (batch.cu).
//
// The Jacobian of the coarsest level is assembled in FP64 into band storage
// with the unknowns numbered node-major along y, p = (i * nny + j) * 3 + c,
// which gives kl = ku = 6 * nny + 8.  It is factored by LU with partial
// pivoting (row interchanges, multipliers kept in place), then the explicit
// inverse is formed column by column.  A V-cycle's coarse solve is one dense
// FP64 matrix-vector product with that inverse.
#pragma once
#include "common.cuh"

namespace dnnmg {

struct Band {
  int n, kl, ku, W;  // W = 2 kl + ku + 1 stored columns per row
};

__host__ __device__ inline Band band_of(const Grid& g) {
  Band b;
  b.n = 3 * g.nn;
  b.kl = b.ku = 6 * g.nny + 8;
  b.W = 2 * b.kl + b.ku + 1;
  return b;
}

// band index of DOF (comp c, node (i, j)) and back
__host__ __device__ inline int bidx(const Grid& g, int c, int i, int j) {
  return (i * g.nny + j) * 3 + c;
}
__host__ __device__ inline int lidx(const Grid& g, int p) {
  const int c = p % 3, node = p / 3;
  const int i = node / g.nny, j = node % g.nny;
  return c * g.nn + j * g.nnx + i;
}

// entry (r, col) of the band matrix
__device__ __forceinline__ double& AB(double* ab, const Band& b, int r, int col) {
  return ab[(size_t)r * b.W + (col - r + b.kl)];
}

// Row `row` of the banded coarse Jacobian (one thread per row).
__device__ __forceinline__ void assemble_row(const Grid& g, const Sten<double>& s,
                                             const double* __restrict__ vb,
                                             double* __restrict__ ab, int row) {
  const Band bd = band_of(g);
  if (row >= bd.n) return;
  for (int k = 0; k < bd.W; ++k) ab[(size_t)row * bd.W + k] = 0.0;
  const int c = row % 3, node = row / 3;
  const int i = node / g.nny, j = node % g.nny;
  const uint8_t f = g.flags[j * g.nnx + i];
  const bool cons = (c < 2) ? (f & kVDir) : (f & kPFix);
  if (cons) {
    AB(ab, bd, row, row) = 1.0;
    return;
  }
  for (int cy = 0; cy < 2; ++cy)
    for (int cx = 0; cx < 2; ++cx) {
      const int ci = i - 1 + cx, cj = j - 1 + cy;
      if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny || g.solid[cj * g.nx + ci]) continue;
      const int al = (1 - cx) + 2 * (1 - cy);
      double bu[4], bv[4];
      load_cell<double, false>(g, vb, ci, cj, 0, bu);
      load_cell<double, false>(g, vb + g.nn, ci, cj, 0, bv);
      GaussData<double> gd;
      gauss_data<double>(bu, bv, gd);
      for (int be = 0; be < 4; ++be) {
        const int ni = ci + (be & 1), nj = cj + (be >> 1);
        const uint8_t fb = g.flags[nj * g.nnx + ni];
        double J[3][3];
        elem_pair<double>(s, gd, al, be, J);
        for (int c2 = 0; c2 < 3; ++c2) {
          const bool cons2 = (c2 < 2) ? (fb & kVDir) : (fb & kPFix);
          if (cons2) continue;
          AB(ab, bd, row, bidx(g, c2, ni, nj)) += J[c][c2];
        }
      }
    }
  if (c == 2) {
    for (int dJ = 0; dJ < 2; ++dJ) {
      const int PJ = (j >> 1) - dJ;
      if (PJ < 0 || PJ >= g.ny / 2 || j - 2 * PJ > 2) continue;
      for (int dI = 0; dI < 2; ++dI) {
        const int PI = (i >> 1) - dI;
        if (PI < 0 || PI >= g.nx / 2 || i - 2 * PI > 2) continue;
        if (g.solid[(2 * PJ) * g.nx + 2 * PI]) continue;
        const int mn = (i - 2 * PI) + 3 * (j - 2 * PJ);
        for (int m = 0; m < 9; ++m) {
          const int ni = 2 * PI + m % 3, nj = 2 * PJ + m / 3;
          if (g.flags[nj * g.nnx + ni] & kPFix) continue;
          AB(ab, bd, row, bidx(g, 2, ni, nj)) += s.S9[mn * 9 + m];
        }
      }
    }
  }
}

// Banded LU with partial pivoting in one thread block (dgbtf2 ordering).
// The rows k..k+kl that elimination step k touches live in a shared-memory
// window of kWin row slots (row r in slot r % kWin, same per-row band offset
// as in global memory); a row is loaded when it enters the window and written
// back once it is final.
// All kLUThreads threads of the block call it; win holds kWin * W doubles.
constexpr int kLUThreads = 1024;
constexpr int kWin = 64;
__device__ __forceinline__ void band_lu_block(const Grid& g, double* __restrict__ ab,
                                              int* __restrict__ piv, int* status, double* win) {
  const Band bd = band_of(g);
  __shared__ int s_p;
  __shared__ double s_d, s_akk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto W = [&](int r, int col) -> double& {
    return win[(size_t)(r % kWin) * bd.W + (col - r + bd.kl)];
  };
  // rows 0..kl enter the window
  for (int r = 0; r <= min(bd.kl, bd.n - 1); ++r)
    for (int e = tid; e < bd.W; e += kLUThreads)
      win[(size_t)(r % kWin) * bd.W + e] = ab[(size_t)r * bd.W + e];
  __syncthreads();
  for (int k = 0; k < bd.n; ++k) {
    const int rmax = min(bd.n - 1, k + bd.kl);
    const int cmax = min(bd.n - 1, k + bd.ku + bd.kl);
    // row k + kl + 1 enters the window at the end of this step (into the
    // slot row k - 1 has left); its global load is issued first so that
    // its latency overlaps the elimination (rows beyond k + kl are untouched)
    const int rn = k + bd.kl + 1;
    const bool pf_on = rn < bd.n && tid < bd.W;
    const double pf = pf_on ? ab[(size_t)rn * bd.W + tid] : 0.0;
    // pivot: largest |entry| of column k in rows k..rmax (lowest row on ties)
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r <= rmax; r += 32) {
        const double v = fabs(W(r, k));
        if (v > best) best = v, bi = r;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) best = ov, bi = oi;
      }
      if (lane == 0) {
        s_p = bi;
        s_d = W(bi, k);
        s_akk = W(k, k);
        piv[k] = bi;
        if (!(best > 0.0)) atomicOr(status, 2);
      }
    }
    __syncthreads();
    const int p = s_p;
    const double d = s_d;
    const double id = d != 0.0 ? 1.0 / d : 0.0;
    // interchange rows k and p right of column k, and form column k of L
    // (row p of it receives the old diagonal entry)
    if (p != k)
      for (int col = k + 1 + tid; col <= cmax; col += kLUThreads) {
        const double t = W(k, col);
        W(k, col) = W(p, col);
        W(p, col) = t;
      }
    for (int r = k + tid; r <= rmax; r += kLUThreads) {
      if (r == k)
        W(k, k) = d;
      else
        W(r, k) = (r == p ? s_akk : W(r, k)) * id;
    }
    __syncthreads();
    const int nr = rmax - k, nc = cmax - k;
    for (int e = tid; e < nr * nc; e += kLUThreads) {
      const int r = k + 1 + e / nc, col = k + 1 + e % nc;
      W(r, col) -= W(r, k) * W(k, col);
    }
    __syncthreads();
    // row k is final: write it back; the prefetched row takes its slot
    for (int e = tid; e < bd.W; e += kLUThreads)
      ab[(size_t)k * bd.W + e] = win[(size_t)(k % kWin) * bd.W + e];
    if (pf_on) win[(size_t)(rn % kWin) * bd.W + tid] = pf;
    __syncthreads();
  }
}

// Columns [col0, col0 + kInvWarps) of the inverse: solve L U x = P e_col,
// one warp per column, the warps of the block in step.  The factor entries
// that step k needs (column k of L with the pivot, then row k of U) are
// shared by all columns: the block streams them into a ring of kInvStages
// shared-memory slots with asynchronous copies issued kInvStages - 1 steps
// ahead, so no step waits on a global load.  All threads of the block call
// it; sm holds inv_block_smem_doubles(n) doubles.
constexpr int kInvWarps = 6;    // columns per block: 149 blocks cover the 891 columns
constexpr int kInvStages = 8;
constexpr int kInvLW = 64;   // >= kl: entries of one L column in a slot
constexpr int kInvUW = 192;  // >= ku + kl + 1: entries of one U row in a slot

__host__ __device__ inline size_t inv_block_smem_doubles(int n) {
  return (size_t)kInvWarps * n + (size_t)kInvStages * (kInvLW + kInvUW + 1);
}

// rd[k] = 1 / U(k, k) of the factored band (one thread per row)
__device__ __forceinline__ void band_diag_recip(const Grid& g, const double* __restrict__ ab,
                                                double* __restrict__ rd, int k) {
  const Band bd = band_of(g);
  if (k < bd.n) rd[k] = 1.0 / ab[(size_t)k * bd.W + bd.kl];
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void band_inverse_block(const Grid& g, const double* __restrict__ ab,
                                                   const int* __restrict__ piv,
                                                   const double* __restrict__ rd,
                                                   double* __restrict__ Ainv, int col0, double* sm) {
  const Band bd = band_of(g);
  const int n = bd.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = blockDim.x;
  double* xs = sm;                                   // [kInvWarps][n]
  double* Lb = sm + (size_t)kInvWarps * n;           // [kInvStages][kInvLW]
  double* Ub = Lb + (size_t)kInvStages * kInvLW;     // [kInvStages][kInvUW]
  int* pb = reinterpret_cast<int*>(Ub + (size_t)kInvStages * kInvUW);  // [kInvStages]
  const int col = col0 + warp;
  double* x = xs + (size_t)warp * n;
  // stage s of the forward sweep: L(s+1 .. s+kl, s) and piv[s]
  auto issue_fwd = [&](int s) {
    if (s < n) {
      const int m = min(bd.kl, n - 1 - s);
      for (int t = tid; t < m; t += nt)
        cp_async8(Lb + (size_t)(s % kInvStages) * kInvLW + t,
                  ab + (size_t)(s + 1 + t) * bd.W + (bd.kl - 1 - t));
      if (tid == nt - 1) cp_async4(pb + s % kInvStages, piv + s);
    }
    cp_async_commit();
  };
  // stage s of the backward sweep (row k = n - 1 - s): 1 / U(k, k) in slot
  // entry 0, U(k, k+1 .. cmax) in entries 1..
  auto issue_bwd = [&](int s) {
    if (s < n) {
      const int k = n - 1 - s;
      const int m = min(bd.ku + bd.kl, n - 1 - k) + 1;
      double* slot = Ub + (size_t)(s % kInvStages) * kInvUW;
      for (int t = tid; t < m; t += nt)
        cp_async8(slot + t, t == 0 ? rd + k : ab + (size_t)k * bd.W + bd.kl + t);
    }
    cp_async_commit();
  };
  if (col < n)
    for (int r = lane; r < n; r += 32) x[r] = (r == col) ? 1.0 : 0.0;
  for (int s = 0; s < kInvStages - 1; ++s) issue_fwd(s);
  for (int k = 0; k < n; ++k) {
    cp_async_wait<kInvStages - 2>();  // stage k has landed (this thread's copies)
    __syncthreads();                   // ... everybody's; slot (k - 1) % S is free
    issue_fwd(k + kInvStages - 1);
    if (col < n) {
      const int p = pb[k % kInvStages];
      if (lane == 0 && p != k) {
        const double t = x[k];
        x[k] = x[p];
        x[p] = t;
      }
      __syncwarp();
      const double xk = x[k];
      if (xk != 0.0) {
        const double* Lk = Lb + (size_t)(k % kInvStages) * kInvLW;
        const int rmax = min(n - 1, k + bd.kl);
        for (int r = k + 1 + lane; r <= rmax; r += 32) x[r] -= Lk[r - k - 1] * xk;
      }
      __syncwarp();
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  for (int s = 0; s < kInvStages - 1; ++s) issue_bwd(s);
  for (int s = 0; s < n; ++s) {
    cp_async_wait<kInvStages - 2>();
    __syncthreads();
    issue_bwd(s + kInvStages - 1);
    if (col < n) {
      const int k = n - 1 - s;
      const double* Uk = Ub + (size_t)(s % kInvStages) * kInvUW;
      const int cmax = min(n - 1, k + bd.ku + bd.kl);
      double acc = 0.0;
      for (int c2 = k + 1 + lane; c2 <= cmax; c2 += 32) acc += Uk[c2 - k] * x[c2];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) x[k] = (x[k] - acc) * Uk[0];
      __syncwarp();
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // Ainv[r][col0 .. col0 + kInvWarps): kInvWarps consecutive doubles per row
  for (int e = tid; e < n * kInvWarps; e += nt) {
    const int r = e / kInvWarps, w = e % kInvWarps;
    if (col0 + w < n) Ainv[(size_t)r * n + col0 + w] = xs[(size_t)w * n + r];
  }
}

// x = Ainv b with the band numbering on both sides; one warp per row.
// Rows [rblock * kSolveWarps, +kSolveWarps) of x; the whole block calls it,
// sb holds n doubles of shared memory.
constexpr int kSolveWarps = 8;
template <typename T>
__device__ __forceinline__ void coarse_solve_rows(const Grid& g, const double* __restrict__ Ainv,
                                                  const T* __restrict__ b, T* __restrict__ x,
                                                  int rblock, double* sb) {
  const Band bd = band_of(g);
  for (int p = threadIdx.x; p < bd.n; p += blockDim.x) sb[p] = (double)b[lidx(g, p)];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = rblock * kSolveWarps + warp;
  if (r >= bd.n) return;
  const double* row = Ainv + (size_t)r * bd.n;
  double acc = 0.0;
  for (int c = lane; c < bd.n; c += 32) acc += row[c] * sb[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[lidx(g, r)] = (T)acc;
}

}  // namespace dnnmg
