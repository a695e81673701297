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

// Stabilisation pieces of the four cells of a 2h patch: S[c][m * 9 + n] =
// alpha kappa^T K_c kappa with K_c the Q1 stiffness of cell c = cx + 2 cy of
// the patch on its 3x3 nodes (the cellwise forms: their own cell blocks).  A
// patch whose cells are partly solid integrates over its fluid cells only,
// so its matrix is the sum of those cells' pieces; whole patches use S9.
struct PatchPieces {
  double S[4][81];
};

// entry (r, col) of the band matrix
__device__ __forceinline__ double& AB(double* ab, const Band& b, int r, int col) {
  return ab[(size_t)r * b.W + (col - r + b.kl)];
}

// Row `row` of the banded coarse Jacobian (one thread per row); pp (may be
// null when every patch is whole) gives the pieces of part-solid patches.
__device__ __forceinline__ void assemble_row(const Grid& g, const Sten<double>& s,
                                             const double* __restrict__ vb,
                                             double* __restrict__ ab, int row,
                                             const PatchPieces* pp = nullptr) {
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
        const int c00 = (2 * PJ) * g.nx + 2 * PI;
        const int fm = (g.solid[c00] ? 0 : 1) | (g.solid[c00 + 1] ? 0 : 2) |
                       (g.solid[c00 + g.nx] ? 0 : 4) | (g.solid[c00 + g.nx + 1] ? 0 : 8);
        const bool whole = fm == 15 || !pp;  // whole patch (or no pieces: lower-left cell decides)
        if (whole && g.solid[c00]) continue;
        if (fm == 0) continue;
        const int mn = (i - 2 * PI) + 3 * (j - 2 * PJ);
        for (int m = 0; m < 9; ++m) {
          const int ni = 2 * PI + m % 3, nj = 2 * PJ + m / 3;
          if (g.flags[nj * g.nnx + ni] & kPFix) continue;
          double v = 0.0;
          if (whole) {
            v = s.S9[mn * 9 + m];
          } else {
            for (int c = 0; c < 4; ++c)
              if (fm & (1 << c)) v += pp->S[c][mn * 9 + m];
          }
          AB(ab, bd, row, bidx(g, 2, ni, nj)) += v;
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
// one warp per column, with no barrier between the warps until the end.
// Each warp streams the factor entries a step needs (column k of L and the
// pivot, then column k of U and 1 / U(k, k)) from global memory into a
// register ring kInvAhead steps ahead, so a step waits neither on a load nor
// on the other warps.  The forward sweep starts at row col - kl: a swap at
// step k touches rows k and piv[k] <= k + kl, so no earlier step reaches the
// nonzero of e_col.  All threads of the block call it; sm holds
// inv_block_smem_doubles(n) doubles.
constexpr int kInvWarps = 6;    // columns per block: 149 blocks cover the 891 columns
constexpr int kInvAhead = 8;    // steps of factor entries in flight per warp

__host__ __device__ inline size_t inv_block_smem_doubles(int n) { return (size_t)kInvWarps * n; }

// rd[k] = 1 / U(k, k) of the factored band (one thread per row)
__device__ __forceinline__ void band_diag_recip(const Grid& g, const double* __restrict__ ab,
                                                double* __restrict__ rd, int k) {
  const Band bd = band_of(g);
  if (k < bd.n) rd[k] = 1.0 / ab[(size_t)k * bd.W + bd.kl];
}

__device__ __forceinline__ void band_inverse_block(const Grid& g, const double* __restrict__ ab,
                                                   const int* __restrict__ piv,
                                                   const double* __restrict__ rd,
                                                   double* __restrict__ Ainv, int col0, double* sm) {
  const Band bd = band_of(g);
  const int n = bd.n, kl = bd.kl, KU2 = bd.ku + bd.kl, W = bd.W;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int col = col0 + warp;
  double* x = sm + (size_t)warp * n;
  constexpr int D = kInvAhead;
  if (col < n) {  // warp-uniform
    for (int r = lane; r < n; r += 32) x[r] = (r == col) ? 1.0 : 0.0;
    __syncwarp();
    // ---- forward: x <- L^{-1} P x; lane holds L(k+1+lane, k), L(k+33+lane, k)
    double la[D], lb[D];
    int pp[D];
    auto load_fwd = [&](int s, double& l0, double& l1, int& pk) {
      l0 = l1 = 0.0;
      pk = 0;
      if (s < n) {
        const int rmax = min(n - 1, s + kl);
        const int r0 = s + 1 + lane, r1 = r0 + 32;
        if (r0 <= rmax) l0 = ab[(size_t)r0 * W + (s - r0 + kl)];
        if (r1 <= rmax) l1 = ab[(size_t)r1 * W + (s - r1 + kl)];
        pk = piv[s];
      }
    };
    const int k0 = max(0, col - kl);
#pragma unroll
    for (int j = 0; j < D; ++j) load_fwd(k0 + j, la[j], lb[j], pp[j]);
    for (int kb = k0; kb < n; kb += D) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int k = kb + j;
        if (k < n) {
          const int p = pp[j];
          if (lane == 0 && p != k) {
            const double t = x[k];
            x[k] = x[p];
            x[p] = t;
          }
          __syncwarp();
          const double xk = x[k];
          const int rmax = min(n - 1, k + kl);
          const int r0 = k + 1 + lane, r1 = r0 + 32;
          if (r0 <= rmax) x[r0] -= la[j] * xk;
          if (r1 <= rmax) x[r1] -= lb[j] * xk;
          __syncwarp();
        }
        load_fwd(k + D, la[j], lb[j], pp[j]);
      }
    }
    // ---- backward: x <- U^{-1} x by columns, k = n-1 .. 0: x[k] /= U(k, k),
    // then x[r] -= U(r, k) x[k] for the rows r = k-1-lane-32i (i < 4, ku + kl
    // <= 128) above it; lane holds those U(r, k) and 1 / U(k, k)
    double u0[D], u1[D], u2[D], u3[D], ri[D];
    auto load_bwd = [&](int k, double& v0, double& v1, double& v2, double& v3, double& rk) {
      v0 = v1 = v2 = v3 = rk = 0.0;
      if (k >= 0) {
        const int rmin = max(0, k - KU2);
        const int r = k - 1 - lane;  // U(r, k) at ab[r W + k - r + kl]
        if (r >= rmin) v0 = ab[(size_t)r * W + (k - r + kl)];
        if (r - 32 >= rmin) v1 = ab[(size_t)(r - 32) * W + (k - r + 32 + kl)];
        if (r - 64 >= rmin) v2 = ab[(size_t)(r - 64) * W + (k - r + 64 + kl)];
        if (r - 96 >= rmin) v3 = ab[(size_t)(r - 96) * W + (k - r + 96 + kl)];
        rk = rd[k];
      }
    };
#pragma unroll
    for (int j = 0; j < D; ++j) load_bwd(n - 1 - j, u0[j], u1[j], u2[j], u3[j], ri[j]);
    for (int kb = n - 1; kb >= 0; kb -= D) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int k = kb - j;
        if (k >= 0) {
          const double xk = x[k] * ri[j];
          __syncwarp();
          if (lane == 0) x[k] = xk;
          const int rmin = max(0, k - KU2), r = k - 1 - lane;
          if (r >= rmin) x[r] -= u0[j] * xk;
          if (r - 32 >= rmin) x[r - 32] -= u1[j] * xk;
          if (r - 64 >= rmin) x[r - 64] -= u2[j] * xk;
          if (r - 96 >= rmin) x[r - 96] -= u3[j] * xk;
          __syncwarp();
        }
        load_bwd(k - D, u0[j], u1[j], u2[j], u3[j], ri[j]);
      }
    }
  }
  __syncthreads();
  // Ainv[r][col0 .. col0 + kInvWarps): kInvWarps consecutive doubles per row
  for (int e = tid; e < n * kInvWarps; e += blockDim.x) {
    const int r = e / kInvWarps, w = e % kInvWarps;
    if (col0 + w < n) Ainv[(size_t)r * n + col0 + w] = sm[(size_t)w * n + r];
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
