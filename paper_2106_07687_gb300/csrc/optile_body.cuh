// Tiled evaluation of the operator rows (Eqs. 4-5 and their linearisation,
// Eq. 6) on a tile of TX x TY nodes: the block stages the field (and the
// linearisation velocity) of the tile plus a two-node halo in shared
// memory, computes the 12 rows of every cell touching the tile once and the
// 9 LPS rows of every patch touching it once, and each thread then sums the
// rows of its node.  A node-wise evaluation recomputes each cell's
// Gauss-point values for each of the cell's four nodes; the tile does it
// once.  All global loads of the tile are issued in one round.
#pragma once
#include "common.cuh"

namespace dnnmg {

template <typename T, int TX, int TY>
struct OpSmem {
  T w[3][TY + 4][TX + 4];
  T vb[2][TY + 4][TX + 4];
  uint8_t fl[TY + 4][TX + 4];
  uint8_t sol[TY + 4][TX + 4];  // solid flag of the cell whose lower-left node this is
  T cres[(TY + 1) * (TX + 1)][12];
  T pres[(TY / 2 + 1) * (TX / 2 + 1)][9];
  int8_t cvalid[(TY + 1) * (TX + 1)];
  int8_t pvalid[(TY / 2 + 1) * (TX / 2 + 1)];
};

// Rows (ru, rv, rp) of the operator at this thread's node of tile (bx, by):
// A(w) if NONLIN, else A'(vb) w; with MASK, constrained entries of w count
// as zero.  Every thread of the NTT-thread block calls it (block barriers
// inside): the first TX * TY threads own a node each, any further ones help
// stage the tile and compute its cell and patch rows.  A thread whose node
// lies outside the level, and every helper, gets n = -1.  Constrained rows
// are returned like free ones (the caller overrides them).  The fields are
// stored as L and converted to the arithmetic type T when staged.
template <class X>
struct op_same {  // keeps a parameter out of template argument deduction
  using type = X;
};
template <typename T, bool NONLIN, bool MASK, int TX, int TY, int NTT = TX * TY, typename L = T>
__device__ __forceinline__ void op_tile_rows(const Grid& g, const Sten<T>& s,
                                             const L* __restrict__ w,
                                             const typename op_same<L>::type* __restrict__ vb,
                                             int bx, int by, OpSmem<T, TX, TY>& S, T& ru, T& rv,
                                             T& rp, int& n) {
  static_assert(TX % 2 == 0 && TY % 2 == 0, "even tile");
  constexpr int kNT = TX * TY, kSX = TX + 4, kSY = TY + 4;
  constexpr int kCX = TX + 1, kCY = TY + 1, kPX = TX / 2 + 1, kPY = TY / 2 + 1;
  const int nn = g.nn;
  const int i0 = bx * TX, j0 = by * TY;  // first node of the tile (even)
  static_assert(NTT >= kNT, "thread group");
  const int t = threadIdx.x;
  // ---- stage nodes [i0-2, i0+TX+2) x [j0-2, j0+TY+2)
  for (int e = t; e < kSX * kSY; e += NTT) {
    const int li = e % kSX, lj = e / kSX;
    const int i = i0 - 2 + li, j = j0 - 2 + lj;
    T u = 0, v = 0, p = 0, bu = 0, bvv = 0;
    uint8_t f = 0xFF, so = 1;
    if (i >= 0 && j >= 0 && i <= g.nx && j <= g.ny) {
      const int m = j * g.nnx + i;
      f = g.flags[m];
      u = T(w[m]);
      v = T(w[nn + m]);
      p = T(w[2 * nn + m]);
      if (!NONLIN) {
        bu = T(vb[m]);
        bvv = T(vb[nn + m]);
      }
      if (i < g.nx && j < g.ny) so = g.solid[j * g.nx + i];
    }
    S.w[0][lj][li] = (MASK && (f & kVDir)) ? T(0) : u;
    S.w[1][lj][li] = (MASK && (f & kVDir)) ? T(0) : v;
    S.w[2][lj][li] = (MASK && (f & kPFix)) ? T(0) : p;
    S.vb[0][lj][li] = bu;
    S.vb[1][lj][li] = bvv;
    S.fl[lj][li] = f;
    S.sol[lj][li] = so;
  }
  __syncthreads();
  // ---- cells [i0-1, i0+TX) x [j0-1, j0+TY): 12 rows each, and the patches
  // I in [i0/2 - 1, i0/2 + TX/2 - 1] (those with 2I <= i <= 2I+2 for a node i
  // of the tile), likewise J: 9 LPS rows each
  const int PI0 = i0 / 2 - 1, PJ0 = j0 / 2 - 1;
  for (int e = t; e < kCX * kCY; e += NTT) {
    const int lc = e % kCX, lr = e / kCX;
    const int ci = i0 - 1 + lc, cj = j0 - 1 + lr;
    const bool ok = ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny && !S.sol[lr + 1][lc + 1];
    S.cvalid[e] = ok;
    if (!ok) continue;
    T wu[4], wv[4], wp[4], bu[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int li = lc + 1 + (a & 1), lj = lr + 1 + (a >> 1);
      wu[a] = S.w[0][lj][li];
      wv[a] = S.w[1][lj][li];
      wp[a] = S.w[2][lj][li];
      bu[a] = S.vb[0][lj][li];
      bv[a] = S.vb[1][lj][li];
    }
    T r[12];
    cell_all_rows<T, NONLIN>(s, wu, wv, wp, bu, bv, r);
#pragma unroll
    for (int k = 0; k < 12; ++k) S.cres[e][k] = r[k];
  }
  // the patches start where the cells left off, on the threads that the
  // cell loop leaves idle (a rotation of the thread index)
  constexpr int kOff = (kCX * kCY) % NTT;
  for (int e = (t + NTT - kOff) % NTT; e < kPX * kPY; e += NTT) {
    const int pi = PI0 + e % kPX, pj = PJ0 + e / kPX;
    const bool ok = pi >= 0 && pj >= 0 && pi < g.nx / 2 && pj < g.ny / 2 &&
                    !S.sol[2 * pj - j0 + 2][2 * pi - i0 + 2];
    S.pvalid[e] = ok;
    if (!ok) continue;
    T p[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) p[m] = S.w[2][2 * pj + m / 3 - j0 + 2][2 * pi + m % 3 - i0 + 2];
#pragma unroll
    for (int mn = 0; mn < 9; ++mn) {
      T acc = 0;
#pragma unroll
      for (int m = 0; m < 9; ++m) acc += s.S9[mn * 9 + m] * p[m];
      S.pres[e][mn] = acc;
    }
  }
  __syncthreads();
  // ---- this thread's node
  const int i = i0 + t % TX, j = j0 + t / TX;
  ru = rv = rp = T(0);
  n = -1;
  if (t >= kNT || i > g.nx || j > g.ny) return;
  n = j * g.nnx + i;
#pragma unroll
  for (int dyy = 0; dyy < 2; ++dyy)
#pragma unroll
    for (int dxx = 0; dxx < 2; ++dxx) {
      const int e = (j - 1 + dyy - (j0 - 1)) * kCX + (i - 1 + dxx - (i0 - 1));
      if (!S.cvalid[e]) continue;
      const int al = (1 - dxx) + 2 * (1 - dyy);
      ru += S.cres[e][al];
      rv += S.cres[e][4 + al];
      rp += S.cres[e][8 + al];
    }
#pragma unroll
  for (int dJ = 0; dJ < 2; ++dJ) {
    const int PJ = (j >> 1) - dJ;
    if (j - 2 * PJ > 2) continue;
#pragma unroll
    for (int dI = 0; dI < 2; ++dI) {
      const int PI = (i >> 1) - dI;
      if (i - 2 * PI > 2) continue;
      const int e = (PJ - PJ0) * kPX + (PI - PI0);
      if (!S.pvalid[e]) continue;
      rp += S.pres[e][(i - 2 * PI) + 3 * (j - 2 * PJ)];
    }
  }
}

// flag bits of this thread's node after op_tile_rows (n >= 0)
template <typename T, int TX, int TY>
__device__ __forceinline__ uint8_t op_tile_flags(const OpSmem<T, TX, TY>& S) {
  return S.fl[threadIdx.x / TX + 2][threadIdx.x % TX + 2];
}

}  // namespace dnnmg
