// Per-thread and per-tile bodies of the Vanka smoother, shared by the
// single-problem kernels (vanka.cu) and the batched kernels (batch.cu).
//
// Setup: for every fluid cell, the restriction of the global Jacobian to the
// cell's 12 DOFs (its 4 nodes x u, v, p), with identity rows/columns on
// constrained DOFs, is inverted by Gauss-Jordan elimination with partial
// pivoting and stored as inv[colour][entry][slot] so that the smoothing pass
// streams it with coalesced loads.
//
// Tiled colour pass: a block owns kTCX x kTCY cells of the colour, i.e. the
// (2 kTCX) x (2 kTCY) nodes they cover.  It stages the masked iterate, vbar
// and the flags of those nodes plus a two-node halo in shared memory,
// computes the 12 rows of every cell touching the tile and the 9 LPS rows of
// every patch touching it once, sums them per node, exchanges each cell's 12
// defects among the cell's four threads by warp shuffles and applies the
// 12x12 inverse.  Cells of one colour share no node; nodes outside the
// colour's fluid cells are copied, so x_out is complete and the next colour
// reads it without races.
#pragma once
#include "common.cuh"

namespace dnnmg {

template <typename T>
__device__ __forceinline__ T vk_abs(T v) {
  return v < T(0) ? -v : v;
}

// Shared memory of one cell's setup (one half-warp): the Gauss-point data of
// the 9 cells around it and the 3x3 element blocks of its 36 (element, a, b)
// triples.
template <typename T>
struct SetupSmem {
  T gd[9][24];  // Bu, Bv, Bux, Buy, Bvx, Bvy at the 4 Gauss points
  T J[36][9];   // J[c][c2] of triple a * 9 + m (see vanka_setup_cell)
  int ok[9];    // the element is a fluid cell of the level
};

// Inverse of the local 12x12 block of the cell of `slot` in `colour`,
// computed by a group of 16 consecutive lanes (a half-warp; every lane of it
// calls this with the same cell and its own W).  The block's entry between
// local nodes a and b sums the element Jacobians of the cells that hold both
// nodes: the 4 cells around a (b = a), the 2 cells on the edge a-b, or the
// cell itself (a, b diagonal) -- 36 (element, a, b) triples over the 9 cells
// around the cell.  Lanes 0..8 form the Gauss-point data of one of those 9
// cells each, the 16 lanes then form the triples' 3x3 element blocks, and
// lane r < 12 sums row r = (c, a) of the block (component c of local node a)
// in the order of the cells around node a (rows first) and keeps it in
// registers.  Gauss-Jordan elimination with partial pivoting then runs
// across the lanes: at step k the unused lane with the largest |A[.][k]|
// (lowest lane on ties) is the pivot row, its normalised row is broadcast by
// shuffles and every other lane eliminates column k.  Rows are never
// swapped; the lane that pivoted on column k ends with row k of the inverse.
template <typename T>
__device__ __forceinline__ void vanka_setup_cell(const Grid& g, const Sten<T>& s,
                                                 const T* __restrict__ vb, T* __restrict__ inv,
                                                 int* status, int colour, int slot,
                                                 SetupSmem<T>& W) {
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1, pitch = vanka_pitch(g);
  const int nslots = vanka_slots(g);
  if (slot >= nslots || slot % pitch >= sx) return;
  const int ci = 2 * (slot % pitch) - cx, cj = 2 * (slot / pitch) - cy;
  if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny || g.solid[cj * g.nx + ci]) return;
  const int lane = threadIdx.x & 15;
  const unsigned mask = 0xFFFFu << (threadIdx.x & 16);  // this half-warp
  const int r = lane < 12 ? lane : 0;                   // lanes 12..15 shadow row 0
  const int c = r >> 2, a = r & 3;
  const int ai = ci + (a & 1), aj = cj + (a >> 1);       // node a

  // ---- Gauss-point data of cell e = ex + 3 ey at (ci - 1 + ex, cj - 1 + ey)
  if (lane < 9) {
    const int Tx = ci - 1 + lane % 3, Ty = cj - 1 + lane / 3;
    const bool ev = Tx >= 0 && Ty >= 0 && Tx < g.nx && Ty < g.ny && !g.solid[Ty * g.nx + Tx];
    W.ok[lane] = ev;
    if (ev) {
      T bu[4], bv[4];
      load_cell<T, false>(g, vb, Tx, Ty, 0, bu);
      load_cell<T, false>(g, vb + g.nn, Tx, Ty, 0, bv);
      GaussData<T> gd;
      gauss_data<T>(bu, bv, gd);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        W.gd[lane][q] = gd.Bu[q];
        W.gd[lane][4 + q] = gd.Bv[q];
        W.gd[lane][8 + q] = gd.Bux[q];
        W.gd[lane][12 + q] = gd.Buy[q];
        W.gd[lane][16 + q] = gd.Bvx[q];
        W.gd[lane][20 + q] = gd.Bvy[q];
      }
    }
  }
  __syncwarp(mask);
  // ---- element blocks of triple t = a * 9 + m: node b = a ^ d and the cell
  // (ex, ey) holding both, with m < 4: d = 0, the 4 cells around a (rows
  // first); m = 4, 5: d = 1, the 2 cells on the x edge (bottom first);
  // m = 6, 7: d = 2, the 2 cells on the y edge (left first); m = 8: d = 3,
  // the cell itself
  for (int t = lane; t < 36; t += 16) {
    const int ta = t / 9, m = t % 9;
    const int tax = ta & 1, tay = ta >> 1;
    int d, ex, ey;
    if (m < 4) {
      d = 0, ex = tax + (m & 1), ey = tay + (m >> 1);
    } else if (m < 6) {
      d = 1, ex = 1, ey = tay + (m - 4);
    } else if (m < 8) {
      d = 2, ex = tax + (m - 6), ey = 1;
    } else {
      d = 3, ex = 1, ey = 1;
    }
    const int tb = ta ^ d, tbx = tb & 1, tby = tb >> 1;
    const int e = ex + 3 * ey;
    T J[3][3];
    if (W.ok[e]) {
      GaussData<T> gd;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        gd.Bu[q] = W.gd[e][q];
        gd.Bv[q] = W.gd[e][4 + q];
        gd.Bux[q] = W.gd[e][8 + q];
        gd.Buy[q] = W.gd[e][12 + q];
        gd.Bvx[q] = W.gd[e][16 + q];
        gd.Bvy[q] = W.gd[e][20 + q];
      }
      elem_pair<T>(s, gd, (tax + 1 - ex) + 2 * (tay + 1 - ey), (tbx + 1 - ex) + 2 * (tby + 1 - ey),
                   J);
#pragma unroll
      for (int k = 0; k < 9; ++k) W.J[t][k] = J[k / 3][k % 3];
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) W.J[t][k] = T(0);
    }
  }
  __syncwarp(mask);
  // ---- row r: column block b sums the triples of (a, b), d = a ^ b: the
  // 4, 2, 2 or 1 consecutive ones from a * 9 + 0, 4, 6 or 8
  T A[24];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int d = a ^ b;
    const int t0 = a * 9 + (d == 0 ? 0 : (d == 1 ? 4 : (d == 2 ? 6 : 8)));
    const int cnt = d == 0 ? 4 : (d == 3 ? 1 : 2);
#pragma unroll
    for (int c2 = 0; c2 < 3; ++c2) A[c2 * 4 + b] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < cnt) {
#pragma unroll
        for (int c2 = 0; c2 < 3; ++c2) A[c2 * 4 + b] += W.J[t0 + k][c * 3 + c2];
      }
  }
#pragma unroll
  for (int k = 12; k < 24; ++k) A[k] = T(0);
  // local projection stabilisation (pressure rows) of the patches
  // containing node pairs: lane l forms the entry of the pressure row of
  // node l / 4 and the pressure column of node l % 4 (the sum over the
  // patches that hold both nodes, rows of patches first), and the lanes of
  // the pressure rows collect their four entries (the pressure-pressure
  // element blocks are zero, so A[8 + b] is 0 before)
  {
    const int la = lane >> 2, lb = lane & 3;
    const int pai = ci + (la & 1), paj = cj + (la >> 1);  // node la
    const int pbi = ci + (lb & 1), pbj = cj + (lb >> 1);  // node lb
    T lps = T(0);
    for (int PJ = (paj - 1) >> 1; PJ <= (paj >> 1); ++PJ)  // patches holding node la
      for (int PI = (pai - 1) >> 1; PI <= (pai >> 1); ++PI) {
        if (PI < 0 || PJ < 0 || PI >= g.nx / 2 || PJ >= g.ny / 2) continue;
        if (g.solid[(2 * PJ) * g.nx + 2 * PI]) continue;
        const int sb = pbi - 2 * PI, tb = pbj - 2 * PJ;
        if (sb < 0 || sb > 2 || tb < 0 || tb > 2) continue;
        lps += s.S9[((pai - 2 * PI) + 3 * (paj - 2 * PJ)) * 9 + sb + 3 * tb];
      }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const T v = __shfl_sync(mask, lps, a * 4 + b, 16);
      if (c == 2) A[8 + b] += v;
    }
  }
  // identity rows and zero columns on constrained DOFs
  uint8_t fl[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) fl[b] = g.flags[(cj + (b >> 1)) * g.nnx + ci + (b & 1)];
  const bool own_cons = g.flags[aj * g.nnx + ai] & (c < 2 ? kVDir : kPFix);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const bool col_cons = fl[k & 3] & (k < 8 ? kVDir : kPFix);
    if (own_cons) A[k] = k == r ? T(1) : T(0);
    else if (col_cons) A[k] = T(0);
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) A[12 + k] = k == r ? T(1) : T(0);

  // Gauss-Jordan elimination with partial pivoting across the lanes, in
  // place: the right half of [A | I] is kept in the columns already
  // eliminated.  Before step k, the identity column of an unused row p is
  // still e_p, so after the step it holds 1 / A[p][k] in row p and
  // -A[i][k] / A[p][k] elsewhere, which column k receives; columns j < k hold
  // the identity column of the row that pivoted on column j (pcol[j]).  The
  // arithmetic is that of the explicit form, entry by entry.
  bool used = lane >= 12, ok = true;
  int my_col = 0;
  int pcol[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    // pivot: the largest |A[k]| among the unused rows, the lowest lane on a tie
    T best;
    int p;
    if constexpr (sizeof(T) == 4) {
      // the bit patterns of non-negative floats order like the floats: one
      // maximum over the half-warp, then the lowest lane that holds it
      const unsigned key = used ? 0u : __float_as_uint(vk_abs(A[k]));
      const unsigned mx = __reduce_max_sync(mask, key);
      p = (__ffs(__ballot_sync(mask, key == mx) & mask) - 1) & 15;
      best = __uint_as_float(mx);
    } else {
      best = used ? T(-1) : vk_abs(A[k]);
      p = lane;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(mask, best, o, 16);
        const int op = __shfl_xor_sync(mask, p, o, 16);
        if (ob > best || (ob == best && op < p)) best = ob, p = op;
      }
    }
    pcol[k] = p;
    ok = ok && best > T(0);  // the same in every lane of the group
    if (ok) {
      const T ip = T(1) / __shfl_sync(mask, A[k], p, 16);
      const T f = A[k];
      const bool piv = lane == p;
#pragma unroll
      for (int cc = 0; cc < 12; ++cc) {
        if (cc == k) continue;
        const T pn = __shfl_sync(mask, A[cc], p, 16) * ip;  // normalised pivot row
        A[cc] = piv ? pn : A[cc] - f * pn;
      }
      A[k] = piv ? ip : T(0) - f * ip;
      if (piv) used = true, my_col = k;
    }
  }
  if (!ok) {
    if (lane == 0) atomicOr(status, 1);
  }
  if (lane >= 12) return;
  // row my_col of the inverse; entry j is its column pcol[j]
  T* out = inv + (size_t)colour * 144 * nslots + slot;
#pragma unroll
  for (int j = 0; j < 12; ++j)
    out[(size_t)(my_col * 12 + pcol[j]) * nslots] = ok ? A[j] : T(0);
}

// Resident blocks per SM the pass kernels ask the compiler for: FP32 passes
// are held to 128 registers per thread so that 512 threads per SM fit.
template <typename T>
constexpr int pass_min_blocks(int threads) {
  return sizeof(T) == 4 ? (512 / threads > 0 ? 512 / threads : 1) : 1;
}

template <typename T, int kTCX, int kTCY>
struct PassSmem {
  T w[3][2 * kTCY + 4][2 * kTCX + 4];
  T vb[2][2 * kTCY + 4][2 * kTCX + 4];
  uint8_t fl[2 * kTCY + 4][2 * kTCX + 4];
  uint8_t sol[2 * kTCY + 4][2 * kTCX + 4];  // solid flag of the cell whose lower-left node this is
  T cres[(2 * kTCY + 1) * (2 * kTCX + 1)][12];
  T pres[(kTCY + 2) * (kTCX + 2)][9];
  int8_t cvalid[(2 * kTCY + 1) * (2 * kTCX + 1)];
  int8_t pvalid[(kTCY + 2) * (kTCX + 2)];
};

// Stage the tile whose first node is (i0, j0) -- nodes [i0-2, i0-2+kSX) x
// [j0-2, j0-2+kSY) with the masked iterate, vbar, flags and the solid flag
// of the cell whose lower-left node each one is -- then compute the 12 rows
// of every cell touching the tile and the 9 LPS rows of every patch touching
// it, once each.  Thread t of NTT; ends with the rows visible to all
// threads of the group (two block barriers).
template <typename T, int kTCX, int kTCY, int NTT>
__device__ __forceinline__ void pass_stage_rows(const Grid& g, const Sten<T>& s,
                                                const T* __restrict__ xin,
                                                const T* __restrict__ vb, int i0, int j0, int t,
                                                PassSmem<T, kTCX, kTCY>& S) {
  constexpr int kSX = 2 * kTCX + 4;
  constexpr int kCX = 2 * kTCX + 1, kCY = 2 * kTCY + 1;
  constexpr int kPX = kTCX + 2, kPY = kTCY + 2;
  constexpr int kSY = 2 * kTCY + 4;
  const int nn = g.nn;
  for (int e = t; e < kSX * kSY; e += NTT) {
    const int li = e % kSX, lj = e / kSX;
    const int i = i0 - 2 + li, j = j0 - 2 + lj;
    T xu1 = 0, xv1 = 0, xp1 = 0, bu = 0, bvv = 0;
    uint8_t f = 0xFF, so = 1;
    if (i >= 0 && j >= 0 && i <= g.nx && j <= g.ny) {
      const int n = j * g.nnx + i;
      f = g.flags[n];
      xu1 = xin[n];
      xv1 = xin[nn + n];
      xp1 = xin[2 * nn + n];
      bu = vb[n];
      bvv = vb[nn + n];
      if (i < g.nx && j < g.ny) so = g.solid[j * g.nx + i];
    }
    S.w[0][lj][li] = (f & kVDir) ? T(0) : xu1;
    S.w[1][lj][li] = (f & kVDir) ? T(0) : xv1;
    S.w[2][lj][li] = (f & kPFix) ? T(0) : xp1;
    S.vb[0][lj][li] = bu;
    S.vb[1][lj][li] = bvv;
    S.fl[lj][li] = f;
    S.sol[lj][li] = so;
  }
  __syncthreads();
  // ---- cells [i0-1, i0-1+kCX) x [j0-1, j0-1+kCY): 12 rows each, then the
  // patches touching the tile: 9 LPS rows each; these are the patches from
  // ceil((i0 - 2) / 2) (also for negative i0) to floor((i0 + 2 kTCX - 1) / 2),
  // likewise in y
  const int PI0 = (i0 - 1) >> 1, PJ0 = (j0 - 1) >> 1;
  const int PI1 = (i0 + 2 * kTCX - 1) >> 1, PJ1 = (j0 + 2 * kTCY - 1) >> 1;
  for (int e = t; e < kCX * kCY; e += NTT) {
    const int lc = e % kCX, lr = e / kCX;
    const int ci = i0 - 1 + lc, cj = j0 - 1 + lr;
    const bool ok = ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny && !S.sol[lr + 1][lc + 1];
    S.cvalid[e] = ok;
    if (!ok) continue;
    T wu[4], wv[4], wp[4], bu[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int li = lc + 1 + (a & 1), lj = lr + 1 + (a >> 1);  // staged coords of the node
      wu[a] = S.w[0][lj][li];
      wv[a] = S.w[1][lj][li];
      wp[a] = S.w[2][lj][li];
      bu[a] = S.vb[0][lj][li];
      bv[a] = S.vb[1][lj][li];
    }
    T r[12];
    cell_all_rows<T, false>(s, wu, wv, wp, bu, bv, r);
#pragma unroll
    for (int k = 0; k < 12; ++k) S.cres[e][k] = r[k];
  }
  // the patches start where the cells left off, on the threads that the
  // cell loop leaves idle (a rotation of the thread index)
  constexpr int kOff = (kCX * kCY) % NTT;
  for (int e = (t + NTT - kOff) % NTT; e < kPX * kPY; e += NTT) {
    const int pi = PI0 + e % kPX, pj = PJ0 + e / kPX;
    const bool ok = pi <= PI1 && pj <= PJ1 && pi >= 0 && pj >= 0 && pi < g.nx / 2 &&
                    pj < g.ny / 2 && !S.sol[2 * pj - j0 + 2][2 * pi - i0 + 2];
    S.pvalid[e] = ok;
    if (!ok) continue;
    T p[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      const int li = 2 * pi + m % 3 - (i0 - 2), lj = 2 * pj + m / 3 - (j0 - 2);
      p[m] = S.w[2][lj][li];
    }
#pragma unroll
    for (int mn = 0; mn < 9; ++mn) {
      T acc = 0;
#pragma unroll
      for (int m = 0; m < 9; ++m) acc += s.S9[mn * 9 + m] * p[m];
      S.pres[e][mn] = acc;
    }
  }
  __syncthreads();
}

// Defect b - A x at node (i, j) of the staged tile with first node (i0, j0)
// from the staged rows (constrained rows: b - x), for a node of a fluid
// colour cell; xu.. and bu0.. are the node's unmasked iterate and
// right-hand side.
template <typename T, int kTCX, int kTCY>
__device__ __forceinline__ void pass_node_defect(int i, int j, int i0, int j0, T xu, T xv, T xp,
                                                 T bu0, T bv0, T bp0,
                                                 const PassSmem<T, kTCX, kTCY>& S, T& du, T& dv,
                                                 T& dp) {
  constexpr int kCX = 2 * kTCX + 1, kPX = kTCX + 2;
  const int PI0 = (i0 - 1) >> 1, PJ0 = (j0 - 1) >> 1;
  T ru = 0, rv = 0, rp = 0;
#pragma unroll
  for (int dyy = 0; dyy < 2; ++dyy)
#pragma unroll
    for (int dxx = 0; dxx < 2; ++dxx) {
      const int lc = i - 1 + dxx - (i0 - 1), lr = j - 1 + dyy - (j0 - 1);
      const int e = lr * kCX + lc;
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
  const uint8_t f = S.fl[j - (j0 - 2)][i - (i0 - 2)];
  du = bu0 - ((f & kVDir) ? xu : ru);
  dv = bv0 - ((f & kVDir) ? xv : rv);
  dp = bp0 - ((f & kPFix) ? xp : rp);
}

// Tile (bx, by) of the colour pass, computed by a group of NTT consecutive
// threads of the block (a block may hold several such groups, each with its
// own S; every thread of the block must call this together because of the
// block barriers).  The first 4 kTCX kTCY threads own one node of a colour
// cell each; with NTT larger, the other threads help stage the tile and
// compute the cell and patch rows, so that those take one round instead of
// two.  A group with active = false takes part in the barriers only and
// writes nothing.
template <typename T, int kTCX, int kTCY, int NTT = 4 * kTCX * kTCY>
__device__ __forceinline__ void vanka_pass_tile(const Grid& g, const Sten<T>& s, int colour,
                                                const T* __restrict__ b, const T* __restrict__ xin,
                                                const T* __restrict__ vb, const T* __restrict__ inv,
                                                T omega, T* __restrict__ xout, int bx, int by,
                                                PassSmem<T, kTCX, kTCY>& S, bool active = true) {
  if (!active) bx = by = 0;
  constexpr int kTileThreads = 4 * kTCX * kTCY;
  static_assert(NTT >= kTileThreads && NTT % 32 == 0 && kTileThreads % 32 == 0, "tile group");
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1, sy = g.ny / 2 + 1;
  const int pitch = vanka_pitch(g), nslots = vanka_slots(g);
  const int nn = g.nn;
  const int tx0 = bx * kTCX, ty0 = by * kTCY;
  const int i0 = 2 * tx0 - cx, j0 = 2 * ty0 - cy;  // first node of the tile
  const int t = threadIdx.x % NTT;
  const bool owner = t < kTileThreads;  // owns a node of a colour cell
  // ---- this thread's node (quad q, local node a) and its loads that do not
  // depend on the defect: b, x_in and its three rows of the cell's inverse,
  // issued first so that their latency overlaps the stencil work below
  const int q = t >> 2, a = t & 3;
  const int ti = tx0 + (q % kTCX), tj = ty0 + (q / kTCX);
  const bool slot_ok = owner && ti < sx && tj < sy;
  const int slot = tj * pitch + ti;
  const int ci = 2 * ti - cx, cj = 2 * tj - cy;
  const int i = ci + (a & 1), j = cj + (a >> 1);
  const bool node_ok = slot_ok && i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
  const int n = node_ok ? j * g.nnx + i : 0;
  // every global load of the tile is issued before the first barrier, none
  // depends on another: the thread's b, x_in and three inverse rows (read
  // even for a solid cell, whose rows are then not used), and the staged
  // nodes' flags, iterate, vbar and cell solid flags
  T xu = 0, xv = 0, xp = 0, bu0 = 0, bv0 = 0, bp0 = 0;
  T iv[36];
  if (node_ok) {
    xu = xin[n], xv = xin[nn + n], xp = xin[2 * nn + n];
    bu0 = b[n], bv0 = b[nn + n], bp0 = b[2 * nn + n];
    const T* row0 = inv + (size_t)colour * 144 * nslots + slot;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 12; ++k) iv[c * 12 + k] = row0[(size_t)((c * 4 + a) * 12 + k) * nslots];
  }
  pass_stage_rows<T, kTCX, kTCY, NTT>(g, s, xin, vb, i0, j0, t, S);
  // own cell (ci, cj) sits at staged index (ci - i0 + 2, cj - j0 + 2)
  const bool cell_ok = slot_ok && ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny &&
                       !S.sol[cj - j0 + 2][ci - i0 + 2];
  if (!owner) return;  // helpers are whole warps past the owners
  T du = 0, dv = 0, dp = 0;
  if (node_ok && cell_ok)
    pass_node_defect<T, kTCX, kTCY>(i, j, i0, j0, xu, xv, xp, bu0, bv0, bp0, S, du, dv, dp);
  const int lane = t & 31, base = lane & ~3;
  T d[12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = __shfl_sync(0xffffffffu, du, base + k);
    d[4 + k] = __shfl_sync(0xffffffffu, dv, base + k);
    d[8 + k] = __shfl_sync(0xffffffffu, dp, base + k);
  }
  if (!node_ok || !active) return;
  if (cell_ok) {
    T acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[c] += iv[c * 12 + k] * d[k];
    }
    xout[n] = xu + omega * acc[0];
    xout[nn + n] = xv + omega * acc[1];
    xout[2 * nn + n] = xp + omega * acc[2];
  } else {
    xout[n] = xu;
    xout[nn + n] = xv;
    xout[2 * nn + n] = xp;
  }
}


// The first colour pass of a smoothing sweep that starts from x = 0, for
// item e = 4 * slot + a (node a of the colour cell of `slot`): the defect is
// then b on every row (b - A 0 = b, and b - x = b on constrained rows), so
// the pass needs neither the iterate nor any operator rows:
// x_out = omega A_c^-1 b on the colour's fluid cells and 0 on every other
// node, bitwise what the tiled pass computes from x = 0, and every node of the
// level is written.  The four items of a cell are consecutive lanes of one
// warp; all 32 lanes call this (valid = false for padding items).
template <typename T>
__device__ __forceinline__ void vanka_pass_zero_node(const Grid& g, int colour,
                                                     const T* __restrict__ b,
                                                     const T* __restrict__ inv, T omega,
                                                     T* __restrict__ xout, int e, bool valid) {
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1, pitch = vanka_pitch(g);
  const int nslots = vanka_slots(g);
  const int nn = g.nn;
  const int slot = e >> 2, a = e & 3;
  const bool slot_ok = valid && slot < nslots && slot % pitch < sx;
  const int ci = 2 * (slot % pitch) - cx, cj = 2 * (slot / pitch) - cy;
  const int i = ci + (a & 1), j = cj + (a >> 1);
  const bool node_ok = slot_ok && i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
  const bool cell_ok = slot_ok && ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny &&
                       !g.solid[cj * g.nx + ci];
  const int n = node_ok ? j * g.nnx + i : 0;
  T du = 0, dv = 0, dp = 0;
  if (node_ok) du = b[n], dv = b[nn + n], dp = b[2 * nn + n];
  const int base = (threadIdx.x & 31) & ~3;
  T d[12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = __shfl_sync(0xffffffffu, du, base + k);
    d[4 + k] = __shfl_sync(0xffffffffu, dv, base + k);
    d[8 + k] = __shfl_sync(0xffffffffu, dp, base + k);
  }
  if (!node_ok) return;
  if (cell_ok) {
    // one row of the inverse at a time (fewer live registers)
    const T* row0 = inv + (size_t)colour * 144 * nslots + slot;
    T acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c] = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k)
        acc[c] += row0[(size_t)((c * 4 + a) * 12 + k) * nslots] * d[k];
    }
    xout[n] = T(0) + omega * acc[0];
    xout[nn + n] = T(0) + omega * acc[1];
    xout[2 * nn + n] = T(0) + omega * acc[2];
  } else {
    xout[n] = T(0);
    xout[nn + n] = T(0);
    xout[2 * nn + n] = T(0);
  }
}

}  // namespace dnnmg
