// Shared device-side definitions of the DNN-MG CUDA path.
//
// Discretisation (Sec. 2.1, Eqs. 4-5): Q1 velocity and pressure on square
// cells of width h, theta-scheme in time, pressure stabilised by local
// projection onto bilinears of the 2h patch mesh.  Unknowns of a level are
// stored [3][ny+1][nx+1] (u, v, p; x index fastest).  Every operator row is
// evaluated matrix-free at its node from the (up to) four cells and four
// patches around it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dnnmg {

constexpr int kMaxLevels = 12;
constexpr uint8_t kVDir = 1;   // velocity Dirichlet node
constexpr uint8_t kPFix = 2;   // pressure fixed (node touches no fluid cell)

// Abscissae of the 2-point Gauss rule on [0, 1]: (1 -+ 1/sqrt(3)) / 2.
constexpr double kG0 = 0.21132486540518711775;
constexpr double kG1 = 0.78867513459481288225;

struct Grid {
  int nx, ny;          // cells
  int nnx, nny, nn;    // nodes
  double h;
  const uint8_t* solid;  // [ny*nx]
  const uint8_t* flags;  // [nn]
};

// Per-level constants of the linear part of the operator.
template <typename T>
struct Sten {
  T E[16];    // (1/k) M + theta nu K  (row a, column b)
  T Dx[16];   // int xi_a d/dx phi_b
  T Dy[16];   // int xi_a d/dy phi_b
  T S9[81];   // alpha kappa^T K9 kappa on the 3x3 nodes of a patch
  T wq;       // theta * h^2 / 4, weight of one Gauss point in the convection
  T ih;       // 1 / h
};

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// A scalar derived once per block by its first thread and shared with the
// block (an FP64 square root or division in every thread would make a
// vector kernel FP64-bound on this GPU).  All threads of the block call it.
template <class F>
__device__ __forceinline__ double block_scalar(F f) {
  __shared__ double v;
  if (threadIdx.x == 0) v = f();
  __syncthreads();
  return v;
}

// A scalar mailbox in mapped pinned host memory.  A kernel stores the values
// the host needs (v, iv), then, after a system-scope fence, the sequence
// number of the post; the host polls seq instead of copying the values back
// and synchronising the stream, which shortens each host round trip of the
// Newton and FGMRES loops.  Posts on one stream carry increasing numbers, so
// seq >= t means that post t and every earlier one have landed.
struct HostMail {
  volatile double v[8];
  volatile int iv[8];
  volatile unsigned long long seq;
};

// Values of the four bilinear shape functions and their derivatives (times
// h) at Gauss point q = qx + 2 qy.
template <typename T>
__device__ __forceinline__ void shape_at(int q, T phi[4], T dx[4], T dy[4]) {
  const T gx = (q & 1) ? T(kG1) : T(kG0);
  const T gy = (q >> 1) ? T(kG1) : T(kG0);
  const T fx[2] = {T(1) - gx, gx};
  const T fy[2] = {T(1) - gy, gy};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int bx = b & 1, by = b >> 1;
    phi[b] = fx[bx] * fy[by];
    dx[b] = (bx ? T(1) : T(-1)) * fy[by];
    dy[b] = fx[bx] * (by ? T(1) : T(-1));
  }
}

// The same values for one local node b (a runtime index: selects, not an
// indexed local array).
template <typename T>
__device__ __forceinline__ void shape_one(int q, int b, T& phi, T& dx, T& dy) {
  const T gx = (q & 1) ? T(kG1) : T(kG0);
  const T gy = (q >> 1) ? T(kG1) : T(kG0);
  const T fx = (b & 1) ? gx : T(1) - gx;
  const T fy = (b >> 1) ? gy : T(1) - gy;
  phi = fx * fy;
  dx = ((b & 1) ? T(1) : T(-1)) * fy;
  dy = fx * ((b >> 1) ? T(1) : T(-1));
}

// Rows of local node a of one fluid cell, added to (ru, rv, rp).
//   NONLIN = true : A(x) with x = (wu, wv, wp) (Eqs. 4-5), convection N(w)w.
//   NONLIN = false: A'(vbar) w (Eq. 6), convection N(vbar)w + (w.grad)vbar.
// The pressure row here holds the divergence only; LPS is added per patch.
template <typename T, bool NONLIN>
__device__ __forceinline__ void cell_rows(const Sten<T>& s, int a, const T wu[4], const T wv[4],
                                          const T wp[4], const T bu[4], const T bv[4], T& ru,
                                          T& rv, T& rp) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    ru += s.E[a * 4 + b] * wu[b] - s.Dx[b * 4 + a] * wp[b];
    rv += s.E[a * 4 + b] * wv[b] - s.Dy[b * 4 + a] * wp[b];
    rp += s.Dx[a * 4 + b] * wu[b] + s.Dy[a * 4 + b] * wv[b];
  }
  T cu_acc = 0, cv_acc = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T phi[4], dx[4], dy[4];
    shape_at<T>(q, phi, dx, dy);
    T Wu = 0, Wv = 0, Wux = 0, Wuy = 0, Wvx = 0, Wvy = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      Wu += phi[b] * wu[b];
      Wv += phi[b] * wv[b];
      Wux += dx[b] * wu[b];
      Wuy += dy[b] * wu[b];
      Wvx += dx[b] * wv[b];
      Wvy += dy[b] * wv[b];
    }
    T cu, cv;
    if (NONLIN) {
      cu = Wu * Wux + Wv * Wuy;
      cv = Wu * Wvx + Wv * Wvy;
    } else {
      T Bu = 0, Bv = 0, Bux = 0, Buy = 0, Bvx = 0, Bvy = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        Bu += phi[b] * bu[b];
        Bv += phi[b] * bv[b];
        Bux += dx[b] * bu[b];
        Buy += dy[b] * bu[b];
        Bvx += dx[b] * bv[b];
        Bvy += dy[b] * bv[b];
      }
      cu = Bu * Wux + Bv * Wuy + Wu * Bux + Wv * Buy;
      cv = Bu * Wvx + Bv * Wvy + Wu * Bvx + Wv * Bvy;
    }
    cu_acc += phi[a] * cu;
    cv_acc += phi[a] * cv;
  }
  // derivatives above are per unit reference length: scale by 1/h
  ru += s.wq * s.ih * cu_acc;
  rv += s.wq * s.ih * cv_acc;
}

// Load one field at the four nodes of cell (ci, cj); MASK zeroes the
// constrained entries (flag bit `bit`).
template <typename T, bool MASK>
__device__ __forceinline__ void load_cell(const Grid& g, const T* __restrict__ f, int ci, int cj,
                                          uint8_t bit, T out[4]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int n = (cj + (b >> 1)) * g.nnx + ci + (b & 1);
    T v = f[n];
    if (MASK && (g.flags[n] & bit)) v = T(0);
    out[b] = v;
  }
}

// Full operator rows (u, v, p) at node (i, j) of a level.
//   w : [3][nn] field (state for NONLIN, direction for the Jacobian)
//   vb: [2][nn] linearisation velocity (Jacobian only)
// With MASK, constrained entries of w are read as zero (the Jacobian acts on
// free DOFs only); constrained rows are handled by the caller.
template <typename T, bool NONLIN, bool MASK>
__device__ __forceinline__ void node_rows(const Grid& g, const Sten<T>& s, int i, int j,
                                          const T* __restrict__ w, const T* __restrict__ vb,
                                          T& ru, T& rv, T& rp) {
  ru = rv = rp = T(0);
  const int nn = g.nn;
#pragma unroll
  for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
    for (int cx = 0; cx < 2; ++cx) {
      const int ci = i - 1 + cx, cj = j - 1 + cy;
      if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) continue;
      if (g.solid[cj * g.nx + ci]) continue;
      const int a = (1 - cx) + 2 * (1 - cy);
      T wu[4], wv[4], wp[4], bu[4], bv[4];
      load_cell<T, MASK>(g, w, ci, cj, kVDir, wu);
      load_cell<T, MASK>(g, w + nn, ci, cj, kVDir, wv);
      load_cell<T, MASK>(g, w + 2 * nn, ci, cj, kPFix, wp);
      if (!NONLIN) {
        load_cell<T, false>(g, vb, ci, cj, 0, bu);
        load_cell<T, false>(g, vb + nn, ci, cj, 0, bv);
      }
      cell_rows<T, NONLIN>(s, a, wu, wv, wp, bu, bv, ru, rv, rp);
    }
  }
  // local projection stabilisation, patches I with 2I <= i <= 2I+2
  const T* p = w + 2 * nn;
  const int npx = g.nx >> 1, npy = g.ny >> 1;
#pragma unroll
  for (int dJ = 0; dJ < 2; ++dJ) {
    const int J = (j >> 1) - dJ;
    if (J < 0 || J >= npy || j - 2 * J > 2) continue;
#pragma unroll
    for (int dI = 0; dI < 2; ++dI) {
      const int I = (i >> 1) - dI;
      if (I < 0 || I >= npx || i - 2 * I > 2) continue;
      if (g.solid[(2 * J) * g.nx + 2 * I]) continue;
      const int mn = (i - 2 * I) + 3 * (j - 2 * J);
      T acc = 0;
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        const int n = (2 * J + m / 3) * g.nnx + 2 * I + m % 3;
        T pv = p[n];
        if (MASK && (g.flags[n] & kPFix)) pv = T(0);
        acc += s.S9[mn * 9 + m] * pv;
      }
      rp += acc;
    }
  }
}

// Gauss-point values of a linearisation velocity on one cell (derivatives
// per unit reference length).
template <typename T>
struct GaussData {
  T Bu[4], Bv[4], Bux[4], Buy[4], Bvx[4], Bvy[4];
};

template <typename T>
__device__ __forceinline__ void gauss_data(const T bu[4], const T bv[4], GaussData<T>& gd) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T phi[4], dx[4], dy[4];
    shape_at<T>(q, phi, dx, dy);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      a0 += phi[b] * bu[b];
      a1 += phi[b] * bv[b];
      a2 += dx[b] * bu[b];
      a3 += dy[b] * bu[b];
      a4 += dx[b] * bv[b];
      a5 += dy[b] * bv[b];
    }
    gd.Bu[q] = a0, gd.Bv[q] = a1, gd.Bux[q] = a2, gd.Buy[q] = a3, gd.Bvx[q] = a4, gd.Bvy[q] = a5;
  }
}

// Element Jacobian A'_T(vbar) entries between local nodes al (row) and be
// (column): J[c][c'] for components (u, v, p) (Eq. 6, before LPS).
template <typename T>
__device__ __forceinline__ void elem_pair(const Sten<T>& s, const GaussData<T>& gd, int al, int be,
                                          T J[3][3]) {
  T N = 0, Cuu = 0, Cuv = 0, Cvu = 0, Cvv = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T pa, dxa, dya, pb, dxb, dyb;
    shape_one<T>(q, al, pa, dxa, dya);
    shape_one<T>(q, be, pb, dxb, dyb);
    const T pab = pa * pb;
    N += pa * (gd.Bu[q] * dxb + gd.Bv[q] * dyb);
    Cuu += pab * gd.Bux[q];
    Cuv += pab * gd.Buy[q];
    Cvu += pab * gd.Bvx[q];
    Cvv += pab * gd.Bvy[q];
  }
  const T sc = s.wq * s.ih;
  const T e = s.E[al * 4 + be];
  J[0][0] = e + sc * (N + Cuu);
  J[0][1] = sc * Cuv;
  J[0][2] = -s.Dx[be * 4 + al];
  J[1][0] = sc * Cvu;
  J[1][1] = e + sc * (N + Cvv);
  J[1][2] = -s.Dy[be * 4 + al];
  J[2][0] = s.Dx[al * 4 + be];
  J[2][1] = s.Dy[al * 4 + be];
  J[2][2] = T(0);
}

// All twelve rows (u0..u3, v0..v3, p0..p3) of one fluid cell's contribution
// to A'(vbar) w (NONLIN = false) or A(w) (NONLIN = true); the Gauss-point
// values are computed once for the cell.  Pressure rows hold the divergence
// only (LPS is added per patch).
template <typename T, bool NONLIN>
__device__ __forceinline__ void cell_all_rows(const Sten<T>& s, const T wu[4], const T wv[4],
                                              const T wp[4], const T bu[4], const T bv[4],
                                              T r[12]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T ru = 0, rv = 0, rp = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      ru += s.E[a * 4 + b] * wu[b] - s.Dx[b * 4 + a] * wp[b];
      rv += s.E[a * 4 + b] * wv[b] - s.Dy[b * 4 + a] * wp[b];
      rp += s.Dx[a * 4 + b] * wu[b] + s.Dy[a * 4 + b] * wv[b];
    }
    r[a] = ru, r[4 + a] = rv, r[8 + a] = rp;
  }
  const T sc = s.wq * s.ih;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T phi[4], dx[4], dy[4];
    shape_at<T>(q, phi, dx, dy);
    T Wu = 0, Wv = 0, Wux = 0, Wuy = 0, Wvx = 0, Wvy = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      Wu += phi[b] * wu[b];
      Wv += phi[b] * wv[b];
      Wux += dx[b] * wu[b];
      Wuy += dy[b] * wu[b];
      Wvx += dx[b] * wv[b];
      Wvy += dy[b] * wv[b];
    }
    T cu, cv;
    if (NONLIN) {
      cu = Wu * Wux + Wv * Wuy;
      cv = Wu * Wvx + Wv * Wvy;
    } else {
      T Bu = 0, Bv = 0, Bux = 0, Buy = 0, Bvx = 0, Bvy = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        Bu += phi[b] * bu[b];
        Bv += phi[b] * bv[b];
        Bux += dx[b] * bu[b];
        Buy += dy[b] * bu[b];
        Bvx += dx[b] * bv[b];
        Bvy += dy[b] * bv[b];
      }
      cu = Bu * Wux + Bv * Wuy + Wu * Bux + Wv * Buy;
      cv = Bu * Wvx + Bv * Wvy + Wu * Bvx + Wv * Bvy;
    }
    cu *= sc;
    cv *= sc;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      r[a] += phi[a] * cu;
      r[4 + a] += phi[a] * cv;
    }
  }
}

}  // namespace dnnmg
