// Per-thread bodies of the multigrid kernels, shared by the one-launch-per-
// stage kernels, the persistent V-cycle kernel and the batched kernels.
#pragma once
#include "common.cuh"

namespace dnnmg {

// One colour pass of the Vanka smoother for global thread `tid` (four
// consecutive threads form the quad of one cell; every lane of a warp must
// call this together because of the shuffles).  See vanka.cu.
template <typename T>
__device__ __forceinline__ void vanka_pass_thread(const Grid& g, const Sten<T>& s, int colour,
                                                  const T* __restrict__ b,
                                                  const T* __restrict__ xin,
                                                  const T* __restrict__ vb,
                                                  const T* __restrict__ inv, T omega,
                                                  T* __restrict__ xout, int tid) {
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1, pitch = vanka_pitch(g);
  const int nslots = vanka_slots(g);
  const int slot = tid >> 2, a = tid & 3;
  const bool slot_ok = slot < nslots && slot % pitch < sx;
  const int ci = 2 * (slot % pitch) - cx, cj = 2 * (slot / pitch) - cy;
  const int i = ci + (a & 1), j = cj + (a >> 1);
  const bool node_ok = slot_ok && i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
  const bool cell_ok = slot_ok && ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny &&
                       !g.solid[(cj < 0 ? 0 : cj) * g.nx + (ci < 0 ? 0 : ci)];
  const int nn = g.nn;
  const int n = node_ok ? j * g.nnx + i : 0;
  // loads independent of the defect first (latency overlaps the stencil)
  T xu = 0, xv = 0, xp = 0, b0 = 0, b1 = 0, b2 = 0;
  T iv[36];
  if (node_ok) {
    xu = xin[n], xv = xin[nn + n], xp = xin[2 * nn + n];
    b0 = b[n], b1 = b[nn + n], b2 = b[2 * nn + n];
  }
  if (node_ok && cell_ok) {
    const T* row0 = inv + (size_t)colour * 144 * nslots + slot;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < 12; ++k) iv[c * 12 + k] = row0[(size_t)((c * 4 + a) * 12 + k) * nslots];
  }
  T du = 0, dv = 0, dp = 0;
  if (node_ok && cell_ok) {
    T ru, rv, rp;
    node_rows<T, false, true>(g, s, i, j, xin, vb, ru, rv, rp);
    const uint8_t f = g.flags[n];
    du = b0 - ((f & kVDir) ? xu : ru);
    dv = b1 - ((f & kVDir) ? xv : rv);
    dp = b2 - ((f & kPFix) ? xp : rp);
  }
  const int lane = threadIdx.x & 31, base = lane & ~3;
  T d[12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = __shfl_sync(0xffffffffu, du, base + k);
    d[4 + k] = __shfl_sync(0xffffffffu, dv, base + k);
    d[8 + k] = __shfl_sync(0xffffffffu, dp, base + k);
  }
  if (!node_ok) return;
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

// d = b - A'(vbar) x at node (i, j); constrained rows: b - x, or 0 if masked.
template <typename T>
__device__ __forceinline__ void defect_node(const Grid& g, const Sten<T>& s, const T* __restrict__ b,
                                            const T* __restrict__ x, const T* __restrict__ vb,
                                            T* __restrict__ d, bool masked, int i, int j) {
  const int n = j * g.nnx + i;
  T ru, rv, rp;
  node_rows<T, false, true>(g, s, i, j, x, vb, ru, rv, rp);
  const uint8_t f = g.flags[n];
  const int nn = g.nn;
  if (f & kVDir) {
    d[n] = masked ? T(0) : b[n] - x[n];
    d[nn + n] = masked ? T(0) : b[nn + n] - x[nn + n];
  } else {
    d[n] = b[n] - ru;
    d[nn + n] = b[nn + n] - rv;
  }
  if (f & kPFix)
    d[2 * nn + n] = masked ? T(0) : b[2 * nn + n] - x[2 * nn + n];
  else
    d[2 * nn + n] = b[2 * nn + n] - rp;
}

__device__ __forceinline__ uint8_t field_bit(int c) { return c < 2 ? kVDir : kPFix; }

// Coarse node (I, J) of R d = P^T d on free DOFs (full-weighting stencil),
// for the first ncomp <= 3 fields.  Every load (flags and the up to 27 fine
// values) is issued in one round before any is used; the sums run in the
// stencil's row order.
template <typename T, bool MASK>
__device__ __forceinline__ void restrict_node(const Grid& f, const Grid& c, const T* __restrict__ d,
                                              T* __restrict__ bc, int ncomp, int I, int J) {
  const int nc = J * c.nnx + I;
  const uint8_t cfl = MASK ? c.flags[nc] : uint8_t(0);
  int nf[9];
  bool in[9];
  uint8_t ffl[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const int i = 2 * I + e % 3 - 1, j = 2 * J + e / 3 - 1;
    in[e] = i >= 0 && i < f.nnx && j >= 0 && j < f.nny;
    nf[e] = in[e] ? j * f.nnx + i : 0;
    ffl[e] = (MASK && in[e]) ? f.flags[nf[e]] : uint8_t(0);
  }
  T v[3][9];
#pragma unroll
  for (int comp = 0; comp < 3; ++comp)
#pragma unroll
    for (int e = 0; e < 9; ++e)
      v[comp][e] = (comp < ncomp && in[e]) ? d[comp * f.nn + nf[e]] : T(0);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    if (comp >= ncomp) break;
    const uint8_t bit = field_bit(comp);
    T acc = 0;
    if (!(MASK && (cfl & bit))) {
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        if (!in[e] || (MASK && (ffl[e] & bit))) continue;
        const int di = e % 3 - 1, dj = e / 3 - 1;
        acc += (di == 0 ? T(1) : T(0.5)) * (dj == 0 ? T(1) : T(0.5)) * v[comp][e];
      }
    }
    bc[comp * c.nn + nc] = acc;
  }
}

// Value of the bilinear interpolant of a coarse field at fine node (i, j).
template <typename T, bool MASK>
__device__ __forceinline__ T interp_node(const Grid& c, const T* __restrict__ xc, uint8_t bit,
                                         int i, int j) {
  const int I0 = i >> 1, J0 = j >> 1;
  const int nI = (i & 1) ? 2 : 1, nJ = (j & 1) ? 2 : 1;
  const T w = T(1) / T(nI * nJ);
  T acc = 0;
  for (int bb = 0; bb < nJ; ++bb)
    for (int aa = 0; aa < nI; ++aa) {
      const int n = (J0 + bb) * c.nnx + I0 + aa;
      if (MASK && (c.flags[n] & bit)) continue;
      acc += xc[n];
    }
  return w * acc;
}

// x += P xc at fine node (i, j) on free DOFs.  The fine flag, the flags and
// values of the up to four coarse nodes and x are loaded in one round; the
// interpolant sums the coarse nodes in the same order as interp_node.
template <typename T>
__device__ __forceinline__ void prolong_add_node(const Grid& f, const Grid& c,
                                                 const T* __restrict__ xc, T* __restrict__ x,
                                                 int i, int j) {
  const int n = j * f.nnx + i;
  const int I0 = i >> 1, J0 = j >> 1;
  const int nI = (i & 1) ? 2 : 1, nJ = (j & 1) ? 2 : 1;
  int m[4];
  bool use[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int aa = e & 1, bb = e >> 1;
    use[e] = aa < nI && bb < nJ;
    m[e] = use[e] ? (J0 + bb) * c.nnx + I0 + aa : 0;
  }
  const uint8_t fl = f.flags[n];
  uint8_t cfl[4];
  T xv[3], cv[3][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) cfl[e] = use[e] ? c.flags[m[e]] : uint8_t(0xFF);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    xv[comp] = x[comp * f.nn + n];
#pragma unroll
    for (int e = 0; e < 4; ++e) cv[comp][e] = use[e] ? xc[comp * c.nn + m[e]] : T(0);
  }
  const T w = T(1) / T(nI * nJ);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    const uint8_t bit = field_bit(comp);
    if (fl & bit) continue;
    T acc = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (!(cfl[e] & bit)) acc += cv[comp][e];
    x[comp * f.nn + n] = xv[comp] + w * acc;
  }
}

// y = A'(vbar) w at node (i, j) on free DOFs, y = w on constrained DOFs.
template <typename T>
__device__ __forceinline__ void apply_node(const Grid& g, const Sten<T>& s, const T* __restrict__ w,
                                           const T* __restrict__ vb, T* __restrict__ y, int i,
                                           int j) {
  const int n = j * g.nnx + i;
  T ru, rv, rp;
  node_rows<T, false, true>(g, s, i, j, w, vb, ru, rv, rp);
  const uint8_t f = g.flags[n];
  y[n] = (f & kVDir) ? w[n] : ru;
  y[g.nn + n] = (f & kVDir) ? w[g.nn + n] : rv;
  y[2 * g.nn + n] = (f & kPFix) ? w[2 * g.nn + n] : rp;
}

// r = f - A(x) at node (i, j) on free DOFs, 0 on constrained DOFs (FP64).
__device__ __forceinline__ void residual64_node(const Grid& g, const Sten<double>& s,
                                                const double* __restrict__ x,
                                                const double* __restrict__ f,
                                                double* __restrict__ r, int i, int j) {
  const int n = j * g.nnx + i;
  double ru, rv, rp;
  node_rows<double, true, false>(g, s, i, j, x, nullptr, ru, rv, rp);
  const uint8_t fl = g.flags[n];
  const int nn = g.nn;
  r[n] = (fl & kVDir) ? 0.0 : f[n] - ru;
  r[nn + n] = (fl & kVDir) ? 0.0 : f[nn + n] - rv;
  r[2 * nn + n] = (fl & kPFix) ? 0.0 : f[2 * nn + n] - rp;
}

// f = (1/k) (v_old, phi) at node (i, j) with the Q1 mass matrix
// (h^2/36) [4 2 2 1] pattern; pressure rows 0.  m = h^2 / 36 / k, formed by
// the caller once (an FP64 division per node is slow on this GPU).
__device__ __forceinline__ void old_rhs64_node(const Grid& g, double m,
                                               const double* __restrict__ x,
                                               double* __restrict__ f, int i, int j) {
  const int n = j * g.nnx + i, nn = g.nn;
  // interior node with four fluid cells: the assembled row, 16 on the node,
  // 4 on its edge neighbours and 1 on its corner neighbours (fewer FP64
  // operations than the sum over the cells; FP64 runs at 1/64 of FP32 here)
  if (i >= 1 && j >= 1 && i < g.nx && j < g.ny && !g.solid[(j - 1) * g.nx + i - 1] &&
      !g.solid[(j - 1) * g.nx + i] && !g.solid[j * g.nx + i - 1] && !g.solid[j * g.nx + i]) {
    const int w = n - 1, e = n + 1, s = n - g.nnx, no = n + g.nnx;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double* xc = x + c * nn;
      const double edges = (xc[w] + xc[e]) + (xc[s] + xc[no]);
      const double corners = (xc[s - 1] + xc[s + 1]) + (xc[no - 1] + xc[no + 1]);
      f[c * nn + n] = m * (16.0 * xc[n] + 4.0 * edges + corners);
    }
    f[2 * nn + n] = 0.0;
    return;
  }
  double fu = 0, fv = 0;
  for (int cy = 0; cy < 2; ++cy)
    for (int cx = 0; cx < 2; ++cx) {
      const int ci = i - 1 + cx, cj = j - 1 + cy;
      if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny || g.solid[cj * g.nx + ci]) continue;
      const int ax = 1 - cx, ay = 1 - cy;
      for (int b = 0; b < 4; ++b) {
        const int bx = b & 1, by = b >> 1;
        const double wgt = (ax == bx ? 2.0 : 1.0) * (ay == by ? 2.0 : 1.0);
        const int nb = (cj + by) * g.nnx + ci + bx;
        fu += wgt * x[nb];
        fv += wgt * x[nn + nb];
      }
    }
  f[n] = m * fu;
  f[nn + n] = m * fv;
  f[2 * nn + n] = 0.0;
}

// f -= coef * [nu (grad v, grad phi) + (v . grad v, phi)] on the velocity
// rows of node (i, j): the explicit part of the theta-scheme (Eq. 5 with
// weight 1 - theta).  sx holds nu K in E, the Gauss weight h^2/4 without
// theta, and no pressure or LPS terms.
__device__ __forceinline__ void explicit_sub64_node(const Grid& g, const Sten<double>& sx,
                                                    double coef, const double* __restrict__ x,
                                                    double* __restrict__ f, int i, int j) {
  const int n = j * g.nnx + i;
  double ru, rv, rp;
  node_rows<double, true, false>(g, sx, i, j, x, nullptr, ru, rv, rp);
  f[n] -= coef * ru;
  f[g.nn + n] -= coef * rv;
}

// coarse (I, J) <- fine (2I, 2J) for ncomp fields
template <typename T>
__device__ __forceinline__ void inject_node(const Grid& f, const Grid& c, const T* __restrict__ xf,
                                            T* __restrict__ xc, int ncomp, int I, int J) {
  for (int comp = 0; comp < ncomp; ++comp)
    xc[comp * c.nn + J * c.nnx + I] = xf[comp * f.nn + (2 * J) * f.nnx + 2 * I];
}

// unmasked bilinear prolongation of ncomp fields at fine node (i, j)
__device__ __forceinline__ void prolong_state_node(const Grid& f, const Grid& c,
                                                   const double* __restrict__ xc,
                                                   double* __restrict__ xf, int ncomp, int i,
                                                   int j) {
  const int n = j * f.nnx + i;
  for (int comp = 0; comp < ncomp; ++comp)
    xf[comp * f.nn + n] = interp_node<double, false>(c, xc + comp * c.nn, 0, i, j);
}

// Band numbering of the coarsest level: DOF p = (i * nny + j) * 3 + c.
__host__ __device__ inline int band_to_level(const Grid& g, int p) {
  const int c = p % 3, node = p / 3;
  const int i = node / g.nny, j = node % g.nny;
  return c * g.nn + j * g.nnx + i;
}

}  // namespace dnnmg
