// Cell-wise Vanka smoother (Sec. 2.2 names multigrid as the preconditioner;
// the smoother is cell-wise Vanka with 12x12 local solves).
//
// Setup: for every fluid cell, the restriction of the global Jacobian to the
// cell's 12 DOFs (its 4 nodes x u, v, p), with identity rows/columns on
// constrained DOFs, is inverted by Gauss-Jordan elimination with partial
// pivoting and stored as inv[colour][entry][slot] so that the smoothing pass
// streams it with coalesced loads.
//
// Pass (one colour): four threads (a quad) own one cell, one node each.  Each
// thread evaluates the three operator rows of its node against x_in, the quad
// exchanges its 12 defects by warp shuffles, and every thread writes its
// node's three updated values to x_out.  Cells of one colour share no node;
// nodes outside the colour's fluid cells are copied, so x_out is complete and
// the next colour reads it without races.
#include "kernels.h"
#include "vbody.cuh"

namespace dnnmg {

namespace {

constexpr int kSetupThreads = 128;
constexpr int kPassThreads = 128;

template <typename T>
__device__ __forceinline__ T tabs(T v) {
  return v < T(0) ? -v : v;
}

template <typename T>
__global__ void __launch_bounds__(kSetupThreads)
    vanka_setup_kernel(Grid g, Sten<T> s, const T* __restrict__ vb, T* __restrict__ inv,
                       int* status) {
  const int colour = blockIdx.y;
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1;
  const int nslots = sx * (g.ny / 2 + 1);
  const int slot = blockIdx.x * kSetupThreads + threadIdx.x;
  if (slot >= nslots) return;
  const int ci = 2 * (slot % sx) - cx, cj = 2 * (slot / sx) - cy;
  if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny || g.solid[cj * g.nx + ci]) return;

  T A[12][24];
#pragma unroll
  for (int r = 0; r < 12; ++r)
#pragma unroll
    for (int c = 0; c < 24; ++c) A[r][c] = T(0);

  // element contributions of the (up to) 9 cells sharing a node with this one
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int tx = ci + dx, ty = cj + dy;
      if (tx < 0 || ty < 0 || tx >= g.nx || ty >= g.ny || g.solid[ty * g.nx + tx]) continue;
      T bu[4], bv[4];
      load_cell<T, false>(g, vb, tx, ty, 0, bu);
      load_cell<T, false>(g, vb + g.nn, tx, ty, 0, bv);
      GaussData<T> gd;
      gauss_data<T>(bu, bv, gd);
      for (int a = 0; a < 4; ++a) {
        const int alx = (a & 1) - dx, aly = (a >> 1) - dy;
        if (alx < 0 || alx > 1 || aly < 0 || aly > 1) continue;
        for (int b = 0; b < 4; ++b) {
          const int bex = (b & 1) - dx, bey = (b >> 1) - dy;
          if (bex < 0 || bex > 1 || bey < 0 || bey > 1) continue;
          T J[3][3];
          elem_pair<T>(s, gd, alx + 2 * aly, bex + 2 * bey, J);
          for (int c = 0; c < 3; ++c)
            for (int c2 = 0; c2 < 3; ++c2) A[c * 4 + a][c2 * 4 + b] += J[c][c2];
        }
      }
    }
  // local projection stabilisation of the patches containing node pairs
  const int PI0 = ci >> 1, PJ0 = cj >> 1;
  for (int dJ = -1; dJ <= 1; ++dJ)
    for (int dI = -1; dI <= 1; ++dI) {
      const int PI = PI0 + dI, PJ = PJ0 + dJ;
      if (PI < 0 || PJ < 0 || PI >= g.nx / 2 || PJ >= g.ny / 2) continue;
      if (g.solid[(2 * PJ) * g.nx + 2 * PI]) continue;
      for (int a = 0; a < 4; ++a) {
        const int sa = ci + (a & 1) - 2 * PI, ta = cj + (a >> 1) - 2 * PJ;
        if (sa < 0 || sa > 2 || ta < 0 || ta > 2) continue;
        for (int b = 0; b < 4; ++b) {
          const int sb = ci + (b & 1) - 2 * PI, tb = cj + (b >> 1) - 2 * PJ;
          if (sb < 0 || sb > 2 || tb < 0 || tb > 2) continue;
          A[8 + a][8 + b] += s.S9[(sa + 3 * ta) * 9 + sb + 3 * tb];
        }
      }
    }
  // identity rows and columns on constrained DOFs
  for (int a = 0; a < 4; ++a) {
    const uint8_t f = g.flags[(cj + (a >> 1)) * g.nnx + ci + (a & 1)];
    for (int c = 0; c < 3; ++c) {
      const bool cons = (c < 2) ? (f & kVDir) : (f & kPFix);
      if (!cons) continue;
      const int r = c * 4 + a;
      for (int k = 0; k < 12; ++k) A[r][k] = A[k][r] = T(0);
      A[r][r] = T(1);
    }
  }
  for (int r = 0; r < 12; ++r) A[r][12 + r] = T(1);

  // Gauss-Jordan elimination with partial pivoting on [A | I]
  bool ok = true;
  for (int k = 0; k < 12; ++k) {
    int p = k;
    T best = tabs(A[k][k]);
    for (int r = k + 1; r < 12; ++r) {
      const T v = tabs(A[r][k]);
      if (v > best) best = v, p = r;
    }
    if (!(best > T(0))) {
      ok = false;
      break;
    }
    if (p != k)
      for (int c = 0; c < 24; ++c) {
        const T t = A[k][c];
        A[k][c] = A[p][c];
        A[p][c] = t;
      }
    const T ip = T(1) / A[k][k];
    for (int c = 0; c < 24; ++c) A[k][c] *= ip;
    for (int r = 0; r < 12; ++r) {
      if (r == k) continue;
      const T f = A[r][k];
      if (f == T(0)) continue;
      for (int c = 0; c < 24; ++c) A[r][c] -= f * A[k][c];
    }
  }
  if (!ok) atomicOr(status, 1);
  T* out = inv + (size_t)colour * 144 * nslots + slot;
  for (int r = 0; r < 12; ++r)
    for (int c = 0; c < 12; ++c) out[(size_t)(r * 12 + c) * nslots] = ok ? A[r][12 + c] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(kPassThreads)
    vanka_pass_kernel(Grid g, Sten<T> s, int colour, const T* __restrict__ b,
                      const T* __restrict__ xin, const T* __restrict__ vb,
                      const T* __restrict__ inv, T omega, T* __restrict__ xout) {
  vanka_pass_thread<T>(g, s, colour, b, xin, vb, inv, omega, xout,
                       blockIdx.x * kPassThreads + threadIdx.x);
}

}  // namespace

template <typename T>
void launch_vanka_setup(const Grid& g, const Sten<T>& s, const T* vb, T* inv, int* status,
                        cudaStream_t st) {
  dim3 grid(cdiv(vanka_slots(g), kSetupThreads), 4);
  note_launch();
  vanka_setup_kernel<T><<<grid, kSetupThreads, 0, st>>>(g, s, vb, inv, status);
}

template <typename T>
void launch_vanka_pass(const Grid& g, const Sten<T>& s, int colour, const T* b, const T* xin,
                       const T* vb, const T* inv, T omega, T* xout, cudaStream_t st) {
  const int threads = 4 * vanka_slots(g);
  note_launch();
  vanka_pass_kernel<T><<<cdiv(threads, kPassThreads), kPassThreads, 0, st>>>(
      g, s, colour, b, xin, vb, inv, omega, xout);
}

template void launch_vanka_setup<float>(const Grid&, const Sten<float>&, const float*, float*,
                                        int*, cudaStream_t);
template void launch_vanka_setup<double>(const Grid&, const Sten<double>&, const double*,
                                         double*, int*, cudaStream_t);
template void launch_vanka_pass<float>(const Grid&, const Sten<float>&, int, const float*,
                                       const float*, const float*, const float*, float, float*,
                                       cudaStream_t);
template void launch_vanka_pass<double>(const Grid&, const Sten<double>&, int, const double*,
                                        const double*, const double*, const double*, double,
                                        double*, cudaStream_t);

}  // namespace dnnmg
