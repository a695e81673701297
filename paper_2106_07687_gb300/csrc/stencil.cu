// Matrix-free operator kernels: Jacobian apply, defect, FP64 nonlinear
// residual and the old-time right-hand side (Sec. 2.1, Eqs. 4-7).
//
// One thread per node; the 2D block of 32x4 threads covers a tile of nodes
// with x fastest, so each warp reads contiguous rows of the SoA fields.
#include "kernels.h"
#include "vbody.cuh"

namespace dnnmg {

namespace {

constexpr int kBX = 32, kBY = 4;

template <typename T>
__global__ void __launch_bounds__(kBX* kBY) apply_kernel(Grid g, Sten<T> s, const T* __restrict__ w,
                                                         const T* __restrict__ vb,
                                                         T* __restrict__ y) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  const int n = j * g.nnx + i;
  T ru, rv, rp;
  node_rows<T, false, true>(g, s, i, j, w, vb, ru, rv, rp);
  const uint8_t f = g.flags[n];
  y[n] = (f & kVDir) ? w[n] : ru;
  y[g.nn + n] = (f & kVDir) ? w[g.nn + n] : rv;
  y[2 * g.nn + n] = (f & kPFix) ? w[2 * g.nn + n] : rp;
}

template <typename T>
__global__ void __launch_bounds__(kBX* kBY)
    defect_kernel(Grid g, Sten<T> s, const T* __restrict__ b, const T* __restrict__ x,
                  const T* __restrict__ vb, T* __restrict__ d, bool masked) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  defect_node<T>(g, s, b, x, vb, d, masked, i, j);
}

__global__ void __launch_bounds__(kBX* kBY)
    residual64_kernel(Grid g, Sten<double> s, const double* __restrict__ x,
                      const double* __restrict__ f, double* __restrict__ r) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  const int n = j * g.nnx + i;
  double ru, rv, rp;
  node_rows<double, true, false>(g, s, i, j, x, nullptr, ru, rv, rp);
  const uint8_t fl = g.flags[n];
  const int nn = g.nn;
  r[n] = (fl & kVDir) ? 0.0 : f[n] - ru;
  r[nn + n] = (fl & kVDir) ? 0.0 : f[nn + n] - rv;
  r[2 * nn + n] = (fl & kPFix) ? 0.0 : f[2 * nn + n] - rp;
}

// (1/k) (v_old, phi) with the Q1 mass matrix (h^2/36) [4 2 2 1] pattern.
__global__ void __launch_bounds__(kBX* kBY)
    old_rhs64_kernel(Grid g, double inv_k, const double* __restrict__ x, double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  const int n = j * g.nnx + i, nn = g.nn;
  const double m = g.h * g.h / 36.0 * inv_k;
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
// rows: the explicit part of the theta-scheme (Eq. 5 with weight 1 - theta).
// sx holds nu K in E, the Gauss weight h^2/4 without theta, and no pressure
// or LPS terms, so the nonlinear rows of sx are exactly that bracket.
__global__ void __launch_bounds__(kBX* kBY)
    explicit_sub64_kernel(Grid g, Sten<double> sx, double coef, const double* __restrict__ x,
                          double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  const int n = j * g.nnx + i;
  double ru, rv, rp;
  node_rows<double, true, false>(g, sx, i, j, x, nullptr, ru, rv, rp);
  f[n] -= coef * ru;
  f[g.nn + n] -= coef * rv;
}

inline dim3 node_grid(const Grid& g) { return dim3(cdiv(g.nnx, kBX), cdiv(g.nny, kBY)); }

}  // namespace

template <typename T>
void launch_apply(const Grid& g, const Sten<T>& s, const T* w, const T* vb, T* y, cudaStream_t st) {
  note_launch();
  apply_kernel<T><<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, s, w, vb, y);
}

template <typename T>
void launch_defect(const Grid& g, const Sten<T>& s, const T* b, const T* x, const T* vb, T* d,
                   bool masked, cudaStream_t st) {
  note_launch();
  defect_kernel<T><<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, s, b, x, vb, d, masked);
}

void launch_residual64(const Grid& g, const Sten<double>& s, const double* x, const double* f,
                       double* r, cudaStream_t st) {
  note_launch();
  residual64_kernel<<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, s, x, f, r);
}

void launch_old_time_rhs64(const Grid& g, double inv_k, const double* x_old, double* f,
                           cudaStream_t st) {
  note_launch();
  old_rhs64_kernel<<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, inv_k, x_old, f);
}

void launch_explicit_sub64(const Grid& g, const Sten<double>& sx, double coef, const double* x,
                           double* f, cudaStream_t st) {
  note_launch();
  explicit_sub64_kernel<<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, sx, coef, x, f);
}

template void launch_apply<float>(const Grid&, const Sten<float>&, const float*, const float*,
                                  float*, cudaStream_t);
template void launch_apply<double>(const Grid&, const Sten<double>&, const double*, const double*,
                                   double*, cudaStream_t);
template void launch_defect<float>(const Grid&, const Sten<float>&, const float*, const float*,
                                   const float*, float*, bool, cudaStream_t);
template void launch_defect<double>(const Grid&, const Sten<double>&, const double*,
                                    const double*, const double*, double*, bool, cudaStream_t);

}  // namespace dnnmg
