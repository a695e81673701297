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
  apply_node<T>(g, s, w, vb, y, i, j);
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
  residual64_node(g, s, x, f, r, i, j);
}

__global__ void __launch_bounds__(kBX* kBY)
    old_rhs64_kernel(Grid g, double inv_k, const double* __restrict__ x, double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  old_rhs64_node(g, inv_k, x, f, i, j);
}

__global__ void __launch_bounds__(kBX* kBY)
    explicit_sub64_kernel(Grid g, Sten<double> sx, double coef, const double* __restrict__ x,
                          double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  explicit_sub64_node(g, sx, coef, x, f, i, j);
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
