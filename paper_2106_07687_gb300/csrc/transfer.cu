// Grid transfers between nested Q1 levels: bilinear prolongation P, its
// transpose R = P^T, and nodal injection (Sec. 2.2, the prolongation and restriction of Algorithm 1).
// Inside the V-cycle both P and R act on free DOFs only; the DNN-MG state and
// right-hand-side transfers use the unmasked operators.
#include "dnnmg_body.cuh"
#include "kernels.h"
#include "vbody.cuh"

namespace dnnmg {

namespace {

constexpr int kBX = 32, kBY = 4;

template <typename T, bool MASK>
__global__ void restrict_kernel(Grid f, Grid c, const T* __restrict__ d, T* __restrict__ bc,
                                int ncomp) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  if (I >= c.nnx || J >= c.nny) return;
  restrict_node<T, MASK>(f, c, d, bc, ncomp, I, J);
}

template <typename T>
__global__ void prolong_add_kernel(Grid f, Grid c, const T* __restrict__ xc, T* __restrict__ x) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= f.nnx || j >= f.nny) return;
  prolong_add_node<T>(f, c, xc, x, i, j);
}

__global__ void prolong_state_kernel(Grid f, Grid c, const double* __restrict__ xc,
                                     double* __restrict__ xf, int ncomp,
                                     double* __restrict__ ximp) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= f.nnx || j >= f.nny) return;
  prolong_state_node(f, c, xc, xf, ncomp, i, j);
  if (ximp) {  // the same field with the Dirichlet values imposed
    const int n = j * f.nnx + i;
    for (int comp = 0; comp < 3; ++comp) ximp[comp * f.nn + n] = xf[comp * f.nn + n];
    impose_dirichlet_node(f, ximp, i, j);
  }
}

template <typename T>
__global__ void inject_kernel(Grid f, Grid c, const T* __restrict__ xf, T* __restrict__ xc,
                              int ncomp) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  if (I >= c.nnx || J >= c.nny) return;
  inject_node<T>(f, c, xf, xc, ncomp, I, J);
}

template <typename T>
__global__ void linearize_levels_kernel(const __grid_constant__ LinLevels<T> L,
                                        const double* x64, T* vbJ, int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0 && status) *status = 0;
  if (t >= L.off[L.nlev]) return;
  int k = 0;
  while (t >= L.off[k + 1]) ++k;
  const int top = L.nlev - 1, m = top - k;
  const int n = t - L.off[k], J = n / L.nnx[k], I = n - J * L.nnx[k];
  const int f = ((J << m) * L.nnx[top]) + (I << m);
  for (int comp = 0; comp < 2; ++comp) {
    const double v = x64[comp * L.nn[top] + f];
    L.vb64[k][comp * L.nn[k] + n] = v;
    L.vb[k][comp * L.nn[k] + n] = static_cast<T>(v);
    if (k == top) vbJ[comp * L.nn[k] + n] = static_cast<T>(v);
  }
}

inline dim3 grid_of(const Grid& g) { return dim3(cdiv(g.nnx, kBX), cdiv(g.nny, kBY)); }

}  // namespace

template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* d, T* bc, cudaStream_t st) {
  note_launch();
  restrict_kernel<T, true><<<grid_of(coarse), dim3(kBX, kBY), 0, st>>>(fine, coarse, d, bc, 3);
}

template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, T* x, cudaStream_t st) {
  note_launch();
  prolong_add_kernel<T><<<grid_of(fine), dim3(kBX, kBY), 0, st>>>(fine, coarse, xc, x);
}

template <typename T>
void launch_inject(const Grid& fine, const Grid& coarse, const T* xf, T* xc, int ncomp,
                   cudaStream_t st) {
  note_launch();
  inject_kernel<T><<<grid_of(coarse), dim3(kBX, kBY), 0, st>>>(fine, coarse, xf, xc, ncomp);
}

template <typename T>
void launch_linearize_levels(const LinLevels<T>& L, const double* x64, T* vbJ, int* status,
                             cudaStream_t st) {
  note_launch();
  const int n = L.off[L.nlev] > 0 ? L.off[L.nlev] : 1;
  linearize_levels_kernel<T><<<cdiv(n, 256), 256, 0, st>>>(L, x64, vbJ, status);
}

void launch_prolong_state64(const Grid& fine, const Grid& coarse, const double* xc, double* xf,
                            int ncomp, cudaStream_t st, double* ximp) {
  note_launch();
  prolong_state_kernel<<<grid_of(fine), dim3(kBX, kBY), 0, st>>>(fine, coarse, xc, xf, ncomp,
                                                                 ncomp == 3 ? ximp : nullptr);
}

void launch_restrict_full64(const Grid& fine, const Grid& coarse, const double* bf, double* bc,
                            int ncomp, cudaStream_t st) {
  note_launch();
  restrict_kernel<double, false><<<grid_of(coarse), dim3(kBX, kBY), 0, st>>>(fine, coarse, bf, bc,
                                                                             ncomp);
}

#define DNNMG_INST(T)                                                                         \
  template void launch_restrict<T>(const Grid&, const Grid&, const T*, T*, cudaStream_t);     \
  template void launch_prolong_add<T>(const Grid&, const Grid&, const T*, T*, cudaStream_t);  \
  template void launch_inject<T>(const Grid&, const Grid&, const T*, T*, int, cudaStream_t);     \
  template void launch_linearize_levels<T>(const LinLevels<T>&, const double*, T*, int*,        \
                                           cudaStream_t);
DNNMG_INST(float)
DNNMG_INST(double)
#undef DNNMG_INST

}  // namespace dnnmg
