// Cell-wise Vanka smoother (Sec. 2.2 names multigrid as the preconditioner;
// the smoother is cell-wise Vanka with 12x12 local solves): the launchers of
// the setup and of one colour pass.  The per-cell and per-tile arithmetic is
// in vanka_body.cuh.
#include "kernels.h"
#include "vanka_body.cuh"

namespace dnnmg {

namespace {


template <typename T>
__global__ void __launch_bounds__(kSetupThreads)
    vanka_setup_kernel(Grid g, Sten<T> s, const T* __restrict__ vb, T* __restrict__ inv,
                       int* status) {
  __shared__ SetupSmem<T> W[kSetupCells];
  vanka_setup_cell<T>(g, s, vb, inv, status, blockIdx.y,
                      blockIdx.x * kSetupCells + threadIdx.x / 16, W[threadIdx.x / 16]);
}

template <typename T, int TCX, int TCY>
__global__ void __launch_bounds__(4 * TCX * TCY, pass_min_blocks<T>(4 * TCX * TCY))
    vanka_pass_tiled_kernel(Grid g, Sten<T> s, int colour, const T* __restrict__ b,
                            const T* __restrict__ xin, const T* __restrict__ vb,
                            const T* __restrict__ inv, T omega, T* __restrict__ xout) {
  extern __shared__ __align__(16) uint8_t smraw[];
  PassSmem<T, TCX, TCY>& S = *reinterpret_cast<PassSmem<T, TCX, TCY>*>(smraw);
  vanka_pass_tile<T, TCX, TCY>(g, s, colour, b, xin, vb, inv, omega, xout, blockIdx.x, blockIdx.y,
                               S);
}

template <typename T, int TCX, int TCY>
void pass_shape(const Grid& g, const Sten<T>& s, int colour, const T* b, const T* xin, const T* vb,
                const T* inv, T omega, T* xout, cudaStream_t st) {
  const dim3 grid(cdiv(g.nx / 2 + 1, TCX), cdiv(g.ny / 2 + 1, TCY));
  const size_t smem = sizeof(PassSmem<T, TCX, TCY>);
  static bool attr = false;
  if (!attr && smem > 48 * 1024) {
    cudaFuncSetAttribute(vanka_pass_tiled_kernel<T, TCX, TCY>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  note_launch();
  vanka_pass_tiled_kernel<T, TCX, TCY><<<grid, 4 * TCX * TCY, smem, st>>>(g, s, colour, b, xin, vb,
                                                                          inv, omega, xout);
}

}  // namespace

template <typename T>
void launch_vanka_setup(const Grid& g, const Sten<T>& s, const T* vb, T* inv, int* status,
                        cudaStream_t st) {
  dim3 grid(cdiv(vanka_slots(g), kSetupCells), 4);
  note_launch();
  vanka_setup_kernel<T><<<grid, kSetupThreads, 0, st>>>(g, s, vb, inv, status);
}

template <typename T>
void launch_vanka_pass(const Grid& g, const Sten<T>& s, int colour, const T* b, const T* xin,
                       const T* vb, const T* inv, T omega, T* xout, cudaStream_t st, int shape) {
  switch (shape) {
    case 1:
      pass_shape<T, 8, 4>(g, s, colour, b, xin, vb, inv, omega, xout, st);
      break;
    case 2:
      pass_shape<T, 8, 8>(g, s, colour, b, xin, vb, inv, omega, xout, st);
      break;
    default:
      pass_shape<T, 16, 4>(g, s, colour, b, xin, vb, inv, omega, xout, st);
      break;
  }
}

template void launch_vanka_setup<float>(const Grid&, const Sten<float>&, const float*, float*,
                                        int*, cudaStream_t);
template void launch_vanka_setup<double>(const Grid&, const Sten<double>&, const double*,
                                         double*, int*, cudaStream_t);
template void launch_vanka_pass<float>(const Grid&, const Sten<float>&, int, const float*,
                                       const float*, const float*, const float*, float, float*,
                                       cudaStream_t, int);
template void launch_vanka_pass<double>(const Grid&, const Sten<double>&, int, const double*,
                                        const double*, const double*, const double*, double,
                                        double*, cudaStream_t, int);

}  // namespace dnnmg
