// One V(nu1, nu2) cycle in a single persistent cooperative launch.
//
// The cycle (Sec. 2.2: multigrid as the GMRES preconditioner) is a fixed
// sequence of phases -- Vanka colour passes, defect, restriction (with the
// coarse iterate zeroed), the coarse direct solve, prolongation -- built once
// per top level on the host.  The kernel walks the phase list; all blocks
// work on a phase with grid-stride loops and meet at a grid-wide barrier
// before the next.  Every phase runs the same per-thread bodies as the
// one-launch-per-stage kernels, so the arithmetic is identical; only the
// ~20 kernel launches per level and cycle disappear.
#include <cooperative_groups.h>

#include "kernels.h"
#include "vbody.cuh"
#include "vcycle.h"

namespace cg = cooperative_groups;

namespace dnnmg {

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads)
    vcycle_kernel(const VLevel<T>* __restrict__ lv, const Phase* __restrict__ ph, int nph, int top,
                  const T* __restrict__ topb, T* __restrict__ topx, const double* __restrict__ Ainv,
                  T omega) {
  extern __shared__ double sbuf[];
  __shared__ Sten<T> ss;
  cg::grid_group grid = cg::this_grid();
  const int nthreads = gridDim.x * kThreads;
  const int gtid = blockIdx.x * kThreads + threadIdx.x;
  for (int p = 0; p < nph; ++p) {
    const Phase f = ph[p];
    const int k = f.level;
    const Grid g = lv[k].g;
    {  // this level's constants into shared memory
      const T* src = reinterpret_cast<const T*>(&lv[k].s);
      T* dst = reinterpret_cast<T*>(&ss);
      for (int e = threadIdx.x; e < (int)(sizeof(Sten<T>) / sizeof(T)); e += kThreads)
        dst[e] = src[e];
      __syncthreads();
    }
    const T* b = k == top ? topb : lv[k].b;
    T* x0 = k == top ? topx : lv[k].x;
    switch (f.type) {
      case kPhasePass: {
        const T* xin = f.in ? lv[k].x2 : x0;
        T* xout = f.out ? lv[k].x2 : x0;
        const int nq = 4 * vanka_slots(g);
        for (int base = blockIdx.x * kThreads; base < nq; base += nthreads)
          vanka_pass_thread<T>(g, ss, f.colour, b, xin, lv[k].vb, lv[k].inv, omega, xout,
                               base + threadIdx.x);
        break;
      }
      case kPhaseDefect: {
        const T* x = f.in ? lv[k].x2 : x0;
        for (int n = gtid; n < g.nn; n += nthreads)
          defect_node<T>(g, ss, b, x, lv[k].vb, lv[k].d, true, n % g.nnx, n / g.nnx);
        break;
      }
      case kPhaseRestrict: {
        const Grid c = lv[k - 1].g;
        T* bc = lv[k - 1].b;
        T* xc = lv[k - 1].x;
        for (int n = gtid; n < c.nn; n += nthreads) {
          restrict_node<T, true>(g, c, lv[k].d, bc, 3, n % c.nnx, n / c.nnx);
          xc[n] = T(0);
          xc[c.nn + n] = T(0);
          xc[2 * c.nn + n] = T(0);
        }
        break;
      }
      case kPhaseCoarse: {
        const int nd = 3 * g.nn;
        for (int q = threadIdx.x; q < nd; q += kThreads) sbuf[q] = (double)b[band_to_level(g, q)];
        __syncthreads();
        const int warp = gtid >> 5, lane = threadIdx.x & 31, nwarps = nthreads >> 5;
        for (int r = warp; r < nd; r += nwarps) {
          const double* row = Ainv + (size_t)r * nd;
          double acc = 0.0;
          for (int c2 = lane; c2 < nd; c2 += 32) acc += row[c2] * sbuf[c2];
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) x0[band_to_level(g, r)] = (T)acc;
        }
        break;
      }
      case kPhaseProlong: {
        const Grid c = lv[k - 1].g;
        T* x = f.in ? lv[k].x2 : x0;
        for (int n = gtid; n < g.nn; n += nthreads)
          prolong_add_node<T>(g, c, lv[k - 1].x, x, n % g.nnx, n / g.nnx);
        break;
      }
      case kPhaseZeroTop: {
        for (int n = gtid; n < 3 * g.nn; n += nthreads) topx[n] = T(0);
        break;
      }
    }
    grid.sync();
  }
}

void build_phases(int k, int top, int nu1, int nu2, std::vector<Phase>& out) {
  if (k == 0) {
    out.push_back({kPhaseCoarse, 0, 0, 0, 0});
    return;
  }
  int cur = 0;
  for (int s = 0; s < nu1; ++s)
    for (int c = 0; c < 4; ++c) {
      out.push_back({kPhasePass, k, c, cur, 1 - cur});
      cur ^= 1;
    }
  out.push_back({kPhaseDefect, k, 0, cur, 0});
  out.push_back({kPhaseRestrict, k, 0, 0, 0});
  build_phases(k - 1, top, nu1, nu2, out);
  out.push_back({kPhaseProlong, k, 0, cur, 0});
  for (int s = 0; s < nu2; ++s)
    for (int c = 0; c < 4; ++c) {
      out.push_back({kPhasePass, k, c, cur, 1 - cur});
      cur ^= 1;
    }
  (void)top;
}

}  // namespace

std::vector<Phase> vcycle_phases(int top, int nu1, int nu2) {
  std::vector<Phase> out;
  out.push_back({kPhaseZeroTop, top, 0, 0, 0});
  build_phases(top, top, nu1, nu2, out);
  return out;
}

template <typename T>
int vcycle_grid(int coarse_nd) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = sizeof(double) * coarse_nd;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vcycle_kernel<T>, kThreads, smem) !=
          cudaSuccess ||
      per <= 0)
    return 0;
  if (per > 4) per = 4;
  return per * sms;
}

template <typename T>
int launch_vcycle_persistent(const VLevel<T>* lv, const Phase* ph, int nph, int top, const T* topb,
                             T* topx, const double* Ainv, T omega, int grid, int coarse_nd,
                             cudaStream_t st) {
  void* args[] = {(void*)&lv, (void*)&ph, (void*)&nph, (void*)&top, (void*)&topb,
                  (void*)&topx, (void*)&Ainv, (void*)&omega};
  note_launch();
  const cudaError_t e =
      cudaLaunchCooperativeKernel((void*)vcycle_kernel<T>, dim3(grid), dim3(kThreads), args,
                                  sizeof(double) * coarse_nd, st);
  return e == cudaSuccess ? 0 : 1;
}

template int vcycle_grid<float>(int);
template int vcycle_grid<double>(int);
template int launch_vcycle_persistent<float>(const VLevel<float>*, const Phase*, int, int,
                                             const float*, float*, const double*, float, int, int,
                                             cudaStream_t);
template int launch_vcycle_persistent<double>(const VLevel<double>*, const Phase*, int, int,
                                              const double*, double*, const double*, double, int,
                                              int, cudaStream_t);

}  // namespace dnnmg
