// One V(nu1, nu2) cycle in a single persistent launch: a cooperative grid,
// or one thread-block cluster (up to 16 blocks on 16 SMs).
//
// The cycle (Sec. 2.2: multigrid as the GMRES preconditioner) is a fixed
// sequence of phases -- Vanka colour passes, defect, restriction (with the
// coarse iterate zeroed), the coarse direct solve, prolongation -- built once
// per top level on the host.  The kernel walks the phase list; all blocks
// work on a phase with grid-stride loops and meet at a barrier (grid-wide,
// or the hardware cluster barrier) before the next.  Every phase runs the same per-thread bodies as the
// one-launch-per-stage kernels, so the arithmetic is identical; only the
// ~20 kernel launches per level and cycle disappear.
#include <cooperative_groups.h>

#include "kernels.h"
#include "vanka_body.cuh"
#include "vbody.cuh"
#include "vcycle.h"

namespace cg = cooperative_groups;

namespace dnnmg {

namespace {

constexpr int kThreads = 256;        // threads per block, cooperative grid
// threads per block of the single-cluster launch (FP64 needs more registers)
template <typename T>
constexpr int cluster_threads() {
  return sizeof(T) == 4 ? 512 : 256;
}

constexpr int kTCX = 16, kTCY = 4;  // colour-pass tile of the persistent kernels
constexpr int kMaxPhases = 160;  // phases of one launch (a V(2,2) cycle from level 8)
constexpr int kMaxVLevels = 10;

// Shared-memory copies of the launch's phase list and level records, loaded
// once so that no phase starts with a dependent global load.
template <typename T>
struct WalkSmem {
  VLevel<T> lv[kMaxVLevels];
  Phase ph[kMaxPhases];
};

// Walk the phase list; `sync` separates phases (a grid-wide barrier for the
// cooperative launch, the cluster barrier for the single-cluster launch).
// Threads of all blocks split every phase with grid-stride loops.
template <typename T, int NT, class Sync>
__device__ __forceinline__ void walk_phases(const VLevel<T>* __restrict__ glv,
                                            const Phase* __restrict__ gph, int nph, int top,
                                            const T* __restrict__ topb, T* __restrict__ topx,
                                            const double* __restrict__ Ainv, T omega,
                                            double* sbuf, PassSmem<T, kTCX, kTCY>* tsm,
                                            WalkSmem<T>& S, Sync sync) {
  const int nthreads = gridDim.x * NT;
  const int gtid = blockIdx.x * NT + threadIdx.x;
  {
    const int nl = top + 1;
    const int* src = reinterpret_cast<const int*>(glv);
    int* dst = reinterpret_cast<int*>(S.lv);
    for (int e = threadIdx.x; e < (int)(nl * sizeof(VLevel<T>) / sizeof(int)); e += NT)
      dst[e] = src[e];
    const int* ps = reinterpret_cast<const int*>(gph);
    int* pd = reinterpret_cast<int*>(S.ph);
    for (int e = threadIdx.x; e < (int)(nph * sizeof(Phase) / sizeof(int)); e += NT) pd[e] = ps[e];
    __syncthreads();
  }
  for (int p = 0; p < nph; ++p) {
    const Phase f = S.ph[p];
    const int k = f.level;
    const VLevel<T>& L = S.lv[k];
    const Grid& g = L.g;
    const Sten<T>& ss = L.s;
    const T* b = k == top ? topb : L.b;
    T* x0 = k == top ? topx : L.x;
    switch (f.type) {
      case kPhasePass: {
        // tiles of kTCX x kTCY colour cells, NT / (4 kTCX kTCY) tiles per block at a time
        const T* xin = f.in ? L.x2 : x0;
        T* xout = f.out ? L.x2 : x0;
        constexpr int kTiles = NT / (4 * kTCX * kTCY);
        const int sub = threadIdx.x / (4 * kTCX * kTCY);
        const int nbx = cdiv(g.nx / 2 + 1, kTCX);
        const int nt = nbx * cdiv(g.ny / 2 + 1, kTCY);
        for (int t0 = blockIdx.x * kTiles; t0 < nt; t0 += gridDim.x * kTiles) {
          const int t = t0 + sub;
          vanka_pass_tile<T, kTCX, kTCY>(g, ss, f.colour, b, xin, L.vb, L.inv, omega, xout,
                                         t % nbx, t / nbx, tsm[sub], t < nt);
          __syncthreads();  // the tile's shared memory is reused by the next tile
        }
        break;
      }
      case kPhaseDefect: {
        const T* x = f.in ? L.x2 : x0;
        for (int n = gtid; n < g.nn; n += nthreads)
          defect_node<T>(g, ss, b, x, L.vb, L.d, true, n % g.nnx, n / g.nnx);
        break;
      }
      case kPhaseRestrict: {
        const VLevel<T>& C = S.lv[k - 1];
        const Grid& c = C.g;
        for (int n = gtid; n < c.nn; n += nthreads) {
          restrict_node<T, true>(g, c, L.d, C.b, 3, n % c.nnx, n / c.nnx);
          C.x[n] = T(0);
          C.x[c.nn + n] = T(0);
          C.x[2 * c.nn + n] = T(0);
        }
        break;
      }
      case kPhaseCoarse: {
        const int nd = 3 * g.nn;
        for (int q = threadIdx.x; q < nd; q += NT) sbuf[q] = (double)b[band_to_level(g, q)];
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
        const VLevel<T>& C = S.lv[k - 1];
        T* x = f.in ? L.x2 : x0;
        for (int n = gtid; n < g.nn; n += nthreads)
          prolong_add_node<T>(g, C.g, C.x, x, n % g.nnx, n / g.nnx);
        break;
      }
      case kPhaseZeroTop: {
        for (int n = gtid; n < 3 * g.nn; n += nthreads) topx[n] = T(0);
        break;
      }
    }
    sync();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    vcycle_kernel(const VLevel<T>* __restrict__ lv, const Phase* __restrict__ ph, int nph, int top,
                  const T* __restrict__ topb, T* __restrict__ topx, const double* __restrict__ Ainv,
                  T omega) {
  extern __shared__ __align__(16) uint8_t dyn[];  // coarse vector or pass tiles
  __shared__ WalkSmem<T> S;
  cg::grid_group grid = cg::this_grid();
  walk_phases<T, kThreads>(lv, ph, nph, top, topb, topx, Ainv, omega,
                           reinterpret_cast<double*>(dyn),
                           reinterpret_cast<PassSmem<T, kTCX, kTCY>*>(dyn), S,
                           [&] { grid.sync(); });
}

// The whole grid is one thread-block cluster; phases are separated by the
// cluster barrier (release / acquire at cluster scope, so the global-memory
// results of one phase are visible to every block of the cluster in the next).
template <typename T>
__global__ void __launch_bounds__(cluster_threads<T>())
    vcycle_cluster_kernel(const VLevel<T>* __restrict__ lv, const Phase* __restrict__ ph, int nph,
                          int top, const T* __restrict__ topb, T* __restrict__ topx,
                          const double* __restrict__ Ainv, T omega) {
  extern __shared__ __align__(16) uint8_t dyn[];  // coarse vector or pass tiles
  __shared__ WalkSmem<T> S;
  cg::cluster_group cl = cg::this_cluster();
  walk_phases<T, cluster_threads<T>()>(lv, ph, nph, top, topb, topx, Ainv, omega,
                                       reinterpret_cast<double*>(dyn),
                                       reinterpret_cast<PassSmem<T, kTCX, kTCY>*>(dyn), S,
                                       [&] { cl.sync(); });
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

namespace {
// dynamic shared memory of a block of nt threads: the coarse right-hand
// side (FP64) or the block's pass tiles, whichever is larger
template <typename T>
size_t walk_smem(int coarse_nd, int nt) {
  const size_t tiles = sizeof(PassSmem<T, kTCX, kTCY>) * (nt / (4 * kTCX * kTCY));
  const size_t cv = sizeof(double) * coarse_nd;
  return tiles > cv ? tiles : cv;
}
}  // namespace

bool vcycle_fits(int nphases, int nlevels) {
  return nphases <= kMaxPhases && nlevels <= kMaxVLevels;
}

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
  const size_t smem = walk_smem<T>(coarse_nd, kThreads);
  if (cudaFuncSetAttribute(vcycle_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
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
                                  walk_smem<T>(coarse_nd, kThreads), st);
  return e == cudaSuccess ? 0 : 1;
}

template <typename T>
int vcycle_cluster_size(int coarse_nd) {
  const size_t smem = walk_smem<T>(coarse_nd, cluster_threads<T>());
  if (cudaFuncSetAttribute(vcycle_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cs : {16, 8}) {
    if (cs > 8 && cudaFuncSetAttribute(vcycle_cluster_kernel<T>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(cluster_threads<T>());
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void*)vcycle_cluster_kernel<T>, &cfg) == cudaSuccess &&
        n > 0)
      return cs;
    cudaGetLastError();
  }
  return 0;
}

template <typename T>
int launch_vcycle_cluster(const VLevel<T>* lv, const Phase* ph, int nph, int top, const T* topb,
                          T* topx, const double* Ainv, T omega, int cluster, int coarse_nd,
                          cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(cluster_threads<T>());
  cfg.dynamicSmemBytes = walk_smem<T>(coarse_nd, cluster_threads<T>());
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, vcycle_cluster_kernel<T>, lv, ph, nph, top, topb,
                                           topx, Ainv, omega);
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
template int vcycle_cluster_size<float>(int);
template int vcycle_cluster_size<double>(int);
template int launch_vcycle_cluster<float>(const VLevel<float>*, const Phase*, int, int,
                                          const float*, float*, const double*, float, int, int,
                                          cudaStream_t);
template int launch_vcycle_cluster<double>(const VLevel<double>*, const Phase*, int, int,
                                           const double*, double*, const double*, double, int,
                                           int, cudaStream_t);

}  // namespace dnnmg
