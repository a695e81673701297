// One V(nu1, nu2) cycle in a single persistent launch: a cooperative grid,
// or one thread-block cluster (up to 16 blocks on 16 SMs).
//
// The cycle (Sec. 2.2: multigrid as the GMRES preconditioner) is a fixed
// sequence of phases -- Vanka colour passes, defect, restriction (with the
// coarse iterate zeroed), the coarse direct solve, prolongation -- built once
// per top level on the host.  The kernel walks the phase list; all blocks
// share every phase and meet at a barrier (grid-wide, or the hardware cluster
// barrier) before the next.  Every phase runs the same per-thread bodies as
// the one-launch-per-stage kernels, so the arithmetic is identical; only the
// ~20 kernel launches per level and cycle disappear.
#include <algorithm>
#include <cooperative_groups.h>

#include "kernels.h"
#include "optile_body.cuh"
#include "vanka_body.cuh"
#include "vbody.cuh"
#include "vcycle.h"

namespace cg = cooperative_groups;

namespace dnnmg {

namespace {

// Colour-pass tiles (colour cells).  The cooperative kernel takes 8 x 4
// tiles, one per block at a time: on the small levels of a sub-cycle the
// tile's cell rows (ALU-bound on one SM) are the longest part of a pass, and
// smaller tiles spread a level over more SMs.  Its blocks have 256 threads:
// 128 own the tile's nodes and 128 help stage it and compute its rows.  The
// single-cluster kernel (16 blocks) keeps 16 x 4 tiles, two per block.
constexpr int kCTX = 8, kCTY = 4;
constexpr int kLTX = 16, kLTY = 4;
constexpr int kCoopOwners = 4 * kCTX * kCTY;
constexpr int kCoopThreads = 2 * kCoopOwners;
constexpr int kClusterOwners = 4 * kLTX * kLTY;
// threads per block of the single-cluster launch (FP64 needs more registers)
template <typename T>
constexpr int cluster_threads() {
  return sizeof(T) == 4 ? 2 * kClusterOwners : kClusterOwners;
}
constexpr int kMaxPhases = 160;  // phases of one launch (a V(2,2) cycle from level 8)
constexpr int kMaxVLevels = 10;

// Shared-memory copies of the launch's phase list and level records, loaded
// once so that no phase starts with a dependent global load.
template <typename T>
struct WalkSmem {
  VLevel<T> lv[kMaxVLevels];
  Phase ph[kMaxPhases];
};

// Item n < count of a node-wise phase for every thread of the grid: chunks
// of 32 consecutive items (one warp, coalesced) go round-robin over the
// blocks first, so that a small level still spreads over all of them.
template <int NT, class F>
__device__ __forceinline__ void for_items(int count, F f) {
  constexpr int kWarps = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nchunks = (count + 31) >> 5;
  for (int c = blockIdx.x + gridDim.x * w; c < nchunks; c += gridDim.x * kWarps) {
    const int n = (c << 5) + lane;
    if (n < count) f(n);
  }
}

// Walk the phase list; `sync` separates phases (a grid-wide barrier for the
// cooperative launch, the cluster barrier for the single-cluster launch).
// Threads of all blocks split every node-wise phase; a colour pass gives each
// group of NTT threads of a block one TCX x TCY tile at a time.
template <typename T, int TCX, int TCY, int NT, int NTT, class Sync>
__device__ __forceinline__ void walk_phases(const VLevel<T>* __restrict__ glv,
                                            const Phase* __restrict__ gph, int nph, int top,
                                            const T* __restrict__ topb, T* __restrict__ topx,
                                            const double* __restrict__ Ainv, T omega,
                                            uint8_t* dyn, WalkSmem<T>& S, Sync sync) {
  // dynamic shared memory: the pass tiles, the defect tile or the coarse vector
  double* sbuf = reinterpret_cast<double*>(dyn);
  PassSmem<T, TCX, TCY>* tsm = reinterpret_cast<PassSmem<T, TCX, TCY>*>(dyn);
  constexpr int kDX = 16, kDY = 8;  // defect tile: owners plus helpers, as a pass tile
  auto& dsm = *reinterpret_cast<OpSmem<T, kDX, kDY>*>(dyn);
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
  constexpr int kTiles = NT / NTT;  // pass tiles in flight per block
  const int sub = threadIdx.x / NTT;
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
        // tiles of TCX x TCY colour cells, kTiles per block at a time
        const T* xin = f.in ? L.x2 : x0;
        T* xout = f.out ? L.x2 : x0;
        const int nbx = cdiv(g.nx / 2 + 1, TCX);
        const int nt = nbx * cdiv(g.ny / 2 + 1, TCY);
        for (int t0 = blockIdx.x * kTiles; t0 < nt; t0 += gridDim.x * kTiles) {
          const int t = t0 + sub;
          vanka_pass_tile<T, TCX, TCY, NTT>(g, ss, f.colour, b, xin, L.vb, L.inv, omega, xout,
                                            t % nbx, t / nbx, tsm[sub], t < nt);
          __syncthreads();  // the tile's shared memory is reused by the next tile
        }
        break;
      }
      case kPhaseDefect: {
        // tiles of kDX x kDY nodes, each cell's rows computed once per tile
        const T* x = f.in ? L.x2 : x0;
        const int ntx = cdiv(g.nnx, kDX), ntiles = ntx * cdiv(g.nny, kDY);
        const int nn = g.nn;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
          T ru, rv, rp;
          int n;
          op_tile_rows<T, false, true, kDX, kDY, NT>(g, ss, x, L.vb, t % ntx, t / ntx, dsm, ru, rv,
                                                     rp, n);
          if (n >= 0) {
            const uint8_t fl = op_tile_flags<T, kDX, kDY>(dsm);
            L.d[n] = (fl & kVDir) ? T(0) : b[n] - ru;
            L.d[nn + n] = (fl & kVDir) ? T(0) : b[nn + n] - rv;
            L.d[2 * nn + n] = (fl & kPFix) ? T(0) : b[2 * nn + n] - rp;
          }
          __syncthreads();  // the tile's shared memory is reused by the next tile
        }
        break;
      }
      case kPhaseRestrict: {
        const VLevel<T>& C = S.lv[k - 1];
        const Grid& c = C.g;
        const bool zero = f.colour == 1;
        for_items<NT>(c.nn, [&](int n) {
          restrict_node<T, true>(g, c, L.d, C.b, 3, n % c.nnx, n / c.nnx);
          if (zero) {
            C.x[n] = T(0);
            C.x[c.nn + n] = T(0);
            C.x[2 * c.nn + n] = T(0);
          }
        });
        break;
      }
      case kPhasePassZero: {
        // four items per colour cell, warp-sized chunks round-robin over the
        // blocks; every lane of a warp takes part in the cell's shuffles
        T* xout = f.out ? L.x2 : x0;
        const int count = 4 * vanka_slots(g);
        const int nchunks = (count + 31) >> 5;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int c = blockIdx.x + gridDim.x * w; c < nchunks; c += gridDim.x * (NT / 32)) {
          const int e = (c << 5) + lane;
          vanka_pass_zero_node<T>(g, f.colour, b, L.inv, omega, xout, e, e < count);
        }
        break;
      }
      case kPhaseCoarse: {
        const int nd = 3 * g.nn;
        for (int q0 = threadIdx.x; q0 < nd; q0 += 4 * NT) {  // four loads in flight
          double v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * NT;
            v[u] = q < nd ? (double)b[band_to_level(g, q)] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u * NT < nd) sbuf[q0 + u * NT] = v[u];
        }
        __syncthreads();
        // one warp per row, rows round-robin over the blocks first
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int r = blockIdx.x + gridDim.x * w; r < nd; r += gridDim.x * (NT / 32)) {
          const double* row = Ainv + (size_t)r * nd;
          // chunks of 16 entries per lane: every load of a chunk is issued
          // before its products are summed, so that a row of up to 512
          // entries costs one round trip to L2 instead of one per entry
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          for (int c0 = lane; c0 < nd; c0 += 16 * 32) {
            double rv[16], sv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int c2 = c0 + 32 * u;
              rv[u] = c2 < nd ? row[c2] : 0.0;
              sv[u] = c2 < nd ? sbuf[c2] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u & 3] += rv[u] * sv[u];
          }
          double a = (acc[0] + acc[1]) + (acc[2] + acc[3]);
          for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          if (lane == 0) x0[band_to_level(g, r)] = (T)a;
        }
        break;
      }
      case kPhaseProlong: {
        const VLevel<T>& C = S.lv[k - 1];
        T* x = f.in ? L.x2 : x0;
        for_items<NT>(g.nn, [&](int n) {
          prolong_add_node<T>(g, C.g, C.x, x, n % g.nnx, n / g.nnx);
        });
        break;
      }
      case kPhaseZeroTop: {
        for_items<NT>(3 * g.nn, [&](int n) { topx[n] = T(0); });
        break;
      }
    }
    sync();
  }
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads)
    vcycle_kernel(const VLevel<T>* __restrict__ lv, const Phase* __restrict__ ph, int nph, int top,
                  const T* __restrict__ topb, T* __restrict__ topx, const double* __restrict__ Ainv,
                  T omega, const int* skip) {
  // a speculative FGMRES iteration after the cycle stopped: every block
  // reads the same flag (set before this launch) and returns before any barrier
  if (skip && *skip) return;
  extern __shared__ __align__(16) uint8_t dyn[];  // coarse vector or pass tiles
  __shared__ WalkSmem<T> S;
  cg::grid_group grid = cg::this_grid();
  walk_phases<T, kCTX, kCTY, kCoopThreads, kCoopThreads>(lv, ph, nph, top, topb, topx, Ainv,
                                                         omega, dyn, S, [&] { grid.sync(); });
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
  walk_phases<T, kLTX, kLTY, cluster_threads<T>(), kClusterOwners>(
      lv, ph, nph, top, topb, topx, Ainv, omega, dyn, S, [&] { cl.sync(); });
}

void build_phases(int k, int top, int nu1, int nu2, std::vector<Phase>& out) {
  if (k == 0) {
    out.push_back({kPhaseCoarse, 0, 0, 0, 0});
    return;
  }
  // with pre-smoothing, the first pass starts from the zero iterate and
  // writes every node, so no level needs zeroing beforehand
  int cur = 0;
  for (int s = 0; s < nu1; ++s)
    for (int c = 0; c < 4; ++c) {
      out.push_back({s == 0 && c == 0 ? kPhasePassZero : kPhasePass, k, c, cur, 1 - cur});
      cur ^= 1;
    }
  out.push_back({kPhaseDefect, k, 0, cur, 0});
  out.push_back({kPhaseRestrict, k, nu1 > 0 ? 0 : 1, 0, 0});
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
// dynamic shared memory of a block with `tiles_in_flight` TCX x TCY pass
// tiles: the largest of the coarse right-hand side (FP64), the pass tiles and
// the 16 x 8-node defect tile
template <typename T, int TCX, int TCY>
size_t walk_smem(int coarse_nd, int tiles_in_flight) {
  size_t m = sizeof(PassSmem<T, TCX, TCY>) * tiles_in_flight;
  m = std::max(m, sizeof(double) * coarse_nd);
  m = std::max(m, sizeof(OpSmem<T, 16, 8>));
  return m;
}
}  // namespace

int vcycle_coop_tiles(const Grid& g) {
  return cdiv(g.nx / 2 + 1, kCTX) * cdiv(g.ny / 2 + 1, kCTY);
}

bool vcycle_fits(int nphases, int nlevels) {
  return nphases <= kMaxPhases && nlevels <= kMaxVLevels;
}

std::vector<Phase> vcycle_phases(int top, int nu1, int nu2) {
  std::vector<Phase> out;
  if (nu1 == 0 || top == 0) out.push_back({kPhaseZeroTop, top, 0, 0, 0});
  build_phases(top, top, nu1, nu2, out);
  return out;
}

template <typename T>
int vcycle_grid(int coarse_nd) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = walk_smem<T, kCTX, kCTY>(coarse_nd, 1);
  if (cudaFuncSetAttribute(vcycle_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vcycle_kernel<T>, kCoopThreads, smem) !=
          cudaSuccess ||
      per <= 0)
    return 0;
  if (per > 4) per = 4;
  return per * sms;
}

template <typename T>
int launch_vcycle_persistent(const VLevel<T>* lv, const Phase* ph, int nph, int top, const T* topb,
                             T* topx, const double* Ainv, T omega, int grid, int coarse_nd,
                             cudaStream_t st, const int* skip) {
  void* args[] = {(void*)&lv,   (void*)&ph,   (void*)&nph,   (void*)&top, (void*)&topb,
                  (void*)&topx, (void*)&Ainv, (void*)&omega, (void*)&skip};
  note_launch();
  const cudaError_t e =
      cudaLaunchCooperativeKernel((void*)vcycle_kernel<T>, dim3(grid), dim3(kCoopThreads), args,
                                  walk_smem<T, kCTX, kCTY>(coarse_nd, 1), st);
  return e == cudaSuccess ? 0 : 1;
}

template <typename T>
int vcycle_cluster_size(int coarse_nd) {
  const size_t smem = walk_smem<T, kLTX, kLTY>(coarse_nd, cluster_threads<T>() / kClusterOwners);
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
  cfg.dynamicSmemBytes = walk_smem<T, kLTX, kLTY>(coarse_nd, cluster_threads<T>() / kClusterOwners);
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
                                             cudaStream_t, const int*);
template int launch_vcycle_persistent<double>(const VLevel<double>*, const Phase*, int, int,
                                              const double*, double*, const double*, double, int,
                                              int, cudaStream_t, const int*);
template int vcycle_cluster_size<float>(int);
template int vcycle_cluster_size<double>(int);
template int launch_vcycle_cluster<float>(const VLevel<float>*, const Phase*, int, int,
                                          const float*, float*, const double*, float, int, int,
                                          cudaStream_t);
template int launch_vcycle_cluster<double>(const VLevel<double>*, const Phase*, int, int,
                                           const double*, double*, const double*, double, int,
                                           int, cudaStream_t);

}  // namespace dnnmg
