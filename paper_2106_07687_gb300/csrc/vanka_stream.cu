// Streaming colour pass of the Vanka smoother for the large levels (FP32).
//
// Persistent blocks (three per SM) walk the colour's tiles of 16 x 4 colour
// cells.  The 12 x 12 inverses of a tile (144 entries x 64 cells, 36 KB, the
// bulk of a pass's memory traffic) arrive in shared memory by one
// tensor-memory-access (TMA) copy per tile, issued as soon as the previous
// tile's products have read the buffer, so that the copy overlaps the
// staging, operator rows and defects of the tile.  The pass is bound by the
// latency of those dependent steps, not by bandwidth: one buffer and three
// resident blocks (24 warps per SM) beat two buffers and two blocks.  The arithmetic of a tile is
// that of vanka_pass_tile (the same staging, rows, defect sums and 12 x 12
// products in the same order), so the result is bitwise the tiled pass's.
//
// Thread layout: thread t owns node a = t / 64 of colour cell q = t % 64 of
// the tile, so that a warp reads one inverse entry of 32 consecutive cells
// (conflict-free in the [entry][cell] box); the four nodes of a cell pass
// their defects through shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kernels.h"
#include "umma.cuh"
#include "vanka_body.cuh"

namespace dnnmg {

namespace {

using namespace umma;

constexpr int kQX = 16, kQY = 4;  // colour cells of a tile
constexpr int kQ = kQX * kQY;
constexpr int kStreamThreads = 4 * kQ;
constexpr uint32_t kBoxBytes = 144u * kQ * sizeof(float);
constexpr uint32_t kStreamPolls = 1u << 24;

constexpr int kBufs = 1;

struct StreamSmem {
  float inv[kBufs][144][kQ];  // inverse rows of the tile, [entry][qy * 16 + qx]
  PassSmem<float, kQX, kQY> p;
  float d[kQ][13];        // the 12 defects of each colour cell (padded row)
  uint64_t bar[2];
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

// 3-D tile copy global -> shared, completion counted on mbar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
      : "memory");
}

__global__ void __launch_bounds__(kStreamThreads, kBufs == 1 ? 3 : 2)
    vanka_pass_stream_kernel(const __grid_constant__ CUtensorMap tmap, Grid g, Sten<float> s,
                             int colour, const float* __restrict__ b,
                             const float* __restrict__ xin, const float* __restrict__ vb,
                             float omega, float* __restrict__ xout, int* status) {
  extern __shared__ __align__(128) uint8_t smraw[];
  StreamSmem& S = *reinterpret_cast<StreamSmem*>(smraw);
  const int cx = colour & 1, cy = colour >> 1;
  const int sx = g.nx / 2 + 1, sy = g.ny / 2 + 1;
  const int nbx = cdiv(sx, kQX), nt = nbx * cdiv(sy, kQY);
  const int nn = g.nn;
  const int t = threadIdx.x;
  const int a = t / kQ, q = t % kQ, qx = q % kQX, qy = q / kQX;
  if (t == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
  }
  __syncthreads();
  auto issue = [&](int tile, int buf) {  // thread 0 only
    mbar_expect_tx(&S.bar[buf], kBoxBytes);
    tma_load_3d(&S.inv[buf][0][0], &tmap, (tile % nbx) * kQX, (tile / nbx) * kQY, colour * 144,
                &S.bar[buf]);
  };
  uint32_t parity[2] = {0u, 0u};
  bool pending[2] = {(int)blockIdx.x < nt, false};  // a copy into the buffer is in flight
  if (t == 0 && pending[0]) issue(blockIdx.x, 0);
  bool failed = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < nt && !failed; tile += gridDim.x, ++it) {
    const int buf = kBufs == 1 ? 0 : (it & 1);
    const int next = tile + gridDim.x;
    if (kBufs == 2 && next < nt) {  // the other buffer was released by the last barrier
      if (t == 0) issue(next, buf ^ 1);
      pending[buf ^ 1] = true;
    }
    const int bx = tile % nbx, by = tile / nbx;
    const int ti = bx * kQX + qx, tj = by * kQY + qy;
    const bool slot_ok = ti < sx && tj < sy;
    const int ci = 2 * ti - cx, cj = 2 * tj - cy;
    const int i = ci + (a & 1), j = cj + (a >> 1);
    const bool node_ok = slot_ok && i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
    const int n = node_ok ? j * g.nnx + i : 0;
    float xu = 0, xv = 0, xp = 0, bu0 = 0, bv0 = 0, bp0 = 0;
    if (node_ok) {
      xu = xin[n], xv = xin[nn + n], xp = xin[2 * nn + n];
      bu0 = b[n], bv0 = b[nn + n], bp0 = b[2 * nn + n];
    }
    const int i0 = 2 * bx * kQX - cx, j0 = 2 * by * kQY - cy;  // first node of the tile
    pass_stage_rows<float, kQX, kQY, kStreamThreads>(g, s, xin, vb, i0, j0, t, S.p);
    const bool cell_ok = slot_ok && ci >= 0 && cj >= 0 && ci < g.nx && cj < g.ny &&
                         !S.p.sol[cj - j0 + 2][ci - i0 + 2];
    float du = 0, dv = 0, dp = 0;
    if (node_ok && cell_ok)
      pass_node_defect<float, kQX, kQY>(i, j, i0, j0, xu, xv, xp, bu0, bv0, bp0, S.p, du, dv, dp);
    S.d[q][a] = du;
    S.d[q][4 + a] = dv;
    S.d[q][8 + a] = dp;
    // the tile's inverse rows (bounded wait; the barrier also publishes S.d)
    const bool got = mbar_wait(&S.bar[buf], parity[buf], kStreamPolls);
    if (got) {
      parity[buf] ^= 1u;
      pending[buf] = false;
    }
    failed = __syncthreads_or(!got);
    if (!failed && node_ok) {
      if (cell_ok) {
        float acc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          acc[c] = 0;
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[c] += S.inv[buf][(c * 4 + a) * 12 + k][q] * S.d[q][k];
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
    __syncthreads();  // the staged tile, the defects and this buffer are reused
    if (kBufs == 1 && !failed && next < nt) {  // the buffer is free again: the next tile
      if (t == 0) issue(next, 0);
      pending[0] = true;
    }
  }
  if (failed) {
    if (t == 0) atomicOr(status, 8);
    // copies still in flight land before the block's shared memory is released
    for (int k = 0; k < kBufs; ++k)
      if (pending[k]) mbar_wait(&S.bar[k], parity[k], kStreamPolls);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool make_vanka_tensor_map(void* map, const float* inv, const Grid& g) {
  static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || !inv || (reinterpret_cast<uintptr_t>(inv) & 15)) return false;
  const int sx = g.nx / 2 + 1, sy = g.ny / 2 + 1, pitch = vanka_pitch(g);
  // inv[colour][entry][tj][ti] as a 3-D array (ti, tj, colour * 144 + entry);
  // rows of pitch floats, so every stride is a multiple of 16 bytes
  const cuuint64_t dims[3] = {(cuuint64_t)sx, (cuuint64_t)sy, 4 * 144};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float),
                                 (cuuint64_t)pitch * sy * sizeof(float)};
  const cuuint32_t box[3] = {kQX, kQY, 144};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
            const_cast<float*>(inv), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int vanka_stream_grid(const Grid& g) {
  static int slots = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = (int)sizeof(StreamSmem);
    if (cudaFuncSetAttribute(vanka_pass_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vanka_pass_stream_kernel,
                                                      kStreamThreads, smem) != cudaSuccess)
      per = 0;
    cudaGetLastError();
    slots = per * sms;
  });
  const int nt = cdiv(g.nx / 2 + 1, kQX) * cdiv(g.ny / 2 + 1, kQY);
  return slots <= 0 ? 0 : (nt < slots ? nt : slots);
}

void launch_vanka_pass_stream(const void* map, const Grid& g, const Sten<float>& s, int colour,
                              const float* b, const float* xin, const float* vb, float omega,
                              float* xout, int* status, cudaStream_t st) {
  const int grid = vanka_stream_grid(g);
  note_launch();
  vanka_pass_stream_kernel<<<grid, kStreamThreads, sizeof(StreamSmem), st>>>(
      *reinterpret_cast<const CUtensorMap*>(map), g, s, colour, b, xin, vb, omega, xout, status);
}

}  // namespace dnnmg
