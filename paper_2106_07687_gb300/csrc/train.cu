// Training of the patch network (Sec. 2.2 / Sec. 3.1): loss of Eq. 7 as a
// mean of squared errors, backpropagation through time over T steps, and
// Adam.  Weight gradients of a layer are sums over all (step, sequence)
// columns of dG^T x, computed as split-K tcgen05 GEMMs on the transposed
// BF16 streams written by the forward and backward passes; a ones row in
// every input stream makes the bias gradient the last output column.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kernels.h"
#include "patchnet.cuh"
#include "train.h"
#include "umma.cuh"

namespace dnnmg {

namespace {

using namespace umma;

constexpr uint32_t kWaitPolls = 1u << 22;
constexpr int kTile = 128;

__device__ __forceinline__ uint16_t f2bf(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// transposed operand: element (n, k) = src[k * ld + n] for k < K_valid
__global__ void pack_transpose_kernel(const float* __restrict__ src, int ld, int N, int K,
                                      int K_valid, uint16_t* __restrict__ dst) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * K; idx += gridDim.x * blockDim.x) {
    const int n = idx / K, k = idx % K;
    const float v = k < K_valid ? src[(size_t)k * ld + n] : 0.0f;
    dst[kmajor_offset(n, k, K) >> 1] = f2bf(v);
  }
}

// Shared memory of the backward kernel: the transposed weights and one
// operand region R of 128 rows, which holds in turn dY (nout columns), dA1
// (128) and the gate gradients [dr | dz | dn | r * dn] of a layer (4m);
// both products of a layer (dG_h W_hh over [dr | dz] and r * dn, dG_i W_ih
// over [dr | dz | dn]) read it.
struct BwdSmem {
  uint32_t w, r, bar, tmem, red, total;
  static __host__ __device__ uint32_t up(uint32_t v) { return (v + 127u) & ~127u; }
  static __host__ __device__ BwdSmem of(const NetDims& d, size_t w_elems) {
    BwdSmem s{};
    uint32_t o = 0;
    s.w = o;    o = up(o + (uint32_t)(w_elems * 2));
    const int kr = 4 * d.hidden > 128 ? 4 * d.hidden : 128;
    s.r = o;    o += kTile * kr * 2;
    s.bar = o;  o += 16;
    s.tmem = o; o += 16;
    s.red = o;  o += 16 * 8;  // one double per warp
    s.total = o;
    return s;
  }
};

template <int U>
__device__ __forceinline__ void store_row(uint8_t* buf, int r, int k0, int K, const float* v) {
#pragma unroll
  for (int h = 0; h < U / 8; ++h) {
    uint32_t p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      p[i] = (uint32_t)f2bf(v[8 * h + 2 * i]) | ((uint32_t)f2bf(v[8 * h + 2 * i + 1]) << 16);
    *reinterpret_cast<uint4*>(buf + kmajor_offset(r, k0 + 8 * h, K)) =
        make_uint4(p[0], p[1], p[2], p[3]);
  }
}

template <int U>
__device__ __forceinline__ void load_f32(const float* src, float* v) {
#pragma unroll
  for (int q = 0; q < U / 4; ++q) {
    const float4 u = reinterpret_cast<const float4*>(src)[q];
    v[4 * q] = u.x, v[4 * q + 1] = u.y, v[4 * q + 2] = u.z, v[4 * q + 3] = u.w;
  }
}

__device__ __forceinline__ void mma_run(uint32_t d_tmem, uint32_t a_addr, int a_K, uint32_t b_addr,
                                        int b_K, int N, int K, bool acc_first) {
  const uint32_t id = idesc_bf16(kTile, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = smem_desc(a_addr + ks * 256, 128, (a_K / 8) * 128);
    const uint64_t db = smem_desc(b_addr + ks * 256, 128, (b_K / 8) * 128);
    mma_bf16(d_tmem, da, db, id, (ks > 0 || acc_first) ? 1u : 0u);
  }
}

// Gradient of one GRU layer for this thread's row, hidden units u0..u0+U-1:
// dh (total gradient of the new state) -> gate gradients (into the operand
// region R as [dr | dz | dn | r * dn] and transposed into giT / ghT) and the
// direct part dh * z of the previous state's gradient.  Rows past the batch
// (valid false) read nothing and give zeros.
template <int H, int U>
__device__ __forceinline__ void gru_backward_chunk(int u0, const float* dh, const float* g,
                                                   const float* hprev, float* dprev, uint8_t* R,
                                                   int row, bool valid, uint16_t* giT,
                                                   uint16_t* ghT, size_t ld) {
  float gr[U], gz[U], gn[U], gh[U];
#pragma unroll
  for (int i = 0; i < U; ++i) gr[i] = gz[i] = gn[i] = gh[i] = 0.0f;
  if (valid) {
    load_f32<U>(g + u0, gr);
    load_f32<U>(g + H + u0, gz);
    load_f32<U>(g + 2 * H + u0, gn);
    load_f32<U>(g + 3 * H + u0, gh);
  }
  float dar[U], daz[U], dan[U], dhn[U];
#pragma unroll
  for (int i = 0; i < U; ++i) {
    const float r = gr[i], z = gz[i], n = gn[i], ghn = gh[i];
    const float dn = dh[i] * (1.0f - z);
    const float dz = dh[i] * (hprev[i] - n);
    const float an = dn * (1.0f - n * n);
    const float dr = an * ghn;
    dar[i] = dr * r * (1.0f - r);
    daz[i] = dz * z * (1.0f - z);
    dan[i] = an;
    dhn[i] = an * r;
    dprev[i] = dh[i] * z;
  }
  store_row<U>(R, row, u0, 4 * H, dar);
  store_row<U>(R, row, H + u0, 4 * H, daz);
  store_row<U>(R, row, 2 * H + u0, 4 * H, dan);
  store_row<U>(R, row, 3 * H + u0, 4 * H, dhn);
  if (valid) {
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int j = u0 + i;
      giT[(size_t)j * ld] = f2bf(dar[i]);
      giT[(size_t)(H + j) * ld] = f2bf(daz[i]);
      giT[(size_t)(2 * H + j) * ld] = f2bf(dan[i]);
      ghT[(size_t)j * ld] = f2bf(dar[i]);
      ghT[(size_t)(H + j) * ld] = f2bf(daz[i]);
      ghT[(size_t)(2 * H + j) * ld] = f2bf(dhn[i]);
    }
  }
}

constexpr int kBwdWG = 4;  // warpgroups: each takes a quarter of every accumulator's columns
constexpr int kBwdThreads = kTile * kBwdWG;

// Backpropagation through time for 128 sequences per tile, steps T-1 .. 0.
// TMEM columns: [0,128) dY W2, [128,128+m) dA1 W1 (the top layer's state
// gradient), then per layer [0,m) dG_h W_hh (the previous state's gradient)
// and [m,2m) dG_i W_ih (the gradient of the layer's input, the state of the
// layer below).
template <int H, int NL>
__global__ void __launch_bounds__(kBwdThreads, 1)
    patchnet_backward_kernel(NetDims d, BwdPack W, const uint16_t* __restrict__ wT, BwdArgs a) {
  constexpr int U = H / 4, KACT = act_size(H, NL), KR = 4 * H;
  extern __shared__ __align__(1024) uint8_t sm[];
  const BwdSmem S = BwdSmem::of(d, W.total);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row = (warp & 3) * 32 + lane;  // patch row of the tile = TMEM lane
  const int cq = warp >> 2;                // column quarter
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + S.bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S.tmem);
  double* red = reinterpret_cast<double*>(sm + S.red);
  {
    const uint4* src = reinterpret_cast<const uint4*>(wT);
    uint4* dst = reinterpret_cast<uint4*>(sm + S.w);
    for (size_t i = t; i < W.total / 8; i += kBwdThreads) dst[i] = src[i];
  }
  if (warp == 0) tmem_alloc(tslot, 256);
  if (t == 0) mbar_init(bar, 1);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t tm = tbase + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t sb = smem_u32(sm);
  uint8_t* R = sm + S.r;
  const uint32_t sw = sb + S.w;
  const int B = a.B, T = a.T, C = d.c_out, NO = d.nout();
  const size_t ld = (size_t)T * B;
  const int u0 = U * cq;  // this thread's hidden units
  uint32_t phase = 0;
  bool failed = false;
  double loss = 0.0;
  const int ntiles = (B + kTile - 1) / kTile;

  auto sync_mma = [&](auto issue) {
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (t == 0) {
      fence_after_sync();
      issue();
      mma_commit(bar);
    }
    if (!mbar_wait(bar, phase, kWaitPolls)) failed = true;
    phase ^= 1;
    failed = __syncthreads_or(failed);
    fence_after_sync();
  };

  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int p = tile * kTile + row;
    const bool valid = p < B;
    float dcar[NL][U];  // gradients w.r.t. the previous step's states (these units)
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int j = 0; j < U; ++j) dcar[l][j] = 0.0f;
#pragma unroll 1
    for (int step = T - 1; step >= 0 && !failed; --step) {
      const size_t col = (size_t)step * B + p;
      const float* act = a.act + col * KACT;
      const float* actp = step > 0 ? act - (size_t)B * KACT : nullptr;
      // ---- loss and dY (Eq. 7 as a mean): dY = 2 (y - Y) / (B T C); output
      // columns 16 cq .. +15 (one 16-column chunk of the nout per warpgroup)
      if (cq < NO / 16) {
        float dy[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) dy[i] = 0.0f;
        if (valid) {
          const size_t o = ((size_t)p * T + step) * C;
          for (int i = 0; i < 16; ++i) {
            const int j = 16 * cq + i;
            if (j >= C) break;
            const float e = a.ypred[o + j] - a.Y[o + j];
            loss += (double)e * e;
            dy[i] = a.scale * e;
            a.dyT[(size_t)j * ld + col] = f2bf(dy[i]);
          }
        }
        store_row<16>(R, row, 16 * cq, NO, dy);
      }
      sync_mma([&] { mma_run(tbase + 0, sb + S.r, NO, sw + 2 * W.w2t, NO, d.k2(), NO, false); });
      if (failed) break;
      float dtop[U];  // gradient of the current layer's new state from above
      if (!d.mlp) {   // a single dense layer: dY W2 is the top state's gradient
        tmem_ld<U>(tm + u0, dtop);
      } else {
      // ---- dense head: da1 = (dY W2) * [a1 > 0], 32 of the 128 units
#pragma unroll
      for (int c = 2 * cq; c < 2 * cq + 2; ++c) {
        float v[16];
        tmem_ld16(tm + c * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = c * 16 + i;
          v[i] = (valid && act[act_a1(H, NL) + j] > 0.0f) ? v[i] : 0.0f;
          if (valid) a.da1T[(size_t)j * ld + col] = f2bf(v[i]);
        }
        store_row<16>(R, row, c * 16, 128, v);
      }
      sync_mma([&] { mma_run(tbase + 128, sb + S.r, 128, sw + 2 * W.w1t, 128, H, 128, false); });
      if (failed) break;
      tmem_ld<U>(tm + 128 + u0, dtop);
      }
      // ---- GRU layers, top to bottom (the first layer's input gradient is
      // not needed)
#pragma unroll
      for (int l = NL - 1; l >= 0; --l) {
        float dh[U], hp[U], dp[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
          dh[i] = valid ? dtop[i] + dcar[l][i] : 0.0f;
          hp[i] = 0.0f;
        }
        if (valid && actp) load_f32<U>(actp + act_h(H, l) + u0, hp);
        gru_backward_chunk<H, U>(u0, dh, act + act_g(H, NL, l), hp, dp, R, row, valid,
                                 a.giT[l] + col, a.ghT[l] + col, ld);
        sync_mma([&] {
          const uint32_t r0 = sb + S.r, wh = sw + 2 * W.whh[l];
          mma_run(tbase + 0, r0, KR, wh, 3 * H, H, 2 * H, false);                 // [dr | dz]
          mma_run(tbase + 0, r0 + 3 * H * 16, KR, wh + 2 * H * 16, 3 * H, H, H, true);  // r * dn
          if (l > 0) mma_run(tbase + H, r0, KR, sw + 2 * W.wih[l], 3 * H, H, 3 * H, false);
        });
        if (failed) break;
        float dm[U];
        tmem_ld<U>(tm + u0, dm);
#pragma unroll
        for (int i = 0; i < U; ++i) dcar[l][i] = dp[i] + dm[i];
        if (l > 0) tmem_ld<U>(tm + H + u0, dtop);
      }
      if (failed) break;
      fence_before_sync();
      __syncthreads();
    }
  }
  // per-CTA loss partial (fixed-order reduction)
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0) red[warp] = loss;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < kBwdThreads / 32; ++w) s += red[w];
    a.loss_partial[blockIdx.x] = s;
  }
  if (failed) {
    if (t == 0) atomicOr(a.status, 4);
    mbar_wait(bar, phase, kWaitPolls);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, 256);
  }
}

// Weight gradients of all layers in one launch: for every job, the partial
// sums Cpart[job][split][M][N] = A[M][k-range] B[N][k-range]^T over a range
// of the K = (steps x patches) columns.  A block owns one 128-row tile of one
// job and one K range; its operands stream through a ring of kWStages
// shared-memory stages filled by asynchronous 16-byte copies, so the copies
// of chunk c + kWStages - 1 overlap the tensor-core MMAs of chunk c (a slot
// is refilled once the MMAs that read it have completed).
constexpr int kKC = 64;
constexpr int kWStages = 4;
constexpr int kWNmax = 144;
constexpr size_t kWStageA = (size_t)kTile * kKC * 2;
constexpr size_t kWStage = kWStageA + (size_t)kWNmax * kKC * 2;
constexpr size_t kWSmem = kWStages * kWStage + 64;

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kTile, 1)
    wgrad_kernel(WGradArgs a, float* __restrict__ Cpart, int* status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kWStages * kWStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + kWStages);
  int jb = 0;
  while (jb + 1 < a.njobs && (int)blockIdx.x >= a.first[jb + 1]) ++jb;
  const WGradJob& J = a.job[jb];
  const int nmt = J.M / kTile;
  const int b = blockIdx.x - a.first[jb];
  const int mt = b % nmt, split = b / nmt;
  const int row0 = mt * kTile;
  const int kbeg = split * a.Ks, kend = min(a.K, kbeg + a.Ks);
  const int nch = kend > kbeg ? (kend - kbeg + kKC - 1) / kKC : 0;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)J.N) ncols <<= 1;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (t == 0)
    for (int q = 0; q < kWStages; ++q) mbar_init(bar + q, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  auto load = [&](int c) {
    if (c < nch) {
      uint8_t* sa = sm + (size_t)(c % kWStages) * kWStage;
      uint8_t* sb = sa + kWStageA;
      const int k0 = kbeg + c * kKC;
      const int q8 = min(kKC, kend - k0) / 8;
      for (int e = t; e < kTile * q8; e += kTile) {
        const int r = e / q8, q = e % q8;
        cp16(sa + kmajor_offset(r, q * 8, kKC), J.A + (size_t)(row0 + r) * J.lda + k0 + q * 8);
      }
      for (int e = t; e < J.N * q8; e += kTile) {
        const int r = e / q8, q = e % q8;
        cp16(sb + kmajor_offset(r, q * 8, kKC), J.B + (size_t)r * J.ldb + k0 + q * 8);
      }
    }
    cp_commit();
  };
  for (int c = 0; c < kWStages - 1; ++c) load(c);
  const uint32_t id = idesc_bf16(kTile, J.N);
  bool failed = false;
  int last = -1;  // last chunk whose MMAs were committed
  for (int c = 0; c < nch && !failed; ++c) {
    cp_wait<kWStages - 2>();  // chunk c has landed (this thread's copies)
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (t == 0) {
      const uint8_t* sa = sm + (size_t)(c % kWStages) * kWStage;
      const uint8_t* sb = sa + kWStageA;
      const int kc = min(kKC, kend - (kbeg + c * kKC));
      for (int ks = 0; ks < kc / 16; ++ks) {
        const uint64_t da = smem_desc(smem_u32(sa) + ks * 256, 128, (kKC / 8) * 128);
        const uint64_t db = smem_desc(smem_u32(sb) + ks * 256, 128, (kKC / 8) * 128);
        mma_bf16(tbase, da, db, id, (c > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(bar + c % kWStages);
    }
    last = c;
    // refill the slot of chunk c - 1 once its MMAs are done
    if (c >= 1 && !mbar_wait(bar + (c - 1) % kWStages, ((c - 1) / kWStages) & 1, kWaitPolls))
      failed = true;
    failed = __syncthreads_or(failed);
    if (!failed) load(c + kWStages - 1);
  }
  if (!failed && last >= 0 &&
      !mbar_wait(bar + last % kWStages, (last / kWStages) & 1, kWaitPolls))
    failed = true;
  failed = __syncthreads_or(failed);
  cp_wait<0>();
  fence_after_sync();
  float* Cp = Cpart + a.coff[jb] + (size_t)split * J.M * J.N;
  const int r = row0 + t;
  if (!failed) {
    for (int c = 0; c < J.N / 16; ++c) {
      float v[16];
      if (nch > 0) tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      for (int i = 0; i < 16; ++i) Cp[(size_t)r * J.N + c * 16 + i] = nch > 0 ? v[i] : 0.0f;
    }
  } else {
    if (t == 0) atomicOr(status, 4);
    // the tensor core may still be working: wait (bounded) for the last commit
    if (last >= 0) mbar_wait(bar + last % kWStages, (last / kWStages) & 1, kWaitPolls);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, ncols);
  }
}

// The same partial sums with the operands copied by the tensor memory
// accelerator (TMA): one thread of the block issues, per 64-column chunk, one
// 2-D tile copy of A (128 rows) and one of B (N rows) into a ring of
// kTStages stages, waits for a stage's bytes on its mbarrier, issues the
// chunk's MMAs and commits them to the stage's release barrier; the copy of
// chunk c + kTStages waits for that release.  A box row is 64 columns (128
// bytes) copied with the 128-byte swizzle, which is the MMA's swizzled
// K-major operand layout (smem_desc_sw128): one copy request per row.
constexpr int kTStages = 6;
constexpr size_t kTStageA = (size_t)kTile * kKC * 2;                 // 16 KB
constexpr size_t kTStage = (kTStageA + (size_t)kWNmax * kKC * 2 + 1023) / 1024 * 1024;
constexpr size_t kTSmem = kTStages * kTStage + 1024 + 256;
constexpr uint32_t kTPolls = 1u << 24;

struct WGradMaps {
  CUtensorMap a[kMaxWGradJobs], b[kMaxWGradJobs];
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(mbar))
      : "memory");
}

__global__ void __launch_bounds__(kTile, 1)
    wgrad_tma_kernel(WGradArgs a, const __grid_constant__ WGradMaps maps,
                     float* __restrict__ Cpart, int* status) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  // stages on a 1024-byte boundary (the copies need 128)
  uint8_t* sm = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kTStages * kTStage);
  uint64_t* empty = full + kTStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + kTStages);
  __shared__ int s_failed;
  int jb = 0;
  while (jb + 1 < a.njobs && (int)blockIdx.x >= a.first[jb + 1]) ++jb;
  const WGradJob& J = a.job[jb];
  const int nmt = J.M / kTile;
  const int b = blockIdx.x - a.first[jb];
  const int mt = b % nmt, split = b / nmt;
  const int row0 = mt * kTile;
  const int kbeg = split * a.Ks, kend = min(a.K, kbeg + a.Ks);
  const int nch = kend > kbeg ? (kend - kbeg + kKC - 1) / kKC : 0;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)J.N) ncols <<= 1;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (t == 0) {
    for (int q = 0; q < kTStages; ++q) {
      mbar_init(full + q, 1);
      mbar_init(empty + q, 1);
    }
    s_failed = 0;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t bytes = (uint32_t)(kTStageA + (size_t)J.N * kKC * 2);
  int last = -1;  // last chunk whose MMAs were committed
  if (t == 0) {
    const CUtensorMap* ma = &maps.a[jb];
    const CUtensorMap* mb = &maps.b[jb];
    auto issue = [&](int c) {
      uint8_t* sa = sm + (size_t)(c % kTStages) * kTStage;
      const int k0 = kbeg + c * kKC;
      mbar_expect_tx(full + c % kTStages, bytes);
      tma_load_2d(sa, ma, k0, row0, full + c % kTStages);
      tma_load_2d(sa + kTStageA, mb, k0, 0, full + c % kTStages);
    };
    const uint32_t id = idesc_bf16(kTile, J.N);
    bool failed = false;
    int issued = 0;
    for (; issued < nch && issued < kTStages; ++issued) issue(issued);
    for (int c = 0; c < nch && !failed; ++c) {
      const int sidx = c % kTStages;
      const uint32_t par = (uint32_t)(c / kTStages) & 1u;
      if (!mbar_wait(full + sidx, par, kTPolls)) {
        failed = true;
        break;
      }
      fence_after_sync();
      const uint32_t sa = smem_u32(sm + (size_t)sidx * kTStage);
      const uint32_t sb = sa + (uint32_t)kTStageA;
      const int kc = min(kKC, kend - (kbeg + c * kKC));
      for (int ks = 0; ks < kc / 16; ++ks) {
        const uint64_t da = smem_desc_sw128(sa + ks * 32);
        const uint64_t db = smem_desc_sw128(sb + ks * 32);
        mma_bf16(tbase, da, db, id, (c > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(empty + sidx);
      last = c;
      if (issued < nch) {  // the stage is free once these MMAs are done
        if (!mbar_wait(empty + sidx, par, kTPolls)) {
          failed = true;
          break;
        }
        issue(issued++);
      }
    }
    if (!failed && last >= 0 &&
        !mbar_wait(empty + last % kTStages, (uint32_t)(last / kTStages) & 1u, kTPolls))
      failed = true;
    if (failed) {
      // copies and MMAs still in flight finish before the block's memory is
      // released: every issued stage's bytes, then the last commit (bounded)
      for (int c = last + 1; c < issued; ++c)
        mbar_wait(full + c % kTStages, (uint32_t)(c / kTStages) & 1u, kTPolls);
      if (last >= 0) mbar_wait(empty + last % kTStages, (uint32_t)(last / kTStages) & 1u, kTPolls);
      s_failed = 1;
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const bool failed = s_failed != 0;
  float* Cp = Cpart + a.coff[jb] + (size_t)split * J.M * J.N;
  const int r = row0 + t;
  if (!failed) {
    for (int c = 0; c < J.N / 16; ++c) {
      float v[16];
      if (nch > 0) tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      for (int i = 0; i < 16; ++i) Cp[(size_t)r * J.N + c * 16 + i] = nch > 0 ? v[i] : 0.0f;
    }
  } else if (t == 0) {
    atomicOr(status, 4);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, ncols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn() {
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

// Tensor map of a BF16 operand [rows][ld] (columns K) with boxes of kKC
// columns x box_rows rows in the 128-byte swizzle; false when it cannot be
// made (alignment, sizes, no driver entry point).
bool wgrad_map(CUtensorMap* m, const uint16_t* p, int rows, size_t ld, int K, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tmap_encode_fn();
  if (!fn || !p || (reinterpret_cast<uintptr_t>(p) & 15) || ld % 8 || K % 8 || box_rows > 256)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(p), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// grad_w[m * n_valid + n] = sum_s Cpart[job][s][m][n] (fixed order, FP64),
// grad_b[m] = sum_s Cpart[job][s][m][bias_col], all jobs in one launch
__global__ void wgrad_reduce_kernel(WGradArgs a, const float* __restrict__ Cpart) {
  const int total = a.eoff[a.njobs];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int jb = 0;
    while (jb + 1 < a.njobs && e >= a.eoff[jb + 1]) ++jb;
    const WGradJob& J = a.job[jb];
    const int le = e - a.eoff[jb];
    const int m = le / (J.n_valid + 1), n = le % (J.n_valid + 1);
    const int cn = n < J.n_valid ? n : J.bias_col;
    const float* Cp = Cpart + a.coff[jb];
    double acc = 0.0;
    for (int sp = 0; sp < a.splits; ++sp) acc += Cp[((size_t)sp * J.M + m) * J.N + cn];
    if (n < J.n_valid)
      J.gw[(size_t)m * J.n_valid + n] = (float)acc;
    else if (J.gb)  // no bias: the ones column's sums are not a parameter
      J.gb[m] = (float)acc;
  }
}

__global__ void loss_kernel(const double* __restrict__ part, int n, double inv, float* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    *out = (float)(s * inv);
  }
}

// Adam with bias correction: w -= lr * mhat / (sqrt(vhat) + eps)
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, size_t n, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

void launch_pack_backward(const NetDims& d, const float* w, uint16_t* wT, cudaStream_t st) {
  const BwdPack W = BwdPack::of(d);
  const NetOffsets o = d.offsets();
  const int H = d.hidden, k2 = d.k2();
  const float* Wih[kMaxLayers] = {};
  const float* Whh[kMaxLayers] = {};
  for (int l = 0; l < d.layers; ++l) {
    Wih[l] = w + o.wih[l];
    Whh[l] = w + o.whh[l];
  }
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(w + o.w2, k2, k2, d.nout(), d.c_out, wT + W.w2t);
  if (d.mlp) {
    note_launch();
    pack_transpose_kernel<<<64, 256, 0, st>>>(w + o.w1, H, H, 128, 128, wT + W.w1t);
  }
  for (int l = 0; l < d.layers; ++l) {
    note_launch();
    pack_transpose_kernel<<<64, 256, 0, st>>>(Whh[l], H, H, 3 * H, 3 * H, wT + W.whh[l]);
    if (l == 0) continue;
    note_launch();
    pack_transpose_kernel<<<64, 256, 0, st>>>(Wih[l], H, H, 3 * H, 3 * H, wT + W.wih[l]);
  }
}

size_t patchnet_backward_smem(const NetDims& d) {
  return BwdSmem::of(d, BwdPack::of(d).total).total;
}

namespace {
template <int H, int NL>
void launch_backward_shape(const NetDims& d, const uint16_t* wT, const BwdArgs& a, int nblocks,
                           cudaStream_t st) {
  const BwdPack W = BwdPack::of(d);
  const BwdSmem S = BwdSmem::of(d, W.total);
  cudaFuncSetAttribute(patchnet_backward_kernel<H, NL>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total);
  note_launch();
  patchnet_backward_kernel<H, NL><<<nblocks, kBwdThreads, S.total, st>>>(d, W, wT, a);
}
}  // namespace

void launch_patchnet_backward(const NetDims& d, const uint16_t* wT, const BwdArgs& a,
                              int nblocks, cudaStream_t st) {
  switch (d.hidden * 10 + d.layers) {
    case 321: launch_backward_shape<32, 1>(d, wT, a, nblocks, st); break;
    case 322: launch_backward_shape<32, 2>(d, wT, a, nblocks, st); break;
    case 323: launch_backward_shape<32, 3>(d, wT, a, nblocks, st); break;
    case 641: launch_backward_shape<64, 1>(d, wT, a, nblocks, st); break;
    case 642: launch_backward_shape<64, 2>(d, wT, a, nblocks, st); break;
    case 643: launch_backward_shape<64, 3>(d, wT, a, nblocks, st); break;
    default: break;  // rejected by net_supported
  }
}

int launch_wgrad(const WGradJob* jobs, int njobs, int K, int splits, float* Cpart, int* status,
                 cudaStream_t st) {
  if (njobs < 1 || njobs > kMaxWGradJobs || K < 16 || K % 16 || splits < 1) return 1;
  WGradArgs a{};
  a.njobs = njobs;
  a.K = K;
  int Ks = (K + splits - 1) / splits;
  Ks = (Ks + kKC - 1) / kKC * kKC;
  a.Ks = Ks;
  a.splits = (K + Ks - 1) / Ks;
  long long coff = 0;
  int blocks = 0, elems = 0;
  for (int q = 0; q < njobs; ++q) {
    const WGradJob& J = jobs[q];
    if (J.M <= 0 || J.M % kTile || J.N < 16 || J.N > kWNmax || J.N % 16 || J.lda % 8 ||
        J.ldb % 8 || J.bias_col >= J.N || J.n_valid >= J.N || J.m_valid > J.M)
      return 1;
    a.job[q] = J;
    a.coff[q] = coff;
    a.first[q] = blocks;
    a.eoff[q] = elems;
    coff += (long long)a.splits * J.M * J.N;
    blocks += (J.M / kTile) * a.splits;
    elems += J.m_valid * (J.n_valid + 1);
  }
  a.first[njobs] = blocks;
  a.eoff[njobs] = elems;
  // the TMA-fed kernel where every operand has a tensor map
  WGradMaps maps;
  bool tma = true;
  for (int q = 0; q < njobs && tma; ++q) {
    const WGradJob& J = jobs[q];
    tma = wgrad_map(&maps.a[q], J.A, J.M, J.lda, K, kTile) &&
          wgrad_map(&maps.b[q], J.B, J.N, J.ldb, K, J.N);
  }
  static const bool tattr =
      cudaFuncSetAttribute(wgrad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kTSmem) == cudaSuccess;
  if (tma && tattr) {
    note_launch();
    wgrad_tma_kernel<<<blocks, kTile, kTSmem, st>>>(a, maps, Cpart, status);
    note_launch();
    wgrad_reduce_kernel<<<cdiv(elems, 256), 256, 0, st>>>(a, Cpart);
    return 0;
  }
  cudaGetLastError();
  static const bool attr =
      cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kWSmem) == cudaSuccess;
  (void)attr;
  note_launch();
  wgrad_kernel<<<blocks, kTile, kWSmem, st>>>(a, Cpart, status);
  note_launch();
  wgrad_reduce_kernel<<<cdiv(elems, 256), 256, 0, st>>>(a, Cpart);
  return 0;
}

size_t wgrad_partials(const WGradJob* jobs, int njobs, int K, int splits) {
  int Ks = (K + splits - 1) / splits;
  Ks = (Ks + kKC - 1) / kKC * kKC;
  const int sp = (K + Ks - 1) / Ks;
  size_t n = 0;
  for (int q = 0; q < njobs; ++q) n += (size_t)sp * jobs[q].M * jobs[q].N;
  return n;
}

void launch_loss(const double* part, int n, double inv, float* out, cudaStream_t st) {
  note_launch();
  loss_kernel<<<1, 256, 0, st>>>(part, n, inv, out);
}

void launch_adam(float* w, const float* g, float* m, float* v, size_t n, float lr, int step,
                 cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  note_launch();
  adam_kernel<<<cdiv((int)n, 256), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, c1, c2, 1e-8f);
}

}  // namespace dnnmg
