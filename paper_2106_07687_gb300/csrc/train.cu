// Training of the patch network (Sec. 2.2 / Sec. 3.1): loss of Eq. 7 as a
// mean of squared errors, backpropagation through time over T steps, and
// Adam.  Weight gradients of a layer are sums over all (step, sequence)
// columns of dG^T x, computed as split-K tcgen05 GEMMs on the transposed
// BF16 streams written by the forward and backward passes; a ones row in
// every input stream makes the bias gradient the last output column.
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

struct BwdSmem {
  uint32_t w, r1, r2, bar, tmem, red, total;
  static __host__ __device__ BwdSmem of() {
    BwdSmem s{};
    uint32_t o = 0;
    s.w = o;    o += (uint32_t)(BwdPack::kTotal * 2);
    s.r1 = o;   o += kTile * 192 * 2;
    s.r2 = o;   o += kTile * 192 * 2;
    s.bar = o;  o += 16;
    s.tmem = o; o += 16;
    s.red = o;  o += 16 * 8;  // one double per warp
    s.total = o;
    return s;
  }
};

__device__ __forceinline__ void store_row16(uint8_t* buf, int r, int k0, int K, const float* v) {
  uint32_t p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = (uint32_t)f2bf(v[2 * i]) | ((uint32_t)f2bf(v[2 * i + 1]) << 16);
  *reinterpret_cast<uint4*>(buf + kmajor_offset(r, k0, K)) = make_uint4(p[0], p[1], p[2], p[3]);
  *reinterpret_cast<uint4*>(buf + kmajor_offset(r, k0 + 8, K)) = make_uint4(p[4], p[5], p[6], p[7]);
}

__device__ __forceinline__ void mma_run(uint32_t d_tmem, uint32_t a_addr, int a_K, uint32_t b_addr,
                                        int b_K, int N, int K) {
  const uint32_t id = idesc_bf16(kTile, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = smem_desc(a_addr + ks * 256, 128, (a_K / 8) * 128);
    const uint64_t db = smem_desc(b_addr + ks * 256, 128, (b_K / 8) * 128);
    mma_bf16(d_tmem, da, db, id, ks > 0 ? 1u : 0u);
  }
}

// Gradient of one GRU layer for this thread's row, hidden units
// c*16..c*16+15: dh (total gradient of the new state) -> gate gradients dgi,
// dgh (rows of the operands in r_gi / r_gh and transposed in HBM) and the
// direct part dh * z of the previous state's gradient.
__device__ __forceinline__ void gru_backward_chunk(int c, const float* dh, const float* g,
                                                   const float* hprev, float* dprev, uint8_t* r_gi,
                                                   uint8_t* r_gh, int row, bool valid,
                                                   uint16_t* giT, uint16_t* ghT, size_t ld) {
  float dar[16], daz[16], dan[16], dhn[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int j = c * 16 + i;
    const float r = g[j], z = g[64 + j], n = g[128 + j], ghn = g[192 + j];
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
  if (r_gi) {
    store_row16(r_gi, row, c * 16, 192, dar);
    store_row16(r_gi, row, 64 + c * 16, 192, daz);
    store_row16(r_gi, row, 128 + c * 16, 192, dan);
  }
  store_row16(r_gh, row, c * 16, 192, dar);
  store_row16(r_gh, row, 64 + c * 16, 192, daz);
  store_row16(r_gh, row, 128 + c * 16, 192, dhn);
  if (valid) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int j = c * 16 + i;
      giT[(size_t)j * ld] = f2bf(dar[i]);
      giT[(size_t)(64 + j) * ld] = f2bf(daz[i]);
      giT[(size_t)(128 + j) * ld] = f2bf(dan[i]);
      ghT[(size_t)j * ld] = f2bf(dar[i]);
      ghT[(size_t)(64 + j) * ld] = f2bf(daz[i]);
      ghT[(size_t)(128 + j) * ld] = f2bf(dhn[i]);
    }
  }
}

constexpr int kBwdWG = 4;  // warpgroups: each takes a quarter of every accumulator's columns
constexpr int kBwdThreads = kTile * kBwdWG;

__global__ void __launch_bounds__(kBwdThreads, 1)
    patchnet_backward_kernel(NetDims d, const uint16_t* __restrict__ wT, BwdArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const BwdSmem S = BwdSmem::of();
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row = (warp & 3) * 32 + lane;  // patch row of the tile = TMEM lane
  const int cq = warp >> 2;                // column quarter
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + S.bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S.tmem);
  double* red = reinterpret_cast<double*>(sm + S.red);
  {
    const uint4* src = reinterpret_cast<const uint4*>(wT);
    uint4* dst = reinterpret_cast<uint4*>(sm + S.w);
    for (int i = t; i < BwdPack::kTotal / 8; i += kBwdThreads) dst[i] = src[i];
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
  uint8_t* R1 = sm + S.r1;
  uint8_t* R2 = sm + S.r2;
  const int B = a.B, T = a.T, C = d.c_out, NO = d.nout();
  const size_t ld = (size_t)T * B;
  const int u0 = 16 * cq;  // this thread's 16 hidden units
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
    float dh0n[16], dh1n[16];  // gradients w.r.t. the previous step's states (these units)
#pragma unroll
    for (int j = 0; j < 16; ++j) dh0n[j] = dh1n[j] = 0.0f;
#pragma unroll 1
    for (int step = T - 1; step >= 0 && !failed; --step) {
      const size_t col = (size_t)step * B + p;
      const float* act = a.act + col * kAct;
      const float* actp = step > 0 ? a.act + (col - B) * kAct : nullptr;
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
        store_row16(R1, row, 16 * cq, NO, dy);
      }
      sync_mma([&] { mma_run(tbase + 0, sb + S.r1, NO, sb + S.w + 2 * BwdPack::kW2T, NO, 128, NO); });
      if (failed) break;
      // ---- dense head: da1 = (dY W2) * [a1 > 0], 32 of the 128 units
#pragma unroll
      for (int c = 2 * cq; c < 2 * cq + 2; ++c) {
        float v[16];
        tmem_ld16(tm + c * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = c * 16 + i;
          v[i] = (valid && act[kActA1 + j] > 0.0f) ? v[i] : 0.0f;
          if (valid) a.da1T[(size_t)j * ld + col] = f2bf(v[i]);
        }
        store_row16(R1, row, c * 16, 128, v);
      }
      sync_mma([&] { mma_run(tbase + 128, sb + S.r1, 128, sb + S.w + 2 * BwdPack::kW1T, 128, 64, 128); });
      if (failed) break;
      // ---- GRU layer 1
      {
        float dh[16], hp[16], dp[16];
        tmem_ld16(tm + 128 + u0, dh);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          dh[i] = valid ? dh[i] + dh1n[i] : 0.0f;
          hp[i] = actp ? actp[kActH1 + u0 + i] : 0.0f;
        }
        gru_backward_chunk(cq, dh, act + kActG1, hp, dp, R1, R2, row, valid, a.gi1T + col,
                           a.gh1T + col, ld);
#pragma unroll
        for (int i = 0; i < 16; ++i) dh1n[i] = dp[i];
      }
      sync_mma([&] {
        mma_run(tbase + 0, sb + S.r2, 192, sb + S.w + 2 * BwdPack::kWhh1T, 192, 64, 192);
        mma_run(tbase + 64, sb + S.r1, 192, sb + S.w + 2 * BwdPack::kWih1T, 192, 64, 192);
      });
      if (failed) break;
      // ---- GRU layer 0 (its input gradient is not needed)
      {
        float dmm[16], dtop[16], hp[16], dp[16];
        tmem_ld16(tm + u0, dmm);
        tmem_ld16(tm + 64 + u0, dtop);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          dh1n[i] += dmm[i];
          dtop[i] = valid ? dtop[i] + dh0n[i] : 0.0f;
          hp[i] = actp ? actp[kActH0 + u0 + i] : 0.0f;
        }
        gru_backward_chunk(cq, dtop, act + kActG0, hp, dp, nullptr, R2, row, valid, a.gi0T + col,
                           a.gh0T + col, ld);
#pragma unroll
        for (int i = 0; i < 16; ++i) dh0n[i] = dp[i];
      }
      sync_mma([&] { mma_run(tbase + 128, sb + S.r2, 192, sb + S.w + 2 * BwdPack::kWhh0T, 192, 64, 192); });
      if (failed) break;
      {
        float dmm[16];
        tmem_ld16(tm + 128 + u0, dmm);
#pragma unroll
        for (int i = 0; i < 16; ++i) dh0n[i] += dmm[i];
      }
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
    else
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
  const int H = d.hidden;
  const float* Wih0 = w;
  const float* Whh0 = Wih0 + (size_t)3 * H * d.c_in;
  const float* Wih1 = Whh0 + (size_t)3 * H * H + 6 * H;
  const float* Whh1 = Wih1 + (size_t)3 * H * H;
  const float* W1 = Whh1 + (size_t)3 * H * H + 6 * H;
  const float* W2 = W1 + (size_t)d.mlp * H + d.mlp;
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(W2, d.mlp, 128, d.nout(), d.c_out, wT + BwdPack::kW2T);
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(W1, H, 64, 128, 128, wT + BwdPack::kW1T);
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(Whh0, H, 64, 192, 192, wT + BwdPack::kWhh0T);
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(Whh1, H, 64, 192, 192, wT + BwdPack::kWhh1T);
  note_launch();
  pack_transpose_kernel<<<64, 256, 0, st>>>(Wih1, H, 64, 192, 192, wT + BwdPack::kWih1T);
}

void launch_patchnet_backward(const NetDims& d, const uint16_t* wT, const BwdArgs& a,
                              int nblocks, cudaStream_t st) {
  const BwdSmem S = BwdSmem::of();
  cudaFuncSetAttribute(patchnet_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)S.total);
  note_launch();
  patchnet_backward_kernel<<<nblocks, kBwdThreads, S.total, st>>>(d, wT, a);
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
