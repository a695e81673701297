// Patch network on fifth-generation tensor cores (Sec. 2.2 / Sec. 3.1: GRU
// cells with memory per patch, then dense layers; inputs and outputs per
// patch as in the network evaluation of Algorithm 1).
//
// patchnet_forward_kernel<TRAIN, m, n>: persistent, one 128-patch tile at a
// time per CTA, 512 threads in four warpgroups.  Patch row r of the tile is
// TMEM lane r; warp w serves lanes 32 (w % 4) .. +31, and warpgroup w / 4
// takes one quarter of every accumulator's columns in the epilogues (m / 4
// hidden units of its row), so that the gate nonlinearities of a tile are
// spread over 16 warps.  All weights live in shared memory as BF16 K-major
// operands; per GRU layer the tensor core accumulates in TMEM (4m FP32
// columns)
//   [0,2m)   x W_ih[r,z]^T + h W_hh[r,z]^T      (gates r and z)
//   [2m,3m)  x W_ih[n]^T                        (input part of gate n)
//   [3m,4m)  h W_hh[n]^T                        (hidden part of gate n)
// and each thread applies the gate nonlinearities to its units in
// registers, writing the new hidden state (FP32) to HBM and (BF16) to shared
// memory as the next GEMM's operand.  The previous state of a layer is read
// back from HBM (the thread's own earlier write), so no layer's state stays
// in registers between layers.  The dense head reuses TMEM columns [0,128)
// and [128,128+N2).
#include "kernels.h"
#include "patchnet.cuh"
#include "umma.cuh"

namespace dnnmg {

namespace {

using namespace umma;

constexpr uint32_t kWaitPolls = 1u << 22;  // bound of every mbarrier wait
constexpr int kTile = 128;
constexpr int kFwdWG = 4;                      // warpgroups of the forward kernel
constexpr int kFwdThreads = kTile * kFwdWG;

__device__ __forceinline__ uint16_t f2bf(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// -- packing -----------------------------------------------------------------
__global__ void pack_block_kernel(const float* __restrict__ src, int ld, int row0, int rows_valid,
                                  int cols_valid, int R, int K, uint16_t* __restrict__ dst) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < R * K; idx += gridDim.x * blockDim.x) {
    const int r = idx / K, k = idx % K;
    const float v = (r < rows_valid && k < cols_valid) ? src[(size_t)(row0 + r) * ld + k] : 0.0f;
    dst[kmajor_offset(r, k, K) >> 1] = f2bf(v);
  }
}

// fused biases; a network without biases gets zeros
__global__ void pack_bias_kernel(const float* __restrict__ w, NetDims d, float* __restrict__ bias) {
  const int H = d.hidden;
  const NetOffsets o = d.offsets();
  for (int l = 0; l < d.layers; ++l) {
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      float* b = bias + (size_t)l * 4 * H;
      if (d.bias) {
        const float* bih = w + o.bih[l];
        const float* bhh = w + o.bhh[l];
        b[j] = bih[j] + bhh[j];
        b[H + j] = bih[H + j] + bhh[H + j];
        b[2 * H + j] = bih[2 * H + j];
        b[3 * H + j] = bhh[2 * H + j];
      } else {
        b[j] = b[H + j] = b[2 * H + j] = b[3 * H + j] = 0.0f;
      }
    }
  }
  float* ob = bias + (size_t)d.layers * 4 * H;
  for (int j = threadIdx.x; j < d.mlp; j += blockDim.x) ob[j] = d.bias ? w[o.b1 + j] : 0.0f;
  for (int j = threadIdx.x; j < d.nout(); j += blockDim.x)
    ob[d.mlp + j] = d.bias && j < d.c_out ? w[o.b2 + j] : 0.0f;
}

// -- shared-memory plan of the forward kernel ---------------------------------
// Operand regions are reused as soon as the MMA that reads them has
// completed:
//   a: x_t (layer 0 input, kx0 columns), then each layer's new state (the
//      next layer's input, m columns; the top layer's is the head's input);
//   b: the previous state of the layer being evaluated (m columns), staged
//      before that layer's MMAs;
//   m: the dense head's hidden layer (128 columns), over a and b.
struct FwdSmem {
  uint32_t w, bias, a, b, m, bar, tmem, total;
  static __host__ __device__ uint32_t up(uint32_t v) { return (v + 127u) & ~127u; }
  static __host__ __device__ FwdSmem of(const NetDims& d, size_t w_elems) {
    FwdSmem s{};
    uint32_t o = 0;
    s.w = o;    o = up(o + (uint32_t)(w_elems * 2));
    s.bias = o; o = up(o + (uint32_t)((d.layers * 4 * d.hidden + d.mlp + d.nout()) * 4));
    const int ka = d.kx0() > d.hidden ? d.kx0() : d.hidden;
    const uint32_t asz = kTile * ka * 2, bsz = kTile * d.hidden * 2, msz = kTile * 128 * 2;
    s.a = o;
    s.b = o + asz;
    s.m = s.a;
    o += asz + bsz > msz ? asz + bsz : msz;
    s.bar = o;  o += 16;
    s.tmem = o; o += 16;
    s.total = o;
    return s;
  }
};

// write U (8 or 16) consecutive values of row r (columns k0..) as BF16 operand
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

// Issue D(+)= A * B^T over K (in 16-wide slices) for one accumulator.
__device__ __forceinline__ void mma_run(uint32_t d_tmem, uint32_t a_addr, int a_K, uint32_t b_addr,
                                        int b_K, int N, int K, bool acc_first) {
  const uint32_t id = idesc_bf16(kTile, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = smem_desc(a_addr + ks * 256, 128, (a_K / 8) * 128);
    const uint64_t db = smem_desc(b_addr + ks * 256, 128, (b_K / 8) * 128);
    mma_bf16(d_tmem, da, db, id, (ks > 0 || acc_first) ? 1u : 0u);
  }
}

template <int U>
__device__ __forceinline__ void store_f32(float* dst, const float* v) {
#pragma unroll
  for (int q = 0; q < U / 4; ++q)
    reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
template <int U>
__device__ __forceinline__ void load_f32(const float* src, float* v) {
#pragma unroll
  for (int q = 0; q < U / 4; ++q) {
    const float4 u = reinterpret_cast<const float4*>(src)[q];
    v[4 * q] = u.x, v[4 * q + 1] = u.y, v[4 * q + 2] = u.z, v[4 * q + 3] = u.w;
  }
}

// One GRU layer's epilogue for U units [u0, u0 + U) of this thread's row:
// gates from TMEM, new hidden state from hprev into `next` (BF16 operand)
// and `hout` (FP32, HBM, the U units).  With `gsave` the gates r, z, n and
// the hidden part of gate n (incl. bias) are stored for the backward pass
// (row layout [r | z | n | hn], m each); with `hT` the new state is also
// written transposed in BF16 (column `col`, row stride ldT).
template <int H, int U>
__device__ __forceinline__ void gru_epilogue(uint32_t tm, const float* bias, const float* hprev,
                                             uint8_t* next, int row, int u0, float* hout,
                                             bool valid, float* gsave, uint16_t* hT, size_t ldT) {
  float rp[U], zp[U], ip[U], hp[U];
  tmem_ld<U>(tm + u0, rp);
  tmem_ld<U>(tm + H + u0, zp);
  tmem_ld<U>(tm + 2 * H + u0, ip);
  tmem_ld<U>(tm + 3 * H + u0, hp);
  float hn[U];
#pragma unroll
  for (int i = 0; i < U; ++i) {
    const int j = u0 + i;
    const float r = sigmoidf_(rp[i] + bias[j]);
    const float z = sigmoidf_(zp[i] + bias[H + j]);
    const float ghn = hp[i] + bias[3 * H + j];
    const float n = tanhf(ip[i] + bias[2 * H + j] + r * ghn);
    hn[i] = (1.0f - z) * n + z * hprev[i];
    rp[i] = r, zp[i] = z, ip[i] = n, hp[i] = ghn;
  }
  store_row<U>(next, row, u0, H, hn);
  if (!valid) return;
  store_f32<U>(hout + u0, hn);
  if (gsave) {
    store_f32<U>(gsave + u0, rp);
    store_f32<U>(gsave + H + u0, zp);
    store_f32<U>(gsave + 2 * H + u0, ip);
    store_f32<U>(gsave + 3 * H + u0, hp);
  }
  if (hT)
#pragma unroll
    for (int i = 0; i < U; ++i) hT[(size_t)(u0 + i) * ldT] = f2bf(hn[i]);
}

// Arguments of the forward kernel.  Inference: T = 1, hidden state read from
// h_in and written to h_out.  Training: the hidden state starts at zero and
// the kernel stores, per (t, p), the activations the backward pass needs
// (act, FP32) and transposed BF16 copies of the GEMM inputs for the weight
// gradients (column index t * P + p).
struct FwdArgs {
  const uint16_t* x;  // [P][T][C_in]
  int P, T;
  const float* h_in;  // [layers][P][m]
  float* h_out;       // [layers][P][m]
  float* out;         // [P][T][C_out]
  float* act;         // [T][P][act_size]
  uint16_t* xT;       // [kx0 + 16][T * P]
  uint16_t* hT[kMaxLayers];  // [m + 16][(T + 1) * P], state of step t at column (t + 1) * P + p
  uint16_t* y1T;      // [144][T * P]
  int* status;
};

template <bool TRAIN, int H, int NL>
__global__ void __launch_bounds__(kFwdThreads, 1)
    patchnet_forward_kernel(NetDims d, PackLayout L, const uint16_t* __restrict__ wimg,
                            const float* __restrict__ bias_g, FwdArgs a) {
  constexpr int U = H / 4;  // hidden units of this thread's row
  constexpr int KACT = act_size(H, NL);
  extern __shared__ __align__(1024) uint8_t sm[];
  const FwdSmem S = FwdSmem::of(d, L.total);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row = (warp & 3) * 32 + lane;  // patch row of the tile = TMEM lane
  const int cq = warp >> 2;                // column quarter of the epilogues
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + S.bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S.tmem);
  float* bias = reinterpret_cast<float*>(sm + S.bias);
  const int P = a.P, T = a.T;

  // weights and biases: one copy per CTA
  {
    const uint4* src = reinterpret_cast<const uint4*>(wimg);
    uint4* dst = reinterpret_cast<uint4*>(sm + S.w);
    for (size_t i = t; i < L.total / 8; i += kFwdThreads) dst[i] = src[i];
    const int nb = NL * 4 * H + d.mlp + d.nout();
    for (int i = t; i < nb; i += kFwdThreads) bias[i] = bias_g[i];
  }
  if (warp == 0) tmem_alloc(tslot, 256);
  if (t == 0) mbar_init(bar, 1);
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t tm = tbase + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
  const uint32_t sbase = smem_u32(sm);
  const int kx0 = d.kx0();
  const int u0 = U * cq;  // this thread's hidden units
  uint32_t phase = 0;
  bool failed = false;
  const int ntiles = (P + kTile - 1) / kTile;
  const size_t HP = (size_t)P * H;
  const size_t ld = (size_t)T * P, ldh = (size_t)(T + 1) * P;

  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int p = tile * kTile + row;
    const bool valid = p < P;
#pragma unroll 1
    for (int step = 0; step < T && !failed; ++step) {
      const size_t col = (size_t)step * P + p;
      float* act = TRAIN ? a.act + col * KACT : nullptr;
      // previous state of layer l (this thread's units): zero at the start
      // of a training sequence, else the thread's own earlier write
      auto load_prev = [&](int l, float* hv) {
#pragma unroll
        for (int i = 0; i < U; ++i) hv[i] = 0.0f;
        if (!valid) return;
        if (TRAIN) {
          if (step > 0) load_f32<U>(act - (size_t)P * KACT + act_h(H, l) + u0, hv);
        } else {
          load_f32<U>(a.h_in + l * HP + (size_t)p * H + u0, hv);
        }
      };
      // ---- stage x_t (BF16, 16-byte chunks spread over the block) and the
      // first layer's previous state (BF16 operand, this thread's units)
      {
        const int nq = kx0 / 8;
        const bool vec = d.c_in % 8 == 0;  // input rows start on 16-byte boundaries
        for (int e = t; e < kTile * nq; e += kFwdThreads) {
          // inference: a thread's neighbours take the next chunks of the
          // same row (coalesced loads); training: the same chunk of the next
          // rows, so that the transposed copy is written coalesced
          const int r = TRAIN ? e % kTile : e / nq, q = TRAIN ? e / kTile : e % nq;
          const int pr = tile * kTile + r;
          uint4 v = make_uint4(0, 0, 0, 0);
          const bool in = pr < P && q * 8 < d.c_in;
          const uint16_t* src = a.x + ((size_t)pr * T + step) * d.c_in;
          if (in && vec) {
            v = reinterpret_cast<const uint4*>(src)[q];
          } else if (in) {  // element by element, zeros past C_in
            uint16_t* ev = reinterpret_cast<uint16_t*>(&v);
            for (int i = 0; i < 8; ++i) ev[i] = q * 8 + i < d.c_in ? src[q * 8 + i] : 0;
          }
          *reinterpret_cast<uint4*>(sm + S.a + kmajor_offset(r, q * 8, kx0)) = v;
          if (TRAIN && in) {
            const uint16_t* ev = reinterpret_cast<const uint16_t*>(&v);
            const size_t cr = (size_t)step * P + pr;
            for (int i = 0; i < 8 && q * 8 + i < d.c_in; ++i)
              a.xT[(size_t)(q * 8 + i) * ld + cr] = ev[i];
          }
        }
      }
      float hprev[U];
      load_prev(0, hprev);
      store_row<U>(sm + S.b, row, u0, H, hprev);
      // ---- the GRU layers (unrolled); layer l reads its input from region
      // a and its previous state from region b and writes its new state into
      // region a
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        const uint32_t ax = sbase + S.a, ah = sbase + S.b;
        const int kx = l == 0 ? kx0 : H;
        if (t == 0) {
          fence_after_sync();
          mma_run(tbase + 0, ax, kx, sbase + S.w + 2 * L.rz[l], kx, 2 * H, kx, false);
          mma_run(tbase + 0, ah, H, sbase + S.w + 2 * L.hrz[l], H, 2 * H, H, true);
          mma_run(tbase + 2 * H, ax, kx, sbase + S.w + 2 * L.in[l], kx, H, kx, false);
          mma_run(tbase + 3 * H, ah, H, sbase + S.w + 2 * L.hn[l], H, H, H, false);
          mma_commit(bar);
        }
        if (!mbar_wait(bar, phase, kWaitPolls)) failed = true;
        phase ^= 1;
        if (__syncthreads_or(failed)) {
          failed = true;
          break;
        }
        fence_after_sync();
        float* hout = TRAIN ? act + act_h(H, l) : a.h_out + l * HP + (size_t)p * H;
        uint16_t* hT = TRAIN ? a.hT[l] + ldh - ld + col : nullptr;
        gru_epilogue<H, U>(tm, bias + l * 4 * H, hprev, sm + S.a, row, u0, hout, valid,
                           TRAIN ? act + act_g(H, NL, l) : nullptr, hT, ldh);
        if (l + 1 < NL) {  // region b is free: stage the next layer's previous state
          load_prev(l + 1, hprev);
          store_row<U>(sm + S.b, row, u0, H, hprev);
        }
      }
      if (failed) break;
      // ---- dense head: relu(h W1^T + b1) W2^T + b2 on the top layer's state,
      // or h W2^T + b2 without the hidden dense layer
      const float* b1 = bias + NL * 4 * H;
      if (d.mlp) {
      fence_async_smem();
      fence_before_sync();
      __syncthreads();
      if (t == 0) {
        fence_after_sync();
        mma_run(tbase + 0, sbase + S.a, H, sbase + S.w + 2 * L.w1, H, 128, H, false);
        mma_commit(bar);
      }
      if (!mbar_wait(bar, phase, kWaitPolls)) failed = true;
      phase ^= 1;
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      fence_after_sync();
#pragma unroll 1
      for (int c = 2 * cq; c < 2 * cq + 2; ++c) {  // 32 of the 128 units
        float v[16];
        tmem_ld16(tm + c * 16, v);
        if (TRAIN && valid) {
          float pre[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) pre[i] = v[i] + b1[c * 16 + i];
          store_f32<16>(act + act_a1(H, NL) + c * 16, pre);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + b1[c * 16 + i], 0.0f);
        store_row<16>(sm + S.m, row, c * 16, 128, v);
        if (TRAIN && valid)
#pragma unroll
          for (int i = 0; i < 16; ++i) a.y1T[(size_t)(c * 16 + i) * ld + col] = f2bf(v[i]);
      }
      }
      fence_async_smem();
      fence_before_sync();
      __syncthreads();
      const int n2 = d.nout();
      if (t == 0) {
        fence_after_sync();
        if (d.mlp)
          mma_run(tbase + 128, sbase + S.m, 128, sbase + S.w + 2 * L.w2, 128, n2, 128, false);
        else  // the single dense layer reads the top state in region a
          mma_run(tbase + 128, sbase + S.a, H, sbase + S.w + 2 * L.w2, H, n2, H, false);
        mma_commit(bar);
      }
      if (!mbar_wait(bar, phase, kWaitPolls)) failed = true;
      phase ^= 1;
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      fence_after_sync();
      const float* b2 = b1 + d.mlp;
      if (cq < n2 / 16) {  // one 16-column chunk of the output per warpgroup
        float v[16];
        tmem_ld16(tm + 128 + cq * 16, v);
        if (valid)
          for (int i = 0; i < 16; ++i) {
            const int j = cq * 16 + i;
            if (j < d.c_out) a.out[((size_t)p * T + step) * d.c_out + j] = v[i] + b2[j];
          }
      }
      fence_before_sync();
      __syncthreads();
    }
  }
  if (failed) {
    if (t == 0) atomicOr(a.status, 4);
    // let MMAs still in flight finish before the accumulator is released
    mbar_wait(bar, phase, kWaitPolls);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, 256);
  }
}

// -- generic GEMM: C = A B^T ----------------------------------------------------
constexpr int kKC = 64;
__global__ void __launch_bounds__(kTile, 1)
    umma_gemm_kernel(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                     float* __restrict__ C, int M, int N, int K, uint32_t ncols, int* status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sa = sm;                       // 128 x kKC
  uint8_t* sb = sm + kTile * kKC * 2;     // N x kKC
  uint64_t* bar = reinterpret_cast<uint64_t*>(sb + 256 * kKC * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (t == 0) mbar_init(bar, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *tslot;
  const int row0 = blockIdx.x * kTile;
  uint32_t phase = 0;
  bool failed = false;
  for (int k0 = 0; k0 < K && !failed; k0 += kKC) {
    const int kc = min(kKC, K - k0);
    for (int e = t; e < kTile * (kc / 8); e += kTile) {
      const int r = e / (kc / 8), q = e % (kc / 8);
      *reinterpret_cast<uint4*>(sa + kmajor_offset(r, q * 8, kc)) =
          *reinterpret_cast<const uint4*>(A + (size_t)(row0 + r) * K + k0 + q * 8);
    }
    for (int e = t; e < N * (kc / 8); e += kTile) {
      const int r = e / (kc / 8), q = e % (kc / 8);
      *reinterpret_cast<uint4*>(sb + kmajor_offset(r, q * 8, kc)) =
          *reinterpret_cast<const uint4*>(B + (size_t)r * K + k0 + q * 8);
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (t == 0) {
      fence_after_sync();
      mma_run(tbase, smem_u32(sa), kc, smem_u32(sb), kc, N, kc, k0 > 0);
      mma_commit(bar);
    }
    if (!mbar_wait(bar, phase, kWaitPolls)) failed = true;
    phase ^= 1;
    failed = __syncthreads_or(failed);
    fence_after_sync();
  }
  if (!failed) {
    const int r = row0 + t;
    for (int c = 0; c < N / 16; ++c) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + c * 16, v);
      for (int i = 0; i < 16; ++i) C[(size_t)r * N + c * 16 + i] = v[i];
    }
  } else {
    if (t == 0) atomicOr(status, 4);
    mbar_wait(bar, phase, kWaitPolls);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, ncols);
  }
}

template <bool TRAIN, int H, int NL>
void launch_forward_shape(const NetDims& d, const PackedNet& pk, const FwdArgs& a,
                          cudaStream_t st) {
  const PackLayout L = PackLayout::of(d);
  const FwdSmem S = FwdSmem::of(d, L.total);
  cudaFuncSetAttribute(patchnet_forward_kernel<TRAIN, H, NL>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (a.P + kTile - 1) / kTile;
  note_launch();
  patchnet_forward_kernel<TRAIN, H, NL><<<ntiles < sms ? ntiles : sms, kFwdThreads, S.total, st>>>(
      d, L, pk.w, pk.bias, a);
}

// one instantiation per network size of Table 1
template <bool TRAIN>
void launch_forward_impl(const NetDims& d, const PackedNet& pk, const FwdArgs& a, cudaStream_t st) {
  switch (d.hidden * 10 + d.layers) {
    case 321: launch_forward_shape<TRAIN, 32, 1>(d, pk, a, st); break;
    case 322: launch_forward_shape<TRAIN, 32, 2>(d, pk, a, st); break;
    case 323: launch_forward_shape<TRAIN, 32, 3>(d, pk, a, st); break;
    case 641: launch_forward_shape<TRAIN, 64, 1>(d, pk, a, st); break;
    case 642: launch_forward_shape<TRAIN, 64, 2>(d, pk, a, st); break;
    case 643: launch_forward_shape<TRAIN, 64, 3>(d, pk, a, st); break;
    default: break;  // rejected by net_supported
  }
}

}  // namespace

size_t patchnet_forward_smem(const NetDims& d) {
  return FwdSmem::of(d, PackLayout::of(d).total).total;
}

bool net_supported(const NetDims& d) {
  // (the input stream of the first layer's weight gradient, C_in + 1 rows
  // with the ones row, must fit the 144-row operand of that GEMM)
  if ((d.hidden != 32 && d.hidden != 64) || d.layers < 1 || d.layers > kMaxLayers ||
      (d.mlp != 128 && d.mlp != 0) || d.c_in < 1 || d.c_in > 127 || d.c_out < 1 ||
      d.c_out > 64 || d.nout() > 16 * kFwdWG || (d.bias != 0 && d.bias != 1))
    return false;
  constexpr size_t kSmemMax = 227 * 1024;
  return patchnet_forward_smem(d) <= kSmemMax && patchnet_backward_smem(d) <= kSmemMax;
}

void launch_pack_weights(const NetDims& d, const float* w, PackedNet& pk, cudaStream_t st) {
  const PackLayout L = PackLayout::of(d);
  const NetOffsets o = d.offsets();
  const int H = d.hidden;
  for (int l = 0; l < d.layers; ++l) {
    const int c = l == 0 ? d.c_in : H;
    const float* Wih = w + o.wih[l];
    const float* Whh = w + o.whh[l];
    const int kx = L.kx[l];
    note_launch();
    pack_block_kernel<<<64, 256, 0, st>>>(Wih, c, 0, 2 * H, c, 2 * H, kx, pk.w + L.rz[l]);
    note_launch();
    pack_block_kernel<<<64, 256, 0, st>>>(Wih, c, 2 * H, H, c, H, kx, pk.w + L.in[l]);
    note_launch();
    pack_block_kernel<<<64, 256, 0, st>>>(Whh, H, 0, 2 * H, H, 2 * H, H, pk.w + L.hrz[l]);
    note_launch();
    pack_block_kernel<<<64, 256, 0, st>>>(Whh, H, 2 * H, H, H, H, H, pk.w + L.hn[l]);
  }
  if (d.mlp) {
    note_launch();
    pack_block_kernel<<<64, 256, 0, st>>>(w + o.w1, H, 0, 128, H, 128, H, pk.w + L.w1);
  }
  const int k2 = d.k2();
  note_launch();
  pack_block_kernel<<<64, 256, 0, st>>>(w + o.w2, k2, 0, d.c_out, k2, d.nout(), k2, pk.w + L.w2);
  note_launch();
  pack_bias_kernel<<<1, 128, 0, st>>>(w, d, pk.bias);
}

void launch_patchnet_forward(const NetDims& d, const PackedNet& pk, const uint16_t* x,
                             const float* h, float* h_out, float* out, int P, int* status,
                             cudaStream_t st) {
  if (P <= 0) return;
  FwdArgs a{};
  a.x = x;
  a.P = P;
  a.T = 1;
  a.h_in = h;
  a.h_out = h_out;
  a.out = out;
  a.status = status;
  launch_forward_impl<false>(d, pk, a, st);
}

void launch_patchnet_train_forward(const NetDims& d, const PackedNet& pk, const uint16_t* x, int B,
                                   int T, float* ypred, const TrainBufs& tb, int* status,
                                   cudaStream_t st) {
  if (B <= 0 || T <= 0) return;
  FwdArgs a{};
  a.x = x;
  a.P = B;
  a.T = T;
  a.out = ypred;
  a.act = tb.act;
  a.xT = tb.xT;
  for (int l = 0; l < kMaxLayers; ++l) a.hT[l] = tb.hT[l];
  a.y1T = tb.y1T;
  a.status = status;
  launch_forward_impl<true>(d, pk, a, st);
}

int launch_umma_gemm(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                     int* status, cudaStream_t st) {
  if (M <= 0 || M % kTile || N < 16 || N > 256 || N % 16 || K < 16 || K % 16) return 1;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)N) ncols <<= 1;
  const size_t smem = (size_t)kTile * kKC * 2 + (size_t)256 * kKC * 2 + 64;
  cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  umma_gemm_kernel<<<M / kTile, kTile, smem, st>>>(A, B, C, M, N, K, ncols, status);
  return 0;
}

}  // namespace dnnmg
