// Matrix-free operator kernels: Jacobian apply, defect, FP64 nonlinear
// residual and the old-time right-hand side (Sec. 2.1, Eqs. 3-6).
//
// Apply, defect and residual run tiled (32 x 8 nodes per block, cell and
// patch rows computed once per tile, optile_body.cuh); the right-hand-side
// kernels run one thread per node with 32 x 4 blocks, x fastest, so each
// warp reads contiguous rows of the SoA fields.
#include "kernels.h"
#include "dfloat.cuh"
#include "krylov_body.cuh"
#include "optile_body.cuh"
#include "vbody.cuh"

namespace dnnmg {

namespace {

constexpr int kBX = 32, kBY = 4;

__global__ void __launch_bounds__(kBX* kBY)
    old_rhs64_kernel(Grid g, double m, const double* __restrict__ x, double* __restrict__ f,
                     double* __restrict__ copy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  old_rhs64_node(g, m, x, f, i, j);
  if (copy) {  // the state itself, saved beside the right-hand side
    const int n = j * g.nnx + i;
    for (int c = 0; c < 3; ++c) copy[c * g.nn + n] = x[c * g.nn + n];
  }
}

__global__ void __launch_bounds__(kBX* kBY)
    explicit_sub64_kernel(Grid g, Sten<double> sx, double coef, const double* __restrict__ x,
                          double* __restrict__ f) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= g.nnx || j >= g.nny) return;
  explicit_sub64_node(g, sx, coef, x, f, i, j);
}

inline dim3 node_grid(const Grid& g) { return dim3(cdiv(g.nnx, kBX), cdiv(g.nny, kBY)); }

// Tiled variants (optile_body.cuh): one block per TX x TY nodes.
constexpr int kTX = 32, kTY = 8;

template <typename T>
__global__ void __launch_bounds__(kTX* kTY)
    apply_tiled_kernel(Grid g, Sten<T> s, const T* __restrict__ w, const T* __restrict__ vb,
                       T* __restrict__ y, const int* skip) {
  if (skip && *skip) return;  // a speculative FGMRES iteration after the cycle stopped
  extern __shared__ __align__(16) uint8_t smraw[];
  auto& S = *reinterpret_cast<OpSmem<T, kTX, kTY>*>(smraw);
  T ru, rv, rp;
  int n;
  op_tile_rows<T, false, true, kTX, kTY>(g, s, w, vb, blockIdx.x, blockIdx.y, S, ru, rv, rp, n);
  if (n < 0) return;
  const uint8_t f = op_tile_flags<T, kTX, kTY>(S);
  y[n] = (f & kVDir) ? w[n] : ru;
  y[g.nn + n] = (f & kVDir) ? w[g.nn + n] : rv;
  y[2 * g.nn + n] = (f & kPFix) ? w[2 * g.nn + n] : rp;
}

template <typename T>
__global__ void __launch_bounds__(kTX* kTY)
    defect_tiled_kernel(Grid g, Sten<T> s, const T* __restrict__ b, const T* __restrict__ x,
                        const T* __restrict__ vb, T* __restrict__ d, bool masked) {
  extern __shared__ __align__(16) uint8_t smraw[];
  auto& S = *reinterpret_cast<OpSmem<T, kTX, kTY>*>(smraw);
  T ru, rv, rp;
  int n;
  op_tile_rows<T, false, true, kTX, kTY>(g, s, x, vb, blockIdx.x, blockIdx.y, S, ru, rv, rp, n);
  if (n < 0) return;
  const uint8_t f = op_tile_flags<T, kTX, kTY>(S);
  const int nn = g.nn;
  if (f & kVDir) {
    d[n] = masked ? T(0) : b[n] - x[n];
    d[nn + n] = masked ? T(0) : b[nn + n] - x[nn + n];
  } else {
    d[n] = b[n] - ru;
    d[nn + n] = b[nn + n] - rv;
  }
  if (f & kPFix)
    d[2 * nn + n] = masked ? T(0) : b[2 * nn + n] - x[2 * nn + n];
  else
    d[2 * nn + n] = b[2 * nn + n] - rp;
}

// |r|^2 over all blocks of the launch (see NormOut); every thread of the
// block calls it with the squares of its node's residual (0 for none)
__device__ __forceinline__ void norm_reduce(double sq, const NormOut& no) {
  __shared__ double sh[32];
  __shared__ bool last;
  const double bs = block_sum(sq, sh);  // valid in thread 0
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    no.partials[b] = bs;
    __threadfence();
    last = atomicAdd(no.counter, 1u) == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) acc += __ldcg(no.partials + q);
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    *no.out = tot;
    *no.counter = 0u;
    if (no.mail) {
      no.mail->v[0] = tot;
      if (no.status)
        for (int i = 0; i < 4; ++i) no.mail->iv[i] = no.status[i];
      mail_post(no.mail, no.seq);
    }
  }
}

__global__ void __launch_bounds__(kTX* kTY)
    residual64_tiled_kernel(Grid g, Sten<double> s, const double* __restrict__ x,
                            const double* __restrict__ f, double* __restrict__ r,
                            const NormOut no) {
  extern __shared__ __align__(16) uint8_t smraw[];
  auto& S = *reinterpret_cast<OpSmem<double, kTX, kTY>*>(smraw);
  double ru, rv, rp;
  int n;
  op_tile_rows<double, true, false, kTX, kTY>(g, s, x, nullptr, blockIdx.x, blockIdx.y, S, ru, rv,
                                              rp, n);
  double sq = 0.0;
  if (n >= 0) {
    const uint8_t fl = op_tile_flags<double, kTX, kTY>(S);
    const int nn = g.nn;
    const double r0 = (fl & kVDir) ? 0.0 : f[n] - ru;
    const double r1 = (fl & kVDir) ? 0.0 : f[nn + n] - rv;
    const double r2 = (fl & kPFix) ? 0.0 : f[2 * nn + n] - rp;
    r[n] = r0, r[nn + n] = r1, r[2 * nn + n] = r2;
    sq = r0 * r0 + r1 * r1 + r2 * r2;
  }
  if (no.partials) norm_reduce(sq, no);
}

// The same residual with the operator evaluated in FP32 (the state rounded
// to FP32, the subtraction from f in FP64): the fine-level residual whose
// only use is the network's input features, which are rounded to BF16.
__global__ void __launch_bounds__(kTX* kTY)
    residual32_tiled_kernel(Grid g, Sten<float> s, const double* __restrict__ x,
                            const double* __restrict__ f, double* __restrict__ r) {
  extern __shared__ __align__(16) uint8_t smraw[];
  auto& S = *reinterpret_cast<OpSmem<float, kTX, kTY>*>(smraw);
  float ru, rv, rp;
  int n;
  op_tile_rows<float, true, false, kTX, kTY, kTX * kTY, double>(g, s, x, nullptr, blockIdx.x,
                                                               blockIdx.y, S, ru, rv, rp, n);
  if (n < 0) return;
  const uint8_t fl = op_tile_flags<float, kTX, kTY>(S);
  const int nn = g.nn;
  r[n] = (fl & kVDir) ? 0.0 : f[n] - (double)ru;
  r[nn + n] = (fl & kVDir) ? 0.0 : f[nn + n] - (double)rv;
  r[2 * nn + n] = (fl & kPFix) ? 0.0 : f[2 * nn + n] - (double)rp;
}

// The same residual with the operator evaluated in double-float arithmetic
// (about 48 significant bits; the subtraction from f in FP64), for
// mixed-precision contexts.
__global__ void __launch_bounds__(kTX* kTY)
    residual_df_tiled_kernel(Grid g, Sten<dfloat> s, const double* __restrict__ x,
                             const double* __restrict__ f, double* __restrict__ r,
                             const NormOut no) {
  extern __shared__ __align__(16) uint8_t smraw[];
  auto& S = *reinterpret_cast<OpSmem<dfloat, kTX, kTY>*>(smraw);
  dfloat ru, rv, rp;
  int n;
  op_tile_rows<dfloat, true, false, kTX, kTY, kTX * kTY, double>(
      g, s, x, nullptr, blockIdx.x, blockIdx.y, S, ru, rv, rp, n);
  double sq = 0.0;
  if (n >= 0) {
    const uint8_t fl = op_tile_flags<dfloat, kTX, kTY>(S);
    const int nn = g.nn;
    const double r0 = (fl & kVDir) ? 0.0 : f[n] - (double)ru;
    const double r1 = (fl & kVDir) ? 0.0 : f[nn + n] - (double)rv;
    const double r2 = (fl & kPFix) ? 0.0 : f[2 * nn + n] - (double)rp;
    r[n] = r0, r[nn + n] = r1, r[2 * nn + n] = r2;
    sq = r0 * r0 + r1 * r1 + r2 * r2;
  }
  if (no.partials) norm_reduce(sq, no);
}

inline dim3 tile_grid(const Grid& g) { return dim3(cdiv(g.nnx, kTX), cdiv(g.nny, kTY)); }

// opt a kernel in to `bytes` of dynamic shared memory; callers keep the
// result in a function-local static, so each launcher does it once
template <typename K>
size_t smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return bytes;
}

}  // namespace

template <typename T>
void launch_apply(const Grid& g, const Sten<T>& s, const T* w, const T* vb, T* y, cudaStream_t st,
                  const int* skip) {
  note_launch();
  static const size_t sm = smem_attr(apply_tiled_kernel<T>, sizeof(OpSmem<T, kTX, kTY>));
  apply_tiled_kernel<T><<<tile_grid(g), kTX * kTY, sm, st>>>(g, s, w, vb, y, skip);
}

template <typename T>
void launch_defect(const Grid& g, const Sten<T>& s, const T* b, const T* x, const T* vb, T* d,
                   bool masked, cudaStream_t st) {
  note_launch();
  static const size_t sm = smem_attr(defect_tiled_kernel<T>, sizeof(OpSmem<T, kTX, kTY>));
  defect_tiled_kernel<T><<<tile_grid(g), kTX * kTY, sm, st>>>(g, s, b, x, vb, d, masked);
}

int residual_blocks(const Grid& g) { return cdiv(g.nnx, kTX) * cdiv(g.nny, kTY); }

void launch_residual64(const Grid& g, const Sten<double>& s, const double* x, const double* f,
                       double* r, cudaStream_t st, bool dfloat_ops, const NormOut& no) {
  if (dfloat_ops) {
    Sten<dfloat> sd;
    for (int e = 0; e < 16; ++e) {
      sd.E[e] = dfloat(s.E[e]);
      sd.Dx[e] = dfloat(s.Dx[e]);
      sd.Dy[e] = dfloat(s.Dy[e]);
    }
    for (int e = 0; e < 81; ++e) sd.S9[e] = dfloat(s.S9[e]);
    sd.wq = dfloat(s.wq);
    sd.ih = dfloat(s.ih);
    note_launch();
    static const size_t smd =
        smem_attr(residual_df_tiled_kernel, sizeof(OpSmem<dfloat, kTX, kTY>));
    residual_df_tiled_kernel<<<tile_grid(g), kTX * kTY, smd, st>>>(g, sd, x, f, r, no);
    return;
  }
  note_launch();
  static const size_t sm = smem_attr(residual64_tiled_kernel, sizeof(OpSmem<double, kTX, kTY>));
  residual64_tiled_kernel<<<tile_grid(g), kTX * kTY, sm, st>>>(g, s, x, f, r, no);
}

void launch_residual_features(const Grid& g, const Sten<double>& s, const double* x,
                              const double* f, double* r, cudaStream_t st, bool fp32_ops) {
  if (!fp32_ops) {
    launch_residual64(g, s, x, f, r, st, false);
    return;
  }
  Sten<float> sf;
  for (int e = 0; e < 16; ++e) {
    sf.E[e] = (float)s.E[e];
    sf.Dx[e] = (float)s.Dx[e];
    sf.Dy[e] = (float)s.Dy[e];
  }
  for (int e = 0; e < 81; ++e) sf.S9[e] = (float)s.S9[e];
  sf.wq = (float)s.wq;
  sf.ih = (float)s.ih;
  note_launch();
  static const size_t sm = smem_attr(residual32_tiled_kernel, sizeof(OpSmem<float, kTX, kTY>));
  residual32_tiled_kernel<<<tile_grid(g), kTX * kTY, sm, st>>>(g, sf, x, f, r);
}

void launch_old_time_rhs64(const Grid& g, double inv_k, const double* x_old, double* f,
                           cudaStream_t st, double* copy) {
  note_launch();
  old_rhs64_kernel<<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, g.h * g.h / 36.0 * inv_k, x_old,
                                                              f, copy);
}

void launch_explicit_sub64(const Grid& g, const Sten<double>& sx, double coef, const double* x,
                           double* f, cudaStream_t st) {
  note_launch();
  explicit_sub64_kernel<<<node_grid(g), dim3(kBX, kBY), 0, st>>>(g, sx, coef, x, f);
}

template void launch_apply<float>(const Grid&, const Sten<float>&, const float*, const float*,
                                  float*, cudaStream_t, const int*);
template void launch_apply<double>(const Grid&, const Sten<double>&, const double*, const double*,
                                   double*, cudaStream_t, const int*);
template void launch_defect<float>(const Grid&, const Sten<float>&, const float*, const float*,
                                   const float*, float*, bool, cudaStream_t);
template void launch_defect<double>(const Grid&, const Sten<double>&, const double*,
                                    const double*, const double*, double*, bool, cudaStream_t);

}  // namespace dnnmg
