// Vector kernels of the flexible GMRES solver (Sec. 2.2: GMRES preconditioned
// by multigrid) and of the Newton update (Eq. 6).  Reductions accumulate in
// FP64 and run in two fixed-order stages, so results are deterministic.
#include <atomic>

#include <cooperative_groups.h>

#include "kernels.h"
#include "krylov_body.cuh"

namespace dnnmg {

namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 296;  // two blocks per SM of a 148+ SM part

template <typename Ts, typename Td>
__global__ void cast_kernel(const Ts* __restrict__ a, Td* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (Td)a[i];
}

// b = a, d = c over n doubles: pairs as 16-byte accesses, the odd last
// element (n odd) by the first thread
__global__ void copy2_kernel(const double* __restrict__ a, double* __restrict__ b,
                             const double* __restrict__ c, double* __restrict__ d, size_t n) {
  const size_t n2 = n / 2;
  const double2* a2 = reinterpret_cast<const double2*>(a);
  const double2* c2 = reinterpret_cast<const double2*>(c);
  double2* b2 = reinterpret_cast<double2*>(b);
  double2* d2 = reinterpret_cast<double2*>(d);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2;
       i += (size_t)gridDim.x * blockDim.x) {
    b2[i] = a2[i];
    d2[i] = c2[i];
  }
  if (n % 2 && blockIdx.x == 0 && threadIdx.x == 0) {
    b[n - 1] = a[n - 1];
    d[n - 1] = c[n - 1];
  }
}

template <typename T>
__global__ void fill_kernel(T* a, T v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// partials[i * gridDim.x + block] = sum over the block's chunk of V[i] . w
template <typename T>
__global__ void __launch_bounds__(kThreads)
    multidot_kernel(const T* __restrict__ V, size_t ld, int k, const T* __restrict__ w, size_t n,
                    double* __restrict__ partials) {
  __shared__ double sh[32];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  for (int i = 0; i < k; ++i) {
    const T* v = V + (size_t)i * ld;
    double acc = 0.0;
    for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) acc += (double)v[e] * (double)w[e];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[(size_t)i * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void post_kernel(HostMail* m, unsigned long long seq, const double* src, int slot,
                            int n, const int* isrc, int islot, int ni) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i) m->v[slot + i] = src[i];
  for (int i = 0; i < ni; ++i) m->iv[islot + i] = isrc[i];
  mail_post(m, seq);
}

__global__ void dots_finish_kernel(const double* __restrict__ partials, int nb, double* out,
                                   HostMail* mail, unsigned long long seq) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[(size_t)blockIdx.x * nb + b];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    out[blockIdx.x] = t;
    if (mail) {  // a single block (k = 1)
      mail->v[0] = t;
      mail_post(mail, seq);
    }
  }
}

template <typename T>
__global__ void multiaxpy_kernel(const T* __restrict__ V, size_t ld, int k,
                                 const double* __restrict__ h, T* __restrict__ w, size_t n) {
  __shared__ double sh[64];
  if (threadIdx.x < k) sh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double acc = (double)w[e];
    for (int i = 0; i < k; ++i) acc -= sh[i] * (double)V[(size_t)i * ld + e];
    w[e] = (T)acc;
  }
}

template <typename T>
__global__ void scale_dev_kernel(const T* __restrict__ x, const double* a, int mode,
                                 T* __restrict__ y, size_t n) {
  const double s = block_scalar([&] {
    double v = *a;
    if (mode == 2) v = sqrt(fmax(v, 0.0));
    if (mode >= 1) v = v != 0.0 ? 1.0 / v : 0.0;
    return v;
  });
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    y[e] = (T)(s * (double)x[e]);
}

template <typename T, typename Tx>
__global__ void combine_kernel(const T* __restrict__ Z, size_t ld, int k,
                               const double* __restrict__ y, double eps, Tx* __restrict__ x,
                               size_t n) {
  __shared__ double sh[64];
  if (threadIdx.x < k) sh[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += sh[i] * (double)Z[(size_t)i * ld + e];
    x[e] = (Tx)((double)x[e] + eps * acc);
  }
}

__global__ void givens_kernel(double* H, int ldh, double* cs, double* sn, double* g,
                              const double* hcol, int j, double* resid) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *resid = givens_column(H, ldh, cs, sn, g, hcol, j);
}

__global__ void backsolve_kernel(const double* H, int ldh, const double* g, int k, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  backsolve_small(H, ldh, g, k, y);
}

template <typename T>
__global__ void gmres_start_kernel(const T* __restrict__ r, const double* nrm2, T* __restrict__ v0,
                                   double* g, size_t n, HostMail* mail, unsigned long long seq) {
  const double beta = block_scalar([&] { return sqrt(fmax(*nrm2, 0.0)); });
  const double s = block_scalar([&] { return beta > 0 ? 1.0 / beta : 0.0; });
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g[0] = beta;
    if (mail) {
      mail->v[1] = *nrm2;
      mail_post(mail, seq);
    }
  }
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    v0[e] = (T)(s * (double)r[e]);
}

// One Arnoldi step (arnoldi_body) in one cooperative launch of kDotBlocks
// blocks.
constexpr int kArnThreads = 512;
template <typename T>
__global__ void __launch_bounds__(kArnThreads) arnoldi_kernel(const ArnoldiArgs<T> a) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  arnoldi_body<T, kArnThreads>(a, [&] { grid.sync(); });
}

// The start of an FGMRES cycle in one cooperative launch of kDotBlocks
// blocks: with init, the right-hand side r64 is rounded to T (rT, and the
// first residual rcur = rT) and the correction wsol cleared; then |rcur|^2
// (the chunks of multidot_kernel; products and per-thread sums in T, the
// sums over threads and over the blocks' partials in FP64, the latter in one
// fixed order repeated by every block), V0 = rcur / |rcur| (scaled in T)
// and g[0] = |rcur|.  hcol[0] = |rcur|^2; with mail it is also posted into
// mail->v[1].  Per element only the rounding of r64 is an FP64 operation.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    fgmres_begin_kernel(const double* __restrict__ r64, T* __restrict__ rT, T* __restrict__ wsol,
                        T* __restrict__ rcur, T* __restrict__ v0, size_t n,
                        double* __restrict__ partials, double* hcol, double* g, int init,
                        HostMail* mail, unsigned long long seq, int* skip, double* target,
                        double rtol) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  __shared__ double nrm2s;
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  T acc = T(0);
  for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    T t;
    if (init) {
      t = (T)r64[e];
      rT[e] = t;
      rcur[e] = t;
      wsol[e] = T(0);
    } else {
      t = rcur[e];
    }
    acc += t * t;
  }
  const double bsum = block_sum((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = bsum;
  grid.sync();
  double a2 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a2 += partials[b];
  const double tot = block_sum(a2, sh);
  if (threadIdx.x == 0) nrm2s = tot;
  __syncthreads();
  const double nrm2 = nrm2s;
  const double beta = block_scalar([&] { return sqrt(fmax(nrm2, 0.0)); });
  const double sc = block_scalar([&] { return beta > 0 ? 1.0 / beta : 0.0; });
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hcol[0] = nrm2;
    g[0] = beta;
    if (skip) {  // a new cycle runs; the first cycle's |r| sets the stopping target
      *skip = 0;
      if (init) *target = rtol * beta;
    }
    if (mail) {
      mail->v[1] = nrm2;
      mail_post(mail, seq);
    }
  }
  // the thread's own elements of rcur (written above by this thread)
  const T sT = (T)sc;
  for (size_t e = lo + threadIdx.x; e < hi; e += blockDim.x) v0[e] = sT * rcur[e];
}

// The end of a converged FGMRES cycle in one launch: y = H^-1 g (the
// k x k back substitution in FP64, repeated by every block), then
// x64 += eps * (wsol + sum_i y_i Z_i) with the combination taken in T (the
// precision of the Krylov vectors) and only the update of x64 in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    fgmres_finish_kernel(const double* __restrict__ H, int ldh, const double* __restrict__ g,
                         int k, const T* __restrict__ Z, size_t ld,
                         const T* __restrict__ wsol, double eps, double* __restrict__ x64,
                         size_t n) {
  __shared__ double y[64];
  __shared__ T yT[64];
  if (threadIdx.x == 0) {
    backsolve_small(H, ldh, g, k, y);
    for (int i = 0; i < k; ++i) yT[i] = (T)y[i];
  }
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    T acc = wsol[e];
    for (int i = 0; i < k; ++i) acc += yT[i] * Z[(size_t)i * ld + e];
    x64[e] += eps * (double)acc;
  }
}

inline int blocks_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

size_t dots_partials(size_t n, int k) { return (size_t)kDotBlocks * (k > 0 ? k : 1); }

template <typename Ts, typename Td>
void launch_cast(const Ts* a, Td* b, size_t n, cudaStream_t st) {
  note_launch();
  cast_kernel<Ts, Td><<<blocks_for(n), kThreads, 0, st>>>(a, b, n);
}

void launch_copy2(const double* a, double* b, const double* c, double* d, size_t n,
                  cudaStream_t st) {
  const bool vec = ((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) % 16 == 0;
  if (!vec) {
    cudaMemcpyAsync(b, a, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d, c, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return;
  }
  note_launch();
  copy2_kernel<<<blocks_for(n / 2 + 1), kThreads, 0, st>>>(a, b, c, d, n);
}

template <typename T>
void launch_fill(T* a, T v, size_t n, cudaStream_t st) {
  note_launch();
  fill_kernel<T><<<blocks_for(n), kThreads, 0, st>>>(a, v, n);
}

template <typename T>
void launch_multidot(const T* V, size_t ld, int k, const T* w, size_t n, double* partials,
                     double* out, cudaStream_t st, HostMail* mail, unsigned long long seq) {
  note_launch();
  multidot_kernel<T><<<kDotBlocks, kThreads, 0, st>>>(V, ld, k, w, n, partials);
  note_launch();
  dots_finish_kernel<<<k, kThreads, 0, st>>>(partials, kDotBlocks, out, k == 1 ? mail : nullptr,
                                             seq);
}

void launch_post(HostMail* mail, unsigned long long seq, const double* src, int slot, int n,
                 const int* isrc, int islot, int ni, cudaStream_t st) {
  note_launch();
  post_kernel<<<1, 32, 0, st>>>(mail, seq, src, slot, n, isrc, islot, ni);
}

template <typename T>
void launch_multiaxpy(const T* V, size_t ld, int k, const double* h, T* w, size_t n,
                      cudaStream_t st) {
  note_launch();
  multiaxpy_kernel<T><<<blocks_for(n), kThreads, 0, st>>>(V, ld, k, h, w, n);
}

template <typename T>
void launch_scale_dev(const T* x, const double* a, int mode, T* y, size_t n, cudaStream_t st) {
  note_launch();
  scale_dev_kernel<T><<<blocks_for(n), kThreads, 0, st>>>(x, a, mode, y, n);
}

template <typename T, typename Tx>
void launch_combine(const T* Z, size_t ld, int k, const double* y, double eps, Tx* x, size_t n,
                    cudaStream_t st) {
  note_launch();
  combine_kernel<T, Tx><<<blocks_for(n), kThreads, 0, st>>>(Z, ld, k, y, eps, x, n);
}

// blocks of the cooperative Arnoldi launch (one per SM), 0 if it cannot run
template <typename T>
int arnoldi_blocks() {
  static const int nblk = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, arnoldi_kernel<T>,
                                                                  kArnThreads, 0) == cudaSuccess &&
                    per >= 1 && sms <= kDotBlocks;
    cudaGetLastError();
    return ok ? sms : 0;
  }();
  return nblk;
}

template <typename T>
bool arnoldi_available() {
  return arnoldi_blocks<T>() > 0;
}

template <typename T>
int launch_arnoldi_step(const T* V, size_t ld, int j, T* w, size_t n, double* partials,
                        double* hcol, double* H, int ldh, double* cs, double* sn, double* gvec,
                        double* resid, cudaStream_t st, HostMail* mail, unsigned long long seq,
                        int slot, int* skip, const double* target, int its, int maxit) {
  if (j + 2 > 64) return 1;  // the second pass holds k + 1 values
  const int nblk = arnoldi_blocks<T>();
  if (nblk == 0) return 1;
  const ArnoldiArgs<T> a{V,  ld, j,    w,    n,    partials, hcol,   H,  ldh,  cs,
                         sn, gvec, resid, mail, seq, slot,     skip,  target, its, maxit};
  void* args[] = {(void*)&a};
  if (cudaLaunchCooperativeKernel((void*)arnoldi_kernel<T>, dim3(nblk), dim3(kArnThreads), args,
                                  0, st) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  note_launch();
  return 0;
}

void launch_givens(double* H, int ldh, double* cs, double* sn, double* gvec, const double* hcol,
                   int j, double* resid, cudaStream_t st) {
  note_launch();
  givens_kernel<<<1, 32, 0, st>>>(H, ldh, cs, sn, gvec, hcol, j, resid);
}

void launch_backsolve(const double* H, int ldh, const double* gvec, int k, double* y,
                      cudaStream_t st) {
  note_launch();
  backsolve_kernel<<<1, 32, 0, st>>>(H, ldh, gvec, k, y);
}

template <typename T>
int launch_fgmres_begin(const double* r64, T* rT, T* wsol, T* rcur, T* v0, size_t n,
                        double* partials, double* hcol, double* gvec, bool init, HostMail* mail,
                        unsigned long long seq, cudaStream_t st, int* skip, double* target,
                        double rtol) {
  static const bool fits = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgmres_begin_kernel<T>,
                                                                  kThreads, 0) == cudaSuccess &&
                    per * sms >= kDotBlocks;
    cudaGetLastError();
    return ok;
  }();
  if (!fits) return 1;
  int in = init ? 1 : 0;
  void* args[] = {(void*)&r64,  (void*)&rT,       (void*)&wsol, (void*)&rcur,
                  (void*)&v0,   (void*)&n,        (void*)&partials, (void*)&hcol,
                  (void*)&gvec, (void*)&in,       (void*)&mail, (void*)&seq,
                  (void*)&skip, (void*)&target,   (void*)&rtol};
  if (cudaLaunchCooperativeKernel((void*)fgmres_begin_kernel<T>, dim3(kDotBlocks), dim3(kThreads),
                                  args, 0, st) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  note_launch();
  return 0;
}

template <typename T>
void launch_fgmres_finish(const double* H, int ldh, const double* gvec, int k, const T* Z,
                          size_t ld, const T* wsol, double eps, double* x64, size_t n,
                          cudaStream_t st) {
  note_launch();
  const int nb = std::min(blocks_for(n), kDotBlocks);
  fgmres_finish_kernel<T><<<nb, kThreads, 0, st>>>(H, ldh, gvec, k, Z, ld, wsol, eps, x64, n);
}

template <typename T>
void launch_gmres_start(const T* r, const double* nrm2, T* v0, double* gvec, size_t n,
                        cudaStream_t st, HostMail* mail, unsigned long long seq) {
  note_launch();
  gmres_start_kernel<T><<<blocks_for(n), kThreads, 0, st>>>(r, nrm2, v0, gvec, n, mail, seq);
}

#define DNNMG_INST(T)                                                                          \
  template void launch_fill<T>(T*, T, size_t, cudaStream_t);                                   \
  template void launch_multidot<T>(const T*, size_t, int, const T*, size_t, double*, double*,  \
                                   cudaStream_t, HostMail*, unsigned long long);               \
  template void launch_multiaxpy<T>(const T*, size_t, int, const double*, T*, size_t,          \
                                    cudaStream_t);                                             \
  template void launch_scale_dev<T>(const T*, const double*, int, T*, size_t, cudaStream_t);  \
  template void launch_gmres_start<T>(const T*, const double*, T*, double*, size_t,            \
                                      cudaStream_t, HostMail*, unsigned long long);            \
  template void launch_combine<T, T>(const T*, size_t, int, const double*, double, T*, size_t, \
                                     cudaStream_t);                                            \
  template int launch_arnoldi_step<T>(const T*, size_t, int, T*, size_t, double*, double*,     \
                                      double*, int, double*, double*, double*, double*,        \
                                      cudaStream_t, HostMail*, unsigned long long, int, int*,  \
                                      const double*, int, int);                                \
  template bool arnoldi_available<T>();                                                       \
  template int launch_fgmres_begin<T>(const double*, T*, T*, T*, T*, size_t, double*, double*, \
                                      double*, bool, HostMail*, unsigned long long,            \
                                      cudaStream_t, int*, double*, double);                    \
  template void launch_fgmres_finish<T>(const double*, int, const double*, int, const T*,      \
                                        size_t, const T*, double, double*, size_t,             \
                                        cudaStream_t);
DNNMG_INST(float)
DNNMG_INST(double)
#undef DNNMG_INST
template void launch_combine<float, double>(const float*, size_t, int, const double*, double,
                                            double*, size_t, cudaStream_t);
template void launch_fill<uint16_t>(uint16_t*, uint16_t, size_t, cudaStream_t);
template void launch_cast<double, float>(const double*, float*, size_t, cudaStream_t);
template void launch_cast<float, double>(const float*, double*, size_t, cudaStream_t);
template void launch_cast<double, double>(const double*, double*, size_t, cudaStream_t);
template void launch_cast<float, float>(const float*, float*, size_t, cudaStream_t);

}  // namespace dnnmg
