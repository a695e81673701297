// Batched stage kernels: one launch covers one stage (a Vanka colour pass, a
// defect, a transfer, a vector operation, ...) of every problem of a batch.
// Each block takes its (problem, block) pair from the stage's work list,
// returns at once if the problem is masked, loads the problem's level record
// and constants and runs the same per-node, per-tile or per-cell body as the
// single-problem kernels (vbody.cuh, vanka_body.cuh, coarse_body.cuh,
// dnnmg_body.cuh, krylov_body.cuh), so the arithmetic is identical.
#include "batch.h"
#include "coarse_body.cuh"
#include "dnnmg_body.cuh"
#include "kernels.h"
#include "krylov_body.cuh"
#include "vanka_body.cuh"
#include "vbody.cuh"

namespace dnnmg {

namespace {

__device__ __forceinline__ bool masked(const int* act, int p) { return act && !act[p]; }

// block-wide copy of a constants record into shared memory
template <typename S>
__device__ __forceinline__ void load_const(S& dst, const S& src) {
  static_assert(sizeof(S) % sizeof(int) == 0, "record size");
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int e = threadIdx.x; e < (int)(sizeof(S) / sizeof(int)); e += blockDim.x) d[e] = s[e];
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ const BLev<T>& lev_of(const BView<T>& v, int p, int k) {
  return v.lev[(size_t)p * v.nL + k];
}

// ---------------------------------------------------------------- V-cycle

template <typename T, int TCX, int TCY>
__global__ void __launch_bounds__(4 * TCX * TCY, pass_min_blocks<T>(4 * TCX * TCY))
    bpass_kernel(BView<T> v, int k, int colour, int in, int out, const T* __restrict__ topb,
                 T* __restrict__ topx, T omega, const int2* __restrict__ work,
                 const int* __restrict__ act) {
  const int2 w = work[blockIdx.x];
  if (masked(act, w.x)) return;
  __shared__ Sten<T> ss;
  extern __shared__ __align__(16) uint8_t smraw[];
  const BLev<T> L = lev_of(v, w.x, k);
  load_const(ss, v.sT[(size_t)w.x * v.nL + k]);
  T* x0 = L.top ? topx + L.off : L.x;
  const T* b = L.top ? topb + L.off : L.b;
  const T* xin = in ? L.x2 : x0;
  T* xout = out ? L.x2 : x0;
  const int nbx = cdiv(L.g.nx / 2 + 1, TCX);
  vanka_pass_tile<T, TCX, TCY>(L.g, ss, colour, b, xin, L.vb, L.inv, omega, xout, w.y % nbx,
                               w.y / nbx, *reinterpret_cast<PassSmem<T, TCX, TCY>*>(smraw));
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bdefect_kernel(BView<T> v, int k, int in, const T* __restrict__ topb, T* __restrict__ topx,
                   const int2* __restrict__ work, const int* __restrict__ act) {
  const int2 w = work[blockIdx.x];
  if (masked(act, w.x)) return;
  __shared__ Sten<T> ss;
  const BLev<T> L = lev_of(v, w.x, k);
  load_const(ss, v.sT[(size_t)w.x * v.nL + k]);
  const int n = w.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  const T* x0 = L.top ? topx + L.off : L.x;
  const T* b = L.top ? topb + L.off : L.b;
  defect_node<T>(L.g, ss, b, in ? L.x2 : x0, L.vb, L.d, true, n % L.g.nnx, n / L.g.nnx);
}

// work: node blocks of level k - 1 of the problems that have level k
template <typename T>
__global__ void __launch_bounds__(kNB)
    brestrict_kernel(BView<T> v, int k, const int2* __restrict__ work,
                     const int* __restrict__ act) {
  const int2 w = work[blockIdx.x];
  if (masked(act, w.x)) return;
  const BLev<T> F = lev_of(v, w.x, k), C = lev_of(v, w.x, k - 1);
  const int n = w.y * kNB + threadIdx.x;
  if (n >= C.g.nn) return;
  restrict_node<T, true>(F.g, C.g, F.d, C.b, 3, n % C.g.nnx, n / C.g.nnx);
  C.x[n] = T(0);
  C.x[C.g.nn + n] = T(0);
  C.x[2 * C.g.nn + n] = T(0);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bprolong_kernel(BView<T> v, int k, int in, T* __restrict__ topx, const int2* __restrict__ work,
                    const int* __restrict__ act) {
  const int2 w = work[blockIdx.x];
  if (masked(act, w.x)) return;
  const BLev<T> F = lev_of(v, w.x, k), C = lev_of(v, w.x, k - 1);
  const int n = w.y * kNB + threadIdx.x;
  if (n >= F.g.nn) return;
  T* x0 = F.top ? topx + F.off : F.x;
  prolong_add_node<T>(F.g, C.g, C.x, in ? F.x2 : x0, n % F.g.nnx, n / F.g.nnx);
}

// grid (row blocks, problems); the coarsest level is level 1 for every problem
template <typename T>
__global__ void __launch_bounds__(32 * kSolveWarps)
    bcoarse_solve_kernel(BView<T> v, const double* __restrict__ Ainv, long long astride,
                         const T* __restrict__ topb, T* __restrict__ topx,
                         const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (masked(act, p)) return;
  extern __shared__ double sb[];
  const BLev<T> C = lev_of(v, p, 1);
  const T* b = C.top ? topb + C.off : C.b;
  T* x = C.top ? topx + C.off : C.x;
  coarse_solve_rows<T>(C.g, Ainv + (size_t)p * astride, b, x, blockIdx.x, sb);
}

// ------------------------------------------------- top- and fine-level nodes

template <typename T>
__device__ __forceinline__ const BLev<T>& own_level(const BView<T>& v, int p, int dl) {
  return lev_of(v, p, v.par[p].L + dl);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bapply_kernel(BView<T> v, const T* __restrict__ w, const T* __restrict__ vbJ,
                  T* __restrict__ y, const int2* __restrict__ work, const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  __shared__ Sten<T> ss;
  const int k = v.par[wk.x].L;
  const BLev<T> L = lev_of(v, wk.x, k);
  load_const(ss, v.sT[(size_t)wk.x * v.nL + k]);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  apply_node<T>(L.g, ss, w + L.off, vbJ + L.off, y + L.off, n % L.g.nnx, n / L.g.nnx);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bdefect_top_kernel(BView<T> v, const T* __restrict__ b, const T* __restrict__ x,
                       const T* __restrict__ vbJ, T* __restrict__ d,
                       const int2* __restrict__ work, const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  __shared__ Sten<T> ss;
  const int k = v.par[wk.x].L;
  const BLev<T> L = lev_of(v, wk.x, k);
  load_const(ss, v.sT[(size_t)wk.x * v.nL + k]);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  defect_node<T>(L.g, ss, b + L.off, x + L.off, vbJ + L.off, d + L.off, false, n % L.g.nnx,
                 n / L.g.nnx);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bresidual64_kernel(BView<T> v, int dl, const double* __restrict__ x,
                       const double* __restrict__ f, double* __restrict__ r,
                       const int2* __restrict__ work, const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  __shared__ Sten<double> ss;
  const int k = v.par[wk.x].L + dl;
  const BLev<T> L = lev_of(v, wk.x, k);
  load_const(ss, v.s64[(size_t)wk.x * v.nL + k]);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  residual64_node(L.g, ss, x + L.off, f + L.off, r + L.off, n % L.g.nnx, n / L.g.nnx);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bold_rhs_kernel(BView<T> v, int dl, const double* __restrict__ xo, double* __restrict__ f,
                    const int2* __restrict__ work, const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  __shared__ Sten<double> ss;
  const BPar pr = v.par[wk.x];
  const int k = pr.L + dl;
  const BLev<T> L = lev_of(v, wk.x, k);
  if (pr.explicit_on) load_const(ss, v.sx[(size_t)wk.x * v.nL + k]);
  const double m = block_scalar([&] { return L.g.h * L.g.h / 36.0 * pr.inv_k; });
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  const int i = n % L.g.nnx, j = n / L.g.nnx;
  old_rhs64_node(L.g, m, xo + L.off, f + L.off, i, j);
  if (pr.explicit_on) explicit_sub64_node(L.g, ss, pr.ecoef, xo + L.off, f + L.off, i, j);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bcopy_impose_kernel(BView<T> v, int dl, const double* __restrict__ src,
                        double* __restrict__ dst, const int2* __restrict__ work,
                        const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> L = own_level(v, wk.x, dl);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  double* x = dst + L.off;
  if (src) {
    const double* s = src + L.off;
    x[n] = s[n];
    x[L.g.nn + n] = s[L.g.nn + n];
    x[2 * L.g.nn + n] = s[2 * L.g.nn + n];
  }
  impose_dirichlet_node(L.g, x, n % L.g.nnx, n / L.g.nnx);
}

// ---------------------------------------------------------- linearisation

template <typename T>
__global__ void __launch_bounds__(kNB)
    btop_vb_kernel(BView<T> v, const double* __restrict__ x64, const int2* __restrict__ work,
                   const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> L = own_level(v, wk.x, 0);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  L.vb64[n] = x64[L.off + n];
  L.vb64[L.g.nn + n] = x64[L.off + L.g.nn + n];
}

// work: node blocks of level k - 1 of the problems that have level k
template <typename T>
__global__ void __launch_bounds__(kNB)
    binject_vb_kernel(BView<T> v, int k, const int2* __restrict__ work,
                      const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> F = lev_of(v, wk.x, k), C = lev_of(v, wk.x, k - 1);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= C.g.nn) return;
  inject_node<double>(F.g, C.g, F.vb64, C.vb64, 2, n % C.g.nnx, n / C.g.nnx);
}

template <typename T>
__global__ void __launch_bounds__(kNB)
    bcast_vb_kernel(BView<T> v, int k, const int2* __restrict__ work,
                    const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> L = lev_of(v, wk.x, k);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= L.g.nn) return;
  L.vb[n] = (T)L.vb64[n];
  L.vb[L.g.nn + n] = (T)L.vb64[L.g.nn + n];
}

// work: (problem, colour * slot_blocks + slot_block)
template <typename T>
__global__ void __launch_bounds__(kSetupThreads)
    bsetup_kernel(BView<T> v, int k, int* __restrict__ status, const int2* __restrict__ work,
                  const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  __shared__ Sten<T> ss;
  const BLev<T> L = lev_of(v, wk.x, k);
  load_const(ss, v.sT[(size_t)wk.x * v.nL + k]);
  const int nsb = cdiv(vanka_slots(L.g), kSetupCells);
  __shared__ SetupSmem<T> W[kSetupCells];
  vanka_setup_cell<T>(L.g, ss, L.vb, L.inv, status + wk.x, wk.y / nsb,
                      (wk.y % nsb) * kSetupCells + threadIdx.x / 16, W[threadIdx.x / 16]);
}

template <typename T>
__global__ void bassemble_kernel(BView<T> v, double* __restrict__ cwork, long long cstride,
                                 const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (masked(act, p)) return;
  const BLev<T> C = lev_of(v, p, 1);
  assemble_row(C.g, v.s64[(size_t)p * v.nL + 1], C.vb64, cwork + (size_t)p * cstride,
               blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kLUThreads)
    blu_kernel(BView<T> v, double* __restrict__ cwork, long long cstride, long long bandsz,
               int* __restrict__ status, const int* __restrict__ act) {
  const int p = blockIdx.x;
  if (masked(act, p)) return;
  extern __shared__ double win[];
  const BLev<T> C = lev_of(v, p, 1);
  double* ab = cwork + (size_t)p * cstride;
  band_lu_block(C.g, ab, reinterpret_cast<int*>(ab + bandsz), status + p, win);
}

// the work area of a problem: band, pivots (n ints in n doubles), 1 / U(k, k)
template <typename T>
__global__ void brecip_kernel(BView<T> v, double* __restrict__ cwork, long long cstride,
                              long long bandsz, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (masked(act, p)) return;
  const BLev<T> C = lev_of(v, p, 1);
  double* ab = cwork + (size_t)p * cstride;
  band_diag_recip(C.g, ab, ab + bandsz + 3 * C.g.nn, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(32 * kInvWarps)
    binverse_kernel(BView<T> v, const double* __restrict__ cwork, long long cstride,
                    long long bandsz, double* __restrict__ Ainv, long long astride,
                    const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (masked(act, p)) return;
  extern __shared__ __align__(16) double sm[];
  const BLev<T> C = lev_of(v, p, 1);
  const double* ab = cwork + (size_t)p * cstride;
  band_inverse_block(C.g, ab, reinterpret_cast<const int*>(ab + bandsz), ab + bandsz + 3 * C.g.nn,
                     Ainv + (size_t)p * astride, blockIdx.x * kInvWarps, sm);
}

// -------------------------------------------------------------- vectors

template <typename T>
__global__ void __launch_bounds__(kVT)
    bmultidot_kernel(const T* __restrict__ V, size_t ld, int nv, const T* __restrict__ w,
                     double* __restrict__ part, int nblk, const int* __restrict__ vinst,
                     const int* __restrict__ act) {
  __shared__ double sh[32];
  if (masked(act, vinst[blockIdx.x])) return;
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
  double wl[kVE];
#pragma unroll
  for (int r = 0; r < kVE; ++r) wl[r] = (double)w[base + r * kVT];
  for (int j = 0; j < nv; ++j) {
    const T* vj = V + (size_t)j * ld + base;
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < kVE; ++r) acc += (double)vj[r * kVT] * wl[r];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)j * nblk + blockIdx.x] = t;
  }
}

// grid (problems, vectors)
__global__ void __launch_bounds__(kVT)
    bdots_finish_kernel(const double* __restrict__ part, int nblk, const int* __restrict__ first,
                        const int* __restrict__ count, double* __restrict__ out, int ostride,
                        const int* __restrict__ act) {
  __shared__ double sh[32];
  const int p = blockIdx.x, j = blockIdx.y;
  if (masked(act, p)) return;
  const double* pj = part + (size_t)j * nblk + first[p];
  double acc = 0.0;
  for (int b = threadIdx.x; b < count[p]; b += kVT) acc += pj[b];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) out[(size_t)p * ostride + j] = t;
}

template <typename T>
__global__ void __launch_bounds__(kVT)
    bmultiaxpy_kernel(const T* __restrict__ V, size_t ld, int nv, const double* __restrict__ h,
                      int hstride, T* __restrict__ w, const int* __restrict__ vinst,
                      const int* __restrict__ act) {
  __shared__ double sh[64];
  const int p = vinst[blockIdx.x];
  if (masked(act, p)) return;
  if (threadIdx.x < nv) sh[threadIdx.x] = h[(size_t)p * hstride + threadIdx.x];
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kVE; ++r) {
    const size_t e = base + r * kVT;
    double acc = (double)w[e];
    for (int j = 0; j < nv; ++j) acc -= sh[j] * (double)V[(size_t)j * ld + e];
    w[e] = (T)acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kVT)
    bscale_kernel(const T* __restrict__ x, const double* __restrict__ a, int astride, int mode,
                  T* __restrict__ y, const int* __restrict__ vinst, const int* __restrict__ act) {
  const int p = vinst[blockIdx.x];
  if (masked(act, p)) return;
  const double s = block_scalar([&] {
    double v = a[(size_t)p * astride];
    if (mode == 2) v = sqrt(fmax(v, 0.0));
    if (mode >= 1) v = v != 0.0 ? 1.0 / v : 0.0;
    return v;
  });
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kVE; ++r) y[base + r * kVT] = (T)(s * (double)x[base + r * kVT]);
}

template <typename T>
__global__ void __launch_bounds__(kVT)
    bstart_kernel(const T* __restrict__ r, const double* __restrict__ nrm2, int nstride,
                  T* __restrict__ v0, double* __restrict__ gv, int gstride,
                  const int* __restrict__ vinst, const int* __restrict__ first,
                  const int* __restrict__ act) {
  const int p = vinst[blockIdx.x];
  if (masked(act, p)) return;
  const double beta = block_scalar([&] { return sqrt(fmax(nrm2[(size_t)p * nstride], 0.0)); });
  const double s = block_scalar([&] { return beta > 0 ? 1.0 / beta : 0.0; });
  if (blockIdx.x == (unsigned)first[p] && threadIdx.x == 0) gv[(size_t)p * gstride] = beta;
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kVE; ++q) v0[base + q * kVT] = (T)(s * (double)r[base + q * kVT]);
}

template <typename T, typename Tx>
__global__ void __launch_bounds__(kVT)
    bcombine_kernel(const T* __restrict__ Z, size_t ld, const int* __restrict__ kcnt,
                    const double* __restrict__ y, int ystride, double eps, Tx* __restrict__ x,
                    const int* __restrict__ vinst, const int* __restrict__ act) {
  __shared__ double sh[64];
  const int p = vinst[blockIdx.x];
  if (masked(act, p)) return;
  const int k = kcnt ? kcnt[p] : 1;
  if (threadIdx.x < k) sh[threadIdx.x] = y[(size_t)p * ystride + threadIdx.x];
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kVE; ++r) {
    const size_t e = base + r * kVT;
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += sh[j] * (double)Z[(size_t)j * ld + e];
    x[e] = (Tx)((double)x[e] + eps * acc);
  }
}

__global__ void __launch_bounds__(kVT)
    bcopy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                 const int* __restrict__ vinst, const int* __restrict__ act) {
  if (masked(act, vinst[blockIdx.x])) return;
  const size_t base = (size_t)blockIdx.x * kVB + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kVE; ++r) dst[base + r * kVT] = src[base + r * kVT];
}

// one thread per problem
__global__ void bgivens_kernel(int nprob, int m, double* __restrict__ H, double* __restrict__ cs,
                               double* __restrict__ sn, double* __restrict__ gv,
                               const double* __restrict__ hcol, int j, double* __restrict__ resid,
                               const double* __restrict__ target, int* __restrict__ kcnt,
                               int* __restrict__ its, int maxit, int* __restrict__ gact) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob || !gact[p]) return;
  const int ldh = m + 1;
  const double r = givens_column(H + (size_t)p * ldh * ldh, ldh, cs + (size_t)p * ldh,
                                 sn + (size_t)p * ldh, gv + (size_t)p * (m + 2),
                                 hcol + (size_t)p * (2 * m + 4), j);
  resid[p] = r;
  kcnt[p] = j + 1;
  its[p] += 1;
  if (!(r > target[p]) || its[p] >= maxit) gact[p] = 0;
}

__global__ void bbacksolve_kernel(int nprob, int m, const double* __restrict__ H,
                                  const double* __restrict__ gv, const int* __restrict__ kcnt,
                                  double* __restrict__ y, const int* __restrict__ act) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob || masked(act, p)) return;
  const int ldh = m + 1;
  backsolve_small(H + (size_t)p * ldh * ldh, ldh, gv + (size_t)p * (m + 2), kcnt[p],
                  y + (size_t)p * ldh);
}

// ---------------------------------------------------------------- DNN-MG

// work: node blocks of level L + dlf; xc in the layout of level L + dlf - 1
// (the top layout for dlf = 1), xf in the layout of level L + dlf
template <typename T>
__global__ void __launch_bounds__(kNB)
    bprolong_state_kernel(BView<T> v, const double* __restrict__ xc, double* __restrict__ xf,
                          int ncomp, int zero_p, int dlf, const int2* __restrict__ work,
                          const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> F = own_level(v, wk.x, dlf), C = own_level(v, wk.x, dlf - 1);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= F.g.nn) return;
  prolong_state_node(F.g, C.g, xc + C.off, xf + F.off, ncomp, n % F.g.nnx, n / F.g.nnx);
  if (zero_p) xf[F.off + 2 * F.g.nn + n] = 0.0;
}

// work: node blocks of level L + dlf - 1; bf in the layout of level L + dlf,
// bc in the layout of level L + dlf - 1
template <typename T>
__global__ void __launch_bounds__(kNB)
    brestrict_full_kernel(BView<T> v, const double* __restrict__ bf, double* __restrict__ bc,
                          int ncomp, int dlf, const int2* __restrict__ work,
                          const int* __restrict__ act) {
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BLev<T> F = own_level(v, wk.x, dlf), C = own_level(v, wk.x, dlf - 1);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= C.g.nn) return;
  restrict_node<double, false>(F.g, C.g, bf + F.off, bc + C.off, ncomp, n % C.g.nnx,
                               n / C.g.nnx);
}

// patches of K x K fine nodes: K = 3 with one replaced level, 5 with two
template <typename T, int K>
__global__ void bgather_kernel(BView<T> v, int P, const int* __restrict__ pinst,
                               const int* __restrict__ pcell, const double* __restrict__ xt,
                               const double* __restrict__ r, const float* __restrict__ mean,
                               const float* __restrict__ stdv, uint16_t* __restrict__ X) {
  constexpr int kR = K == 3 ? 1 : 2, kCin = 4 * K * K + 4;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const int p = pinst[q];
  const BPar pr = v.par[p];
  const BLev<T>& L = lev_of(v, p, pr.L);
  const BLev<T>& F = lev_of(v, p, pr.L + kR);
  const FeatConsts fc{pr.feat_h, pr.feat_k, pr.feat_pe};
  gather_patch<false, K>(L.g, F.g, pcell[q], xt + F.off, r + F.off, mean, stdv, fc,
                         X + (size_t)q * kCin, nullptr);
}

template <typename T, int K>
__global__ void __launch_bounds__(kNB)
    bscatter_kernel(BView<T> v, const int* __restrict__ cell_patch, const float* __restrict__ out,
                    int c_out, const double* __restrict__ xt, double* __restrict__ vcorr,
                    const int2* __restrict__ work, const int* __restrict__ act) {
  constexpr int kR = K == 3 ? 1 : 2;
  const int2 wk = work[blockIdx.x];
  if (masked(act, wk.x)) return;
  const BPar pr = v.par[wk.x];
  const BLev<T> F = lev_of(v, wk.x, pr.L + kR), L = lev_of(v, wk.x, pr.L);
  const int n = wk.y * kNB + threadIdx.x;
  if (n >= F.g.nn) return;
  scatter_node<K>(L.g, F.g, cell_patch + pr.coff, out, c_out, xt + F.off, vcorr + F.off,
                  n % F.g.nnx, n / F.g.nnx);
}

template <typename T, int TCX, int TCY>
void pass_launch(const BView<T>& v, int k, int colour, int in, int out, const T* topb, T* topx,
                 T omega, Work w, const int* act, cudaStream_t st) {
  const size_t smem = sizeof(PassSmem<T, TCX, TCY>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(bpass_kernel<T, TCX, TCY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  note_launch();
  bpass_kernel<T, TCX, TCY><<<w.n, 4 * TCX * TCY, smem, st>>>(v, k, colour, in, out, topb, topx,
                                                              omega, w.d, act);
}

inline int vblocks(const VecTab& vt) { return vt.nblk; }

}  // namespace

void pass_shape_dims(int s, int* tcx, int* tcy) {
  switch (s) {
    case 1: *tcx = 8, *tcy = 4; break;
    case 2: *tcx = 8, *tcy = 8; break;
    default: *tcx = 16, *tcy = 4; break;
  }
}

template <typename T>
void bk_pass(const BView<T>& v, int k, int colour, int in, int out, const T* topb, T* topx,
             T omega, Work w, int shape, const int* act, cudaStream_t st) {
  if (w.n <= 0) return;
  switch (shape) {
    case 1: pass_launch<T, 8, 4>(v, k, colour, in, out, topb, topx, omega, w, act, st); break;
    case 2: pass_launch<T, 8, 8>(v, k, colour, in, out, topb, topx, omega, w, act, st); break;
    default: pass_launch<T, 16, 4>(v, k, colour, in, out, topb, topx, omega, w, act, st); break;
  }
}

#define NODE_LAUNCH(kernel, ...)                                  \
  do {                                                            \
    if (w.n <= 0) return;                                         \
    note_launch();                                                \
    kernel<<<w.n, kNB, 0, st>>>(__VA_ARGS__, w.d, act);           \
  } while (0)

template <typename T>
void bk_defect(const BView<T>& v, int k, int in, const T* topb, T* topx, Work w, const int* act,
               cudaStream_t st) {
  NODE_LAUNCH(bdefect_kernel<T>, v, k, in, topb, topx);
}

template <typename T>
void bk_restrict(const BView<T>& v, int k, Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(brestrict_kernel<T>, v, k);
}

template <typename T>
void bk_prolong(const BView<T>& v, int k, int in, T* topx, Work w, const int* act,
                cudaStream_t st) {
  NODE_LAUNCH(bprolong_kernel<T>, v, k, in, topx);
}

template <typename T>
void bk_coarse_solve(const BView<T>& v, int nprob, int n1, const double* Ainv, long long astride,
                     const T* topb, T* topx, const int* act, cudaStream_t st) {
  note_launch();
  bcoarse_solve_kernel<T><<<dim3(cdiv(n1, kSolveWarps), nprob), 32 * kSolveWarps,
                            sizeof(double) * n1, st>>>(v, Ainv, astride, topb, topx, act);
}

template <typename T>
void bk_apply(const BView<T>& v, const T* wv, const T* vbJ, T* y, Work w, const int* act,
              cudaStream_t st) {
  NODE_LAUNCH(bapply_kernel<T>, v, wv, vbJ, y);
}

template <typename T>
void bk_defect_top(const BView<T>& v, const T* b, const T* x, const T* vbJ, T* d, Work w,
                   const int* act, cudaStream_t st) {
  NODE_LAUNCH(bdefect_top_kernel<T>, v, b, x, vbJ, d);
}

template <typename T>
void bk_residual64(const BView<T>& v, int dl, const double* x, const double* f, double* r,
                   Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(bresidual64_kernel<T>, v, dl, x, f, r);
}

template <typename T>
void bk_old_rhs(const BView<T>& v, int dl, const double* xo, double* f, Work w, const int* act,
                cudaStream_t st) {
  NODE_LAUNCH(bold_rhs_kernel<T>, v, dl, xo, f);
}

template <typename T>
void bk_copy_impose(const BView<T>& v, int dl, const double* src, double* dst, Work w,
                    const int* act, cudaStream_t st) {
  NODE_LAUNCH(bcopy_impose_kernel<T>, v, dl, src, dst);
}

template <typename T>
void bk_top_vb(const BView<T>& v, const double* x64, Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(btop_vb_kernel<T>, v, x64);
}

template <typename T>
void bk_inject_vb(const BView<T>& v, int k, Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(binject_vb_kernel<T>, v, k);
}

template <typename T>
void bk_cast_vb(const BView<T>& v, int k, Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(bcast_vb_kernel<T>, v, k);
}

template <typename T>
void bk_setup(const BView<T>& v, int k, int* status, Work w, const int* act, cudaStream_t st) {
  if (w.n <= 0) return;
  note_launch();
  bsetup_kernel<T><<<w.n, kSetupThreads, 0, st>>>(v, k, status, w.d, act);
}

template <typename T>
void bk_coarse_factor(const BView<T>& v, int nprob, int n1, double* cwork, long long cstride,
                      long long bandsz, double* Ainv, long long astride, int* status,
                      const int* act, cudaStream_t st) {
  note_launch();
  bassemble_kernel<T><<<dim3(cdiv(n1, 128), nprob), 128, 0, st>>>(v, cwork, cstride, act);
  const int W = (int)(bandsz / n1);
  const size_t win_bytes = sizeof(double) * kWin * W;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(blu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)win_bytes);
    attr = true;
  }
  note_launch();
  blu_kernel<T><<<nprob, kLUThreads, win_bytes, st>>>(v, cwork, cstride, bandsz, status, act);
  note_launch();
  brecip_kernel<T><<<dim3(cdiv(n1, 128), nprob), 128, 0, st>>>(v, cwork, cstride, bandsz, act);
  const size_t ism = sizeof(double) * inv_block_smem_doubles(n1);
  static const bool inv_attr =
      cudaFuncSetAttribute(binverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ism) == cudaSuccess;
  (void)inv_attr;
  note_launch();
  binverse_kernel<T><<<dim3(cdiv(n1, kInvWarps), nprob), 32 * kInvWarps, ism, st>>>(
      v, cwork, cstride, bandsz, Ainv, astride, act);
}

template <typename T>
void bk_multidot(const T* V, size_t ld, int nv, const T* wv, double* part, const VecTab& vt,
                 double* out, int ostride, const int* act, cudaStream_t st) {
  note_launch();
  bmultidot_kernel<T><<<vblocks(vt), kVT, 0, st>>>(V, ld, nv, wv, part, vt.nblk, vt.inst, act);
  note_launch();
  bdots_finish_kernel<<<dim3(vt.nprob, nv), kVT, 0, st>>>(part, vt.nblk, vt.first, vt.count, out,
                                                          ostride, act);
}

template <typename T>
void bk_multiaxpy(const T* V, size_t ld, int nv, const double* h, int hstride, T* wv,
                  const VecTab& vt, const int* act, cudaStream_t st) {
  note_launch();
  bmultiaxpy_kernel<T><<<vblocks(vt), kVT, 0, st>>>(V, ld, nv, h, hstride, wv, vt.inst, act);
}

template <typename T>
void bk_scale(const T* x, const double* a, int astride, int mode, T* y, const VecTab& vt,
              const int* act, cudaStream_t st) {
  note_launch();
  bscale_kernel<T><<<vblocks(vt), kVT, 0, st>>>(x, a, astride, mode, y, vt.inst, act);
}

template <typename T>
void bk_start(const T* r, const double* nrm2, int nstride, T* v0, double* gv, int gstride,
              const VecTab& vt, const int* act, cudaStream_t st) {
  note_launch();
  bstart_kernel<T><<<vblocks(vt), kVT, 0, st>>>(r, nrm2, nstride, v0, gv, gstride, vt.inst,
                                                vt.first, act);
}

template <typename T, typename Tx>
void bk_combine(const T* Z, size_t ld, const int* kcnt, const double* y, int ystride, double eps,
                Tx* x, const VecTab& vt, const int* act, cudaStream_t st) {
  note_launch();
  bcombine_kernel<T, Tx><<<vblocks(vt), kVT, 0, st>>>(Z, ld, kcnt, y, ystride, eps, x, vt.inst,
                                                      act);
}

void bk_copy(const double* src, double* dst, const VecTab& vt, const int* act, cudaStream_t st) {
  note_launch();
  bcopy_kernel<<<vblocks(vt), kVT, 0, st>>>(src, dst, vt.inst, act);
}

void bk_givens(int nprob, int m, double* H, double* cs, double* sn, double* gv,
               const double* hcol, int j, double* resid, const double* target, int* kcnt,
               int* its, int maxit, int* gact, cudaStream_t st) {
  note_launch();
  bgivens_kernel<<<cdiv(nprob, 64), 64, 0, st>>>(nprob, m, H, cs, sn, gv, hcol, j, resid, target,
                                                 kcnt, its, maxit, gact);
}

void bk_backsolve(int nprob, int m, const double* H, const double* gv, const int* kcnt, double* y,
                  const int* act, cudaStream_t st) {
  note_launch();
  bbacksolve_kernel<<<cdiv(nprob, 64), 64, 0, st>>>(nprob, m, H, gv, kcnt, y, act);
}

template <typename T>
void bk_prolong_state(const BView<T>& v, const double* xc, double* xf, int ncomp, int zero_p,
                      int dlf, Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(bprolong_state_kernel<T>, v, xc, xf, ncomp, zero_p, dlf);
}

template <typename T>
void bk_restrict_full(const BView<T>& v, const double* bf, double* bc, int ncomp, int dlf,
                      Work w, const int* act, cudaStream_t st) {
  NODE_LAUNCH(brestrict_full_kernel<T>, v, bf, bc, ncomp, dlf);
}

template <typename T>
void bk_gather(const BView<T>& v, int K, int P, const int* pinst, const int* pcell,
               const double* xt, const double* r, const float* mean, const float* stdv,
               uint16_t* X, cudaStream_t st) {
  if (P <= 0) return;
  note_launch();
  if (K == 5)
    bgather_kernel<T, 5><<<cdiv(P, 128), 128, 0, st>>>(v, P, pinst, pcell, xt, r, mean, stdv, X);
  else
    bgather_kernel<T, 3><<<cdiv(P, 128), 128, 0, st>>>(v, P, pinst, pcell, xt, r, mean, stdv, X);
}

template <typename T>
void bk_scatter(const BView<T>& v, int K, const int* cell_patch, const float* out, int c_out,
                const double* xt, double* vcorr, Work w, const int* act, cudaStream_t st) {
  if (K == 5) {
    NODE_LAUNCH((bscatter_kernel<T, 5>), v, cell_patch, out, c_out, xt, vcorr);
  } else {
    NODE_LAUNCH((bscatter_kernel<T, 3>), v, cell_patch, out, c_out, xt, vcorr);
  }
}

#undef NODE_LAUNCH

#define BK_INST(T)                                                                              \
  template void bk_pass<T>(const BView<T>&, int, int, int, int, const T*, T*, T, Work, int,     \
                           const int*, cudaStream_t);                                           \
  template void bk_defect<T>(const BView<T>&, int, int, const T*, T*, Work, const int*,         \
                             cudaStream_t);                                                     \
  template void bk_restrict<T>(const BView<T>&, int, Work, const int*, cudaStream_t);           \
  template void bk_prolong<T>(const BView<T>&, int, int, T*, Work, const int*, cudaStream_t);   \
  template void bk_coarse_solve<T>(const BView<T>&, int, int, const double*, long long,         \
                                   const T*, T*, const int*, cudaStream_t);                     \
  template void bk_apply<T>(const BView<T>&, const T*, const T*, T*, Work, const int*,          \
                            cudaStream_t);                                                      \
  template void bk_defect_top<T>(const BView<T>&, const T*, const T*, const T*, T*, Work,       \
                                 const int*, cudaStream_t);                                     \
  template void bk_residual64<T>(const BView<T>&, int, const double*, const double*, double*,   \
                                 Work, const int*, cudaStream_t);                               \
  template void bk_old_rhs<T>(const BView<T>&, int, const double*, double*, Work, const int*,   \
                              cudaStream_t);                                                    \
  template void bk_copy_impose<T>(const BView<T>&, int, const double*, double*, Work,           \
                                  const int*, cudaStream_t);                                    \
  template void bk_top_vb<T>(const BView<T>&, const double*, Work, const int*, cudaStream_t);   \
  template void bk_inject_vb<T>(const BView<T>&, int, Work, const int*, cudaStream_t);          \
  template void bk_cast_vb<T>(const BView<T>&, int, Work, const int*, cudaStream_t);            \
  template void bk_setup<T>(const BView<T>&, int, int*, Work, const int*, cudaStream_t);        \
  template void bk_coarse_factor<T>(const BView<T>&, int, int, double*, long long, long long,   \
                                    double*, long long, int*, const int*, cudaStream_t);        \
  template void bk_multidot<T>(const T*, size_t, int, const T*, double*, const VecTab&,         \
                               double*, int, const int*, cudaStream_t);                         \
  template void bk_multiaxpy<T>(const T*, size_t, int, const double*, int, T*, const VecTab&,   \
                                const int*, cudaStream_t);                                      \
  template void bk_scale<T>(const T*, const double*, int, int, T*, const VecTab&, const int*,   \
                            cudaStream_t);                                                      \
  template void bk_start<T>(const T*, const double*, int, T*, double*, int, const VecTab&,       \
                            const int*, cudaStream_t);                                          \
  template void bk_combine<T, T>(const T*, size_t, const int*, const double*, int, double, T*,  \
                                 const VecTab&, const int*, cudaStream_t);                      \
  template void bk_prolong_state<T>(const BView<T>&, const double*, double*, int, int, int,    \
                                    Work, const int*, cudaStream_t);                            \
  template void bk_restrict_full<T>(const BView<T>&, const double*, double*, int, int, Work,    \
                                    const int*, cudaStream_t);                                  \
  template void bk_gather<T>(const BView<T>&, int, int, const int*, const int*, const double*,  \
                             const double*, const float*, const float*, uint16_t*,              \
                             cudaStream_t);                                                     \
  template void bk_scatter<T>(const BView<T>&, int, const int*, const float*, int,              \
                              const double*, double*, Work, const int*, cudaStream_t);
BK_INST(float)
BK_INST(double)
#undef BK_INST
template void bk_combine<float, double>(const float*, size_t, const int*, const double*, int,
                                        double, double*, const VecTab&, const int*,
                                        cudaStream_t);

}  // namespace dnnmg
