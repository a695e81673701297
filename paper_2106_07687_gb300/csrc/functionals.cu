// Functionals of a discrete solution (Sec. 3.4), FP64.
//
//  * J_div = int_Omega |div v|^2 dx over the fluid cells (2x2 Gauss).
//  * Drag and lift on the obstacle, J_e = -int_Gamma (nu grad v - p I) n . e ds
//    with n pointing into the obstacle, in residual (volume) form: minus the
//    backward-Euler momentum rows (1/k) M (v - v_old) + nu K v + N(v) v
//    - (p, div phi) summed over the nodes of Gamma (the velocity-Dirichlet
//    nodes strictly inside the channel; only those touching a fluid cell get
//    a contribution).  Without v_old the time term is left out.
//  * Relative l2 errors of velocity and pressure against a reference.
//
// One pass over the cells with per-block partial sums, then one block sums
// the partials; both in a fixed order, so repeated calls agree bit for bit.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "krylov_body.cuh"

namespace dnnmg {
namespace {

constexpr int kFnThreads = 256;

__global__ void __launch_bounds__(kFnThreads)
    functionals_kernel(const Grid g, const FnConsts c, const double* __restrict__ x,
                       const double* __restrict__ xo, double* __restrict__ part) {
  __shared__ double sh[32];
  const int nn = g.nn;
  const double wg = 0.25 * g.h * g.h, ih = 1.0 / g.h;
  double jdiv = 0.0, fx = 0.0, fy = 0.0;
  const int ncell = g.nx * g.ny;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
       cell += gridDim.x * blockDim.x) {
    if (g.solid[cell]) continue;
    const int ci = cell % g.nx, cj = cell / g.nx;
    double wu[4], wv[4], wp[4];
    bool gam[4], any = false;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ci + (a & 1), j = cj + (a >> 1), n = j * g.nnx + i;
      wu[a] = x[n];
      wv[a] = x[nn + n];
      wp[a] = x[2 * nn + n];
      gam[a] = (g.flags[n] & kVDir) && i > 0 && i < g.nx && j > 0 && j < g.ny;
      any |= gam[a];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double phi[4], dx[4], dy[4];
      shape_at<double>(q, phi, dx, dy);
      double div = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) div += dx[b] * wu[b] + dy[b] * wv[b];
      div *= ih;
      jdiv += wg * div * div;
    }
    if (!any) continue;
    double r[12];
    cell_all_rows<double, true>(c.s, wu, wv, wp, wu, wv, r);
    double ou[4], ov[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int n = (cj + (a >> 1)) * g.nnx + ci + (a & 1);
      ou[a] = xo ? xo[n] : wu[a];
      ov[a] = xo ? xo[nn + n] : wv[a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!gam[a]) continue;
      double mu = 0.0, mv = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        mu += c.mk[a * 4 + b] * ou[b];
        mv += c.mk[a * 4 + b] * ov[b];
      }
      fx -= r[a] - mu;
      fy -= r[4 + a] - mv;
    }
  }
  jdiv = block_sum(jdiv, sh);
  fx = block_sum(fx, sh);
  fy = block_sum(fy, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = jdiv;
    part[3 * blockIdx.x + 1] = fx;
    part[3 * blockIdx.x + 2] = fy;
  }
}

__global__ void __launch_bounds__(kFnThreads)
    rel_err_kernel(int nn, const double* __restrict__ x, const double* __restrict__ xr,
                   double* __restrict__ part) {
  __shared__ double sh[32];
  double ev = 0.0, rv = 0.0, ep = 0.0, rp = 0.0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
    const double du = x[n] - xr[n], dv = x[nn + n] - xr[nn + n];
    const double dp = x[2 * nn + n] - xr[2 * nn + n];
    ev += du * du + dv * dv;
    rv += xr[n] * xr[n] + xr[nn + n] * xr[nn + n];
    ep += dp * dp;
    rp += xr[2 * nn + n] * xr[2 * nn + n];
  }
  ev = block_sum(ev, sh);
  rv = block_sum(rv, sh);
  ep = block_sum(ep, sh);
  rp = block_sum(rp, sh);
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x + 0] = ev;
    part[4 * blockIdx.x + 1] = rv;
    part[4 * blockIdx.x + 2] = ep;
    part[4 * blockIdx.x + 3] = rp;
  }
}

// out[k] = sum over blocks b of part[b * nval + k], k < nval <= 4
__global__ void __launch_bounds__(kFnThreads)
    partial_sum_kernel(const double* __restrict__ part, int nblocks, int nval,
                       double* __restrict__ out) {
  __shared__ double sh[32];
  for (int k = 0; k < nval; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += part[b * nval + k];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[k] = v;
  }
}

int fn_blocks(long long work) {
  const long long nb = (work + kFnThreads - 1) / kFnThreads;
  return (int)std::max<long long>(1, std::min<long long>(kFnBlocks, nb));
}

}  // namespace

void launch_functionals(const Grid& g, const FnConsts& c, const double* x, const double* x_old,
                        double* part, double* out, cudaStream_t st) {
  const int nb = fn_blocks((long long)g.nx * g.ny);
  functionals_kernel<<<nb, kFnThreads, 0, st>>>(g, c, x, x_old, part);
  partial_sum_kernel<<<1, kFnThreads, 0, st>>>(part, nb, 3, out);
  note_launches(2);
}

void launch_rel_errors(const Grid& g, const double* x, const double* x_ref, double* part,
                       double* out, cudaStream_t st) {
  const int nb = fn_blocks(g.nn);
  rel_err_kernel<<<nb, kFnThreads, 0, st>>>(g.nn, x, x_ref, part);
  partial_sum_kernel<<<1, kFnThreads, 0, st>>>(part, nb, 4, out);
  note_launches(2);
}

}  // namespace dnnmg
