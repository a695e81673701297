// Host runtime and C ABI of libdnnmg: level hierarchy, stencil constants,
// V-cycle, flexible GMRES and Newton orchestration (Sec. 2.2, Algorithm 1).
// All arithmetic of the method runs in the kernels of this library; the host
// code only sequences launches and reads back convergence scalars.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dnnmg.h"
#include "kernels.h"
#include "dnnmg_step.h"
#include "coarse_body.cuh"
#include "runtime.h"

using namespace dnnmg;

namespace dnnmg {

// ---------------------------------------------------------------------------
// Geometry of one level (host side), Sec. 2.1 / Eq. 2 with the channel
// reading: obstacle = square of 2x2 level-0 cells whose lower-left corner
// is the corner of cell (oi0, oj0) of level olev (0 or 1; on level 1 it is
// 4x4 cells), no-slip on walls and on every node of a solid cell, parabolic
// inflow at x = 0, do-nothing at x = 4.  A cell of a level coarser than olev
// is solid when all its descendants on level olev are.
HostLevel make_level(int ell, int oi0, int oj0, int olev) {
  HostLevel L;
  L.ell = ell;
  Grid& g = L.g;
  g.nx = 16 << ell;
  g.ny = 4 << ell;
  g.nnx = g.nx + 1;
  g.nny = g.ny + 1;
  g.nn = g.nnx * g.nny;
  g.h = 4.0 / g.nx;
  L.solid.assign((size_t)g.nx * g.ny, 0);
  if (oi0 >= 0)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const int B = 2 << olev;  // the block's width in level-olev cells
        bool in;
        if (ell >= olev) {
          const int I = i >> (ell - olev), J = j >> (ell - olev);
          in = I >= oi0 && I < oi0 + B && J >= oj0 && J < oj0 + B;
        } else {  // the cell's descendants on level olev: [i s, (i + 1) s)
          const int sc = 1 << (olev - ell);
          in = i * sc >= oi0 && (i + 1) * sc <= oi0 + B && j * sc >= oj0 && (j + 1) * sc <= oj0 + B;
        }
        if (in) L.solid[(size_t)j * g.nx + i] = 1;
      }
  L.flags.assign(g.nn, 0);
  for (int j = 0; j <= g.ny; ++j)
    for (int i = 0; i <= g.nx; ++i) {
      bool touch_solid = false, touch_fluid = false;
      for (int cy = -1; cy <= 0; ++cy)
        for (int cx = -1; cx <= 0; ++cx) {
          const int ci = i + cx, cj = j + cy;
          if (ci < 0 || cj < 0 || ci >= g.nx || cj >= g.ny) continue;
          if (L.solid[(size_t)cj * g.nx + ci])
            touch_solid = true;
          else
            touch_fluid = true;
        }
      uint8_t f = 0;
      if (touch_solid || i == 0 || j == 0 || j == g.ny) f |= kVDir;
      if (!touch_fluid) f |= kPFix;
      L.flags[(size_t)j * g.nnx + i] = f;
    }
  return L;
}

// Q1 element constants from 1D tensor products on a cell of width h:
// 1D mass h/6 [2 1; 1 2], 1D stiffness 1/h [1 -1; -1 1],
// 1D int phi_i phi_j' = [-1/2 1/2; -1/2 1/2].
template <typename T>
Sten<T> make_sten(double h, const dnnmg_config& c) {
  const double m1[2][2] = {{h / 3, h / 6}, {h / 6, h / 3}};
  const double k1[2][2] = {{1 / h, -1 / h}, {-1 / h, 1 / h}};
  const double c1[2][2] = {{-0.5, 0.5}, {-0.5, 0.5}};
  double M[4][4], K[4][4], Dx[4][4], Dy[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int ax = a & 1, ay = a >> 1, bx = b & 1, by = b >> 1;
      M[a][b] = m1[ax][bx] * m1[ay][by];
      K[a][b] = k1[ax][bx] * m1[ay][by] + m1[ax][bx] * k1[ay][by];
      Dx[a][b] = c1[ax][bx] * m1[ay][by];
      Dy[a][b] = m1[ax][bx] * c1[ay][by];
    }
  Sten<T> s;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      s.E[a * 4 + b] = (T)(M[a][b] / c.dt + c.theta * c.nu * K[a][b]);
      s.Dx[a * 4 + b] = (T)Dx[a][b];
      s.Dy[a * 4 + b] = (T)Dy[a][b];
    }
  // LPS on a 2x2-cell patch: S9 = alpha kappa^T K9 kappa, kappa = I - Pi,
  // Pi = bilinear interpolation from the patch corners.
  double K9[9][9] = {};
  for (int cy = 0; cy < 2; ++cy)
    for (int cx = 0; cx < 2; ++cx)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          const int ma = (cx + (a & 1)) + 3 * (cy + (a >> 1));
          const int mb = (cx + (b & 1)) + 3 * (cy + (b >> 1));
          K9[ma][mb] += K[a][b];
        }
  double kap[9][9] = {};
  for (int m = 0; m < 9; ++m) {
    const int sx = m % 3, sy = m / 3;
    kap[m][m] += 1.0;
    for (int cy = 0; cy <= 2; cy += 2)
      for (int cx = 0; cx <= 2; cx += 2) {
        const double w = (1.0 - std::abs(sx - cx) / 2.0) * (1.0 - std::abs(sy - cy) / 2.0);
        kap[m][cx + 3 * cy] -= w;
      }
  }
  const double alpha = c.alpha0 * h * h / c.nu;
  for (int m = 0; m < 9; ++m)
    for (int n = 0; n < 9; ++n) {
      double acc = 0;
      for (int p = 0; p < 9; ++p)
        for (int q = 0; q < 9; ++q) acc += kap[p][m] * K9[p][q] * kap[q][n];
      s.S9[m * 9 + n] = (T)(alpha * acc);
    }
  // Cellwise forms.  Each fluid cell lies in exactly one patch and patches
  // are all fluid or all solid on every multigrid level, so a patch matrix
  // that is the sum of its four cells' blocks gives the cellwise operator.
  if (c.lps_mode == 1) {
    // projection onto cellwise constants: grad pi p = 0, S = alpha K
    for (int m = 0; m < 9; ++m)
      for (int n = 0; n < 9; ++n) s.S9[m * 9 + n] = (T)(alpha * K9[m][n]);
  } else if (c.lps_mode == 2) {
    // projection of the gradient onto its cell mean: on a square Q1 cell
    // the rest is alpha / 6 times the outer product of the bilinear mode
    // c = (1, -1, -1, 1)
    double S9c[9][9] = {};
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            const double ca = ((a & 1) == (a >> 1)) ? 1.0 : -1.0;
            const double cb = ((b & 1) == (b >> 1)) ? 1.0 : -1.0;
            const int ma = (cx + (a & 1)) + 3 * (cy + (a >> 1));
            const int mb = (cx + (b & 1)) + 3 * (cy + (b >> 1));
            S9c[ma][mb] += alpha / 6.0 * ca * cb;
          }
    for (int m = 0; m < 9; ++m)
      for (int n = 0; n < 9; ++n) s.S9[m * 9 + n] = (T)S9c[m][n];
  }
  s.wq = (T)(c.theta * h * h / 4.0);
  s.ih = (T)(1.0 / h);
  return s;
}

// The stabilisation of each cell of a 2h patch on the patch's 3x3 nodes
// (the summands of S9 above, cell c = cx + 2 cy): a part-solid patch sums the
// pieces of its fluid cells (its integral runs over those cells only).
PatchPieces make_patch_pieces(double h, const dnnmg_config& c) {
  const double m1[2][2] = {{h / 3, h / 6}, {h / 6, h / 3}};
  const double k1[2][2] = {{1 / h, -1 / h}, {-1 / h, 1 / h}};
  double K[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int ax = a & 1, ay = a >> 1, bx = b & 1, by = b >> 1;
      K[a][b] = k1[ax][bx] * m1[ay][by] + m1[ax][bx] * k1[ay][by];
    }
  double kap[9][9] = {};
  for (int m = 0; m < 9; ++m) {
    const int sx = m % 3, sy = m / 3;
    kap[m][m] += 1.0;
    for (int cy = 0; cy <= 2; cy += 2)
      for (int cx = 0; cx <= 2; cx += 2)
        kap[m][cx + 3 * cy] -= (1.0 - std::abs(sx - cx) / 2.0) * (1.0 - std::abs(sy - cy) / 2.0);
  }
  const double alpha = c.alpha0 * h * h / c.nu;
  PatchPieces pp{};
  for (int cc = 0; cc < 4; ++cc) {
    const int cx = cc & 1, cy = cc >> 1;
    double Kc[9][9] = {}, Mc[9][9] = {};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const int ma = (cx + (a & 1)) + 3 * (cy + (a >> 1));
        const int mb = (cx + (b & 1)) + 3 * (cy + (b >> 1));
        Kc[ma][mb] += K[a][b];
        const double ca = ((a & 1) == (a >> 1)) ? 1.0 : -1.0;
        const double cb = ((b & 1) == (b >> 1)) ? 1.0 : -1.0;
        Mc[ma][mb] += alpha / 6.0 * ca * cb;
      }
    for (int m = 0; m < 9; ++m)
      for (int n = 0; n < 9; ++n) {
        double v;
        if (c.lps_mode == 1) {
          v = alpha * Kc[m][n];
        } else if (c.lps_mode == 2) {
          v = Mc[m][n];
        } else {
          double acc = 0;
          for (int p = 0; p < 9; ++p)
            for (int q = 0; q < 9; ++q) acc += kap[p][m] * Kc[p][q] * kap[q][n];
          v = alpha * acc;
        }
        pp.S[cc][m * 9 + n] = v;
      }
  }
  return pp;
}

bool part_solid_patches(const HostLevel& L) {
  const Grid& g = L.g;
  for (int J = 0; J < g.ny / 2; ++J)
    for (int I = 0; I < g.nx / 2; ++I) {
      const size_t c = (size_t)(2 * J) * g.nx + 2 * I;
      const int n = L.solid[c] + L.solid[c + 1] + L.solid[c + g.nx] + L.solid[c + g.nx + 1];
      if (n != 0 && n != 4) return true;
    }
  return false;
}

// Constants of the explicit old-time bracket nu (grad v, grad phi) + (v.grad v, phi)
// of the theta-scheme: E = nu K, no mass, no pressure, no LPS, Gauss weight h^2/4.
Sten<double> make_explicit_sten(double h, const dnnmg_config& c) {
  dnnmg_config e = c;
  e.theta = 1.0;
  Sten<double> s = make_sten<double>(h, e);
  const double k1[2][2] = {{1 / h, -1 / h}, {-1 / h, 1 / h}};
  const double m1[2][2] = {{h / 3, h / 6}, {h / 6, h / 3}};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int ax = a & 1, ay = a >> 1, bx = b & 1, by = b >> 1;
      s.E[a * 4 + b] = c.nu * (k1[ax][bx] * m1[ay][by] + m1[ax][bx] * k1[ay][by]);
      s.Dx[a * 4 + b] = s.Dy[a * 4 + b] = 0.0;
    }
  for (int m = 0; m < 81; ++m) s.S9[m] = 0.0;
  s.wq = h * h / 4.0;
  return s;
}

template Sten<float> make_sten<float>(double, const dnnmg_config&);
template Sten<double> make_sten<double>(double, const dnnmg_config&);

}  // namespace dnnmg

// ---------------------------------------------------------------------------
// C ABI

namespace {
thread_local std::string g_setup_error;  // message of this thread's last context-free failure
}

namespace dnnmg {
void set_thread_error(const char* msg) { g_setup_error = msg; }
}

extern "C" {

int dnnmg_default_config(dnnmg_config* c) {
  if (!c) return DNNMG_ERR_ARG;
  std::memset(c, 0, sizeof(*c));
  c->nu = 0.01;
  c->dt = 0.01;
  c->theta = 1.0;
  c->alpha0 = 0.1;
  c->newton_tol = 1e-10;
  c->gmres_rtol = 1e-4;
  c->omega = 0.8;
  c->eps_damp = 1.0;
  c->obstacle_i0 = 2;
  c->obstacle_j0 = 1;
  c->level_solve = 3;
  c->level_coarse = 1;
  c->replaced_levels = 1;
  c->precision = DNNMG_FP64;
  c->newton_max = 20;
  c->gmres_m = 20;
  c->gmres_maxit = 200;
  c->nu1 = 2;
  c->nu2 = 2;
  c->hidden = 64;
  c->gru_layers = 2;
  c->mlp_width = 128;
  c->fallback_newton_its = 8;
  c->coarse_refresh = 32;
  c->persistent_vcycle = -1;
  c->precond_lag = 1;
  c->persistent_mode = -1;
  c->stream_pass = 0;
  c->net_bias = 1;
  c->net_inputs = 0;
  c->obstacle_level = 0;
  return DNNMG_OK;
}

int dnnmg_setup(const dnnmg_config* cfg, void* stream, dnnmg_ctx** out) {
  if (!out) return DNNMG_ERR_ARG;
  *out = nullptr;
  if (!cfg) return DNNMG_ERR_ARG;
  std::unique_ptr<dnnmg_ctx> ctx(new dnnmg_ctx());
  ctx->cfg = *cfg;
  ctx->st = (cudaStream_t)stream;
  int rc = ctx->init();
  if (rc != DNNMG_OK) {
    g_setup_error = ctx->err;
    return rc;
  }
  g_setup_error.clear();
  *out = ctx.release();
  return DNNMG_OK;
}

int dnnmg_destroy(dnnmg_ctx* ctx) {
  delete ctx;
  return DNNMG_OK;
}

const char* dnnmg_last_error(const dnnmg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_error.c_str();
}

int dnnmg_level_dims(const dnnmg_ctx* ctx, int level, int* nx, int* ny) {
  if (!ctx || !nx || !ny || level < 0 || level >= (int)ctx->lv.size()) return DNNMG_ERR_ARG;
  *nx = ctx->lv[level].g.nx;
  *ny = ctx->lv[level].g.ny;
  return DNNMG_OK;
}

int dnnmg_get_state(dnnmg_ctx* ctx, double* x) {
  if (!ctx || !x) return DNNMG_ERR_ARG;
  return ctx->get_state(x);
}

int dnnmg_set_state(dnnmg_ctx* ctx, const double* x) {
  if (!ctx || !x) return DNNMG_ERR_ARG;
  return ctx->set_state(x);
}

int dnnmg_linearize(dnnmg_ctx* ctx, const double* x) {
  if (!ctx || !x) return DNNMG_ERR_ARG;
  return ctx->linearize_api(x);
}

int dnnmg_apply(dnnmg_ctx* ctx, int level, const void* w, void* y, int precision) {
  if (!ctx || !w || !y) return DNNMG_ERR_ARG;
  return ctx->apply_api(level, w, y, precision);
}

int dnnmg_vcycle(dnnmg_ctx* ctx, int level, const void* b, void* x, int precision) {
  if (!ctx || !b || !x) return DNNMG_ERR_ARG;
  return ctx->vcycle_api(level, b, x, precision);
}

int dnnmg_residual(dnnmg_ctx* ctx, const double* x, const double* f, double* r) {
  if (!ctx || !x || !f || !r) return DNNMG_ERR_ARG;
  return ctx->residual_api(x, f, r);
}

int dnnmg_step(dnnmg_ctx* ctx, int mode, dnnmg_step_stats* stats) {
  if (!ctx) return DNNMG_ERR_ARG;
  if (mode != DNNMG_PLAIN && mode != DNNMG_NET) return ctx->fail(DNNMG_ERR_ARG, "unknown mode");
  return ctx->step(mode, stats);
}

int dnnmg_step_io(dnnmg_ctx* ctx, int mode, const double* x_in, double* x_out,
                  dnnmg_step_stats* stats) {
  if (!ctx) return DNNMG_ERR_ARG;
  if (mode != DNNMG_PLAIN && mode != DNNMG_NET) return ctx->fail(DNNMG_ERR_ARG, "unknown mode");
  const size_t bytes = 3 * sizeof(double) * ctx->grid(ctx->L()).nn;
  if (x_in) {
    cudaMemcpyAsync(ctx->x64, x_in, bytes, cudaMemcpyHostToDevice, ctx->st);
    dnnmg::launch_impose_dirichlet64(ctx->grid(ctx->L()), ctx->x64, ctx->st);
  }
  int rc = ctx->step(mode, stats);
  if (x_out && (rc == DNNMG_OK || rc == DNNMG_ERR_NOT_CONVERGED)) {
    cudaMemcpyAsync(x_out, ctx->x64, bytes, cudaMemcpyDeviceToHost, ctx->st);
    if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return ctx->check("step_io");
  }
  return rc;
}

int dnnmg_prolongate(dnnmg_ctx* ctx, int level, const double* xc, double* xf) {
  if (!ctx || !xc || !xf) return DNNMG_ERR_ARG;
  if (level < 0 || level + 1 >= (int)ctx->lv.size())
    return ctx->fail(DNNMG_ERR_ARG, "level out of range");
  dnnmg::launch_prolong_state64(ctx->grid(level + 1), ctx->grid(level), xc, xf, 3, ctx->st);
  return ctx->check("prolongate");
}

int dnnmg_functionals(dnnmg_ctx* ctx, int level, const double* x, const double* x_old,
                      double* out) {
  if (!ctx || !x || !out) return DNNMG_ERR_ARG;
  if (level < 0 || level >= (int)ctx->lv.size())
    return ctx->fail(DNNMG_ERR_ARG, "level out of range");
  return ctx->functionals(level, x, x_old, out);
}

int dnnmg_relative_errors(dnnmg_ctx* ctx, int level, const double* x, const double* x_ref,
                          double* out) {
  if (!ctx || !x || !x_ref || !out) return DNNMG_ERR_ARG;
  if (level < 0 || level >= (int)ctx->lv.size())
    return ctx->fail(DNNMG_ERR_ARG, "level out of range");
  return ctx->rel_errors(level, x, x_ref, out);
}

int dnnmg_profile(dnnmg_ctx* ctx, int enable) {
  if (!ctx) return DNNMG_ERR_ARG;
  ctx->prof.enable(enable != 0);
  return DNNMG_OK;
}

int dnnmg_profile_read(dnnmg_ctx* ctx, int stage, int level, int64_t* launches, double* ms) {
  if (!ctx || stage < 0 || stage >= kStages || level < -1 || level >= kMaxLevels)
    return DNNMG_ERR_ARG;
  ctx->prof.collect(ctx->st);
  long long n = 0;
  double t = 0;
  for (int l = 0; l < kMaxLevels; ++l)
    if (level < 0 || l == level) {
      n += ctx->prof.count(stage, l);
      t += ctx->prof.ms(stage, l);
    }
  if (launches) *launches = n;
  if (ms) *ms = t;
  return DNNMG_OK;
}

uint64_t dnnmg_kernel_launches(void) { return dnnmg::launches(); }

int dnnmg_vcycle_split(const dnnmg_ctx* ctx) {
  return ctx && ctx->solver ? ctx->solver->split_level() : -1;
}

int dnnmg_vcycle_plan(const dnnmg_ctx* ctx, int level, int* split_level, int* split_mode,
                      int* pass_shape) {
  if (!ctx || !ctx->solver || !split_level || !split_mode || !pass_shape) return DNNMG_ERR_ARG;
  *split_level = ctx->solver->split_level();
  *split_mode = ctx->solver->split_mode();
  *pass_shape = ctx->solver->pass_shape(level);
  return DNNMG_OK;
}

size_t dnnmg_num_params(const dnnmg_ctx* ctx) { return ctx ? ctx->nd.num_params() : 0; }

int dnnmg_net_dims(const dnnmg_ctx* ctx, int* c_in, int* c_out) {
  if (!ctx || !c_in || !c_out) return DNNMG_ERR_ARG;
  *c_in = ctx->nd.c_in;
  *c_out = ctx->nd.c_out;
  return DNNMG_OK;
}

int dnnmg_set_weights(dnnmg_ctx* ctx, const float* w) {
  if (!ctx || !w) return DNNMG_ERR_ARG;
  return ctx->set_weights(w);
}

int dnnmg_get_weights(dnnmg_ctx* ctx, float* w) {
  if (!ctx || !w) return DNNMG_ERR_ARG;
  return ctx->get_weights(w);
}

int dnnmg_patch_infer(dnnmg_ctx* ctx, const uint16_t* x, float* h, float* out, int P) {
  if (!ctx || (P > 0 && (!x || !h || !out))) return DNNMG_ERR_ARG;
  return ctx->patch_infer(x, h, out, P);
}

int dnnmg_num_patches(const dnnmg_ctx* ctx) { return ctx ? ctx->P : 0; }

int dnnmg_set_feature_stats(dnnmg_ctx* ctx, const float* mean, const float* stdv) {
  if (!ctx || !mean || !stdv) return DNNMG_ERR_ARG;
  return ctx->set_feature_stats(mean, stdv);
}

int dnnmg_get_fine_velocity(dnnmg_ctx* ctx, double* v) {
  if (!ctx || !v) return DNNMG_ERR_ARG;
  return ctx->get_fine_velocity(v);
}

int dnnmg_get_patch_inputs(dnnmg_ctx* ctx, uint16_t* x) {
  if (!ctx || !x) return DNNMG_ERR_ARG;
  return ctx->get_patch_inputs(x);
}

int dnnmg_train_grad(dnnmg_ctx* ctx, const uint16_t* X, const float* Y, int B, int T, float* grad,
                     float* loss) {
  if (!ctx || !X || !Y) return DNNMG_ERR_ARG;
  return ctx->train_grad(X, Y, B, T, grad, loss);
}

int dnnmg_train_step(dnnmg_ctx* ctx, const uint16_t* X, const float* Y, int B, int T, float lr,
                     float* loss) {
  if (!ctx || !X || !Y || !(lr >= 0.0f)) return DNNMG_ERR_ARG;
  return ctx->train_step(X, Y, B, T, lr, loss);
}

int dnnmg_reset_optimizer(dnnmg_ctx* ctx) {
  if (!ctx) return DNNMG_ERR_ARG;
  return ctx->reset_optimizer();
}

int dnnmg_make_sample(dnnmg_ctx* ctx, const double* xf_prev, const double* xf_next, float* X,
                      float* Y, dnnmg_step_stats* stats) {
  if (!ctx || !xf_prev || !xf_next || !X || !Y) return DNNMG_ERR_ARG;
  return ctx->make_sample(xf_prev, xf_next, X, Y, stats);
}

int dnnmg_make_corpus(dnnmg_ctx* ctx, int n_traj, const double* nu, int spinup_steps,
                      double spinup_dt, int relax_steps, int T, float* X, float* Y) {
  if (!ctx || !nu || !X || !Y) return DNNMG_ERR_ARG;
  return ctx->make_corpus(n_traj, nu, spinup_steps, spinup_dt, relax_steps, T, X, Y);
}

int dnnmg_feature_stats(dnnmg_ctx* ctx, const float* X, int64_t rows, float* mean, float* stdv) {
  if (!ctx || !X) return DNNMG_ERR_ARG;
  return ctx->feature_stats(X, rows, mean, stdv);
}

int dnnmg_gather_batch(dnnmg_ctx* ctx, const float* X, const float* Y, const int* idx, int B,
                       int T, int64_t stride, uint16_t* Xb, float* Yb) {
  if (!ctx || !X || !Y || !idx || !Xb || !Yb) return DNNMG_ERR_ARG;
  return ctx->gather_batch(X, Y, idx, B, T, stride, Xb, Yb);
}

int dnnmg_gemm_bf16(dnnmg_ctx* ctx, const uint16_t* A, const uint16_t* B, float* C, int M, int N,
                    int K) {
  if (!ctx || !A || !B || !C) return DNNMG_ERR_ARG;
  if (!ctx->net_status) return ctx->fail(DNNMG_ERR_STATE, "no tensor-core status word");
  if (dnnmg::launch_umma_gemm(A, B, C, M, N, K, ctx->net_status, ctx->st))
    return ctx->fail(DNNMG_ERR_ARG, "gemm: need M % 128 == 0, 16 <= N <= 256, N % 16 == 0, K % 16 == 0");
  return ctx->net_check("gemm");
}

}  // extern "C"
