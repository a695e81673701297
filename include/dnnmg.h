/*
 * dnnmg.h - C ABI of the GB300 (sm_103a) DNN-MG hot path.
 *
 * The library advances the 2D incompressible Navier-Stokes equations
 * (Sec. 2.1, Eq. 1 with the boundary conditions of Eq. 2) in a channel
 * [0,4] x [0,1] with a block obstacle, discretised by Q1/Q1 finite elements
 * with local projection stabilisation (Eqs. 4-5) on a hierarchy of uniformly
 * refined meshes.  Each time step solves A_n(x_n) = f_n (Eq. 3) by Newton's
 * method (Eq. 6) whose linear systems are solved by flexible GMRES
 * preconditioned with one geometric multigrid V-cycle (Sec. 2.2, the Newton
 * iteration of Algorithm 1).  In DNN-MG mode a patch-wise recurrent network (stacked GRUs +
 * dense layers, Sec. 2.2 and Sec. 3.1) predicts a velocity correction on the
 * level(s) above the finest solved one, which enters the next step through
 * the restricted right-hand side (the network correction of Algorithm 1);
 * the network is trained with the loss of Eq. 7.
 *
 * Conventions
 *  - Every function returns a status code (DNNMG_OK = 0).  On failure the
 *    context keeps a message, read with dnnmg_last_error().  Nothing prints
 *    and nothing aborts.
 *  - The context owns all device memory it needs; it allocates it in
 *    dnnmg_setup() and frees it in dnnmg_destroy().  Apart from the calls that
 *    say otherwise, calls do not allocate.
 *  - Pointer arguments marked "device" are device pointers of the current
 *    CUDA device, borrowed for the duration of the call.  Work is issued on
 *    the stream given to dnnmg_setup(); functions that return results to the
 *    host synchronise that stream.
 *  - A field on mesh level l is stored as [3][ny+1][nx+1] (u, v, p; x index
 *    fastest) with nx = 16 * 2^l, ny = 4 * 2^l: node (i, j) of component c at
 *    c * (nx+1)(ny+1) + j * (nx+1) + i.  Velocity-only fields are [2][..].
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef DNNMG_H
#define DNNMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DNNMG_OK 0
#define DNNMG_ERR_ARG 1            /* invalid argument or configuration */
#define DNNMG_ERR_CUDA 2           /* a CUDA call failed */
#define DNNMG_ERR_NOT_CONVERGED 3  /* Newton hit its iteration cap; the step is still taken */
#define DNNMG_ERR_NUMERICAL 4      /* NaN/Inf or a singular local/coarse matrix */
#define DNNMG_ERR_TIMEOUT 5        /* a device loop hit its iteration cap */
#define DNNMG_ERR_STATE 6          /* call not valid in the context's current state */

/* precision modes */
#define DNNMG_FP64 0   /* everything in FP64 */
#define DNNMG_MIXED 1  /* V-cycle and GMRES in FP32 inside FP64 Newton (defect correction) */

/* time-step modes */
#define DNNMG_PLAIN 0  /* classical Newton-Krylov-multigrid step (Newton part of Algorithm 1) */
#define DNNMG_NET 1    /* DNN-MG step (Algorithm 1) */

typedef struct dnnmg_ctx dnnmg_ctx;

/* Configuration (plain old data).  Start from dnnmg_default_config(). */
typedef struct dnnmg_config {
  double nu;          /* kinematic viscosity, 1/Re (Eq. 1) */
  double dt;          /* time step k (Eq. 5) */
  double theta;       /* time scheme weight: 1 = backward Euler, 0.5 = Crank-Nicolson (Eq. 5) */
  double alpha0;      /* LPS parameter, alpha_T = alpha0 * Re * h_T^2 (Sec. 2.1) */
  double newton_tol;  /* stop when the l2 norm of f_n - A_n(x) over free DOFs <= newton_tol;
                         in DNNMG_MIXED the operator of that residual is evaluated in
                         double-float (about 48 bits): its rounding floor is about
                         1e-12 on the small channels, so smaller tolerances are
                         not reached there */
  double gmres_rtol;  /* relative residual reduction of FGMRES per Newton step */
  double omega;       /* damping of the Vanka update */
  double eps_damp;    /* Newton damping epsilon (the damped update of Algorithm 1) */
  int32_t obstacle_i0, obstacle_j0; /* lower-left cell, on level obstacle_level, of the
                                       solid square of 2x2 level-0 cells; -1 = none */
  int32_t level_solve;     /* finest level L solved by multigrid */
  int32_t level_coarse;    /* coarsest multigrid level (direct solve), >= 1 */
  int32_t replaced_levels; /* levels above L replaced by the network (1 or 2; 0 = none) */
  int32_t precision;       /* DNNMG_FP64 or DNNMG_MIXED */
  int32_t newton_max;      /* Newton iteration cap */
  int32_t gmres_m;         /* FGMRES restart length (<= 40) */
  int32_t gmres_maxit;     /* total FGMRES iteration cap per Newton step */
  int32_t nu1, nu2;        /* pre- and post-smoothing sweeps of the V(nu1, nu2) cycle */
  int32_t hidden;          /* GRU hidden size m: 32 or 64 (default 64) */
  int32_t gru_layers;      /* stacked GRU cells n: 1, 2 or 3 (default 2); m x n are
                              the sizes of Table 1 */
  int32_t mlp_width;       /* width of the hidden dense layer: 128 (default), or 0 for a
                              single dense layer m -> C_out after the GRUs (Table 1) */
  int32_t fallback_newton_its; /* DNN-MG step redone without the network if Newton needs more */
  int32_t train_batch;     /* largest training batch B (sequences) of dnnmg_train_*, 0 = none */
  int32_t train_seq;       /* largest training sequence length T */
  int32_t coarse_refresh;  /* time steps between refactorisations of the coarse level (>= 1) */
  int32_t persistent_vcycle; /* levels <= this one run their part of a V-cycle as one
                                persistent launch; 0: none; -1: chosen by timing */
  int32_t precond_lag;     /* 1: the multigrid preconditioner keeps the linearisation of a
                              step's first Newton iteration (the matvec is always current) */
  int32_t persistent_mode; /* that launch: 0 = cooperative grid, 1 = one thread-block
                              cluster, -1 = chosen by timing */
  int32_t lps_mode;        /* projection pi_h of the pressure stabilisation (Sec. 2.1):
                              0 = bilinear interpolation on the 2h patch mesh (default);
                              1 = onto cellwise constants, so s is alpha times the
                              pressure Laplacian (not consistent: O(alpha h) terms on
                              the boundary for linear p; slower V-cycle contraction);
                              2 = the gradient onto its cell mean, which penalises only
                              each cell's bilinear mode and leaves the line pressure
                              mode (-1)^i free: the Jacobian is singular and the solver
                              does not converge with it (operator, residual and
                              functionals only, for comparisons) */
  int32_t stream_pass;     /* FP32 colour passes of the levels outside the persistent
                              launch: 0 = the streaming kernel (inverses copied by TMA
                              one tile ahead) where the autotuner finds it faster
                              (default), 1 = always where it can run, -1 = never */
  int32_t net_bias;        /* 1: the GRUs and dense layers have biases (default); 0: none,
                              as the networks of Table 1 */
  int32_t net_inputs;      /* inputs C_in of the network: 0 = the patch features of
                              Sec. 2.2 (4 K^2 + 4 for K x K patch nodes, default); any
                              other value (1..127) makes a network for dnnmg_patch_infer
                              and training only (DNN-MG steps and samples need the
                              patch features); Table 1's networks have 51 */
  int32_t obstacle_level;  /* level whose cells place the obstacle square (Sec. 2.1 gives no
                              geometry): 0 = level-0 cells, 1 <= i0 <= 13, j0 = 1 (default);
                              1 = snapped to level-1 cells (the square is 4x4 of them),
                              2 <= i0 <= 27, 1 <= j0 <= 3, and j0 = 2 or i0 odd (the other
                              positions leave a one-cell fluid strip along the inflow or
                              a wall with no free velocity node on level 1, and the
                              coarse problem is singular there).  At odd level-1 offsets the 2h
                              stabilisation patches of level 1 along the square are partly
                              solid (their term integrates over the fluid cells only); the
                              coarse direct solve assembles them, and dnnmg_apply refuses
                              level 1 there; level 0 keeps only its fully covered cells.
                              Levels >= 2 see the square exactly, as whole patches.  Single
                              contexts only (not the batched engine nor the allocation-free
                              call). */
} dnnmg_config;

/* Per-step statistics returned by dnnmg_step(). */
typedef struct dnnmg_step_stats {
  int32_t newton_its;
  int32_t gmres_its;   /* total FGMRES iterations = V-cycles */
  int32_t fallback;    /* 1 if the network correction was dropped for this step */
  int32_t status;      /* status code of the step */
  double res0;         /* initial nonlinear residual norm */
  double res_final;    /* final nonlinear residual norm */
  double ms;           /* device time of the step in milliseconds */
} dnnmg_step_stats;

/* Fill *cfg with the defaults: nu = 0.01, dt = 0.01, theta = 1, alpha0 = 0.1,
 * newton_tol = 1e-10, gmres_rtol = 1e-4, omega = 0.8, eps_damp = 1,
 * obstacle at level-0 cell (2, 1), L = 3, coarse level 1, replaced_levels = 1,
 * FP64, newton_max = 20, gmres_m = 20, gmres_maxit = 200, V(2,2), GRU 2 x 64,
 * dense width 128, fallback_newton_its = 8, coarse_refresh = 32,
 * persistent_vcycle = -1, precond_lag = 1.  Returns DNNMG_ERR_ARG if cfg is
 * NULL. */
int dnnmg_default_config(dnnmg_config* cfg);

/* Create a context: builds the level hierarchy coarse..L (and L+1..L+r for the
 * network), boundary masks, stencil constants and all workspaces, and sets the
 * state to the impulsive start (zero interior velocity and pressure, parabolic
 * inflow u = 6y(1-y)).  `stream` is a cudaStream_t (NULL = legacy default).
 * Errors: DNNMG_ERR_ARG for an invalid configuration (levels out of range,
 * obstacle not inside the channel, unsupported sizes), DNNMG_ERR_CUDA if an
 * allocation fails; *out is NULL then. */
int dnnmg_setup(const dnnmg_config* cfg, void* stream, dnnmg_ctx** out);

/* Free everything owned by ctx.  NULL is allowed. */
int dnnmg_destroy(dnnmg_ctx* ctx);

/* Message of the last failure on ctx ("" if none), owned by ctx.  With
 * ctx = NULL: the message of this thread's last failed dnnmg_setup() or
 * dnnmg_coarse_solve_noalloc() call. */
const char* dnnmg_last_error(const dnnmg_ctx* ctx);

/* Cells of mesh level `level` (any level from 0 to L + replaced_levels). */
int dnnmg_level_dims(const dnnmg_ctx* ctx, int level, int* nx, int* ny);

/* Copy the FP64 state x_n of the finest solved level L to/from device
 * buffer x ([3][nn] doubles).  set_state imposes the Dirichlet values on the
 * constrained DOFs and clears the network's stored right-hand side and
 * hidden state. */
int dnnmg_get_state(dnnmg_ctx* ctx, double* x);
int dnnmg_set_state(dnnmg_ctx* ctx, const double* x);

/* Linearise the multigrid hierarchy at the velocity of the FP64 device state
 * x ([3][nn] doubles on level L): the velocity is injected nodally to every
 * coarser level, every level's Jacobian A'(vbar) (Eq. 6) is set up (Vanka
 * inverses, coarse-level LU and inverse).  Needed before dnnmg_apply() and
 * dnnmg_vcycle(); dnnmg_step() does it itself.
 * Errors: DNNMG_ERR_NUMERICAL if a local Vanka matrix or the coarse matrix
 * is singular. */
int dnnmg_linearize(dnnmg_ctx* ctx, const double* x);

/* y = A'(vbar) w on level `level` (coarse <= level <= L) at the current
 * linearisation, with identity rows and columns on constrained DOFs.
 * w, y: device [3][nn] arrays of double (precision = DNNMG_FP64) or float
 * (DNNMG_MIXED); precision must equal the context's. */
int dnnmg_apply(dnnmg_ctx* ctx, int level, const void* w, void* y, int precision);

/* One V(nu1, nu2) cycle (Sec. 2.2; cell-wise Vanka smoother, bilinear
 * transfers, direct coarse solve) on level `level` for A'(vbar) x = b,
 * starting from x = 0.  b, x: device [3][nn] arrays of the context's
 * precision (see dnnmg_apply).  b should vanish on constrained DOFs. */
int dnnmg_vcycle(dnnmg_ctx* ctx, int level, const void* b, void* x, int precision);

/* r = f - A_n(x) (Eqs. 4-5) on level L in FP64, zero on constrained DOFs.
 * x, f, r: device [3][nn] doubles. */
int dnnmg_residual(dnnmg_ctx* ctx, const double* x, const double* f, double* r);

/* One time step (Eq. 3) from the context's state.  mode = DNNMG_PLAIN: the
 * right-hand side is the old-time term of Eq. 5; mode = DNNMG_NET: the step
 * uses the restricted right-hand side left by the previous DNN-MG step (if
 * any) and ends with the network correction of Algorithm 1 (prolongation, network, Rhs,
 * restriction).  If the Newton iteration count exceeds the fallback threshold
 * the step is recomputed without the network right-hand side (Sec. 3.3).
 * stats (host pointer, may be NULL) receives the step statistics.
 * Returns DNNMG_ERR_NOT_CONVERGED if Newton hit newton_max (the step is still
 * taken), DNNMG_ERR_NUMERICAL on NaN/Inf. */
int dnnmg_step(dnnmg_ctx* ctx, int mode, dnnmg_step_stats* stats);

/* One time step with the level-L state exchanged through HOST memory (the
 * coupling of a host-resident application, e.g. an FE code that owns the
 * state): x_in ([3][nn] doubles, host, pinned for best speed) becomes the
 * state v^L_{n-1} (Dirichlet values imposed; the network's hidden state and
 * stored right-hand side are kept), the step runs as dnnmg_step(), and the new
 * state is copied to x_out (host).  Either pointer may be NULL to skip that
 * copy. */
int dnnmg_step_io(dnnmg_ctx* ctx, int mode, const double* x_in, double* x_out,
                  dnnmg_step_stats* stats);

/* Unmasked bilinear prolongation P of all three fields from level `level`
 * to level + 1 (the prolongation P of Algorithm 1): xc device [3][nn(level)]
 * doubles, xf device [3][nn(level + 1)] doubles; level + 1 <= L + replaced_levels. */
int dnnmg_prolongate(dnnmg_ctx* ctx, int level, const double* xc, double* xf);

/* ---- functionals (Sec. 3.4) ---------------------------------------------------
 * dnnmg_functionals: out (host, 3 doubles) = {J_div, J_drag, J_lift} of the
 * state x (device [3][nn(level)] doubles, any level 0 .. L + replaced_levels)
 * with the context's nu and dt:
 *   J_div  = int |div v|^2 dx over the fluid cells (2x2 Gauss per cell);
 *   J_drag = -int_Gamma (nu grad v - p I) n . e_x ds, J_lift the same with
 *            e_y, Gamma the obstacle boundary, n pointing into the obstacle.
 * Drag and lift are evaluated in residual (volume) form: minus the
 * backward-Euler momentum rows (1/k) M (v - v_old) + nu K v + N(v) v
 * - (p, div phi) summed over the obstacle's boundary nodes.  x_old (device,
 * same layout, velocity used) is the state one time step earlier; NULL drops
 * the time-derivative term (steady form).  Fixed-order sums: repeated calls
 * return identical values.  Synchronous on the context's stream.
 *
 * dnnmg_relative_errors: out (host, 2 doubles) = relative l2 errors of the
 * velocity and of the pressure of x against x_ref (both device
 * [3][nn(level)] doubles).  DNNMG_ERR_NUMERICAL if a reference part is zero. */
int dnnmg_functionals(dnnmg_ctx* ctx, int level, const double* x, const double* x_old,
                      double* out);
int dnnmg_relative_errors(dnnmg_ctx* ctx, int level, const double* x, const double* x_ref,
                          double* out);

/* ---- patch network (Sec. 2.2, Sec. 3.1, Table 1) ------------------------------
 * n stacked GRU cells of hidden size m (config gru_layers, hidden; m x n in
 * {32, 64} x {1, 2, 3}, Table 1; default 64 x 2; PyTorch gate convention r,
 * z, n) and a dense head Linear(m, 128) + ReLU + Linear(128, C_out), applied
 * to every patch independently.  A patch is one level-L cell; with r
 * replaced levels it covers K x K nodes of level L + r (K = 3 for r = 1, 5
 * for r = 2): C_in = 4 K^2 + 4 inputs (prolongated velocity u, v and fine
 * velocity residual r_u, r_v at its K x K fine nodes, then 4 geometry/flow
 * features: 40 or 104), C_out = 2 K^2 outputs (velocity correction u, v at
 * the nodes: 18 or 50).  Every size runs with C_in = 40; with C_in = 104 the
 * 64 x 3 network does not fit the kernel's shared memory and its network
 * calls return DNNMG_ERR_ARG.  Weights are BF16 on the tensor cores with
 * FP32 accumulation; the hidden state is FP32.
 * Flat FP32 parameter order (PyTorch's): per GRU layer W_ih [3m][C_l],
 * W_hh [3m][m], b_ih [3m], b_hh [3m] (C_0 = C_in, C_l = m above); then
 * W1 [128][m], b1 [128], W2 [C_out][128], b2 [C_out].  A new context has
 * all weights zero. */

/* Number of network parameters (55,954 for 64 x 2 with C_in = 40, C_out =
 * 18; 72,370 for 64 x 2 with C_in = 104, C_out = 50). */
size_t dnnmg_num_params(const dnnmg_ctx* ctx);

/* Network input and output widths of the context. */
int dnnmg_net_dims(const dnnmg_ctx* ctx, int* c_in, int* c_out);

/* Copy the FP32 parameters from / to HOST memory (dnnmg_num_params floats).
 * set_weights re-packs the BF16 tensor-core copy. */
int dnnmg_set_weights(dnnmg_ctx* ctx, const float* w);
int dnnmg_get_weights(dnnmg_ctx* ctx, float* w);

/* One recurrent step of the network for P patches (the network evaluation of Algorithm 1):
 *   x   : device [P][C_in] bfloat16 (raw uint16 bits), normalised inputs
 *   h   : device [gru_layers][P][hidden] float, hidden state, updated in place
 *   out : device [P][C_out] float, predicted correction
 * P = 0 is a no-op.  Errors: DNNMG_ERR_ARG (unsupported network shape),
 * DNNMG_ERR_TIMEOUT (a tensor-core completion wait hit its bound). */
int dnnmg_patch_infer(dnnmg_ctx* ctx, const uint16_t* x, float* h, float* out, int P);

/* C = A B^T on the tensor cores: A device [M][K], B device [N][K] bfloat16
 * row-major, C device [M][N] float row-major; M % 128 == 0,
 * 16 <= N <= 256 with N % 16 == 0, K % 16 == 0 (else DNNMG_ERR_ARG). */
int dnnmg_gemm_bf16(dnnmg_ctx* ctx, const uint16_t* A, const uint16_t* B, float* C, int M, int N,
                    int K);

/* ---- DNN-MG state (the network correction of Algorithm 1) -----------------------------------
 * A DNNMG_NET step ends with: v~ = P(v^L) on the fine level F = L + r (P
 * applied once per replaced level); the fine residual r = f - A(v~, P p^L)
 * of Eq. 3 on level F with f built from the previous corrected fine
 * velocity; the patch inputs; one network step (the hidden state persists
 * across steps); v_corr = v~ + d with d averaged over the patches sharing a
 * node and zero on Dirichlet nodes; b^F = Rhs(v_corr) = (1/k) M v_corr; and
 * b^L = R b^F (R once per replaced level), the velocity right-hand side of
 * the next step.  Patches are the fluid cells of level L in cell order
 * (j * nx + i). */

/* Number of patches (fluid cells of level L). */
int dnnmg_num_patches(const dnnmg_ctx* ctx);

/* Per-feature standardisation of the network inputs, host arrays [C_in]:
 * input = (feature - mean) / std.  Default mean 0, std 1. */
int dnnmg_set_feature_stats(dnnmg_ctx* ctx, const float* mean, const float* std);

/* Corrected fine velocity v_corr of the last DNN-MG step: device
 * [2][nn of level L + replaced_levels] doubles.  DNNMG_ERR_STATE before the
 * first one. */
int dnnmg_get_fine_velocity(dnnmg_ctx* ctx, double* v);

/* Network inputs of the last DNN-MG step: device [P][C_in] bfloat16. */
int dnnmg_get_patch_inputs(dnnmg_ctx* ctx, uint16_t* x);

/* ---- training (Eq. 7, Sec. 3.1) -------------------------------------------------
 * One batch = B patch sequences of T steps; the hidden state starts at zero
 * for every sequence.  Loss = mean over (b, t, outputs) of (y - Y)^2 (Eq. 7
 * as a mean).  Gradients by backpropagation through time on the tensor
 * cores (BF16 operands, FP32 accumulation); weight gradients are split-K
 * GEMMs with a fixed-order reduction (deterministic).  The workspace is
 * allocated by dnnmg_setup() for cfg.train_batch x cfg.train_seq.
 *   X : device [B][T][C_in] bfloat16     Y : device [B][T][C_out] float
 * Requirements: B % 16 == 0, 16 <= B <= train_batch, 1 <= T <= train_seq
 * (else DNNMG_ERR_ARG; DNNMG_ERR_STATE without a training workspace). */

/* Loss (host *loss) and gradient (device grad, dnnmg_num_params floats, in
 * the flat parameter order) at the current weights; no update. */
int dnnmg_train_grad(dnnmg_ctx* ctx, const uint16_t* X, const float* Y, int B, int T, float* grad,
                     float* loss);

/* One Adam step (beta = (0.9, 0.999), eps = 1e-8, bias-corrected) with
 * learning rate lr on the FP32 weights; the BF16 copies are re-packed.
 * *loss (host, may be NULL) receives the loss before the update. */
int dnnmg_train_step(dnnmg_ctx* ctx, const uint16_t* X, const float* Y, int B, int T, float lr,
                     float* loss);

/* Zero the Adam moments and step count. */
int dnnmg_reset_optimizer(dnnmg_ctx* ctx);

/* ---- training corpus from plain fine-level trajectories (Sec. 3.1) ----------
 * Training data comes from high-fidelity solutions on level L+1, localised
 * to the time steps and patches.  Given two consecutive fine states
 * x^F_{n-1}, x^F_n on the fine level F = L + replaced_levels (device
 * [3][nn of level F] doubles, e.g. from a second context with
 * level_solve = F), dnnmg_make_sample injects x^F_{n-1} to level L, solves
 * the level-L step with the right-hand side an exact correction would give,
 * b^L = R (1/k) M^F v^F_{n-1} (R once per replaced level), and writes for
 * every patch the raw (unstandardised) inputs at P(v^L_n) (device [P][C_in]
 * float) and the targets v^F_n - P(v^L_n) at its fine nodes, zero on
 * Dirichlet nodes (device [P][C_out] float).  It overwrites the context's
 * level-L state and clears its DNN-MG state. */
int dnnmg_make_sample(dnnmg_ctx* ctx, const double* xf_prev, const double* xf_next, float* X,
                      float* Y, dnnmg_step_stats* stats);

/* The whole corpus of Sec. 3.1 on the device: n_traj plain trajectories of
 * the context's channel (its obstacle), trajectory k with viscosity nu[k]
 * (host array).  Each starts from rest: spinup_steps plain steps of the
 * level-L solver with time step spinup_dt, the state prolongated (P, once
 * per replaced level) to the fine level F = L + replaced_levels, then
 * relax_steps plain fine-level steps with the configured dt, then T more
 * fine steps; after fine step n the pair (x^F_{n-1}, x^F_n) gives one
 * dnnmg_make_sample into slot s = k * T + n.
 *   X: device [n_traj][T][P][C_in] float (raw inputs, row = s * P + patch),
 *   Y: device [n_traj][T][P][C_out] float (targets); the layout
 *      dnnmg_gather_batch reads with stride = P.
 * The first call creates (allocates) a plain solver on level F inside the
 * context; later calls reuse it.  On return the context's nu and dt are the
 * configured ones again and its state is the impulsive start (network
 * state cleared).  Errors: DNNMG_ERR_ARG (counts < 1, negative steps,
 * non-positive nu or spinup_dt), DNNMG_ERR_STATE (no DNN-MG network), and
 * the errors of the steps; a step that stops at its Newton cap is kept. */
int dnnmg_make_corpus(dnnmg_ctx* ctx, int n_traj, const double* nu, int spinup_steps,
                      double spinup_dt, int relax_steps, int T, float* X, float* Y);

/* Per-feature mean and standard deviation (population, FP64 sums in fixed
 * order) of `rows` raw input rows (device [rows][C_in] float); they become the
 * context's standardisation (features with zero spread get std 1).  mean /
 * std (host [C_in], may be NULL) receive them. */
int dnnmg_feature_stats(dnnmg_ctx* ctx, const float* X, int64_t rows, float* mean, float* std);

/* Assemble a training batch from a raw corpus laid out row = s * stride + p
 * (s: time-step slot, p: patch): sequence b takes rows
 * (idx[2b] + t) * stride + idx[2b+1], t = 0..T-1.  idx: device [B][2] int32.
 * Writes Xb (device [B][T][C_in] bfloat16, standardised) and Yb (device
 * [B][T][C_out] float). */
int dnnmg_gather_batch(dnnmg_ctx* ctx, const float* X, const float* Y, const int* idx, int B,
                       int T, int64_t stride, uint16_t* Xb, float* Yb);

/* Direct solve of the coarsest multigrid level without any device allocation
 * (the paper has no counterpart: this is a deployment variant).
 *
 * For callers that cannot call cudaMalloc - e.g. code that runs under an
 * external memory manager owning the whole device heap, or inside a
 * real-time loop where an allocation and the synchronisation it may cause
 * are not allowed - and therefore cannot create a context.  It assembles the
 * linearised operator A'(vbar) of level cfg->level_coarse, factors it
 * by banded LU with partial pivoting and returns x = A'(vbar)^{-1} b: the
 * same operator the coarse level of dnnmg_vcycle() inverts.
 *   cfg  : host pointer; uses nu, dt, theta (must be 1), alpha0, obstacle_i0,
 *          obstacle_j0 and level_coarse.
 *   vbar : device, [2][nn] doubles, linearisation velocity on that level.
 *   b, x : device, [3][nn] doubles on that level (b and x may not alias).
 *   stream: cudaStream_t to issue the work on; the call synchronises it.
 * Working memory is one file-scope __device__ array of 2 MiB that every GPU
 * which loads this library holds until the process exits; it fits level 1
 * only (891 unknowns, ~1.34 MB).  Larger levels return DNNMG_ERR_ARG.
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  All
 * calls share the array and it keeps the last call's contents, so calls that
 * overlap on the GPU (other streams, other threads) race: serialise them.
 * Errors: DNNMG_ERR_ARG, DNNMG_ERR_CUDA (also when a CUDA error of earlier
 * work was already pending on entry: it is left pending), DNNMG_ERR_NUMERICAL
 * (singular matrix); the message is read with dnnmg_last_error(NULL). */
int dnnmg_coarse_solve_noalloc(const dnnmg_config* cfg, const double* vbar, const double* b,
                               double* x, void* stream);

/* Per-stage device timers (tracing).  Stages: */
#define DNNMG_STAGE_VANKA_PASS 0    /* one colour pass of the Vanka smoother */
#define DNNMG_STAGE_VANKA_SETUP 1   /* local 12x12 inverses of one level */
#define DNNMG_STAGE_APPLY 2         /* Jacobian apply inside FGMRES */
#define DNNMG_STAGE_DEFECT 3        /* defect before restriction */
#define DNNMG_STAGE_TRANSFER 4      /* restriction / prolongation */
#define DNNMG_STAGE_COARSE_FACTOR 5 /* coarse-level LU and inverse */
#define DNNMG_STAGE_COARSE_SOLVE 6  /* coarse-level solve in the V-cycle */
#define DNNMG_STAGE_KRYLOV 7        /* FGMRES orthogonalisation and updates */
#define DNNMG_STAGE_RESIDUAL 8      /* FP64 nonlinear residual */
#define DNNMG_STAGE_NETWORK 9       /* DNN-MG gather, patch network, scatter and Rhs */
#define DNNMG_STAGE_TRAIN 10        /* training forward, backward and optimiser */
#define DNNMG_STAGE_VCYCLE 11       /* one persistent V-cycle launch (all of the above in it) */

/* enable != 0: reset the timers and record CUDA events around the launches
 * of each stage from now on; enable = 0: stop recording.  Recording costs one
 * event pair per timed launch group; results are exact device times. */
int dnnmg_profile(dnnmg_ctx* ctx, int enable);

/* Accumulated device time (ms) and number of timed launch groups of `stage`
 * on mesh level `level` (level = -1: all levels) since the last reset.
 * Synchronises the context's stream. */
int dnnmg_profile_read(dnnmg_ctx* ctx, int stage, int level, int64_t* launches, double* ms);

/* Level from which the V-cycle runs as one persistent launch (0: none),
 * as configured or chosen by timing at the first linearisation; -1 on error. */
int dnnmg_vcycle_split(const dnnmg_ctx* ctx);

/* The autotuned plan of the V-cycle (valid after the first linearisation):
 * the split level as above; the kind of persistent launch below it (0: one
 * cooperative grid with grid-wide barriers, 1: one thread-block cluster of
 * up to 16 blocks with cluster barriers); and the tile of colour cells per
 * block of the colour pass on `level` (0: 16x4, 1: 8x4, 2: 8x8, 3: the
 * streaming pass of 16x4 tiles; -1 if the level is not in the hierarchy). */
int dnnmg_vcycle_plan(const dnnmg_ctx* ctx, int level, int* split_level, int* split_mode,
                      int* pass_shape);

/* ------------------------------------------------------------------------
 * Batched problems
 *
 * A batch advances many independent channel problems of uneven size in
 * lock-step with the algorithm of a single context (Newton, FGMRES, one
 * V-cycle per Krylov step; DNN-MG steps add the network correction of
 * Algorithm 1 with one network evaluation over the patches of all problems).
 * Every stage (a Vanka colour pass on level k, a defect, a transfer, a
 * Krylov vector operation, ...) is one kernel launch over a work list of
 * the blocks of all problems that take part in it; problems that have
 * converged are masked.  One FGMRES iteration is replayed as a CUDA graph.
 *
 * Problems may differ in nu, dt, theta, alpha0, the obstacle and
 * level_solve; all other fields must be equal.  DNN-MG needs
 * replaced_levels = 1 and one network shared by all problems.
 *
 * The finest solved level of every problem lives in concatenated vectors
 * of `length` elements: problem p occupies [offset_p, offset_p + 3 nn_p)
 * ([3][ny+1][nx+1] layout of its level), padded with zeros to the next
 * problem.  The batch runs on an internal stream: each call waits for the
 * stream given to dnnmg_batch_setup() first and returns with its own work
 * complete.
 * ------------------------------------------------------------------------ */
typedef struct dnnmg_batch dnnmg_batch;

/* Set up n >= 1 problems from cfgs[0..n) (validated like dnnmg_setup).  On
 * failure *out is NULL and dnnmg_batch_last_error(NULL) holds the reason. */
int dnnmg_batch_setup(const dnnmg_config* cfgs, int n, void* stream, dnnmg_batch** out);
int dnnmg_batch_destroy(dnnmg_batch* b);
/* message of the last failure of b (b = NULL: of this thread's last setup) */
const char* dnnmg_batch_last_error(const dnnmg_batch* b);
/* number of problems and length of the concatenated top-level vectors */
int dnnmg_batch_size(const dnnmg_batch* b, int* n, int64_t* length);
/* finest solved level and offset of problem `inst` in the concatenated vectors */
int dnnmg_batch_layout(const dnnmg_batch* b, int inst, int* level, int64_t* offset);
/* FP64 state of problem `inst` ([3][..] of its level, device) */
int dnnmg_batch_get_state(dnnmg_batch* b, int inst, double* x);
/* replaces the state (Dirichlet values re-imposed); resets the DNN-MG
 * history of the batch and forces a coarse refactorisation at the next step */
int dnnmg_batch_set_state(dnnmg_batch* b, int inst, const double* x);
/* linearise every problem's hierarchy at its current state (like
 * dnnmg_linearize of a single context) */
int dnnmg_batch_linearize(dnnmg_batch* b);
/* one V(nu1, nu2) cycle of every problem on its finest solved level from
 * x = 0: rhs, x are concatenated device vectors of `length` elements in the
 * batch precision (double for DNNMG_FP64, float for DNNMG_MIXED) */
int dnnmg_batch_vcycle(dnnmg_batch* b, const void* rhs, void* x);
/* One V(nu1, nu2) cycle (Sec. 2.2) of problem `inst` alone on its finest
 * solved level, from x = 0, at the batch's current linearisation: rhs, x are
 * that problem's own device vectors ([3][nn] of its level, batch precision),
 * not the concatenated ones.  The instance form of dnnmg_vcycle.
 * Errors: DNNMG_ERR_ARG (inst out of range), DNNMG_ERR_STATE (not
 * linearised). */
int dnnmg_batch_vcycle_inst(dnnmg_batch* b, int inst, const void* rhs, void* x);
/* One time step of every problem; stats[0..n) (nullable) receive each
 * problem's counts and status (ms: the batch's step time).  Returns
 * DNNMG_OK or the first non-OK problem status. */
int dnnmg_batch_step(dnnmg_batch* b, int mode, dnnmg_step_stats* stats);
/* shared network weights (host, flat order of dnnmg_set_weights) and
 * feature standardisation (host, C_in floats each) */
int dnnmg_batch_set_weights(dnnmg_batch* b, const float* w);
int dnnmg_batch_set_feature_stats(dnnmg_batch* b, const float* mean, const float* std);
/* corrected fine velocity of problem `inst` after a DNN-MG step ([2][..] of
 * level L + replaced_levels, device) */
int dnnmg_batch_get_fine_velocity(dnnmg_batch* b, int inst, double* v);
/* on != 0 (default): replay FGMRES iterations as CUDA graphs */
int dnnmg_batch_graphs(dnnmg_batch* b, int on);
/* stage timers as dnnmg_profile / dnnmg_profile_read (levels are absolute) */
int dnnmg_batch_profile(dnnmg_batch* b, int enable);
int dnnmg_batch_profile_read(dnnmg_batch* b, int stage, int level, int64_t* launches, double* ms);

/* Number of kernels this library has launched in this process so far. */
uint64_t dnnmg_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* DNNMG_H */
