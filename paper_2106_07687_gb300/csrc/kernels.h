// Host-side launchers of the solver kernels (internal to libdnnmg).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace dnnmg {

// Process-wide count of kernels launched by this library.
void note_launch();
void note_launches(unsigned long long n);  // kernels of a replayed graph
unsigned long long launches();

// Operator rows (stencil.cu) ---------------------------------------------
// y = A'(vbar) w on free DOFs, y = w on constrained DOFs (Eq. 6); nothing
// when skip is set and *skip != 0 at the launch's start.
template <typename T>
void launch_apply(const Grid& g, const Sten<T>& s, const T* w, const T* vb, T* y, cudaStream_t st,
                  const int* skip = nullptr);
// d = b - A'(vbar) x with the same constrained handling; if `masked`,
// d is zeroed on constrained DOFs (input of the restriction).
template <typename T>
void launch_defect(const Grid& g, const Sten<T>& s, const T* b, const T* x, const T* vb, T* d,
                   bool masked, cudaStream_t st);
// r = f - A(x) on free DOFs, 0 on constrained DOFs (FP64 nonlinear residual).
// With dfloat_ops, A(x) is evaluated in double-float arithmetic (about 48
// significant bits, FP32 units) and only f - A(x) in FP64.
// With no.partials set, the launch also forms |r|^2: every block's sum in a
// fixed order, then the last block to finish adds the blocks' sums in block
// order, stores the total in *no.out, posts it into no.mail->v[0] (as post
// no.seq, when mail is set) and resets *no.counter (zero between launches).
// no.partials holds residual_blocks(g) doubles.
struct NormOut {
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* out = nullptr;
  HostMail* mail = nullptr;
  unsigned long long seq = 0;
  const int* status = nullptr;  // when set, status[0..3] is posted too (mail->iv[0..3])
};
int residual_blocks(const Grid& g);
void launch_residual64(const Grid& g, const Sten<double>& s, const double* x, const double* f,
                       double* r, cudaStream_t st, bool dfloat_ops = false,
                       const NormOut& no = NormOut{});
// The fine-level residual f - A(x) whose only use is the network's input
// features (rounded to BF16): the operator in FP32 when fp32_ops (mixed
// precision contexts), else launch_residual64 in FP64.
void launch_residual_features(const Grid& g, const Sten<double>& s, const double* x,
                              const double* f, double* r, cudaStream_t st, bool fp32_ops);
// f = (1/k) M v_old on the velocity rows, 0 on the pressure rows.
// With copy, also copy = x_old (all three fields) in the same launch.
void launch_old_time_rhs64(const Grid& g, double inv_k, const double* x_old, double* f,
                           cudaStream_t st, double* copy = nullptr);

// f -= coef * (explicit transport + diffusion of x) on the velocity rows
// (theta-scheme old-time terms); sx from make_explicit_sten
void launch_explicit_sub64(const Grid& g, const Sten<double>& sx, double coef, const double* x,
                           double* f, cudaStream_t st);

// Transfers (transfer.cu) ----------------------------------------------------
// bc = R d (R = P^T on free DOFs, coarse constrained rows zeroed)
template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* d, T* bc, cudaStream_t st);
// x += P xc on free fine DOFs
template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, T* x, cudaStream_t st);
// coarse (I, J) <- fine (2I, 2J), ncomp fields
template <typename T>
void launch_inject(const Grid& fine, const Grid& coarse, const T* xf, T* xc, int ncomp,
                   cudaStream_t st);
// Every level's linearisation point from the finest velocity at once: level
// k of nlev (the last the finest) takes the fine node (2^m I, 2^m J), m =
// nlev-1-k, which is the nodal injection applied m times.  Writes vb64 (FP64)
// and vb (T) of each level, vbJ (T) of the finest, and clears *status when
// status is not null.  One launch; results equal inject + cast bit for bit.
template <typename T>
struct LinLevels {
  int nlev;
  int nnx[kMaxLevels], nn[kMaxLevels], off[kMaxLevels + 1];  // off: prefix of nn
  double* vb64[kMaxLevels];
  T* vb[kMaxLevels];
};
template <typename T>
void launch_linearize_levels(const LinLevels<T>& L, const double* x64, T* vbJ, int* status,
                             cudaStream_t st);
// Unmasked bilinear prolongation of ncomp fields (DNN-MG state transfer).
// With ximp (ncomp = 3), also ximp = xf with the Dirichlet values imposed.
void launch_prolong_state64(const Grid& fine, const Grid& coarse, const double* xc, double* xf,
                            int ncomp, cudaStream_t st, double* ximp = nullptr);
// Unmasked R = P^T of ncomp fields (DNN-MG right-hand side restriction).
void launch_restrict_full64(const Grid& fine, const Grid& coarse, const double* bf, double* bc,
                            int ncomp, cudaStream_t st);

// Vanka (vanka.cu) -----------------------------------------------------------
// inverse of the 12x12 restriction of A'(vbar) to every fluid cell, stored
// inv[colour][144][slot], slot = tj * (nx/2 + 1) + ti, cell (2ti - ci, 2tj - cj)
template <typename T>
void launch_vanka_setup(const Grid& g, const Sten<T>& s, const T* vb, T* inv, int* status,
                        cudaStream_t st);
// one colour pass: xout = xin + omega A_c^{-1} (b - A xin)_c on the colour's cells;
// `shape` picks the tile of colour cells a block owns: 0 = 16x4, 1 = 8x4, 2 = 8x8
constexpr int kPassShapes = 3;
constexpr int kPassStream = 3;  // plan code of the streaming pass (vanka_stream.cu)
template <typename T>
void launch_vanka_pass(const Grid& g, const Sten<T>& s, int colour, const T* b, const T* xin,
                       const T* vb, const T* inv, T omega, T* xout, cudaStream_t st,
                       int shape = 0);
// Slots of a colour's cells: slot (ti, tj) = cell (2 ti - cx, 2 tj - cy) of
// colour (cx, cy), for ti < nx/2 + 1, tj < ny/2 + 1.  A row of slots is padded
// to a multiple of 4 (16 bytes of FP32), so that a row of the inverse array
// inv[colour][entry][tj][ti] starts on a 16-byte boundary (tensor-memory-
// access copies need that); padding slots are never written or used.
__host__ __device__ inline int vanka_pitch(const Grid& g) { return ((g.nx / 2 + 1) + 3) & ~3; }
__host__ __device__ inline int vanka_slots(const Grid& g) { return vanka_pitch(g) * (g.ny / 2 + 1); }
// Streaming FP32 colour pass for large levels (vanka_stream.cu): the same
// result as launch_vanka_pass, with the tile's inverses copied by TMA one
// tile ahead.  map: a tensor map of the level's inverse array made by
// make_vanka_tensor_map (false if the driver cannot make one);
// vanka_stream_grid is 0 when the kernel cannot be resident.  A copy that
// does not arrive within the poll limit sets bit 8 of *status.
constexpr int kTensorMapBytes = 128;
bool make_vanka_tensor_map(void* map, const float* inv, const Grid& g);
int vanka_stream_grid(const Grid& g);
void launch_vanka_pass_stream(const void* map, const Grid& g, const Sten<float>& s, int colour,
                              const float* b, const float* xin, const float* vb, float omega,
                              float* xout, int* status, cudaStream_t st);
// Vanka setup kernels: 16 lanes per cell, kSetupCells cells per block
constexpr int kSetupThreads = 128;
constexpr int kSetupCells = kSetupThreads / 16;

// Coarse direct solve (coarse.cu) -------------------------------------------
// Assemble the banded Jacobian of the coarsest level (FP64), factor it with
// partial pivoting and form the explicit inverse Ainv (ndof x ndof, FP64,
// unknowns in band order).  `work` needs coarse_work_doubles(g) doubles.
size_t coarse_work_doubles(const Grid& g);
bool coarse_supported(const Grid& g);  // band fits the shared-memory window
// Assemble + factor into caller-provided band storage (coarse_band_doubles(g)
// doubles) and pivots (3 nn ints), and solve with those factors.
size_t coarse_band_doubles(const Grid& g);
void launch_coarse_lu(const Grid& g, const Sten<double>& s, const double* vb, double* band,
                      int* piv, int* status, cudaStream_t st);
void launch_coarse_lu_solve(const Grid& g, const double* band, const int* piv, const double* b,
                            double* x, cudaStream_t st);
struct PatchPieces;  // coarse_body.cuh
// pp: stabilisation pieces of part-solid patches (null: every patch is whole)
void launch_coarse_factor(const Grid& g, const Sten<double>& s, const double* vb, double* work,
                          double* Ainv, int* status, cudaStream_t st,
                          const PatchPieces* pp = nullptr);
// x = Ainv b, b and x in the [3][nn] layout of the level
template <typename T>
void launch_coarse_solve(const Grid& g, const double* Ainv, const T* b, T* x, cudaStream_t st);

// Vectors (vec.cu) ----------------------------------------------------------
// Post n doubles from src (device) into v[slot..] and ni ints from isrc into
// iv[islot..] as post number seq (one thread; src/isrc may be null).
void launch_post(HostMail* mail, unsigned long long seq, const double* src, int slot, int n,
                 const int* isrc, int islot, int ni, cudaStream_t st);
template <typename Ts, typename Td>
void launch_cast(const Ts* a, Td* b, size_t n, cudaStream_t st);
template <typename T>
void launch_fill(T* a, T v, size_t n, cudaStream_t st);
// b = a and d = c, n doubles each, in one launch
void launch_copy2(const double* a, double* b, const double* c, double* d, size_t n,
                  cudaStream_t st);
// partial dot products of w against k vectors V[i] (stride ld); out[k] after
// launch_dots_finish.  partials needs dots_partials(n, k) doubles.
// With mail (k = 1 only), out[0] is also posted into mail->v[0] as post seq.
template <typename T>
void launch_multidot(const T* V, size_t ld, int k, const T* w, size_t n, double* partials,
                     double* out, cudaStream_t st, HostMail* mail = nullptr,
                     unsigned long long seq = 0);
// w -= sum_i h[i] V[i]
template <typename T>
void launch_multiaxpy(const T* V, size_t ld, int k, const double* h, T* w, size_t n,
                      cudaStream_t st);
// y = s * x with s = a, 1/a or 1/sqrt(a) (mode 0, 1, 2), a read on the device
template <typename T>
void launch_scale_dev(const T* x, const double* a, int mode, T* y, size_t n, cudaStream_t st);
// x += eps * (sum_i y[i] Z[i]) in FP64 accumulation, result type Tx
template <typename T, typename Tx>
void launch_combine(const T* Z, size_t ld, int k, const double* y, double eps, Tx* x, size_t n,
                    cudaStream_t st);
size_t dots_partials(size_t n, int k);
// One Arnoldi step (CGS2 against V[0..j], normalisation, Givens update of
// column j, resid = |g[j+1]|) in one cooperative launch; products in the
// vectors' precision, sums over threads and blocks in FP64.  Returns nonzero
// (nothing launched) when the cooperative grid cannot be resident.  partials needs (2 j + 3) x
// dots_partials(n, 1) doubles, hcol 2 j + 3.  With mail, resid is also
// posted into mail->v[0] as post seq.
template <typename T>
int launch_arnoldi_step(const T* V, size_t ld, int j, T* w, size_t n, double* partials,
                        double* hcol, double* H, int ldh, double* cs, double* sn, double* gvec,
                        double* resid, cudaStream_t st, HostMail* mail = nullptr,
                        unsigned long long seq = 0, int slot = 0, int* skip = nullptr,
                        const double* target = nullptr, int its = 0, int maxit = 0);
// whether launch_arnoldi_step can launch (its cooperative grid is resident)
template <typename T>
bool arnoldi_available();
// FGMRES small-matrix kernels: Hessenberg column j (from h[0..j+1]) is
// rotated, the new Givens rotation stored and g updated; resid = |g[j+1]|.
void launch_givens(double* H, int ldh, double* cs, double* sn, double* gvec, const double* hcol,
                   int j, double* resid, cudaStream_t st);
// y = H[0:k,0:k]^{-1} g[0:k] (back substitution)
void launch_backsolve(const double* H, int ldh, const double* gvec, int k, double* y,
                      cudaStream_t st);
// The start of an FGMRES cycle (one cooperative launch; nonzero return:
// nothing launched, the grid cannot be resident): with init, rT = (T) r64,
// rcur = rT, wsol = 0; then hcol[0] = |rcur|^2 (products in T, sums in
// FP64), V0 = rcur / |rcur|, gvec[0] = |rcur|, and with mail |rcur|^2 posted
// into mail->v[1].  With skip, *skip = 0 (the cycle's iterations run) and,
// with init, *target = rtol |rcur| (see launch_arnoldi_step).  partials
// needs dots_partials(n, 1) doubles.
template <typename T>
int launch_fgmres_begin(const double* r64, T* rT, T* wsol, T* rcur, T* v0, size_t n,
                        double* partials, double* hcol, double* gvec, bool init, HostMail* mail,
                        unsigned long long seq, cudaStream_t st, int* skip = nullptr,
                        double* target = nullptr, double rtol = 0.0);
// The end of a converged FGMRES cycle: y = H[0:k,0:k]^{-1} g[0:k] (FP64),
// then x64 += eps * (wsol + sum_i y[i] Z[i]), the combination in T.
template <typename T>
void launch_fgmres_finish(const double* H, int ldh, const double* gvec, int k, const T* Z,
                          size_t ld, const T* wsol, double eps, double* x64, size_t n,
                          cudaStream_t st);
// set V0 = r / ||r|| with norm from nrm2[0]; g[0] = ||r||.  With mail,
// nrm2[0] is also posted into mail->v[1] as post seq.
template <typename T>
void launch_gmres_start(const T* r, const double* nrm2, T* v0, double* gvec, size_t n,
                        cudaStream_t st, HostMail* mail = nullptr, unsigned long long seq = 0);

// ---- functionals of Sec. 3.4 (functionals.cu) --------------------------------
// Backward-Euler constants of a level (theta = 1) and its mass matrix over k.
struct FnConsts {
  Sten<double> s;
  double mk[16];
};
constexpr int kFnBlocks = 304;  // partial sums: part needs kFnBlocks * 4 doubles
// out (device) = {J_div, J_drag, J_lift} of state x; x_old may be null (steady form)
void launch_functionals(const Grid& g, const FnConsts& c, const double* x, const double* x_old,
                        double* part, double* out, cudaStream_t st);
// out (device) = {|v - v_ref|^2, |v_ref|^2, |p - p_ref|^2, |p_ref|^2}
void launch_rel_errors(const Grid& g, const double* x, const double* x_ref, double* part,
                       double* out, cudaStream_t st);

}  // namespace dnnmg
