// Batched engine (internal): many independent channel problems of uneven
// size stepped in lock-step, one kernel launch per V-cycle stage for all of
// them.
//
// Every level of every problem is described by a BLev record in device
// memory.  A stage kernel is launched over a work list of (problem, block)
// pairs, built once at setup for that stage's level and block shape, so a
// launch covers exactly the tiles or node blocks of the problems that have
// the level and no block idles.  Problems that have converged are masked by
// a per-problem active flag that every block reads first.
//
// The finest solved level of every problem (its "top" level) lives in
// concatenated vectors: problem i occupies [off_i, off_i + 3 nn_i), padded to
// a multiple of kVB elements so that a vector block never straddles two
// problems.  Krylov bases, the FP64 state and the Newton residual use this
// layout.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dnnmg.h"
#include "common.cuh"

namespace dnnmg {

constexpr int kNB = 256;        // nodes (threads) per block of the node kernels
constexpr int kVT = 256;        // threads per block of the vector kernels
constexpr int kVE = 4;          // elements per thread of the vector kernels
constexpr int kVB = kVT * kVE;  // elements per vector block (padding unit)

template <typename T>
struct BLev {
  Grid g;
  T *x, *x2, *b, *d, *vb, *inv;  // multigrid buffers (x, b unused on the top level)
  double* vb64;                  // FP64 linearisation point (velocity)
  long long off;                 // offset of the problem in the top-level vectors
  int top;                       // 1 on the problem's finest solved level
  int pad;
};

// Per-problem scalars read by the batched kernels.
struct BPar {
  double inv_k;   // 1 / dt
  double ecoef;   // 1 - theta (weight of the explicit old-time terms)
  double nu, dt;
  long long coff;  // offset of the problem's level-L cells in the cell -> patch table
  int L;           // finest solved level
  int explicit_on;
  float feat_h, feat_k;  // patch features h_L / 0.25 and k / h_L
  float feat_pe;         // h_L / (K^2 nu), the Peclet number's factor
};

// Device-side view of all problems (arrays indexed [problem * nL + level]).
template <typename T>
struct BView {
  const BLev<T>* lev;
  const Sten<T>* sT;         // multigrid constants in the V-cycle precision
  const Sten<double>* s64;   // FP64 constants (residual, coarse assembly)
  const Sten<double>* sx;    // explicit theta-scheme bracket (FP64)
  const BPar* par;           // [problem]
  int nL;
};

// Work list of a stage: (problem, block of that problem) per launched block.
struct Work {
  const int2* d = nullptr;
  int n = 0;
};

// Blocks of the concatenated top-level vectors: the problem of every block
// and every problem's first block and block count.
struct VecTab {
  const int* inst = nullptr;
  const int* first = nullptr;
  const int* count = nullptr;
  int nblk = 0, nprob = 0;
};

// Launchers (batch_kernels.cu).  `act` (nullable) masks problems: a block of
// a problem with act[problem] == 0 returns at once.  dl selects the level of
// the node kernels that run on a problem's own levels: 0 = finest solved
// level L, 1 = level L + 1 (the DNN-MG fine level).
template <typename T>
void bk_pass(const BView<T>& v, int k, int colour, int in, int out, const T* topb, T* topx,
             T omega, Work w, int shape, const int* act, cudaStream_t st);
template <typename T>
void bk_defect(const BView<T>& v, int k, int in, const T* topb, T* topx, Work w, const int* act,
               cudaStream_t st);
template <typename T>
void bk_restrict(const BView<T>& v, int k, Work w, const int* act, cudaStream_t st);
template <typename T>
void bk_prolong(const BView<T>& v, int k, int in, T* topx, Work w, const int* act,
                cudaStream_t st);
template <typename T>
void bk_coarse_solve(const BView<T>& v, int nprob, int n1, const double* Ainv, long long astride,
                     const T* topb, T* topx, const int* act, cudaStream_t st);
template <typename T>
void bk_apply(const BView<T>& v, const T* w, const T* vbJ, T* y, Work wk, const int* act,
              cudaStream_t st);
template <typename T>
void bk_defect_top(const BView<T>& v, const T* b, const T* x, const T* vbJ, T* d, Work wk,
                   const int* act, cudaStream_t st);
template <typename T>
void bk_residual64(const BView<T>& v, int dl, const double* x, const double* f, double* r,
                   Work wk, const int* act, cudaStream_t st);
template <typename T>
void bk_old_rhs(const BView<T>& v, int dl, const double* xo, double* f, Work wk, const int* act,
                cudaStream_t st);
template <typename T>
void bk_copy_impose(const BView<T>& v, int dl, const double* src, double* dst, Work wk,
                    const int* act, cudaStream_t st);
template <typename T>
void bk_top_vb(const BView<T>& v, const double* x64, Work wk, const int* act, cudaStream_t st);
template <typename T>
void bk_inject_vb(const BView<T>& v, int k, Work wk, const int* act, cudaStream_t st);
template <typename T>
void bk_cast_vb(const BView<T>& v, int k, Work wk, const int* act, cudaStream_t st);
template <typename T>
void bk_setup(const BView<T>& v, int k, int* status, Work wk, const int* act, cudaStream_t st);
template <typename T>
void bk_coarse_factor(const BView<T>& v, int nprob, int n1, double* cwork, long long cstride,
                      long long bandsz, double* Ainv, long long astride, int* status,
                      const int* act, cudaStream_t st);
template <typename T>
void bk_multidot(const T* V, size_t ld, int nv, const T* w, double* part, const VecTab& vt,
                 double* out, int ostride, const int* act, cudaStream_t st);
template <typename T>
void bk_multiaxpy(const T* V, size_t ld, int nv, const double* h, int hstride, T* w,
                  const VecTab& vt, const int* act, cudaStream_t st);
template <typename T>
void bk_scale(const T* x, const double* a, int astride, int mode, T* y, const VecTab& vt,
              const int* act, cudaStream_t st);
template <typename T>
void bk_start(const T* r, const double* nrm2, int nstride, T* v0, double* gv, int gstride,
              const VecTab& vt, const int* act, cudaStream_t st);
// x += eps * sum_{j < kcnt[p]} y[p][j] Z_j (kcnt == nullptr: one term)
template <typename T, typename Tx>
void bk_combine(const T* Z, size_t ld, const int* kcnt, const double* y, int ystride, double eps,
                Tx* x, const VecTab& vt, const int* act, cudaStream_t st);
void bk_copy(const double* src, double* dst, const VecTab& vt, const int* act, cudaStream_t st);
// Givens update of Hessenberg column j for every active problem; a problem
// whose residual estimate reaches its target (or maxit, or is not finite)
// is deactivated in gact.
void bk_givens(int nprob, int m, double* H, double* cs, double* sn, double* gv,
               const double* hcol, int j, double* resid, const double* target, int* kcnt,
               int* its, int maxit, int* gact, cudaStream_t st);
void bk_backsolve(int nprob, int m, const double* H, const double* gv, const int* kcnt, double* y,
                  const int* act, cudaStream_t st);
// P from level L + dlf - 1 to level L + dlf (work: node blocks of L + dlf)
template <typename T>
void bk_prolong_state(const BView<T>& v, const double* xc, double* xf, int ncomp, int zero_p,
                      int dlf, Work wk, const int* act, cudaStream_t st);
// R = P^T from level L + dlf to level L + dlf - 1 (work: node blocks of L + dlf - 1)
template <typename T>
void bk_restrict_full(const BView<T>& v, const double* bf, double* bc, int ncomp, int dlf,
                      Work wk, const int* act, cudaStream_t st);
// patch inputs of K x K-node patches (K = 3 or 5) on level L + (K == 3 ? 1 : 2)
template <typename T>
void bk_gather(const BView<T>& v, int K, int P, const int* pinst, const int* pcell,
               const double* xt, const double* r, const float* mean, const float* stdv,
               uint16_t* X, cudaStream_t st);
template <typename T>
void bk_scatter(const BView<T>& v, int K, const int* cell_patch, const float* out, int c_out,
                const double* xt, double* vcorr, Work wk, const int* act, cudaStream_t st);
// tile shape (cells per block) of pass shape s
void pass_shape_dims(int s, int* tcx, int* tcy);

class BatchBase {
 public:
  virtual ~BatchBase() = default;
  virtual int init() = 0;
  virtual int step(int mode, dnnmg_step_stats* stats) = 0;
  virtual int linearize(const double* x64) = 0;
  virtual int vcycle(const void* b, void* x) = 0;
  virtual int precision() const = 0;
};

}  // namespace dnnmg

struct dnnmg_batch;
std::unique_ptr<dnnmg::BatchBase> make_batch_engine(dnnmg_batch* b);
