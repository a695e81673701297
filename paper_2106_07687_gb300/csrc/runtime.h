// Host runtime of libdnnmg (internal): the context, its level hierarchy and
// the precision-templated multigrid / Krylov / Newton engine.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "../../include/dnnmg.h"
#include "kernels.h"
#include "patchnet.cuh"
#include "train.h"

namespace dnnmg {

struct HostLevel {
  int ell = 0;
  Grid g{};
  std::vector<uint8_t> solid, flags;
};

HostLevel make_level(int ell, int oi0, int oj0, int olev);
// whether some 2h stabilisation patch of the level is part solid
bool part_solid_patches(const HostLevel& L);
struct PatchPieces;
PatchPieces make_patch_pieces(double h, const dnnmg_config& c);
// DNNMG_OK, or an error code with the reason in err
int check_config(const dnnmg_config& c, std::string& err);
// impulsive start on a level: zero state with the inflow profile on x = 0
std::vector<double> initial_state(const Grid& g);
template <typename T>
Sten<T> make_sten(double h, const dnnmg_config& c);
Sten<double> make_explicit_sten(double h, const dnnmg_config& c);

// Owns device allocations; frees them on destruction.
class DevMem {
 public:
  ~DevMem() {
    for (void* p : ptrs_) cudaFree(p);
  }
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T) + 16) != cudaSuccess) {
      ok_ = false;
      return nullptr;
    }
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  bool ok() const { return ok_; }

 private:
  std::vector<void*> ptrs_;
  bool ok_ = true;
};

// Per-stage device timers: CUDA events recorded on the context's stream
// around kernel launches, read back after the stream has synchronised.
constexpr int kStages = 12;
class Prof {
 public:
  ~Prof() {
    for (cudaEvent_t e : ev_) cudaEventDestroy(e);
  }
  void enable(bool on) {
    on_ = on;
    reset();
    if (on && ev_.empty()) {
      ev_.resize(kPool);
      for (auto& e : ev_) cudaEventCreate(&e);
    }
  }
  bool on() const { return on_; }
  void reset() {
    recs_.clear();
    used_ = 0;
    for (auto& r : ms_) for (auto& v : r) v = 0;
    for (auto& r : cnt_) for (auto& v : r) v = 0;
  }
  // returns the record slot or -1
  int begin(int stage, int level, cudaStream_t st) {
    if (!on_ || used_ + 2 > kPool) return -1;
    const int e0 = used_;
    used_ += 2;
    cudaEventRecord(ev_[e0], st);
    recs_.push_back({stage, level, e0});
    return e0;
  }
  void end(int e0, cudaStream_t st) {
    if (e0 >= 0) cudaEventRecord(ev_[e0 + 1], st);
  }
  // records [from, to) of launches that turned out to do nothing (a
  // speculative FGMRES iteration after the cycle stopped) are not counted
  size_t mark() const { return recs_.size(); }
  void drop(size_t from, size_t to) {
    if (from < to && to <= recs_.size()) recs_.erase(recs_.begin() + from, recs_.begin() + to);
  }
  void collect(cudaStream_t st) {
    if (recs_.empty()) return;
    cudaStreamSynchronize(st);
    for (const Rec& r : recs_) {
      float t = 0;
      cudaEventElapsedTime(&t, ev_[r.e0], ev_[r.e0 + 1]);
      ms_[r.stage][r.level] += t;
      cnt_[r.stage][r.level] += 1;
    }
    recs_.clear();
    used_ = 0;
  }
  double ms(int stage, int level) const { return ms_[stage][level]; }
  long long count(int stage, int level) const { return cnt_[stage][level]; }

 private:
  struct Rec {
    int stage, level, e0;
  };
  static constexpr int kPool = 1 << 14;
  bool on_ = false;
  std::vector<cudaEvent_t> ev_;
  std::vector<Rec> recs_;
  int used_ = 0;
  double ms_[kStages][kMaxLevels] = {};
  long long cnt_[kStages][kMaxLevels] = {};
};

// Precision-independent interface of the solver engine.
class SolverBase {
 public:
  virtual ~SolverBase() = default;
  // coarse = false keeps the coarse-level factorisation of the previous call;
  // precond = false only updates the Jacobian of the FGMRES matvec.  With
  // report = false the setups' singularity flags are not read back (no host
  // synchronisation); they accumulate on the device until device_status.
  virtual int linearize(const double* x64, bool coarse, bool precond, bool report = true) = 0;
  virtual int apply(int k, const void* w, void* y) = 0;
  virtual int vcycle(int k, const void* b, void* x) = 0;
  // FGMRES on the finest level: w64 += eps * A'^{-1} r64 (approximately)
  virtual int solve(const double* r64, double* x64, double eps, int* its) = 0;
  virtual int precision() const = 0;
  // level from which the V-cycle runs as one persistent launch (0: none),
  // the kind of that launch (0: cooperative grid, 1: single cluster), and
  // the colour-pass tile shape chosen for a level
  virtual int split_level() const = 0;
  virtual int split_mode() const = 0;
  virtual int pass_shape(int level) const = 0;
  // recompute every level's stencil constants from the context's nu and dt
  // (after a change of either); the next linearisation refactors the coarse level
  virtual void set_physics() = 0;
  // device-side error bits of the smoother kernels (0: none; -1: CUDA error);
  // *setup receives the setups' singularity bits accumulated since
  // clear_setup_status (1: a local Vanka matrix, 2: the coarse matrix)
  virtual int device_status(int* setup = nullptr) = 0;
  virtual void clear_setup_status() = 0;
  // the device status words (4 ints) and the same answer as device_status
  // from their values already read (posted with a later residual norm)
  virtual const int* status_words() const = 0;
  virtual int status_from(const int st[4], int* setup) = 0;
};

std::unique_ptr<SolverBase> make_solver(struct ::dnnmg_ctx* ctx);

}  // namespace dnnmg

struct dnnmg_ctx {
  dnnmg_config cfg{};
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<dnnmg::HostLevel> lv;  // levels 0 .. L + replaced_levels
  std::vector<uint8_t*> d_solid, d_flags;
  dnnmg::DevMem mem;
  std::unique_ptr<dnnmg::SolverBase> solver;
  dnnmg::Sten<double> s64L{};  // FP64 constants of the finest solved level
  dnnmg::Sten<double> sxL{}, sxF{};  // explicit theta-scheme bracket on levels L, L+1
  // FP64 state of level L
  double* x64 = nullptr;
  double* xold64 = nullptr;
  double* f64 = nullptr;
  double* r64 = nullptr;
  double* dots = nullptr;      // small device scratch for reductions
  double* partials = nullptr;  // reduction partials
  double* h_scalars = nullptr; // pinned host scalars
  dnnmg::HostMail* mail_h = nullptr;  // mapped pinned mailbox: host view
  dnnmg::HostMail* mail_d = nullptr;  // and device view
  unsigned long long mail_seq = 0;  // number of the last post issued on st
  double *fpart = nullptr, *fout = nullptr;  // functionals: partial sums, results
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  dnnmg::Prof prof;
  long long steps_taken = 0;   // time steps since setup (coarse refresh schedule)
  int last_newton_its = 1;     // Newton iterations of the last Newton solve
  // patch network
  dnnmg::NetDims nd{};
  bool net_ok = false;
  float* w_master = nullptr;   // FP32 flat parameters
  dnnmg::PackedNet pk{};
  int* net_status = nullptr;
  // DNN-MG correction state (level L+1 fields)
  int P = 0;                       // patches = fluid cells of level L
  int* patch_cell = nullptr;       // [P] cell id of each patch
  int* cell_patch = nullptr;       // [nx_L * ny_L] patch id or -1
  dnnmg::Sten<double> s64F{};
  double *xtF = nullptr, *ximpF = nullptr, *fF = nullptr, *rF = nullptr, *vcorr = nullptr,
         *bF = nullptr, *bL = nullptr;
  double* midF = nullptr;  // level L+1 transfer buffer with two replaced levels
  uint16_t* X = nullptr;
  float *net_out = nullptr, *hid = nullptr, *feat_mean = nullptr, *feat_std = nullptr;
  bool have_net_rhs = false, have_vcorr = false;
  bool net_status_posted = false;  // the correction's status waits in mailbox iv[4]
  double* stat_partial = nullptr;  // [128][C_in][2] feature-statistics partials
  // training workspace (capacity cfg.train_batch x cfg.train_seq)
  dnnmg::TrainBufs tb{};
  float *tr_ypred = nullptr, *loss_dev = nullptr, *grad = nullptr, *adam_m = nullptr,
        *adam_v = nullptr, *cpart = nullptr;
  uint16_t *dyT = nullptr, *da1T = nullptr, *wT = nullptr;
  uint16_t* giT[dnnmg::kMaxLayers] = {};  // gate gradients of each layer (input side)
  uint16_t* ghT[dnnmg::kMaxLayers] = {};  // (hidden side)
  double* loss_part = nullptr;
  int tr_layout_B = -1, tr_layout_T = -1, adam_step = 0, tr_blocks_max = 0, tr_splits_max = 0;
  size_t cpart_floats = 0;

  ~dnnmg_ctx();
  int init();
  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  int check(const char* what);
  // the number of the next post on st
  unsigned long long mail_ticket() { return ++mail_seq; }
  // wait (host poll, bounded by the stream's progress) until post t landed
  int mail_wait(unsigned long long t, const char* what);
  dnnmg::Grid grid(int level) const { return lv[level].g; }
  int L() const { return cfg.level_solve; }
  // the level the network corrects: L + replaced_levels
  int fine_level() const { return cfg.level_solve + cfg.replaced_levels; }
  int lc() const { return cfg.level_coarse; }
  // mixed precision: the FP64 residuals evaluate the operator in double-float
  bool mixed() const { return cfg.precision == DNNMG_MIXED; }
  // r64 = f - A(x64) with |r64| posted to the mailbox (returns the post's
  // number), and the wait for it
  unsigned long long residual_norm_begin(const double* f, bool with_status = false);
  int residual_norm_end(unsigned long long t, double* nrm);
  double* norm_partials = nullptr;  // per-block sums of the residual launch
  unsigned* norm_counter = nullptr; // blocks done (zero between launches)

  int get_state(double* x);
  int set_state(const double* x);
  int linearize_api(const double* x);
  int apply_api(int level, const void* w, void* y, int precision);
  int vcycle_api(int level, const void* b, void* x, int precision);
  int residual_api(const double* x, const double* f, double* r);
  int step(int mode, dnnmg_step_stats* stats);
  int init_net();
  int set_weights(const float* w_host);
  int get_weights(float* w_host);
  int patch_infer(const uint16_t* x, float* h, float* out, int P);
  int net_check(const char* what);
  int init_dnnmg();
  // f = old-time right-hand side of Eq. 5 from x_old on level `level`
  void old_rhs(int level, const double* x_old, double* f, double* copy = nullptr);
  int dnnmg_correction();
  // xf = P xc (each replaced level once); with ximp, also ximp = xf with the
  // Dirichlet values imposed
  void prolong_up(const double* xc, double* xf, int ncomp, double* ximp = nullptr);
  void restrict_down(const double* bf, double* bc);
  int set_feature_stats(const float* mean, const float* stdv);
  int get_fine_velocity(double* v);
  int functionals(int level, const double* x, const double* x_old, double* out_host);
  int rel_errors(int level, const double* x, const double* x_ref, double* out_host);
  int get_patch_inputs(uint16_t* x);
  int init_train();
  int train_grad_impl(const uint16_t* X, const float* Y, int B, int T);
  int train_grad(const uint16_t* X, const float* Y, int B, int T, float* g, float* loss);
  int train_step(const uint16_t* X, const float* Y, int B, int T, float lr, float* loss);
  int reset_optimizer();
  int make_sample(const double* xf_prev, const double* xf_next, float* Xraw, float* Y,
                  dnnmg_step_stats* s);
  int feature_stats(const float* Xraw, long long rows, float* mean_h, float* std_h);
  int gather_batch(const float* Xraw, const float* Yc, const int* idx, int B, int T,
                   long long stride, uint16_t* Xb, float* Yb);
  int newton(const double* f, dnnmg_step_stats* st);
  // nu and dt of every stencil of this context (and of its corpus solver)
  void set_physics(double nu, double dt);
  // plain solver on the fine level, made by the first make_corpus call
  std::unique_ptr<dnnmg_ctx> corpus_fine;
  int make_corpus(int n_traj, const double* nu, int spinup_steps, double spinup_dt,
                  int relax_steps, int T, float* Xraw, float* Y);
};
