// Batched engine: many independent channel problems of uneven size (own
// obstacle, viscosity, time step and finest level each) advanced by the same
// time-step algorithm as a single context -- Newton's method (Eq. 6) with
// right-preconditioned FGMRES and a multigrid V-cycle (Sec. 2.2), and for
// DNN-MG steps the network correction of Algorithm 1 -- with every
// stage of every problem issued as one launch for the whole batch.
//
// Lock-step control: all problems run Newton and FGMRES iterations together;
// a problem that has converged (or failed) is masked out of the following
// launches by its active flag.  The V-cycle is walked level by level from
// the finest level of the batch down to level 1; a launch at level k covers
// the problems that have level k, so each problem sees exactly its own
// V-cycle.  One FGMRES iteration (V-cycle, matvec, orthogonalisation, Givens
// update) is captured once per Krylov index as a CUDA graph and replayed;
// the host reads the per-problem active flags after each iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "batch.h"
#include "dnnmg_body.cuh"
#include "coarse_body.cuh"
#include "runtime.h"

using namespace dnnmg;

struct dnnmg_batch {
  std::vector<dnnmg_config> cfg;
  cudaStream_t st = nullptr;
  std::string err;
  std::unique_ptr<dnnmg::BatchBase> eng;
  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
};

namespace dnnmg {

namespace {

long long pad_to(long long n, long long q) { return (n + q - 1) / q * q; }

template <typename T>
class Batch final : public BatchBase {
 public:
  explicit Batch(dnnmg_batch* b) : B_(b), ust_(b->st) {}
  ~Batch() override {
    if (st_) cudaStreamSynchronize(st_);
    for (auto& g : graphs_)
      if (g) cudaGraphExecDestroy(g);
    if (st_) cudaStreamDestroy(st_);
    if (h_pin_) cudaFreeHost(h_pin_);
    if (h_mask_) cudaFreeHost(h_mask_);
    if (ev0_) cudaEventDestroy(ev0_);
    if (ev1_) cudaEventDestroy(ev1_);
  }

  int precision() const override { return sizeof(T) == 8 ? DNNMG_FP64 : DNNMG_MIXED; }

  int init() override;
  int step(int mode, dnnmg_step_stats* stats) override;
  int linearize(const double* x64) override;
  int vcycle(const void* b, void* x) override;

  int nprob() const { return n_; }
  long long length() const { return N_; }
  int level_of(int p) const { return L_[p]; }
  long long offset_of(int p) const { return off_[p]; }
  int get_state(int p, double* x);
  int set_state(int p, const double* x);
  int vcycle_one(int p, const void* b, void* x);
  int set_weights(const float* w);
  int set_feature_stats(const float* mean, const float* stdv);
  int get_fine_velocity(int p, double* v);
  Prof& prof() { return prof_; }
  int set_graphs(int on) {
    use_graphs_ = on != 0;
    return DNNMG_OK;
  }

 private:
  struct Table {
    int2* d = nullptr;
    int n = 0;
    Work w() const { return Work{d, n}; }
  };

  int fail(int code, const std::string& m) { return B_->fail(code, m); }
  // Work runs on an internal non-blocking stream (graph capture needs one);
  // every call first waits for the caller's stream, and every call returns
  // with the internal stream drained.
  void sync_in() {
    if (ust_) cudaStreamSynchronize(ust_);
    else cudaDeviceSynchronize();
  }
  int check(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DNNMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return DNNMG_OK;
  }
  Table make_table(const std::vector<int2>& items) {
    Table t;
    t.n = (int)items.size();
    if (t.n == 0) return t;
    t.d = mem_.alloc<int2>(items.size());
    if (t.d) cudaMemcpyAsync(t.d, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st_);
    return t;
  }
  // node blocks of level k of the problems with L >= k + m
  Table node_table(int k, int m) {
    std::vector<int2> it;
    for (int p = 0; p < n_; ++p)
      if (L_[p] >= k + m)
        for (int b = 0; b < cdiv(hl_[p][k].g.nn, kNB); ++b) it.push_back(make_int2(p, b));
    return make_table(it);
  }
  // node blocks of every problem's own level L + dl
  Table own_table(int dl) {
    std::vector<int2> it;
    for (int p = 0; p < n_; ++p)
      for (int b = 0; b < cdiv(hl_[p][L_[p] + dl].g.nn, kNB); ++b) it.push_back(make_int2(p, b));
    return make_table(it);
  }
  Table tile_table(int k, int shape) {
    int tcx = 16, tcy = 4;
    pass_shape_dims(shape, &tcx, &tcy);
    std::vector<int2> it;
    for (int p = 0; p < n_; ++p)
      if (L_[p] >= k) {
        const Grid& g = hl_[p][k].g;
        const int nt = cdiv(g.nx / 2 + 1, tcx) * cdiv(g.ny / 2 + 1, tcy);
        for (int b = 0; b < nt; ++b) it.push_back(make_int2(p, b));
      }
    return make_table(it);
  }
  Table setup_table(int k) {
    std::vector<int2> it;
    for (int p = 0; p < n_; ++p)
      if (L_[p] >= k) {
        const int nsb = cdiv(vanka_slots(hl_[p][k].g), kSetupCells);
        for (int b = 0; b < 4 * nsb; ++b) it.push_back(make_int2(p, b));
      }
    return make_table(it);
  }

  // synchronous, so that the pinned staging buffer can be reused at once
  int* upload_mask(const std::vector<int>& m, int* dst) {
    std::memcpy(h_mask_, m.data(), sizeof(int) * n_);
    cudaMemcpyAsync(dst, h_mask_, sizeof(int) * n_, cudaMemcpyHostToDevice, st_);
    cudaStreamSynchronize(st_);
    return dst;
  }
  int sync_read(const void* dev, void* host, size_t bytes) {
    cudaMemcpyAsync(h_pin_, dev, bytes, cudaMemcpyDeviceToHost, st_);
    if (cudaStreamSynchronize(st_) != cudaSuccess) return check("sync");
    std::memcpy(host, h_pin_, bytes);
    return DNNMG_OK;
  }

  void vcycle_all(const T* b, T* x, const int* act);
  void smooth(int k, const T* b, T* x, int sweeps, const int* act);
  void fgmres_iteration(int j);
  int linearize_masked(const int* act, bool coarse, bool precond);
  int solve(const int* nact_d, const std::vector<int>& nact, std::vector<int>& gits);
  int newton(const std::vector<int>& mask, std::vector<dnnmg_step_stats>& s);
  int norms(const double* v, const int* act, std::vector<double>& out);
  void old_rhs_top(const double* xo, double* f, const int* act);
  void correction();

  dnnmg_batch* B_;
  cudaStream_t ust_ = nullptr, st_ = nullptr;
  int n_ = 0, Lmax_ = 0, nL_ = 0, R_ = 0, m_ = 0, n1_ = 0;
  dnnmg_config c0_{};
  std::vector<int> L_;
  std::vector<std::vector<HostLevel>> hl_;
  std::vector<long long> off_, offF_, offM_;  // top, fine (L + R) and, for R = 2, L + 1
  long long N_ = 0, NF_ = 0, NM_ = 0;
  DevMem mem_;
  std::vector<BLev<T>> hlev_;
  BView<T> v_{};
  // work lists
  std::map<int, Table> node0_, node1_, tiles_, setup_;
  Table top_, fine_, mid_;
  int shape_ = 0;
  VecTab vt_{};
  // concatenated top-level vectors
  double *x64_ = nullptr, *xold64_ = nullptr, *f64_ = nullptr, *r64_ = nullptr;
  T *V_ = nullptr, *Z_ = nullptr, *wsol_ = nullptr, *rT_ = nullptr, *rcur_ = nullptr,
    *vbJ_ = nullptr;
  double* part_ = nullptr;
  // per-problem Krylov scalars
  double *H_ = nullptr, *cs_ = nullptr, *sn_ = nullptr, *gv_ = nullptr, *hcol_ = nullptr,
         *y_ = nullptr, *resid_ = nullptr, *target_ = nullptr, *one_ = nullptr, *nrm_ = nullptr;
  int *kcnt_ = nullptr, *its_ = nullptr, *gact_ = nullptr, *cact_ = nullptr, *nact_ = nullptr,
      *sel_ = nullptr, *status_ = nullptr;
  // coarse level
  double *cwork_ = nullptr, *Ainv_ = nullptr;
  long long cstride_ = 0, bandsz_ = 0, astride_ = 0;
  bool linearized_ = false, coarse_done_ = false;
  long long steps_taken_ = 0;
  // host staging
  void* h_pin_ = nullptr;
  int* h_mask_ = nullptr;
  cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
  Prof prof_;
  // graphs of one FGMRES iteration per Krylov index
  std::vector<cudaGraphExec_t> graphs_;
  std::vector<int> seen_;                 // eager runs of iteration j so far
  std::vector<unsigned long long> glaunch_;  // kernels in graph j
  bool use_graphs_ = true;
  // DNN-MG
  NetDims nd_{};
  bool net_ok_ = false;
  float* w_master_ = nullptr;
  PackedNet pk_{};
  int* net_status_ = nullptr;
  int P_ = 0;
  int *pinst_ = nullptr, *pcell_ = nullptr, *cell_patch_ = nullptr;
  double *xtF_ = nullptr, *ximpF_ = nullptr, *fF_ = nullptr, *rF_ = nullptr, *vcorr_ = nullptr,
         *bF_ = nullptr, *bL_ = nullptr, *midF_ = nullptr;  // midF_: level L + 1 (R = 2)
  uint16_t* X_ = nullptr;
  float *net_out_ = nullptr, *hid_ = nullptr, *feat_mean_ = nullptr, *feat_std_ = nullptr;
  bool have_vcorr_ = false, have_net_rhs_ = false;
};

template <typename T>
int Batch<T>::init() {
  const std::vector<dnnmg_config>& cf = B_->cfg;
  n_ = (int)cf.size();
  c0_ = cf[0];
  for (int p = 0; p < n_; ++p) {
    std::string e;
    if (int rc = check_config(cf[p], e)) return fail(rc, "problem " + std::to_string(p) + ": " + e);
    if (cf[p].obstacle_level != 0)
      return fail(DNNMG_ERR_ARG, "problem " + std::to_string(p) + ": only level-0 obstacle blocks");
    const dnnmg_config& c = cf[p];
    if (c.precision != c0_.precision || c.replaced_levels != c0_.replaced_levels ||
        c.gmres_m != c0_.gmres_m || c.gmres_maxit != c0_.gmres_maxit ||
        c.newton_max != c0_.newton_max || c.nu1 != c0_.nu1 || c.nu2 != c0_.nu2 ||
        c.omega != c0_.omega || c.eps_damp != c0_.eps_damp || c.newton_tol != c0_.newton_tol ||
        c.gmres_rtol != c0_.gmres_rtol || c.coarse_refresh != c0_.coarse_refresh ||
        c.precond_lag != c0_.precond_lag || c.fallback_newton_its != c0_.fallback_newton_its ||
        c.hidden != c0_.hidden || c.gru_layers != c0_.gru_layers ||
        c.mlp_width != c0_.mlp_width || c.net_bias != c0_.net_bias || c.net_inputs != 0)
      return fail(DNNMG_ERR_ARG, "problems of a batch may differ only in nu, dt, theta, alpha0, "
                                 "obstacle and level_solve (and take the patch features as "
                                 "network inputs)");
  }

  R_ = c0_.replaced_levels;
  m_ = c0_.gmres_m;
  L_.resize(n_);
  for (int p = 0; p < n_; ++p) {
    L_[p] = cf[p].level_solve;
    Lmax_ = std::max(Lmax_, L_[p]);
  }
  nL_ = Lmax_ + std::max(2, R_ + 1);
  if (cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking) != cudaSuccess)
    return fail(DNNMG_ERR_CUDA, "stream creation failed");
  if (cudaMallocHost(&h_pin_, (size_t)n_ * (2 * m_ + 4) * sizeof(double) + 4096) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&h_mask_), sizeof(int) * n_) != cudaSuccess)
    return fail(DNNMG_ERR_CUDA, "pinned allocation failed");
  cudaEventCreate(&ev0_);
  cudaEventCreate(&ev1_);
  // ---- levels and masks
  hl_.resize(n_);
  for (int p = 0; p < n_; ++p) {
    const int top = L_[p] + R_;
    for (int l = 0; l <= top; ++l) {
      hl_[p].push_back(make_level(l, cf[p].obstacle_i0, cf[p].obstacle_j0, 0));
      Grid& g = hl_[p].back().g;
      uint8_t* s = mem_.alloc<uint8_t>((size_t)g.nx * g.ny);
      uint8_t* f = mem_.alloc<uint8_t>(g.nn);
      if (!mem_.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
      cudaMemcpyAsync(s, hl_[p].back().solid.data(), hl_[p].back().solid.size(), cudaMemcpyHostToDevice, st_);
      cudaMemcpyAsync(f, hl_[p].back().flags.data(), hl_[p].back().flags.size(), cudaMemcpyHostToDevice, st_);
      g.solid = s;
      g.flags = f;
    }
  }
  // ---- offsets of the concatenated vectors
  off_.resize(n_);
  offF_.assign(n_, 0);
  offM_.assign(n_, 0);
  for (int p = 0; p < n_; ++p) {
    off_[p] = N_;
    N_ += pad_to(3LL * hl_[p][L_[p]].g.nn, kVB);
    if (R_) {
      offF_[p] = NF_;
      NF_ += pad_to(3LL * hl_[p][L_[p] + R_].g.nn, kVB);
    }
    if (R_ == 2) {
      offM_[p] = NM_;
      NM_ += pad_to(3LL * hl_[p][L_[p] + 1].g.nn, kVB);
    }
  }
  // ---- per-level records and constants
  hlev_.assign((size_t)n_ * nL_, BLev<T>{});
  std::vector<Sten<T>> hsT((size_t)n_ * nL_);
  std::vector<Sten<double>> hs64((size_t)n_ * nL_), hsx((size_t)n_ * nL_);
  std::vector<BPar> hpar(n_);
  for (int p = 0; p < n_; ++p) {
    const dnnmg_config& c = cf[p];
    for (int k = 1; k <= L_[p] + R_; ++k) {
      BLev<T>& l = hlev_[(size_t)p * nL_ + k];
      const Grid& g = hl_[p][k].g;
      l.g = g;
      hsT[(size_t)p * nL_ + k] = make_sten<T>(g.h, c);
      hs64[(size_t)p * nL_ + k] = make_sten<double>(g.h, c);
      hsx[(size_t)p * nL_ + k] = make_explicit_sten(g.h, c);
      if (k > L_[p]) {  // DNN-MG levels: geometry and offset only
        l.off = k == L_[p] + R_ ? offF_[p] : offM_[p];
        continue;
      }
      const size_t n3 = 3 * (size_t)g.nn, n2 = 2 * (size_t)g.nn;
      l.top = k == L_[p];
      l.off = l.top ? off_[p] : 0;
      if (!l.top) {
        l.x = mem_.alloc<T>(n3);
        l.b = mem_.alloc<T>(n3);
      }
      l.x2 = mem_.alloc<T>(n3);
      l.d = mem_.alloc<T>(n3);
      l.vb = mem_.alloc<T>(n2);
      l.vb64 = mem_.alloc<double>(n2);
      if (k >= 2) l.inv = mem_.alloc<T>((size_t)4 * 144 * vanka_slots(g));
    }
    BPar& pr = hpar[p];
    pr.inv_k = 1.0 / c.dt;
    pr.ecoef = 1.0 - c.theta;
    pr.nu = c.nu;
    pr.dt = c.dt;
    pr.L = L_[p];
    pr.explicit_on = c.theta != 1.0;
    {
      const FeatConsts fc = feat_consts(hl_[p][L_[p]].g.h, c.nu, c.dt, (1 << (R_ > 0 ? R_ : 1)) + 1);
      pr.feat_h = fc.h_rel;
      pr.feat_k = fc.k_rel;
      pr.feat_pe = fc.pe;
    }
  }
  if (!mem_.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  const Grid& g1 = hl_[0][1].g;
  if (!coarse_supported(g1)) return fail(DNNMG_ERR_ARG, "coarse level too large");
  n1_ = 3 * g1.nn;
  cstride_ = (long long)coarse_work_doubles(g1);
  bandsz_ = (long long)coarse_band_doubles(g1);
  astride_ = (long long)n1_ * n1_;
  cwork_ = mem_.alloc<double>((size_t)n_ * cstride_);
  Ainv_ = mem_.alloc<double>((size_t)n_ * astride_);
  // ---- top-level vectors and Krylov scalars
  x64_ = mem_.alloc<double>(N_);
  xold64_ = mem_.alloc<double>(N_);
  f64_ = mem_.alloc<double>(N_);
  r64_ = mem_.alloc<double>(N_);
  V_ = mem_.alloc<T>((size_t)(m_ + 1) * N_);
  Z_ = mem_.alloc<T>((size_t)m_ * N_);
  wsol_ = mem_.alloc<T>(N_);
  rT_ = mem_.alloc<T>(N_);
  rcur_ = mem_.alloc<T>(N_);
  vbJ_ = mem_.alloc<T>(N_);
  const int nblk = (int)(N_ / kVB);
  part_ = mem_.alloc<double>((size_t)(m_ + 1) * nblk);
  H_ = mem_.alloc<double>((size_t)n_ * (m_ + 1) * (m_ + 1));
  cs_ = mem_.alloc<double>((size_t)n_ * (m_ + 1));
  sn_ = mem_.alloc<double>((size_t)n_ * (m_ + 1));
  gv_ = mem_.alloc<double>((size_t)n_ * (m_ + 2));
  hcol_ = mem_.alloc<double>((size_t)n_ * (2 * m_ + 4));
  y_ = mem_.alloc<double>((size_t)n_ * (m_ + 1));
  resid_ = mem_.alloc<double>(n_);
  target_ = mem_.alloc<double>(n_);
  nrm_ = mem_.alloc<double>(n_);
  one_ = mem_.alloc<double>(1);
  kcnt_ = mem_.alloc<int>(n_);
  its_ = mem_.alloc<int>(n_);
  gact_ = mem_.alloc<int>(n_);
  cact_ = mem_.alloc<int>(n_);
  nact_ = mem_.alloc<int>(n_);
  sel_ = mem_.alloc<int>(n_);
  status_ = mem_.alloc<int>(n_);
  // vector blocks
  std::vector<int> vinst(nblk), vfirst(n_), vcount(n_);
  for (int p = 0; p < n_; ++p) {
    const long long len = pad_to(3LL * hl_[p][L_[p]].g.nn, kVB);
    vfirst[p] = (int)(off_[p] / kVB);
    vcount[p] = (int)(len / kVB);
    for (int b = 0; b < vcount[p]; ++b) vinst[vfirst[p] + b] = p;
  }
  int* dvi = mem_.alloc<int>(nblk);
  int* dvf = mem_.alloc<int>(n_);
  int* dvc = mem_.alloc<int>(n_);
  if (!mem_.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  cudaMemcpyAsync(dvi, vinst.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dvf, vfirst.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dvc, vcount.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, st_);
  vt_ = VecTab{dvi, dvf, dvc, nblk, n_};
  // ---- work lists
  for (int k = 1; k <= Lmax_; ++k) {
    node0_[k] = node_table(k, 0);
    node1_[k] = node_table(k, 1);
    if (k >= 2) {
      tiles_[k] = tile_table(k, shape_);
      setup_[k] = setup_table(k);
    }
  }
  top_ = own_table(0);
  // ---- DNN-MG state
  if (R_ >= 1) {
    fine_ = own_table(R_);
    if (R_ == 2) mid_ = own_table(1);
    const int K = (1 << R_) + 1;
    nd_.c_in = 4 * K * K + 4;
    nd_.c_out = 2 * K * K;
    nd_.hidden = c0_.hidden;
    nd_.layers = c0_.gru_layers;
    nd_.mlp = c0_.mlp_width;
    nd_.bias = c0_.net_bias;
    net_ok_ = net_supported(nd_);
    if (net_ok_) {
      std::vector<int> pi, pc, cp;
      for (int p = 0; p < n_; ++p) {
        const HostLevel& h = hl_[p][L_[p]];
        hpar[p].coff = (long long)cp.size();
        for (size_t c = 0; c < h.solid.size(); ++c) {
          if (h.solid[c]) {
            cp.push_back(-1);
            continue;
          }
          cp.push_back((int)pi.size());
          pi.push_back(p);
          pc.push_back((int)c);
        }
      }
      P_ = (int)pi.size();
      pinst_ = mem_.alloc<int>(P_);
      pcell_ = mem_.alloc<int>(P_);
      cell_patch_ = mem_.alloc<int>(cp.size());
      xtF_ = mem_.alloc<double>(NF_);
      ximpF_ = mem_.alloc<double>(NF_);
      fF_ = mem_.alloc<double>(NF_);
      rF_ = mem_.alloc<double>(NF_);
      vcorr_ = mem_.alloc<double>(NF_);
      bF_ = mem_.alloc<double>(NF_);
      if (R_ == 2) midF_ = mem_.alloc<double>(NM_);
      bL_ = mem_.alloc<double>(N_);
      X_ = mem_.alloc<uint16_t>((size_t)P_ * nd_.c_in);
      net_out_ = mem_.alloc<float>((size_t)P_ * nd_.c_out);
      hid_ = mem_.alloc<float>((size_t)nd_.layers * P_ * nd_.hidden);
      feat_mean_ = mem_.alloc<float>(nd_.c_in);
      feat_std_ = mem_.alloc<float>(nd_.c_in);
      const PackLayout pl = PackLayout::of(nd_);
      w_master_ = mem_.alloc<float>(nd_.num_params());
      pk_.w = mem_.alloc<uint16_t>(pl.total);
      pk_.w_elems = pl.total;
      pk_.bias_elems = (size_t)nd_.layers * 4 * nd_.hidden + nd_.mlp + nd_.nout();
      pk_.bias = mem_.alloc<float>(pk_.bias_elems);
      net_status_ = mem_.alloc<int>(4);
      if (!mem_.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
      cudaMemcpyAsync(pinst_, pi.data(), sizeof(int) * P_, cudaMemcpyHostToDevice, st_);
      cudaMemcpyAsync(pcell_, pc.data(), sizeof(int) * P_, cudaMemcpyHostToDevice, st_);
      cudaMemcpyAsync(cell_patch_, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice, st_);
      std::vector<float> zero(nd_.c_in, 0.0f), one(nd_.c_in, 1.0f);
      cudaMemcpyAsync(feat_mean_, zero.data(), sizeof(float) * nd_.c_in, cudaMemcpyHostToDevice, st_);
      cudaMemcpyAsync(feat_std_, one.data(), sizeof(float) * nd_.c_in, cudaMemcpyHostToDevice, st_);
      cudaMemsetAsync(hid_, 0, sizeof(float) * nd_.layers * P_ * nd_.hidden, st_);
      cudaMemsetAsync(w_master_, 0, sizeof(float) * nd_.num_params(), st_);
      cudaMemsetAsync(net_status_, 0, sizeof(int) * 4, st_);
      launch_pack_weights(nd_, w_master_, pk_, st_);
      cudaStreamSynchronize(st_);  // host vectors above go out of scope
    }
  }
  // ---- device records
  BLev<T>* dl = mem_.alloc<BLev<T>>(hlev_.size());
  Sten<T>* dsT = mem_.alloc<Sten<T>>(hsT.size());
  Sten<double>* ds64 = mem_.alloc<Sten<double>>(hs64.size());
  Sten<double>* dsx = mem_.alloc<Sten<double>>(hsx.size());
  BPar* dpar = mem_.alloc<BPar>(n_);
  if (!mem_.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  cudaMemcpyAsync(dl, hlev_.data(), sizeof(BLev<T>) * hlev_.size(), cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dsT, hsT.data(), sizeof(Sten<T>) * hsT.size(), cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(ds64, hs64.data(), sizeof(Sten<double>) * hs64.size(), cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dsx, hsx.data(), sizeof(Sten<double>) * hsx.size(), cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(dpar, hpar.data(), sizeof(BPar) * n_, cudaMemcpyHostToDevice, st_);
  v_ = BView<T>{dl, dsT, ds64, dsx, dpar, nL_};
  // ---- initial states (impulsive start) and zeroed Krylov storage
  cudaMemsetAsync(x64_, 0, sizeof(double) * N_, st_);
  cudaMemsetAsync(V_, 0, sizeof(T) * (size_t)(m_ + 1) * N_, st_);
  cudaMemsetAsync(Z_, 0, sizeof(T) * (size_t)m_ * N_, st_);
  for (T* a : {wsol_, rT_, rcur_, vbJ_}) cudaMemsetAsync(a, 0, sizeof(T) * N_, st_);
  for (double* a : {xold64_, f64_, r64_}) cudaMemsetAsync(a, 0, sizeof(double) * N_, st_);
  if (R_ >= 1 && net_ok_)
    for (double* a : {xtF_, ximpF_, fF_, rF_, vcorr_, bF_}) cudaMemsetAsync(a, 0, sizeof(double) * NF_, st_);
  for (int p = 0; p < n_; ++p) {
    const std::vector<double> x0 = initial_state(hl_[p][L_[p]].g);
    cudaMemcpyAsync(x64_ + off_[p], x0.data(), sizeof(double) * x0.size(), cudaMemcpyHostToDevice, st_);
    cudaStreamSynchronize(st_);
  }
  for (int* a : {kcnt_, its_, gact_, cact_, nact_, sel_, status_}) cudaMemsetAsync(a, 0, sizeof(int) * n_, st_);
  for (double* a : {resid_, target_, nrm_}) cudaMemsetAsync(a, 0, sizeof(double) * n_, st_);
  const double one = 1.0;
  cudaMemcpyAsync(one_, &one, sizeof(double), cudaMemcpyHostToDevice, st_);
  cudaStreamSynchronize(st_);
  graphs_.assign(m_, nullptr);
  seen_.assign(m_, 0);
  glaunch_.assign(m_, 0);
  return check("batch setup");
}

template <typename T>
void Batch<T>::smooth(int k, const T* b, T* x, int sweeps, const int* act) {
  int cur = 0;
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 4; ++colour) {
      const int p = prof_.begin(DNNMG_STAGE_VANKA_PASS, k, st_);
      bk_pass<T>(v_, k, colour, cur, 1 - cur, b, x, (T)c0_.omega, tiles_[k].w(), shape_, act, st_);
      prof_.end(p, st_);
      cur ^= 1;
    }
}

// One V(nu1, nu2) cycle of every active problem on its own finest level with
// x = 0 on entry (b, x in the top-level layout).
template <typename T>
void Batch<T>::vcycle_all(const T* b, T* x, const int* act) {
  for (int k = Lmax_; k >= 2; --k) {
    smooth(k, b, x, c0_.nu1, act);
    int p = prof_.begin(DNNMG_STAGE_DEFECT, k, st_);
    bk_defect<T>(v_, k, 0, b, x, node0_[k].w(), act, st_);
    prof_.end(p, st_);
    p = prof_.begin(DNNMG_STAGE_TRANSFER, k, st_);
    bk_restrict<T>(v_, k, node1_[k - 1].w(), act, st_);
    prof_.end(p, st_);
  }
  int p = prof_.begin(DNNMG_STAGE_COARSE_SOLVE, 1, st_);
  bk_coarse_solve<T>(v_, n_, n1_, Ainv_, astride_, b, x, act, st_);
  prof_.end(p, st_);
  for (int k = 2; k <= Lmax_; ++k) {
    p = prof_.begin(DNNMG_STAGE_TRANSFER, k, st_);
    bk_prolong<T>(v_, k, 0, x, node0_[k].w(), act, st_);
    prof_.end(p, st_);
    smooth(k, b, x, c0_.nu2, act);
  }
}

// Linearise the active problems at their current state: the FGMRES matvec
// always, the multigrid hierarchy (injection, Vanka inverses) if `precond`,
// the coarse factorisation if `coarse`.
template <typename T>
int Batch<T>::linearize_masked(const int* act, bool coarse, bool precond) {
  launch_cast<double, T>(x64_, vbJ_, N_, st_);
  if (!precond && linearized_) return check("linearize");
  bk_top_vb<T>(v_, x64_, top_.w(), act, st_);
  for (int k = Lmax_; k >= 2; --k) bk_inject_vb<T>(v_, k, node1_[k - 1].w(), act, st_);
  cudaMemsetAsync(status_, 0, sizeof(int) * n_, st_);
  for (int k = 1; k <= Lmax_; ++k) {
    bk_cast_vb<T>(v_, k, node0_[k].w(), act, st_);
    if (k >= 2) {
      const int p = prof_.begin(DNNMG_STAGE_VANKA_SETUP, k, st_);
      bk_setup<T>(v_, k, status_, setup_[k].w(), act, st_);
      prof_.end(p, st_);
    }
  }
  if (coarse || !coarse_done_) {
    const int p = prof_.begin(DNNMG_STAGE_COARSE_FACTOR, 1, st_);
    bk_coarse_factor<T>(v_, n_, n1_, cwork_, cstride_, bandsz_, Ainv_, astride_, status_, act, st_);
    prof_.end(p, st_);
    coarse_done_ = true;
  }
  linearized_ = true;
  return check("linearize");
}

template <typename T>
int Batch<T>::linearize(const double* x64) {
  (void)x64;
  sync_in();
  if (int rc = linearize_masked(nullptr, true, true)) return rc;
  std::vector<int> status(n_);
  if (int rc = sync_read(status_, status.data(), sizeof(int) * n_)) return rc;
  for (int p = 0; p < n_; ++p) {
    if (status[p] & 1) return fail(DNNMG_ERR_NUMERICAL, "singular local Vanka matrix");
    if (status[p] & 2) return fail(DNNMG_ERR_NUMERICAL, "singular coarse-level matrix");
  }
  return DNNMG_OK;
}

template <typename T>
int Batch<T>::vcycle(const void* b, void* x) {
  if (!linearized_) return fail(DNNMG_ERR_STATE, "vcycle before linearize");
  sync_in();
  launch_fill<T>(static_cast<T*>(x), T(0), N_, st_);
  vcycle_all(static_cast<const T*>(b), static_cast<T*>(x), nullptr);
  cudaStreamSynchronize(st_);
  return check("vcycle");
}

// FGMRES iteration j of every problem still active in gact_: Z_j = M^{-1}
// V_j (one V-cycle), V_{j+1} = A' Z_j orthogonalised by two CGS passes,
// Givens update and convergence test.
template <typename T>
void Batch<T>::fgmres_iteration(int j) {
  T* vj = V_ + (size_t)j * N_;
  T* zj = Z_ + (size_t)j * N_;
  T* w = V_ + (size_t)(j + 1) * N_;
  const int hs = 2 * m_ + 4;
  launch_fill<T>(zj, T(0), N_, st_);
  vcycle_all(vj, zj, gact_);
  int p = prof_.begin(DNNMG_STAGE_APPLY, Lmax_, st_);
  bk_apply<T>(v_, zj, vbJ_, w, top_.w(), gact_, st_);
  prof_.end(p, st_);
  p = prof_.begin(DNNMG_STAGE_KRYLOV, Lmax_, st_);
  bk_multidot<T>(V_, N_, j + 1, w, part_, vt_, hcol_, hs, gact_, st_);
  bk_multiaxpy<T>(V_, N_, j + 1, hcol_, hs, w, vt_, gact_, st_);
  bk_multidot<T>(V_, N_, j + 1, w, part_, vt_, hcol_ + j + 1, hs, gact_, st_);
  bk_multiaxpy<T>(V_, N_, j + 1, hcol_ + j + 1, hs, w, vt_, gact_, st_);
  bk_multidot<T>(w, N_, 1, w, part_, vt_, hcol_ + 2 * j + 2, hs, gact_, st_);
  // scale before the Givens update may deactivate a problem; the scaled
  // vector of a problem that has just converged is not used again
  bk_scale<T>(w, hcol_ + 2 * j + 2, hs, 2, w, vt_, gact_, st_);
  bk_givens(n_, m_, H_, cs_, sn_, gv_, hcol_, j, resid_, target_, kcnt_, its_, c0_.gmres_maxit,
            gact_, st_);
  prof_.end(p, st_);
}

// FGMRES(m) on the top level of the problems in nact: x64 += eps * w.
template <typename T>
int Batch<T>::solve(const int* nact_d, const std::vector<int>& nact, std::vector<int>& gits) {
  launch_cast<double, T>(r64_, rT_, N_, st_);
  launch_fill<T>(wsol_, T(0), N_, st_);
  cudaMemcpyAsync(rcur_, rT_, sizeof(T) * N_, cudaMemcpyDeviceToDevice, st_);
  cudaMemsetAsync(its_, 0, sizeof(int) * n_, st_);
  cudaMemcpyAsync(gact_, nact_d, sizeof(int) * n_, cudaMemcpyDeviceToDevice, st_);
  std::vector<int> gact(nact);
  bool first = true;
  const int hs = 2 * m_ + 4;
  while (true) {
    if (std::none_of(gact.begin(), gact.end(), [](int a) { return a != 0; })) break;
    cudaMemcpyAsync(cact_, gact_, sizeof(int) * n_, cudaMemcpyDeviceToDevice, st_);
    bk_multidot<T>(rcur_, N_, 1, rcur_, part_, vt_, hcol_, hs, gact_, st_);
    bk_start<T>(rcur_, hcol_, hs, V_, gv_, m_ + 2, vt_, gact_, st_);
    if (first) {
      first = false;
      std::vector<double> hc((size_t)n_ * hs);
      if (int rc = sync_read(hcol_, hc.data(), sizeof(double) * hc.size())) return rc;
      std::vector<double> tgt(n_, 0.0);
      bool changed = false;
      for (int p = 0; p < n_; ++p) {
        if (!gact[p]) continue;
        const double b2 = hc[(size_t)p * hs];
        if (!std::isfinite(b2)) return fail(DNNMG_ERR_NUMERICAL, "non-finite residual");
        tgt[p] = c0_.gmres_rtol * std::sqrt(b2);
        if (!(b2 > 0)) gact[p] = 0, changed = true;
      }
      std::memcpy(h_pin_, tgt.data(), sizeof(double) * n_);
      cudaMemcpyAsync(target_, h_pin_, sizeof(double) * n_, cudaMemcpyHostToDevice, st_);
      if (changed) {
        upload_mask(gact, gact_);
        cudaMemcpyAsync(cact_, gact_, sizeof(int) * n_, cudaMemcpyDeviceToDevice, st_);
      }
      cudaStreamSynchronize(st_);
      if (std::none_of(gact.begin(), gact.end(), [](int a) { return a != 0; })) break;
    }
    for (int j = 0; j < m_; ++j) {
      // the first run of iteration j is eager (it also sets kernel
      // attributes); later runs replay a graph captured on the second
      if (use_graphs_ && !prof_.on() && seen_[j] > 0) {
        if (!graphs_[j]) {
          cudaGraph_t g = nullptr;
          const unsigned long long l0 = launches();
          if (cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return check("graph capture");
          fgmres_iteration(j);
          if (cudaStreamEndCapture(st_, &g) != cudaSuccess) return check("graph capture");
          glaunch_[j] = launches() - l0;
          const cudaError_t e = cudaGraphInstantiate(&graphs_[j], g, 0);
          cudaGraphDestroy(g);
          if (e != cudaSuccess) return check("graph instantiate");
        } else {
          note_launches(glaunch_[j]);
        }
        cudaGraphLaunch(graphs_[j], st_);
      } else {
        fgmres_iteration(j);
        ++seen_[j];
      }
      if (int rc = sync_read(gact_, gact.data(), sizeof(int) * n_)) return rc;
      if (std::none_of(gact.begin(), gact.end(), [](int a) { return a != 0; })) break;
    }
    bk_backsolve(n_, m_, H_, gv_, kcnt_, y_, cact_, st_);
    bk_combine<T, T>(Z_, N_, kcnt_, y_, m_ + 1, 1.0, wsol_, vt_, cact_, st_);
    // restart from the true residual of the current iterate
    bk_defect_top<T>(v_, rT_, wsol_, vbJ_, rcur_, top_.w(), gact_, st_);
  }
  std::vector<double> res(n_);
  if (int rc = sync_read(resid_, res.data(), sizeof(double) * n_)) return rc;
  std::vector<int> its(n_);
  if (int rc = sync_read(its_, its.data(), sizeof(int) * n_)) return rc;
  for (int p = 0; p < n_; ++p)
    if (nact[p]) {
      gits[p] += its[p];
      if (its[p] > 0 && !std::isfinite(res[p]))
        return fail(DNNMG_ERR_NUMERICAL, "non-finite GMRES residual");
    }
  bk_combine<T, double>(wsol_, N_, nullptr, one_, 0, c0_.eps_damp, x64_, vt_, nact_d, st_);
  return check("fgmres");
}

template <typename T>
int Batch<T>::norms(const double* v, const int* act, std::vector<double>& out) {
  bk_multidot<double>(v, N_, 1, v, part_, vt_, nrm_, 1, act, st_);
  out.assign(n_, 0.0);
  if (int rc = sync_read(nrm_, out.data(), sizeof(double) * n_)) return rc;
  for (double& x : out) x = std::sqrt(x);
  return DNNMG_OK;
}

template <typename T>
void Batch<T>::old_rhs_top(const double* xo, double* f, const int* act) {
  bk_old_rhs<T>(v_, 0, xo, f, top_.w(), act, st_);
}

// Lock-step Newton on the problems with mask[p] != 0 (f64_ holds their
// right-hand sides).
template <typename T>
int Batch<T>::newton(const std::vector<int>& mask, std::vector<dnnmg_step_stats>& s) {
  std::vector<int> act(mask);
  int* act_d = upload_mask(act, nact_);
  int p = prof_.begin(DNNMG_STAGE_RESIDUAL, Lmax_, st_);
  bk_residual64<T>(v_, 0, x64_, f64_, r64_, top_.w(), act_d, st_);
  prof_.end(p, st_);
  std::vector<double> nrm;
  if (int rc = norms(r64_, act_d, nrm)) return rc;
  std::vector<int> gits(n_, 0), nits(n_, 0);
  for (int q = 0; q < n_; ++q)
    if (act[q]) s[q].res0 = nrm[q];
  int it = 0;
  while (true) {
    bool any = false;
    for (int q = 0; q < n_; ++q) {
      if (!act[q]) continue;
      if (!std::isfinite(nrm[q])) {
        s[q].status = DNNMG_ERR_NUMERICAL;
        act[q] = 0;
      } else if (nrm[q] <= c0_.newton_tol || nits[q] >= c0_.newton_max) {
        act[q] = 0;
      }
      any = any || act[q];
    }
    if (!any) break;
    act_d = upload_mask(act, nact_);
    const bool refresh = it == 0 && steps_taken_ % c0_.coarse_refresh == 0;
    const bool precond = it == 0 || !c0_.precond_lag;
    if (int rc = linearize_masked(act_d, refresh, precond)) return rc;
    if (precond) {
      std::vector<int> status(n_);
      if (int rc = sync_read(status_, status.data(), sizeof(int) * n_)) return rc;
      bool changed = false;
      for (int q = 0; q < n_; ++q)
        if (act[q] && status[q]) {
          s[q].status = DNNMG_ERR_NUMERICAL;
          act[q] = 0;
          changed = true;
        }
      if (changed) act_d = upload_mask(act, nact_);
    }
    if (int rc = solve(act_d, act, gits)) return rc;
    p = prof_.begin(DNNMG_STAGE_RESIDUAL, Lmax_, st_);
    bk_residual64<T>(v_, 0, x64_, f64_, r64_, top_.w(), act_d, st_);
    prof_.end(p, st_);
    std::vector<double> nn;
    if (int rc = norms(r64_, act_d, nn)) return rc;
    for (int q = 0; q < n_; ++q)
      if (act[q]) {
        nrm[q] = nn[q];
        ++nits[q];
      }
    ++it;
  }
  for (int q = 0; q < n_; ++q) {
    if (!mask[q]) continue;
    s[q].newton_its += nits[q];
    s[q].gmres_its += gits[q];
    s[q].res_final = nrm[q];
    if (s[q].status == DNNMG_OK && nrm[q] > c0_.newton_tol) s[q].status = DNNMG_ERR_NOT_CONVERGED;
  }
  return check("newton");
}

// the network correction of Algorithm 1 for every problem after the level-L solves.
template <typename T>
void Batch<T>::correction() {
  const Work wf = fine_.w();
  const int K = (1 << R_) + 1;
  const int pr = prof_.begin(DNNMG_STAGE_NETWORK, Lmax_, st_);
  // P once per replaced level (through level L + 1 when two are replaced)
  auto prolong_up = [&](const double* xc, double* xf, int ncomp, int zero_p) {
    if (R_ == 2) {
      bk_prolong_state<T>(v_, xc, midF_, ncomp, 0, 1, mid_.w(), nullptr, st_);
      bk_prolong_state<T>(v_, midF_, xf, ncomp, zero_p, 2, wf, nullptr, st_);
    } else {
      bk_prolong_state<T>(v_, xc, xf, ncomp, zero_p, 1, wf, nullptr, st_);
    }
  };
  if (!have_vcorr_) prolong_up(xold64_, vcorr_, 2, 1);
  prolong_up(x64_, xtF_, 3, 0);                                        // P
  bk_old_rhs<T>(v_, R_, vcorr_, fF_, wf, nullptr, st_);
  bk_copy_impose<T>(v_, R_, xtF_, ximpF_, wf, nullptr, st_);
  bk_residual64<T>(v_, R_, ximpF_, fF_, rF_, wf, nullptr, st_);      // input: fine residual
  bk_gather<T>(v_, K, P_, pinst_, pcell_, xtF_, rF_, feat_mean_, feat_std_, X_, st_);
  launch_patchnet_forward(nd_, pk_, X_, hid_, hid_, net_out_, P_, net_status_, st_);  // network
  bk_scatter<T>(v_, K, cell_patch_, net_out_, nd_.c_out, xtF_, vcorr_, wf, nullptr, st_);
  bk_old_rhs<T>(v_, R_, vcorr_, bF_, wf, nullptr, st_);               // Rhs
  cudaMemsetAsync(bL_, 0, sizeof(double) * N_, st_);
  if (R_ == 2) {                                                       // R, twice
    cudaMemsetAsync(midF_, 0, sizeof(double) * NM_, st_);
    bk_restrict_full<T>(v_, bF_, midF_, 2, 2, mid_.w(), nullptr, st_);
    bk_restrict_full<T>(v_, midF_, bL_, 2, 1, top_.w(), nullptr, st_);
  } else {
    bk_restrict_full<T>(v_, bF_, bL_, 2, 1, top_.w(), nullptr, st_);  // R
  }
  prof_.end(pr, st_);
  have_vcorr_ = have_net_rhs_ = true;
}

template <typename T>
int Batch<T>::step(int mode, dnnmg_step_stats* stats) {
  if (mode == DNNMG_NET && (R_ < 1 || !net_ok_))
    return fail(DNNMG_ERR_ARG, "DNN-MG steps need replaced_levels 1 or 2 and the default network");
  sync_in();
  std::vector<dnnmg_step_stats> s(n_);
  for (auto& x : s) x = dnnmg_step_stats{};
  cudaEventRecord(ev0_, st_);
  cudaMemcpyAsync(xold64_, x64_, sizeof(double) * N_, cudaMemcpyDeviceToDevice, st_);
  const bool use_net_rhs = mode == DNNMG_NET && have_net_rhs_;
  if (use_net_rhs)
    cudaMemcpyAsync(f64_, bL_, sizeof(double) * N_, cudaMemcpyDeviceToDevice, st_);
  else
    old_rhs_top(xold64_, f64_, nullptr);
  const std::vector<int> all(n_, 1);
  int rc = newton(all, s);
  if (rc == DNNMG_OK && use_net_rhs) {
    // problems whose corrected right-hand side slowed Newton down redo the
    // step without it
    std::vector<int> fb(n_, 0);
    bool any = false;
    for (int q = 0; q < n_; ++q)
      if (s[q].status != DNNMG_OK || s[q].newton_its > c0_.fallback_newton_its) {
        fb[q] = 1;
        any = true;
        s[q].fallback = 1;
        s[q].status = DNNMG_OK;
      }
    if (any) {
      int* fb_d = upload_mask(fb, sel_);
      bk_copy(xold64_, x64_, vt_, fb_d, st_);
      old_rhs_top(xold64_, f64_, fb_d);
      rc = newton(fb, s);
    }
  }
  if (rc == DNNMG_OK && mode == DNNMG_NET) {
    correction();
    if (int r2 = check("dnnmg correction")) rc = r2;
  }
  ++steps_taken_;
  cudaEventRecord(ev1_, st_);
  cudaEventSynchronize(ev1_);
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0_, ev1_);
  prof_.collect(st_);
  int worst = rc;
  for (int q = 0; q < n_; ++q) {
    s[q].ms = ms;
    if (rc != DNNMG_OK) s[q].status = rc;
    if (worst == DNNMG_OK && s[q].status != DNNMG_OK) worst = s[q].status;
  }
  if (stats) std::memcpy(stats, s.data(), sizeof(dnnmg_step_stats) * n_);
  if (mode == DNNMG_NET && rc == DNNMG_OK) {
    int ns = 0;
    cudaMemcpyAsync(h_pin_, net_status_, sizeof(int), cudaMemcpyDeviceToHost, st_);
    cudaStreamSynchronize(st_);
    std::memcpy(&ns, h_pin_, sizeof(int));
    if (ns & 4) {
      cudaMemsetAsync(net_status_, 0, sizeof(int), st_);
      return fail(DNNMG_ERR_TIMEOUT, "network: tensor-core wait timed out");
    }
  }
  return worst;
}

// One V-cycle of problem p alone: its right-hand side is placed at its
// offset in the first FGMRES basis vector, the cycle runs with only p active
// (the other problems' work is masked out) into the first search vector,
// and p's part is copied out.  Both vectors are free between steps.
template <typename T>
int Batch<T>::vcycle_one(int p, const void* b, void* x) {
  if (!linearized_) return fail(DNNMG_ERR_STATE, "vcycle before linearize");
  sync_in();
  const size_t n3 = 3 * (size_t)hl_[p][L_[p]].g.nn;
  std::vector<int> one(n_, 0);
  one[p] = 1;
  const int* act = upload_mask(one, sel_);
  T* bb = V_;
  T* xx = Z_;
  launch_fill<T>(xx, T(0), N_, st_);
  cudaMemcpyAsync(bb + off_[p], b, sizeof(T) * n3, cudaMemcpyDeviceToDevice, st_);
  vcycle_all(bb, xx, act);
  cudaMemcpyAsync(x, xx + off_[p], sizeof(T) * n3, cudaMemcpyDeviceToDevice, st_);
  cudaStreamSynchronize(st_);
  return check("vcycle_one");
}

template <typename T>
int Batch<T>::get_state(int p, double* x) {
  sync_in();
  cudaMemcpyAsync(x, x64_ + off_[p], sizeof(double) * 3 * hl_[p][L_[p]].g.nn,
                  cudaMemcpyDeviceToDevice, st_);
  cudaStreamSynchronize(st_);
  return check("get_state");
}

template <typename T>
int Batch<T>::set_state(int p, const double* x) {
  sync_in();
  cudaMemcpyAsync(x64_ + off_[p], x, sizeof(double) * 3 * hl_[p][L_[p]].g.nn,
                  cudaMemcpyDeviceToDevice, st_);
  std::vector<int> one(n_, 0);
  one[p] = 1;
  bk_copy_impose<T>(v_, 0, nullptr, x64_, top_.w(), upload_mask(one, sel_), st_);
  have_net_rhs_ = have_vcorr_ = false;
  steps_taken_ = 0;  // the next step refactors the coarse level
  if (hid_) cudaMemsetAsync(hid_, 0, sizeof(float) * nd_.layers * P_ * nd_.hidden, st_);
  cudaStreamSynchronize(st_);
  return check("set_state");
}

template <typename T>
int Batch<T>::set_weights(const float* w) {
  if (!net_ok_) return fail(DNNMG_ERR_STATE, "no DNN-MG network in this batch");
  cudaMemcpyAsync(w_master_, w, sizeof(float) * nd_.num_params(), cudaMemcpyHostToDevice, st_);
  launch_pack_weights(nd_, w_master_, pk_, st_);
  cudaStreamSynchronize(st_);
  return check("set_weights");
}

template <typename T>
int Batch<T>::set_feature_stats(const float* mean, const float* stdv) {
  if (!net_ok_) return fail(DNNMG_ERR_STATE, "no DNN-MG network in this batch");
  for (int k = 0; k < nd_.c_in; ++k)
    if (!(stdv[k] > 0.0f)) return fail(DNNMG_ERR_ARG, "feature std must be positive");
  cudaMemcpyAsync(feat_mean_, mean, sizeof(float) * nd_.c_in, cudaMemcpyHostToDevice, st_);
  cudaMemcpyAsync(feat_std_, stdv, sizeof(float) * nd_.c_in, cudaMemcpyHostToDevice, st_);
  cudaStreamSynchronize(st_);
  return check("set_feature_stats");
}

template <typename T>
int Batch<T>::get_fine_velocity(int p, double* v) {
  if (!have_vcorr_) return fail(DNNMG_ERR_STATE, "no DNN-MG step taken yet");
  sync_in();
  cudaMemcpyAsync(v, vcorr_ + offF_[p], sizeof(double) * 2 * hl_[p][L_[p] + R_].g.nn,
                  cudaMemcpyDeviceToDevice, st_);
  cudaStreamSynchronize(st_);
  return check("get_fine_velocity");
}

}  // namespace

}  // namespace dnnmg

std::unique_ptr<dnnmg::BatchBase> make_batch_engine(dnnmg_batch* b) {
  std::unique_ptr<dnnmg::BatchBase> e;
  if (b->cfg[0].precision == DNNMG_FP64)
    e = std::make_unique<dnnmg::Batch<double>>(b);
  else
    e = std::make_unique<dnnmg::Batch<float>>(b);
  return e;
}

// ---------------------------------------------------------------------------
// C ABI of the batched engine

namespace {
thread_local std::string g_batch_error;

// dispatch on the engine's precision
template <typename F>
int with_engine(dnnmg_batch* b, F&& f) {
  if (b->cfg[0].precision == DNNMG_FP64) return f(*static_cast<Batch<double>*>(b->eng.get()));
  return f(*static_cast<Batch<float>*>(b->eng.get()));
}
template <typename F>
int with_engine_c(const dnnmg_batch* b, F&& f) {
  if (b->cfg[0].precision == DNNMG_FP64)
    return f(*static_cast<const Batch<double>*>(b->eng.get()));
  return f(*static_cast<const Batch<float>*>(b->eng.get()));
}
}  // namespace

extern "C" {

int dnnmg_batch_setup(const dnnmg_config* cfgs, int n, void* stream, dnnmg_batch** out) {
  if (!out) return DNNMG_ERR_ARG;
  *out = nullptr;
  if (!cfgs || n < 1 || n > 4096) {
    g_batch_error = "need 1 <= n <= 4096 configurations";
    return DNNMG_ERR_ARG;
  }
  std::unique_ptr<dnnmg_batch> b(new dnnmg_batch());
  b->cfg.assign(cfgs, cfgs + n);
  b->st = (cudaStream_t)stream;
  b->eng = make_batch_engine(b.get());
  const int rc = b->eng->init();
  if (rc != DNNMG_OK) {
    g_batch_error = b->err;
    return rc;
  }
  g_batch_error.clear();
  *out = b.release();
  return DNNMG_OK;
}

int dnnmg_batch_destroy(dnnmg_batch* b) {
  delete b;
  return DNNMG_OK;
}

const char* dnnmg_batch_last_error(const dnnmg_batch* b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

int dnnmg_batch_size(const dnnmg_batch* b, int* n, int64_t* length) {
  if (!b || !n || !length) return DNNMG_ERR_ARG;
  return with_engine_c(b, [&](const auto& e) {
    *n = e.nprob();
    *length = e.length();
    return DNNMG_OK;
  });
}

int dnnmg_batch_layout(const dnnmg_batch* b, int inst, int* level, int64_t* offset) {
  if (!b || !level || !offset || inst < 0 || inst >= (int)b->cfg.size()) return DNNMG_ERR_ARG;
  return with_engine_c(b, [&](const auto& e) {
    *level = e.level_of(inst);
    *offset = e.offset_of(inst);
    return DNNMG_OK;
  });
}

int dnnmg_batch_get_state(dnnmg_batch* b, int inst, double* x) {
  if (!b || !x || inst < 0 || inst >= (int)b->cfg.size()) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.get_state(inst, x); });
}

int dnnmg_batch_set_state(dnnmg_batch* b, int inst, const double* x) {
  if (!b || !x || inst < 0 || inst >= (int)b->cfg.size()) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.set_state(inst, x); });
}

int dnnmg_batch_linearize(dnnmg_batch* b) {
  if (!b) return DNNMG_ERR_ARG;
  return b->eng->linearize(nullptr);
}

int dnnmg_batch_vcycle(dnnmg_batch* b, const void* rhs, void* x) {
  if (!b || !rhs || !x) return DNNMG_ERR_ARG;
  return b->eng->vcycle(rhs, x);
}

int dnnmg_batch_vcycle_inst(dnnmg_batch* b, int inst, const void* rhs, void* x) {
  if (!b || !rhs || !x || inst < 0 || inst >= (int)b->cfg.size()) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.vcycle_one(inst, rhs, x); });
}

int dnnmg_batch_step(dnnmg_batch* b, int mode, dnnmg_step_stats* stats) {
  if (!b) return DNNMG_ERR_ARG;
  if (mode != DNNMG_PLAIN && mode != DNNMG_NET) return b->fail(DNNMG_ERR_ARG, "unknown mode");
  return b->eng->step(mode, stats);
}

int dnnmg_batch_set_weights(dnnmg_batch* b, const float* w_host) {
  if (!b || !w_host) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.set_weights(w_host); });
}

int dnnmg_batch_set_feature_stats(dnnmg_batch* b, const float* mean_host, const float* std_host) {
  if (!b || !mean_host || !std_host) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.set_feature_stats(mean_host, std_host); });
}

int dnnmg_batch_get_fine_velocity(dnnmg_batch* b, int inst, double* v) {
  if (!b || !v || inst < 0 || inst >= (int)b->cfg.size()) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.get_fine_velocity(inst, v); });
}

int dnnmg_batch_graphs(dnnmg_batch* b, int on) {
  if (!b) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) { return e.set_graphs(on); });
}

int dnnmg_batch_profile(dnnmg_batch* b, int on) {
  if (!b) return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) {
    e.prof().enable(on != 0);
    return DNNMG_OK;
  });
}

int dnnmg_batch_profile_read(dnnmg_batch* b, int stage, int level, int64_t* launches,
                             double* ms) {
  if (!b || !ms || !launches || stage < 0 || stage >= dnnmg::kStages || level < -1 ||
      level >= dnnmg::kMaxLevels)
    return DNNMG_ERR_ARG;
  return with_engine(b, [&](auto& e) {
    double t = 0;
    long long c = 0;
    for (int l = 0; l < dnnmg::kMaxLevels; ++l)
      if (level < 0 || l == level) {
        t += e.prof().ms(stage, l);
        c += e.prof().count(stage, l);
      }
    *ms = t;
    *launches = c;
    return DNNMG_OK;
  });
}

}  // extern "C"
