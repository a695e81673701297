// Host runtime: multigrid V-cycle, flexible GMRES and Newton time step
// (Sec. 2.2, Eq. 6, the Newton iteration of Algorithm 1), sequencing the kernels of this
// library on the context's stream.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "coarse_body.cuh"
#include "dnnmg_step.h"
#include "runtime.h"
#include "vcycle.h"

using namespace dnnmg;

namespace dnnmg {

namespace {

template <typename T>
class Solver final : public SolverBase {
 public:
  explicit Solver(dnnmg_ctx* c) : c_(c) {}
  ~Solver() override {
    for (cudaStream_t s : side_) cudaStreamDestroy(s);
    for (cudaEvent_t e : side_ev_) cudaEventDestroy(e);
    if (fork_ev_) cudaEventDestroy(fork_ev_);
  }

  int init() {
    const dnnmg_config& cfg = c_->cfg;
    st_ = c_->st;
    K_ = cfg.level_solve - cfg.level_coarse;
    lv_.resize(K_ + 1);
    for (int k = 0; k <= K_; ++k) {
      Lev& l = lv_[k];
      l.level = cfg.level_coarse + k;
      l.g = c_->grid(l.level);
      const size_t n3 = 3 * (size_t)l.g.nn, n2 = 2 * (size_t)l.g.nn;
      l.s = make_sten<T>(l.g.h, cfg);
      l.s64 = make_sten<double>(l.g.h, cfg);
      l.x = c_->mem.alloc<T>(n3);
      l.x2 = c_->mem.alloc<T>(n3);
      l.b = c_->mem.alloc<T>(n3);
      l.d = c_->mem.alloc<T>(n3);
      l.vb = c_->mem.alloc<T>(n2);
      l.vb64 = c_->mem.alloc<double>(n2);
      if (k > 0) l.inv = c_->mem.alloc<T>((size_t)4 * 144 * vanka_slots(l.g));
    }
    // streaming colour passes (FP32): a tensor map of every level's inverses
    if constexpr (sizeof(T) == 4) {
      for (int k = 1; k <= K_; ++k)
        lv_[k].stream_ok = lv_[k].inv && vanka_stream_grid(lv_[k].g) > 0 &&
                           make_vanka_tensor_map(lv_[k].tmap, (const float*)lv_[k].inv, lv_[k].g);
    }
    lin_.nlev = K_ + 1;
    lin_.off[0] = 0;
    for (int k = 0; k <= K_; ++k) {
      lin_.nnx[k] = lv_[k].g.nnx;
      lin_.nn[k] = lv_[k].g.nn;
      lin_.off[k + 1] = lin_.off[k] + lv_[k].g.nn;
      lin_.vb64[k] = lv_[k].vb64;
      lin_.vb[k] = lv_[k].vb;
    }
    const Grid& g0 = lv_[0].g;
    if (!coarse_supported(g0)) return c_->fail(DNNMG_ERR_ARG, "coarse level too large");
    // a level-1 obstacle at odd offsets leaves part-solid patches on the coarse level
    part_solid_ = part_solid_patches(c_->lv[lv_[0].level]);
    if (part_solid_) pieces_ = make_patch_pieces(g0.h, cfg);
    coarse_work_ = c_->mem.alloc<double>(coarse_work_doubles(g0));
    ainv_ = c_->mem.alloc<double>((size_t)9 * g0.nn * g0.nn);
    status_ = c_->mem.alloc<int>(4);
    if (status_) cudaMemsetAsync(status_, 0, 4 * sizeof(int), st_);  // fresh memory is not zero
    m_ = cfg.gmres_m;
    n_ = 3 * (size_t)lv_[K_].g.nn;
    V_ = c_->mem.alloc<T>((m_ + 1) * n_);
    Z_ = c_->mem.alloc<T>(m_ * n_);
    wsol_ = c_->mem.alloc<T>(n_);
    rT_ = c_->mem.alloc<T>(n_);
    rcur_ = c_->mem.alloc<T>(n_);
    H_ = c_->mem.alloc<double>((m_ + 1) * (m_ + 1));
    cs_ = c_->mem.alloc<double>(m_ + 1);
    sn_ = c_->mem.alloc<double>(m_ + 1);
    gv_ = c_->mem.alloc<double>(m_ + 2);
    hcol_ = c_->mem.alloc<double>(2 * m_ + 4);
    y_ = c_->mem.alloc<double>(m_ + 1);
    vbJ_ = c_->mem.alloc<T>(2 * (size_t)lv_[K_].g.nn);
    partials_ = c_->mem.alloc<double>(dots_partials(n_, 2 * m_ + 4));
    skip_ = c_->mem.alloc<int>(1);
    target_dev_ = c_->mem.alloc<double>(1);
    if (!c_->mem.ok()) return c_->fail(DNNMG_ERR_CUDA, "device allocation failed");
    // persistent sub-cycles: level table and one phase list per possible top level
    if (cfg.persistent_vcycle != 0) {
      std::vector<VLevel<T>> hv(K_ + 1);
      for (int k = 0; k <= K_; ++k)
        hv[k] = VLevel<T>{lv_[k].g, lv_[k].s, lv_[k].x, lv_[k].x2, lv_[k].b, lv_[k].d,
                          lv_[k].vb, lv_[k].inv};
      dlv_ = c_->mem.alloc<VLevel<T>>(K_ + 1);
      std::vector<Phase> all;
      for (int k = 0; k <= K_; ++k) {
        const std::vector<Phase> p = vcycle_phases(k, cfg.nu1, cfg.nu2);
        ph_off_.push_back((int)all.size());
        ph_n_.push_back((int)p.size());
        all.insert(all.end(), p.begin(), p.end());
      }
      dph_ = c_->mem.alloc<Phase>(all.size());
      if (!c_->mem.ok()) return c_->fail(DNNMG_ERR_CUDA, "device allocation failed");
      cudaMemcpyAsync(dlv_, hv.data(), sizeof(VLevel<T>) * hv.size(), cudaMemcpyHostToDevice, st_);
      cudaMemcpyAsync(dph_, all.data(), sizeof(Phase) * all.size(), cudaMemcpyHostToDevice, st_);
      cudaStreamSynchronize(st_);
      coarse_nd_ = 3 * lv_[0].g.nn;
      bool fits = true;
      for (int k = 0; k <= K_; ++k) fits = fits && vcycle_fits(ph_n_[k], k + 1);
      vgrid_ = fits ? vcycle_grid<T>(coarse_nd_) : 0;
      cluster_ = fits ? vcycle_cluster_size<T>(coarse_nd_) : 0;
      split_ = cfg.persistent_vcycle > 0 ? cfg.persistent_vcycle : -1;  // -1: tune later
      split_mode_ = cfg.persistent_mode >= 0 ? cfg.persistent_mode : (vgrid_ > 0 ? 0 : 1);
    }
    shape_.assign(K_ + 1, 0);
    {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev);
    }
    // side streams and events of the concurrent Vanka setups (levels 1..K-1)
    if (K_ > 1) {
      if (cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming) != cudaSuccess)
        return c_->fail(DNNMG_ERR_CUDA, "event creation failed");
      for (int k = 1; k < K_; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
          return c_->fail(DNNMG_ERR_CUDA, "stream creation failed");
        side_.push_back(s);
        side_ev_.push_back(e);
      }
    }
    return c_->check("solver init");
  }

  int precision() const override { return sizeof(T) == 8 ? DNNMG_FP64 : DNNMG_MIXED; }

  // Linearise every level at the velocity of x64 (level L): nodal injection
  // down the hierarchy, Vanka inverses, coarse LU and inverse.
  int linearize(const double* x64, bool coarse, bool precond, bool report) override {
    // the Jacobian of the FGMRES matvec always follows the current iterate
    linearized_j_ = true;
    if (!precond && linearized_) {
      launch_cast<double, T>(x64, vbJ_, 2 * (size_t)lv_[K_].g.nn, st_);
      return c_->check("linearize");
    }
    // every level's point (injection down the hierarchy, FP64 and T copies)
    // and the matvec's, in one launch
    launch_linearize_levels<T>(lin_, x64, vbJ_, report || !tuned_ ? status_ : nullptr, st_);
    // the levels' setups are independent and each leaves most of the GPU
    // idle: levels below the top run on side streams beside it
    const int p = c_->prof.begin(DNNMG_STAGE_VANKA_SETUP, lv_[K_].level, st_);
    const bool fork = !side_.empty() && !capturing();
    if (fork) cudaEventRecord(fork_ev_, st_);
    for (int k = K_; k > 0; --k) {
      cudaStream_t s = st_;
      if (fork && k < K_) {
        s = side_[k - 1];
        cudaStreamWaitEvent(s, fork_ev_, 0);
      }
      launch_vanka_setup<T>(lv_[k].g, lv_[k].s, lv_[k].vb, lv_[k].inv, status_, s);
      if (s != st_) {
        cudaEventRecord(side_ev_[k - 1], s);
        cudaStreamWaitEvent(st_, side_ev_[k - 1], 0);
      }
    }
    c_->prof.end(p, st_);
    if (coarse || !coarse_done_) {
      const int p = c_->prof.begin(DNNMG_STAGE_COARSE_FACTOR, lv_[0].level, st_);
      launch_coarse_factor(lv_[0].g, lv_[0].s64, lv_[0].vb64, coarse_work_, ainv_, status_, st_,
                           part_solid_ ? &pieces_ : nullptr);
      c_->prof.end(p, st_);
      coarse_done_ = true;
    }
    if (!report && tuned_) {
      linearized_ = true;
      return c_->check("linearize");
    }
    int status = 0;
    cudaMemcpyAsync(c_->h_scalars, status_, sizeof(int), cudaMemcpyDeviceToHost, st_);
    if (int rc = c_->check("linearize")) return rc;
    cudaStreamSynchronize(st_);
    std::memcpy(&status, c_->h_scalars, sizeof(int));
    linearized_ = true;
    if (!tuned_) {
      tune_split();
      tuned_ = true;
    }
    if (status & 1) return c_->fail(DNNMG_ERR_NUMERICAL, "singular local Vanka matrix");
    if (status & 2) return c_->fail(DNNMG_ERR_NUMERICAL, "singular coarse-level matrix");
    return DNNMG_OK;
  }

  int apply(int k, const void* w, void* y) override {
    if (!linearized_) return c_->fail(DNNMG_ERR_STATE, "apply before linearize");
    launch_apply<T>(lv_[k].g, lv_[k].s, static_cast<const T*>(w), k == K_ ? vbJ_ : lv_[k].vb,
                    static_cast<T*>(y), st_);
    return c_->check("apply");
  }

  int vcycle(int k, const void* b, void* x) override {
    if (!linearized_) return c_->fail(DNNMG_ERR_STATE, "vcycle before linearize");
    if (!cycle_ignores_x(k)) launch_fill<T>(static_cast<T*>(x), T(0), 3 * (size_t)lv_[k].g.nn, st_);
    cycle(k, static_cast<const T*>(b), static_cast<T*>(x));
    return c_->check("vcycle");
  }

  // FGMRES(m) with right preconditioning by one V-cycle; CGS with one
  // re-orthogonalisation; x64 += eps * w at the end.
  int solve(const double* r64, double* x64, double eps, int* its_out) override {
    const dnnmg_config& cfg = c_->cfg;
    int its = 0;
    double target = -1.0;
    bool done = false;
    while (!done) {
      // |r|^2 of the first cycle travels to the host beside the first
      // iteration's residual estimate (one wait for both)
      bool first = target < 0;
      HostMail* mail = first ? c_->mail_d : nullptr;
      const unsigned long long t0 = first ? c_->mail_ticket() : 0;
      // rounding of r, zero correction, |r|, V0 in one launch where the
      // cooperative grid fits, else the separate steps.  The fused start also
      // resets the device-side stop flag and sets the stopping target, which
      // lets the iterations run one ahead of the host (spec) where every
      // launch of an iteration can skip itself: the whole cycle one
      // cooperative launch and the cooperative Arnoldi step.
      bool spec = arnoldi_available<T>() && cycle_one_coop_launch(K_);
      if (launch_fgmres_begin<T>(r64, rT_, wsol_, rcur_, V_, n_, partials_, hcol_, gv_, first,
                                 mail, t0, st_, skip_, target_dev_, cfg.gmres_rtol) != 0) {
        spec = false;
        if (first) {
          launch_cast<double, T>(r64, rT_, n_, st_);
          launch_fill<T>(wsol_, T(0), n_, st_);
          cudaMemcpyAsync(rcur_, rT_, n_ * sizeof(T), cudaMemcpyDeviceToDevice, st_);
        }
        launch_multidot<T>(rcur_, n_, 1, rcur_, n_, partials_, hcol_, st_);
        launch_gmres_start<T>(rcur_, hcol_, V_, gv_, n_, st_, mail, t0);
      }
      // one iteration: preconditioner, matvec and Arnoldi step, whose
      // residual estimate goes to mailbox slot 2 + (jj & 1); with spec each
      // launch does nothing once an earlier iteration stopped the cycle on
      // the device (the same test as the host's below)
      auto enqueue = [&](int jj, int its_after) -> unsigned long long {
        T* vj = V_ + (size_t)jj * n_;
        T* zj = Z_ + (size_t)jj * n_;
        T* w = V_ + (size_t)(jj + 1) * n_;
        int* sk = spec ? skip_ : nullptr;
        if (!cycle_ignores_x(K_)) launch_fill<T>(zj, T(0), n_, st_);
        cycle(K_, vj, zj, sk);
        int p = c_->prof.begin(DNNMG_STAGE_APPLY, lv_[K_].level, st_);
        launch_apply<T>(lv_[K_].g, lv_[K_].s, zj, vbJ_, w, st_, sk);
        c_->prof.end(p, st_);
        p = c_->prof.begin(DNNMG_STAGE_KRYLOV, lv_[K_].level, st_);
        const unsigned long long ticket = c_->mail_ticket();
        const int slot = 2 + (jj & 1);
        if (launch_arnoldi_step<T>(V_, n_, jj, w, n_, partials_, hcol_, H_, m_ + 1, cs_, sn_, gv_,
                                   y_ + m_, st_, c_->mail_d, ticket, slot, sk, target_dev_,
                                   its_after, cfg.gmres_maxit) != 0) {
          launch_multidot<T>(V_, n_, jj + 1, w, n_, partials_, hcol_, st_);
          launch_multiaxpy<T>(V_, n_, jj + 1, hcol_, w, n_, st_);
          launch_multidot<T>(V_, n_, jj + 1, w, n_, partials_, hcol_ + jj + 1, st_);
          launch_multiaxpy<T>(V_, n_, jj + 1, hcol_ + jj + 1, w, n_, st_);
          launch_multidot<T>(w, n_, 1, w, n_, partials_, hcol_ + 2 * jj + 2, st_);
          launch_givens(H_, m_ + 1, cs_, sn_, gv_, hcol_, jj, y_ + m_, st_);
          launch_scale_dev<T>(w, hcol_ + 2 * jj + 2, 2, w, n_, st_);
          launch_post(c_->mail_d, ticket, y_ + m_, slot, 1, nullptr, 0, 0, st_);
        }
        c_->prof.end(p, st_);
        return ticket;
      };
      int k = 0;
      const int its0 = its;
      unsigned long long tcur = enqueue(0, its0 + 1);
      for (int j = 0; j < m_; ++j) {
        // is there an iteration after this one unless it converges?
        const bool ahead = j + 1 < m_ && its0 + j + 1 < cfg.gmres_maxit;
        unsigned long long tnext = 0;
        size_t rec0 = 0, rec1 = 0;  // its stage-timer records
        if (spec && ahead) {  // before the host's wait
          rec0 = c_->prof.mark();
          tnext = enqueue(j + 1, its0 + j + 2);
          rec1 = c_->prof.mark();
        }
        ++its;
        k = j + 1;
        // the residual estimate (and, in the first cycle, |r|^2 posted
        // by the cycle's start) from the host mailbox
        if (int rc = c_->mail_wait(tcur, "fgmres")) return rc;
        const double res = c_->mail_h->v[2 + (j & 1)];
        if (first) {
          first = false;
          const double b2 = c_->mail_h->v[1];
          if (!(b2 > 0)) {  // zero right-hand side: no update (the iteration is discarded)
            its = 0;
            k = 0;
            done = true;
            c_->prof.drop(rec0, rec1);
            break;
          }
          if (!std::isfinite(b2)) return c_->fail(DNNMG_ERR_NUMERICAL, "non-finite residual");
          target = cfg.gmres_rtol * std::sqrt(b2);
        }
        if (!std::isfinite(res)) return c_->fail(DNNMG_ERR_NUMERICAL, "non-finite GMRES residual");
        if (res <= target || its >= cfg.gmres_maxit) {
          done = true;
          c_->prof.drop(rec0, rec1);  // the iteration ahead did nothing
          break;
        }
        if (!spec && ahead) tnext = enqueue(j + 1, its0 + j + 2);
        tcur = tnext;
      }
      if (k == 0) break;
      if (done) {
        // y = H^-1 g and x64 += eps (wsol + Z y) in one launch
        launch_fgmres_finish<T>(H_, m_ + 1, gv_, k, Z_, n_, wsol_, eps, x64, n_, st_);
        break;
      }
      launch_backsolve(H_, m_ + 1, gv_, k, y_, st_);
      launch_combine<T, T>(Z_, n_, k, y_, 1.0, wsol_, n_, st_);
      // restart from the true residual of the current iterate
      launch_defect<T>(lv_[K_].g, lv_[K_].s, rT_, wsol_, vbJ_, rcur_, false, st_);
    }
    if (its_out) *its_out = its;
    return c_->check("fgmres");
  }

 private:
  struct Lev {
    int level = 0;
    Grid g{};
    Sten<T> s{};
    Sten<double> s64{};
    T *x = nullptr, *x2 = nullptr, *b = nullptr, *d = nullptr, *vb = nullptr, *inv = nullptr;
    double* vb64 = nullptr;
    alignas(64) unsigned char tmap[kTensorMapBytes] = {};  // TMA map of inv (FP32)
    bool stream_ok = false;  // the streaming colour pass can run on this level
    bool stream = false;     // and the autotuner chose it
  };

  // nu sweeps of four colour passes, ping-ponging between x and the level's
  // second buffer; an even number of passes leaves the result in x.
  void smooth(int k, const T* b, T* x, int sweeps) {
    Lev& l = lv_[k];
    T* cur = x;
    T* nxt = l.x2;
    for (int s = 0; s < sweeps; ++s)
      for (int colour = 0; colour < 4; ++colour) {
        const int p = c_->prof.begin(DNNMG_STAGE_VANKA_PASS, l.level, st_);
        if constexpr (sizeof(T) == 4) {
          if (l.stream)
            launch_vanka_pass_stream(l.tmap, l.g, l.s, colour, b, cur, l.vb, (T)c_->cfg.omega,
                                     nxt, status_ + 2, st_);
          else
            launch_vanka_pass<T>(l.g, l.s, colour, b, cur, l.vb, l.inv, (T)c_->cfg.omega, nxt,
                                 st_, shape_[k]);
        } else {
          launch_vanka_pass<T>(l.g, l.s, colour, b, cur, l.vb, l.inv, (T)c_->cfg.omega, nxt, st_,
                               shape_[k]);
        }
        c_->prof.end(p, st_);
        T* t = cur;
        cur = nxt;
        nxt = t;
      }
  }

  void set_physics() override {
    const dnnmg_config& cfg = c_->cfg;
    for (Lev& l : lv_) {
      l.s = make_sten<T>(l.g.h, cfg);
      l.s64 = make_sten<double>(l.g.h, cfg);
    }
    if (part_solid_) pieces_ = make_patch_pieces(lv_[0].g.h, cfg);
    if (dlv_) {
      std::vector<VLevel<T>> hv(K_ + 1);
      for (int k = 0; k <= K_; ++k)
        hv[k] = VLevel<T>{lv_[k].g, lv_[k].s, lv_[k].x, lv_[k].x2, lv_[k].b, lv_[k].d,
                          lv_[k].vb, lv_[k].inv};
      cudaMemcpyAsync(dlv_, hv.data(), sizeof(VLevel<T>) * hv.size(), cudaMemcpyHostToDevice, st_);
      cudaStreamSynchronize(st_);
    }
    coarse_done_ = false;
    linearized_ = linearized_j_ = false;
  }

  int split_level() const override { return split_ > 0 ? split_ : 0; }
  int split_mode() const override { return split_mode_; }
  int pass_shape(int level) const override {
    const int k = level - lv_[0].level;
    return k >= 0 && k <= K_ ? (lv_[k].stream ? kPassStream : shape_[k]) : -1;
  }
  int device_status(int* setup) override {
    int st[4] = {0, 0, 0, 0};
    const unsigned long long t = c_->mail_ticket();
    launch_post(c_->mail_d, t, nullptr, 0, 0, status_, 0, 4, st_);
    if (c_->mail_wait(t, "status") != DNNMG_OK) return -1;
    for (int i = 0; i < 4; ++i) st[i] = c_->mail_h->iv[i];
    return status_from(st, setup);
  }
  const int* status_words() const override { return status_; }
  int status_from(const int st[4], int* setup) override {
    if (st[2]) cudaMemsetAsync(status_ + 2, 0, sizeof(int), st_);  // reported once
    if (setup) *setup = st[0];
    return st[2];
  }
  void clear_setup_status() override { cudaMemsetAsync(status_, 0, sizeof(int), st_); }

  // Autotuner, run once at the first linearisation: (1) the tile shape of
  // the colour pass on every level, by timing four passes per shape; (2) the
  // level from which the cycle runs as one persistent launch and the kind of
  // that launch (cooperative grid or single cluster), by timing whole cycles
  // of the top level for every candidate (0 = one launch per stage); a lower
  // split replaces a higher one only when it is more than 2 % faster.
  void tune_split() {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof_on = c_->prof.on();
    if (prof_on) c_->prof.enable(false);
    auto time_ms = [&](auto&& f, int reps) {
      f();  // warm-up
      cudaEventRecord(e0, st_);
      for (int r = 0; r < reps; ++r) f();
      cudaEventRecord(e1, st_);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      return cudaGetLastError() == cudaSuccess ? ms : 1e30f;
    };
    for (int k = 1; k <= K_; ++k) {
      float best = 1e30f;
      int best_s = 0;
      lv_[k].stream = false;
      for (int sh = 0; sh < kPassShapes; ++sh) {
        shape_[k] = sh;
        const float ms = time_ms([&] { smooth(k, lv_[k].d, lv_[k].x, 1); }, 3);
        if (ms < best) best = ms, best_s = sh;
      }
      shape_[k] = best_s;
      if (lv_[k].stream_ok && c_->cfg.stream_pass >= 0) {
        lv_[k].stream = true;
        const float ms = time_ms([&] { smooth(k, lv_[k].d, lv_[k].x, 1); }, 3);
        lv_[k].stream = c_->cfg.stream_pass == 1 || ms < best;
      }
    }
    const int top = K_;
    if (split_ == -1) {
      split_ = 0;
      T* b = lv_[top].d;
      T* x = wsol_;
      launch_fill<T>(b, T(0), 3 * (size_t)lv_[top].g.nn, st_);
      float best = 1e30f;
      int best_s = 0, best_m = 0, best_cap = 0;
      for (int cand = lv_[top].level; cand >= 0; --cand) {
        if (cand > 0 && cand < lv_[0].level + 1) continue;
        for (int mode = 0; mode < 2; ++mode) {
          if (cand == 0 && mode == 1) continue;
          if (cand > 0 && c_->cfg.persistent_mode >= 0 && mode != c_->cfg.persistent_mode) continue;
          if (cand > 0 && ((mode == 0 && vgrid_ <= 0) || (mode == 1 && cluster_ <= 0))) continue;
          split_ = cand;
          split_mode_ = mode;
          // cooperative grids: also fewer blocks than tiles (cheaper grid
          // barriers, more tiles per block); 0 = one block per tile
          for (int cap : {0, 2, 1}) {
            if (cap > 0 && (mode != 0 || cand == 0)) continue;
            coop_cap_ = cap * sms_;
            persistent_failed_ = false;
            float ms = time_ms([&] { cycle(top, b, x); }, 5);
            if (persistent_failed_) ms = 1e30f;
            // candidates come from the highest split down: a lower split (more
            // launches) or a capped grid must be faster by more than the timing noise
            if (ms < 0.98f * best) best = ms, best_s = cand, best_m = mode, best_cap = coop_cap_;
          }
        }
      }
      split_ = best_s;
      split_mode_ = best_m;
      coop_cap_ = best_cap;
      persistent_failed_ = false;
    }
    if (prof_on) c_->prof.enable(true);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  // Whether cycle(k, ...) runs as one persistent launch whose first pass
  // starts from the zero iterate without reading x (then x need not be
  // zeroed on entry; a failed launch zeroes it before the per-stage cycle).
  bool cycle_ignores_x(int k) const {
    return split_ > 0 && lv_[k].level <= split_ && !persistent_failed_ &&
           (split_mode_ == 0 ? vgrid_ > 0 : cluster_ > 0) && c_->cfg.nu1 > 0 && k > 0;
  }

  // Whether the whole cycle on level k is one cooperative launch (which
  // can skip itself on the device; the per-stage launches of the levels
  // above a split cannot).
  bool cycle_one_coop_launch(int k) const {
    return split_ > 0 && lv_[k].level <= split_ && !persistent_failed_ && split_mode_ == 0 &&
           vgrid_ > 0;
  }

  // One V(nu1, nu2) cycle on level k for A x = b with x = 0 on entry (or any
  // x when cycle_ignores_x(k)).  Levels at or below split_ run their whole
  // sub-cycle as one cooperative launch; with skip, that launch does nothing
  // when *skip is set at its start (a speculative FGMRES iteration).
  void cycle(int k, const T* b, T* x, const int* skip = nullptr) {
    if (split_ > 0 && lv_[k].level <= split_ && !persistent_failed_ &&
        (split_mode_ == 0 ? vgrid_ > 0 : cluster_ > 0)) {
      const int p = c_->prof.begin(DNNMG_STAGE_VCYCLE, lv_[k].level, st_);
      int rc;
      if (split_mode_ == 0) {
        // one block per colour-pass tile of the sub-cycle's top level
        int blocks = vcycle_coop_tiles(lv_[k].g);
        blocks = blocks < 64 ? 64 : blocks;
        if (coop_cap_ > 0 && blocks > coop_cap_) blocks = coop_cap_;
        blocks = blocks > vgrid_ ? vgrid_ : blocks;
        rc = launch_vcycle_persistent<T>(dlv_, dph_ + ph_off_[k], ph_n_[k], k, b, x, ainv_,
                                         (T)c_->cfg.omega, blocks, coarse_nd_, st_, skip);
      } else {
        rc = launch_vcycle_cluster<T>(dlv_, dph_ + ph_off_[k], ph_n_[k], k, b, x, ainv_,
                                      (T)c_->cfg.omega, cluster_, coarse_nd_, st_);
      }
      c_->prof.end(p, st_);
      if (rc == 0) return;
      persistent_failed_ = true;  // fall back to one launch per stage
      cudaGetLastError();
      launch_fill<T>(x, T(0), 3 * (size_t)lv_[k].g.nn, st_);
    }
    Lev& l = lv_[k];
    if (k == 0) {
      const int p = c_->prof.begin(DNNMG_STAGE_COARSE_SOLVE, l.level, st_);
      launch_coarse_solve<T>(l.g, ainv_, b, x, st_);
      c_->prof.end(p, st_);
      return;
    }
    Lev& lc = lv_[k - 1];
    smooth(k, b, x, c_->cfg.nu1);
    int p = c_->prof.begin(DNNMG_STAGE_DEFECT, l.level, st_);
    launch_defect<T>(l.g, l.s, b, x, l.vb, l.d, true, st_);
    c_->prof.end(p, st_);
    p = c_->prof.begin(DNNMG_STAGE_TRANSFER, l.level, st_);
    launch_restrict<T>(l.g, lc.g, l.d, lc.b, st_);
    launch_fill<T>(lc.x, T(0), 3 * (size_t)lc.g.nn, st_);
    c_->prof.end(p, st_);
    cycle(k - 1, lc.b, lc.x);
    p = c_->prof.begin(DNNMG_STAGE_TRANSFER, l.level, st_);
    launch_prolong_add<T>(l.g, lc.g, lc.x, x, st_);
    c_->prof.end(p, st_);
    smooth(k, b, x, c_->cfg.nu2);
  }

  dnnmg_ctx* c_;
  cudaStream_t st_ = nullptr;
  int K_ = 0, m_ = 0;
  size_t n_ = 0;
  std::vector<Lev> lv_;
  double *coarse_work_ = nullptr, *ainv_ = nullptr;
  bool part_solid_ = false;  // the coarse level has part-solid stabilisation patches
  PatchPieces pieces_{};
  int* status_ = nullptr;
  T *V_ = nullptr, *Z_ = nullptr, *wsol_ = nullptr, *rT_ = nullptr, *rcur_ = nullptr;
  double *H_ = nullptr, *cs_ = nullptr, *sn_ = nullptr, *gv_ = nullptr, *hcol_ = nullptr,
         *y_ = nullptr, *partials_ = nullptr;
  int* skip_ = nullptr;            // device-side stop flag of an FGMRES cycle
  double* target_dev_ = nullptr;   // its stopping target rtol |r0|
  bool linearized_ = false, linearized_j_ = false;
  bool coarse_done_ = false;
  T* vbJ_ = nullptr;  // top-level linearisation of the FGMRES matvec
  LinLevels<T> lin_ = {};  // every level's linearisation buffers
  VLevel<T>* dlv_ = nullptr;
  std::vector<cudaStream_t> side_;   // side_[k - 1]: setup of level k < K
  std::vector<cudaEvent_t> side_ev_;
  cudaEvent_t fork_ev_ = nullptr;
  bool capturing() const {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st_, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
  }
  Phase* dph_ = nullptr;
  std::vector<int> ph_off_, ph_n_;
  int vgrid_ = 0, coarse_nd_ = 0, cluster_ = 0;
  int split_ = 0;  // levels <= split_ (> 0) run as one persistent launch; -1: not tuned yet
  int split_mode_ = 0;        // 0: cooperative grid, 1: single cluster
  int coop_cap_ = 0;          // most blocks of the cooperative grid (0: one per tile)
  int sms_ = 0;               // multiprocessors of the device
  std::vector<int> shape_;    // colour-pass tile shape per level
  bool tuned_ = false;
  bool persistent_failed_ = false;
};

}  // namespace

std::unique_ptr<SolverBase> make_solver(dnnmg_ctx* ctx) {
  if (ctx->cfg.precision == DNNMG_FP64) {
    auto s = std::make_unique<Solver<double>>(ctx);
    if (s->init() != DNNMG_OK) return nullptr;
    return s;
  }
  auto s = std::make_unique<Solver<float>>(ctx);
  if (s->init() != DNNMG_OK) return nullptr;
  return s;
}

}  // namespace dnnmg

// ---------------------------------------------------------------------------
// context

dnnmg_ctx::~dnnmg_ctx() {
  if (st) cudaStreamSynchronize(st);
  solver.reset();
  if (h_scalars) cudaFreeHost(h_scalars);
  if (mail_h) cudaFreeHost(mail_h);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

int dnnmg_ctx::check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DNNMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return DNNMG_OK;
}

namespace dnnmg {

namespace {
int fail_msg(std::string& err, int code, const char* msg) {
  err = msg;
  return code;
}
}  // namespace

int check_config(const dnnmg_config& c, std::string& err) {
  if (!(c.nu > 0) || !(c.dt > 0) || !(c.alpha0 >= 0) || !(c.theta > 0 && c.theta <= 1))
    return fail_msg(err, DNNMG_ERR_ARG, "nu, dt, theta or alpha0 out of range");
  if (c.level_coarse < 1 || c.level_coarse > c.level_solve || c.level_solve > 9)
    return fail_msg(err, DNNMG_ERR_ARG, "need 1 <= level_coarse <= level_solve <= 9");
  if (c.level_coarse != 1) return fail_msg(err, DNNMG_ERR_ARG, "the coarse direct solve supports level 1");
  if (c.replaced_levels < 0 || c.replaced_levels > 2 || c.level_solve + c.replaced_levels > 10)
    return fail_msg(err, DNNMG_ERR_ARG, "replaced_levels must be 0, 1 or 2");
  if (c.obstacle_level != 0 && c.obstacle_level != 1)
    return fail_msg(err, DNNMG_ERR_ARG, "obstacle_level must be 0 or 1");
  if (c.obstacle_level == 0 && c.obstacle_i0 >= 0 &&
      (c.obstacle_i0 < 1 || c.obstacle_i0 > 13 || c.obstacle_j0 < 1 || c.obstacle_j0 > 1))
    return fail_msg(err, DNNMG_ERR_ARG, "obstacle must be a 2x2 level-0 block with 1 <= i0 <= 13, j0 = 1");
  // a one-cell strip between the square and the inflow, or between the
  // square and a wall with the square at an even level-1 offset along it,
  // has no free velocity node on level 1 and leaves the coarse problem
  // singular: those positions are refused
  if (c.obstacle_level == 1 && c.obstacle_i0 >= 0 &&
      (c.obstacle_i0 < 2 || c.obstacle_i0 > 27 || c.obstacle_j0 < 1 || c.obstacle_j0 > 3 ||
       (c.obstacle_j0 != 2 && c.obstacle_i0 % 2 == 0)))
    return fail_msg(err, DNNMG_ERR_ARG,
                    "an obstacle snapped to level 1 needs 2 <= i0 <= 27, 1 <= j0 <= 3 and j0 = 2 or "
                    "i0 odd (level-1 cells; other positions make the level-1 problem singular)");
  if (c.obstacle_level == 1 && c.level_solve < 2)
    return fail_msg(err, DNNMG_ERR_ARG, "a level-1 obstacle needs level_solve >= 2");
  if (c.precision != DNNMG_FP64 && c.precision != DNNMG_MIXED)
    return fail_msg(err, DNNMG_ERR_ARG, "unknown precision");
  if (c.gmres_m < 1 || c.gmres_m > 40 || c.gmres_maxit < 1 || c.newton_max < 1 || c.nu1 < 0 ||
      c.nu2 < 0 || c.coarse_refresh < 1 || c.persistent_mode < -1 || c.persistent_mode > 1 ||
      c.lps_mode < 0 || c.lps_mode > 2)
    return fail_msg(err, DNNMG_ERR_ARG, "solver parameters out of range");
  return DNNMG_OK;
}

std::vector<double> initial_state(const Grid& g) {
  // impulsive start: zero state, then the inflow profile on x = 0
  std::vector<double> x0(3 * (size_t)g.nn, 0.0);
  for (int j = 0; j <= g.ny; ++j) {
    const double y = j * g.h;
    x0[(size_t)j * g.nnx] = 6.0 * y * (1.0 - y);
  }
  return x0;
}

}  // namespace dnnmg

int dnnmg_ctx::init() {
  const dnnmg_config& c = cfg;
  if (int rc = check_config(c, err)) return rc;
  const int nlev = c.level_solve + c.replaced_levels + 1;
  for (int l = 0; l < nlev; ++l)
    lv.push_back(make_level(l, c.obstacle_i0, c.obstacle_j0, c.obstacle_level));
  for (int l = 0; l < nlev; ++l) {
    Grid& g = lv[l].g;
    uint8_t* s = mem.alloc<uint8_t>((size_t)g.nx * g.ny);
    uint8_t* f = mem.alloc<uint8_t>(g.nn);
    if (!mem.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
    cudaMemcpyAsync(s, lv[l].solid.data(), lv[l].solid.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(f, lv[l].flags.data(), lv[l].flags.size(), cudaMemcpyHostToDevice, st);
    g.solid = s;
    g.flags = f;
  }
  if (cudaMallocHost(&h_scalars, 64 * sizeof(double)) != cudaSuccess)
    return fail(DNNMG_ERR_CUDA, "pinned allocation failed");
  if (cudaHostAlloc(&mail_h, sizeof(HostMail), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(&mail_d, mail_h, 0) != cudaSuccess)
    return fail(DNNMG_ERR_CUDA, "mapped pinned allocation failed");
  mail_h->seq = 0;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  const Grid gL = grid(L());
  const size_t n3 = 3 * (size_t)gL.nn;
  x64 = mem.alloc<double>(n3);
  xold64 = mem.alloc<double>(n3);
  f64 = mem.alloc<double>(n3);
  r64 = mem.alloc<double>(n3);
  dots = mem.alloc<double>(64);
  partials = mem.alloc<double>(dots_partials(n3, 4));
  fpart = mem.alloc<double>(4 * kFnBlocks);
  fout = mem.alloc<double>(4);
  norm_partials = mem.alloc<double>(residual_blocks(gL));
  norm_counter = mem.alloc<unsigned>(1);
  if (!mem.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  cudaMemsetAsync(norm_counter, 0, sizeof(unsigned), st);
  s64L = make_sten<double>(gL.h, cfg);
  sxL = make_explicit_sten(gL.h, cfg);
  if (cfg.replaced_levels > 0) sxF = make_explicit_sten(grid(fine_level()).h, cfg);
  const std::vector<double> x0 = initial_state(gL);
  cudaMemcpyAsync(x64, x0.data(), n3 * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  if (int rc = check("setup")) return rc;
  solver = make_solver(this);
  if (!solver) return err.empty() ? fail(DNNMG_ERR_CUDA, "solver setup failed") : DNNMG_ERR_CUDA;
  if (int rc = init_net()) return rc;
  if (int rc = init_dnnmg()) return rc;
  if (int rc = init_train()) return rc;
  return check("setup");
}

int dnnmg_ctx::init_train() {
  if (cfg.train_batch <= 0 || cfg.train_seq <= 0 || !net_ok) return DNNMG_OK;
  const size_t B = cfg.train_batch, T = cfg.train_seq, K = B * T, Kh = (T + 1) * B;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  tr_blocks_max = sms;
  tr_splits_max = 160;
  const int H = nd.hidden, NL = nd.layers, MG = gate_rows(nd);
  tb.act = mem.alloc<float>(K * act_size(H, NL));
  tb.xT = mem.alloc<uint16_t>((size_t)(nd.kx0() + 16) * K);
  for (int l = 0; l < NL; ++l) tb.hT[l] = mem.alloc<uint16_t>((size_t)(H + 16) * Kh);
  tb.y1T = mem.alloc<uint16_t>(144 * K);
  tr_ypred = mem.alloc<float>(K * nd.c_out);
  dyT = mem.alloc<uint16_t>(128 * K);
  da1T = mem.alloc<uint16_t>(128 * K);
  for (int l = 0; l < NL; ++l) {
    giT[l] = mem.alloc<uint16_t>((size_t)MG * K);
    ghT[l] = mem.alloc<uint16_t>((size_t)MG * K);
  }
  loss_part = mem.alloc<double>(tr_blocks_max);
  loss_dev = mem.alloc<float>(4);
  grad = mem.alloc<float>(nd.num_params());
  adam_m = mem.alloc<float>(nd.num_params());
  adam_v = mem.alloc<float>(nd.num_params());
  cpart_floats = (size_t)tr_splits_max * 256 * 144;
  cpart = mem.alloc<float>(cpart_floats);
  wT = mem.alloc<uint16_t>(BwdPack::of(nd).total);
  if (!mem.ok()) return fail(DNNMG_ERR_CUDA, "training workspace allocation failed");
  return reset_optimizer();
}

int dnnmg_ctx::reset_optimizer() {
  if (!adam_m) return fail(DNNMG_ERR_STATE, "no training workspace (set train_batch, train_seq)");
  cudaMemsetAsync(adam_m, 0, sizeof(float) * nd.num_params(), st);
  cudaMemsetAsync(adam_v, 0, sizeof(float) * nd.num_params(), st);
  adam_step = 0;
  return check("reset_optimizer");
}

namespace {
// BF16 one in rows [r0, r1) of a row-major [rows][ld] array
void fill_rows_one(uint16_t* a, size_t ld, int r0, int r1, cudaStream_t st) {
  launch_fill<uint16_t>(a + (size_t)r0 * ld, (uint16_t)0x3F80, (size_t)(r1 - r0) * ld, st);
}
}  // namespace

int dnnmg_ctx::train_grad_impl(const uint16_t* Xd, const float* Yd, int B, int T) {
  if (!grad) return fail(DNNMG_ERR_STATE, "no training workspace (set train_batch, train_seq)");
  if (B < 16 || B % 16 || B > cfg.train_batch || T < 1 || T > cfg.train_seq)
    return fail(DNNMG_ERR_ARG, "need B % 16 == 0, 16 <= B <= train_batch, 1 <= T <= train_seq");
  const size_t K = (size_t)B * T, Kh = (size_t)(T + 1) * B;
  const int H = nd.hidden, NL = nd.layers, MG = gate_rows(nd);
  if (B != tr_layout_B || T != tr_layout_T) {
    cudaMemsetAsync(tb.xT, 0, 2 * (size_t)(nd.kx0() + 16) * K, st);
    for (int l = 0; l < NL; ++l) {
      cudaMemsetAsync(tb.hT[l], 0, 2 * (size_t)(H + 16) * Kh, st);
      cudaMemsetAsync(giT[l], 0, 2 * (size_t)MG * K, st);
      cudaMemsetAsync(ghT[l], 0, 2 * (size_t)MG * K, st);
      fill_rows_one(tb.hT[l], Kh, H, H + 1, st);
    }
    cudaMemsetAsync(tb.y1T, 0, 2 * 144 * K, st);
    cudaMemsetAsync(dyT, 0, 2 * 128 * K, st);
    fill_rows_one(tb.xT, K, nd.c_in, nd.c_in + 1, st);
    fill_rows_one(tb.y1T, K, 128, 129, st);
    tr_layout_B = B;
    tr_layout_T = T;
  }
  const int p = prof.begin(DNNMG_STAGE_TRAIN, 0, st);
  launch_pack_backward(nd, w_master, wT, st);
  launch_patchnet_train_forward(nd, pk, Xd, B, T, tr_ypred, tb, net_status, st);
  BwdArgs a{};
  a.act = tb.act;
  a.ypred = tr_ypred;
  a.Y = Yd;
  a.B = B;
  a.T = T;
  a.scale = (float)(2.0 / ((double)B * T * nd.c_out));
  a.dyT = dyT;
  a.da1T = da1T;
  for (int l = 0; l < NL; ++l) {
    a.giT[l] = giT[l];
    a.ghT[l] = ghT[l];
  }
  a.loss_partial = loss_part;
  a.status = net_status;
  const int nb = std::min((B + 127) / 128, tr_blocks_max);
  launch_patchnet_backward(nd, wT, a, nb, st);
  launch_loss(loss_part, nb, 1.0 / ((double)B * T * nd.c_out), loss_dev, st);
  // weight gradients: dW = sum over columns of dG^T x (split-K), bias = ones
  // row; per layer W_ih against the layer's input (x, or the state of the
  // layer below at the same step: the shifted view of its stream) and W_hh
  // against the layer's previous state (the unshifted view)
  WGradJob jobs[kMaxWGradJobs];
  int njobs = 0;
  const NetOffsets o = nd.offsets();
  auto gb = [&](size_t off) { return off == kNoParam ? nullptr : grad + off; };  // bias gradient
  for (int l = 0; l < NL; ++l) {
    if (l == 0)
      jobs[njobs++] = {giT[0], tb.xT, K, K, MG, (nd.c_in + 1 + 15) / 16 * 16, 3 * H, nd.c_in,
                       nd.c_in, grad + o.wih[0], gb(o.bih[0])};
    else
      jobs[njobs++] = {giT[l], tb.hT[l - 1] + B, K, Kh, MG, H + 16, 3 * H, H, H,
                       grad + o.wih[l], gb(o.bih[l])};
    jobs[njobs++] = {ghT[l], tb.hT[l], K, Kh, MG, H + 16, 3 * H, H, H, grad + o.whh[l],
                     gb(o.bhh[l])};
  }
  if (nd.mlp) {
    jobs[njobs++] = {da1T, tb.hT[NL - 1] + B, K, Kh, 128, H + 16, nd.mlp, H, H, grad + o.w1,
                     gb(o.b1)};
    jobs[njobs++] = {dyT, tb.y1T, K, K, 128, 144, nd.c_out, nd.mlp, nd.mlp, grad + o.w2,
                     gb(o.b2)};
  } else {  // a single dense layer: W2 against the top layer's new state
    jobs[njobs++] = {dyT, tb.hT[NL - 1] + B, K, Kh, 128, H + 16, nd.c_out, H, H, grad + o.w2,
                     gb(o.b2)};
  }
  // one wave: a block per SM at most (a block's 4-stage ring fills most of
  // an SM's shared memory), at least four K chunks of 64 per block
  int tiles = 0;
  for (int q = 0; q < njobs; ++q) tiles += jobs[q].M / 128;
  int splits = std::max(1, std::min(tr_blocks_max / tiles, (int)(K / 256)));
  while (splits > 1 && wgrad_partials(jobs, njobs, (int)K, splits) > cpart_floats) --splits;
  if (launch_wgrad(jobs, njobs, (int)K, splits, cpart, net_status, st))
    return fail(DNNMG_ERR_ARG, "weight-gradient GEMM shape");
  prof.end(p, st);
  return net_check("train");
}

int dnnmg_ctx::train_grad(const uint16_t* X, const float* Y, int B, int T, float* g, float* loss) {
  if (int rc = train_grad_impl(X, Y, B, T)) return rc;
  if (g) cudaMemcpyAsync(g, grad, sizeof(float) * nd.num_params(), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(h_scalars, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (loss) std::memcpy(loss, h_scalars, sizeof(float));
  return check("train_grad");
}

int dnnmg_ctx::train_step(const uint16_t* X, const float* Y, int B, int T, float lr, float* loss) {
  if (int rc = train_grad_impl(X, Y, B, T)) return rc;
  ++adam_step;
  launch_adam(w_master, grad, adam_m, adam_v, nd.num_params(), lr, adam_step, st);
  launch_pack_weights(nd, w_master, pk, st);
  cudaMemcpyAsync(h_scalars, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (loss) std::memcpy(loss, h_scalars, sizeof(float));
  return check("train_step");
}

// Patch lists and level L+1 buffers of the DNN-MG correction.
int dnnmg_ctx::init_dnnmg() {
  // NET steps, samples and corpora report the missing parts
  if (cfg.replaced_levels < 1 || !net_ok || cfg.net_inputs > 0) return DNNMG_OK;
  const HostLevel& hl = lv[L()];
  std::vector<int> pc, cp(hl.solid.size(), -1);
  for (size_t c = 0; c < hl.solid.size(); ++c)
    if (!hl.solid[c]) {
      cp[c] = (int)pc.size();
      pc.push_back((int)c);
    }
  P = (int)pc.size();
  const Grid gF = grid(fine_level());
  const size_t n3 = 3 * (size_t)gF.nn;
  if (cfg.replaced_levels == 2) {  // intermediate level L+1 of the transfers
    midF = mem.alloc<double>(3 * (size_t)grid(L() + 1).nn);
    if (!midF) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  }
  patch_cell = mem.alloc<int>(P);
  cell_patch = mem.alloc<int>(cp.size());
  xtF = mem.alloc<double>(n3);
  ximpF = mem.alloc<double>(n3);
  fF = mem.alloc<double>(n3);
  rF = mem.alloc<double>(n3);
  vcorr = mem.alloc<double>(n3);
  bF = mem.alloc<double>(n3);
  bL = mem.alloc<double>(3 * (size_t)grid(L()).nn);
  X = mem.alloc<uint16_t>((size_t)P * nd.c_in);
  net_out = mem.alloc<float>((size_t)P * nd.c_out);
  hid = mem.alloc<float>((size_t)nd.layers * P * nd.hidden);
  feat_mean = mem.alloc<float>(nd.c_in);
  feat_std = mem.alloc<float>(nd.c_in);
  stat_partial = mem.alloc<double>((size_t)128 * nd.c_in * 2);
  if (!mem.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  cudaMemcpyAsync(patch_cell, pc.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(cell_patch, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice, st);
  std::vector<float> zero(nd.c_in, 0.0f), one(nd.c_in, 1.0f);
  cudaMemcpyAsync(feat_mean, zero.data(), sizeof(float) * nd.c_in, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(feat_std, one.data(), sizeof(float) * nd.c_in, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(hid, 0, sizeof(float) * nd.layers * P * nd.hidden, st);
  s64F = make_sten<double>(gF.h, cfg);
  cudaStreamSynchronize(st);
  return check("dnnmg setup");
}

// P applied once per replaced level: xc on level L -> xf on the fine level
// (ncomp fields; midF holds the level L+1 values when two levels are replaced)
void dnnmg_ctx::prolong_up(const double* xc, double* xf, int ncomp, double* ximp) {
  const Grid gL = grid(L()), gF = grid(fine_level());
  if (cfg.replaced_levels == 2) {
    const Grid gM = grid(L() + 1);
    launch_prolong_state64(gM, gL, xc, midF, ncomp, st);
    launch_prolong_state64(gF, gM, midF, xf, ncomp, st, ximp);
  } else {
    launch_prolong_state64(gF, gL, xc, xf, ncomp, st, ximp);
  }
}

// R = P^T once per replaced level, velocity fields: bf on the fine level ->
// bc on level L (pressure rows 0)
void dnnmg_ctx::restrict_down(const double* bf, double* bc) {
  const Grid gL = grid(L()), gF = grid(fine_level());
  cudaMemsetAsync(bc, 0, 3 * sizeof(double) * gL.nn, st);
  if (cfg.replaced_levels == 2) {
    const Grid gM = grid(L() + 1);
    cudaMemsetAsync(midF, 0, 3 * sizeof(double) * gM.nn, st);
    launch_restrict_full64(gF, gM, bf, midF, 2, st);
    launch_restrict_full64(gM, gL, midF, bc, 2, st);
  } else {
    launch_restrict_full64(gF, gL, bf, bc, 2, st);
  }
}

// the network correction of Algorithm 1 after the level-L solve of this step (x64 = v^L_n).
int dnnmg_ctx::dnnmg_correction() {
  const Grid gL = grid(L()), gF = grid(fine_level());
  const int K = (1 << cfg.replaced_levels) + 1;
  const int pr = prof.begin(DNNMG_STAGE_NETWORK, L(), st);
  if (!have_vcorr) {  // first correction: the previous fine velocity is P(v^L_{n-1})
    prolong_up(xold64, vcorr, 2);
    cudaMemsetAsync(vcorr + 2 * gF.nn, 0, sizeof(double) * gF.nn, st);
  }
  prolong_up(x64, xtF, 3, ximpF);  // P, and the same with the Dirichlet values imposed
  old_rhs(fine_level(), vcorr, fF);
  launch_residual_features(gF, s64F, ximpF, fF, rF, st, mixed());  // input: fine residual
  launch_gather(gL, gF, K, patch_cell, P, xtF, rF, feat_mean, feat_std, cfg.nu, cfg.dt, X, st);
  launch_patchnet_forward(nd, pk, X, hid, hid, net_out, P, net_status, st);  // network
  launch_scatter(gL, gF, K, cell_patch, net_out, nd.c_out, xtF, vcorr, st);
  old_rhs(fine_level(), vcorr, bF);                                   // Rhs
  restrict_down(bF, bL);                                              // R
  prof.end(pr, st);
  have_vcorr = have_net_rhs = true;
  // the network's status goes to the mailbox and is read once the step's
  // work is complete (step() synchronises at its end anyway)
  if (int rc = check("dnnmg correction")) return rc;
  launch_post(mail_d, mail_ticket(), nullptr, 0, 0, net_status, 4, 1, st);
  net_status_posted = true;
  return DNNMG_OK;
}

// One training sample per patch (corpus generation): the level-L step from
// the injected fine state x^{L+1}_{n-1} with the right-hand side the DNN-MG
// correction would produce if it were exact, b^L = R (1/k) M^{L+1} v^{L+1}_{n-1};
// then the network inputs at P(v^L_n) and the targets v^{L+1}_n - P(v^L_n).
int dnnmg_ctx::make_sample(const double* xf_prev, const double* xf_next, float* Xraw, float* Y,
                           dnnmg_step_stats* s) {
  if (!X)
    return fail(DNNMG_ERR_STATE,
                "DNN-MG needs replaced_levels 1 or 2 and a network on the patch features");
  const Grid gL = grid(L()), gF = grid(fine_level());
  const size_t n3L = 3 * (size_t)gL.nn;
  const int K = (1 << cfg.replaced_levels) + 1;
  if (cfg.replaced_levels == 2) {  // nodal injection fine -> L+1 -> L
    const Grid gM = grid(L() + 1);
    launch_inject<double>(gF, gM, xf_prev, midF, 3, st);
    launch_inject<double>(gM, gL, midF, x64, 3, st);
  } else {
    launch_inject<double>(gF, gL, xf_prev, x64, 3, st);
  }
  launch_impose_dirichlet64(gL, x64, st);
  cudaMemcpyAsync(xold64, x64, n3L * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(vcorr, xf_prev, 2 * sizeof(double) * gF.nn, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(vcorr + 2 * gF.nn, 0, sizeof(double) * gF.nn, st);
  old_rhs(fine_level(), vcorr, fF);
  restrict_down(fF, f64);
  dnnmg_step_stats tmp{};
  steps_taken = 0;  // a new state: refactor the coarse level
  int rc = newton(f64, s ? s : &tmp);
  if (rc != DNNMG_OK && rc != DNNMG_ERR_NOT_CONVERGED) return rc;
  prolong_up(x64, xtF, 3);
  cudaMemcpyAsync(ximpF, xtF, 3 * sizeof(double) * gF.nn, cudaMemcpyDeviceToDevice, st);
  launch_impose_dirichlet64(gF, ximpF, st);
  launch_residual_features(gF, s64F, ximpF, fF, rF, st, mixed());
  launch_gather_raw(gL, gF, K, patch_cell, P, xtF, rF, cfg.nu, cfg.dt, Xraw, st);
  launch_targets(gL, gF, K, patch_cell, P, xf_next, xtF, Y, st);
  have_net_rhs = have_vcorr = false;
  steps_taken = 0;
  cudaStreamSynchronize(st);
  return check("make_sample");
}

void dnnmg_ctx::set_physics(double nu, double dt) {
  cfg.nu = nu;
  cfg.dt = dt;
  const Grid gL = grid(L());
  s64L = make_sten<double>(gL.h, cfg);
  sxL = make_explicit_sten(gL.h, cfg);
  if (cfg.replaced_levels > 0) {
    sxF = make_explicit_sten(grid(fine_level()).h, cfg);
    s64F = make_sten<double>(grid(fine_level()).h, cfg);
  }
  solver->set_physics();
  steps_taken = 0;
}

// Corpus of Sec. 3.1 from plain trajectories: per trajectory a viscosity,
// a spin-up of the level-L solver from the impulsive start (larger time
// step), the prolongated state relaxed by plain fine-level steps, then T
// fine steps with one make_sample per step.
int dnnmg_ctx::make_corpus(int n_traj, const double* nus, int spinup_steps, double spinup_dt,
                           int relax_steps, int T, float* Xraw, float* Y) {
  if (!X)
    return fail(DNNMG_ERR_STATE,
                "DNN-MG needs replaced_levels 1 or 2 and a network on the patch features");
  if (n_traj < 1 || T < 1 || spinup_steps < 0 || relax_steps < 0 || !(spinup_dt > 0))
    return fail(DNNMG_ERR_ARG, "make_corpus: bad trajectory counts or spin-up time step");
  for (int k = 0; k < n_traj; ++k)
    if (!(nus[k] > 0)) return fail(DNNMG_ERR_ARG, "make_corpus: viscosities must be positive");
  if (!corpus_fine) {
    auto f = std::make_unique<dnnmg_ctx>();
    f->cfg = cfg;
    f->cfg.level_solve = fine_level();
    f->cfg.replaced_levels = 0;
    f->cfg.train_batch = 0;
    f->cfg.train_seq = 0;
    f->st = st;
    if (int rc = f->init()) return fail(rc, "make_corpus: fine-level solver: " + f->err);
    corpus_fine = std::move(f);
  }
  dnnmg_ctx& fine = *corpus_fine;
  const double nu0 = cfg.nu, dt0 = cfg.dt;
  const Grid gL = grid(L()), gF = grid(fine_level());
  const std::vector<double> x0 = initial_state(gL);
  const size_t rows = (size_t)P;
  int rc = DNNMG_OK;
  auto ok = [](int r) { return r == DNNMG_OK || r == DNNMG_ERR_NOT_CONVERGED; };
  for (int k = 0; k < n_traj && rc == DNNMG_OK; ++k) {
    set_physics(nus[k], spinup_dt);
    cudaMemcpyAsync(x64, x0.data(), x0.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    have_net_rhs = have_vcorr = false;
    for (int s = 0; s < spinup_steps; ++s) {
      const int r = step(DNNMG_PLAIN, nullptr);
      if (!ok(r)) return r;
    }
    set_physics(nus[k], dt0);
    fine.set_physics(nus[k], dt0);
    prolong_up(x64, fine.x64, 3);
    if (int r = fine.set_state(fine.x64)) return fail(r, "make_corpus: " + fine.err);
    for (int s = 0; s < relax_steps; ++s) {
      const int r = fine.step(DNNMG_PLAIN, nullptr);
      if (!ok(r)) return fail(r, "make_corpus: " + fine.err);
    }
    for (int n = 0; n < T; ++n) {
      // the fine step leaves its previous state in xold64
      const int r = fine.step(DNNMG_PLAIN, nullptr);
      if (!ok(r)) return fail(r, "make_corpus: " + fine.err);
      const size_t slot = (size_t)k * T + n;
      const int r2 = make_sample(fine.xold64, fine.x64, Xraw + slot * rows * nd.c_in,
                                 Y + slot * rows * nd.c_out, nullptr);
      if (!ok(r2)) return r2;
    }
  }
  (void)gF;
  // back to the configured physics and the impulsive start
  set_physics(nu0, dt0);
  fine.set_physics(nu0, dt0);
  cudaMemcpyAsync(x64, x0.data(), x0.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  have_net_rhs = have_vcorr = false;
  if (hid) cudaMemsetAsync(hid, 0, sizeof(float) * nd.layers * P * nd.hidden, st);
  cudaStreamSynchronize(st);
  return check("make_corpus");
}

int dnnmg_ctx::feature_stats(const float* Xraw, long long rows, float* mean_h, float* std_h) {
  if (!feat_mean) return fail(DNNMG_ERR_STATE, "no DNN-MG network in this context");
  if (rows <= 0) return fail(DNNMG_ERR_ARG, "no rows");
  launch_feature_stats(Xraw, rows, nd.c_in, stat_partial, 128, feat_mean, feat_std, st);
  if (mean_h) cudaMemcpyAsync(mean_h, feat_mean, sizeof(float) * nd.c_in, cudaMemcpyDeviceToHost, st);
  if (std_h) cudaMemcpyAsync(std_h, feat_std, sizeof(float) * nd.c_in, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return check("feature_stats");
}

int dnnmg_ctx::gather_batch(const float* Xraw, const float* Yc, const int* idx, int B, int T,
                            long long stride, uint16_t* Xb, float* Yb) {
  if (!feat_mean) return fail(DNNMG_ERR_STATE, "no DNN-MG network in this context");
  if (B <= 0 || T <= 0 || stride <= 0) return fail(DNNMG_ERR_ARG, "bad batch shape");
  launch_gather_batch(Xraw, Yc, idx, B, T, stride, nd.c_in, nd.c_out, feat_mean, feat_std, Xb, Yb,
                      st);
  return check("gather_batch");
}

int dnnmg_ctx::set_feature_stats(const float* mean, const float* stdv) {
  if (!feat_mean) return fail(DNNMG_ERR_STATE, "no DNN-MG network in this context");
  for (int k = 0; k < nd.c_in; ++k)
    if (!(stdv[k] > 0.0f)) return fail(DNNMG_ERR_ARG, "feature std must be positive");
  cudaMemcpyAsync(feat_mean, mean, sizeof(float) * nd.c_in, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(feat_std, stdv, sizeof(float) * nd.c_in, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return check("set_feature_stats");
}

int dnnmg_ctx::functionals(int level, const double* x, const double* x_old, double* out_host) {
  const Grid g = grid(level);
  dnnmg_config be = cfg;
  be.theta = 1.0;
  FnConsts c{};
  c.s = make_sten<double>(g.h, be);
  const double m1[2][2] = {{g.h / 3, g.h / 6}, {g.h / 6, g.h / 3}};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      c.mk[a * 4 + b] = m1[a & 1][b & 1] * m1[a >> 1][b >> 1] / cfg.dt;
  launch_functionals(g, c, x, x_old, fpart, fout, st);
  cudaMemcpyAsync(out_host, fout, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return check("functionals");
  return check("functionals");
}

int dnnmg_ctx::rel_errors(int level, const double* x, const double* x_ref, double* out_host) {
  double s4[4];
  launch_rel_errors(grid(level), x, x_ref, fpart, fout, st);
  cudaMemcpyAsync(s4, fout, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return check("relative_errors");
  if (int rc = check("relative_errors")) return rc;
  if (!(s4[1] > 0.0) || !(s4[3] > 0.0)) return fail(DNNMG_ERR_NUMERICAL, "reference state is zero");
  out_host[0] = std::sqrt(s4[0] / s4[1]);
  out_host[1] = std::sqrt(s4[2] / s4[3]);
  return DNNMG_OK;
}

int dnnmg_ctx::get_fine_velocity(double* v) {
  if (!have_vcorr) return fail(DNNMG_ERR_STATE, "no DNN-MG step taken yet");
  cudaMemcpyAsync(v, vcorr, 2 * sizeof(double) * grid(fine_level()).nn, cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  return check("get_fine_velocity");
}

int dnnmg_ctx::get_patch_inputs(uint16_t* x) {
  if (!have_vcorr) return fail(DNNMG_ERR_STATE, "no DNN-MG step taken yet");
  cudaMemcpyAsync(x, X, sizeof(uint16_t) * P * nd.c_in, cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  return check("get_patch_inputs");
}

// Network dimensions follow the patch: one level-L cell covers
// (2^r + 1)^2 nodes of level L + r; inputs are the prolongated velocity and
// the fine residual at those nodes plus 4 geometry features.
int dnnmg_ctx::init_net() {
  const int r = cfg.replaced_levels > 0 ? cfg.replaced_levels : 1;
  const int k = (1 << r) + 1;
  nd.c_in = cfg.net_inputs > 0 ? cfg.net_inputs : 4 * k * k + 4;
  nd.c_out = 2 * k * k;
  nd.hidden = cfg.hidden;
  nd.layers = cfg.gru_layers;
  nd.mlp = cfg.mlp_width;
  nd.bias = cfg.net_bias;
  net_ok = net_supported(nd);
  if (!net_ok) return DNNMG_OK;  // network calls report the unsupported shape
  const PackLayout L = PackLayout::of(nd);
  w_master = mem.alloc<float>(nd.num_params());
  pk.w = mem.alloc<uint16_t>(L.total);
  pk.w_elems = L.total;
  pk.bias_elems = (size_t)nd.layers * 4 * nd.hidden + nd.mlp + nd.nout();
  pk.bias = mem.alloc<float>(pk.bias_elems);
  net_status = mem.alloc<int>(4);
  if (!mem.ok()) return fail(DNNMG_ERR_CUDA, "device allocation failed");
  cudaMemsetAsync(w_master, 0, sizeof(float) * nd.num_params(), st);
  cudaMemsetAsync(net_status, 0, sizeof(int) * 4, st);
  launch_pack_weights(nd, w_master, pk, st);
  return check("network setup");
}

int dnnmg_ctx::mail_wait(unsigned long long t, const char* what) {
  if (int rc = check(what)) return rc;  // a failed launch never posts
  for (unsigned polls = 1;; ++polls) {
    if (__atomic_load_n(&mail_h->seq, __ATOMIC_ACQUIRE) >= t) return DNNMG_OK;
    if (polls % 1024 == 0) {
      // every kernel before the post has ended (or failed) once the stream
      // is idle: the post is then either visible or never comes
      const cudaError_t e = cudaStreamQuery(st);
      if (e == cudaErrorNotReady) continue;
      if (__atomic_load_n(&mail_h->seq, __ATOMIC_ACQUIRE) >= t) return DNNMG_OK;
      if (e != cudaSuccess) return check(what);
      return fail(DNNMG_ERR_CUDA, std::string(what) + ": the device posted no value");
    }
  }
}

int dnnmg_ctx::net_check(const char* what) {
  if (int rc = check(what)) return rc;
  const unsigned long long t = mail_ticket();
  launch_post(mail_d, t, nullptr, 0, 0, net_status, 0, 1, st);
  if (int rc = mail_wait(t, what)) return rc;
  const int s = mail_h->iv[0];
  if (s & 4) {
    cudaMemsetAsync(net_status, 0, sizeof(int), st);
    return fail(DNNMG_ERR_TIMEOUT, std::string(what) + ": tensor-core wait timed out");
  }
  return DNNMG_OK;
}

int dnnmg_ctx::set_weights(const float* w_host) {
  if (!net_ok) return fail(DNNMG_ERR_ARG, "network shape not supported");
  cudaMemcpyAsync(w_master, w_host, sizeof(float) * nd.num_params(), cudaMemcpyHostToDevice, st);
  launch_pack_weights(nd, w_master, pk, st);
  cudaStreamSynchronize(st);
  return check("set_weights");
}

int dnnmg_ctx::get_weights(float* w_host) {
  if (!net_ok) return fail(DNNMG_ERR_ARG, "network shape not supported");
  cudaMemcpyAsync(w_host, w_master, sizeof(float) * nd.num_params(), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  return check("get_weights");
}

int dnnmg_ctx::patch_infer(const uint16_t* x, float* h, float* out, int P) {
  if (!net_ok) return fail(DNNMG_ERR_ARG, "network shape not supported");
  if (P < 0) return fail(DNNMG_ERR_ARG, "negative patch count");
  if (P == 0) return DNNMG_OK;
  const int p = prof.begin(DNNMG_STAGE_NETWORK, 0, st);
  launch_patchnet_forward(nd, pk, x, h, h, out, P, net_status, st);
  prof.end(p, st);
  return net_check("patch_infer");
}

void dnnmg_ctx::old_rhs(int level, const double* x_old, double* f, double* copy) {
  const Grid g = grid(level);
  launch_old_time_rhs64(g, 1.0 / cfg.dt, x_old, f, st, copy);
  if (cfg.theta != 1.0)
    launch_explicit_sub64(g, level == L() ? sxL : sxF, 1.0 - cfg.theta, x_old, f, st);
}

int dnnmg_ctx::get_state(double* x) {
  cudaMemcpyAsync(x, x64, 3 * sizeof(double) * grid(L()).nn, cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  return check("get_state");
}

int dnnmg_ctx::set_state(const double* x) {
  cudaMemcpyAsync(x64, x, 3 * sizeof(double) * grid(L()).nn, cudaMemcpyDeviceToDevice, st);
  launch_impose_dirichlet64(grid(L()), x64, st);
  have_net_rhs = have_vcorr = false;
  steps_taken = 0;  // the next step refactors the coarse level
  if (hid) cudaMemsetAsync(hid, 0, sizeof(float) * nd.layers * P * nd.hidden, st);
  cudaStreamSynchronize(st);
  return check("set_state");
}

int dnnmg_ctx::linearize_api(const double* x) { return solver->linearize(x, true, true); }

int dnnmg_ctx::apply_api(int level, const void* w, void* y, int precision) {
  if (level < lc() || level > L()) return fail(DNNMG_ERR_ARG, "level out of range");
  if (part_solid_patches(lv[level]))
    return fail(DNNMG_ERR_ARG, "the operator kernels need whole stabilisation patches on this level");
  if (precision != solver->precision()) return fail(DNNMG_ERR_ARG, "precision mismatch");
  return solver->apply(level - lc(), w, y);
}

int dnnmg_ctx::vcycle_api(int level, const void* b, void* x, int precision) {
  if (level < lc() || level > L()) return fail(DNNMG_ERR_ARG, "level out of range");
  if (precision != solver->precision()) return fail(DNNMG_ERR_ARG, "precision mismatch");
  return solver->vcycle(level - lc(), b, x);
}

int dnnmg_ctx::residual_api(const double* x, const double* f, double* r) {
  launch_residual64(grid(L()), s64L, x, f, r, st, mixed());
  return check("residual");
}

// r64 = f - A(x64) and its norm (formed by the residual launch and read
// through the host mailbox): enqueue, returning the post's number, and wait
unsigned long long dnnmg_ctx::residual_norm_begin(const double* f, bool with_status) {
  const Grid gL = grid(L());
  NormOut no;
  no.partials = norm_partials;
  no.counter = norm_counter;
  no.out = dots;
  no.mail = mail_d;
  no.seq = mail_ticket();
  if (with_status) no.status = solver->status_words();
  const int p = prof.begin(DNNMG_STAGE_RESIDUAL, L(), st);
  launch_residual64(gL, s64L, x64, f, r64, st, mixed(), no);
  prof.end(p, st);
  return no.seq;
}

int dnnmg_ctx::residual_norm_end(unsigned long long t, double* nrm) {
  if (int rc = mail_wait(t, "residual norm")) return rc;
  *nrm = std::sqrt(mail_h->v[0]);
  return DNNMG_OK;
}

int dnnmg_ctx::newton(const double* f, dnnmg_step_stats* s) {
  const unsigned long long t0 = residual_norm_begin(f);
  // the linearisations' singularity flags are read once, after the loop
  solver->clear_setup_status();
  // the first Newton iteration's linearisation does not depend on the
  // residual: it is enqueued before the host waits for the norm, so that
  // the setups run during that round trip (it is wasted when the state
  // already meets the tolerance, so not after a step that needed no iteration)
  const bool lin0 = cfg.newton_max > 0 && last_newton_its > 0;
  if (lin0)
    if (int rc = solver->linearize(x64, steps_taken % cfg.coarse_refresh == 0, true, false))
      return rc;
  double nrm = 0;
  if (int rc = residual_norm_end(t0, &nrm)) return rc;
  s->res0 = nrm;
  int it = 0, gits = 0;
  while (nrm > cfg.newton_tol && it < cfg.newton_max) {
    if (!std::isfinite(nrm)) return fail(DNNMG_ERR_NUMERICAL, "non-finite Newton residual");
    // the coarse-level factorisation is refreshed at the first Newton step of
    // every coarse_refresh-th time step (a lagged preconditioner component)
    const bool refresh = it == 0 && steps_taken % cfg.coarse_refresh == 0;
    // with precond_lag the multigrid preconditioner keeps the linearisation
    // of the step's first Newton iteration; the matvec always uses the current one
    const bool precond = it == 0 || !cfg.precond_lag;
    if (!(it == 0 && lin0))
      if (int rc = solver->linearize(x64, refresh, precond, false)) return rc;
    int its = 0;
    if (int rc = solver->solve(r64, x64, cfg.eps_damp, &its)) return rc;
    gits += its;
    // the smoothers' and setups' status words travel with this norm
    if (int rc = residual_norm_end(residual_norm_begin(f, true), &nrm)) return rc;
    ++it;
  }
  s->newton_its = it;
  s->gmres_its = gits;
  last_newton_its = it;
  s->res_final = nrm;
  int setup = 0;
  int words[4];
  for (int i = 0; i < 4; ++i) words[i] = mail_h->iv[i];
  // after an iteration the status words came with the last norm; else read them now
  if (const int ds = it > 0 ? solver->status_from(words, &setup) : solver->device_status(&setup))
    return ds < 0 ? check("newton") : fail(DNNMG_ERR_TIMEOUT, "a colour pass's inverse copy timed out");
  if (setup & 1) return fail(DNNMG_ERR_NUMERICAL, "singular local Vanka matrix");
  if (setup & 2) return fail(DNNMG_ERR_NUMERICAL, "singular coarse-level matrix");
  if (!std::isfinite(nrm)) return fail(DNNMG_ERR_NUMERICAL, "non-finite Newton residual");
  if (nrm > cfg.newton_tol) return DNNMG_ERR_NOT_CONVERGED;
  return check("newton");
}

int dnnmg_ctx::step(int mode, dnnmg_step_stats* stats) {
  dnnmg_step_stats s{};
  const Grid gL = grid(L());
  const size_t n3 = 3 * (size_t)gL.nn;
  if (mode == DNNMG_NET && (cfg.replaced_levels < 1 || !net_ok || !X))
    return fail(DNNMG_ERR_ARG,
                "DNN-MG steps need replaced_levels 1 or 2 and a network on the patch features");
  cudaEventRecord(ev0, st);
  const bool use_net_rhs = mode == DNNMG_NET && have_net_rhs;
  if (use_net_rhs) {
    launch_copy2(x64, xold64, bL, f64, n3, st);  // both copies in one launch
  } else {
    old_rhs(L(), x64, f64, xold64);  // and xold64 = x64 in the same launch
  }
  int rc = newton(f64, &s);
  if (use_net_rhs && (rc != DNNMG_OK || s.newton_its > cfg.fallback_newton_its)) {
    // the corrected right-hand side slowed Newton down: redo the step without it
    cudaMemcpyAsync(x64, xold64, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    old_rhs(L(), xold64, f64);
    const int first_its = s.newton_its, first_gits = s.gmres_its;
    rc = newton(f64, &s);
    s.newton_its += first_its;
    s.gmres_its += first_gits;
    s.fallback = 1;
  }
  if (mode == DNNMG_NET && (rc == DNNMG_OK || rc == DNNMG_ERR_NOT_CONVERGED)) {
    const int rc2 = dnnmg_correction();
    if (rc2 != DNNMG_OK) rc = rc2;
  }
  ++steps_taken;
  cudaEventRecord(ev1, st);
  if (cudaEventSynchronize(ev1) != cudaSuccess) {  // a fault in the step's kernels
    net_status_posted = false;
    const int rc3 = check("step");
    return rc3 ? rc3 : fail(DNNMG_ERR_CUDA, "step: stream synchronisation failed");
  }
  if (net_status_posted) {  // the correction's status, complete with the step
    net_status_posted = false;
    if (mail_h->iv[4] & 4) {
      cudaMemsetAsync(net_status, 0, sizeof(int), st);
      if (rc == DNNMG_OK || rc == DNNMG_ERR_NOT_CONVERGED)
        rc = fail(DNNMG_ERR_TIMEOUT, "dnnmg correction: tensor-core wait timed out");
    }
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  s.ms = ms;
  s.status = rc;
  prof.collect(st);
  (void)mode;
  if (stats) *stats = s;
  return rc;
}
