"""Benchmark of the DNN-MG hot path on one GB300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode step|vcycle|net|coarse|periodic]

Workload (the DNN-MG configuration): multigrid solve on the 512x128 channel
(level 5, 198,531 DOFs) and the patch network on the 1024x256 level
(61,440 patches, 2-layer GRU with hidden size 64 + MLP 128, BF16 with FP32
accumulation); held-out viscosity nu = 0.0065, dt = 0.005, mixed FP32/FP64
solver, obstacle seeded.  Before the timed region the network is trained by
the library's own kernels (10-step windows) on the device corpus of 32 plain
fine trajectories (seeded obstacle, nu uniform in [0.004, 0.01]).  All
methods start from the same developed flow at t ~ 1 s (level-5 spin-up),
then W untimed and K timed steps: DNN-MG, plain MG(L), plain FP64 MG(L+1)
(the reference of the errors) and plain mixed-precision MG(L+1) at a sweep of
Newton / FGMRES tolerances, each step timed alone with L2 flushed before it;
the equal-error block reads off MG(L+1)'s time per step at DNN-MG's velocity
error.  `value` = DNN-MG time steps per second over all ranks.  Also: the
plain FP64 128x32 workload beside the oracle, the plain mixed 1024x256
workload with its per-step error against an FP64 run, held-out trajectories,
the batched, large and network-size workloads.  One JSON line is printed by
rank 0.  --impl reference times the FP64 CPU oracle (DNN-MG step of the same
workload) on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time/step & V-cycle DOF/s: DNN-MG vs plain MG on 1 GB300 at equal L2 err; %HBM/TC peak"
L, NU, DT = 5, 0.0065, 0.005
NU_RANGE = (0.004, 0.01)                 # viscosities of the corpus and held-out trajectories
CORPUS_SEEDS = tuple(range(2000, 2032))  # 32 plain fine trajectories
HELDOUT_SEEDS = tuple(range(2032, 2036))
SPIN_STEPS, SPIN_DT, RELAX_STEPS = 50, 0.02, 4  # level-L spin-up to t = 1 s, fine relaxation
# untimed steps of every method before the timed ones, at least: the
# network's GRU memory is zero after the state is set, and DNN-MG's third
# and fourth steps from there take a third Newton iteration (11 FGMRES
# iterations) while it fills; from the fifth on the step is steady
NET_WARMUP = 5
# end-to-end steps: one period of the coarse level's refactorisation (every
# 32nd step by default), so that the window holds exactly one
E2E_STEPS = 32
# training batch: 152 tiles of 128 sequences, one per SM of the GB300
CORPUS_T, TRAIN_ITERS, TRAIN_B, TRAIN_T = 16, 400, 19456, 10
LARGE_CORPUS_STEPS, LARGE_TRAIN_ITERS = 16, 100  # two replaced levels
# plain MG(L+1) tolerance sweep: (Newton tolerance, FGMRES relative tolerance,
# Newton cap, FGMRES cap); the last point is one Newton step with one V-cycle
SWEEP = ((1e-10, 1e-4, 20, 200), (1e-8, 1e-3, 20, 200), (1e-6, 1e-2, 20, 200),
         (1e-5, 1e-1, 20, 200), (1e-4, 0.3, 20, 200), (1e-3, 0.5, 20, 200), (0.0, 0.5, 1, 1))
WORKLOAD = ("DNN-MG time step: multigrid on the 512x128 channel (level 5, 198,531 DOFs) + patch "
            "network on 1024x256 (level 6, 61,440 patches, GRU 2x64 + MLP 128, BF16), nu=0.0065, "
            "dt=0.005, mixed FP32/FP64, developed flow (t ~ 1 s)")
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture, keyed by the hash of the kernel's sources (source_hash) at the
# capture; after a change of those sources the figure no longer describes
# the kernel and is not reported (traffic = null) until a new capture is
# entered here.
NCU_TRAFFIC = {"5af723181ebd87da": {"vcycle_kernel<float>@split5": 60213248 + 942336}}
L2_BYTES = 129 * 2 ** 20


def source_hash(unit="vcycle.cu"):
    """First 16 hex digits of the SHA-256 of one translation unit of the
    library and every header it includes from the project (recursively,
    sorted by name): the sources a kernel's traffic capture belongs to."""
    csrc = os.path.join(ROOT, "paper_2106_07687_gb300", "csrc")
    found, todo = set(), [os.path.join(csrc, unit)]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in found or not os.path.exists(f):
            continue
        found.add(f)
        with open(f) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith("#include \""):
                    todo.append(os.path.join(os.path.dirname(f), line.split('"')[1]))
    h = hashlib.sha256()
    for f in sorted(found):
        h.update(os.path.relpath(f, ROOT).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ndof(level):
    return 3 * (16 * 2 ** level + 1) * (4 * 2 ** level + 1)


def nnodes(level):
    return ndof(level) // 3


def fluid_cells(level):
    return 16 * 4 * 4 ** level - 4 * 4 ** level


def vcycle_bytes(top, coarsest=1, sweeps=4):
    """Algorithmic HBM bytes of one V(2,2) cycle with top level `top` (FP32
    vectors, FP32 12x12 Vanka inverses, FP64 coarse inverse): per smoothing
    level 4 colour passes per sweep, each streaming the colour's inverses
    (576 B per cell) and b, x_in, x_out, vbar (44 B per node); the defect
    (44 B per node), restriction (12 B per fine node + 24 B per coarse node),
    prolongation (24 B per fine node + 12 B per coarse node); the coarse
    solve reads its 891 x 891 FP64 inverse once."""
    total = 12 * nnodes(top)                      # zeroing of the top iterate
    for lev in range(coarsest + 1, top + 1):
        per_pass = fluid_cells(lev) / 4 * 576 + nnodes(lev) * 44
        total += 4 * sweeps * per_pass + nnodes(lev) * 44
        total += nnodes(lev) * 12 + nnodes(lev - 1) * 24 + nnodes(lev) * 24 + nnodes(lev - 1) * 12
    nd = 3 * nnodes(coarsest)
    return total + 8 * nd * nd + 8 * nd


_ORACLE_STEP = """
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
import synthetic
from oracle import dnnmg, fem, mesh, net, newton
ob = synthetic.obstacle_block(1000)
levels = mesh.hierarchy({level}, obstacle=ob)
fine = mesh.Level({level} + 1, obstacle=ob)
prm = fem.Params(nu={nu}, dt={dt})
opt = newton.SolverOptions()
spec = net.NetSpec()
params = spec.unflatten(synthetic.random_weights(1, spec.num_params(), 0.02))
x = mesh.initial_state(levels[-1])
state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
for _ in range({warm}):
    x, state, _ = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt)
times = []
t_end = time.perf_counter() + {budget}
for k in range({steps}):
    t = time.perf_counter()
    x, state, _ = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt)
    times.append(time.perf_counter() - t)
    if time.perf_counter() > t_end:
        break
print(json.dumps(times))
"""


def oracle_dnnmg_steps(level, steps=1, warm=0, threads=1, budget=1e9):
    """Seconds per FP64 oracle DNN-MG step (level-L solve + fine residual,
    features, network, scatter, Rhs, restriction), consecutive steps from
    the impulsive start in a fresh process with `threads` BLAS/OpenMP
    threads; stops after `budget` seconds of timed steps (at least one)."""
    code = _ORACLE_STEP.format(root=ROOT, level=level, nu=NU, dt=DT, warm=warm, steps=steps,
                               budget=budget)
    n = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline():
    """One oracle DNN-MG step of the benchmarked workload (solve on level 5,
    network on level 6), the first step from the impulsive start, timed
    single-threaded and with every host core."""
    cores = os.cpu_count() or 1
    one = oracle_dnnmg_steps(L, threads=1)[0]
    allc = oracle_dnnmg_steps(L, threads=cores)[0]
    best = min(one, allc)
    return {"value": 1.0 / best, "unit": "time steps/s", "cores": cores if allc <= one else 1,
            "kind": "oracle",
            "single_thread": {"value": 1.0 / one, "s_per_step": one},
            "all_cores": {"value": 1.0 / allc, "s_per_step": allc, "threads": cores},
            "sample": f"the first DNN-MG time step of the FP64 oracle from the impulsive start on "
                      f"the benchmarked workload (solve on 512x128, level {L}; network on "
                      f"1024x256): {one:.1f} s single-threaded, {allc:.1f} s with {cores} "
                      f"BLAS/OpenMP threads; value = the faster"}


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = sorted(float(r[0]) for r in self.rows if num(r[0]))
        mx = max(float(r[1]) for r in self.rows if num(r[1]))
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p.get("bf16_tflops_sustained", p["bf16_tflops"]), \
            "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def l2_bandwidth(torch, stream, mib=24, reps=200):
    """L2 bandwidth measured here: repeated copies between two buffers of
    `mib` MiB each, both resident in the 129 MB L2 after the first pass
    (bytes read plus written per copy over CUDA-event time)."""
    n = mib * 2 ** 20 // 4
    a = torch.ones(n, device="cuda")
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        b.copy_(a)
    e1.record(stream)
    torch.cuda.synchronize()
    return 2 * 4 * n * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9


def net_flops(c_in=40, H=64, mlp=128, c_out=18):
    """FLOPs (2 per multiply-add) per patch and step: forward, and forward +
    backward (activation gradients of all but the first layer's input, weight
    gradients of every layer)."""
    fwd = 3 * H * c_in + 3 * H * H + 3 * H * H + 3 * H * H + mlp * H + c_out * mlp
    act = c_out * mlp + mlp * H + 3 * H * H + 3 * H * H + 3 * H * H
    return 2 * fwd, 2 * (fwd + act + fwd)


def rest_corpus(dn, torch, common, level, replaced, nus_train, corpus_steps):
    """Training samples from plain trajectories on level `level + replaced`
    started from rest (one per viscosity in nus_train, `corpus_steps` steps
    each), made by the library's kernels.  Returns (X, Y) stacked over
    steps."""
    Xs, Ys = [], []
    for v in nus_train:
        fctx = dn.Context(level_solve=level + replaced, nu=v, **common)
        sctx = dn.Context(level_solve=level, nu=v, replaced_levels=replaced, **common)
        prev = fctx.get_state()
        for _ in range(corpus_steps):
            fctx.step(dn.PLAIN)
            cur = fctx.get_state()
            X, Y = sctx.make_sample(prev, cur)
            Xs.append(X)
            Ys.append(Y)
            prev = cur
        fctx.close()
        sctx.close()
    return torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous()


def device_corpus(dn, torch, precision):
    """The corpus of Sec. 3.1 at the configured scale: 32 plain trajectories
    (seeds CORPUS_SEEDS: seeded obstacle, nu uniform in NU_RANGE), each spun
    up on level L to t = 1 s, relaxed on level L+1 and sampled over CORPUS_T
    fine steps by dnnmg_make_corpus.  Trajectories are grouped by obstacle
    position (one context per position).  Returns (X [32*T*P, 40],
    Y [32*T*P, 18], seconds)."""
    import synthetic
    groups = {}
    for sd in CORPUS_SEEDS:
        groups.setdefault(synthetic.obstacle_block(sd), []).append(
            synthetic.viscosity(sd, *NU_RANGE))
    n = len(CORPUS_SEEDS)
    P = None
    X = Y = None
    k = 0
    t0 = time.perf_counter()
    for ob, nus in sorted(groups.items()):
        ctx = dn.Context(level_solve=L, replaced_levels=1, precision=precision, nu=NU, dt=DT,
                         obstacle_i0=ob[0], obstacle_j0=ob[1])
        if X is None:
            P = ctx.num_patches()
            ci, co = ctx.net_dims()
            X = torch.empty(n, CORPUS_T, P, ci, dtype=torch.float32, device="cuda")
            Y = torch.empty(n, CORPUS_T, P, co, dtype=torch.float32, device="cuda")
        ctx.make_corpus(nus, SPIN_STEPS, SPIN_DT, RELAX_STEPS, CORPUS_T, X[k:k + len(nus)],
                        Y[k:k + len(nus)])
        k += len(nus)
        ctx.close()
    torch.cuda.synchronize()
    return X.view(n * CORPUS_T * P, -1), Y.view(n * CORPUS_T * P, -1), time.perf_counter() - t0


def train_on(dn, torch, stream, common, level, replaced, nu, corpus, n_traj, corpus_steps, iters,
             **net):
    """A network (sizes in `net`: hidden, gru_layers) trained by `iters` Adam
    steps at batch TRAIN_B x TRAIN_T on the corpus, with its feature
    statistics.  Returns (context, mean, std, losses, ms per training step)."""
    import numpy as np
    import synthetic
    Xc, Yc = corpus
    net_ctx = dn.Context(level_solve=level, nu=nu, replaced_levels=replaced, train_batch=TRAIN_B,
                         train_seq=TRAIN_T, **net, **common)
    P = net_ctx.num_patches()
    feat_mean, feat_std = net_ctx.feature_stats(Xc)
    net_ctx.set_weights(synthetic.random_weights(77, net_ctx.num_params(), 0.05).astype(np.float32))
    rng = np.random.default_rng(3)
    idx_all = []
    for _ in range(iters):
        tid = rng.integers(0, n_traj, TRAIN_B)
        start = rng.integers(0, corpus_steps - TRAIN_T + 1, TRAIN_B)
        idx_all.append(np.stack([tid * corpus_steps + start, rng.integers(0, P, TRAIN_B)], 1))
    idx_dev = torch.from_numpy(np.stack(idx_all).astype(np.int32)).cuda()
    losses = []
    for it in range(5):   # warm-up
        Xb, Yb = net_ctx.gather_batch(Xc, Yc, idx_dev[it].contiguous(), TRAIN_T, P)
        losses.append(net_ctx.train_step(Xb, Yb, TRAIN_B, TRAIN_T, 2e-3))
    torch.cuda.synchronize()
    te0, te1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    te0.record(stream)
    for it in range(5, iters):
        Xb, Yb = net_ctx.gather_batch(Xc, Yc, idx_dev[it].contiguous(), TRAIN_T, P)
        lr = 2e-3 if it < 0.7 * iters else 5e-4
        losses.append(net_ctx.train_step(Xb, Yb, TRAIN_B, TRAIN_T, lr))
    te1.record(stream)
    torch.cuda.synchronize()
    train_ms = te0.elapsed_time(te1) / (iters - 5)
    del idx_dev
    return net_ctx, feat_mean, feat_std, losses, train_ms


def spun_up_state(dn, nu, ob, precision):
    """The developed flow the timed steps start from: SPIN_STEPS plain
    level-L steps from rest with time step SPIN_DT (t = 1 s), then P to level
    L+1.  Returns (level-L state, level-L+1 state) as device FP64 vectors."""
    c = dn.Context(level_solve=L, replaced_levels=1, nu=nu, dt=SPIN_DT, precision=precision,
                   obstacle_i0=ob[0], obstacle_j0=ob[1])
    for _ in range(SPIN_STEPS):
        c.step(dn.PLAIN)
    x5 = c.get_state().clone()
    x6 = c.prolongate(L, x5).clone()
    c.close()
    return x5, x6


def time_infer(ctx, torch, stream, P, c_in, c_out, layers, hidden, reps=20):
    """Mean time of one dnnmg_patch_infer over P patches (ms)."""
    xin = torch.randn(P, c_in, device="cuda").to(torch.bfloat16)
    hin = torch.zeros(layers, P, hidden, device="cuda")
    out = torch.empty(P, c_out, device="cuda")
    for _ in range(3):
        ctx.patch_infer(xin, hin, out)
    torch.cuda.synchronize()
    te0, te1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    te0.record(stream)
    for _ in range(reps):
        ctx.patch_infer(xin, hin, out)
    te1.record(stream)
    torch.cuda.synchronize()
    return te0.elapsed_time(te1) / reps


def on_fine_level(c, net, ref, top):
    """State of context c on level `top` (at or above its solved level): the
    solution prolongated by the library's bilinear P (through the reference
    context's hierarchy above c's own), with the network-corrected fine
    velocity in place of the prolongated one for DNN-MG."""
    lev = c.cfg.level_solve
    x = c.get_state().clone()
    for k in range(top - lev):
        x = (c if k == 0 else ref).prolongate(lev + k, x)
    if net:
        nf = x.numel() // 3
        x[:2 * nf] = c.get_fine_velocity()
    return x


def compare_runs(runs, ref_name, ref, lev, steps_up, stream, flush, torch, K, count,
                 on_step=None):
    """K steps of every run, each timed alone with CUDA events (L2 flushed
    before each), then, untimed, every run's state on the reference's level:
    velocity and pressure relative l2 errors against the reference and the
    drag, lift and J_div functionals (Sec. 3.4), all by the library's
    kernels.  Returns per-run times (ms, summed), error and functional
    series, step statistics and the library's kernel launches inside the
    timed steps (count() is the library's launch counter)."""
    top = lev + steps_up
    fine = lambda name, c, mode: on_fine_level(c, mode == 1, ref, top)
    prev = {name: fine(name, c, mode) for name, (c, mode) in runs.items()}
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    times = {k: 0.0 for k in runs}
    series = {k: {"vel_err": [], "p_err": [], "drag": [], "lift": [], "div": []} for k in runs}
    stats = {k: [] for k in runs}
    counts = {k: 0 for k in runs}
    for _ in range(K):
        for name, (c, mode) in runs.items():
            flush.zero_()
            if on_step:
                on_step(name, True)
            n0 = count()
            ev[0].record(stream)
            stats[name].append(c.step(mode))
            ev[1].record(stream)
            counts[name] += count() - n0
            if on_step:
                on_step(name, False)
            torch.cuda.synchronize()
            times[name] += ev[0].elapsed_time(ev[1])
        cur = {name: fine(name, c, mode) for name, (c, mode) in runs.items()}
        for name in runs:
            ve, pe = ((0.0, 0.0) if name == ref_name else
                      ref.relative_errors(top, cur[name], cur[ref_name]))
            jd, fd, fl = ref.functionals(top, cur[name], prev[name])
            for key, v in zip(("vel_err", "p_err", "drag", "lift", "div"), (ve, pe, fd, fl, jd)):
                series[name][key].append(v)
        prev = cur
    return times, series, stats, counts


def summarize_series(series, ref_name):
    """Mean errors, last functional values and the force drift: the mean
    over steps of |F - F_ref| / |F_ref| with F = (drag, lift)."""
    mean = lambda v: sum(v) / len(v)
    r = series[ref_name]
    out = {}
    for name, s in series.items():
        drift = [((d - dr) ** 2 + (l - lr) ** 2) ** 0.5 / max((dr * dr + lr * lr) ** 0.5, 1e-300)
                 for d, l, dr, lr in zip(s["drag"], s["lift"], r["drag"], r["lift"])]
        out[name] = {"vel_l2_err_mean": mean(s["vel_err"]), "vel_l2_err_last": s["vel_err"][-1],
                     "p_l2_err_mean": mean(s["p_err"]), "p_l2_err_last": s["p_err"][-1],
                     "drag_last": s["drag"][-1], "lift_last": s["lift"][-1],
                     "div_last": s["div"][-1], "force_drift_mean": mean(drift)}
    return out


def run_large(dn, torch, stream, flush, args, common):
    """Large DNN-MG: solve on the 512x128 channel (level 5), the network
    replaces levels 6 and 7 (5x5-node patches of the 2048x512 level, 104
    inputs, 50 outputs); nu = 0.002, dt = 0.002.  Trained on a bounded
    corpus of plain level-7 trajectories (nu 0.0016 and 0.0025); then K
    timed steps each of DNN-MG, plain mixed-precision MG on level 5 and plain
    FP64 MG on level 7 (the reference) from the impulsive start, with the
    errors, functionals and force drift of each against the reference."""
    lev, rep, nu, dt = 5, 2, 0.002, 0.002
    com = dict(common, dt=dt)
    nus_train = (0.0016, 0.0025)
    corpus = rest_corpus(dn, torch, com, lev, rep, nus_train, LARGE_CORPUS_STEPS)
    net_ctx, _, _, losses, train_ms = train_on(dn, torch, stream, com, lev, rep, nu, corpus,
                                               len(nus_train), LARGE_CORPUS_STEPS,
                                               LARGE_TRAIN_ITERS)
    del corpus
    torch.cuda.empty_cache()
    ref = dn.Context(level_solve=lev + rep, nu=nu, **dict(com, precision=dn.FP64))
    coarse = dn.Context(level_solve=lev, nu=nu, **com)
    runs = {"dnnmg": (net_ctx, dn.NET), "mg_L": (coarse, dn.PLAIN), "mg_L+2": (ref, dn.PLAIN)}
    for c, mode in runs.values():
        for _ in range(max(1, args.warmup)):
            c.step(mode)
    K = args.steps
    times, series, _, _ = compare_runs(runs, "mg_L+2", ref, lev, rep, stream, flush, torch, K,
                                       dn.kernel_launches)
    out = {"workload": "solve 512x128 (level 5), network replaces 1024x256 and 2048x512 "
                       "(5x5-node patches, 104 inputs, 50 outputs), nu=0.002, dt=0.002, mixed "
                       "FP32/FP64; reference: plain FP64 MG on 2048x512",
           "patches": net_ctx.num_patches(), "dofs_L": ndof(lev), "dofs_L+2": ndof(lev + rep),
           "steps": K,
           "ms_per_step": {k: times[k] / K for k in runs},
           "vs_mg_L+2": summarize_series(series, "mg_L+2"),
           "train_ms_per_iter": train_ms, "loss_first": losses[0], "loss_last": losses[-1],
           "training": f"{LARGE_TRAIN_ITERS} Adam steps, B={TRAIN_B}, T={TRAIN_T}, corpus 2 "
                       f"level-7 trajectories x {LARGE_CORPUS_STEPS} steps (nu 0.0016, 0.0025)"}
    for c in (net_ctx, ref, coarse):
        c.close()
    torch.cuda.empty_cache()
    return out


TABLE1_SIZES = [(32, 1), (64, 1), (32, 2), (64, 2), (32, 3), (64, 3)]


def run_sizes(dn, torch, stream, flush, args, common, corpus, start):
    """The network sizes of Table 1 (m x n: GRU hidden size m, n stacked
    cells) on the default DNN-MG workload.  Each is trained on the same
    corpus with the same batches and schedule; reported: parameters,
    training time per Adam step (and its factor against 32 x 1, the columns
    of Table 1), forward time over all patches, the last training loss, and
    K DNN-MG steps from the developed flow `start` = (level-L state,
    level-L+1 state) against plain mixed-precision MG on the finer level
    (time per step, velocity and pressure errors, force drift)."""
    out = []
    base = None
    x5, x6 = start
    for m, n in TABLE1_SIZES:
        ctx, _, _, losses, train_ms = train_on(
            dn, torch, stream, common, L, 1, NU, corpus, len(CORPUS_SEEDS), CORPUS_T,
            TRAIN_ITERS, hidden=m, gru_layers=n)
        infer_ms = time_infer(ctx, torch, stream, ctx.num_patches(), 40, 18, n, m)
        ref = dn.Context(level_solve=L + 1, nu=NU, **common)
        ctx.set_state(x5)
        ref.set_state(x6)
        runs = {"dnnmg": (ctx, dn.NET), "mg_L+1": (ref, dn.PLAIN)}
        for c, mode in runs.values():
            for _ in range(max(NET_WARMUP, args.warmup)):
                c.step(mode)
        K = args.steps
        times, series, stats, _ = compare_runs(runs, "mg_L+1", ref, L, 1, stream, flush, torch,
                                               K, dn.kernel_launches)
        err = summarize_series(series, "mg_L+1")["dnnmg"]
        if base is None:
            base = (ctx.num_params(), train_ms)
        out.append({"size": f"{m}x{n}", "params": ctx.num_params(),
                    "params_factor": ctx.num_params() / base[0],
                    "train_ms_per_iter": train_ms, "train_factor": train_ms / base[1],
                    "forward_ms": infer_ms, "loss_first": losses[0], "loss_last": losses[-1],
                    "dnnmg_ms_per_step": times["dnnmg"] / K,
                    "fallbacks": sum(st["fallback"] for st in stats["dnnmg"]),
                    "vel_l2_err_mean": err["vel_l2_err_mean"],
                    "p_l2_err_mean": err["p_l2_err_mean"],
                    "force_drift_mean": err["force_drift_mean"]})
        for c in (ctx, ref):
            c.close()
        torch.cuda.empty_cache()
    return out


def slowest_rank_ms(ms, world, device):
    """The largest of the ranks' times (the whole job ends with its slowest
    rank), by an all-reduce over the process group; the local time for one
    rank."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms, steps, world):
    """Whole-job time steps per second: every one of the world's ranks
    stepped its own problem `steps` times in `ms` milliseconds."""
    return world * steps / (ms * 1e-3)


def equal_error(times, summary, K, names, target="dnnmg"):
    """MG(L+1)'s time per step at the target method's mean velocity error:
    the sweep points (mean velocity error, ms per step) sorted by error, and
    log(time) interpolated linearly in log(error) between the two points
    that bracket the target's error.  When every point is more accurate
    than the target, the fastest of them bounds MG(L+1)'s time at equal
    error from above (bracketed = false)."""
    import math
    e_t = summary[target]["vel_l2_err_mean"]
    pts = sorted((summary[n]["vel_l2_err_mean"], times[n] / K, n) for n in names)
    out = {"target": target, "target_vel_l2_err_mean": e_t,
           "target_ms_per_step": times[target] / K,
           "sweep": [{"run": n, "vel_l2_err_mean": e, "ms_per_step": t} for e, t, n in pts]}
    lo = [p for p in pts if p[0] <= e_t]
    hi = [p for p in pts if p[0] > e_t]
    if lo and hi:
        (e0, t0, n0), (e1, t1, n1) = lo[-1], hi[0]
        w = (math.log(e_t) - math.log(max(e0, 1e-300))) / (math.log(e1) - math.log(max(e0, 1e-300)))
        t_eq = math.exp(math.log(t0) + w * (math.log(t1) - math.log(t0)))
        out.update(bracketed=True, between=[n0, n1], mg_fine_ms_at_equal_error=t_eq)
    elif lo:
        e0, t0, n0 = min(lo, key=lambda p: p[1])
        out.update(bracketed=False, between=[n0, None], mg_fine_ms_at_equal_error=t0,
                   note="every MG(L+1) point is more accurate than the target; the fastest "
                        "point's time bounds MG(L+1)'s time at equal error from above")
    else:
        out.update(bracketed=False, between=[None, pts[0][2]], mg_fine_ms_at_equal_error=None,
                   note="the target is more accurate than every MG(L+1) point")
    t_eq = out["mg_fine_ms_at_equal_error"]
    out["speedup_vs_mg_fine"] = t_eq / out["target_ms_per_step"] if t_eq else None
    return out


def start_runs(runs, x5, x6, fine_names, warmup):
    """Every run starts from the developed flow (level-L runs from x5, the
    others from x6), then `warmup` untimed steps."""
    for name, (c, mode) in runs.items():
        c.set_state(x6 if name in fine_names else x5)
    for name, (c, mode) in runs.items():
        for _ in range(warmup):
            c.step(mode)


def run_heldout(dn, torch, stream, flush, args, weights, feat_mean, feat_std):
    """Learning gain on held-out trajectories (seeds HELDOUT_SEEDS: own
    obstacle and viscosity, not in the corpus): from each developed flow,
    DNN-MG with the trained network and plain MG(L) against plain FP64
    MG(L+1), mean velocity and pressure errors over the steps."""
    import synthetic
    out = []
    K = max(2, min(args.steps, 10))
    for sd in HELDOUT_SEEDS:
        nu, ob = synthetic.viscosity(sd, *NU_RANGE), synthetic.obstacle_block(sd)
        com = dict(precision=dn.MIXED, dt=DT, obstacle_i0=ob[0], obstacle_j0=ob[1])
        x5, x6 = spun_up_state(dn, nu, ob, dn.MIXED)
        d = dn.Context(level_solve=L, replaced_levels=1, nu=nu, **com)
        d.set_weights(weights)
        d.set_feature_stats(feat_mean, feat_std)
        c = dn.Context(level_solve=L, nu=nu, **com)
        r = dn.Context(level_solve=L + 1, nu=nu, **dict(com, precision=dn.FP64))
        runs = {"dnnmg": (d, dn.NET), "mg_L": (c, dn.PLAIN), "mg_L+1_fp64": (r, dn.PLAIN)}
        start_runs(runs, x5, x6, ("mg_L+1_fp64",), max(1, args.warmup))
        _, series, stats, _ = compare_runs(runs, "mg_L+1_fp64", r, L, 1, stream, flush, torch, K,
                                           dn.kernel_launches)
        sm = summarize_series(series, "mg_L+1_fp64")
        out.append({"seed": sd, "nu": nu, "obstacle_block": list(ob), "steps": K,
                    "dnnmg_vel_err": sm["dnnmg"]["vel_l2_err_mean"],
                    "mg_L_vel_err": sm["mg_L"]["vel_l2_err_mean"],
                    "dnnmg_p_err": sm["dnnmg"]["p_l2_err_mean"],
                    "mg_L_p_err": sm["mg_L"]["p_l2_err_mean"],
                    "gain": sm["mg_L"]["vel_l2_err_mean"] / sm["dnnmg"]["vel_l2_err_mean"],
                    "fallbacks": sum(s["fallback"] for s in stats["dnnmg"])})
        for ctx in (d, c, r):
            ctx.close()
        torch.cuda.empty_cache()
    return {"trajectories": out,
            "mean_gain": sum(t["gain"] for t in out) / len(out),
            "setup": f"seeds {HELDOUT_SEEDS[0]}-{HELDOUT_SEEDS[-1]} (nu uniform in {NU_RANGE}, "
                     f"seeded obstacle), developed flow, {K} steps after "
                     f"{max(1, args.warmup)} warm-up steps; errors against plain FP64 MG(L+1)"}


def run_plain_fine(dn, torch, stream, flush, rank, steps=200):
    """The plain mixed-precision workload: the 1024x256 channel (level 6),
    nu = 0.005, dt = 0.005, seeded obstacle, `steps` steps from the impulsive
    start, with the velocity l2 error of every step against the FP64 build
    of the same solver stepping beside it (whose own parity with the oracle
    is 1e-10 in the tests)."""
    import synthetic
    ob = synthetic.obstacle_block(1000 + rank)
    com = dict(level_solve=6, nu=0.005, dt=0.005, obstacle_i0=ob[0], obstacle_j0=ob[1])
    mx = dn.Context(precision=dn.MIXED, **com)
    fp = dn.Context(precision=dn.FP64, **com)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t_mx = t_fp = 0.0
    err, pe, its = [], [], []
    for _ in range(steps):
        for c, acc in ((mx, 0), (fp, 1)):
            flush.zero_()
            ev[0].record(stream)
            st = c.step(dn.PLAIN)
            ev[1].record(stream)
            torch.cuda.synchronize()
            if acc == 0:
                t_mx += ev[0].elapsed_time(ev[1])
                its.append((st["newton_its"], st["gmres_its"]))
            else:
                t_fp += ev[0].elapsed_time(ev[1])
        ve, p_e = fp.relative_errors(6, mx.get_state(), fp.get_state())
        err.append(ve)
        pe.append(p_e)
    out = {"workload": "plain MG, 1024x256 channel (level 6, 790,275 DOFs), nu=0.005, dt=0.005, "
                       "seeded obstacle, from the impulsive start; FP32 V-cycle in FP64 Newton",
           "steps": steps, "ms_per_step_mixed": t_mx / steps, "ms_per_step_fp64": t_fp / steps,
           "steps_per_s_mixed": steps / (t_mx * 1e-3),
           "newton_its_mean": sum(a for a, _ in its) / steps,
           "gmres_its_mean": sum(b for _, b in its) / steps,
           "vel_l2_err_vs_fp64": {"max": max(err), "mean": sum(err) / steps, "last": err[-1],
                                  "every_20th": err[19::20]},
           "p_l2_err_vs_fp64": {"max": max(pe), "mean": sum(pe) / steps},
           "error_reference": "the FP64 build of the same solver (oracle parity 1e-10 in "
                              "tests/test_gpu_solver.py); the CPU oracle would take minutes "
                              "per step at this size"}
    mx.close()
    fp.close()
    return out


def run_plain_small(dn, torch, stream, rank, steps=20):
    """The plain FP64 workload: the 128x32 channel (level 3), nu = 0.01,
    dt = 0.01, seeded obstacle, Newton tolerance 1e-10, `steps` steps from
    the impulsive start.  Returns the block and the per-step states (host)
    for the comparison with the oracle."""
    import synthetic
    ob = synthetic.obstacle_block(1000 + rank)
    c = dn.Context(level_solve=3, precision=dn.FP64, nu=0.01, dt=0.01, newton_tol=1e-10,
                   obstacle_i0=ob[0], obstacle_j0=ob[1])
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t, states, its = 0.0, [], []
    for _ in range(steps):
        ev[0].record(stream)
        st = c.step(dn.PLAIN)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t += ev[0].elapsed_time(ev[1])
        its.append((st["newton_its"], st["gmres_its"]))
        states.append(c.get_state().cpu().numpy())
    c.close()
    return {"workload": "plain MG, FP64, 128x32 channel (level 3, 12,771 DOFs), nu=0.01, "
                        "dt=0.01, seeded obstacle, Newton tolerance 1e-10, from the impulsive "
                        "start",
            "obstacle_block": list(ob), "steps": steps, "ms_per_step": t / steps,
            "newton_its_mean": sum(a for a, _ in its) / steps,
            "gmres_its_mean": sum(b for _, b in its) / steps}, states


_ORACLE_PLAIN = """
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import fem, mesh, newton
levels = mesh.hierarchy(3, obstacle=({i0}, {j0}))
prm = fem.Params(nu=0.01, dt=0.01)
opt = newton.SolverOptions(newton_tol=1e-10)
x = mesh.initial_state(levels[-1])
times, xs = [], []
for _ in range({steps}):
    t = time.perf_counter()
    x, nit, git, nrm = newton.time_step(levels, x, prm, opt)
    times.append(time.perf_counter() - t)
    xs.append(x)
np.save({path!r}, np.array(xs))
print(json.dumps(times))
"""


def oracle_plain_small(block, states):
    """The oracle beside the plain FP64 128x32 workload: the same steps in a
    single-threaded process, timed; the GPU's state after every step is
    compared with the oracle's (relative l2)."""
    import tempfile
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "x.npy")
        code = _ORACLE_PLAIN.format(root=ROOT, i0=block["obstacle_block"][0],
                                    j0=block["obstacle_block"][1], steps=block["steps"], path=path)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             env=env, check=True)
        times = json.loads(out.stdout.strip().splitlines()[-1])
        xs = np.load(path)
    errs = [float(np.linalg.norm(g - o) / np.linalg.norm(o)) for g, o in zip(states, xs)]
    s = sum(times)
    return {"ms_per_step": 1e3 * s / len(times), "cores": 1,
            "gpu_vs_oracle_rel_l2_max": max(errs), "gpu_vs_oracle_rel_l2_last": errs[-1],
            "gpu_speedup": (1e3 * s / len(times)) / block["ms_per_step"]}


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    import synthetic

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ob = synthetic.obstacle_block(1000 + rank)
    common = dict(precision=dn.MIXED, dt=DT, obstacle_i0=ob[0], obstacle_j0=ob[1])
    if args.split >= 0:  # a fixed V-cycle plan instead of the autotuned one
        common.update(persistent_vcycle=args.split, persistent_mode=args.split_mode)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    hbm, bf16, bf16_sus, peak_kind = peaks()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device corpus of 32 trajectories and training (untimed setup) -------
    Xc, Yc, corpus_s = device_corpus(dn, torch, dn.MIXED)
    corpus = (Xc, Yc)
    net_ctx, feat_mean, feat_std, losses, train_ms = train_on(
        dn, torch, stream, common, L, 1, NU, corpus, len(CORPUS_SEEDS), CORPUS_T, TRAIN_ITERS)
    P = net_ctx.num_patches()
    infer_ms = time_infer(net_ctx, torch, stream, P, 40, 18, 2, 64)

    # ---- timed comparison from the developed flow ---------------------------
    x5, x6 = spun_up_state(dn, NU, ob, dn.MIXED)
    ref_ctx = dn.Context(level_solve=L + 1, nu=NU, **dict(common, precision=dn.FP64))
    coarse_ctx = dn.Context(level_solve=L, nu=NU, **common)
    sweep = {}
    for tol, rtol, nmax, gmax in SWEEP:
        name = f"mg_L+1@{tol:g}" if nmax > 1 else "mg_L+1@one_newton_one_vcycle"
        sweep[name] = dn.Context(level_solve=L + 1, nu=NU, newton_tol=tol, gmres_rtol=rtol,
                                 newton_max=nmax, gmres_maxit=gmax, **common)
    runs = {"dnnmg": (net_ctx, dn.NET), "mg_L": (coarse_ctx, dn.PLAIN),
            "mg_L+1_fp64": (ref_ctx, dn.PLAIN), **{k: (c, dn.PLAIN) for k, c in sweep.items()}}
    fine_names = ("mg_L+1_fp64",) + tuple(sweep)
    warm = max(NET_WARMUP, args.warmup)
    start_runs(runs, x5, x6, fine_names, warm)
    barrier()

    def nvtx(name, begin):  # kernel profilers select the DNN-MG launches by this range
        if name == "dnnmg":
            torch.cuda.nvtx.range_push("dnnmg_step") if begin else torch.cuda.nvtx.range_pop()

    with ClockSampler(dev) as clk:
        times, series, stats, counts = compare_runs(runs, "mg_L+1_fp64", ref_ctx, L, 1, stream,
                                                    flush, torch, args.steps, dn.kernel_launches,
                                                    nvtx)
    barrier()
    launches = counts["dnnmg"]
    K = args.steps
    summary = summarize_series(series, "mg_L+1_fp64")
    eq = equal_error(times, summary, K, list(sweep))
    # stage breakdown: more DNN-MG steps with per-stage events (untimed; the
    # events would perturb the timed steps)
    net_ctx.profile(True)
    for k in range(args.steps):
        net_ctx.step(dn.NET)
    stage = {}
    for sid, nm in enumerate(dn.STAGES):
        n, t = net_ctx.profile_read(sid)
        stage[nm] = {"launches": n, "ms": round(t, 4)}
    vp_n, vp_ms = net_ctx.profile_read(0, L)
    vs_n, vs_ms = net_ctx.profile_read(11)  # persistent sub-cycle launches
    net_ctx.profile(False)

    # ---- V-cycle throughput at levels 6 and 5 (current linearisations) -----------
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def vcycle_ms(c, level):
        x = c.get_state()
        c.linearize(x)
        b = torch.from_numpy(synthetic.random_vector(7, ndof(level))).float().cuda()
        xv = torch.empty_like(b)
        for _ in range(3):
            c.vcycle(level, b, xv)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(10):
            c.vcycle(level, b, xv)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 10
    fine_mixed = sweep["mg_L+1@1e-10"]
    vc6, vc5 = vcycle_ms(fine_mixed, L + 1), vcycle_ms(coarse_ctx, L)

    # ---- end to end: DNN-MG steps with the state exchanged through host memory ----
    host_in = torch.empty(ndof(L), dtype=torch.float64).pin_memory()
    host_out = torch.empty(ndof(L), dtype=torch.float64).pin_memory()
    host_in.copy_(net_ctx.get_state().cpu())
    E = E2E_STEPS
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for _ in range(E):
        net_ctx.step_io(dn.NET, host_in, host_out)
        host_in, host_out = host_out, host_in
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t_e2e) / E
    plan_dnnmg, plan_fine = net_ctx.vcycle_plan(), fine_mixed.vcycle_plan()
    weights = net_ctx.get_weights()
    for c in [ref_ctx, coarse_ctx] + list(sweep.values()):
        c.close()
    torch.cuda.empty_cache()

    # ---- held-out trajectories: what the trained network gains ---------------
    heldout = run_heldout(dn, torch, stream, flush, args, weights, feat_mean, feat_std)
    # ---- the plain workloads: FP64 128x32, mixed 1024x256 ----------------------
    small, small_states = run_plain_small(dn, torch, stream, rank)
    plain_fine = run_plain_fine(dn, torch, stream, flush, rank)
    # ---- batched problems: 64 uneven channels, one launch per stage ---------
    batched = run_batched(dn, torch, stream, flush, args, weights, feat_mean, feat_std, rank)
    # ---- large DNN-MG: the network replaces two levels -----------------------
    large = run_large(dn, torch, stream, flush, args, common)
    # ---- the network sizes of Table 1 on the same corpus ---------------------
    sizes = run_sizes(dn, torch, stream, flush, args, common, corpus, (x5, x6))
    del corpus, Xc, Yc
    torch.cuda.empty_cache()

    ms = slowest_rank_ms(times["dnnmg"], world, "cuda")
    if rank != 0:
        return None
    bytes_per_pass = fluid_cells(L) / 4 * 576 + nnodes(L) * 44
    avg_pass_ms = vp_ms / max(vp_n, 1)
    pass_gbs = bytes_per_pass / (avg_pass_ms * 1e-3) / 1e9 if vp_n else 0.0
    # the dominant kernel of the DNN-MG step: the persistent sub-cycle of the
    # small levels (if the plan has one and it takes longer), else the colour pass
    build_id = source_hash()
    if vs_n and vs_ms > vp_ms:
        split = plan_dnnmg["split_level"]
        kname = ("vcycle_kernel<float>" if plan_dnnmg["split_mode"] == 0 else
                 "vcycle_cluster_kernel<float>")
        dom = {"kernel": f"{kname} (V(2,2) sub-cycle of levels {split}..1, one launch)",
               "algorithmic_bytes_per_launch": vcycle_bytes(split), "avg_launch_ms": vs_ms / vs_n,
               "launches": vs_n,
               "traffic": NCU_TRAFFIC.get(build_id, {}).get(f"{kname}@split{split}")}
    else:
        dom = {"kernel": f"vanka_pass_tiled_kernel<float> (level {L}, one colour pass)",
               "algorithmic_bytes_per_launch": bytes_per_pass, "avg_launch_ms": avg_pass_ms,
               "launches": vp_n, "traffic": None}
    achieved = dom["algorithmic_bytes_per_launch"] / (dom["avg_launch_ms"] * 1e-3) / 1e9
    l2_gbs = l2_bandwidth(torch, stream)
    f_fwd, f_train = net_flops()
    mean = lambda v: sum(v) / len(v)
    comparison = {
        name: {"ms_per_step": times[name] / K,
               "newton_its": mean([s["newton_its"] for s in stats[name]]),
               "gmres_its": mean([s["gmres_its"] for s in stats[name]]),
               "fallbacks": sum(s["fallback"] for s in stats[name]),
               **summary[name]}
        for name in runs}
    return {
        "metric": METRIC,
        "value": job_throughput(ms, K, world),
        "unit": "time steps/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 solver, bf16 network", "data": "synthetic",
        "config": {"workload": WORKLOAD, "level_solve": L, "level_net": L + 1, "dofs_L": ndof(L),
                   "dofs_L+1": ndof(L + 1), "patches": P, "obstacle_block": list(ob),
                   "nu": NU, "dt": DT, "l2": "flushed (256 MB write) before every step",
                   "start": f"developed flow: {SPIN_STEPS} level-{L} steps of {SPIN_DT} s from "
                            f"rest (t = 1 s), P to level {L + 1}, then {warm} untimed steps "
                            f"of every method (at least {NET_WARMUP}: the network's GRU memory "
                            f"starts at zero; DNN-MG's third and fourth steps take a third "
                            f"Newton iteration while it fills)",
                   "parallelism": f"independent replicas x{world}",
                   "network_training": f"{TRAIN_ITERS} Adam steps, B={TRAIN_B}, T={TRAIN_T} "
                                       f"windows, device corpus of {len(CORPUS_SEEDS)} "
                                       f"trajectories x {CORPUS_T} fine steps"},
        "comparison": comparison,
        "equal_error": eq,
        "corpus": {"trajectories": len(CORPUS_SEEDS), "steps_per_trajectory": CORPUS_T,
                   "seeds": [CORPUS_SEEDS[0], CORPUS_SEEDS[-1]], "nu_range": list(NU_RANGE),
                   "rows": len(CORPUS_SEEDS) * CORPUS_T * P,
                   "spinup": f"{SPIN_STEPS} level-{L} steps of {SPIN_DT} s, {RELAX_STEPS} "
                             f"relaxation steps on level {L + 1}",
                   "seconds": corpus_s},
        "heldout": heldout,
        "plain_fp64_small": small,
        "plain_mixed_fine": plain_fine,
        "vcycle": {"split_level_dnnmg": plan_dnnmg["split_level"],
                   "split_level_fine": plan_fine["split_level"],
                   "plan_dnnmg": plan_dnnmg, "plan_fine": plan_fine,
                   "level6_ms": vc6, "level6_dof_per_s": ndof(6) / (vc6 * 1e-3),
                   "level6_gbs": vcycle_bytes(6) / (vc6 * 1e-3) / 1e9,
                   "level5_ms": vc5, "level5_dof_per_s": ndof(5) / (vc5 * 1e-3),
                   "level5_gbs": vcycle_bytes(5) / (vc5 * 1e-3) / 1e9},
        "stages_ms_dnnmg": stage,
        "roofline": {"kernel": dom["kernel"], "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": dom["traffic"], "build": build_id,
                     "algorithmic_bytes_per_launch": dom["algorithmic_bytes_per_launch"],
                     "avg_launch_ms": dom["avg_launch_ms"], "launches": dom["launches"],
                     "timing": "CUDA events around each launch in a repeat of the timed steps",
                     # the level-5 cycle's data live in L2 between its phases: the same
                     # algorithmic bytes against the L2 bandwidth measured by a copy here
                     "l2": {"achieved": achieved, "peak": l2_gbs, "unit": "GB/s",
                            "frac": achieved / l2_gbs,
                            "peak_kind": "measured here: copies between two 24 MiB buffers resident in L2"},
                     "others": {
                         **({f"vanka_pass_tiled_kernel<float> level {L}": {
                             "achieved_gbs": pass_gbs, "frac": pass_gbs / hbm,
                             "avg_launch_ms": avg_pass_ms, "bytes_per_launch": bytes_per_pass}}
                            if vp_n else {}),           # not launched when level L is persistent
                         "V(2,2) cycle level 5 (whole cycle)": {
                             "achieved_gbs": vcycle_bytes(5) / (vc5 * 1e-3) / 1e9,
                             "frac": vcycle_bytes(5) / (vc5 * 1e-3) / 1e9 / hbm},
                         "V(2,2) cycle level 6 (whole cycle)": {
                             "achieved_gbs": vcycle_bytes(6) / (vc6 * 1e-3) / 1e9,
                             "frac": vcycle_bytes(6) / (vc6 * 1e-3) / 1e9 / hbm}}},
        "network": {"forward_ms": infer_ms, "patches": P,
                    "forward_tflops": f_fwd * P / (infer_ms * 1e-3) / 1e12,
                    "forward_frac_bf16": f_fwd * P / (infer_ms * 1e-3) / 1e12 / bf16,
                    "forward_hbm_gbs": P * (80 + 1024 + 72) / (infer_ms * 1e-3) / 1e9,
                    "forward_frac_hbm": P * (80 + 1024 + 72) / (infer_ms * 1e-3) / 1e9 / hbm,
                    "train_ms_per_iter": train_ms,
                    "train_patch_steps_per_s": TRAIN_B * TRAIN_T / (train_ms * 1e-3),
                    "train_tflops": f_train * TRAIN_B * TRAIN_T / (train_ms * 1e-3) / 1e12,
                    "train_frac_bf16_sustained":
                        f_train * TRAIN_B * TRAIN_T / (train_ms * 1e-3) / 1e12 / bf16_sus,
                    "loss_first": losses[0], "loss_last": losses[-1]},
        "batched": batched,
        "large_dnnmg": large,
        "network_sizes": {"sizes": sizes,
                          "setup": f"each trained {TRAIN_ITERS} Adam steps on the corpus of "
                                   f"the default network; {args.steps} DNN-MG steps vs plain MG "
                                   f"on level {L + 1} from the developed flow after "
                                   f"{max(NET_WARMUP, args.warmup)} warm-up steps"},
        "clocks": clk.summary(),
        "e2e": {"value": 1.0 / t_e2e, "unit": "time steps/s",
                "h2d_bytes_per_step": 8 * ndof(L), "d2h_bytes_per_step": 8 * ndof(L),
                "steps": E2E_STEPS,
                "note": "dnnmg_step_io steps with the state from and to pinned host memory, "
                        "one coarse refactorisation period (it holds exactly one)"},
        "gpu_launches": int(launches),
        "_small_states": small_states,
    }


BATCH_N, BATCH_SEED = 64, 5000


def batch_problems(dn, mode_levels, precision):
    """64 channels with seeded obstacles and nu in [0.005, 0.02]; finest
    solved levels cycle through mode_levels (uneven sizes)."""
    import numpy as np
    import synthetic
    rng = np.random.default_rng(BATCH_SEED)
    cfgs = []
    for p in range(BATCH_N):
        ob = synthetic.obstacle_block(BATCH_SEED + p)
        cfgs.append(dn.default_config(level_solve=mode_levels[p % len(mode_levels)],
                                      precision=precision, nu=float(rng.uniform(0.005, 0.02)),
                                      dt=DT, obstacle_i0=ob[0], obstacle_j0=ob[1]))
    return cfgs


def run_batched(dn, torch, stream, flush, args, weights, feat_mean, feat_std, rank):
    """Batched engine on 64 uneven problems: DNN-MG steps (solve on levels
    3-5, network on 4-6: finest grids 256x64 .. 1024x256) and plain MG steps
    (levels 4-6), each a lock-step batch with one launch per stage; plain MG
    also run problem by problem with single contexts for comparison."""
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    out = {}
    K = max(2, min(args.steps, 4))
    for name, levels, mode in (("dnnmg", (3, 4, 5), dn.NET), ("plain", (4, 5, 6), dn.PLAIN)):
        cfgs = batch_problems(dn, levels, dn.MIXED)
        B = dn.Batch(cfgs)
        if mode == dn.NET:
            B.set_weights(weights)
            B.set_feature_stats(feat_mean, feat_std)
        for _ in range(max(2, args.warmup)):
            B.step(mode)
        torch.cuda.synchronize()
        l0 = dn.kernel_launches()
        t = 0.0
        its = []
        for _ in range(K):
            flush.zero_()
            ev[0].record(stream)
            st = B.step(mode)
            ev[1].record(stream)
            torch.cuda.synchronize()
            t += ev[0].elapsed_time(ev[1])
            its.append(sum(s["gmres_its"] for s in st) / len(st))
        launches = dn.kernel_launches() - l0
        B.profile(True)
        B.step(mode)
        stage = {}
        for sid, nm in enumerate(dn.STAGES):
            n, tt = B.profile_read(sid)
            if n:
                stage[nm] = {"launches": n, "ms": round(tt, 3)}
        B.profile(False)
        dofs = sum(ndof(c.level_solve) for c in cfgs)
        out[name] = {"problems": len(cfgs), "levels_solved": list(levels),
                     "dofs_solved": dofs, "ms_per_step": t / K,
                     "problem_steps_per_s": len(cfgs) * K / (t * 1e-3),
                     "dof_steps_per_s": dofs * K / (t * 1e-3),
                     "mean_gmres_its_per_problem": sum(its) / len(its),
                     "launches_per_step": launches / K, "stage_ms_one_step": stage}
        del B
        torch.cuda.empty_cache()
    # the same plain problems one by one (single contexts, one timed step each)
    cfgs = batch_problems(dn, (4, 5, 6), dn.MIXED)
    t = 0.0
    for c in cfgs:
        ctx = dn.Context(cfg=c)
        ctx.step(dn.PLAIN)
        ctx.step(dn.PLAIN)
        torch.cuda.synchronize()
        flush.zero_()
        ev[0].record(stream)
        ctx.step(dn.PLAIN)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t += ev[0].elapsed_time(ev[1])
        ctx.close()
    out["plain_sequential_ms_per_step"] = t
    out["plain_batched_speedup"] = t / out["plain"]["ms_per_step"]
    out["workload"] = ("64 channels, seeded obstacle, nu uniform in [0.005, 0.02], dt=0.005, "
                       "mixed FP32/FP64; finest levels cycle 256x64, 512x128, 1024x256")
    return out


def run_vcycles(args):
    """V-cycles on one level only (after --warmup untimed ones): a short
    command for kernel profilers.  --level picks the level (default 6),
    --split the persistent sub-cycle level (-1: autotuned)."""
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    import synthetic
    build.build()
    lev = args.level
    ob = synthetic.obstacle_block(1000)
    kw = {} if args.split < 0 else dict(persistent_vcycle=args.split,
                                        persistent_mode=args.split_mode)
    ctx = dn.Context(level_solve=lev, precision=dn.MIXED, nu=0.005, dt=DT, obstacle_i0=ob[0],
                     obstacle_j0=ob[1], stream_pass=args.stream_pass, **kw)
    x = ctx.get_state()
    ctx.linearize(x)
    b = torch.from_numpy(synthetic.random_vector(7, ndof(lev))).float().cuda()
    xv = torch.empty_like(b)
    for _ in range(args.warmup):
        ctx.vcycle(lev, b, xv)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("vcycles")  # kernel profilers select these launches
    for _ in range(args.steps):
        ctx.vcycle(lev, b, xv)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"mode": "vcycle", "level": lev, "cycles": args.warmup + args.steps,
                      "plan": ctx.vcycle_plan(), "norm": float(xv.norm())}))


def run_net(args):
    """Patch network only: --warmup + --steps inference passes over the
    61,440 patches of the 1024x256 level, then as many training steps at the
    benchmark's batch (random weights and data): a short command for kernel
    profilers."""
    import numpy as np
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    import synthetic
    build.build()
    ctx = dn.Context(level_solve=L, precision=dn.MIXED, nu=NU, dt=DT, train_batch=TRAIN_B,
                     train_seq=TRAIN_T)
    ctx.set_weights(synthetic.random_weights(77, ctx.num_params(), 0.05).astype(np.float32))
    P = ctx.num_patches()
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(P, 40, device="cuda", generator=g).to(torch.bfloat16)
    h = torch.zeros(2, P, 64, device="cuda")
    out = torch.empty(P, 18, device="cuda")
    X = torch.randn(TRAIN_B, TRAIN_T, 40, device="cuda", generator=g).to(torch.bfloat16)
    Y = 0.01 * torch.randn(TRAIN_B, TRAIN_T, 18, device="cuda", generator=g)
    for _ in range(args.warmup + args.steps):
        ctx.patch_infer(x, h, out)
    loss = [ctx.train_step(X, Y, TRAIN_B, TRAIN_T, 1e-4) for _ in range(args.warmup + args.steps)]
    torch.cuda.synchronize()
    print(json.dumps({"mode": "net", "patches": P, "train_batch": TRAIN_B, "train_seq": TRAIN_T,
                      "loss_last": loss[-1]}))


PERIODIC_T = 10.0              # end time (s) of the long run, as in Sec. 3.4
PERIODIC_WINDOW = 1.0          # compared over [T - 1 s, T]
PERIODIC_TRAIN = (1.0, 8.0)    # training windows are cut from the reference in this interval
PERIODIC_WINDOWS, PERIODIC_WIN_STEPS, PERIODIC_ITERS = 8, 20, 300


def series_summary(t, drag, lift):
    """Mean and half peak-to-peak of drag and lift, and, when the lift
    oscillates, its period from the upward crossings of its mean."""
    import numpy as np
    d, l = np.asarray(drag), np.asarray(lift)
    out = {"drag_mean": float(d.mean()), "drag_amp": float((d.max() - d.min()) / 2),
           "lift_mean": float(l.mean()), "lift_amp": float((l.max() - l.min()) / 2)}
    z = l - l.mean()
    up = [t[i] - z[i] * (t[i + 1] - t[i]) / (z[i + 1] - z[i])
          for i in range(len(z) - 1) if z[i] < 0 <= z[i + 1]]
    out["lift_period"] = float(np.diff(up).mean()) if len(up) >= 2 else None
    return out


def first_max(v):
    """Index of the first interior local maximum of v (None if none)."""
    for i in range(1, len(v) - 1):
        if v[i] > v[i - 1] and v[i] >= v[i + 1]:
            return i
    return None


def run_periodic(args):
    """Long horizon (Sec. 3.4): the default DNN-MG workload from the
    impulsive start to t = 10 s.  The plain multigrid reference on the finer
    level runs first; it supplies the training corpus (windows of
    consecutive steps cut from t in [1, 8] s) and its states over the
    compared window [9, 10] s.  The network is trained on that corpus; then
    DNN-MG and plain multigrid on the coarse level run from t = 0.  Printed:
    per method the velocity and pressure errors against the reference over
    the window, drag and lift means, amplitudes and lift period, and, when
    the lift oscillates, the drag and lift differences after aligning the
    phases on the first lift maximum of the window (the paper's procedure);
    with --steps the series are printed every that many steps."""
    import numpy as np
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    import synthetic
    build.build()
    stream = torch.cuda.current_stream()
    ob = synthetic.obstacle_block(1000)
    common = dict(precision=dn.MIXED, dt=DT, obstacle_i0=ob[0], obstacle_j0=ob[1])
    nsteps = int(round(PERIODIC_T / DT))
    w0 = nsteps - int(round(PERIODIC_WINDOW / DT))
    top = L + 1
    ref = dn.Context(level_solve=top, nu=NU, **common)
    sctx = dn.Context(level_solve=L, nu=NU, replaced_levels=1, **common)
    starts = np.linspace(PERIODIC_TRAIN[0] / DT, PERIODIC_TRAIN[1] / DT - PERIODIC_WIN_STEPS,
                         PERIODIC_WINDOWS).astype(int)
    sample_steps = set()
    for s0 in starts:
        sample_steps.update(range(int(s0), int(s0) + PERIODIC_WIN_STEPS))
    Xs, Ys, ref_states = [], [], []
    series = {k: {"drag": [], "lift": [], "div": [], "vel_err": [], "p_err": []}
              for k in ("mg_L+1", "dnnmg", "mg_L")}
    t_run = {}
    prev = ref.get_state().clone()
    t0 = time.perf_counter()
    for n in range(nsteps):
        ref.step(dn.PLAIN)
        cur = ref.get_state().clone()
        if n in sample_steps:
            X, Y = sctx.make_sample(prev, cur)
            Xs.append(X)
            Ys.append(Y)
        if n >= w0:
            ref_states.append(cur)
            jd, fd, fl = ref.functionals(top, cur, prev)
            for key, v in zip(("drag", "lift", "div", "vel_err", "p_err"), (fd, fl, jd, 0.0, 0.0)):
                series["mg_L+1"][key].append(v)
        prev = cur
    torch.cuda.synchronize()
    t_run["mg_L+1"] = time.perf_counter() - t0
    sctx.close()
    corpus = (torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous())
    del Xs, Ys
    net_ctx, _, _, losses, train_ms = train_on(dn, torch, stream, common, L, 1, NU, corpus,
                                               PERIODIC_WINDOWS, PERIODIC_WIN_STEPS,
                                               PERIODIC_ITERS)
    del corpus
    torch.cuda.empty_cache()
    coarse = dn.Context(level_solve=L, nu=NU, **common)
    fallbacks = 0
    for name, c, mode in (("dnnmg", net_ctx, dn.NET), ("mg_L", coarse, dn.PLAIN)):
        prev = None  # the state before the window, taken at step w0 - 1
        t0 = time.perf_counter()
        for n in range(nsteps):
            st = c.step(mode)
            if mode == dn.NET:
                fallbacks += st["fallback"]
            if n >= w0 - 1:
                cur = on_fine_level(c, mode == dn.NET, ref, top)
                if n >= w0:
                    ve, pe = ref.relative_errors(top, cur, ref_states[n - w0])
                    jd, fd, fl = ref.functionals(top, cur, prev)
                    for key, v in zip(("drag", "lift", "div", "vel_err", "p_err"),
                                      (fd, fl, jd, ve, pe)):
                        series[name][key].append(v)
                prev = cur
        torch.cuda.synchronize()
        t_run[name] = time.perf_counter() - t0
    t = [(w0 + 1 + i) * DT for i in range(nsteps - w0)]
    r = series["mg_L+1"]
    periodic = series_summary(t, r["drag"], r["lift"])["lift_amp"] > 1e-3 * abs(np.mean(r["drag"]))
    out = {"mode": "periodic", "workload": WORKLOAD, "t_end": PERIODIC_T,
           "window": [PERIODIC_T - PERIODIC_WINDOW, PERIODIC_T], "steps": nsteps,
           "training": f"{PERIODIC_ITERS} Adam steps on {PERIODIC_WINDOWS} windows of "
                       f"{PERIODIC_WIN_STEPS} consecutive reference steps in t = "
                       f"{PERIODIC_TRAIN[0]}..{PERIODIC_TRAIN[1]} s",
           "loss_first": losses[0], "loss_last": losses[-1], "train_ms_per_iter": train_ms,
           "dnnmg_fallbacks": fallbacks, "lift_oscillates": bool(periodic), "methods": {}}
    i_ref = first_max(r["lift"]) if periodic else None
    for name, sr in series.items():
        m = {"wall_s": t_run[name], **series_summary(t, sr["drag"], sr["lift"]),
             "vel_l2_err_mean": float(np.mean(sr["vel_err"])),
             "p_l2_err_mean": float(np.mean(sr["p_err"])),
             "div_mean": float(np.mean(sr["div"])),
             "drag_rel_diff_mean": float(np.mean(np.abs(np.subtract(sr["drag"], r["drag"])))
                                         / abs(np.mean(r["drag"])))}
        if periodic:
            i_m = first_max(sr["lift"])
            if i_m is not None and i_ref is not None:
                sh = i_m - i_ref
                a0, a1 = max(0, -sh), min(len(t), len(t) - sh)
                dd = [sr["drag"][i + sh] - r["drag"][i] for i in range(a0, a1)]
                dl = [sr["lift"][i + sh] - r["lift"][i] for i in range(a0, a1)]
                m.update({"phase_shift_s": sh * DT,
                          "aligned_drag_maxdiff": float(np.max(np.abs(dd))),
                          "aligned_lift_maxdiff": float(np.max(np.abs(dl)))})
        if args.steps > 1:
            m["series_every"] = args.steps
            m["drag"] = sr["drag"][::args.steps]
            m["lift"] = sr["lift"][::args.steps]
        out["methods"][name] = m
    print(json.dumps(out))


def run_dnnmg_steps(args):
    """DNN-MG steps only (seeded weights, no corpus): --warmup untimed and
    --steps timed steps of the default workload from the developed flow,
    each inside an NVTX range "dnnmg_step" that kernel profilers select; a
    short command for launch lists of the step."""
    import numpy as np
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    import synthetic
    build.build()
    ob = synthetic.obstacle_block(1000)
    ctx = dn.Context(level_solve=L, replaced_levels=1, precision=dn.MIXED, nu=NU, dt=DT,
                     obstacle_i0=ob[0], obstacle_j0=ob[1])
    ctx.set_weights(synthetic.random_weights(77, ctx.num_params(), 0.02).astype(np.float32))
    x5, _ = spun_up_state(dn, NU, ob, dn.MIXED)
    ctx.set_state(x5)
    for _ in range(args.warmup):
        ctx.step(dn.NET)
    torch.cuda.synchronize()
    stats = []
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("dnnmg_step")
        stats.append(ctx.step(dn.NET))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    print(json.dumps({"mode": "dnnmg", "steps": args.steps,
                      "ms": [round(s["ms"], 3) for s in stats], "plan": ctx.vcycle_plan()}))


def run_coarse(args):
    """Coarse level only: --warmup + --steps refactorisations of the level-1
    Jacobian (assembly, cluster band LU, explicit inverse) through
    dnnmg_linearize on the state of the DNN-MG workload after three plain
    steps; prints the mean time of one linearisation (CUDA events)."""
    import torch
    from paper_2106_07687_gb300 import build, dnnmg as dn
    build.build()
    ctx = dn.Context(level_solve=L, precision=dn.MIXED, nu=NU, dt=DT)
    for _ in range(3):
        ctx.step(dn.PLAIN)
    x = ctx.get_state()
    for _ in range(args.warmup):
        ctx.linearize(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.linearize(x)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "coarse", "level": 1, "linearize_ms":
                      e0.elapsed_time(e1) / max(args.steps, 1)}))


def summarize_launches(path):
    """Per-kernel launches, total time and share of an ncu CSV launch list
    (gpu__time_duration.sum per launch)."""
    import collections
    import csv
    import re

    def name(full):
        t = full.replace("(anonymous namespace)", "").replace("<unnamed>", "")
        t = re.sub(r"\(.*$", "", t)
        t = re.sub(r"^void\s+", "", t.strip())
        base = t.split("<")[0]
        return base.split("::")[-1] + t[len(base):]

    rows = list(csv.reader(open(path)))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value",
                                           "Metric Unit"))
    scale = {"nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[hdr + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        a = agg[name(r[ki])]
        a[0] += 1
        a[1] += float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total_us':>10s} {'share':>6s}")
    for k, (n, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k[:44]:44s} {n:8d} {t:10.1f} {100 * t / tot:5.1f}%")


REF_BUDGET_S = 150.0  # the reference arm's timed oracle steps stop after this long


def run_reference(args, rank, world):
    """The FP64 oracle on the benchmarked workload: consecutive DNN-MG steps
    (solve on level 5, network on level 6) from the impulsive start on the
    host cores, single-threaded.  The oracle keeps no caches, so the warm-up
    is one untimed step at most; the timed steps stop after REF_BUDGET_S
    seconds (at least one step), so that the run ends within a few minutes."""
    if rank != 0:
        return None
    t = time.perf_counter()
    per = oracle_dnnmg_steps(L, steps=args.steps, warm=min(args.warmup, 1), threads=1,
                             budget=REF_BUDGET_S)
    mean = sum(per) / len(per)
    v = 1.0 / mean
    sample = (f"{len(per)} consecutive DNN-MG time steps (of the {args.steps} requested) of the "
              f"FP64 oracle on the benchmarked workload (solve on 512x128, level {L}; network "
              f"on 1024x256), after {min(args.warmup, 1)} untimed step(s) from the impulsive "
              f"start; single-threaded; stopped after {REF_BUDGET_S:.0f} s of timed steps")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "time steps/s",
            "n_gpus": world, "steps": len(per), "warmup": min(args.warmup, 1),
            "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "level_solve": L, "dofs_L": ndof(L)},
            "cpu_baseline": {"value": v, "unit": "time steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "time steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--level", type=int, default=6, help="--mode vcycle: level")
    ap.add_argument("--split", type=int, default=-1,
                    help="fixed persistent V-cycle split level (-1: autotuned; 0: none)")
    ap.add_argument("--stream-pass", type=int, default=0, choices=[-1, 0, 1],
                    help="--mode vcycle: streaming colour pass never (-1), autotuned (0), "
                         "always (1)")
    ap.add_argument("--split-mode", type=int, default=-1,
                    help="with --split: 0 cooperative grid, 1 single cluster, -1 autotuned")
    ap.add_argument("--summarize-launches", metavar="CSV", default=None,
                    help="print the per-kernel table of an ncu launch list and exit")
    ap.add_argument("--mode", choices=["step", "vcycle", "net", "coarse", "periodic", "dnnmg"],
                    default="step",
                    help="vcycle: only V-cycles on --level; net: only the patch network; "
                         "coarse: only coarse-level factorisations; dnnmg: only DNN-MG steps "
                         "(short runs for kernel profilers); periodic: the long run to "
                         "t = 10 s with the functionals over the last second")
    args = ap.parse_args()
    if args.summarize_launches:
        summarize_launches(args.summarize_launches)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.mode == "vcycle":
        run_vcycles(args)
        return
    if args.mode == "net":
        run_net(args)
        return
    if args.mode == "coarse":
        run_coarse(args)
        return
    if args.mode == "dnnmg":
        run_dnnmg_steps(args)
        return
    if args.mode == "periodic":
        run_periodic(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world)
        small_states = out.pop("_small_states") if out is not None else None
        if out is not None and world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
            out["plain_fp64_small"]["oracle"] = oracle_plain_small(out["plain_fp64_small"],
                                                                   small_states)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
