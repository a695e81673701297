"""Benchmark of the DNN-MG hot path on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: a mixed-precision plain multigrid time step on the 1024x256
channel (level 6, 790,275 DOFs, nu = 0.005, dt = 0.005; obstacle seeded);
the input is the solver state already resident in HBM.  One JSON line is
printed by rank 0.  --impl reference times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time/step & V-cycle DOF/s: DNN-MG vs plain MG on 1 GB300 at equal L2 err; %HBM/TC peak"
LEVEL, NU, DT = 6, 0.005, 0.005
WORKLOAD = "plain MG time step, 1024x256 channel (level 6, 790,275 DOFs), nu=0.005, dt=0.005, mixed FP32/FP64"
ORACLE_LEVEL = 5          # bounded CPU sample: one oracle step on 512x128, scaled by DOFs
L2_BYTES = 129 * 2 ** 20


def ndof(level):
    return 3 * (16 * 2 ** level + 1) * (4 * 2 ** level + 1)


def fluid_cells(level):
    n = 16 * 4 * 4 ** level
    return n - 4 * 4 ** level


def oracle_step_seconds(level, steps=1, warm=1):
    """Time the FP64 oracle on `steps` plain time steps (after `warm`) in a
    fresh single-threaded process; returns seconds per step."""
    code = f"""
import time, sys
sys.path.insert(0, {ROOT!r})
import synthetic
from oracle import fem, mesh, newton
ob = synthetic.obstacle_block(1000)
levels = mesh.hierarchy({level}, obstacle=ob)
prm = fem.Params(nu={NU}, dt={DT})
opt = newton.SolverOptions()
x = mesh.initial_state(levels[-1])
for _ in range({warm}):
    x, *_ = newton.time_step(levels, x, prm, opt)
t = time.perf_counter()
for _ in range({steps}):
    x, *_ = newton.time_step(levels, x, prm, opt)
print((time.perf_counter() - t) / {steps})
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         check=True)
    return float(out.stdout.strip().splitlines()[-1])


def cpu_baseline(steps=1):
    s = oracle_step_seconds(ORACLE_LEVEL, steps=steps)
    scale = ndof(LEVEL) / ndof(ORACLE_LEVEL)
    return {"value": 1.0 / (s * scale), "unit": "time steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} plain time step(s) of the FP64 oracle on the 512x128 channel "
                      f"(level {ORACLE_LEVEL}, {ndof(ORACLE_LEVEL)} DOFs, same physics) after one "
                      f"warm-up step, {s:.2f} s/step, scaled by the DOF ratio "
                      f"{scale:.3f} to level {LEVEL}; single-threaded"}


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
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = max(float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p.get("bf16_tflops"), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


def run_ours(args, rank, world):
    import torch
    from paper_2106_07687_gb300 import build, dnnmg
    import synthetic

    build.build()
    lib = dnnmg.load()
    lib.dnnmg_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.dnnmg_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]
    lib.dnnmg_kernel_launches.restype = ctypes.c_uint64
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ob = synthetic.obstacle_block(1000 + rank)
    ctx = dnnmg.Context(level_solve=LEVEL, precision=dnnmg.MIXED, nu=NU, dt=DT,
                        obstacle_i0=ob[0], obstacle_j0=ob[1])
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stats = []
    for _ in range(args.warmup):
        ctx.step(dnnmg.PLAIN)
    barrier()
    lib.dnnmg_profile(ctx.h, 1)
    launches0 = lib.dnnmg_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            stats.append(ctx.step(dnnmg.PLAIN))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier()
    launches = lib.dnnmg_kernel_launches() - launches0
    ms_steps = sum(a.elapsed_time(b) for a, b in ev)
    stage = {}
    names = ["vanka_pass", "vanka_setup", "apply", "defect", "transfer", "coarse_factor",
             "coarse_solve", "krylov", "residual64"]
    for sid, nm in enumerate(names):
        n, t = ctypes.c_int64(), ctypes.c_double()
        lib.dnnmg_profile_read(ctx.h, sid, -1, ctypes.byref(n), ctypes.byref(t))
        stage[nm] = {"launches": n.value, "ms": round(t.value, 4)}
    n, t = ctypes.c_int64(), ctypes.c_double()
    lib.dnnmg_profile_read(ctx.h, 0, LEVEL, ctypes.byref(n), ctypes.byref(t))
    vp_launches, vp_ms = n.value, t.value
    lib.dnnmg_profile(ctx.h, 0)

    # V-cycle throughput on level 6 at the current linearisation
    x = ctx.get_state()
    ctx.linearize(x)
    b = torch.from_numpy(synthetic.random_vector(7, ndof(LEVEL))).float().cuda()
    xv = torch.empty_like(b)
    for _ in range(3):
        ctx.vcycle(LEVEL, b, xv)
    R = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(R):
        ctx.vcycle(LEVEL, b, xv)
    e1.record(stream)
    torch.cuda.synchronize()
    vcycle_ms = e0.elapsed_time(e1) / R

    # end to end through the public API with host buffers: H2D state, step, D2H state
    host_x = torch.empty(ndof(LEVEL), dtype=torch.float64).pin_memory()
    host_x.copy_(x.cpu())
    dev_x = torch.empty_like(x)
    E = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for _ in range(E):
        dev_x.copy_(host_x, non_blocking=True)
        ctx.set_state(dev_x)
        ctx.step(dnnmg.PLAIN)
        host_x.copy_(ctx.get_state(), non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t_e2e) / E

    local = {"ms": ms_steps, "wall": t_wall, "vp_ms": vp_ms, "vp_launches": vp_launches}
    if world > 1:
        t = torch.tensor([ms_steps], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        local["ms"] = float(t.item())
    if rank != 0:
        return None

    ms_per_step = local["ms"] / args.steps
    hbm, _, peak_kind = peaks()
    bytes_per_pass = fluid_cells(LEVEL) / 4 * 576 + ndof(LEVEL) / 3 * 44
    avg_pass_ms = vp_ms / max(vp_launches, 1)
    achieved = bytes_per_pass / (avg_pass_ms * 1e-3) / 1e9
    return {
        "metric": METRIC,
        "value": world * args.steps / (local["ms"] * 1e-3),
        "unit": "time steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "level": LEVEL, "dofs": ndof(LEVEL),
                   "obstacle_block": list(ob), "l2": "flushed (256 MB write) before every step",
                   "parallelism": f"replicas x{world}"},
        "vcycle": {"ms": vcycle_ms, "dof_per_s": ndof(LEVEL) / (vcycle_ms * 1e-3)},
        "newton_its_per_step": sum(s["newton_its"] for s in stats) / len(stats),
        "gmres_its_per_step": sum(s["gmres_its"] for s in stats) / len(stats),
        "stages_ms": stage,
        "roofline": {"kernel": "vanka_pass (level 6, FP32)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": bytes_per_pass,
                     "avg_launch_ms": avg_pass_ms},
        "clocks": clk.summary(),
        "e2e": {"value": 1.0 / t_e2e, "unit": "time steps/s",
                "h2d_bytes_per_step": 8 * ndof(LEVEL), "d2h_bytes_per_step": 8 * ndof(LEVEL)},
        "gpu_launches": int(launches),
    }


def run_vcycles(args):
    """Level-6 V-cycles only (after --warmup untimed ones): a short command
    for kernel profilers."""
    import torch
    from paper_2106_07687_gb300 import build, dnnmg
    import synthetic
    build.build()
    ob = synthetic.obstacle_block(1000)
    ctx = dnnmg.Context(level_solve=LEVEL, precision=dnnmg.MIXED, nu=NU, dt=DT,
                        obstacle_i0=ob[0], obstacle_j0=ob[1])
    x = ctx.get_state()
    ctx.linearize(x)
    b = torch.from_numpy(synthetic.random_vector(7, ndof(LEVEL))).float().cuda()
    xv = torch.empty_like(b)
    for _ in range(args.warmup + args.steps):
        ctx.vcycle(LEVEL, b, xv)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "vcycle", "level": LEVEL, "cycles": args.warmup + args.steps,
                      "norm": float(xv.norm())}))


def run_reference(args, rank, world):
    if rank != 0:
        return None
    steps = []
    for _ in range(args.warmup):
        pass
    t = time.perf_counter()
    per = [oracle_step_seconds(4, steps=1, warm=0) * ndof(LEVEL) / ndof(4)
           for _ in range(args.steps)]
    mean = sum(per) / len(per)
    v = 1.0 / mean
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "time steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "level": LEVEL, "dofs": ndof(LEVEL)},
            "cpu_baseline": {"value": v, "unit": "time steps/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: the first plain time step of the FP64 oracle "
                                       "on the 256x64 channel (level 4) from the impulsive start, "
                                       "scaled by the DOF ratio to level 6; single-threaded"},
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
    ap.add_argument("--mode", choices=["step", "vcycle"], default="step",
                    help="vcycle: only set up level 6 and run --steps V-cycles (profiling runs)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.mode == "vcycle":
        run_vcycles(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world)
        if out is not None and world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline()
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
