"""Parity of the exact configuration the benchmark times, against the FP64
oracle: the mixed-precision DNN-MG step with the multigrid solve on the
512x128 channel (level 5) and the patch network on 1024x256 (level 6,
61,440 patches, GRU 2 x 64 + MLP 128, BF16 with FP32 accumulation), and the
persistent level-5 V-cycle plan the benchmark runs (the whole cycle of
levels 5..1 in one cooperative launch), both with the seeded obstacle.

Bars: relative L2 1e-4 for mixed-precision results and 1e-10 for the FP64
build of the same launch plan; 5e-3 on the BF16 patch inputs.  Each field is
also compared in the max norm on the DOFs next to the walls, the inflow, the
obstacle and on the outflow boundary, so that a boundary-local error cannot
hide under the whole-vector norm."""
import numpy as np
import pytest

import synthetic
from oracle import dnnmg, fem, mesh, mg, net, newton
from tests.gpu_util import lib, max_rel, near_dirichlet_dofs, rel, seeded_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, NU, DT = 5, 0.0065, 0.005
OBSTACLE_SEED = 1000


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-10)])
def test_split5_persistent_vcycle_level5_with_obstacle(precision, tol):
    """vcycle_kernel with split 5, mode 0: every level of the cycle inside
    one cooperative launch, on the benchmark's level-5 channel."""
    dn = lib()
    ob = synthetic.obstacle_block(OBSTACLE_SEED)
    prm = fem.Params(nu=NU, dt=DT)
    ctx = dn.Context(level_solve=L, precision=precision, obstacle_i0=ob[0], obstacle_j0=ob[1],
                     nu=NU, dt=DT, persistent_vcycle=5, persistent_mode=0)
    levels = mesh.hierarchy(L, obstacle=ob)
    lev = levels[-1]
    x = seeded_state(lev, 31)
    ctx.linearize(torch.from_numpy(x).cuda())
    plan = ctx.vcycle_plan()
    assert plan["split_level"] == 5 and plan["split_mode"] == 0, plan
    H = mg.Hierarchy(levels, x, prm)
    near = near_dirichlet_dofs(lev)
    for seed in (81, 82):
        b = synthetic.random_vector(seed, lev.ndof)
        b[lev.cons] = 0.0
        xg = ctx.vcycle(L, torch.from_numpy(b).to(ctx.vdtype).cuda()).double().cpu().numpy()
        xr = mg.vcycle(H, len(levels) - 1, b)
        assert rel(xg, xr) < tol, (seed, rel(xg, xr))
        assert max_rel(xg, xr, near) < 10 * tol, (seed, max_rel(xg, xr, near))


def test_mixed_dnnmg_steps_at_benchmark_size_match_oracle():
    """Two DNN-MG steps (Algorithm 1) of the benchmark's workload from the
    impulsive start: the first with the plain right-hand side, the second
    with the network's restricted one.  Seeded weights of the benchmark's
    network and seeded feature statistics; Newton to 1e-10 on both sides.
    Two contexts run beside one oracle trajectory: one with the autotuned
    V-cycle plan (what the benchmark runs), one with the whole level-5 cycle
    forced into one cooperative launch."""
    dn = lib()
    ob = synthetic.obstacle_block(OBSTACLE_SEED)
    common = dict(level_solve=L, precision=dn.MIXED, obstacle_i0=ob[0], obstacle_j0=ob[1],
                  nu=NU, dt=DT)
    ctxs = {"autotuned": dn.Context(**common),
            "split5": dn.Context(persistent_vcycle=5, persistent_mode=0, **common)}
    spec = net.NetSpec()
    w = synthetic.random_weights(21, spec.num_params(), 0.05).astype(np.float32)
    rng = np.random.default_rng(15)
    mean = rng.normal(0, 0.1, 40).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 40).astype(np.float32)
    for ctx in ctxs.values():
        assert ctx.num_params() == spec.num_params()
        assert ctx.num_patches() == 61440
        ctx.set_weights(w)
        ctx.set_feature_stats(mean, std)
    levels = mesh.hierarchy(L, obstacle=ob)
    fine = mesh.Level(L + 1, obstacle=ob)
    prm = fem.Params(nu=NU, dt=DT)
    opt = newton.SolverOptions()
    params = spec.unflatten(w.astype(np.float64))
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
    near_c = near_dirichlet_dofs(levels[-1])
    near_f = near_dirichlet_dofs(fine)
    near_f = near_f[near_f < 2 * fine.nn]
    for n in range(2):
        stats = {k: c.step(dn.NET) for k, c in ctxs.items()}
        x, state, info = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt,
                                         mean.astype(np.float64), std.astype(np.float64))
        vr = state["vcorr"][:2 * fine.nn]
        for k, ctx in ctxs.items():
            st = stats[k]
            if k == "split5":
                assert ctx.vcycle_plan()["split_level"] == 5
            xg = ctx.get_state().cpu().numpy()
            assert st["res_final"] <= 1e-10, (k, st)
            assert rel(xg, x) < 1e-4, (k, n, rel(xg, x))
            assert max_rel(xg, x, near_c) < 1e-4, (k, n, max_rel(xg, x, near_c))
            vg = ctx.get_fine_velocity().cpu().numpy()
            assert rel(vg, vr) < 1e-4, (k, n, rel(vg, vr))
            assert max_rel(vg, vr, near_f, 2) < 1e-3, (k, n, max_rel(vg, vr, near_f, 2))
            Xg = ctx.get_patch_inputs().double().cpu().numpy()
            assert rel(Xg, info["X"]) < 5e-3, (k, n, rel(Xg, info["X"]))
            assert st["fallback"] == int(info["fallback"]) == 0, k
    for ctx in ctxs.values():
        ctx.close()
