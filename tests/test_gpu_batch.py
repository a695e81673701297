"""Parity of the batched engine (many problems, one launch per stage) with
single-problem contexts and with the oracle.

Three problems of uneven size -- finest solved levels 2, 4 and 3 (64x16,
256x64 and 128x32 channels), each with its own seeded obstacle, viscosity
and time step -- are advanced in lock-step.  Each problem must reproduce
what a single context (itself pinned to the oracle by test_gpu_solver.py and
test_gpu_dnnmg.py) computes for it, and the smallest problem is also
checked against the oracle directly.  FP64 bars: 1e-12 for one V-cycle
(identical arithmetic up to summation order), 1e-10 for time steps (both
sides iterate Newton to 1e-12); mixed precision: 1e-5 for one FP32 V-cycle
and 1e-4 for steps."""
import numpy as np
import pytest

import synthetic
from oracle import fem, mesh, newton
from tests.gpu_util import lib, rel, seeded_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (finest level, nu, dt, obstacle seed)
PROBS = [(2, 0.01, 0.01, 1001), (4, 0.02, 0.005, 1002), (3, 0.005, 0.01, 1003)]


def _cfgs(dn, precision, **kw):
    out = []
    for L, nu, dt, seed in PROBS:
        ob = synthetic.obstacle_block(seed)
        out.append(dn.default_config(level_solve=L, precision=precision, obstacle_i0=ob[0],
                                     obstacle_j0=ob[1], nu=nu, dt=dt, newton_tol=1e-12, **kw))
    return out


def _slice(vec, batch, i):
    lev, off = batch.layout(i)
    return vec[off:off + 3 * (16 * 2 ** lev + 1) * (4 * 2 ** lev + 1)]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_batched_vcycle_matches_single_contexts(precision, tol):
    dn = lib()
    cfgs = _cfgs(dn, precision)
    B = dn.Batch(cfgs)
    assert B.n == len(cfgs)
    bvec = torch.zeros(B.length, dtype=B.vdtype, device="cuda")
    singles = []
    for i, c in enumerate(cfgs):
        lev = mesh.Level(c.level_solve, obstacle=(c.obstacle_i0, c.obstacle_j0))
        x = torch.tensor(seeded_state(lev, 50 + i), device="cuda")
        B.set_state(i, x)
        ctx = dn.Context(cfg=c)
        ctx.set_state(x)
        ctx.linearize(ctx.get_state())
        b = torch.tensor(synthetic.random_vector(70 + i, 3 * lev.nn), dtype=B.vdtype,
                         device="cuda")
        _slice(bvec, B, i).copy_(b)
        singles.append((ctx, c.level_solve, b))
    B.linearize()
    xb = B.vcycle(bvec)
    for i, (ctx, L, b) in enumerate(singles):
        xs = ctx.vcycle(L, b)
        assert rel(_slice(xb, B, i).cpu().numpy(), xs.cpu().numpy()) < tol, i
    # one problem alone (the instance form of the V-cycle) gives that
    # problem's part of the batch cycle
    for i, (ctx, L, b) in enumerate(singles):
        xi = B.vcycle_inst(i, b.contiguous())
        assert rel(xi.cpu().numpy(), _slice(xb, B, i).cpu().numpy()) < tol, i
    with pytest.raises(dn.DnnmgError):
        B.vcycle_inst(B.n, singles[0][2].contiguous())
    # the padding between problems stays zero
    mask = torch.ones(B.length, dtype=torch.bool, device="cuda")
    for i in range(B.n):
        lev, off = B.layout(i)
        mask[off:off + 3 * (16 * 2 ** lev + 1) * (4 * 2 ** lev + 1)] = False
    assert float(xb[mask].abs().max().item() if mask.any() else 0.0) == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_plain_steps_match_single_contexts_and_oracle(precision):
    dn = lib()
    cfgs = _cfgs(dn, precision)
    B = dn.Batch(cfgs)
    ctxs = [dn.Context(cfg=c) for c in cfgs]
    c0 = cfgs[0]
    ob0 = (c0.obstacle_i0, c0.obstacle_j0)
    levels = mesh.hierarchy(c0.level_solve, obstacle=ob0)
    prm = fem.Params(nu=c0.nu, dt=c0.dt)
    opt = newton.SolverOptions(newton_tol=1e-12)
    x0 = mesh.initial_state(levels[-1])
    tol = 1e-10 if precision == 0 else 1e-4
    for n in range(3):
        stats = B.step(dn.PLAIN)
        assert len(stats) == B.n
        x0, _, _, _ = newton.time_step(levels, x0, prm, opt)
        for i, ctx in enumerate(ctxs):
            ss = ctx.step(dn.PLAIN)
            xb = B.get_state(i).cpu().numpy()
            xs = ctx.get_state().cpu().numpy()
            assert stats[i]["res_final"] <= 1e-12, (n, i, stats[i])
            assert stats[i]["newton_its"] >= 1
            assert rel(xb, xs) < tol, (n, i, rel(xb, xs), stats[i], ss)
        assert rel(B.get_state(0).cpu().numpy(), x0) < tol, n


@pytest.mark.parametrize("replaced", [1, 2])
def test_batched_dnnmg_steps_match_single_contexts(replaced):
    """DNN-MG steps with a random network (shared weights and feature
    statistics): the corrected fine velocities and the level-L states of all
    problems equal those of single contexts; with one replaced level (3x3-node
    patches, 40 inputs) and with two (5x5-node patches, 104 inputs, P and R
    applied twice)."""
    dn = lib()
    cfgs = _cfgs(dn, 0, replaced_levels=replaced)
    B = dn.Batch(cfgs)
    ctxs = [dn.Context(cfg=c) for c in cfgs]
    npar = ctxs[0].num_params()
    c_in = ctxs[0].net_dims()[0]
    assert c_in == (40 if replaced == 1 else 104)
    w = synthetic.random_weights(11, npar, 0.05).astype(np.float32)
    rng = np.random.default_rng(5)
    mean = rng.normal(0, 0.1, c_in).astype(np.float32)
    std = rng.uniform(0.5, 2.0, c_in).astype(np.float32)
    B.set_weights(w)
    B.set_feature_stats(mean, std)
    for ctx in ctxs:
        ctx.set_weights(w)
        ctx.set_feature_stats(mean, std)
    for n in range(3):
        stats = B.step(dn.NET)
        for i, ctx in enumerate(ctxs):
            ss = ctx.step(dn.NET)
            assert stats[i]["fallback"] == ss["fallback"], (n, i)
            xb, xs = B.get_state(i).cpu().numpy(), ctx.get_state().cpu().numpy()
            assert rel(xb, xs) < 1e-9, (n, i, rel(xb, xs))
            vb = B.get_fine_velocity(i).cpu().numpy()
            vs = ctx.get_fine_velocity().cpu().numpy()
            assert rel(vb, vs) < 1e-9, (n, i, rel(vb, vs))


def test_batched_crank_nicolson_and_graph_toggle():
    """theta = 1/2 on one problem of the batch, and the same steps with the
    FGMRES graphs switched off give the same states."""
    dn = lib()
    cfgs = _cfgs(dn, 0)
    cfgs[1].theta = 0.5
    A, B = dn.Batch(cfgs), dn.Batch(cfgs)
    B.graphs(False)
    ctx = dn.Context(cfg=cfgs[1])
    for n in range(2):
        A.step(dn.PLAIN)
        B.step(dn.PLAIN)
        ctx.step(dn.PLAIN)
        for i in range(A.n):
            assert rel(A.get_state(i).cpu().numpy(), B.get_state(i).cpu().numpy()) < 1e-12
        assert rel(A.get_state(1).cpu().numpy(), ctx.get_state().cpu().numpy()) < 1e-10
