"""Corpus generation against the oracle, and what a trained network gains.

make_sample: the level-L step from an injected fine state with the
right-hand side an exact correction would give, then raw inputs and targets
per patch -- compared with the oracle's composition of the same steps
(FP32 outputs: relative L2 1e-5 for inputs, 1e-4 for targets).

Learning gain: a network trained by this library's kernels on samples from
plain fine trajectories (two viscosities) must bring the DNN-MG velocity
closer to the fine-level solution than plain multigrid on level L, on a
held-out viscosity (the paper's claim that the correction improves the coarse
solution, Sec. 3.4).  Small channel: L = 2 (64x16), fine level 3."""
import numpy as np
import pytest

import synthetic
from oracle import dnnmg, fem, mesh, mg, newton
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, DT = 2, 0.01


@pytest.mark.parametrize("replaced", [1, 2])
def test_make_sample_matches_oracle(replaced):
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    nu = 0.01
    fine_ctx = dn.Context(level_solve=L + replaced, precision=dn.FP64, obstacle_i0=ob[0],
                          obstacle_j0=ob[1], nu=nu, dt=DT, newton_tol=1e-12)
    ctx = dn.Context(level_solve=L, precision=dn.FP64, obstacle_i0=ob[0], obstacle_j0=ob[1],
                     nu=nu, dt=DT, newton_tol=1e-12, replaced_levels=replaced)
    for _ in range(2):
        fine_ctx.step(dn.PLAIN)
    xp = fine_ctx.get_state()
    fine_ctx.step(dn.PLAIN)
    xn = fine_ctx.get_state()
    X, Y = ctx.make_sample(xp, xn)
    # oracle
    levels = mesh.hierarchy(L, obstacle=ob)
    chain = [levels[-1]] + [mesh.Level(L + k, obstacle=ob) for k in range(1, replaced + 1)]
    coarse, fine = chain[0], chain[-1]
    ratio = 2 ** replaced
    prm = fem.Params(nu=nu, dt=DT)
    xp_h, xn_h = xp.cpu().numpy(), xn.cpu().numpy()
    xL = xp_h
    for k in range(replaced, 0, -1):   # nodal injection, one level at a time
        xL = mg.inject(xL, chain[k - 1], chain[k], 3)
    vprev = xp_h.copy()
    vprev[2 * fine.nn:] = 0.0
    _, bL = dnnmg.rhs_and_restrict(coarse, fine, chain, vprev, prm)
    x, *_ = newton.newton_solve(levels, xL, bL, prm, newton.SolverOptions(newton_tol=1e-12))
    xt = dnnmg.prolongate_chain(chain, x)
    r = dnnmg.fine_residual(fine, xt, vprev, prm)
    Xr = dnnmg.patch_features(coarse, fine, ratio, xt, r, prm)
    nodes = dnnmg.patch_nodes(coarse, fine, ratio)
    vd = fine.vdir.ravel()[nodes]
    Yr = np.concatenate([np.where(vd, 0, xn_h[:fine.nn][nodes] - xt[:fine.nn][nodes]),
                         np.where(vd, 0, xn_h[fine.nn:2 * fine.nn][nodes] - xt[fine.nn:2 * fine.nn][nodes])],
                        axis=1)
    assert rel(X.double().cpu().numpy(), Xr) < 1e-5
    assert rel(Y.double().cpu().numpy(), Yr) < 1e-4
    np.testing.assert_allclose(ctx.get_state().cpu().numpy(), x, rtol=0, atol=1e-9)


def _trajectory(dn, ob, nu, steps):
    c = dn.Context(level_solve=L + 1, precision=dn.MIXED, obstacle_i0=ob[0], obstacle_j0=ob[1],
                   nu=nu, dt=DT)
    states = [c.get_state()]
    for _ in range(steps):
        c.step(dn.PLAIN)
        states.append(c.get_state())
    return states


def test_trained_network_beats_plain_coarse_multigrid():
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    steps, T, B = 40, 8, 256
    train_nus, test_nu = (0.008, 0.012), 0.01
    ctx = dn.Context(level_solve=L, precision=dn.MIXED, obstacle_i0=ob[0], obstacle_j0=ob[1],
                     nu=test_nu, dt=DT, train_batch=B, train_seq=T)
    P = ctx.num_patches()
    Xs, Ys = [], []
    for nu in train_nus:
        sctx = dn.Context(level_solve=L, precision=dn.MIXED, obstacle_i0=ob[0], obstacle_j0=ob[1],
                          nu=nu, dt=DT)
        traj = _trajectory(dn, ob, nu, steps)
        for n in range(1, steps + 1):
            X, Y = sctx.make_sample(traj[n - 1], traj[n])
            Xs.append(X)
            Ys.append(Y)
    Xc = torch.cat(Xs).contiguous()
    Yc = torch.cat(Ys).contiguous()
    ctx.feature_stats(Xc)
    spec_n = ctx.num_params()
    ctx.set_weights(synthetic.random_weights(77, spec_n, 0.08).astype(np.float32))
    rng = np.random.default_rng(3)
    losses = []
    for it in range(400):
        traj_id = rng.integers(0, len(train_nus), B)
        start = rng.integers(0, steps - T + 1, B)
        idx = np.stack([traj_id * steps + start, rng.integers(0, P, B)], axis=1).astype(np.int32)
        Xb, Yb = ctx.gather_batch(Xc, Yc, torch.from_numpy(idx).cuda(), T, P)
        losses.append(ctx.train_step(Xb, Yb, B, T, 2e-3 if it < 300 else 5e-4))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20]), (losses[:3], losses[-3:])
    # held-out viscosity: DNN-MG vs plain MG(L) against the fine solution
    ref = _trajectory(dn, ob, test_nu, 20)
    plain = dn.Context(level_solve=L, precision=dn.MIXED, obstacle_i0=ob[0], obstacle_j0=ob[1],
                       nu=test_nu, dt=DT)
    fine = mesh.Level(L + 1, obstacle=ob)
    coarse = mesh.Level(L, obstacle=ob)
    e_net, e_plain = [], []
    for n in range(1, 21):
        ctx.step(dn.NET)
        plain.step(dn.PLAIN)
        vr = ref[n].cpu().numpy()[:2 * fine.nn]
        vn = ctx.get_fine_velocity().cpu().numpy()
        vp = dnnmg.prolongate_state(coarse, fine, plain.get_state().cpu().numpy())[:2 * fine.nn]
        e_net.append(np.linalg.norm(vn - vr) / np.linalg.norm(vr))
        e_plain.append(np.linalg.norm(vp - vr) / np.linalg.norm(vr))
    assert np.mean(e_net[5:]) < 0.8 * np.mean(e_plain[5:]), (e_net, e_plain)
