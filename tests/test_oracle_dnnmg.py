"""Pins of the oracle's DNN-MG pieces (the network correction of Algorithm 1): with a zero
network correction the restricted right-hand side is exactly the coarse
level's own old-time term (nested Q1 spaces, exact quadrature), so a DNN-MG
step reduces to a plain MG(L) step; scatter averaging and patch features
behave as defined on closed-form inputs."""
import numpy as np
import pytest

from oracle import dnnmg, fem, mesh, newton


@pytest.mark.parametrize("replaced", [1, 2])
def test_zero_correction_gives_coarse_old_time_term(replaced):
    L = 2
    prm = fem.Params(nu=0.01, dt=0.01)
    chain = [mesh.Level(L + k, obstacle=(3, 1)) for k in range(replaced + 1)]
    coarse, fine = chain[0], chain[-1]
    rng = np.random.default_rng(0)
    xL = rng.standard_normal(coarse.ndof)
    xt = xL
    for k in range(replaced):
        xt = dnnmg.prolongate_state(chain[k], chain[k + 1], xt)
    _, bL = dnnmg.rhs_and_restrict(coarse, fine, chain, xt, prm)
    ref = fem.old_time_rhs(coarse, xL, prm)
    free = coarse.free.copy()
    free[2 * coarse.nn:] = False
    np.testing.assert_allclose(bL[free], ref[free], rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_dnnmg_step_with_zero_network_equals_plain_step():
    levels = mesh.hierarchy(2, obstacle=(2, 1))
    coarse = levels[-1]
    fine = mesh.Level(3, obstacle=(2, 1))
    prm = fem.Params(nu=0.01, dt=0.01)
    opt = newton.SolverOptions(newton_tol=1e-12)
    x0 = mesh.initial_state(coarse)
    x1, *_ = newton.time_step(levels, x0, prm, opt)
    # the network correction of Algorithm 1 with d = 0, then the next step from b^L
    xt = dnnmg.prolongate_state(coarse, fine, x1)
    _, bL = dnnmg.rhs_and_restrict(coarse, fine, [coarse, fine], xt, prm)
    x2_dnn, *_ = newton.newton_solve(levels, x1, bL, prm, opt)
    x2_plain, *_ = newton.time_step(levels, x1, prm, opt)
    assert np.linalg.norm(x2_dnn - x2_plain) < 1e-10 * np.linalg.norm(x2_plain)


def test_scatter_average_of_constant_prediction():
    coarse, fine = mesh.Level(2, obstacle=(2, 1)), mesh.Level(3, obstacle=(2, 1))
    P = len(coarse.fluid_cells)
    d = np.concatenate([np.full((P, 9), 0.7), np.full((P, 9), -0.2)], axis=1)
    out = dnnmg.scatter_average(coarse, fine, 2, d)
    covered = np.zeros(fine.nn, bool)
    covered[dnnmg.patch_nodes(coarse, fine, 2).ravel()] = True
    ok = covered & ~fine.vdir.ravel()
    np.testing.assert_allclose(out[:fine.nn][ok], 0.7, rtol=1e-15)
    np.testing.assert_allclose(out[fine.nn:][ok], -0.2, rtol=1e-15)
    assert (out[:fine.nn][~ok] == 0).all()
    # a linear field of per-patch values averages to the node's mean
    d2 = np.zeros((P, 18))
    d2[:, 4] = np.arange(P)          # patch centres are unshared nodes
    out2 = dnnmg.scatter_average(coarse, fine, 2, d2)
    centres = dnnmg.patch_nodes(coarse, fine, 2)[:, 4]
    np.testing.assert_allclose(out2[centres], np.arange(P) * ~fine.vdir.ravel()[centres])


def test_patch_features_for_uniform_flow():
    coarse, fine = mesh.Level(1, obstacle=None), mesh.Level(2, obstacle=None)
    prm = fem.Params(nu=0.02, dt=0.005)
    xt = np.concatenate([np.full(fine.nn, 0.6), np.full(fine.nn, 0.8), np.zeros(fine.nn)])
    r = np.zeros(fine.ndof)
    X = dnnmg.patch_features(coarse, fine, 2, xt, r, prm)
    assert X.shape == (coarse.nx * coarse.ny, 40)
    np.testing.assert_allclose(X[:, :9], 0.6)
    np.testing.assert_allclose(X[:, 9:18], 0.8)
    np.testing.assert_allclose(X[:, 36], coarse.h / 0.25)
    np.testing.assert_allclose(X[:, 37], 1.0)
    np.testing.assert_allclose(X[:, 38], 1.0 * coarse.h / prm.nu)
    np.testing.assert_allclose(X[:, 39], prm.dt / coarse.h)


def test_patch_count_of_the_dnnmg_workload():
    """One patch per level-5 cell: 512 x 128 = 65,536 cells, of which the
    2x2 level-0 obstacle covers 4 * 32^2 = 4,096."""
    coarse = mesh.Level(5, obstacle=(2, 1))
    assert coarse.nx * coarse.ny == 65536
    assert len(coarse.fluid_cells) == 65536 - 4096


def test_two_replaced_levels_step_with_zero_network_equals_plain_step():
    """Algorithm 1 with the network replacing two levels (5x5-node patches,
    104 inputs, 50 outputs) and an all-zero network: the step after the
    first one uses b^L = R R Rhs(P P v^L), which is the plain old-time term,
    so the trajectory equals plain MG(L)."""
    from oracle import net
    levels = mesh.hierarchy(2, obstacle=(2, 1))
    chain = [mesh.Level(3, obstacle=(2, 1)), mesh.Level(4, obstacle=(2, 1))]
    prm = fem.Params(nu=0.01, dt=0.01)
    opt = newton.SolverOptions(newton_tol=1e-12)
    spec = net.NetSpec(c_in=104, c_out=50)
    params = spec.unflatten(np.zeros(spec.num_params()))
    P = len(levels[-1].fluid_cells)
    state = dict(bL=None, vcorr=None, h=np.zeros((2, P, 64)))
    x_dnn = x_plain = mesh.initial_state(levels[-1])
    for n in range(3):
        x_dnn, state, info = dnnmg.time_step(levels, chain, x_dnn, state, spec, params, prm, opt)
        x_plain, *_ = newton.time_step(levels, x_plain, prm, opt)
        assert info["X"].shape == (P, 104) and info["y"].shape == (P, 50)
        assert not info["fallback"]
        assert np.linalg.norm(x_dnn - x_plain) < 1e-10 * np.linalg.norm(x_plain), n


def test_five_by_five_patches_and_scatter():
    """Two replaced levels: a patch is one level-L cell = 4x4 cells = 5x5
    nodes of level L+2; interior nodes shared by 1, 2 or 4 patches; a
    constant prediction scatters to the same constant."""
    coarse, fine = mesh.Level(1, obstacle=None), mesh.Level(3, obstacle=None)
    nodes = dnnmg.patch_nodes(coarse, fine, 4)
    assert nodes.shape == (coarse.nx * coarse.ny, 25)
    # lower-left patch: nodes (s, t), s, t in 0..4 of the fine level
    np.testing.assert_array_equal(nodes[0], [t * fine.nnx + s for t in range(5) for s in range(5)])
    cnt = np.bincount(nodes.ravel(), minlength=fine.nn)
    i, j = np.arange(fine.nn) % fine.nnx, np.arange(fine.nn) // fine.nnx
    on_x = (i % 4 == 0) & (i > 0) & (i < fine.nx)
    on_y = (j % 4 == 0) & (j > 0) & (j < fine.ny)
    expect = np.where(on_x & on_y, 4, np.where(on_x | on_y, 2, 1))
    np.testing.assert_array_equal(cnt, expect)
    P = nodes.shape[0]
    d = np.concatenate([np.full((P, 25), 0.3), np.full((P, 25), -1.1)], axis=1)
    out = dnnmg.scatter_average(coarse, fine, 4, d)
    ok = ~fine.vdir.ravel()
    np.testing.assert_allclose(out[:fine.nn][ok], 0.3, rtol=1e-15)
    np.testing.assert_allclose(out[fine.nn:][ok], -1.1, rtol=1e-15)
    xt = np.concatenate([np.full(fine.nn, 0.6), np.full(fine.nn, 0.8), np.zeros(fine.nn)])
    prm = fem.Params(nu=0.02, dt=0.005)
    X = dnnmg.patch_features(coarse, fine, 4, xt, np.zeros(fine.ndof), prm)
    assert X.shape == (P, 104)
    np.testing.assert_allclose(X[:, :25], 0.6)
    np.testing.assert_allclose(X[:, 25:50], 0.8)
    np.testing.assert_allclose(X[:, 100], coarse.h / 0.25)
    np.testing.assert_allclose(X[:, 102], 1.0 * coarse.h / prm.nu)
    np.testing.assert_allclose(X[:, 103], prm.dt / coarse.h)
