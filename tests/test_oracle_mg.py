"""Pins of the oracle's multigrid pieces (Sec. 2.2): transfers reproduce
bilinears, the Vanka colouring is node-disjoint, the coarse solve is exact,
and the V-cycle contracts at an h-independent rate."""
import numpy as np
import pytest

from oracle import fem, mesh, mg


def test_prolongation_reproduces_bilinears_and_restriction_is_adjoint():
    coarse, fine = mesh.Level(1), mesh.Level(2)
    Pn = mg.prolongation_nodes(coarse, fine)
    Xc, Yc = coarse.coords()
    Xf, Yf = fine.coords()
    for f in (lambda X, Y: 1 + 0 * X, lambda X, Y: X, lambda X, Y: Y, lambda X, Y: X * Y - 2 * X + 3):
        np.testing.assert_allclose(Pn @ f(Xc, Yc).ravel(), f(Xf, Yf).ravel(), atol=1e-14)
    # a quadratic is not reproduced at midpoints
    assert np.abs(Pn @ (Xc ** 2).ravel() - (Xf ** 2).ravel()).max() > 1e-3
    rng = np.random.default_rng(0)
    P = mg.prolongation_masked(coarse, fine)
    r, x = rng.standard_normal(fine.ndof), rng.standard_normal(coarse.ndof)
    assert abs((P.T @ r) @ x - r @ (P @ x)) < 1e-12 * np.linalg.norm(r) * np.linalg.norm(x)


def test_injection_samples_coinciding_nodes():
    """Nodal injection (the linearisation point of the coarse levels) takes
    the fine value at the coinciding node: a field sampled on the fine nodes
    injects to the same field sampled on the coarse nodes, for any field,
    component by component; after a bilinear prolongation it gives the
    coarse vector back."""
    coarse, fine = mesh.Level(2, obstacle=(2, 1)), mesh.Level(3, obstacle=(2, 1))
    f = lambda X, Y: np.sin(3.1 * X + 0.7) * np.cos(2.3 * Y) + X * X * Y
    g = lambda X, Y: np.exp(-X) + 5.0 * Y ** 3
    Xf, Yf = fine.coords()
    Xc, Yc = coarse.coords()
    xf = np.concatenate([f(Xf, Yf).ravel(), g(Xf, Yf).ravel()])
    xc = mg.inject(xf, coarse, fine, 2)
    np.testing.assert_array_equal(xc, np.concatenate([f(Xc, Yc).ravel(), g(Xc, Yc).ravel()]))
    rng = np.random.default_rng(9)
    v = rng.standard_normal(coarse.nn)
    Pn = mg.prolongation_nodes(coarse, fine)
    np.testing.assert_allclose(mg.inject(Pn @ v, coarse, fine, 1), v, rtol=0, atol=1e-15)


def test_vanka_update_of_a_lone_cell_scales_its_defect_by_one_minus_omega():
    """A colour pass restricted to one cell changes x only on that cell's 12
    DOFs, by omega A_c^-1 d_c, so the new defect on those DOFs is exactly
    (1 - omega) d_c: pins the relaxation factor and that A_c is the block of
    the global matrix on the cell's DOFs (a wrong omega, a transposed or
    misindexed block would leave a different defect)."""
    from oracle import fem
    levels = mesh.hierarchy(2, obstacle=(2, 1))
    prm = fem.Params(nu=0.01, dt=0.01)
    rng = np.random.default_rng(12)
    lev = levels[-1]
    x0 = rng.standard_normal(lev.ndof) * 0.3
    x0[lev.cons] = lev.dirichlet_values[lev.cons]
    H = mg.Hierarchy(levels, x0, prm)
    op = H.ops[-1]
    b = rng.standard_normal(lev.ndof)
    x = rng.standard_normal(lev.ndof)
    cell = int(op.colour_cells[1][7])
    saved = op.colour_cells
    op.colour_cells = [np.array([cell])]
    try:
        dofs = lev.cell_dofs[cell]
        free = lev.free[dofs]
        d_old = (b - op.A @ x)[dofs]
        for omega in (0.8, 0.5):
            x1 = mg.vanka_sweep(op, b, x.copy(), omega)
            d_new = (b - op.A @ x1)[dofs]
            changed = np.flatnonzero(x1 != x)
            assert set(changed) <= set(dofs.tolist())
            np.testing.assert_allclose(d_new[free], (1 - omega) * d_old[free], rtol=1e-9,
                                       atol=1e-12)
    finally:
        op.colour_cells = saved


def test_vanka_colours_are_node_disjoint_and_cover_all_fluid_cells():
    lev = mesh.Level(2)
    op = mg.LevelOp(lev, np.zeros(lev.ndof), fem.Params(), coarsest=False)
    seen = np.zeros(lev.nx * lev.ny, dtype=int)
    for cells in op.colour_cells:
        nodes = lev.cell_nodes[cells].ravel()
        assert len(np.unique(nodes)) == len(nodes)
        seen[cells] += 1
    assert (seen[lev.fluid_cells] == 1).all()
    assert seen.sum() == len(lev.fluid_cells)


def test_vanka_block_is_the_dense_submatrix():
    lev = mesh.Level(2)
    rng = np.random.default_rng(1)
    vb = rng.standard_normal(lev.ndof)
    op = mg.LevelOp(lev, vb, fem.Params(), coarsest=False)
    A = op.A.toarray()
    for c in (0, 37, 200, lev.nx * lev.ny - 1):
        d = lev.cell_dofs[c]
        np.testing.assert_array_equal(op.blocks[c], A[np.ix_(d, d)])


def test_coarse_solve_is_exact():
    lev = mesh.Level(1)
    rng = np.random.default_rng(2)
    op = mg.LevelOp(lev, rng.standard_normal(lev.ndof), fem.Params(), coarsest=True)
    b = rng.standard_normal(lev.ndof)
    x = mg.coarse_solve(op, b)
    assert np.linalg.norm(op.A @ x - b) < 1e-11 * np.linalg.norm(b)


def test_level0_is_singular_with_the_obstacle():
    """The reason the cycle stops at level 1: with a 2x2 block of level-0
    cells in a 4-cell-high channel every node beside the obstacle is no-slip,
    so level 0 has a pressure null space upstream of the obstacle."""
    lev = mesh.Level(0, obstacle=(2, 1))
    X, Y = lev.coords()
    vb = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(2 * lev.nn)])
    s = np.linalg.svd(fem.jacobian(lev, vb, fem.Params()).toarray(), compute_uv=False)
    assert s[-1] < 1e-12 * s[0]
    lev1 = mesh.Level(1, obstacle=(2, 1))
    X, Y = lev1.coords()
    vb = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(2 * lev1.nn)])
    s1 = np.linalg.svd(fem.jacobian(lev1, vb, fem.Params()).toarray(), compute_uv=False)
    assert s1[-1] > 1e-8 * s1[0]


def _rho(L, obstacle, omega=0.8, alpha0=0.1):
    levels = mesh.hierarchy(L, obstacle=obstacle)
    lev = levels[-1]
    X, Y = lev.coords()
    vb = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(2 * lev.nn)])
    H = mg.Hierarchy(levels, vb, fem.Params(nu=0.01, dt=0.01, alpha0=alpha0), omega=omega)
    A = H.ops[-1].A
    rng = np.random.default_rng(5)
    b = np.zeros(lev.ndof)
    x = rng.standard_normal(lev.ndof)
    x[lev.cons] = 0.0
    res = []
    for _ in range(7):
        x = mg.vcycle(H, len(levels) - 1, b, x)
        res.append(np.linalg.norm(A @ x))
    return (res[-1] / res[2]) ** 0.25


def test_vcycle_contraction_is_small_and_h_independent():
    rhos = [_rho(L, (2, 1)) for L in (2, 3, 4)]
    assert max(rhos) < 0.3, rhos
    assert max(rhos) - min(rhos) < 0.1, rhos


def test_vcycle_is_a_linear_map():
    levels = mesh.hierarchy(3)
    lev = levels[-1]
    rng = np.random.default_rng(9)
    H = mg.Hierarchy(levels, rng.standard_normal(lev.ndof) * 0.5, fem.Params())
    b1, b2 = rng.standard_normal(lev.ndof), rng.standard_normal(lev.ndof)
    k = len(levels) - 1
    lhs = mg.vcycle(H, k, 2.0 * b1 - 3.0 * b2)
    rhs = 2.0 * mg.vcycle(H, k, b1) - 3.0 * mg.vcycle(H, k, b2)
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(lhs)


@pytest.mark.parametrize("alpha0,bound", [(0.05, 0.2), (0.1, 0.2), (0.5, 0.6)])
def test_vcycle_contraction_over_the_stabilisation_parameter(alpha0, bound):
    """alpha_0 of Sec. 2.1 is not given by the paper (0.1 here): the
    V(2,2) Vanka cycle contracts by at most 0.2 per cycle for alpha_0 <=
    0.1 and degrades, without diverging, for a stabilisation five times
    stronger (measured 0.38-0.52 at alpha_0 = 0.5)."""
    rhos = [_rho(L, (2, 1), alpha0=alpha0) for L in (2, 3)]
    assert max(rhos) < bound, rhos
