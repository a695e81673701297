"""Pins of the oracle's discretisation (Sec. 2.1, Eqs. 3-6) to facts that do
not come from the oracle itself: textbook Q1 element matrices, exact symbolic
integrals, the discrete Poiseuille solution, finite differences and discrete
mass conservation."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, mesh, mg, newton


def test_q1_element_matrices_match_textbook():
    h = 0.37
    el = fem.Element(h)
    M_ref = h * h / 36.0 * np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]])
    K_ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    # 1D: int phi_i phi_j' over [0,h] = [[-1/2, 1/2], [-1/2, 1/2]]; 1D mass h/6 [[2,1],[1,2]]
    C = np.array([[-0.5, 0.5], [-0.5, 0.5]])
    m = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    Dx_ref = np.array([[C[a & 1, b & 1] * m[a >> 1, b >> 1] for b in range(4)] for a in range(4)])
    Dy_ref = np.array([[m[a & 1, b & 1] * C[a >> 1, b >> 1] for b in range(4)] for a in range(4)])
    np.testing.assert_allclose(el.M, M_ref, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(el.K, K_ref, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(el.Dx, Dx_ref, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(el.Dy, Dy_ref, rtol=1e-14, atol=1e-16)


def test_convection_terms_match_exact_integration():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    h = sympy.Rational(3, 10)
    phis = [(1 - x / h if a & 1 == 0 else x / h) * (1 - y / h if a >> 1 == 0 else y / h)
            for a in range(4)]
    rng = np.random.default_rng(7)
    ub, vb = rng.standard_normal(4), rng.standard_normal(4)
    U = sum(sympy.Float(ub[a]) * phis[a] for a in range(4))
    V = sum(sympy.Float(vb[a]) * phis[a] for a in range(4))
    N_ex = np.zeros((4, 4))
    G_ex = np.zeros((4, 4))
    for a in range(4):
        for b in range(4):
            e = phis[a] * (U * sympy.diff(phis[b], x) + V * sympy.diff(phis[b], y))
            N_ex[a, b] = float(sympy.integrate(e, (x, 0, h), (y, 0, h)))
            g = phis[a] * phis[b] * sympy.diff(U, y)
            G_ex[a, b] = float(sympy.integrate(g, (x, 0, h), (y, 0, h)))
    el = fem.Element(0.3)
    np.testing.assert_allclose(el.convection(ub[None], vb[None])[0], N_ex, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(el.grad_mass(ub[None], el.DY)[0], G_ex, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("lps", ["patch", "cellgrad"])
@pytest.mark.parametrize("ell", [1, 2, 3, 4])
def test_discrete_poiseuille_is_a_fixed_point(ell, lps):
    """u = 6y(1-y), v = 0, p = 12 nu (4 - x) solves the discrete steady and
    backward-Euler problem exactly: 1D linear elements are nodally exact for
    -nu u'' = const, convection vanishes, the mass terms cancel, the LPS
    fluctuation of a linear pressure is zero and p(4) = 0 matches the
    do-nothing outflow."""
    lev = mesh.Level(ell, obstacle=None)
    prm = fem.Params(nu=0.01, dt=0.01, lps=lps)
    X, Y = lev.coords()
    x = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(lev.nn), (12 * prm.nu * (4 - X)).ravel()])
    f = fem.old_time_rhs(lev, x, prm)
    r = fem.residual(lev, x, f, prm)
    assert np.abs(r).max() < 1e-13


def test_poiseuille_breaks_with_wrong_pressure_sign():
    lev = mesh.Level(2, obstacle=None)
    prm = fem.Params(nu=0.01, dt=0.01)
    X, Y = lev.coords()
    x = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(lev.nn), (-12 * prm.nu * (4 - X)).ravel()])
    r = fem.residual(lev, x, fem.old_time_rhs(lev, x, prm), prm)
    assert np.abs(r).max() > 1e-4


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_jacobian_matches_central_differences(theta):
    """The operator is quadratic, so central differences are exact up to
    rounding: A(x + e w) - A(x - e w) = 2 e A'(x) w."""
    lev = mesh.Level(2)
    prm = fem.Params(nu=0.007, dt=0.02, theta=theta)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(lev.ndof)
    w = rng.standard_normal(lev.ndof)
    w[lev.cons] = 0.0
    J = fem.jacobian(lev, x, prm)
    e = 1e-3
    fd = (fem.operator(lev, x + e * w, prm) - fem.operator(lev, x - e * w, prm)) / (2 * e)
    fd[lev.cons] = 0.0
    Jw = J @ w
    assert np.linalg.norm(fd - Jw) / np.linalg.norm(Jw) < 1e-10


def test_lps_vanishes_on_patch_bilinear_pressure_only():
    prm = fem.Params(nu=0.01)
    fine, coarse = mesh.Level(3), mesh.Level(2)
    S = fem.lps_matrix(fine, prm)
    Pn = mg.prolongation_nodes(coarse, fine)
    rng = np.random.default_rng(0)
    p = Pn @ rng.standard_normal(coarse.nn)
    x = np.zeros(fine.ndof)
    x[2 * fine.nn:] = p
    assert np.abs(S @ x).max() < 1e-13 * np.abs(p).max()
    # the line checkerboard (-1)^i is not bilinear on patches and is seen
    x[2 * fine.nn:] = ((-1.0) ** np.arange(fine.nnx))[None, :].repeat(fine.nny, 0).ravel()
    assert x @ (S @ x) > 1e-3 * fem.lps_alpha(fine, prm)
    # and S is symmetric positive semi-definite
    Sd = S.toarray()
    assert np.abs(Sd - Sd.T).max() < 1e-15
    assert np.linalg.eigvalsh(Sd[2 * fine.nn:, 2 * fine.nn:]).min() > -1e-14


@pytest.mark.parametrize("obstacle", [None, (2, 1)])
def test_cellwise_lps_is_the_bilinear_mode_penalty(obstacle):
    """The projection of the gradient onto cellwise constants: on a square Q1 cell the stiffness matrix minus
    the mean-gradient part is (1/6) c c^T with c = (1, -1, -1, 1), the cell's
    bilinear mode, so p^T S p = alpha / 6 * sum over fluid cells of
    (p_00 - p_10 - p_01 + p_11)^2; it vanishes on linear pressures and sees
    p = x y."""
    lev = mesh.Level(2, obstacle=obstacle)
    prm = fem.Params(nu=0.02, lps="cellgrad")
    S = fem.lps_matrix(lev, prm)
    alpha = fem.lps_alpha(lev, prm)
    rng = np.random.default_rng(3)
    p = rng.standard_normal(lev.nn)
    x = np.zeros(lev.ndof)
    x[2 * lev.nn:] = p
    P = p.reshape(lev.nny, lev.nnx)
    expect = 0.0
    for cj in range(lev.ny):
        for ci in range(lev.nx):
            if lev.cell_solid[cj, ci]:
                continue
            m = P[cj, ci] - P[cj, ci + 1] - P[cj + 1, ci] + P[cj + 1, ci + 1]
            expect += alpha / 6.0 * m * m
    assert x @ (S @ x) == pytest.approx(expect, rel=1e-12)
    X, Y = lev.coords()
    for lin in (np.ones_like(X), X, Y, 2 * X - 3 * Y + 1):
        x[2 * lev.nn:] = lin.ravel()
        assert np.abs(S @ x).max() < 1e-13
    x[2 * lev.nn:] = (X * Y).ravel()
    assert x @ (S @ x) > 0.1 * alpha * lev.h ** 4
    Sd = S.toarray()
    assert np.abs(Sd - Sd.T).max() < 1e-15
    # only pressure rows and columns
    assert np.abs(Sd[:2 * lev.nn]).max() == 0 and np.abs(Sd[:, :2 * lev.nn]).max() == 0


def test_cellwise_gradient_lps_leaves_the_line_mode_free():
    """The line pressure mode p = (-1)^i (constant in y) has zero bilinear
    part on every cell, so the stabilisation with the cell mean of the
    gradient does not see it; the Q1/Q1 divergence does not either, so it is
    a null vector of the whole Jacobian and the coarsest-level matrix is
    singular.  The patch projection and the projection onto cellwise
    constants penalise it and keep the matrix regular."""
    lev = mesh.hierarchy(1, obstacle=(2, 1))[-1]
    x = mesh.initial_state(lev)
    z = np.zeros(lev.ndof)
    z[2 * lev.nn:] = np.tile((-1.0) ** np.arange(lev.nnx), lev.nny)
    z[lev.cons] = 0.0                     # pressure nodes inside the obstacle
    cond = {}
    for lps in ("patch", "cell", "cellgrad"):
        prm = fem.Params(nu=0.01, dt=0.01, lps=lps)
        J = fem.jacobian(lev, x, prm)
        s = np.linalg.svd(J.toarray(), compute_uv=False)
        cond[lps] = s[0] / s[-1]
        seen = z @ (fem.lps_matrix(lev, prm) @ z)
        if lps == "cellgrad":
            assert abs(seen) < 1e-12 and np.linalg.norm(J @ z) < 1e-14 * np.linalg.norm(z)
        else:
            assert seen > 1.0 and np.linalg.norm(J @ z) > 0.1 * np.linalg.norm(z)
    assert cond["patch"] < 1e6 and cond["cell"] < 1e6 and cond["cellgrad"] > 1e14, cond


@pytest.mark.parametrize("obstacle", [None, (2, 1), (3, 1)])
def test_cellwise_constant_lps_is_the_pressure_laplacian(obstacle):
    """Projection onto cellwise constants: s(p, xi) = alpha (grad p, grad xi)
    over the fluid cells.  For linear p = a + b x + c y the divergence
    theorem gives (S p)_i = alpha * int over the fluid boundary of
    xi_i (b, c) . n, built here from the mesh alone: each boundary edge of a
    fluid cell (facing a solid cell or the outside) gives half its length
    times alpha (b, c) . n to both of its nodes.  S is symmetric positive
    semi-definite and its null space on the fluid pressures is the
    constants."""
    lev = mesh.Level(2, obstacle=obstacle)
    prm = fem.Params(nu=0.02, lps="cell")
    S = fem.lps_matrix(lev, prm).toarray()[2 * lev.nn:, 2 * lev.nn:]
    alpha, h = fem.lps_alpha(lev, prm), lev.h
    X, Y = lev.coords()
    a, b, c = 0.7, -1.3, 2.1
    got = S @ (a + b * X + c * Y).ravel()
    expect = np.zeros(lev.nn)
    solid = lambda cj, ci: (not (0 <= ci < lev.nx and 0 <= cj < lev.ny)) or lev.cell_solid[cj, ci]
    node = lambda j, i: j * lev.nnx + i
    for cj in range(lev.ny):
        for ci in range(lev.nx):
            if lev.cell_solid[cj, ci]:
                continue
            sides = [((0, -1), -b, [(cj, ci), (cj + 1, ci)]),          # left, n = (-1, 0)
                     ((0, 1), b, [(cj, ci + 1), (cj + 1, ci + 1)]),     # right
                     ((-1, 0), -c, [(cj, ci), (cj, ci + 1)]),           # bottom
                     ((1, 0), c, [(cj + 1, ci), (cj + 1, ci + 1)])]     # top
            for (dj, di), flux, ends in sides:
                if solid(cj + dj, ci + di):
                    for (j, i) in ends:
                        expect[node(j, i)] += alpha * flux * h / 2
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-13 * alpha)
    assert np.abs(expect).max() > 0.1 * alpha * h
    assert np.abs(S - S.T).max() < 1e-15
    fluid = np.abs(S).sum(axis=1) > 0
    ev = np.linalg.eigvalsh(S[np.ix_(fluid, fluid)])
    assert ev[0] > -1e-13 * ev[-1] and abs(ev[0]) < 1e-13 * ev[-1] and ev[1] > 1e-6 * ev[-1]


@pytest.mark.parametrize("ell", [1, 3])
def test_poiseuille_under_cellwise_constant_lps_misses_by_the_boundary_term(ell):
    """With the pressure Laplacian as stabilisation the Poiseuille flow is a
    fixed point except on the inflow and outflow pressure rows, where the
    residual is -(S p)_i = -alpha * int xi_i dp/dx n_x (p = 12 nu (4 - x):
    dp/dx = -12 nu), O(alpha h)."""
    lev = mesh.Level(ell, obstacle=None)
    prm = fem.Params(nu=0.01, dt=0.01, lps="cell")
    X, Y = lev.coords()
    x = np.concatenate([(6 * Y * (1 - Y)).ravel(), np.zeros(lev.nn), (12 * prm.nu * (4 - X)).ravel()])
    r = fem.residual(lev, x, fem.old_time_rhs(lev, x, prm), prm)
    alpha, h = fem.lps_alpha(lev, prm), lev.h
    expect = np.zeros(lev.ndof)
    w = np.full(lev.nny, h)
    w[[0, -1]] = h / 2                    # int xi_i dy along a vertical edge
    rp = expect[2 * lev.nn:].reshape(lev.nny, lev.nnx)
    rp[:, 0] = alpha * 12 * prm.nu * w    # (S p)_i on the inflow, n_x = -1
    rp[:, -1] = -alpha * 12 * prm.nu * w  # outflow, n_x = +1
    # residual = f - A(x): the stabilisation enters A with a plus sign
    np.testing.assert_allclose(r, -expect, rtol=0, atol=1e-13)


def test_mass_conservation_after_newton_step():
    """Summing all pressure rows (sum of xi_i = 1, LPS vanishes on constants)
    gives int div v = outflow flux - inflow flux, so a converged step carries
    the same flux out of the channel as it brings in (Q1 traces integrate
    exactly by the trapezoid rule)."""
    levels = mesh.hierarchy(3, obstacle=(3, 1))
    lev = levels[-1]
    prm = fem.Params(nu=0.01, dt=0.01)
    opt = newton.SolverOptions(newton_tol=1e-12)
    x0 = mesh.initial_state(lev)
    x1, nit, _, nrm = newton.time_step(levels, x0, prm, opt)
    assert nrm <= 1e-12
    u = x1[:lev.nn].reshape(lev.nny, lev.nnx)
    trap = lambda f: lev.h * (f.sum() - 0.5 * (f[0] + f[-1]))
    q_in, q_out = trap(u[:, 0]), trap(u[:, -1])
    assert abs(q_out - q_in) < 1e-10
    assert abs(q_in - 1.0) < 1e-3     # nodal parabola integrates to ~1


def test_newton_mg_matches_direct_solve():
    """Newton with FGMRES + V-cycle reaches the same discrete solution as
    Newton with a sparse direct solve (the solver is only a route)."""
    levels = mesh.hierarchy(2, obstacle=(2, 1))
    lev = levels[-1]
    prm = fem.Params(nu=0.01, dt=0.02)
    opt = newton.SolverOptions(newton_tol=1e-12)
    x0 = mesh.initial_state(lev)
    f = fem.old_time_rhs(lev, x0, prm)
    x_mg, *_ = newton.newton_solve(levels, x0, f, prm, opt)
    x = x0.copy()
    for _ in range(20):
        r = fem.residual(lev, x, f, prm)
        if np.linalg.norm(r) < 1e-13:
            break
        x = x + spla.spsolve(fem.jacobian(lev, x, prm).tocsc(), r)
    assert np.linalg.norm(x_mg - x) / np.linalg.norm(x) < 1e-11
