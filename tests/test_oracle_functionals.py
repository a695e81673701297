"""Pins of the oracle's functionals (Sec. 3.4): the divergence functional on
velocities whose integral is known in closed form, drag and lift in residual
form against integrals done by hand for fields that switch on one term of
the momentum rows at a time (pressure, time derivative, convection,
viscosity), the mirror symmetry of the channel, and a converged time step.
"""
import numpy as np
import pytest

from oracle import fem, functionals as fn, mesh, newton

OB = (2, 1)          # x in [0.5, 1.0], y in [0.25, 0.75]: symmetric about y = 1/2
B_AREA = 0.25


def _state(level, u, v, p):
    return np.concatenate([np.ravel(u), np.ravel(v), np.ravel(p)]).astype(float)


def _pairs(level):
    """(Gamma node, fluid cell containing it) incidences."""
    gam = fn.obstacle_boundary(level)
    nodes = level.cell_nodes[level.fluid_cells]
    return int(gam[nodes].sum())


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_divergence_closed_forms(ell):
    lev = mesh.Level(ell, obstacle=OB)
    X, Y = lev.coords()
    z = np.zeros_like(X)
    fluid = 4.0 - B_AREA
    assert fn.divergence(lev, _state(lev, X, Y, z)) == pytest.approx(4.0 * fluid, rel=1e-13)
    assert abs(fn.divergence(lev, _state(lev, X, -Y, z))) < 1e-24
    # (d/dx (x y))^2 = y^2 over the channel minus the block
    expect = 4.0 / 3.0 - 0.5 * (0.75 ** 3 - 0.25 ** 3) / 3.0
    assert fn.divergence(lev, _state(lev, X * Y, z, z)) == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_gamma_count_and_pressure_force(ell):
    """v = 0, p = x: -(p, d/dx Psi) integrates by parts to -int Psi plus the
    boundary term -|B|; p = y likewise for lift; the cross terms vanish."""
    lev = mesh.Level(ell, obstacle=OB)
    a = 2 << ell                                  # block side in cells
    assert fn.obstacle_boundary(lev).sum() == 4 * a
    assert _pairs(lev) == 8 * a + 4               # corners in 3 fluid cells, edges in 2
    int_psi = lev.h ** 2 / 4 * (8 * a + 4)
    X, Y = lev.coords()
    z = np.zeros_like(X)
    prm = fem.Params(nu=0.3, dt=0.1)
    d, l = fn.forces(lev, _state(lev, z, z, X), prm)
    assert d == pytest.approx(-B_AREA - int_psi, rel=1e-13)
    assert abs(l) < 1e-13
    d, l = fn.forces(lev, _state(lev, z, z, Y), prm)
    assert abs(d) < 1e-13
    assert l == pytest.approx(-B_AREA - int_psi, rel=1e-13)


def test_time_derivative_force():
    """Uniform velocity, v - v_old = k (a, b): J = -(a, b) int Psi."""
    lev = mesh.Level(2, obstacle=OB)
    prm = fem.Params(nu=0.02, dt=0.04)
    a_, b_ = 0.7, -1.3
    one = np.ones((lev.nny, lev.nnx))
    x = _state(lev, 0.4 * one, 0.9 * one, 0 * one)
    x_old = x - prm.dt * _state(lev, a_ * one, b_ * one, 0 * one)
    int_psi = lev.h ** 2 / 4 * _pairs(lev)
    d, l = fn.forces(lev, x, prm, x_old)
    assert d == pytest.approx(-a_ * int_psi, rel=1e-12)
    assert l == pytest.approx(-b_ * int_psi, rel=1e-12)
    # steady form: no time term, uniform flow exerts no force
    d, l = fn.forces(lev, x, prm)
    assert abs(d) < 1e-13 and abs(l) < 1e-13


def _hat_moments(lev):
    """int_F x Psi and int_F y Psi, by exact 1D integrals of the hat
    functions: on a cell to the right of node i, int x (1 - (x - x_i)/h) dx
    = x_i h / 2 + h^2 / 6; to the left, x_i h / 2 - h^2 / 6."""
    h = lev.h
    gam = fn.obstacle_boundary(lev).reshape(lev.nny, lev.nnx)
    mx = my = 0.0
    for cj in range(lev.ny):
        for ci in range(lev.nx):
            if lev.cell_solid[cj, ci]:
                continue
            for dj in (0, 1):
                for di in (0, 1):
                    i, j = ci + di, cj + dj
                    if not gam[j, i]:
                        continue
                    sx = 1.0 if di == 0 else -1.0     # cell right (+) or left (-) of the node
                    sy = 1.0 if dj == 0 else -1.0
                    mx += (i * h * h / 2 + sx * h * h / 6) * (h / 2)
                    my += (j * h * h / 2 + sy * h * h / 6) * (h / 2)
    return mx, my


def test_convection_force():
    """v = (x, -y): v . grad v = (x, y), and the viscous term of a linear
    field integrates to a closed-curve integral of n, i.e. zero."""
    lev = mesh.Level(2, obstacle=OB)
    X, Y = lev.coords()
    prm = fem.Params(nu=0.37, dt=0.1)
    d, l = fn.forces(lev, _state(lev, X, -Y, 0 * X), prm)
    mx, my = _hat_moments(lev)
    assert d == pytest.approx(-mx, rel=1e-12)
    assert l == pytest.approx(-my, rel=1e-12)


def test_viscous_force():
    """u = nodal interpolant of y^2 (linear in y on each cell row, slope
    2 y_j + h), v = 0, p = 0: only nu (d_y u, d_y Psi) remains, and
    int_cell d_y Psi = h/2 (Psi_TL + Psi_TR - Psi_BL - Psi_BR)."""
    lev = mesh.Level(2, obstacle=OB)
    X, Y = lev.coords()
    nu = 0.7
    prm = fem.Params(nu=nu, dt=0.1)
    d, l = fn.forces(lev, _state(lev, Y ** 2, 0 * X, 0 * X), prm)
    psi = fn.obstacle_boundary(lev).reshape(lev.nny, lev.nnx).astype(float)
    h = lev.h
    expect = 0.0
    for cj in range(lev.ny):
        for ci in range(lev.nx):
            if lev.cell_solid[cj, ci]:
                continue
            dpsi = h / 2 * (psi[cj + 1, ci] + psi[cj + 1, ci + 1] - psi[cj, ci] - psi[cj, ci + 1])
            expect += (2 * cj * h + h) * dpsi
    assert d == pytest.approx(-nu * expect, rel=1e-12)
    assert abs(l) < 1e-13


def test_mirror_symmetry():
    """Reflecting a state about y = 1/2 (v -> -v) keeps J_div and drag and
    flips the sign of lift; the block (2, 1) is symmetric."""
    lev = mesh.Level(2, obstacle=OB)
    rng = np.random.default_rng(4)
    prm = fem.Params(nu=0.01, dt=0.02)
    x = rng.standard_normal(lev.ndof)
    xo = rng.standard_normal(lev.ndof)

    def mirror(s):
        u, v, p = (c.reshape(lev.nny, lev.nnx)[::-1] for c in np.split(s, 3))
        return _state(lev, u, -v, p)

    d, l = fn.forces(lev, x, prm, xo)
    dm, lm = fn.forces(lev, mirror(x), prm, mirror(xo))
    assert abs(l) > 1e-3
    assert dm == pytest.approx(d, rel=1e-12)
    assert lm == pytest.approx(-l, rel=1e-12)
    assert fn.divergence(lev, mirror(x)) == pytest.approx(fn.divergence(lev, x), rel=1e-12)


def test_forces_of_converged_steps():
    """After backward-Euler steps from the impulsive start: the momentum
    residual of the functional vanishes at every free node (so any other
    extension of Psi off Gamma gives the same value), the symmetric channel
    has no lift, and the flow pushes the block downstream."""
    levels = mesh.hierarchy(2, obstacle=OB)
    lev = levels[-1]
    prm = fem.Params(nu=0.05, dt=0.05)
    opt = newton.SolverOptions(newton_tol=1e-11)
    x = mesh.initial_state(lev)
    for _ in range(2):
        x_old = x
        x, *_ = newton.time_step(levels, x, prm, opt)
    ru, rv = fn.momentum_residual(lev, x, prm, x_old)
    free_v = ~lev.vdir.ravel()
    assert np.abs(ru[free_v]).max() < 1e-10 and np.abs(rv[free_v]).max() < 1e-10
    d, l = fn.forces(lev, x, prm, x_old)
    assert d > 0.1
    assert abs(l) < 1e-8 * d
    e_v, e_p = fn.relative_errors(lev, x, x)
    assert e_v == 0 and e_p == 0
    e_v, e_p = fn.relative_errors(lev, 1.01 * x, x)
    assert e_v == pytest.approx(0.01) and e_p == pytest.approx(0.01)
