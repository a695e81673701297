"""Functionals of a discrete solution, Sec. 3.4 (oracle, test only).

* J_div(v) = int_Omega |div v|^2 dx over the fluid cells, 2x2 Gauss per
  cell (exact: div v of a Q1 velocity is linear in each coordinate).
* Drag and lift: J_e = -int_Gamma (nu grad v - p I) n . e ds on the
  obstacle boundary Gamma, n pointing into the obstacle, e = e_x (drag) or
  e_y (lift).  Evaluated in the residual (volume) form: with the discrete
  test function Psi_e = e * sum_{i on Gamma} phi_i,
      J_e = -[ ((v - v_old)/k, Psi) + (v . grad v, Psi) + nu (grad v, grad Psi)
               - (p, div Psi) ],
  i.e. minus the momentum rows of the backward-Euler operator at time t_n,
  summed over the nodes of Gamma.  Psi vanishes on the outer boundary, and
  the do-nothing outflow adds no term, so for fields satisfying the momentum
  equation Green's formula turns this into the boundary integral above
  (the outward normal of the fluid on Gamma points into the obstacle).
  With x_old = None the time-derivative term is left out (steady form).
* Relative l2 errors of velocity and pressure against a reference state.

Gamma = the velocity-Dirichlet nodes strictly inside the channel that touch
a fluid cell (the obstacle's boundary nodes); the solid-interior nodes touch
no fluid cell and would contribute nothing.
"""
import numpy as np
import scipy.sparse as sp

from . import fem


def obstacle_boundary(level):
    """Boolean [nn]: the nodes of Gamma."""
    i = np.arange(level.nn) % level.nnx
    j = np.arange(level.nn) // level.nnx
    inner = (i > 0) & (i < level.nx) & (j > 0) & (j < level.ny)
    return level.vdir.ravel() & level.node_touch_fluid.ravel() & inner


def divergence(level, x):
    """J_div of the velocity of state x (Sec. 3.4)."""
    el = fem.Element(level.h)
    nn = level.nn
    nodes = level.cell_nodes[level.fluid_cells]
    div = x[:nn][nodes] @ el.DX.T + x[nn:2 * nn][nodes] @ el.DY.T   # [cell, gauss point]
    return float(np.sum(div ** 2 @ el.W))


def momentum_residual(level, x, prm, x_old=None):
    """Momentum rows (ru, rv) of the backward-Euler operator at every node:
    (1/k) M (v - v_old) + nu K v + N(v) v - (p, div phi), with no constraint
    handling.  x_old = None drops the time-derivative term."""
    be = fem.Params(nu=prm.nu, dt=prm.dt, theta=1.0, alpha0=prm.alpha0, lps=prm.lps)
    # the LPS term lives in the pressure rows only, which are not returned
    A = fem.operator(level, x, be, S=sp.csr_matrix((level.ndof, level.ndof)))
    nn = level.nn
    Mg = fem.mass_matrix(level)
    old = x if x_old is None else x_old
    ru = A[:nn] - Mg @ old[:nn] / prm.dt
    rv = A[nn:2 * nn] - Mg @ old[nn:2 * nn] / prm.dt
    return ru, rv


def forces(level, x, prm, x_old=None):
    """(J_drag, J_lift) of state x (Sec. 3.4), residual form."""
    ru, rv = momentum_residual(level, x, prm, x_old)
    gam = obstacle_boundary(level)
    return -float(ru[gam].sum()), -float(rv[gam].sum())


def relative_errors(level, x, x_ref):
    """(velocity, pressure) relative l2 errors of x against x_ref (Sec. 3.4)."""
    nn = level.nn
    dv = np.linalg.norm(x[:2 * nn] - x_ref[:2 * nn]) / np.linalg.norm(x_ref[:2 * nn])
    dp = np.linalg.norm(x[2 * nn:] - x_ref[2 * nn:]) / np.linalg.norm(x_ref[2 * nn:])
    return float(dv), float(dp)
