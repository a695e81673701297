"""Newton time stepping of the discrete Navier-Stokes system (oracle, test only).

Eq. 3 / Eq. 6: each time step solves A_n(x_n) = f_n by Newton's method from
the initial guess x_{n-1}; every Newton correction w solves
A'_n(x^{(l-1)}) w = f_n - A_n(x^{(l-1)}) by FGMRES preconditioned with one
multigrid V-cycle (Sec. 2.2, the Newton iteration of Algorithm 1), and the update is
damped, z <- z + eps * w (the damped update of Algorithm 1).

Readings: the iteration stops when the Euclidean norm of the nonlinear
residual over free DOFs is at most newton_tol (absolute; default 1e-10), with
a cap of newton_max iterations; FGMRES(m=20) reduces the linear residual by
gmres_rtol = 1e-4 per Newton step; eps = 1 by default.
"""
import numpy as np

from . import fem, mg
from .krylov import fgmres


class SolverOptions:
    def __init__(self, newton_tol=1e-10, newton_max=20, gmres_m=20, gmres_rtol=1e-4,
                 gmres_maxit=200, nu1=2, nu2=2, omega=0.8, eps=1.0):
        self.newton_tol, self.newton_max = newton_tol, newton_max
        self.gmres_m, self.gmres_rtol, self.gmres_maxit = gmres_m, gmres_rtol, gmres_maxit
        self.nu1, self.nu2, self.omega, self.eps = nu1, nu2, omega, eps


def newton_solve(levels, x_init, f, prm, opt, record=None):
    """Solve A_n(x) = f on the finest of `levels` starting at x_init.

    Returns (x, newton_iterations, total_gmres_iterations, final_norm).
    """
    lev = levels[-1]
    S = fem.lps_matrix(lev, prm)
    x = x_init.copy()
    x[lev.cons] = lev.dirichlet_values[lev.cons]
    r = fem.residual(lev, x, f, prm, S)
    norm = np.linalg.norm(r)
    nit, git = 0, 0
    if record is not None:
        record.append(norm)
    while norm > opt.newton_tol and nit < opt.newton_max:
        H = mg.Hierarchy(levels, x, prm, opt.nu1, opt.nu2, opt.omega)
        A = H.ops[-1].A
        L = len(levels) - 1
        w, its, _ = fgmres(lambda z: A @ z, lambda v: mg.vcycle(H, L, v), r,
                           m=opt.gmres_m, rtol=opt.gmres_rtol, maxit=opt.gmres_maxit)
        x = x + opt.eps * w
        r = fem.residual(lev, x, f, prm, S)
        norm = np.linalg.norm(r)
        nit += 1
        git += its
        if record is not None:
            record.append(norm)
    return x, nit, git, norm


def time_step(levels, x_old, prm, opt, f=None):
    """One time step of the plain method: f_n from x_{n-1} (Eq. 5) unless a
    right-hand side is given, then Newton from x_{n-1}."""
    if f is None:
        f = fem.old_time_rhs(levels[-1], x_old, prm)
    return newton_solve(levels, x_old, f, prm, opt)
