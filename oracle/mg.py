"""Geometric multigrid with cell-wise Vanka smoothing (oracle, test only).

Sec. 2.2 preconditions GMRES with one geometric multigrid cycle per
application (the preconditioned solve of Algorithm 1) but does not say which smoother, transfers
or coarse solver it uses.  Readings:
  * operators on every level are rediscretised (fem.jacobian) at the
    linearisation point injected nodally from the finest solved level;
  * prolongation P is bilinear interpolation between nested Q1 spaces,
    restriction R = P^T; inside the cycle both act on free DOFs only
    (P is followed and preceded by zeroing constrained DOFs);
  * smoother: multiplicative cell-wise Vanka over four colours of cells
    ((i mod 2, j mod 2) in the order (0,0), (1,0), (0,1), (1,1)).  In one
    colour all cells take their local defect from the same iterate and are
    updated together; cells of one colour share no node.  The local matrix
    A_c is the restriction of the global Jacobian to the cell's 12 DOFs and
    the update is x_c += omega * A_c^{-1} (b - A x)_c.  Solid cells are
    skipped;
  * the coarsest level of the cycle is solved directly by dense LU with
    partial pivoting.  It is level 1 (32x8 cells, 891 unknowns), not level 0:
    with a 2x2 block of level-0 cells as obstacle in a 4-cell-high channel,
    level 0 has no free velocity node beside the obstacle, so the flow is
    blocked there and the pressure upstream is undetermined (singular);
  * V(nu1, nu2) cycle, zero initial guess when used as preconditioner.
"""
import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from . import fem

COLOURS = ((0, 0), (1, 0), (0, 1), (1, 1))


def prolongation_nodes(coarse, fine):
    """Bilinear interpolation of nodal values, (fine.nn x coarse.nn)."""
    rows, cols, vals = [], [], []
    for j in range(fine.nny):
        for i in range(fine.nnx):
            r = j * fine.nnx + i
            I0, J0 = i // 2, j // 2
            wi = [(I0, 1.0)] if i % 2 == 0 else [(I0, 0.5), (I0 + 1, 0.5)]
            wj = [(J0, 1.0)] if j % 2 == 0 else [(J0, 0.5), (J0 + 1, 0.5)]
            for (I, a) in wi:
                for (J, b) in wj:
                    rows.append(r)
                    cols.append(J * coarse.nnx + I)
                    vals.append(a * b)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.nn, coarse.nn))


def prolongation(coarse, fine):
    """Bilinear prolongation of all three fields (unmasked)."""
    Pn = prolongation_nodes(coarse, fine)
    return sp.block_diag([Pn, Pn, Pn]).tocsr()


def prolongation_masked(coarse, fine):
    """P restricted to free DOFs on both sides, as used inside the cycle."""
    P = prolongation(coarse, fine)
    return (sp.diags(fine.free.astype(float)) @ P @ sp.diags(coarse.free.astype(float))).tocsr()


def inject(fine_x, coarse, fine, ncomp=2):
    """Nodal injection of the first ncomp fields: coarse node (I,J) takes the
    value of fine node (2I, 2J)."""
    out = []
    for c in range(ncomp):
        f = fine_x[c * fine.nn:(c + 1) * fine.nn].reshape(fine.nny, fine.nnx)
        out.append(f[::2, ::2].ravel())
    return np.concatenate(out)


def vanka_blocks(level, A):
    """A_c = A[dofs_c, dofs_c] for every cell (12x12, FP64)."""
    dofs = level.cell_dofs
    n = dofs.shape[0]
    r = np.repeat(dofs[:, :, None], 12, axis=2).ravel()
    c = np.repeat(dofs[:, None, :], 12, axis=1).ravel()
    vals = np.asarray(A[r, c]).ravel()
    return vals.reshape(n, 12, 12)


class LevelOp:
    """Everything the cycle needs on one level for one linearisation."""

    def __init__(self, level, vbar, prm, coarsest):
        self.level = level
        self.A = fem.jacobian(level, vbar, prm)
        if coarsest:
            self.lu = sla.lu_factor(self.A.toarray())
        else:
            self.blocks = vanka_blocks(level, self.A)
            cs = level.cell_solid
            jj, ii = np.meshgrid(np.arange(level.ny), np.arange(level.nx), indexing="ij")
            self.colour_cells = [np.flatnonzero(((ii % 2 == ci) & (jj % 2 == cj) & ~cs).ravel())
                                 for (ci, cj) in COLOURS]


class Hierarchy:
    """Cycle levels (levels[0] is the directly solved coarsest one) with
    operators linearised at vbar, given on the finest level levels[-1]."""

    def __init__(self, levels, vbar_L, prm, nu1=2, nu2=2, omega=0.8):
        self.levels = levels
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        L = len(levels) - 1
        vb = [None] * (L + 1)
        vb[L] = vbar_L[:2 * levels[L].nn]
        for k in range(L, 0, -1):
            vb[k - 1] = inject(vb[k], levels[k - 1], levels[k])
        self.vbar = vb
        self.ops = []
        for k in range(L + 1):
            full = np.zeros(levels[k].ndof)
            full[:2 * levels[k].nn] = vb[k]
            self.ops.append(LevelOp(levels[k], full, prm, coarsest=(k == 0)))
        self.P = [None] + [prolongation_masked(levels[k - 1], levels[k]) for k in range(1, L + 1)]


def vanka_sweep(op, b, x, omega):
    """One multiplicative four-colour Vanka sweep, in place on x."""
    dofs = op.level.cell_dofs
    for cells in op.colour_cells:
        d = b - op.A @ x
        idx = dofs[cells]
        delta = np.linalg.solve(op.blocks[cells], d[idx][..., None])[..., 0]
        x[idx] += omega * delta
    return x


def coarse_solve(op, b):
    """Direct solve on the coarsest cycle level by LU with partial pivoting."""
    return sla.lu_solve(op.lu, b)


def vcycle(H, ell, b, x=None):
    """One V(nu1, nu2) cycle on cycle level ell (index into H.levels) for
    A x = b; returns x."""
    op = H.ops[ell]
    if x is None:
        x = np.zeros_like(b)
    else:
        x = x.copy()
    if ell == 0:
        return coarse_solve(op, b)
    for _ in range(H.nu1):
        vanka_sweep(op, b, x, H.omega)
    d = b - op.A @ x
    bc = H.P[ell].T @ d
    xc = vcycle(H, ell - 1, bc)
    x += H.P[ell] @ xc
    for _ in range(H.nu2):
        vanka_sweep(op, b, x, H.omega)
    return x
