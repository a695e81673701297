"""Q1/Q1 finite elements with local projection stabilisation (oracle, test only).

Follows Sec. 2.1: velocity and pressure in the same continuous space
(Eq. 3 and the text around it), pressure stabilised by the local projection
term sum_T alpha_T (grad(p - pi p), grad(xi - pi xi))_T with
alpha_T = alpha_0 * Re * h_T^2 (Re = 1/nu), the pressure rows of Eq. 4 and the
velocity rows of Eq. 5, written as a theta-scheme (theta = 1/2 is the
Crank-Nicolson form printed in Eq. 5, theta = 1 is backward Euler).

Readings:
  * the element is Q1 (bilinear): the DOF counts of Sec. 3.1 (2560 elements,
    8088 DOFs; 640 elements, 2124 DOFs) are three unknowns per vertex;
  * pi is bilinear interpolation on the patch mesh of width 2h (2x2 blocks
    of cells, i.e. the cells of the parent level), so kappa = id - pi
    vanishes on bilinear p.  The integral runs over the fluid cells of each
    patch; on level >= 1 a patch is all fluid or all solid when the
    obstacle is made of level-0 cells, and on level 0 a patch may be partly
    solid; with an obstacle of level-1 cells at odd level-1 offsets the
    patches of level 1 (the coarse level of the cycle) are partly solid too;
  * all integrals use 2x2 Gauss quadrature per cell, exact here for mass,
    stiffness, divergence and the Q1 convection term on square cells;
  * constrained DOFs (velocity Dirichlet nodes, fixed pressures) get identity
    rows and columns in the Jacobian; the nonlinear residual is zero on them.

Element DOF order (u0..u3, v0..v3, p0..p3), local node a = ax + 2 ay.
"""
import numpy as np
import scipy.sparse as sp

GAUSS = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
QXI = np.array([GAUSS[0], GAUSS[1], GAUSS[0], GAUSS[1]])
QETA = np.array([GAUSS[0], GAUSS[0], GAUSS[1], GAUSS[1]])
QW = np.full(4, 0.25)


def _basis(xi, eta):
    """Bilinear shape functions on [0,1]^2 and their reference derivatives."""
    phi, dxi, deta = np.zeros(4), np.zeros(4), np.zeros(4)
    for a in range(4):
        ax, ay = a & 1, a >> 1
        fx, dfx = (xi, 1.0) if ax else (1.0 - xi, -1.0)
        fy, dfy = (eta, 1.0) if ay else (1.0 - eta, -1.0)
        phi[a], dxi[a], deta[a] = fx * fy, dfx * fy, fx * dfy
    return phi, dxi, deta


_B = [_basis(QXI[q], QETA[q]) for q in range(4)]
PHI = np.array([b[0] for b in _B])      # [q, a]
DXI = np.array([b[1] for b in _B])
DETA = np.array([b[2] for b in _B])


class Params:
    """Physical and discretisation parameters of one time step.  lps selects
    the projection pi_h of the stabilisation (Sec. 2.1): "patch" (bilinear
    interpolation on the 2h patch mesh), "cell" (onto cellwise constants, so
    grad pi_h p = 0 and s is the pressure Laplacian) or "cellgrad" (the cell
    mean of the gradient)."""

    def __init__(self, nu=0.01, dt=0.01, theta=1.0, alpha0=0.1, lps="patch"):
        self.nu, self.dt, self.theta, self.alpha0 = nu, dt, theta, alpha0
        self.lps = lps


class Element:
    """Constant element matrices of a square cell of width h."""

    def __init__(self, h):
        self.h = h
        self.W = QW * h * h
        self.DX, self.DY = DXI / h, DETA / h
        W, P = self.W, PHI
        self.M = np.einsum("q,qa,qb->ab", W, P, P)
        self.K = (np.einsum("q,qa,qb->ab", W, self.DX, self.DX)
                  + np.einsum("q,qa,qb->ab", W, self.DY, self.DY))
        # Dx[a, b] = int xi_a d/dx phi_b   (pressure test a, velocity trial b)
        self.Dx = np.einsum("q,qa,qb->ab", W, P, self.DX)
        self.Dy = np.einsum("q,qa,qb->ab", W, P, self.DY)

    def convection(self, ub, vb):
        """N[n,a,b] = int phi_a (vbar . grad phi_b) for cells with nodal vbar."""
        U, V = ub @ PHI.T, vb @ PHI.T                        # [n, q]
        return (np.einsum("q,qa,nq,qb->nab", self.W, PHI, U, self.DX)
                + np.einsum("q,qa,nq,qb->nab", self.W, PHI, V, self.DY))

    def grad_mass(self, fb, D):
        """C[n,a,b] = int phi_a phi_b (d fbar) with d = D (DX or DY)."""
        G = fb @ D.T                                         # [n, q]
        return np.einsum("q,qa,qb,nq->nab", self.W, PHI, PHI, G)


def element_jacobians(level, vbar, prm):
    """12x12 Jacobians A'(vbar) of all fluid cells (Eq. 6), before LPS."""
    el = Element(level.h)
    cells = level.fluid_cells
    nodes = level.cell_nodes[cells]
    u = vbar[:level.nn][nodes]
    v = vbar[level.nn:2 * level.nn][nodes]
    n = len(cells)
    th, ik = prm.theta, 1.0 / prm.dt
    N = el.convection(u, v)
    base = ik * el.M[None] + th * (prm.nu * el.K[None] + N)
    J = np.zeros((n, 12, 12))
    J[:, 0:4, 0:4] = base + th * el.grad_mass(u, el.DX)
    J[:, 0:4, 4:8] = th * el.grad_mass(u, el.DY)
    J[:, 4:8, 0:4] = th * el.grad_mass(v, el.DX)
    J[:, 4:8, 4:8] = base + th * el.grad_mass(v, el.DY)
    J[:, 0:4, 8:12] = -el.Dx.T[None]
    J[:, 4:8, 8:12] = -el.Dy.T[None]
    J[:, 8:12, 0:4] = el.Dx[None]
    J[:, 8:12, 4:8] = el.Dy[None]
    return J


def lps_alpha(level, prm):
    """alpha_T = alpha_0 * Re * h_T^2 with Re = 1/nu (Sec. 2.1)."""
    return prm.alpha0 * level.h * level.h / prm.nu


def _interp_2h():
    """Pi[m, n]: value at parent-local node m of the bilinear interpolant of
    the four parent corners (corners are the nodes with even s and t)."""
    Pi = np.zeros((9, 9))
    for t in range(3):
        for s in range(3):
            for ct in (0, 2):
                for cs in (0, 2):
                    Pi[s + 3 * t, cs + 3 * ct] = (1 - abs(s - cs) / 2) * (1 - abs(t - ct) / 2)
    return Pi


def _cellwise(level, Sc):
    """Sum of the 4x4 pressure block Sc over the fluid cells of the level."""
    nodes = level.cell_nodes[level.fluid_cells] + 2 * level.nn
    rows = np.repeat(nodes[:, :, None], 4, axis=2).ravel()
    cols = np.repeat(nodes[:, None, :], 4, axis=1).ravel()
    vals = np.broadcast_to(Sc, (len(nodes), 4, 4)).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(level.ndof, level.ndof)).tocsr()


def lps_matrix_cell(level, prm):
    """Projection onto cellwise constants (pi_h into W^(1) read as the
    piecewise constants, Sec. 2.1): grad pi_h p = 0 inside each cell, so
    s(p, xi) = sum_K alpha (grad p, grad xi)_K over the fluid cells, the Q1
    stiffness matrix of the pressure scaled by alpha.  It does not vanish on
    linear p: by the divergence theorem S p = alpha int_dOmega xi grad p . n."""
    return _cellwise(level, lps_alpha(level, prm) * Element(level.h).K)


def lps_matrix_cellgrad(level, prm):
    """Projection of the gradient onto cellwise constants:
    s(p, xi) = sum_K alpha (grad p - pi_K grad p, grad xi - pi_K grad xi)_K,
    pi_K the mean over the fluid cell K, i.e. per cell alpha (K - g g^T / |K|)
    with g_a = int_K grad phi_a (2x2 Gauss, exact for Q1)."""
    alpha = lps_alpha(level, prm)
    el = Element(level.h)
    g = np.stack([el.W @ el.DX, el.W @ el.DY], axis=1)       # [a, 2]
    return _cellwise(level, alpha * (el.K - g @ g.T / (level.h * level.h)))


def lps_matrix(level, prm):
    """Pressure-pressure stabilisation matrix s(p, xi) on the whole level
    (patch projection; prm.lps == "cell" or "cellgrad" selects the
    cellwise forms above).

    Patches are 2x2 blocks of cells (the cells of the parent level); on each
    patch K, s_K = alpha kappa^T K9 kappa with K9 the Q1 stiffness matrix of
    the patch's fluid cells on its 3x3 nodes and kappa = I - Pi.
    """
    lps = getattr(prm, "lps", "patch")
    if lps == "cell":
        return lps_matrix_cell(level, prm)
    if lps == "cellgrad":
        return lps_matrix_cellgrad(level, prm)
    assert lps == "patch", lps
    alpha = lps_alpha(level, prm)
    el = Element(level.h)
    nn, nnx = level.nn, level.nnx
    kappa = np.eye(9) - _interp_2h()
    npx, npy = level.nx // 2, level.ny // 2
    blocks, ps = [], []
    for J in range(npy):
        for I in range(npx):
            K9 = np.zeros((9, 9))
            for cy in (0, 1):
                for cx in (0, 1):
                    if level.cell_solid[2 * J + cy, 2 * I + cx]:
                        continue
                    loc = [(cx + (a & 1)) + 3 * (cy + (a >> 1)) for a in range(4)]
                    K9[np.ix_(loc, loc)] += el.K
            if not K9.any():
                continue
            blocks.append(alpha * kappa.T @ K9 @ kappa)
            ps.append([2 * nn + (2 * J + t) * nnx + 2 * I + s
                       for t in range(3) for s in range(3)])
    dofs = np.array(ps)
    rows = np.repeat(dofs[:, :, None], 9, axis=2).ravel()
    cols = np.repeat(dofs[:, None, :], 9, axis=1).ravel()
    vals = np.array(blocks).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(level.ndof, level.ndof)).tocsr()


def _assemble(level, Je):
    dofs = level.cell_dofs[level.fluid_cells]
    rows = np.repeat(dofs[:, :, None], 12, axis=2).ravel()
    cols = np.repeat(dofs[:, None, :], 12, axis=1).ravel()
    return sp.coo_matrix((Je.ravel(), (rows, cols)), shape=(level.ndof, level.ndof)).tocsr()


def constrain(level, A):
    """Identity rows and columns on constrained DOFs."""
    Q = sp.diags(level.free.astype(float))
    return (Q @ A @ Q + sp.diags(level.cons.astype(float))).tocsr()


def jacobian(level, vbar, prm):
    """Global Jacobian A'_n(vbar) (Eq. 6) with LPS, constrained, CSR FP64."""
    A = _assemble(level, element_jacobians(level, vbar, prm)) + lps_matrix(level, prm)
    return constrain(level, A)


def mass_matrix(level):
    """Scalar Q1 mass matrix over the fluid cells (nn x nn)."""
    el = Element(level.h)
    nodes = level.cell_nodes[level.fluid_cells]
    rows = np.repeat(nodes[:, :, None], 4, axis=2).ravel()
    cols = np.repeat(nodes[:, None, :], 4, axis=1).ravel()
    vals = np.broadcast_to(el.M, (len(nodes), 4, 4)).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(level.nn, level.nn)).tocsr()


def _scatter(level, cellvals, ncomp_offset):
    out = np.zeros(level.nn)
    np.add.at(out, level.cell_nodes[level.fluid_cells], cellvals)
    return out


def transport_diffusion(level, x, prm):
    """Per component: nu (grad v_c, grad phi) + (v . grad v_c, phi), all nodes."""
    el = Element(level.h)
    nodes = level.cell_nodes[level.fluid_cells]
    u = x[:level.nn][nodes]
    v = x[level.nn:2 * level.nn][nodes]
    N = el.convection(u, v)
    out = []
    for f in (u, v):
        cv = prm.nu * f @ el.K.T + np.einsum("nab,nb->na", N, f)
        out.append(_scatter(level, cv, 0))
    return out


def operator(level, x, prm, S=None):
    """Nonlinear map A_n(x) of Eqs. 4-5 on all rows (no constraint handling)."""
    el = Element(level.h)
    nn = level.nn
    nodes = level.cell_nodes[level.fluid_cells]
    u, v, p = x[:nn][nodes], x[nn:2 * nn][nodes], x[2 * nn:][nodes]
    td_u, td_v = transport_diffusion(level, x, prm)
    Mg = mass_matrix(level)
    ik, th = 1.0 / prm.dt, prm.theta
    Au = ik * (Mg @ x[:nn]) + th * td_u - _scatter(level, p @ el.Dx, 0)
    Av = ik * (Mg @ x[nn:2 * nn]) + th * td_v - _scatter(level, p @ el.Dy, 0)
    Ap = _scatter(level, u @ el.Dx.T + v @ el.Dy.T, 0)
    if S is None:
        S = lps_matrix(level, prm)
    out = np.concatenate([Au, Av, Ap])
    return out + S @ x


def old_time_rhs(level, x_old, prm):
    """f_n of Eq. 5 without external force: (1/k)(v_{n-1}, phi)
    - (1 - theta)[(v_{n-1} . grad v_{n-1}, phi) + nu (grad v_{n-1}, grad phi)]."""
    nn = level.nn
    Mg = mass_matrix(level)
    f = np.zeros(level.ndof)
    f[:nn] = Mg @ x_old[:nn] / prm.dt
    f[nn:2 * nn] = Mg @ x_old[nn:2 * nn] / prm.dt
    if prm.theta != 1.0:
        td_u, td_v = transport_diffusion(level, x_old, prm)
        f[:nn] -= (1.0 - prm.theta) * td_u
        f[nn:2 * nn] -= (1.0 - prm.theta) * td_v
    return f


def residual(level, x, f, prm, S=None):
    """Nonlinear residual f_n - A_n(x) (Eq. 6 right-hand side), zero on
    constrained DOFs."""
    r = f - operator(level, x, prm, S)
    r[level.cons] = 0.0
    return r
