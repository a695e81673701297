"""Flexible GMRES with restarts (oracle, test only).

Sec. 2.2 solves each Newton step (Eq. 6) with GMRES preconditioned by
geometric multigrid.  Because one V-cycle is used as the preconditioner (and
in mixed precision it is not exactly a fixed linear map), the flexible,
right-preconditioned variant is used: x = x0 + Z y with z_j = M^{-1} v_j.
Arnoldi by modified Gram-Schmidt, least squares by Givens rotations.
"""
import numpy as np


def fgmres(matvec, precond, b, x0=None, m=20, rtol=1e-4, atol=0.0, maxit=200):
    """Solve A x = b; returns (x, iterations, final residual norm estimate).

    Stops when ||b - A x|| <= max(rtol * ||b - A x0||, atol) or after maxit
    Arnoldi steps in total.
    """
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    its = 0
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    target = max(rtol * beta, atol)
    if beta <= target:
        return x, 0, beta
    while True:
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= target or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + Z[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= target or its >= maxit:
            return x, its, beta
