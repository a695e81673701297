"""Helpers shared by the GPU parity tests: building the CUDA library, making
contexts, and seeded states that satisfy the boundary conditions."""
import numpy as np
import pytest

import synthetic
from oracle import mesh


def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07687_gb300 import build, dnnmg
    build.build()
    dnnmg.load()
    return dnnmg


def seeded_state(lev, seed, amp=0.3, p_scale=0.1):
    """A velocity field with the channel's boundary values plus a smooth
    random perturbation, and a random pressure (FP64, [3][nn])."""
    X, Y = lev.coords()
    u, v = synthetic.random_velocity_field(seed, lev.nny, lev.nnx, amp)
    u = u + 6 * Y * (1 - Y)
    p = p_scale * synthetic.random_vector(seed + 17, lev.nn)
    x = np.concatenate([u.ravel(), v.ravel(), p])
    x[lev.cons] = lev.dirichlet_values[lev.cons]
    return x


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def near_dirichlet_dofs(lev):
    """Free DOFs whose node lies next to a velocity-Dirichlet node (walls,
    inflow, obstacle; 8-neighbourhood) or on the outflow boundary: where a
    localised boundary error would hide under a whole-vector norm."""
    vd = lev.vdir
    near = np.zeros_like(vd)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            s = np.roll(np.roll(vd, dj, axis=0), di, axis=1)
            if dj == 1:
                s[0, :] = False
            if dj == -1:
                s[-1, :] = False
            if di == 1:
                s[:, 0] = False
            if di == -1:
                s[:, -1] = False
            near |= s
    near[:, -1] = True
    m = np.concatenate([near.ravel()] * 3)
    return np.flatnonzero(m & lev.free)


def max_rel(a, b, idx, ncomp=3):
    """Largest |a - b| over the DOFs idx, relative to the largest |b| of the
    same field (each of the ncomp fields separately; returns the worst)."""
    n = b.size // ncomp
    worst = 0.0
    for c in range(ncomp):
        sel = idx[(idx >= c * n) & (idx < (c + 1) * n)]
        if sel.size == 0:
            continue
        scale = max(np.abs(b[c * n:(c + 1) * n]).max(), 1e-300)
        worst = max(worst, float(np.abs(a[sel] - b[sel]).max() / scale))
    return worst
