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
