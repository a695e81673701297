"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws random numbers
(obstacle positions, viscosities, random fields, random network weights and
patch inputs) from seeds, so that the CUDA path and the oracle can be fed the
same inputs.  The channel workload it describes stands in for the obstacle
benchmark of Sec. 3.1 (elliptic obstacles in a channel), whose geometry and
data are not available.
"""
import numpy as np

# Channel [0, 4] x [0, 1], coarse mesh of 16 x 4 square cells of width 0.25.
LX, LY = 4.0, 1.0
NX0, NY0 = 16, 4

# Allowed obstacle centres: a 2x2 block of coarse cells centred at
# x in [0.6, 1.2], y in [0.35, 0.65] can only sit at x_c in {0.75, 1.0},
# y_c = 0.5 when aligned with the coarse cells.
OBSTACLE_CENTRES_X = (0.75, 1.0)


def obstacle_block(seed):
    """Lower-left coarse cell (i0, j0) of the 2x2 solid block for a seed."""
    rng = np.random.default_rng(1_000_003 + int(seed))
    xc = OBSTACLE_CENTRES_X[int(rng.integers(0, len(OBSTACLE_CENTRES_X)))]
    i0 = int(round(xc / 0.25)) - 1
    j0 = 1
    return (i0, j0)


def viscosity(seed, lo, hi):
    """nu drawn uniformly from [lo, hi] for a seed."""
    rng = np.random.default_rng(2_000_003 + int(seed))
    return float(rng.uniform(lo, hi))


def random_vector(seed, n, scale=1.0):
    """Standard normal FP64 vector of length n."""
    rng = np.random.default_rng(3_000_017 + int(seed))
    return scale * rng.standard_normal(n)


def random_velocity_field(seed, nny, nnx, amp=0.3):
    """Smooth random velocity perturbation (u, v) on a node grid, FP64.

    A handful of low Fourier modes with random amplitudes: it has the
    spatial structure of a developing channel flow rather than white noise.
    """
    rng = np.random.default_rng(4_000_037 + int(seed))
    y = np.linspace(0.0, 1.0, nny)[:, None]
    x = np.linspace(0.0, 4.0, nnx)[None, :]
    u = np.zeros((nny, nnx))
    v = np.zeros((nny, nnx))
    for kx in range(1, 4):
        for ky in range(1, 3):
            a, b, c, d = rng.standard_normal(4)
            u += amp * a * np.sin(kx * np.pi * x / 4 + c) * np.sin(ky * np.pi * y)
            v += amp * b * np.sin(kx * np.pi * x / 4 + d) * np.sin(ky * np.pi * y)
    return u, v


def random_weights(seed, n, scale=0.1):
    """Flat FP64 parameter vector drawn uniformly from [-scale, scale]."""
    rng = np.random.default_rng(5_000_011 + int(seed))
    return rng.uniform(-scale, scale, n)


def random_patch_inputs(seed, shape, scale=1.0):
    """Standard-normal patch features of the given shape, FP64."""
    rng = np.random.default_rng(6_000_001 + int(seed))
    return scale * rng.standard_normal(shape)
