"""Pins of the oracle's obstacle variants (Sec. 2.1 leaves the geometry open):
the square snapped to level-1 cells against the level-0 block it must
reproduce at even offsets, its exact extent and nesting on every level, and the local
projection stabilisation of part-solid 2h patches against a brute-force
quadrature of its defining integral over the patch's fluid cells."""
import numpy as np
import pytest

from oracle import fem, mesh, mg


@pytest.mark.parametrize("i0,j0", [(2, 1), (3, 1), (1, 1), (13, 1)])
def test_level1_block_at_even_offsets_is_the_level0_block(i0, j0):
    for ell in range(0, 5):
        a = mesh.Level(ell, obstacle=(i0, j0)).cell_solid
        b = mesh.Level(ell, obstacle=(2 * i0, 2 * j0, 1)).cell_solid
        assert np.array_equal(a, b), ell


@pytest.mark.parametrize("i0,j0", [(5, 3), (4, 2), (7, 1), (1, 1), (27, 3), (6, 3)])
def test_level1_square_extent_and_nesting(i0, j0):
    ob = (i0, j0, 1)
    h1 = 0.125
    for ell in range(1, 5):
        lev = mesh.Level(ell, obstacle=ob)
        s = lev.cell_solid
        assert s.sum() == 16 * 4 ** (ell - 1)
        # the solid cells fill [i0 h1, i0 h1 + 0.5] x [j0 h1, j0 h1 + 0.5] exactly
        jj, ii = np.nonzero(s)
        assert np.isclose(ii.min() * lev.h, i0 * h1) and np.isclose((ii.max() + 1) * lev.h, i0 * h1 + 0.5)
        assert np.isclose(jj.min() * lev.h, j0 * h1) and np.isclose((jj.max() + 1) * lev.h, j0 * h1 + 0.5)
        # nested: the next level's solid cells are the children of these
        finer = mesh.Level(ell + 1, obstacle=ob).cell_solid
        assert np.array_equal(finer, np.kron(s, np.ones((2, 2), dtype=bool)))
    # level 0 keeps only the cells all of whose children are solid: a
    # 0.5-wide interval from an odd level-1 offset covers one level-0 cell
    s0 = mesh.Level(0, obstacle=ob).cell_solid
    assert s0.sum() == (2 if i0 % 2 == 0 else 1) * (2 if j0 % 2 == 0 else 1)


def _patch_solid_counts(lev):
    s = lev.cell_solid.astype(int)
    return s[0::2, 0::2] + s[1::2, 0::2] + s[0::2, 1::2] + s[1::2, 1::2]


def test_odd_level1_block_splits_only_level1_patches():
    ob = (5, 3, 1)
    n1 = _patch_solid_counts(mesh.Level(1, obstacle=ob))
    # the square covers level-1 cells 5..8 x 3..6: patch columns 2, 3, 4 and
    # rows 1, 2, 3, the middle one whole, the ring of eight partly solid
    assert ((n1 > 0) & (n1 < 4)).sum() == 8 and (n1 == 4).sum() == 1
    for ell in (2, 3, 4):
        n = _patch_solid_counts(mesh.Level(ell, obstacle=ob))
        assert set(np.unique(n)) <= {0, 4}


def _brute_force_lps_energy(lev, p, alpha):
    """alpha * sum over patches K, over the fluid cells T of K, of the
    integral over T of |grad(p_h - pi_K p_h)|^2, with p_h bilinear on each
    cell, pi_K p_h the bilinear interpolant of p_h's values at the corners of
    K, and 3x3 Gauss quadrature per cell (exact for these integrands)."""
    g, w = np.polynomial.legendre.leggauss(3)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    P = p.reshape(lev.nny, lev.nnx)
    h = lev.h
    total = 0.0
    for J in range(lev.ny // 2):
        for I in range(lev.nx // 2):
            c = [[P[2 * J + 2 * b, 2 * I + 2 * a] for a in (0, 1)] for b in (0, 1)]
            for cy in (0, 1):
                for cx in (0, 1):
                    if lev.cell_solid[2 * J + cy, 2 * I + cx]:
                        continue
                    i, j = 2 * I + cx, 2 * J + cy
                    v = [[P[j + b, i + a] for a in (0, 1)] for b in (0, 1)]
                    for qy, wy in zip(g, w):
                        for qx, wx in zip(g, w):
                            # cell-local derivatives of the cell's bilinear p
                            dpx = ((1 - qy) * (v[0][1] - v[0][0]) + qy * (v[1][1] - v[1][0])) / h
                            dpy = ((1 - qx) * (v[1][0] - v[0][0]) + qx * (v[1][1] - v[0][1])) / h
                            # the same point in patch coordinates (width 2h)
                            X, Y = (cx + qx) / 2.0, (cy + qy) / 2.0
                            dix = ((1 - Y) * (c[0][1] - c[0][0]) + Y * (c[1][1] - c[1][0])) / (2 * h)
                            diy = ((1 - X) * (c[1][0] - c[0][0]) + X * (c[1][1] - c[0][1])) / (2 * h)
                            total += wx * wy * h * h * ((dpx - dix) ** 2 + (dpy - diy) ** 2)
    return alpha * total


@pytest.mark.parametrize("ob", [(5, 3, 1), (4, 2, 1), (2, 1), (6, 1, 1)])
def test_lps_on_part_solid_patches_matches_brute_force(ob):
    prm = fem.Params(nu=0.01)
    lev = mesh.Level(1, obstacle=ob)
    S = fem.lps_matrix(lev, prm)
    rng = np.random.default_rng(7)
    p = rng.standard_normal(lev.nn)
    x = np.zeros(lev.ndof)
    x[2 * lev.nn:] = p
    e = float(x @ (S @ x))
    ref = _brute_force_lps_energy(lev, p, fem.lps_alpha(lev, prm))
    assert abs(e - ref) < 1e-12 * abs(ref)
    # dropping a part-solid patch, or integrating over its solid cell too,
    # would change the energy: the level-1 block at odd offsets has such patches
    if len(ob) == 3 and ob[0] % 2:
        whole = _brute_force_lps_energy(mesh.Level(1, obstacle=None), p, fem.lps_alpha(lev, prm))
        assert abs(e - whole) > 1e-6 * abs(ref)


def test_lps_with_part_solid_patches_vanishes_on_patch_bilinear_pressure():
    prm = fem.Params(nu=0.01)
    lev, parent = mesh.Level(1, obstacle=(5, 3, 1)), mesh.Level(0, obstacle=None)
    S = fem.lps_matrix(lev, prm)
    Pn = mg.prolongation_nodes(parent, lev)
    p = Pn @ np.random.default_rng(1).standard_normal(parent.nn)
    x = np.zeros(lev.ndof)
    x[2 * lev.nn:] = p
    assert np.abs(S @ x).max() < 1e-13 * np.abs(p).max()
    Sd = S.toarray()[2 * lev.nn:, 2 * lev.nn:]
    assert np.abs(Sd - Sd.T).max() < 1e-15
    assert np.linalg.eigvalsh(Sd).min() > -1e-14


@pytest.mark.parametrize("i0,j0,regular", [(5, 3, True), (5, 1, True), (6, 2, True), (2, 2, True),
                                           (6, 1, False), (4, 3, False), (1, 2, False)])
def test_level1_problem_is_singular_with_a_one_cell_strip(i0, j0, regular):
    """The level-1 Jacobian (the coarse direct solve's matrix) with the
    square snapped to level 1: a one-cell fluid strip between the square and
    the inflow, or between the square and a wall at an even level-1 offset,
    has no free velocity node and a pressure mode the whole patches'
    stabilisation does not see, so the matrix is singular; the library
    refuses those positions."""
    from tests.gpu_util import seeded_state
    prm = fem.Params(nu=0.01, dt=0.01)
    lev = mesh.Level(1, obstacle=(i0, j0, 1))
    A = fem.jacobian(lev, seeded_state(lev, 31), prm).toarray()
    s = np.linalg.svd(A, compute_uv=False)
    assert (s[-1] / s[0] > 1e-10) == regular, s[-1] / s[0]
