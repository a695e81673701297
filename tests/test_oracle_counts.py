"""The element pair from the paper's DOF counts (Sec. 3.1: 640 cells with
2,124 unknowns, refined once to 2,560 cells with 8,088 unknowns).  For a
quadrilateral mesh of a domain with one hole (the channel around the
obstacle), Euler's formula V - E + F = 0 with 4F = 2 E_interior + E_boundary
gives V = F + E_b / 2 vertices; uniform refinement makes F four times and
E_b twice as large.  Three unknowns per vertex (equal-order Q1/Q1) fit both
counts with one boundary-edge count; Q2 velocity with Q1 pressure does not."""
from oracle import mesh


def _vertices(F, Eb):
    return F + Eb // 2


def test_paper_dof_counts_are_q1_q1():
    F0, N0, F1, N1 = 640, 2124, 2560, 8088
    assert N0 % 3 == 0
    Eb = 2 * (N0 // 3 - F0)                       # boundary edges of the coarse mesh
    assert Eb == 136
    assert 3 * _vertices(F1, 2 * Eb) == N1        # the refined count follows
    # Q2 velocity (vertices + edge midpoints + cell centres) and Q1 pressure
    V0 = _vertices(F0, Eb)
    E0 = (4 * F0 + Eb) // 2
    assert 2 * (V0 + E0 + F0) + V0 != N0


def test_oracle_levels_carry_three_unknowns_per_vertex():
    for ell in (0, 1, 3):
        lev = mesh.Level(ell)
        assert lev.ndof == 3 * lev.nn == 3 * (lev.nx + 1) * (lev.ny + 1)
        assert (lev.nx, lev.ny) == (16 * 2 ** ell, 4 * 2 ** ell)
