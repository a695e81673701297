"""Mesh hierarchy of the channel and its boundary masks (oracle, test only).

Sec. 2.1 states the problem on a domain with Dirichlet boundary Gamma^D and
a do-nothing outflow Gamma^N (Eq. 2); Sec. 2.2 uses a hierarchy of nested,
uniformly refined meshes Omega_0 c ... c Omega_L c Omega_{L+1}.

Readings (the paper gives no geometry for this channel):
  * domain [0,4]x[0,1], level l has (16*2^l) x (4*2^l) square cells of
    width h_l = 0.25 * 2^-l;
  * the obstacle is a 2x2 block of level-0 cells, so it is resolved exactly
    on every level; or (obstacle = (i0, j0, 1)) the same square snapped to
    level-1 cells (4x4 of them from cell (i0, j0)), resolved exactly on
    levels >= 1, where a level-0 cell is solid only when all four of its
    level-1 children are (the coarser level sees a smaller obstacle);
  * velocity Dirichlet nodes: the inflow x=0 (u = 6y(1-y), v = 0), the walls
    y=0 and y=1 and every node of a solid cell (no slip, also the obstacle
    interior); the outflow x=4 is do-nothing (natural);
  * pressure is an unknown at every node of a fluid cell; nodes with no
    fluid cell have their pressure fixed to 0 (identity rows).

Unknown vectors are laid out [3][ny+1][nx+1] (u, v, p; x index fastest).
"""
import numpy as np

NX0, NY0, LX = 16, 4, 4.0


def inflow_profile(y):
    """Parabolic inflow with mean speed 1 (Eq. 2, v = v^D on Gamma^D)."""
    return 6.0 * y * (1.0 - y)


class Level:
    """One mesh level: sizes, solid cells and the constrained-DOF masks."""

    def __init__(self, ell, obstacle=(2, 1)):
        self.ell = ell
        self.nx, self.ny = NX0 << ell, NY0 << ell
        self.h = LX / self.nx
        self.nnx, self.nny = self.nx + 1, self.ny + 1
        self.nn = self.nnx * self.nny
        self.ndof = 3 * self.nn
        self.obstacle = obstacle

        if obstacle is None:
            solid = np.zeros((self.ny, self.nx), dtype=bool)
        else:
            i0, j0 = obstacle[0], obstacle[1]
            olev = obstacle[2] if len(obstacle) > 2 else 0
            B = 2 << olev                     # the square's width in level-olev cells
            if ell >= olev:
                # the level-olev cell containing each cell of this level
                ci = np.arange(self.nx) >> (ell - olev)
                cj = np.arange(self.ny) >> (ell - olev)
                solid = ((ci[None, :] >= i0) & (ci[None, :] < i0 + B)
                         & (cj[:, None] >= j0) & (cj[:, None] < j0 + B))
            else:
                # the descendants [s i, s (i + 1)) on level olev all in the square
                sc = 1 << (olev - ell)
                ci = np.arange(self.nx)
                cj = np.arange(self.ny)
                solid = ((sc * ci[None, :] >= i0) & (sc * (ci[None, :] + 1) <= i0 + B)
                         & (sc * cj[:, None] >= j0) & (sc * (cj[:, None] + 1) <= j0 + B))
        self.cell_solid = solid

        # A node touches the (up to four) cells around it.
        touch_solid = np.zeros((self.nny, self.nnx), dtype=bool)
        touch_fluid = np.zeros((self.nny, self.nnx), dtype=bool)
        for dj in (0, 1):
            for di in (0, 1):
                touch_solid[dj:dj + self.ny, di:di + self.nx] |= solid
                touch_fluid[dj:dj + self.ny, di:di + self.nx] |= ~solid
        self.node_touch_fluid = touch_fluid

        vdir = touch_solid.copy()
        vdir[:, 0] = True
        vdir[0, :] = True
        vdir[-1, :] = True
        self.vdir = vdir                      # [nny, nnx] bool
        self.pfix = ~touch_fluid              # [nny, nnx] bool
        self.cons = np.concatenate([vdir.ravel(), vdir.ravel(), self.pfix.ravel()])
        self.free = ~self.cons

        y = np.arange(self.nny) * self.h
        g = np.zeros((3, self.nny, self.nnx))
        g[0, :, 0] = inflow_profile(y)      # zero at the two wall corners
        self.dirichlet_values = g.ravel()     # values of constrained DOFs

        # Cell -> global DOF map, local order (u0..u3, v0..v3, p0..p3) with
        # local node a = ax + 2*ay at (i+ax, j+ay).
        jj, ii = np.meshgrid(np.arange(self.ny), np.arange(self.nx), indexing="ij")
        nodes = np.stack([jj * self.nnx + ii, jj * self.nnx + ii + 1,
                          (jj + 1) * self.nnx + ii, (jj + 1) * self.nnx + ii + 1],
                         axis=-1).reshape(-1, 4)
        self.cell_nodes = nodes               # [ncell, 4], cell id = j*nx + i
        self.cell_dofs = np.concatenate([nodes, nodes + self.nn, nodes + 2 * self.nn], axis=1)
        self.fluid_cells = np.flatnonzero(~solid.ravel())

    def node_index(self, i, j):
        return j * self.nnx + i

    def coords(self):
        x = np.arange(self.nnx) * self.h
        y = np.arange(self.nny) * self.h
        return np.meshgrid(x, y)


COARSEST = 1


def hierarchy(L, obstacle=(2, 1), coarsest=COARSEST):
    """Levels coarsest..L of the channel (the multigrid cycle's levels)."""
    return [Level(ell, obstacle) for ell in range(coarsest, L + 1)]


def initial_state(level):
    """Impulsive start: zero interior velocity and pressure, Dirichlet data on
    the boundary (Eq. 2 gives v_0 without a value)."""
    x = np.zeros(level.ndof)
    x[level.cons] = level.dirichlet_values[level.cons]
    return x
