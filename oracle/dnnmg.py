"""The DNN-MG additions to a time step (oracle, test only).

the network correction of Algorithm 1 and Sec. 2.2: after the Newton solve on level L,
  6  v~^{L+1} = P(v^L)                      (prolongation to level L+1)
  7  d^{L+1}  = N(v~^{L+1}, Omega_L, Omega_{L+1})   (network, per patch)
  8  b^{L+1}_{n+1} = Rhs(v~^{L+1} + d^{L+1}, f_n, f_{n+1})
  9  b^L_{n+1} = R(b^{L+1}_{n+1})            (restriction to level L)
The network input of a patch is the residual of Eq. 3 on level L+1, the
prolongated velocity, geometric properties (aspect ratio) and the Peclet
number over the patch; the output is a velocity correction only.

Readings:
  * a patch is one level-L cell; with one replaced level it covers 2x2 fine
    cells = 3x3 fine nodes (local index m = s + 3t), with two replaced
    levels 4x4 cells = 5x5 nodes of level L+2 (then "fine" below is L+2 and
    P is applied twice).  Patches on solid cells are skipped;
  * the fine residual is r = f^{fine} - A^{fine}(v~, P p^L) on velocity rows,
    zero on Dirichlet rows, with f^{fine} = (1/k) M^{fine} v_corr,n-1 the
    old-time term built from the previous corrected fine velocity;
  * input features per patch, in this order: v~_u at the patch nodes, v~_v,
    r_u, r_v, then [h_L / 0.25, aspect ratio h_x/h_y, Pe, k / h_L] with
    Pe = |mean of v~ over the patch nodes| * h_L / nu; each feature is then
    standardised, (value - mean) / std, with statistics of the corpus;
  * the correction at a fine node is the mean of the predictions of all
    patches containing it, and zero on velocity Dirichlet nodes;
  * Rhs (the right-hand side Rhs of Algorithm 1) for backward Euler is (1/k) M^{fine} (v~ + d)
    (theta-scheme: minus (1-theta) times the explicit transport and
    diffusion of v~ + d), external force f = 0; R = P^T per component;
    Dirichlet rows of b^L are irrelevant (the Newton solve overwrites them).
"""
import numpy as np

from . import fem, mg


def prolongate_state(coarse, fine, x):
    """Bilinear P of all three fields (unmasked)."""
    Pn = mg.prolongation_nodes(coarse, fine)
    return np.concatenate([Pn @ x[c * coarse.nn:(c + 1) * coarse.nn] for c in range(3)])


def patch_nodes(coarse, fine, ratio):
    """[P, (ratio+1)^2] fine node indices of every fluid level-L cell (patch),
    patches in cell-id order, nodes with s (x) fastest."""
    cells = coarse.fluid_cells
    I, J = cells % coarse.nx, cells // coarse.nx
    k = ratio + 1
    s = np.arange(k)
    ii = ratio * I[:, None, None] + s[None, None, :]
    jj = ratio * J[:, None, None] + s[None, :, None]
    return (jj * fine.nnx + ii).reshape(len(cells), k * k)


def fine_residual(fine, xt, v_corr_prev, prm):
    """Residual of Eq. 3 on the fine level at (v~, P p), velocity rows."""
    f = fem.old_time_rhs(fine, v_corr_prev, prm)
    f[2 * fine.nn:] = 0.0
    x = xt.copy()
    x[fine.cons] = fine.dirichlet_values[fine.cons]
    return fem.residual(fine, x, f, prm)


def patch_features(coarse, fine, ratio, xt, r, prm, mean=None, std=None):
    """[P, 4 (ratio+1)^2 + 4] network inputs (raw if mean/std are None)."""
    nodes = patch_nodes(coarse, fine, ratio)
    nn = fine.nn
    ut, vt = xt[:nn][nodes], xt[nn:2 * nn][nodes]
    ru, rv = r[:nn][nodes], r[nn:2 * nn][nodes]
    hL = coarse.h
    speed = np.hypot(ut.mean(1), vt.mean(1))
    geo = np.stack([np.full(len(nodes), hL / 0.25), np.ones(len(nodes)),
                    speed * hL / prm.nu, np.full(len(nodes), prm.dt / hL)], axis=1)
    X = np.concatenate([ut, vt, ru, rv, geo], axis=1)
    if mean is not None:
        X = (X - mean) / std
    return X


def scatter_average(coarse, fine, ratio, d):
    """Mean over containing patches of the per-patch corrections d
    [P, 2 (ratio+1)^2] -> fine velocity correction (2 nn), zero on Dirichlet."""
    nodes = patch_nodes(coarse, fine, ratio)
    k2 = nodes.shape[1]
    nn = fine.nn
    cnt = np.bincount(nodes.ravel(), minlength=nn).astype(float)
    out = np.zeros(2 * nn)
    for c in range(2):
        s = np.bincount(nodes.ravel(), weights=d[:, c * k2:(c + 1) * k2].ravel(), minlength=nn)
        out[c * nn:(c + 1) * nn] = np.where(cnt > 0, s / np.maximum(cnt, 1), 0.0)
    vd = fine.vdir.ravel()
    out[:nn][vd] = 0.0
    out[nn:][vd] = 0.0
    return out


def rhs_and_restrict(coarse, fine, levels_between, v_corr, prm):
    """b^{fine} = Rhs(v_corr) and b^L = R b^{fine} (Algorithm 1).

    levels_between lists the levels from L to the fine level, so that R is
    applied once per replaced level.  Returns (b_fine, b_L) as full vectors
    (pressure rows zero)."""
    b = fem.old_time_rhs(fine, v_corr, prm)
    b[2 * fine.nn:] = 0.0
    bL = b
    for k in range(len(levels_between) - 1, 0, -1):
        f, c = levels_between[k], levels_between[k - 1]
        Pn = mg.prolongation_nodes(c, f)
        bL = np.concatenate([Pn.T @ bL[i * f.nn:(i + 1) * f.nn] for i in range(3)])
    return b, bL


def prolongate_chain(chain, x):
    """P applied once per level step of chain = [L, L+1, ..., fine]."""
    for k in range(len(chain) - 1):
        x = prolongate_state(chain[k], chain[k + 1], x)
    return x


def time_step(levels, fine, x_old, state, spec, params, prm, opt, mean=None, std=None,
              fallback_its=8, bf16=True):
    """One DNN-MG time step (Algorithm 1): Newton on level L with the
    restricted right-hand side of the previous step (if any; otherwise the
    plain old-time term), redone without it if Newton needs more than
    `fallback_its` iterations (Sec. 3.3), then the network correction.

    fine: the level above L (one replaced level) or the list of levels
    [L+1, ..., L+r] that the network replaces (Sec. 2.2: one or multiple
    finest levels); P and R are then applied once per replaced level and a
    patch covers (2^r + 1)^2 nodes of level L+r.

    state: dict(bL, vcorr, h) from the previous step (None, None, zeros at
    the start).  Returns (x_new, new_state, info)."""
    from . import net, newton
    coarse = levels[-1]
    chain = [coarse] + (list(fine) if isinstance(fine, (list, tuple)) else [fine])
    fine = chain[-1]
    ratio = 2 ** (len(chain) - 1)
    plain_f = fem.old_time_rhs(coarse, x_old, prm)
    f = state["bL"] if state["bL"] is not None else plain_f
    x, nit, git, nrm = newton.newton_solve(levels, x_old, f, prm, opt)
    fallback = False
    if state["bL"] is not None and (nrm > opt.newton_tol or nit > fallback_its):
        x, nit2, git2, nrm = newton.newton_solve(levels, x_old, plain_f, prm, opt)
        nit, git, fallback = nit + nit2, git + git2, True
    nn = fine.nn
    if state["vcorr"] is not None:
        vprev = state["vcorr"]
    else:
        vprev = prolongate_chain(chain, x_old)
        vprev[2 * nn:] = 0.0
    xt = prolongate_chain(chain, x)
    r = fine_residual(fine, xt, vprev, prm)
    X = patch_features(coarse, fine, ratio, xt, r, prm, mean, std)
    if bf16:
        X = net.bf16_round(X)
    y, h = net.step_forward(spec, params, X, state["h"], bf16)
    d = scatter_average(coarse, fine, ratio, y)
    vcorr = xt.copy()
    vcorr[:2 * nn] += d
    vcorr[2 * nn:] = 0.0
    _, bL = rhs_and_restrict(coarse, fine, chain, vcorr, prm)
    info = dict(newton_its=nit, gmres_its=git, res=nrm, fallback=fallback, X=X, y=y)
    return x, dict(bL=bL, vcorr=vcorr, h=h), info
