"""Host-side test helpers: ghost filling, block conversion and oracle-side initial conserved
variables.  Nothing here is part of the product path."""
import numpy as np

import oracle as O


def to_oracle(bi):
    return O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)


def _wrap_axis(a, axis, n, g, staggered):
    """Periodic ghost copy along one array axis (axis order z, y, x)."""
    a = np.moveaxis(a, axis, 0)
    if staggered:   # indices -g..n+g, face/vertex i == i+n
        for t in range(g):
            a[t] = a[n + t]                    # -g+t <- n-g+t
        for t in range(g + 1):
            a[n + g + t] = a[g + t]            # n+t <- t
    else:           # indices -g..n+g-1, cell i == i+n
        for t in range(g):
            a[t] = a[n + t]
            a[n + g + t] = a[g + t]
    return np.moveaxis(a, 0, axis)


def fill_periodic_cells(a, n, g):
    """a: (..., Nz, Ny, Nx) cell array."""
    for d in range(3):
        ax = a.ndim - 1 - d
        _wrap_axis(a, ax, n[d], g, False)
    return a


def fill_periodic_faces(B, n, g):
    for f in range(3):
        for d in range(3):
            _wrap_axis(B[f], 2 - d, n[d], g, d == f)
    return B


def fill_periodic_vertices(m, n, g):
    for d in range(3):
        _wrap_axis(m, m.ndim - 1 - d, n[d], g, True)
    return m


def cell_metric(bi, order=2):
    """Cell-centre metric (Nz, Ny, Nx, 16) on every cell where it is computable (others NaN)."""
    blk = to_oracle(bi)
    g = bi.ng
    n = bi.n
    e = 0 if order == 2 else 1
    lo = tuple(-g + e for _ in range(3))
    hi = tuple(n[d] + g - e for d in range(3))
    val, _ = O.interp_cells(blk, order, lo, hi)
    N = [v + 2 * g for v in n]
    out = np.full((N[2], N[1], N[0], 16), np.nan)
    sh = [hi[d] - lo[d] for d in range(3)]
    out[e:N[2] - e, e:N[1] - e, e:N[0] - e] = val.reshape(sh[2], sh[1], sh[0], 16)
    return out


def cell_B(bi):
    """Densitised cell-centred field, mean of the two faces, (Nz, Ny, Nx, 3)."""
    Bx, By, Bz = bi.B
    return np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]),
                     0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                     0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], axis=-1)


def cons_from_prims(bi, P: O.Params, order=2):
    """Conserved variables (5 or 6, Nz, Ny, Nx) from the block's prims with the oracle's prim2con;
    cells without a computable metric are left 0."""
    cm = cell_metric(bi, order)
    Bc = cell_B(bi)
    W = np.moveaxis(bi.W, 0, -1)
    ok = np.isfinite(cm[..., 0])
    q = np.zeros(W.shape[:-1] + (P.nq,))
    q[ok] = O.prim2con(cm[ok], W[ok], Bc[ok], P)
    return np.ascontiguousarray(np.moveaxis(q, -1, 0))


def interior(a, n, g):
    return a[..., g:g + n[2], g:g + n[1], g:g + n[0]]


def interior_faces(B, n, g):
    Bx, By, Bz = B
    return [Bx[g:g + n[2], g:g + n[1], g:g + n[0] + 1],
            By[g:g + n[2], g:g + n[1] + 1, g:g + n[0]],
            Bz[g:g + n[2] + 1, g:g + n[1], g:g + n[0]]]


def fill_outflow_x_periodic_yz(bi):
    """Copy ghosts: outflow (zero-gradient) along x, periodic along y and z."""
    n, g = bi.n, bi.ng
    W = bi.W
    for t in range(g):
        W[..., t] = W[..., g]
        W[..., n[0] + g + t] = W[..., n[0] + g - 1]
    Bx, By, Bz = bi.B
    for t in range(g):
        Bx[..., t] = Bx[..., g]
        Bx[..., n[0] + g + 1 + t] = Bx[..., n[0] + g]
        By[..., t] = By[..., g]; By[..., n[0] + g + t] = By[..., n[0] + g - 1]
        Bz[..., t] = Bz[..., g]; Bz[..., n[0] + g + t] = Bz[..., n[0] + g - 1]
    for d in (1, 2):
        ax = 2 - d
        _wrap_axis(W, W.ndim - 1 - d, n[d], g, False)
        for f in range(3):
            _wrap_axis(bi.B[f], ax, n[d], g, f == d)
    return bi


RK = {2: [(0.0, 1.0, 1.0), (0.5, 0.5, 0.5)],
      3: [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)]}


def evolve(bi, P, dt, nsteps, fill, order=2, rk=2):
    """Shu-Osher RK steps of the oracle stage; ``fill(bi)`` fills ghosts of W and B in place."""
    import copy
    U = cons_from_prims(bi, P, order)
    for _ in range(nsteps):
        U0, B0 = U.copy(), [b.copy() for b in bi.B]
        for (g0, g1, beta) in RK[rk]:
            Ps = copy.copy(P)
            Ps.rk_g0, Ps.rk_g1, Ps.rk_beta = g0, g1, beta
            U, Bo, Wo, st = O.stage_block(to_oracle(bi), U, U0, B0, dt, Ps)
            bi.W = Wo
            bi.B = Bo
            fill(bi)
    return U, bi
