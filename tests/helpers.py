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


def two_level_periodic(seed=0, g=3, bmag=0.05):
    """A periodic two-level mesh: one coarse block C (8^3 cells of 2h) and four fine blocks F (8^3 cells
    of h, a 2 x 2 layer along y, z) on its +x side, on [0, 24h) x [0, 16h)^2, h = 1/16.  Every field is
    generated once on the fine grid (periodic, ghost width 2g) and each block takes its window: fine
    blocks directly, the coarse block as means over 2^3 cells (W), 2^2 faces (B, from a vector potential
    whose coarse edge values are means of the two fine edge values, so that the coarse faces equal the
    means of the fine faces to rounding) and every second vertex (metric).  Ghosts come from the same
    global field (an AMR code would fill the fine ghosts by prolongation).
    Returns (blocks [C, F00, F10, F01, F11], records) with records (coarse, fine, d, side, o1, o2)."""
    from paper_2311_04989_gb300.inputs import BlockInput
    rng = np.random.default_rng(seed)
    h = 1.0 / 16
    nf = (24, 16, 16)
    G = 2 * g                        # ghost width of the global fine arrays
    L = (nf[0] * h, nf[1] * h, nf[2] * h)
    ph = rng.uniform(0, 2 * np.pi, 16)
    modes = rng.integers(-1, 2, (16, 2, 3))
    modes[:, :, 0] = np.where(np.all(modes == 0, axis=2), 1, modes[:, :, 0])

    def wave(x, y, z, k):
        """two plane waves with integer mode numbers on each axis's own period (periodic)"""
        out = 0.0
        for q in range(2):
            m = modes[k, q]
            out = out + np.sin(2 * np.pi * (m[0] * x / L[0] + m[1] * y / L[1] + m[2] * z / L[2]) + ph[k] + q)
        return 0.5 * out

    ax = [(np.arange(-G, nf[a] + G) + 0.5) * h for a in range(3)]      # cell centres
    av = [np.arange(-G, nf[a] + G + 1) * h for a in range(3)]          # vertices
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    W = np.zeros((5,) + X.shape)
    W[0] = 1e-3 * (1 + 0.3 * wave(X, Y, Z, 0))
    W[1] = 0.1 * wave(X, Y, Z, 3)
    W[2] = 0.1 * wave(X, Y, Z, 6)
    W[3] = 0.05 * wave(X, Y, Z, 9)
    W[4] = 1e-4 * (1 + 0.3 * wave(X, Y, Z, 1))
    Zv, Yv, Xv = np.meshgrid(av[2], av[1], av[0], indexing="ij")
    M = np.zeros((16,) + Xv.shape)
    M[0] = 1 + 0.01 * wave(Xv, Yv, Zv, 2)
    M[4] = M[7] = M[9] = 1 + 0.01 * wave(Xv, Yv, Zv, 4)
    M[5] = 0.002 * wave(Xv, Yv, Zv, 5)
    # edge vector potential (periodic): A_x at (cell x, vertex y, vertex z), A_y at (vertex x, cell y,
    # vertex z), A_z at (vertex x, vertex y, cell z)
    def pot(comp, Xe, Ye, Ze):
        return bmag * h * 16 * wave(Xe, Ye, Ze, 7 + comp) / (2 * np.pi)
    Zz, Yy, Xx = np.meshgrid(av[2], av[1], ax[0], indexing="ij"); Axf = pot(0, Xx, Yy, Zz)
    Zz, Yy, Xx = np.meshgrid(av[2], ax[1], av[0], indexing="ij"); Ayf = pot(1, Xx, Yy, Zz)
    Zz, Yy, Xx = np.meshgrid(ax[2], av[1], av[0], indexing="ij"); Azf = pot(2, Xx, Yy, Zz)

    def curl(Ax, Ay, Az, d):
        Bx = (Az[:, 1:, :] - Az[:, :-1, :]) / d - (Ay[1:, :, :] - Ay[:-1, :, :]) / d
        By = (Ax[1:, :, :] - Ax[:-1, :, :]) / d - (Az[:, :, 1:] - Az[:, :, :-1]) / d
        Bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / d - (Ax[:, 1:, :] - Ax[:, :-1, :]) / d
        return [Bx, By, Bz]

    Bf = curl(Axf, Ayf, Azf, h)
    # coarse potentials: means of the two fine edges along each coarse edge (coarse vertex = even fine
    # vertex); the coarse grid starts at fine index 0, with G/2 = g coarse ghosts
    Axc = 0.5 * (Axf[::2, ::2, 0::2] + Axf[::2, ::2, 1::2])
    Ayc = 0.5 * (Ayf[::2, 0::2, ::2] + Ayf[::2, 1::2, ::2])
    Azc = 0.5 * (Azf[0::2, ::2, ::2] + Azf[1::2, ::2, ::2])
    Bc = curl(Axc, Ayc, Azc, 2 * h)
    Wc = W.reshape(5, W.shape[1] // 2, 2, W.shape[2] // 2, 2, W.shape[3] // 2, 2)
    Wc = 0.125 * (((Wc[:, :, 0, :, 0, :, 0] + Wc[:, :, 0, :, 0, :, 1]) + (Wc[:, :, 0, :, 1, :, 0] + Wc[:, :, 0, :, 1, :, 1]))
                  + ((Wc[:, :, 1, :, 0, :, 0] + Wc[:, :, 1, :, 0, :, 1]) + (Wc[:, :, 1, :, 1, :, 0] + Wc[:, :, 1, :, 1, :, 1])))
    Mc = M[:, ::2, ::2, ::2]

    def cut(a, lo, n, Goff, stag=(0, 0, 0)):
        s = tuple(slice(lo[ax_] - g + Goff, lo[ax_] + n[ax_] + g + stag[ax_] + Goff) for ax_ in (2, 1, 0))
        return np.ascontiguousarray(a[(Ellipsis,) + s])

    blocks = []
    n = (8, 8, 8)
    gc_off = G // 2                   # coarse global arrays: index 0 is coarse position -g
    blocks.append(BlockInput(n, g, (0.0, 0.0, 0.0), (2 * h,) * 3, cut(Mc, (0, 0, 0), n, gc_off, (1, 1, 1)),
                             cut(Wc, (0, 0, 0), n, gc_off),
                             [cut(Bc[d], (0, 0, 0), n, gc_off, tuple(int(a == d) for a in range(3))) for d in range(3)]))
    records = []
    for k in (0, 1):
        for j in (0, 1):
            lo = (16, 8 * j, 8 * k)
            blocks.append(BlockInput(n, g, (lo[0] * h, lo[1] * h, lo[2] * h), (h,) * 3,
                                     cut(M, lo, n, G, (1, 1, 1)), cut(W, lo, n, G),
                                     [cut(Bf[d], lo, n, G, tuple(int(a == d) for a in range(3))) for d in range(3)]))
            f = len(blocks) - 1
            records.append((0, f, 0, +1, 4 * j, 4 * k))
            records.append((0, f, 0, -1, 4 * j, 4 * k))   # periodic wrap: the fine +x side meets the coarse -x side
    return blocks, records


def two_level_periodic_tables():
    """Ghost-fill tables of two_level_periodic's mesh (coarse block 0, fine blocks 1 + j + 2k):
    the same-level neighbour table (sides toward the other level -1), the restriction maps that fill
    the coarse block's x ghosts from the fine layer (periodic images included), the prolongation maps
    that fill the fine blocks' x ghost slabs from the coarse block, and the level-face records.
    Period: 12 coarse cells along x (8 coarse + 4 under the fine layer), 8 along y and z."""
    from paper_2311_04989_gb300.inputs import neighbour_slot
    fid = lambda j, k: 1 + (j % 2) + 2 * (k % 2)
    nbr = np.full((5, 27), -1, np.int32)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            s = neighbour_slot(0, oy, oz)
            nbr[0, s] = 0
            for k in (0, 1):
                for j in (0, 1):
                    nbr[fid(j, k), s] = fid(j + oy, k + oz)
    pieces = [((-3, 0), 1, -4), ((0, 4), 0, 0), ((4, 8), 1, 4), ((8, 11), 0, 8)]   # (range, fine index, offset)
    rmaps = []
    for (xlo, xhi), offx in (((8, 11), 8), ((-3, 0), -4)):
        for (ylo, yhi), j, offy in pieces:
            for (zlo, zhi), k, offz in pieces:
                rmaps.append((0, fid(j, k), (offx, offy, offz), (xlo, ylo, zlo), (xhi, yhi, zhi)))
    pmaps = []
    for k in (0, 1):
        for j in (0, 1):
            pmaps.append((0, fid(j, k), (8, 4 * j, 4 * k), (-3, -3, -3), (0, 11, 11)))
            pmaps.append((0, fid(j, k), (-4, 4 * j, 4 * k), (8, -3, -3), (11, 11, 11)))
    records = []
    for k in (0, 1):
        for j in (0, 1):
            records.append((0, fid(j, k), 0, +1, 4 * j, 4 * k))
            records.append((0, fid(j, k), 0, -1, 4 * j, 4 * k))
    return nbr, rmaps, pmaps, records
