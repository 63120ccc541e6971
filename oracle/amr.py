"""Level-boundary operators of a refined mesh (Sec. 3.3, last paragraph: divergence- and
curl-preserving restriction and prolongation of the face field, and the flux and electric-field
corrections at refinement boundaries).

TEST INFRASTRUCTURE ONLY (part of the oracle: only tests/, smoke() and bench.py's CPU legs use it).
Plain numpy loops over small regions.  Arrays are ghost-padded block arrays: cell (i, j, k) of a block
with ghost width g at index [..., k + g, j + g, i + g]; the d-face array has one more point along d;
vertices (edges) one more along every axis.  A fine block's cell i along an axis covers half of coarse
cell off + floor(i / 2) (refinement ratio 2).

Readings (the paper cites the operators without formulas):
* restriction: a coarse cell value is the mean of its 8 fine cells (the conserved variables are
  densitised, so this conserves them); a coarse face value is the mean of the 4 fine faces on it (the
  same flux through the face, so a divergence-free fine field restricts to a divergence-free one)
* cell prolongation: limited linear, u_fine = u_c + (s_x dx + s_y dy + s_z dz) / 4 with s_d = +-1 the
  side of the fine cell and dx.. the minmod of the two one-sided differences of the coarse neighbours;
  the 8 fine cells average to u_c
* face prolongation: a fine face lying on a coarse face takes the coarse value plus the limited
  transverse slopes of the coarse face plane (the 4 average to the coarse face); the 12 fine faces
  inside a coarse cell are the mean of the two opposite outer fine faces plus the minimal-norm
  correction that makes all 8 fine cells divergence-free (solved in fluxes: value x face area)
* flux correction: a coarse face on a level boundary takes the mean of the 4 fine-face fluxes on it
* EMF correction: a coarse edge on a level boundary takes the mean of the 2 fine edge EMFs along it
"""
from __future__ import annotations

import numpy as np

import oracle as O


def _minmod(a, b):
    return 0.0 if a * b <= 0.0 else (a if abs(a) < abs(b) else b)


def _fdiv(i):
    """coarse index and side (-1 low half, +1 high half) of fine index i (floor division by 2)"""
    c = i // 2
    return c, (1 if i - 2 * c else -1)


# ---------------------------------------------------------------------------------------------
# restriction
# ---------------------------------------------------------------------------------------------
def restrict_cells(fine, gf, coarse, gc, off, lo, hi):
    """coarse[..., cells lo..hi-1 (coarse indices)] = mean of the 8 fine cells each covers.
    fine/coarse: (nvar, Nz, Ny, Nx) arrays."""
    for k in range(lo[2], hi[2]):
        for j in range(lo[1], hi[1]):
            for i in range(lo[0], hi[0]):
                fi, fj, fk = 2 * (i - off[0]), 2 * (j - off[1]), 2 * (k - off[2])
                s = 0.0
                for dk in (0, 1):
                    for dj in (0, 1):
                        for di in (0, 1):
                            s = s + fine[..., fk + dk + gf, fj + dj + gf, fi + di + gf]
                coarse[..., k + gc, j + gc, i + gc] = 0.125 * s


def _ghost_plane(lo, hi, n, d, p):
    """A range wholly outside the destination block along d leaves the block's own d-face planes."""
    return n is not None and (hi[d] <= 0 or lo[d] >= n[d]) and p[d] in (0, n[d])


def restrict_faces(fineB, gf, coarseB, gc, off, lo, hi, nc=None):
    """Coarse d-faces with index lo..hi-1 (hi along d inclusive of the last face: hi[d] + 1) = mean of
    the 4 fine d-faces on each.  nc: the coarse block size (ghost-slab rule of _ghost_plane)."""
    for d in range(3):
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        hid = list(hi)
        hid[d] += 1
        for k in range(lo[2], hid[2]):
            for j in range(lo[1], hid[1]):
                for i in range(lo[0], hid[0]):
                    c = (i, j, k)
                    if _ghost_plane(lo, hi, nc, d, c):
                        continue
                    f0 = [2 * (c[a] - off[a]) for a in range(3)]
                    s = 0.0
                    for u in (0, 1):
                        for v in (0, 1):
                            f = list(f0)
                            f[t1] += u
                            f[t2] += v
                            s = s + fineB[d][f[2] + gf, f[1] + gf, f[0] + gf]
                    coarseB[d][k + gc, j + gc, i + gc] = 0.25 * s


# ---------------------------------------------------------------------------------------------
# prolongation
# ---------------------------------------------------------------------------------------------
def prolong_cells(coarse, gc, fine, gf, off, lo, hi):
    """fine[..., cells lo..hi-1 (fine indices)] from the limited linear reconstruction of the coarse
    cells (each coarse cell used needs its 6 face neighbours in the coarse array)."""
    nvar = coarse.shape[0]
    for k in range(lo[2], hi[2]):
        for j in range(lo[1], hi[1]):
            for i in range(lo[0], hi[0]):
                (ci, si), (cj, sj), (ck, sk) = _fdiv(i), _fdiv(j), _fdiv(k)
                c = (ci + off[0], cj + off[1], ck + off[2])
                sides = (si, sj, sk)
                for v in range(nvar):
                    u0 = coarse[v, c[2] + gc, c[1] + gc, c[0] + gc]
                    val = u0
                    for a in range(3):
                        lo_c, hi_c = list(c), list(c)
                        lo_c[a] -= 1
                        hi_c[a] += 1
                        um = coarse[v, lo_c[2] + gc, lo_c[1] + gc, lo_c[0] + gc]
                        up = coarse[v, hi_c[2] + gc, hi_c[1] + gc, hi_c[0] + gc]
                        val = val + 0.25 * sides[a] * _minmod(up - u0, u0 - um)
                    fine[v, k + gf, j + gf, i + gf] = val


def _outer_face(coarseB, gc, d, cf):
    """Values of the 4 fine d-faces on coarse d-face cf (coarse indices, cf[d] = the face's plane),
    as a dict {(s1, s2): value} over the transverse sides s1 (along t1), s2 (along t2)."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    B = coarseB[d]
    at = lambda p: B[p[2] + gc, p[1] + gc, p[0] + gc]
    b0 = at(cf)
    slopes = []
    for t in (t1, t2):
        m, p = list(cf), list(cf)
        m[t] -= 1
        p[t] += 1
        slopes.append(_minmod(at(p) - b0, b0 - at(m)))
    return {(s1, s2): b0 + 0.25 * s1 * slopes[0] + 0.25 * s2 * slopes[1] for s1 in (-1, 1) for s2 in (-1, 1)}


def prolong_cell_faces(coarseB, gc, c, dxf):
    """The 36 fine faces of coarse cell c: {(d, a, b, cc): value} with (a, b, cc) the fine face's
    position in the cell: along d one of -1 (low outer), 0 (interior), +1 (high outer); across d the
    side -1/+1.  dxf: fine spacings (face areas for the divergence-free solve)."""
    area = (dxf[1] * dxf[2], dxf[0] * dxf[2], dxf[0] * dxf[1])
    val = {}
    for d in range(3):
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        for side in (-1, 1):
            cf = list(c)
            cf[d] += 1 if side > 0 else 0
            for (s1, s2), v in _outer_face(coarseB, gc, d, cf).items():
                pos = [0, 0, 0]
                pos[d], pos[t1], pos[t2] = side, s1, s2
                val[(d,) + tuple(pos)] = v
    # fluxes (value x area) of the outer faces; D_d at the transverse position of a fine face
    phi = {k: v * area[k[0]] for k, v in val.items()}

    def D(d, pos):   # high outer minus low outer flux at transverse position pos (pos[d] ignored)
        hp, lp = list(pos), list(pos)
        hp[d], lp[d] = 1, -1
        return phi[(d,) + tuple(hp)] - phi[(d,) + tuple(lp)]

    # R_abc = (Dx(b,c) + Dy(a,c) + Dz(a,b)) / 2 for the fine cell at sides (a, b, c)
    R = {}
    for a in (-1, 1):
        for b in (-1, 1):
            for cc in (-1, 1):
                p = [a, b, cc]
                R[(a, b, cc)] = 0.5 * (D(0, p) + D(1, p) + D(2, p))
    mono = {"a": lambda a, b, c: a, "b": lambda a, b, c: b, "c": lambda a, b, c: c,
            "ab": lambda a, b, c: a * b, "ac": lambda a, b, c: a * c, "bc": lambda a, b, c: b * c,
            "abc": lambda a, b, c: a * b * c}
    r = {m: sum(R[k] * f(*k) for k in R) / 8.0 for m, f in mono.items()}
    # interior corrections (minimal-norm split of the shared monomials)
    for (b, cc) in ((-1, -1), (-1, 1), (1, -1), (1, 1)):
        X = r["a"] + 0.5 * r["ab"] * b + 0.5 * r["ac"] * cc + r["abc"] / 3.0 * b * cc
        phi[(0, 0, b, cc)] = 0.5 * (phi[(0, -1, b, cc)] + phi[(0, 1, b, cc)]) + X
    for (a, cc) in ((-1, -1), (-1, 1), (1, -1), (1, 1)):
        Y = r["b"] + 0.5 * r["ab"] * a + 0.5 * r["bc"] * cc + r["abc"] / 3.0 * a * cc
        phi[(1, a, 0, cc)] = 0.5 * (phi[(1, a, -1, cc)] + phi[(1, a, 1, cc)]) + Y
    for (a, b) in ((-1, -1), (-1, 1), (1, -1), (1, 1)):
        Z = r["c"] + 0.5 * r["ac"] * a + 0.5 * r["bc"] * b + r["abc"] / 3.0 * a * b
        phi[(2, a, b, 0)] = 0.5 * (phi[(2, a, b, -1)] + phi[(2, a, b, 1)]) + Z
    return {k: v / area[k[0]] for k, v in phi.items()}


def prolong_faces(coarseB, gc, fineB, gf, off, lo, hi, dxf, nf=None):
    """Fine d-faces of fine cells lo..hi-1 (fine indices; the high face of the last cell along d
    included) from the divergence-preserving prolongation of the coarse faces.  A fine face on a
    coarse face plane (even index along d) depends on that coarse plane only; a fine face inside a
    coarse cell (odd index) on all six faces of the cell.  nf: the fine block size (ghost-slab rule
    of _ghost_plane)."""
    cache = {}
    for d in range(3):
        t1, t2 = (d + 1) % 3, (d + 2) % 3
        hid = list(hi)
        hid[d] += 1
        for k in range(lo[2], hid[2]):
            for j in range(lo[1], hid[1]):
                for i in range(lo[0], hid[0]):
                    f = (i, j, k)
                    if _ghost_plane(lo, hi, nf, d, f):
                        continue
                    if f[d] % 2 == 0:
                        cf = [0, 0, 0]
                        cf[d] = f[d] // 2 + off[d]
                        c1, s1 = _fdiv(f[t1])
                        c2, s2 = _fdiv(f[t2])
                        cf[t1], cf[t2] = c1 + off[t1], c2 + off[t2]
                        val = _outer_face(coarseB, gc, d, cf)[(s1, s2)]
                    else:
                        c, pos = [0, 0, 0], [0, 0, 0]
                        for a in range(3):
                            if a == d:
                                c[a], pos[a] = f[a] // 2 + off[a], 0
                            else:
                                ca, pos[a] = _fdiv(f[a])
                                c[a] = ca + off[a]
                        key = tuple(c)
                        if key not in cache:
                            cache[key] = prolong_cell_faces(coarseB, gc, key, dxf)
                        val = cache[key][(d,) + tuple(pos)]
                    fineB[d][k + gf, j + gf, i + gf] = val


# ---------------------------------------------------------------------------------------------
# flux and EMF corrections at a level boundary
# ---------------------------------------------------------------------------------------------
def correct_level_face(Fc, Ec, nc, gc, Ff, Ef, nf, gf, d, side, o1, o2):
    """Replace the coarse block's fluxes Fc[d] and EMFs Ec on the patch of its side-`side` d-face that a
    fine block covers (coarse transverse cells o1.. along t1, o2.. along t2) by the restricted fine
    values.  nc, nf: coarse and fine block sizes.  Fc/Ff, Ec/Ef as returned by oracle.stage_fluxes."""
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    nc1, nc2 = nf[t1] // 2, nf[t2] // 2

    def cidx(pd, p1, p2, arr_g):
        p = [0, 0, 0]
        p[d], p[t1], p[t2] = pd, p1, p2
        return p[2] + arr_g, p[1] + arr_g, p[0] + arr_g

    nqv = Fc[d].shape[0]
    # plane index along d: coarse n_d (side +1) or 0; fine 0 (side +1) or n_f[d]
    pc = nc[d] if side > 0 else 0
    pf = 0 if side > 0 else nf[d]
    for J in range(o1, o1 + nc1):
        for K in range(o2, o2 + nc2):
            for v in range(nqv):
                s = 0.0
                for u in (0, 1):
                    for w in (0, 1):
                        s = s + Ff[d][(v,) + cidx(pf, 2 * (J - o1) + u, 2 * (K - o2) + w, gf)]
                Fc[d][(v,) + cidx(pc, J, K, gc)] = 0.25 * s
    # edges on the plane: E_t1 (along t1) at cells J along t1, vertices K along t2; E_t2 likewise
    for J in range(o1, o1 + nc1):
        for K in range(o2, o2 + nc2 + 1):
            fa = Ef[t1][cidx(pf, 2 * (J - o1), 2 * (K - o2), gf)]
            fb = Ef[t1][cidx(pf, 2 * (J - o1) + 1, 2 * (K - o2), gf)]
            Ec[t1][cidx(pc, J, K, gc)] = 0.5 * (fa + fb)
    for J in range(o1, o1 + nc1 + 1):
        for K in range(o2, o2 + nc2):
            fa = Ef[t2][cidx(pf, 2 * (J - o1), 2 * (K - o2), gf)]
            fb = Ef[t2][cidx(pf, 2 * (J - o1), 2 * (K - o2) + 1, gf)]
            Ec[t2][cidx(pc, J, K, gc)] = 0.5 * (fa + fb)


def two_level_stage(blocks, U, records, P: O.Params, dt, correct=True, U0=None, B0=None):
    """One stage of every block of a two-level mesh with the level-boundary corrections.
    records: (coarse, fine, d, side, o1, o2) per fine block touching a coarse block's face; U0, B0:
    the RK registers (default: the stage input).  Returns [(U', B', W', status)] per block."""
    U0 = U0 if U0 is not None else U
    B0 = B0 if B0 is not None else [bi.B for bi in blocks]
    F, E = [], []
    for b, bi in enumerate(blocks):
        f, e = O.stage_fluxes(O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B), U[b], U0[b], B0[b], dt, P)
        F.append(f)
        E.append(e)
    if correct:
        for (c, f, d, side, o1, o2) in records:
            correct_level_face(F[c], E[c], blocks[c].n, blocks[c].ng, F[f], E[f], blocks[f].n, blocks[f].ng, d, side,
                               o1, o2)
    out = []
    for b, bi in enumerate(blocks):
        out.append(O.stage_block_with(O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B), U[b], U0[b], B0[b], dt, P,
                                      F[b], E[b]))
    return out


def fill_two_level(blocks, nbr, restrict_maps, prolong_maps):
    """Ghosts of a two-level mesh: same-level copies (neighbour table; sides toward the other level
    are -1), then the restriction maps, then the prolongation maps (primitives and B).
    maps: (coarse, fine, off, lo, hi)."""
    from oracle import driver as DR
    n, g = blocks[0].n, blocks[0].ng
    DR.ghost_fill([b.W for b in blocks], [b.B for b in blocks], nbr, n, g)
    for (c, f, off, lo, hi) in restrict_maps:
        cb, fb = blocks[c], blocks[f]
        restrict_cells(fb.W, fb.ng, cb.W, cb.ng, off, lo, hi)
        restrict_faces(fb.B, fb.ng, cb.B, cb.ng, off, lo, hi, nc=cb.n)
    for (c, f, off, lo, hi) in prolong_maps:
        cb, fb = blocks[c], blocks[f]
        prolong_cells(cb.W, cb.ng, fb.W, fb.ng, off, lo, hi)
        prolong_faces(cb.B, cb.ng, fb.B, fb.ng, off, lo, hi, fb.dx, nf=fb.n)


def two_level_rk_step(blocks, U, nbr, restrict_maps, prolong_maps, records, P: O.Params, cfl, order=3):
    """One RK step of a two-level mesh (ghost fill of fill_two_level before every stage, the grid time
    step of the finest spacing, SSP-RK stages with the level-boundary corrections), in place of the
    blocks' W, B and U.  Returns dt."""
    from oracle import driver as DR
    fill_two_level(blocks, nbr, restrict_maps, prolong_maps)
    dt = DR.grid_dt(blocks, cfl)
    U0 = [u.copy() for u in U]
    B0 = [[f.copy() for f in b.B] for b in blocks]
    for s_i, (g0, g1, beta) in enumerate(DR.RK_STAGES[order]):
        if s_i > 0:
            fill_two_level(blocks, nbr, restrict_maps, prolong_maps)
        Pst = O.Params(**{**P.__dict__, "rk_g0": g0, "rk_g1": g1, "rk_beta": beta})
        out = two_level_stage(blocks, U, records, Pst, dt, U0=U0, B0=B0)
        for b, (Uo, Bo, Wo, st) in enumerate(out):
            U[b][...] = Uo
            blocks[b].W[...] = Wo
            for d in range(3):
                blocks[b].B[d][...] = Bo[d]
    return dt
