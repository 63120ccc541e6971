"""One Runge-Kutta step of a set of same-level MeshBlocks: ghost exchange, time step, stages.

The third-order Runge-Kutta integrator is the one stated at the start of Sec. 4 for every test of the
paper; the global time step is the CFL factor times the finest grid spacing (Sec. 3.1); each stage is
the method-of-lines update of Sec. 3.2-3.5.

TEST INFRASTRUCTURE ONLY (part of the oracle: only tests/, smoke() and bench.py's CPU legs use it).
Plain numpy around the oracle's stage: every ghost cell and ghost face is copied from the block the
neighbour table names (or, at an outflow boundary, from the nearest interior element of the same
block); dt is either CFL min dx over the blocks (dt_mode "grid", Sec. 3.1) or CFL min over interior
cells and directions of dx_d / max |lambda_d| (dt_mode "signal"); the stages are the Shu-Osher forms
of SSP-RK2 and SSP-RK3.
"""
from __future__ import annotations

import numpy as np

import oracle as O

# (g0, g1, beta) of U' = g0 U^n + g1 U + beta dt L(U), per stage
RK_STAGES = {2: [(0.0, 1.0, 1.0), (0.5, 0.5, 0.5)],
             3: [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)]}


def _slot(ox, oy, oz):
    return (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)


def _side(i, n):
    return -1 if i < 0 else (1 if i >= n else 0)


def ghost_fill(W, B, nbr, n, g):
    """W: list of (nw, Nz, Ny, Nx) cell arrays, B: list of [Bx, By, Bz] face arrays (all blocks with the
    same n and g); fills every ghost cell and ghost face in place."""
    N = [v + 2 * g for v in n]
    W0 = [w.copy() for w in W]
    B0 = [[f.copy() for f in bb] for bb in B]
    for b in range(len(W)):
        # cells
        for k in range(-g, n[2] + g):
            for j in range(-g, n[1] + g):
                for i in range(-g, n[0] + g):
                    o = (_side(i, n[0]), _side(j, n[1]), _side(k, n[2]))
                    if o == (0, 0, 0):
                        continue
                    src = nbr[b, _slot(*o)]
                    if src >= 0:
                        si, sj, sk, sb = i - o[0] * n[0], j - o[1] * n[1], k - o[2] * n[2], src
                    else:   # outflow: nearest interior cell of this block
                        si, sj, sk, sb = min(max(i, 0), n[0] - 1), min(max(j, 0), n[1] - 1), min(max(k, 0), n[2] - 1), b
                    W[b][:, k + g, j + g, i + g] = W0[sb][:, sk + g, sj + g, si + g]
        # faces: the d-face array has n_d + 1 owned faces (0..n_d) along d
        for d in range(3):
            nd = [n[0] + (d == 0), n[1] + (d == 1), n[2] + (d == 2)]
            for k in range(-g, nd[2] + g - (d == 2) * 0):
                if k + g >= N[2] + (d == 2):
                    continue
                for j in range(-g, nd[1] + g):
                    if j + g >= N[1] + (d == 1):
                        continue
                    for i in range(-g, nd[0] + g):
                        if i + g >= N[0] + (d == 0):
                            continue
                        o = (_side(i, nd[0]), _side(j, nd[1]), _side(k, nd[2]))
                        if o == (0, 0, 0):
                            continue
                        src = nbr[b, _slot(*o)]
                        if src >= 0:
                            si, sj, sk, sb = i - o[0] * n[0], j - o[1] * n[1], k - o[2] * n[2], src
                        else:
                            si = min(max(i, 0), nd[0] - 1); sj = min(max(j, 0), nd[1] - 1)
                            sk = min(max(k, 0), nd[2] - 1); sb = b
                        B[b][d][k + g, j + g, i + g] = B0[sb][d][sk + g, sj + g, si + g]
    return W, B


def cfl_dt(blocks, W, B, P: O.Params, cfl):
    """dt = cfl * min over interior cells and directions of dx_d / max(|lambda-_d|, |lambda+_d|), the
    fast speeds of Sec. 2.2 at the cell state (cell field = mean of the two densitised faces)."""
    rate = 0.0
    for b, bi in enumerate(blocks):
        n, g = bi.n, bi.ng
        blk = O.Block(n, g, bi.dx, bi.metric, W[b], B[b])
        cm, _ = O.interp_cells(blk, P.interp_order, 0, tuple(n))
        w = W[b][:, g:g + n[2], g:g + n[1], g:g + n[0]].reshape(W[b].shape[0], -1).T
        Bx, By, Bz = B[b]
        Bc = np.stack([0.5 * (Bx[g:g + n[2], g:g + n[1], g:g + n[0]] + Bx[g:g + n[2], g:g + n[1], g + 1:g + n[0] + 1]),
                       0.5 * (By[g:g + n[2], g:g + n[1], g:g + n[0]] + By[g:g + n[2], g + 1:g + n[1] + 1, g:g + n[0]]),
                       0.5 * (Bz[g:g + n[2], g:g + n[1], g:g + n[0]] + Bz[g + 1:g + n[2] + 1, g:g + n[1], g:g + n[0]])],
                      -1).reshape(-1, 3)
        for d in range(3):
            _, _, lam = O.flux_points(d, cm, w, Bc, P)
            rate = max(rate, float(np.max(np.abs(lam))) / bi.dx[d])
    return cfl / rate


def grid_dt(blocks, cfl):
    """dt = cfl * the finest grid spacing over the blocks (Sec. 3.1)."""
    return cfl * min(min(bi.dx) for bi in blocks)


def rk_step(blocks, U, nbr, P: O.Params, cfl, order=3, dt_mode="signal"):
    """One RK step in place of the blocks' W, B and the conserved U (list of (nq, Nz, Ny, Nx)).
    Returns (dt, statuses of the last stage)."""
    n, g = blocks[0].n, blocks[0].ng
    W = [bi.W for bi in blocks]
    Bf = [bi.B for bi in blocks]
    ghost_fill(W, Bf, nbr, n, g)
    dt = cfl_dt(blocks, W, Bf, P, cfl) if dt_mode == "signal" else grid_dt(blocks, cfl)
    U0 = [u.copy() for u in U]
    B0 = [[f.copy() for f in bb] for bb in Bf]
    st = None
    for s_i, (g0, g1, beta) in enumerate(RK_STAGES[order]):
        if s_i > 0:
            ghost_fill(W, Bf, nbr, n, g)
        Pst = O.Params(**{**P.__dict__, "rk_g0": g0, "rk_g1": g1, "rk_beta": beta})
        st = []
        for b, bi in enumerate(blocks):
            blk = O.Block(n, g, bi.dx, bi.metric, W[b], Bf[b])
            Uo, Bo, Wo, s = O.stage_block(blk, U[b], U0[b], B0[b], dt, Pst)
            U[b][...] = Uo
            W[b][...] = Wo
            for d in range(3):
                Bf[b][d][...] = Bo[d]
            st.append(s)
    return dt, st
