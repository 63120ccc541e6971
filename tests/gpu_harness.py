"""GPU-side test harness: pack seeded blocks into device pools, run the C-ABI stage, unpack, and
compare with the oracle.  Inputs of both sides come from ``paper_2311_04989_gb300.inputs`` and the
oracle's prim2con; nothing flows from the CUDA path into the oracle."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2311_04989_gb300 import grstage as G
from tests import helpers as H

_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        _ctx = G.gr_context_create(0)
    return _ctx


_eos = {}


def eos_handle(table):
    """gr_eos of an EOS table object (created once per table object and kept alive)."""
    key = id(table)
    if key not in _eos:
        _eos[key] = (table, G.gr_eos_create(ctx(), table))
    return _eos[key][1]


def gr_params_from(P: O.Params, precision=G.GR_PREC_FP64, c2p_guess=G.GR_GUESS_NONE):
    c = P.c()
    p = G.gr_params_default(recon=P.recon, precision=precision, emf=P.emf, ceiling=P.ceiling, c2p_guess=c2p_guess,
                            max_iter=P.max_iter, gamma_ad=P.gamma_ad, rho_atm=P.rho_atm, p_atm=c.p_atm,
                            f_thr=P.f_thr, W_max=P.W_max, M_max=P.M_max, tol=P.tol, weno_eps=P.weno_eps,
                            rk_g0=P.rk_g0, rk_g1=P.rk_g1, rk_beta=P.rk_beta, atm_band=P.atm_band)
    if P.table is not None:
        p.eos = G.GR_EOS_TABLE
        p.table = int(eos_handle(P.table))
        p.T_atm = P.T_atm
        p.Ye_atm = P.Ye_atm
    return p


def mixed_params(P: O.Params) -> O.Params:
    """The parameters of P with the mixed path's atmosphere band (gr_params.atm_band =
    GR_MIXED_ATM_BAND), for the mixed stage and for the oracle run it is compared with."""
    import dataclasses
    return dataclasses.replace(P, atm_band=G.GR_MIXED_ATM_BAND)


class Pools:
    """Device pools of a list of BlockInput-like objects (numpy arrays per block)."""

    def __init__(self, blocks, device="cuda"):
        import torch
        self.torch = torch
        self.blocks = blocks
        self.L = G.Layout.of(blocks)
        self.device = device

    # numpy (per block, padded shape) -> device pool
    def cells(self, per_block, nvar, dtype=np.float64):
        L = self.L
        h = np.zeros((nvar, max(L.ncell, 1)), dtype)
        for b, a in enumerate(per_block):
            a = np.asarray(a).reshape(nvar, -1) if nvar > 1 else np.asarray(a).reshape(1, -1)
            h[:, L.cell_off[b]:L.cell_off[b] + a.shape[1]] = a
        return self.torch.from_numpy(h).to(self.device)

    def faces(self, per_block):
        L = self.L
        out = []
        for d in range(3):
            h = np.zeros(max(L.nface[d], 1))
            for b, B in enumerate(per_block):
                a = np.asarray(B[d]).ravel()
                h[L.face_off[b, d]:L.face_off[b, d] + a.size] = a
            out.append(self.torch.from_numpy(h).to(self.device))
        return out

    def verts(self, per_block):
        L = self.L
        h = np.zeros((16, max(L.nvert, 1)))
        for b, m in enumerate(per_block):
            a = np.asarray(m).reshape(16, -1)
            h[:, L.vert_off[b]:L.vert_off[b] + a.shape[1]] = a
        return self.torch.from_numpy(h).to(self.device)

    # device pool -> numpy per block
    def unpack_cells(self, t, nvar):
        h = t.cpu().numpy()
        out = []
        for b, bi in enumerate(self.blocks):
            N = [bi.n[a] + 2 * bi.ng for a in range(3)]
            sz = N[0] * N[1] * N[2]
            a = h[..., self.L.cell_off[b]:self.L.cell_off[b] + sz]
            out.append(a.reshape((nvar,) + (N[2], N[1], N[0])) if nvar > 1 else a.reshape(N[2], N[1], N[0]))
        return out

    def unpack_faces(self, ts):
        hs = [t.cpu().numpy() for t in ts]
        out = []
        for b, bi in enumerate(self.blocks):
            N = [bi.n[a] + 2 * bi.ng for a in range(3)]
            fb = []
            for d in range(3):
                sh = (N[2] + (d == 2), N[1] + (d == 1), N[0] + (d == 0))
                sz = sh[0] * sh[1] * sh[2]
                fb.append(hs[d][self.L.face_off[b, d]:self.L.face_off[b, d] + sz].reshape(sh))
            out.append(fb)
        return out


def gpu_stage(blocks, P: O.Params, dt, precision=G.GR_PREC_FP64, U=None, U0=None, B0=None, order=None,
              k_zero=True, return_pools=False, c2p_guess=G.GR_GUESS_NONE, shapes=None, autotune=False,
              level_faces=None):
    """Run gr_stage on a batch; returns a list of (Uo, Bo, Wo, status) per block (numpy)."""
    import torch
    order = order or P.interp_order
    if U is None:
        U = [H.cons_from_prims(bi, P, order) for bi in blocks]
    pools = Pools(blocks)
    nq, nw = P.nq, P.nw
    Ud = pools.cells(U, nq)
    U0d = pools.cells(U0 if U0 is not None else U, nq)
    Wd = pools.cells([bi.W for bi in blocks], nw)
    Bd = pools.faces([bi.B for bi in blocks])
    B0d = pools.faces(B0 if B0 is not None else [bi.B for bi in blocks])
    Md = pools.verts([bi.metric for bi in blocks])
    Uo = Ud.clone(); Wo = Wd.clone(); Bo = [b.clone() for b in Bd]
    st = torch.zeros(max(pools.L.ncell, 1), dtype=torch.uint8, device="cuda")
    mesh = G.gr_mesh_create(ctx(), pools.L.descriptors())
    try:
        metric = G.metric_struct(Md, order=order, k_zero=k_zero)
        state = G.state_struct(Ud, U0d, Bd, B0d, Wd, Uo, Bo, Wo, st)
        gp = gr_params_from(P, precision, c2p_guess)
        if shapes is not None:
            G.gr_mesh_set_shapes(mesh, precision, gp.eos, shapes)
        if level_faces:
            G.gr_mesh_set_levels(mesh, faces=level_faces)
        if autotune:
            G.gr_autotune(mesh, metric, state, dt, gp, 1, torch.cuda.current_stream())
        G.gr_stage(mesh, metric, state, dt, gp, torch.cuda.current_stream())
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    Uo_b = pools.unpack_cells(Uo, nq)
    Wo_b = pools.unpack_cells(Wo, nw)
    st_b = pools.unpack_cells(st, 1)
    Bo_b = pools.unpack_faces(Bo)
    out = [dict(U=Uo_b[b], B=Bo_b[b], W=Wo_b[b], status=st_b[b]) for b in range(len(blocks))]
    return (out, pools) if return_pools else out


def oracle_stage(blocks, P: O.Params, dt, U=None, U0=None, B0=None):
    out = []
    for b, bi in enumerate(blocks):
        Ub = U[b] if U is not None else H.cons_from_prims(bi, P, P.interp_order)
        U0b = U0[b] if U0 is not None else Ub
        B0b = B0[b] if B0 is not None else bi.B
        Uo, Bo, Wo, st = O.stage_block(H.to_oracle(bi), Ub, U0b, B0b, dt, P)
        out.append(dict(U=Uo, B=Bo, W=Wo, status=st))
    return out


REL_FLOOR = {"W0": 0.0, "W4": 0.0}   # rho, p: plain relative


def compare(gpu, ref, blocks=None, skip=(), floors=None):
    """Max relative error per variable over interior cells / faces of all blocks, and the number of
    status mismatches.  Denominators:
      D, rho, p           |ref| (plain relative)
      S_j, tau            max(|ref|, D + |tau|): Eq. consB_def forms S_j and tau from terms of the
                          size of the cell's energy density, so rounding differences scale with it
                          (e.g. tau ~ p/(Gamma-1) ~ 1e-30 in the atmosphere is a difference of
                          terms ~ rho ~ 1e-16; S' in a star in equilibrium is a small residual)
      u~^i, B faces       max(|ref|, 1e-3 max|ref| of the block) (they pass through zero)
      D Y_e, Y_e, T       plain relative (table).  Variables named in skip are left out; floors
                          overrides the 1e-3 of a variable (name -> fraction of the block maximum)."""
    errs = {}
    nmis = 0
    for b, (g, r) in enumerate(zip(gpu, ref)):
        n, ng = _geom(g, r, blocks, b)
        for key in ("U", "W"):
            gi = H.interior(g[key], n, ng)
            ri = H.interior(r[key], n, ng)
            if not ri.size:
                continue
            for v in range(ri.shape[0]):
                name = f"{key}{v}"
                if name in skip:
                    continue
                if (key == "U" and v in (0, 5)) or (key == "W" and v >= 5):
                    den = np.maximum(np.abs(ri[v]), 1e-300)
                elif key == "U":
                    den = np.maximum(np.abs(ri[v]), np.abs(ri[0]) + np.abs(ri[4]))
                else:
                    scale = np.max(np.abs(ri[v]))
                    fl = (floors or {}).get(name, REL_FLOOR.get(name, 1e-3))
                    den = np.maximum(np.abs(ri[v]), max(fl * scale, 1e-300))
                e = float(np.max(np.abs(gi[v] - ri[v]) / den))
                errs[name] = max(errs.get(name, 0.0), e)
        for d, (gf, rf) in enumerate(zip(H.interior_faces(g["B"], n, ng), H.interior_faces(r["B"], n, ng))):
            scale = np.max(np.abs(rf)) if rf.size else 0.0
            den = np.maximum(np.abs(rf), max(1e-3 * scale, 1e-300))
            e = float(np.max(np.abs(gf - rf) / den)) if rf.size else 0.0
            errs[f"B{d}"] = max(errs.get(f"B{d}", 0.0), e)
        # the oracle has no bracket proposal; compare the physics bits only
        nmis += int(np.sum((H.interior(g["status"], n, ng) & 0x3F) != H.interior(r["status"], n, ng)))
    errs["status_mismatch"] = nmis
    return errs


def mixed_errors(gpu, ref, blocks):
    """Per-variable error of a mixed-path output against the oracle's, over interior cells / faces of all
    blocks, each in the measure natural to it:
      D, rho, p (and D Y_e, T with a table)   relative |x - x_ref| / |x_ref|
      S_j, tau                                 relative to the cell's energy scale, max(|x_ref|, D + |tau|)
      u~^i (and Y_e)                           absolute (u~ = W v in units of c): they pass through zero, and
                                               the rounding of an FP32 flux moves them by an amount set by
                                               the flux, not by their own size
      B^d                                      |B - B_ref| / max |B_ref| of the block
    and the number of cells whose status (physics bits) differs."""
    names_u = ["D", "S_x", "S_y", "S_z", "tau", "DYe"]
    names_w = ["rho", "u_x", "u_y", "u_z", "p", "Ye", "T"]
    errs = {}
    nmis = 0
    for b, (g, r) in enumerate(zip(gpu, ref)):
        n, ng = _geom(g, r, blocks, b)
        gu, ru = H.interior(g["U"], n, ng), H.interior(r["U"], n, ng)
        gw, rw = H.interior(g["W"], n, ng), H.interior(r["W"], n, ng)
        if not ru.size:
            continue
        for v in range(ru.shape[0]):
            if v in (0, 5):
                den = np.maximum(np.abs(ru[v]), 1e-300)
            else:
                den = np.maximum(np.abs(ru[v]), np.abs(ru[0]) + np.abs(ru[4]))
            errs[names_u[v]] = max(errs.get(names_u[v], 0.0), float(np.max(np.abs(gu[v] - ru[v]) / den)))
        for v in range(rw.shape[0]):
            d = np.abs(gw[v] - rw[v])
            e = float(np.max(d)) if v in (1, 2, 3, 5) else float(np.max(d / np.maximum(np.abs(rw[v]), 1e-300)))
            errs[names_w[v]] = max(errs.get(names_w[v], 0.0), e)
        for d, (gf, rf) in enumerate(zip(H.interior_faces(g["B"], n, ng), H.interior_faces(r["B"], n, ng))):
            scale = max(float(np.max(np.abs(rf))), 1e-300) if rf.size else 1.0
            e = float(np.max(np.abs(gf - rf))) / scale if rf.size else 0.0
            errs[f"B_{'xyz'[d]}"] = max(errs.get(f"B_{'xyz'[d]}", 0.0), e)
        nmis += int(np.sum((H.interior(g["status"], n, ng) & 0x3F) != H.interior(r["status"], n, ng)))
    errs["status_mismatch"] = nmis
    return errs


# Bounds of the mixed path (FP32 reconstruction, HLLE and EMFs; FP64 accumulation, CT and con2prim)
# against the FP64 oracle at the same atmosphere band, in mixed_errors()'s measures, per kind of
# workload.  rho and D carry the stated 1e-6; the others sit a few times above what the GPU measured
# (every test prints its numbers).  An FP32 flux carries a relative rounding of ~1e-7 of its largest
# terms, which reaches the conserved variables scaled by dt/dx, the pressure through con2prim's
# conditioning (cold gas, where p is a small part of the energy, magnifies it), and the velocities as an
# absolute amount.  Static stars add one more effect: the corner EMF takes its upwind correction from the
# side the face mass flux points to, and in a star in equilibrium that flux is rounding noise, whose sign
# differs between FP32 and FP64 fluxes; the two choices differ by the correction itself, so B' there
# agrees to the size of the upwind correction (a truncation-level amount, ~1e-4 of max |B|), not to
# rounding (test_single_64cubed_star_fp64_and_mixed shows the plain-mean EMF, which has no switch,
# agreeing to rounding).
_M = dict(D=1e-6, rho=1e-6, S_x=2e-7, S_y=2e-7, S_z=2e-7, tau=3e-7)
MIXED_BOUNDS = {
    # measured (GB300): u~ <= 3.4e-8, p <= 5.3e-6, B <= 3.3e-8, S <= 3.4e-8, tau <= 4.4e-8
    "random": dict(_M, u_x=1e-7, u_y=1e-7, u_z=1e-7, p=2e-5, B_x=1e-7, B_y=1e-7, B_z=1e-7),
    # one RK3 step: u~ <= 1.8e-8, p <= 2.1e-6, B <= 1.6e-8
    "driver": dict(_M, u_x=1e-7, u_y=1e-7, u_z=1e-7, p=1e-5, B_x=1e-7, B_y=1e-7, B_z=1e-7),
    # u~ <= 6.4e-8, p <= 1.2e-5, T <= 1.0e-5, Y_e <= 3.6e-8, D Y_e <= 2.7e-7, S <= 7.2e-8, tau <= 9.5e-8
    "table": dict(_M, DYe=1e-6, u_x=2e-7, u_y=2e-7, u_z=2e-7, p=5e-5, Ye=1e-7, T=5e-5, B_x=1e-7, B_y=1e-7,
                  B_z=1e-7),
    # stars in equilibrium: p <= 9.1e-4 (cold outer layers), B <= 5.2e-4 (EMF upwind switch), u~ <= 9.1e-9
    "star": dict(_M, u_x=1e-7, u_y=1e-7, u_z=1e-7, p=3e-3, B_x=2e-3, B_y=2e-3, B_z=2e-3),
    # PPM's limiter can take the other branch where two candidates agree to FP32 rounding (star surface):
    # rho <= 5.2e-6, p <= 1.8e-4, B <= 3.4e-4, u~ <= 4.1e-8
    "star_ppm": dict(_M, D=2e-5, rho=2e-5, u_x=2e-7, u_y=2e-7, u_z=2e-7, p=1e-3, B_x=1e-3, B_y=1e-3, B_z=1e-3),
}


def check_mixed(out, ref, blocks, bounds, label=""):
    """Mixed-path output against the oracle's: statuses equal (physics bits), and every variable named
    in bounds within its bound (mixed_errors()'s measures).  Prints the per-variable errors; returns
    them."""
    e = mixed_errors(out, ref, blocks)
    mis = e.pop("status_mismatch")
    print(f"{label}: " + ", ".join(f"{k} {v:.1e}" for k, v in e.items()) + f"; status mismatches {mis}")
    assert mis == 0, (label, mis)
    bad = {k: (e[k], b) for k, b in bounds.items() if k in e and not e[k] < b}
    assert not bad, (label, bad)
    return e


def _geom(g, r, blocks, b):
    if blocks is not None:
        return blocks[b].n, blocks[b].ng
    # infer from shapes: status (Nz,Ny,Nx); assume ng = 3
    Nz, Ny, Nx = r["status"].shape
    return (Nx - 6, Ny - 6, Nz - 6), 3


def backward_error(out, bi, P: O.Params, order=2):
    """How well the primitives of a stage output solve its own conserved variables: max over the
    interior cells of a regular solve (status 0; cells under a floor, clamp or the atmosphere are set by
    closed-form policies and compared forward) of |prim2con(W', cell field of B') - U'| (the oracle's
    prim2con and cell metric), with the
    conserved-variable denominators of compare().  Recovering the primitives from the conserved
    variables is ill-conditioned where the pressure is a small part of the energy (cold, low-density
    gas) or a velocity passes through zero, so two FP64 implementations whose conserved variables agree
    to rounding can differ there by far more in W; the backward error is the well-conditioned check."""
    n, g = bi.n, bi.ng
    cm = H.cell_metric(bi, order)[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 16)
    Bx, By, Bz = out["B"]
    cb = np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]), 0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                   0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], axis=-1)[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 3)
    w = H.interior(out["W"], n, g).reshape(out["W"].shape[0], -1).T
    u = H.interior(out["U"], n, g).reshape(out["U"].shape[0], -1).T
    ok = H.interior(out["status"], n, g).ravel() == 0
    if not ok.any():
        return 0.0
    q = O.prim2con(cm[ok], w[ok, :P.nw], cb[ok], P)
    u = u[ok]
    err = 0.0
    for v in range(q.shape[1]):
        den = np.abs(u[:, 0]) if v in (0, 5) else np.maximum(np.abs(u[:, v]), np.abs(u[:, 0]) + np.abs(u[:, 4]))
        err = max(err, float(np.max(np.abs(q[:, v] - u[:, v]) / np.maximum(den, 1e-300))))
    return err


def policy_cells_error(got, ref, bi):
    """Largest relative difference of the primitives on interior cells that a floor, clamp or the
    atmosphere set (status != 0 in the reference), denominator max(|ref|, 1e-300)."""
    n, g = bi.n, bi.ng
    m = H.interior(ref["status"], n, g) != 0
    if not m.any():
        return 0.0
    gw, rw = H.interior(got["W"], n, g), H.interior(ref["W"], n, g)
    return float(max(np.max(np.abs(gw[v][m] - rw[v][m]) / np.maximum(np.abs(rw[v][m]), 1e-300))
                     for v in range(rw.shape[0])))
