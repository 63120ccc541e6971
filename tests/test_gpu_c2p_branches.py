"""Every branch of the conservative-to-primitive step (Sec. 3.5, App. A) on the GPU against the oracle,
cell by cell: one block whose x-columns are set to the degenerate cases of the method -- a Lorentz factor
above the ceiling (clamped, and reset to the atmosphere with the other ceiling rule), tau below the cold
static value (floor), B^2/D above M_max (D rescaled), a non-finite conserved variable (failure), D below
the atmosphere threshold, D at the threshold itself (the knife edge the band decides), a cell with no
field -- beside ordinary cells.  Statuses must be identical, the primitives and the conserved variables
that the floors rewrite within 1e-12 (FP64 path; gr_con2prim), with and without the FP32 bracket
proposal."""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from tests import gpu_harness as GH
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


def branch_block(P):
    """(block, conserved U (5, Nz, Ny, Nx)) with the degenerate cases along x (columns 0..8)."""
    bi = I.random_block(n=(10, 6, 6), g=3, seed=140, metric_amp=0.03, rho_range=(1e-6, 1e-3), u_max=0.4)
    g = bi.ng
    # column 0: u~^x = 30 (W above W_max = sqrt(1 + 20^2))
    bi.W[1][:, :, g + 0] = 30.0
    # column 8: no field (all faces of its cells zero)
    bi.B[0][:, :, g + 8:g + 10] = 0.0
    bi.B[1][:, :, g + 8] = 0.0
    bi.B[2][:, :, g + 8] = 0.0
    U = H.cons_from_prims(bi, P)
    cm, cb = H.cell_metric(bi), H.cell_B(bi)
    sg = np.sqrt(np.linalg.det(np.stack([np.stack([cm[..., 4], cm[..., 5], cm[..., 6]], -1),
                                         np.stack([cm[..., 5], cm[..., 7], cm[..., 8]], -1),
                                         np.stack([cm[..., 6], cm[..., 8], cm[..., 9]], -1)], -2)))
    gam = cm[..., 4:10]
    Bu = cb / sg[..., None]
    BB = (gam[..., 0] * Bu[..., 0] ** 2 + gam[..., 3] * Bu[..., 1] ** 2 + gam[..., 5] * Bu[..., 2] ** 2
          + 2 * (gam[..., 1] * Bu[..., 0] * Bu[..., 1] + gam[..., 2] * Bu[..., 0] * Bu[..., 2]
                 + gam[..., 4] * Bu[..., 1] * Bu[..., 2]))
    c = (slice(None), slice(None))
    # column 1: tau below the cold static value B^2 / 2 (densitised): tau = 0.1 of it
    U[4][c + (slice(g + 1, g + 2),)] = 0.1 * 0.5 * (BB * sg)[c + (slice(g + 1, g + 2),)]
    # column 2: B^2 / D above M_max: D = B^2 / (10 M_max) (densitised)
    U[0][c + (slice(g + 2, g + 3),)] = ((BB / (10.0 * P.M_max)) * sg)[c + (slice(g + 2, g + 3),)]
    # column 3: a non-finite momentum
    U[2][c + (slice(g + 3, g + 4),)] = np.nan
    # column 4: D below the atmosphere threshold
    U[0][c + (slice(g + 4, g + 5),)] = (0.5 * P.f_thr * P.rho_atm * sg)[c + (slice(g + 4, g + 5),)]
    # column 5: D exactly at the threshold (reset within the band)
    U[0][c + (slice(g + 5, g + 6),)] = (P.f_thr * P.rho_atm * sg)[c + (slice(g + 5, g + 6),)]
    return bi, U, cm, cb


@pytest.mark.parametrize("ceiling", [0, 1])
@pytest.mark.parametrize("guess", [G.GR_GUESS_NONE, G.GR_GUESS_FP32])
def test_every_con2prim_branch_matches_the_oracle(ceiling, guess):
    import torch
    P = O.Params(gamma_ad=2.0, rho_atm=1e-9, tol=1e-14, M_max=10.0, ceiling=ceiling)
    bi, U, cm, cb = branch_block(P)
    n, g = bi.n, bi.ng
    pools = GH.Pools([bi])
    Ud = pools.cells([U], 5)
    Bd, Md = pools.faces([bi.B]), pools.verts([bi.metric])
    Wd = torch.zeros((5, Ud.shape[1]), dtype=torch.float64, device="cuda")
    st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        G.gr_con2prim(mesh, G.metric_struct(Md), list(Ud), Bd, list(Wd), st, GH.gr_params_from(P, c2p_guess=guess))
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    Ug = H.interior(pools.unpack_cells(Ud, 5)[0], n, g)
    Wg = H.interior(pools.unpack_cells(Wd, 5)[0], n, g)
    Sg = H.interior(pools.unpack_cells(st, 1)[0], n, g) & 0x3F
    # the oracle on every interior cell
    met = cm[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 16)
    bd = cb[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 3)
    q = np.moveaxis(H.interior(U, n, g), 0, -1).reshape(-1, 5)
    w_ref, q_ref, st_ref, _ = O.con2prim(met, q, bd, P)
    st_g = Sg.reshape(-1)
    assert np.array_equal(st_g, st_ref), np.unique(st_g[st_g != st_ref])
    # every branch was taken somewhere
    bits = np.bitwise_or.reduce(st_ref)
    assert bits & G.GR_ST_W_CLAMPED and bits & G.GR_ST_TAU_FLOOR and bits & G.GR_ST_BD_LIMIT
    assert bits & G.GR_ST_FAILED and bits & G.GR_ST_ATM_THRESHOLD and np.any(st_ref == 0)
    wg = np.moveaxis(Wg, 0, -1).reshape(-1, 5)
    ug = np.moveaxis(Ug, 0, -1).reshape(-1, 5)
    for v in range(5):
        den = np.maximum(np.abs(w_ref[:, v]), 1e-3 * np.max(np.abs(w_ref[:, v])) + 1e-300)
        assert np.max(np.abs(wg[:, v] - w_ref[:, v]) / den) < 1e-12, ("W", v)
        den = np.maximum(np.abs(q_ref[:, v]), np.abs(q_ref[:, 0]) + np.abs(q_ref[:, 4]))
        assert np.max(np.abs(ug[:, v] - q_ref[:, v]) / den) < 1e-12, ("U", v)


@pytest.mark.parametrize("ceiling", [0, 1])
def test_every_con2prim_branch_in_the_mixed_stage(ceiling):
    """The same cells through the mixed stage with dt = 0 (U' = U): its atmosphere test on the FP32
    sqrt(gamma) in k_update and its con2prim form (FP32 bracket top, two-division master function) in
    k_c2p, against the oracle at the mixed atmosphere band.  Statuses identical; primitives and the
    conserved variables of solved cells within 1e-12; the atmosphere cells' conserved variables, formed
    with the FP32 metric and cell field, within 1e-6."""
    P = GH.mixed_params(O.Params(gamma_ad=2.0, rho_atm=1e-9, tol=1e-14, M_max=10.0, ceiling=ceiling))
    bi, U, cm, cb = branch_block(P)
    n, g = bi.n, bi.ng
    out = GH.gpu_stage([bi], P, 0.0, precision=G.GR_PREC_MIXED, U=[U])[0]
    met = cm[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 16)
    bd = cb[g:g + n[2], g:g + n[1], g:g + n[0]].reshape(-1, 3)
    q = np.moveaxis(H.interior(U, n, g), 0, -1).reshape(-1, 5)
    w_ref, q_ref, st_ref, _ = O.con2prim(met, q, bd, P)
    st_g = (H.interior(out["status"], n, g) & 0x3F).reshape(-1)
    assert np.array_equal(st_g, st_ref), np.unique(st_g[st_g != st_ref])
    bits = np.bitwise_or.reduce(st_ref)
    assert bits & G.GR_ST_W_CLAMPED and bits & G.GR_ST_TAU_FLOOR and bits & G.GR_ST_BD_LIMIT
    assert bits & G.GR_ST_FAILED and bits & G.GR_ST_ATM_THRESHOLD and np.any(st_ref == 0)
    wg = np.moveaxis(H.interior(out["W"], n, g), 0, -1).reshape(-1, 5)
    ug = np.moveaxis(H.interior(out["U"], n, g), 0, -1).reshape(-1, 5)
    atm = (st_ref & (G.GR_ST_ATM_THRESHOLD | G.GR_ST_FAILED)) != 0
    for v in range(5):
        den = np.maximum(np.abs(w_ref[:, v]), 1e-3 * np.max(np.abs(w_ref[:, v])) + 1e-300)
        assert np.max(np.abs(wg[:, v] - w_ref[:, v]) / den) < 1e-12, ("W", v)
        den = np.maximum(np.abs(q_ref[:, v]), np.abs(q_ref[:, 0]) + np.abs(q_ref[:, 4]))
        e = np.abs(ug[:, v] - q_ref[:, v]) / den
        assert np.max(e[~atm]) < 1e-12, ("U", v)
        assert np.max(e[atm]) < 1e-6, ("U atmosphere", v)
