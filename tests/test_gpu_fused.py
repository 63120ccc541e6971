"""The fused sweep of the mixed path (k_fused: reconstruction, HLLE fluxes, corner EMFs, CT update and flux
divergence of a block in one pass, fluxes and EMFs in shared memory) and the tiled face sweep (k_faces_tile:
face fluxes from stencils and metric staged in shared memory) against the separate kernels: the paths must
give bitwise the same stage (U', W', status, B' and the FP32 copies of W', B'), on uneven
blocks of every size the sweep takes (ragged x-y extents up to 16, any length in z), for every
reconstruction method, both RK forms and both corner-EMF rules, on smooth random states and across a star
surface (atmosphere resets and root-find cells in one block).  And against the oracle on the bench's
two-star blocks."""
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


def _run(blocks, P, path, dt, rk=False):
    import torch
    pools = GH.Pools(blocks)
    U = pools.cells([H.cons_from_prims(b, P) for b in blocks], 5)
    W, B, M = pools.cells([b.W for b in blocks], 5), pools.faces([b.B for b in blocks]), pools.verts(
        [b.metric for b in blocks])
    # an RK register stage: U0, B0 differ from U, B
    U0 = U * (1 + 1e-3) if rk else U
    B0 = [b * (1 - 1e-3) for b in B] if rk else B
    Uo, Wo, Bo = torch.zeros_like(U), torch.zeros_like(W), [torch.zeros_like(b) for b in B]
    Wo32, Bo32 = torch.zeros(W.shape, dtype=torch.float32, device="cuda"), [
        torch.zeros(b.shape, dtype=torch.float32, device="cuda") for b in B]
    st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        gp = GH.gr_params_from(P, G.GR_PREC_MIXED, G.GR_GUESS_FP32)
        if rk:
            gp.rk_g0, gp.rk_g1, gp.rk_beta = 0.75, 0.25, 0.25
        state = G.state_struct(U, U0, B, B0, W, Uo, Bo, Wo, st)
        G.set_fp32_copies(state, Wo32=Wo32, Bo32=Bo32)
        G.gr_mesh_set_path(mesh, path)
        assert G.gr_mesh_get_path(mesh) == path
        G.gr_stage(mesh, G.metric_struct(M), state, dt, gp, torch.cuda.current_stream())
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    return [Uo.cpu(), Wo.cpu(), st.cpu(), Wo32.cpu()] + [b.cpu() for b in Bo] + [b.cpu() for b in Bo32], pools


def _same(a, b):
    import torch
    for x, y in zip(a, b):
        assert torch.equal(x, y), (x - y).abs().max()


@pytest.mark.parametrize("recon", [0, 1, 2, 3])
@pytest.mark.parametrize("rk", [False, True])
def test_fused_sweep_equals_the_separate_kernels_bitwise(recon, rk):
    shapes = [(16, 16, 16), (8, 12, 5), (16, 7, 9), (3, 3, 16), (1, 2, 3), (13, 16, 2)]
    blocks = [I.random_block(n=n, g=3, seed=120 + k, metric_amp=0.03) for k, n in enumerate(shapes)]
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-14, tol=1e-12))
    dt = 0.2 * min(min(b.dx) for b in blocks)
    sep, _ = _run(blocks, P, G.GR_PATH_SEPARATE, dt, rk)
    for path in (G.GR_PATH_FUSED, G.GR_PATH_TILED_FACES):
        _same(sep, _run(blocks, P, path, dt, rk)[0])


@pytest.mark.parametrize("emf", [0, 1])
def test_fused_sweep_across_a_star_surface_bitwise(emf):
    tov = I.solve_tov()
    star = I.star_block(n=(32, 32, 32), g=3, half_width=10.02, tov=tov, A_b=0.05)
    blocks = I.split_block(star, (2, 2, 2))
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-13 * tov.rho[0], tol=1e-10, emf=emf))
    dt = 0.25 * star.dx[0]
    sep, pools = _run(blocks, P, G.GR_PATH_SEPARATE, dt)
    st = sep[2].numpy()
    assert np.any(st & 1) and np.any(st == 0)     # both atmosphere resets and solved cells
    for path in (G.GR_PATH_FUSED, G.GR_PATH_TILED_FACES):
        _same(sep, _run(blocks, P, path, dt)[0])


def _same_nan(a, b):
    """Bitwise equality that takes NaN for NaN (the positions must match)."""
    import torch
    for x, y in zip(a, b):
        if x.is_floating_point():
            mx, my = torch.isnan(x), torch.isnan(y)
            assert torch.equal(mx, my), int((mx != my).sum())
            assert torch.equal(x[~mx], y[~my]), (x[~mx] - y[~my]).abs().max()
        else:
            assert torch.equal(x, y), int((x != y).sum())


@pytest.mark.parametrize("face_b", [3e18, 3e19])
def test_paths_agree_bitwise_beside_an_overflowing_field(face_b):
    """One x-face in the atmosphere corner of a star block carries a field so large that the FP32 momentum
    and energy fluxes about it reach ~1e36 (first case) or overflow (second case) while the atmosphere
    around it stays below the threshold.  The cells beside it must take the same decision (atmosphere
    reset, or failed for a non-finite update of S_j or tau) on the separate kernels -- whose atmosphere
    test reads the fluxes of S_j and tau only in a block that the face kernel flagged -- and on the tiled
    faces, as on the fused sweep, which always reads them."""
    tov = I.solve_tov()
    star = I.star_block(n=(32, 32, 32), g=3, half_width=10.02, tov=tov, A_b=0.05)
    g = star.ng
    star.B[0][g + 1, g + 1, g + 2] = face_b
    blocks = I.split_block(star, (2, 2, 2))
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-13 * tov.rho[0], tol=1e-10))
    dt = 0.25 * star.dx[0]
    sep, _ = _run(blocks, P, G.GR_PATH_SEPARATE, dt)
    st = sep[2].numpy()
    print("statuses beside the planted face:", np.unique(st, return_counts=True))
    assert np.any(st & G.GR_ST_ATM_THRESHOLD)
    for path in (G.GR_PATH_FUSED, G.GR_PATH_TILED_FACES):
        _same_nan(sep, _run(blocks, P, path, dt)[0])


def test_fused_sweep_refuses_blocks_it_does_not_take():
    big = [I.random_block(n=(24, 8, 8), g=3, seed=5)]
    pools = GH.Pools(big)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        for path in (G.GR_PATH_FUSED, G.GR_PATH_TILED_FACES):
            with pytest.raises(G.GrstageError, match="wider than 16"):
                G.gr_mesh_set_path(mesh, path)
        assert G.gr_mesh_get_path(mesh) == G.GR_PATH_SEPARATE
    finally:
        G.gr_mesh_destroy(mesh)


def test_fused_sweep_on_two_star_blocks_against_the_oracle():
    """Sampled 16^3 blocks of the bench's two-star workload (star centre, surface, atmosphere) through the
    fused sweep, per variable against the oracle at the same atmosphere band."""
    mi = I.BinaryStarMesh(nb=16, n=16)
    centre = lambda x: int((x + 32) // 4)
    pick = lambda i, j, k: i + 16 * (j + 16 * k)
    sample = [pick(centre(-20), 8, 8), pick(centre(20) + 2, 8, 8), pick(8, 8, 8)]
    blocks = [mi.block(b) for b in sample]
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=1, rho_atm=mi.rho_atm, p_atm=mi.p_atm, tol=1e-10))
    dt = 0.25 * mi.dx
    got, pools = _run(blocks, P, G.GR_PATH_FUSED, dt)
    Uo, Wo, st = (pools.unpack_cells(got[k].cuda(), n) for k, n in ((0, 5), (1, 5), (2, 1)))
    Bo = pools.unpack_faces([x.cuda() for x in got[4:7]])
    out = [dict(U=Uo[b], W=Wo[b], B=Bo[b], status=st[b]) for b in range(len(blocks))]
    ref = GH.oracle_stage(blocks, P, dt)
    GH.check_mixed(out, ref, blocks, GH.MIXED_BOUNDS["star"], "two-star blocks, fused sweep")
