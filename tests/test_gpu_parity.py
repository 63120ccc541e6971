"""GPU parity: the CUDA stage (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bar: FP64 path within 1e-12 relative per variable (denominators in tests/gpu_harness.compare) and
identical status; the uniform state bitwise; the mixed path (FP32 reconstruction/HLLE/EMF, FP64
accumulation and con2prim) within 1e-6 relative in rho with div B at round-off."""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from tests import gpu_harness as GH
from tests import helpers as H

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


def check64(gpu, ref, blocks, tol=TOL64):
    e = GH.compare(gpu, ref, blocks)
    bad = {k: v for k, v in e.items() if k != "status_mismatch" and v > tol}
    assert not bad and e["status_mismatch"] == 0, e
    return e


@pytest.mark.parametrize("recon", [0, 1, 2, 3])
def test_uniform_state_bitwise(recon):
    bi = I.uniform_block(n=(9, 7, 5))
    P = O.Params(gamma_ad=5.0 / 3.0, recon=recon, rho_atm=1e-10, tol=1e-15)
    U = H.cons_from_prims(bi, P)
    out = GH.gpu_stage([bi], P, 0.05, U=[U])[0]
    n, g = bi.n, bi.ng
    assert np.array_equal(H.interior(out["U"], n, g), H.interior(U, n, g))
    for a, b in zip(H.interior_faces(out["B"], n, g), H.interior_faces(bi.B, n, g)):
        assert np.array_equal(a, b)
    assert np.all(H.interior(out["status"], n, g) == 0)


@pytest.mark.parametrize("recon", [0, 1, 2, 3])
def test_random_block_fp64_parity(recon):
    bi = I.random_block(n=(16, 12, 10), g=3, seed=21, metric_amp=0.02)
    P = O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-14, tol=1e-15, rk_g0=0.5, rk_g1=0.5, rk_beta=0.5)
    U = H.cons_from_prims(bi, P)
    U0 = 1.0001 * U
    dt = 0.2 * bi.dx[0]
    check64(GH.gpu_stage([bi], P, dt, U=[U], U0=[U0]), GH.oracle_stage([bi], P, dt, U=[U], U0=[U0]), [bi])


def test_batch_of_uneven_blocks_fp64_parity():
    """Several block sizes in one launch, incl. a non-cubic block with a ragged last tile."""
    sizes = [(8, 8, 8), (12, 12, 12), (16, 16, 16), (13, 7, 9)]
    fields = I.make_fields(np.random.default_rng(5), 1.0, shared_metric=True)
    blocks = [I.random_block(n=s, g=3, x0=(0.1 * k, 0.05, 0.2), dx=(1 / 64,) * 3, seed=30, fields=fields)
              for k, s in enumerate(sizes)]
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-15)
    dt = 0.2 / 64
    check64(GH.gpu_stage(blocks, P, dt), GH.oracle_stage(blocks, P, dt), blocks)


def test_cellprep_sweep_tilings_fp64_parity():
    """The order-2 cell preparation walks each block along z in tiles of its x-y cell plane (at most 32
    columns, 256 cells): two x tiles of 23 (N0 = 46) with a ragged y tile, x tiles of 20 and 19 (N0 = 39)
    with ragged y tiles, and a thin block of one 7-column tile (N0 = 7)."""
    sizes = [(40, 6, 5), (33, 9, 3), (1, 20, 4)]
    fields = I.make_fields(np.random.default_rng(6), 1.0, shared_metric=True)
    blocks = [I.random_block(n=s, g=3, x0=(0.1 * k, 0.05, 0.2), dx=(1 / 64,) * 3, seed=31, fields=fields)
              for k, s in enumerate(sizes)]
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-15)
    dt = 0.2 / 64
    check64(GH.gpu_stage(blocks, P, dt), GH.oracle_stage(blocks, P, dt), blocks)


def test_shock_tube_block_fp64_parity():
    """The 1D magnetised shock tube on a 16^3 block (Gamma 5/3, PLM), first stage."""
    bi = I.shock_tube_block(n=(16, 16, 16), g=3)
    P = O.Params(gamma_ad=5.0 / 3.0, recon=0, rho_atm=1e-10, tol=1e-15)
    dt = 0.4 * bi.dx[0]
    check64(GH.gpu_stage([bi], P, dt), GH.oracle_stage([bi], P, dt), [bi])


def test_magnetised_star_fp64_parity():
    """Static Gamma=2 polytrope in its isotropic TOV metric with a poloidal field and atmosphere,
    WENOZ (a reduced 32^3 version of the 64^3 star)."""
    tov = I.solve_tov()
    bi = I.star_block(n=(32, 32, 32), g=3, half_width=10.02, tov=tov, A_b=0.05)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-13 * tov.rho[0], tol=1e-15)
    dt = 0.25 * bi.dx[0]
    check64(GH.gpu_stage([bi], P, dt), GH.oracle_stage([bi], P, dt), [bi])


def test_order4_interpolation_fp64_parity():
    bi = I.random_block(n=(10, 10, 10), g=4, seed=41, metric_amp=0.05)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-15, interp_order=4)
    dt = 0.2 * bi.dx[0]
    check64(GH.gpu_stage([bi], P, dt), GH.oracle_stage([bi], P, dt), [bi])


def test_nonzero_extrinsic_curvature_fp64_parity():
    bi = I.random_block(n=(8, 8, 8), g=3, seed=43, metric_amp=0.05, with_K=True)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-15)
    dt = 0.2 * bi.dx[0]
    check64(GH.gpu_stage([bi], P, dt, k_zero=False), GH.oracle_stage([bi], P, dt), [bi])


@pytest.mark.parametrize("recon", [1, 2, 3])
def test_mixed_precision_error_bounds(recon):
    """FP32 reconstruction/HLLE/EMF with FP64 accumulation against the FP64 oracle at the same
    atmosphere band: every variable within its stated bound (rho and D 1e-6), statuses equal, div B at
    FP64 round-off (WENOZ, WENO5, PPM)."""
    bi = I.random_block(n=(16, 16, 16), g=3, seed=22, metric_amp=0.02)
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-14, tol=1e-15))
    dt = 0.2 * bi.dx[0]
    out = GH.gpu_stage([bi], P, dt, precision=G.GR_PREC_MIXED, c2p_guess=G.GR_GUESS_FP32)
    ref = GH.oracle_stage([bi], P, dt)
    GH.check_mixed(out, ref, [bi], GH.MIXED_BOUNDS["random"], f"random block, mixed, recon {recon}")
    n, g = bi.n, bi.ng
    d = O.divb(n, g, bi.dx, out[0]["B"])
    Bmax = max(np.max(np.abs(b)) for b in H.interior_faces(out[0]["B"], n, g))
    assert np.max(np.abs(H.interior(d, n, g))) * bi.dx[0] / Bmax < 1e-14


@pytest.mark.parametrize("recon", [1, 3])
def test_mixed_precision_on_a_star_surface(recon):
    """The mixed path across the surface of the magnetised star, where a reconstruction stencil spans
    ~11 decades in density (star against atmosphere): rho within 1e-6 of the FP64 oracle, the same
    cells set to atmosphere, div B at round-off (WENOZ and PPM).  PPM's limiter takes sign decisions on
    products of differences; at the surface an FP32 rounding can flip one and move a face value by a
    limiter correction instead of a rounding, so its bound is 1e-5 (WENOZ's weights vary smoothly)."""
    tov = I.solve_tov()
    bi = I.star_block(n=(32, 32, 32), g=3, half_width=10.02, tov=tov, A_b=0.05)
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-13 * tov.rho[0], tol=1e-10))
    dt = 0.25 * bi.dx[0]
    out = GH.gpu_stage([bi], P, dt, precision=G.GR_PREC_MIXED, c2p_guess=G.GR_GUESS_FP32)
    ref = GH.oracle_stage([bi], P, dt)
    GH.check_mixed(out, ref, [bi], GH.MIXED_BOUNDS["star" if recon == 1 else "star_ppm"],
                   f"star surface, mixed, recon {recon}")
    n, g = bi.n, bi.ng
    d = O.divb(n, g, bi.dx, out[0]["B"])
    Bmax = max(np.max(np.abs(b)) for b in H.interior_faces(out[0]["B"], n, g))
    assert np.max(np.abs(H.interior(d, n, g))) * bi.dx[0] / Bmax < 1e-14


@pytest.mark.parametrize("umax", [0.5, 6.0])
def test_fp32_presolve_bracket_gives_the_same_root(umax):
    """con2prim with an FP32 pre-solve proposing the bracket converges to the oracle's root
    (tight tolerance), and rejects nothing on smooth states."""
    bi = I.random_block(n=(12, 12, 12), g=3, seed=23, metric_amp=0.05, u_max=umax)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-15)
    dt = 0.2 * bi.dx[0]
    out = GH.gpu_stage([bi], P, dt, c2p_guess=G.GR_GUESS_FP32)
    ref = GH.oracle_stage([bi], P, dt)
    # The iteration path differs from the oracle's (other bracket), so mu agrees to a few ulp; p is
    # recovered through eps = W (qbar - mu rbar^2) + ..., which cancels by ~W/eps (~1e4 here), so p
    # is held to 1e-10 and every other variable to 1e-12.
    e = GH.compare(out, ref, [bi])
    assert e["W4"] < 1e-10 and e["status_mismatch"] == 0, e
    assert all(v < TOL64 for k, v in e.items() if k not in ("W4", "status_mismatch")), e
    st = H.interior(out[0]["status"], bi.n, bi.ng)
    assert np.mean((st & G.GR_ST_GUESS_REJECTED) != 0) < 0.01


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_the_direct_stage_bitwise(precision):
    import torch
    bi = I.random_block(n=(12, 12, 12), g=3, seed=24, metric_amp=0.02)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-12)
    U = H.cons_from_prims(bi, P)
    pools = GH.Pools([bi])
    Ud, Wd, Bd, Md = pools.cells([U], 5), pools.cells([bi.W], 5), pools.faces([bi.B]), pools.verts([bi.metric])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    metric = G.metric_struct(Md)
    gp = GH.gr_params_from(P, precision, G.GR_GUESS_FP32 if precision else G.GR_GUESS_NONE)
    outs = []
    for use_graph in (False, True):
        Uo, Wo, Bo = Ud.clone(), Wd.clone(), [b.clone() for b in Bd]
        st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
        state = G.state_struct(Ud, Ud, Bd, Bd, Wd, Uo, Bo, Wo, st)
        if use_graph:
            g = G.gr_graph_capture(mesh, metric, state, 0.01, gp)
            G.gr_graph_launch(g, torch.cuda.current_stream())
            G.gr_graph_launch(g, torch.cuda.current_stream())    # replays are idempotent
            torch.cuda.synchronize()
            G.gr_graph_destroy(g)
        else:
            G.gr_stage(mesh, metric, state, 0.01, gp, torch.cuda.current_stream())
            torch.cuda.synchronize()
        outs.append([Uo.cpu(), Wo.cpu(), st.cpu()] + [b.cpu() for b in Bo])
    G.gr_mesh_destroy(mesh)
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("recon", [1, 0])
def test_fp32_copies_give_bitwise_the_same_mixed_stage(recon):
    """The mixed stage from caller-given FP32 copies of W, B and the metric (gr_cast_f32 of the FP64
    inputs) equals the stage that converts them itself, bitwise, on uneven blocks; the FP32 copies of
    its outputs it is asked to write are gr_cast_f32 of the FP64 outputs wherever those are written, and
    untouched elsewhere."""
    import torch
    blocks = [I.random_block(n=n, g=3, seed=90 + k, metric_amp=0.02) for k, n in
              enumerate([(8, 8, 8), (16, 8, 12), (12, 12, 12)])]
    P = GH.mixed_params(O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-14, tol=1e-12))
    pools = GH.Pools(blocks)
    U = pools.cells([H.cons_from_prims(b, P) for b in blocks], 5)
    W, B, M = pools.cells([b.W for b in blocks], 5), pools.faces([b.B for b in blocks]), pools.verts(
        [b.metric for b in blocks])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    gp = GH.gr_params_from(P, G.GR_PREC_MIXED, G.GR_GUESS_FP32)
    s = torch.cuda.current_stream()

    def f32(x):
        y = torch.empty(x.shape, dtype=torch.float32, device="cuda")
        G.gr_cast_f32(x.contiguous(), y, s)
        return y

    W32, B32, M32 = f32(W), [f32(b) for b in B], f32(M)
    outs = []
    try:
        for copies in (False, True):
            Uo, Wo, Bo = U.clone(), W.clone(), [b.clone() for b in B]
            st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
            state = G.state_struct(U, U, B, B, W, Uo, Bo, Wo, st)
            metric = G.metric_struct(M, metric32=M32 if copies else None)
            sentinel = -7.0
            Wo32 = torch.full(W.shape, sentinel, dtype=torch.float32, device="cuda")
            Bo32 = [torch.full(b.shape, sentinel, dtype=torch.float32, device="cuda") for b in B]
            if copies:
                G.set_fp32_copies(state, W32=W32, B32=B32, Wo32=Wo32, Bo32=Bo32)
            G.gr_stage(mesh, metric, state, 0.01, gp, s)
            torch.cuda.synchronize()
            outs.append([Uo.cpu(), Wo.cpu(), st.cpu()] + [b.cpu() for b in Bo])
    finally:
        G.gr_mesh_destroy(mesh)
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    # the written FP32 copies: the conversion of the outputs on interior cells / faces of interior cells
    inter = torch.zeros(pools.L.ncell, dtype=torch.bool)
    for b_, bi in enumerate(blocks):
        g, n = bi.ng, bi.n
        m = torch.zeros((n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g), dtype=torch.bool)
        m[g:g + n[2], g:g + n[1], g:g + n[0]] = True
        inter[int(pools.L.cell_off[b_]):int(pools.L.cell_off[b_]) + m.numel()] = m.view(-1)
    Wo64 = outs[1][1].cuda()
    ref32 = f32(Wo64).cpu()
    got32 = Wo32.cpu()
    assert torch.equal(got32[:, inter], ref32[:, inter])
    assert torch.all(got32[:, ~inter] == sentinel)
    for d in range(3):
        written = Bo32[d].cpu() != sentinel
        assert torch.equal(Bo32[d].cpu()[written], f32(outs[1][3 + d].cuda()).cpu()[written])
        assert int(written.sum()) == sum((b.n[0] + (d == 0)) * (b.n[1] + (d == 1)) * (b.n[2] + (d == 2))
                                         for b in blocks)


@pytest.mark.parametrize("precision,nbatch,rk", [(G.GR_PREC_FP64, 1, False), (G.GR_PREC_MIXED, 3, False),
                                                  (G.GR_PREC_MIXED, 2, True)])
def test_host_stage_equals_the_device_stage_bitwise(precision, nbatch, rk):
    # gr_host_stage on pinned host pools (batched transfers in, stages, transfers out on three streams)
    # gives gr_stage's results on device copies of the same data, for uneven blocks and an RK register
    # stage, ghosts of the outputs untouched
    import torch
    blocks = [I.random_block(n=n, g=3, seed=70 + k, metric_amp=0.02) for k, n in
              enumerate([(8, 8, 8), (16, 8, 12), (12, 12, 12), (8, 16, 8)])]
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-14, tol=1e-12)
    if rk:
        P.rk_g0, P.rk_g1, P.rk_beta = 0.75, 0.25, 0.25
    pools = GH.Pools(blocks)
    U = pools.cells([H.cons_from_prims(b, P) for b in blocks], 5)
    U0 = U * (1 + 1e-3) if rk else U
    Wd, Bd, Md = pools.cells([b.W for b in blocks], 5), pools.faces([b.B for b in blocks]), pools.verts(
        [b.metric for b in blocks])
    B0 = [b * (1 - 1e-3) for b in Bd] if rk else Bd
    gp = GH.gr_params_from(P, precision, G.GR_GUESS_FP32 if precision else G.GR_GUESS_NONE)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        # device stage
        Uo, Wo, Bo = U.clone(), Wd.clone(), [b.clone() for b in Bd]
        st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
        G.gr_stage(mesh, G.metric_struct(Md), G.state_struct(U, U0, Bd, B0, Wd, Uo, Bo, Wo, st), 0.01, gp,
                   torch.cuda.current_stream())
        torch.cuda.synchronize()
        ref = [Uo.cpu(), Wo.cpu(), st.cpu()] + [b.cpu() for b in Bo]
        # the same on pinned host pools
        pin = lambda t: t.cpu().pin_memory()
        hU, hW, hM = pin(U), pin(Wd), pin(Md)
        hU0 = pin(U0) if rk else hU
        hB = [pin(b) for b in Bd]
        hB0 = [pin(b) for b in B0] if rk else hB
        # outputs start as the device outputs did (the stages write interior elements only)
        hUo, hWo = pin(U), pin(Wd)
        hBo = [pin(b) for b in Bd]
        hst = torch.zeros(pools.L.ncell, dtype=torch.uint8).pin_memory()
        if not rk:   # pageable host pools are refused before anything runs
            with pytest.raises(G.GrstageError):
                G.gr_host_stage(mesh, G.metric_struct(hM), G.state_struct(U.cpu(), U.cpu(), hB, hB, hW, hUo, hBo, hWo,
                                                                          hst), 0.01, gp, nbatch)
        for _ in range(2):   # the second call reuses the staging pools and batches
            G.gr_host_stage(mesh, G.metric_struct(hM), G.state_struct(hU, hU0, hB, hB0, hW, hUo, hBo, hWo, hst), 0.01,
                            gp, nbatch, torch.cuda.current_stream())
            torch.cuda.synchronize()
            got = [hUo, hWo, hst] + hBo
            for a, b in zip(ref, got):
                assert torch.equal(a, b)
    finally:
        G.gr_mesh_destroy(mesh)


def test_invalid_arguments_are_rejected():
    import torch
    bi = I.uniform_block(n=(4, 4, 4), g=2)
    P = O.Params(gamma_ad=2.0, recon=1)
    with pytest.raises(G.GrstageError, match="ghost width"):
        GH.gpu_stage([bi], P, 0.01)
    with pytest.raises(G.GrstageError, match="invalid argument"):
        G.gr_mesh_create(GH.ctx(), [G.gr_block((G.C.c_int32 * 3)(0, 4, 4), 3)])


def test_empty_mesh_is_a_no_op():
    import torch
    mesh = G.gr_mesh_create(GH.ctx(), [])
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.zeros(8, dtype=torch.uint8, device="cuda")
    m = G.metric_struct(torch.zeros((16, 8), dtype=torch.float64, device="cuda"))
    s = G.state_struct([x] * 5, None, [x] * 3, None, [x] * 5, [x.clone() for _ in range(5)],
                       [x.clone() for _ in range(3)], [x.clone() for _ in range(5)], st)
    G.gr_stage(mesh, m, s, 0.1, G.gr_params_default())
    G.gr_mesh_destroy(mesh)


def test_prim2con_and_con2prim_entries():
    import torch
    bi = I.random_block(n=(12, 10, 8), g=3, seed=51, metric_amp=0.05)
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-15)
    pools = GH.Pools([bi])
    Wd = pools.cells([bi.W], 5)
    Bd = pools.faces([bi.B])
    Md = pools.verts([bi.metric])
    Ud = torch.zeros_like(Wd)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    m = G.metric_struct(Md)
    gp = GH.gr_params_from(P)
    G.gr_prim2con(mesh, m, list(Wd), Bd, list(Ud), gp)
    Uref = H.cons_from_prims(bi, P)
    Ug = pools.unpack_cells(Ud, 5)[0]
    n, g = bi.n, bi.ng
    for v in range(5):
        r = H.interior(Uref[v], n, g)
        den = np.maximum(np.abs(r), 1e-3 * np.max(np.abs(r)))
        assert np.max(np.abs(H.interior(Ug[v], n, g) - r) / den) < 1e-13, v
    W2 = torch.zeros_like(Wd)
    st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
    G.gr_con2prim(mesh, m, list(Ud), Bd, list(W2), st, gp)
    Wg = pools.unpack_cells(W2, 5)[0]
    assert np.max(np.abs(H.interior(Wg[0] - bi.W[0], n, g)) / H.interior(bi.W[0], n, g)) < 1e-12
    G.gr_mesh_destroy(mesh)


def test_diag_mass_and_divB():
    import torch
    bi = I.random_block(n=(16, 16, 16), g=3, seed=52)
    P = O.Params(gamma_ad=2.0)
    U = H.cons_from_prims(bi, P)
    pools = GH.Pools([bi])
    Ud = pools.cells([U], 5)
    Bd = pools.faces([bi.B])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    out = G.gr_diag(mesh, list(Ud), Bd)
    G.gr_mesh_destroy(mesh)
    n, g = bi.n, bi.ng
    Mb = np.sum(H.interior(U[0], n, g)) * np.prod(bi.dx)
    assert abs(out[0] - Mb) < 1e-12 * Mb
    assert out[1] < 1e-14 and out[2] < 1e-14


@pytest.mark.parametrize("precision", [G.GR_PREC_FP64, G.GR_PREC_MIXED])
def test_every_launch_shape_gives_bitwise_the_same_stage(precision):
    """CTA size, work-list order and persistent grids only change who computes what: every shape, and
    the autotuner's choice, give bitwise the same outputs (uneven batch with star matter and atmosphere)."""
    blocks = [I.random_block(n=s, g=3, seed=90 + k, rho_range=(1e-14, 1e-3)) for k, s in
              enumerate([(16, 16, 16), (24, 16, 8), (8, 8, 8), (5, 7, 9)])]
    P = O.Params(gamma_ad=2.0, rho_atm=1e-12, tol=1e-10)
    dt = 0.1 * min(blocks[0].dx)
    guess = G.GR_GUESS_FP32 if precision == G.GR_PREC_MIXED else G.GR_GUESS_NONE
    ref = GH.gpu_stage(blocks, P, dt, precision=precision, c2p_guess=guess)
    assert any(np.any(r["status"] == 1) for r in ref) and any(np.any(r["status"] == 0) for r in ref)
    variants = [[(64, 0, 0)] * 6, [(256, 1, 1)] * 6, [(128, 1, 0)] * 6,
                [(64, 1, 1), (256, 0, 0), (128, 1, 1), (64, 0, 1), (256, 1, 0), (64, 0, 1)]]
    for shp in variants:
        out = GH.gpu_stage(blocks, P, dt, precision=precision, c2p_guess=guess, shapes=shp)
        for a, b in zip(out, ref):
            for key in ("U", "W", "status"):
                assert np.array_equal(a[key], b[key]), (shp, key)
            for d in range(3):
                assert np.array_equal(a["B"][d], b["B"][d]), (shp, d)
    out = GH.gpu_stage(blocks, P, dt, precision=precision, c2p_guess=guess, autotune=True)
    for a, b in zip(out, ref):
        assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["W"], b["W"])


def test_autotune_and_shape_arguments():
    import torch
    blocks = [I.random_block(n=(8, 8, 8), g=3, seed=95)]
    pools = GH.Pools(blocks)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        assert G.gr_mesh_get_shapes(mesh, G.GR_PREC_MIXED) == [(128, 0, 0)] * 6
        with pytest.raises(G.GrstageError):
            G.gr_mesh_set_shapes(mesh, G.GR_PREC_MIXED, 0, [(96, 0, 0)] * 6)
        with pytest.raises(G.GrstageError):
            G.gr_mesh_set_shapes(mesh, 7, 0, [(64, 0, 0)] * 6)
        P = O.Params()
        U = H.cons_from_prims(blocks[0], P)
        Ud, Wd = pools.cells([U], 5), pools.cells([blocks[0].W], 5)
        Bd, Md = pools.faces([blocks[0].B]), pools.verts([blocks[0].metric])
        Uo, Wo, Bo = Ud.clone(), Wd.clone(), [b.clone() for b in Bd]
        st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
        state = G.state_struct(Ud, Ud, Bd, Bd, Wd, Uo, Bo, Wo, st)
        gp = GH.gr_params_from(P, G.GR_PREC_MIXED)
        shapes, ms = G.gr_autotune(mesh, G.metric_struct(Md), state, 0.01, gp, 2)
        assert len(shapes) == 6 and all(t in (64, 128, 256) and o in (0, 1) and p in (0, 1) for t, o, p in shapes)
        assert all(m >= 0 for m in ms)
        assert G.gr_mesh_get_shapes(mesh, G.GR_PREC_FP64) == [(128, 0, 0)] * 6   # other precision untouched
    finally:
        G.gr_mesh_destroy(mesh)


def test_autotuned_bracket_proposal_is_one_of_the_two_and_gives_its_stage():
    """GR_GUESS_AUTO: gr_autotune times the stage with no proposal and with the FP32 pre-solve and keeps the
    faster for the mesh (none before tuning); a stage with AUTO then equals, bitwise, the stage run with the
    chosen proposal explicitly."""
    import torch
    blocks = [I.random_block(n=s, g=3, seed=120 + k, rho_range=(1e-14, 1e-3)) for k, s in
              enumerate([(16, 16, 16), (12, 8, 10)])]
    P = O.Params(gamma_ad=2.0, rho_atm=1e-12, tol=1e-10)
    pools = GH.Pools(blocks)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        assert G.gr_mesh_get_guess(mesh, G.GR_PREC_MIXED, 0) == G.GR_GUESS_NONE
        assert G.gr_mesh_get_guess(mesh, 5, 0) == -1
        U = pools.cells([H.cons_from_prims(b, P) for b in blocks], 5)
        W, B, M = pools.cells([b.W for b in blocks], 5), pools.faces([b.B for b in blocks]), pools.verts(
            [b.metric for b in blocks])
        metric = G.metric_struct(M)
        dt = 0.1 * min(blocks[0].dx)

        def run(guess, tune=False):
            Uo, Wo, Bo = U.clone(), W.clone(), [x.clone() for x in B]
            st = torch.zeros(pools.L.ncell, dtype=torch.uint8, device="cuda")
            state = G.state_struct(U, U, B, B, W, Uo, Bo, Wo, st)
            gp = GH.gr_params_from(GH.mixed_params(P), G.GR_PREC_MIXED, guess)
            if tune:
                G.gr_autotune(mesh, metric, state, dt, gp, 2)
            G.gr_stage(mesh, metric, state, dt, gp)
            torch.cuda.synchronize()
            return [t.cpu().numpy() for t in (Uo, Wo, st)] + [b.cpu().numpy() for b in Bo]

        auto = run(G.GR_GUESS_AUTO, tune=True)
        chosen = G.gr_mesh_get_guess(mesh, G.GR_PREC_MIXED, 0)
        assert chosen in (G.GR_GUESS_NONE, G.GR_GUESS_FP32)
        assert G.gr_mesh_get_guess(mesh, G.GR_PREC_FP64, 0) == G.GR_GUESS_NONE   # other precision untouched
        explicit = run(chosen)
        for a, b in zip(auto, explicit):
            assert np.array_equal(a, b)
    finally:
        G.gr_mesh_destroy(mesh)
