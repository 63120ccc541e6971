"""Multi-block RK step on the GPU (ghost exchange, time step, SSP-RK2/RK3 stages) against the oracle's
driver, through the C ABI.

* the ghost fill gives bitwise the oracle's ghost cells and ghost faces, periodic and outflow
* one FP64 driver step (RK2 and RK3, grid or wave-speed dt) within 1e-12 of the oracle's step
* a captured driver step replays bitwise like the direct step
* the mixed-precision driver step keeps rho within 1e-6 of the oracle and div B at round-off
* neighbour tables that would copy ghosts from ghosts (blocks thinner than the ghost width) and
  malformed tables are rejected"""
import copy

import numpy as np
import pytest

import oracle as O
from oracle import driver as DR
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from tests import gpu_harness as GH
from tests import helpers as H
from tests.test_oracle_driver import periodic_global

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


class Run:
    """Device pools of a set of same-level blocks and a driver on them."""

    def __init__(self, blocks, nbr, P: O.Params, U=None):
        import torch
        self.blocks = blocks
        self.pools = GH.Pools(blocks)
        self.P = P
        U = U if U is not None else [H.cons_from_prims(b, P, P.interp_order) for b in blocks]
        self.U = self.pools.cells(U, P.nq)
        self.W = self.pools.cells([b.W for b in blocks], P.nw)
        self.B = self.pools.faces([b.B for b in blocks])
        self.M = self.pools.verts([b.metric for b in blocks])
        self.st = torch.zeros(max(self.pools.L.ncell, 1), dtype=torch.uint8, device="cuda")
        self.mesh = G.gr_mesh_create(GH.ctx(), self.pools.L.descriptors())
        self.drv = G.gr_driver_create(self.mesh, nbr)
        self.metric = G.metric_struct(self.M, order=P.interp_order)

    def close(self):
        G.gr_driver_destroy(self.drv)
        G.gr_mesh_destroy(self.mesh)

    def rows(self, t, n):
        return [t[v] for v in range(n)]

    def step(self, cfl, dt_mode, order, precision=G.GR_PREC_FP64):
        import torch
        gp = GH.gr_params_from(self.P, precision)
        G.gr_driver_step(self.drv, self.metric, self.rows(self.U, self.P.nq), self.rows(self.W, self.P.nw), self.B,
                         self.st, gp, cfl, dt_mode, order, torch.cuda.current_stream())

    def result(self):
        import torch
        torch.cuda.synchronize()
        U = self.pools.unpack_cells(self.U, self.P.nq)
        W = self.pools.unpack_cells(self.W, self.P.nw)
        B = self.pools.unpack_faces(self.B)
        st = self.pools.unpack_cells(self.st, 1)
        return [dict(U=U[b], W=W[b], B=B[b], status=st[b]) for b in range(len(self.blocks))]


def _scramble_ghosts(blocks, seed):
    """Overwrite every ghost cell and ghost face with noise, so that a ghost the fill misses shows."""
    rng = np.random.default_rng(seed)
    for bi in blocks:
        n, g = bi.n, bi.ng
        keep = H.interior(bi.W, n, g).copy()
        bi.W[...] = rng.uniform(0.5, 2.0, bi.W.shape)
        bi.W[:, g:g + n[2], g:g + n[1], g:g + n[0]] = keep
        for d in range(3):
            f = bi.B[d]
            sl = (slice(g, g + n[2] + (d == 2)), slice(g, g + n[1] + (d == 1)), slice(g, g + n[0] + (d == 0)))
            keep = f[sl].copy()
            f[...] = rng.uniform(-1.0, 1.0, f.shape)
            f[sl] = keep


@pytest.mark.parametrize("periodic", [True, False])
def test_ghost_fill_matches_the_oracle_bitwise(periodic):
    import torch
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14)
    parts = I.split_block(periodic_global(n=(16, 8, 8), seed=50), (2, 2, 1))
    _scramble_ghosts(parts, 51)
    nbr = I.block_grid_neighbours((2, 2, 1), periodic=(periodic, True, periodic))
    run = Run(parts, nbr, P)
    try:
        G.gr_ghost_fill(run.drv, run.rows(run.W, P.nw), run.B, torch.cuda.current_stream())
        got = run.result()
    finally:
        run.close()
    n, g = parts[0].n, parts[0].ng
    W = [b.W.copy() for b in parts]
    B = [[f.copy() for f in b.B] for b in parts]
    DR.ghost_fill(W, B, nbr, n, g)
    for b in range(len(parts)):
        assert np.array_equal(got[b]["W"], W[b])
        for d in range(3):
            assert np.array_equal(got[b]["B"][d], B[b][d])


CASES = [  # (rk order, dt mode, recon, periodic)
    (3, G.GR_DT_GRID, 1, True),
    (3, G.GR_DT_SIGNAL, 1, True),
    (2, G.GR_DT_SIGNAL, 0, False),
    (3, G.GR_DT_GRID, 3, True),
]


@pytest.mark.parametrize("order,dt_mode,recon,periodic", CASES)
def test_driver_steps_match_the_oracle(order, dt_mode, recon, periodic):
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14, recon=recon)
    whole = periodic_global(n=(16, 8, 8), seed=52 + recon)
    parts = I.split_block(whole, (2, 2, 1))
    nbr = I.block_grid_neighbours((2, 2, 1), periodic=(periodic, True, True))
    ref = copy.deepcopy(parts)
    Uref = [H.cons_from_prims(b, P, P.interp_order) for b in ref]
    run = Run(parts, nbr, P, U=[u.copy() for u in Uref])
    cfl = 0.25
    mode = "grid" if dt_mode == G.GR_DT_GRID else "signal"
    try:
        for _ in range(2):
            run.step(cfl, dt_mode, order)
            got = run.result()
            dt_gpu = G.gr_driver_dt(run.drv)
            dt_ref, st_ref = DR.rk_step(ref, Uref, nbr, P, cfl, order=order, dt_mode=mode)
            assert abs(dt_gpu - dt_ref) <= 1e-13 * dt_ref
    finally:
        run.close()
    refs = [dict(U=Uref[b], W=ref[b].W, B=ref[b].B, status=st_ref[b]) for b in range(len(ref))]
    errs = GH.compare(got, refs, blocks=parts)
    print(f"driver RK{order} {mode} recon {recon} periodic {periodic}: max err "
          f"{max(v for k, v in errs.items() if k != 'status_mismatch'):.2e}")
    assert errs.pop("status_mismatch") == 0
    assert max(errs.values()) < TOL64, errs


@pytest.mark.parametrize("dt_mode", [G.GR_DT_GRID, G.GR_DT_SIGNAL])
def test_captured_driver_step_replays_bitwise(dt_mode):
    import torch
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14, recon=1)
    parts = I.split_block(periodic_global(n=(16, 8, 8), seed=56), (2, 2, 1))
    nbr = I.block_grid_neighbours((2, 2, 1))
    a = Run(copy.deepcopy(parts), nbr, P)
    b = Run(copy.deepcopy(parts), nbr, P)
    try:
        gp = GH.gr_params_from(P, G.GR_PREC_MIXED)
        graph = G.gr_driver_capture(a.drv, a.metric, a.rows(a.U, P.nq), a.rows(a.W, P.nw), a.B, a.st, gp, 0.25,
                                    dt_mode, 3)
        try:
            for _ in range(3):
                G.gr_graph_launch(graph, torch.cuda.current_stream())
                b.step(0.25, dt_mode, 3, G.GR_PREC_MIXED)
        finally:
            G.gr_graph_destroy(graph)
        ra, rb = a.result(), b.result()
        assert G.gr_driver_dt(a.drv) == G.gr_driver_dt(b.drv)
    finally:
        a.close()
        b.close()
    for x, y in zip(ra, rb):
        assert np.array_equal(x["U"], y["U"]) and np.array_equal(x["W"], y["W"])
        assert np.array_equal(x["status"], y["status"])
        for d in range(3):
            assert np.array_equal(x["B"][d], y["B"][d])


def test_mixed_driver_step_error_and_div_b():
    """One mixed RK3 step of the driver against the oracle driver's step at the same atmosphere band:
    every variable within the stated bounds, div B at round-off."""
    P = GH.mixed_params(O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14, recon=1))
    parts = I.split_block(periodic_global(n=(16, 8, 8), seed=57), (2, 2, 1))
    nbr = I.block_grid_neighbours((2, 2, 1))
    ref = copy.deepcopy(parts)
    Uref = [H.cons_from_prims(b, P, P.interp_order) for b in ref]
    run = Run(parts, nbr, P, U=[u.copy() for u in Uref])
    try:
        run.step(0.25, G.GR_DT_GRID, 3, G.GR_PREC_MIXED)
        got = run.result()
    finally:
        run.close()
    _, st = DR.rk_step(ref, Uref, nbr, P, 0.25, order=3, dt_mode="grid")
    refs = [dict(U=Uref[b], W=ref[b].W, B=ref[b].B, status=st[b]) for b in range(len(parts))]
    GH.check_mixed(got, refs, parts, GH.MIXED_BOUNDS["driver"], "mixed RK3 driver step")
    for b, bi in enumerate(parts):
        n, g = bi.n, bi.ng
        div = O.divb(n, g, bi.dx, got[b]["B"])
        bmax = max(np.max(np.abs(f)) for f in got[b]["B"])
        assert np.max(np.abs(H.interior(div, n, g))) * bi.dx[0] / bmax < 1e-14


def test_driver_rejects_bad_tables():
    thin = I.split_block(I.uniform_block(n=(4, 8, 8), g=3), (2, 1, 1))   # 2 cells < 3 ghosts along x
    pools = GH.Pools(thin)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        with pytest.raises(G.GrstageError):
            G.gr_driver_create(mesh, I.block_grid_neighbours((2, 1, 1)))
        # outflow everywhere is fine: no copy from a neighbour crosses the thin axis
        alone = np.full((2, 27), -1, np.int32)
        alone[:, 13] = (0, 1)
        G.gr_driver_destroy(G.gr_driver_create(mesh, alone))
        bad = I.block_grid_neighbours((2, 1, 1), periodic=(False, True, True))
        bad[0, 13] = 1
        with pytest.raises(G.GrstageError):
            G.gr_driver_create(mesh, bad)
        bad = I.block_grid_neighbours((2, 1, 1), periodic=(False, True, True))
        bad[1, 0] = 7
        with pytest.raises(G.GrstageError):
            G.gr_driver_create(mesh, bad)
    finally:
        G.gr_mesh_destroy(mesh)



def test_driver_step_with_the_table_matches_the_oracle():
    # the driver with the tabulated EOS (7 primitive pools exchanged, D Y_e advected): two RK2 steps,
    # grid time step, periodic split domain, against the oracle's driver
    eos = I.SyntheticEOS()
    tab = eos.table(n=(80, 64, 24))
    n, g = (16, 8, 8), 3
    bi = I.random_block(n=n, g=g, seed=58, dx=tuple(1.0 / v for v in n), L=1.0, eos=eos, rho_range=(1e-7, 1e-3),
                        T_range=(1e-3, 3e-2), ye_range=(0.1, 0.45), u_max=0.3, sigma_range=(1e-3, 0.3),
                        fields=I.make_fields(np.random.default_rng(I.SEED_BASE + 58), 1.0, shared_metric=True),
                        metric_amp=0.01)
    H.fill_periodic_cells(bi.W, n, g)
    H.fill_periodic_faces(bi.B, n, g)
    H.fill_periodic_vertices(bi.metric, n, g)
    parts = I.split_block(bi, (2, 2, 1))
    nbr = I.block_grid_neighbours((2, 2, 1))
    P = O.Params(table=tab, rho_atm=1e-12, tol=1e-14, recon=1)
    ref = copy.deepcopy(parts)
    Uref = [H.cons_from_prims(b, P, P.interp_order) for b in ref]
    run = Run(parts, nbr, P, U=[u.copy() for u in Uref])
    try:
        for _ in range(2):
            run.step(0.25, G.GR_DT_GRID, 2)
            got = run.result()
            _, st_ref = DR.rk_step(ref, Uref, nbr, P, 0.25, order=2, dt_mode="grid")
    finally:
        run.close()
    refs = [dict(U=Uref[b], W=ref[b].W, B=ref[b].B, status=st_ref[b]) for b in range(len(ref))]
    # u~^i pass through zero; con2prim recovers them from O(1) quantities (W ~ 1), rounding ~1e-16
    # absolute: their floor is 1e-2 of the block maximum (as in the refined-mesh tests)
    errs = GH.compare(got, refs, blocks=parts, floors={"W1": 1e-2, "W2": 1e-2, "W3": 1e-2})
    print("driver RK2 with the table: " + ", ".join(f"{k} {v:.1e}" for k, v in sorted(errs.items())))
    assert errs.pop("status_mismatch") == 0
    # T is the inverse of the table's piecewise-linear interpolant in log T, ill-conditioned where the
    # cold part dominates the pressure: held to 1e-10 as in the table stage parity test
    for k, v in errs.items():
        assert v < (1e-10 if k == "W6" else TOL64), (k, v)
