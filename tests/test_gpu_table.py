"""Tabulated EOS on the GPU (Sec. 2.2.1; App. A) against the FP64 oracle, through the C ABI.

* gr_prim2con / gr_con2prim with the table: same conserved variables, primitives, Y_e, T and status
  as the oracle, including temperature-floor, Y_e-clamp, limit and atmosphere cells
* one stage on table blocks (uneven batch): FP64 path within 1e-12 of the oracle; the mixed path
  within its error bound and with div B at round-off
* a table whose log rho axis does not cover the state's densities takes the nearest density's
  specific quantities on both sides
* the learned bracket trained on table solves of other seeds gives the same roots with fewer FP64
  master-function evaluations"""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from paper_2311_04989_gb300 import learned_bracket as LB
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


@pytest.fixture(scope="module")
def eos():
    return I.SyntheticEOS()


@pytest.fixture(scope="module")
def tab(eos):
    return eos.table()            # 200 x 128 x 64, the size of the con2prim-heavy workload


def table_block(eos, n, seed, **kw):
    args = dict(rho_range=(1e-8, 1e-3), T_range=(1e-3, 5e-2), ye_range=(0.05, 0.5), u_max=0.6,
                sigma_range=(1e-3, 1.0), metric_amp=0.02)
    args.update(kw)
    return I.random_block(n=n, g=3, seed=seed, eos=eos, **args)


def _interior_mask(L, blocks):
    m = np.zeros(L.ncell, bool)
    for b, bi in enumerate(blocks):
        a = np.zeros(tuple(v + 2 * bi.ng for v in bi.n[::-1]), bool)
        a[bi.ng:-bi.ng, bi.ng:-bi.ng, bi.ng:-bi.ng] = True
        m[L.cell_off[b]:L.cell_off[b] + a.size] = a.ravel()
    return m


def test_table_prim2con_and_con2prim_match_the_oracle(eos, tab):
    import torch
    blocks = [table_block(eos, (12, 10, 8), 300), table_block(eos, (6, 6, 6), 301, u_max=3.0,
                                                            sigma_range=(1e-2, 1e3))]
    P = O.Params(table=tab, rho_atm=1e-12, T_atm=2e-3, tol=1e-14)
    gp = GH.gr_params_from(P)
    pools = GH.Pools(blocks)
    Wd = pools.cells([bi.W for bi in blocks], 7)
    Bd = pools.faces([bi.B for bi in blocks])
    Md = pools.verts([bi.metric for bi in blocks])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    metric = G.metric_struct(Md)
    U = torch.zeros((6, Wd.shape[1]), dtype=torch.float64, device="cuda")
    G.gr_prim2con(mesh, metric, list(Wd), Bd, list(U), gp)
    U_p2c = U.cpu().numpy()
    # perturb: some cells below the atmosphere, some with Y_e outside the table
    Uh = U_p2c.copy()
    inter = _interior_mask(pools.L, blocks)
    idx = np.flatnonzero(inter)
    rng = np.random.default_rng(5)
    Uh[0, idx[rng.choice(idx.size, 10, replace=False)]] *= 1e-9
    sel = idx[rng.choice(idx.size, 10, replace=False)]
    Uh[5, sel] = 0.9 * Uh[0, sel]
    U = torch.from_numpy(Uh).cuda()
    Uc = U.clone()
    W2 = torch.zeros((7, Wd.shape[1]), dtype=torch.float64, device="cuda")
    st = torch.zeros(Wd.shape[1], dtype=torch.uint8, device="cuda")
    G.gr_con2prim(mesh, metric, list(Uc), Bd, list(W2), st, gp)
    torch.cuda.synchronize()
    G.gr_mesh_destroy(mesh)
    # oracle on the same interior cells
    Ug, Wg, Sg = U.cpu().numpy(), W2.cpu().numpy(), st.cpu().numpy()
    Uog = Uc.cpu().numpy()
    for b, bi in enumerate(blocks):
        n, g = bi.n, bi.ng
        cm = H.interior(np.moveaxis(H.cell_metric(bi), -1, 0), n, g).reshape(16, -1).T
        Bc = H.interior(np.moveaxis(H.cell_B(bi), -1, 0), n, g).reshape(3, -1).T
        sl = slice(pools.L.cell_off[b], pools.L.cell_off[b] + np.prod(bi.N))
        shape = (-1,) + tuple(bi.N[::-1])
        w_in = H.interior(np.asarray(bi.W), n, g).reshape(7, -1).T
        q_ref = O.prim2con(cm, w_in, Bc, P)
        # prim2con parity
        q_p2c = H.interior(U_p2c[:, sl].reshape(shape), n, g).reshape(6, -1).T
        scale = q_ref[:, 0] + np.abs(q_ref[:, 4])
        assert np.max(np.abs(q_p2c[:, 0] / q_ref[:, 0] - 1)) < 1e-13
        for k in (1, 2, 3, 4):
            d = np.abs(q_p2c[:, k] - q_ref[:, k]) / np.maximum(np.abs(q_ref[:, k]), scale)
            assert d.max() < 1e-12, (k, d.max())
        assert np.max(np.abs(q_p2c[:, 5] / q_ref[:, 5] - 1)) < 1e-13
        q_gpu = H.interior(Ug[:, sl].reshape(shape), n, g).reshape(6, -1).T     # perturbed input
        # con2prim parity on every cell (the oracle starts from the GPU's perturbed input U)
        w_ref, qo_ref, st_ref, _ = O.con2prim(cm, q_gpu, Bc, P)
        w_gpu = H.interior(Wg[:, sl].reshape(shape), n, g).reshape(7, -1).T
        qo_gpu = H.interior(Uog[:, sl].reshape(shape), n, g).reshape(6, -1).T
        s_gpu = H.interior(Sg[sl].reshape(bi.N[::-1]), n, g).ravel()
        assert np.array_equal(s_gpu & 0x3F, st_ref)
        assert np.any(st_ref & 1) and np.any(st_ref & 32)
        for k in range(7):
            floor = 1e-3 * np.max(np.abs(w_ref[:, k])) if 1 <= k <= 3 else 1e-300
            d = np.abs(w_gpu[:, k] - w_ref[:, k]) / np.maximum(np.abs(w_ref[:, k]), floor)
            assert d.max() < (1e-10 if k == 6 else 1e-12), (b, k, d.max())
        sc = qo_ref[:, 0] + np.abs(qo_ref[:, 4])
        for k in range(6):
            den = np.maximum(np.abs(qo_ref[:, k]), sc if 1 <= k <= 4 else 1e-300)
            assert np.max(np.abs(qo_gpu[:, k] - qo_ref[:, k]) / den) < 1e-12, k


def test_table_stage_fp64_parity_on_an_uneven_batch(eos, tab):
    blocks = [table_block(eos, (10, 8, 6), 310), table_block(eos, (6, 7, 8), 311),
              table_block(eos, (8, 8, 8), 312, u_max=2.0, sigma_range=(1e-2, 30.0))]
    P = O.Params(table=tab, rho_atm=1e-12, T_atm=1e-4, tol=1e-13)
    dt = 0.2 * min(blocks[0].dx)
    gpu = GH.gpu_stage(blocks, P, dt)
    ref = GH.oracle_stage(blocks, P, dt)
    e = GH.compare(gpu, ref, blocks)
    assert e["status_mismatch"] == 0
    for k, v in e.items():
        if k != "status_mismatch":
            assert v < (1e-10 if k == "W6" else 1e-12), (k, v)


def test_table_density_outside_the_table_takes_the_nearest_density(eos):
    tab = eos.table(n=(40, 64, 16), rho_range=(1e-6, 1e-2))   # the block reaches down to 1e-8
    blocks = [table_block(eos, (8, 6, 6), 320)]
    P = O.Params(table=tab, rho_atm=1e-12, T_atm=1e-4, tol=1e-13)
    dt = 0.2 * min(blocks[0].dx)
    e = GH.compare(GH.gpu_stage(blocks, P, dt), GH.oracle_stage(blocks, P, dt), blocks)
    assert e["status_mismatch"] == 0
    assert max(v for k, v in e.items() if k not in ("status_mismatch", "W6")) < 1e-12, e


def test_table_stage_mixed_precision_error_bound(eos, tab):
    import torch
    blocks = [table_block(eos, (16, 16, 16), 330), table_block(eos, (12, 16, 10), 331)]
    P = GH.mixed_params(O.Params(table=tab, rho_atm=1e-12, T_atm=1e-4, tol=1e-10))
    dt = 0.2 * min(blocks[0].dx)
    gmx = GH.gpu_stage(blocks, P, dt, precision=G.GR_PREC_MIXED, c2p_guess=G.GR_GUESS_FP32)
    ref = GH.oracle_stage(blocks, P, dt)
    GH.check_mixed(gmx, ref, blocks, GH.MIXED_BOUNDS["table"], "table stage, mixed vs the oracle")
    for b, bi in enumerate(blocks):
        div = O.divb(bi.n, bi.ng, bi.dx, gmx[b]["B"])
        bmax = max(np.max(np.abs(x)) for x in gmx[b]["B"])
        assert np.max(np.abs(H.interior(div, bi.n, bi.ng))) * min(bi.dx) / bmax < 1e-14


def test_table_learned_bracket_saves_evaluations(eos, tab):
    import torch
    ctx = GH.ctx()
    P = O.Params(table=tab, rho_atm=1e-12, T_atm=1e-5, tol=1e-10)
    gp = GH.gr_params_from(P)
    kw = dict(rho_range=(1e-11, 1e-3), T_range=(1e-4, 5e-2), u_max=3.0, sigma_range=(1e-4, 1e2))
    train_blocks = [table_block(eos, (16, 16, 16), 400 + k, **kw) for k in range(64)]
    x, t = LB.collect(ctx, train_blocks, gp)
    assert x.shape[0] > 200000
    # the table's root depends on six features: more samples and epochs than the ideal gas needs
    Pm, losses, delta = LB.train(x, t, epochs=400, batch=2048, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0], losses
    test_blocks = [table_block(eos, (16, 16, 16), 500 + k, **kw) for k in range(3)]
    L, W, B, M = G.pack_blocks(test_blocks)
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    metric = G.metric_struct(M)
    U = torch.zeros((6, W.shape[1]), dtype=torch.float64, device="cuda")
    G.gr_prim2con(mesh, metric, list(W), B, list(U), gp)
    out = {}
    for name, guess in (("none", G.GR_GUESS_NONE), ("mlp", G.GR_GUESS_MLP)):
        Uc = U.clone(); Wc = torch.zeros((7, W.shape[1]), dtype=torch.float64, device="cuda")
        st = torch.zeros(L.ncell, dtype=torch.uint8, device="cuda")
        ev = torch.zeros(L.ncell, dtype=torch.int32, device="cuda")
        p = GH.gr_params_from(P, c2p_guess=guess)
        p.mlp = int(Pm.data_ptr())
        G.gr_con2prim(mesh, metric, list(Uc), B, list(Wc), st, p, evals=ev)
        torch.cuda.synchronize()
        out[name] = (Wc.cpu().numpy(), st.cpu().numpy(), ev.cpu().numpy())
    G.gr_mesh_destroy(mesh)
    inter = _interior_mask(L, test_blocks)
    W0, s0, e0 = (a[..., inter] for a in out["none"])
    W1, s1, e1 = (a[..., inter] for a in out["mlp"])
    solved = (s0 & 0x3F) == 0
    assert np.array_equal(s0 & 0x3F, s1 & 0x3F)
    rejected = np.mean((s1[solved] & G.GR_ST_GUESS_REJECTED) != 0)
    assert rejected < 0.05, rejected
    rel = np.abs(W1[0][solved] - W0[0][solved]) / W0[0][solved]
    assert rel.max() < 1e-8
    gain = e0[solved].mean() / e1[solved].mean()
    print(f"table learned bracket: {e0[solved].mean():.2f} -> {e1[solved].mean():.2f} FP64 master evaluations "
          f"per solved cell (x{gain:.2f}), {100 * rejected:.2f}% rejected, first step {delta:.2e}")
    assert gain > 1.15
