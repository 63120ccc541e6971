"""Learned con2prim bracket on the GPU (not in the paper: a bracket proposal for the root find of Sec. 3.5).

* the sampler's features and log mu equal the oracle's for the same conserved states
* the network's forward pass and its backpropagated gradient equal the FP64 oracle's
* training on solves of the method lowers the loss, and on held-out states the learned bracket
  gives the same primitives as the plain bracket with fewer FP64 master-function evaluations"""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from paper_2311_04989_gb300 import learned_bracket as LB
from tests import gpu_harness as GH
from tests import helpers as H

pytestmark = pytest.mark.gpu

WIDE = dict(rho_range=(1e-12, 1e-2), theta_range=(1e-4, 1.0), u_max=3.0, sigma_range=(1e-4, 1e2),
            metric_amp=0.05)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


def test_sampler_matches_the_oracle():
    import torch
    bi = I.random_block(n=(12, 10, 8), g=3, seed=70, **WIDE)
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-15)
    U = H.cons_from_prims(bi, P)
    pools = GH.Pools([bi])
    Ud, Bd, Md = pools.cells([U], 5), pools.faces([bi.B]), pools.verts([bi.metric])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    nc = pools.L.ncell
    feats = [torch.zeros(nc, dtype=torch.float32, device="cuda") for _ in range(G.GR_MLP_NIN)]
    target = torch.zeros(nc, dtype=torch.float32, device="cuda")
    valid = torch.zeros(nc, dtype=torch.uint8, device="cuda")
    G.gr_c2p_samples(mesh, G.metric_struct(Md), list(Ud), Bd, GH.gr_params_from(P), feats, target, valid)
    G.gr_mesh_destroy(mesh)
    n, g = bi.n, bi.ng
    f_g = np.stack([H.interior(pools.unpack_cells(f.view(1, -1).double(), 1)[0], n, g).ravel() for f in feats], 1)
    t_g = H.interior(pools.unpack_cells(target.view(1, -1).double(), 1)[0], n, g).ravel()
    v_g = H.interior(pools.unpack_cells(valid, 1)[0], n, g).ravel().astype(bool)
    cm = H.interior(np.moveaxis(H.cell_metric(bi), -1, 0), n, g).reshape(16, -1).T
    Bc = H.interior(np.moveaxis(H.cell_B(bi), -1, 0), n, g).reshape(3, -1).T
    q = H.interior(U, n, g).reshape(5, -1).T
    f_r, t_r, v_r = O.c2p_samples(cm, q, Bc, P)
    assert np.array_equal(v_g, v_r) and v_r.mean() > 0.9
    assert np.max(np.abs(f_g[v_r] - f_r[v_r]) / np.maximum(np.abs(f_r[v_r]), 1e-3)) < 1e-6
    assert np.max(np.abs(t_g[v_r] - t_r[v_r])) < 1e-6


def test_forward_and_gradient_match_the_oracle():
    import torch
    rng = np.random.default_rng(71)
    P = np.zeros(G.GR_MLP_NPARAM)
    nin = G.GR_MLP_NIN
    P[G.MLP_MEAN:G.MLP_MEAN + nin] = rng.normal(0, 1, nin)
    P[G.MLP_ISTD:G.MLP_ISTD + nin] = rng.uniform(0.5, 2, nin)
    P[G.MLP_TMEAN], P[G.MLP_TSTD] = -0.7, 0.4
    P[16:] = rng.normal(0, 0.3, G.GR_MLP_NPARAM - 16)
    P = P.astype(np.float32).astype(np.float64)     # the values the GPU sees
    x = rng.normal(0, 1, (1000, nin)).astype(np.float32).astype(np.float64)
    t = rng.normal(-0.7, 0.5, 1000).astype(np.float32).astype(np.float64)
    Pd = torch.tensor(P, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    tg = G.gr_mlp_forward(Pd, xd).double().cpu().numpy()
    assert np.max(np.abs(tg - O.mlp_forward(P, x))) < 1e-5
    loss_g, grad_g = G.gr_mlp_grad(Pd, xd, td)
    loss_r, grad_r = O.mlp_loss_grad(P, x, t)
    assert abs(loss_g - loss_r) < 1e-5 * loss_r
    gg = grad_g.double().cpu().numpy()
    assert np.linalg.norm(gg - grad_r) < 1e-4 * np.linalg.norm(grad_r)
    assert np.max(np.abs(gg - grad_r)) < 1e-4 * np.max(np.abs(grad_r))


def test_training_lowers_the_loss_and_the_bracket_saves_evaluations():
    import torch
    ctx = GH.ctx()
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-10)
    gp = GH.gr_params_from(P)
    train_blocks = [I.random_block(n=(16, 16, 16), g=3, seed=100 + k, **WIDE) for k in range(32)]
    x, t = LB.collect(ctx, train_blocks, gp)
    assert x.shape[0] > 100000
    Pm, losses, delta = LB.train(x, t, epochs=60, batch=1024, lr=2e-3)
    assert losses[-1] < 0.05 * losses[0], losses
    assert 1e-5 <= delta < 0.05
    # held-out states: plain bracket versus learned bracket
    test_blocks = [I.random_block(n=(16, 16, 16), g=3, seed=200 + k, **WIDE) for k in range(3)]
    L, W, B, M = G.pack_blocks(test_blocks)
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    metric = G.metric_struct(M)
    U = torch.zeros_like(W)
    G.gr_prim2con(mesh, metric, list(W), B, list(U), gp)
    out = {}
    for name, guess in (("none", G.GR_GUESS_NONE), ("mlp", G.GR_GUESS_MLP)):
        Uc = U.clone(); Wc = torch.zeros_like(W)
        st = torch.zeros(L.ncell, dtype=torch.uint8, device="cuda")
        ev = torch.zeros(L.ncell, dtype=torch.int32, device="cuda")
        p = GH.gr_params_from(P, c2p_guess=guess)
        p.mlp = int(Pm.data_ptr())
        G.gr_con2prim(mesh, metric, list(Uc), B, list(Wc), st, p, evals=ev)
        torch.cuda.synchronize()
        out[name] = (Wc.cpu().numpy(), st.cpu().numpy(), ev.cpu().numpy())
    G.gr_mesh_destroy(mesh)
    interior = np.zeros(L.ncell, bool)
    for b, bi in enumerate(test_blocks):
        m = np.zeros(tuple(v + 2 * bi.ng for v in bi.n[::-1]), bool)
        m[bi.ng:-bi.ng, bi.ng:-bi.ng, bi.ng:-bi.ng] = True
        interior[L.cell_off[b]:L.cell_off[b] + m.size] = m.ravel()
    W0, s0, e0 = (a[..., interior] for a in out["none"])
    W1, s1, e1 = (a[..., interior] for a in out["mlp"])
    solved = (s0 & 0x3F) == 0
    assert np.array_equal(s0 & 0x3F, s1 & 0x3F)
    rejected = np.mean((s1[solved] & G.GR_ST_GUESS_REJECTED) != 0)
    assert rejected < 0.05, rejected
    # same root to the solve tolerance: rho = D/W, W^2 amplification of tol 1e-10
    rel = np.abs(W1[0][solved] - W0[0][solved]) / W0[0][solved]
    assert rel.max() < 1e-8
    gain = e0[solved].mean() / e1[solved].mean()
    print(f"learned bracket: {e0[solved].mean():.2f} -> {e1[solved].mean():.2f} FP64 master evaluations per "
          f"solved cell (x{gain:.2f}), {100 * rejected:.2f}% brackets rejected, first step {delta:.2e}")
    assert gain > 1.15
