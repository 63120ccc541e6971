"""Learned con2prim bracket: collect samples of the bracketed solves, train the network on the GPU,
and set its bracket half-width.

All arithmetic runs in the library's kernels (gr_prim2con, gr_c2p_samples, gr_mlp_train,
gr_mlp_forward); this module only moves tensors: it compacts the valid samples, takes the
normalisation statistics of the features and targets, and chooses the half-width from the
residuals of a held-out set.  The parameter layout is the one documented in include/grstage.h.
"""
from __future__ import annotations

import numpy as np

from . import grstage as G

NW = G.GR_MLP_NPARAM - 16


def collect(ctx, blocks, params: G.gr_params, device="cuda"):
    """Features (n,6) and log mu (n,) of the plain bracketed solves of the interior cells of blocks
    (their conserved variables formed from the blocks' primitives by gr_prim2con)."""
    import torch
    L, W, B, M = G.pack_blocks(blocks, device)
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    try:
        metric = G.metric_struct(M)
        U = torch.zeros((6 if params.eos == G.GR_EOS_TABLE else 5, W.shape[1]), dtype=W.dtype, device=W.device)
        G.gr_prim2con(mesh, metric, list(W), B, list(U), params)
        feats = [torch.zeros(L.ncell, dtype=torch.float32, device=device) for _ in range(G.GR_MLP_NIN)]
        target = torch.zeros(L.ncell, dtype=torch.float32, device=device)
        valid = torch.zeros(L.ncell, dtype=torch.uint8, device=device)
        G.gr_c2p_samples(mesh, metric, list(U), B, params, feats, target, valid)
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    return samples_from(feats, target, valid)


def samples_from(feats, target, valid):
    import torch
    m = valid.bool()
    x = torch.stack([f[m] for f in feats], 1).contiguous()
    return x, target[m].contiguous()


def init_params(x, t, seed=0, device="cuda"):
    """Parameter vector with the data's normalisation statistics and seeded random weights
    (Glorot-uniform scale per layer)."""
    import torch
    P = np.zeros(G.GR_MLP_NPARAM, np.float32)
    nin = G.GR_MLP_NIN
    xm = x.mean(0).cpu().numpy(); xs = x.std(0).cpu().numpy()
    P[G.MLP_MEAN:G.MLP_MEAN + nin] = xm
    P[G.MLP_ISTD:G.MLP_ISTD + nin] = 1.0 / np.maximum(xs, 1e-6)
    P[G.MLP_TMEAN] = float(t.mean().item())
    P[G.MLP_TSTD] = max(float(t.std().item()), 1e-6)
    P[G.MLP_STEP] = 1.0
    rng = np.random.default_rng(2311_04989 + seed)
    off = 16
    for (nout, nin) in ((64, nin), (64, 64), (1, 64)):
        lim = np.sqrt(6.0 / (nin + nout))
        P[off:off + nout * nin] = rng.uniform(-lim, lim, nout * nin)
        off += nout * nin + nout          # biases stay 0
    return torch.from_numpy(P).to(device)


def set_step(P, x, t, quantile=0.75, floor=1e-5):
    """First bracket step delta = the given quantile of |predicted - true log mu| on (x, t) (a
    typical error: larger ones are reached by the doubling steps), at least floor."""
    r = (G.gr_mlp_forward(P, x) - t).abs()
    q = float(np.quantile(r.cpu().numpy(), quantile))
    P[G.MLP_STEP] = max(q, floor)
    return float(P[G.MLP_STEP].item())


def train(x, t, epochs=60, batch=1024, lr=2e-3, seed=0, holdout=0.1):
    """Shuffle (seeded), fit on (1 - holdout) of the samples, set the first step on the rest.
    Returns (P, per-epoch losses, delta)."""
    import torch
    n = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(2311_04989 + seed)
    perm = torch.randperm(n, generator=g).to(x.device)
    x, t = x[perm].contiguous(), t[perm].contiguous()
    nh = max(1, int(holdout * n))
    xt, tt, xh, th = x[nh:].contiguous(), t[nh:].contiguous(), x[:nh].contiguous(), t[:nh].contiguous()
    P = init_params(xt, tt, seed, x.device)
    losses = G.gr_mlp_train(P, xt, tt, epochs, batch, lr)
    delta = set_step(P, xh, th)
    return P, losses, delta
