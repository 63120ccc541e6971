"""Matter sources of the spacetime equations on the GPU (rho_ADM, S_i, S_ij of Sec. 2.1-2.2 at the
owned vertices, cell-to-vertex interpolation of Sec. 3.2) against the oracle, through the C ABI.

* a batch of uneven blocks (8^3 .. 32^3, the widest needing several shared-memory slabs) within 1e-12
  of the oracle for vertex-interpolation orders 2 and 4 and metric orders 2 and 4
* the tabulated EOS within 1e-12
* the FP32-arithmetic variant: rho_ADM within 1e-6 pointwise, every source within 1e-6 of its scale
* vertices outside the owned range are left untouched
* too small a ghost width and a bad order are rejected"""
import numpy as np
import pytest
from scipy.ndimage import maximum_filter

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


def gpu_adm(blocks, P: O.Params, vc_order, metric_order, precision=G.GR_PREC_FP64):
    import torch
    pools = GH.Pools(blocks)
    W = pools.cells([b.W for b in blocks], P.nw)
    Bd = pools.faces([b.B for b in blocks])
    M = pools.verts([b.metric for b in blocks])
    out = torch.full((10, max(pools.L.nvert, 1)), float("nan"), dtype=torch.float64, device="cuda")
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        metric = G.metric_struct(M, order=metric_order)
        gp = GH.gr_params_from(P, precision)
        G.gr_adm_sources(mesh, metric, [W[v] for v in range(min(P.nw, 6))], Bd, gp, vc_order, [out[c] for c in range(10)],
                         torch.cuda.current_stream())
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    h = out.cpu().numpy()
    res = []
    for b, bi in enumerate(blocks):
        N = [bi.n[a] + 2 * bi.ng + 1 for a in range(3)]
        sz = N[0] * N[1] * N[2]
        o = pools.L.vert_off[b]
        res.append(h[:, o:o + sz].reshape(10, N[2], N[1], N[0]))
    return res


def owned(bi):
    g = bi.ng
    return (slice(None), slice(g, g + bi.n[2] + 1), slice(g, g + bi.n[1] + 1), slice(g, g + bi.n[0] + 1))


def max_rel(got, ref, bi):
    sl = owned(bi)
    g, r = got[sl], ref[sl]
    err = 0.0
    for c in range(10):
        scale = np.max(np.abs(r[c]))
        den = np.maximum(np.abs(r[c]), max(1e-3 * scale, 1e-300))
        err = max(err, float(np.max(np.abs(g[c] - r[c]) / den)))
    return err


def uneven_batch(seed=60):
    sizes = [(8, 8, 8), (16, 12, 8), (32, 32, 32), (12, 16, 24), (16, 16, 16)]
    return [I.random_block(n=n, g=3, seed=seed + k, rho_range=(1e-6, 1e-2), u_max=0.5, sigma_range=(1e-2, 3.0),
                           metric_amp=0.02) for k, n in enumerate(sizes)]


@pytest.mark.parametrize("vc_order,metric_order", [(2, 2), (4, 2), (4, 4)])
def test_adm_sources_match_the_oracle(vc_order, metric_order):
    blocks = uneven_batch()
    P = O.Params(gamma_ad=2.0, interp_order=metric_order)
    got = gpu_adm(blocks, P, vc_order, metric_order)
    err = 0.0
    for b, bi in enumerate(blocks):
        ref = O.adm_block(H.to_oracle(bi), P, vc_order)
        err = max(err, max_rel(got[b], ref, bi))
        mask = np.ones(got[b].shape[1:], bool)
        mask[owned(bi)[1:]] = False
        assert np.all(np.isnan(got[b][:, mask]))
    print(f"ADM sources, vertex order {vc_order}, metric order {metric_order}: max rel err {err:.2e}")
    assert err < TOL64


def test_adm_sources_with_the_table_match_the_oracle():
    eos = I.SyntheticEOS()
    tab = eos.table(n=(80, 64, 24))
    blocks = [I.random_block(n=n, g=3, seed=70 + k, eos=eos, rho_range=(1e-8, 1e-3), T_range=(1e-3, 5e-2),
                             ye_range=(0.05, 0.5), u_max=0.5, sigma_range=(1e-3, 1.0), metric_amp=0.02)
              for k, n in enumerate([(8, 8, 8), (16, 8, 12)])]
    P = O.Params(table=tab)
    got = gpu_adm(blocks, P, 4, 2)
    err = max(max_rel(got[b], O.adm_block(H.to_oracle(bi), P, 4), bi) for b, bi in enumerate(blocks))
    print(f"ADM sources with the table: max rel err {err:.2e}")
    assert err < TOL64


@pytest.mark.parametrize("vc_order", [2, 4])
def test_mixed_adm_sources_error_bound(vc_order):
    # FP32 rounding is relative to the size of the terms each source sums: rho_ADM is a sum of
    # same-sign terms at a cell (pointwise bound), while S_i and S_ij are differences of terms of the
    # block's energy-density scale (bound relative to the component's largest magnitude in the block)
    blocks = uneven_batch(seed=90)
    P = O.Params(gamma_ad=2.0)
    got = gpu_adm(blocks, P, vc_order, 2, G.GR_PREC_MIXED)
    e_rho = e_scale = 0.0
    for b, bi in enumerate(blocks):
        sl = owned(bi)
        g, r = got[b][sl], O.adm_block(H.to_oracle(bi), P, vc_order)[sl]
        # the order-4 interpolant has negative weights: its rounding scales with the stencil's values,
        # bounded here by the largest |rho_ADM| within two vertices
        den = np.abs(r[0]) if vc_order == 2 else maximum_filter(np.abs(r[0]), size=5, mode="nearest")
        e_rho = max(e_rho, float(np.max(np.abs(g[0] - r[0]) / den)))
        for c in range(10):
            e_scale = max(e_scale, float(np.max(np.abs(g[c] - r[c])) / np.max(np.abs(r[c]))))
    print(f"ADM sources, FP32 arithmetic, vertex order {vc_order}: rho_ADM pointwise {e_rho:.2e}, "
          f"every component vs its block scale {e_scale:.2e}")
    assert e_rho < 1e-6 and e_scale < 1e-6


def test_adm_sources_reject_bad_arguments():
    import torch
    bi = I.random_block(n=(8, 8, 8), g=1, seed=80)
    P = O.Params(gamma_ad=2.0)
    pools = GH.Pools([bi])
    W = pools.cells([bi.W], 5)
    Bd = pools.faces([bi.B])
    M = pools.verts([bi.metric])
    out = torch.zeros((10, pools.L.nvert), dtype=torch.float64, device="cuda")
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        gp = GH.gr_params_from(P)
        args = (list(W), Bd, gp)
        with pytest.raises(G.GrstageError):   # order 4 needs two ghost cells
            G.gr_adm_sources(mesh, G.metric_struct(M, order=2), *args, 4, list(out))
        with pytest.raises(G.GrstageError):
            G.gr_adm_sources(mesh, G.metric_struct(M, order=2), *args, 3, list(out))
        G.gr_adm_sources(mesh, G.metric_struct(M, order=2), *args, 2, list(out))
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
