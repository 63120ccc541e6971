"""gr_diag_noalloc: the diagnostics entry point for callers that cannot allocate device memory (an
application that owns the device memory pool, or an in-situ hook that must not change the device
footprint).  It must give gr_diag's results, call after call, through the C ABI.

Collected last on purpose (file name), so a stop-at-first-failure run has already run every other
test before this one."""
import numpy as np
import pytest

from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()
    return torch


def _pools(torch, blocks, seed):
    """Device pools with a face field that is not divergence-free (so the div B norms are O(1))."""
    rng = np.random.default_rng(seed)
    L = G.Layout.of(blocks)
    D = np.zeros((5, L.ncell))
    for b, bi in enumerate(blocks):
        a = rng.uniform(0.5, 2.0, bi.W[0].size)
        D[0, L.cell_off[b]:L.cell_off[b] + a.size] = a
    Bp = []
    for d in range(3):
        h = np.zeros(L.nface[d])
        for b, bi in enumerate(blocks):
            f = bi.B[d].ravel() + 1e-3 * rng.standard_normal(bi.B[d].size)
            h[L.face_off[b, d]:L.face_off[b, d] + f.size] = f
        Bp.append(torch.from_numpy(h).cuda())
    return L, torch.from_numpy(D).cuda(), Bp


def _check(ref, got):
    assert got[0] == pytest.approx(ref[0], rel=1e-12)
    assert got[1] == pytest.approx(ref[1], rel=1e-12)
    assert got[2] == pytest.approx(ref[2], rel=1e-12)
    assert got[3] == ref[3]


def test_noalloc_diag_matches_gr_diag_on_two_calls_in_a_row(dev):
    torch = dev
    blocks = [I.random_block(n=s, g=3, seed=60 + k) for k, s in enumerate([(16, 16, 16), (8, 12, 10), (5, 5, 5)])]
    ctx = G.gr_context_create(0)
    for call, seed in enumerate((1, 2)):       # the second call sees different data
        L, U, B = _pools(torch, blocks, seed)
        mesh = G.gr_mesh_create(ctx, L.descriptors())
        ref = G.gr_diag(mesh, list(U), B)
        G.gr_mesh_destroy(mesh)
        got = G.gr_diag_noalloc(L.descriptors(), list(U), B)
        _check(ref, got)
        assert got[1] > 1e-3          # a field with real divergence: the norms are exercised
    G.gr_context_destroy(ctx)


def test_noalloc_diag_matches_gr_diag_beyond_one_pass_of_its_grid(dev):
    """More interior cells than the partial-sum grid has threads (512 CTAs x 256), so every thread runs
    several grid-stride iterations and the block search crosses many blocks per thread: 64 blocks of
    16^3 mixed with ragged blocks (270k interior cells)."""
    torch = dev
    shapes = [(16, 16, 16)] * 64 + [(7, 9, 11), (3, 5, 2), (12, 4, 8), (1, 1, 1)]
    blocks = [I.random_block(n=s, g=3, seed=80 + k) for k, s in enumerate(shapes)]
    ctx = G.gr_context_create(0)
    L, U, B = _pools(torch, blocks, 4)
    assert L.interior_cells() > 512 * 256
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    ref = G.gr_diag(mesh, list(U), B)
    G.gr_mesh_destroy(mesh)
    for _ in range(2):
        _check(ref, G.gr_diag_noalloc(L.descriptors(), list(U), B))
    G.gr_context_destroy(ctx)


def test_noalloc_diag_reports_a_nan_face_like_gr_diag(dev):
    """A single NaN face value must reach max |div B|, the integrated norm and max |B| in both entry
    points (a maximum that drops NaN would report a blown-up field as finite)."""
    torch = dev
    blocks = [I.random_block(n=s, g=3, seed=90 + k) for k, s in enumerate([(16, 16, 16), (8, 12, 10)])]
    ctx = G.gr_context_create(0)
    L, U, B = _pools(torch, blocks, 5)
    b1 = blocks[1]
    # an interior y-face of the second block: cell (3, 4, 5)
    g, N = b1.ng, [b1.n[a] + 2 * b1.ng for a in range(3)]
    fy = int(L.face_off[1, 1]) + ((5 + g) * (N[1] + 1) + (4 + g)) * N[0] + (3 + g)
    B[1][fy] = float("nan")
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    ref = G.gr_diag(mesh, list(U), B)
    G.gr_mesh_destroy(mesh)
    got = G.gr_diag_noalloc(L.descriptors(), list(U), B)
    G.gr_context_destroy(ctx)
    assert np.isfinite(ref[0]) and got[0] == pytest.approx(ref[0], rel=1e-12)
    for k in (1, 2, 3):
        assert np.isnan(ref[k]) and np.isnan(got[k]), (k, ref, got)


def test_noalloc_diag_rejects_more_blocks_than_its_fixed_scratch_allows(dev):
    torch = dev
    blocks = [I.uniform_block(n=(2, 2, 2), g=1) for _ in range(257)]
    L, U, B = _pools(torch, blocks, 3)
    with pytest.raises(G.GrstageError, match=r"nblocks must be in \[1, 256\]"):
        G.gr_diag_noalloc(L.descriptors(), list(U), B)
    got = G.gr_diag_noalloc(L.descriptors()[:256], list(U), B)   # the maximum itself is accepted
    assert np.isfinite(got[0])
