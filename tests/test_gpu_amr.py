"""Level-boundary operators on the GPU (Sec. 3.3, last paragraph) against the oracle, through the C ABI.

* restriction of cells and faces, prolongation of cells (limited linear) and of faces (divergence
  preserving), into the fine interior and ghosts, within 1e-14 of the oracle; the prolonged fine cells
  are divergence-free
* one stage on a periodic two-level mesh with the flux and EMF corrections: within 1e-12 of the
  oracle's two-level stage (FP64); total D conserved and the level faces consistent to FP64 rounding;
  the mixed path conserves and stays consistent to its FP32 workspace rounding
* malformed level tables are rejected"""
import numpy as np
import pytest

import oracle as O
from oracle import amr as A
from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300.inputs import BlockInput
from tests import gpu_harness as GH
from tests import helpers as H
from tests.test_oracle_amr import _coarse_faces_from_potential

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


def _pair(rng, nvar=3):
    """a coarse 4^3 block (g = 2) and a fine 8^3 block (g = 2) over the coarse interior, random data"""
    g = 2
    dxc, dxf = (0.2, 0.1, 0.4), (0.1, 0.05, 0.2)
    Wc = rng.uniform(0.5, 2.0, (nvar, 8, 8, 8))
    Bc = _coarse_faces_from_potential(rng, (4, 4, 4), g, dxc)
    Wf = rng.uniform(0.5, 2.0, (nvar, 12, 12, 12))
    Bf = _coarse_faces_from_potential(rng, (8, 8, 8), g, dxf)
    mc = np.zeros((16, 9, 9, 9))
    mf = np.zeros((16, 13, 13, 13))
    c = BlockInput((4, 4, 4), g, (0, 0, 0), dxc, mc, Wc, Bc)
    f = BlockInput((8, 8, 8), g, (0, 0, 0), dxf, mf, Wf, Bf)
    return c, f


def _run(blocks, nvar, restrict_maps=(), prolong_maps=(), prolong=False):
    import torch
    pools = GH.Pools(blocks)
    W = pools.cells([b.W for b in blocks], nvar)
    Bd = pools.faces([b.B for b in blocks])
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        G.gr_mesh_set_levels(mesh, restrict_maps=restrict_maps, prolong_maps=prolong_maps)
        fn = G.gr_prolong if prolong else G.gr_restrict
        fn(mesh, [W[v] for v in range(nvar)], Bd, torch.cuda.current_stream())
        torch.cuda.synchronize()
    finally:
        G.gr_mesh_destroy(mesh)
    return pools.unpack_cells(W, nvar), pools.unpack_faces(Bd)


def test_restriction_matches_the_oracle():
    rng = np.random.default_rng(11)
    c, f = _pair(rng)
    W, B = _run([c, f], 3, restrict_maps=[(0, 1, (0, 0, 0), (0, 0, 0), (4, 4, 4))])
    refW = c.W.copy()
    refB = [b.copy() for b in c.B]
    A.restrict_cells(f.W, 2, refW, 2, (0, 0, 0), (0, 0, 0), (4, 4, 4))
    A.restrict_faces(f.B, 2, refB, 2, (0, 0, 0), (0, 0, 0), (4, 4, 4))
    assert np.max(np.abs(W[0] - refW)) <= 1e-15 * np.max(np.abs(refW))
    for d in range(3):
        assert np.max(np.abs(B[0][d] - refB[d])) <= 1e-14 * np.max(np.abs(refB[d]))


def test_prolongation_matches_the_oracle_into_interior_and_ghosts():
    rng = np.random.default_rng(12)
    c, f = _pair(rng)
    lo, hi = (-2, -2, -2), (10, 10, 10)
    W, B = _run([c, f], 3, prolong_maps=[(0, 1, (0, 0, 0), lo, hi)], prolong=True)
    refW = f.W.copy()
    refB = [b.copy() for b in f.B]
    A.prolong_cells(c.W, 2, refW, 2, (0, 0, 0), lo, hi)
    A.prolong_faces(c.B, 2, refB, 2, (0, 0, 0), lo, hi, f.dx)
    assert np.max(np.abs(W[1] - refW)) <= 1e-14 * np.max(np.abs(refW))
    for d in range(3):
        assert np.max(np.abs(B[1][d] - refB[d])) <= 1e-13 * np.max(np.abs(refB[d]))
    div = O.divb(f.n, f.ng, f.dx, B[1])
    scale = max(np.max(np.abs(b)) for b in B[1]) / min(f.dx)
    assert np.max(np.abs(div)) < 1e-13 * scale


def _level_faces(records):
    return [(c, f, d, s, o1, o2) for (c, f, d, s, o1, o2) in records]


def _mass(blocks, U):
    return sum(np.sum(H.interior(u[0], b.n, b.ng)) * np.prod(b.dx) for u, b in zip(U, blocks))


def _face_mismatch(blocks, out, records):
    g = blocks[0].ng
    worst = 0.0
    for (c, f, d, side, o1, o2) in records:
        pc, pf = (8, 0) if side > 0 else (0, 8)
        cB = out[c]["B"][0][g + o2:g + o2 + 4, g + o1:g + o1 + 4, g + pc]
        fB = out[f]["B"][0][g:g + 8, g:g + 8, g + pf]
        fm = 0.25 * ((fB[0::2, 0::2] + fB[0::2, 1::2]) + (fB[1::2, 0::2] + fB[1::2, 1::2]))
        worst = max(worst, float(np.max(np.abs(cB - fm)) / np.max(np.abs(cB))))
    return worst


def test_two_level_stage_matches_the_oracle_and_conserves():
    blocks, records = H.two_level_periodic(seed=5)
    P = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-12, tol=1e-14, recon=1)
    U = [H.cons_from_prims(b, P) for b in blocks]
    dt = 0.25 * blocks[1].dx[0]
    got = GH.gpu_stage(blocks, P, dt, U=U, level_faces=_level_faces(records))
    ref = A.two_level_stage(blocks, U, records, P, dt)
    refs = [dict(U=r[0], B=r[1], W=r[2], status=r[3]) for r in ref]
    # u~^i here are smooth waves of amplitude ~0.1 through zero; con2prim recovers them from O(1)
    # quantities (W ~ 1), so their rounding is ~1e-16 absolute, which the default floor (1e-3 of the
    # block maximum, ~1e-4) would read as 1e-12: their floor is 1e-2 of the maximum
    errs = GH.compare(got, refs, blocks=blocks, floors={"W1": 1e-2, "W2": 1e-2, "W3": 1e-2})
    dm = abs(_mass(blocks, [g["U"] for g in got]) / _mass(blocks, U) - 1)
    mis = _face_mismatch(blocks, got, records)
    print(f"two-level GPU stage (FP64): max err vs oracle "
          f"{max(v for k, v in errs.items() if k != 'status_mismatch'):.2e}, mass change {dm:.2e}, "
          f"level-face mismatch {mis:.2e}; per variable " +
          ", ".join(f"{k} {v:.1e}" for k, v in sorted(errs.items()) if k != "status_mismatch"))
    assert errs.pop("status_mismatch") == 0
    assert max(errs.values()) < 1e-12, errs
    assert dm < 1e-14 and mis < 1e-13


def test_mixed_two_level_stage_conserves_to_its_workspace_rounding():
    blocks, records = H.two_level_periodic(seed=6)
    P = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-12, tol=1e-14, recon=1)
    U = [H.cons_from_prims(b, P) for b in blocks]
    dt = 0.25 * blocks[1].dx[0]
    got = GH.gpu_stage(blocks, P, dt, U=U, precision=G.GR_PREC_MIXED, level_faces=_level_faces(records))
    plain = GH.gpu_stage(blocks, P, dt, U=U, precision=G.GR_PREC_MIXED)
    m0 = _mass(blocks, U)
    dm = abs(_mass(blocks, [g["U"] for g in got]) / m0 - 1)
    dm_plain = abs(_mass(blocks, [g["U"] for g in plain]) / m0 - 1)
    mis, mis_plain = _face_mismatch(blocks, got, records), _face_mismatch(blocks, plain, records)
    print(f"two-level GPU stage (mixed): mass change {dm:.2e} (uncorrected {dm_plain:.2e}), level-face mismatch "
          f"{mis:.2e} (uncorrected {mis_plain:.2e})")
    assert dm < 1e-10 and mis < 1e-6
    assert dm_plain > 100 * dm and mis_plain > 100 * mis


def test_level_tables_are_checked():
    blocks, records = H.two_level_periodic(seed=7)
    pools = GH.Pools(blocks)
    mesh = G.gr_mesh_create(GH.ctx(), pools.L.descriptors())
    try:
        G.gr_mesh_set_levels(mesh, faces=_level_faces(records))
        bad = [
            [(0, 1, 3, 1, 0, 0)],            # no such direction
            [(0, 1, 0, 2, 0, 0)],            # side must be +-1
            [(0, 1, 0, 1, 5, 0)],            # patch beyond the coarse face
            [(1, 2, 0, 1, 0, 0)],            # same spacing: not a coarse / fine pair
            [(0, 9, 0, 1, 0, 0)],            # no such block
        ]
        for faces in bad:
            with pytest.raises(G.GrstageError):
                G.gr_mesh_set_levels(mesh, faces=faces)
        with pytest.raises(G.GrstageError):   # prolongation would read beyond the coarse ghosts
            G.gr_mesh_set_levels(mesh, prolong_maps=[(0, 1, (0, 0, 0), (-4, 0, 0), (8, 8, 8))])
        G.gr_mesh_set_levels(mesh)            # clears
    finally:
        G.gr_mesh_destroy(mesh)


def test_two_level_driver_steps_match_the_oracle_and_keep_div_b():
    # the RK driver on a refined mesh: cross-level ghost fill (same-level copies, restriction,
    # prolongation) before every stage and the level corrections inside it; two RK3 steps against the
    # oracle's two-level RK step, then the invariants on the GPU's own state
    import copy
    from tests.helpers import two_level_periodic_tables
    from tests.test_gpu_driver import Run
    blocks, _ = H.two_level_periodic(seed=9)
    nbr, rmaps, pmaps, records = two_level_periodic_tables()
    P = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-12, tol=1e-14, recon=1)
    ref = copy.deepcopy(blocks)
    Uref = [H.cons_from_prims(b, P) for b in ref]
    run = Run(blocks, nbr, P, U=[u.copy() for u in Uref])
    m0 = _mass(ref, Uref)
    try:
        G.gr_mesh_set_levels(run.mesh, faces=_level_faces(records), restrict_maps=rmaps, prolong_maps=pmaps)
        for _ in range(2):
            run.step(0.25, G.GR_DT_GRID, 3)
            got = run.result()
            dt_ref = A.two_level_rk_step(ref, Uref, nbr, rmaps, pmaps, records, P, 0.25, order=3)
            assert G.gr_driver_dt(run.drv) == dt_ref
    finally:
        run.close()
    refs = [dict(U=Uref[b], B=ref[b].B, W=ref[b].W, status=np.zeros_like(got[b]["status"])) for b in range(len(ref))]
    errs = GH.compare(got, refs, blocks=blocks, floors={"W1": 1e-2, "W2": 1e-2, "W3": 1e-2})
    dm = abs(_mass(blocks, [g["U"] for g in got]) / m0 - 1)
    divs = []
    for b, g in zip(blocks, got):
        div = O.divb(b.n, b.ng, b.dx, g["B"])
        divs.append(np.max(np.abs(H.interior(div, b.n, b.ng))) * min(b.dx) / max(np.max(np.abs(f)) for f in g["B"]))
    mis = _face_mismatch(blocks, got, records)
    print(f"two-level GPU driver, 2 RK3 steps: max err vs oracle "
          f"{max(v for k, v in errs.items() if k != 'status_mismatch'):.2e}, mass change {dm:.2e}, "
          f"max div B {max(divs):.2e}, level faces {mis:.2e}")
    assert errs.pop("status_mismatch") == 0
    assert max(errs.values()) < 1e-12, errs
    assert dm < 1e-14 and max(divs) < 1e-14 and mis < 1e-13
