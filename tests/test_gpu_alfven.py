"""The circularly polarised SRMHD Alfven wave (an exact nonlinear solution; tests/test_oracle_alfven.py
derives it) through the GPU RK driver, FP64 and mixed precision: the GPU converges to the exact solution
at second order like the oracle, and its FP64 errors equal the oracle's errors (the FP64 path follows the
oracle's arithmetic), while the mixed path's errors stay within a few percent of them (its FP32 flux
rounding is far below the truncation error at these resolutions)."""
import numpy as np
import pytest

from paper_2311_04989_gb300 import grstage as G
from paper_2311_04989_gb300 import inputs as I
from tests import gpu_harness as GH
from tests import test_oracle_alfven as A
from tests.test_gpu_driver import Run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()


def gpu_errors(nx, t_end, precision):
    import oracle as O
    bi, xc = A.wave_block(nx)
    P = O.Params(gamma_ad=A.GAMMA, recon=0, rho_atm=1e-10, tol=1e-14)
    if precision == G.GR_PREC_MIXED:
        P = GH.mixed_params(P)
    run = Run([bi], I.block_grid_neighbours((1, 1, 1)), P)
    try:
        # the same steps as the oracle run: dt = t_end / steps with the grid rule dt = cfl dx
        steps = int(np.ceil(t_end / (0.3 * bi.dx[0])))
        cfl = t_end / steps / bi.dx[0]
        for _ in range(steps):
            run.step(cfl, G.GR_DT_GRID, 3, precision)
        out = run.result()[0]
    finally:
        run.close()
    g, n = bi.ng, bi.n
    by_e, _, uy_e, uz_e = A.exact(xc[g:g + n[0]], t_end)
    by = out["B"][1][g, g, g:g + n[0]]
    uy, uz = out["W"][2][g, g, g:g + n[0]], out["W"][3][g, g, g:g + n[0]]
    assert np.all(out["status"][g:g + n[2], g:g + n[1], g:g + n[0]] == 0)
    return float(np.mean(np.abs(by - by_e))), float(np.mean(np.abs(uy - uy_e)) + np.mean(np.abs(uz - uz_e)))


def test_gpu_alfven_wave_converges_like_the_oracle():
    t_end = 0.5
    ref = [A.errors(nx, t_end) for nx in (32, 64)]
    g64 = [gpu_errors(nx, t_end, G.GR_PREC_FP64) for nx in (32, 64)]
    gmx = [gpu_errors(nx, t_end, G.GR_PREC_MIXED) for nx in (32, 64)]
    print("Alfven wave L1 errors (B^y, u~): oracle", ref, "GPU FP64", g64, "GPU mixed", gmx)
    for r, a, m in zip(ref, g64, gmx):
        for k in range(2):
            assert a[k] == pytest.approx(r[k], rel=1e-9)     # the FP64 path: the oracle's errors
            assert m[k] == pytest.approx(r[k], rel=0.03)     # the mixed path: within 3 %
    for e in (g64, gmx):
        assert e[0][0] / e[1][0] > 3.0 and e[0][1] / e[1][1] > 3.0   # second order
