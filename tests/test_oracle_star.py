"""Static polytropic star (K = 100, Gamma = 2, rho_c = 1.28e-3; Sec. 4.1) in its own fixed isotropic
TOV metric: the flux divergence and the geometric sources of Eq. hydsrc_def balance, so the stage's
right-hand side in the star interior vanishes at second order in the grid spacing.  A dropped or
mis-signed source term leaves an O(1) residual."""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H


@pytest.fixture(scope="module")
def tov():
    return I.solve_tov()


def residual(tov, n, recon):
    bi = I.star_block(n=(n, n, n), g=3, half_width=10.02, tov=tov)
    P = O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-13 * tov.rho[0])
    U = H.cons_from_prims(bi, P)
    dt = 1e-3
    Uo, _, _, st = O.stage_block(H.to_oracle(bi), U, U, bi.B, dt, P)
    L = (H.interior(Uo, bi.n, 3) - H.interior(U, bi.n, 3)) / dt
    X, Y, Z = I.grid(bi.n, 0, bi.x0, bi.dx)
    inside = np.sqrt(X ** 2 + Y ** 2 + Z ** 2) < 0.6 * tov.R_iso
    return np.mean(np.abs(L[1:4][:, inside])), np.mean(np.abs(L[0][inside]))


def test_tov_solution_matches_the_paper_model(tov):
    """Gravitational mass 1.400 (Sec. 4.1) for rho_c = 1.28e-3, K = 100, Gamma = 2."""
    assert abs(tov.M - 1.400) < 2e-3


@pytest.mark.parametrize("recon", [0, 1])
def test_static_star_residual_converges_at_second_order(tov, recon):
    rS32, rD32 = residual(tov, 32, recon)
    rS48, rD48 = residual(tov, 48, recon)
    order = np.log(rS32 / rS48) / np.log(1.5)
    assert order > 1.7, order
    assert np.log(rD32 / rD48) / np.log(1.5) > 1.5
