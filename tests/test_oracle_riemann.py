"""The oracle's stage converges to the exact solution of a relativistic shock tube (flat metric,
B = 0, Gamma = 5/3), the hydrodynamic part of the 1D shock-tube workload."""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H
from tests import riemann_exact as R


def test_exact_solver_satisfies_jump_conditions():
    """Rankine-Hugoniot [F] = V_s [U] across the right shock of the exact solution."""
    G = 5.0 / 3.0
    left, right = (1.0, 1.0, 0.0), (0.125, 0.1, 0.0)
    sol = R.solve(G, left, right)
    gas = R.Gas(G)
    rs, vs, Vs = R._shock(gas, *right, sol.p_star, +1)

    def UF(rho, p, v):
        W = 1 / np.sqrt(1 - v * v); h = gas.h(rho, p)
        U = np.array([rho * W, rho * h * W * W * v, rho * h * W * W - p - rho * W])
        F = np.array([rho * W * v, rho * h * W * W * v * v + p, rho * h * W * W * v - rho * W * v])
        return U, F
    Ua, Fa = UF(*right)
    Ub, Fb = UF(rs, sol.p_star, vs)
    assert np.allclose(Fb - Fa, Vs * (Ub - Ua), rtol=1e-10, atol=1e-12)
    assert abs(vs - sol.v_star) < 1e-12


def run_tube(N, recon, tend=0.4):
    G = 5.0 / 3.0
    bi = I.shock_tube_block(n=(N, 1, 1), g=3, left=(1.0, 1.0, 0.0), right=(0.125, 0.1, 0.0), Bx=0.0)
    P = O.Params(gamma_ad=G, recon=recon, rho_atm=1e-12, p_atm=1e-14)
    dx = bi.dx[0]
    dt = 0.4 * dx
    nsteps = int(round(tend / dt))
    U, bi = H.evolve(bi, P, dt, nsteps, H.fill_outflow_x_periodic_yz)
    g = bi.ng
    rho = bi.W[0, g, g, g:g + N]
    x = -0.5 + (np.arange(N) + 0.5) * dx
    sol = R.solve(G, (1.0, 1.0, 0.0), (0.125, 0.1, 0.0))
    ex = np.array([sol(xi / (nsteps * dt))[0] for xi in x])
    return np.mean(np.abs(rho - ex))


@pytest.mark.parametrize("recon", [0, 1])
def test_shock_tube_converges_to_exact_solution(recon):
    e = [run_tube(N, recon) for N in (32, 64, 128)]
    order = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert e[-1] < 0.01
    assert np.all(order > 0.5), (e, order)
