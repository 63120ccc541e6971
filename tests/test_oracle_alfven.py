"""Pin of the oracle's magnetised flux terms by an exact nonlinear solution: the circularly polarised
Alfven wave of special-relativistic MHD.

With uniform rho, p, B^x = B0 and v^x = 0, the transverse field B_t = eta B0 (cos phi, sin phi),
phi = k (x - v_A t), and the transverse velocity v_t = -v_A B_t / B0 solve the ideal SRMHD equations
(the flat-space, alpha = 1, beta = 0 case of Eq. consB_def and Eq. fluxB_def) for any amplitude eta:

* induction: d_t B^y + d_x (v^x B^y - v^y B^x) = -v_A f' + B0 (v_A / B0) f' = 0 for B^y = f(x - v_A t);
* x-momentum, energy and mass: their fluxes are uniform (v^x = 0, |B_t|, |v_t|, W constant);
* y-momentum: S_y = (rho h + b^2) W^2 v_y - b^0 b_y and its flux T^xy = -b^x b^y are both multiples of
  B^y, with b^0 = W (B.v) = -W v_A eta^2 B0, b^x = B0 / W, b^y = B^y (1/W + W v_A^2 eta^2),
  b^2 = B0^2 (1 + eta^2 - v_A^2 eta^2) and W^2 = 1 / (1 - v_A^2 eta^2); d_t S_y + d_x T^xy = 0 then
  reduces to (rho h + b^2) v_A^2 = B0^2, i.e. eta^2 B0^2 x^2 - (rho h + B0^2 (1 + eta^2)) x + B0^2 = 0 for
  x = v_A^2 (the smaller root; it tends to the Alfven speed B0^2 / (rho h + B0^2) as eta -> 0).

(This derivation is written out here; the paper does not print the wave.)  A dropped or sign-flipped
b^0 b_j or b^i b^j term in the oracle's fluxes, or a wrong b^2, changes the propagation speed or the
transverse coupling, so the error would not converge.  The test runs the oracle's stage with SSP-RK3
on a periodic box of one wavelength at three resolutions and checks that the error of B^y and of the
transverse velocity against the exact solution falls at second order (PLM), and is small."""
import numpy as np
import pytest

import oracle as O
from oracle import driver as DR
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H

RHO, P_GAS, B0, ETA, GAMMA = 1.0, 1.0, 1.0, 1.0, 5.0 / 3.0


def alfven_speed(rho=RHO, p=P_GAS, b0=B0, eta=ETA, gamma=GAMMA):
    h = 1.0 + gamma / (gamma - 1.0) * p / rho
    a = rho * h + b0 ** 2 * (1.0 + eta ** 2)
    x = 2.0 * b0 ** 2 / (a + np.sqrt(a * a - 4.0 * eta ** 2 * b0 ** 4))
    return np.sqrt(x)


def exact(x, t):
    """(B^y, B^z, u~^y, u~^z) of the wave at positions x, time t (wavelength 1)."""
    va = alfven_speed()
    ph = 2.0 * np.pi * (x - va * t)
    by, bz = ETA * B0 * np.cos(ph), ETA * B0 * np.sin(ph)
    w = 1.0 / np.sqrt(1.0 - va ** 2 * ETA ** 2)
    return by, bz, -w * va * by / B0, -w * va * bz / B0


def wave_block(nx, g=3, nt=4):
    """One wavelength along x (nx cells), nt cells along y and z (a 1D problem, periodic)."""
    n = (nx, nt, nt)
    dx = 1.0 / nx
    N = [v + 2 * g for v in n]
    xc = (np.arange(N[0]) - g + 0.5) * dx       # cell centres (and y-, z-face centres) along x
    by, bz, uy, uz = exact(xc, 0.0)
    W = np.zeros((5, N[2], N[1], N[0]))
    W[0] = RHO
    W[2] = uy[None, None, :]
    W[3] = uz[None, None, :]
    W[4] = P_GAS
    Bx = np.full((N[2], N[1], N[0] + 1), B0)
    By = np.broadcast_to(by[None, None, :], (N[2], N[1] + 1, N[0])).copy()
    Bz = np.broadcast_to(bz[None, None, :], (N[2] + 1, N[1], N[0])).copy()
    return I.BlockInput(n, g, (0.0, 0.0, 0.0), (dx, dx, dx), I.metric_flat(n, g), W, [Bx, By, Bz]), xc


def evolve(nx, t_end, cfl=0.3, recon=0):
    bi, xc = wave_block(nx)
    n, g = bi.n, bi.ng
    P = O.Params(gamma_ad=GAMMA, recon=recon, rho_atm=1e-10, tol=1e-14)
    U = H.cons_from_prims(bi, P)
    steps = int(np.ceil(t_end / (cfl * bi.dx[0])))
    dt = t_end / steps
    for _ in range(steps):
        U0 = U.copy()
        B0f = [f.copy() for f in bi.B]
        for g0, g1, beta in DR.RK_STAGES[3]:
            H.fill_periodic_cells(bi.W, n, g)
            H.fill_periodic_faces(bi.B, n, g)
            Pst = O.Params(**{**P.__dict__, "rk_g0": g0, "rk_g1": g1, "rk_beta": beta})
            blk = O.Block(n, g, bi.dx, bi.metric, bi.W, bi.B)
            Uo, Bo, Wo, st = O.stage_block(blk, U, U0, B0f, dt, Pst)
            assert np.all(H.interior(st, n, g) == 0)
            U[...] = Uo
            bi.W[...] = Wo
            for d in range(3):
                bi.B[d][...] = Bo[d]
    return bi, xc


def errors(nx, t_end):
    bi, xc = evolve(nx, t_end)
    g, n = bi.ng, bi.n
    by_e, bz_e, uy_e, uz_e = exact(xc[g:g + n[0]], t_end)
    by = bi.B[1][g:g + n[2], g:g + n[1], g:g + n[0]]
    uy = bi.W[2][g:g + n[2], g:g + n[1], g:g + n[0]]
    uz = bi.W[3][g:g + n[2], g:g + n[1], g:g + n[0]]
    # the problem is 1D: every (y, z) row carries the same solution
    assert np.max(np.abs(by - by[0:1, 0:1, :])) < 1e-12
    eb = float(np.mean(np.abs(by[0, 0] - by_e)))
    eu = float(np.mean(np.abs(uy[0, 0] - uy_e)) + np.mean(np.abs(uz[0, 0] - uz_e)))
    return eb, eu


def test_alfven_speed_is_the_root_of_the_momentum_balance():
    """The quadratic's root satisfies (rho h + b^2) v_A^2 = B0^2 and reduces to the linear Alfven speed."""
    va = alfven_speed()
    h = 1.0 + GAMMA / (GAMMA - 1.0) * P_GAS / RHO
    b2 = B0 ** 2 * (1.0 + ETA ** 2 - va ** 2 * ETA ** 2)
    assert (RHO * h + b2) * va ** 2 == pytest.approx(B0 ** 2, rel=1e-14)
    small = alfven_speed(eta=1e-6)
    assert small ** 2 == pytest.approx(B0 ** 2 / (RHO * h + B0 ** 2), rel=1e-10)
    assert 0.0 < va < 1.0


def test_alfven_wave_converges_to_the_exact_solution():
    t_end = 0.5
    res = [errors(nx, t_end) for nx in (16, 32, 64)]
    eb = [r[0] for r in res]
    eu = [r[1] for r in res]
    print("circularly polarised Alfven wave, L1 errors of B^y:", eb, "of u~^y + u~^z:", eu)
    # second order (PLM with RK3): each halving of dx cuts the error by ~4
    for k in range(2):
        assert eb[k] / eb[k + 1] > 3.0, eb
        assert eu[k] / eu[k + 1] > 3.0, eu
    assert eb[-1] < 2e-2 * ETA * B0 and eu[-1] < 2e-2
