"""Pins of the oracle's multi-block RK step (ghost exchange, CFL time step, SSP-RK2/RK3 stages).

* a periodic domain split into blocks evolves bitwise like the undivided domain (the ghost exchange
  gives every block exactly the data the undivided stage sees)
* a uniform state stays bitwise uniform, periodic or outflow
* total D is conserved on a periodic domain and div B stays at round-off over RK3 steps
* dt = CFL dx / c_s for a static unmagnetised fluid in flat space (the fast speed is the sound speed)"""
import numpy as np
import pytest

import oracle as O
from oracle import driver as DR
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H


def periodic_global(n=(16, 8, 8), g=3, seed=40):
    # the box is one period of the smooth fields in every direction, so the periodic fill keeps the
    # discrete div B = 0 of the curl-built field
    bi = I.random_block(n=n, g=g, seed=seed, dx=tuple(1.0 / v for v in n), L=1.0, rho_range=(1e-5, 1e-3),
                        fields=I.make_fields(np.random.default_rng(I.SEED_BASE + seed), 1.0, shared_metric=True),
                        metric_amp=0.01, u_max=0.4, sigma_range=(1e-2, 1.0))
    H.fill_periodic_cells(bi.W, n, g)
    H.fill_periodic_faces(bi.B, n, g)
    H.fill_periodic_vertices(bi.metric, n, g)
    return bi


def test_split_domain_evolves_bitwise_like_the_whole_domain():
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14, recon=1)
    whole = periodic_global()
    parts = I.split_block(whole, (2, 1, 1))
    Uw = [H.cons_from_prims(whole, P)]
    Up = [H.cons_from_prims(b, P) for b in parts]
    nbr_w = I.block_grid_neighbours((1, 1, 1))
    nbr_p = I.block_grid_neighbours((2, 1, 1))
    for _ in range(2):
        dtw, _ = DR.rk_step([whole], Uw, nbr_w, P, 0.3, order=3)
        dtp, _ = DR.rk_step(parts, Up, nbr_p, P, 0.3, order=3)
        assert dtw == dtp
    g, n = whole.ng, parts[0].n
    for b, part in enumerate(parts):
        sl = slice(g + b * n[0], g + (b + 1) * n[0])
        assert np.array_equal(H.interior(Up[b], n, g), Uw[0][:, g:g + n[2], g:g + n[1], sl])
        assert np.array_equal(H.interior(part.W, n, g), whole.W[:, g:g + n[2], g:g + n[1], sl])
        assert np.array_equal(part.B[0][g:g + n[2], g:g + n[1], g:g + n[0] + 1],
                              whole.B[0][g:g + n[2], g:g + n[1], g + b * n[0]:g + (b + 1) * n[0] + 1])


@pytest.mark.parametrize("periodic", [True, False])
def test_uniform_state_stays_uniform(periodic):
    bi = I.uniform_block(n=(8, 8, 8), g=3, dx=(0.1,) * 3)
    parts = I.split_block(bi, (2, 2, 1))
    P = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-10, tol=1e-15)
    U = [H.cons_from_prims(b, P) for b in parts]
    U_init = [u.copy() for u in U]
    nbr = I.block_grid_neighbours((2, 2, 1), periodic=(periodic,) * 3)
    for _ in range(2):
        DR.rk_step(parts, U, nbr, P, 0.4, order=2)
    for u, u0, b in zip(U, U_init, parts):
        assert np.array_equal(H.interior(u, b.n, b.ng), H.interior(u0, b.n, b.ng))


def test_mass_conserved_and_divb_at_roundoff_over_rk3_steps():
    P = O.Params(gamma_ad=2.0, rho_atm=1e-14, tol=1e-14, recon=3)
    parts = I.split_block(periodic_global(seed=41), (2, 1, 1))
    U = [H.cons_from_prims(b, P) for b in parts]
    nbr = I.block_grid_neighbours((2, 1, 1))
    mass0 = sum(H.interior(u[0], b.n, b.ng).sum() for u, b in zip(U, parts))
    for _ in range(3):
        dt, st = DR.rk_step(parts, U, nbr, P, 0.3, order=3)
        assert all(np.all(H.interior(s, b.n, b.ng) == 0) for s, b in zip(st, parts))
    mass = sum(H.interior(u[0], b.n, b.ng).sum() for u, b in zip(U, parts))
    assert abs(mass / mass0 - 1) < 1e-14
    for b in parts:
        div = O.divb(b.n, b.ng, b.dx, b.B)
        bmax = max(np.max(np.abs(f)) for f in b.B)
        assert np.max(np.abs(H.interior(div, b.n, b.ng))) * b.dx[0] / bmax < 1e-14


def test_cfl_dt_of_a_static_fluid_is_the_sound_crossing_time():
    rho, p, gam = 0.7, 0.2, 5.0 / 3.0
    bi = I.uniform_block(n=(6, 6, 6), g=3, dx=(0.1, 0.05, 0.2), rho=rho, u=(0, 0, 0), p=p, B=(0, 0, 0))
    P = O.Params(gamma_ad=gam, rho_atm=1e-10)
    h = 1 + gam / (gam - 1) * p / rho
    cs = np.sqrt(gam * p / (rho * h))
    dt = DR.cfl_dt([bi], [bi.W], [bi.B], P, 0.3)
    assert abs(dt / (0.3 * 0.05 / cs) - 1) < 1e-14


@pytest.mark.parametrize("order", [2, 3])
def test_rk_stages_reproduce_the_taylor_polynomial_of_a_linear_ode(order):
    # on u' = lam u an explicit s-stage method of order s = 2, 3 is exactly the degree-s Taylor
    # polynomial of exp(z), z = lam dt (a dropped or misplaced coefficient changes it)
    for z in (-0.7, -0.1, 0.3, 1.2):
        u0, u = 1.0, 1.0
        for g0, g1, beta in DR.RK_STAGES[order]:
            u = g0 * u0 + g1 * u + beta * z * u
        taylor = sum(z ** k / np.prod(range(1, k + 1)) for k in range(order + 1))
        assert abs(u - taylor) < 1e-15


def test_grid_dt_is_the_cfl_factor_times_the_finest_spacing():
    a = I.uniform_block(n=(4, 4, 4), g=3, dx=(0.1, 0.05, 0.2))
    b = I.uniform_block(n=(4, 4, 4), g=3, dx=(0.025, 0.3, 0.1))
    assert DR.grid_dt([a, b], 0.25) == 0.25 * 0.025
