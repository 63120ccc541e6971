"""Whole-stage pins of the oracle: exact invariants of the discretisation.

* a uniform state is a fixed point, bitwise (flat metric, and a constant curved metric with shift)
* constrained transport keeps div B: div B' = g0 div B0 + g1 div B to round-off (Eq. gausslaw, Sec. 3.3)
* on a plane-parallel problem the corner electric field reduces to the face flux, so the 3D
  face update of B^y equals the 1D conservative update with the x-face induction flux (the
  defining property of the upwinded corner average, reading c9); the plain mean fails it
* periodic blocks conserve D (and S, tau in flat space) to round-off (Eq. claw, Eq. Mb)
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H


def run_stage(bi, P, dt, U=None, U0=None, B0=None, order=2, iters=False):
    if U is None:
        U = H.cons_from_prims(bi, P, order)
    if U0 is None:
        U0 = U
    if B0 is None:
        B0 = bi.B
    return O.stage_block(H.to_oracle(bi), U, U0, B0, dt, P, return_iters=iters)


@pytest.mark.parametrize("recon", [0, 1])
@pytest.mark.parametrize("order", [2, 4])
def test_uniform_state_is_a_fixed_point_bitwise(recon, order):
    g = 4 if order == 4 else 3
    bi = I.uniform_block(n=(6, 5, 4), g=g)
    P = O.Params(gamma_ad=5.0 / 3.0, recon=recon, interp_order=order, rho_atm=1e-10, tol=1e-15)
    U = H.cons_from_prims(bi, P, order)
    Uo, Bo, Wo, st = run_stage(bi, P, 0.05, U=U, order=order)
    n, g = bi.n, bi.ng
    assert np.array_equal(H.interior(Uo, n, g), H.interior(U, n, g))
    for a, b in zip(H.interior_faces(Bo, n, g), H.interior_faces(bi.B, n, g)):
        assert np.array_equal(a, b)
    assert np.all(H.interior(st, n, g) == 0)
    assert np.max(np.abs(H.interior(Wo, n, g) - H.interior(bi.W, n, g))) < 1e-13


def test_uniform_state_in_constant_curved_metric_with_shift():
    m = np.zeros(16)
    m[0] = 0.8; m[1:4] = (0.1, -0.05, 0.2)
    m[4:10] = (1.2, 0.05, -0.03, 0.9, 0.02, 1.1)
    bi = I.uniform_block(n=(5, 5, 5), metric=m)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-10)
    U = H.cons_from_prims(bi, P)
    Uo, Bo, _, _ = run_stage(bi, P, 0.05, U=U)
    n, g = bi.n, bi.ng
    assert np.array_equal(H.interior(Uo, n, g), H.interior(U, n, g))
    for a, b in zip(H.interior_faces(Bo, n, g), H.interior_faces(bi.B, n, g)):
        assert np.array_equal(a, b)


def test_uniform_state_would_change_if_a_flux_term_were_dropped():
    """Guards the fixed-point test: a non-uniform metric breaks the balance, so the update is
    non-zero (the test above is not passing for a trivial reason)."""
    bi = I.random_block(n=(6, 6, 6), seed=5, metric_amp=0.05)
    bi.W[1:4] = 0.0
    bi.W[0] = 1e-3; bi.W[4] = 1e-5
    for b in bi.B:
        b[:] = 0.0
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-12)
    U = H.cons_from_prims(bi, P)
    Uo, _, _, _ = run_stage(bi, P, 0.01, U=U)
    n, g = bi.n, bi.ng
    assert np.max(np.abs(H.interior(Uo - U, n, g)[1:4])) > 0


@pytest.mark.parametrize("recon", [0, 1])
def test_constrained_transport_keeps_div_B(recon):
    bi = I.random_block(n=(8, 8, 8), seed=6, metric_amp=0.02)
    P = O.Params(gamma_ad=2.0, recon=recon, rho_atm=1e-14, rk_g0=0.5, rk_g1=0.5, rk_beta=0.5)
    n, g = bi.n, bi.ng
    d0 = O.divb(n, g, bi.dx, bi.B)
    Bmax = max(np.max(np.abs(b)) for b in bi.B)
    assert np.max(np.abs(H.interior(d0, n, g))) * bi.dx[0] / Bmax < 1e-14
    Uo, Bo, _, st = run_stage(bi, P, 0.2 * bi.dx[0])
    d1 = O.divb(n, g, bi.dx, Bo)
    assert np.max(np.abs(H.interior(d1, n, g))) * bi.dx[0] / Bmax < 1e-14
    # and the field really changed
    assert max(np.max(np.abs(a - b)) for a, b in zip(H.interior_faces(Bo, n, g),
                                                     H.interior_faces(bi.B, n, g))) > 1e-6 * Bmax


def _plane_parallel_By_update(bi, P, dt, Bo):
    """B^y after the stage from the 1D update with the x-face induction flux F^x_{B^y}."""
    n, g = bi.n, bi.ng
    j, k = g, g                            # any column
    W = bi.W[:, k, j, :]                   # (5, Nx)
    Bx = bi.B[0][k, j, :]                  # (Nx+1,)
    Byc = 0.5 * (bi.B[1][k, j, :] + bi.B[1][k, j + 1, :])
    Bzc = 0.5 * (bi.B[2][k, j, :] + bi.B[2][k + 1, j, :])
    rec = [O.recon1d(P.recon, W[v], P.weno_eps) for v in range(5)]
    rby = O.recon1d(P.recon, Byc, P.weno_eps)
    rbz = O.recon1d(P.recon, Bzc, P.weno_eps)
    faces = np.arange(g, g + n[0] + 1)       # array index of x-faces 0..n
    wL = np.stack([rec[v][0][faces] for v in range(5)], 1)
    wR = np.stack([rec[v][1][faces] for v in range(5)], 1)
    BL = np.stack([Bx[faces], rby[0][faces], rbz[0][faces]], 1)
    BR = np.stack([Bx[faces], rby[1][faces], rbz[1][faces]], 1)
    m = np.zeros((len(faces), 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    F = O.face_flux(0, m, wL, BL, wR, BR, P)
    FBy = F[:, 5]
    By0 = bi.B[1][k, j, g:g + n[0]]
    By1 = P.rk_g1 * By0 - P.rk_beta * dt * (FBy[1:] - FBy[:-1]) / bi.dx[0]
    return By1, Bo[1][k, j, g:g + n[0]]


@pytest.mark.parametrize("recon", [0, 1])
def test_plane_parallel_corner_emf_reduces_to_face_flux(recon):
    bi = I.shock_tube_block(n=(16, 4, 4), g=3)
    P = O.Params(gamma_ad=5.0 / 3.0, recon=recon, rho_atm=1e-10, tol=1e-15)
    dt = 0.4 * bi.dx[0]
    Uo, Bo, Wo, st = run_stage(bi, P, dt)
    n, g = bi.n, bi.ng
    # every y-z column identical, bitwise
    Ui = H.interior(Uo, n, g)
    assert np.array_equal(Ui, np.broadcast_to(Ui[:, :1, :1, :], Ui.shape))
    By1, By_stage = _plane_parallel_By_update(bi, P, dt, Bo)
    scale = np.max(np.abs(By1))
    assert np.max(np.abs(By_stage - By1)) < 1e-14 * scale
    # the B^x faces do not change in a plane-parallel problem
    assert np.array_equal(H.interior_faces(Bo, n, g)[0], H.interior_faces(bi.B, n, g)[0])
    # the plain mean of the four face values does not have this property
    Pa = O.Params(gamma_ad=5.0 / 3.0, recon=recon, rho_atm=1e-10, tol=1e-15, emf=1)
    _, Bo_a, _, _ = run_stage(bi, Pa, dt)
    By1a, By_a = _plane_parallel_By_update(bi, Pa, dt, Bo_a)
    assert np.max(np.abs(By_a - By1a)) > 1e-6 * scale


def periodic_block(n=8, seed=7, flat=False, g=3):
    L = 1.0
    bi = I.random_block(n=(n, n, n), g=g, seed=seed, L=L, flat=flat, rho_range=(1e-4, 1e-3),
                        u_max=0.3, theta_range=(1e-2, 1e-1), sigma_range=(1e-2, 1.0))
    H.fill_periodic_cells(bi.W, bi.n, g)
    H.fill_periodic_faces(bi.B, bi.n, g)
    H.fill_periodic_vertices(bi.metric, bi.n, g)
    return bi


@pytest.mark.parametrize("flat", [True, False])
def test_periodic_block_conserves(flat):
    bi = periodic_block(flat=flat)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-12)
    U = H.cons_from_prims(bi, P)
    Uo, Bo, _, st = run_stage(bi, P, 0.2 * bi.dx[0], U=U)
    n, g = bi.n, bi.ng
    assert np.all(H.interior(st, n, g) == 0)
    s0 = H.interior(U, n, g).reshape(5, -1).sum(1)
    s1 = H.interior(Uo, n, g).reshape(5, -1).sum(1)
    scale = np.abs(H.interior(U, n, g)).reshape(5, -1).sum(1)
    assert abs(s1[0] - s0[0]) < 1e-14 * scale[0]
    if flat:
        assert np.all(np.abs(s1 - s0) < 1e-14 * scale)
    d = H.interior(Uo - U, n, g)
    assert np.max(np.abs(d[0])) > 1e-8 * np.max(np.abs(H.interior(U, n, g)[0]))   # it did evolve


def test_operation_counts_split_con2prim_by_kind_of_cell():
    """The counting build of the stage (algorithmic operations per phase, for the rooflines) books the
    con2prim of cells reset to the atmosphere without a root find apart from the cells it solves."""
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=1e-10, tol=1e-12)
    matter = I.uniform_block(n=(4, 4, 4), g=3, rho=1e-3, p=1e-5)
    atm = I.uniform_block(n=(4, 4, 4), g=3, rho=1e-10, u=(0.0, 0.0, 0.0), p=P.K_poly * 1e-20, B=(0.0, 0.0, 0.0))
    for bi, solved in ((matter, True), (atm, False)):
        U = H.cons_from_prims(bi, P)
        c = O.stage_block_count(H.to_oracle(bi), U, U, bi.B, 0.01, P)
        assert set(c) == set(O.PHASES)
        n_solve, n_atm = sum(c["con2prim"]), sum(c["con2prim_atmosphere"])
        assert (n_solve > 0, n_atm == 0) == (solved, solved), (bi is matter, c)
        assert sum(c["faces"]) > 0 and sum(c["update_and_sources"]) > 0
        Uo, Bo, Wo, st = run_stage(bi, P, 0.01, U=U)
        assert bool(np.any(H.interior(st, bi.n, bi.ng) & 1)) != solved
