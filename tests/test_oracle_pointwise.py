"""Pins of the oracle's pointwise physics against closed forms and 4D-covariant identities.

Eq. consB_def, Eq. fluxB_def, Eq. EMT_MHD, Eq. hydsrc_def (Sec. 2); wave speeds (Sec. 2.2, reading c2);
HLLE (reading c1); con2prim with the App. A policy (Sec. 3.5, App. A)."""
import numpy as np
import pytest

import oracle as O
from tests import fourd

GAMMA = 2.0


def random_metric(rng, n, amp=0.2, K=False):
    m = np.zeros((n, 16))
    m[:, 0] = 1 + amp * rng.uniform(-1, 1, n)
    m[:, 1:4] = amp * rng.uniform(-1, 1, (n, 3))
    for c, (i, j) in enumerate(fourd.SYM):
        m[:, 4 + c] = (1.0 if i == j else 0.0) + amp * rng.uniform(-0.5, 0.5, n)
    if K:
        m[:, 10:16] = amp * rng.uniform(-1, 1, (n, 6))
    return m


def random_prims(rng, n, umax=2.0, rho=(1e-6, 1e-2), theta=(1e-3, 1.0)):
    w = np.zeros((n, 5))
    w[:, 0] = np.exp(rng.uniform(np.log(rho[0]), np.log(rho[1]), n))
    w[:, 1:4] = rng.uniform(-umax, umax, (n, 3))
    w[:, 4] = w[:, 0] * np.exp(rng.uniform(np.log(theta[0]), np.log(theta[1]), n))
    return w


def random_B(rng, w, sigma=(1e-3, 10.0)):
    n = w.shape[0]
    s = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), n))
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * np.sqrt(s * w[:, 4])[:, None]


def rel(a, b, floor):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


# ------------------------------------------------------------------------------------------
# prim -> cons
# ------------------------------------------------------------------------------------------
def test_p2c_fluid_at_rest_closed_form():
    """v = 0, B = 0:  D = sqrt(gamma) rho, S = 0, tau = sqrt(gamma) rho eps (Eq. cons_def)."""
    rng = np.random.default_rng(1)
    m = random_metric(rng, 50)
    w = random_prims(rng, 50)
    w[:, 1:4] = 0
    P = O.Params(gamma_ad=GAMMA)
    q = O.prim2con(m, w, np.zeros((50, 3)), P)
    sg = np.array([np.sqrt(np.linalg.det(fourd.unpack(x)[2])) for x in m])
    eps = w[:, 4] / ((GAMMA - 1) * w[:, 0])
    assert rel(q[:, 0], sg * w[:, 0], 1e-300) < 1e-14
    assert np.max(np.abs(q[:, 1:4])) == 0.0
    assert rel(q[:, 4], sg * w[:, 0] * eps, 1e-300) < 1e-13


def test_p2c_flat_special_relativistic_mhd():
    """Flat metric: S_i = (rho h W^2 + B^2) v_i - (B.v) B_i,
    tau = rho h W^2 - p - rho W + B^2 (1 + v^2)/2 - (B.v)^2/2 (textbook SRMHD)."""
    rng = np.random.default_rng(2)
    n = 200
    m = np.zeros((n, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    q = O.prim2con(m, w, B, P)
    ut = w[:, 1:4]
    W = np.sqrt(1 + np.sum(ut * ut, 1))
    v = ut / W[:, None]
    h = 1 + w[:, 4] / ((GAMMA - 1) * w[:, 0]) + w[:, 4] / w[:, 0]
    Bv = np.sum(B * v, 1); B2 = np.sum(B * B, 1); v2 = np.sum(v * v, 1)
    S = (w[:, 0] * h * W ** 2 + B2)[:, None] * v - Bv[:, None] * B
    tau = w[:, 0] * h * W ** 2 - w[:, 4] - w[:, 0] * W + 0.5 * B2 * (1 + v2) - 0.5 * Bv ** 2
    assert rel(q[:, 0], w[:, 0] * W, 1e-300) < 1e-14
    scale = np.max(np.abs(S))
    assert np.max(np.abs(q[:, 1:4] - S)) < 1e-12 * scale
    assert rel(q[:, 4], tau, 1e-30) < 1e-11


def test_p2c_matches_covariant_stress_tensor():
    """General metric with shift: D, S_j, tau from the 4D stress tensor of Eq. EMT_MHD."""
    rng = np.random.default_rng(3)
    n = 100
    m = random_metric(rng, n)
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    q = O.prim2con(m, w, B, P)
    ref = np.array([fourd.cons(fourd.state(m[k], w[k], B[k], GAMMA)) for k in range(n)])
    for c in range(5):
        assert rel(q[:, c], ref[:, c], 1e-12 * np.max(np.abs(ref[:, c]))) < 1e-10, c


# ------------------------------------------------------------------------------------------
# fluxes, speeds, HLLE
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_matches_covariant_form(d):
    rng = np.random.default_rng(10 + d)
    n = 100
    m = random_metric(rng, n)
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    U, F, lam = O.flux_points(d, m, w, B, P)
    ref = np.array([fourd.flux(fourd.state(m[k], w[k], B[k], GAMMA), d) for k in range(n)])
    for c in range(7):
        scale = np.max(np.abs(ref[:, c]))
        assert np.max(np.abs(F[:, c] - ref[:, c])) < 1e-11 * scale, c


@pytest.mark.parametrize("d", [0, 1, 2])
def test_speeds_match_covariant_dispersion_relation(d):
    rng = np.random.default_rng(20 + d)
    n = 100
    m = random_metric(rng, n)
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    _, _, lam = O.flux_points(d, m, w, B, P)
    ref = np.array([fourd.speeds(fourd.state(m[k], w[k], B[k], GAMMA), d, GAMMA) for k in range(n)])
    assert np.max(np.abs(lam - ref)) < 1e-9


def test_speeds_flat_relativistic_velocity_addition():
    """Flat metric, motion along x, B = 0: lam = (v -+ c_s)/(1 -+ v c_s)."""
    P = O.Params(gamma_ad=5.0 / 3.0)
    n = 20
    m = np.zeros((n, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    w = np.zeros((n, 5)); w[:, 0] = 1.0; w[:, 4] = np.linspace(0.01, 10, n)
    ut = np.linspace(-3, 3, n)
    w[:, 1] = ut
    _, _, lam = O.flux_points(0, m, w, np.zeros((n, 3)), P)
    v = ut / np.sqrt(1 + ut ** 2)
    eps = w[:, 4] / ((P.gamma_ad - 1) * w[:, 0])
    h = 1 + eps + w[:, 4] / w[:, 0]
    cs = np.sqrt(P.gamma_ad * w[:, 4] / (w[:, 0] * h))
    assert np.allclose(lam[:, 0], (v - cs) / (1 - v * cs), rtol=1e-13, atol=1e-15)
    assert np.allclose(lam[:, 1], (v + cs) / (1 + v * cs), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlle_consistency(d):
    """F_HLLE(U, U) = F(U)."""
    rng = np.random.default_rng(30 + d)
    n = 100
    m = random_metric(rng, n)
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    _, F, _ = O.flux_points(d, m, w, B, P)
    Fh = O.face_flux(d, m, w, B, w, B, P)
    for c in range(7):
        scale = np.max(np.abs(F[:, c]))
        assert np.max(np.abs(Fh[:, c] - F[:, c])) < 1e-13 * scale, c


def test_hlle_supersonic_states_take_upwind_flux():
    """All speeds of both states positive -> F = F_L; all negative -> F = F_R."""
    P = O.Params(gamma_ad=GAMMA)
    n = 10
    m = np.zeros((n, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    rng = np.random.default_rng(40)
    wL = random_prims(rng, n, umax=0.0, theta=(1e-4, 1e-3)); wL[:, 1] = 30.0
    wR = random_prims(rng, n, umax=0.0, theta=(1e-4, 1e-3)); wR[:, 1] = 25.0
    B = np.zeros((n, 3))
    _, FL, lamL = O.flux_points(0, m, wL, B, P)
    _, FR, lamR = O.flux_points(0, m, wR, B, P)
    assert np.all(lamL[:, 0] > 0) and np.all(lamR[:, 0] > 0)
    Fh = O.face_flux(0, m, wL, B, wR, B, P)
    assert np.max(np.abs(Fh - FL) / np.maximum(np.abs(FL), 1e-300)) < 1e-14
    wL[:, 1] *= -1; wR[:, 1] *= -1
    _, FR, _ = O.flux_points(0, m, wR, B, P)
    Fh = O.face_flux(0, m, wL, B, wR, B, P)
    assert np.max(np.abs(Fh - FR) / np.maximum(np.abs(FR), 1e-300)) < 1e-14


# ------------------------------------------------------------------------------------------
# sources
# ------------------------------------------------------------------------------------------
def test_sources_match_covariant_form_stationary_metric():
    """Eq. hydsrc_def against (1/2) alpha sqrt(gamma) T^{mu nu} d_j g_{mu nu} and the energy
    source with Gamma^0_{mu nu}, for a stationary metric whose K_ij follows from the shift."""
    rng = np.random.default_rng(50)
    n = 60
    m = random_metric(rng, n)
    dm = np.zeros((n, 3, 16))
    dm[:, :, :10] = 0.3 * rng.uniform(-1, 1, (n, 3, 10))
    for k in range(n):
        K = fourd.stationary_K(m[k], dm[k])
        for c, (i, j) in enumerate(fourd.SYM):
            m[k, 10 + c] = K[i, j]
    w = random_prims(rng, n)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA)
    s = O.sources(m, dm, w, B, P)
    ref = np.array([fourd.sources_stationary(fourd.state(m[k], w[k], B[k], GAMMA), dm[k]) for k in range(n)])
    assert np.all(s[:, 0] == 0)
    for c in range(1, 5):
        scale = np.max(np.abs(ref[:, c]))
        assert np.max(np.abs(s[:, c] - ref[:, c])) < 1e-10 * scale, c


def test_sources_vanish_in_flat_space():
    rng = np.random.default_rng(51)
    n = 20
    m = np.zeros((n, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    w = random_prims(rng, n); B = random_B(rng, w)
    s = O.sources(m, np.zeros((n, 3, 16)), w, B, O.Params(gamma_ad=GAMMA))
    assert np.all(s == 0)


# ------------------------------------------------------------------------------------------
# con2prim
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("umax", [1.0, 30.0])
@pytest.mark.parametrize("tol", [1e-10, 1e-15])
def test_con2prim_round_trip(umax, tol):
    """prim -> cons -> prim on magnetised states in a curved metric with shift.  The relative
    error in rho is bounded by the bracket tolerance times W^2 (rho = D/W with v^2 = mu^2 rbar^2);
    at a tight tolerance it is within the 1e-10 that App. A reports for all but W ~ 1e3."""
    rng = np.random.default_rng(60)
    n = 2000
    m = random_metric(rng, n, amp=0.1)
    w = random_prims(rng, n, umax=umax, rho=(1e-12, 1e-2))
    B = random_B(rng, w, sigma=(1e-4, 100.0))
    P = O.Params(gamma_ad=GAMMA, rho_atm=1e-20, W_max=1e4, M_max=1e8, tol=tol)
    q = O.prim2con(m, w, B, P)
    w2, q2, st, it = O.con2prim(m, q, B, P)
    assert np.all(st == 0)
    assert np.all(q2 == q)
    W = np.array([np.sqrt(1 + w[k, 1:4] @ fourd.unpack(m[k])[2] @ w[k, 1:4]) for k in range(n)])
    bound = 2 * tol * W ** 2 + 1e-10
    erho = np.abs(w2[:, 0] - w[:, 0]) / w[:, 0]
    assert np.all(erho < bound)
    if tol < 1e-14:
        assert erho.max() < 1e-10
        assert rel(w2[:, 4], w[:, 4], 1e-300) < 1e-8
    u = np.linalg.norm(w[:, 1:4], axis=1)
    for c in range(1, 4):
        assert np.max(np.abs(w2[:, c] - w[:, c]) / np.maximum(u, 1e-3)) < 2 * tol * W.max() ** 2 + 1e-10
    assert it.max() < 30


def test_con2prim_tight_tolerance_reaches_round_off():
    rng = np.random.default_rng(61)
    n = 500
    m = random_metric(rng, n, amp=0.1)
    w = random_prims(rng, n, umax=3.0)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA, rho_atm=1e-20, tol=1e-15)
    q = O.prim2con(m, w, B, P)
    w2, _, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st == 0)
    assert rel(w2[:, 0], w[:, 0], 1e-300) < 1e-13


def test_con2prim_atmosphere_threshold_resets_and_recomputes_cons():
    """D below f_thr rho_atm -> atmosphere prims and cons recomputed from them (Sec. 3.5)."""
    rng = np.random.default_rng(62)
    n = 20
    m = random_metric(rng, n, amp=0.1)
    w = random_prims(rng, n, rho=(1e-16, 1e-15))
    B = random_B(rng, w)
    P = O.Params(gamma_ad=GAMMA, rho_atm=1e-13, p_atm=1e-24)
    q = O.prim2con(m, w, B, P)
    w2, q2, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st & 1)
    assert np.all(w2[:, 0] == 1e-13) and np.all(w2[:, 1:4] == 0) and np.all(w2[:, 4] == 1e-24)
    qa = O.prim2con(m, w2, B, P)
    assert np.array_equal(q2, qa)


def test_con2prim_nan_is_a_failure_status():
    m = np.zeros((2, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    q = np.array([[np.nan, 0, 0, 0, 1.0], [1.0, np.inf, 0, 0, 1.0]])
    P = O.Params(gamma_ad=GAMMA)
    w, q2, st, _ = O.con2prim(m, q, np.zeros((2, 3)), P)
    assert np.all(st & 2)
    assert np.all(np.isfinite(q2)) and np.all(w[:, 0] == P.rho_atm)


def test_con2prim_tau_floor_and_B_over_D_limit():
    """tau below the cold static value B^2/2 is raised to it (status 8); B^2/D above M_max
    rescales D (status 16) (App. A)."""
    P = O.Params(gamma_ad=GAMMA, rho_atm=1e-20, M_max=100.0)
    m = np.zeros((2, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    B = np.array([[0.1, 0, 0], [1.0, 0.0, 0.0]])
    q = np.array([[1.0, 0, 0, 0, 0.001], [1e-4, 0, 0, 0, 1.0]])
    w, q2, st, _ = O.con2prim(m, q, B, P)
    assert st[0] & 8 and q2[0, 4] == pytest.approx(0.5 * 0.1 ** 2, rel=1e-15)
    assert st[1] & 16 and q2[1, 0] == pytest.approx(1.0 / 100.0, rel=1e-15)


def test_con2prim_lorentz_factor_clamp():
    """W above W_max is reset to W_max (status 4) without touching the conserved variables."""
    rng = np.random.default_rng(63)
    n = 50
    m = random_metric(rng, n, amp=0.05)
    w = random_prims(rng, n, umax=0.0, theta=(1e-3, 1e-2))
    w[:, 1] = 100.0
    B = np.zeros((n, 3))
    P = O.Params(gamma_ad=GAMMA, rho_atm=1e-20)
    q = O.prim2con(m, w, B, P)
    w2, q2, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st & 4)
    assert np.array_equal(q2, q)
    W = np.array([np.sqrt(1 + w2[k, 1:4] @ fourd.unpack(m[k])[2] @ w2[k, 1:4]) for k in range(n)])
    assert np.allclose(W, P.W_max, rtol=1e-12)
    P2 = O.Params(gamma_ad=GAMMA, rho_atm=1e-20, ceiling=1)
    w3, q3, st3, _ = O.con2prim(m, q, B, P2)
    assert np.all(st3 & 4) and np.all(w3[:, 0] == P2.rho_atm)


def test_con2prim_cells_at_the_atmosphere_density_are_reset_deterministically():
    """Sec. 3.5 resets a cell whose density falls below f_thr rho_atm.  At the default band (1e-12)
    cells equal to the threshold up to FP64 rounding take the atmosphere branch and every cell above
    it by more than that is solved (1 + 1e-9 included); a wider band, passed as a parameter (the mixed
    path's FP32 sqrt(gamma) classification tolerance, 1e-6), takes the cells within it too."""
    n = 7
    m = np.zeros((n, 16)); m[:, 0] = 1; m[:, 4] = m[:, 7] = m[:, 9] = 1
    w = np.zeros((n, 5))
    w[:, 0] = 1e-13 * np.array([1 - 1e-15, 1.0, 1 + 1e-15, 1 + 1e-9, 1 + 5e-7, 1 + 1e-5, 2.0])
    w[:, 4] = 1e-24
    for band, expect in ((None, [1, 1, 1, 0, 0, 0, 0]), (1e-6, [1, 1, 1, 1, 1, 0, 0])):
        P = O.Params(gamma_ad=GAMMA, rho_atm=1e-13, p_atm=1e-24)
        if band is not None:
            P.atm_band = band
        q = O.prim2con(m, w, np.zeros((n, 3)), P)
        w2, q2, st, _ = O.con2prim(m, q, np.zeros((n, 3)), P)
        assert list(st & 1) == expect, (band, st)
        k = int(np.sum(expect))
        assert np.all(w2[:k, 4] == 1e-24) and np.all(w2[:k, 0] == 1e-13)
        # solved cells keep their density (flat metric, at rest: rho = D exactly up to the solve)
        assert np.allclose(w2[k:, 0], w[k:, 0], rtol=1e-12, atol=0)
