"""Pins of the oracle's tabulated EOS (Sec. 2.2.1; App. A for the nested temperature root and the
error policy).

* trilinear interpolation in (log rho, log T, Y_e) reproduces a function that is trilinear in those
  variables exactly, and the temperature recovered from (rho, p, Y_e) is exact for it
* on the synthetic table the interpolant equals the sampled EOS at the nodes and converges at
  second order between them
* a table of the Gamma = 5/3 ideal gas (p = rho T, eps = 3T/2) gives the ideal-gas con2prim and
  the ideal-gas stage, to the table's interpolation error: this ties the table path to the
  independently pinned ideal-gas path
* prim -> cons -> prim round trips; the conserved variables of the recovered state reproduce the
  input; Y_e is carried as D Y_e; the temperature floor, the Y_e clamp and the atmosphere
  follow App. A
* in a stage, a uniform Y_e stays uniform and the total D Y_e is conserved on a periodic block"""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I
from tests import helpers as H
from tests.test_oracle_pointwise import random_metric, random_B


class _Tab:
    """A table object with given node arrays (same attributes as inputs.EosTable)."""
    def __init__(self, n, x0, dx, lp, le, cs2):
        self.n, self.x0, self.dx, self.lp, self.le, self.cs2 = n, x0, dx, lp, le, cs2


def _axes(n, x0, dx):
    return [x0[a] + dx[a] * np.arange(n[a]) for a in range(3)]


def trilinear_table(rng):
    """log p, log e, c_s^2 trilinear in (log rho, log T, Y_e), log p and log e increasing in log T."""
    n, x0, dx = (7, 9, 5), (np.log(1e-10), np.log(1e-5), 0.05), (2.0, 0.7, 0.1)
    lr, lT, ye = _axes(n, x0, dx)
    Y, T, R = np.meshgrid(ye, lT, lr, indexing="ij")

    def f(c):
        return (c[0] + c[1] * R + c[2] * T + c[3] * Y + c[4] * R * T + c[5] * R * Y + c[6] * T * Y
                + c[7] * R * T * Y)
    cp = np.array([1.0, 1.0, 2.0, 0.3, 0.01, 0.05, 0.1, 0.002])
    ce = np.array([1.0, 1.0, 0.02, 0.1, 0.0005, 0.001, 0.002, 0.0001])   # e > rho: eps well conditioned
    cc = np.array([0.2, 0.001, 0.01, 0.05, 0.0, 0.001, 0.002, 0.0])
    return _Tab(n, x0, dx, f(cp), f(ce), f(cc)), (cp, ce, cc)


def test_trilinear_function_is_reproduced_and_inverted_exactly():
    rng = np.random.default_rng(0)
    tab, (cp, ce, cc) = trilinear_table(rng)
    P = O.Params(table=tab)
    m = 500
    lo = [tab.x0[a] for a in range(3)]
    hi = [tab.x0[a] + (tab.n[a] - 1) * tab.dx[a] for a in range(3)]
    R, T, Y = (rng.uniform(lo[a], hi[a], m) for a in range(3))
    p, eps, cs2, Tr = O.table_eval(P, np.exp(R), np.exp(T), Y)

    def f(c):
        return (c[0] + c[1] * R + c[2] * T + c[3] * Y + c[4] * R * T + c[5] * R * Y + c[6] * T * Y
                + c[7] * R * T * Y)
    assert np.max(np.abs(np.log(p) - f(cp))) < 1e-12
    assert np.max(np.abs(np.log(np.exp(R) * (1 + eps)) - f(ce))) < 1e-12
    assert np.max(np.abs(cs2 - f(cc))) < 1e-13
    assert np.max(np.abs(np.log(Tr) - T)) < 1e-12


def test_synthetic_table_matches_its_eos_at_nodes_and_converges_at_second_order():
    eos = I.SyntheticEOS()
    rng = np.random.default_rng(1)
    errs = []
    for k, n in enumerate([(20, 16, 4), (39, 31, 7)]):
        tab = eos.table(n=n, rho_range=(1e-12, 1e-2), T_range=(1e-5, 1e-1), ye_range=(0.05, 0.55))
        P = O.Params(table=tab)
        if k == 0:   # nodes
            lr, lT, ye = _axes(tab.n, tab.x0, tab.dx)
            R = np.exp(lr[rng.integers(0, n[0], 50)]); T = np.exp(lT[rng.integers(0, n[1], 50)])
            Y = ye[rng.integers(0, n[2], 50)]
            p, eps, cs2, _ = O.table_eval(P, R, T, Y)
            assert np.max(np.abs(p / eos.p(R, T, Y) - 1)) < 1e-13
            e_true = R * (1 + eos.eps(R, T, Y))
            assert np.max(np.abs(R * (1 + eps) / e_true - 1)) < 1e-13    # e, not eps: e/rho - 1 cancels
            assert np.max(np.abs(cs2 - eos.cs2(R, T, Y))) < 1e-15
        pts = np.random.default_rng(2)
        R = np.exp(pts.uniform(np.log(2e-12), np.log(5e-3), 2000))
        T = np.exp(pts.uniform(np.log(2e-5), np.log(5e-2), 2000))
        Y = pts.uniform(0.1, 0.5, 2000)
        p, _, _, _ = O.table_eval(P, R, T, Y)
        errs.append(np.max(np.abs(np.log(p / eos.p(R, T, Y)))))
    assert 3.0 < errs[0] / errs[1] < 5.0, errs     # halving the spacing: ~4x smaller


def ideal_gas_table(nT=4000):
    """p = rho T, eps = 3T/2: the Gamma = 5/3 ideal gas as a table.  log p and log e are linear in
    log rho, so only the T direction carries interpolation error."""
    n, x0 = (3, nT, 2), (np.log(1e-16), np.log(1e-5), 0.0)
    dx = ((np.log(10.0) - x0[0]) / (n[0] - 1), (np.log(20.0) - x0[1]) / (n[1] - 1), 1.0)
    lr, lT, ye = _axes(n, x0, dx)
    Y, T, R = np.meshgrid(ye, np.exp(lT), np.exp(lr), indexing="ij")
    lp = np.log(R * T)
    le = np.log(R * (1 + 1.5 * T))
    cs2 = (5.0 / 3.0) * T / (1 + 2.5 * T) + 0 * R
    return _Tab(n, x0, dx, lp, le, cs2)


def _table_prims(w5, ye=0.5):
    w = np.zeros((w5.shape[0], 7))
    w[:, :5] = w5
    w[:, 5] = ye
    return w


def test_ideal_gas_table_gives_the_ideal_gas_con2prim():
    rng = np.random.default_rng(3)
    n = 400
    m = random_metric(rng, n, amp=0.1)
    w5 = np.zeros((n, 5))
    w5[:, 0] = np.exp(rng.uniform(np.log(1e-8), np.log(1e-2), n))
    w5[:, 1:4] = rng.uniform(-2, 2, (n, 3))
    w5[:, 4] = w5[:, 0] * np.exp(rng.uniform(np.log(1e-3), np.log(1.0), n))
    B = random_B(rng, w5)
    Pi = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-14, tol=1e-13)
    Pt = O.Params(table=ideal_gas_table(), rho_atm=1e-14, T_atm=1e-5, tol=1e-13)
    q5 = O.prim2con(m, w5, B, Pi)
    q6 = O.prim2con(m, _table_prims(w5), B, Pt)
    # same conserved variables up to the interpolation error of log(1 + 3T/2) in log T
    assert np.max(np.abs(q6[:, :5] - q5) / np.maximum(np.abs(q5), q5[:, [0]] + np.abs(q5[:, [4]]))) < 1e-6
    assert np.allclose(q6[:, 5], 0.5 * q6[:, 0], rtol=1e-15)
    wi, _, si, _ = O.con2prim(m, q5, B, Pi)
    wt, _, st, _ = O.con2prim(m, np.c_[q5, 0.5 * q5[:, 0]], B, Pt)
    ok = (si == 0) & (st == 0)
    assert ok.mean() > 0.95
    for k in range(5):
        floor = 1e-3 * np.max(np.abs(wi[ok, k])) if 1 <= k <= 3 else 0
        err = np.abs(wt[ok, k] - wi[ok, k]) / np.maximum(np.abs(wi[ok, k]), floor)
        assert err.max() < 1e-5, (k, err.max())
    # the derived temperature is p / rho for this gas
    assert np.max(np.abs(wt[ok, 6] / (wt[ok, 4] / wt[ok, 0]) - 1)) < 1e-6


def test_ideal_gas_table_gives_the_ideal_gas_stage():
    bi = I.random_block(n=(8, 8, 8), g=3, seed=11, rho_range=(1e-6, 1e-3), theta_range=(1e-2, 0.5),
                        u_max=0.6, sigma_range=(1e-2, 1.0))
    Pi = O.Params(gamma_ad=5.0 / 3.0, rho_atm=1e-14, tol=1e-13)
    Pt = O.Params(table=ideal_gas_table(), rho_atm=1e-14, T_atm=1e-5, tol=1e-13)
    U5 = H.cons_from_prims(bi, Pi)
    blk_i = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
    Wt = np.concatenate([bi.W, 0.5 + 0 * bi.W[:1], 0 * bi.W[:1]])
    blk_t = O.Block(bi.n, bi.ng, bi.dx, bi.metric, Wt, bi.B)
    U6 = np.concatenate([U5, 0.5 * U5[:1]])
    dt = 0.2 * min(bi.dx)
    Ui, Bi, Wi, si = O.stage_block(blk_i, U5, U5, bi.B, dt, Pi)
    Ut, Bt, Wt2, st = O.stage_block(blk_t, U6, U6, bi.B, dt, Pt)
    n, g = bi.n, bi.ng
    assert np.array_equal(H.interior(si, n, g), H.interior(st, n, g))
    scale = H.interior(Ui[0] + np.abs(Ui[4]), n, g)
    for v in range(5):
        d = np.abs(H.interior(Ut[v] - Ui[v], n, g)) / np.maximum(np.abs(H.interior(Ui[v], n, g)), scale)
        assert d.max() < 2e-6, (v, d.max())
    for d_ in range(3):
        assert np.max(np.abs(Bt[d_] - Bi[d_])) <= 2e-6 * np.max(np.abs(Bi[d_]))
    # uniform Y_e stays uniform
    assert np.max(np.abs(H.interior(Ut[5] / Ut[0], n, g) - 0.5)) < 1e-14
    assert np.max(np.abs(H.interior(Wt2[5], n, g) - 0.5)) < 1e-14


@pytest.fixture(scope="module")
def tab():
    return I.SyntheticEOS().table(n=(60, 48, 12))


def test_round_trip_and_conserved_reproduction(tab):
    rng = np.random.default_rng(4)
    n = 600
    m = random_metric(rng, n, amp=0.1)
    w = np.zeros((n, 7))
    w[:, 0] = np.exp(rng.uniform(np.log(1e-11), np.log(5e-3), n))
    w[:, 1:4] = rng.uniform(-3, 3, (n, 3))
    w[:, 5] = rng.uniform(0.05, 0.55, n)
    T = np.exp(rng.uniform(np.log(1e-5), np.log(5e-2), n))
    w[:, 4] = tab.eos.p(w[:, 0], T, w[:, 5])
    B = random_B(rng, w[:, :5], sigma=(1e-3, 1.0))
    P = O.Params(table=tab, rho_atm=1e-13, T_atm=1e-6, tol=1e-13)
    q = O.prim2con(m, w, B, P)
    assert np.allclose(q[:, 5], q[:, 0] * w[:, 5], rtol=1e-15)
    w2, q2, st, it = O.con2prim(m, q, B, P)
    ok = st == 0
    assert ok.mean() > 0.9
    Wl = np.sqrt(1 + np.sum(w[:, 1:4] ** 2, 1))     # approximate (metric amp 0.1): error scale
    for k in (0, 1, 2, 3, 5):
        err = np.abs(w2[ok, k] - w[ok, k]) / np.maximum(np.abs(w[ok, k]), 1e-3 if 1 <= k <= 3 else 0)
        assert np.all(err < 1e-11 * Wl[ok] ** 2 + 1e-12), (k, err.max())
    # the recovered state reproduces the conserved variables (S, tau on the energy scale)
    q3 = O.prim2con(m, w2, B, P)
    scale = q[ok, 0] + np.abs(q[ok, 4])
    assert np.max(np.abs(q3[ok, 0] - q[ok, 0]) / q[ok, 0]) < 1e-12
    for k in (1, 2, 3, 4):
        assert np.max(np.abs(q3[ok, k] - q[ok, k]) / np.maximum(np.abs(q[ok, k]), scale)) < 1e-10
    # T output is the table temperature of (rho, p, Y_e)
    _, _, _, Tr = O.table_eval(P, w2[ok, 0], w2[ok, 6], w2[ok, 5])
    assert np.max(np.abs(Tr / w2[ok, 6] - 1)) < 1e-9


def test_temperature_floor_ye_clamp_and_atmosphere(tab):
    rng = np.random.default_rng(5)
    n = 30
    m = random_metric(rng, n, amp=0.05)
    w = np.zeros((n, 7))
    w[:, 0] = 1e-5
    w[:, 1] = 0.3
    w[:, 5] = 0.3
    w[:, 4] = tab.eos.p(1e-5, 1e-6, 0.3)        # T = 1e-6 < T_atm = 1e-4
    B = np.zeros((n, 3))
    P = O.Params(table=tab, rho_atm=1e-13, T_atm=1e-4, tol=1e-13)
    q = O.prim2con(m, w, B, P)
    w2, q2, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st == 32)
    assert np.allclose(w2[:, 6], 1e-4, rtol=1e-15)
    p_floor, _, _, _ = O.table_eval(P, w2[:, 0], np.full(n, 1e-4), w2[:, 5])
    assert np.allclose(w2[:, 4], p_floor, rtol=1e-14)
    assert np.allclose(O.prim2con(m, w2, B, P), q2, rtol=1e-13, atol=0)     # conserved rebuilt
    # Y_e outside the table: moved to its end, D Y_e rewritten
    w3 = w.copy(); w3[:, 4] = tab.eos.p(1e-5, 1e-3, 0.3)
    q = O.prim2con(m, w3, B, P)
    q[:, 5] = 0.9 * q[:, 0]
    w4, q4, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st == 32)
    assert np.allclose(w4[:, 5], tab.ye_range[1], rtol=1e-15)
    assert np.allclose(q4[:, 5], q4[:, 0] * tab.ye_range[1], rtol=1e-15)
    # atmosphere: rho_atm, T_atm, Y_e_atm, u = 0
    q = O.prim2con(m, w3, B, P)
    q[:, 0] = 1e-20; q[:, 5] = 1e-20 * 0.3
    w5, q5, st, _ = O.con2prim(m, q, B, P)
    assert np.all(st == 1)
    assert np.allclose(w5[:, 0], 1e-13) and np.all(w5[:, 1:4] == 0)
    assert np.allclose(w5[:, 5], P.Ye_atm) and np.allclose(w5[:, 6], 1e-4)
    assert np.allclose(O.prim2con(m, w5, B, P), q5, rtol=1e-12, atol=0)


def test_ye_is_conserved_on_a_periodic_block(tab):
    bi = I.random_block(n=(10, 8, 6), g=3, seed=12, eos=tab.eos, rho_range=(1e-6, 1e-3), T_range=(1e-4, 1e-2),
                        u_max=0.5, sigma_range=(1e-3, 0.1), flat=True)
    H.fill_periodic_cells(bi.W, bi.n, bi.ng)
    H.fill_periodic_faces(bi.B, bi.n, bi.ng)
    P = O.Params(table=tab, rho_atm=1e-13, T_atm=1e-6, tol=1e-13)
    U = H.cons_from_prims(bi, P)
    blk = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
    Uo, Bo, Wo, st = O.stage_block(blk, U, U, bi.B, 0.2 * min(bi.dx), P)
    n, g = bi.n, bi.ng
    assert np.all(H.interior(st, n, g) & 0x3 == 0)
    for v in (0, 5):
        before, after = H.interior(U[v], n, g).sum(), H.interior(Uo[v], n, g).sum()
        assert abs(after - before) <= 1e-13 * H.interior(np.abs(U[v]), n, g).sum(), v
    ye = H.interior(Wo[5], n, g)
    assert ye.min() >= 0.05 - 1e-3 and ye.max() <= 0.5 + 1e-3


@pytest.mark.parametrize("vx", [0.3, -0.3])
def test_ye_flux_is_the_mass_flux_times_the_upwind_state(tab, vx):
    """Uniform flow along x with a Y_e profile: the D flux is the same on every face, so the stage moves
    Y_e by the difference of the upwind reconstructed Y_e (left state for vx > 0, right for vx < 0)."""
    n, g = (12, 2, 2), 3
    bi = I.uniform_block(n=n, g=g, dx=(0.1, 0.1, 0.1), rho=1e-4, u=(vx, 0.0, 0.0), p=1e-6, B=(0.0, 0.0, 0.0))
    N = bi.N
    x = np.arange(N[0]) - g
    ye_line = 0.25 + 0.15 * np.tanh((x - 5.0) / 1.5) + 0.02 * np.sin(0.9 * x)
    W = np.zeros((7,) + bi.W.shape[1:])
    W[:5] = bi.W
    W[4] = tab.eos.p(1e-4, 1e-3, 0.3)
    W[5] = ye_line[None, None, :]
    P = O.Params(table=tab, rho_atm=1e-13, T_atm=1e-6, tol=1e-14, recon=0)
    bt = I.BlockInput(bi.n, g, bi.x0, bi.dx, bi.metric, W, bi.B)
    U = H.cons_from_prims(bt, P)
    blk = O.Block(bt.n, g, bt.dx, bt.metric, W, bt.B)
    dt = 0.05
    Uo, _, Wo, st = O.stage_block(blk, U, U, bt.B, dt, P)
    L, R = O.recon1d(0, ye_line)
    up = L if vx > 0 else R                       # face f between cells f-1 and f (array index)
    D = U[0, g, g, g]
    FD = D * vx / np.sqrt(1 + vx * vx)            # flat metric, uniform state: D v^x, v^x = u~^x / W
    i = np.arange(g, g + n[0])
    ye_new = (D * ye_line[i] - dt / bt.dx[0] * FD * (up[i + 1] - up[i])) / D
    got = Uo[5, g, g, g:g + n[0]] / Uo[0, g, g, g:g + n[0]]
    assert np.max(np.abs(got - ye_new)) < 1e-14
    other = R if vx > 0 else L
    ye_wrong = (D * ye_line[i] - dt / bt.dx[0] * FD * (other[i + 1] - other[i])) / D
    assert np.max(np.abs(ye_wrong - ye_new)) > 1e-4      # the test distinguishes the two sides
