"""Pins of the oracle's reconstruction (Sec. 3.4, readings c4/c5) and vertex-to-cell/face metric
interpolation (Sec. 3.2, reading c10) against exact polynomial reproduction and convergence order."""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I


def test_plm_exact_on_linear_data():
    x = np.arange(20) * 0.1
    w = 3.0 - 2.0 * x
    L, R = O.recon1d(0, w)
    f = np.arange(3, 18)
    xf = (f - 0.5) * 0.1
    assert np.allclose(L[f], 3.0 - 2.0 * xf, rtol=0, atol=1e-14)
    assert np.allclose(R[f], 3.0 - 2.0 * xf, rtol=0, atol=1e-14)


def test_plm_is_bounded_by_neighbours():
    rng = np.random.default_rng(0)
    w = rng.uniform(0, 1, 200)
    L, R = O.recon1d(0, w)
    for f in range(3, 198):
        lo, hi = min(w[f - 2], w[f - 1], w[f]), max(w[f - 2], w[f - 1], w[f])
        assert lo - 1e-15 <= L[f] <= hi + 1e-15
        lo, hi = min(w[f - 1], w[f], w[f + 1]), max(w[f - 1], w[f], w[f + 1])
        assert lo - 1e-15 <= R[f] <= hi + 1e-15
    # extremum: zero slope
    L, R = O.recon1d(0, np.array([0, 0, 0, 1.0, 0, 0, 0, 0]))
    assert L[4] == 1.0 and R[3] == 1.0


def cell_avg(F, xl, xr):
    return (F(xr) - F(xl)) / (xr - xl)


@pytest.mark.parametrize("coef", [(1.0, 0, 0), (0.3, -2.0, 0), (0.5, 1.0, 4.0)])
def test_wenoz_exact_on_quadratic_cell_averages(coef):
    a, b, c = coef
    F = lambda x: a * x + b * x ** 2 / 2 + c * x ** 3 / 3       # antiderivative
    f = lambda x: a + b * x + c * x ** 2
    h = 0.05
    xe = np.arange(31) * h
    w = cell_avg(F, xe[:-1], xe[1:])
    L, R = O.recon1d(1, w, eps=1e-40)
    for k in range(3, 28):
        assert abs(L[k] - f(xe[k])) < 1e-12
        assert abs(R[k] - f(xe[k])) < 1e-12


def test_wenoz_fifth_order_on_smooth_data():
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        xe = np.arange(n + 1) * h
        w = cell_avg(lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi), xe[:-1], xe[1:])
        L, R = O.recon1d(1, w, eps=1e-40)
        k = np.arange(3, n - 2)
        errs.append(max(np.max(np.abs(L[k] - np.sin(2 * np.pi * xe[k]))),
                        np.max(np.abs(R[k] - np.sin(2 * np.pi * xe[k])))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.5), orders


def test_wenoz_mirror_symmetry():
    rng = np.random.default_rng(1)
    w = rng.uniform(0, 1, 40)
    L, R = O.recon1d(1, w)
    L2, R2 = O.recon1d(1, w[::-1].copy())
    n = 40
    for f in range(3, n - 2):
        assert L[f] == R2[n - f] and R[f] == L2[n - f]


def test_wenoz_non_oscillatory_at_a_jump():
    w = np.where(np.arange(40) < 20, 1.0, 0.0)
    L, R = O.recon1d(1, w)
    k = np.arange(3, 38)
    assert np.all(L[k] > -1e-12) and np.all(L[k] < 1 + 1e-12)
    assert np.all(R[k] > -1e-12) and np.all(R[k] < 1 + 1e-12)


def poly_metric_block(order, seed=3):
    """Metric components set to a random polynomial of degree order-1 in each coordinate."""
    rng = np.random.default_rng(seed)
    n, g = (5, 6, 7), 3
    dx = (0.3, 0.2, 0.25)
    x0 = (0.1, -0.2, 0.3)
    X, Y, Z = I.grid(n, g, x0, dx, (1, 1, 1))
    deg = order - 1
    coefs = rng.uniform(-1, 1, (16, deg + 1, deg + 1, deg + 1))

    def P(c, X, Y, Z):
        out = np.zeros_like(X)
        for a in range(deg + 1):
            for b in range(deg + 1):
                for e in range(deg + 1):
                    out += coefs[c, a, b, e] * X ** a * Y ** b * Z ** e
        return out

    def dP(c, k, X, Y, Z):
        out = np.zeros_like(X)
        for a in range(deg + 1):
            for b in range(deg + 1):
                for e in range(deg + 1):
                    pw = [a, b, e]
                    if pw[k] == 0:
                        continue
                    t = coefs[c, a, b, e] * pw[k]
                    pw[k] -= 1
                    out += t * X ** pw[0] * Y ** pw[1] * Z ** pw[2]
        return out

    metric = np.stack([P(c, X, Y, Z) for c in range(16)])
    W = np.zeros((5,) + tuple(v + 2 * g for v in n[::-1]))
    blk = O.Block(n, g, dx, metric, W)
    return blk, P, dP, (n, g, x0, dx)


@pytest.mark.parametrize("order", [2, 4])
def test_interpolation_exact_on_tensor_polynomials(order):
    blk, P, dP, (n, g, x0, dx) = poly_metric_block(order)
    lo, hi = -1, 4
    val, dval = O.interp_cells(blk, order, lo, hi)
    ax = [x0[d] + (np.arange(lo, hi) + 0.5) * dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    for c in range(16):
        assert np.max(np.abs(val[:, c] - P(c, X, Y, Z))) < 1e-12
        for k in range(3):
            assert np.max(np.abs(dval[:, k, c] - dP(c, k, X, Y, Z))) < 1e-11
    for d in range(3):
        fv = O.interp_faces(blk, order, d, lo, hi)
        axf = [x0[e] + (np.arange(lo, hi) + (0.0 if e == d else 0.5)) * dx[e] for e in range(3)]
        Zf, Yf, Xf = np.meshgrid(axf[2], axf[1], axf[0], indexing="ij")
        for c in range(16):
            assert np.max(np.abs(fv[:, c] - P(c, Xf.ravel(), Yf.ravel(), Zf.ravel()))) < 1e-12


def test_order2_interpolation_is_not_exact_on_quadratics():
    """Guards the test above: a degree-2 polynomial is only approximated at order 2."""
    blk, P, dP, (n, g, x0, dx) = poly_metric_block(3)
    val, _ = O.interp_cells(blk, 2, 0, 3)
    ax = [x0[d] + (np.arange(0, 3) + 0.5) * dx[d] for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    assert np.max(np.abs(val[:, 0] - P(0, X.ravel(), Y.ravel(), Z.ravel()))) > 1e-6


# ---- WENO5 (Jiang & Shu) and PPM (Colella-Sekora limited) ------------------------------------------
def test_weno5_is_the_linear_fifth_order_formula_on_linear_data():
    """On linear data the three smoothness indicators are equal, so the weights are the linear ones and
    the value is the upwind fifth-order formula (2 v0 - 13 v1 + 47 v2 + 27 v3 - 3 v4)/60."""
    rng = np.random.default_rng(4)
    w = 0.7 + 0.3 * np.arange(20) + 0 * rng.uniform(size=20)
    L, R = O.recon1d(2, w, eps=1e-40)
    for f in range(3, 18):
        v = w[f - 3:f + 2]
        lin = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60
        assert abs(L[f] - lin) < 1e-13


@pytest.mark.parametrize("method", [2, 3])
@pytest.mark.parametrize("coef", [(1.0, 0, 0), (0.3, -2.0, 0), (0.5, 1.0, 4.0)])
def test_weno5_and_ppm_exact_on_monotone_quadratic_cell_averages(method, coef):
    """Cell averages of a monotone quadratic: every WENO sub-stencil and the fourth-order PPM interface
    value are exact, and no PPM limiter engages (no extremum, no overshoot)."""
    a, b, c = coef
    F = lambda x: a * x + b * x ** 2 / 2 + c * x ** 3 / 3
    f = lambda x: a + b * x + c * x ** 2
    h = 0.02
    xe = 0.01 + np.arange(31) * h     # f' = b + 2 c x keeps one sign on [0.01, 0.63] for these coefficients
    w = cell_avg(F, xe[:-1], xe[1:])
    L, R = O.recon1d(method, w, eps=1e-40)
    for k in range(3, 28):
        assert abs(L[k] - f(xe[k])) < 1e-12, (k, L[k], f(xe[k]))
        assert abs(R[k] - f(xe[k])) < 1e-12


@pytest.mark.parametrize("method,min_order", [(2, 4.5), (3, 2.8)])
def test_weno5_fifth_and_ppm_third_order_on_smooth_data(method, min_order):
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        xe = np.arange(n + 1) * h
        w = cell_avg(lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi), xe[:-1], xe[1:])
        L, R = O.recon1d(method, w, eps=1e-40)
        k = np.arange(3, n - 2)
        errs.append(np.mean(np.abs(L[k] - np.sin(2 * np.pi * xe[k])) + np.abs(R[k] - np.sin(2 * np.pi * xe[k]))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > min_order), orders


@pytest.mark.parametrize("method", [2, 3])
def test_weno5_and_ppm_mirror_symmetric(method):
    rng = np.random.default_rng(2)
    w = rng.uniform(0, 1, 40)
    L, R = O.recon1d(method, w)
    L2, R2 = O.recon1d(method, w[::-1].copy())
    for f in range(3, 38):
        assert abs(L[f] - R2[40 - f]) < 1e-15 and abs(R[f] - L2[40 - f]) < 1e-15


def test_ppm_is_monotone_at_a_jump_and_flat_at_an_extremum():
    w = np.where(np.arange(40) < 20, 1.0, 0.0)
    L, R = O.recon1d(3, w)
    k = np.arange(3, 38)
    assert np.all((L[k] >= 0) & (L[k] <= 1) & (R[k] >= 0) & (R[k] <= 1))
    # a single-cell spike: the spike cell's parabola is flattened (no overshoot above the spike)
    s = np.zeros(20); s[10] = 1.0
    L, R = O.recon1d(3, s)
    assert L[11] <= 1.0 and R[10] <= 1.0 and np.all(L[3:18] >= 0) and np.all(R[3:18] >= 0)
