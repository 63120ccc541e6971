"""Pins of the oracle's matter sources of the spacetime equations (Sec. 2.1, 2.2) and of their
cell-to-vertex interpolation (Sec. 3.2).

* the closed forms equal the projections n_mu n_nu T^{mu nu}, -gamma_{i mu} n_nu T^{mu nu} and
  gamma_{i mu} gamma_{j nu} T^{mu nu} of the stress-energy tensor built from 4-vectors, with b^mu
  formed as the projection orthogonal to u of the Eulerian field (an independent construction)
* rho_ADM = (tau + D)/sqrt(gamma) and S_i = S_i^cons/sqrt(gamma) against the oracle's conserved
  variables, ideal gas and table
* a static unmagnetised fluid in flat space: rho_ADM = rho (1 + eps), S_i = 0, S_ij = p delta_ij
* the cell-to-vertex interpolation reproduces per-axis polynomials of degree 1 (order 2) and 3
  (order 4) exactly and writes only the owned vertices"""
import numpy as np
import pytest

import oracle as O
from paper_2311_04989_gb300 import inputs as I

SYM = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


def random_points(rng, n, magnetised=True):
    metric = np.zeros((n, 16))
    metric[:, 0] = rng.uniform(0.6, 1.2, n)
    metric[:, 1:4] = rng.uniform(-0.2, 0.2, (n, 3))
    A = rng.uniform(-0.15, 0.15, (n, 3, 3))
    g = np.eye(3)[None] + 0.5 * (A + A.transpose(0, 2, 1))
    for i in range(3):
        for j in range(i, 3):
            metric[:, 4 + SYM[i][j]] = g[:, i, j]
    prims = np.zeros((n, 5))
    prims[:, 0] = 10 ** rng.uniform(-6, -2, n)
    prims[:, 1:4] = rng.uniform(-1.5, 1.5, (n, 3))
    prims[:, 4] = prims[:, 0] * 10 ** rng.uniform(-3, 0, n)
    B = rng.uniform(-1, 1, (n, 3)) * np.sqrt(prims[:, 4:5]) * (3.0 if magnetised else 0.0)
    return metric, prims, B


def four_tensor_sources(metric, prims, B, gamma_ad):
    """The projections of T^{mu nu} = (rho h + b^2) u u + (p + b^2/2) g^{-1} - b b, built from 4-vectors."""
    out = np.zeros((len(prims), 10))
    for n in range(len(prims)):
        a = metric[n, 0]
        beta = metric[n, 1:4]
        gam = np.array([[metric[n, 4 + SYM[i][j]] for j in range(3)] for i in range(3)])
        g4 = np.zeros((4, 4))
        g4[0, 0] = -a * a + beta @ gam @ beta
        g4[0, 1:] = g4[1:, 0] = gam @ beta
        g4[1:, 1:] = gam
        g4u = np.linalg.inv(g4)
        rho, ut, p = prims[n, 0], prims[n, 1:4], prims[n, 4]
        W = np.sqrt(1 + ut @ gam @ ut)
        u = np.concatenate([[W / a], ut - W * beta / a])          # u^mu
        ul = g4 @ u
        Bcal = B[n] / np.sqrt(np.linalg.det(gam))                  # undensitised Eulerian field
        Bmu = np.concatenate([[0.0], Bcal])
        b = (Bmu + (ul @ Bmu) * u) / W                             # projection orthogonal to u, / W
        bl = g4 @ b
        b2 = b @ bl
        assert abs(ul @ b) < 1e-12 * (1 + np.abs(b).max() * W)
        h = 1 + gamma_ad / (gamma_ad - 1) * p / rho
        T = (rho * h + b2) * np.outer(u, u) + (p + b2 / 2) * g4u - np.outer(b, b)
        nl = np.array([-a, 0, 0, 0])
        out[n, 0] = nl @ T @ nl
        TL = g4 @ T @ g4                                            # T_{mu nu}
        nu = g4u @ nl                                               # n^mu
        # S_i = -gamma_i^mu n^nu T_{mu nu}, S_ij = gamma_i^mu gamma_j^nu T_{mu nu}; gamma_i^mu = delta + n^mu n_i
        proj = np.eye(4) + np.outer(nl, nu)                         # proj[i, mu] = gamma_i^mu (rows: lower)
        for i in range(3):
            out[n, 1 + i] = -(proj[1 + i] @ TL @ nu)
            for j in range(i, 3):
                out[n, 4 + SYM[i][j]] = proj[1 + i] @ TL @ proj[1 + j]
    return out


@pytest.mark.parametrize("magnetised", [False, True])
def test_closed_forms_are_the_projections_of_the_stress_energy_tensor(magnetised):
    rng = np.random.default_rng(7)
    metric, prims, B = random_points(rng, 200, magnetised)
    P = O.Params(gamma_ad=5.0 / 3.0)
    got = O.adm_points(metric, prims, B, P)
    ref = four_tensor_sources(metric, prims, B, P.gamma_ad)
    scale = np.abs(ref[:, :1]) + np.abs(ref).max(axis=1, keepdims=True) * 1e-3
    assert np.max(np.abs(got - ref) / scale) < 1e-11


def test_energy_and_momentum_densities_follow_from_the_conserved_variables():
    rng = np.random.default_rng(8)
    metric, prims, B = random_points(rng, 300)
    P = O.Params(gamma_ad=2.0)
    adm = O.adm_points(metric, prims, B, P)
    q = O.prim2con(metric, prims, B, P)
    sg = np.array([np.sqrt(np.linalg.det(np.array([[m[4 + SYM[i][j]] for j in range(3)] for i in range(3)])))
                   for m in metric])
    assert np.allclose(adm[:, 0], (q[:, 4] + q[:, 0]) / sg, rtol=1e-12, atol=0)
    for i in range(3):
        assert np.allclose(adm[:, 1 + i], q[:, 1 + i] / sg, rtol=1e-11, atol=1e-13 * np.abs(adm[:, :1]).max())


def test_table_sources_match_the_conserved_variables():
    eos = I.SyntheticEOS()
    tab = eos.table(n=(60, 40, 16))
    rng = np.random.default_rng(9)
    n = 200
    metric, p5, B = random_points(rng, n)
    rho = 10 ** rng.uniform(-7, -3, n)
    T = 10 ** rng.uniform(-3, -1.5, n)
    ye = rng.uniform(0.1, 0.5, n)
    prims = np.zeros((n, 7))
    prims[:, 0] = rho
    prims[:, 1:4] = p5[:, 1:4]
    prims[:, 4] = eos.p(rho, T, ye)
    prims[:, 5] = ye
    prims[:, 6] = T
    P = O.Params(table=tab)
    adm = O.adm_points(metric, prims, B * np.sqrt(rho)[:, None] * 0.1, P)
    q = O.prim2con(metric, prims, B * np.sqrt(rho)[:, None] * 0.1, P)
    sg = np.array([np.sqrt(np.linalg.det(np.array([[m[4 + SYM[i][j]] for j in range(3)] for i in range(3)])))
                   for m in metric])
    assert np.allclose(adm[:, 0], (q[:, 4] + q[:, 0]) / sg, rtol=1e-12, atol=0)


def test_static_fluid_in_flat_space():
    n = 20
    rng = np.random.default_rng(10)
    metric = np.zeros((n, 16))
    metric[:, 0] = 1.0
    metric[:, 4] = metric[:, 7] = metric[:, 9] = 1.0
    prims = np.zeros((n, 5))
    prims[:, 0] = rng.uniform(0.1, 2, n)
    prims[:, 4] = rng.uniform(0.01, 1, n)
    P = O.Params(gamma_ad=4.0 / 3.0)
    adm = O.adm_points(metric, prims, np.zeros((n, 3)), P)
    eps = prims[:, 4] / ((P.gamma_ad - 1) * prims[:, 0])
    assert np.allclose(adm[:, 0], prims[:, 0] * (1 + eps), rtol=1e-15)
    assert np.all(adm[:, 1:4] == 0)
    for c, diag in zip(range(4, 10), (1, 0, 0, 1, 0, 1)):
        assert np.allclose(adm[:, c], prims[:, 4] * diag, rtol=1e-15, atol=0)


@pytest.mark.parametrize("vc_order,deg", [(2, 1), (4, 3)])
def test_cell_to_vertex_interpolation_is_exact_on_polynomials(vc_order, deg):
    # static fluid, flat metric, ideal gas: rho_ADM = rho + p/(Gamma-1) is the polynomial in rho
    n, g = (6, 5, 7), 3
    bi = I.uniform_block(n=n, g=g, dx=(0.1, 0.2, 0.15), rho=1.0, u=(0.0, 0.0, 0.0), p=0.3, B=(0.0, 0.0, 0.0))
    x = [(np.arange(-g, n[d] + g) + 0.5) * bi.dx[d] for d in range(3)]
    rng = np.random.default_rng(11)
    coef = [rng.uniform(-0.3, 0.3, deg + 1) for _ in range(3)]
    poly = lambda c, t: sum(ck * t ** k for k, ck in enumerate(c))
    f = 2.0 + poly(coef[2], x[2])[:, None, None] * poly(coef[1], x[1])[None, :, None] * poly(coef[0], x[0])[None, None, :]
    bi.W[0] = f
    bi.W[1:4] = 0.0
    for d in range(3):
        bi.B[d][...] = 0.0
    P = O.Params(gamma_ad=5.0 / 3.0, interp_order=2)
    out = O.adm_block(O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B), P, vc_order)
    xv = [np.arange(-g, n[d] + g + 1) * bi.dx[d] for d in range(3)]
    fv = 2.0 + poly(coef[2], xv[2])[:, None, None] * poly(coef[1], xv[1])[None, :, None] * \
        poly(coef[0], xv[0])[None, None, :]
    own = (slice(g, g + n[2] + 1), slice(g, g + n[1] + 1), slice(g, g + n[0] + 1))
    assert np.max(np.abs(out[0][own] - (fv[own] + 0.3 / (P.gamma_ad - 1)))) < 1e-13
    assert np.allclose(out[4][own], 0.3, rtol=1e-14) and np.all(out[5][own] == 0)
    mask = np.ones(out.shape[1:], bool)
    mask[own] = False
    assert np.all(np.isnan(out[:, mask]))
