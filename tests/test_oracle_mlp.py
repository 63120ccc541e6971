"""Pins of the oracle's learned-bracket pieces (not in the paper: a bracket proposal for the root find of Sec. 3.5):
backpropagated gradients against central finite differences, and the recorded root equal to the
definition mu = 1/(h W) of the state the conserved variables came from."""
import numpy as np

import oracle as O
from tests.test_oracle_pointwise import random_metric, random_prims, random_B


def random_params(rng, scale=0.5):
    P = np.zeros(O.MLP_OFF + O.MLP_NW)
    P[O.MLP_MEAN:O.MLP_MEAN + O.MLP_IN] = rng.normal(0, 1, O.MLP_IN)
    P[O.MLP_ISTD:O.MLP_ISTD + O.MLP_IN] = rng.uniform(0.5, 2.0, O.MLP_IN)
    P[O.MLP_TMEAN], P[O.MLP_TSTD] = -0.5, 0.7
    P[O.MLP_OFF:] = rng.normal(0, scale, O.MLP_NW)
    return P


def test_parameter_count():
    assert O.mlp_nparam() == 16 + 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_backprop_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = random_params(rng)
    x = rng.normal(0, 1, (17, O.MLP_IN))
    t = rng.normal(0, 1, 17)
    L, g = O.mlp_loss_grad(P, x, t)
    assert L > 0
    nw1 = 64 * O.MLP_IN
    idx = np.concatenate([rng.choice(O.MLP_NW, 60, replace=False), [0, nw1 - 1, nw1 + 63, O.MLP_NW - 1]])
    h = 1e-4

    def loss_at(k, dx):
        Pk = P.copy(); Pk[O.MLP_OFF + k] += dx
        return O.mlp_loss_grad(Pk, x, t)[0]
    for k in idx:   # fourth-order central difference
        fd = (-loss_at(k, 2 * h) + 8 * loss_at(k, h) - 8 * loss_at(k, -h) + loss_at(k, -2 * h)) / (12 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3), (k, fd, g[k])


def test_forward_is_the_affine_output_of_the_loss_network():
    """The loss uses z = (t_hat - mean)/std, so a target equal to the prediction gives zero loss."""
    rng = np.random.default_rng(1)
    P = random_params(rng)
    x = rng.normal(0, 1, (9, O.MLP_IN))
    t = O.mlp_forward(P, x)
    L, g = O.mlp_loss_grad(P, x, t)
    assert L < 1e-28 and np.max(np.abs(g)) < 1e-14


def test_samples_record_the_root_and_the_invariants():
    rng = np.random.default_rng(2)
    n = 300
    m = random_metric(rng, n, amp=0.1)
    w = random_prims(rng, n, umax=3.0)
    B = random_B(rng, w)
    P = O.Params(gamma_ad=2.0, rho_atm=1e-20, tol=1e-15)
    q = O.prim2con(m, w, B, P)
    f, t, valid = O.c2p_samples(m, q, B, P)
    assert np.all(valid)
    # mu = 1/(h W) of the original state
    g6 = m[:, 4:10]
    ut = w[:, 1:4]
    gxx, gxy, gxz, gyy, gyz, gzz = g6.T
    uu = (gxx * ut[:, 0] ** 2 + gyy * ut[:, 1] ** 2 + gzz * ut[:, 2] ** 2 +
          2 * (gxy * ut[:, 0] * ut[:, 1] + gxz * ut[:, 0] * ut[:, 2] + gyz * ut[:, 1] * ut[:, 2]))
    W = np.sqrt(1 + uu)
    h = 1 + 2.0 / (2.0 - 1) * w[:, 4] / w[:, 0]
    assert np.max(np.abs(t - np.log(1 / (h * W)))) < 1e-12
    # q = tau/D feature
    assert np.allclose(f[:, 0], np.log1p(q[:, 4] / q[:, 0]), rtol=1e-12, atol=0)
    assert np.all((f[:, 3] >= 0) & (f[:, 3] <= 1 + 1e-12))
    assert np.all(f[:, 4:] == 0)     # the ideal gas is scale-free: no density or composition feature
    # atmosphere cells are not samples
    q2 = q.copy(); q2[:5, 0] = 1e-30
    _, _, v2 = O.c2p_samples(m, q2, B, P)
    assert not np.any(v2[:5]) and np.all(v2[5:])


def test_table_samples_carry_density_and_composition_features():
    from paper_2311_04989_gb300 import inputs as I
    tab = I.SyntheticEOS().table(n=(40, 30, 6))
    rng = np.random.default_rng(3)
    n = 200
    m = random_metric(rng, n, amp=0.1)
    w = np.zeros((n, 7))
    w[:, 0] = np.exp(rng.uniform(np.log(1e-8), np.log(1e-3), n))
    w[:, 1:4] = rng.normal(0, 0.5, (n, 3))
    w[:, 5] = rng.uniform(0.1, 0.5, n)
    w[:, 4] = tab.eos.p(w[:, 0], 1e-3, w[:, 5])
    B = random_B(rng, w[:, :5])
    P = O.Params(table=tab, rho_atm=1e-12, tol=1e-14)
    q = O.prim2con(m, w, B, P)
    f, t, valid = O.c2p_samples(m, q, B, P)
    assert valid.mean() > 0.95
    sg = np.sqrt(np.linalg.det(np.stack([m[:, [4, 5, 6]], m[:, [5, 7, 8]], m[:, [6, 8, 9]]], 1)))
    Dt = q[:, 0] / sg
    ok = valid & (Dt * 1e4 > 2 * np.einsum("ni,ni->n", B, B) / sg ** 2)      # B^2/D limit inactive
    assert np.allclose(f[ok, 4], np.log(Dt[ok]), rtol=0, atol=1e-12)
    assert np.allclose(f[ok, 5], w[ok, 5], rtol=1e-12, atol=0)
