"""Exact solution of the 1D special-relativistic hydrodynamic Riemann problem, ideal gas, no
tangential velocity (test helper).

Written from the relations of relativistic gas dynamics: across a rarefaction the Riemann invariant
artanh(v) +- A(c_s) is constant, with A(c) = ln((sqrt(G-1) + c)/(sqrt(G-1) - c))/sqrt(G-1) for the
isentropic ideal gas; across a shock the Taub adiabat [h^2] = (h_a/rho_a + h/rho)[p] and the
mass flux j^2 = -[p]/[h/rho] fix the post-shock state.  The pressure p* in the star region makes
the two post-wave velocities equal.
"""
import numpy as np
from scipy.optimize import brentq


class Gas:
    def __init__(self, G):
        self.G = G
        self.s = np.sqrt(G - 1)

    def h(self, rho, p):
        return 1 + self.G / (self.G - 1) * p / rho

    def cs(self, rho, p):
        return np.sqrt(self.G * p / (rho * self.h(rho, p)))

    def A(self, c):
        return np.log((self.s + c) / (self.s - c)) / self.s


def _rarefaction(gas, rho, p, v, ps, sign):
    """Post-wave (rho*, v*) of a rarefaction; sign=-1 left-facing, +1 right-facing."""
    K = p / rho ** gas.G
    rs = (ps / K) ** (1 / gas.G)
    cs_a, cs_b = gas.cs(rho, p), gas.cs(rs, ps)
    # left fan: artanh v + A(c) constant; right fan: artanh v - A(c) constant
    if sign < 0:
        z = np.arctanh(v) + gas.A(cs_a) - gas.A(cs_b)
    else:
        z = np.arctanh(v) - gas.A(cs_a) + gas.A(cs_b)
    return rs, np.tanh(z)


def _shock(gas, rho, p, v, ps, sign):
    """Post-shock (rho*, v*, shock speed); sign=-1 left-facing, +1 right-facing."""
    G = gas.G
    ha = gas.h(rho, p)
    dp = ps - p
    # Taub adiabat as a quadratic in h*
    a = 1 - (G - 1) * dp / (G * ps)
    b = (G - 1) * dp / (G * ps)
    c = -ha * ha - ha / rho * dp
    hs = (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)
    rs = G * ps / ((G - 1) * (hs - 1))
    j = np.sqrt(-dp / (hs / rs - ha / rho)) * sign
    Wa = 1 / np.sqrt(1 - v * v)
    r2w2 = rho * rho * Wa * Wa
    Vs = (r2w2 * v + j * np.sqrt(j * j + r2w2 * (1 - v * v))) / (r2w2 + j * j)
    Ws = 1 / np.sqrt(1 - Vs * Vs)
    vs = (ha * Wa * v + Ws * dp / j) / (ha * Wa + dp * (Ws * v / j + 1 / (rho * Wa)))
    return rs, vs, Vs


def _post(gas, st, ps, sign):
    rho, p, v = st
    if ps > p:
        rs, vs, _ = _shock(gas, rho, p, v, ps, sign)
    else:
        rs, vs = _rarefaction(gas, rho, p, v, ps, sign)
    return rs, vs


def solve(G, left, right):
    """left/right = (rho, p, v).  Returns a function (xi = x/t) -> (rho, p, v)."""
    gas = Gas(G)
    f = lambda ps: _post(gas, left, ps, -1)[1] - _post(gas, right, ps, +1)[1]
    lo, hi = 1e-12 * min(left[1], right[1]), 10 * max(left[1], right[1])
    ps = brentq(f, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=500)
    rLs, vs = _post(gas, left, ps, -1)
    rRs, _ = _post(gas, right, ps, +1)

    def wave_edges(st, rs, sign):
        rho, p, v = st
        if ps > p:
            _, _, Vs = _shock(gas, rho, p, v, ps, sign)
            return Vs, Vs
        ca, cb = gas.cs(rho, p), gas.cs(rs, ps)
        if sign < 0:
            return (v - ca) / (1 - v * ca), (vs - cb) / (1 - vs * cb)
        return (vs + cb) / (1 + vs * cb), (v + ca) / (1 + v * ca)

    Lh, Lt = wave_edges(left, rLs, -1)
    Rt, Rh = wave_edges(right, rRs, +1)

    def fan(st, xi, sign):
        rho, p, v = st
        K = p / rho ** G
        ca = gas.cs(rho, p)
        # characteristic speed (v + sign c)/(1 + sign v c) = xi with the invariant held
        Ja = np.arctanh(v) + (gas.A(ca) if sign < 0 else -gas.A(ca))

        def resid(c):
            vv = np.tanh(Ja - gas.A(c)) if sign < 0 else np.tanh(Ja + gas.A(c))
            return (vv + sign * c) / (1 + sign * vv * c) - xi

        c = brentq(resid, 1e-14, gas.s * (1 - 1e-14), xtol=1e-15)
        vv = np.tanh(Ja - gas.A(c)) if sign < 0 else np.tanh(Ja + gas.A(c))
        # c^2 = G p/(rho h) with p = K rho^G -> solve for rho
        r = brentq(lambda r: gas.cs(r, K * r ** G) - c, 1e-300, 1e10, xtol=1e-300, rtol=1e-14)
        return r, K * r ** G, vv

    def sample(xi):
        if xi <= Lh:
            return left
        if xi < Lt:
            return fan(left, xi, -1)
        if xi < vs:
            return (rLs, ps, vs)
        if xi < Rt:
            return (rRs, ps, vs)
        if xi < Rh:
            return fan(right, xi, +1)
        return right

    sample.p_star, sample.v_star = ps, vs
    return sample
