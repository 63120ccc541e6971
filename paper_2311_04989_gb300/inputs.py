"""Seeded synthetic inputs for the GRMHD stage (numpy only).

This module is shared by the tests, the CPU oracle's callers and ``bench.py``.  It holds none of the
stage's arithmetic: it draws smooth random fields, solves the TOV equations for star initial data,
and forms the face field as the discrete curl of an edge vector potential so that it is
divergence-free by construction (the initial-data recipe of Sec. 4.4, Eq. Apotential).

Array layout of one MeshBlock with ``n`` interior cells per direction and ``g`` ghosts
(``N = n + 2g``, x fastest):

* vertex metric ``(16, Nz+1, Ny+1, Nx+1)``: alpha, beta^i, gamma_{xx,xy,xz,yy,yz,zz}, K_ij
* primitives ``(5, Nz, Ny, Nx)``: rho, u~^x, u~^y, u~^z, p; with a tabulated EOS ``(7, ...)``: rho, u~^i,
  p, Y_e, T (T as drawn; the stage derives its own from (rho, p, Y_e))
* faces: ``Bx (Nz, Ny, Nx+1)``, ``By (Nz, Ny+1, Nx)``, ``Bz (Nz+1, Ny, Nx)`` (densitised B^i)

Cell index ``i`` in ``[-g, n+g-1]`` has centre ``x0 + (i + 1/2) dx``; vertex and face index ``i`` in
``[-g, n+g]`` sit at ``x0 + i dx``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2311_04989


@dataclass
class BlockInput:
    n: tuple            # interior cells (nx, ny, nz)
    ng: int
    x0: tuple           # coordinate of vertex index 0
    dx: tuple
    metric: np.ndarray  # (16, Nz+1, Ny+1, Nx+1)
    W: np.ndarray       # (5, Nz, Ny, Nx)
    B: list = field(default_factory=list)   # [Bx, By, Bz]

    @property
    def N(self):
        return tuple(v + 2 * self.ng for v in self.n)


# ---------------------------------------------------------------------------------------------
# coordinates
# ---------------------------------------------------------------------------------------------
def _axis(n, g, x0, dx, stagger):
    """1D coordinates: stagger=0 -> cell centres, 1 -> vertices/faces."""
    if stagger:
        return x0 + np.arange(-g, n + g + 1) * dx
    return x0 + (np.arange(-g, n + g) + 0.5) * dx


def grid(n, g, x0, dx, stag=(0, 0, 0)):
    """Meshgrid (Z, Y, X) arrays of the requested staggering, shaped (z, y, x)."""
    ax = [_axis(n[d], g, x0[d], dx[d], stag[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


# ---------------------------------------------------------------------------------------------
# smooth random fields
# ---------------------------------------------------------------------------------------------
class SmoothField:
    """Sum of a few random Fourier modes on a box of size L, scaled to lie within [-1, 1]."""

    def __init__(self, rng: np.random.Generator, L: float, nmodes: int = 8, kmax: int = 3):
        self.k = rng.integers(-kmax, kmax + 1, size=(nmodes, 3)).astype(float) * (2 * np.pi / L)
        self.k[np.all(self.k == 0, axis=1)] = 2 * np.pi / L
        self.ph = rng.uniform(0, 2 * np.pi, nmodes)
        self.a = rng.uniform(0.5, 1.0, nmodes)
        self.a /= self.a.sum()

    def __call__(self, X, Y, Z):
        out = np.zeros_like(X)
        for k, ph, a in zip(self.k, self.ph, self.a):
            out += a * np.sin(k[0] * X + k[1] * Y + k[2] * Z + ph)
        return out


def metric_flat(n, g):
    m = np.zeros((16,) + tuple(v + 2 * g + 1 for v in n[::-1]))
    m[0] = 1.0
    m[4] = m[7] = m[9] = 1.0
    return m


def metric_perturbed(n, g, x0, dx, rng, amp=1e-2, L=1.0, with_K=False):
    """Flat metric plus smooth perturbations |delta g| <= amp of alpha, beta^i and gamma_ij."""
    X, Y, Z = grid(n, g, x0, dx, (1, 1, 1))
    m = metric_flat(n, g)
    for c in range(10):
        m[c] = m[c] + amp * SmoothField(rng, L)(X, Y, Z)
    if with_K:
        for c in range(10, 16):
            m[c] = amp * SmoothField(rng, L)(X, Y, Z)
    return m


def curl_B(n, g, x0, dx, A):
    """Face field B = curl A (discrete) from an edge vector potential.

    ``A(comp, X, Y, Z)`` returns A_comp; A_x lives on x-edges (cell centre in x, vertices in y,z),
    and cyclically.  The discrete divergence of the result vanishes to round-off."""
    Nx, Ny, Nz = (v + 2 * g for v in n)
    # edge arrays over the whole padded range
    Xe, Ye, Ze = grid(n, g, x0, dx, (0, 1, 1)); Ax = A(0, Xe, Ye, Ze)   # (Nz+1, Ny+1, Nx)
    Xe, Ye, Ze = grid(n, g, x0, dx, (1, 0, 1)); Ay = A(1, Xe, Ye, Ze)   # (Nz+1, Ny, Nx+1)
    Xe, Ye, Ze = grid(n, g, x0, dx, (1, 1, 0)); Az = A(2, Xe, Ye, Ze)   # (Nz, Ny+1, Nx+1)
    Bx = (Az[:, 1:, :] - Az[:, :-1, :]) / dx[1] - (Ay[1:, :, :] - Ay[:-1, :, :]) / dx[2]
    By = (Ax[1:, :, :] - Ax[:-1, :, :]) / dx[2] - (Az[:, :, 1:] - Az[:, :, :-1]) / dx[0]
    Bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / dx[0] - (Ax[:, 1:, :] - Ax[:, :-1, :]) / dx[1]
    assert Bx.shape == (Nz, Ny, Nx + 1) and By.shape == (Nz, Ny + 1, Nx) and Bz.shape == (Nz + 1, Ny, Nx)
    return [np.ascontiguousarray(Bx), np.ascontiguousarray(By), np.ascontiguousarray(Bz)]


def random_block(n=(16, 16, 16), g=3, x0=(0.0, 0.0, 0.0), dx=None, seed=0, L=1.0,
                 rho_range=(1e-10, 1e-3), u_max=0.5, theta_range=(1e-3, 1e-1),
                 sigma_range=(1e-3, 10.0), metric_amp=1e-2, with_K=False, flat=False,
                 fields=None, eos=None, T_range=(1e-5, 1e-2), ye_range=(0.05, 0.5)):
    """Smooth random block.  ``fields`` (a dict of SmoothField) lets several blocks sample the
    same global functions, so neighbouring blocks agree in their overlap.

    ``eos`` (a SyntheticEOS): tabulated-EOS block; T and Y_e are drawn as smooth fields in
    ``T_range`` (log-uniform) and ``ye_range`` and p = p(rho, T, Y_e) of that EOS (``theta_range``
    is then unused)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    if dx is None:
        dx = tuple(L / v for v in n)
    if fields is None:
        fields = make_fields(rng, L)
    X, Y, Z = grid(n, g, x0, dx)
    lr = np.log(rho_range)
    rho = np.exp(lr[0] + (lr[1] - lr[0]) * 0.5 * (1 + fields["rho"](X, Y, Z)))
    lt = np.log(theta_range)
    if eos is not None:
        if "temp" not in fields:
            rng2 = np.random.default_rng(SEED_BASE + seed + 104729)
            fields = dict(fields, temp=SmoothField(rng2, L), ye=SmoothField(rng2, L))
        lT = np.log(T_range)

        def thermo(Xe, Ye, Ze, rr):
            T = np.exp(lT[0] + (lT[1] - lT[0]) * 0.5 * (1 + fields["temp"](Xe, Ye, Ze)))
            ye = ye_range[0] + (ye_range[1] - ye_range[0]) * 0.5 * (1 + fields["ye"](Xe, Ye, Ze))
            return eos.p(rr, T, ye), T, ye
    else:
        def thermo(Xe, Ye, Ze, rr):
            tt = np.exp(lt[0] + (lt[1] - lt[0]) * 0.5 * (1 + fields["theta"](Xe, Ye, Ze)))
            return rr * tt, None, None
    p, T, ye = thermo(X, Y, Z, rho)
    W = np.zeros((5 if eos is None else 7,) + X.shape)
    W[0] = rho
    for c in range(3):
        W[1 + c] = u_max * fields[f"u{c}"](X, Y, Z) / np.sqrt(3.0)
    W[4] = p
    if eos is not None:
        W[5] = ye
        W[6] = T
    # field: A_i = sqrt(sigma p) a_i(x) / k, so that |B|^2 ~ sigma p in order of magnitude
    ls = np.log(sigma_range)
    kk = 2 * np.pi / L

    def A(comp, Xe, Ye, Ze):
        rr = np.exp(lr[0] + (lr[1] - lr[0]) * 0.5 * (1 + fields["rho"](Xe, Ye, Ze)))
        pp = thermo(Xe, Ye, Ze, rr)[0]
        ss = np.exp(ls[0] + (ls[1] - ls[0]) * 0.5 * (1 + fields["sigma"](Xe, Ye, Ze)))
        return np.sqrt(ss * pp) * fields[f"a{comp}"](Xe, Ye, Ze) / kk

    B = curl_B(n, g, x0, dx, A)
    if flat:
        metric = metric_flat(n, g)
    else:
        metric = metric_perturbed(n, g, x0, dx, np.random.default_rng(SEED_BASE + seed + 7919),
                                  amp=metric_amp, L=L, with_K=with_K)
        if fields.get("metric") is not None:
            Xv, Yv, Zv = grid(n, g, x0, dx, (1, 1, 1))
            metric = metric_flat(n, g)
            for c in range(16 if with_K else 10):
                base = 0.0 if c >= 10 else metric[c]
                metric[c] = base + metric_amp * fields["metric"][c](Xv, Yv, Zv)
    return BlockInput(tuple(n), g, tuple(x0), tuple(dx), metric, np.ascontiguousarray(W), B)


def make_fields(rng, L, shared_metric=False):
    f = {k: SmoothField(rng, L) for k in ("rho", "theta", "sigma", "u0", "u1", "u2", "a0", "a1", "a2")}
    f["metric"] = [SmoothField(rng, L) for _ in range(16)] if shared_metric else None
    return f


def uniform_block(n=(8, 8, 8), g=3, dx=(0.1, 0.1, 0.1), rho=1.0, u=(0.1, -0.2, 0.05), p=0.5,
                  B=(0.3, -0.2, 0.4), metric=None):
    """A uniform state; ``metric`` is an optional 16-vector of constant metric values."""
    N = tuple(v + 2 * g for v in n)
    W = np.zeros((5, N[2], N[1], N[0]))
    W[0] = rho
    for c in range(3):
        W[1 + c] = u[c]
    W[4] = p
    m = metric_flat(n, g)
    if metric is not None:
        for c in range(16):
            m[c] = metric[c]
    Bx = np.full((N[2], N[1], N[0] + 1), B[0])
    By = np.full((N[2], N[1] + 1, N[0]), B[1])
    Bz = np.full((N[2] + 1, N[1], N[0]), B[2])
    return BlockInput(tuple(n), g, (0.0, 0.0, 0.0), tuple(dx), m, W, [Bx, By, Bz])


# ---------------------------------------------------------------------------------------------
# 1D magnetised shock tube along x (16^3 block, Gamma = 5/3)
# ---------------------------------------------------------------------------------------------
def shock_tube_block(n=(16, 16, 16), g=3, left=(1.0, 1.0, 1.0), right=(0.125, 0.1, -1.0), Bx=0.5,
                     x_range=(-0.5, 0.5)):
    """left/right = (rho, p, B^y); Bx constant; u~ = 0; flat metric; discontinuity at x = 0."""
    L = x_range[1] - x_range[0]
    dx = (L / n[0], L / n[0], L / n[0])
    x0 = (x_range[0], 0.0, 0.0)
    N = tuple(v + 2 * g for v in n)
    X, _, _ = grid(n, g, x0, dx)
    W = np.zeros((5, N[2], N[1], N[0]))
    isL = X < 0
    W[0] = np.where(isL, left[0], right[0])
    W[4] = np.where(isL, left[1], right[1])
    Bxa = np.full((N[2], N[1], N[0] + 1), Bx)
    Xy, _, _ = grid(n, g, x0, dx, (0, 1, 0))
    By = np.where(Xy < 0, left[2], right[2]).astype(float)
    Bz = np.zeros((N[2] + 1, N[1], N[0]))
    return BlockInput(tuple(n), g, x0, dx, metric_flat(n, g), W, [Bxa, np.ascontiguousarray(By), Bz])


# ---------------------------------------------------------------------------------------------
# TOV star in isotropic coordinates (initial data of Sec. 4.1: K = 100, Gamma = 2)
# ---------------------------------------------------------------------------------------------
@dataclass
class TOV:
    rbar: np.ndarray     # isotropic radius grid (interior, increasing)
    rho: np.ndarray
    p: np.ndarray
    alpha: np.ndarray
    psi4: np.ndarray     # conformal factor^4
    R_iso: float         # isotropic surface radius
    M: float             # gravitational mass
    K: float
    Gamma: float

    def at(self, r):
        """(rho, p, alpha, psi4) at isotropic radius r (array)."""
        r = np.asarray(r, float)
        inside = r < self.R_iso
        rho = np.where(inside, np.interp(r, self.rbar, self.rho), 0.0)
        p = np.where(inside, np.interp(r, self.rbar, self.p), 0.0)
        rr = np.maximum(r, 0.5 * self.R_iso)   # exterior formulas are used only outside the star
        a_out = (1 - self.M / (2 * rr)) / (1 + self.M / (2 * rr))
        psi4_out = (1 + self.M / (2 * rr)) ** 4
        alpha = np.where(inside, np.interp(r, self.rbar, self.alpha), a_out)
        psi4 = np.where(inside, np.interp(r, self.rbar, self.psi4), psi4_out)
        return rho, p, alpha, psi4


def solve_tov(rho_c=1.28e-3, K=100.0, Gamma=2.0, npts=4000):
    """TOV equations in Schwarzschild radius, then mapped to isotropic radius and matched to
    isotropic Schwarzschild outside."""
    from scipy.integrate import solve_ivp

    def eps_of(p):
        rho = (p / K) ** (1 / Gamma)
        return rho, rho + p / (Gamma - 1)          # rest-mass and total energy density

    p_c = K * rho_c ** Gamma

    def rhs(r, y):
        m, p, phi, lnrb = y
        p = max(p, 0.0)
        rho, e = eps_of(p)
        if r == 0:
            return [0, 0, 0, 0]
        den = r * (r - 2 * m)
        dp = -(e + p) * (m + 4 * np.pi * r ** 3 * p) / den
        return [4 * np.pi * r ** 2 * e, dp, (m + 4 * np.pi * r ** 3 * p) / den,
                1 / (r * np.sqrt(1 - 2 * m / r))]

    def surface(r, y):
        return y[1] - 1e-14 * p_c
    surface.terminal = True
    r0 = 1e-6
    rho0, e0 = eps_of(p_c)
    y0 = [4 / 3 * np.pi * r0 ** 3 * e0, p_c, 0.0, np.log(r0)]
    sol = solve_ivp(rhs, (r0, 100.0), y0, events=surface, rtol=1e-11, atol=1e-14, dense_output=True,
                    max_step=0.01)
    R = sol.t[-1]
    r = np.linspace(r0, R, npts)
    m, p, phi, lnrb = sol.sol(r)
    M = m[-1]
    # isotropic radius: match rbar(R) to the exterior relation r = rbar (1 + M/(2 rbar))^2
    Rb = 0.5 * (R - M + np.sqrt(R * R - 2 * M * R))
    rbar = np.exp(lnrb - lnrb[-1]) * Rb
    # lapse: e^phi with phi(R) = 0.5 ln(1 - 2M/R)
    phi = phi - phi[-1] + 0.5 * np.log(1 - 2 * M / R)
    p = np.maximum(p, 0.0)
    rho = (p / K) ** (1 / Gamma)
    psi4 = (r / rbar) ** 2
    rbar = np.concatenate([[0.0], rbar])
    rho = np.concatenate([[rho_c], rho]); p = np.concatenate([[p_c], p])
    alpha = np.concatenate([[np.exp(phi[0])], np.exp(phi)])
    psi4 = np.concatenate([[psi4[0]], psi4])
    return TOV(rbar, rho, p, alpha, psi4, float(Rb), float(M), K, Gamma)


def star_block(n=(64, 64, 64), g=3, half_width=10.02, tov: TOV | None = None, centres=((0.0, 0.0, 0.0),),
               x0=None, dx=None, A_b=None, B_over_rho=None, f_atm=1e-13, rho_max=None):
    """Static star(s) in a conformally flat metric with gamma_ij = psi^4 delta_ij, beta = 0, K = 0.

    Several centres superpose the stars as psi = 1 + sum(psi_a - 1), alpha psi = 1 + sum(alpha_a psi_a - 1)
    (the reading of the paper's analytic superposition of the two stars' metrics).  The poloidal field is the curl of
    A = (-y A_phi, x A_phi, 0) with A_phi = A_b max(p - 0.04 p_max, 0) (Eq. Apotential), taken about each
    centre.  Density below the atmosphere f_atm rho_max is raised to it."""
    if tov is None:
        tov = solve_tov()
    if dx is None:
        dx = (2 * half_width / n[0],) * 3
    if x0 is None:
        x0 = (-half_width,) * 3
    rho_max = tov.rho[0] if rho_max is None else rho_max
    rho_atm = f_atm * rho_max
    p_atm = tov.K * rho_atm ** tov.Gamma

    def fields_at(X, Y, Z):
        rho = np.zeros_like(X); p = np.zeros_like(X)
        psi = np.ones_like(X); apsi = np.ones_like(X)
        for c in centres:
            r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
            r_, p_, a_, q4 = tov.at(r)
            rho += r_; p += p_
            ps = q4 ** 0.25
            psi += ps - 1; apsi += a_ * ps - 1
        return rho, p, apsi / psi, psi ** 4

    Xv, Yv, Zv = grid(n, g, x0, dx, (1, 1, 1))
    _, _, al, q4 = fields_at(Xv, Yv, Zv)
    assert np.all(al > 0)
    m = metric_flat(n, g)
    m[0] = al
    m[4] = m[7] = m[9] = q4
    X, Y, Z = grid(n, g, x0, dx)
    rho, p, _, _ = fields_at(X, Y, Z)
    rho = np.maximum(rho, rho_atm)
    p = np.maximum(p, p_atm)
    W = np.zeros((5,) + X.shape)
    W[0] = rho
    W[4] = p
    p_max = tov.p[0]
    if A_b is None:
        A_b = 0.0

    def A(comp, Xe, Ye, Ze):
        out = np.zeros_like(Xe)
        if comp == 2:
            return out
        for c in centres:
            r = np.sqrt((Xe - c[0]) ** 2 + (Ye - c[1]) ** 2 + (Ze - c[2]) ** 2)
            _, pp, _, _ = tov.at(r)
            Aphi = A_b * np.maximum(pp - 0.04 * p_max, 0.0)
            out += (-(Ye - c[1]) * Aphi) if comp == 0 else ((Xe - c[0]) * Aphi)
        return out

    B = curl_B(n, g, x0, dx, A)
    return BlockInput(tuple(n), g, tuple(x0), tuple(dx), m, np.ascontiguousarray(W), B)


# ---------------------------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------------------------
def amr_like_batch(nblocks=1024, sizes=(16, 24, 32), g=3, seed=3, L=1.0, levels=3, workers=1, **kw):
    """Blocks of uneven sizes drawn from ``sizes``, at ``levels`` refinement levels (dx, dx/2, dx/4),
    placed at random positions; all sample the same global smooth fields.  The sizes and positions are
    drawn in order from one seeded generator, then the blocks are built (in ``workers`` processes; the
    result does not depend on it)."""
    rng = np.random.default_rng(SEED_BASE + seed)
    fields = make_fields(rng, L, shared_metric=True)
    spec = []
    for b in range(nblocks):
        n = int(rng.choice(sizes))
        lev = int(rng.integers(0, levels))
        dxb = (L / 64) / (2 ** lev)
        x0 = tuple(rng.uniform(0, L - n * dxb, 3))
        spec.append((n, x0, dxb))
    args = [((sp[0],) * 3, g, sp[1], (sp[2],) * 3, seed, L, fields, kw) for sp in spec]
    if workers <= 1:
        return [_amr_block(a) for a in args]
    # worker processes (spawned: safe whatever the parent has initialised); numpy-bound in pieces too
    # small for threads to help
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_amr_block, args, chunksize=max(1, len(args) // (4 * workers))))


def _amr_block(a):
    n, g, x0, dx, seed, L, fields, kw = a
    return random_block(n, g, x0, dx, seed=seed, L=L, fields=fields, **kw)


# ---------------------------------------------------------------------------------------------
# full-stage throughput workload: two static stars in a superposed metric, nb^3 blocks of n^3
# ---------------------------------------------------------------------------------------------
class _Geom:
    def __init__(self, n, ng, dx):
        self.n, self.ng, self.dx = n, ng, dx


class BinaryStarMesh:
    """Two Gamma = 2, K = 100 TOV stars (rho_c = 1e-3) at x = +-sep/2 on [-L/2, L/2]^3, cut into
    nb^3 blocks of n^3 cells with ng ghosts.  Metric: conformally flat superposition (beta = 0,
    K_ij = 0); field: the poloidal vector potential of Eq. Apotential about each star, scaled so
    that max b^2 / max rho = b2_over_rho; atmosphere f_atm rho_max.  Fields are evaluated once on
    the global ghost-extended grid and sliced per block."""

    def __init__(self, nb=16, n=16, ng=3, L=64.0, rho_c=1e-3, sep=40.0, b2_over_rho=1e-2, f_atm=1e-13,
                 K=100.0, Gamma=2.0):
        self.nb, self.n, self.ng, self.L = nb, n, ng, L
        self.dx = L / (nb * n)
        self.tov = solve_tov(rho_c=rho_c, K=K, Gamma=Gamma)
        self.rho_max = rho_c
        self.rho_atm = f_atm * rho_c
        self.p_atm = K * self.rho_atm ** Gamma
        self.K, self.Gamma = K, Gamma
        centres = ((-sep / 2, 0.0, 0.0), (sep / 2, 0.0, 0.0))
        Ntot = nb * n
        x0 = -L / 2
        # global axes (ghost-extended)
        ac = x0 + (np.arange(-ng, Ntot + ng) + 0.5) * self.dx      # cells
        av = x0 + np.arange(-ng, Ntot + ng + 1) * self.dx          # vertices / faces

        def star_fields(X, Y, Z, what):
            out = [np.zeros_like(X) for _ in what]
            psi = np.ones_like(X) if ("alpha" in what or "psi4" in what) else None
            apsi = np.ones_like(X) if "alpha" in what else None
            for c in centres:
                r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
                r_, p_, a_, q4 = self.tov.at(r)
                for k, w in enumerate(what):
                    if w == "rho":
                        out[k] += r_
                    elif w == "p":
                        out[k] += p_
                if psi is not None:
                    ps = q4 ** 0.25
                    psi += ps - 1
                    if apsi is not None:
                        apsi += a_ * ps - 1
            for k, w in enumerate(what):
                if w == "alpha":
                    out[k] = apsi / psi
                elif w == "psi4":
                    out[k] = psi ** 4
            return out

        Z, Y, X = np.meshgrid(ac, ac, ac, indexing="ij")
        rho, p = star_fields(X, Y, Z, ("rho", "p"))
        del X, Y, Z
        self.rho = np.maximum(rho, self.rho_atm)
        self.p = np.maximum(p, self.p_atm)
        Z, Y, X = np.meshgrid(av, av, av, indexing="ij")
        self.alpha, self.psi4 = star_fields(X, Y, Z, ("alpha", "psi4"))
        del X, Y, Z
        assert np.all(self.alpha > 0)
        p_max = self.tov.p[0]

        def A(comp, X, Y, Z):
            out = np.zeros_like(X)
            for c in centres:
                r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
                _, pp, _, _ = self.tov.at(r)
                Aphi = np.maximum(pp - 0.04 * p_max, 0.0)
                out += (-(Y - c[1]) * Aphi) if comp == 0 else ((X - c[0]) * Aphi)
            return out

        # edge potentials on the global grid (A_z = 0)
        Ze, Ye, Xe = np.meshgrid(av, av, ac, indexing="ij"); Ax = A(0, Xe, Ye, Ze)   # (V, V, C)
        Ze, Ye, Xe = np.meshgrid(av, ac, av, indexing="ij"); Ay = A(1, Xe, Ye, Ze)   # (V, C, V)
        del Xe, Ye, Ze
        d = self.dx
        Bx = -(Ay[1:, :, :] - Ay[:-1, :, :]) / d                         # (C, C, V)
        By = (Ax[1:, :, :] - Ax[:-1, :, :]) / d                          # (C, V, C)
        Bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / d - (Ax[:, 1:, :] - Ax[:, :-1, :]) / d   # (V, C, C)
        del Ax, Ay
        # b^2 of the static fluid = |calB|^2_gamma = |B|^2 / psi^8 (B densitised, gamma = psi^4 delta)
        Bc2 = (0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1])) ** 2 + (0.5 * (By[:, 1:, :] + By[:, :-1, :])) ** 2 + \
              (0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])) ** 2
        psi4c = 0.125 * sum(self.psi4[a:a + Ntot + 2 * ng, b:b + Ntot + 2 * ng, c:c + Ntot + 2 * ng]
                            for a in (0, 1) for b in (0, 1) for c in (0, 1))
        b2max = np.max(Bc2 / psi4c ** 2)
        s = np.sqrt(b2_over_rho * self.rho.max() / b2max) if b2max > 0 else 0.0
        self.B = [Bx * s, By * s, Bz * s]
        self.A_b = s

    def blocks(self):
        """Per-block geometry objects (n, ng, dx), block id = bi + nb (bj + nb bk)."""
        return [_Geom((self.n,) * 3, self.ng, (self.dx,) * 3) for _ in range(self.nb ** 3)]

    def _slices(self, b, stag=(0, 0, 0)):
        nb, n, ng = self.nb, self.n, self.ng
        bi, bj, bk = b % nb, (b // nb) % nb, b // (nb * nb)
        N = n + 2 * ng
        return tuple(slice(o * n, o * n + N + s) for o, s in ((bk, stag[2]), (bj, stag[1]), (bi, stag[0])))

    def block(self, b) -> BlockInput:
        """Materialise block b as a BlockInput (for the oracle)."""
        n, ng = self.n, self.ng
        sc = self._slices(b)
        sv = self._slices(b, (1, 1, 1))
        W = np.zeros((5,) + (n + 2 * ng,) * 3)
        W[0] = self.rho[sc]
        W[4] = self.p[sc]
        m = np.zeros((16,) + (n + 2 * ng + 1,) * 3)
        m[0] = self.alpha[sv]
        m[4] = m[7] = m[9] = self.psi4[sv]
        B = [np.ascontiguousarray(self.B[d][self._slices(b, tuple(int(a == d) for a in range(3)))])
             for d in range(3)]
        bi, bj, bk = b % self.nb, (b // self.nb) % self.nb, b // (self.nb * self.nb)
        x0 = tuple(-self.L / 2 + o * n * self.dx for o in (bi, bj, bk))
        return BlockInput((n,) * 3, ng, x0, (self.dx,) * 3, m, W, B)

    def pack(self, layout):
        """numpy pools in the library layout: W (5, ncell), B [3 x nface], metric (10, nvert)."""
        nbk = self.nb ** 3
        W = np.zeros((5, layout.ncell))
        Bp = [np.zeros(layout.nface[d]) for d in range(3)]
        M = np.zeros((10, layout.nvert))
        for b in range(nbk):
            sc = self._slices(b)
            sv = self._slices(b, (1, 1, 1))
            c0 = layout.cell_off[b]
            r = self.rho[sc].ravel(); W[0, c0:c0 + r.size] = r
            W[4, c0:c0 + r.size] = self.p[sc].ravel()
            v0 = layout.vert_off[b]
            a = self.alpha[sv].ravel(); M[0, v0:v0 + a.size] = a
            q = self.psi4[sv].ravel()
            for c in (4, 7, 9):
                M[c, v0:v0 + q.size] = q
            for d in range(3):
                f = self.B[d][self._slices(b, tuple(int(a_ == d) for a_ in range(3)))].ravel()
                f0 = layout.face_off[b, d]
                Bp[d][f0:f0 + f.size] = f
        return W, Bp, M


# ---------------------------------------------------------------------------------------------
# synthetic tabulated EOS (stand-in for the CompOSE table of Sec. 2.2.1, which is not available)
# ---------------------------------------------------------------------------------------------
@dataclass
class EosTable:
    """Nodes of log p, log e (e = rho (1 + eps)) and c_s^2 on a uniform grid in (log rho, log T, Y_e)
    (natural logarithms).  Arrays are (n_Ye, n_T, n_rho), rho fastest."""
    n: tuple
    x0: tuple
    dx: tuple
    lp: np.ndarray
    le: np.ndarray
    cs2: np.ndarray
    eos: object = None       # the analytic EOS the nodes were sampled from (input generation only)

    def axis(self, a):
        return self.x0[a] + self.dx[a] * np.arange(self.n[a])

    @property
    def rho_range(self):
        return float(np.exp(self.x0[0])), float(np.exp(self.x0[0] + (self.n[0] - 1) * self.dx[0]))

    @property
    def T_range(self):
        return float(np.exp(self.x0[1])), float(np.exp(self.x0[1] + (self.n[1] - 1) * self.dx[1]))

    @property
    def ye_range(self):
        return float(self.x0[2]), float(self.x0[2] + (self.n[2] - 1) * self.dx[2])


class SyntheticEOS:
    """Cold polytrope + ideal gas + radiation with a composition dependence:

        p = K_Y rho^Gamma + rho T + a T^4,   K_Y = K (1 + 0.1 (Y_e - 0.25)),
        eps = K_Y rho^(Gamma-1)/(Gamma-1) + 1.5 T + 3 a T^4 / rho,

    T in units of the baryon mass.  eps satisfies the first law (d eps/d rho at fixed T equals
    (p - T dp/dT)/rho^2), p and e are increasing in T, and c_s^2 = (dp/drho at fixed entropy)/h
    with h = 1 + eps + p/rho."""

    def __init__(self, K=100.0, Gamma=2.0, a_rad=1.0):
        self.K, self.Gamma, self.a = K, Gamma, a_rad

    def KY(self, ye):
        return self.K * (1 + 0.1 * (ye - 0.25))

    def p(self, rho, T, ye):
        return self.KY(ye) * rho ** self.Gamma + rho * T + self.a * T ** 4

    def eps(self, rho, T, ye):
        return self.KY(ye) * rho ** (self.Gamma - 1) / (self.Gamma - 1) + 1.5 * T + 3 * self.a * T ** 4 / rho

    def cs2(self, rho, T, ye):
        G, a, KY = self.Gamma, self.a, self.KY(ye)
        p, eps = self.p(rho, T, ye), self.eps(rho, T, ye)
        dp_drho = G * KY * rho ** (G - 1) + T
        dp_dT = rho + 4 * a * T ** 3
        deps_drho = KY * rho ** (G - 2) - 3 * a * T ** 4 / rho ** 2
        deps_dT = 1.5 + 12 * a * T ** 3 / rho
        dT_drho_s = (p / rho ** 2 - deps_drho) / deps_dT      # along d eps = (p/rho^2) d rho
        return (dp_drho + dp_dT * dT_drho_s) / (1 + eps + p / rho)

    def table(self, n=(200, 128, 64), rho_range=(1e-15, 1e-2), T_range=(1e-7, 1e-1), ye_range=(0.01, 0.6)):
        x0 = (float(np.log(rho_range[0])), float(np.log(T_range[0])), float(ye_range[0]))
        dx = (float((np.log(rho_range[1]) - np.log(rho_range[0])) / (n[0] - 1)),
              float((np.log(T_range[1]) - np.log(T_range[0])) / (n[1] - 1)),
              float((ye_range[1] - ye_range[0]) / (n[2] - 1)))
        lr = x0[0] + dx[0] * np.arange(n[0])
        lT = x0[1] + dx[1] * np.arange(n[1])
        ye = x0[2] + dx[2] * np.arange(n[2])
        Y, T, R = np.meshgrid(ye, np.exp(lT), np.exp(lr), indexing="ij")
        lp = np.log(self.p(R, T, Y))
        le = np.log(R * (1 + self.eps(R, T, Y)))
        cs2 = self.cs2(R, T, Y)
        return EosTable(tuple(n), x0, dx, np.ascontiguousarray(lp), np.ascontiguousarray(le),
                        np.ascontiguousarray(cs2), self)


# ---------------------------------------------------------------------------------------------
# same-level block topology (ghost exchange of a multi-block RK step)
# ---------------------------------------------------------------------------------------------
def neighbour_slot(ox, oy, oz):
    """Index of the direction (ox, oy, oz) in {-1,0,1}^3 within a block's 27 neighbour entries."""
    return (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)


def block_grid_neighbours(nb, periodic=(True, True, True)):
    """Neighbour table of an nb[0] x nb[1] x nb[2] grid of equal blocks, block index
    (bz * nb[1] + by) * nb[0] + bx: nbr[b, neighbour_slot(o)] = the block adjacent in direction o, or -1
    at a non-periodic (outflow) boundary.  Slot 13 (o = 0) is the block itself."""
    nbx, nby, nbz = nb
    nbr = np.full((nbx * nby * nbz, 27), -1, np.int32)
    for bz in range(nbz):
        for by in range(nby):
            for bx in range(nbx):
                b = (bz * nby + by) * nbx + bx
                for oz in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for ox in (-1, 0, 1):
                            c = [bx + ox, by + oy, bz + oz]
                            ok = True
                            for a in range(3):
                                if not 0 <= c[a] < nb[a]:
                                    if periodic[a]:
                                        c[a] %= nb[a]
                                    else:
                                        ok = False
                            if ok:
                                nbr[b, neighbour_slot(ox, oy, oz)] = (c[2] * nby + c[1]) * nbx + c[0]
    return nbr


def split_block(bi: BlockInput, nb):
    """Cut a ghost-padded block into nb[0] x nb[1] x nb[2] equal sub-blocks (same ghost width) by copying
    windows of its arrays: ghost regions of the pieces are the neighbours' interiors (or the big block's
    own ghosts at its boundary).  Block order as in block_grid_neighbours."""
    n = [bi.n[a] // nb[a] for a in range(3)]
    assert all(n[a] * nb[a] == bi.n[a] for a in range(3))
    g = bi.ng
    out = []
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                o = (bx * n[0], by * n[1], bz * n[2])
                sc = (slice(o[2], o[2] + n[2] + 2 * g), slice(o[1], o[1] + n[1] + 2 * g), slice(o[0], o[0] + n[0] + 2 * g))
                sv = tuple(slice(s.start, s.stop + 1) for s in sc)
                W = np.ascontiguousarray(bi.W[(slice(None),) + sc])
                M = np.ascontiguousarray(bi.metric[(slice(None),) + sv])
                B = []
                for d in range(3):
                    sf = list(sc)
                    ax = 2 - d
                    sf[ax] = slice(sc[ax].start, sc[ax].stop + 1)
                    B.append(np.ascontiguousarray(bi.B[d][tuple(sf)]))
                x0 = tuple(bi.x0[a] + o[a] * bi.dx[a] for a in range(3))
                out.append(BlockInput(tuple(n), g, x0, bi.dx, M, W, B))
    return out
