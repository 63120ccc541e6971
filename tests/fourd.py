"""Independent 4D-covariant restatements used to pin the oracle (test helper).

Nothing here follows the oracle's 3+1 formulas.  Everything is built from the 4-metric g_{mu nu},
the 4-velocity and the projected comoving field b^mu = (calB^mu + (calB.u) u^mu)/W, then the
conserved variables, fluxes and sources are read off standard covariant identities:

  D = sqrt(gamma) rho W,  S_j = alpha sqrt(gamma) T^0_j,  tau = alpha^2 sqrt(gamma) T^00 - D,
  F^i_D = alpha sqrt(gamma) rho u^i,  F^i_{S_j} = alpha sqrt(gamma) T^i_j,
  F^i_tau = sqrt(gamma) (alpha^2 T^{0i} - alpha rho u^i),
  F^i_{B^k} = alpha sqrt(gamma) (b^k u^i - b^i u^k),
  s_{S_j} = (1/2) alpha sqrt(gamma) T^{mu nu} d_j g_{mu nu}   (stationary metric),
  s_tau = alpha sqrt(gamma) (T^{mu 0} d_mu alpha - alpha T^{mu nu} Gamma^0_{mu nu}).
"""
import numpy as np

SYM = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def unpack(m16):
    a = m16[0]
    beta = np.array(m16[1:4])
    g = np.zeros((3, 3)); K = np.zeros((3, 3))
    for c, (i, j) in enumerate(SYM):
        g[i, j] = g[j, i] = m16[4 + c]
        K[i, j] = K[j, i] = m16[10 + c]
    return a, beta, g, K


def four_metric(a, beta, g):
    bl = g @ beta
    g4 = np.zeros((4, 4))
    g4[0, 0] = -a * a + beta @ bl
    g4[0, 1:] = g4[1:, 0] = bl
    g4[1:, 1:] = g
    return g4


def state(m16, w, Bdens, Gamma):
    """4D objects of one point: g4, g4 inverse, u^mu, b^mu, T^{mu nu}, sqrt(gamma)."""
    a, beta, g, K = unpack(m16)
    g4 = four_metric(a, beta, g)
    g4u = np.linalg.inv(g4)
    sg = np.sqrt(np.linalg.det(g))
    rho, ut, p = w[0], np.array(w[1:4]), w[4]
    W = np.sqrt(1 + ut @ g @ ut)
    u = np.zeros(4)
    u[0] = W / a
    u[1:] = ut - W * beta / a
    calB = np.zeros(4)
    calB[1:] = np.array(Bdens) / sg
    Bu = calB @ g4 @ u
    b = (calB + Bu * u) / W
    b2 = b @ g4 @ b
    eps = p / ((Gamma - 1) * rho)
    h = 1 + eps + p / rho
    T = (rho * h + b2) * np.outer(u, u) + (p + 0.5 * b2) * g4u - np.outer(b, b)
    return dict(a=a, beta=beta, g=g, K=K, g4=g4, g4u=g4u, sg=sg, u=u, b=b, b2=b2, T=T, rho=rho,
                p=p, h=h, W=W, eps=eps)


def cons(S):
    a, sg, T, g4 = S["a"], S["sg"], S["T"], S["g4"]
    D = sg * S["rho"] * S["W"]
    Tmix = T @ g4           # T^mu_nu
    Sj = a * sg * Tmix[0, 1:]
    tau = a * a * sg * T[0, 0] - D
    return np.array([D, *Sj, tau])


def flux(S, d):
    a, sg, T, g4, u, b = S["a"], S["sg"], S["T"], S["g4"], S["u"], S["b"]
    i = d + 1
    Tmix = T @ g4
    FD = a * sg * S["rho"] * u[i]
    FS = a * sg * Tmix[i, 1:]
    Ft = sg * (a * a * T[0, i] - a * S["rho"] * u[i])
    t1, t2 = (d + 1) % 3 + 1, (d + 2) % 3 + 1
    FB = [a * sg * (b[k] * u[i] - b[i] * u[k]) for k in (t1, t2)]
    return np.array([FD, *FS, Ft, *FB])


def speeds(S, d, Gamma):
    """Roots of (k.u)^2 (1 - c^2) = c^2 k.k for k_mu = (-lam, delta^d_i)."""
    cs2 = Gamma * S["p"] / (S["rho"] * S["h"])
    ca2 = S["b2"] / (S["rho"] * S["h"] + S["b2"])
    c2 = cs2 + ca2 - cs2 * ca2
    u, gu = S["u"], S["g4u"]
    i = d + 1
    # (u^i - lam u^0)^2 (1 - c2) - c2 (gu00 lam^2 - 2 gu0i lam + guii) = 0
    A = u[0] ** 2 * (1 - c2) - c2 * gu[0, 0]
    Bc = -2 * u[0] * u[i] * (1 - c2) + 2 * c2 * gu[0, i]
    Cc = u[i] ** 2 * (1 - c2) - c2 * gu[i, i]
    r = np.roots([A, Bc, Cc])
    r = np.sort(r.real)
    return r[0], r[1]


def christoffel0(g4, dg4):
    """Gamma^0_{mu nu} from g and its derivatives dg4[l] = d_l g_{mu nu} (l = 0..3)."""
    g4u = np.linalg.inv(g4)
    G = np.zeros((4, 4))
    for m in range(4):
        for n in range(4):
            G[m, n] = 0.5 * sum(g4u[0, l] * (dg4[m][l, n] + dg4[n][l, m] - dg4[l][m, n]) for l in range(4))
    return G


def sources_stationary(S, dm):
    """Sources of a stationary metric.  dm[k] = d_k of the 16 metric components (k = x,y,z)."""
    a, beta, g = S["a"], S["beta"], S["g"]
    dg4 = [np.zeros((4, 4))]       # d_t g = 0
    for k in range(3):
        da, dbeta, dg, _ = unpack(dm[k])
        # d_k of g4 components
        bl = g @ beta
        dbl = dg @ beta + g @ dbeta
        G = np.zeros((4, 4))
        G[0, 0] = -2 * a * da + dbeta @ bl + beta @ dbl
        G[0, 1:] = G[1:, 0] = dbl
        G[1:, 1:] = dg
        dg4.append(G)
    T, sg = S["T"], S["sg"]
    sS = [0.5 * a * sg * np.sum(T * dg4[1 + k]) for k in range(3)]
    dalpha = np.array([0.0] + [unpack(dm[k])[0] for k in range(3)])
    G0 = christoffel0(S["g4"], dg4)
    stau = a * sg * (T[:, 0] @ dalpha - a * np.sum(T * G0))
    return np.array([0.0, *sS, stau])


def stationary_K(m16, dm):
    """K_ij of a stationary slicing: d_t gamma_ij = 0 = -2 alpha K_ij + D_i beta_j + D_j beta_i."""
    a, beta, g, _ = unpack(m16)
    gu = np.linalg.inv(g)
    dg = np.array([unpack(dm[k])[2] for k in range(3)])        # dg[k][i][j]
    dbeta = np.array([unpack(dm[k])[1] for k in range(3)])     # dbeta[k][i] = d_k beta^i
    # 3-Christoffel Gamma^l_{ij}
    Gam = np.zeros((3, 3, 3))
    for l in range(3):
        for i in range(3):
            for j in range(3):
                Gam[l, i, j] = 0.5 * sum(gu[l, m] * (dg[i][m, j] + dg[j][m, i] - dg[m][i, j]) for m in range(3))
    bl = g @ beta
    # d_i beta_j = d_i (g_jk beta^k)
    dbl = np.array([[dg[i][j] @ beta + g[j] @ dbeta[i] for j in range(3)] for i in range(3)])
    Db = dbl - np.einsum("lij,l->ij", Gam, bl)
    return (Db + Db.T) / (2 * a)
