"""FP64 CPU oracle for one GRMHD Runge-Kutta stage (arXiv:2311.04989, Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py`` may import this package.  The product path (the CUDA library and its
binding) never does, and it shares no code with it.

The numerical work lives in ``grmhd_oracle.cpp`` (plain C++ restating the paper's equations); this
module compiles it with ``g++`` into ``oracle/_lib/liboracle.so`` and marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grmhd_oracle.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle (FP64, no FMA contraction) if the source is newer than the library."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_LIBC = os.path.join(_LIBDIR, "liboracle_count.so")


def build_count(force: bool = False) -> str:
    """Operation-counting build of the stage (``real`` = an op-counting scalar, see flopcount.h)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    hdr = os.path.join(_HERE, "flopcount.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if force or not os.path.exists(_LIBC) or os.path.getmtime(_LIBC) < newest:
        tmp = _LIBC + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-DORACLE_COUNT_FLOPS", "-I", _HERE, "-o", tmp, _SRC])
        os.replace(tmp, _LIBC)
    return _LIBC


PHASES = ["cell_metric_and_field", "faces", "cell_efield", "corner_emf", "update_and_sources", "ct",
          "con2prim", "con2prim_atmosphere"]


class OGeom(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("ng", C.c_int32), ("dx", C.c_double * 3)]


class OTable(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("pad_", C.c_int32), ("x0", C.c_double * 3), ("dx", C.c_double * 3),
                ("lp", C.POINTER(C.c_double)), ("le", C.POINTER(C.c_double)), ("cs2", C.POINTER(C.c_double))]


class OParams(C.Structure):
    _fields_ = [("gamma_ad", C.c_double), ("rho_atm", C.c_double), ("p_atm", C.c_double),
                ("f_thr", C.c_double), ("W_max", C.c_double), ("M_max", C.c_double),
                ("tol", C.c_double), ("weno_eps", C.c_double), ("rk_g0", C.c_double),
                ("rk_g1", C.c_double), ("rk_beta", C.c_double), ("max_iter", C.c_int32),
                ("recon", C.c_int32), ("emf", C.c_int32), ("ceiling", C.c_int32),
                ("interp_order", C.c_int32), ("pad_", C.c_int32),
                ("eos", C.c_int32), ("pad2_", C.c_int32), ("T_atm", C.c_double), ("Ye_atm", C.c_double),
                ("h0", C.c_double), ("table", C.POINTER(OTable)), ("atm_band", C.c_double)]


def otable(tab) -> OTable:
    """C view of an EOS table object (attributes n, x0, dx, lp, le, cs2 with lp/le/cs2 float64 arrays
    of shape (n_Ye, n_T, n_rho)); the arrays are kept alive on the returned struct."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (tab.lp, tab.le, tab.cs2)]
    for a in arrs:
        assert a.shape == (tab.n[2], tab.n[1], tab.n[0])
    t = OTable((C.c_int32 * 3)(*tab.n), 0, (C.c_double * 3)(*tab.x0), (C.c_double * 3)(*tab.dx),
               *(a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs))
    t._keep = arrs
    return t


def table_hmin(tab) -> float:
    """Minimum specific enthalpy (e + p)/rho over the table's nodes."""
    t = otable(tab)
    return float(lib().oracle_table_hmin(C.byref(t)))


@dataclass
class Params:
    """Physical and numerical parameters of the stage (names follow the paper)."""
    gamma_ad: float = 2.0
    rho_atm: float = 1e-13          # f_atm * rho_max   (Sec. 3.5)
    p_atm: float | None = None      # p(rho_atm); None -> K rho_atm^Gamma
    K_poly: float = 100.0           # polytropic K used for p_atm (Sec. 2.2.1)
    f_thr: float = 1.0              # Sec. 3.5
    W_max: float = float(np.sqrt(1.0 + 20.0 ** 2))   # u~ <= 20 (Sec. 3.5)
    M_max: float = 1e4              # B^2/D ceiling (App. A; value is a reading)
    tol: float = 1e-10              # bracketing tolerance (Sec. 3.5)
    weno_eps: float = 1e-40
    rk_g0: float = 0.0
    rk_g1: float = 1.0
    rk_beta: float = 1.0
    max_iter: int = 100
    recon: int = 1                  # 0 PLM, 1 WENOZ, 2 WENO5, 3 PPM
    emf: int = 0                    # 0 upwinded corner average, 1 plain mean
    ceiling: int = 0                # 0 clamp W, 1 atmosphere
    interp_order: int = 2
    table: object = None            # EOS table (Sec. 2.2.1); None -> ideal gas
    T_atm: float = 1e-6             # atmosphere temperature (table)
    Ye_atm: float = 0.5             # atmosphere electron fraction (table)
    atm_band: float = 1e-12         # relative band above f_thr rho_atm that counts as reached (Sec. 3.5)

    @property
    def eos(self) -> int:
        return 0 if self.table is None else 1

    @property
    def nw(self) -> int:            # primitives per point
        return 7 if self.table is not None else 5

    @property
    def nq(self) -> int:            # conserved per point
        return 6 if self.table is not None else 5

    def c(self) -> OParams:
        p_atm = self.p_atm if self.p_atm is not None else self.K_poly * self.rho_atm ** self.gamma_ad
        o = OParams(self.gamma_ad, self.rho_atm, p_atm, self.f_thr, self.W_max, self.M_max,
                    self.tol, self.weno_eps, self.rk_g0, self.rk_g1, self.rk_beta,
                    self.max_iter, self.recon, self.emf, self.ceiling, self.interp_order, 0)
        o.atm_band = self.atm_band
        if self.table is not None:
            t = otable(self.table)
            h0 = getattr(self.table, "_oracle_h0", None)
            if h0 is None:
                h0 = float(lib().oracle_table_hmin(C.byref(t)))
                self.table._oracle_h0 = h0
            o.eos, o.T_atm, o.Ye_atm, o.h0 = 1, self.T_atm, self.Ye_atm, h0
            o.table = C.pointer(t)
            o._keep = t
        return o


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        u8 = C.POINTER(C.c_uint8)
        i32 = C.POINTER(C.c_int32)
        pp = C.POINTER(OParams)
        L.oracle_prim2con.argtypes = [C.c_int, dp, dp, dp, pp, dp]
        L.oracle_con2prim.argtypes = [C.c_int, dp, dp, dp, pp, dp, u8, i32]
        L.oracle_flux_points.argtypes = [C.c_int, C.c_int, dp, dp, dp, pp, dp, dp, dp]
        L.oracle_face_flux.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, pp, dp]
        L.oracle_sources.argtypes = [C.c_int, dp, dp, dp, dp, pp, dp]
        L.oracle_recon1d.argtypes = [C.c_int, C.c_int, dp, C.c_double, dp, dp]
        ip = C.POINTER(C.c_int32)
        L.oracle_interp_cells.argtypes = [C.POINTER(OGeom), dp, C.c_int, ip, ip, dp, dp]
        L.oracle_interp_faces.argtypes = [C.POINTER(OGeom), dp, C.c_int, C.c_int, ip, ip, dp]
        L.oracle_stage_block.argtypes = [C.POINTER(OGeom), dp, dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                         C.c_double, pp, dp, dp, dp, dp, dp, u8, i32]
        L.oracle_stage_block.restype = C.c_int
        L.oracle_stage_block_ex.argtypes = L.oracle_stage_block.argtypes + [dp, dp, dp, dp]
        L.oracle_stage_block_ex.restype = C.c_int
        L.oracle_divb_block.argtypes = [C.POINTER(OGeom), dp, dp, dp, dp]
        L.oracle_c2p_samples.argtypes = [C.c_int, dp, dp, dp, pp, dp, dp, u8]
        L.oracle_mlp_nparam.restype = C.c_int
        L.oracle_mlp_forward.argtypes = [dp, dp, C.c_int, dp]
        L.oracle_mlp_loss_grad.argtypes = [dp, dp, dp, C.c_int, dp, dp]
        L.oracle_table_eval.argtypes = [C.c_int, pp, dp, dp, dp, dp]
        L.oracle_table_hmin.argtypes = [C.POINTER(OTable)]
        L.oracle_table_hmin.restype = C.c_double
        L.oracle_adm_points.argtypes = [C.c_int, dp, dp, dp, pp, dp]
        L.oracle_adm_block.argtypes = [C.POINTER(OGeom), dp, dp, dp, dp, dp, pp, C.c_int, dp]
        L.oracle_adm_block.restype = C.c_int
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# pointwise entries
# ---------------------------------------------------------------------------------------------
def prim2con(metric, prims, Bdens, P: Params):
    """Eq. consB_def at points.  metric (n,16), prims (n,5), Bdens (n,3) -> q (n,5); with a table
    prims (n,7) = (rho, u~^i, p, Y_e, T; T unread) -> q (n,6)."""
    metric, prims, Bdens = _f64(metric), _f64(prims), _f64(Bdens)
    n = prims.shape[0]
    assert prims.shape[1] == P.nw
    q = np.zeros((n, P.nq))
    cp = P.c()
    lib().oracle_prim2con(n, _d(metric), _d(prims), _d(Bdens), C.byref(cp), _d(q))
    return q


def con2prim(metric, q, Bdens, P: Params):
    """Con2prim at points.  Returns (prims (n,nw), q_out (n,nq), status (n,), iterations (n,))."""
    metric, Bdens = _f64(metric), _f64(Bdens)
    q = _f64(q).copy()
    n = q.shape[0]
    assert q.shape[1] == P.nq
    w = np.zeros((n, P.nw))
    st = np.zeros(n, np.uint8)
    it = np.zeros(n, np.int32)
    cp = P.c()
    lib().oracle_con2prim(n, _d(metric), _d(q), _d(Bdens), C.byref(cp), _d(w),
                          st.ctypes.data_as(C.POINTER(C.c_uint8)),
                          it.ctypes.data_as(C.POINTER(C.c_int32)))
    return w, q, st, it


def flux_points(d, metric, prims, Bdens, P: Params):
    """Physical U (n,7), F^d (n,7) and (lam-, lam+) (n,2) of Eq. fluxB_def at points."""
    metric, prims, Bdens = _f64(metric), _f64(prims), _f64(Bdens)
    n = prims.shape[0]
    U = np.zeros((n, 7)); F = np.zeros((n, 7)); lam = np.zeros((n, 2))
    cp = P.c()
    lib().oracle_flux_points(n, d, _d(metric), _d(prims), _d(Bdens), C.byref(cp), _d(U), _d(F), _d(lam))
    return U, F, lam


def face_flux(d, metric, wL, BL, wR, BR, P: Params):
    """HLLE flux (n,7) at faces from left/right states; with a table (n,8), the D Y_e flux last."""
    metric, wL, BL, wR, BR = map(_f64, (metric, wL, BL, wR, BR))
    n = wL.shape[0]
    assert wL.shape[1] == P.nw
    F = np.zeros((n, 8 if P.table is not None else 7))
    cp = P.c()
    lib().oracle_face_flux(n, d, _d(metric), _d(wL), _d(BL), _d(wR), _d(BR), C.byref(cp), _d(F))
    return F


def sources(metric, dmetric, prims, Bdens, P: Params):
    """Eq. hydsrc_def at points.  dmetric (n,3,16)."""
    metric, dmetric, prims, Bdens = map(_f64, (metric, dmetric, prims, Bdens))
    n = prims.shape[0]
    s = np.zeros((n, 5))
    cp = P.c()
    lib().oracle_sources(n, _d(metric), _d(dmetric), _d(prims), _d(Bdens), C.byref(cp), _d(s))
    return s


def recon1d(method, w, eps=1e-40):
    """Face states L[f], R[f] between cells f-1 and f, for f in [3, n-3]."""
    w = _f64(w)
    n = w.shape[0]
    L = np.full(n, np.nan); R = np.full(n, np.nan)
    lib().oracle_recon1d(method, n, _d(w), eps, _d(L), _d(R))
    return L, R


# ---------------------------------------------------------------------------------------------
# block entries
# ---------------------------------------------------------------------------------------------
@dataclass
class Block:
    """One ghost-padded MeshBlock in the oracle's layout (see grmhd_oracle.cpp header)."""
    n: tuple
    ng: int
    dx: tuple
    metric: np.ndarray          # (16, Nz+1, Ny+1, Nx+1)
    W: np.ndarray               # (5, Nz, Ny, Nx)
    B: list = field(default_factory=list)   # [Bx (Nz,Ny,Nx+1), By (Nz,Ny+1,Nx), Bz (Nz+1,Ny,Nx)]

    def geom(self) -> OGeom:
        return OGeom((C.c_int32 * 3)(*self.n), self.ng, (C.c_double * 3)(*self.dx))


def _rng3(lo, hi):
    lo = (lo,) * 3 if np.isscalar(lo) else tuple(lo)
    hi = (hi,) * 3 if np.isscalar(hi) else tuple(hi)
    return (C.c_int32 * 3)(*lo), (C.c_int32 * 3)(*hi), int(np.prod(np.subtract(hi, lo)))


def interp_cells(blk: Block, order, lo, hi):
    """Metric values (m,16) and derivatives (m,3,16) at cell centres with index in [lo, hi)
    per direction (scalars or 3-tuples), x fastest."""
    g = blk.geom()
    clo, chi, m = _rng3(lo, hi)
    val = np.zeros((m, 16)); dval = np.zeros((m, 3, 16))
    lib().oracle_interp_cells(C.byref(g), _d(_f64(blk.metric)), order, clo, chi, _d(val), _d(dval))
    return val, dval


def interp_faces(blk: Block, order, d, lo, hi):
    g = blk.geom()
    clo, chi, m = _rng3(lo, hi)
    val = np.zeros((m, 16))
    lib().oracle_interp_faces(C.byref(g), _d(_f64(blk.metric)), order, d, clo, chi, _d(val))
    return val


def stage_block(blk: Block, U, U0, B0, dt, P: Params, return_iters=False):
    """One RK stage on one block.  Returns (U', [B'x,B'y,B'z], W', status[, iters]).

    Outputs keep the input's ghost-padded shape; ghost entries of U', B', W' are copies of the
    inputs (U, B, W) and status is 0 there."""
    g = blk.geom()
    metric = _f64(blk.metric)
    W = _f64(blk.W)
    B = [_f64(b) for b in blk.B]
    U = _f64(U); U0 = _f64(U0); B0 = [_f64(b) for b in B0]
    Uo = U.copy(); Wo = W.copy(); Bo = [b.copy() for b in B]
    st = np.zeros(W.shape[1:], np.uint8)
    it = np.zeros(W.shape[1:], np.int32)
    cp = P.c()
    r = lib().oracle_stage_block(C.byref(g), _d(metric), _d(W), _d(B[0]), _d(B[1]), _d(B[2]),
                                 _d(U), _d(U0), _d(B0[0]), _d(B0[1]), _d(B0[2]), float(dt),
                                 C.byref(cp), _d(Uo), _d(Bo[0]), _d(Bo[1]), _d(Bo[2]), _d(Wo),
                                 st.ctypes.data_as(C.POINTER(C.c_uint8)),
                                 it.ctypes.data_as(C.POINTER(C.c_int32)))
    if r != 0:
        raise ValueError("oracle_stage_block: ghost width too small for the stencil")
    if return_iters:
        return Uo, Bo, Wo, st, it
    return Uo, Bo, Wo, st


def stage_fluxes(blk: Block, U, U0, B0, dt, P: Params):
    """The face fluxes and corner EMFs one stage of this block computes: (F, E) with F[d] of shape
    (nq, *d-face array shape) and E[m] of the vertex-array shape (edge indexed by its low corner)."""
    return _stage_ex(blk, U, U0, B0, dt, P, None, None)[4:]


def stage_block_with(blk: Block, U, U0, B0, dt, P: Params, F, E):
    """One RK stage with the face fluxes F and corner EMFs E (layouts of stage_fluxes) taking the place
    of the block's own; returns (U', B', W', status) like stage_block."""
    return _stage_ex(blk, U, U0, B0, dt, P, F, E)[:4]


def _stage_ex(blk, U, U0, B0, dt, P, F_in, E_in):
    g = blk.geom()
    metric = _f64(blk.metric)
    W = _f64(blk.W)
    B = [_f64(b) for b in blk.B]
    U = _f64(U); U0 = _f64(U0); B0 = [_f64(b) for b in B0]
    Uo = U.copy(); Wo = W.copy(); Bo = [b.copy() for b in B]
    st = np.zeros(W.shape[1:], np.uint8)
    it = np.zeros(W.shape[1:], np.int32)
    nq = P.nq
    N = [v + 2 * blk.ng for v in blk.n]
    fshape = [(N[2] + (d == 2), N[1] + (d == 1), N[0] + (d == 0)) for d in range(3)]
    vshape = (N[2] + 1, N[1] + 1, N[0] + 1)
    Fout = np.zeros(sum(nq * int(np.prod(f)) for f in fshape))
    Eout = np.zeros(3 * int(np.prod(vshape)))
    Fin = np.concatenate([_f64(F_in[d]).ravel() for d in range(3)]) if F_in is not None else None
    Ein = np.concatenate([_f64(E_in[m]).ravel() for m in range(3)]) if E_in is not None else None
    cp = P.c()
    r = lib().oracle_stage_block_ex(C.byref(g), _d(metric), _d(W), _d(B[0]), _d(B[1]), _d(B[2]),
                                    _d(U), _d(U0), _d(B0[0]), _d(B0[1]), _d(B0[2]), float(dt),
                                    C.byref(cp), _d(Uo), _d(Bo[0]), _d(Bo[1]), _d(Bo[2]), _d(Wo),
                                    st.ctypes.data_as(C.POINTER(C.c_uint8)),
                                    it.ctypes.data_as(C.POINTER(C.c_int32)), _d(Fout), _d(Eout),
                                    _d(Fin) if Fin is not None else None, _d(Ein) if Ein is not None else None)
    if r != 0:
        raise ValueError("oracle_stage_block_ex: ghost width too small for the stencil")
    F, o = [], 0
    for d in range(3):
        sz = nq * int(np.prod(fshape[d]))
        F.append(Fout[o:o + sz].reshape((nq,) + fshape[d]))
        o += sz
    E = [Eout[m * int(np.prod(vshape)):(m + 1) * int(np.prod(vshape))].reshape(vshape) for m in range(3)]
    return Uo, Bo, Wo, st, F, E


_libc = None


def stage_block_count(blk: Block, U, U0, B0, dt, P: Params):
    """Run the counting build of the stage on one block; returns {phase: (add, mul, div, sqrt)}."""
    global _libc
    if _libc is None:
        L = C.CDLL(build_count())
        dp = C.POINTER(C.c_double)
        L.oracle_stage_block.argtypes = lib().oracle_stage_block.argtypes
        L.oracle_stage_block.restype = C.c_int
        L.oracle_flops_get.argtypes = [dp, C.c_int]
        _libc = L
    L = _libc
    g = blk.geom()
    metric, W = _f64(blk.metric), _f64(blk.W)
    B = [_f64(b) for b in blk.B]
    U = _f64(U); U0 = _f64(U0); B0 = [_f64(b) for b in B0]
    Uo = U.copy(); Wo = W.copy(); Bo = [b.copy() for b in B]
    st = np.zeros(W.shape[1:], np.uint8)
    it = np.zeros(W.shape[1:], np.int32)
    out = np.zeros(40)
    L.oracle_flops_get(_d(out), 1)
    cp = P.c()
    r = L.oracle_stage_block(C.byref(g), _d(metric), _d(W), _d(B[0]), _d(B[1]), _d(B[2]), _d(U), _d(U0),
                             _d(B0[0]), _d(B0[1]), _d(B0[2]), float(dt), C.byref(cp), _d(Uo), _d(Bo[0]),
                             _d(Bo[1]), _d(Bo[2]), _d(Wo), st.ctypes.data_as(C.POINTER(C.c_uint8)),
                             it.ctypes.data_as(C.POINTER(C.c_int32)))
    if r != 0:
        raise ValueError("oracle_stage_block (count build) failed")
    L.oracle_flops_get(_d(out), 1)
    return {ph: tuple(out[5 * k:5 * k + 4]) for k, ph in enumerate(PHASES)}


def divb(blk_n, ng, dx, B):
    g = OGeom((C.c_int32 * 3)(*blk_n), ng, (C.c_double * 3)(*dx))
    B = [_f64(b) for b in B]
    out = np.zeros((blk_n[2] + 2 * ng, blk_n[1] + 2 * ng, blk_n[0] + 2 * ng))
    lib().oracle_divb_block(C.byref(g), _d(B[0]), _d(B[1]), _d(B[2]), _d(out))
    return out


# ---------------------------------------------------------------------------------------------
# learned con2prim bracket (FP64 reference of the MLP and its training data)
# ---------------------------------------------------------------------------------------------
MLP_H, MLP_IN, MLP_OFF = 64, 6, 16
MLP_NW = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1
MLP_MEAN, MLP_ISTD, MLP_TMEAN, MLP_TSTD, MLP_STEP = 0, 6, 12, 13, 14


def c2p_samples(metric, q, Bdens, P: Params):
    """(features (n,6), log mu at the root (n,), valid (n,) bool) of the bracketed solves."""
    metric, q, Bdens = _f64(metric), _f64(q), _f64(Bdens)
    n = q.shape[0]
    assert q.shape[1] == P.nq
    f = np.zeros((n, MLP_IN)); t = np.zeros(n); v = np.zeros(n, np.uint8)
    cp = P.c()
    lib().oracle_c2p_samples(n, _d(metric), _d(q), _d(Bdens), C.byref(cp), _d(f), _d(t),
                             v.ctypes.data_as(C.POINTER(C.c_uint8)))
    return f, t, v.astype(bool)


def mlp_nparam():
    return int(lib().oracle_mlp_nparam())


def mlp_forward(P, x):
    P, x = _f64(P), _f64(x)
    t = np.zeros(x.shape[0])
    lib().oracle_mlp_forward(_d(P), _d(x), x.shape[0], _d(t))
    return t


def mlp_loss_grad(P, x, t):
    """Mean-squared-error loss in normalised units and its gradient w.r.t. the network weights."""
    P, x, t = _f64(P), _f64(x), _f64(t)
    g = np.zeros(MLP_NW)
    L = C.c_double()
    lib().oracle_mlp_loss_grad(_d(P), _d(x), _d(t), x.shape[0], _d(g), C.byref(L))
    return L.value, g


# ---------------------------------------------------------------------------------------------
# tabulated EOS lookups (Sec. 2.2.1)
# ---------------------------------------------------------------------------------------------
def table_eval(P: Params, rho, T, ye):
    """(p, eps, c_s^2) at (rho, T, Y_e) from the table and the temperature recovered from (rho, p, Y_e)."""
    rho, T, ye = _f64(rho), _f64(T), _f64(ye)
    n = rho.shape[0]
    out = np.zeros((n, 4))
    cp = P.c()
    lib().oracle_table_eval(n, C.byref(cp), _d(rho), _d(T), _d(ye), _d(out))
    return out[:, 0], out[:, 1], out[:, 2], out[:, 3]


# ---------------------------------------------------------------------------------------------
# matter sources of the spacetime equations (Sec. 2.1, 2.2) and their cell-to-vertex
# interpolation (Sec. 3.2)
# ---------------------------------------------------------------------------------------------
ADM_NAMES = ("rho_ADM", "S_x", "S_y", "S_z", "S_xx", "S_xy", "S_xz", "S_yy", "S_yz", "S_zz")


def adm_points(metric, prims, Bdens, P: Params):
    """(rho_ADM, S_i, S_ij) at points (n,10); layouts as prim2con."""
    metric, prims, Bdens = _f64(metric), _f64(prims), _f64(Bdens)
    n = prims.shape[0]
    assert prims.shape[1] == P.nw
    out = np.zeros((n, 10))
    cp = P.c()
    lib().oracle_adm_points(n, _d(metric), _d(prims), _d(Bdens), C.byref(cp), _d(out))
    return out


def adm_block(blk: Block, P: Params, vc_order: int = 2):
    """Matter sources of a block at its owned vertices (10, Nz+1, Ny+1, Nx+1); other vertices NaN."""
    g = blk.geom()
    N = [v + 2 * blk.ng for v in blk.n]
    out = np.full((10, N[2] + 1, N[1] + 1, N[0] + 1), np.nan)
    W = _f64(blk.W)
    assert W.shape[0] == P.nw
    Bx, By, Bz = (_f64(b) for b in blk.B)
    cp = P.c()
    rc = lib().oracle_adm_block(C.byref(g), _d(_f64(blk.metric)), _d(W), _d(Bx), _d(By), _d(Bz), C.byref(cp),
                                int(vc_order), _d(out))
    if rc != 0:
        raise ValueError("adm_block: ghost width too small for the interpolation orders")
    return out
