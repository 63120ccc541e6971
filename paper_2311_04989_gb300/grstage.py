"""Thin ctypes binding of libgrstage.so (include/grstage.h), same names as the C ABI.

Argument marshalling only: every step of the stage runs in the library's CUDA kernels.  PyTorch
supplies device memory and streams.  Importing works without a GPU; calling a ``gr_*`` function
loads the library and raises ``GrstageError`` if it is missing or a call fails -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgrstage.so")

GR_OK, GR_EINVAL, GR_ECUDA, GR_ENOMEM, GR_ETIMEOUT, GR_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
GR_RECON_PLM, GR_RECON_WENOZ, GR_RECON_WENO5, GR_RECON_PPM = 0, 1, 2, 3
GR_PREC_FP64, GR_PREC_MIXED = 0, 1
GR_EMF_UPWIND, GR_EMF_MEAN = 0, 1
GR_CEIL_CLAMP, GR_CEIL_ATMOSPHERE = 0, 1
GR_EOS_IDEAL, GR_EOS_TABLE = 0, 1
GR_ST_ATM_THRESHOLD, GR_ST_FAILED, GR_ST_W_CLAMPED = 0x01, 0x02, 0x04
GR_ST_TAU_FLOOR, GR_ST_BD_LIMIT, GR_ST_EOS_CLAMP = 0x08, 0x10, 0x20
GR_ST_GUESS_REJECTED = 0x40
GR_GUESS_NONE, GR_GUESS_FP32, GR_GUESS_MLP, GR_GUESS_AUTO = 0, 1, 2, 3

# every symbol include/grstage.h declares
EXPORTS = ["gr_strerror", "gr_last_error", "gr_abi_version", "gr_params_default", "gr_context_create",
           "gr_context_destroy", "gr_mesh_create", "gr_mesh_destroy", "gr_mesh_workspace_bytes",
           "gr_stage", "gr_prim2con", "gr_con2prim", "gr_diag", "gr_profile_begin", "gr_profile_end",
           "gr_diag_noalloc", "gr_noalloc_last_error", "gr_mlp_nparam", "gr_mlp_last_error", "gr_c2p_samples",
           "gr_mlp_forward", "gr_mlp_grad", "gr_mlp_train", "gr_graph_capture", "gr_graph_launch",
           "gr_graph_destroy", "gr_eos_create", "gr_eos_destroy", "gr_eos_bytes", "gr_eos_h0", "gr_autotune",
           "gr_mesh_get_shapes", "gr_mesh_set_shapes", "gr_driver_create", "gr_driver_destroy", "gr_ghost_fill",
           "gr_cfl_dt", "gr_driver_step", "gr_driver_capture", "gr_driver_dt", "gr_driver_dt_device",
           "gr_adm_sources", "gr_mesh_set_levels", "gr_restrict", "gr_prolong", "gr_host_stage", "gr_cast_f32",
           "gr_peak_alu", "gr_mesh_set_path", "gr_mesh_get_path", "gr_mesh_get_guess"]
GR_ABI_VERSION = 3
GR_MLP_NPARAM = 4689
GR_MLP_NIN = 6
MLP_MEAN, MLP_ISTD, MLP_TMEAN, MLP_TSTD, MLP_STEP = 0, 6, 12, 13, 14
GR_NKERNELS = 7
GR_NSTAGE_KERNELS = 6
GR_DT_GRID, GR_DT_SIGNAL = 0, 1
GR_MIXED_ATM_BAND = 1e-6
KERNEL_NAMES = ["k_cast", "k_cellprep", "k_faces", "k_edges", "k_ct", "k_update", "k_c2p"]


class GrstageError(RuntimeError):
    pass


class gr_block(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("ng", C.c_int32), ("dx", C.c_double * 3),
                ("cell_off", C.c_int64), ("face_off", C.c_int64 * 3), ("vert_off", C.c_int64)]


class gr_metric(C.Structure):
    _fields_ = [("v", C.c_void_p * 16), ("order", C.c_int32), ("k_zero", C.c_int32), ("v32", C.c_void_p * 16)]


class gr_state(C.Structure):
    _fields_ = [("U", C.c_void_p * 6), ("U0", C.c_void_p * 6), ("B", C.c_void_p * 3), ("B0", C.c_void_p * 3),
                ("W", C.c_void_p * 7), ("Uo", C.c_void_p * 6), ("Bo", C.c_void_p * 3), ("Wo", C.c_void_p * 7),
                ("status", C.c_void_p), ("W32", C.c_void_p * 6), ("B32", C.c_void_p * 3), ("Wo32", C.c_void_p * 6),
                ("Bo32", C.c_void_p * 3)]


class gr_shape(C.Structure):
    _fields_ = [("tile", C.c_int32), ("order", C.c_int32), ("persistent", C.c_int32)]


class gr_level_face(C.Structure):
    _fields_ = [("coarse", C.c_int32), ("fine", C.c_int32), ("dir", C.c_int32), ("side", C.c_int32),
                ("o1", C.c_int32), ("o2", C.c_int32)]


class gr_level_map(C.Structure):
    _fields_ = [("coarse", C.c_int32), ("fine", C.c_int32), ("off", C.c_int32 * 3), ("lo", C.c_int32 * 3),
                ("hi", C.c_int32 * 3)]


class gr_eos_table(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("pad_", C.c_int32), ("x0", C.c_double * 3), ("dx", C.c_double * 3),
                ("log_p", C.c_void_p), ("log_e", C.c_void_p), ("cs2", C.c_void_p)]


class gr_params(C.Structure):
    _fields_ = [("size", C.c_uint32), ("recon", C.c_int32), ("precision", C.c_int32), ("emf", C.c_int32),
                ("ceiling", C.c_int32), ("max_iter", C.c_int32), ("c2p_guess", C.c_int32), ("gamma_ad", C.c_double),
                ("rho_atm", C.c_double), ("p_atm", C.c_double), ("f_thr", C.c_double), ("W_max", C.c_double),
                ("M_max", C.c_double), ("tol", C.c_double), ("weno_eps", C.c_double), ("rk_g0", C.c_double),
                ("rk_g1", C.c_double), ("rk_beta", C.c_double), ("mlp", C.c_void_p), ("eos", C.c_int32),
                ("pad_", C.c_int32), ("table", C.c_void_p), ("T_atm", C.c_double), ("Ye_atm", C.c_double),
                ("atm_band", C.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgrstage.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise GrstageError(f"libgrstage.so not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, i32 = C.c_void_p, C.c_int32
    L.gr_strerror.restype = C.c_char_p
    L.gr_strerror.argtypes = [C.c_int]
    L.gr_last_error.restype = C.c_char_p
    L.gr_abi_version.restype = C.c_int
    L.gr_params_default.argtypes = [C.POINTER(gr_params)]
    L.gr_context_create.argtypes = [C.POINTER(vp), C.c_int]
    L.gr_context_destroy.argtypes = [vp]
    L.gr_mesh_create.argtypes = [vp, C.POINTER(gr_block), i32, i32, C.POINTER(vp)]
    L.gr_mesh_destroy.argtypes = [vp]
    L.gr_mesh_workspace_bytes.argtypes = [vp]
    L.gr_mesh_workspace_bytes.restype = C.c_int64
    L.gr_stage.argtypes = [vp, C.POINTER(gr_metric), C.POINTER(gr_state), C.c_double, C.POINTER(gr_params), vp]
    L.gr_prim2con.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 7, C.c_void_p * 3, C.c_void_p * 6,
                              C.POINTER(gr_params), vp]
    L.gr_con2prim.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 6, C.c_void_p * 3, C.c_void_p * 7, vp, vp,
                              C.POINTER(gr_params), vp]
    L.gr_autotune.argtypes = [vp, C.POINTER(gr_metric), C.POINTER(gr_state), C.c_double, C.POINTER(gr_params), i32,
                              vp, C.POINTER(C.c_double)]
    L.gr_mesh_get_shapes.argtypes = [vp, i32, i32, C.POINTER(gr_shape)]
    L.gr_mesh_set_shapes.argtypes = [vp, i32, i32, C.POINTER(gr_shape)]
    L.gr_eos_create.argtypes = [vp, C.POINTER(gr_eos_table), C.POINTER(vp)]
    L.gr_eos_destroy.argtypes = [vp]
    L.gr_eos_bytes.argtypes = [vp]
    L.gr_eos_bytes.restype = C.c_int64
    L.gr_eos_h0.argtypes = [vp]
    L.gr_eos_h0.restype = C.c_double
    L.gr_diag.argtypes = [vp, C.c_void_p * 5, C.c_void_p * 3, C.POINTER(C.c_double), vp]
    L.gr_cast_f32.argtypes = [vp, vp, C.c_int64, vp]
    L.gr_mesh_set_path.argtypes = [vp, i32]
    L.gr_mesh_get_path.argtypes = [vp]
    L.gr_mesh_get_guess.argtypes = [vp, i32, i32]
    L.gr_peak_alu.argtypes = [i32, i32, i32, C.c_int64, vp, C.POINTER(C.c_double), vp]
    L.gr_diag_noalloc.argtypes = [C.POINTER(gr_block), i32, C.c_void_p * 5, C.c_void_p * 3,
                                  C.POINTER(C.c_double), vp]
    L.gr_noalloc_last_error.restype = C.c_char_p
    L.gr_mlp_nparam.restype = C.c_int
    L.gr_mlp_last_error.restype = C.c_char_p
    L.gr_c2p_samples.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 6, C.c_void_p * 3, C.POINTER(gr_params),
                                 C.c_void_p * 6, vp, vp, vp]
    L.gr_mlp_forward.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.gr_mlp_grad.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp]
    L.gr_mlp_train.argtypes = [vp, vp, vp, C.c_int64, i32, i32, C.c_float, C.POINTER(C.c_float), vp]
    L.gr_graph_capture.argtypes = [vp, C.POINTER(gr_metric), C.POINTER(gr_state), C.c_double, C.POINTER(gr_params),
                                   C.POINTER(vp)]
    L.gr_graph_launch.argtypes = [vp, vp]
    L.gr_graph_destroy.argtypes = [vp]
    L.gr_profile_begin.argtypes = [vp, i32]
    L.gr_profile_end.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i32)]
    L.gr_driver_create.argtypes = [vp, vp, C.POINTER(vp)]
    L.gr_driver_destroy.argtypes = [vp]
    L.gr_ghost_fill.argtypes = [vp, C.c_void_p * 7, i32, C.c_void_p * 3, vp]
    L.gr_cfl_dt.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 7, C.c_void_p * 3, C.POINTER(gr_params),
                            C.c_double, vp, vp]
    L.gr_driver_step.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 6, C.c_void_p * 7, C.c_void_p * 3, vp,
                                 C.POINTER(gr_params), C.c_double, i32, i32, vp]
    L.gr_driver_capture.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 6, C.c_void_p * 7, C.c_void_p * 3, vp,
                                    C.POINTER(gr_params), C.c_double, i32, i32, C.POINTER(vp)]
    L.gr_driver_dt.argtypes = [vp, C.POINTER(C.c_double)]
    L.gr_driver_dt_device.argtypes = [vp]
    L.gr_driver_dt_device.restype = vp
    L.gr_host_stage.argtypes = [vp, C.POINTER(gr_metric), C.POINTER(gr_state), C.c_double, C.POINTER(gr_params), i32,
                                vp]
    L.gr_mesh_set_levels.argtypes = [vp, C.POINTER(gr_level_face), i32, C.POINTER(gr_level_map), i32,
                                     C.POINTER(gr_level_map), i32]
    L.gr_restrict.argtypes = [vp, C.c_void_p * 8, i32, vp, vp]
    L.gr_prolong.argtypes = [vp, C.c_void_p * 8, i32, vp, vp]
    L.gr_adm_sources.argtypes = [vp, C.POINTER(gr_metric), C.c_void_p * 7, C.c_void_p * 3, C.POINTER(gr_params), i32,
                                 C.c_void_p * 10, vp]
    for f in EXPORTS:
        if not hasattr(L, f):
            raise GrstageError(f"libgrstage.so lacks {f}")
    if L.gr_abi_version() != GR_ABI_VERSION:
        raise GrstageError("libgrstage.so ABI version mismatch")
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != GR_OK:
        L = load()
        raise GrstageError(f"{what}: {L.gr_strerror(rc).decode()} ({L.gr_last_error().decode()})")


def gr_params_default(**kw) -> gr_params:
    p = gr_params()
    load().gr_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def gr_context_create(device: int = 0):
    h = C.c_void_p()
    _check(load().gr_context_create(C.byref(h), device), "gr_context_create")
    return h


def gr_context_destroy(ctx):
    load().gr_context_destroy(ctx)


def gr_mesh_create(ctx, blocks: list[gr_block]):
    arr = (gr_block * max(1, len(blocks)))(*blocks)
    h = C.c_void_p()
    _check(load().gr_mesh_create(ctx, arr, len(blocks), 0, C.byref(h)), "gr_mesh_create")
    return h


def gr_mesh_destroy(mesh):
    load().gr_mesh_destroy(mesh)


def gr_mesh_workspace_bytes(mesh) -> int:
    return int(load().gr_mesh_workspace_bytes(mesh))


def _stream(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def gr_stage(mesh, metric: gr_metric, state: gr_state, dt: float, params: gr_params, stream=None):
    _check(load().gr_stage(mesh, C.byref(metric), C.byref(state), float(dt), C.byref(params), _stream(stream)),
           "gr_stage")


def _ptrs(n, ts):
    """Pointer array of n entries from tensors (or ints); missing trailing entries are NULL."""
    ts = list(ts)[:n]
    vals = [int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t) for t in ts]
    return (C.c_void_p * n)(*(vals + [0] * (n - len(vals))))


def gr_prim2con(mesh, metric: gr_metric, W, B, U, params: gr_params, stream=None):
    """W: 5 (ideal gas) or 6-7 (table: rho, u~^i, p, Y_e[, T]) cell pools; U: 5 or 6."""
    _check(load().gr_prim2con(mesh, C.byref(metric), _ptrs(7, W), _ptrs(3, B), _ptrs(6, U), C.byref(params),
                              _stream(stream)), "gr_prim2con")


def gr_con2prim(mesh, metric: gr_metric, U, B, W, status, params: gr_params, stream=None, evals=None):
    st = int(status.data_ptr()) if status is not None else 0
    ev = int(evals.data_ptr()) if evals is not None else 0
    _check(load().gr_con2prim(mesh, C.byref(metric), _ptrs(6, U), _ptrs(3, B), _ptrs(7, W), st, ev,
                              C.byref(params), _stream(stream)), "gr_con2prim")


class EosHandle:
    """gr_eos on a device; keep it alive while params reference it."""

    def __init__(self, h, nbytes, h0):
        self.h, self.nbytes, self.h0 = h, nbytes, h0

    def __int__(self):
        return int(self.h.value)


def gr_eos_create(ctx, table) -> EosHandle:
    """table: object with n, x0, dx and float64 arrays lp, le, cs2 of shape (n_Ye, n_T, n_rho)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (table.lp, table.le, table.cs2)]
    for a in arrs:
        assert a.shape == (table.n[2], table.n[1], table.n[0])
    t = gr_eos_table((C.c_int32 * 3)(*table.n), 0, (C.c_double * 3)(*table.x0), (C.c_double * 3)(*table.dx),
                     *(a.ctypes.data for a in arrs))
    h = C.c_void_p()
    L = load()
    _check(L.gr_eos_create(ctx, C.byref(t), C.byref(h)), "gr_eos_create")
    return EosHandle(h, int(L.gr_eos_bytes(h)), float(L.gr_eos_h0(h)))


def gr_eos_destroy(eos: EosHandle):
    load().gr_eos_destroy(eos.h)


def gr_diag(mesh, U, B, stream=None):
    out = (C.c_double * 4)()
    _check(load().gr_diag(mesh, _ptrs(5, list(U)[:5]), _ptrs(3, B), out, _stream(stream)), "gr_diag")
    return list(out)


def gr_cast_f32(src, dst, stream=None):
    """dst[:] = FP32 copy of the FP64 device tensor src (same number of elements), by the mixed path's
    conversion (IEEE round to nearest even)."""
    n = src.numel()
    if dst.numel() != n:
        raise ValueError("gr_cast_f32: size mismatch")
    _check(load().gr_cast_f32(C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()), C.c_int64(n),
                              _stream(stream)), "gr_cast_f32")


GR_PATH_SEPARATE, GR_PATH_FUSED, GR_PATH_TILED_FACES = 0, 1, 2
PATH_NAMES = {GR_PATH_SEPARATE: "separate kernels", GR_PATH_FUSED: "fused sweep", GR_PATH_TILED_FACES: "tiled face sweep"}


def gr_mesh_set_path(mesh, path: int):
    _check(load().gr_mesh_set_path(mesh, int(path)), "gr_mesh_set_path")


def gr_mesh_get_path(mesh) -> int:
    return int(load().gr_mesh_get_path(mesh))


def gr_mesh_get_guess(mesh, precision: int, eos: int = 0) -> int:
    """The bracket proposal GR_GUESS_AUTO stands for on this mesh (set by gr_autotune)."""
    return int(load().gr_mesh_get_guess(mesh, int(precision), int(eos)))


def gr_peak_alu(kind: int, blocks: int, threads: int, iters: int, sink, stream=None) -> float:
    """Launch one throughput loop (0 FP32 FMA, 1 packed FP32x2 FMA, 2 FP64 FMA); returns its flops."""
    f = C.c_double()
    rc = load().gr_peak_alu(kind, blocks, threads, C.c_int64(iters), C.c_void_p(sink.data_ptr()), C.byref(f),
                            _stream(stream))
    if rc != GR_OK:
        raise GrstageError(f"gr_peak_alu: {load().gr_strerror(rc).decode()}")
    return f.value


def gr_diag_noalloc(blocks: list[gr_block], U, B, stream=None):
    """gr_diag for at most 256 blocks without any device allocation (see include/grstage.h)."""
    arr = (gr_block * max(1, len(blocks)))(*blocks)
    out = (C.c_double * 4)()
    L = load()
    rc = L.gr_diag_noalloc(arr, len(blocks), _ptrs(5, list(U)[:5]), _ptrs(3, B), out, _stream(stream))
    if rc != GR_OK:
        raise GrstageError(f"gr_diag_noalloc: {L.gr_strerror(rc).decode()} ({L.gr_noalloc_last_error().decode()})")
    return list(out)


def gr_host_stage(mesh, metric: gr_metric, state: gr_state, dt: float, params: gr_params, nbatch: int = 8,
                  stream=None):
    """gr_stage on host-resident (pinned) pools: metric and state hold host pointers (see include/grstage.h)."""
    _check(load().gr_host_stage(mesh, C.byref(metric), C.byref(state), float(dt), C.byref(params), int(nbatch),
                                _stream(stream)), "gr_host_stage")


def gr_graph_capture(mesh, metric: gr_metric, state: gr_state, dt: float, params: gr_params):
    h = C.c_void_p()
    _check(load().gr_graph_capture(mesh, C.byref(metric), C.byref(state), float(dt), C.byref(params), C.byref(h)),
           "gr_graph_capture")
    return h


def gr_autotune(mesh, metric: gr_metric, state: gr_state, dt: float, params: gr_params, reps: int = 3, stream=None):
    """Pick the fastest launch shape of each stage kernel (see include/grstage.h); returns the chosen
    shapes as (tile, order, persistent) tuples and the mean ms of each kernel with its shape."""
    ms = (C.c_double * GR_NSTAGE_KERNELS)()
    _check(load().gr_autotune(mesh, C.byref(metric), C.byref(state), float(dt), C.byref(params), int(reps),
                              _stream(stream), ms), "gr_autotune")
    return gr_mesh_get_shapes(mesh, params.precision, params.eos), list(ms)


def gr_mesh_get_shapes(mesh, precision, eos=GR_EOS_IDEAL):
    arr = (gr_shape * GR_NSTAGE_KERNELS)()
    _check(load().gr_mesh_get_shapes(mesh, int(precision), int(eos), arr), "gr_mesh_get_shapes")
    return [(a.tile, a.order, a.persistent) for a in arr]


def gr_mesh_set_shapes(mesh, precision, eos, shapes):
    arr = (gr_shape * GR_NSTAGE_KERNELS)(*[gr_shape(*t) for t in shapes])
    _check(load().gr_mesh_set_shapes(mesh, int(precision), int(eos), arr), "gr_mesh_set_shapes")


def gr_graph_launch(graph, stream=None):
    _check(load().gr_graph_launch(graph, _stream(stream)), "gr_graph_launch")


def gr_graph_destroy(graph):
    load().gr_graph_destroy(graph)


ADM_NAMES = ("rho_ADM", "S_x", "S_y", "S_z", "S_xx", "S_xy", "S_xz", "S_yy", "S_yz", "S_zz")


def gr_adm_sources(mesh, metric: gr_metric, W, B, params: gr_params, vc_order, out, stream=None):
    """rho_ADM, S_i, S_ij at the owned vertices into the 10 vertex pools ``out`` (see include/grstage.h)."""
    _check(load().gr_adm_sources(mesh, C.byref(metric), _ptrs(7, W), _ptrs(3, B), C.byref(params), int(vc_order),
                                 _ptrs(10, out), _stream(stream)), "gr_adm_sources")


def _level_array(cls, items):
    items = list(items)
    arr = (cls * max(1, len(items)))()
    for k, it in enumerate(items):
        arr[k] = it if isinstance(it, cls) else cls(*[(C.c_int32 * 3)(*x) if isinstance(x, (tuple, list)) else x
                                                     for x in it])
    return arr, len(items)


def gr_mesh_set_levels(mesh, faces=(), restrict_maps=(), prolong_maps=()):
    """faces: (coarse, fine, dir, side, o1, o2) tuples; maps: (coarse, fine, off, lo, hi) with 3-tuples."""
    fa, nf = _level_array(gr_level_face, faces)
    ra, nr = _level_array(gr_level_map, restrict_maps)
    pa, npr = _level_array(gr_level_map, prolong_maps)
    _check(load().gr_mesh_set_levels(mesh, fa, nf, ra, nr, pa, npr), "gr_mesh_set_levels")


def _amr(fn, name, mesh, cells, B, stream):
    cells = list(cells)
    bp = _ptrs(3, B) if B is not None else None
    _check(fn(mesh, _ptrs(8, cells), len(cells), C.cast(bp, C.c_void_p) if bp is not None else None,
              _stream(stream)), name)


def gr_restrict(mesh, cells, B=None, stream=None):
    _amr(load().gr_restrict, "gr_restrict", mesh, cells, B, stream)


def gr_prolong(mesh, cells, B=None, stream=None):
    _amr(load().gr_prolong, "gr_prolong", mesh, cells, B, stream)


def gr_driver_create(mesh, nbr):
    """nbr: int32 array (n_blocks, 27) on the host; slot (oz+1)*9 + (oy+1)*3 + (ox+1) names the block
    across that face, edge or corner, -1 for an outflow side."""
    a = np.ascontiguousarray(nbr, dtype=np.int32)
    h = C.c_void_p()
    _check(load().gr_driver_create(mesh, a.ctypes.data, C.byref(h)), "gr_driver_create")
    return h


def gr_driver_destroy(driver):
    load().gr_driver_destroy(driver)


def gr_ghost_fill(driver, W, B, stream=None):
    W = list(W)
    _check(load().gr_ghost_fill(driver, _ptrs(7, W), len(W), _ptrs(3, B), _stream(stream)), "gr_ghost_fill")


def gr_cfl_dt(driver, metric: gr_metric, W, B, params: gr_params, cfl: float, dt_dev=None, stream=None):
    dp = int(dt_dev.data_ptr()) if dt_dev is not None else 0
    _check(load().gr_cfl_dt(driver, C.byref(metric), _ptrs(7, W), _ptrs(3, B), C.byref(params), float(cfl), dp,
                            _stream(stream)), "gr_cfl_dt")


def _step_args(metric, U, W, B, status, params, cfl, dt_mode, rk_order):
    st = int(status.data_ptr()) if status is not None else 0
    return (C.byref(metric), _ptrs(6, U), _ptrs(7, W), _ptrs(3, B), st, C.byref(params), float(cfl), int(dt_mode),
            int(rk_order))


def gr_driver_step(driver, metric: gr_metric, U, W, B, status, params: gr_params, cfl: float,
                   dt_mode: int = GR_DT_GRID, rk_order: int = 3, stream=None):
    _check(load().gr_driver_step(driver, *_step_args(metric, U, W, B, status, params, cfl, dt_mode, rk_order),
                                 _stream(stream)), "gr_driver_step")


def gr_driver_capture(driver, metric: gr_metric, U, W, B, status, params: gr_params, cfl: float,
                      dt_mode: int = GR_DT_GRID, rk_order: int = 3):
    h = C.c_void_p()
    _check(load().gr_driver_capture(driver, *_step_args(metric, U, W, B, status, params, cfl, dt_mode, rk_order),
                                    C.byref(h)), "gr_driver_capture")
    return h


def gr_driver_dt(driver) -> float:
    """dt of the driver's last step (synchronises with the device)."""
    v = C.c_double()
    _check(load().gr_driver_dt(driver, C.byref(v)), "gr_driver_dt")
    return float(v.value)


def gr_driver_dt_device(driver) -> int:
    return int(load().gr_driver_dt_device(driver) or 0)


def _mcheck(rc, what):
    if rc != GR_OK:
        L = load()
        raise GrstageError(f"{what}: {L.gr_strerror(rc).decode()} ({L.gr_mlp_last_error().decode()})")


def gr_c2p_samples(mesh, metric: gr_metric, U, B, params: gr_params, feats, target, valid, stream=None):
    _check(load().gr_c2p_samples(mesh, C.byref(metric), _ptrs(6, U), _ptrs(3, B), C.byref(params), _ptrs(6, feats),
                                 int(target.data_ptr()), int(valid.data_ptr()), _stream(stream)), "gr_c2p_samples")


def gr_mlp_forward(P, x, stream=None):
    import torch
    t = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _mcheck(load().gr_mlp_forward(int(P.data_ptr()), int(x.data_ptr()), x.shape[0], int(t.data_ptr()),
                                  _stream(stream)), "gr_mlp_forward")
    return t


def gr_mlp_grad(P, x, t, stream=None):
    import torch
    g = torch.empty(GR_MLP_NPARAM - 16, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _mcheck(load().gr_mlp_grad(int(P.data_ptr()), int(x.data_ptr()), int(t.data_ptr()), x.shape[0],
                               int(g.data_ptr()), int(loss.data_ptr()), _stream(stream)), "gr_mlp_grad")
    return float(loss.item()), g


def gr_mlp_train(P, x, t, epochs, batch=16384, lr=1e-3, stream=None):
    losses = (C.c_float * epochs)()
    _mcheck(load().gr_mlp_train(int(P.data_ptr()), int(x.data_ptr()), int(t.data_ptr()), x.shape[0], int(epochs),
                                int(batch), float(lr), losses, _stream(stream)), "gr_mlp_train")
    return list(losses)


def gr_profile_begin(mesh, max_stages: int):
    _check(load().gr_profile_begin(mesh, int(max_stages)), "gr_profile_begin")


def gr_profile_end(mesh):
    """Returns (ms per kernel summed over the profiled stages, number of stages)."""
    ms = (C.c_double * GR_NKERNELS)()
    n = C.c_int32()
    _check(load().gr_profile_end(mesh, ms, C.byref(n)), "gr_profile_end")
    return list(ms), int(n.value)


# ---------------------------------------------------------------------------------------------
# pool packing (device memory layout of a batch of blocks)
# ---------------------------------------------------------------------------------------------
@dataclass
class Layout:
    """Element offsets of every block in the cell / face / vertex pools."""
    n: list
    ng: list
    dx: list
    cell_off: np.ndarray
    face_off: np.ndarray   # (nb, 3)
    vert_off: np.ndarray
    ncell: int
    nface: tuple
    nvert: int

    @staticmethod
    def of(blocks, align: int = 32):
        """blocks: iterable of objects with .n (3-tuple), .ng, .dx.  Offsets are rounded up to
        ``align`` elements (256 B for FP64) so every block starts on an aligned address."""
        n, ng, dx = [], [], []
        co, fo, vo = [], [], []
        c = 0; f = [0, 0, 0]; v = 0
        up = lambda x: (x + align - 1) // align * align
        for b in blocks:
            N = [b.n[a] + 2 * b.ng for a in range(3)]
            n.append(tuple(b.n)); ng.append(b.ng); dx.append(tuple(b.dx))
            co.append(c); c = up(c + N[0] * N[1] * N[2])
            fo.append(tuple(f))
            for a in range(3):
                f[a] = up(f[a] + (N[0] + (a == 0)) * (N[1] + (a == 1)) * (N[2] + (a == 2)))
            vo.append(v); v = up(v + (N[0] + 1) * (N[1] + 1) * (N[2] + 1))
        return Layout(n, ng, dx, np.array(co, np.int64), np.array(fo, np.int64).reshape(-1, 3),
                      np.array(vo, np.int64), c, tuple(f), v)

    def descriptors(self) -> list[gr_block]:
        out = []
        for b in range(len(self.n)):
            out.append(gr_block((C.c_int32 * 3)(*self.n[b]), self.ng[b], (C.c_double * 3)(*self.dx[b]),
                                int(self.cell_off[b]), (C.c_int64 * 3)(*[int(x) for x in self.face_off[b]]),
                                int(self.vert_off[b])))
        return out

    def interior_cells(self) -> int:
        return int(sum(n[0] * n[1] * n[2] for n in self.n))


def metric_struct(metric_pool, order: int = 2, k_zero: bool = True, metric32=None) -> gr_metric:
    """metric_pool: (16, nvert) device tensor; metric32: optional FP32 copy of it (mixed path)."""
    m = gr_metric()
    for c in range(16):
        m.v[c] = int(metric_pool[c].data_ptr())
        if metric32 is not None:
            m.v32[c] = int(metric32[c].data_ptr())
    m.order = order
    m.k_zero = 1 if k_zero else 0
    return m


def set_fp32_copies(state: gr_state, W32=None, B32=None, Wo32=None, Bo32=None) -> gr_state:
    """Point the optional FP32 copies of a gr_state (mixed path) at device tensors: W32 / Wo32 up to 6
    cell pools, B32 / Bo32 three face pools (None leaves a group unset)."""
    if W32 is not None:
        for v in range(min(6, len(W32))):
            state.W32[v] = int(W32[v].data_ptr())
        for d in range(3):
            state.B32[d] = int(B32[d].data_ptr())
    if Wo32 is not None:
        for v in range(min(6, len(Wo32))):
            state.Wo32[v] = int(Wo32[v].data_ptr())
        for d in range(3):
            state.Bo32[d] = int(Bo32[d].data_ptr())
    return state


def state_struct(U, U0, B, B0, W, Uo, Bo, Wo, status) -> gr_state:
    """U, U0, Uo: 5 (or 6 with a table) cell pools; W, Wo: 5 (or 7) cell pools."""
    s = gr_state()
    for v in range(len(U)):
        s.U[v] = int(U[v].data_ptr())
        s.U0[v] = int(U0[v].data_ptr()) if U0 is not None else 0
        s.Uo[v] = int(Uo[v].data_ptr())
    for v in range(len(W)):
        s.W[v] = int(W[v].data_ptr())
        s.Wo[v] = int(Wo[v].data_ptr())
    for d in range(3):
        s.B[d] = int(B[d].data_ptr())
        s.B0[d] = int(B0[d].data_ptr()) if B0 is not None else 0
        s.Bo[d] = int(Bo[d].data_ptr())
    s.status = int(status.data_ptr())
    return s


def pack_blocks(blocks, device="cuda"):
    """Device pools (torch) of a list of blocks with numpy arrays W (5 or 7,...), B [3], metric (16,...).
    Returns (layout, W pool, [B pools], metric pool)."""
    import torch
    L = Layout.of(blocks)
    nw = np.asarray(blocks[0].W).shape[0] if len(blocks) else 5
    W = np.zeros((nw, max(L.ncell, 1)))
    M = np.zeros((16, max(L.nvert, 1)))
    Bp = [np.zeros(max(L.nface[d], 1)) for d in range(3)]
    for b, bi in enumerate(blocks):
        w = np.asarray(bi.W).reshape(nw, -1)
        W[:, L.cell_off[b]:L.cell_off[b] + w.shape[1]] = w
        m = np.asarray(bi.metric).reshape(16, -1)
        M[:, L.vert_off[b]:L.vert_off[b] + m.shape[1]] = m
        for d in range(3):
            f = np.asarray(bi.B[d]).ravel()
            Bp[d][L.face_off[b, d]:L.face_off[b, d] + f.size] = f
    to = lambda a: torch.from_numpy(a).to(device)
    return L, to(W), [to(x) for x in Bp], to(M)
