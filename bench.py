#!/usr/bin/env python
"""Benchmark: GRMHD cell-updates/s per Runge-Kutta stage on one GB300.

Workload (full-stage throughput): 256^3 cells as 4096 MeshBlocks of 16^3 (3 ghosts) on [-32, 32]^3,
two Gamma = 2, K = 100 TOV stars (rho_c = 1e-3) at x = +-20 in their superposed conformally flat
metric, poloidal field with max b^2 / max rho = 1e-2, atmosphere 1e-13 rho_max, WENOZ + HLLE.
A step is one gr_stage call over all blocks (metric interpolation, reconstruction, HLLE, corner
EMFs, CT update, flux divergence + sources, con2prim).  Inputs are synthetic (seeded/analytic) and
resident in HBM (~25 GB, far larger than L2, so no flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is the mixed-precision path (FP32 reconstruction / HLLE / EMF,
FP64 accumulation, CT and con2prim); the plain FP64 path is reported beside it.  Multi-GPU runs are
independent replicas (the stage needs no exchange inside a step); value sums all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GRMHD cell-updates/s per RK stage"
UNIT = "cell-updates/s"
GUESS_NAMES = {0: "none", 1: "fp32"}
WORKLOAD = "two-star full-stage throughput: 4096 blocks of 16^3 (ng=3), WENOZ+HLLE, CT, con2prim"
# con2prim bracket proposal of the timed mixed stage (--guess; the con2prim_guess / con2prim_table
# sections time every proposal on their own workloads)
MIXED_GUESS = 3   # GR_GUESS_AUTO, set from --guess in main()
FP64_NOMINAL_TFLOPS = 1.25      # nominal dense FP64 of the GB300 (context only; the roofline uses the measured rate)


def _hbm_peak():
    """Measured copy bandwidth of this machine's GPUs (GB/s) and where it came from."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


MEASURED_HBM_GBS, HBM_PEAK_SOURCE = _hbm_peak()


def env_rank():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def max_over_ranks(ms, dist, dev):
    """The job's time: the slowest rank's (an all-reduce MAX; the value itself on one process)."""
    import torch
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed (replicas: the same per rank) over the job's
    time in ms."""
    return units_per_rank * world / (ms / 1e3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nb", type=int, default=16, help="blocks per dimension (16 -> 4096 blocks)")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-c2p", action="store_true", help="skip the con2prim bracket-guess timings")
    ap.add_argument("--no-table", action="store_true", help="skip the tabulated-EOS con2prim workload")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of gr_autotune's")
    ap.add_argument("--no-rk", action="store_true", help="skip the timing of a whole RK3 driver step")
    ap.add_argument("--no-adm", action="store_true", help="skip the timing of the matter-source outputs")
    ap.add_argument("--no-configs", action="store_true", help="skip the smaller configurations (C1-C3)")
    ap.add_argument("--path", default="auto", choices=["auto", "separate", "fused", "tiled"],
                    help="path of the mixed stage: the autotuner's choice, or one forced")
    ap.add_argument("--e2e-batches", type=int, default=8, help="block batches of the host-buffer stage")
    ap.add_argument("--only-config", default=None, choices=["C1", "C2", "C3"],
                    help="time only this smaller configuration (GPU, --precision, --no-autotune honoured) and "
                         "print its figures (no headline line); for profiling one configuration's kernels")
    ap.add_argument("--config-blocks", type=int, default=1024, help="blocks of the AMR-like batch (C3)")
    ap.add_argument("--guess", default="auto", choices=["auto", "none", "fp32"],
                    help="con2prim bracket proposal of the mixed stage (headline and smaller configurations); "
                         "auto: the autotuner times none and the FP32 pre-solve on the workload and keeps the faster")
    a = ap.parse_args()
    if a.warmup < 3:
        a.warmup = 3
    return a


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# arithmetic-pipe peaks, measured on this GPU (FFMA, packed FFMA2, DFMA throughput loops)
# ---------------------------------------------------------------------------------------------
def measure_alu_peaks(G, torch, dev, seconds=1.5):
    """Peak FP32 (FFMA and packed FFMA2) and FP64 (DFMA) rates of the GPU: gr_peak_alu's loops of
    independent FMA chains on every SM (8 CTAs of 256 threads per SM), sized to run ~0.3 s per launch,
    timed with CUDA events over ~`seconds` per pipe, with the SM clock sampled meanwhile."""
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    blocks, threads = 8 * nsm, 256
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {"sm_count": nsm, "blocks": blocks, "threads": threads, "source": "measured: gr_peak_alu loops"}
    names = {0: "fp32_ffma", 1: "fp32x2_ffma2", 2: "fp64_dfma"}
    clk = ClockSampler(dev.index if dev.index is not None else 0)
    clk.start()
    for kind, name in names.items():
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        iters = 1 << 12
        while True:   # calibrate: one launch of ~0.3 s
            e0.record(stream)
            G.gr_peak_alu(kind, blocks, threads, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if ms > 100 or iters > (1 << 30):
                break
            iters *= 4
        iters = max(1, int(iters * 300.0 / ms))
        reps = max(1, int(seconds * 1e3 / 300.0))
        fl = 0.0
        e0.record(stream)
        for _ in range(reps):
            fl += G.gr_peak_alu(kind, blocks, threads, iters, sink, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"tflops": fl / (ms / 1e3) / 1e12, "ms": ms, "launches": reps}
    out["clocks"] = clk.stop()
    mhz = out["clocks"].get("sm_mhz")
    if mhz:
        for name in names.values():
            out[name]["flops_per_sm_per_clock"] = out[name]["tflops"] * 1e12 / (nsm * mhz * 1e6)
    out["fp32_tflops"] = max(out["fp32_ffma"]["tflops"], out["fp32x2_ffma2"]["tflops"])
    out["fp64_tflops"] = out["fp64_dfma"]["tflops"]
    return out


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on host cores
# ---------------------------------------------------------------------------------------------
def oracle_sample(mesh, seconds, nthreads):
    """Time the oracle's stage on a seeded random sample of blocks with nthreads host threads (the
    ctypes call releases the GIL).  Returns (cell-updates/s, cells, wall seconds, blocks)."""
    import concurrent.futures as cf

    import numpy as np

    import oracle as O
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=mesh.rho_atm, p_atm=mesh.p_atm, tol=1e-10)
    dt = 0.25 * mesh.dx
    rng = np.random.default_rng(2311_04989)
    order = rng.permutation(mesh.nb ** 3)

    def prep(b):
        bi = mesh.block(int(b))
        blk = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
        g = bi.ng
        val, _ = O.interp_cells(blk, 2, (-g,) * 3, tuple(v + g for v in bi.n))
        Bx, By, Bz = bi.B
        Bc = np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]), 0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                       0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], -1).reshape(-1, 3)
        q = O.prim2con(val, np.moveaxis(bi.W, 0, -1).reshape(-1, 5), Bc, P)
        U = np.ascontiguousarray(np.moveaxis(q.reshape(bi.W.shape[1:] + (5,)), -1, 0))
        return blk, U

    def one(item):
        blk, U = item
        O.stage_block(blk, U, U, blk.B, dt, P)
        return blk.n[0] * blk.n[1] * blk.n[2]

    O.lib()
    # estimate the per-block cost on one prepared block, then size the sample to the budget
    probe = prep(order[0])
    t = time.perf_counter()
    one(probe)
    per_block = max(time.perf_counter() - t, 1e-4)
    done = int(min(len(order), max(nthreads, seconds * nthreads / per_block)))
    items = [probe] + [prep(b) for b in order[1:done]]
    t1 = time.perf_counter()
    with cf.ThreadPoolExecutor(nthreads) as ex:
        cells = sum(ex.map(one, items))
    wall = time.perf_counter() - t1
    return cells / wall, cells, wall, done


def oracle_errors(torch, mesh_in, L, got, dt):
    """Per-variable error of the mixed stage output (device pools `got` = (W, B faces, U, status)) against
    the FP64 oracle's stage at the same atmosphere band (1e-6) and tolerance (1e-10), on sampled blocks of
    the workload: both star centres, a star-surface block, atmosphere blocks and corners (the measures of
    MEASURES, over those blocks).  Runs the oracle (the CPU-baseline leg's program) once per block."""
    import numpy as np

    import oracle as O
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10, atm_band=1e-6)
    nb = mesh_in.nb
    centre = lambda x: int((x + mesh_in.L / 2) // (mesh_in.L / nb))
    pick = lambda i, j, k: i + nb * (j + nb * k)
    h = nb // 2
    sample = sorted({pick(centre(-20), h, h), pick(centre(20), h - 1, h - 1), pick(min(nb - 1, centre(20) + 2), h, h),
                     pick(h, h, h), pick(0, 0, 0), pick(nb - 1, nb - 1, nb - 1)})
    Wg, Bg, Ug, sg = got
    acc = {}
    for b in sample:
        bi = mesh_in.block(b)
        g, n = bi.ng, bi.n
        N = [n[d] + 2 * g for d in range(3)]
        blk = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
        val, _ = O.interp_cells(blk, 2, (-g,) * 3, tuple(v + g for v in n))
        Bx, By, Bz = bi.B
        Bc = np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]), 0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                       0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], -1).reshape(-1, 3)
        q = O.prim2con(val, np.moveaxis(bi.W, 0, -1).reshape(-1, 5), Bc, P)
        U = np.ascontiguousarray(np.moveaxis(q.reshape(bi.W.shape[1:] + (5,)), -1, 0))
        Uo, Bo, Wo, st = O.stage_block(blk, U, U, blk.B, dt, P)
        c0, nc = int(L.cell_off[b]), N[0] * N[1] * N[2]
        sl = (slice(g, g + n[2]), slice(g, g + n[1]), slice(g, g + n[0]))
        gU = Ug[:, c0:c0 + nc].cpu().numpy().reshape(5, N[2], N[1], N[0])
        gW = Wg[:5, c0:c0 + nc].cpu().numpy().reshape(5, N[2], N[1], N[0])
        gs = sg[c0:c0 + nc].cpu().numpy().reshape(N[2], N[1], N[0])
        ru, gu, rw, gw = Uo[(slice(None),) + sl], gU[(slice(None),) + sl], Wo[(slice(None),) + sl], gW[(slice(None),) + sl]
        e = {}
        scale = np.abs(ru[0]) + np.abs(ru[4])
        for v, name in enumerate(("D", "S_x", "S_y", "S_z", "tau")):
            den = np.maximum(np.abs(ru[v]), 1e-300) if v == 0 else np.maximum(np.abs(ru[v]), scale)
            e[name] = float(np.max(np.abs(gu[v] - ru[v]) / den))
        for v, name in enumerate(("rho", "u_x", "u_y", "u_z", "p")):
            d = np.abs(gw[v] - rw[v])
            e[name] = float(np.max(d if v in (1, 2, 3) else d / np.maximum(np.abs(rw[v]), 1e-300)))
        for d_, name in enumerate(("B_x", "B_y", "B_z")):
            sh = (N[2] + (d_ == 2), N[1] + (d_ == 1), N[0] + (d_ == 0))
            f0 = int(L.face_off[b, d_])
            gf = Bg[d_][f0:f0 + sh[0] * sh[1] * sh[2]].cpu().numpy().reshape(sh)
            fs = (slice(g, g + n[2] + (d_ == 2)), slice(g, g + n[1] + (d_ == 1)), slice(g, g + n[0] + (d_ == 0)))
            rf, gf = Bo[d_][fs], gf[fs]
            e[name] = float(np.max(np.abs(gf - rf)) / max(float(np.max(np.abs(rf))), 1e-300))
        e["status_mismatch"] = int(np.sum((gs[sl] & 0x3F) != st[sl]))
        for k, v in e.items():
            acc[k] = max(acc.get(k, 0), v)
    acc["blocks"] = sample
    acc["measures"] = MEASURES + " (B^d: of the block's max |B|)"
    acc["oracle"] = "FP64 oracle stage, atmosphere band 1e-6, tol 1e-10, same seeded inputs"
    return acc


def run_reference(a):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from paper_2311_04989_gb300 import inputs as I
    mesh = I.BinaryStarMesh(nb=a.nb, n=16)
    nthreads = os.cpu_count() or 1
    per_step = max(1.0, 60.0 / max(1, a.steps + a.warmup))
    vals = []
    for s in range(a.warmup + a.steps):
        v, cells, wall, nblk = oracle_sample(mesh, per_step, nthreads)
        if s >= a.warmup:
            vals.append((v, cells, wall, nblk))
    value = statistics.median([v[0] for v in vals])
    ms = statistics.median([v[2] / v[1] * (16 ** 3 * a.nb ** 3) * 1e3 for v in vals])
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD + " (bounded random sample of blocks per step)",
                      "blocks": a.nb ** 3, "parallelism": "replicas"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                            "sample": f"{vals[-1][3]} random blocks of 16^3 per step (~{per_step:.0f} s of "
                                      f"work), oracle FP64 C++ stage, {nthreads} threads"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
# the sources the stage kernels are compiled from (a change to any of them invalidates the
# committed DRAM traffic; the driver, matter-source and level-boundary kernels do not enter)
STAGE_SOURCES = ("eos.cuh", "faces_core.cuh", "faces_f32.cu", "faces_f64.cu", "faces_impl.cuh", "internal.h", "mlp.cuh",
                 "physics.cuh", "stage_common.cuh", "stage_kernels.cu", "update_common.cuh")


def strip_comments(src):
    """C/C++ source with its comments removed and each line's trailing blanks dropped (string and
    character literals kept whole), so that an edit of the comments alone keeps the hash below."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    lines = (l.rstrip() for l in "".join(out).split("\n"))
    return "\n".join(l for l in lines if l)


def kernel_source_hash():
    """Hash of the stage kernels' code (comments and blank lines excluded)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2311_04989_gb300", "csrc")
    for f in STAGE_SOURCES:
        h.update(strip_comments(open(os.path.join(d, f), encoding="utf-8").read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def load_traffic(kernel, precision):
    """DRAM bytes per launch of a kernel from the committed ncu summary, only if it was taken on
    the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(f"{kernel}:{precision}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("bytes_per_launch")


MEASURES = ("D, rho, p: max |x - x_ref| / |x_ref|; S_j, tau: relative to max(|x_ref|, D + |tau|) (the cell's "
            "energy scale); u~^i: absolute (units of c); B^d: max |B - B_ref| / max |B_ref| over the faces of "
            "interior cells; over interior cells; status_mismatch: cells whose physics status bits differ")


def interior_mask(L, geoms, dev):
    """Boolean mask of the interior cells in the cell pools."""
    import torch
    m = torch.zeros(L.ncell, dtype=torch.bool, device=dev)
    cache = {}
    for b, gm in enumerate(geoms):
        key = (tuple(gm.n), gm.ng)
        if key not in cache:
            g, n = gm.ng, gm.n
            t = torch.zeros((n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g), dtype=torch.bool, device=dev)
            t[g:g + n[2], g:g + n[1], g:g + n[0]] = True
            cache[key] = t.view(-1)
        t = cache[key]
        o = int(L.cell_off[b])
        m[o:o + t.numel()] = t
    return m


def per_variable_errors(torch, got, ref, interior):
    """Per-variable error of one stage output against another over the whole mesh (device tensors:
    (W, B faces, U, status) each), in the measures of MEASURES."""
    Wg, Bg, Ug, sg = got
    Wr, Br, Ur, sr = ref
    out = {}
    Ui = Ur[:, interior]
    scale = Ui[0].abs() + Ui[4].abs()
    for v, name in enumerate(("D", "S_x", "S_y", "S_z", "tau")):
        den = Ui[v].abs().clamp_min(1e-300) if v == 0 else torch.maximum(Ui[v].abs(), scale)
        out[name] = float(((Ug[v, interior] - Ui[v]).abs() / den).max().item())
    for v, name in enumerate(("rho", "u_x", "u_y", "u_z", "p")):
        d = (Wg[v, interior] - Wr[v, interior]).abs()
        out[name] = float((d if v in (1, 2, 3) else d / Wr[v, interior].abs().clamp_min(1e-300)).max().item())
    for d_, name in enumerate(("B_x", "B_y", "B_z")):
        out[name] = float(((Bg[d_] - Br[d_]).abs().max() / Br[d_].abs().max().clamp_min(1e-300)).item())
    out["status_mismatch"] = int(((sg[interior].to(torch.int32) & 0x3F) != (sr[interior].to(torch.int32) & 0x3F))
                                 .sum().item())
    return out


def config_inputs(I, only=None, c3_blocks=1024):
    """The smaller benchmark configurations as seeded inputs: (name, blocks, oracle-style parameters);
    only = "C1" / "C2" / "C3" builds that one alone (c3_blocks: the AMR-like batch's block count)."""
    out = []
    tov = I.solve_tov() if only in (None, "C2") else None
    if only in (None, "C1"):
        out.append(("C1 shock tube, 1 block of 16^3, PLM, Gamma 5/3", [I.shock_tube_block(n=(16, 16, 16), g=3)],
                    dict(gamma=5.0 / 3.0, recon=0, rho_atm=1e-10)))
    if only in (None, "C2"):
        out.append(("C2 magnetised 64^3 star (A0), WENOZ",
                    [I.star_block(n=(64, 64, 64), g=3, half_width=10.02, tov=tov, A_b=0.05)],
                    dict(gamma=2.0, recon=1, rho_atm=1e-13 * tov.rho[0])))
    if only in (None, "C3"):
        out.append((f"C3 AMR-like batch, {c3_blocks} blocks of 16^3/24^3/32^3, WENOZ",
                    I.amr_like_batch(nblocks=c3_blocks, workers=os.cpu_count() or 4),
                    dict(gamma=5.0 / 3.0, recon=1, rho_atm=1e-14)))
    return out


def config_timings(a, ctx, dev, G, configs):
    """Stage throughput of the smaller configurations on the GPU, FP64 and mixed (or the one --precision
    names), autotuned launch shapes unless --no-autotune, a step = one gr_stage over all blocks of the
    configuration, inputs resident (C1 and C2 fit in L2, so theirs are L2-warm figures; C3's inputs,
    several GB, do not); the mixed stage in its steady state, as for the headline (FP32 copies of W, B and
    the metric in, of W' and B' out)."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for name, blocks, cp in configs:
        L, W, B, M = G.pack_blocks(blocks, dev)
        mesh = G.gr_mesh_create(ctx, L.descriptors())
        metric = G.metric_struct(M)
        U = torch.zeros_like(W)
        cells = L.interior_cells()
        dt = 0.25 * min(min(b.dx) for b in blocks)
        row = {"cells": cells, "blocks": len(blocks)}
        for prec in ("fp64", "mixed"):
            if a.precision not in ("both", prec):
                continue
            mixed = prec == "mixed"
            p = G.gr_params_default(recon=cp["recon"], gamma_ad=cp["gamma"], rho_atm=cp["rho_atm"],
                                    p_atm=100.0 * cp["rho_atm"] ** cp["gamma"], tol=1e-10,
                                    precision=G.GR_PREC_MIXED if mixed else G.GR_PREC_FP64,
                                    c2p_guess=MIXED_GUESS if mixed else G.GR_GUESS_NONE,
                                    atm_band=G.GR_MIXED_ATM_BAND if mixed else 1e-12)
            G.gr_prim2con(mesh, metric, list(W), B, list(U), p, stream)
            Uo, Wo, Bo = torch.zeros_like(U), torch.zeros_like(W), [torch.zeros_like(x) for x in B]
            st = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
            state = G.state_struct(U, U, B, B, W, Uo, Bo, Wo, st)
            mt = metric
            if mixed:   # the steady state, as for the headline: FP32 copies of the inputs in, of W' and B' out
                def f32(x):
                    y = torch.empty(x.shape, dtype=torch.float32, device=dev)
                    G.gr_cast_f32(x.contiguous(), y, stream)
                    return y
                M32 = f32(M)
                mt = G.metric_struct(M, metric32=M32)
                W32, B32 = f32(W), [f32(x) for x in B]
                G.set_fp32_copies(state, W32=W32, B32=B32, Wo32=torch.empty_like(W32),
                                  Bo32=[torch.empty_like(x) for x in B32])
            metric_run = mt
            if not a.no_autotune:
                G.gr_autotune(mesh, metric_run, state, dt, p, 1, stream)
            for _ in range(a.warmup):
                G.gr_stage(mesh, metric_run, state, dt, p, stream)
            steps = max(a.steps, 10)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            G.gr_profile_begin(mesh, steps)
            e0.record(stream)
            for _ in range(steps):
                G.gr_stage(mesh, metric_run, state, dt, p, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            kms, nst = G.gr_profile_end(mesh)
            ms = e0.elapsed_time(e1) / steps
            stv = st.to(torch.int32)
            row[prec] = {"ms_per_stage": ms, "cell_updates_per_s": cells / (ms / 1e3),
                         "atmosphere_fraction": float(((stv & 1) != 0).sum().item()) / cells,
                         "kernel_ms": dict(zip(G.KERNEL_NAMES, [k / max(1, nst) for k in kms])),
                         "path": G.PATH_NAMES[G.gr_mesh_get_path(mesh)] if mixed else "separate kernels"}
            if mixed:
                row[prec]["c2p_guess"] = GUESS_NAMES[G.gr_mesh_get_guess(mesh, G.GR_PREC_MIXED, 0)] \
                    if a.guess == "auto" else a.guess
                row[prec]["guess_rejected"] = int(((stv & 64) != 0).sum().item())
            del Uo, Wo, Bo, st, state
        if "fp64" in row and "mixed" in row:
            row["ratio_mixed_over_fp64"] = row["fp64"]["ms_per_stage"] / row["mixed"]["ms_per_stage"]
        G.gr_mesh_destroy(mesh)
        out[name] = row
        del L, W, B, M, U
        torch.cuda.empty_cache()
    return out


def config_oracle_timings(configs, seconds):
    """The FP64 oracle's stage on each smaller configuration, on 1 core and on all host cores (a bounded
    sample of blocks for the batch), in cell-updates/s."""
    import concurrent.futures as cf

    import numpy as np

    import oracle as O
    out = {}
    nthreads = os.cpu_count() or 1
    for name, blocks, cp in configs:
        P = O.Params(gamma_ad=cp["gamma"], recon=cp["recon"], rho_atm=cp["rho_atm"], tol=1e-10)
        dt = 0.25 * min(min(b.dx) for b in blocks)
        rng = np.random.default_rng(7)
        order = rng.permutation(len(blocks))

        def prep(b):
            bi = blocks[int(b)]
            blk = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
            g = bi.ng
            val, _ = O.interp_cells(blk, 2, (-g,) * 3, tuple(v + g for v in bi.n))
            Bx, By, Bz = bi.B
            Bc = np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]), 0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                           0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], -1).reshape(-1, 3)
            q = O.prim2con(val, np.moveaxis(bi.W, 0, -1).reshape(-1, 5), Bc, P)
            return blk, np.ascontiguousarray(np.moveaxis(q.reshape(bi.W.shape[1:] + (5,)), -1, 0))

        def one(item):
            blk, U = item
            O.stage_block(blk, U, U, blk.B, dt, P)
            return blk.n[0] * blk.n[1] * blk.n[2]

        row = {}
        probe = prep(order[0])
        t0 = time.perf_counter()
        one(probe)
        per_block = max(time.perf_counter() - t0, 1e-4)
        prepared = [probe]
        for threads in (1, nthreads):
            # blocks for ~`seconds` of work; a configuration with fewer blocks repeats its blocks
            ncall = int(min(10000, max(threads, seconds * threads / per_block)))
            while len(prepared) < min(ncall, len(order)):
                prepared.append(prep(order[len(prepared)]))
            items = [prepared[i % len(prepared)] for i in range(ncall)]
            t1 = time.perf_counter()
            with cf.ThreadPoolExecutor(threads) as ex:
                cells = sum(ex.map(one, items))
            t_used = time.perf_counter() - t1
            row[f"{threads}_cores" if threads > 1 else "1_core"] = {"cell_updates_per_s": cells / t_used, "cells": cells,
                                                                  "block_stages": len(items), "s": round(t_used, 2)}
        out[name] = row
    return out


def con2prim_table_workload(a, ctx, dev, G, I):
    """Con2prim-heavy workload with the tabulated EOS: 256 blocks of 32^3 (one ghost), synthetic
    200 x 128 x 64 table, densities from rho_atm to 1e-3, Lorentz factors up to ~5, |B|^2/p from 1e-3
    to 1e5 (about 30 % of the cells near the atmosphere or with |B|^2/rho >= 1).  gr_con2prim is timed with no bracket proposal, the FP32 pre-solve and the learned bracket
    (trained on the solves of 64 blocks of other seeds)."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    from paper_2311_04989_gb300 import learned_bracket as LB
    eos = I.SyntheticEOS()
    tab = eos.table()
    h = G.gr_eos_create(ctx, tab)
    rho_atm, T_atm = 1e-12, 1e-5
    kw = dict(rho_range=(rho_atm, 1e-3), T_range=(1e-4, 5e-2), ye_range=(0.05, 0.5), u_max=3.0,
              sigma_range=(1e-3, 1e5), metric_amp=0.02)
    t_gen = time.time()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        blocks = list(ex.map(lambda k: I.random_block(n=(32, 32, 32), g=1, seed=600 + k, eos=eos, **kw), range(256)))
        train = list(ex.map(lambda k: I.random_block(n=(16, 16, 16), g=1, seed=900 + k, eos=eos, **kw), range(64)))
    t_gen = time.time() - t_gen
    rho = np.concatenate([b.W[0, 1:-1, 1:-1, 1:-1].ravel() for b in blocks])
    sig = np.concatenate([(((b.B[0][1:-1, 1:-1, 1:-2] + b.B[0][1:-1, 1:-1, 2:-1]) ** 2 +
                            (b.B[1][1:-1, 1:-2, 1:-1] + b.B[1][1:-1, 2:-1, 1:-1]) ** 2 +
                            (b.B[2][1:-2, 1:-1, 1:-1] + b.B[2][2:-1, 1:-1, 1:-1]) ** 2) / 4 /
                           b.W[0, 1:-1, 1:-1, 1:-1]).ravel() for b in blocks])
    hard = float(np.mean((rho < 10 * rho_atm) | (sig >= 1.0)))
    p = G.gr_params_default(eos=G.GR_EOS_TABLE, table=int(h), rho_atm=rho_atm, T_atm=T_atm, Ye_atm=0.5, tol=1e-10)
    Pm, losses, delta = None, [0.0], 0.0
    t_train = time.time()
    x, t = LB.collect(ctx, train, p, device=dev)
    Pm, losses, delta = LB.train(x, t, epochs=400, batch=2048, lr=3e-3)
    t_train = time.time() - t_train
    L, W, B, M = G.pack_blocks(blocks, dev)
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    metric = G.metric_struct(M)
    stream = torch.cuda.current_stream()
    U = torch.zeros((6, W.shape[1]), dtype=torch.float64, device=dev)
    G.gr_prim2con(mesh, metric, list(W), B, list(U), p, stream)
    inter = torch.zeros(L.ncell, dtype=torch.bool, device=dev)
    m = torch.zeros((34, 34, 34), dtype=torch.bool, device=dev)
    m[1:-1, 1:-1, 1:-1] = True
    for b in range(len(blocks)):
        inter[int(L.cell_off[b]):int(L.cell_off[b]) + m.numel()] = m.view(-1)
    cells = L.interior_cells()
    out = {"workload": "256 blocks of 32^3, tabulated EOS 200x128x64 (synthetic), |B|^2/p 1e-3..1e5, u~ <= 3",
           "cells": cells, "hard_cell_fraction": hard, "input_gen_s": round(t_gen, 1),
           "mlp_training": {"training_samples": int(x.shape[0]), "train_s": round(t_train, 2), "first_step": delta,
                            "loss_first_last": [losses[0], losses[-1]]}}
    for name, guess in (("none", G.GR_GUESS_NONE), ("fp32", G.GR_GUESS_FP32), ("mlp", G.GR_GUESS_MLP)):
        p.c2p_guess = guess
        p.mlp = int(Pm.data_ptr())
        Uc = U.clone()
        Wc = torch.zeros((7, W.shape[1]), dtype=torch.float64, device=dev)
        st = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
        ev = torch.zeros(L.ncell, dtype=torch.int32, device=dev)
        for _ in range(a.warmup):
            Uc.copy_(U)
            G.gr_con2prim(mesh, metric, list(Uc), B, list(Wc), st, p, stream, evals=ev)
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(a.steps):
            Uc.copy_(U)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.gr_con2prim(mesh, metric, list(Uc), B, list(Wc), st, p, stream, evals=ev)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        solved = ((st.to(torch.int32) & 0x3F) == 0) & inter
        ms = tot / a.steps
        out[name] = {"ms": ms, "cells_per_s": cells / (ms / 1e3),
                     "fp64_evals_per_solved_cell": float(ev[solved].double().mean().item()),
                     "solved_cells": int(solved.sum().item()),
                     "rejected": int(((st.to(torch.int32) & 64) != 0).sum().item())}
    G.gr_mesh_destroy(mesh)
    G.gr_eos_destroy(h)
    return out


def main():
    global MIXED_GUESS
    a = parse()
    MIXED_GUESS = {"none": 0, "fp32": 1, "auto": 3}[a.guess]   # GR_GUESS_NONE, GR_GUESS_FP32, GR_GUESS_AUTO
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch

    from paper_2311_04989_gb300 import build as Bld
    from paper_2311_04989_gb300 import grstage as G
    from paper_2311_04989_gb300 import inputs as I

    rank, world, lrank = env_rank()
    torch.cuda.set_device(lrank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    if rank == 0 or world == 1:
        Bld.build()
    if dist:
        dist.barrier()

    def barrier():
        if dist:
            dist.barrier()

    if a.only_config:
        ctx = G.gr_context_create(lrank)
        cfg = config_inputs(I, a.only_config, a.config_blocks)
        res = config_timings(a, ctx, torch.device("cuda", lrank), G, cfg)
        G.gr_context_destroy(ctx)
        if rank == 0:
            print(json.dumps({"configs": res}))
        return

    # ---- workload ------------------------------------------------------------------------------
    t_gen = time.time()
    mesh_in = I.BinaryStarMesh(nb=a.nb, n=16)
    geoms = mesh_in.blocks()
    L = G.Layout.of(geoms)
    Wh, Bh, Mh = mesh_in.pack(L)
    dev = torch.device("cuda", lrank)
    W = torch.from_numpy(Wh).to(dev)
    B = [torch.from_numpy(x).to(dev) for x in Bh]
    M = torch.from_numpy(Mh).to(dev)
    del Wh, Bh, Mh
    t_gen = time.time() - t_gen
    Mfull = [M[c] for c in range(10)] + [M[0]] * 6          # K_ij unread (k_zero)
    metric = G.gr_metric()
    for c in range(16):
        metric.v[c] = int(Mfull[c].data_ptr())
    metric.order, metric.k_zero = 2, 1
    ctx = G.gr_context_create(lrank)
    mesh = G.gr_mesh_create(ctx, L.descriptors())
    ws_bytes = G.gr_mesh_workspace_bytes(mesh)
    stream = torch.cuda.current_stream()
    U = torch.zeros_like(W)
    P64 = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=G.GR_PREC_FP64, gamma_ad=2.0,
                              rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10)
    G.gr_prim2con(mesh, metric, list(W), B, list(U), P64, stream)
    Uo = torch.zeros_like(U); Wo = torch.zeros_like(W); Bo = [torch.zeros_like(x) for x in B]
    st = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
    state = G.state_struct(U, U, B, B, W, Uo, Bo, Wo, st)
    dt = 0.25 * mesh_in.dx
    cells = L.interior_cells()

    # The mixed path's steady state: a stage reads FP32 copies of W and B that the previous stage wrote
    # (Wo32 / Bo32) and writes the copies of its own outputs for the next one; the metric of this workload
    # is static, so its FP32 copy is made once.  Here the input copies are made once with gr_cast_f32 (the
    # conversion a previous stage's output writes give); every timed stage writes its output copies.
    def f32(x):
        y = torch.empty(x.shape, dtype=torch.float32, device=dev)
        G.gr_cast_f32(x.contiguous(), y, stream)
        return y

    W32, B32 = f32(W), [f32(x) for x in B]
    M32 = f32(M)
    M32full = [M32[c] for c in range(10)] + [M32[0]] * 6
    metric32 = G.gr_metric()
    for c in range(16):
        metric32.v[c] = metric.v[c]
        metric32.v32[c] = int(M32full[c].data_ptr())
    metric32.order, metric32.k_zero = 2, 1
    Wo32, Bo32 = torch.empty_like(W32), [torch.empty_like(x) for x in B32]
    state32 = G.state_struct(U, U, B, B, W, Uo, Bo, Wo, st)
    G.set_fp32_copies(state32, W32=W32, B32=B32, Wo32=Wo32, Bo32=Bo32)

    def timed(precision, copies=False):
        mt, stt = (metric32, state32) if copies else (metric, state)
        guess = MIXED_GUESS if precision == G.GR_PREC_MIXED else G.GR_GUESS_NONE
        p = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=precision, gamma_ad=2.0, c2p_guess=guess,
                                rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10,
                                atm_band=G.GR_MIXED_ATM_BAND if precision == G.GR_PREC_MIXED else 1e-12)
        # launch shapes per kernel from the library's autotuner (untimed; it runs the stage itself)
        shapes = None
        if not a.no_autotune:
            shapes, _ = G.gr_autotune(mesh, mt, stt, dt, p, 1 if precision == G.GR_PREC_FP64 else 3, stream)
        if a.path != "auto" and precision == G.GR_PREC_MIXED:
            G.gr_mesh_set_path(mesh, {"separate": G.GR_PATH_SEPARATE, "fused": G.GR_PATH_FUSED,
                                      "tiled": G.GR_PATH_TILED_FACES}[a.path])
        for _ in range(a.warmup):
            G.gr_stage(mesh, mt, stt, dt, p, stream)
        torch.cuda.synchronize()
        barrier()
        clk = ClockSampler(lrank)
        clk.start()
        G.gr_profile_begin(mesh, a.steps)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        for _ in range(a.steps):
            G.gr_stage(mesh, mt, stt, dt, p, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        kms, nst = G.gr_profile_end(mesh)
        return max_over_ranks(ms, dist, dev) / a.steps, [k / max(1, nst) for k in kms], clocks, shapes

    # measured arithmetic peaks of this GPU (the ALU rooflines divide by them)
    peaks = measure_alu_peaks(G, torch, dev)
    results = {}
    precs = {"both": ["fp64", "mixed_convert", "mixed"], "fp64": ["fp64"],
             "mixed": ["mixed_convert", "mixed"]}[a.precision]
    snap = {}
    for name in precs:
        prec = G.GR_PREC_FP64 if name == "fp64" else G.GR_PREC_MIXED
        ms, kms, clocks, shapes = timed(prec, copies=name == "mixed")
        results[name] = dict(ms=ms, kernel_ms=kms, clocks=clocks,
                             shapes=dict(zip(G.KERNEL_NAMES[1:], shapes)) if shapes else None)
        if prec == G.GR_PREC_MIXED:   # the bracket proposal the stage ran with (auto: the autotuner's choice)
            results[name]["c2p_guess"] = GUESS_NAMES[G.gr_mesh_get_guess(mesh, prec, 0)] if a.guess == "auto" \
                else a.guess
        snap[name] = (Wo.clone(), [x.clone() for x in Bo], Uo.clone(), st.clone())
        stv = st.to(torch.int32)
        results[name]["status"] = {"atmosphere": int(((stv & 1) != 0).sum().item()),
                                   "failed": int(((stv & 2) != 0).sum().item()),
                                   "guess_rejected": int(((stv & 64) != 0).sum().item())}
    # error of the mixed path against the FP64 path (which matches the oracle to 1e-12)
    err = None
    interior = interior_mask(L, geoms, dev)
    if "fp64" in snap and "mixed" in snap:
        err = per_variable_errors(torch, snap["mixed"], snap["fp64"], interior)
        d = G.gr_diag(mesh, list(snap["mixed"][2]), snap["mixed"][1], stream)
        err["divB_rel_max"] = d[1]
        err["divB_integrated"] = d[2]
        err["measures"] = MEASURES
    head = "mixed" if "mixed" in results else "fp64"
    ms_head = results[head]["ms"]
    value = job_value(cells, world, ms_head)

    # ---- the mixed stage through each path: separate kernels and the fused sweep ------------------
    paths = None
    if "mixed" in results:
        chosen = G.gr_mesh_get_path(mesh)
        pm = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=G.GR_PREC_MIXED, c2p_guess=MIXED_GUESS,
                                 gamma_ad=2.0, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10,
                                 atm_band=G.GR_MIXED_ATM_BAND)
        paths = {"autotuner_chose": G.PATH_NAMES[chosen]}
        for name_, f in (("separate_kernels", G.GR_PATH_SEPARATE), ("fused_sweep", G.GR_PATH_FUSED),
                         ("tiled_face_sweep", G.GR_PATH_TILED_FACES)):
            try:
                G.gr_mesh_set_path(mesh, f)
                for _ in range(a.warmup):
                    G.gr_stage(mesh, metric32, state32, dt, pm, stream)
                G.gr_profile_begin(mesh, a.steps)
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(a.steps):
                    G.gr_stage(mesh, metric32, state32, dt, pm, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                kms_, nst_ = G.gr_profile_end(mesh)
                paths[name_] = {"ms_per_step": e0.elapsed_time(e1) / a.steps,
                                "kernel_ms": dict(zip(G.KERNEL_NAMES, [k / max(1, nst_) for k in kms_]))}
            except G.GrstageError as ex:
                paths[name_] = {"unavailable": str(ex)}
        G.gr_mesh_set_path(mesh, chosen)

    # ---- end to end through the C ABI with host buffers ---------------------------------------
    e2e = None
    if not a.no_e2e:
        hm = head == "mixed"
        p = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=(G.GR_PREC_MIXED if hm else G.GR_PREC_FP64),
                                c2p_guess=(MIXED_GUESS if hm else G.GR_GUESS_NONE),
                                gamma_ad=2.0, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10,
                                atm_band=G.GR_MIXED_ATM_BAND if hm else 1e-12)
        # the host-buffer entry: pinned host pools in, pinned host pools out; the library copies batches
        # of blocks in, runs their stages and copies them out on three overlapping streams
        hU, hW, hM = U.cpu().pin_memory(), W.cpu().pin_memory(), M.cpu().pin_memory()
        hB = [x.cpu().pin_memory() for x in B]
        hUo, hWo = torch.empty_like(hU).pin_memory(), torch.empty_like(hW).pin_memory()
        hBo = [torch.empty_like(x).pin_memory() for x in hB]
        hst = torch.empty(st.shape, dtype=st.dtype, pin_memory=True)
        hmetric = G.gr_metric()
        for c in range(10):
            hmetric.v[c] = int(hM[c].data_ptr())
        hmetric.order, hmetric.k_zero = 2, 1
        hstate = G.state_struct(hU, hU, hB, hB, hW, hUo, hBo, hWo, hst)
        # bytes that cross the host link per step: W, B and the metric whole (ghosts included), U on
        # interior cells; out: U', W', status on interior cells, B' on the faces of interior cells
        nint = L.interior_cells()
        nctf = sum((gm.n[0] + (d == 0)) * (gm.n[1] + (d == 1)) * (gm.n[2] + (d == 2)) for gm in geoms for d in range(3))
        bin_ = sum(x.numel() * x.element_size() for x in [hW, hM] + hB) + hU.shape[0] * nint * 8
        bout = (hUo.shape[0] + hWo.shape[0]) * nint * 8 + nint + nctf * 8
        nbatch = a.e2e_batches

        def e2e_step():
            G.gr_host_stage(mesh, hmetric, hstate, dt, p, nbatch, stream)

        for _ in range(a.warmup):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e = max_over_ranks(e0.elapsed_time(e1) / a.steps, dist, dev)
        e2e = {"value": job_value(cells, world, ms_e), "unit": UNIT, "h2d_bytes_per_step": bin_,
               "d2h_bytes_per_step": bout, "ms_per_step": ms_e, "api": "gr_host_stage",
               "batches": nbatch}
        del hU, hW, hM, hB, hUo, hWo, hBo, hst

    # ---- the same stage replayed as a CUDA graph ------------------------------------------------
    graph_ms = None
    if head == "mixed":
        pg = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=G.GR_PREC_MIXED, c2p_guess=MIXED_GUESS,
                                 gamma_ad=2.0, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10,
                                 atm_band=G.GR_MIXED_ATM_BAND)
        gph = G.gr_graph_capture(mesh, metric, state, dt, pg)
        for _ in range(a.warmup):
            G.gr_graph_launch(gph, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            G.gr_graph_launch(gph, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1) / a.steps
        G.gr_graph_destroy(gph)

    # ---- a whole RK3 step (ghost exchange + dt + 3 stages) replayed as one CUDA graph -------------
    rk = None
    if head == "mixed" and not a.no_rk:
        pr = G.gr_params_default(recon=G.GR_RECON_WENOZ, precision=G.GR_PREC_MIXED, c2p_guess=MIXED_GUESS,
                                 gamma_ad=2.0, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm, tol=1e-10,
                                 atm_band=G.GR_MIXED_ATM_BAND)
        nbr = I.block_grid_neighbours((a.nb,) * 3, periodic=(False,) * 3)
        drv = G.gr_driver_create(mesh, nbr)
        Ur, Wr, Br = U.clone(), W.clone(), [x.clone() for x in B]
        str_ = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
        gph = G.gr_driver_capture(drv, metric32, list(Ur), list(Wr), Br, str_, pr, 0.25, G.GR_DT_GRID, 3)
        for _ in range(a.warmup):
            G.gr_graph_launch(gph, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            G.gr_graph_launch(gph, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_rk = e0.elapsed_time(e1) / a.steps
        # the ghost exchange alone: algorithmic bytes = every ghost element read once and written once
        e0.record(stream)
        for _ in range(a.steps):
            G.gr_ghost_fill(drv, list(Wr), Br, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_gf = e0.elapsed_time(e1) / a.steps
        gb = 0
        for gm in geoms:
            Nn = [gm.n[d] + 2 * gm.ng for d in range(3)]
            gb += 5 * 16 * (Nn[0] * Nn[1] * Nn[2] - gm.n[0] * gm.n[1] * gm.n[2])
            for d in range(3):
                F_ = [Nn[x] + (x == d) for x in range(3)]
                O_ = [gm.n[x] + (x == d) for x in range(3)]
                gb += 16 * (F_[0] * F_[1] * F_[2] - O_[0] * O_[1] * O_[2])
        stv = str_.to(torch.int32)
        rk = {"ms_per_rk3_step": ms_rk, "stages": 3, "cfl": 0.25, "dt": G.gr_driver_dt(drv),
              "cell_updates_per_s_per_stage": 3 * cells * world / (ms_rk / 1e3),
              "launches_per_step": 1 + 1 + 1 + 3 * 6 + 2 * 1,
              "ghost_fill": {"ms": ms_gf, "bytes": gb, "GB_per_s": gb / (ms_gf / 1e3) / 1e9},
              "failed_cells_after": int(((stv & 2) != 0).sum().item()),
              "note": "graph of ghost fill (1 kernel) + grid dt (1) + the FP32 conversion of W and B (1) + 3 x (6 stage "
                      "kernels) + 2 inter-stage ghost fills (FP64 and FP32 copies together); the later stages read "
                      "the FP32 copies their predecessors wrote; static metric given with its FP32 copy; outflow "
                      "boundaries; the state evolves over warm-up and timed steps"}
        G.gr_graph_destroy(gph)
        G.gr_driver_destroy(drv)
        del Ur, Wr, Br, str_
        torch.cuda.empty_cache()

    # ---- matter sources of the spacetime equations at the vertices ------------------------------
    adm = None
    if not a.no_adm:
        outv = torch.empty((10, L.nvert), dtype=torch.float64, device=dev)
        adm = {}
        for vo, pname in ((2, "fp64"), (4, "fp64"), (2, "mixed"), (4, "mixed")):
            pa = G.gr_params_default(recon=G.GR_RECON_WENOZ, gamma_ad=2.0, rho_atm=mesh_in.rho_atm,
                                     p_atm=mesh_in.p_atm,
                                     precision=G.GR_PREC_FP64 if pname == "fp64" else G.GR_PREC_MIXED)
            G.gr_adm_sources(mesh, metric, list(W), B, pa, vo, list(outv), stream)   # first call makes the lists
            for _ in range(a.warmup):
                G.gr_adm_sources(mesh, metric, list(W), B, pa, vo, list(outv), stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.steps):
                G.gr_adm_sources(mesh, metric, list(W), B, pa, vo, list(outv), stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_a = e0.elapsed_time(e1) / a.steps
            nv = sum((gm.n[0] + 1) * (gm.n[1] + 1) * (gm.n[2] + 1) for gm in geoms)
            adm[f"{pname}_order{vo}"] = {"ms": ms_a, "owned_vertices": nv, "vertices_per_s": nv / (ms_a / 1e3)}
        del outv
        torch.cuda.empty_cache()

    # ---- con2prim with and without a proposed bracket on the stage's output ------------------
    c2p = None
    if not a.no_c2p:
        from paper_2311_04989_gb300 import learned_bracket as LB
        # the stage output is the mixed path's: its atmosphere cells sit at the threshold up to its FP32
        # sqrt(gamma), so con2prim classifies them with the mixed path's band
        p64 = G.gr_params_default(recon=G.GR_RECON_WENOZ, gamma_ad=2.0, rho_atm=mesh_in.rho_atm, p_atm=mesh_in.p_atm,
                                  tol=1e-10, atm_band=G.GR_MIXED_ATM_BAND)
        Uref = snap[head][2]
        Bref = snap[head][1]
        # training samples: the solves of this workload's stage output ("prior solves" of the run)
        feats = [torch.zeros(L.ncell, dtype=torch.float32, device=dev) for _ in range(G.GR_MLP_NIN)]
        tgt = torch.zeros(L.ncell, dtype=torch.float32, device=dev)
        val = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
        G.gr_c2p_samples(mesh, metric, list(Uref), Bref, p64, feats, tgt, val, stream)
        xs, ts = LB.samples_from(feats, tgt, val)
        t_train = time.time()
        Pm, losses, delta = LB.train(xs, ts, epochs=20, batch=1024, lr=2e-3)
        t_train = time.time() - t_train
        c2p = {"training_samples": int(xs.shape[0]), "mlp_train_s": round(t_train, 2), "mlp_first_step": delta,
               "mlp_loss_first_last": [losses[0], losses[-1]]}
        for name, guess in (("none", G.GR_GUESS_NONE), ("fp32", G.GR_GUESS_FP32), ("mlp", G.GR_GUESS_MLP)):
            pc = G.gr_params_default(recon=G.GR_RECON_WENOZ, gamma_ad=2.0, rho_atm=mesh_in.rho_atm,
                                     p_atm=mesh_in.p_atm, tol=1e-10, c2p_guess=guess, atm_band=G.GR_MIXED_ATM_BAND)
            pc.mlp = int(Pm.data_ptr())
            Uc = Uref.clone(); Wc = torch.zeros_like(W)
            stc = torch.zeros(L.ncell, dtype=torch.uint8, device=dev)
            ev = torch.zeros(L.ncell, dtype=torch.int32, device=dev)
            for _ in range(a.warmup):
                Uc.copy_(Uref)
                G.gr_con2prim(mesh, metric, list(Uc), Bref, list(Wc), stc, pc, stream, evals=ev)
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(a.steps):
                Uc.copy_(Uref)
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                G.gr_con2prim(mesh, metric, list(Uc), Bref, list(Wc), stc, pc, stream, evals=ev)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            solved = ((stc.to(torch.int32) & 0x3F) == 0) & interior
            c2p[name] = {"ms": tot / a.steps, "fp64_evals_per_solved_cell": float(ev[solved].double().mean().item()),
                         "solved_cells": int(solved.sum().item()),
                         "rejected": int(((stc.to(torch.int32) & 64) != 0).sum().item())}

    # ---- con2prim-heavy workload with the tabulated EOS ------------------------------------------
    c2p_table = None
    if not a.no_table and not a.no_c2p:
        c2p_table = con2prim_table_workload(a, ctx, dev, G, I)

    # ---- the smaller configurations: shock tube, 64^3 star, AMR-like batch -----------------------
    configs_out = None
    if not a.no_configs and world == 1:
        cfg = config_inputs(I)
        configs_out = {"gpu": config_timings(a, ctx, dev, G, cfg)}
        if not a.no_cpu and rank == 0:
            configs_out["oracle"] = config_oracle_timings(cfg, 5.0)
        del cfg

    # ---- roofline of the dominant kernel ---------------------------------------------------------
    flops = json.load(open(os.path.join(ROOT, "tests", "golden", "flops_binary_star_16cubed.json")))
    ph = flops["phases"]

    def ph_flops(*names):
        return sum(ph[n]["add"] + ph[n]["mul"] + ph[n]["div"] + ph[n]["sqrt"] for n in names)

    scale = (a.nb ** 3) / 4096.0
    # phases of the oracle's count -> the kernel that runs them, and the pipe they run on
    # FP64 path: every phase in FP64; the atmosphere resets are decided and done in k_update
    phases64 = {"k_cellprep": ("cell_metric_and_field", "cell_efield"), "k_faces": ("faces",),
                "k_edges": ("corner_emf",), "k_ct": ("ct",), "k_update": ("update_and_sources", "con2prim_atmosphere"),
                "k_c2p": ("con2prim",)}

    def kernel_ops(kn, mixed, solved_frac):
        """(FP32 ops, FP64 ops) of one launch of kernel kn on this workload (oracle-counted).  Mixed
        path: the cell prep, faces and corner EMFs run in FP32; CT, con2prim and the atmosphere resets
        in FP64; the flux divergence and sources of the solved (matter) cells run in k_c2p (sources in
        FP32, accumulation in FP64: counted as FP32), those of the atmosphere cells are skipped (their
        reset overrides them)."""
        if not mixed:
            return 0.0, sum(ph_flops(p_) for p_ in phases64.get(kn, ())) * scale
        if kn in ("k_cellprep", "k_faces", "k_edges"):
            return sum(ph_flops(p_) for p_ in phases64[kn]) * scale, 0.0
        if kn == "k_ct":
            return 0.0, ph_flops("ct") * scale
        if kn == "k_update":
            return 0.0, ph_flops("con2prim_atmosphere") * scale
        if kn == "k_c2p":
            return ph_flops("update_and_sources") * solved_frac * scale, ph_flops("con2prim") * scale
        return 0.0, 0.0

    def kernel_rooflines(name, peaks):
        """ALU roofline of every stage kernel against the measured FP32 and FP64 peaks: the time lower
        bound is FP32 ops / FP32 peak + FP64 ops / FP64 peak, and peak is the matching effective rate."""
        kms = results[name]["kernel_ms"]
        mixed = name == "mixed"
        stc = results[name]["status"]
        solved_frac = max(0.0, 1.0 - (stc["atmosphere"] + stc["failed"]) / cells)
        rows = {}
        for i, kn in enumerate(G.KERNEL_NAMES):
            # the cell prep (plane sums carried along z) and the atmosphere resets do fewer operations than
            # the oracle's plain per-cell form, so the oracle's count is no measure of their work
            if kn in ("k_cellprep", "k_update"):
                continue
            f32, f64 = kernel_ops(kn, mixed, solved_frac)
            if f32 + f64 <= 0 or kms[i] <= 0:
                continue
            t_lb = f32 / (peaks["fp32_tflops"] * 1e12) + f64 / (peaks["fp64_tflops"] * 1e12)
            fl = f32 + f64
            rows[kn] = {"ms": kms[i], "fp32_flops": f32, "fp64_flops": f64, "achieved_tflops": fl / (kms[i] / 1e3) / 1e12,
                        "peak_tflops": fl / t_lb / 1e12, "frac": t_lb / (kms[i] / 1e3)}
        return rows

    def roofline(name, peaks):
        """The dominant kernel's ALU roofline (of measured peaks)."""
        rows = kernel_rooflines(name, peaks)
        kms = results[name]["kernel_ms"]
        kn = max(rows, key=lambda k: rows[k]["ms"])
        r = rows[kn]
        return {"bound": "alu", "achieved": r["achieved_tflops"], "peak": r["peak_tflops"], "unit": "TFLOP/s",
                "frac": r["frac"], "traffic": load_traffic(kn, name), "kernel": kn,
                "peak_source": "measured",
                "peak_kind": (f"measured FP32 {peaks['fp32_tflops']:.2f} TFLOP/s and FP64 {peaks['fp64_tflops']:.3f} "
                              "TFLOP/s (gr_peak_alu loops on this GPU), combined as the time lower bound of the "
                              "kernel's oracle-counted FP32 and FP64 operations"),
                "flops_per_launch": r["fp32_flops"] + r["fp64_flops"], "fp32_flops": r["fp32_flops"],
                "fp64_flops": r["fp64_flops"], "kernel_ms": r["ms"], "kernel_share": r["ms"] / sum(kms)}

    def stage_hbm(name):
        """The whole stage against the measured copy bandwidth, with the compulsory bytes of this
        workload: U (5), B (3), W (5) read and U', B', W' (13 words) and the status byte written per
        interior cell, plus the 10 metric words per vertex (K_ij declared zero and unread; one vertex per
        cell, the mesh's unique vertices); the first RK stage form (g0 = 0) reads no U0 / B0."""
        nvert = (a.nb * 16 + 1) ** 3
        bytes_ = cells * (13 * 8 + 13 * 8 + 1) + nvert * 10 * 8
        ms = results[name]["ms"]
        ach = bytes_ / (ms / 1e3) / 1e9
        pk = MEASURED_HBM_GBS
        return {"compulsory_bytes": bytes_, "bytes_per_cell": bytes_ / cells, "achieved_GBps": ach, "peak_GBps": pk,
                "frac": ach / pk, "peak_source": f"{HBM_PEAK_SOURCE} copy bandwidth (hbm_gbs)"}

    # ---- CPU baseline (rank 0, N = 1) ------------------------------------------------------------
    cpu = None
    mixed_vs_oracle = None
    if not a.no_cpu and world == 1 and rank == 0:
        nthreads = os.cpu_count() or 1
        v, ncell, wall, nblk = oracle_sample(mesh_in, a.cpu_seconds, nthreads)
        cpu = {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"{nblk} seeded-random blocks of the same workload, FP64 oracle stage, "
                         f"{nthreads} threads, {wall:.1f} s"}
        # the same oracle on one core (single-thread rate of the reference program)
        v1, _, wall1, nblk1 = oracle_sample(mesh_in, min(a.cpu_seconds, 10.0), 1)
        cpu["one_core"] = {"value": v1, "cores": 1, "sample": f"{nblk1} blocks, {wall1:.1f} s"}
        if "mixed" in snap:
            mixed_vs_oracle = oracle_errors(torch, mesh_in, L, snap["mixed"], dt)

    # cell prep, faces, edges, CT, update, con2prim (+ the FP32 cast on the mixed path) per stage
    # cell prep, faces, edges, CT, update, con2prim per stage (the steady-state mixed stage converts nothing)
    launches = a.steps * 6
    fp64 = None
    if "fp64" in results and head != "fp64":
        fp64 = {"value": cells * world / (results["fp64"]["ms"] / 1e3), "ms_per_step": results["fp64"]["ms"],
                "kernel_ms": dict(zip(G.KERNEL_NAMES, results["fp64"]["kernel_ms"])),
                "roofline": roofline("fp64", peaks), "kernel_rooflines": kernel_rooflines("fp64", peaks),
                "stage_hbm": stage_hbm("fp64"), "clocks": results["fp64"]["clocks"]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": ms_head, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "blocks": a.nb ** 3, "cells_per_gpu": cells, "recon": "WENOZ",
                      "riemann": "HLLE", "precision": head, "parallelism": "replicas" if world > 1 else "single",
                      "l2": "inputs ~25 GB >> L2 (no flush)", "workspace_bytes": ws_bytes,
                      "fp32_copies": ("mixed stage in its steady state: reads FP32 copies of W and B (as the previous "
                                      "stage writes them) and of the static metric (made once), writes FP64 outputs "
                                      "and the FP32 copies of W' and B' for the next stage"),
                      "c2p_guess": (results[head].get("c2p_guess", a.guess) + (" (autotuned)" if a.guess == "auto" else ""))
                                   if head == "mixed" else "none",
                      "atmosphere_fraction": (results[head]["status"]["atmosphere"] / cells),
                      "input_gen_s": round(t_gen, 1)},
           "roofline": roofline(head, peaks), "clocks": results[head]["clocks"], "alu_peaks": peaks,
           "stage_hbm": stage_hbm(head), "kernel_rooflines": kernel_rooflines(head, peaks), "e2e": e2e, "gpu_launches": launches,
           "cpu_baseline": cpu, "kernel_ms": dict(zip(G.KERNEL_NAMES, results[head]["kernel_ms"])),
           "fp64": fp64, "mixed_error_vs_fp64": err,
           "mixed_error_vs_oracle": mixed_vs_oracle, "configs": configs_out, "stage_paths": paths, "status_counts": results[head].get("status"),
           "graph_ms_per_step": graph_ms, "rk3_driver": rk, "adm_sources": adm, "con2prim_guess": c2p, "con2prim_table": c2p_table,
           "launch_shapes": {k: v.get("shapes") for k, v in results.items()},
           "ratio_mixed_over_fp64": (results["fp64"]["ms"] / results["mixed"]["ms"]) if fp64 else None,
           "mixed_with_input_conversion": ({"ms_per_step": results["mixed_convert"]["ms"],
                                            "value": cells * world / (results["mixed_convert"]["ms"] / 1e3),
                                            "kernel_ms": dict(zip(G.KERNEL_NAMES, results["mixed_convert"]["kernel_ms"])),
                                            "note": "the same stage converting W, B and the metric to FP32 itself "
                                                    "(k_cast) instead of reading the FP32 copies"}
                                           if "mixed_convert" in results else None)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    G.gr_mesh_destroy(mesh)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
