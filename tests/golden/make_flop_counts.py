"""Write the algorithmic operation counts of the full-stage throughput workload.

Runs the operation-counting build of the oracle's stage (oracle/flopcount.h) on the two-star
workload (4096 blocks of 16^3, WENOZ + HLLE, FP64) and writes, per phase of the stage, the summed
adds, multiplies, divides and square roots over all blocks, together with the unit counts the GPU
kernels process.  Blocks whose cells and ghosts are all untouched atmosphere (uniform rho_atm,
p_atm, u~ = 0, B = 0) take identical branches, so one of them is counted and multiplied by their
number; every other block is counted individually.  Calls only oracle/ and the input generators.

    python tests/golden/make_flop_counts.py [--nb 16]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2311_04989_gb300 import inputs as I  # noqa: E402


def cons(bi, P):
    """Conserved variables of a block from its prims with the oracle's prim2con (all cells)."""
    n, g = bi.n, bi.ng
    blk = O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B)
    lo, hi = (-g,) * 3, tuple(n[d] + g for d in range(3))
    val, _ = O.interp_cells(blk, 2, lo, hi)
    Bx, By, Bz = bi.B
    Bc = np.stack([0.5 * (Bx[:, :, 1:] + Bx[:, :, :-1]), 0.5 * (By[:, 1:, :] + By[:, :-1, :]),
                   0.5 * (Bz[1:, :, :] + Bz[:-1, :, :])], -1).reshape(-1, 3)
    W = np.moveaxis(bi.W, 0, -1).reshape(-1, 5)
    q = O.prim2con(val, W, Bc, P)
    return np.ascontiguousarray(np.moveaxis(q.reshape(bi.W.shape[1:] + (5,)), -1, 0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nb", type=int, default=16)
    ap.add_argument("--out", default=os.path.join(HERE, "flops_binary_star_16cubed.json"))
    a = ap.parse_args()
    t0 = time.time()
    mesh = I.BinaryStarMesh(nb=a.nb, n=16)
    P = O.Params(gamma_ad=2.0, recon=1, rho_atm=mesh.rho_atm, p_atm=mesh.p_atm, tol=1e-10)
    dt = 0.25 * mesh.dx
    nbk = a.nb ** 3
    total = {ph: np.zeros(4) for ph in O.PHASES}
    atm_counts, n_atm, n_counted = None, 0, 0
    for b in range(nbk):
        bi = mesh.block(b)
        quiet = np.all(bi.W[0] == mesh.rho_atm) and all(np.all(x == 0) for x in bi.B)
        if quiet and atm_counts is not None:
            n_atm += 1
            continue
        U = cons(bi, P)
        c = O.stage_block_count(O.Block(bi.n, bi.ng, bi.dx, bi.metric, bi.W, bi.B), U, U, bi.B, dt, P)
        if quiet:
            atm_counts, n_atm = c, 1
        else:
            n_counted += 1
            for ph in O.PHASES:
                total[ph] += np.array(c[ph])
    for ph in O.PHASES:
        total[ph] += n_atm * np.array(atm_counts[ph])
    n, g = 16, 3
    units = {"cells_interior": nbk * n ** 3, "cells_padded": nbk * (n + 2 * g) ** 3,
             "faces_extended": nbk * 3 * (n + 1) * (n + 2) ** 2, "edges": nbk * 3 * n * (n + 1) ** 2,
             "ct_faces": nbk * 3 * (n + 1) * n * n}
    res = {"workload": f"two TOV stars, {nbk} blocks of 16^3 (ng=3), WENOZ+HLLE, FP64, tol 1e-10",
           "blocks_counted_individually": n_counted, "quiet_atmosphere_blocks": n_atm,
           "phases": {ph: dict(zip(("add", "mul", "div", "sqrt"), map(float, total[ph]))) for ph in O.PHASES},
           "units": units, "seconds": round(time.time() - t0, 1)}
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
