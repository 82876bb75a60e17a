"""Writes c2_oracle.npz: the FP64 oracle's NNCP-HALS run on the 512 x 512 x 512,
R = 32 workload (rank-32 U[0,1) model + U[0, 0.01) noise, tensor seed 0,
initial factors seed 1), 50 outer iterations through the dimension tree with
root split 1 (Alg. 1 / Alg. 3, HALS update of Sec. II-B, fit of Sec. IV-B).

Stored: the fit of every iteration, and lambda and the column-normalised
factors after iterations 1, 5, 20 and 50 (factors rounded to float32 to keep
the file small; the tests compare them at 1e-3); and, for the initial
factors, rows 0, 1, 255, 300 and 511 of every mode's MTTKRP (Sec. II-A
definition), against which the benchmark states each precision's error.
Only ``oracle`` and the seeded generators are called.

    python tests/golden/make_c2_oracle.py
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1806_07985_gb300 import synth  # noqa: E402

DIMS, R, ITERS, CHECK = (512, 512, 512), 32, 50, (1, 5, 20, 50)
ROWS = (0, 1, 255, 300, 511)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle.npz")


def main():
    x, _ = synth.lowrank_plus_noise(DIMS, R, seed=0)
    H0 = synth.init_factors(DIMS, R, seed=1)
    snaps = {}
    count = {"inner": 0}

    def cb(event, n, H, lam, **_):
        count["inner"] += 1
        if n == len(DIMS) - 1:
            k = count["inner"] // len(DIMS)
            if k in CHECK:
                snaps[k] = ([h.astype(np.float32) for h in H], np.array(lam, dtype=np.float64))

    ref = oracle.nncp_hals(x.astype(np.float64), DIMS, [h.astype(np.float64) for h in H0],
                           max_iters=ITERS, use_dimtree=True, s=1, callback=cb)
    arrays = {"fits": np.array(ref["fits"], dtype=np.float64), "check": np.array(CHECK),
              "rows": np.array(ROWS)}
    xd = x.astype(np.float64)
    H0d = [h.astype(np.float64) for h in H0]
    for n in range(len(DIMS)):
        arrays[f"M{n}_rows"] = oracle.mttkrp_rows(xd, DIMS, H0d, n, ROWS)
    for k in CHECK:
        Hk, lamk = snaps[k]
        arrays[f"lam_{k}"] = lamk
        for n, h in enumerate(Hk):
            arrays[f"H{n}_{k}"] = h
    np.savez_compressed(OUT, **arrays)
    print("wrote", OUT, "final fit", ref["fits"][-1])


if __name__ == "__main__":
    main()
