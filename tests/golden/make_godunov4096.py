"""Write tests/golden/godunov4096_seed1_10steps.txt from the oracle (CPU, ~2-3 min, ~5 GB).

The 4096^2 FP32-bulk workload is too large for the oracle inside a GPU test,
so its FP64 oracle result is stored here at sampled cells: 1024 cells drawn
by a seeded generator plus every 8th cell of rows 1000 and 3000 (lines across
both Sod interfaces).  Also stored: the 10 time steps and the exact (fsum)
totals of the four conserved fields after 10 steps.  Only oracle/ and the
seeded input generator are used.
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1710_08774_gb300 import inputs as I  # noqa: E402

N, STEPS, SEED = 4096, 10, 1
OUT = os.path.join(HERE, "godunov4096_seed1_10steps.txt")


def sample_points():
    rng = np.random.default_rng(2024)
    pts = [(int(j), int(i)) for j, i in zip(rng.integers(0, N, 1024), rng.integers(0, N, 1024))]
    for j in (1000, 3000):
        pts += [(j, i) for i in range(0, N, 8)]
    return pts


def main():
    U = I.sod_state(N, N, seed=SEED)
    W, dts, st = oracle.godunov(U, STEPS)
    assert st.floor_hits == 0 and st.newton_nonconv == 0
    with open(OUT, "w") as f:
        f.write("# oracle FP64 Godunov, 4096x4096 Sod-like seed 1, CFL 0.5, 10 steps (x then y sweep)\n")
        f.write("# written by tests/golden/make_godunov4096.py; rows: j i rho rhou rhov E\n")
        f.write("dt " + " ".join(f"{x:.17e}" for x in dts) + "\n")
        f.write("totals " + " ".join(f"{math.fsum(W[k].ravel().tolist()):.17e}" for k in range(4)) + "\n")
        f.write("absmax " + " ".join(f"{np.max(np.abs(W[k])):.17e}" for k in range(4)) + "\n")
        for j, i in sample_points():
            f.write(f"{j} {i} " + " ".join(f"{W[k, j, i]:.17e}" for k in range(4)) + "\n")


if __name__ == "__main__":
    main()
