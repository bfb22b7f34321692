"""Write the full-size expected barcodes under tests/golden/ using only the CPU
oracle (oracle/). The input points are stored with the barcodes, so a test on
another machine feeds the GPU path exactly these float32 points.

    python tests/golden/make_golden.py [torus2000] [sphere192] [torus300_cohom]

torus2000:      the 2000-point noisy torus (seed 0), full filtration, H0-H1
                (oracle COHOM_CLEAR, about 3 minutes on 8 cores).
sphere192:      192 points on S^3 (seed 0), full filtration, H0-H2
                (oracle COHOM_CLEAR).
torus300_cohom: 300 points of the noisy torus (seed 3), full filtration,
                H0-H1, by the coboundary reduction WITHOUT clearing (oracle
                COHOM: Alg. 1 on every column of the coboundary matrix, no
                Kruskal, no clearing lemma; about 2.5 minutes on 8 cores), so
                that a full-size comparison does not rest only on the two
                shortcuts the GPU path shares with COHOM_CLEAR.
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2003_07989_gb300 import inputs as I  # noqa: E402

CASES = {
    "torus2000": (lambda: I.noisy_torus(2000, seed=0), 1, O.MODE_COHOM_CLEAR),
    "sphere192": (lambda: I.sphere_s3(192, seed=0), 2, O.MODE_COHOM_CLEAR),
    "torus300_cohom": (lambda: I.noisy_torus(300, seed=3), 1, O.MODE_COHOM),
}
MODE_NAMES = {O.MODE_HOM: "HOM", O.MODE_COHOM: "COHOM", O.MODE_COHOM_CLEAR: "COHOM_CLEAR"}


def make(name):
    gen, max_dim, mode = CASES[name]
    X = gen()
    D = O.distance_matrix(X)
    t0 = time.time()
    P = O.barcodes(D, max_dim, math.inf, mode)
    dt = time.time() - t0
    out = {"points": X, "max_dim": np.array(max_dim), "oracle_seconds": np.array(dt),
           "oracle_additions": np.array(P.additions), "oracle_mode": np.array(MODE_NAMES[mode])}
    for q in range(max_dim + 1):
        out[f"H{q}"] = P.barcode(q)
    path = os.path.join(HERE, f"{name}.npz")
    np.savez_compressed(path, **out)
    print(name, "written", path, f"{dt:.1f} s", [len(out[f'H{q}']) for q in range(max_dim + 1)])


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        make(name)
