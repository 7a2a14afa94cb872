"""Write the golden fixtures under tests/golden/ (calls only oracle/).

odd_6x9x4.txt -- the shape of the worked example in Sec. III-B of the paper
(4 images of 6 rows x 9 columns).  The paper prints no values for it, so the
input is a seeded synthetic scan stored verbatim, and the expected output is
the FP64 oracle's, which the pins in tests/test_oracle_pins.py tie to brute
force and closed forms.  The file fixes the oracle against regressions and
gives the CUDA path an odd-width case (9 columns: no 16-byte row pitch).

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from tests.gen import synth as S  # noqa: E402


def odd_case():
    sc = S.tiny_scan(seed=5, rows=6, cols=9, K=4,
                     roi_origin=(29, 27), det_rows=64, det_cols=64)
    edges = S.bin_edges(0.0, 20.0, 1.0)
    return sc, edges


def write_odd():
    sc, edges = odd_case()
    out = O.reconstruct(sc.geom, sc.wires, sc.images, edges)
    path = os.path.join(HERE, "odd_6x9x4.txt")
    with open(path, "w") as f:
        f.write("# Shape of the worked example of Sec. III-B (4 images x 6 rows x 9 cols).\n")
        f.write("# Seeded synthetic input (tiny_scan seed 5, ROI at (29, 27) of 64x64),\n")
        f.write("# bins of 1 um with centres 0..20 um; expected output = FP64 oracle.\n")
        f.write(f"K {sc.K} rows 6 cols 9 bins {edges.shape[0] - 1}\n")
        f.write("images\n")
        for v in sc.images.reshape(-1):
            f.write(f"{int(v)}\n")
        f.write("edges\n")
        for v in edges:
            f.write(f"{v:.17g}\n")
        f.write("out\n")
        for v in out.reshape(-1):
            f.write(f"{v:.17g}\n")
    return path


def read_odd():
    path = os.path.join(HERE, "odd_6x9x4.txt")
    lines = [ln.strip() for ln in open(path) if not ln.startswith("#")]
    hdr = lines[0].split()
    K, rows, cols, B = int(hdr[1]), int(hdr[3]), int(hdr[5]), int(hdr[7])
    i = lines.index("images") + 1
    images = np.array([int(x) for x in lines[i:i + K * rows * cols]],
                      dtype=np.uint16).reshape(K, rows, cols)
    i = lines.index("edges") + 1
    edges = np.array([float(x) for x in lines[i:i + B + 1]])
    i = lines.index("out") + 1
    out = np.array([float(x) for x in lines[i:i + B * rows * cols]]).reshape(B, rows, cols)
    return images, edges, out


if __name__ == "__main__":
    print(write_odd())
