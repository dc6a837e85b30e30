"""Writes the stored oracle values of tests/golden/ (calls only oracle/ and
the input generators).  The paper prints no worked example to match (its
accuracy tables are absent from the source), so these fixtures freeze the
oracle's own output: a later change to the oracle's arithmetic must rerun
this script in the same commit and name the passage that justifies it.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402
import workloads as W  # noqa: E402

TARGETS = [0, 1, 77, 130, 255, 256, 400, 511]


def compute():
    """Starfish 1 + 0.25 cos 5t, 32 panels, k = 5, p = 8, sigma = cos 3t +
    0.5 i sin t (the 32-panel parity workload): S, D and grad S, interior
    PV, at TARGETS."""
    wl = W.cfg1()
    g = oracle.geometry(wl.curve, wl.curve.edges(wl.M), 16, 64)
    dens = W.density_cfg1(g["t_tgt"])
    sel = np.array(TARGETS)
    rows = []
    for op, name in ((oracle.OP_S, "S"), (oracle.OP_D, "D"), (oracle.OP_GRAD_S, "GRAD_S")):
        v = oracle.apply(g, op, oracle.SIDE_INT, oracle.LIMIT_PV, wl.k, wl.p, dens, sel=sel)
        v = v.reshape(len(TARGETS), -1)
        for i, t in enumerate(TARGETS):
            for c in range(v.shape[1]):
                rows.append((name, t, c, v[i, c].real, v[i, c].imag))
    return rows


def main():
    path = os.path.join(HERE, "starfish32_k5_p8_int_pv.txt")
    with open(path, "w") as f:
        f.write("# oracle output: starfish 1+0.25cos5t, 32 panels, k=5, p=8, interior PV, sigma=cos3t+0.5i sin t\n")
        f.write("# written by tests/golden/make_golden.py; columns: op target component re im\n")
        for name, t, c, re, im in compute():
            f.write(f"{name} {t} {c} {re:.17e} {im:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
