"""Writes the stored expected values under tests/golden/ by running the oracle
(and nothing else) on small seeded workloads:

  cuboid_prec32.txt / cuboid_prec64.txt
      The 2x2x10 um cuboid of 1,920 Kuhn tets, A + B <-> C (kf = 1e6 /M/s,
      kb = 10 /s, D = 1e-11 m^2/s), 5,000 A and 5,000 B placed by volume,
      simulation seed 3, run to 10 ms (13 full windows and a shortened one),
      mean-occupancy trial counts. prec32: the kernel-precision mode (float
      propensities); prec64: all FP64.

Usage: python tests/golden/make_golden.py   (from the repository root)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1610_02258_gb300 import inputs as I  # noqa: E402


def cuboid(prec: int):
    w = I.config1()
    o = oracle.from_workload(w, prec=prec)
    o.run(w.t_end)
    return w, o


def write(path, w, o, prec):
    c = o.get_counts()
    with open(path, "w") as f:
        f.write(f"# {w.name}: oracle prec={prec}, seed {w.seed}, t_end {w.t_end!r} s\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write(f"windows {o.windows}\n")
        f.write(f"tau {o.tau!r}\n")
        f.write(f"shape {c.shape[0]} {c.shape[1]}\n")
        f.write("totals " + " ".join(str(int(x)) for x in c.sum(axis=1)) + "\n")
        for row in c:
            f.write(" ".join(str(int(x)) for x in row) + "\n")


def read(path):
    meta, rows = {}, []
    for line in open(path):
        if line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key in ("windows", "tau", "shape", "totals"):
            meta[key] = rest.split()
        else:
            rows.append([int(x) for x in line.split()])
    return {"windows": int(meta["windows"][0]), "tau": float(meta["tau"][0]),
            "totals": [int(x) for x in meta["totals"]], "counts": np.array(rows, np.int32)}


if __name__ == "__main__":
    from oracle.build import build
    build()
    for prec in (32, 64):
        w, o = cuboid(prec)
        write(os.path.join(HERE, f"cuboid_prec{prec}.txt"), w, o, prec)
        print(f"wrote cuboid_prec{prec}.txt: {o.windows} windows")
