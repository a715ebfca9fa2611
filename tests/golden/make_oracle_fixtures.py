"""Writes oracle_regression.json: sampled states of the CPU oracle on two
workloads with piecewise-constant initial data (no transcendental functions,
so the values do not depend on the platform's libm), stored as exact
hexadecimal doubles.  It calls only the oracle and the input generators.

    python tests/golden/make_oracle_fixtures.py

The stored values guard the oracle against unintended change: a deliberate
change of its arithmetic regenerates this file in the same commit, whose
message names the passage of the paper that justifies it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2501_02317_gb300 import workloads as wl  # noqa: E402

CASES = {
    # Sec. 4.2: the Sod shock tube, 512 cells, outflow walls, t = 0.2
    "sod_512_t0.2": dict(make=lambda: wl.sod(512), t_end=0.2, max_steps=1 << 40, stride=16),
    # Sec. 4.4, Eq. 7: the implosion on 48^2 cells, 60 steps
    "implosion_48_60_steps": dict(make=lambda: wl.liska_wendroff(48), t_end=2.5, max_steps=60, stride=37),
}


def compute(name):
    c = CASES[name]
    mesh, W = c["make"]()
    U, t, steps, flags = oracle.run(mesh, oracle.prim_to_cons(mesh, W), 0.0, c["t_end"], c["max_steps"])
    flat = U.reshape(mesh.nvar, -1)
    idx = list(range(0, flat.shape[1], c["stride"]))
    return {
        "steps": int(steps), "t": float(t).hex(), "flags": int(flags),
        "cells": idx,
        "U": [[float(flat[q, i]).hex() for i in idx] for q in range(mesh.nvar)],
        "totals": [float(v).hex() for v in oracle.totals(mesh, U)],
    }


def main():
    out = {"about": "oracle states written by make_oracle_fixtures.py (exact doubles as hex)"}
    for name in CASES:
        out[name] = compute(name)
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
