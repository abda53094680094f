#!/usr/bin/env python3
"""Write the oracle's results for the reduced shapes of the two large
workloads, which the dense oracle takes minutes to hours to compute, so that
the GPU parity tests can compare against them without recomputing.

Only ``oracle/`` (dense LU steps, Appendices A-B) and the seeded input
generators of ``workloads/`` are called here; nothing comes from the CUDA
path.  Each file holds the objective G, the gradient dG/dalpha and the final
states rho_i(T) of one problem, as JSON (floats written with repr, so they
round-trip exactly):

  qudits_4x2_full.json   the four-qudit workload's structure (chain
                         cross-Kerr, 2 carriers x 30 splines, dt = 0.0125 ns)
                         at 2 levels per qudit (vec 256), 3 random pure
                         states, all 40000 steps of its 500 ns horizon;
  qudits_4x3_prefix.json the same at 3 levels per qudit (vec 6561), the first
                         24 steps (controls those of the 500 ns horizon);
  qutrits_6x2_prefix.json the six-qutrit workload's structure (ring
                         cross-Kerr, 2 carriers x 40 splines, dt = 0.015 ns)
                         at 2 levels per subsystem (vec 4096), 4 random pure
                         states, the first 24 steps (controls those of the
                         300 ns horizon).

Usage: python tests/golden/make_oracle_references.py [name ...]
"""

from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import imr  # noqa: E402


def qudits_4x2_full():
    return W.config4(levels=(2, 2, 2, 2), n_states=3, n_steps=40000)


def qudits_4x3_prefix():
    return W.prefix(W.config4(levels=(3, 3, 3, 3), n_states=3, n_steps=40000), 24)


def qutrits_6x2_prefix():
    return W.prefix(W.config5(levels=(2,) * 6, n_states=4, n_steps=20000), 24)


PROBLEMS = {"qudits_4x2_full": qudits_4x2_full, "qudits_4x3_prefix": qudits_4x3_prefix,
            "qutrits_6x2_prefix": qutrits_6x2_prefix}


def write(name: str) -> None:
    p = PROBLEMS[name]()
    t0 = time.perf_counter()
    G, g, fw = imr.gradient(p)
    rhoT = np.asarray(fw["rhoT"])
    out = {
        "problem": name,
        "doc": PROBLEMS[name].__name__,
        "n_steps": int(p.system.n_steps),
        "T_ns": float(p.system.T_ns),
        "G": float(G),
        "grad": [float(x) for x in g],
        "rhoT_re": [float(x) for x in rhoT.real.ravel()],
        "rhoT_im": [float(x) for x in rhoT.imag.ravel()],
        "rhoT_shape": list(rhoT.shape),
        "oracle_seconds": time.perf_counter() - t0,
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f)
    print(name, "G =", repr(float(G)), f"{out['oracle_seconds']:.0f} s", flush=True)


def load(name: str):
    """(G, grad, rhoT) of a stored reference."""
    d = json.load(open(os.path.join(HERE, name + ".json")))
    rho = (np.array(d["rhoT_re"]) + 1j * np.array(d["rhoT_im"])).reshape(d["rhoT_shape"])
    return d["G"], np.array(d["grad"]), rho


if __name__ == "__main__":
    for n in sys.argv[1:] or list(PROBLEMS):
        write(n)
