"""Writes the regression fixtures of tests/golden/ from the FP64 oracle
(oracle/ and the seeded input generator only; no CUDA path).  The paper
prints no worked example, so these values are not the paper's: they freeze
the oracle's outputs on small seeded cases so that a later change to its
arithmetic shows up as a failing test (and must be justified).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import confined as oc  # noqa: E402
from oracle import cv as ocv  # noqa: E402
from paper_2312_02990_gb300 import inputs  # noqa: E402


def bulk_case():
    """N=108 FCC + jitter: forces of 5 atoms, U, virial (Eq. 6, Eq. 7)."""
    N = 108
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    st = inputs.jittered_states(N, 1, seed=4242, amp=0.08)[0]
    F, W, U = oracle.forces(b, st, 0.7)
    return {"cite": "Eq. 6 (WCA, Lees-Edwards offset 0.7), Eq. 7 virial", "N": N, "delta": 0.7,
            "seed": 4242, "F_first5": F[:, :5].tolist(), "W": list(map(float, W)), "U": float(U)}


def daughter_case():
    """Four mapped daughters of one N=108 state, 20 steps at gamma = 0.1:
    Omega(0) and B(s) = P_xy(s) (Eq. 3, 5, 7)."""
    N = 108
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    st = inputs.jittered_states(N, 1, seed=77, amp=0.05)
    B, Om = oracle.daughters(b, st, np.array([0.13]), 0.1, 20)
    return {"cite": "Eq. 3 mappings, Eq. 5 SLLOD/Nose-Hoover, Eq. 7 Omega and P_xy", "N": N,
            "seed": 77, "alpha0": 0.13, "gamma": 0.1, "Omega": Om.tolist(), "B": B.tolist()}


def confined_case():
    """Small channel, 10 steps at gamma = 0.05: wall stresses, slab totals
    and the inner wall layers' p_x sums of the four mapped daughters (Eq. 9,
    10, 11)."""
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=11)
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]), vwall=0.05 * 5.0)
    B, Om = oc.daughters(sy, s["state"][None], s["lattice"], np.zeros(1), 10, 5)
    ns = oc.N_SLAB
    return {"cite": "Eq. 9 potential, Eq. 10 dynamics, Eq. 11 Omega; v = gamma h / 2", "seed": 11,
            "Omega": Om.tolist(), "wall_stress": B[:, :, :2].tolist(),
            "slab_px_total": B[:, :, 2:2 + ns].sum(axis=2).tolist(),
            "slab_n": B[:, :, 2 + ns:2 + 2 * ns].tolist(),
            "wall_layer_px": B[:, :, 2 + 2 * ns:].tolist()}


def cv_case():
    """Forward pass of a seeded network in FP64 with BF16 weights."""
    rng = np.random.default_rng(9)
    p = (rng.standard_normal(ocv.N_PARAMS) * 0.1).astype(np.float32)
    X = rng.standard_normal((4, ocv.N_FEAT)).astype(np.float32)
    y = ocv.forward(ocv.bf16(p), X)[0]
    return {"cite": "control-variate network 32-128-128-1 (not in the paper)", "seed": 9,
            "y": np.asarray(y, np.float64).ravel().tolist()}


def main():
    cases = {"bulk_forces": bulk_case, "bulk_daughters": daughter_case,
             "confined_daughters": confined_case, "cv_forward": cv_case}
    for name, fn in cases.items():
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main()
