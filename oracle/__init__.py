"""Plain FP64 CPU oracle of the TTCF daughter ensemble (arXiv:2312.02990).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2312_02990_gb300``) and neither imports the other;
both take their seeded inputs from ``paper_2312_02990_gb300.inputs``.

``ttcf_oracle.c`` holds the molecular dynamics (Eq. 3, 5, 6, 7; Algorithm 2;
the same equations under planar elongational flow),
``reduce.py`` the ensemble averages (Eq. 1, 2, 4, 8), ``cv.py`` the learned
control variate (not in the paper).
"""
from .core import (Bulk, build, lib, wca, forces, pressure, apply_mapping,
                   trajectory, mother, daughter, daughters, trajectory_elong,
                   daughter_elong, daughters_elong)
from .reduce import responses, viscosity, autocorrelation, green_kubo
from . import cv

__all__ = ["Bulk", "build", "lib", "wca", "forces", "pressure", "apply_mapping",
           "trajectory", "mother", "daughter", "daughters", "trajectory_elong",
           "daughter_elong", "daughters_elong", "responses", "viscosity",
           "autocorrelation", "green_kubo", "cv"]
