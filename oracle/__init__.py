"""FP64 CPU oracle for the per-frame irradiance-volume update, selection and packing.

TEST INFRASTRUCTURE ONLY. This package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` and by nothing else: the CUDA library never calls it and shares no
code with it. It is a plain, slow restatement of the method of Sections 3.2-3.4
of "A Distributed, Decoupled System for Losslessly Streaming Dynamic Light
Probes to Thin Clients" (arXiv 2103.05875), in float64 numpy, with each step
citing the passage it follows.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, brute force or the paper's printed
numbers; none is "parity unpinned".
"""
from . import blend, numerics, octahedral, select_pack  # noqa: F401
from .volume import Frame, OracleVolume  # noqa: F401
