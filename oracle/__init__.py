"""CPU FP64 oracle for the finite-element Bloch-Torrey solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import it: only the
tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg and
reference arm use it.
It shares no code with the CUDA library; both read the same seeded inputs from
``geom``.
"""
from .btoracle import (assemble, doubling, interface_faces, periodic_master, pgse_tables,
                       q_from_b, run, run_lab, run_transformed, sequence, signal_weights)
from .mf1d import mf_interval_signal

__all__ = ["assemble", "doubling", "interface_faces", "periodic_master", "pgse_tables",
           "q_from_b", "run", "run_lab", "run_transformed", "sequence", "signal_weights",
           "mf_interval_signal"]
