"""CPU oracle of the SAT sampler's hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it and
shares no code with it.

Contents (each function cites the passage of the paper it restates):

* ``dimacs``     — DIMACS reader and plain CNF evaluation (Section II-A, Fig. 1(a)).
* ``transform``  — Algorithm 1 and its fallback (Section III-A).
* ``relax.c``    — FP64 relaxation, l2 loss, adjoint, GD/Adam, threshold, Boolean
                   evaluation, CNF check, Philox4x32-10 (Table 1, Eqs. 5-9).
* ``sampler``    — orchestration of rounds, verification and deduplication.
* ``mlp``        — FP64 proposal network: forward, BCE, gradients, IMLE selection.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_PATH = _HERE / "liborc.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile relax.c into liborc.so (gcc, -O2, OpenMP)."""
    src = _HERE / "relax.c"
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < src.stat().st_mtime:
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", str(src), "-o", str(_LIB_PATH), "-lm"])
    return _LIB_PATH


class OrcCircuit(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int), ("n_instr", ctypes.c_int),
        ("ins_out", ctypes.c_void_p), ("ins_op", ctypes.c_void_p), ("ins_neg", ctypes.c_void_p),
        ("ins_off", ctypes.c_void_p), ("ins_cnt", ctypes.c_void_p),
        ("lit_node", ctypes.c_void_p), ("lit_neg", ctypes.c_void_p),
        ("n_pi", ctypes.c_int), ("pi_node", ctypes.c_void_p),
        ("n_out", ctypes.c_int), ("out_node", ctypes.c_void_p), ("target", ctypes.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        L.orc_threads.restype = ctypes.c_int
        L.orc_forward.argtypes = [P, ctypes.c_int, P, P, P]
        L.orc_backward.argtypes = [P, ctypes.c_int, P, P, P]
        L.orc_backward_mag.argtypes = [P, ctypes.c_int, P, P, P]
        L.orc_gd.argtypes = [ctypes.c_long, P, P, ctypes.c_double]
        L.orc_adam.argtypes = [ctypes.c_long, P, P, P, P, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_hard.argtypes = [P, ctypes.c_int, P, P]
        L.orc_cnf_check.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_init_normal.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_double, P]
        _lib = L
    return _lib


def ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


from .dimacs import parse_dimacs, cnf_satisfied, DimacsError  # noqa: E402,F401
from .transform import factorize, direct_circuit, Circuit, Definition  # noqa: E402,F401
from .sampler import (  # noqa: E402,F401
    FlatCircuit, flatten, forward, backward, backward_magnitude, adam_step, gd_step, hard_eval,
    full_assignment, cnf_check, solution_hash, philox4x32_10, init_normal,
    sample_round, verify, Oracle,
)
