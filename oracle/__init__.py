"""FP64 CPU oracle for stochastic convolutional sparse coding (SCSC).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow statement of what
the GPU library computes: the CSC objective (Eq. 1), the subsampled code
problem (Eq. 3) solved by proximal gradient, the up-projection (Eq. 4), the
batch dictionary step (Eq. 5), the online surrogates (Eq. 7, Eq. 8), the
ADMM and Gauss-Seidel solvers (Sec. 3.2), inpainting (Sec. 4.3) and safe
screening of the code problem (Sec. 5) of
Xiong, Richtarik & Heidrich, "Stochastic Convolutional Sparse Coding" (2019).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.

The arithmetic lives in ``scsc_oracle.c`` (plain C, FP64), compiled by
:func:`build` with gcc; :mod:`oracle.reference` composes it per batch.
Parity status: pinned (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scsc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, OpenMP) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB)
        for p in (_SRC, os.path.join(_HERE, "scsc_oracle.h")))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        # -ffp-contract=off: every product and sum is rounded on its own, as
        # written; no FMA contraction in the oracle.
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i, u32, u64, dbl = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
            sig = {
                "orc_splitmix64": (u64, [u64]),
                "orc_is_sampled": (i, [u64, u64, u64, i, i, i, i, i, u32, u32]),
                "orc_mask_image": (None, [u64, u64, u64, i, i, i, u32, u32, P]),
                "orc_synthesis": (None, [i, i, i, i, P, P, P]),
                "orc_adjoint": (None, [i, i, i, i, P, P, P]),
                "orc_filter_gradient": (None, [i, i, i, i, P, P, P]),
                "orc_soft_threshold": (dbl, [dbl, dbl]),
                "orc_project_filters": (None, [i, i, P]),
                "orc_objective_image": (dbl, [i, i, i, i, P, P, P, dbl]),
                "orc_code_update_image": (None, [i, i, i, i, P, P, P, P, dbl, dbl, i]),
                "orc_code_update_image_keep": (None, [i, i, i, i, P, P, P, P, dbl, dbl, i]),
                "orc_objective_image_observed": (dbl, [i, i, i, i, P, P, P, P, dbl]),
                "orc_code_update_image_observed": (None, [i, i, i, i, P, P, P, P, P, dbl, dbl,
                                                          i]),
                "orc_power_ddt": (dbl, [i, i, i, i, P, u64, u64, i]),
                "orc_power_ztz": (dbl, [i, P, P, P, i, i, P, u64, u64, i]),
                "orc_power_dense": (dbl, [i, P, u64, u64, i]),
                "orc_surrogate_accumulate": (None, [i, i, i, i, P, P, dbl, P, P]),
                "orc_admm_image": (None, [i, i, i, i, P, P, P, P, dbl, dbl, dbl, i, i]),
                "orc_screen_image": (ctypes.c_int64, [i, i, i, i, P, P, P, P, dbl, P, P]),
                "orc_code_update_image_screened": (ctypes.c_int64, [i, i, i, i, P, P, P, P, dbl,
                                                                    dbl, i, i, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib
