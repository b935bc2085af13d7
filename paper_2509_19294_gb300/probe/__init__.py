"""Binding of libnbody_probe.so: measured per-SM issue rates behind the force
kernel's roofline (see probe/pipe_rates.h).  A measurement aid for bench.py,
not part of the force library; like the force library it has no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "libnbody_probe.so")
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (build.py builds both libraries)")
        lib = ctypes.CDLL(path)
        lib.nbody_measure_pipes.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        lib.nbody_measure_pipes.restype = ctypes.c_int
        _lib = lib
    return _lib


def measure_pipes() -> dict:
    """FP32 f32x2 lanes, MUFU rsqrt, force-kernel pair arithmetic (pairs) and
    FP64 FMA per clock per SM of the current GPU."""
    out = (ctypes.c_double * 4)()
    rc = load().nbody_measure_pipes(out, 4)
    if rc != 0:
        raise RuntimeError(f"nbody_measure_pipes failed with status {rc}")
    return {"fp32_lanes_per_clk_sm": out[0], "mufu_rsqrt_per_clk_sm": out[1],
            "pair_arith_pairs_per_clk_sm": out[2], "fp64_fma_per_clk_sm": out[3]}
