"""Seeded synthetic inputs (uniform and varden-like points, query boxes,
index samples).

A module of its own: it draws random inputs and holds none of the kd-tree
method's arithmetic, so the CUDA path and the CPU oracle can both take their
inputs from it.  The generators are written in C (``inputs.c``), integer-only
and therefore identical on x86-64 and AArch64 for a given seed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inputs.c")
_LIB = os.path.join(_HERE, "libpkdinputs.so")

# Seeds of the benchmark workloads: data, queries, insert batch, delete ids.
SEED_DATA, SEED_QUERY, SEED_INSERT, SEED_DELETE = 1, 2, 3, 4
SEED_VARDEN = 11

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _l():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp = C.c_void_p
        L.pkdin_uniform.argtypes = [vp, C.c_uint64, C.c_int, C.c_uint64]
        L.pkdin_varden.argtypes = [vp, C.c_uint64, C.c_int, C.c_uint64]
        L.pkdin_sample_indices.restype = C.c_int
        L.pkdin_sample_indices.argtypes = [vp, C.c_uint64, C.c_uint64, C.c_uint64]
        L.pkdin_boxes.argtypes = [vp, vp, C.c_uint64, C.c_int, C.c_uint32, C.c_uint64]
        L.pkdin_splitmix64_first.restype = C.c_uint64
        L.pkdin_splitmix64_first.argtypes = [C.c_uint64]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def uniform(n: int, d: int, seed: int = SEED_DATA) -> np.ndarray:
    """int32 [n, d], each coordinate uniform in [0, 2^30)."""
    out = np.empty((n, d), np.int32)
    _l().pkdin_uniform(_p(out), n, d, seed)
    return out


def varden(n: int, d: int, seed: int = SEED_VARDEN) -> np.ndarray:
    """int32 [n, d], one clamped random walk with rare uniform restarts."""
    out = np.empty((n, d), np.int32)
    _l().pkdin_varden(_p(out), n, d, seed)
    return out


def points(kind: str, n: int, d: int, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform(n, d, seed)
    if kind == "varden":
        return varden(n, d, seed)
    raise ValueError(kind)


def sample_indices(k: int, n: int, seed: int = SEED_DELETE) -> np.ndarray:
    """k distinct indices of [0, n), uint32."""
    out = np.empty(k, np.uint32)
    if _l().pkdin_sample_indices(_p(out), k, n, seed):
        raise MemoryError("sample_indices")
    return out


def boxes(q: int, d: int, max_side: int, seed: int = SEED_QUERY):
    """q closed boxes (lo, hi), int32 [q, d] each."""
    lo = np.empty((q, d), np.int32)
    hi = np.empty((q, d), np.int32)
    _l().pkdin_boxes(_p(lo), _p(hi), q, d, max_side, seed)
    return lo, hi


def splitmix64_first(seed: int) -> int:
    return int(_l().pkdin_splitmix64_first(seed))
