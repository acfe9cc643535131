"""Pkd-tree CPU oracle -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``oracle.c``: a plain single-threaded C restatement of
the construction (Alg. 1), batch insertion (Alg. 2), batch deletion (Sec. 4.2)
and the k-NN / range-count queries (Sec. 5) of "Parallel kd-tree with Batch
Updates".  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the CUDA library never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C, -O2, no vendor code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("d", C.c_int),
        ("phi", C.c_int),
        ("lam", C.c_int),
        ("sigma_log2", C.c_int),
        ("sigma_os", C.c_int),
        ("count_mode", C.c_int),
        ("alpha_num", C.c_int),
        ("alpha_den", C.c_int),
        ("seed", C.c_uint64),
    ]


@dataclass
class Params:
    """Pkd-tree parameters (Sec. 5 "Parameter Choosing": lambda=6, phi=32,
    sigma=32, alpha=0.3).  ``sigma_log2`` is the sample-rate exponent of rate
    mode (rate 2^-sigma_log2); ``count_mode`` switches to about
    2^lambda * sigma_os samples per subproblem as in Alg. 1."""

    d: int
    phi: int = 32
    lam: int = 6
    sigma_log2: int = 6
    sigma_os: int = 32
    count_mode: int = 0
    alpha_num: int = 3
    alpha_den: int = 10
    seed: int = 1

    def c(self) -> _Params:
        return _Params(self.d, self.phi, self.lam, self.sigma_log2, self.sigma_os,
                       self.count_mode, self.alpha_num, self.alpha_den, self.seed)


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        vp = C.c_void_p
        L.orc_build.restype = vp
        L.orc_build.argtypes = [vp, vp, C.c_uint64, P(_Params), P(C.c_int)]
        L.orc_build_at_depth.restype = vp
        L.orc_build_at_depth.argtypes = [vp, vp, C.c_uint64, P(_Params), C.c_uint32, P(C.c_int)]
        L.orc_insert.restype = C.c_int
        L.orc_insert.argtypes = [vp, vp, vp, C.c_uint64]
        L.orc_delete.restype = C.c_int
        L.orc_delete.argtypes = [vp, vp, C.c_uint64, P(C.c_uint64)]
        L.orc_free.argtypes = [vp]
        L.orc_size.restype = C.c_uint64
        L.orc_size.argtypes = [vp]
        L.orc_height.restype = C.c_int
        L.orc_height.argtypes = [vp]
        L.orc_export.restype = C.c_int
        L.orc_export.argtypes = [vp, vp, vp, vp, P(C.c_uint64), vp, vp, P(C.c_uint64)]
        L.orc_points.argtypes = [vp, vp, vp]
        for f in ("orc_knn_brute", "orc_knn_tree"):
            getattr(L, f).argtypes = [vp, vp, C.c_uint64, C.c_int, vp, vp]
        for f in ("orc_range_count_brute", "orc_range_count_tree"):
            getattr(L, f).argtypes = [vp, vp, vp, C.c_uint64, vp]
        L.orc_mix64.restype = C.c_uint64
        L.orc_mix64.argtypes = [C.c_uint64]
        L.orc_sample_hash.restype = C.c_uint64
        L.orc_sample_hash.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.orc_sample_shift.restype = C.c_int
        L.orc_sample_shift.argtypes = [P(_Params), C.c_uint64]
        L.orc_is_sampled.restype = C.c_int
        L.orc_is_sampled.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int]
        L.orc_split_rule.restype = C.c_int
        L.orc_split_rule.argtypes = [vp, C.c_uint64, C.c_int, P(C.c_int), P(C.c_int32)]
        L.orc_balanced.restype = C.c_int
        L.orc_balanced.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _coords(a, d: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a.reshape(-1, d)


class OracleError(RuntimeError):
    pass


class OracleTree:
    """A Pkd-tree held by the CPU oracle."""

    def __init__(self, coords, ids=None, params: Params | None = None, depth: int = 0):
        assert params is not None
        self.params = params
        self._pc = params.c()
        c = _coords(coords, params.d)
        i = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
        err = C.c_int(0)
        h = lib().orc_build_at_depth(_ptr(c), _ptr(i), c.shape[0], C.byref(self._pc), depth,
                                     C.byref(err))
        if not h:
            raise OracleError(f"orc_build failed: {err.value}")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def size(self) -> int:
        return int(lib().orc_size(self._h))

    @property
    def height(self) -> int:
        return int(lib().orc_height(self._h))

    def insert(self, coords, ids):
        c = _coords(coords, self.params.d)
        i = np.ascontiguousarray(ids, dtype=np.uint32)
        r = lib().orc_insert(self._h, _ptr(c), _ptr(i), c.shape[0])
        if r:
            raise OracleError(f"orc_insert failed: {r}")

    def delete(self, ids) -> int:
        """Delete the points named by ids (Sec. 4.2 with the id as the key);
        unknown and repeated ids are skipped.  Returns the points removed."""
        i = np.ascontiguousarray(ids, dtype=np.uint32).reshape(-1)
        nd = C.c_uint64(0)
        r = lib().orc_delete(self._h, _ptr(i), i.shape[0], C.byref(nd))
        if r:
            raise OracleError(f"orc_delete failed: {r}")
        return int(nd.value)

    def export(self) -> dict:
        nn, nl = C.c_uint64(0), C.c_uint64(0)
        lib().orc_export(self._h, None, None, None, C.byref(nn), None, None, C.byref(nl))
        dims = np.empty(nn.value, np.uint8)
        splits = np.empty(nn.value, np.int32)
        sizes = np.empty(nn.value, np.uint64)
        offs = np.empty(nl.value + 1, np.uint64)
        lids = np.empty(self.size, np.uint32)
        lib().orc_export(self._h, _ptr(dims), _ptr(splits), _ptr(sizes), C.byref(nn),
                         _ptr(lids), _ptr(offs), C.byref(nl))
        return dict(dims=dims, splits=splits, sizes=sizes, leaf_ids=lids, leaf_offsets=offs)

    def points(self):
        n = self.size
        ids = np.empty(n, np.uint32)
        xs = np.empty((n, self.params.d), np.int32)
        lib().orc_points(self._h, _ptr(ids), _ptr(xs))
        return ids, xs

    def knn(self, queries, k: int, brute: bool = False):
        q = _coords(queries, self.params.d)
        ids = np.empty((q.shape[0], k), np.uint32)
        d2 = np.empty((q.shape[0], k), np.int64)
        f = lib().orc_knn_brute if brute else lib().orc_knn_tree
        f(self._h, _ptr(q), q.shape[0], k, _ptr(ids), _ptr(d2))
        return ids, d2

    def range_count(self, lo, hi, brute: bool = False):
        lo = _coords(lo, self.params.d)
        hi = _coords(hi, self.params.d)
        out = np.empty(lo.shape[0], np.uint64)
        f = lib().orc_range_count_brute if brute else lib().orc_range_count_tree
        f(self._h, _ptr(lo), _ptr(hi), lo.shape[0], _ptr(out))
        return out

    def range_report(self, lo, hi) -> list:
        """Range report (Sec. 5, reporting form of the range query) by its
        definition: for each closed box, the sorted ids of the stored points
        with lo <= x <= hi in every dimension."""
        ids, X = self.points()
        return range_report(X, ids, lo, hi)


def range_report(points, ids, lo, hi) -> list:
    """Sorted ids of the points inside each closed box (brute force)."""
    P = np.asarray(points).reshape(len(ids), -1)
    i = np.asarray(ids, dtype=np.uint32)
    out = []
    for a, b in zip(np.asarray(lo), np.asarray(hi)):
        inside = np.all((P >= a) & (P <= b), axis=1)
        out.append(np.sort(i[inside]))
    return out


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def sample_hash(seed: int, depth: int, id_: int) -> int:
    return int(lib().orc_sample_hash(seed, depth, id_))


def sample_shift(params: Params, n: int) -> int:
    pc = params.c()
    return int(lib().orc_sample_shift(C.byref(pc), n))


def is_sampled(seed: int, depth: int, id_: int, shift: int) -> bool:
    return bool(lib().orc_is_sampled(seed, depth, id_, shift))


def split_rule(pts) -> tuple[int, int] | None:
    p = np.ascontiguousarray(pts, dtype=np.int32)
    if p.ndim == 1:
        p = p.reshape(-1, 1)
    dim, x = C.c_int(0), C.c_int32(0)
    r = lib().orc_split_rule(_ptr(p), p.shape[0], p.shape[1], C.byref(dim), C.byref(x))
    return None if r else (int(dim.value), int(x.value))


def balanced(left: int, total: int, alpha_num: int, alpha_den: int) -> bool:
    return bool(lib().orc_balanced(left, total, alpha_num, alpha_den))
