"""Thin ctypes binding of ``libpkd.so`` (the C ABI in ``include/pkd.h``).

Argument marshalling only: every step of every call runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (torch supplies device
memory and streams).  The library must be built (``_native.build()`` or
``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _native

PKD_OK, PKD_EINVAL, PKD_ENOMEM, PKD_ECUDA, PKD_ETIMEOUT, PKD_EINTERNAL = range(6)


class PkdError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class pkd_params(C.Structure):
    _fields_ = [("d", C.c_int), ("phi", C.c_int), ("lambda_", C.c_int), ("sigma_log2", C.c_int),
                ("sigma_os", C.c_int), ("count_mode", C.c_int), ("alpha_num", C.c_int),
                ("alpha_den", C.c_int), ("seed", C.c_uint64)]


@dataclass
class Params:
    """Build parameters (see pkd.h).  Defaults follow the paper's Sec. 5:
    lambda = 6, phi = 32, sigma_os = 32, alpha = 3/10; the sample rate is
    2^-sigma_log2 (1/64)."""

    d: int
    phi: int = 32
    lam: int = 6
    sigma_log2: int = 6
    sigma_os: int = 32
    count_mode: int = 0
    alpha_num: int = 3
    alpha_den: int = 10
    seed: int = 1

    def c(self) -> pkd_params:
        return pkd_params(self.d, self.phi, self.lam, self.sigma_log2, self.sigma_os,
                          self.count_mode, self.alpha_num, self.alpha_den, self.seed)


_lib = None


def lib():
    """Load libpkd.so; fail loudly when it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_native.LIB):
            raise ImportError(f"{_native.LIB} is not built; run __graft_entry__.build()")
        L = C.CDLL(_native.LIB)
        vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int
        P = C.POINTER
        L.pkd_build.argtypes = [vp, vp, u64, P(pkd_params), vp, P(vp)]
        L.pkd_batch_insert.argtypes = [vp, vp, vp, u64, vp]
        L.pkd_batch_delete.argtypes = [vp, vp, u64, P(u64), vp]
        L.pkd_knn.argtypes = [vp, vp, u64, i32, vp, vp, vp]
        L.pkd_range_count.argtypes = [vp, vp, vp, u64, vp, vp]
        L.pkd_knn_ids_noalloc.argtypes = [vp, vp, u64, i32, vp, vp]
        L.pkd_range_report.argtypes = [vp, vp, vp, u64, vp, vp, u64, P(u64), vp]
        L.pkd_build_forest.argtypes = [vp, vp, P(u64), C.c_uint32, P(pkd_params), vp, P(vp)]
        L.pkd_forest_trees.restype = C.c_uint32
        L.pkd_forest_trees.argtypes = [vp]
        L.pkd_forest_size.restype = u64
        L.pkd_forest_size.argtypes = [vp, C.c_uint32]
        L.pkd_forest_export.argtypes = [vp, C.c_uint32, vp, vp, vp, P(u64), vp, vp, P(u64)]
        L.pkd_forest_knn.argtypes = [vp, C.c_uint32, vp, u64, i32, vp, vp, vp]
        L.pkd_forest_free.argtypes = [vp]
        L.pkd_forest_free.restype = None
        L.pkd_export.argtypes = [vp, vp, vp, vp, P(u64), vp, vp, P(u64)]
        L.pkd_set_bounding_boxes.argtypes = [vp, i32, vp]
        L.pkd_mem_info.argtypes = [P(u64), P(u64), P(u64), P(u64), P(u64)]
        L.pkd_export_boxes.argtypes = [vp, vp, vp, u64]
        L.pkd_size.restype = u64
        L.pkd_size.argtypes = [vp]
        L.pkd_height.argtypes = [vp, P(i32)]
        L.pkd_free.argtypes = [vp]
        L.pkd_free.restype = None
        L.pkd_strerror.restype = C.c_char_p
        L.pkd_strerror.argtypes = [i32]
        L.pkd_set_option.argtypes = [C.c_char_p, C.c_int64]
        L.pkd_kernel_timing.argtypes = [i32]
        L.pkd_kernel_stats.argtypes = [C.c_char_p, P(u64), P(C.c_double), P(u64)]
        for f in ("pkd_build", "pkd_batch_insert", "pkd_batch_delete", "pkd_knn", "pkd_range_count",
                  "pkd_knn_ids_noalloc", "pkd_range_report", "pkd_set_bounding_boxes", "pkd_export_boxes", "pkd_mem_info", "pkd_build_forest", "pkd_forest_export", "pkd_forest_knn", "pkd_export", "pkd_height", "pkd_set_option", "pkd_kernel_timing",
                  "pkd_kernel_stats"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().pkd_strerror(code).decode()


def _check(code: int, what: str):
    if code != PKD_OK:
        raise PkdError(code, what)


def _dptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# --- the C ABI, one function per entry point --------------------------------

def pkd_build(coords: torch.Tensor, ids: torch.Tensor | None, params: Params, stream=None):
    """Build a tree over coords [n, d] int32 (device), ids [n] int32/uint32 or None."""
    assert coords.dtype == torch.int32 and coords.dim() == 2 and coords.shape[1] == params.d
    if ids is not None:
        assert ids.dtype in (torch.int32, torch.uint32) and ids.numel() == coords.shape[0]
    h = C.c_void_p()
    pc = params.c()
    _check(lib().pkd_build(_dptr(coords), _dptr(ids), coords.shape[0], C.byref(pc),
                           _stream(stream), C.byref(h)), "pkd_build")
    return h


def pkd_batch_insert(tree, coords: torch.Tensor, ids: torch.Tensor, stream=None):
    _check(lib().pkd_batch_insert(tree, _dptr(coords), _dptr(ids), coords.shape[0],
                                  _stream(stream)), "pkd_batch_insert")


def pkd_batch_delete(tree, ids: torch.Tensor, stream=None) -> int:
    """Delete the points named by ids [m] int32/uint32 (device); returns
    the number removed (unknown and repeated ids are skipped)."""
    nd = C.c_uint64(0)
    _check(lib().pkd_batch_delete(tree, _dptr(ids), ids.numel(), C.byref(nd), _stream(stream)),
           "pkd_batch_delete")
    return int(nd.value)


def pkd_knn(tree, queries: torch.Tensor, k: int, out_ids: torch.Tensor, out_d2: torch.Tensor,
            stream=None):
    _check(lib().pkd_knn(tree, _dptr(queries), queries.shape[0], k, _dptr(out_ids), _dptr(out_d2),
                         _stream(stream)), "pkd_knn")


def pkd_knn_ids_noalloc(tree, queries: torch.Tensor, k: int, out_ids: torch.Tensor, stream=None):
    """k-NN ids through the library's fixed scratch (no allocation in the call)."""
    _check(lib().pkd_knn_ids_noalloc(tree, _dptr(queries), queries.shape[0], k, _dptr(out_ids),
                                     _stream(stream)), "pkd_knn_ids_noalloc")


def pkd_range_count(tree, lo: torch.Tensor, hi: torch.Tensor, out: torch.Tensor, stream=None):
    _check(lib().pkd_range_count(tree, _dptr(lo), _dptr(hi), lo.shape[0], _dptr(out),
                                 _stream(stream)), "pkd_range_count")


def pkd_export(tree) -> dict:
    nn, nl = C.c_uint64(0), C.c_uint64(0)
    _check(lib().pkd_export(tree, None, None, None, C.byref(nn), None, None, C.byref(nl)), "pkd_export")
    n = int(lib().pkd_size(tree))
    dims = np.empty(nn.value, np.uint8)
    splits = np.empty(nn.value, np.int32)
    sizes = np.empty(nn.value, np.uint64)
    lids = np.empty(max(n, 1), np.uint32)
    offs = np.empty(nl.value + 1, np.uint64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(lib().pkd_export(tree, p(dims), p(splits), p(sizes), C.byref(nn), p(lids), p(offs),
                            C.byref(nl)), "pkd_export")
    return dict(dims=dims, splits=splits, sizes=sizes, leaf_ids=lids[:n], leaf_offsets=offs)


def pkd_range_report(tree, lo: torch.Tensor, hi: torch.Tensor, stream=None):
    """Ids of the points inside each box: (offsets [q+1] int64, ids) on the
    device; sizes the id buffer with a first call."""
    q = lo.shape[0]
    offsets = torch.empty(q + 1, dtype=torch.int64, device=lo.device)
    tot = C.c_uint64(0)
    r = lib().pkd_range_report(tree, _dptr(lo), _dptr(hi), q, _dptr(offsets), None, 0, C.byref(tot),
                               _stream(stream))
    if r != PKD_OK and not (r == PKD_EINVAL and tot.value > 0):
        _check(r, "pkd_range_report")
    ids = torch.empty(max(int(tot.value), 1), dtype=torch.int32, device=lo.device)
    _check(lib().pkd_range_report(tree, _dptr(lo), _dptr(hi), q, _dptr(offsets), _dptr(ids), ids.numel(),
                                  C.byref(tot), _stream(stream)), "pkd_range_report")
    return offsets, ids[:int(tot.value)]


def pkd_build_forest(coords: torch.Tensor, ids: torch.Tensor | None, offsets, params: Params, stream=None):
    """Build len(offsets) - 1 independent trees over coords [n, d] in one pass;
    offsets is a host sequence of n_trees + 1 point offsets."""
    assert coords.dtype == torch.int32 and coords.dim() == 2 and coords.shape[1] == params.d
    if ids is not None:
        assert ids.dtype in (torch.int32, torch.uint32) and ids.numel() == coords.shape[0]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    assert off.ndim == 1 and off.size >= 2 and int(off[-1]) == coords.shape[0]
    h = C.c_void_p()
    pc = params.c()
    _check(lib().pkd_build_forest(_dptr(coords), _dptr(ids), off.ctypes.data_as(C.POINTER(C.c_uint64)),
                                  off.size - 1, C.byref(pc), _stream(stream), C.byref(h)), "pkd_build_forest")
    return h


def pkd_forest_export(forest, tree: int) -> dict:
    nn, nl = C.c_uint64(0), C.c_uint64(0)
    _check(lib().pkd_forest_export(forest, tree, None, None, None, C.byref(nn), None, None, C.byref(nl)),
           "pkd_forest_export")
    n = int(lib().pkd_forest_size(forest, tree))
    dims = np.empty(nn.value, np.uint8)
    splits = np.empty(nn.value, np.int32)
    sizes = np.empty(nn.value, np.uint64)
    lids = np.empty(max(n, 1), np.uint32)
    offs = np.empty(nl.value + 1, np.uint64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(lib().pkd_forest_export(forest, tree, p(dims), p(splits), p(sizes), C.byref(nn), p(lids), p(offs),
                                   C.byref(nl)), "pkd_forest_export")
    return dict(dims=dims, splits=splits, sizes=sizes, leaf_ids=lids[:n], leaf_offsets=offs)


def pkd_forest_knn(forest, tree: int, queries: torch.Tensor, k: int, out_ids: torch.Tensor,
                   out_d2: torch.Tensor, stream=None):
    _check(lib().pkd_forest_knn(forest, tree, _dptr(queries), queries.shape[0], k, _dptr(out_ids),
                                _dptr(out_d2), _stream(stream)), "pkd_forest_knn")


def pkd_forest_free(forest):
    lib().pkd_forest_free(forest)


def pkd_set_bounding_boxes(tree, enable: bool, stream=None):
    """Keep (True) or drop (False) the tight box of every node (Pkd-bb)."""
    _check(lib().pkd_set_bounding_boxes(tree, 1 if enable else 0, _stream(stream)), "pkd_set_bounding_boxes")


def pkd_export_boxes(tree, n_nodes: int, d: int):
    """The stored boxes in pre-order: (lo, hi), each [n_nodes, d] int32."""
    lo = np.empty((n_nodes, d), np.int32)
    hi = np.empty((n_nodes, d), np.int32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(lib().pkd_export_boxes(tree, p(lo), p(hi), n_nodes), "pkd_export_boxes")
    return lo, hi


def pkd_mem_info() -> dict:
    """Device memory as the library sees it (bytes): free, pool_reserved,
    pool_used, cached and available (free + unused pool + cache)."""
    v = [C.c_uint64(0) for _ in range(5)]
    _check(lib().pkd_mem_info(*[C.byref(x) for x in v]), "pkd_mem_info")
    return dict(zip(("free", "pool_reserved", "pool_used", "cached", "available"), (int(x.value) for x in v)))


def pkd_size(tree) -> int:
    return int(lib().pkd_size(tree))


def pkd_height(tree) -> int:
    h = C.c_int(0)
    _check(lib().pkd_height(tree, C.byref(h)), "pkd_height")
    return int(h.value)


def pkd_free(tree):
    lib().pkd_free(tree)


def pkd_set_option(name: str, value: int):
    _check(lib().pkd_set_option(name.encode(), int(value)), f"pkd_set_option({name})")


def pkd_kernel_timing(enable: bool):
    _check(lib().pkd_kernel_timing(1 if enable else 0), "pkd_kernel_timing")


def pkd_kernel_stats(name: str):
    n, it = C.c_uint64(0), C.c_uint64(0)
    ms = C.c_double(0)
    _check(lib().pkd_kernel_stats(name.encode(), C.byref(n), C.byref(ms), C.byref(it)),
           "pkd_kernel_stats")
    return int(n.value), float(ms.value), int(it.value)


# --- convenience wrapper -----------------------------------------------------

class Tree:
    """A Pkd-tree on the current CUDA device."""

    def __init__(self, coords: torch.Tensor, ids: torch.Tensor | None, params: Params, stream=None):
        self.params = params
        self._h = pkd_build(coords, ids, params, stream)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            pkd_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def size(self) -> int:
        return pkd_size(self._h)

    @property
    def height(self) -> int:
        return pkd_height(self._h)

    def insert(self, coords, ids, stream=None):
        pkd_batch_insert(self._h, coords, ids, stream)

    def delete(self, ids, stream=None) -> int:
        return pkd_batch_delete(self._h, ids, stream)

    def knn(self, queries: torch.Tensor, k: int, stream=None):
        out_i = torch.empty((queries.shape[0], k), dtype=torch.int32, device=queries.device)
        out_d = torch.empty((queries.shape[0], k), dtype=torch.int64, device=queries.device)
        pkd_knn(self._h, queries, k, out_i, out_d, stream)
        return out_i, out_d

    def range_count(self, lo: torch.Tensor, hi: torch.Tensor, stream=None):
        out = torch.empty(lo.shape[0], dtype=torch.int64, device=lo.device)
        pkd_range_count(self._h, lo, hi, out, stream)
        return out

    def export(self) -> dict:
        return pkd_export(self._h)
