"""The C-ABI library loads and exports every entry point that include/pkd.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

from paper_2411_09275_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pkd.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pkd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pkd_build", "pkd_batch_insert", "pkd_batch_delete", "pkd_knn", "pkd_range_count",
              "pkd_export", "pkd_free", "pkd_size", "pkd_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _native.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (pkd_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"not exported: {missing}"
    L = ctypes.CDLL(lib)
    for n in _declared():
        assert getattr(L, n) is not None
    L.pkd_strerror.restype = ctypes.c_char_p
    assert L.pkd_strerror(1) == b"invalid argument"
