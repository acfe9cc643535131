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


def _lib_and_params():
    lib = ctypes.CDLL(_native.build())

    class P(ctypes.Structure):
        _fields_ = [("d", ctypes.c_int), ("phi", ctypes.c_int), ("lambda_", ctypes.c_int),
                    ("sigma_log2", ctypes.c_int), ("sigma_os", ctypes.c_int), ("count_mode", ctypes.c_int),
                    ("alpha_num", ctypes.c_int), ("alpha_den", ctypes.c_int), ("seed", ctypes.c_uint64)]

    lib.pkd_build.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(P), ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_void_p)]
    lib.pkd_set_option.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    return lib, P


def test_build_rejects_bad_parameters_before_any_device_work():
    # parameter checks are host-only and come first (pkd.h: PKD_EINVAL)
    lib, P = _lib_and_params()
    good = dict(d=3, phi=32, lambda_=6, sigma_log2=6, sigma_os=32, count_mode=0, alpha_num=3, alpha_den=10, seed=1)
    bad = [dict(d=0), dict(d=9), dict(phi=0), dict(lambda_=0), dict(lambda_=11), dict(sigma_log2=-1),
           dict(sigma_log2=31), dict(sigma_os=0), dict(count_mode=2), dict(alpha_den=0), dict(alpha_den=(1 << 20) + 1),
           dict(alpha_num=-1), dict(alpha_num=6, alpha_den=10)]
    h = ctypes.c_void_p()
    for b in bad:
        p = P(**dict(good, **b))
        assert lib.pkd_build(None, None, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1, b
        assert h.value is None
    p = P(**good)
    assert lib.pkd_build(None, None, 0, ctypes.byref(p), None, None) == 1          # no output slot
    assert lib.pkd_build(None, None, 1 << 31, ctypes.byref(p), None, ctypes.byref(h)) == 1  # n too large
    assert lib.pkd_build(None, None, 10, ctypes.byref(p), None, ctypes.byref(h)) == 1        # no coordinates
    assert lib.pkd_build(None, None, 0, None, None, ctypes.byref(h)) == 1                     # no parameters


def test_null_tree_and_option_ranges():
    lib, _ = _lib_and_params()
    for f in ("pkd_batch_insert", "pkd_batch_delete", "pkd_knn", "pkd_range_count", "pkd_export", "pkd_height"):
        getattr(lib, f).restype = ctypes.c_int
    assert lib.pkd_batch_insert(None, None, None, ctypes.c_uint64(5), None) == 1
    assert lib.pkd_batch_delete(None, None, ctypes.c_uint64(5), None, None) == 1
    assert lib.pkd_knn(None, None, ctypes.c_uint64(1), 1, None, None, None) == 1
    assert lib.pkd_range_count(None, None, None, ctypes.c_uint64(1), None, None) == 1
    assert lib.pkd_export(None, None, None, None, None, None, None, None) == 1
    assert lib.pkd_height(None, None) == 1
    # tuning options: unknown names and out-of-range values are rejected
    for name, v in ((b"no_such_option", 1), (b"fail_alloc_after", -2), (b"tile", 100), (b"tile", 3000), (b"tile", 8192), (b"base_cap", 32),
                    (b"base_cap", 20000), (b"skel_cap", 63), (b"sieve_kernel", 3), (b"sieve_kernel", -1),
                    (b"base_kernel", 2)):
        assert lib.pkd_set_option(name, v) == 1, (name, v)
    assert lib.pkd_set_option(None, 0) == 1
    # accepted values, then the defaults back
    for name, v in ((b"tile", 512), (b"base_cap", 1024), (b"skel_cap", 256), (b"sieve_kernel", 2), (b"base_kernel", 1)):
        assert lib.pkd_set_option(name, v) == 0, (name, v)
    for name, v in ((b"tile", 2048), (b"base_cap", 0), (b"skel_cap", 0), (b"sieve_kernel", 0), (b"base_kernel", 0)):
        assert lib.pkd_set_option(name, v) == 0
