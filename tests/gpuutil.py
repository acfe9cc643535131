"""Helpers shared by the GPU tests (marshalling only)."""
from __future__ import annotations

import contextlib

import numpy as np

import oracle as O
from paper_2411_09275_gb300 import inputs as I


def dev():
    import torch

    return torch.device("cuda:0")


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def ids_dev(a):
    import torch

    a = np.asarray(a)
    assert a.min(initial=0) >= 0 and a.max(initial=0) < (1 << 32)
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(dev())


def oparams(p) -> O.Params:
    return O.Params(d=p.d, phi=p.phi, lam=p.lam, sigma_log2=p.sigma_log2, sigma_os=p.sigma_os,
                    count_mode=p.count_mode, alpha_num=p.alpha_num, alpha_den=p.alpha_den,
                    seed=p.seed)


# library options whose default is not 0
DEFAULTS = {"tile": 2048, "wait_cycles": 4_000_000_000, "fail_alloc_after": -1, "graph_rounds": 1}


@contextlib.contextmanager
def knobs(**kw):
    from paper_2411_09275_gb300 import pkd

    try:
        for k, v in kw.items():
            pkd.pkd_set_option(k, v)
        yield
    finally:
        for k in kw:
            pkd.pkd_set_option(k, DEFAULTS.get(k, 0))


def make_points(kind: str, n: int, d: int, seed: int) -> np.ndarray:
    if kind == "dups":
        return (I.uniform(n, d, seed) % 5).astype(np.int32)
    if kind == "dups_big":
        X = I.uniform(n, d, seed)
        X[: n // 2] = X[0]  # half the points identical
        return X
    if kind == "line":
        X = I.uniform(n, d, seed)
        X[:, 1:] = 7  # all extent in dimension 0
        return X
    return I.points(kind, n, d, seed)
