"""Autotuner for the build: picks lambda (skeleton levels per sieve round),
the sample rate 2^-sigma_log2 and the sieve tile size by timing pkd_build on
a sample of the workload.

lambda and the sample rate change the tree (they are parameters of Alg. 1;
the paper fixes lambda = 6 and sigma = 32 by a similar sweep, Sec. 5
"Parameter Choosing"), so whatever is chosen is recorded with the results
and parity is checked with the chosen values.  The tile size is a tuning
knob that never changes the tree.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np
import torch

from . import pkd


@dataclasses.dataclass(frozen=True)
class Candidate:
    lam: int
    sigma_log2: int
    tile: int

    def params(self, d: int, **kw) -> pkd.Params:
        return pkd.Params(d=d, lam=self.lam, sigma_log2=self.sigma_log2, **kw)


def grid(lambdas=(5, 6, 7, 8), sigma_log2s=(5, 6, 7, 8), tiles=(1024, 2048, 4096)) -> list[Candidate]:
    """Every combination, lambda in [1, 10], sigma_log2 in [0, 30], tiles
    powers of two in [256, 4096] (the library's ranges)."""
    out = []
    for lam, sl, tile in itertools.product(lambdas, sigma_log2s, tiles):
        if not (1 <= lam <= 10 and 0 <= sl <= 30 and 256 <= tile <= 4096 and tile & (tile - 1) == 0):
            raise ValueError(f"candidate out of range: lam={lam} sigma_log2={sl} tile={tile}")
        out.append(Candidate(lam, sl, tile))
    return out


def pick(times: dict[Candidate, float]) -> Candidate:
    """The fastest candidate; ties go to the earliest in (lam, sigma_log2,
    tile) order, so the choice is reproducible."""
    return min(times, key=lambda c: (times[c], c.lam, c.sigma_log2, c.tile))


def time_build(coords: torch.Tensor, cand: Candidate, reps: int = 2, stream=None) -> float:
    """Median device time (ms) of pkd_build with the candidate's parameters."""
    d = coords.shape[1]
    st = stream or torch.cuda.current_stream()
    pkd.pkd_set_option("tile", cand.tile)
    try:
        pkd.pkd_free(pkd.pkd_build(coords, None, cand.params(d), st))  # warm-up
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            h = pkd.pkd_build(coords, None, cand.params(d), st)
            b.record(st)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            pkd.pkd_free(h)
        return float(np.median(ts))
    finally:
        pkd.pkd_set_option("tile", 2048)


def tune(coords: torch.Tensor, candidates: list[Candidate] | None = None, reps: int = 2) -> dict:
    """Time every candidate on `coords` (a device [n, d] int32 sample of the
    workload) and return the choice with the whole table."""
    cands = candidates or grid()
    times = {c: time_build(coords, c, reps) for c in cands}
    best = pick(times)
    return {"best": dataclasses.asdict(best), "sample_points": int(coords.shape[0]),
            "table": [dict(dataclasses.asdict(c), ms=t) for c, t in sorted(times.items(), key=lambda kv: kv[1])]}
