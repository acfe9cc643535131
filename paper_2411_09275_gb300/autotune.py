"""Autotuner for the build: picks lambda (skeleton levels per sieve round),
the sample rate 2^-sigma_log2, the leaf wrap phi, the sieve tile size and the
shared-memory base-case cutoff by timing pkd_build on a sample of the
workload.

lambda, the sample rate and phi change the tree (they are parameters of
Alg. 1; the paper fixes lambda = 6, sigma = 32 and phi = 32 by a similar
sweep, Sec. 5 "Parameter Choosing"), so whatever is chosen is recorded with
the results and parity is checked with the chosen values.  The tile size and
the base-case cutoff (the largest subproblem finished by one CTA in shared
memory; 0 = as large as shared memory allows) are tuning knobs that never
change the tree.
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
    phi: int = 32
    base_cap: int = 0

    def params(self, d: int, **kw) -> pkd.Params:
        return pkd.Params(d=d, lam=self.lam, sigma_log2=self.sigma_log2, phi=self.phi, **kw)


def grid(lambdas=(5, 6, 7, 8), sigma_log2s=(5, 6, 7, 8), tiles=(1024, 2048, 4096), phis=(32,),
         base_caps=(0,)) -> list[Candidate]:
    """Every combination, lambda in [1, 10], sigma_log2 in [0, 30], tiles
    powers of two in [256, 4096], phi >= 1, base_cap 0 or in [64, 16384]
    (the library's ranges)."""
    out = []
    for lam, sl, tile, phi, bc in itertools.product(lambdas, sigma_log2s, tiles, phis, base_caps):
        if not (1 <= lam <= 10 and 0 <= sl <= 30 and 256 <= tile <= 4096 and tile & (tile - 1) == 0
                and phi >= 1 and (bc == 0 or 64 <= bc <= 16384)):
            raise ValueError(f"candidate out of range: lam={lam} sigma_log2={sl} tile={tile} phi={phi} "
                             f"base_cap={bc}")
        out.append(Candidate(lam, sl, tile, phi, bc))
    return out


def pick(times: dict[Candidate, float]) -> Candidate:
    """The fastest candidate; ties go to the earliest in (lam, sigma_log2,
    tile, phi, base_cap) order, so the choice is reproducible."""
    return min(times, key=lambda c: (times[c], c.lam, c.sigma_log2, c.tile, c.phi, c.base_cap))


def time_build(coords: torch.Tensor, cand: Candidate, reps: int = 2, stream=None) -> float:
    """Median device time (ms) of pkd_build with the candidate's parameters."""
    d = coords.shape[1]
    st = stream or torch.cuda.current_stream()
    pkd.pkd_set_option("tile", cand.tile)
    pkd.pkd_set_option("base_cap", cand.base_cap)
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
        pkd.pkd_set_option("base_cap", 0)


def tune(coords: torch.Tensor, candidates: list[Candidate] | None = None, reps: int = 2) -> dict:
    """Time every candidate on `coords` (a device [n, d] int32 sample of the
    workload) and return the choice with the whole table."""
    cands = candidates or grid()
    times = {c: time_build(coords, c, reps) for c in cands}
    best = pick(times)
    return {"best": dataclasses.asdict(best), "sample_points": int(coords.shape[0]),
            "table": [dict(dataclasses.asdict(c), ms=t) for c, t in sorted(times.items(), key=lambda kv: kv[1])]}
