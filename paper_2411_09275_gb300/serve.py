"""Serving loop over one resident Pkd-tree with continuous batching.

Requests arrive over time (insert a batch, delete a batch, or a k-NN query
batch).  The loop admits them in arrival order:

- k-NN batches between two updates run concurrently, each on its own CUDA
  stream (up to `streams` in flight); they only read the tree;
- an update (BatchInsert, Alg. 2, or BatchDelete, Sec. 4.2) waits for every
  query admitted before it, then runs alone, so updates are linearised in
  admission order and every query sees exactly the updates admitted before
  it;
- a request is admitted only while the device has room for it (free HBM
  above the request's estimated working set plus a reserve); otherwise the
  loop first drains the queries in flight.

Latency of a request = completion time - arrival time (query completions
are timed by CUDA events on their streams).  Every step runs in the
library's kernels through the C ABI; this module only orders the calls.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import pkd


@dataclasses.dataclass
class Request:
    kind: str                    # "insert", "delete" or "knn"
    arrival: float               # seconds after the start of the stream
    coords: torch.Tensor | None  # device [m, d] int32: points (insert) or queries (knn); None for deletes
    ids: torch.Tensor | None = None  # device [m] int32 view of uint32 ids (updates)
    k: int = 10                  # knn

    @property
    def size(self) -> int:
        return int(self.ids.numel()) if self.kind == "delete" else int(self.coords.shape[0])


@dataclasses.dataclass
class Result:
    kind: str
    size: int
    arrival: float
    done: float = 0.0
    n_deleted: int | None = None
    knn_ids: torch.Tensor | None = None
    knn_d2: torch.Tensor | None = None

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.done - self.arrival)


def working_set_bytes(r: Request, d: int) -> int:
    """Device bytes a request may need beyond the tree (routing buffers and
    rebuild scratch for updates, outputs for queries); an estimate."""
    m = r.size
    if r.kind == "knn":
        return m * r.k * 12 + m * 4 * d
    return m * (4 * d + 4) * 24


class Server:
    def __init__(self, tree: pkd.Tree, streams: int = 4, reserve_bytes: int = 1 << 30, realtime: bool = True):
        self.tree = tree
        self.d = tree.params.d
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.reserve = reserve_bytes
        self.realtime = realtime

    def _free_bytes(self) -> int:
        return torch.cuda.mem_get_info()[0]

    def run(self, requests: list[Request]) -> list[Result]:
        reqs = sorted(requests, key=lambda r: r.arrival)
        results: list[Result] = []
        inflight: list[tuple[Result, torch.cuda.Event, int]] = []  # (result, done event, stream)
        base = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        base.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = 0

        def now() -> float:
            return time.perf_counter() - t0

        def retire(all_: bool):
            keep = []
            for res, ev, si in inflight:
                if all_ or ev.query():
                    ev.synchronize()
                    res.done = base.elapsed_time(ev) / 1e3
                else:
                    keep.append((res, ev, si))
            inflight[:] = keep

        for r in reqs:
            if self.realtime:
                wait = r.arrival - now()
                while wait > 0:  # idle until the request arrives (retiring queries meanwhile)
                    retire(False)
                    time.sleep(min(wait, 1e-4))
                    wait = r.arrival - now()
            need = working_set_bytes(r, self.d)
            if self._free_bytes() < need + self.reserve:
                retire(True)
            res = Result(r.kind, r.size, r.arrival)
            results.append(res)
            if r.kind == "knn":
                retire(False)
                if len(inflight) >= len(self.streams):
                    # the oldest query's stream becomes free
                    oldest = inflight[0]
                    oldest[1].synchronize()
                    retire(False)
                busy = {si for _, _, si in inflight}
                si = next(i for i in range(len(self.streams)) if i not in busy)
                st = self.streams[si]
                st.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(st):
                    out_i = torch.empty((r.coords.shape[0], r.k), dtype=torch.int32, device=r.coords.device)
                    out_d = torch.empty((r.coords.shape[0], r.k), dtype=torch.int64, device=r.coords.device)
                    pkd.pkd_knn(self.tree._h, r.coords, r.k, out_i, out_d, st)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(st)
                res.knn_ids, res.knn_d2 = out_i, out_d
                inflight.append((res, ev, si))
            else:
                retire(True)  # linearise: every earlier query has finished
                s = torch.cuda.current_stream()
                if r.kind == "insert":
                    pkd.pkd_batch_insert(self.tree._h, r.coords, r.ids, s)
                else:
                    res.n_deleted = pkd.pkd_batch_delete(self.tree._h, r.ids, s)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(s)
                ev.synchronize()
                res.done = base.elapsed_time(ev) / 1e3
        retire(True)
        return results


def summarize(results: list[Result], wall_s: float) -> dict:
    """p50 / p99 latency per request kind and overall, and Mpts/s (points
    inserted + deleted + queries answered, over the wall time)."""
    out = {}
    lat_all = np.array([r.latency_ms for r in results])
    for kind in ("insert", "delete", "knn"):
        lat = np.array([r.latency_ms for r in results if r.kind == kind])
        if lat.size:
            out[kind] = {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99))}
    pts = sum(r.size for r in results)
    out["all"] = {"count": int(lat_all.size), "p50_ms": float(np.percentile(lat_all, 50)),
                  "p99_ms": float(np.percentile(lat_all, 99))}
    out["mpts_per_s"] = pts / wall_s / 1e6
    return out
