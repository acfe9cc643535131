"""Serving loop over one resident Pkd-tree with continuous batching.

Requests arrive over time (insert a batch, delete a batch, or a k-NN query
batch).  The loop admits them in arrival order and never waits on the host
for an update:

- updates (BatchInsert, Alg. 2, or BatchDelete, Sec. 4.2) run one after
  another, in admission order, on an update thread and one CUDA stream of
  their own; before update k the update stream waits (on the device) for
  every query admitted before it;
- a k-NN batch admitted after update k runs on one of `streams` query
  streams once update k has been issued, ordered after it by an event; a
  batch that arrives while update k is still running is admitted (its
  result slot and bookkeeping made) and released as soon as update k's
  event exists, without stopping the admission of later requests;
- k-NN batches between the same two updates run concurrently (they only
  read the tree);
- a request is admitted only while the library has room for it
  (pkd_mem_info's available bytes above the request's estimated working
  set plus a reserve); otherwise the loop first lets the work in flight
  finish.

So every query sees exactly the updates admitted before it, and updates
are linearised in admission order.  Latency of a request = completion time
(a CUDA event on its stream) - arrival time.  Every step runs in the
library's kernels through the C ABI; this module only orders the calls.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
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
    admitted: float = 0.0        # host time the loop accepted the request
    epoch: int = 0               # updates admitted before this request
    n_deleted: int | None = None
    knn_ids: torch.Tensor | None = None
    knn_d2: torch.Tensor | None = None
    error: str | None = None

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
        self.update_stream = torch.cuda.Stream()
        self.reserve = reserve_bytes
        self.realtime = realtime

    def _available_bytes(self) -> int:
        return pkd.pkd_mem_info()["available"]

    def run(self, requests: list[Request]) -> list[Result]:
        reqs = sorted(requests, key=lambda r: r.arrival)
        results: list[Result] = []
        inflight: list[tuple[Result, torch.cuda.Event, int]] = []  # queries on the device
        pending: list[tuple[Result, Request]] = []                  # queries waiting for their update
        epoch_events: dict[int, list[torch.cuda.Event]] = {}        # epoch -> events of its queries
        epoch_open: dict[int, int] = {}                             # epoch -> its queries not yet launched
        deps_ready: dict[int, threading.Event] = {}                 # update k may start
        done_event: dict[int, torch.cuda.Event] = {}                # update k issued: its end event
        lock = threading.Lock()
        work: queue.Queue = queue.Queue()
        failure: list[BaseException] = []
        base = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        base.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def now() -> float:
            return time.perf_counter() - t0

        dev = torch.cuda.current_device()
        abort = threading.Event()

        def worker():
            torch.cuda.set_device(dev)
            while True:
                item = work.get()
                if item is None:
                    return
                k, r, res = item
                deps_ready[k].wait()
                if abort.is_set():
                    return
                us = self.update_stream
                with lock:
                    deps = list(epoch_events.get(k, []))
                for ev in deps:
                    us.wait_event(ev)
                try:
                    with torch.cuda.stream(us):
                        if r.kind == "insert":
                            pkd.pkd_batch_insert(self.tree._h, r.coords, r.ids, us)
                        else:
                            res.n_deleted = pkd.pkd_batch_delete(self.tree._h, r.ids, us)
                except BaseException as e:  # reported after the stream has been served
                    failure.append(e)
                    res.error = str(e)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(us)
                with lock:
                    done_event[k] = ev

        th = threading.Thread(target=worker, daemon=True)
        th.start()
        n_updates = 0

        def retire(all_: bool):
            keep = []
            for res, ev, si in inflight:
                if all_ or ev.query():
                    ev.synchronize()
                    res.done = base.elapsed_time(ev) / 1e3
                else:
                    keep.append((res, ev, si))
            inflight[:] = keep

        def close_epochs():
            # update k may start once every query admitted before it has
            # been launched (its events are then known)
            for k in range(n_updates):
                if not deps_ready[k].is_set() and all(epoch_open.get(e, 0) == 0 for e in range(k + 1)):
                    deps_ready[k].set()

        def launch(res: Result, r: Request):
            if len(inflight) >= len(self.streams):
                inflight[0][1].synchronize()  # the oldest query's stream becomes free
                retire(False)
            busy = {si for _, _, si in inflight}
            si = next(i for i in range(len(self.streams)) if i not in busy)
            st = self.streams[si]
            if res.epoch > 0:
                with lock:
                    st.wait_event(done_event[res.epoch - 1])
            with torch.cuda.stream(st):
                out_i = torch.empty((r.coords.shape[0], r.k), dtype=torch.int32, device=r.coords.device)
                out_d = torch.empty((r.coords.shape[0], r.k), dtype=torch.int64, device=r.coords.device)
                pkd.pkd_knn(self.tree._h, r.coords, r.k, out_i, out_d, st)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(st)
            res.knn_ids, res.knn_d2 = out_i, out_d
            inflight.append((res, ev, si))
            with lock:
                epoch_events.setdefault(res.epoch, []).append(ev)
            epoch_open[res.epoch] -= 1

        def release_pending():
            keep = []
            for res, r in pending:
                with lock:
                    ready = res.epoch == 0 or (res.epoch - 1) in done_event
                if ready:
                    launch(res, r)
                else:
                    keep.append((res, r))
            pending[:] = keep
            close_epochs()

        def drain():
            # every update handed to the worker and every query admitted so far
            while pending or any(not deps_ready[k].is_set() or k not in done_event for k in range(n_updates)):
                release_pending()
                retire(False)
                time.sleep(5e-5)
            retire(True)
            with lock:
                evs = list(done_event.values())
            for ev in evs:
                ev.synchronize()

        try:
            for r in reqs:
                if self.realtime:
                    wait = r.arrival - now()
                    while wait > 0:  # idle until the request arrives (queries move on meanwhile)
                        release_pending()
                        retire(False)
                        time.sleep(min(wait, 1e-4))
                        wait = r.arrival - now()
                release_pending()
                if self._available_bytes() < working_set_bytes(r, self.d) + self.reserve:
                    drain()
                res = Result(r.kind, r.size, r.arrival, admitted=now(), epoch=n_updates)
                results.append(res)
                if r.kind == "knn":
                    epoch_open[res.epoch] = epoch_open.get(res.epoch, 0) + 1
                    pending.append((res, r))
                    release_pending()
                else:
                    k = n_updates
                    n_updates += 1
                    deps_ready[k] = threading.Event()
                    work.put((k, r, res))
                    close_epochs()
            drain()
        except BaseException:
            abort.set()
            for ev in deps_ready.values():
                ev.set()
            raise
        finally:
            work.put(None)
            th.join()
        for k, res in enumerate(x for x in results if x.kind != "knn"):
            res.done = base.elapsed_time(done_event[k]) / 1e3
        if failure:
            raise failure[0]
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
