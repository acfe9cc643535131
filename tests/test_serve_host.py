"""Host logic of the serving loop, on the CPU: the library calls and CUDA
streams/events are replaced by fakes that record what the loop asks for.

Checked: updates run in arrival order and only after every query admitted
before them has completed; queries run on at most `streams` streams at once
and never on a busy stream; a request that does not fit in free device
memory first drains the queries in flight; results keep arrival order."""
import contextlib

import pytest
import torch

from paper_2411_09275_gb300 import serve


class FakeStream:
    n = 0

    def __init__(self):
        FakeStream.n += 1
        self.name = f"s{FakeStream.n}"

    def wait_stream(self, other):
        pass


class World:
    """Fake device: events complete when synchronised (or when the test says)."""

    def __init__(self, free_bytes):
        self.free = free_bytes
        self.log = []          # (op, detail)
        self.inflight = {}     # event -> (request index, stream name)
        self.current = FakeStream()


class FakeEvent:
    world = None

    def __init__(self, enable_timing=False):
        self.done = False
        self.stream = None

    def record(self, stream=None):
        self.stream = stream

    def query(self):
        return self.done

    def synchronize(self):
        if not self.done:
            self.done = True
            w = FakeEvent.world
            if self in w.inflight:
                w.log.append(("complete", w.inflight.pop(self)))

    def elapsed_time(self, other):
        return 1.0


class FakeTree:
    class P:
        d = 2

    params = P()
    _h = object()


@pytest.fixture
def world(monkeypatch):
    w = World(free_bytes=8 << 30)
    FakeEvent.world = w
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: w.current)
    monkeypatch.setattr(torch.cuda, "stream", lambda st: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a, **k: (w.free, 1 << 40))

    def knn(h, coords, k, oi, od, st):
        w.log.append(("knn", (int(coords[0, 0]), st.name)))

    def ins(h, coords, ids, st):
        w.log.append(("insert", int(coords[0, 0])))

    def dele(h, ids, st):
        w.log.append(("delete", int(ids[0])))
        return int(ids.numel())

    monkeypatch.setattr(serve.pkd, "pkd_knn", knn)
    monkeypatch.setattr(serve.pkd, "pkd_batch_insert", ins)
    monkeypatch.setattr(serve.pkd, "pkd_batch_delete", dele)
    # a query's event is in flight until synchronised; remember which request it ends
    orig_record = FakeEvent.record

    def record(self, stream=None):
        orig_record(self, stream)
        calls = [e for e in w.log if e[0] in ("knn", "insert", "delete")]
        if calls and calls[-1][0] == "knn" and calls[-1][1] not in w.inflight.values():
            w.inflight[self] = calls[-1][1]

    monkeypatch.setattr(FakeEvent, "record", record)
    return w


def _req(kind, idx, m=4, k=3):
    c = torch.full((m, 2), idx, dtype=torch.int32) if kind != "delete" else None
    ids = None
    if kind == "insert":
        ids = torch.arange(m, dtype=torch.int32)
    elif kind == "delete":
        ids = torch.full((m,), idx, dtype=torch.int32)  # the log reads the request number from ids[0]
    return serve.Request(kind, 0.001 * idx, c, ids, k)


def test_updates_linearised_after_earlier_queries(world):
    kinds = ["knn", "knn", "insert", "knn", "delete", "knn", "knn", "knn", "insert"]
    reqs = [_req(kd, i) for i, kd in enumerate(kinds)]
    out = serve.Server(FakeTree(), streams=2, realtime=False).run(reqs)
    assert [r.kind for r in out] == kinds
    log = world.log
    # every update runs after the completion of every query that arrived before it
    for pos, (op, det) in enumerate(log):
        if op in ("insert", "delete"):
            earlier_q = [i for i, kd in enumerate(kinds) if kd == "knn" and i < det]
            done = {d[0] for o, d in log[:pos] if o == "complete"}
            assert set(earlier_q) <= done, (op, det)
    # updates in arrival order
    assert [d for o, d in log if o in ("insert", "delete")] == [2, 4, 8]
    # every query completes exactly once
    assert sorted(d[0] for o, d in log if o == "complete") == [i for i, kd in enumerate(kinds) if kd == "knn"]


def test_at_most_streams_queries_in_flight_on_distinct_streams(world):
    reqs = [_req("knn", i) for i in range(9)]
    serve.Server(FakeTree(), streams=3, realtime=False).run(reqs)
    busy = {}
    for op, det in world.log:
        if op == "knn":
            idx, st = det
            assert st not in busy.values(), "a query went to a busy stream"
            busy[idx] = st
            assert len(busy) <= 3
        elif op == "complete":
            busy.pop(det[0])
    assert not busy


def test_admission_waits_for_memory(world):
    # free memory below any request's need plus the reserve: every admission
    # first drains the queries in flight, so at most one is ever in flight
    world.free = 1 << 20
    reqs = [_req("knn", i) for i in range(5)]
    serve.Server(FakeTree(), streams=4, realtime=False, reserve_bytes=1 << 30).run(reqs)
    inflight = 0
    for op, det in world.log:
        if op == "knn":
            inflight += 1
            assert inflight == 1
        elif op == "complete":
            inflight -= 1


def test_summary_counts_and_rates():
    rs = [serve.Result("knn", 100, 0.0, 0.002), serve.Result("insert", 1000, 0.001, 0.004),
          serve.Result("delete", 50, 0.002, 0.003)]
    s = serve.summarize(rs, 0.01)
    assert s["all"]["count"] == 3
    assert s["knn"]["count"] == 1 and s["insert"]["count"] == 1 and s["delete"]["count"] == 1
    assert s["mpts_per_s"] == pytest.approx(1150 / 0.01 / 1e6)
    assert s["insert"]["p50_ms"] == pytest.approx(3.0)
