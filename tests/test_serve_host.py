"""Host logic of the serving loop, on the CPU: the library calls and CUDA
streams/events are replaced by fakes that record what the loop asks for.

Checked: updates run in arrival order, each on the update stream after a
device-side wait for the queries admitted since the previous update; every
query admitted after update k waits for update k's event; queries run on at
most `streams` streams at once and never on a busy stream; a request that
does not fit in the library's available memory first drains the work in
flight; a query that arrives while an update runs is admitted before that
update finishes (the loop does not wait for updates); results keep arrival
order."""
import contextlib
import threading
import time

import pytest
import torch

from paper_2411_09275_gb300 import serve


class World:
    """Fake device: events complete when synchronised."""

    def __init__(self, available):
        self.available = available
        self.log = []          # (op, detail), appended under self.lock
        self.lock = threading.Lock()
        self.inflight = {}     # query event -> request index
        self.current = None
        self.update_gate = None  # threading.Event an update waits for, if set
        self.update_started = threading.Event()

    def add(self, op, det):
        with self.lock:
            self.log.append((op, det))


class FakeStream:
    n = 0
    world = None

    def __init__(self):
        FakeStream.n += 1
        self.name = f"s{FakeStream.n}"

    def wait_stream(self, other):
        pass

    def wait_event(self, ev):
        FakeStream.world.add("wait", (self.name, ev.tag))


class FakeEvent:
    world = None
    n = 0

    def __init__(self, enable_timing=False):
        FakeEvent.n += 1
        self.tag = f"e{FakeEvent.n}"
        self.done = False

    def record(self, stream=None):
        self.stream = stream

    def query(self):
        return self.done

    def synchronize(self):
        w = FakeEvent.world
        with w.lock:
            if not self.done:
                self.done = True
                if self in w.inflight:
                    w.log.append(("complete", w.inflight.pop(self)))

    def elapsed_time(self, other):
        return 1.0


class FakeTree:
    class P:
        d = 2

    params = P()
    _h = object()


class FakeQuery:
    """Stands in for a device tensor of m queries tagged with the request number."""

    device = "cpu"

    def __init__(self, idx, m=4):
        self.idx, self.m = idx, m

    @property
    def shape(self):
        return (self.m, 2)

    def __getitem__(self, key):
        return self.idx


@pytest.fixture
def world(monkeypatch):
    w = World(available=8 << 30)
    FakeEvent.world = w
    FakeStream.world = w
    w.current = FakeStream()
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a, **k: w.current)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda st: contextlib.nullcontext())
    monkeypatch.setattr(serve.pkd, "pkd_mem_info", lambda: {"available": w.available})
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: real_empty(0) if k.get("device") == "cpu" else real_empty(*a, **k))

    def knn(h, coords, k, oi, od, st):
        w.add("knn", (coords.idx, st.name))

    def upd(kind, idx, st):
        w.add(kind, (idx, st.name))
        w.update_started.set()
        if w.update_gate is not None:
            assert w.update_gate.wait(5.0)

    monkeypatch.setattr(serve.pkd, "pkd_knn", knn)
    monkeypatch.setattr(serve.pkd, "pkd_batch_insert",
                        lambda h, coords, ids, st: upd("insert", int(coords[0, 0]), st))
    monkeypatch.setattr(serve.pkd, "pkd_batch_delete", lambda h, ids, st: upd("delete", int(ids[0]), st) or 0)
    # remember which request each recorded event ends
    orig_record = FakeEvent.record

    def record(self, stream=None):
        orig_record(self, stream)
        with w.lock:
            calls = [e for e in w.log if e[0] in ("knn", "insert", "delete")]
            if not calls:
                return
            op, det = calls[-1]
            if op == "knn" and det[0] not in w.inflight.values() and det[0] not in w.recorded:
                w.inflight[self] = det[0]
                w.recorded.add(det[0])
            elif op in ("insert", "delete") and det[0] not in w.update_events:
                w.update_events[det[0]] = self.tag

    w.recorded = set()
    w.update_events = {}
    monkeypatch.setattr(FakeEvent, "record", record)
    return w


def _req(kind, idx, m=4, k=3):
    if kind == "knn":
        return serve.Request(kind, 0.001 * idx, FakeQuery(idx, m), None, k)
    if kind == "insert":
        return serve.Request(kind, 0.001 * idx, torch.full((m, 2), idx, dtype=torch.int32),
                             torch.arange(m, dtype=torch.int32), k)
    return serve.Request(kind, 0.001 * idx, None, torch.full((m,), idx, dtype=torch.int32), k)


def test_updates_ordered_after_earlier_queries_and_before_later_ones(world):
    kinds = ["knn", "knn", "insert", "knn", "delete", "knn", "knn", "knn", "insert", "knn"]
    reqs = [_req(kd, i) for i, kd in enumerate(kinds)]
    out = serve.Server(FakeTree(), streams=2, realtime=False).run(reqs)
    assert [r.kind for r in out] == kinds
    assert [r.epoch for r in out] == [0, 0, 0, 1, 1, 2, 2, 2, 2, 3]
    log = world.log
    updates = [d[0] for o, d in log if o in ("insert", "delete")]
    assert updates == [2, 4, 8]  # arrival order
    upd_stream = next(d[1] for o, d in log if o == "insert")
    # before each update, its stream waits for as many query events as
    # queries were admitted since the previous update
    for k, u in enumerate(updates):
        pos_u = next(pos for pos, (o, d) in enumerate(log) if o in ("insert", "delete") and d[0] == u)
        prev_pos = (next(pos for pos, (o, d) in enumerate(log) if o in ("insert", "delete") and d[0] == updates[k - 1])
                    if k else -1)
        prev = updates[k - 1] if k else -1
        mine = [i for i, kd in enumerate(kinds) if kd == "knn" and prev < i < u]
        waits = [d for pos, (o, d) in enumerate(log) if prev_pos < pos < pos_u and o == "wait" and d[0] == upd_stream]
        assert len(waits) == len(mine), (u, waits, mine)
    # every query after an update waits for that update's end event before it runs
    for i, kd in enumerate(kinds):
        before = [u for u in updates if u < i]
        if kd != "knn" or not before:
            continue
        pos_q = next(pos for pos, (o, d) in enumerate(log) if o == "knn" and d[0] == i)
        assert any(o == "wait" and d[1] == world.update_events[before[-1]] for o, d in log[:pos_q]), i
    # every query completes exactly once
    assert sorted(d for o, d in log if o == "complete") == [i for i, kd in enumerate(kinds) if kd == "knn"]


def test_queries_are_admitted_while_an_update_runs(world):
    # the update blocks until the test releases it: the loop must admit the
    # queries that arrive meanwhile (not wait for the update), and launch
    # them only once the update has been issued
    world.update_gate = threading.Event()
    kinds = ["knn", "insert", "knn", "knn", "knn"]
    reqs = [_req(kd, i) for i, kd in enumerate(kinds)]
    box = {}

    def run():
        box["out"] = serve.Server(FakeTree(), streams=4, realtime=False).run(reqs)

    th = threading.Thread(target=run)
    th.start()
    assert world.update_started.wait(5.0)
    time.sleep(0.2)  # the loop keeps going while the update is held
    with world.lock:
        launched = [d[0] for o, d in world.log if o == "knn"]
    assert launched == [0]  # the later queries wait for the update
    held = time.perf_counter()
    world.update_gate.set()
    th.join(10.0)
    out = box["out"]
    assert [r.kind for r in out] == kinds
    # all three were admitted before the update was let go
    assert max(r.admitted for r in out) < out[1].admitted + (time.perf_counter() - held) + 0.2
    assert all(r.epoch == 1 for r in out[2:])
    with world.lock:
        launched = [d[0] for o, d in world.log if o == "knn"]
    assert launched == [0, 2, 3, 4]


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
            busy.pop(det)
    assert not busy


def test_admission_waits_for_memory(world):
    # available memory below any request's need plus the reserve: every
    # admission first drains the work in flight, so at most one query is
    # ever in flight
    world.available = 1 << 20
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
