"""GPU tests of the serving loop: a resident tree under a mixed stream of
inserts, deletes and k-NN batches.  Every query's answer equals the oracle's
on the tree state made by the updates admitted before it (a replay of the
same linearised sequence), and the answers are the same whether the queries
run one at a time or overlapped on several streams."""
import numpy as np
import pytest

import oracle as O
from paper_2411_09275_gb300 import inputs as I
from tests.gpuutil import ids_dev, make_points, oparams, to_dev

pytestmark = pytest.mark.gpu


def _mods():
    from paper_2411_09275_gb300 import pkd, serve

    return pkd, serve


def _workload(n, d, count, seed):
    """A request list (arrival order) plus the host data to replay it."""
    rng = np.random.default_rng(seed)
    X = make_points("uniform", n, d, seed)
    live = list(range(n))
    nxt = n
    reqs = []
    t = 0.0
    for q in range(count):
        t += rng.exponential(1e-3)
        kind = rng.choice(["insert", "delete", "knn"], p=[0.4, 0.2, 0.4])
        if kind == "insert":
            m = int(rng.integers(50, 1500))
            Y = I.uniform(m, d, seed * 100 + q)
            ids = np.arange(nxt, nxt + m, dtype=np.uint32)
            live.extend(range(nxt, nxt + m))
            nxt += m
            reqs.append(("insert", t, Y, ids, 0))
        elif kind == "delete":
            m = int(rng.integers(20, 800))
            sel = rng.choice(len(live), size=min(m, len(live)), replace=False)
            ids = np.array([live[i] for i in sel], np.uint32)
            keep = np.ones(len(live), bool)
            keep[sel] = False
            live = [v for v, kp in zip(live, keep) if kp]
            reqs.append(("delete", t, None, ids, 0))
        else:
            m = int(rng.integers(10, 400))
            Q = I.uniform(m, d, seed * 1000 + q)
            reqs.append(("knn", t, Q, None, int(rng.choice([1, 5, 10]))))
    return X, reqs


def _run(pkd, serve, X, reqs, streams, realtime=False):
    d = X.shape[1]
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)
    tree = pkd.Tree(to_dev(X), None, p)
    R = [serve.Request(kind, t, to_dev(C) if C is not None else None, ids_dev(ids) if ids is not None else None, k)
         for kind, t, C, ids, k in reqs]
    out = serve.Server(tree, streams=streams, realtime=realtime).run(R)
    tree.close()
    return p, out


def test_serving_results_equal_oracle_replay():
    pkd, serve = _mods()
    X, reqs = _workload(20000, 3, 40, 5)
    p, out = _run(pkd, serve, X, reqs, streams=4)
    o = O.OracleTree(X, None, oparams(p))
    for (kind, _, C, ids, k), res in zip(reqs, out):
        assert res.kind == kind
        if kind == "insert":
            o.insert(C, ids)
        elif kind == "delete":
            assert res.n_deleted == o.delete(ids) == len(ids)
        else:
            wi, wd = o.knn(C, k)
            assert np.array_equal(res.knn_d2.cpu().numpy(), wd)
            assert np.array_equal(res.knn_ids.cpu().numpy().view(np.uint32), wi)
    o.close()


def test_queries_alone_and_overlapped_agree():
    pkd, serve = _mods()
    X, reqs = _workload(15000, 2, 30, 9)
    _, alone = _run(pkd, serve, X, reqs, streams=1)
    _, mixed = _run(pkd, serve, X, reqs, streams=4)
    for a, b in zip(alone, mixed):
        assert a.kind == b.kind
        if a.kind == "knn":
            assert np.array_equal(a.knn_ids.cpu().numpy(), b.knn_ids.cpu().numpy())
            assert np.array_equal(a.knn_d2.cpu().numpy(), b.knn_d2.cpu().numpy())
        if a.kind == "delete":
            assert a.n_deleted == b.n_deleted


def test_summary_has_percentiles():
    _, serve = _mods()
    X, reqs = _workload(8000, 3, 20, 13)
    from paper_2411_09275_gb300 import pkd

    _, out = _run(pkd, serve, X, reqs, streams=2, realtime=True)
    s = serve.summarize(out, 1.0)
    assert s["all"]["count"] == 20 and s["all"]["p99_ms"] >= s["all"]["p50_ms"] >= 0


def test_queries_admitted_during_an_update_see_exactly_the_earlier_updates():
    # a large insert, then k-NN batches that arrive while it runs, then a
    # delete and more queries: the batches are admitted before the insert
    # finishes (the loop does not wait for updates) and each answer equals
    # the oracle's on the updates admitted before it
    pkd, serve = _mods()
    d, n = 3, 400000
    X = make_points("uniform", n, d, 21)
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)
    Y = I.uniform(300000, d, 22)
    yid = np.arange(n, n + 300000, dtype=np.uint32)
    kill = np.arange(0, n, 5, dtype=np.uint32)
    plan = [("insert", 0.0, Y, yid, 0)]
    plan += [("knn", 1e-4 * (q + 1), I.uniform(500, d, 30 + q), None, 10) for q in range(6)]
    plan += [("delete", 2e-3, None, kill, 0)]
    plan += [("knn", 2e-3 + 1e-4 * (q + 1), I.uniform(500, d, 40 + q), None, 5) for q in range(4)]
    tree = pkd.Tree(to_dev(X), None, p)
    R = [serve.Request(kind, t, to_dev(C) if C is not None else None, ids_dev(ids) if ids is not None else None, k)
         for kind, t, C, ids, k in plan]
    out = serve.Server(tree, streams=4, realtime=True).run(R)
    tree.close()
    ins = out[0]
    during = [r for r in out[1:7] if r.admitted < ins.done]
    assert during, "no query was admitted while the insert ran"
    o = O.OracleTree(X, None, oparams(p))
    for (kind, _, C, ids, k), res in zip(plan, out):
        if kind == "insert":
            o.insert(C, ids)
        elif kind == "delete":
            assert res.n_deleted == o.delete(ids) == len(ids)
        else:
            wi, wd = o.knn(C, k)
            assert np.array_equal(res.knn_d2.cpu().numpy(), wd)
            assert np.array_equal(res.knn_ids.cpu().numpy().view(np.uint32), wi)
    o.close()
