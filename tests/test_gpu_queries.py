"""GPU parity of the queries (Sec. 5): k-NN returns exactly the k smallest
(squared distance, id) pairs, range count the exact number of points in each
closed box; both checked against the oracle (itself pinned to brute force)."""
import numpy as np
import pytest

import oracle as O
from paper_2411_09275_gb300 import inputs as I
from tests import treeutil as U
from tests.gpuutil import ids_dev, knobs, make_points, oparams, to_dev

pytestmark = pytest.mark.gpu


def _pkd():
    from paper_2411_09275_gb300 import pkd

    return pkd


@pytest.mark.parametrize("d,kind", [(1, "uniform"), (2, "uniform"), (3, "varden"), (5, "dups"), (8, "uniform")])
@pytest.mark.parametrize("k", [1, 10, 33, 128])
def test_knn_matches_oracle(d, kind, k):
    pkd = _pkd()
    n = 30000
    X = make_points(kind, n, d, 61 + d)
    ids = np.arange(n, dtype=np.uint32)[::-1].copy()
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=2, sigma_os=4)
    with knobs(base_cap=1024):
        t = pkd.Tree(to_dev(X), ids_dev(ids), p)
    o = O.OracleTree(X, ids, oparams(p))
    Q = np.concatenate([I.uniform(500, d, 62), X[:300]])
    gi, gd = t.knn(to_dev(Q), k)
    wi, wd = o.knn(Q, k)
    assert np.array_equal(gd.cpu().numpy(), wd)
    assert np.array_equal(gi.cpu().numpy().view(np.uint32), wi)


def test_knn_pads_and_tie_case():
    pkd = _pkd()
    X = np.array([[3, 4], [5, 0], [100, 0]], np.int32)
    ids = np.array([50, 1, 3], np.uint32)
    t = pkd.Tree(to_dev(X), ids_dev(ids), pkd.Params(d=2, phi=1, lam=1, sigma_log2=0, sigma_os=1))
    gi, gd = t.knn(to_dev(np.array([[0, 0]], np.int32)), 5)
    assert list(gi.cpu().numpy().view(np.uint32)[0]) == [1, 50, 3, 0xFFFFFFFF, 0xFFFFFFFF]
    assert list(gd.cpu().numpy()[0][:3]) == [25, 25, 10000]
    assert gd.cpu().numpy()[0][3] == np.iinfo(np.int64).max


@pytest.mark.parametrize("d", [1, 2, 3, 6])
def test_range_count_matches_oracle(d):
    pkd = _pkd()
    n = 50000
    X = make_points("varden" if d == 3 else "uniform", n, d, 71)
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)
    t = pkd.Tree(to_dev(X), None, p)
    o = O.OracleTree(X, None, oparams(p))
    for side in (1 << 12, 1 << 24, 1 << 29, 1 << 30):
        lo, hi = I.boxes(400, d, side, 72 + side % 97)
        got = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.uint64)
        assert np.array_equal(got, o.range_count(lo, hi))


def test_queries_after_updates_and_config1_knn():
    # 1e6 uniform 2-D points, k-NN k=10 for 1e4 uniform queries
    pkd = _pkd()
    X = I.uniform(1_000_000, 2, 1)
    p = pkd.Params(d=2)
    t = pkd.Tree(to_dev(X), None, p)
    o = O.OracleTree(X, None, oparams(p))
    Q = I.uniform(10_000, 2, 2)
    gi, gd = t.knn(to_dev(Q), 10)
    wi, wd = o.knn(Q, 10)
    assert np.array_equal(gd.cpu().numpy(), wd) and np.array_equal(gi.cpu().numpy().view(np.uint32), wi)
    # after a batch of inserts and deletes
    Y = I.uniform(100_000, 2, 3)
    yid = np.arange(1_000_000, 1_100_000, dtype=np.uint32)
    t.insert(to_dev(Y), ids_dev(yid))
    o.insert(Y, yid)
    sel = I.sample_indices(50_000, 1_000_000, 4)
    assert t.delete(ids_dev(sel)) == o.delete(sel) == 50_000
    gi, gd = t.knn(to_dev(Q[:2000]), 10)
    wi, wd = o.knn(Q[:2000], 10)
    assert np.array_equal(gd.cpu().numpy(), wd) and np.array_equal(gi.cpu().numpy().view(np.uint32), wi)
    lo, hi = I.boxes(2000, 2, 1 << 26, 5)
    got = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, o.range_count(lo, hi))


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_range_report_matches_brute_force(d):
    pkd = _pkd()
    n = 40000
    X = make_points("varden" if d == 3 else "uniform", n, d, 91)
    ids = ((np.arange(n, dtype=np.uint64) * 2246822519) % (1 << 32)).astype(np.uint32)
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)
    t = pkd.Tree(to_dev(X), ids_dev(ids), p)
    for side in (1 << 10, 1 << 22, 1 << 30):
        lo, hi = I.boxes(300, d, side, 92 + side % 89)
        off, got = pkd.pkd_range_report(t._h, to_dev(lo), to_dev(hi))
        off = off.cpu().numpy().astype(np.int64)
        got = got.cpu().numpy().view(np.uint32)
        cnt = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.int64)
        assert np.array_equal(np.diff(off), cnt) and off[0] == 0 and off[-1] == got.size
        want = O.range_report(X, ids, lo, hi)
        for i in range(len(lo)):
            assert np.array_equal(np.sort(got[off[i]:off[i + 1]]), want[i])
    t.close()


def test_range_report_after_updates():
    pkd = _pkd()
    d, n = 2, 20000
    X = make_points("uniform", n, d, 93)
    t = pkd.Tree(to_dev(X), None, pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4))
    Y = I.uniform(5000, d, 94)
    yid = np.arange(n, n + 5000, dtype=np.uint32)
    t.insert(to_dev(Y), ids_dev(yid))
    kill = np.arange(0, n, 3)
    t.delete(ids_dev(kill.astype(np.uint32)))
    o = O.OracleTree(X, None, O.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4))
    o.insert(Y, yid)
    o.delete(kill.astype(np.uint32))
    lo, hi = I.boxes(200, d, 1 << 27, 95)
    off, got = pkd.pkd_range_report(t._h, to_dev(lo), to_dev(hi))
    off = off.cpu().numpy().astype(np.int64)
    got = got.cpu().numpy().view(np.uint32)
    want = o.range_report(lo, hi)
    for i in range(len(lo)):
        assert np.array_equal(np.sort(got[off[i]:off[i + 1]]), want[i])
    o.close()
    t.close()


def test_queries_on_a_tree_deeper_than_the_local_stack():
    """alpha = 1/2 never rebuilds an interior node, so batches that always
    land right of every stored point grow one path by two levels per batch
    (the rightmost leaf plus the batch is rebuilt below it).  Past height
    126 the searches keep their stacks in global scratch, a chunk of queries
    at a time; every answer still equals the oracle's, with and without
    stored boxes."""
    import torch

    pkd = _pkd()
    d = 1
    p = pkd.Params(d=d, phi=2, lam=2, sigma_log2=0, sigma_os=1, alpha_num=1, alpha_den=2)
    X = (np.arange(8, dtype=np.int32) * 7).reshape(8, 1)
    ids = np.arange(8, dtype=np.uint32)
    t = pkd.Tree(to_dev(X), ids_dev(ids), p)
    o = O.OracleTree(X, ids, oparams(p))
    nxt, top = 8, 100
    for r in range(80):
        Y = (top + np.array([3, 1, 2], dtype=np.int32)).reshape(3, 1)
        yid = np.arange(nxt, nxt + 3, dtype=np.uint32)
        t.insert(to_dev(Y), ids_dev(yid))
        o.insert(Y, yid)
        nxt += 3
        top += 10
    assert t.height > 130
    pts = o.points()[1]
    Q = np.concatenate([I.uniform(200, d, 71) % (top + 50), pts[::7]]).astype(np.int32)
    lo, hi = I.boxes(100, d, 300, 72)
    lo, hi = lo % top, hi % top
    hi = np.maximum(lo, hi)
    for boxes in (False, True):
        pkd.pkd_set_bounding_boxes(t._h, boxes)
        for k in (1, 5, 40):
            gi, gd = t.knn(to_dev(Q), k)
            wi, wd = o.knn(Q, k)
            assert np.array_equal(gd.cpu().numpy(), wd) and np.array_equal(gi.cpu().numpy().view(np.uint32), wi)
        cnt = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.uint64)
        assert np.array_equal(cnt, o.range_count(lo, hi))
        off, got = pkd.pkd_range_report(t._h, to_dev(lo), to_dev(hi))
        off = off.cpu().numpy().astype(np.int64)
        got = got.cpu().numpy().view(np.uint32)
        want = o.range_report(lo, hi)
        for i in range(len(lo)):
            assert np.array_equal(np.sort(got[off[i]:off[i + 1]]), want[i])
    # the no-allocation search has no scratch for a deep tree: it refuses
    out = torch.empty((len(Q), 5), dtype=torch.int32, device="cuda")
    with pytest.raises(Exception):
        pkd.pkd_knn_ids_noalloc(t._h, to_dev(Q), 5, out)
    t.close()
