"""GPU tests of the stored-bounding-box variant (Pkd-bb, Sec. 6 of the
paper): every node's stored box is the tight box of the points below it
(checked node by node against the exported leaves), it stays so after batch
updates, and k-NN, range count and range report give exactly the oracle's
answers with the boxes on, as they do with them off."""
import numpy as np
import pytest

import oracle as O
from paper_2411_09275_gb300 import inputs as I
from tests.gpuutil import ids_dev, make_points, oparams, to_dev

pytestmark = pytest.mark.gpu

INT_MAX, INT_MIN = 2**31 - 1, -2**31


def _pkd():
    from paper_2411_09275_gb300 import pkd

    return pkd


def _node_leaf_ranges(dims):
    """For every pre-order node, the range [first, last) of leaf numbers in
    its subtree (leaves are numbered in pre-order = in-order)."""
    n = len(dims)
    first = np.zeros(n, np.int64)
    last = np.zeros(n, np.int64)
    leaf_no = np.cumsum(dims == 0xFF) - (dims == 0xFF)
    end = np.zeros(n, np.int64)
    kids = {}
    stack = []
    for i in range(n):
        if stack:
            p = stack[-1]
            kids.setdefault(p, []).append(i)
            if len(kids[p]) == 2:
                stack.pop()
        if dims[i] != 0xFF:
            stack.append(i)
    for i in range(n - 1, -1, -1):
        if dims[i] == 0xFF:
            first[i], last[i] = leaf_no[i], leaf_no[i] + 1
        else:
            a, b = kids[i]
            first[i], last[i] = first[a], last[b]
    return first, last


def _check_boxes(t, xyz, d):
    pkd = _pkd()
    ex = t.export()
    lo, hi = pkd.pkd_export_boxes(t._h, len(ex["dims"]), d)
    first, last = _node_leaf_ranges(ex["dims"])
    offs = ex["leaf_offsets"].astype(np.int64)
    ids = ex["leaf_ids"]
    for v in range(len(ex["dims"])):
        pid = ids[offs[first[v]]:offs[last[v]]]
        if len(pid) == 0:
            assert (lo[v] == INT_MAX).all() and (hi[v] == INT_MIN).all(), v
            continue
        P = np.array([xyz[int(i)] for i in pid], np.int64).reshape(-1, d)
        assert np.array_equal(lo[v], P.min(axis=0)) and np.array_equal(hi[v], P.max(axis=0)), v


def _check_queries(t, o, d, seed):
    pkd = _pkd()
    Q = np.concatenate([I.uniform(300, d, seed), o.points()[1][:200]])
    for k in (1, 10, 33):
        gi, gd = t.knn(to_dev(Q), k)
        wi, wd = o.knn(Q, k)
        assert np.array_equal(gd.cpu().numpy(), wd) and np.array_equal(gi.cpu().numpy().view(np.uint32), wi)
    for side in (1 << 12, 1 << 24, 1 << 30):
        lo, hi = I.boxes(150, d, side, seed + side % 97)
        cnt = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.uint64)
        assert np.array_equal(cnt, o.range_count(lo, hi))
        off, got = pkd.pkd_range_report(t._h, to_dev(lo), to_dev(hi))
        off = off.cpu().numpy().astype(np.int64)
        got = got.cpu().numpy().view(np.uint32)
        want = o.range_report(lo, hi)
        for i in range(len(lo)):
            assert np.array_equal(np.sort(got[off[i]:off[i + 1]]), want[i])


@pytest.mark.parametrize("d,kind", [(1, "uniform"), (2, "varden"), (3, "uniform"), (3, "dups"), (5, "varden")])
def test_boxes_tight_and_queries_exact_through_updates(d, kind):
    pkd = _pkd()
    n = 30000
    X = make_points(kind, n, d, 201 + d)
    ids = np.arange(n, dtype=np.uint32) * 3 + 1
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8, alpha_num=1, alpha_den=2)
    t = pkd.Tree(to_dev(X), ids_dev(ids), p)
    o = O.OracleTree(X, ids, oparams(p))
    xyz = {int(i): tuple(x) for i, x in zip(ids, X.tolist())}
    _check_queries(t, o, d, 210)                # boxes off (the Pkd form)
    pkd.pkd_set_bounding_boxes(t._h, True)
    _check_boxes(t, xyz, d)
    _check_queries(t, o, d, 211)
    rng = np.random.default_rng(d)
    nxt = 3 * n + 10
    for r in range(3):
        Y = make_points(kind, 4000, d, 220 + r)
        yid = np.arange(nxt, nxt + 4000, dtype=np.uint32)
        nxt += 4000
        t.insert(to_dev(Y), ids_dev(yid))
        o.insert(Y, yid)
        xyz.update({int(i): tuple(x) for i, x in zip(yid, Y.tolist())})
        live = np.array(sorted(xyz), dtype=np.uint32)
        # skewed delete: the lowest first coordinates, so that whole subtrees
        # empty out (alpha = 1/2 keeps empty children)
        kill = live[np.argsort([xyz[int(i)][0] for i in live])[:5000]]
        kill = np.concatenate([kill, rng.choice(live, 500, replace=False)])
        assert t.delete(ids_dev(kill)) == o.delete(kill)
        for i in kill:
            xyz.pop(int(i), None)
        _check_boxes(t, xyz, d)
        _check_queries(t, o, d, 230 + r)
    pkd.pkd_set_bounding_boxes(t._h, False)
    _check_queries(t, o, d, 240)
    t.close()


def test_boxes_on_empty_and_tiny_trees():
    pkd = _pkd()
    d = 2
    p = pkd.Params(d=d, phi=4)
    t = pkd.Tree(to_dev(np.zeros((0, d), np.int32)), None, p)
    pkd.pkd_set_bounding_boxes(t._h, True)
    _check_boxes(t, {}, d)
    Y = I.uniform(50, d, 250)
    t.insert(to_dev(Y), ids_dev(np.arange(50, dtype=np.uint32)))
    _check_boxes(t, {i: tuple(x) for i, x in enumerate(Y.tolist())}, d)
    assert t.delete(ids_dev(np.arange(50, dtype=np.uint32))) == 50
    _check_boxes(t, {}, d)
    t.close()
