"""The benchmark's own workload at full size, in the launch configuration
bench.py times (default parameters, the same input generators and seeds):
build 1e8 3-D points, insert 1e7 new points, delete 1e7 random existing ids,
on uniform and on varden-like inputs.

- Exact parity with the oracle: the SHA-256 of the GPU tree's canonical
  export after the delete, and of its 10-NN answer for 1e4 queries, equal the
  values that tests/golden/make_fullsize_golden.py computed from the CPU
  oracle alone on the same inputs (tests/golden/fullsize_*.txt).
- Properties that hold at any size, checked independently of the oracle:
  the exported tree holds every live id exactly once, each leaf at most phi
  points unless all its points are identical, every internal node's size
  equals the sum of its children's; every point of every sampled leaf lies
  inside the leaf's subspace (the box cut by the splitters above it, left =
  strictly below); k-NN for sampled queries and range counts for sampled
  boxes equal brute force over all live points (numpy, one query at a time).
"""
import numpy as np
import pytest

import bench
from paper_2411_09275_gb300 import inputs as I
from tests.golden import make_fullsize_golden as G
from tests.gpuutil import ids_dev, to_dev

pytestmark = pytest.mark.gpu


def _leaf_boxes(ex, d, want_leaves):
    """Subspace box of every leaf in want_leaves (leaf numbers in leaf
    order), from the pre-order export: node i's left child is i + 1 and its
    right child follows the left subtree."""
    dims = ex["dims"].tolist()
    splits = ex["splits"].tolist()
    n_nodes = len(dims)
    # subtree node counts, from the last node backwards
    cnt = [0] * n_nodes
    stack = []
    for i in range(n_nodes - 1, -1, -1):
        if dims[i] == 0xFF:
            cnt[i] = 1
        else:
            left = stack.pop()
            right = stack.pop()
            cnt[i] = 1 + left + right
        stack.append(cnt[i])
    # an internal node's size is the sum of its children's
    sizes = ex["sizes"].tolist()
    for i in range(n_nodes):
        if dims[i] != 0xFF:
            assert sizes[i] == sizes[i + 1] + sizes[i + 1 + cnt[i + 1]], i
    boxes = {}
    leaf = 0
    todo = [(0, [0] * d, [(1 << 30) - 1] * d)]
    while todo:
        i, lo, hi = todo.pop()
        if dims[i] == 0xFF:
            if leaf in want_leaves:
                boxes[leaf] = (np.array(lo), np.array(hi))
            leaf += 1
            continue
        j, x = dims[i], splits[i]
        rlo = list(lo)
        rlo[j] = max(rlo[j], x)
        lhi = list(hi)
        lhi[j] = min(lhi[j], x - 1)
        todo.append((i + 1 + cnt[i + 1], rlo, list(hi)))
        todo.append((i + 1, list(lo), lhi))
    return boxes


def test_full_size_bench_workload_properties():
    from paper_2411_09275_gb300 import pkd

    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    n, d, m = wl["n"], wl["d"], wl["m"]
    X, Y, yid, zid = bench.make_inputs(wl, 0)
    params = pkd.Params(d=d)
    t = pkd.Tree(to_dev(X), None, params)
    t.insert(to_dev(Y), ids_dev(yid))
    assert t.delete(ids_dev(zid)) == m
    assert t.size == n
    allX = np.concatenate([X, Y])
    alive = np.ones(n + m, bool)
    alive[zid.astype(np.int64)] = False
    live = np.flatnonzero(alive)

    ex = t.export()
    # every live id exactly once
    assert np.array_equal(np.sort(ex["leaf_ids"]), live.astype(np.uint32))
    dims, sizes = ex["dims"], ex["sizes"].astype(np.int64)
    leaf_sizes = sizes[dims == 0xFF]
    assert leaf_sizes.sum() == n
    offs = ex["leaf_offsets"].astype(np.int64)
    assert np.array_equal(np.diff(offs), leaf_sizes)
    # leaves above phi must be heavy (all points identical)
    big = np.flatnonzero(leaf_sizes > params.phi)
    for k in big[:50]:
        pts = allX[ex["leaf_ids"][offs[k]:offs[k + 1]].astype(np.int64)]
        assert (pts == pts[0]).all()
    # sampled leaves lie inside their subspaces
    rng = np.random.default_rng(7)
    nleaves = len(leaf_sizes)
    want = set(int(x) for x in rng.choice(nleaves, size=200, replace=False))
    boxes = _leaf_boxes(ex, d, want)
    assert len(boxes) == len(want)
    for k, (blo, bhi) in boxes.items():
        pts = allX[ex["leaf_ids"][offs[k]:offs[k + 1]].astype(np.int64)]
        assert (pts >= blo).all() and (pts <= bhi).all()

    # k-NN and range counts against brute force on sampled queries
    P = allX[live]
    pid = live.astype(np.uint32)
    Q = np.concatenate([I.uniform(6, d, 2), X[rng.choice(n, 6, replace=False)]])
    k = 10
    gi, gd = t.knn(to_dev(Q), k)
    gi = gi.cpu().numpy().view(np.uint32)
    gd = gd.cpu().numpy()
    for qi in range(len(Q)):
        d2 = np.zeros(len(P), np.int64)
        for j in range(d):
            dj = P[:, j].astype(np.int64) - int(Q[qi, j])
            d2 += dj * dj
        kth = np.partition(d2, k - 1)[k - 1]
        cand = np.flatnonzero(d2 <= kth)
        order = cand[np.lexsort((pid[cand], d2[cand]))][:k]
        assert np.array_equal(gd[qi], d2[order]) and np.array_equal(gi[qi], pid[order])
    lo, hi = I.boxes(8, d, 1 << 26, 5)
    cnt = t.range_count(to_dev(lo), to_dev(hi)).cpu().numpy().astype(np.int64)
    for bi in range(len(lo)):
        assert cnt[bi] == int(np.all((P >= lo[bi]) & (P <= hi[bi]), axis=1).sum())
    t.close()


def _golden():
    want = {}
    with open(G.OUT) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            kind, key, *rest = ln.split()
            want.setdefault(kind, {})[key] = rest
    return want


@pytest.mark.parametrize("kind", ["uniform", "varden"])
def test_full_size_equals_oracle_golden(kind):
    from paper_2411_09275_gb300 import pkd

    wl = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD], kind=kind)
    assert (wl["n"], wl["d"], wl["m"]) == (G.N, G.D, G.M)
    X, Y, yid, zid = bench.make_inputs(wl, 0)
    gX, gY, gyid, gzid, gQ = G.workload(kind)  # the golden script's own draw of the inputs
    assert np.array_equal(X, gX) and np.array_equal(Y, gY) and np.array_equal(yid, gyid)
    assert np.array_equal(zid, gzid)
    del gX, gY
    t = pkd.Tree(to_dev(X), None, pkd.Params(d=wl["d"]))
    t.insert(to_dev(Y), ids_dev(yid))
    assert t.delete(ids_dev(zid)) == wl["m"]
    ex = t.export()
    qi, qd = t.knn(to_dev(gQ), G.K)
    qi = qi.cpu().numpy().view(np.uint32)
    qd = qd.cpu().numpy()
    t.close()
    want = _golden()[kind]
    nodes, leaves = int(want["nodes"][0]), int(want["nodes"][2])
    assert (len(ex["dims"]), len(ex["leaf_offsets"]) - 1) == (nodes, leaves)
    assert G.export_digest(ex) == want["export_sha256"][0]
    row0 = " ".join(f"{int(a)}:{int(b)}" for a, b in zip(qi[0], qd[0]))
    assert row0 == " ".join(want["knn_row0"])
    assert G.knn_digest(qi, qd) == want["knn_sha256"][0]
