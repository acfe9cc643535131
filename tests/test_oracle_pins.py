"""Pins for the CPU oracle against things other than itself: a published
random-number test vector, hand-worked splitter cases, a naive textbook
kd-tree, brute-force numpy definitions of the queries, set algebra for the
updates and the kd-tree invariants of Sec. 2."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2411_09275_gb300 import inputs as I
from tests import treeutil as U

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _gold_lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.strip() for l in f if l.strip() and not l.startswith("#")]


# --------------------------------------------------------------------------
# Sampling hash
# --------------------------------------------------------------------------

def test_mix64_matches_published_splitmix64_vector():
    want = [int(v) for v in _gold_lines("splitmix64_seed1234567.txt")]
    got = [O.mix64((1234567 + (k + 1) * GAMMA) & M64) for k in range(len(want))]
    assert got == want


def test_sample_rate_and_depth_independence():
    # Rate mode draws a point with probability 2^-s, independently per depth.
    n, s = 200_000, 4
    ids = np.arange(n, dtype=np.uint32)
    a = np.array([O.is_sampled(7, 3, int(i), s) for i in ids[:50_000]])
    b = np.array([O.is_sampled(7, 4, int(i), s) for i in ids[:50_000]])
    p = 2.0 ** -s
    sd = np.sqrt(p * (1 - p) / len(a))
    assert abs(a.mean() - p) < 5 * sd
    assert abs(b.mean() - p) < 5 * sd
    both = (a & b).mean()
    assert abs(both - p * p) < 5 * np.sqrt(p * p / len(a))
    assert all(O.is_sampled(1, 0, int(i), 0) for i in ids[:100])  # s = 0: every point


def test_count_mode_shift():
    # about 2^lambda * sigma_os samples: s = max(0, floor(log2(n / (2^lambda sigma_os))))
    p = O.Params(d=2, lam=6, sigma_os=32, count_mode=1)
    base = 64 * 32
    assert O.sample_shift(p, 1) == 0
    assert O.sample_shift(p, base - 1) == 0
    assert O.sample_shift(p, base) == 0
    assert O.sample_shift(p, 2 * base - 1) == 0
    assert O.sample_shift(p, 2 * base) == 1
    assert O.sample_shift(p, 1024 * base) == 10
    assert O.sample_shift(p, 1024 * base + 5) == 10
    assert O.sample_shift(O.Params(d=2, sigma_log2=6), 10 ** 8) == 6  # rate mode: fixed


# --------------------------------------------------------------------------
# Splitter rule and balance test
# --------------------------------------------------------------------------

def test_split_rule_hand_cases():
    for line in _gold_lines("split_rule_cases.txt"):
        d, pts, dim, x, nleft = [f.strip() for f in line.split("|")]
        d = int(d)
        P = np.array([[int(v) for v in t.split(",")] for t in pts.split()], np.int32)
        assert P.shape[1] == d
        got = O.split_rule(P)
        assert got == (int(dim), int(x)), line
        assert int((P[:, got[0]] < got[1]).sum()) == int(nleft), line


def test_split_rule_properties_random():
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(2, 60))
        d = int(rng.integers(1, 5))
        P = rng.integers(0, int(rng.choice([3, 50, 1 << 30])), size=(n, d)).astype(np.int32)
        got = O.split_rule(P)
        if (P == P[0]).all():
            assert got is None
            continue
        j, x = got
        ext = P.max(0).astype(np.int64) - P.min(0)
        assert ext[j] == ext.max() and (ext[:j] < ext.max()).all()
        left = (P[:, j] < x).sum()
        assert 0 < left < n  # both sides non-empty
        v = np.sort(P[:, j])
        if v[0] != v[n // 2]:
            assert x == v[n // 2]  # the rank-floor(n/2) element
        else:
            assert x == v[v > v[0]].min()


def test_balance_boundaries():
    # alpha = 3/10: balanced iff 0.2 <= L/N <= 0.8, inclusive.
    assert O.balanced(20, 100, 3, 10) and O.balanced(80, 100, 3, 10)
    assert not O.balanced(19, 100, 3, 10) and not O.balanced(81, 100, 3, 10)
    assert O.balanced(50, 100, 3, 10)
    assert O.balanced(1, 5, 3, 10) and not O.balanced(0, 5, 3, 10)
    # alpha = 0: exactly half only; alpha = 1/2: always.
    assert O.balanced(5, 10, 0, 1) and not O.balanced(4, 10, 0, 1) and not O.balanced(3, 7, 0, 1)
    assert all(O.balanced(L, 9, 1, 2) for L in range(10))


# --------------------------------------------------------------------------
# Construction
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d,phi,sigma_os,kind", [
    (1, 4, 4, "uniform"), (2, 32, 32, "uniform"), (2, 4, 4, "dups"),
    (3, 8, 8, "varden"), (5, 6, 4, "uniform"), (2, 1, 1, "dups"),
])
def test_sample_all_equals_textbook_kdtree(d, phi, sigma_os, kind):
    # With every point sampled (s = 0) and 2*sigma_os > phi, every splitter of
    # Alg. 1 is the exact median of its node's own points, so the tree must be
    # the plain kd-tree of Sec. 2, whatever the skeleton height.
    n = 3000
    if kind == "uniform":
        X = I.uniform(n, d, 21)
    elif kind == "varden":
        X = I.varden(n, d, 22)
    else:
        X = (I.uniform(n, d, 23) % 7).astype(np.int32)
    ids = np.arange(n, dtype=np.uint32)[::-1].copy()
    for lam in (1, 3, 6):
        p = O.Params(d=d, phi=phi, lam=lam, sigma_log2=0, sigma_os=sigma_os, seed=9)
        got = O.OracleTree(X, ids, p).export()
        U.assert_exports_equal(got, U.textbook_kdtree(X, ids, phi))


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("kind", ["uniform", "varden", "dups"])
def test_build_invariants(d, kind):
    n = 4000
    if kind == "uniform":
        X = I.uniform(n, d, 31)
    elif kind == "varden":
        X = I.varden(n, d, 32)
    else:
        X = (I.uniform(n, d, 33) % 3).astype(np.int32)
    ids = (np.arange(n, dtype=np.uint32) * 7 + 3)
    for p in (O.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4),
              O.Params(d=d, phi=32, lam=6, sigma_log2=6, sigma_os=32),
              O.Params(d=d, phi=5, lam=4, sigma_os=8, count_mode=1)):
        e = O.OracleTree(X, ids, p).export()
        U.check_invariants(e, X, ids, p.phi)


def test_one_dimension_leaves_are_sorted():
    # d = 1: the kd-tree is a search tree, so in-order leaves are sorted with
    # every leaf strictly below the next (equal keys never straddle a split).
    X = (I.uniform(5000, 1, 41) % 1000).astype(np.int32)
    ids = np.arange(5000, dtype=np.uint32)
    t = O.OracleTree(X, ids, O.Params(d=1, phi=8, lam=4, sigma_log2=3, sigma_os=4))
    sets = U.leaf_sets(t.export())
    prev_max = -1
    for s in sets:
        v = X[s.astype(np.int64), 0]
        assert v.min() > prev_max
        prev_max = v.max()


def test_special_cases():
    p = O.Params(d=2, phi=32)
    e = O.OracleTree(np.zeros((0, 2), np.int32), None, p).export()
    assert list(e["dims"]) == [0xFF] and list(e["leaf_offsets"]) == [0, 0]
    X = I.uniform(32, 2, 1)
    e = O.OracleTree(X, None, p).export()
    assert list(e["dims"]) == [0xFF] and e["sizes"][0] == 32
    X = np.full((1000, 2), 77, np.int32)
    e = O.OracleTree(X, None, p).export()  # all identical: one heavy leaf
    assert list(e["dims"]) == [0xFF] and e["sizes"][0] == 1000
    X = np.zeros((1000, 2), np.int32)
    X[::2, 1] = 5  # two distinct values on one dimension
    e = O.OracleTree(X, None, p).export()
    assert e["dims"][0] == 1 and e["splits"][0] == 5
    assert len(e["dims"]) == 3 and list(e["sizes"]) == [1000, 500, 500]


def test_root_splitter_rederived_from_sample():
    # The root splitter is the rule applied to the root sample (the points
    # whose hash at depth 0 passes), not to the points themselves.
    n, d = 20000, 3
    X = I.uniform(n, d, 51)
    p = O.Params(d=d, phi=32, lam=6, sigma_log2=5, sigma_os=32, seed=1234)
    e = O.OracleTree(X, None, p).export()
    S = X[[i for i in range(n) if O.is_sampled(p.seed, 0, i, 5)]]
    assert len(S) >= 2 * p.sigma_os
    assert (int(e["dims"][0]), int(e["splits"][0])) == O.split_rule(S)
    # and its exact-median counterpart differs (the sample matters)
    assert O.split_rule(X) != O.split_rule(S)


def test_height_bound_uniform():
    # Lemma 3.2: height O(log n); sampled medians keep it near log2(n/phi).
    n = 100_000
    X = I.uniform(n, 2, 61)
    t = O.OracleTree(X, None, O.Params(d=2))
    assert t.height <= int(np.ceil(np.log2(n / 32))) + 3


# --------------------------------------------------------------------------
# Queries
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_knn_tree_and_brute_match_numpy_definition(d):
    n = 3000
    X = I.varden(n, d, 71) if d == 3 else I.uniform(n, d, 71)
    X[::10] = X[1::10]  # duplicates force distance ties
    ids = np.arange(n, dtype=np.uint32)[::-1].copy()
    t = O.OracleTree(X, ids, O.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4))
    Q = np.concatenate([I.uniform(40, d, 72), X[:20]])
    for k in (1, 10, 37):
        want = U.knn_numpy(X, ids, Q, k)
        for brute in (False, True):
            gi, gd = t.knn(Q, k, brute=brute)
            assert np.array_equal(gd, want[1]) and np.array_equal(gi, want[0])
    # k larger than the tree: padded
    gi, gd = O.OracleTree(X[:5], ids[:5], O.Params(d=d)).knn(Q[:3], 8)
    assert (gi[:, 5:] == 0xFFFFFFFF).all() and (gd[:, 5:] == np.iinfo(np.int64).max).all()


@pytest.mark.parametrize("d", [1, 2, 3])
def test_range_count_matches_numpy_definition(d):
    n = 5000
    X = I.uniform(n, d, 81)
    t = O.OracleTree(X, None, O.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8))
    for side in (1 << 20, 1 << 28, 1 << 30):
        lo, hi = I.boxes(60, d, side, 82)
        want = U.range_count_numpy(X, lo, hi)
        assert np.array_equal(t.range_count(lo, hi), want)
        assert np.array_equal(t.range_count(lo, hi, brute=True), want)


# --------------------------------------------------------------------------
# Batch updates
# --------------------------------------------------------------------------

def _multiset(ids, xs):
    return sorted(zip(ids.tolist(), map(tuple, xs.tolist())))


@pytest.mark.parametrize("kind", ["uniform", "varden"])
def test_updates_set_algebra_and_invariants(kind):
    d, n, m = 3, 6000, 1500
    X = I.points(kind, n, d, 91)
    ids = np.arange(n, dtype=np.uint32)
    p = O.Params(d=d, phi=16, lam=3, sigma_log2=3, sigma_os=8)
    t = O.OracleTree(X, ids, p)
    Y = I.points(kind, m, d, 92)
    yid = np.arange(n, n + m, dtype=np.uint32)
    t.insert(Y, yid)
    allX, allI = np.concatenate([X, Y]), np.concatenate([ids, yid])
    assert _multiset(*t.points()) == _multiset(allI, allX)
    U.check_invariants(t.export(), allX, allI, p.phi, built_fresh=False)
    # delete: some present points, repeats, and ids that name no point
    sel = I.sample_indices(2000, n + m, 93)
    di = allI[sel].copy()
    di = np.concatenate([di, di[:50], di[50:80], np.full(10, 10 ** 9, np.uint32)])
    nd = t.delete(di)
    keep = np.ones(n + m, bool)
    keep[sel] = False
    assert nd == 2000 and t.size == n + m - 2000
    assert _multiset(*t.points()) == _multiset(allI[keep], allX[keep])
    U.check_invariants(t.export(), allX[keep], allI[keep], p.phi, built_fresh=False)


def test_exact_median_updates_keep_every_node_balanced():
    # With every point sampled and distinct coordinates, a fresh build splits
    # at exact medians, so every node is alpha-balanced; Alg. 2 and Sec. 4.2
    # must keep it so after any sequence of batches.
    d, n = 2, 4000
    X = I.uniform(n, d, 101)
    ids = np.arange(n, dtype=np.uint32)
    p = O.Params(d=d, phi=8, lam=3, sigma_log2=0, sigma_os=8)
    t = O.OracleTree(X, ids, p)
    nxt = n
    live_X, live_I = [X], [ids]
    rng = np.random.default_rng(3)
    for r in range(6):
        # skewed insert: all in a corner, to force rebuilds
        Y = (I.uniform(700, d, 200 + r) // 8).astype(np.int32)
        yid = np.arange(nxt, nxt + 700, dtype=np.uint32)
        nxt += 700
        t.insert(Y, yid)
        live_X.append(Y)
        live_I.append(yid)
        AX, AI = np.concatenate(live_X), np.concatenate(live_I)
        # skewed delete: the largest x0 first
        sel = np.argsort(-AX[:, 0])[:500]
        assert t.delete(AI[sel]) == 500
        keep = np.ones(len(AI), bool)
        keep[sel] = False
        live_X, live_I = [AX[keep]], [AI[keep]]
        e = t.export()
        # check every interior node: L/N within [0.2, 0.8]
        dims, sizes = e["dims"], e["sizes"]
        stack, kids = [], {}
        for i in range(len(dims)):
            if stack:
                q = stack[-1]
                kids.setdefault(q, []).append(i)
                if len(kids[q]) == 2:
                    stack.pop()
            if dims[i] != 0xFF:
                stack.append(i)
        for i, (a, b) in kids.items():
            assert O.balanced(int(sizes[a]), int(sizes[i]), 3, 10), (r, i)


def test_alpha_half_never_rebuilds_interior_nodes():
    d, n = 2, 5000
    X = I.uniform(n, d, 111)
    p = O.Params(d=d, phi=16, lam=4, sigma_log2=2, sigma_os=8, alpha_num=1, alpha_den=2)
    t = O.OracleTree(X, None, p)
    before = t.export()
    t.insert((I.uniform(3000, d, 112) // 16).astype(np.int32), np.arange(n, n + 3000, dtype=np.uint32))
    after = t.export()
    # the splitters above the old leaves survive: the old pre-order interior
    # sequence is a subsequence of the new one at the same nodes
    old_int = [(int(a), int(b)) for a, b in zip(before["dims"], before["splits"]) if a != 0xFF]
    new_int = [(int(a), int(b)) for a, b in zip(after["dims"], after["splits"]) if a != 0xFF]
    it = iter(new_int)
    assert all(any(x == y for y in it) for x in old_int)
    assert after["sizes"][0] == n + 3000


def test_alpha_zero_root_rebuild_equals_fresh_build():
    # alpha = 0: a root of odd size can never be exactly balanced, so
    # insertion rebuilds the root: the tree equals Build(union) at depth 0.
    d, n, m = 2, 3001, 1000
    X = I.uniform(n, d, 121)
    Y = I.uniform(m, d, 122)
    ids = np.arange(n + m, dtype=np.uint32)
    p = O.Params(d=d, phi=16, lam=3, sigma_log2=2, sigma_os=8, alpha_num=0, alpha_den=1)
    t = O.OracleTree(X, ids[:n], p)
    t.insert(Y, ids[n:])
    fresh = O.OracleTree(np.concatenate([X, Y]), ids, p)
    U.assert_exports_equal(t.export(), fresh.export())


def test_insert_into_leaf_root_and_delete_to_empty():
    d = 2
    p = O.Params(d=d, phi=32)
    X = I.uniform(10, d, 131)
    t = O.OracleTree(X, np.arange(10, dtype=np.uint32), p)
    Y = I.uniform(500, d, 132)
    t.insert(Y, np.arange(10, 510, dtype=np.uint32))
    fresh = O.OracleTree(np.concatenate([X, Y]), np.arange(510, dtype=np.uint32), p)
    U.assert_exports_equal(t.export(), fresh.export())  # leaf root: Build(T u P)
    allX = np.concatenate([X, Y])
    assert t.delete(np.arange(510, dtype=np.uint32)) == 510
    e = t.export()
    assert list(e["dims"]) == [0xFF] and t.size == 0
    assert t.delete(np.arange(5, dtype=np.uint32)) == 0


def test_invalid_inputs_rejected():
    with pytest.raises(O.OracleError):
        O.OracleTree(np.array([[1 << 30, 0]], np.int32), None, O.Params(d=2))
    with pytest.raises(O.OracleError):
        O.OracleTree(np.array([[-1, 0]], np.int32), None, O.Params(d=2))
    with pytest.raises(O.OracleError):
        O.OracleTree(np.zeros((3, 2), np.int32), None, O.Params(d=2, alpha_num=3, alpha_den=5))
    with pytest.raises(O.OracleError):
        O.OracleTree(np.zeros((3, 9), np.int32), None, O.Params(d=9))


# --------------------------------------------------------------------------
# Top-down re-derivation of builds and updates
# --------------------------------------------------------------------------

def _xyz(X, ids):
    return {int(i): tuple(int(v) for v in x) for i, x in zip(ids, X)}


@pytest.mark.parametrize("cfg", [
    dict(d=2, phi=8, lam=3, sigma_log2=2, sigma_os=4, kind="uniform"),
    dict(d=3, phi=4, lam=2, sigma_log2=1, sigma_os=3, kind="varden"),
    dict(d=2, phi=6, lam=4, sigma_os=4, count_mode=1, kind="dups"),
    dict(d=1, phi=3, lam=1, sigma_log2=3, sigma_os=2, kind="uniform"),
])
def test_build_rederived_top_down(cfg):
    cfg = dict(cfg)
    kind = cfg.pop("kind")
    P = O.Params(seed=77, **cfg)
    n = 2500
    X = I.points("uniform" if kind == "dups" else kind, n, P.d, 141)
    if kind == "dups":
        X = (X % 5).astype(np.int32)
    ids = (np.arange(n, dtype=np.uint32) * 13 + 1)
    for depth in (0, 3):
        tree = U.parse(O.OracleTree(X, ids, P, depth=depth).export())
        U.rederive_build(tree, _xyz(X, ids), P, O.split_rule, O.is_sampled, O.sample_shift,
                         depth=depth)


@pytest.mark.parametrize("kind,alpha", [("uniform", (3, 10)), ("varden", (3, 10)),
                                        ("uniform", (1, 10)), ("varden", (0, 1))])
def test_updates_rederived_node_by_node(kind, alpha):
    d, n = 2, 3000
    P = O.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4, alpha_num=alpha[0],
                 alpha_den=alpha[1], seed=5)
    X = I.points(kind, n, d, 151)
    ids = np.arange(n, dtype=np.uint32)
    xyz = _xyz(X, ids)
    t = O.OracleTree(X, ids, P)

    def build_at(bids, depth):
        c = np.array([xyz[int(i)] for i in bids], np.int32).reshape(len(bids), d)
        return U.parse(O.OracleTree(c, bids, P, depth=depth).export())

    nxt = n
    rng = np.random.default_rng(9)
    for r in range(4):
        before = U.parse(t.export())
        # skewed batch: a band of the space gets most of the new points
        Y = I.points(kind, 600, d, 160 + r)
        Y[: 400, 0] = (Y[: 400, 0] // 16).astype(np.int32)
        yid = np.arange(nxt, nxt + 600, dtype=np.uint32)
        nxt += 600
        xyz.update(_xyz(Y, yid))
        want = U.expect_insert(before, xyz, Y, yid, P, build_at, O.balanced)
        t.insert(Y, yid)
        U.assert_exports_equal(t.export(), U.unparse(want))

        before = U.parse(t.export())
        live = before["ids"]
        sel = live[np.argsort([xyz[int(i)][1] for i in live])[:500]]  # the 500 lowest x1
        sel = np.concatenate([sel, rng.choice(live, 50, replace=False)])
        want = U.expect_delete(before, set(int(i) for i in sel), P, build_at, O.balanced)
        t.delete(sel)
        U.assert_exports_equal(t.export(), U.unparse(want))


def test_knn_equal_distance_tie_across_a_split():
    # Hand-built: the root splits x at 5 (widest dimension x, rank-1 element of
    # {3, 5, 100}); query (0,0) meets A=(3,4) (d2 25, id 50) in the near half
    # first, and B=(5,0) (d2 25, id 1) lies in the far half whose box is at
    # squared distance exactly 25: the far half must still be searched, and B
    # wins the tie on its smaller id.
    X = np.array([[3, 4], [5, 0], [100, 0]], np.int32)
    ids = np.array([50, 1, 3], np.uint32)
    t = O.OracleTree(X, ids, O.Params(d=2, phi=1, lam=1, sigma_log2=0, sigma_os=1))
    e = t.export()
    assert (int(e["dims"][0]), int(e["splits"][0])) == (0, 5)
    gi, gd = t.knn(np.array([[0, 0]], np.int32), 1)
    assert gi[0, 0] == 1 and gd[0, 0] == 25
    gi, gd = t.knn(np.array([[0, 0]], np.int32), 2)
    assert list(gi[0]) == [1, 50] and list(gd[0]) == [25, 25]


def test_range_report_hand_example_and_count_consistency():
    # five 2-D points; closed boxes include their boundary
    X = np.array([[0, 0], [5, 5], [5, 9], [10, 0], [7, 7]], np.int32)
    ids = np.array([40, 11, 12, 3, 9], np.uint32)
    lo = np.array([[0, 0], [5, 5], [8, 8], [0, 0]], np.int32)
    hi = np.array([[5, 5], [7, 9], [9, 9], [10, 10]], np.int32)
    got = O.range_report(X, ids, lo, hi)
    assert [list(g) for g in got] == [[11, 40], [9, 11, 12], [], [3, 9, 11, 12, 40]]
    # the tree's report agrees with its own count on random boxes
    rng = np.random.default_rng(3)
    P = rng.integers(0, 1 << 20, size=(3000, 3)).astype(np.int32)
    t = O.OracleTree(P, None, O.Params(d=3, phi=8, lam=3, sigma_log2=2, sigma_os=4))
    lo = rng.integers(0, 1 << 19, size=(50, 3)).astype(np.int32)
    hi = lo + rng.integers(0, 1 << 19, size=(50, 3)).astype(np.int32)
    rep = t.range_report(lo, hi)
    assert [len(r) for r in rep] == list(t.range_count(lo, hi).astype(int))
    t.close()


# --------------------------------------------------------------------------
# Reading R5: a node no update reaches is not re-tested
# --------------------------------------------------------------------------

def _pre_order(e):
    """(children, depth, end of subtree) per pre-order node index."""
    dims = e["dims"]
    n = len(dims)
    kids, stack = {}, []
    depth = np.zeros(n, int)
    for i in range(n):
        if stack:
            p = stack[-1]
            kids.setdefault(p, []).append(i)
            depth[i] = depth[p] + 1
            if len(kids[p]) == 2:
                stack.pop()
        if dims[i] != 0xFF:
            stack.append(i)
    end = np.zeros(n, int)
    for i in range(n - 1, -1, -1):
        end[i] = i + 1 if dims[i] == 0xFF else end[kids[i][1]]
    return kids, depth, end


def test_untouched_unbalanced_node_is_kept_r5():
    # 60 points on a line, rate-1/2 samples, lambda = 2, phi = 2, alpha = 3/10.
    # The node at pre-order 14 (depth 3) was split on its ancestor's sample at
    # 139, below which only one of its ten points lies: 2*10*1 = 20 is below
    # (10 - 6)*10 = 40, so it is already outside the alpha band after the
    # build.  Inserting one point at the far right end (x = 999, right of the
    # root's splitter) reaches none of that subtree: Sec. 4.1 rebuilds only a
    # node that becomes unbalanced after insertion, so the subtree must come
    # out unchanged, although Build on its ten points at depth 3 (what
    # re-testing every node of Alg. 2's skeletons would do) draws a new
    # sample and gives a different subtree.
    X = np.random.default_rng(3).integers(0, 1000, size=(60, 1)).astype(np.int32)
    ids = np.arange(60, dtype=np.uint32)
    P = O.Params(d=1, phi=2, lam=2, sigma_log2=1, sigma_os=1, alpha_num=3, alpha_den=10, seed=3)
    t = O.OracleTree(X, ids, P)
    e = t.export()
    kids, depth, end = _pre_order(e)
    u = 14
    assert e["dims"][u] == 0 and depth[u] == 3 and int(e["splits"][u]) == 139
    assert int(e["sizes"][u]) == 10 and int(e["sizes"][kids[u][0]]) == 1
    assert not O.balanced(1, 10, 3, 10)
    # u's ten points: the leaves of its pre-order span
    leaf_no = np.cumsum(e["dims"] == 0xFF) - 1
    offs = e["leaf_offsets"].astype(int)
    uid = np.concatenate([e["leaf_ids"][offs[leaf_no[i]]:offs[leaf_no[i] + 1]]
                          for i in range(u, end[u]) if e["dims"][i] == 0xFF])
    assert sorted(X[uid, 0].tolist()) == [113, 139, 159, 172, 179, 181, 190, 236, 244, 254]
    assert 999 >= int(e["splits"][0]) and e["dims"][0] == 0  # the new point goes right at the root
    span = {k: e[k][u:end[u]].copy() for k in ("dims", "splits", "sizes")}
    t.insert(np.array([[999]], np.int32), np.array([60], np.uint32))
    e2 = t.export()
    for k in span:  # u lies in the root's left subtree: same pre-order positions
        assert np.array_equal(e2[k][u:end[u]], span[k]), k
    alt = O.OracleTree(X[uid], uid, P, depth=3).export()
    assert not (len(alt["dims"]) == len(span["dims"])
                and all(np.array_equal(alt[k], span[k]) for k in span))


# --------------------------------------------------------------------------
# Reading R9 (ids name points) and R6 (delete by id)
# --------------------------------------------------------------------------

def test_ids_are_unique_and_insert_rejects_whole_batches():
    d = 2
    p = O.Params(d=d, phi=4, lam=2, sigma_log2=1, sigma_os=2)
    X = I.uniform(300, d, 171)
    with pytest.raises(O.OracleError):  # a repeated id in a build
        O.OracleTree(X, np.r_[np.arange(299), [5]].astype(np.uint32), p)
    with pytest.raises(O.OracleError):  # the k-NN padding id
        O.OracleTree(X, np.r_[np.arange(299), [0xFFFFFFFF]].astype(np.uint32), p)
    t = O.OracleTree(X, np.arange(300, dtype=np.uint32), p)
    before = t.export()
    Y = I.uniform(20, d, 172)
    for bad in (np.r_[np.arange(300, 319), [7]],        # 7 is stored
                np.r_[np.arange(300, 319), [300]],      # repeated in the batch
                np.r_[np.arange(300, 319), [0xFFFFFFFF]]):
        with pytest.raises(O.OracleError):
            t.insert(Y, bad.astype(np.uint32))
        U.assert_exports_equal(t.export(), before)     # rejected whole
    t.insert(Y, np.arange(300, 320, dtype=np.uint32))
    assert t.size == 320


def test_delete_by_id_skips_unknown_dead_and_repeated_ids():
    d = 3
    p = O.Params(d=d, phi=4, lam=2, sigma_log2=1, sigma_os=2)
    X = I.uniform(500, d, 181)
    ids = (np.arange(500, dtype=np.uint32) * 7 + 3)  # sparse labels
    t = O.OracleTree(X, ids, p)
    # 40 stored ids, each twice, plus labels that name nothing
    sel = ids[::12][:40]
    batch = np.r_[sel, sel[::-1], [0, 1, 2, 4, 10 ** 9]].astype(np.uint32)
    assert t.delete(batch) == 40 and t.size == 460
    got_ids, got_x = t.points()
    keep = ~np.isin(ids, sel)
    assert sorted(zip(got_ids.tolist(), map(tuple, got_x.tolist()))) == \
        sorted(zip(ids[keep].tolist(), map(tuple, X[keep].tolist())))
    # deleted ids are gone: deleting them again removes nothing
    assert t.delete(sel) == 0
    # a deleted id may be inserted again, with new coordinates
    Y = I.uniform(3, d, 182)
    t.insert(Y, sel[:3])
    assert t.size == 463
    gi, gx = t.points()
    assert {int(i): tuple(x) for i, x in zip(gi, gx.tolist())}[int(sel[1])] == tuple(Y[1].tolist())
    assert t.delete(sel[:3]) == 3
