"""Helpers for checking canonical tree exports against the definitions of a
kd-tree (Sec. 2 of the paper).  Pure numpy; independent of both the oracle
and the CUDA path."""
from __future__ import annotations

import numpy as np

COORD_MAX = (1 << 30) - 1


def walk(export: dict, d: int):
    """Yield (kind, node_index, depth, lo[d], hi[d], leaf_index) for every
    node of a pre-order export; lo/hi is the node's subspace implied by the
    splitters above it (closed box, left = strictly below the split)."""
    dims, splits = export["dims"], export["splits"]
    stack = [(0, np.zeros(d, np.int64), np.full(d, COORD_MAX, np.int64))]
    i = 0
    leaf = 0
    while stack:
        depth, lo, hi = stack.pop()
        if dims[i] == 0xFF:
            yield ("leaf", i, depth, lo, hi, leaf)
            leaf += 1
        else:
            j, x = int(dims[i]), int(splits[i])
            yield ("node", i, depth, lo, hi, None)
            llo, lhi = lo.copy(), hi.copy()
            lhi[j] = min(lhi[j], x - 1)
            rlo, rhi = lo.copy(), hi.copy()
            rlo[j] = max(rlo[j], x)
            stack.append((depth + 1, rlo, rhi))  # right after left
            stack.append((depth + 1, llo, lhi))
        i += 1
    assert i == len(dims), "export is not a complete pre-order binary tree"


def leaf_sets(export: dict):
    offs = export["leaf_offsets"].astype(np.int64)
    ids = export["leaf_ids"]
    return [ids[offs[k]:offs[k + 1]] for k in range(len(offs) - 1)]


def check_invariants(export: dict, coords: np.ndarray, ids: np.ndarray, phi: int,
                     built_fresh: bool = True):
    """The kd-tree definitions: every id exactly once; every point inside its
    leaf's subspace; leaves of at most phi points unless all identical; every
    interior size is the sum of its leaves; fresh builds have no empty child."""
    d = coords.shape[1]
    by_id = {int(i): k for k, i in enumerate(ids)}
    sets = leaf_sets(export)
    allids = np.concatenate(sets) if sets else np.zeros(0, np.uint32)
    assert len(allids) == len(ids)
    assert np.array_equal(np.sort(allids), np.sort(ids)), "ids differ from the input set"
    sizes = export["sizes"]
    dims = export["dims"]
    nodes = list(walk(export, d))
    # subtree sizes: recompute bottom-up over the pre-order
    n = len(dims)
    sub = np.zeros(n, np.int64)
    children = {}
    stack = []
    for i in range(n):
        if stack:
            p = stack[-1]
            children.setdefault(p, []).append(i)
            if len(children[p]) == 2:
                stack.pop()
        if dims[i] != 0xFF:
            stack.append(i)
    leaf_k = 0
    leaf_of_node = {}
    for kind, i, depth, lo, hi, lk in nodes:
        if kind == "leaf":
            leaf_of_node[i] = lk
    for i in range(n - 1, -1, -1):
        if dims[i] == 0xFF:
            sub[i] = len(sets[leaf_of_node[i]])
        else:
            a, b = children[i]
            sub[i] = sub[a] + sub[b]
            if built_fresh:
                assert sub[a] > 0 and sub[b] > 0, "empty child in a fresh build"
    assert np.array_equal(sub, sizes.astype(np.int64)), "stored sizes differ from leaf counts"
    for kind, i, depth, lo, hi, lk in nodes:
        if kind != "leaf":
            continue
        s = sets[lk]
        if len(s) == 0:
            continue
        pts = coords[[by_id[int(v)] for v in s]]
        assert (pts >= lo).all() and (pts <= hi).all(), f"leaf {lk} holds a point outside its box"
        if len(s) > phi:
            assert (pts == pts[0]).all(), f"leaf {lk} exceeds phi without being heavy"


def height(export: dict) -> int:
    return max(depth for kind, i, depth, lo, hi, lk in walk(export, 1))


def textbook_kdtree(coords: np.ndarray, ids: np.ndarray, phi: int) -> dict:
    """The plain kd-tree of Sec. 2 / the start of Sec. 3, written naively:
    leaf at <= phi points or all points identical; otherwise split on the
    widest dimension (lowest on ties) at the element of rank floor(n/2), or
    at the next larger distinct value when nothing lies below it; strictly
    smaller goes left.  Returns a canonical export."""
    dims, splits, sizes, leaf_ids, offs = [], [], [], [], [0]

    def rec(P, I):
        n = len(P)
        if n <= phi or (P == P[0]).all():
            dims.append(0xFF)
            splits.append(0)
            sizes.append(n)
            leaf_ids.extend(sorted(int(v) for v in I))
            offs.append(len(leaf_ids))
            return
        ext = P.max(axis=0).astype(np.int64) - P.min(axis=0)
        j = int(np.argmax(ext))
        v = np.sort(P[:, j])
        x = int(v[n // 2])
        if v[0] == x:
            x = int(v[v > v[0]].min())
        dims.append(j)
        splits.append(x)
        sizes.append(n)
        m = P[:, j] < x
        rec(P[m], I[m])
        rec(P[~m], I[~m])

    if len(coords) == 0:
        dims, splits, sizes, offs = [0xFF], [0], [0], [0, 0]
    else:
        rec(coords, ids)
    return dict(dims=np.array(dims, np.uint8), splits=np.array(splits, np.int32),
                sizes=np.array(sizes, np.uint64), leaf_ids=np.array(leaf_ids, np.uint32),
                leaf_offsets=np.array(offs, np.uint64))


def exports_equal(a: dict, b: dict) -> bool:
    return all(np.array_equal(a[k], b[k]) for k in
               ("dims", "splits", "sizes", "leaf_ids", "leaf_offsets"))


def assert_exports_equal(a: dict, b: dict):
    for k in ("dims", "splits", "sizes", "leaf_offsets", "leaf_ids"):
        x, y = a[k], b[k]
        assert len(x) == len(y), f"{k}: length {len(x)} != {len(y)}"
        if not np.array_equal(x, y):
            bad = np.nonzero(x != y)[0]
            raise AssertionError(f"{k}: {len(bad)} mismatches, first at {bad[0]}: {x[bad[0]]} != {y[bad[0]]}")


def knn_numpy(coords: np.ndarray, ids: np.ndarray, q: np.ndarray, k: int):
    """k-NN by definition: the k smallest (squared distance, id) pairs."""
    out_i = np.full((len(q), k), 0xFFFFFFFF, np.uint32)
    out_d = np.full((len(q), k), np.iinfo(np.int64).max, np.int64)
    c = coords.astype(np.int64)
    for r in range(len(q)):
        d2 = ((c - q[r].astype(np.int64)) ** 2).sum(axis=1)
        o = np.lexsort((ids, d2))[:k]
        out_i[r, :len(o)] = ids[o]
        out_d[r, :len(o)] = d2[o]
    return out_i, out_d


def range_count_numpy(coords, lo, hi):
    return np.array([((coords >= lo[r]) & (coords <= hi[r])).all(axis=1).sum()
                     for r in range(len(lo))], np.uint64)


# --------------------------------------------------------------------------
# Nested view of an export, and checkers that re-derive a tree top-down from
# the rules (used to pin the oracle's composition of its building blocks)
# --------------------------------------------------------------------------

def parse(export: dict):
    """Pre-order export -> nested dicts {leaf, dim, split, size, l, r, ids}."""
    dims, splits, sizes = export["dims"], export["splits"], export["sizes"]
    sets = leaf_sets(export)
    pos, leaf = [0], [0]

    def rec():
        i = pos[0]
        pos[0] += 1
        if dims[i] == 0xFF:
            s = sets[leaf[0]]
            leaf[0] += 1
            return dict(leaf=True, ids=np.asarray(s, np.uint32), size=int(sizes[i]))
        l = rec()
        r = rec()
        return dict(leaf=False, dim=int(dims[i]), split=int(splits[i]), size=int(sizes[i]),
                    l=l, r=r, ids=np.concatenate([l["ids"], r["ids"]]))

    return rec()


def unparse(tree) -> dict:
    dims, splits, sizes, lids, offs = [], [], [], [], [0]

    def rec(v):
        if v["leaf"]:
            dims.append(0xFF)
            splits.append(0)
            sizes.append(v["size"])
            lids.extend(sorted(int(x) for x in v["ids"]))
            offs.append(len(lids))
            return
        dims.append(v["dim"])
        splits.append(v["split"])
        sizes.append(v["size"])
        rec(v["l"])
        rec(v["r"])

    rec(tree)
    return dict(dims=np.array(dims, np.uint8), splits=np.array(splits, np.int32),
                sizes=np.array(sizes, np.uint64), leaf_ids=np.array(lids, np.uint32),
                leaf_offsets=np.array(offs, np.uint64))


def rederive_build(tree, xyz: dict, P, split_rule, is_sampled, sample_shift, depth=0):
    """Check every node of a built (sub)tree against Alg. 1's rules, top-down:
    a Build(P, t) root is a leaf iff |P| <= phi or P is all identical;
    otherwise its sample is drawn at depth t and the first lambda levels are
    the skeleton on that sample (a node splits while it has >= 2 sigma_os
    distinct samples), each bucket at local depth j being Build(P_b, t + j),
    or, when the skeleton root is a bucket, one exact split of P itself.
    ``xyz`` maps id -> coordinate tuple; P carries the parameters."""
    def coords(ids):
        return np.array([xyz[int(i)] for i in ids], np.int32).reshape(len(ids), P.d)

    def identical(ids):
        c = coords(ids)
        return len(c) == 0 or bool((c == c[0]).all())

    def build_root(v, t):
        n = len(v["ids"])
        assert v["size"] == n
        if n <= P.phi or identical(v["ids"]):
            assert v["leaf"], f"depth {t}: expected a leaf of {n} points"
            return
        assert not v["leaf"], f"depth {t}: {n} points must be split"
        s = sample_shift(P, n)
        S = np.array([i for i in v["ids"] if is_sampled(P.seed, t, int(i), s)], np.uint32)
        skeleton(v, S, 0, t)

    def skeleton(v, S, j, t):
        if j < P.lam and len(S) >= 2 * P.sigma_os and not identical(S):
            assert not v["leaf"]
            cs = coords(S)
            assert (v["dim"], v["split"]) == split_rule(cs), f"skeleton node at depth {t + j}"
            m = cs[:, v["dim"]] < v["split"]
            skeleton(v["l"], S[m], j + 1, t)
            skeleton(v["r"], S[~m], j + 1, t)
        elif j == 0:
            assert (v["dim"], v["split"]) == split_rule(coords(v["ids"])), f"exact split at depth {t}"
            build_root(v["l"], t + 1)
            build_root(v["r"], t + 1)
        else:
            build_root(v, t + j)

    build_root(tree, depth)


def expect_insert(tree, xyz: dict, bc, bi, P, build_at, balanced):
    """Alg. 2 node by node: a leaf takes Build(leaf + new, t); an interior node
    that receives new points stays (and recurses) when it is still
    alpha-balanced, else it is rebuilt with all its points and the new ones."""
    def rec(v, B, t):
        if len(B) == 0:
            return v
        if v["leaf"]:
            return build_at(np.concatenate([v["ids"], bi[B]]), t)
        m = bc[B, v["dim"]] < v["split"]
        N, L = v["size"] + len(B), v["l"]["size"] + int(m.sum())
        if balanced(L, N, P.alpha_num, P.alpha_den):
            l, r = rec(v["l"], B[m], t + 1), rec(v["r"], B[~m], t + 1)
            return dict(leaf=False, dim=v["dim"], split=v["split"], size=N, l=l, r=r,
                        ids=np.concatenate([l["ids"], r["ids"]]))
        return build_at(np.concatenate([v["ids"], bi[B]]), t)

    return rec(tree, np.arange(len(bi)), 0)


def expect_delete(tree, dead: set, P, build_at, balanced):
    """Sec. 4.2 node by node with exact post-deletion sizes: a node without
    deleted points stays; one that empties becomes an empty leaf; a leaf
    keeps its survivors; an interior node stays (and recurses) when still
    alpha-balanced, else it is rebuilt from its survivors."""
    def ndead(v):
        return sum(1 for i in v["ids"] if int(i) in dead)

    def live(v):
        return np.array([i for i in v["ids"] if int(i) not in dead], np.uint32)

    def rec(v, t):
        k = ndead(v)
        if k == 0:
            return v
        N = v["size"] - k
        if N == 0:
            return dict(leaf=True, ids=np.zeros(0, np.uint32), size=0)
        if v["leaf"]:
            return build_at(live(v), t)
        L = v["l"]["size"] - ndead(v["l"])
        if balanced(L, N, P.alpha_num, P.alpha_den):
            l, r = rec(v["l"], t + 1), rec(v["r"], t + 1)
            return dict(leaf=False, dim=v["dim"], split=v["split"], size=N, l=l, r=r,
                        ids=np.concatenate([l["ids"], r["ids"]]))
        return build_at(live(v), t)

    return rec(tree, 0)
