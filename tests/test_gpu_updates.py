"""GPU parity of BatchInsert (Alg. 2) and BatchDelete (Sec. 4.2): after every
batch the canonical export of the GPU tree equals the oracle's."""
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


class Pair:
    """A GPU tree and an oracle tree driven through the same batches."""

    def __init__(self, X, ids, p):
        pkd = _pkd()
        self.p = p
        self.g = pkd.Tree(to_dev(X), ids_dev(ids), p)
        self.o = O.OracleTree(X, ids, oparams(p))
        self.xyz = {int(i): tuple(x) for i, x in zip(ids, X.tolist())}

    def insert(self, Y, yid):
        self.g.insert(to_dev(Y), ids_dev(yid))
        self.o.insert(Y, yid)
        self.xyz.update({int(i): tuple(x) for i, x in zip(yid, Y.tolist())})
        self.check("insert")

    def delete(self, zid):
        nd = self.g.delete(ids_dev(zid))
        assert nd == self.o.delete(zid)
        self.check("delete")
        for i in zid:
            self.xyz.pop(int(i), None)
        return nd

    def check(self, what):
        assert self.g.size == self.o.size, what
        U.assert_exports_equal(self.g.export(), self.o.export())


def _ids(n, base=0):
    return (np.arange(base, base + n, dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32)


@pytest.mark.parametrize("kind", ["uniform", "varden"])
def test_insert_delete_small_tree(kind):
    pkd = _pkd()
    d = 2
    X = make_points(kind, 2000, d, 11)
    pr = Pair(X, _ids(2000), pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4))
    pr.insert(make_points(kind, 500, d, 12), _ids(500, 2000))
    live = np.array(sorted(pr.xyz))
    sel = live[I.sample_indices(600, len(live), 13)]
    assert pr.delete(sel) == 600


@pytest.mark.parametrize("sieve_kernel", [0, 1, 2], ids=["stream", "tiles", "stream-rewalk"])
@pytest.mark.parametrize("alpha", [(3, 10), (0, 1), (1, 2), (1, 10)])
def test_update_sequences_forced_rounds(alpha, sieve_kernel):
    pkd = _pkd()
    d, n = 3, 20000
    X = make_points("uniform", n, d, 21)
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4, alpha_num=alpha[0], alpha_den=alpha[1])
    with knobs(base_cap=256, skel_cap=64, tile=512, sieve_kernel=sieve_kernel):
        pr = Pair(X, _ids(n), p)
        nxt = n
        rng = np.random.default_rng(5)
        for r in range(3):
            Y = make_points("uniform", 3000, d, 30 + r)
            Y[:2000, 0] //= 64  # skewed: forces rebuilds on the left
            pr.insert(Y, _ids(3000, nxt))
            nxt += 3000
            live = np.array(sorted(pr.xyz))
            sel = rng.choice(live, 2500, replace=False)
            # repeats, and ids that name nothing (never inserted)
            zid = np.concatenate([sel, sel[:100], sel[100:150], _ids(50, 10 ** 8)]).astype(np.uint32)
            assert pr.delete(rng.permutation(zid)) == 2500


def test_heavy_leaves_and_duplicates():
    pkd = _pkd()
    d, n = 2, 8000
    X = make_points("dups", n, d, 41)  # coordinates in {0..4}^2: heavy leaves
    pr = Pair(X, _ids(n), pkd.Params(d=d, phi=16, lam=4, sigma_log2=2, sigma_os=4))
    Y = make_points("dups", 3000, d, 42)
    pr.insert(Y, _ids(3000, n))
    zid = np.concatenate([_ids(1000), _ids(500, n)])
    assert pr.delete(zid) == 1500


def test_empty_tree_grow_and_delete_everything():
    pkd = _pkd()
    d = 3
    p = pkd.Params(d=d, phi=32)
    pr = Pair(np.zeros((0, d), np.int32), np.zeros(0, np.uint32), p)
    Y = make_points("uniform", 20000, d, 51)  # larger than the initial arena: it must grow
    pr.insert(Y, _ids(20000))
    assert pr.delete(_ids(20000)) == 20000
    assert pr.g.size == 0
    pr.insert(Y[:100], _ids(100))


def test_config2_scaled_uniform_and_varden():
    # the 1e8-point build-and-update workload at 1/100 scale: 1e6 points d=3, insert 1e5 new
    # points, delete 1e5 random existing ids, alpha = 3/10, default params
    pkd = _pkd()
    d, n, m = 3, 1_000_000, 100_000
    for kind, seed in (("uniform", 1), ("varden", 11)):
        X = I.points(kind, n, d, seed)
        pr = Pair(X, np.arange(n, dtype=np.uint32), pkd.Params(d=d))
        Y = I.points(kind, m, d, 3 + seed)
        pr.insert(Y, np.arange(n, n + m, dtype=np.uint32))
        sel = I.sample_indices(m, n + m, 4)
        assert pr.delete(sel.astype(np.uint32)) == m


def test_flatten_overflow_is_redone_with_room():
    # The lists that flatten the rebuilt subtrees start at 64 entries: the
    # skewed batches below rebuild interior subtrees far larger than that, so
    # the first attempt overflows and the update redoes the flatten with room
    # for every node; the trees still match the oracle.
    pkd = _pkd()
    d, n = 3, 200_000
    X = make_points("uniform", n, d, 61)
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4)
    pr = Pair(X, _ids(n), p)
    Y = make_points("uniform", 40_000, d, 62)
    Y[:, 0] //= 64  # a slab of new points: interior subtrees become unbalanced
    pkd.pkd_kernel_timing(True)
    try:
        with knobs(front_cap=64):
            pr.insert(Y, _ids(40_000, n))
            pr.delete(_ids(60_000))
        retries = pkd.pkd_kernel_stats("front_retries")[0]
    finally:
        pkd.pkd_kernel_timing(False)
    assert retries >= 1


def test_delete_scratch_recycled_between_trees():
    # Trees of 4e6 points built and freed one after the other, each deleting
    # a batch: a released tree's per-slot delete scratch (all zero again
    # after every delete) goes back to the block cache as zeroed, and a later
    # tree's first delete may take it without a fill.  Every tree matches
    # the oracle.
    pkd = _pkd()
    d, n, m = 3, 4_000_000, 200_000
    p = pkd.Params(d=d)
    pkd.pkd_kernel_timing(True)
    try:
        for seed in (21, 22, 23):
            X = I.points("uniform", n, d, seed)
            ids = np.arange(n, dtype=np.uint32)
            t = pkd.Tree(to_dev(X), ids_dev(ids), p)
            o = O.OracleTree(X, ids, oparams(p))
            zid = I.sample_indices(m, n, seed + 5).astype(np.uint32)
            assert t.delete(ids_dev(zid)) == o.delete(zid)
            U.assert_exports_equal(t.export(), o.export())
            t.close()
        reused = pkd.pkd_kernel_stats("scratch_zeroed")[0]
    finally:
        pkd.pkd_kernel_timing(False)
    print("zeroed scratch taken by", reused, "of 2 later trees")


def _rejects(fn):
    pkd = _pkd()
    with pytest.raises(pkd.PkdError) as e:
        fn()
    assert e.value.code == pkd.PKD_EINVAL


def test_id_rules_match_the_oracle():
    # ids name points: repeated or reserved ids are rejected (builds), a batch
    # that names a stored point or repeats an id is rejected whole (inserts);
    # deletes skip ids that name nothing, repeats and deleted ids; a deleted
    # id may come back with new coordinates
    pkd = _pkd()
    d, n = 3, 6000
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4)
    X = make_points("uniform", n, d, 61)
    ids = _ids(n)
    _rejects(lambda: pkd.Tree(to_dev(X), ids_dev(np.r_[ids[:-1], ids[:1]]), p))
    _rejects(lambda: pkd.Tree(to_dev(X), ids_dev(np.r_[ids[:-1], [0xFFFFFFFF]]), p))
    pr = Pair(X, ids, p)
    before = pr.g.export()
    Y = make_points("uniform", 400, d, 62)
    for bad in (np.r_[_ids(399, n), ids[17:18]],            # a stored id
                np.r_[_ids(399, n), _ids(1, n + 5)],        # repeated in the batch
                np.r_[_ids(399, n), [0xFFFFFFFF]]):        # the reserved id
        _rejects(lambda: pr.g.insert(to_dev(Y), ids_dev(bad)))
        with pytest.raises(O.OracleError):
            pr.o.insert(Y, bad.astype(np.uint32))
        U.assert_exports_equal(pr.g.export(), before)
    pr.insert(Y, _ids(400, n))
    kill = np.r_[ids[::7], _ids(400, n)[::3]]
    assert pr.delete(np.r_[kill, kill[:50], [12345678, 0xFFFFFFFF]].astype(np.uint32)) == len(kill)
    assert pr.delete(kill[:100]) == 0  # deleted already
    Z = make_points("uniform", 100, d, 63)
    pr.insert(Z, kill[:100])  # deleted ids come back with new coordinates
    assert pr.delete(kill[:100]) == 100


def test_sparse_random_ids_and_table_growth():
    # labels drawn at random from the whole 32-bit range (the id table's
    # probing path), a tree that starts small and grows through many inserts
    pkd = _pkd()
    d = 2
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4)
    rng = np.random.default_rng(71)
    labels = rng.permutation(np.unique(rng.integers(0, 0xFFFFFFFF, size=70000, dtype=np.uint64)))[:60000]
    labels = labels.astype(np.uint32)
    X = make_points("varden", 1000, d, 72)
    pr = Pair(X, labels[:1000], p)
    at = 1000
    for r in range(5):
        m = 1000 * 3 ** r // 3 + 500
        Y = make_points("varden", m, d, 73 + r)
        pr.insert(Y, labels[at:at + m])
        at += m
        live = np.array(sorted(pr.xyz), dtype=np.uint32)
        pr.delete(rng.choice(live, len(live) // 4, replace=False))
