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

    def delete(self, Z, zid):
        nd = self.g.delete(to_dev(Z), ids_dev(zid))
        assert nd == self.o.delete(Z, zid)
        self.check("delete")
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
    Z = np.array([pr.xyz[int(i)] for i in sel], np.int32)
    assert pr.delete(Z, sel) == 600


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
            Z = np.array([pr.xyz[int(i)] for i in sel], np.int32)
            Z = np.concatenate([Z, Z[:100], Z[100:150] + 1])  # duplicates and absent points
            zid = np.concatenate([sel, sel[:100], sel[100:150]]).astype(np.uint32)
            assert pr.delete(Z, zid) == 2500
            for i in sel:
                del pr.xyz[int(i)]


def test_heavy_leaves_and_duplicates():
    pkd = _pkd()
    d, n = 2, 8000
    X = make_points("dups", n, d, 41)  # coordinates in {0..4}^2: heavy leaves
    pr = Pair(X, _ids(n), pkd.Params(d=d, phi=16, lam=4, sigma_log2=2, sigma_os=4))
    Y = make_points("dups", 3000, d, 42)
    pr.insert(Y, _ids(3000, n))
    Z = np.concatenate([X[:1000], Y[:500]])
    zid = np.concatenate([_ids(1000), _ids(500, n)])
    assert pr.delete(Z, zid) == 1500


def test_empty_tree_grow_and_delete_everything():
    pkd = _pkd()
    d = 3
    p = pkd.Params(d=d, phi=32)
    pr = Pair(np.zeros((0, d), np.int32), np.zeros(0, np.uint32), p)
    Y = make_points("uniform", 20000, d, 51)  # larger than the initial arena: it must grow
    pr.insert(Y, _ids(20000))
    assert pr.delete(Y, _ids(20000)) == 20000
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
        allX = np.concatenate([X, Y])
        assert pr.delete(allX[sel], sel) == m
