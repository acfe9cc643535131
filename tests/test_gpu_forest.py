"""GPU parity of the batched build (pkd_build_forest): every tree of a
forest, built in one pass with the others, equals the oracle's build of that
tree's points alone (canonical export byte for byte), and k-NN on a forest
tree equals the oracle's."""
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


def _forest_inputs(sizes, d, kind, seed):
    X = make_points(kind, int(sum(sizes)), d, seed) if sum(sizes) else np.zeros((0, d), np.int32)
    ids = ((np.arange(len(X), dtype=np.uint64) * 2654435761 + 17) % (1 << 32)).astype(np.uint32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    return X, ids, off


CASES = [
    # (name, sizes, d, kind, params overrides, knobs)
    ("mixed-defaults", [0, 1, 2, 33, 200, 1000, 5000, 30000, 0, 7, 12000], 3, "uniform", {}, {}),
    ("mixed-forced-rounds", [20000, 3, 0, 700, 15000, 64, 9000], 2, "varden",
     dict(phi=8, lam=3, sigma_log2=2, sigma_os=4), dict(base_cap=256, skel_cap=64)),
    ("duplicates", [5000, 2000, 40], 3, "dups", dict(phi=4, lam=2, sigma_log2=3, sigma_os=2),
     dict(base_cap=512)),
    ("many-small", [int(x) for x in np.random.default_rng(21).integers(0, 400, 300)], 3, "uniform", {}, {}),
]


@pytest.mark.parametrize("graph_rounds", [1, 0], ids=["device-rounds", "host-rounds"])
@pytest.mark.parametrize("name,sizes,d,kind,over,kn", CASES, ids=[c[0] for c in CASES])
def test_forest_trees_match_their_own_oracle_builds(name, sizes, d, kind, over, kn, graph_rounds):
    pkd = _pkd()
    X, ids, off = _forest_inputs(sizes, d, kind, 500 + len(sizes))
    p = pkd.Params(d=d, seed=7, **over)
    g0 = pkd.pkd_kernel_stats("graph_builds")[0]
    with knobs(graph_rounds=graph_rounds, **kn):
        f = pkd.pkd_build_forest(to_dev(X), ids_dev(ids), off, p)
    # every tree's rounds, as extra roots of one build, ran from one graph
    # launch with no host synchronisation between rounds (device rounds)
    assert pkd.pkd_kernel_stats("graph_builds")[0] - g0 == graph_rounds
    try:
        assert pkd.lib().pkd_forest_trees(f) == len(sizes)
        for t in range(len(sizes)):
            a, b = int(off[t]), int(off[t + 1])
            assert pkd.lib().pkd_forest_size(f, t) == b - a
            want = O.OracleTree(X[a:b], ids[a:b], oparams(p)).export()
            U.assert_exports_equal(pkd.pkd_forest_export(f, t), want)
    finally:
        pkd.pkd_forest_free(f)


def test_forest_knn_matches_oracle():
    import torch

    pkd = _pkd()
    sizes = [3000, 0, 25000, 5]
    X, ids, off = _forest_inputs(sizes, 3, "varden", 77)
    p = pkd.Params(d=3)
    f = pkd.pkd_build_forest(to_dev(X), ids_dev(ids), off, p)
    try:
        Q = np.concatenate([I.uniform(300, 3, 78), X[:100]])
        for t, k in ((0, 10), (1, 3), (2, 33), (3, 8)):
            a, b = int(off[t]), int(off[t + 1])
            oi = torch.empty((len(Q), k), dtype=torch.int32, device="cuda")
            od = torch.empty((len(Q), k), dtype=torch.int64, device="cuda")
            pkd.pkd_forest_knn(f, t, to_dev(Q), k, oi, od)
            wi, wd = O.OracleTree(X[a:b], ids[a:b], oparams(p)).knn(Q, k)
            assert np.array_equal(od.cpu().numpy(), wd)
            assert np.array_equal(oi.cpu().numpy().view(np.uint32), wi)
    finally:
        pkd.pkd_forest_free(f)


def test_forest_rejects_bad_offsets():
    pkd = _pkd()
    X = make_points("uniform", 100, 2, 3)
    p = pkd.Params(d=2)
    lib = pkd.lib()
    import ctypes as C

    h = C.c_void_p()
    pc = p.c()
    for off in ([0, 60, 40, 100], [5, 50, 100]):
        o = np.asarray(off, np.uint64)
        r = lib.pkd_build_forest(pkd._dptr(to_dev(X)), None, o.ctypes.data_as(C.POINTER(C.c_uint64)), len(o) - 1,
                                 C.byref(pc), pkd._stream(None), C.byref(h))
        assert r == pkd.PKD_EINVAL
