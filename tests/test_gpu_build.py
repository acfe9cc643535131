"""GPU parity of the build path (Alg. 1): the canonical export of the tree
built by the CUDA kernels (through the C ABI) must equal the CPU oracle's,
byte for byte (splitters in pre-order, sizes, sorted leaf id sets)."""
import numpy as np
import pytest

import oracle as O
from tests import treeutil as U
from tests.gpuutil import ids_dev, knobs, make_points, oparams, to_dev

pytestmark = pytest.mark.gpu


def _pkd():
    from paper_2411_09275_gb300 import pkd

    return pkd


CASES = [
    # (name, n, d, kind, params overrides, knobs)
    ("base-only-2d", 1000, 2, "uniform", {}, {}),
    ("base-skeleton-levels", 6000, 3, "varden", dict(phi=8, lam=3, sigma_log2=2, sigma_os=4), {}),
    ("rounds-2d", 20000, 2, "uniform", dict(phi=16, lam=4, sigma_log2=2, sigma_os=8),
     dict(base_cap=256, skel_cap=64)),
    ("rounds-3d-varden", 30000, 3, "varden", dict(phi=8, lam=3, sigma_log2=1, sigma_os=4),
     dict(base_cap=512, skel_cap=128)),
    ("rounds-dups-heavy", 20000, 2, "dups", dict(phi=4, lam=2, sigma_log2=3, sigma_os=2),
     dict(base_cap=256, skel_cap=64)),
    ("rounds-half-identical", 20000, 3, "dups_big", dict(phi=16, lam=5, sigma_log2=3, sigma_os=4),
     dict(base_cap=256, skel_cap=64)),
    ("rounds-line", 20000, 3, "line", dict(phi=16, lam=6, sigma_log2=2, sigma_os=8),
     dict(base_cap=256)),
    ("count-mode", 40000, 2, "uniform", dict(phi=8, lam=4, sigma_os=8, count_mode=1),
     dict(base_cap=1024, skel_cap=256)),
    ("d1", 20000, 1, "uniform", dict(phi=8, lam=5, sigma_log2=2, sigma_os=4), dict(base_cap=512)),
    ("d5", 20000, 5, "uniform", dict(phi=8, lam=3, sigma_log2=2, sigma_os=4), dict(base_cap=512)),
    ("d8", 20000, 8, "varden", dict(phi=8, lam=3, sigma_log2=2, sigma_os=4), dict(base_cap=512)),
    ("lambda10", 60000, 2, "uniform", dict(phi=4, lam=10, sigma_log2=0, sigma_os=4),
     dict(base_cap=2048, skel_cap=1024)),
    ("lambda8-256-buckets", 60000, 3, "varden", dict(phi=4, lam=8, sigma_log2=0, sigma_os=4),
     dict(base_cap=2048, skel_cap=1024)),
    ("sample-all-tiles", 50000, 2, "uniform", dict(phi=32, lam=6, sigma_log2=0, sigma_os=32),
     dict(base_cap=1024, tile=512)),
    ("defaults-100k", 100000, 2, "uniform", {}, {}),
    ("defaults-forced-rounds", 100000, 3, "uniform", {}, dict(base_cap=1024, skel_cap=256)),
]


# graph_rounds 1: every round decided on the device (one graph launch);
# 0: the same kernels sequenced by the host
@pytest.mark.parametrize("base_kernel,sieve_kernel,graph_rounds", [(0, 0, 1), (0, 2, 1), (1, 1, 1), (0, 0, 0), (1, 1, 0)],
                         ids=["sorted-stream", "sorted-stream-rewalk", "select-tiles", "sorted-stream-host",
                              "select-tiles-host"])
@pytest.mark.parametrize("name,n,d,kind,over,kn", CASES, ids=[c[0] for c in CASES])
def test_build_matches_oracle(name, n, d, kind, over, kn, base_kernel, sieve_kernel, graph_rounds):
    pkd = _pkd()
    X = make_points(kind, n, d, 1000 + n + d)
    ids = ((np.arange(n, dtype=np.uint64) * 2654435761) % (1 << 32)).astype(np.uint32)
    p = pkd.Params(d=d, seed=42, **over)
    g0 = pkd.pkd_kernel_stats("graph_builds")[0]
    with knobs(base_kernel=base_kernel, sieve_kernel=sieve_kernel, graph_rounds=graph_rounds, **kn):
        t = pkd.Tree(to_dev(X), ids_dev(ids), p)
        got = t.export()
    want = O.OracleTree(X, ids, oparams(p)).export()
    U.assert_exports_equal(got, want)
    assert t.size == n
    # the build's rounds ran from one graph launch exactly when asked
    assert pkd.pkd_kernel_stats("graph_builds")[0] - g0 == graph_rounds
    t.close()


@pytest.mark.parametrize("n", [0, 1, 2, 32, 33, 65, 1000])
def test_build_tiny_sizes(n):
    pkd = _pkd()
    d = 2
    X = make_points("uniform", max(n, 1), d, 7)[:n]
    p = pkd.Params(d=d)
    t = pkd.Tree(to_dev(X.reshape(n, d)), None, p)
    U.assert_exports_equal(t.export(), O.OracleTree(X.reshape(n, d), None, oparams(p)).export())
    t.close()


def test_build_rejects_bad_input():
    pkd = _pkd()
    X = np.zeros((10, 2), np.int32)
    X[3, 1] = 1 << 30
    with pytest.raises(pkd.PkdError) as e:
        pkd.Tree(to_dev(X), None, pkd.Params(d=2))
    assert e.value.code == pkd.PKD_EINVAL
    with pytest.raises(pkd.PkdError):
        pkd.Tree(to_dev(np.zeros((10, 2), np.int32)), None, pkd.Params(d=2, alpha_num=4, alpha_den=5))


def test_build_deterministic_and_config1():
    # n = 1e6, d = 2 uniform in [0, 2^30), phi 32, lambda 6, rate 1/64.
    pkd = _pkd()
    from paper_2411_09275_gb300 import inputs as I

    X = I.uniform(1_000_000, 2, 1)
    p = pkd.Params(d=2)
    a = pkd.Tree(to_dev(X), None, p).export()
    b = pkd.Tree(to_dev(X), None, p).export()
    U.assert_exports_equal(a, b)
    U.assert_exports_equal(a, O.OracleTree(X, None, oparams(p)).export())


@pytest.mark.parametrize("n", [1, 3, 6, 37, 1000, 100003])
def test_build_validation_every_position_and_alignment(n):
    # The range check reads a scalar head up to a 16-byte boundary, 16-byte
    # vectors, then a scalar tail: a bad value is caught wherever it sits
    # and whatever the buffer's alignment; in-range extremes pass.
    import torch

    pkd = _pkd()
    d = 2
    base = make_points("uniform", n, d, 11).reshape(-1)
    base[0] = 0
    base[-1] = (1 << 30) - 1
    for off in range(4):
        buf = torch.zeros(n * d + 4, dtype=torch.int32, device="cuda")
        view = buf[off:off + n * d]
        view.copy_(torch.from_numpy(base))
        t = pkd.Tree(view.view(n, d), None, pkd.Params(d=d))
        assert t.size == n
        t.close()
        for pos in sorted({0, 1, 2, 3, n * d // 2, n * d - 2, n * d - 1} & set(range(n * d))):
            for bad in (-1, 1 << 30, -(1 << 31)):
                view.copy_(torch.from_numpy(base))
                view[pos] = bad
                with pytest.raises(pkd.PkdError) as e:
                    pkd.Tree(view.view(n, d), None, pkd.Params(d=d))
                assert e.value.code == pkd.PKD_EINVAL


def test_recorded_build_graph_relaunched_on_new_data():
    """A build whose arguments all equal an earlier build's (same input
    buffer, same sizes: the pool tends to hand out the same scratch) launches
    the earlier build's graph again; the graph reads the data at run time, so
    new coordinates in the same buffer still give the oracle's tree."""
    import torch

    pkd = _pkd()
    n, d = 60000, 3
    p = pkd.Params(d=d, phi=8, lam=4, sigma_log2=2, sigma_os=4)
    buf = torch.empty((n, d), dtype=torch.int32, device="cuda")
    reused = 0
    with knobs(base_cap=1024, skel_cap=256):
        for r in range(4):
            X = make_points("varden" if r % 2 else "uniform", n, d, 900 + r)
            buf.copy_(torch.from_numpy(X))
            g0, u0 = pkd.pkd_kernel_stats("graph_builds")[0], pkd.pkd_kernel_stats("graph_builds")[2]
            t = pkd.Tree(buf, None, p)
            g1, u1 = pkd.pkd_kernel_stats("graph_builds")[0], pkd.pkd_kernel_stats("graph_builds")[2]
            assert g1 - g0 == 1
            reused += u1 - u0
            U.assert_exports_equal(t.export(), O.OracleTree(X, None, oparams(p)).export())
            t.close()
    # the same sizes four times: at least one build found its graph recorded
    assert reused >= 1


def test_recorded_graphs_evicted_and_relaunched_stay_correct():
    """More distinct build shapes than the recorded-graph cache holds (16):
    every build records or relaunches a graph, evicted graphs are destroyed
    only once their launches have completed, and every tree still equals
    the oracle's."""
    pkd = _pkd()
    d = 2
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4)
    sizes = [3000 + 1700 * i for i in range(20)]
    with knobs(base_cap=256, skel_cap=64):
        for rep in range(2):
            for i, n in enumerate(sizes):
                if rep and i % 3:
                    continue
                X = make_points("varden" if i % 2 else "uniform", n, d, 4000 + n)
                t = pkd.Tree(to_dev(X), None, p)
                U.assert_exports_equal(t.export(), O.OracleTree(X, None, oparams(p)).export())
                t.close()
