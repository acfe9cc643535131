"""Failure detection without a GPU fault (host-side fault injection):

- out of device memory: the library's allocations are made to fail after k
  successful ones (option fail_alloc_after), for every k until the call
  succeeds; every failing insert or delete returns PKD_ENOMEM and leaves the
  tree exactly as it was (same export, same size, still usable), and the
  final successful call gives the oracle's tree;
- a device-side wait that runs out: the limit of the streaming sieve's
  mbarrier waits (option wait_cycles) is set to 0, so the first wait that
  is not already satisfied gives up; the call returns PKD_ETIMEOUT (the
  kernels that would consume the unfinished counts do nothing), and a fresh
  tree built afterwards with the default limit is correct."""
import numpy as np
import pytest

import oracle as O
from tests import treeutil as U
from tests.gpuutil import ids_dev, knobs, make_points, oparams, to_dev

pytestmark = pytest.mark.gpu

FORCED = dict(base_cap=256, skel_cap=64, tile=512)  # sieve rounds and skeleton jobs on a small input


def _pkd():
    from paper_2411_09275_gb300 import pkd

    return pkd


def _sweep_until_success(call, t, before):
    """Run call() with fail_alloc_after = 0, 1, 2, ... until it succeeds;
    returns the number of failures seen (all PKD_ENOMEM, tree unchanged)."""
    pkd = _pkd()
    fails = 0
    for k in range(0, 2000):
        try:
            with knobs(fail_alloc_after=k):
                call()
            return fails
        except pkd.PkdError as e:
            assert e.code == pkd.PKD_ENOMEM, (k, e.code)
            fails += 1
            U.assert_exports_equal(t.export(), before)
    raise AssertionError("the call never succeeded")


@pytest.mark.parametrize("kind", ["uniform", "varden"])
def test_out_of_memory_leaves_the_tree_unchanged(kind):
    pkd = _pkd()
    d, n = 3, 20000
    X = make_points(kind, n, d, 401)
    ids = np.arange(n, dtype=np.uint32)
    p = pkd.Params(d=d, phi=8, lam=3, sigma_log2=2, sigma_os=4)
    with knobs(**FORCED):
        # a build that cannot allocate makes no tree
        with knobs(fail_alloc_after=3):
            with pytest.raises(pkd.PkdError) as e:
                pkd.Tree(to_dev(X), ids_dev(ids), p)
        assert e.value.code == pkd.PKD_ENOMEM
        t = pkd.Tree(to_dev(X), ids_dev(ids), p)
        o = O.OracleTree(X, ids, oparams(p))
        Y = make_points(kind, 4000, d, 402)
        Y[:3000, 0] //= 32  # skewed: subtrees are rebuilt, not only leaves
        yid = np.arange(n, n + 4000, dtype=np.uint32)
        fails = _sweep_until_success(lambda: t.insert(to_dev(Y), ids_dev(yid)), t, t.export())
        assert fails > 5  # allocations before, inside and after the routing rounds all failed once
        o.insert(Y, yid)
        U.assert_exports_equal(t.export(), o.export())
        kill = np.concatenate([np.arange(0, n, 3), yid[:2500]]).astype(np.uint32)
        fails = _sweep_until_success(lambda: t.delete(ids_dev(kill)), t, t.export())
        assert fails > 5
        o.delete(kill)
        U.assert_exports_equal(t.export(), o.export())
        assert t.size == o.size
        t.close()


def test_wait_timeout_is_reported_and_a_fresh_tree_is_correct():
    pkd = _pkd()
    d, n = 3, 300000
    X = make_points("uniform", n, d, 411)
    p = pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)
    with knobs(**FORCED):
        with knobs(wait_cycles=0):
            with pytest.raises(pkd.PkdError) as e:
                pkd.Tree(to_dev(X), None, p)
        assert e.value.code == pkd.PKD_ETIMEOUT
        t = pkd.Tree(to_dev(X), None, p)
        Y = make_points("uniform", 50000, d, 412)
        yid = np.arange(n, n + 50000, dtype=np.uint32)
        with knobs(wait_cycles=0):
            with pytest.raises(pkd.PkdError) as e:
                t.insert(to_dev(Y), ids_dev(yid))
        assert e.value.code == pkd.PKD_ETIMEOUT
        t.close()  # a tree whose wait ran out is freed
        t = pkd.Tree(to_dev(X), None, p)
        U.assert_exports_equal(t.export(), O.OracleTree(X, None, oparams(p)).export())
        t.close()
