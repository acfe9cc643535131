"""pkd_knn_ids_noalloc: the k-NN entry point whose scratch is a fixed array
compiled into the library.  Its ids must equal pkd_knn's on the same tree and
queries, on consecutive calls (the scratch is reused, and the coordinate-check
flag in it must be cleared by every call), up to the stated maximum of q * k
pairs; larger batches are refused.  The file is named to be collected last, so
it also runs after every other GPU test in the same process."""
import numpy as np
import pytest

from paper_2411_09275_gb300 import inputs as I
from tests.gpuutil import ids_dev, make_points, to_dev

pytestmark = pytest.mark.gpu


def _pkd():
    from paper_2411_09275_gb300 import pkd

    return pkd


def _tree(d=3, n=60000, seed=81):
    pkd = _pkd()
    X = make_points("varden" if d == 3 else "uniform", n, d, seed)
    ids = (np.arange(n, dtype=np.uint64) * 7919 % (1 << 32)).astype(np.uint32)
    return pkd.Tree(to_dev(X), ids_dev(ids), pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8)), X


def _noalloc(t, Q, k):
    import torch

    pkd = _pkd()
    out = torch.full((Q.shape[0], k), -7, dtype=torch.int32, device=Q.device)
    pkd.pkd_knn_ids_noalloc(t._h, Q, k, out)
    return out


def test_noalloc_equals_knn_on_two_calls_in_a_row():
    t, X = _tree()
    Q1 = to_dev(np.concatenate([I.uniform(1500, 3, 82), X[:500]]))
    Q2 = to_dev(np.concatenate([X[1000:1700], I.uniform(2300, 3, 83)]))
    want1, _ = t.knn(Q1, 10)
    want2, _ = t.knn(Q2, 33)
    got1 = _noalloc(t, Q1, 10)
    got2 = _noalloc(t, Q2, 33)
    assert (got1 == want1).all().item()
    assert (got2 == want2).all().item()
    # the same batch again, after a different one, gives the same ids
    again = _noalloc(t, Q1, 10)
    assert (again == want1).all().item()


@pytest.mark.parametrize("d", [1, 5])
def test_noalloc_other_dimensions(d):
    t, X = _tree(d=d, n=20000, seed=84 + d)
    Q = to_dev(np.concatenate([I.uniform(700, d, 85), X[:300]]))
    for k in (1, 16, 128):
        want, _ = t.knn(Q, k)
        assert (_noalloc(t, Q, k) == want).all().item()


def test_noalloc_at_the_maximum_and_past_it():
    pkd = _pkd()
    t, _ = _tree()
    k = 16
    q = (1 << 20) // k  # PKD_NOALLOC_MAX_PAIRS of pkd.h, in (query, neighbour) pairs
    Q = to_dev(I.uniform(q, 3, 86))
    want, _ = t.knn(Q, k)
    assert (_noalloc(t, Q, k) == want).all().item()
    Q1 = to_dev(I.uniform(q + 1, 3, 87))
    with pytest.raises(pkd.PkdError) as e:
        _noalloc(t, Q1, k)
    assert e.value.code == pkd.PKD_EINVAL


def test_noalloc_rejects_bad_input_then_recovers():
    import torch

    pkd = _pkd()
    t, X = _tree()
    Q = to_dev(I.uniform(1000, 3, 88))
    want, _ = t.knn(Q, 5)
    bad = Q.clone()
    bad[417, 2] = 1 << 30
    for k in (0, 129):
        with pytest.raises(pkd.PkdError):
            _noalloc(t, Q, k)
    with pytest.raises(pkd.PkdError) as e:
        _noalloc(t, bad, 5)
    assert e.value.code == pkd.PKD_EINVAL
    # the flag set by the rejected batch must not leak into the next call
    assert (_noalloc(t, Q, 5) == want).all().item()
    empty = torch.empty((0, 3), dtype=torch.int32, device=Q.device)
    assert _noalloc(t, empty, 5).numel() == 0


_FRESH = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2411_09275_gb300 import inputs as I, pkd

dev = torch.device("cuda:0")
pkd.lib()
trees, queries = {}, {}
for d in (3, 8):
    X = I.uniform(30000, d, 90 + d)
    trees[d] = pkd.Tree(torch.from_numpy(X).to(dev), None, pkd.Params(d=d, phi=16, lam=4, sigma_log2=3, sigma_os=8))
    queries[d] = torch.from_numpy(np.concatenate([I.uniform(1000, d, 95 + d), X[:200]])).to(dev)
out3 = torch.empty((1200, 5), dtype=torch.int32, device=dev)
out8 = torch.empty((1200, 128), dtype=torch.int32, device=dev)
torch.cuda.synchronize()
# first call on the device: the set-up (d = 3, k = 5 uses the small-k kernel only)
pkd.pkd_knn_ids_noalloc(trees[3]._h, queries[3], 5, out3)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
alloc0 = pkd.pkd_kernel_stats("allocations")[0]
# first d = 8, k = 128 search of the process: a kernel with far more local memory
pkd.pkd_knn_ids_noalloc(trees[8]._h, queries[8], 128, out8)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
alloc1 = pkd.pkd_kernel_stats("allocations")[0]
want, _ = trees[8].knn(queries[8], 128)
torch.cuda.synchronize()
ok = bool((want == out8).all().item())
print("RESULT", free0, free1, alloc0, alloc1, ok)
'''


def test_noalloc_call_allocates_nothing_after_its_set_up():
    # in a fresh process, so that no earlier test has loaded the kernels or
    # grown the local-memory reservation: after the set-up call, a call that
    # uses a kernel never launched before in the process (d = 8, k = 128)
    # leaves the device's free memory and the library's allocation count
    # unchanged, and returns pkd_knn's ids
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")]
    assert r.returncode == 0 and line, r.stdout[-2000:] + r.stderr[-2000:]
    _, free0, free1, alloc0, alloc1, ok = line[0].split()
    assert ok == "True"
    assert int(alloc1) == int(alloc0), (alloc0, alloc1)
    assert int(free1) == int(free0), (free0, free1)
