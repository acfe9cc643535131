"""Freeing a tree is ordered after the work queued on it, not after the
whole device: pkd_free records nothing itself, it makes the legacy default
stream wait for the last use of the tree on every stream a call used (an
event each call records) and frees there.  A long k-NN batch queued on a side
stream, the tree freed at once and a new tree built in the same memory on
another stream: the batch's answers are still the first tree's."""
import numpy as np
import pytest

import oracle as O
from paper_2411_09275_gb300 import inputs as I
from tests.gpuutil import oparams, to_dev

pytestmark = pytest.mark.gpu


def test_free_waits_for_queries_in_flight_on_other_streams():
    import torch

    from paper_2411_09275_gb300 import pkd

    n, d, k = 400_000, 3, 64
    p = pkd.Params(d=d)
    X = I.uniform(n, d, 301)
    Q = I.uniform(200_000, d, 302)
    gX, gQ = to_dev(X), to_dev(Q)
    side = torch.cuda.Stream()
    t = pkd.Tree(gX, None, p)
    torch.cuda.synchronize()
    oi = torch.empty((len(Q), k), dtype=torch.int32, device="cuda")
    od = torch.empty((len(Q), k), dtype=torch.int64, device="cuda")
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        pkd.pkd_knn(t._h, gQ, k, oi, od, side)
    t.close()  # returns at once; the memory is released after the batch
    X2 = I.uniform(n, d, 303)
    t2 = pkd.Tree(to_dev(X2), None, p)  # same sizes: the pool hands out the same blocks
    torch.cuda.synchronize()
    wi, wd = O.OracleTree(X, None, oparams(p)).knn(Q[:2000], k)
    assert np.array_equal(od[:2000].cpu().numpy(), wd)
    assert np.array_equal(oi[:2000].cpu().numpy().view(np.uint32), wi)
    t2.close()
