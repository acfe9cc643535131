"""GPU check of the autotuner: it times real builds, and the tree built with
the parameters it chose equals the oracle's tree for those parameters."""
import pytest

import oracle as O
from tests import treeutil as U
from tests.gpuutil import make_points, oparams, to_dev

pytestmark = pytest.mark.gpu


def test_tune_then_build_with_choice_matches_oracle():
    from paper_2411_09275_gb300 import autotune as A
    from paper_2411_09275_gb300 import pkd

    X = make_points("varden", 60000, 2, 41)
    g = to_dev(X)
    res = A.tune(g, A.grid((4, 6), (3, 6), (1024, 2048), phis=(16, 32), base_caps=(0, 1024)), reps=1)
    assert len(res["table"]) == 32 and all(r["ms"] > 0 for r in res["table"])
    best = A.Candidate(**res["best"])
    assert res["table"][0]["ms"] == min(r["ms"] for r in res["table"])
    p = best.params(2)
    t = pkd.Tree(g, None, p)
    U.assert_exports_equal(t.export(), O.OracleTree(X, None, oparams(p)).export())
    t.close()
