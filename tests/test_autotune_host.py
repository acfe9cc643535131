"""Host logic of the autotuner (no GPU): the candidate grid respects the
library's parameter ranges and the choice is the fastest, with a
reproducible tie-break."""
import pytest

from paper_2411_09275_gb300 import autotune as A


def test_grid_is_the_cartesian_product_in_range():
    g = A.grid((5, 6), (6, 7, 8), (1024, 2048))
    assert len(g) == 12 and len(set(g)) == 12
    assert all(1 <= c.lam <= 10 and 0 <= c.sigma_log2 <= 30 and c.tile in (1024, 2048) for c in g)
    with pytest.raises(ValueError):
        A.grid((11,), (6,), (2048,))
    with pytest.raises(ValueError):
        A.grid((6,), (6,), (3000,))
    with pytest.raises(ValueError):
        A.grid((6,), (6,), (2048,), phis=(0,))
    with pytest.raises(ValueError):
        A.grid((6,), (6,), (2048,), base_caps=(32,))
    g = A.grid((6,), (6,), (2048,), phis=(16, 32), base_caps=(0, 1024))
    assert len(g) == 4 and {(c.phi, c.base_cap) for c in g} == {(16, 0), (16, 1024), (32, 0), (32, 1024)}


def test_pick_fastest_then_smallest_parameters():
    c1, c2, c3 = A.Candidate(6, 6, 2048), A.Candidate(5, 7, 4096), A.Candidate(7, 5, 1024)
    assert A.pick({c1: 3.0, c2: 2.0, c3: 2.5}) == c2
    assert A.pick({c1: 2.0, c2: 2.0, c3: 2.0}) == A.Candidate(5, 7, 4096)


def test_candidate_params_carry_the_choice():
    p = A.Candidate(7, 5, 1024, phi=16).params(3)
    assert (p.d, p.lam, p.sigma_log2, p.phi) == (3, 7, 5, 16)
