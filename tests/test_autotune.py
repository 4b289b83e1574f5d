"""The tile-shape autotuner: candidate shapes fit the grid, and tuning a
small workload returns one of them with a positive step time (the deposit
integers do not depend on the tile shape, see test_parity_gpu)."""
import pytest

from paper_1908_10793_gb300 import inputs as I


def test_candidates_fit_the_grid():
    from paper_1908_10793_gb300 import autotune
    for w in (I.sbox3d("small"), I.box2d("small"), I.si2d_instance(0), I.cyldisk("small")):
        cands = autotune.candidate_tiles(w)
        assert cands and len(set(cands)) == len(cands)
        for t in cands:
            for d in range(3):
                assert 1 <= t[d] <= max(1, w.n[d])
                if w.n[d] == 1:
                    assert t[d] == 1


@pytest.mark.gpu
def test_tuning_returns_a_timed_candidate():
    from paper_1908_10793_gb300 import autotune
    w = I.si2d_instance(2, "small")
    best, times = autotune.tune_tile(w, steps=2)
    assert best in autotune.candidate_tiles(w)
    assert times[best] == min(times.values()) and all(t > 0 for t in times.values())


def test_batch_candidates_start_with_the_default_and_cover_modes():
    from paper_1908_10793_gb300 import autotune
    ws = [I.si2d_instance(k, "small") for k in range(3)]
    cands = autotune.batch_candidates(ws)
    assert cands[0] == (None, 1, 0)
    assert len(set(cands)) == len(cands)
    assert {m for _, _, m in cands} == {0, 1}
    # the graph path sorts every step
    assert all(k == 1 for _, k, m in cands if m == 1)
    assert {k for _, k, m in cands if m == 0} == {1, 2}
