"""Host logic of the bare-mass search (paper_1202_2462_gb300.tune.find_m0):
with sigma_min replaced by a known function of m0 (linear in the distance
to a critical mass on the physical side, overestimated by up to 10% as
inverse iteration overestimates it), the search lands within 25% of the
target, never steps past the critical mass, and stops with an error when
sigma_min rises instead of falling."""

import pytest

tune = pytest.importorskip("paper_1202_2462_gb300.tune")


class _Ctx:
    def close(self):
        pass


def _fake(monkeypatch, m_c, slope, over):
    seen = []

    def sigma(m0):
        return slope * abs(m0 - m_c)

    def fake_sigma_min(solver, shape, iters=12, seed=0):
        s = sigma(solver.m0) * (1.0 + over(len(seen)))
        seen.append(solver.m0)
        return [s]

    def make(m0):
        c = _Ctx()
        c.m0 = m0
        return c

    monkeypatch.setattr(tune, "sigma_min", fake_sigma_min)
    return make, seen, sigma


@pytest.mark.parametrize("slope,over", [(0.9, lambda k: 0.0), (1.1, lambda k: 0.1), (0.8, lambda k: 0.05 * (k % 2))])
def test_search_lands_near_the_target_on_the_physical_side(monkeypatch, slope, over):
    m_c, target = -0.98, 1e-3
    make, seen, sigma = _fake(monkeypatch, m_c, slope, over)
    m0, sig, pts = tune.find_m0(make, None, -0.85, target)
    assert all(m > m_c for m in seen)
    assert abs(sig - target) <= 0.25 * target
    assert sigma(m0) <= 1.25 * target and m0 > m_c
    assert len(pts) <= 8


def test_search_stops_when_sigma_rises(monkeypatch):
    # a start past the critical mass: moving "towards" it raises sigma_min
    make, seen, _ = _fake(monkeypatch, -0.98, 0.9, lambda k: 0.0)
    with pytest.raises(RuntimeError, match="did not fall"):
        tune.find_m0(make, None, -1.2, 1e-3)
