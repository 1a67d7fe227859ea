"""Host logic of the cavity stability sweep (no GPU): the threshold search on the tau grid
1/2 + k dtau against fake stability oracles."""
from types import SimpleNamespace

import pytest

from paper_2410_09739_gb300 import cavity_study as S


class FakeProber:
    def __init__(self, stable_fn):
        self.fn = stable_fn
        self.calls = []

    def stable(self, tau):
        self.calls.append(tau)
        return self.fn(tau)


ARGS = SimpleNamespace(dtau=5e-5, tau_hi=0.52, verify=10)


def k_of(tau):
    return round((tau - 0.5) / ARGS.dtau)


@pytest.mark.parametrize("k_star", [2, 17, 399, 400, 401, 1234])
def test_monotone_threshold_is_found_exactly(k_star):
    p = FakeProber(lambda t: k_of(t) >= k_star)
    tau, note = S.threshold(p, ARGS)
    assert note == "ok" and k_of(tau) == k_star
    assert len(p.calls) < 40  # bisection, not a scan


def test_isolated_stable_point_below_the_threshold_is_rejected():
    # k = 300 (the bisection's second probe) is stable by chance; the threshold is 350
    p = FakeProber(lambda t: k_of(t) == 300 or k_of(t) >= 350)
    tau, _ = S.threshold(p, ARGS)
    assert 0.5 + 300 * ARGS.dtau in p.calls
    assert k_of(tau) == 350


def test_stable_everywhere_and_nowhere():
    assert S.threshold(FakeProber(lambda t: True), ARGS)[1] == "stable at the smallest tau tried"
    tau, note = S.threshold(FakeProber(lambda t: False), ARGS)
    assert tau is None and "no stable" in note
