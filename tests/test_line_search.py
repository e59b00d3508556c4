"""The Hager-Zhang line search of the reconstruction driver (Sec. 6 uses it for mu_a) on 1-D
functions whose minimisers are known: the accepted step meets the Wolfe or the approximate Wolfe
conditions, the bracketing phase grows a tiny first trial and bisection shrinks a huge one, and
an exhausted budget falls back to the best step with a sufficient decrease."""
import math

import pytest

from paper_1608_05238_gb300.inversion import HZParams, hager_zhang


def _conditions(f0, g0, a, fa, ga, p):
    wolfe = fa - f0 <= p.delta * a * g0 and ga >= p.sigma * g0
    approx = (2 * p.delta - 1) * g0 >= ga >= p.sigma * g0 and fa <= f0 + p.epsilon * abs(f0)
    return wolfe or approx


def _counted(fn):
    calls = []

    def phi(a):
        calls.append(a)
        return fn(a)
    return phi, calls


CASES = [
    # phi(a), phi'(a), minimiser
    (lambda a: ((a - 3.0) ** 2 - 9.0, 2 * (a - 3.0)), 3.0),
    (lambda a: (math.exp(a) - 5.0 * a, math.exp(a) - 5.0), math.log(5.0)),
    (lambda a: ((a - 0.02) ** 4 - 0.02 ** 4 - 1e-3 * a, 4 * (a - 0.02) ** 3 - 1e-3), None),
    (lambda a: (-a / (1 + a * a), -(1 - a * a) / (1 + a * a) ** 2), 1.0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("c", [1e-4, 0.5, 40.0])
def test_accepted_step_meets_the_wolfe_conditions(case, c):
    fn, _ = CASES[case]
    p = HZParams(max_evals=40)
    f0, g0 = fn(0.0)
    assert g0 < 0
    phi, calls = _counted(lambda a: fn(a))
    a, fa, ga, n = hager_zhang(phi, f0, g0, c, p)
    assert a is not None and a > 0 and n == len(calls) <= p.max_evals
    assert (fa, ga) == fn(a)
    assert _conditions(f0, g0, a, fa, ga, p), (a, fa, ga)
    assert fa < f0


def test_exact_first_trial_is_accepted_at_once():
    fn, a_star = CASES[0]
    phi, calls = _counted(fn)
    a, _, _, n = hager_zhang(phi, *fn(0.0), a_star)
    assert a == a_star and n == 1 and calls == [a_star]


def test_exhausted_budget_falls_back_to_sufficient_decrease_or_none():
    fn, _ = CASES[1]
    f0, g0 = fn(0.0)
    # one evaluation far beyond the minimiser: no Wolfe point, no sufficient decrease
    a, fa, ga, n = hager_zhang(fn, f0, g0, 50.0, HZParams(max_evals=1))
    assert a is None and n == 1 and (fa, ga) == (f0, g0)
    # a tiny step that decreases phi but whose slope is still too negative is the fallback
    a, fa, ga, n = hager_zhang(fn, f0, g0, 1e-3, HZParams(max_evals=1))
    assert a == 1e-3 and fa < f0 and n == 1
