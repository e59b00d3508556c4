"""The Hager-Zhang line search of the reconstruction driver (Sec. 6 uses it for mu_a) on 1-D
functions whose minimisers are known: the accepted step meets the Wolfe or the approximate Wolfe
conditions, the bracketing phase grows a tiny first trial and bisection shrinks a huge one, and
an exhausted budget falls back to the best step with a sufficient decrease."""
import math

import pytest
import torch

from paper_1608_05238_gb300.inversion import lbfgs_direction, HZParams, hager_zhang


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


# ------------------------------------------------------------------ L-BFGS two-loop recursion
def _cpu_dot(us, vs):
    return sum(float((u.double() * v.double()).sum()) for u, v in zip(us, vs) if u is not None and v is not None)


def _quadratic(n, seed):
    g = torch.Generator().manual_seed(seed)
    Q = torch.randn(n, n, generator=g, dtype=torch.float64)
    A = Q @ Q.T + n * torch.eye(n, dtype=torch.float64)
    b = torch.randn(n, generator=g, dtype=torch.float64)
    return A, b


def test_lbfgs_direction_meets_the_secant_condition():
    """The BFGS inverse-Hessian estimate maps the newest y to the newest s: -direction(y) = s."""
    A, _ = _quadratic(6, 1)
    g = torch.Generator().manual_seed(2)
    pairs = []
    for _ in range(4):
        s_ = torch.randn(6, generator=g, dtype=torch.float64)
        y_ = A @ s_
        pairs.append(([s_, None], [y_, None], 1.0 / float(s_ @ y_)))
    d = lbfgs_direction([pairs[-1][1][0], None], pairs, dot=_cpu_dot)
    assert d[1] is None
    assert torch.allclose(-d[0], pairs[-1][0][0], rtol=1e-10, atol=1e-12)


def test_lbfgs_with_exact_line_search_minimises_a_quadratic():
    """With exact line searches on a strictly convex quadratic, BFGS directions are conjugate and
    the minimiser of an n-dimensional quadratic is reached in n steps (memory >= n)."""
    n = 5
    A, b = _quadratic(n, 3)
    x = torch.zeros(n, dtype=torch.float64)
    pairs = []
    grad = lambda v: A @ v - b
    for _ in range(n):
        gx = grad(x)
        d = lbfgs_direction([gx], pairs, dot=_cpu_dot)[0] if pairs else -gx
        alpha = -float(gx @ d) / float(d @ (A @ d))  # exact minimiser along d
        x_new = x + alpha * d
        s_, y_ = x_new - x, grad(x_new) - gx
        pairs.append(([s_], [y_], 1.0 / float(s_ @ y_)))
        x = x_new
    assert torch.allclose(x, torch.linalg.solve(A, b), rtol=1e-8, atol=1e-10)


def test_lbfgs_with_a_diagonal_initial_inverse_hessian():
    """A diagonal H_0 (the fluence preconditioner's role): without pairs the direction is -H_0 g,
    which on a diagonal quadratic with H_0 its inverse Hessian is the Newton step to the minimiser;
    with pairs the secant condition still holds for the newest pair, and a tensor entry without a
    diagonal (None in h0) keeps the gamma I scaling."""
    g = torch.Generator().manual_seed(5)
    diag = torch.rand(7, generator=g, dtype=torch.float64) * 100 + 0.01
    b = torch.randn(7, generator=g, dtype=torch.float64)
    x = torch.zeros(7, dtype=torch.float64)
    gx = diag * x - b
    d = lbfgs_direction([gx], [], dot=_cpu_dot, h0=[1.0 / diag])[0]
    assert torch.allclose(x + d, b / diag, rtol=1e-12, atol=0)
    A, _ = _quadratic(6, 4)
    h = torch.rand(6, generator=g, dtype=torch.float64) + 0.5
    pairs = []
    for _ in range(3):
        s_ = torch.randn(6, generator=g, dtype=torch.float64)
        pairs.append(([s_, s_[:2].clone()], [A @ s_, 3.0 * s_[:2]], 1.0 / (float(s_ @ (A @ s_)) + 3.0 * float(s_[:2] @ s_[:2]))))
    s_new, y_new = pairs[-1][0], pairs[-1][1]
    d = lbfgs_direction(y_new, pairs, dot=_cpu_dot, h0=[h, None])
    assert torch.allclose(-d[0], s_new[0], rtol=1e-10, atol=1e-12)
    assert torch.allclose(-d[1], s_new[1], rtol=1e-10, atol=1e-12)
    # without pairs, the None entry is scaled by gamma = 1
    d0 = lbfgs_direction([gx, b[:2]], [], dot=_cpu_dot, h0=[1.0 / diag, None])
    assert torch.equal(d0[1], -b[:2])
