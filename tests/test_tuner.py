"""Rebuild-interval auto-tuning (Sec. 2.6, Appendix C) against closed forms and brute force,
and the Brent minimisation behind the critical separation of groups (Sec. 2.4).

Host-only code of the library: runs without a GPU.
"""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def g():
    from paper_1610_07279_gb300 import build, gothic
    build.build()
    gothic.load()
    return gothic


def _mean_time(t_make, model, coef, n):
    i = np.arange(n)
    if model == 0:
        t = coef[0] + i * coef[1]
    elif model == 1:
        t = coef[0] * coef[1] ** i
    else:
        t = coef[0] + i * coef[1] + i * i * coef[2]
    return (t_make + t.sum()) / n


def test_linear_growth_closed_form(g):
    t = 1.0 + 0.1 * np.arange(12)          # t1 = 1, dt = 0.1 (Eq. 9)
    model, n_opt, coef = g.gt_rebuild_interval(t, 5.0)
    assert model == 0
    np.testing.assert_allclose(coef[:2], [1.0, 0.1], rtol=1e-10)
    assert math.isclose(n_opt, math.sqrt(2 * 5.0 / 0.1), rel_tol=1e-9)   # Eq. (12)


def test_power_law_growth_closed_form(g):
    t1, r, t_make = 0.5, 1.05, 3.0
    t = t1 * r ** np.arange(15)
    model, n_opt, coef = g.gt_rebuild_interval(t, t_make)
    assert model == 1
    np.testing.assert_allclose(coef[:2], [t1, r], rtol=1e-9)
    # Appendix C: (n ln r - 1) r^n = (r - 1) t_make / t1 - 1
    lhs = (n_opt * math.log(r) - 1.0) * r ** n_opt
    assert math.isclose(lhs, (r - 1.0) * t_make / t1 - 1.0, rel_tol=1e-7, abs_tol=1e-9)
    # and it is the minimum of the mean time per step over integers (within one)
    best = min(range(1, 200), key=lambda n: _mean_time(t_make, 1, [t1, r], n))
    assert abs(n_opt - best) <= 1.0


def test_parabolic_growth_closed_form(g):
    t1, b, a, t_make = 1.0, 0.02, 0.003, 4.0
    i = np.arange(14)
    t = t1 + i * b + i * i * a
    model, n_opt, coef = g.gt_rebuild_interval(t, t_make)
    assert model == 2
    np.testing.assert_allclose(coef, [t1, b, a], rtol=1e-8, atol=1e-12)
    # Appendix C: n^2 = t_make / (b/2 + (4n - 3) a / 6)
    assert math.isclose(n_opt * n_opt, t_make / (b / 2 + (4 * n_opt - 3) * a / 6), rel_tol=1e-7)
    assert (2 * n_opt - 1) * a + b >= 0
    best = min(range(1, 200), key=lambda n: _mean_time(t_make, 2, [t1, b, a], n))
    assert abs(n_opt - best) <= 1.0


def test_no_growth_means_no_rebuild(g):
    model, n_opt, _ = g.gt_rebuild_interval(2.0 - 0.01 * np.arange(8), 1.0)
    assert n_opt >= 1e6


def test_model_choice_by_reduced_chi2(g):
    rng = np.random.default_rng(0)
    i = np.arange(30)
    lin = 1.0 + 0.05 * i + rng.normal(0, 1e-4, i.size)
    assert g.gt_rebuild_interval(lin, 2.0)[0] == 0
    pw = 0.2 * 1.1 ** i * (1 + rng.normal(0, 1e-5, i.size))
    assert g.gt_rebuild_interval(pw, 2.0)[0] == 1


# ---------------------------------------------------------------- Brent (Sec. 2.4)
def test_brent_finds_parabola_vertex_quickly(g):
    calls = []
    x, fx, ev = g.gt_brent_minimize(lambda t: calls.append(t) or (t - 0.7312) ** 2 + 3.0, -5.0, 4.0,
                                    tol=1e-9, max_evals=100)
    assert abs(x - 0.7312) < 1e-6 and abs(fx - 3.0) < 1e-10
    assert min(abs(c - 0.7312) for c in calls[:4]) < 1e-12  # a parabolic step lands on the vertex
    golden = math.ceil(math.log(9.0 / 1e-9) / math.log((1 + 5 ** 0.5) / 2))
    assert ev < golden  # fewer evaluations than golden-section search to the same bracket


def test_brent_on_nonsmooth_and_edge_minima(g):
    x, _, ev = g.gt_brent_minimize(lambda t: abs(t - 1.25) ** 0.5, 0.0, 10.0, tol=1e-8, max_evals=200)
    assert abs(x - 1.25) < 1e-6  # cusp: golden-section steps still shrink the bracket
    x, _, _ = g.gt_brent_minimize(lambda t: t, 2.0, 3.0, tol=1e-8, max_evals=200)
    assert x - 2.0 < 1e-6  # a monotone function: the minimum is at the lower end
    x, _, _ = g.gt_brent_minimize(lambda t: np.cos(t), 2.0, 4.5, tol=1e-10, max_evals=200)
    assert abs(x - np.pi) < 1e-5


def test_brent_respects_the_evaluation_budget(g):
    calls = []
    g.gt_brent_minimize(lambda t: calls.append(t) or (t - 0.3) ** 4, -1.0, 1.0, tol=1e-14, max_evals=7)
    assert len(calls) <= 7 and all(-1.0 <= t <= 1.0 for t in calls)
