"""Pins of the oracle's direct summation (Eq. 1) to closed forms and invariants."""
import numpy as np
import pytest

from paper_1610_07279_gb300 import ics


def _p4(pos, mass):
    p4 = np.zeros((len(mass), 4), np.float32)
    p4[:, :3] = pos
    p4[:, 3] = mass
    return p4


@pytest.mark.parametrize("sep", [(0.75, 0.0, 0.0), (0.5, 0.25, -0.125), (-3.0, 2.0, 1.5)])
def test_two_body_closed_form(oracle_lib, sep):
    O = oracle_lib
    eps, G = 1.0 / 64.0, 1.0
    m1, m2 = 0.5, 0.25
    p4 = _p4(np.array([[0.0, 0.0, 0.0], sep]), np.array([m1, m2]))
    out = O.direct(p4, eps, G)
    d = np.array(sep, dtype=np.float64)
    r2 = float(d @ d) + eps * eps
    # a_1 = G m_2 d / (r^2 + eps^2)^{3/2}, a_2 = -G m_1 d / (...)^{3/2}
    a1 = G * m2 * d / r2 ** 1.5
    a2 = -G * m1 * d / r2 ** 1.5
    np.testing.assert_allclose(out[0, :3], a1, rtol=1e-15, atol=0)
    np.testing.assert_allclose(out[1, :3], a2, rtol=1e-15, atol=0)
    np.testing.assert_allclose(out[0, 3], -G * m2 / r2 ** 0.5, rtol=1e-15)
    np.testing.assert_allclose(out[1, 3], -G * m1 / r2 ** 0.5, rtol=1e-15)


def test_G_scales_linearly(oracle_lib):
    pos, vel, m, eps = ics.plummer(256, seed=11)
    p4 = _p4(pos, m)
    a1 = oracle_lib.direct(p4, eps, 1.0)
    a3 = oracle_lib.direct(p4, eps, 3.0)
    np.testing.assert_allclose(a3, 3.0 * a1, rtol=1e-14)


def test_momentum_conservation(oracle_lib):
    pos, vel, m, eps = ics.plummer(1024, seed=7)
    m = m * (1.0 + np.random.default_rng(0).uniform(0, 1, m.size)).astype(np.float32)
    p4 = _p4(pos, m)
    a = oracle_lib.direct(p4, eps)
    mom = (p4[:, 3:4].astype(np.float64) * a[:, :3]).sum(axis=0)
    scale = (p4[:, 3].astype(np.float64) * np.linalg.norm(a[:, :3], axis=1)).sum()
    assert np.all(np.abs(mom) <= 1e-13 * scale)


def test_plummer_analytic_field(oracle_lib):
    """Radial field of a Plummer sphere, a(r) = -G M r / (r^2 + a^2)^{3/2} (G=M=a=1)."""
    n = 1 << 13
    pos, vel, m, eps = ics.plummer(n, seed=1)
    p4 = _p4(pos, m)
    a = oracle_lib.direct(p4, eps)
    r = np.linalg.norm(pos, axis=1)
    ar = (a[:, :3] * pos).sum(axis=1) / r
    ana = -r / (r * r + 1.0) ** 1.5
    edges = np.array([0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 5.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        ratio = (ar[sel] / ana[sel]).mean()
        noise = 3.0 / np.sqrt(sel.sum()) + 0.01
        assert abs(ratio - 1.0) < noise, (lo, hi, ratio, sel.sum())


def test_potential_excludes_self(oracle_lib):
    p4 = _p4(np.array([[0.0, 0.0, 0.0]]), np.array([1.0]))
    out = oracle_lib.direct(p4, 0.1)
    assert np.all(out == 0.0)
