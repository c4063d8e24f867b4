"""Pins of the oracle's heating epilogue (§5, Eqs. G0_eff, gamma_uv, gamma_cr).

The efficiency of Wolfire et al. (1995) has two terms with known limits: for
a weak field (x = G0_eff sqrt(T) / n_e -> 0) both denominators are 1; at
x = 1925 the first term is halved; for x -> infinity both vanish.  The
cosmic-ray rate is linear in n with no screening; the UV rate vanishes with
chi and is linear in n at fixed x.
"""
import numpy as np
import pytest

import oracle


def test_efficiency_limits():
    T = np.array([10.0, 100.0, 1e4, 8000.0])
    # weak field: x = 1e-12
    eps = oracle.heating_efficiency(1e-12, T, np.sqrt(T))
    assert np.allclose(eps, 0.049 + 0.037 * (T / 1e4) ** 0.7, rtol=1e-9)
    # T = 1e4 K: the second term's temperature factor is one
    assert oracle.heating_efficiency(1e-12, 1e4, 1.0) == pytest.approx(0.086, rel=1e-9)
    # x = 1925 exactly: first term 0.049 / 2; second 0.037 (T/1e4)^0.7 / (1 + 0.385)
    T0 = 100.0
    ne = 1.0
    g0 = 1925.0 / np.sqrt(T0)
    want = 0.0245 + 0.037 * 0.01 ** 0.7 / 1.385
    assert oracle.heating_efficiency(g0, T0, ne) == pytest.approx(want, rel=1e-12)
    # strong field: both terms fall off, the first as x^-0.73, the second as 1/x
    x = np.array([1e14, 1e16])
    e = oracle.heating_efficiency(x / 100.0, 1e4, 1.0)
    assert np.all(e < 1e-4)
    assert e[0] / e[1] == pytest.approx(100 ** 0.73, rel=1e-2)


def test_efficiency_decreases_with_field_and_rates():
    g0 = np.logspace(-3, 3, 50)
    eps = oracle.heating_efficiency(g0, 80.0, 0.01)
    assert np.all(np.diff(eps) < 0)
    n = np.full(50, 30.0)
    g, uv, cr = oracle.heating(g0 / oracle.G0_DRAINE, n, 80.0, 0.01)
    assert np.allclose(g, g0, rtol=1e-14)
    assert np.all(np.diff(uv) > 0)                  # eps falls slower than G0 rises
    assert np.all(cr == 1e-27 * 30.0)


def test_heating_special_cases():
    n = np.array([1.0, 10.0, 1000.0])
    # no screening (chi = 1, the optically thin run of §5): G0_eff = G0 = 1.7
    g, uv, cr = oracle.heating(np.ones(3), n, 8000.0, 0.02 * n)
    assert np.all(g == 1.7)
    assert np.array_equal(cr, 1e-27 * n)
    # x depends on n_e only: scaling n with n_e fixed scales Gamma_UV linearly
    _, uv2, _ = oracle.heating(np.ones(3), 2 * n, 8000.0, 0.02 * n)
    assert np.allclose(uv2, 2 * uv, rtol=1e-14)
    # full screening: no UV heating, cosmic rays unchanged
    g, uv, cr = oracle.heating(np.zeros(3), n, 8000.0, 0.02 * n)
    assert np.all(g == 0) and np.all(uv == 0) and np.array_equal(cr, 1e-27 * n)
    # a worked value: chi = 0.5, n = 100, T = 100 K, n_e = 0.01, G0 = 1.7
    x = 0.85 * 10.0 / 0.01
    eps = 0.049 / (1 + (x / 1925) ** 0.73) + 0.037 * 0.01 ** 0.7 / (1 + x / 5000)
    g, uv, cr = oracle.heating(0.5, 100.0, 100.0, 0.01)
    assert g == pytest.approx(0.85, rel=1e-15)
    assert uv == pytest.approx(1e-24 * eps * 0.85 * 100.0, rel=1e-14)
    assert cr == pytest.approx(1e-25, rel=1e-15)
