"""Pins of the oracle's filter primitives against facts the paper and mathematics fix.

* g_hat against a trapezoid rule of g (spectrally exact for smooth periodic functions):
  Lemma Periodic_Gaussian_FC ties the two formulas; a wrong normalisation, sign, or a dropped
  periodic image fails.
* Lemma Decay_of_Periodic_Gaussian's pointwise bound.
* Lemma Periodic_Gaussian_Decay's passband floor tau.
"""
import math

import numpy as np
import pytest

from oracle.dsft import g_hat, g_periodic, make_plan, SQRT_2PI


@pytest.mark.parametrize("c1", [0.004, 0.03, 0.2, 0.6, 1.0, 1.7])
def test_ghat_matches_trapezoid_of_g(c1):
    M = 8192
    x = -math.pi + 2 * math.pi * np.arange(M) / M
    gx = g_periodic(x, c1)
    w = np.arange(-40, 41)
    # (1/2pi) int g(x) e^{-iwx} dx by the M-point trapezoid rule on one period
    trap = (np.exp(-1j * np.outer(w, x)) @ gx) / M
    ref = g_hat(w, c1)
    assert np.max(np.abs(trap - ref)) < 1e-13
    assert np.max(np.abs(trap.imag)) < 1e-13


def test_ghat_needs_the_periodic_images():
    # for wide Gaussians the images n = +-1 carry weight: dropping them changes g_hat_0
    c1 = 1.0
    M = 4096
    x = -math.pi + 2 * math.pi * np.arange(M) / M
    central = np.exp(-x ** 2 / (2 * c1 * c1)) / c1
    assert abs(central.mean() - g_hat(0, c1)) > 1e-4
    assert abs(g_periodic(x, c1).mean() - g_hat(0, c1)) < 1e-13


@pytest.mark.parametrize("c1", [0.01, 0.1, 0.5, 1.0, 2.0])
def test_decay_bound(c1):
    x = np.linspace(-math.pi, math.pi, 20001)
    bound = (3.0 / c1 + 1.0 / SQRT_2PI) * np.exp(-x ** 2 / (2 * c1 * c1))
    g = g_periodic(x, c1)
    assert np.all(g <= bound * (1 + 1e-12))
    assert np.all(g >= 0) and g[len(g) // 2] > 0


@pytest.mark.parametrize("N", [2 ** 10, 3 ** 7, 4093, 2 ** 16, 2 ** 26])
@pytest.mark.parametrize("tau", [1 / 3, 0.2, 0.05])
@pytest.mark.parametrize("alpha", [1.0, 1.5, 4.0])
def test_passband_floor(N, tau, alpha):
    lnN = math.log(N)
    beta = alpha * math.sqrt(math.log(1 / (tau * SQRT_2PI)) / 2)
    c1 = beta * math.sqrt(lnN) / N
    edge = math.ceil(N / (alpha * math.sqrt(lnN)))
    w = np.arange(-edge, edge + 1)
    gh = g_hat(w, c1)
    assert gh.min() >= tau
    assert gh.max() <= 1 / SQRT_2PI + 1e-16
    # monotone in |w|
    assert np.all(np.diff(g_hat(np.arange(0, edge), c1)) <= 0)


def test_passband_floor_fails_when_beta_too_large():
    # beta above the lemma's ceiling violates the floor at the band edge: the pin has teeth
    N, tau, alpha = 2 ** 16, 1 / 3, 1.5
    lnN = math.log(N)
    beta = 3.0 * alpha * math.sqrt(math.log(1 / (tau * SQRT_2PI)) / 2)
    c1 = beta * math.sqrt(lnN) / N
    edge = math.ceil(N / (alpha * math.sqrt(lnN)))
    assert g_hat(edge, c1) < tau


@pytest.mark.parametrize("N", [17, 100, 2 ** 12, 65521, 2 ** 22, 2 ** 26])
def test_shift_schedule_tiles_B(N):
    """Algorithm 1: the ceil(c2) bands [q - L, q + L) are disjoint and cover B."""
    plan = make_plan(N, 2, kappa=4, primes=[101, 103, 107], small=None)
    lo, hi = -((N + 1) // 2) + 1, N // 2
    L = plan.L
    assert len(plan.shifts) == math.ceil(1.5 * math.sqrt(math.log(N)) / 2)
    starts = [q - L for q in plan.shifts]
    assert starts[0] == lo
    for a, b in zip(plan.shifts, plan.shifts[1:]):
        assert b - a == 2 * L
    assert plan.shifts[-1] + L - 1 >= hi
