"""Pins of the oracle's resampling step (Section 3.1) against closed forms.

For a trigonometric polynomial f with support S in B, expanding eq. UntruncatedFiniteSum with
g_q(x) = e^{iqx} g(x) gives, exactly,

    (1/N) sum_{j=0}^{N-1} f(y_j) g_q(x - y_j) = sum_{w in S} c_w sum_k (-1)^{kN} g_hat_{w+kN-q} e^{i(w+kN)x},

and the true convolution is (g_q * f)(x) = sum_{w in S} c_w g_hat_{w-q} e^{iwx}.

* with a window covering all N grid points (odd N, 2 kappa + 1 = N) the oracle must equal the first
  form to rounding, for any beta: this pins weights, phases, the modulation sign and window
  placement;
* with Theorem total_convolution_error's parameters (c1 = 6 sqrt(r ln N)/N, half-width
  ceil(6 r ln N / (sqrt 2 pi)) + 1) the oracle must be within 3 ||f||_inf N^{-r} of the second;
* node k of modulus p and node k t of modulus p t (the same point) give the same sample, as the
  subset moduli p_j t_l of the measurements require.
"""
import math

import numpy as np
import pytest

from oracle.dsft import Plan, g_hat, g_periodic, nearest_grid, resample


def _plan(N, kappa, beta):
    lnN = math.log(N)
    c1 = beta * math.sqrt(lnN) / N
    return Plan(N=N, s=1, kappa=kappa, alpha=beta, beta=beta, c1=c1, L=N, shifts=[0],
                primes=[N + 2], small=[])


def _trig(N, S, c):
    y = -math.pi + 2 * math.pi * np.arange(N) / N
    return np.exp(1j * np.outer(y, S)) @ c


def _nodes(P):
    return -math.pi + 2 * math.pi * np.arange(P) / P


@pytest.mark.parametrize("N", [101, 257, 1001])
@pytest.mark.parametrize("beta", [0.8, 1.5, 4.0])
def test_full_window_equals_semidiscrete_closed_form(N, beta):
    rng = np.random.default_rng(N)
    lo, hi = -((N + 1) // 2) + 1, N // 2
    S = rng.choice(np.arange(lo, hi + 1), size=5, replace=False)
    c = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    f = _trig(N, S, c)
    plan = _plan(N, (N - 1) // 2, beta)
    for q in [0, 7, -(N // 3), N // 2]:
        for P in [13, 37]:
            h = resample(f, plan, P, np.arange(P), q)
            x = _nodes(P)
            ref = np.zeros(P, complex)
            for w, cw in zip(S, c):
                for k in range(-6, 7):
                    n = w + k * N
                    ref += cw * (-1) ** (k * N) * g_hat(n - q, plan.c1) * np.exp(1j * n * x)
            assert np.max(np.abs(h - ref)) < 1e-12 * np.sum(np.abs(c))


@pytest.mark.parametrize("N,r", [(2 ** 12, 1), (2 ** 12, 2), (3 ** 8, 2), (65521, 2)])
def test_theorem_total_convolution_error(N, r):
    lnN = math.log(N)
    beta = 6 * math.sqrt(r)
    kappa = math.ceil(6 * r * lnN / (math.sqrt(2) * math.pi)) + 1
    plan = _plan(N, kappa, beta)
    rng = np.random.default_rng(r * N)
    lo, hi = -((N + 1) // 2) + 1, N // 2
    S = rng.choice(np.arange(lo, hi + 1), size=6, replace=False)
    c = np.exp(2j * math.pi * rng.uniform(size=6))
    f = _trig(N, S, c)
    finf = np.max(np.abs(f))
    P = 211
    x = _nodes(P)
    for q in [0, S[0], -N // 4]:
        h = resample(f, plan, P, np.arange(P), int(q))
        exact = np.exp(1j * np.outer(x, S)) @ (c * g_hat(S - q, plan.c1))
        assert np.max(np.abs(h - exact)) <= 3 * finf * N ** (-r)


def test_wrong_modulation_sign_is_detected():
    # the closed form centres the filter on +q: the mirrored filter misses by O(1)
    N, r = 2 ** 12, 1
    lnN = math.log(N)
    plan = _plan(N, math.ceil(6 * r * lnN / (math.sqrt(2) * math.pi)) + 1, 6.0)
    S = np.array([300])
    c = np.array([1.0 + 0j])
    f = _trig(N, S, c)
    x = _nodes(31)
    h = resample(f, plan, 31, np.arange(31), 300)
    right = np.exp(1j * np.outer(x, S)) @ (c * g_hat(S - 300, plan.c1))
    mirrored = np.exp(1j * np.outer(x, S)) @ (c * g_hat(S + 300, plan.c1))
    assert np.max(np.abs(h - right)) < 1e-3
    assert np.max(np.abs(h - mirrored)) > 0.1


@pytest.mark.parametrize("N,P", [(16, 6), (100, 7), (2 ** 20, 3001), (65521, 4099),
                                 (10, 4), (6, 4), (1026, 4), (2 ** 20 + 6, 12)])
def test_nearest_grid_is_argmin_with_ties_up(N, P):
    k = np.arange(P, dtype=np.int64)
    jp = nearest_grid(N, P, k)
    # |kN/P - j'| <= 1/2, exactly, in integers: |2kN - 2j'P| <= P, and ties (= P) take the larger j
    d2 = 2 * k * N - 2 * jp * P
    assert np.all(np.abs(d2) <= P)
    assert np.all(d2 != P)          # a tie would have been rounded up, leaving d2 == -P


@pytest.mark.parametrize("N,P", [(10, 4), (6, 4), (1026, 4), (2 ** 20 + 6, 12)])
def test_nearest_grid_ties_go_up(N, P):
    """Where kN/P is a half-integer both neighbours are nearest; the reading taken (R6) rounds up."""
    k = np.arange(P, dtype=np.int64)
    ties = [kk for kk in k if (2 * kk * N) % (2 * P) == P]
    assert ties, "this case must contain ties"
    for kk in ties:
        assert nearest_grid(N, P, np.array([kk]))[0] == (kk * N + P // 2) // P
        assert 2 * kk * N - 2 * nearest_grid(N, P, np.array([kk]))[0] * P == -P


@pytest.mark.parametrize("N,P,kappa", [(101, 37, 3), (256, 97, 4), (255, 61, 6)])
@pytest.mark.parametrize("q", [0, 5, -17])
def test_window_is_the_nearest_samples_brute_force(N, P, kappa, q):
    """Lemma fewer_points_error's window: for each node x, the 2 kappa + 1 grid points nearest to
    x (found by sorting all N circular distances), each weighted g(x - y_j) e^{iq(x - y_j)} / N,
    summed directly.  Nodes where the choice of nearest points ties are skipped.  A window shifted
    by one sample, a wrong width or a phase of the wrong sign fails this."""
    rng = np.random.default_rng(N * 7 + P + q)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c1 = 1.5 * math.sqrt(math.log(N)) / N
    plan = Plan(N=N, s=1, kappa=kappa, alpha=1.5, beta=1.5, c1=c1, L=N, shifts=[0],
                primes=[P], small=[])
    k = np.arange(P)
    h = resample(f, plan, P, k, q)
    y = -math.pi + 2 * math.pi * np.arange(N) / N
    checked = 0
    for kk in k:
        x = -math.pi + 2 * math.pi * kk / P
        diff = x - y
        dist = np.abs(np.angle(np.exp(1j * diff)))            # circular distance
        order = np.argsort(dist, kind="stable")
        w = 2 * kappa + 1
        if abs(dist[order[w - 1]] - dist[order[w]]) < 1e-9:   # a tie at the window's edge
            continue
        sel = order[:w]
        dd = np.angle(np.exp(1j * diff[sel]))                 # x - y_j in (-pi, pi]
        ref = np.sum(f[sel] * g_periodic(dd, c1) * np.exp(1j * q * dd)) / N
        assert abs(h[kk] - ref) <= 1e-12 * np.sum(np.abs(f[sel]) * g_periodic(dd, c1)) / N, kk
        checked += 1
    assert checked >= P // 2


@pytest.mark.parametrize("N,p,t", [(4099, 101, 3), (2 ** 14, 211, 5), (65521, 97, 13),
                                   (2 ** 20 + 6, 3001, 2)])
@pytest.mark.parametrize("q", [0, 37, -1234])
def test_nodes_of_p_are_the_nodes_kt_of_pt(N, p, t, q):
    """Node k of modulus p and node k t of modulus p t are the same point -pi + 2 pi k / p, and
    the integers of the window (j', d = k N - j P, q d mod P N) scale by t, so the oracle's
    samples agree either way up to the rounding of 2 pi d (a few ulp); a modulus taken as P in
    one place and p in another, or a node index not scaled, gives an error of order one."""
    rng = np.random.default_rng(N + p + t)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    plan = _plan(N, 6, 1.5)
    k = np.arange(p)
    assert np.array_equal(nearest_grid(N, p, k), nearest_grid(N, p * t, k * t))
    a = resample(f, plan, p, k, q)
    b = resample(f, plan, p * t, k * t, q)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
    c = resample(f, plan, p * t, k * t + 1, q)               # the neighbouring nodes differ
    assert np.max(np.abs(a - c)) > 1e-3 * np.max(np.abs(a))
