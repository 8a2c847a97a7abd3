"""Pins of the oracle against the paper's error bounds (Section 3.1 and Appendix B).

* Lemma truncation_error: the filter g against its Fourier series cut to the band B,
  |g(x - y_j) - sum_{n in B} g_hat_n e^{i n (x - y_j)}| < N^{1 - beta^2/18} / (beta sqrt(ln N)),
  with c1 = beta sqrt(ln N) / N (odd N = 2M + 1, B = [-M, M]).  A filter of the wrong width or
  normalisation, or g_hat not its Fourier series, misses the bound by orders of magnitude.
* Lemma fewer_points_error: the oracle's window of 2 kappa + 1 samples around j' against its sum
  over all N samples, within 2 ||f|| N^{-2 pi^2 gamma^2 / beta^2} for beta >= 4, N >= beta^2 and
  kappa = ceil(gamma ln N) + 1.  The lemma's proof ends with ||f||_p times a factor that is below 1
  for every p >= 1, p = infinity included, so the check takes the smallest norm, ||f||_inf.
* eq. E_approx_error_to_GKlam: noise n on the samples moves each measurement E_h by
  (1/P) sum_k n_k e^{-2 pi i k h / P}, at most ||n||_inf; a noise e^{+2 pi i k h / P} attains the
  bound at bin h, which pins the measurement's 1/P normalisation and the sign of its exponent.
"""
import math

import numpy as np
import pytest

from oracle.dsft import Plan, dft_bins, g_hat, g_periodic, resample


def _plan(N, kappa, beta):
    c1 = beta * math.sqrt(math.log(N)) / N
    return Plan(N=N, s=1, kappa=kappa, alpha=beta, beta=beta, c1=c1, L=N, shifts=[0],
                primes=[N + 2], small=[])


@pytest.mark.parametrize("N", [257, 1025, 4097])
@pytest.mark.parametrize("beta", [4.5, 6.0, 8.0])
def test_lemma_truncation_error(N, beta):
    M = (N - 1) // 2
    c1 = beta * math.sqrt(math.log(N)) / N
    rng = np.random.default_rng(N + int(10 * beta))
    x = rng.uniform(-math.pi, math.pi, 64)
    j = rng.integers(0, N, 64)
    d = x - (-math.pi + 2 * math.pi * j / N)
    n = np.arange(-M, M + 1)
    series = (g_hat(n, c1)[None, :] * np.exp(1j * np.outer(d, n))).sum(axis=1)
    err = np.max(np.abs(g_periodic(d, c1) - series))
    bound = N ** (1 - beta ** 2 / 18) / (beta * math.sqrt(math.log(N)))
    assert err < bound, (err, bound)


def test_lemma_truncation_error_detects_a_filter_of_the_wrong_width():
    N, beta = 1025, 6.0
    M = (N - 1) // 2
    c1 = beta * math.sqrt(math.log(N)) / N
    d = np.linspace(-math.pi, math.pi, 33)
    n = np.arange(-M, M + 1)
    series = (g_hat(n, c1)[None, :] * np.exp(1j * np.outer(d, n))).sum(axis=1)
    bound = N ** (1 - beta ** 2 / 18) / (beta * math.sqrt(math.log(N)))
    wrong = g_periodic(d, c1 * 1.01)
    assert np.max(np.abs(wrong - series)) > 1e3 * bound


@pytest.mark.parametrize("N,beta,kappa", [(1001, 4.0, 6), (1001, 4.0, 4), (4097, 4.0, 6),
                                          (4097, 5.0, 8), (16385, 4.0, 6)])
def test_lemma_fewer_points_error(N, beta, kappa):
    assert beta >= 4 and N >= beta ** 2
    gamma = (kappa - 1) / math.log(N)                  # the largest gamma with this kappa
    assert math.ceil(gamma * math.log(N) - 1e-12) + 1 == kappa
    rng = np.random.default_rng(N + kappa)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    full = _plan(N, (N - 1) // 2, beta)                # the window covers all N samples
    cut = _plan(N, kappa, beta)
    bound = 2 * np.max(np.abs(f)) * N ** (-2 * math.pi ** 2 * gamma ** 2 / beta ** 2)
    for P in (97, 331):
        k = np.arange(P)
        err = np.max(np.abs(resample(f, full, P, k, 0) - resample(f, cut, P, k, 0)))
        assert err <= bound, (P, err, bound)


def test_lemma_fewer_points_error_window_converges():
    """The truncation error falls as kappa grows (each step adds the next Gaussian tail terms)."""
    N, beta = 4097, 4.0
    rng = np.random.default_rng(7)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    k = np.arange(97)
    full = resample(f, _plan(N, (N - 1) // 2, beta), 97, k, 0)
    errs = [np.max(np.abs(full - resample(f, _plan(N, kap, beta), 97, k, 0))) for kap in (2, 4, 6, 8)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


@pytest.mark.parametrize("P", [7, 97, 331])
def test_noise_moves_each_measurement_by_at_most_its_sup_norm(P):
    rng = np.random.default_rng(P)
    h = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    for _ in range(5):
        noise = rng.uniform(-1, 1, P) + 1j * rng.uniform(-1, 1, P)
        delta = dft_bins(h + noise) - dft_bins(h)
        assert np.max(np.abs(delta)) <= np.max(np.abs(noise)) * (1 + 1e-12)
    # attained: noise of modulus eps aligned with bin b moves that bin by exactly eps
    eps = 1e-3
    for b in (0, 1, P // 2, P - 1):
        noise = eps * np.exp(2j * math.pi * np.arange(P) * b / P)
        delta = dft_bins(h + noise) - dft_bins(h)
        assert abs(abs(delta[b]) - eps) < 1e-12
        others = np.delete(np.abs(delta), b)
        assert np.max(others) < 1e-12
