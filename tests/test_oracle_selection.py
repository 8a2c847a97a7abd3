"""Pins of the oracle's plan and selections (Algorithm 1, Section 2).

* The s-term choice (R_s^opt's rule: the s largest magnitudes, ties to the smaller frequency)
  against a brute-force sort on constructed exact ties; Algorithm 1's per-shift R_temp and its
  final choice both use it, and R_temp holds s terms when a shift finds more.
* The band of Algorithm 1 is half-open, [q - L, q + L): a frequency exactly on the edge between
  two bands is pooled once, from the shift whose band starts there.
* The small moduli: the shortest run of primes not among the p_j whose product with p_1 reaches N
  (sufficient, and one fewer is not), including a case where the product equals N exactly.
* c1 = beta sqrt(ln N) / N through make_plan: with alpha != beta, Theorem total_convolution_error's
  parameters bound the resampling error by 3 ||f||_inf N^{-r}; a c1 taken from alpha breaks it.
"""
import math

import numpy as np
import pytest

from oracle import dsft as O


def _sorted_choice(w, c, s):
    items = sorted(zip(w.tolist(), c.tolist()), key=lambda t: (-abs(t[1]), t[0]))[:s]
    return [t[0] for t in items]


@pytest.mark.parametrize("s", [1, 2, 3, 5, 9])
def test_s_term_choice_breaks_exact_ties_toward_the_smaller_frequency(s):
    w = np.array([5, -3, 2, 7, -1, 0, 4, -6], dtype=np.int64)
    c = np.array([1, 2, -2, 1j, 2j, -1, 0.5, 2], dtype=np.complex128)   # |c| ties exactly
    got_w, got_c = O.best_s_term(w, c, s)
    assert got_w.tolist() == _sorted_choice(w, c, s)
    assert np.array_equal(np.abs(got_c), np.sort(np.abs(c))[::-1][: min(s, len(c))])
    if s == 3:
        assert got_w.tolist() == [-6, -3, -1]


def _sparse_signal(N, S, c):
    f = np.zeros(N, dtype=np.complex128)
    y = -math.pi + 2 * math.pi * np.arange(N) / N
    for w, cw in zip(S, c):
        f += cw * np.exp(1j * w * y)
    return f


def test_per_shift_choice_keeps_s_terms_when_a_shift_finds_more():
    N, s = 4099, 2
    plan = O.make_plan(N, s, K=5, c_p=8.0, seed=3)
    q = plan.shifts[1]
    S = np.array([q - 40, q - 5, q + 17, q + 60])           # four frequencies in one band
    c = np.array([1.0, 0.9, 0.8, 0.7]) * np.exp(1j * np.array([0.3, 1.1, 2.0, -0.7]))
    sr = O.ussft_shift(_sparse_signal(N, S, c), plan, q)
    assert len(sr.voted) >= 4
    assert len(sr.temp_w) == s
    assert sr.temp_w.tolist() == _sorted_choice(sr.voted, sr.z, s)


def test_band_edge_is_pooled_once_from_the_band_that_starts_there():
    N, s = 2 ** 14 + 1, 3
    plan = O.make_plan(N, s, K=5, c_p=8.0, seed=5)
    L, q1 = plan.L, plan.shifts[1]
    edge = q1 - L                                            # = q0 + L: closes band 0, opens band 1
    assert edge == plan.shifts[0] + L
    S = np.array([edge, q1 + 31, plan.shifts[0] - 77])
    c = np.array([1.0, 0.8, 0.6]) * np.exp(1j * np.array([0.4, -1.3, 2.2]))
    res = O.dsft(_sparse_signal(N, S, c), plan)
    hits = np.nonzero(res.pool_w == edge)[0]
    assert len(hits) == 1 and res.pool_q[hits[0]] == q1
    assert sorted(res.freqs.tolist()) == sorted(S.tolist())


@pytest.mark.parametrize("N,p1,others", [(210, 7, [11, 13]), (1001, 11, [13, 17]),
                                         (30030 * 17, 17, [19, 23]), (2 ** 20, 3001, [3011])])
def test_small_moduli_are_the_shortest_sufficient_run(N, p1, others):
    primes = [p1] + others
    T = O.choose_small_moduli(N, primes)
    assert all(O.is_prime(t) and t not in primes for t in T)
    assert T == sorted(T)
    assert p1 * math.prod(T) >= N
    assert not T or p1 * math.prod(T[:-1]) < N
    run = [t for t in range(2, T[-1] + 1) if O.is_prime(t) and t not in primes] if T else []
    assert T == run                                          # no prime skipped


@pytest.mark.parametrize("N,r", [(4097, 1), (2 ** 12, 2)])
def test_c1_comes_from_beta_through_make_plan(N, r):
    lnN = math.log(N)
    beta = 6 * math.sqrt(r)
    kappa = math.ceil(6 * r * lnN / (math.sqrt(2) * math.pi)) + 1
    plan = O.make_plan(N, 2, kappa=kappa, alpha=1.0, beta=beta, primes=[4099, 4111], small=[])
    assert abs(plan.c1 * N / math.sqrt(lnN) - beta) < 1e-12
    rng = np.random.default_rng(N + r)
    lo, hi = -((N + 1) // 2) + 1, N // 2
    S = rng.choice(np.arange(lo, hi + 1), size=6, replace=False)
    c = np.exp(2j * math.pi * rng.uniform(size=6))
    f = _sparse_signal(N, S, c)
    P = 211
    x = -math.pi + 2 * math.pi * np.arange(P) / P
    for q in [0, plan.shifts[0]]:                            # shifts of Algorithm 1's schedule
        h = O.resample(f, plan, P, np.arange(P), q)
        exact = np.exp(1j * np.outer(x, S)) @ (c * O.g_hat(S - q, plan.c1))
        assert np.max(np.abs(h - exact)) <= 3 * np.max(np.abs(f)) * N ** (-r)


def test_final_choice_is_the_s_term_choice_of_the_pool():
    """Algorithm 1 returns s terms: with more frequencies pooled than s, the s largest of the pool
    (ties to the smaller frequency)."""
    N, s = 2 ** 13 + 3, 3
    plan = O.make_plan(N, s, K=5, c_p=8.0, seed=7)
    S = np.array([plan.shifts[0] + 9, plan.shifts[0] - 200, plan.shifts[1] + 50,
                  plan.shifts[1] - 3, 3000, -5])
    assert np.all((S > -((N + 1) // 2)) & (S <= N // 2))     # all in B
    c = np.array([1.0, 0.5, 0.9, 0.4, 0.8, 0.3]) * np.exp(1j * np.arange(6))
    res = O.dsft(_sparse_signal(N, S, c), plan)
    assert len(res.pool_w) > s
    assert len(res.freqs) == s
    assert res.freqs.tolist() == _sorted_choice(res.pool_w, res.pool_c, s)
    assert sorted(res.freqs.tolist()) == sorted(S[np.argsort(-np.abs(c))[:s]].tolist())
