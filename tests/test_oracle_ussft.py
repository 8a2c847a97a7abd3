"""Pins of the oracle's inner SFT (Appendix B reading) and of Algorithm 1 end to end.

* measurement bins obey the aliasing identity X[c] = sum_{n = c mod P} (-1)^n h_hat_n for exact
  samples of a trigonometric polynomial (eq. DFT_GKlam_Comp at nodes -pi + 2 pi k / P);
* CRT reconstruction is the unique solution (exhaustive on small coprime moduli);
* the map into B is the unique representative (exhaustive);
* the componentwise median survives a corrupted minority of moduli (the "more than half" of
  Appendix B and the sqrt(2) of eq. GSFT_Estimate);
* exactly s-sparse, well-separated inputs are recovered exactly (support) and to rounding
  (coefficients), and the output equals R_s^opt of the brute-force O(N^2) DFT (Section 2);
* Theorem MainTHM's bound holds on a compressible input;
* plan invariants: primes prime and distinct, small moduli coprime, p_1 prod(T) >= N.
"""
import math

import numpy as np
import pytest

from oracle import dsft as O
from synth.signals import make_signal


def _trig_samples(n_freqs, coefs, x):
    return np.exp(1j * np.outer(x, n_freqs)) @ coefs


@pytest.mark.parametrize("P", [7, 30, 101, 210])
def test_aliasing_identity(P):
    rng = np.random.default_rng(P)
    n = rng.integers(-5 * P, 5 * P, size=9)
    c = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    x = -math.pi + 2 * math.pi * np.arange(P) / P
    X = O.dft_bins(_trig_samples(n, c, x))
    ref = np.zeros(P, complex)
    for nn, cc in zip(n, c):
        ref[nn % P] += (-1) ** int(nn % 2) * cc
    assert np.max(np.abs(X - ref)) < 1e-12


@pytest.mark.parametrize("moduli", [(5, 2, 3), (7, 3, 4), (11, 2, 3, 5), (13, 9, 8, 5)])
def test_crt_exhaustive(moduli):
    M = math.prod(moduli)
    seen = set()
    for x in range(M):
        r = [x % m for m in moduli]
        y = O.crt(r, list(moduli))
        assert y == x
        seen.add(tuple(r))
    assert len(seen) == M  # residue map is a bijection


@pytest.mark.parametrize("N,M", [(10, 10), (11, 11), (10, 15), (11, 30), (64, 66)])
def test_to_band_exhaustive(N, M):
    lo, hi = -((N + 1) // 2) + 1, N // 2
    for x in range(M):
        w = O.to_band(x, M, N)
        members = [v for v in range(lo, hi + 1) if (v - x) % M == 0]
        if members:
            assert w == members[0] and len(members) == 1
        else:
            assert w is None


def test_median_survives_minority_corruption():
    rng = np.random.default_rng(3)
    primes = [11, 13, 17, 19, 23]
    w = 1234
    true = 0.7 - 0.2j
    Y = []
    for p in primes:
        y = rng.standard_normal(p) + 1j * rng.standard_normal(p)
        y[w % p] = (-1) ** (w % 2) * true
        Y.append(y)
    assert abs(O.median_estimate(Y, primes, w) - true) < 1e-15
    # corrupt two of five (a minority): still exact
    Y[1][w % 13] += 5 + 5j
    Y[4][w % 23] -= 3 - 7j
    assert abs(O.median_estimate(Y, primes, w) - true) < 1e-15
    # each component perturbed by at most delta on a majority -> error <= sqrt(2) delta
    delta = 1e-3
    for jj, p in enumerate(primes[:3]):
        Y[jj][w % p] = (-1) ** (w % 2) * (true + delta * np.exp(1j * rng.uniform(0, 6.3)))
    assert abs(O.median_estimate(Y, primes, w) - true) <= math.sqrt(2) * delta + 1e-15
    # a majority corrupted the same way breaks it: the pin has teeth
    Y[0][w % 11] += 9
    Y[2][w % 17] += 9
    Y[3][w % 19] += 9
    assert abs(O.median_estimate(Y, primes, w) - true) > 1


def test_plan_invariants():
    for (N, s, seed) in [(2 ** 16, 8, 0), (2 ** 22, 64, 1), (2 ** 26, 1000, 2), (4194301, 64, 5),
                         (1000003, 2, 9)]:
        plan = O.make_plan(N, s, K=5, c_p=3, seed=seed)
        assert len(set(plan.primes)) == 5 and all(O.is_prime(p) for p in plan.primes)
        assert min(plan.primes) >= 3 * s
        assert all(O.is_prime(t) for t in plan.small)
        assert not set(plan.small) & set(plan.primes)
        assert plan.primes[0] * math.prod(plan.small) >= N
        if plan.small:
            assert plan.primes[0] * math.prod(plan.small[:-1]) < N  # minimal
    with pytest.raises(ValueError):
        O.make_plan(2 ** 16, 8, primes=[101, 103, 107], small=[2, 4])
    with pytest.raises(ValueError):
        O.make_plan(2 ** 16, 8, primes=[101, 103, 107], small=[2, 3])   # product too small
    with pytest.raises(ValueError):
        O.make_plan(9, 2, kappa=6)


def test_splitmix64_published_vector():
    # first outputs for seed 1234567 as given with the generator's reference implementation
    state = 1234567
    outs = []
    for _ in range(3):
        state, z = O.splitmix64(state)
        outs.append(z)
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def _recover(N, s, seed, K=5, c_p=8.0, kappa=6):
    sig = make_signal(N, s, seed, "unit", None)
    plan = O.make_plan(N, s, kappa=kappa, K=K, c_p=c_p, seed=seed)
    return sig, plan, O.dsft(sig.f, plan)


@pytest.mark.parametrize("N,s,seed", [(2 ** 12, 3, 1), (3 ** 7, 4, 2), (4093, 3, 3),
                                      (2 ** 16, 8, 1002)])
def test_exact_recovery_of_sparse_inputs(N, s, seed):
    sig, plan, res = _recover(N, s, seed)
    assert sorted(res.freqs.tolist()) == sorted(sig.omega.tolist())
    truth = dict(zip(sig.omega.tolist(), sig.coef))
    err = max(abs(c - truth[int(w)]) for w, c in zip(res.freqs, res.coefs))
    assert err < 1e-9


@pytest.mark.parametrize("N", [512, 729, 509])
def test_matches_brute_force_best_s_term(N):
    """P1: on an s-sparse input plus a small dense tail, the output support is R_s^opt of the
    brute-force DFT and the coefficients agree within the tail's influence."""
    s = 3
    sig = make_signal(N, s, 77 + N, "unit", 40.0)
    w, fh = O.dft_matrix_apply(sig.f)
    bw, bc = O.best_s_term(w, fh, s)
    plan = O.make_plan(N, s, kappa=6, K=7, c_p=10.0, seed=N)
    res = O.dsft(sig.f, plan)
    assert res.freqs.tolist() == bw.tolist()
    tail = np.sort(np.abs(fh))[::-1][s:].sum()
    assert np.max(np.abs(res.coefs - bc)) < 4 * tail / 0.24


def test_brute_force_dft_convention():
    # F f reproduces the spectrum the generator used (odd, even and prime N)
    for N in [64, 81, 97]:
        sig = make_signal(N, 5, N, "loguniform", None)
        w, fh = O.dft_matrix_apply(sig.f)
        spec = np.zeros(N, complex)
        spec[sig.omega - w[0]] = sig.coef
        assert np.max(np.abs(fh - spec)) < 1e-12


def test_main_theorem_bound_on_compressible_input():
    """Theorem MainTHM: ||f_hat - v||_2 <= ||f_hat - f_hat_s^opt||_2 + 33/sqrt(s) ||.||_1
    + 198 sqrt(s) ||f||_inf N^{-r}; checked with r = 1 on a power-law spectrum."""
    N, s = 1024, 4
    rng = np.random.default_rng(11)
    lo = -((N + 1) // 2) + 1
    spec = np.zeros(N, complex)
    idx = rng.permutation(N)
    spec[idx] = (np.arange(1, N + 1) ** -2.0) * np.exp(2j * math.pi * rng.uniform(size=N))
    from synth.signals import samples_from_spectrum
    w_all = np.arange(lo, N // 2 + 1)
    f = samples_from_spectrum(N, w_all, spec)
    w, fh = O.dft_matrix_apply(f)
    plan = O.make_plan(N, s, kappa=6, K=7, c_p=10.0, seed=5)
    res = O.dsft(f, plan)
    v = np.zeros(N, complex)
    v[res.freqs - lo] = res.coefs
    _, best = O.best_s_term(w, fh, s)
    tail = np.sort(np.abs(fh))[::-1][s:]
    bound = (np.sqrt(np.sum(tail ** 2)) + 33 / math.sqrt(s) * tail.sum()
             + 198 * math.sqrt(s) * np.max(np.abs(f)) / N)
    assert np.linalg.norm(fh - v) <= bound
