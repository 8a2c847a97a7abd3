"""Pins of the deterministic inner SFT (Algorithm 3 of the cited work, first paragraph of Lemma
SFT_Ident_Coef_Est_in_Noise): the K smallest primes >= max(ceil(c_p s), 5), K = 2 (s - 1) L + 1,
L = floor(log_{p_1}(N - 1)).

* the pair-collision bound that the choice of K rests on, checked by brute force over every pair
  of frequencies of B: no two distinct frequencies share a residue modulo more than L of the
  primes, so each of s frequencies is alone in its bin for a strict majority of them;
* exact recovery of exactly s-sparse inputs for every input tried, including adversarial spectra
  whose frequencies all coincide modulo the first primes (inputs on which a random draw of a few
  primes can fail);
* the library's host-side choice equals the oracle's.
"""
import math

import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from oracle import dsft as O
from synth.signals import samples_from_spectrum


def _B(N):
    return np.arange(-((N + 1) // 2) + 1, N // 2 + 1, dtype=np.int64)


@pytest.mark.parametrize("N,s,c_p", [(2 ** 10, 3, 2.0), (729, 4, 1.0), (1009, 2, 3.0),
                                     (2 ** 12, 5, 1.0)])
def test_no_pair_collides_modulo_more_than_L_primes(N, s, c_p):
    primes = O.deterministic_primes(N, s, c_p)
    p1 = primes[0]
    L = 0
    while p1 ** (L + 1) <= N - 1:
        L += 1
    assert len(primes) == 2 * (s - 1) * L + 1
    assert primes == O.primes_from(max(math.ceil(c_p * s), 5), len(primes))
    B = _B(N)
    counts = np.zeros((len(B), len(B)), dtype=np.int32)
    for p in primes:
        r = np.mod(B, p)
        counts += (r[:, None] == r[None, :]).astype(np.int32)
    np.fill_diagonal(counts, 0)
    assert counts.max() <= L
    # hence every frequency of any s-subset is isolated in more than K/2 of the primes
    K = len(primes)
    assert K - (s - 1) * counts.max() > K / 2


def _adversarial(N, s, primes):
    """s frequencies of B that all share their residues modulo the first primes."""
    step = primes[0] * primes[1] if primes[0] * primes[1] * (s - 1) < N // 2 else primes[0]
    w = np.array([(i - s // 2) * step for i in range(s)], dtype=np.int64)
    rng = np.random.default_rng(s)
    coef = np.exp(2j * np.pi * rng.random(s))
    return w, coef


@pytest.mark.parametrize("N,s", [(2 ** 12, 4), (3 ** 7, 3), (4093, 5)])
def test_exact_recovery_including_adversarial_spectra(N, s):
    c_p = 2.0
    plan = O.make_plan(N, s, kappa=6, c_p=c_p, deterministic=True)
    assert plan.primes == O.deterministic_primes(N, s, c_p)
    spectra = [_adversarial(N, s, plan.primes)]
    rng = np.random.default_rng(N)
    for _ in range(3):
        w = rng.choice(_B(N), size=s, replace=False)
        spectra.append((w, np.exp(2j * np.pi * rng.random(s))))
    for w, coef in spectra:
        f = samples_from_spectrum(N, w, coef)
        res = O.dsft(f, plan)
        assert sorted(res.freqs.tolist()) == sorted(w.tolist())
        truth = dict(zip(w.tolist(), coef))
        assert max(abs(c - truth[int(x)]) for x, c in zip(res.freqs, res.coefs)) < 1e-8


@pytest.mark.parametrize("N,s,c_p", [(2 ** 12, 4, 2.0), (2 ** 16, 8, 3.0), (4194301, 50, 3.0),
                                     (2 ** 22, 6, 1.0)])
def test_host_choice_matches_oracle(N, s, c_p):
    from paper_1706_02740_gb300 import build as sft_build
    sft_build.build()
    primes, small = sft.sft_choose_moduli_deterministic(N, s, c_p)
    assert primes == O.deterministic_primes(N, s, c_p)
    assert small == O.choose_small_moduli(N, primes)


def test_host_choice_rejects_too_many_primes():
    from paper_1706_02740_gb300 import build as sft_build
    sft_build.build()
    with pytest.raises(sft.SftError):
        sft.sft_choose_moduli_deterministic(2 ** 30, 400, 1.0)
