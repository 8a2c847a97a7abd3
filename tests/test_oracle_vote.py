"""Pins of the inner SFT's identification rules (Appendix B), through oracle.ussft_shift itself.

The measurements are replaced by constructed bins, so the test decides which moduli see which
frequency:

* a frequency is kept when more than half of the K prime moduli reconstruct it ("more than half of
  the j" in the identification step of Appendix B): with K = 5 one seen by 3 moduli is kept and one
  seen by 2 is not; with K = 4 one seen by 3 is kept and one seen by 2 is not;
* each kept frequency carries the number of moduli that found it;
* the median estimate of a frequency present in a majority of the moduli is its exact value
  (eq. GSFT_Estimate, the other moduli hold zero in that bin);
* an exact tie between sub-bins of a small modulus resolves to the smallest sub-bin index u
  (the tie rule this build reads into the argmax): a bin holding two frequencies of equal
  magnitude gets the residue of the one at the smaller u, and an all-zero bin b (every sub-bin
  ties) gets u = 0, so its candidate is b itself.

The measured bins follow the aliasing identity of eq. DFT_GKlam_Comp at the nodes -pi + 2 pi k/P:
X[c] = sum over planted w with w = c (mod P) of (-1)^w a_w.
"""
import math

import numpy as np
import pytest

from oracle import dsft as O


def _fake_measure(plan, planted):
    """planted[j] = {w: a_w} for prime index j; a length-P measurement with P = p_j t or p_j
    holds prime j's planted frequencies at their aliased bins."""

    def measure(f, plan_, q, P):
        j = [jj for jj, p in enumerate(plan.primes) if P % p == 0]
        assert len(j) == 1
        X = np.zeros(P, dtype=np.complex128)
        for w, a in planted[j[0]].items():
            X[w % P] += (-1) ** (w % 2) * a
        return X

    return measure


def _run(monkeypatch, plan, planted):
    monkeypatch.setattr(O, "measure", _fake_measure(plan, planted))
    return O.ussft_shift(np.zeros(plan.N, complex), plan, plan.shifts[0])


def _distinct_mod_each(primes, ws):
    return all(len({w % p for w in ws}) == len(ws) for p in primes)


def test_vote_keeps_majority_rejects_minority_k5(monkeypatch):
    N = 2000
    primes = [11, 13, 17, 19, 23]
    plan = O.make_plan(N, 4, kappa=2, primes=primes)
    assert plan.small == [2, 3, 5, 7]
    w_all, w_maj, w_min = 700, -651, 903
    assert _distinct_mod_each(primes, [w_all, w_maj, w_min])
    a_all, a_maj, a_min = 0.5 - 0.25j, -0.75 + 0.5j, 2.0 + 1.0j
    planted = [dict() for _ in primes]
    for j in range(5):
        planted[j][w_all] = a_all
    for j in (0, 2, 4):                 # 3 of 5: more than half
        planted[j][w_maj] = a_maj
    for j in (1, 3):                    # 2 of 5: a minority, however strong
        planted[j][w_min] = a_min
    sr = _run(monkeypatch, plan, planted)
    voted = dict(zip(sr.voted.tolist(), sr.votes.tolist()))
    assert voted.get(w_all) == 5
    assert voted.get(w_maj) == 3
    assert w_min not in voted
    # each modulus that holds w_min does reconstruct it: the rejection is the vote's
    assert sr.cand[1][w_min % 13] == w_min and sr.cand[3][w_min % 19] == w_min
    # medians over all K moduli: the majority's common value is exact
    z = dict(zip(sr.voted.tolist(), sr.z))
    assert abs(z[w_all] - a_all) < 1e-15
    assert abs(z[w_maj] - a_maj) < 1e-15


def test_vote_even_k_needs_more_than_half(monkeypatch):
    N = 2000
    primes = [11, 13, 17, 19]
    plan = O.make_plan(N, 4, kappa=2, primes=primes)
    w3, w2 = 555, -777
    assert _distinct_mod_each(primes, [w3, w2])
    planted = [dict() for _ in primes]
    for j in (0, 1, 3):                 # 3 of 4
        planted[j][w3] = 1.0 + 0j
    for j in (1, 2):                    # exactly half: not more than half
        planted[j][w2] = 3.0 + 0j
    sr = _run(monkeypatch, plan, planted)
    voted = dict(zip(sr.voted.tolist(), sr.votes.tolist()))
    assert voted.get(w3) == 3
    assert w2 not in voted
    # even K: the median of four values is the mean of the two middle ones (three equal 1, one 0)
    z = dict(zip(sr.voted.tolist(), sr.z))
    assert abs(z[w3] - 1.0) < 1e-15


def test_single_modulus_vote(monkeypatch):
    """K = 1: more than half of one modulus is that modulus."""
    N = 500
    plan = O.make_plan(N, 2, kappa=2, primes=[31])
    w = 201
    sr = _run(monkeypatch, plan, [{w: 1.0 + 0j}])
    assert dict(zip(sr.voted.tolist(), sr.votes.tolist())).get(w) == 1


def test_subbin_tie_takes_smallest_u(monkeypatch):
    N = 2000
    primes = [11, 13, 17, 19, 23]
    plan = O.make_plan(N, 4, kappa=2, primes=primes)
    p, j = 13, 1
    # two frequencies in the same bin b of p = 13 with equal magnitude; they differ modulo every
    # small modulus, so for each t they sit in different sub-bins u of the length 13 t measurement
    w1, w2 = 40, 40 + 13 * 29
    assert w1 % p == w2 % p and w2 <= N // 2
    b = w1 % p
    planted = [dict() for _ in primes]
    planted[j][w1] = 1.0 + 0j
    planted[j][w2] = 1j                 # |a| equal, both magnitudes exactly 1
    sr = _run(monkeypatch, plan, planted)
    for l, t in enumerate(plan.small):
        u1, u2 = (w1 % (p * t)) // p, (w2 % (p * t)) // p
        assert u1 != u2
        u = min(u1, u2)
        assert sr.residues[j][l, b] == (b + p * u) % t
        assert sr.margins[j][l, b] == 0.0
    # all-zero bins: every sub-bin ties at 0, u = 0, residue b mod t, candidate b
    for jj, pp in enumerate(primes):
        for bb in range(pp):
            if jj == j and bb == b:
                continue
            assert sr.cand[jj][bb] == bb


def test_tie_rule_changes_the_candidate(monkeypatch):
    """The rule matters: taking the larger u instead reconstructs a different frequency."""
    N = 2000
    primes = [11, 13, 17, 19, 23]
    plan = O.make_plan(N, 4, kappa=2, primes=primes)
    w1, w2 = 40, 40 + 13 * 29
    planted = [dict() for _ in primes]
    planted[1][w1] = 1.0 + 0j
    planted[1][w2] = 1j
    sr = _run(monkeypatch, plan, planted)
    b = w1 % 13
    got = sr.cand[1][b]
    # the smaller u of each small modulus picks one frequency's residue mod t; the candidate is
    # the CRT of those residues, not the frequency with the larger u in every modulus
    res_small = [min(((w1 % (13 * t)) // 13, (w2 % (13 * t)) // 13)) for t in plan.small]
    expect = O.to_band(O.crt([b] + [(b + 13 * u) % t for u, t in zip(res_small, plan.small)],
                             [13] + plan.small), 13 * math.prod(plan.small), N)
    assert got == expect
    res_large = [max(((w1 % (13 * t)) // 13, (w2 % (13 * t)) // 13)) for t in plan.small]
    other = O.to_band(O.crt([b] + [(b + 13 * u) % t for u, t in zip(res_large, plan.small)],
                            [13] + plan.small), 13 * math.prod(plan.small), N)
    assert other != got
