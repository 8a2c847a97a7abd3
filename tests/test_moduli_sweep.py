"""CPU sweep of the library's host-side choice of moduli (sft_choose_moduli_pool, no device work)
against the oracle's choose_primes and choose_small_moduli, over seeded random arguments across the
call's domain (2 <= N < 2^31, 1 <= s <= N, both prime pools, 64-bit seeds), beside the hand-picked
cases of test_abi.py.  Both sides draw K primes by SplitMix64 and a partial Fisher-Yates shuffle
(Lemma SFT_Ident_Coef_Est_in_Noise's random subset of moduli) and then the shortest run of small
primes t != p_j with p_1 prod(t) >= N, so any difference in the pool, the draw, the rounding of
c_p s or the stopping rule shows as unequal lists."""
import math

import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from oracle import dsft as O
from paper_1706_02740_gb300 import build as sft_build


@pytest.fixture(scope="module")
def lib():
    sft_build.build()
    return sft.load()


def _cases(seed, n, max_cps, max_k):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        N = int(round(math.exp(rng.uniform(math.log(2), math.log(2 ** 31 - 1)))))
        N = min(max(N, 2), 2 ** 31 - 1)
        s = int(round(math.exp(rng.uniform(0.0, math.log(min(N, 50000))))))
        s = min(max(s, 1), N)
        c_p = float(rng.choice([rng.uniform(0.5, 10.0), float(rng.integers(1, 9)), 2.5]))
        if c_p * s > max_cps:
            c_p = max_cps / s
        K = int(rng.integers(1, max_k + 1))
        seed64 = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        out.append((N, s, K, c_p, seed64))
    return out


@pytest.mark.parametrize("case", _cases(2024, 240, 2.0e5, 48))
def test_whole_pool_choice_matches_oracle(lib, case):
    N, s, K, c_p, seed = case
    primes, small = sft.sft_choose_moduli_pool(N, s, K, c_p, seed, sft.SFT_POOL_ALL)
    want = O.choose_primes(s, K, c_p, seed)
    assert primes == want
    assert small == O.choose_small_moduli(N, want)


@pytest.mark.parametrize("case", _cases(2025, 60, 2.0e4, 12))
def test_smooth_pool_choice_matches_oracle(lib, case):
    N, s, K, c_p, seed = case
    primes, small = sft.sft_choose_moduli_pool(N, s, K, c_p, seed, sft.SFT_POOL_SMOOTH)
    want = O.choose_primes(s, K, c_p, seed, "smooth")
    assert primes == want
    assert small == O.choose_small_moduli(N, want)


@pytest.mark.parametrize("s,c_p", [(1000, 3.0), (3, 10.0 / 3.0), (7, 1.0 / 7.0), (999, 1.001)])
def test_lower_end_of_the_pool_is_the_rounded_up_product(lib, s, c_p):
    """lo = max(ceil(c_p s), 5) in double arithmetic on both sides, including products that land on
    or near an integer."""
    primes, _ = sft.sft_choose_moduli_pool(2 ** 30, s, 4, c_p, 9, sft.SFT_POOL_ALL)
    lo = max(int(math.ceil(c_p * s)), 5)
    assert min(primes) >= lo
    assert primes == O.choose_primes(s, 4, c_p, 9)


def _det_cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        N = int(round(math.exp(rng.uniform(math.log(4), math.log(2 ** 31 - 1)))))
        N = min(max(N, 4), 2 ** 31 - 1)
        s = int(rng.integers(1, min(N, 150) + 1))
        c_p = float(rng.uniform(0.5, 8.0))
        out.append((N, s, c_p))
    return out


@pytest.mark.parametrize("case", _det_cases(2026, 80))
def test_deterministic_choice_matches_oracle_or_is_refused_alike(lib, case):
    """The deterministic inner SFT's K = 2 (s - 1) L + 1 smallest primes; the library refuses
    exactly when that K exceeds its 512 moduli."""
    N, s, c_p = case
    want = O.deterministic_primes(N, s, c_p)
    if len(want) > sft.SFT_MAX_K:
        with pytest.raises(sft.SftError):
            sft.sft_choose_moduli_deterministic(N, s, c_p)
        return
    primes, small = sft.sft_choose_moduli_deterministic(N, s, c_p)
    assert primes == want
    assert small == O.choose_small_moduli(N, want)
