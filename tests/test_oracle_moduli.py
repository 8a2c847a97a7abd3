"""Pins of the oracle's moduli pools.

* is_smooth agrees with the largest prime factor from a sieve (no prime factor above 13);
* smooth_primes_from returns exactly the smallest primes p >= lo with p - 1 smooth (brute force
  over the range), with known members and non-members;
* choose_primes over either pool draws K distinct members of that pool, the same ones for the
  same seed, and the draw is the published partial Fisher-Yates with SplitMix64 (checked by
  replaying it on the pool by hand).
"""
import pytest

from oracle import dsft as O


def _largest_prime_factor_table(n_max):
    lpf = list(range(n_max + 1))
    for i in range(2, n_max + 1):
        if lpf[i] == i:                     # i is prime: it is the largest factor of its multiples so far
            for j in range(2 * i, n_max + 1, i):
                lpf[j] = i
    # the sieve above leaves the largest prime factor in lpf[j] since primes come in increasing order
    return lpf


def test_is_smooth_against_a_sieve():
    lpf = _largest_prime_factor_table(20000)
    for n in range(2, 20001):
        assert O.is_smooth(n) == (lpf[n] <= 13), n
    assert O.is_smooth(1)


@pytest.mark.parametrize("p,smooth", [(3001, True), (3137, True), (3011, False), (12289, True),
                                      (65537, True), (8191, True), (4093, False), (3361, True),
                                      (3457, True), (4099, False)])
def test_known_members(p, smooth):
    assert O.is_prime(p)
    assert (p in O.smooth_primes_from(p, 1)) == smooth


@pytest.mark.parametrize("lo,count", [(5, 12), (24, 20), (300, 20), (3000, 20), (12000, 8)])
def test_smooth_pool_is_the_smallest_qualifying_primes(lo, count):
    got = O.smooth_primes_from(lo, count)
    brute = [n for n in range(lo, got[-1] + 1) if O.is_prime(n) and O.is_smooth(n - 1)]
    assert got == brute[:count] and len(brute) == count
    lpf = _largest_prime_factor_table(got[-1])
    assert all(lpf[p - 1] <= 13 for p in got)


@pytest.mark.parametrize("pool,lister", [("all", O.primes_from), ("smooth", O.smooth_primes_from)])
@pytest.mark.parametrize("s,K,c_p,seed", [(1000, 5, 3.0, 1), (64, 7, 3.0, 9), (8, 3, 4.0, 2 ** 63 + 11)])
def test_choice_draws_from_the_pool(pool, lister, s, K, c_p, seed):
    lo = max(-(-int(c_p * s * 1000) // 1000), 5)
    cands = lister(lo, 4 * K)
    got = O.choose_primes(s, K, c_p, seed, pool)
    assert got == sorted(got) and len(set(got)) == K and set(got) <= set(cands)
    assert O.choose_primes(s, K, c_p, seed, pool) == got
    # replay the partial Fisher-Yates shuffle by hand
    state, arr = seed & O.MASK64, list(cands)
    for i in range(K):
        state, r = O.splitmix64(state)
        j = i + r % (len(arr) - i)
        arr[i], arr[j] = arr[j], arr[i]
    assert sorted(arr[:K]) == got


def test_pools_differ_and_seeds_differ():
    a = O.choose_primes(1000, 5, 3.0, 1, "all")
    b = O.choose_primes(1000, 5, 3.0, 1, "smooth")
    assert a != b and all(O.is_smooth(p - 1) for p in b)
    assert O.choose_primes(1000, 5, 3.0, 2, "smooth") != b
    with pytest.raises(ValueError):
        O.choose_primes(1000, 5, 3.0, 1, "other")
