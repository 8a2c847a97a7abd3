"""CPU FP64 oracle for the Gaussian-filtered discrete sparse Fourier transform (Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import or run this module; the product path never does.  It shares no code with the CUDA path.

It is the method written out in the paper's order and notation, slow and plain:

* parameters c1, c2, L and the shifts q (Algorithm 1, its set-up and shift loop);
* the periodic Gaussian g (eq. Def_Periodic_Gaussian) and its Fourier coefficients
  g_hat_w = exp(-c1^2 w^2 / 2) / sqrt(2 pi) (Lemma Periodic_Gaussian_FC);
* resampling: the truncated semi-discrete convolution (eq. UntruncatedFiniteSum cut to the window
  j' - kappa .. j' + kappa of Lemma fewer_points_error) with the modulated filter;
* the unequally spaced SFT A, read from Appendix B as: prime-modulus DFT measurements E_j
  (eq. DFT_GKlam_Comp) at nodes -pi + 2 pi k / P, identification of each bin's frequency from its
  residues modulo small coprime moduli plus the Chinese remainder theorem, a majority vote over the
  prime moduli ("more than half of the j"), and componentwise median estimates (the sqrt(2) of
  eq. GSFT_Estimate);
* band restriction, division by the filter's Fourier coefficient, and the global top-s.

Readings of passages the paper leaves open (modulation sign, node sign, which bins are candidates,
window-centre ties, even N, median of an even count) are the ones listed in the design notes;
each is marked "reading" where it is used below.

Library primitives used as single steps: numpy.fft.fft (a DFT), numpy.median, numpy.lexsort.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
SQRT_2PI = math.sqrt(2.0 * math.pi)


# --------------------------------------------------------------------------------------------
# Seeded choice of the prime moduli (randomized variant of A, Lemma SFT_Ident_Coef_Est_in_Noise)
# --------------------------------------------------------------------------------------------
def splitmix64(state: int):
    """One step of the SplitMix64 generator (Steele, Lea, Flood 2014; constants as published by
    Vigna).  Returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, (z ^ (z >> 31)) & MASK64


def is_prime(n: int) -> bool:
    """Trial division (plain and exact for the sizes used here)."""
    if n < 2:
        return False
    if n < 4:
        return True
    if n % 2 == 0:
        return False
    i = 3
    while i * i <= n:
        if n % i == 0:
            return False
        i += 2
    return True


def primes_from(lo: int, count: int) -> list[int]:
    out, n = [], max(2, lo)
    while len(out) < count:
        if is_prime(n):
            out.append(n)
        n += 1
    return out


SMOOTH_FACTORS = (2, 3, 5, 7, 11, 13)


def is_smooth(n: int, factors=SMOOTH_FACTORS) -> bool:
    """True when n >= 1 has no prime factor outside `factors` (trial division)."""
    if n < 1:
        return False
    for t in factors:
        while n % t == 0:
            n //= t
    return n == 1


def smooth_primes_from(lo: int, count: int) -> list[int]:
    """The `count` smallest primes p >= lo whose p - 1 has no prime factor above 13."""
    out, n = [], max(3, lo)
    while len(out) < count:
        if is_prime(n) and is_smooth(n - 1):
            out.append(n)
        n += 1
    return out


def choose_primes(s: int, K: int, c_p: float, seed: int, pool: str = "all") -> list[int]:
    """K distinct primes drawn by a seeded partial Fisher-Yates shuffle from a pool of 4K primes
    >= max(ceil(c_p * s), 5); returned ascending.  The Monte Carlo variant reads a random subset of
    the deterministic algorithm's moduli (Lemma SFT_Ident_Coef_Est_in_Noise, second paragraph).
    pool "all": the 4K smallest primes; pool "smooth" (a choice of this implementation, not the
    paper's): the 4K smallest primes whose p - 1 has no prime factor above 13 (the measurements
    are then DFTs of prime length p whose p - 1 is a product of small radices)."""
    lo = max(int(math.ceil(c_p * s)), 5)
    if pool == "all":
        cands = primes_from(lo, 4 * K)
    elif pool == "smooth":
        cands = smooth_primes_from(lo, 4 * K)
    else:
        raise ValueError(pool)
    state = seed & MASK64
    for i in range(K):
        state, r = splitmix64(state)
        j = i + (r % (len(cands) - i))
        cands[i], cands[j] = cands[j], cands[i]
    return sorted(cands[:K])


def deterministic_primes(N: int, s: int, c_p: float) -> list[int]:
    """The deterministic inner SFT's moduli (Algorithm 3 of the cited work, first paragraph of
    Lemma SFT_Ident_Coef_Est_in_Noise): the K smallest primes >= max(ceil(c_p * s), 5) with
    K = 2 (s - 1) L + 1, where L is the largest integer with p_1^L <= N - 1.  A product of L + 1 of
    these primes exceeds N - 1, so two distinct frequencies of B (which differ by less than N) share
    a residue modulo at most L of them; with s frequencies each one is alone in its bin for at
    least K - (s - 1) L > K / 2 of the primes."""
    lo = max(int(math.ceil(c_p * s)), 5)
    p1 = primes_from(lo, 1)[0]
    L, pw = 0, p1
    while pw <= N - 1:
        L += 1
        pw *= p1
    K = 2 * (s - 1) * L + 1
    return primes_from(lo, K)


def choose_small_moduli(N: int, primes: list[int]) -> list[int]:
    """Smallest primes t (ascending), none equal to a p_j, until p_1 * prod(t) >= N, so that the
    CRT residue system of every p_j has a modulus M_j = p_j * prod(t) >= N (unique w in B)."""
    T, prod, t = [], primes[0], 2
    while prod < N:
        if is_prime(t) and t not in primes:
            T.append(t)
            prod *= t
        t += 1
    return T


# --------------------------------------------------------------------------------------------
# Plan (Algorithm 1, set-up)
# --------------------------------------------------------------------------------------------
@dataclass
class Plan:
    N: int
    s: int
    kappa: int
    alpha: float
    beta: float
    c1: float
    L: int
    shifts: list[int]
    primes: list[int]
    small: list[int]
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return len(self.primes)


def ceil_half(N: int) -> int:
    return (N + 1) // 2


def make_plan(N: int, s: int, kappa: int = 6, alpha: float = 1.5, beta: float = 1.5,
              K: int = 5, c_p: float = 3.0, seed: int = 0, primes=None, small=None,
              n_shifts: int | None = None, deterministic: bool = False,
              pool: str = "all") -> Plan:
    """c1 = beta sqrt(ln N) / N, c2 = alpha sqrt(ln N) / 2, L = ceil(N / (alpha sqrt(ln N))),
    q_j = -ceil(N/2) + 1 + (2j - 1) L for j = 1..ceil(c2)  (Algorithm 1)."""
    if N < 2 or not (1 <= s <= N):
        raise ValueError("need N >= 2 and 1 <= s <= N")
    if 2 * kappa + 1 > N:
        raise ValueError("window 2*kappa+1 must not exceed N")
    lnN = math.log(N)
    c1 = beta * math.sqrt(lnN) / N
    L = int(math.ceil(N / (alpha * math.sqrt(lnN))))
    nq = int(math.ceil(alpha * math.sqrt(lnN) / 2.0)) if n_shifts is None else int(n_shifts)
    if 2 * nq * L < N:
        raise ValueError("the bands [q-L, q+L) do not cover B")
    shifts = [-ceil_half(N) + 1 + (2 * j - 1) * L for j in range(1, nq + 1)]
    if primes is None:
        primes = (deterministic_primes(N, s, c_p) if deterministic
                  else choose_primes(s, K, c_p, seed, pool))
    primes = sorted(int(p) for p in primes)
    if small is None:
        small = choose_small_moduli(N, primes)
    small = [int(t) for t in small]
    for a in range(len(small)):
        for b in range(a + 1, len(small)):
            if math.gcd(small[a], small[b]) != 1:
                raise ValueError("small moduli must be pairwise coprime")
    for p in primes:
        for t in small:
            if math.gcd(p, t) != 1:
                raise ValueError("every p_j must be coprime to every small modulus")
    if primes[0] * math.prod(small) < N:
        raise ValueError("p_1 * prod(T) must be >= N")
    return Plan(N, s, kappa, alpha, beta, c1, L, shifts, primes, small)


# --------------------------------------------------------------------------------------------
# The periodic Gaussian filter (Section 2.1)
# --------------------------------------------------------------------------------------------
def g_periodic(x, c1: float):
    """g(x) = (1/c1) sum_n exp(-(x - 2 pi n)^2 / (2 c1^2))  (eq. Def_Periodic_Gaussian); the sum
    is cut where its terms are below double precision for |x| <= pi."""
    x = np.asarray(x, dtype=np.float64)
    nmax = 2 + int(math.ceil(10.0 * c1))
    total = np.zeros_like(x)
    for n in range(-nmax, nmax + 1):
        total += np.exp(-((x - 2.0 * math.pi * n) ** 2) / (2.0 * c1 * c1))
    return total / c1


def g_hat(w, c1: float):
    """Fourier series coefficients of g (Lemma Periodic_Gaussian_FC)."""
    w = np.asarray(w, dtype=np.float64)
    return np.exp(-(c1 * c1) * w * w / 2.0) / SQRT_2PI


# --------------------------------------------------------------------------------------------
# Resampling: (g_q * f)(x) from f by a truncated semi-discrete convolution (Section 3.1)
# --------------------------------------------------------------------------------------------
def nearest_grid(N: int, P: int, k):
    """j' = argmin_j |x - y_j| for x = -pi + 2 pi k / P, y_j = -pi + 2 pi j / N: the rounding of
    kN/P, ties rounded up (reading of the argmin of Lemma fewer_points_error)."""
    k = np.asarray(k, dtype=np.int64)
    return (2 * k * N + P) // (2 * P)


def resample(f: np.ndarray, plan: Plan, P: int, k, q: int) -> np.ndarray:
    """h_q(x_k) ~= (1/N) sum_{j=j'-kappa}^{j'+kappa} f_j g_q(x_k - y_j), indices of f mod N.

    The modulated filter is g_q(x) = exp(+i q x) g(x), whose Fourier coefficients are
    g_hat_{w - q} (reading of the modulation of Algorithm 1 and Section 4; the band kept and the
    division both centre on +q).  x - y_j is formed exactly as 2 pi d / (P N) with the integer
    d = kN - jP, and the phase q (x - y_j) is reduced exactly as the integer q d mod P N.
    """
    N = plan.N
    k = np.asarray(k, dtype=np.int64)
    jp = nearest_grid(N, P, k)
    PN = P * N
    h = np.zeros(k.shape, dtype=np.complex128)
    for i in range(-plan.kappa, plan.kappa + 1):
        j = jp + i
        d = k * N - j * P
        delta = 2.0 * math.pi * d.astype(np.float64) / PN
        w = g_periodic(delta, plan.c1) / N
        r = np.mod(q * d, PN)
        phase = 2.0 * math.pi * r.astype(np.float64) / PN
        h += f[np.mod(j, N)] * w * np.exp(1j * phase)
    return h


# --------------------------------------------------------------------------------------------
# Chinese remainder reconstruction (identification step of A)
# --------------------------------------------------------------------------------------------
def crt(residues, moduli) -> int:
    """Garner's mixed-radix reconstruction of the unique x in [0, prod(moduli)) with
    x = residues[i] mod moduli[i] (moduli pairwise coprime)."""
    x, M = 0, 1
    for a, m in zip(residues, moduli):
        v = ((int(a) - x) * pow(M, -1, m)) % m
        x += M * v
        M *= m
    return x


def to_band(wt: int, M: int, N: int):
    """Map a residue class representative wt in [0, M), M >= N, to the member of
    B = (-ceil(N/2), floor(N/2)], or None if that class has no member of B."""
    w = wt if wt <= N // 2 else wt - M
    return w if w > -ceil_half(N) else None


def parity_sign(w) -> np.ndarray:
    """(-1)^w for integer w (exact, from the parity)."""
    w = np.asarray(w, dtype=np.int64)
    return np.where(np.mod(w, 2) == 0, 1.0, -1.0)


# --------------------------------------------------------------------------------------------
# The unequally spaced SFT A on one shift's filtered samples (Appendix B)
# --------------------------------------------------------------------------------------------
@dataclass
class ShiftResult:
    q: int
    Y: list                  # Y[j]: length-p_j DFT of the p_j samples, / p_j
    residues: list           # residues[j]: int array [|T|, p_j]
    margins: list            # margins[j]: float array [|T|, p_j], (|X_1st|^2-|X_2nd|^2)/|X_1st|^2
    cand: list               # cand[j]: object array [p_j] of int or None
    voted: np.ndarray        # int64 voted frequencies (ascending)
    votes: np.ndarray        # vote count of each voted frequency
    z: np.ndarray            # complex128 median estimates of the voted frequencies
    temp_w: np.ndarray       # R_temp: top-s of the voted set by |z|
    temp_z: np.ndarray


def dft_bins(samples: np.ndarray) -> np.ndarray:
    """E_h = (1/P) sum_k samples[k] exp(-2 pi i k h / P), h = 0..P-1 (eq. DFT_GKlam_Comp with
    s_j = P), for samples taken at the nodes -pi + 2 pi k / P."""
    return np.fft.fft(samples) / len(samples)


def measure(f: np.ndarray, plan: Plan, q: int, P: int) -> np.ndarray:
    """The length-P measurement of the shift-q filtered function: resample at the P nodes, then
    take the normalised DFT."""
    return dft_bins(resample(f, plan, P, np.arange(P, dtype=np.int64), q))


def median_estimate(Y: list, primes: list, w: int) -> complex:
    """z_w = (-1)^w (median_j Re Y_j[w mod p_j] + i median_j Im Y_j[w mod p_j]) over all moduli
    (estimation step, eq. GSFT_Estimate; numpy's median of an even count is the mean of the two
    middle values)."""
    vals = np.array([Y[jj][int(w) % p] for jj, p in enumerate(primes)])
    return complex(parity_sign(w) * (np.median(vals.real) + 1j * np.median(vals.imag)))


def majority_vote(cand: list, K: int):
    """Vote of the identification step (Appendix B, "more than half of the j"): w counts once for
    every modulus j one of whose bins reconstructed exactly w (cand[j][b] is the frequency bin b
    of modulus j reconstructed, or None); the w found by more than half of the K moduli are kept.
    Returns the kept frequencies, ascending, and how many moduli found each."""
    found = {}
    for jj, cj in enumerate(cand):
        for w in cj:
            if w is not None:
                found.setdefault(int(w), set()).add(jj)
    need = K // 2 + 1
    voted = sorted(w for w, js in found.items() if len(js) >= need)
    voted = np.array(voted, dtype=np.int64)
    votes = np.array([len(found[int(w)]) for w in voted], dtype=np.int64)
    return voted, votes


def ussft_shift(f: np.ndarray, plan: Plan, q: int) -> ShiftResult:
    N, K = plan.N, plan.K
    Y, residues, margins, cand = [], [], [], []
    for p in plan.primes:
        Yj = measure(f, plan, q, p)
        Y.append(Yj)
        res = np.zeros((len(plan.small), p), dtype=np.int64)
        mar = np.ones((len(plan.small), p), dtype=np.float64)
        b = np.arange(p, dtype=np.int64)
        for l, t in enumerate(plan.small):
            X = measure(f, plan, q, p * t)
            sub = X.reshape(t, p)                     # sub[u, b] = X[b + p u]
            mag = np.abs(sub) ** 2
            ustar = np.argmax(mag, axis=0)           # first maximum: ties go to the smallest u
            res[l] = np.mod(b + p * ustar, t)
            if t > 1:
                srt = np.sort(mag, axis=0)
                top, second = srt[-1], srt[-2]
                with np.errstate(invalid="ignore", divide="ignore"):
                    mar[l] = np.where(top > 0, (top - second) / top, 0.0)
        residues.append(res)
        margins.append(mar)
        M = p * math.prod(plan.small)
        cj = np.empty(p, dtype=object)
        for bb in range(p):
            wt = crt([bb] + [int(res[l, bb]) for l in range(len(plan.small))],
                     [p] + plan.small)
            cj[bb] = to_band(wt, M, N)
        cand.append(cj)

    voted, votes = majority_vote(cand, K)

    # Estimate: componentwise medians over all K moduli of the bin holding w (eq. GSFT_Estimate),
    # times (-1)^w because the nodes start at -pi (reading of the node sign).
    z = np.array([median_estimate(Y, plan.primes, int(w)) for w in voted], dtype=np.complex128)

    # R_temp: an s-sparse approximation, the s largest |z| (ties: smaller w first, Section 2).
    temp_w, temp_z = best_s_term(voted, z, plan.s)
    return ShiftResult(q, Y, residues, margins, cand, voted, votes, z, temp_w, temp_z)


# --------------------------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------------------------
@dataclass
class Result:
    freqs: np.ndarray        # int64, at most s, sorted by |coef| descending, ties w ascending
    coefs: np.ndarray        # complex128
    shifts: list             # ShiftResult per q
    pool_w: np.ndarray       # R-hat before the final top-s
    pool_c: np.ndarray
    pool_q: np.ndarray


def dsft(f: np.ndarray, plan: Plan) -> Result:
    f = np.asarray(f, dtype=np.complex128)
    if f.shape != (plan.N,):
        raise ValueError("f must have length N")
    N, L = plan.N, plan.L
    lo, hi = -ceil_half(N) + 1, N // 2
    pool_w, pool_c, pool_q, shifts = [], [], [], []
    for q in plan.shifts:
        sr = ussft_shift(f, plan, q)
        shifts.append(sr)
        for w, zw in zip(sr.temp_w, sr.temp_z):
            w = int(w)
            if q - L <= w < q + L and lo <= w <= hi:
                # divide by the modulated filter's coefficient g_hat_{w - q}
                pool_w.append(w)
                pool_c.append(zw / g_hat(w - q, plan.c1))
                pool_q.append(q)
    pool_w = np.array(pool_w, dtype=np.int64)
    pool_c = np.array(pool_c, dtype=np.complex128)
    pool_q = np.array(pool_q, dtype=np.int64)
    out_w, out_c = best_s_term(pool_w, pool_c, plan.s)      # the final choice of Algorithm 1
    return Result(out_w, out_c, shifts, pool_w, pool_c, pool_q)


# --------------------------------------------------------------------------------------------
# Plain definitions used as pins
# --------------------------------------------------------------------------------------------
def dft_matrix_apply(f: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """f_hat = F f with F[w, j] = (-1)^w exp(-2 pi i w j / N) / N, w in B (eq. Disc_Fourier_Def),
    by the O(N^2) sum; returns (w, f_hat)."""
    N = len(f)
    w = np.arange(-ceil_half(N) + 1, N // 2 + 1, dtype=np.int64)
    j = np.arange(N, dtype=np.int64)
    E = np.exp(-2j * math.pi * np.mod(np.outer(w, j), N) / N)
    return w, parity_sign(w) * (E @ f) / N


def best_s_term(w: np.ndarray, fh: np.ndarray, s: int):
    """R_s^opt: the s largest |f_hat_w|, ties broken by the smaller w (Section 2)."""
    order = np.lexsort((w, -np.abs(fh)))[:s]
    return w[order], fh[order]
