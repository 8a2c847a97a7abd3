"""Seeded synthetic input signals shaped like the paper's experiments (Section 5.1, 5.4).

This module only draws random inputs; it contains none of the sparse Fourier transform's
arithmetic.  Both the CPU oracle and the CUDA path consume the arrays it returns.

Conventions (Section 2): the frequency set is B = (-ceil(N/2), floor(N/2)] and the DFT matrix is
F[w, j] = (-1)^w exp(-2 pi i w j / N) / N, so a spectrum {c_w} is realised as the sample vector
f_j = sum_w c_w (-1)^w exp(2 pi i w j / N), j = 0..N-1, i.e. F f = c.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def band_lo(N: int) -> int:
    """Smallest element of B = (-ceil(N/2), floor(N/2)] (Section 2)."""
    return -((N + 1) // 2) + 1


@dataclass
class SparseSignal:
    N: int
    omega: np.ndarray      # int64, frequencies in B (sorted ascending)
    coef: np.ndarray       # complex128, Fourier coefficients of f at omega
    f: np.ndarray          # complex128 samples f_j = f(-pi + 2 pi j / N), noise included
    noise_norm: float      # ||n||_2 of the added noise (0 when noiseless)


def draw_spectrum(N: int, s: int, seed: int, magnitude: str = "unit",
                  mag_range: tuple[float, float] = (1e-2, 1.0)):
    """s distinct frequencies uniform over B, random phase, unit or log-uniform magnitude.

    Section 5.1 draws frequencies from [0, N); they are mapped into B by w -> w - N for
    w > floor(N/2), which is the same set of DFT entries.
    """
    if not (1 <= s <= N):
        raise ValueError("need 1 <= s <= N")
    rng = np.random.default_rng(seed)
    raw = rng.choice(N, size=s, replace=False).astype(np.int64)
    omega = np.where(raw > N // 2, raw - N, raw)
    omega.sort()
    phase = rng.uniform(0.0, 2.0 * math.pi, size=s)
    if magnitude == "unit":
        mag = np.ones(s)
    elif magnitude == "loguniform":
        lo, hi = mag_range
        mag = np.exp(rng.uniform(math.log(lo), math.log(hi), size=s))
    else:
        raise ValueError(magnitude)
    coef = mag * np.exp(1j * phase)
    return omega, coef


def samples_from_spectrum(N: int, omega: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """f = F^{-1} c via one inverse FFT (the input is defined by its spectrum)."""
    a = np.zeros(N, dtype=np.complex128)
    sign = np.where(omega % 2 == 0, 1.0, -1.0)
    np.add.at(a, np.mod(omega, N), coef * sign)
    return np.fft.ifft(a) * N


def complex_gaussian_noise(N: int, target_norm: float, seed: int) -> np.ndarray:
    """i.i.d. mean-zero complex Gaussian vector rescaled to the exact 2-norm target_norm."""
    rng = np.random.default_rng(seed ^ 0x5EED5EED)
    n = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    nn = np.linalg.norm(n)
    return n * (target_norm / nn) if nn > 0 else n


def make_signal(N: int, s: int, seed: int, magnitude: str = "unit",
                snr_db: float | None = None,
                mag_range: tuple[float, float] = (1e-2, 1.0)) -> SparseSignal:
    """Section 5.1 generator plus the Section 5.4 noise model.

    SNR = 20 log10(||f||_2 / ||n||_2) (footnote of Section 5.4, log read as log10).
    """
    omega, coef = draw_spectrum(N, s, seed, magnitude, mag_range)
    f = samples_from_spectrum(N, omega, coef)
    noise_norm = 0.0
    if snr_db is not None:
        noise_norm = float(np.linalg.norm(f)) * 10.0 ** (-snr_db / 20.0)
        f = f + complex_gaussian_noise(N, noise_norm, seed)
    return SparseSignal(N=N, omega=omega, coef=coef, f=f, noise_norm=noise_norm)


def as_complex64(f: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(f.astype(np.complex64))


def upcast(f32: np.ndarray) -> np.ndarray:
    """Exact complex64 -> complex128 widening (both paths then see identical values)."""
    return f32.astype(np.complex128)


# Workload recipes for the five configurations (seed = 1000 * config + trial).
def config_signal(config: int, trial: int = 0, N: int | None = None, s: int | None = None):
    seed = 1000 * config + trial
    if config == 1:
        return make_signal(N or 2 ** 16, s or 8, seed, "unit", None)
    if config == 2:
        return make_signal(N or 2 ** 22, s or 64, seed, "unit", 20.0)
    if config == 3:
        return make_signal(N or 2 ** 26, s or 1000, seed, "loguniform", 30.0)
    raise ValueError("configs 4 and 5 are drawn by draw_batch / draw_stream")


def draw_batch_shapes(count: int, seed: int, n_lo: int = 2 ** 18, n_hi: int = 2 ** 24,
                      s_lo: int = 16, s_hi: int = 512):
    """Mixed sizes for the batched launch: N log-uniform over [n_lo, n_hi] with a quarter of the
    signals at a non-power-of-two length (some of them prime), s uniform over [s_lo, s_hi]."""
    rng = np.random.default_rng(seed)
    shapes = []
    for i in range(count):
        e = rng.uniform(math.log2(n_lo), math.log2(n_hi))
        if rng.uniform() < 0.25:
            n = max(n_lo, min(n_hi, int(round(2.0 ** e))))
            if rng.uniform() < 0.5:
                n = _next_prime(n)          # may exceed n_hi by a prime gap
            elif n & (n - 1) == 0:
                n += 1
        else:
            n = 2 ** int(round(e))
        s = int(rng.integers(s_lo, s_hi + 1))
        shapes.append((n, min(s, n)))
    return shapes


def draw_stream(count: int, seed: int, rate_hz: float, n_lo: int = 2 ** 16, n_hi: int = 2 ** 27,
                s_lo: int = 8, s_hi: int = 2048, snr_lo: float = 10.0, snr_hi: float = 40.0):
    """Poisson arrivals of requests with N log-uniform (arbitrary integers), s log-uniform and
    SNR uniform; returns a list of (arrival_time_s, N, s, snr_db)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_hz)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        s = int(round(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        snr = float(rng.uniform(snr_lo, snr_hi))
        out.append((t, n, min(s, n), snr))
    return out


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    i = 3
    while i * i <= n:
        if n % i == 0:
            return False
        i += 2
    return True


def _next_prime(n: int) -> int:
    while not _is_prime(n):
        n += 1
    return n
