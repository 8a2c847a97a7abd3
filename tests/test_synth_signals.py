"""CPU checks of the seeded input generators (synth/signals.py) against the workload recipe: the
spectra of Section 5.1 (s distinct frequencies in B = (-ceil(N/2), floor(N/2)], unit or
log-uniform magnitudes on [1e-2, 1], uniform phases), the samples as F^{-1} c in Section 2's
convention (checked by brute force against the DFT matrix F[w, j] = (-1)^w e^{-2 pi i w j / N} / N),
the noise of Section 5.4 (SNR = 20 log10(||f|| / ||n||) exactly, zero-mean circular Gaussian), the
per-configuration seeds, the mixed batch shapes and the Poisson request stream; and the device-side
generator (run on the CPU device) against the host one."""
import math

import numpy as np
import pytest

from synth.signals import (as_complex64, band_lo, config_signal, draw_batch_shapes, draw_spectrum,
                           draw_stream, make_signal, samples_from_spectrum, upcast)


@pytest.mark.parametrize("N", [1, 2, 7, 16, 1001, 2 ** 20])
def test_spectrum_frequencies_are_distinct_and_in_B(N):
    s = min(N, 64)
    w, c = draw_spectrum(N, s, seed=N, magnitude="unit")
    assert len(np.unique(w)) == s and np.all(np.diff(w) > 0)
    assert np.all(w >= band_lo(N)) and np.all(w <= N // 2)
    assert np.allclose(np.abs(c), 1.0, rtol=0, atol=1e-15)


def test_band_lo_is_the_smallest_element_of_B():
    for N in range(1, 40):
        B = [w for w in range(-N, N + 1) if -math.ceil(N / 2) < w <= N // 2]
        assert band_lo(N) == min(B) and len(B) == N


def test_whole_band_is_drawn_when_s_equals_N():
    for N in (5, 6, 13):
        w, _ = draw_spectrum(N, N, seed=3)
        assert w.tolist() == list(range(band_lo(N), N // 2 + 1))


def test_loguniform_magnitudes_and_uniform_phases():
    _, c = draw_spectrum(2 ** 24, 20000, seed=11, magnitude="loguniform")
    m = np.abs(c)
    assert m.min() >= 1e-2 and m.max() <= 1.0
    lower_decade = np.mean(m < 0.1)                  # log-uniform over two decades: half below 0.1
    assert abs(lower_decade - 0.5) < 0.02
    assert abs(np.mean(c / m)) < 0.03                # uniform phase: the mean unit phasor vanishes


@pytest.mark.parametrize("N", [1, 2, 15, 16, 30])
def test_samples_realise_the_spectrum_in_the_papers_dft_convention(N):
    s = min(N, 5)
    w, c = draw_spectrum(N, s, seed=7 + N, magnitude="loguniform")
    f = samples_from_spectrum(N, w, c)
    B = np.arange(band_lo(N), N // 2 + 1)
    j = np.arange(N)
    F = ((-1.0) ** B)[:, None] * np.exp(-2j * math.pi * np.outer(B, j) / N) / N
    fhat = F @ f
    want = np.zeros(N, dtype=np.complex128)
    want[w - band_lo(N)] = c
    assert np.max(np.abs(fhat - want)) < 1e-13


@pytest.mark.parametrize("snr", [10.0, 20.0, 30.0, 40.0])
def test_noise_meets_the_snr_exactly_and_is_circular_gaussian(snr):
    N, s = 2 ** 16, 32
    clean = make_signal(N, s, seed=5, magnitude="unit")
    noisy = make_signal(N, s, seed=5, magnitude="unit", snr_db=snr)
    n = noisy.f - clean.f
    assert abs(np.linalg.norm(n) - noisy.noise_norm) <= 1e-12 * noisy.noise_norm
    assert abs(20 * math.log10(np.linalg.norm(clean.f) / np.linalg.norm(n)) - snr) < 1e-9
    z = n / (np.linalg.norm(n) / math.sqrt(N))       # unit variance per complex sample
    assert abs(np.mean(z)) < 5 / math.sqrt(N)
    assert abs(np.var(z.real) - 0.5) < 0.02 and abs(np.var(z.imag) - 0.5) < 0.02
    assert abs(np.mean(z.real * z.imag)) < 0.02
    assert np.array_equal(noisy.omega, clean.omega) and np.array_equal(noisy.coef, clean.coef)


def test_seeds_reproduce_and_configurations_use_1000_config_plus_trial():
    a = make_signal(4096, 8, seed=3, magnitude="loguniform", snr_db=20.0)
    b = make_signal(4096, 8, seed=3, magnitude="loguniform", snr_db=20.0)
    c = make_signal(4096, 8, seed=4, magnitude="loguniform", snr_db=20.0)
    assert np.array_equal(a.f, b.f) and not np.array_equal(a.f, c.f)
    for config, trial, N, s, mag, snr in [(1, 0, 2 ** 10, 8, "unit", None),
                                          (2, 3, 2 ** 11, 16, "unit", 20.0),
                                          (3, 9, 2 ** 12, 20, "loguniform", 30.0)]:
        got = config_signal(config, trial, N=N, s=s)
        want = make_signal(N, s, 1000 * config + trial, mag, snr)
        assert np.array_equal(got.f, want.f) and np.array_equal(got.omega, want.omega)


def test_complex64_round_trip_is_exact():
    f = make_signal(1000, 5, seed=1, snr_db=30.0).f
    f32 = as_complex64(f)
    assert f32.dtype == np.complex64 and f32.flags.c_contiguous
    assert np.array_equal(upcast(f32).astype(np.complex64), f32)


def _is_pow2(n):
    return n & (n - 1) == 0


def _is_prime(n):
    return n > 1 and all(n % d for d in range(2, int(n ** 0.5) + 1))


def test_batch_shapes_mix_lengths_as_stated():
    shapes = draw_batch_shapes(4096, seed=4000)
    Ns = np.array([n for n, _ in shapes])
    ss = np.array([s for _, s in shapes])
    assert Ns.min() >= 2 ** 18 and Ns.max() <= 2 ** 24 + 200          # a prime gap above the top
    odd = [n for n in Ns if not _is_pow2(int(n))]
    assert 0.22 < len(odd) / len(Ns) < 0.28
    primes = sum(_is_prime(int(n)) for n in odd[:400])
    assert 0.35 < primes / min(400, len(odd)) < 0.65                  # about half of them prime
    assert ss.min() >= 16 and ss.max() <= 512 and np.all(ss <= Ns)
    e = np.log2(Ns[[_is_pow2(int(n)) for n in Ns]])
    assert e.min() == 18 and e.max() == 24 and abs(np.mean(e) - 21) < 0.2   # log-uniform


def test_request_stream_is_poisson_with_the_stated_ranges():
    rate = 500.0
    st = draw_stream(8000, seed=5000, rate_hz=rate)
    t = np.array([r[0] for r in st])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(np.mean(gaps) * rate - 1) < 0.04
    assert abs(np.std(gaps) / np.mean(gaps) - 1) < 0.05                 # exponential: cv = 1
    N = np.array([r[1] for r in st])
    s = np.array([r[2] for r in st])
    snr = np.array([r[3] for r in st])
    assert N.min() >= 2 ** 16 and N.max() <= 2 ** 27
    assert abs(np.mean(np.log2(N)) - 21.5) < 0.1                       # log-uniform over 11 octaves
    assert s.min() >= 8 and s.max() <= 2048 and np.all(s <= N)
    assert snr.min() >= 10 and snr.max() <= 40 and abs(np.mean(snr) - 25) < 0.5
    assert np.mean(N % 2 == 1) > 0.4                                   # arbitrary integers


@pytest.mark.parametrize("N,s,mag", [(1024, 8, "unit"), (3 ** 7, 12, "loguniform"),
                                     (4099, 5, "unit")])
def test_device_generator_follows_the_same_recipe(N, s, mag):
    """synth.device_signals (run here on the CPU device): noiseless it is the host generator's
    signal; with noise it keeps the spectrum and meets the SNR exactly; the FFT-free direct sum
    (any N up to 2^31 - 1) gives the same samples, across chunk boundaries."""
    torch = pytest.importorskip("torch")
    from synth.device_signals import make_device_signal, make_device_sparse_signal_direct
    host = make_signal(N, s, seed=N + 1, magnitude=mag)
    f, w, c = make_device_signal(N, s, N + 1, mag, None, device="cpu", dtype=torch.complex128)
    assert np.array_equal(w, host.omega) and np.array_equal(c, host.coef)
    assert np.max(np.abs(f.numpy() - host.f)) <= 1e-12 * np.max(np.abs(host.f))
    fn, _, _ = make_device_signal(N, s, N + 1, mag, 20.0, device="cpu", dtype=torch.complex128)
    noise = fn.numpy() - f.numpy()
    assert abs(20 * math.log10(np.linalg.norm(f.numpy()) / np.linalg.norm(noise)) - 20.0) < 1e-9
    d = make_device_sparse_signal_direct(N, w, c, device="cpu", chunk=1000)
    assert d.dtype == torch.complex64
    assert np.max(np.abs(d.numpy() - host.f)) <= 1e-6 * np.max(np.abs(host.f))
