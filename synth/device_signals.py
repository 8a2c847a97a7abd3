"""Seeded synthetic signals generated directly in device memory (for large N, where building the
input on the host would dominate a benchmark's set-up time).  Same recipe as synth.signals:
s distinct frequencies uniform over B, random phase, unit or log-uniform magnitude, f = F^{-1} c
by one inverse FFT, plus i.i.d. complex Gaussian noise rescaled to an exact SNR.  Contains none of
the sparse Fourier transform's arithmetic."""
from __future__ import annotations

import numpy as np

from synth.signals import draw_spectrum


def make_device_signal(N: int, s: int, seed: int, magnitude: str = "loguniform",
                       snr_db: float | None = 30.0, device="cuda", dtype=None):
    import torch
    dtype = dtype or torch.complex64
    omega, coef = draw_spectrum(N, s, seed, magnitude)
    a = torch.zeros(N, dtype=torch.complex128, device=device)
    sign = np.where(omega % 2 == 0, 1.0, -1.0)
    a[torch.from_numpy(np.mod(omega, N)).to(device)] = torch.from_numpy(coef * sign).to(device)
    f = torch.fft.ifft(a) * N
    del a
    if snr_db is not None:
        g = torch.Generator(device=device)
        g.manual_seed(seed ^ 0x5EED5EED)
        n = torch.complex(torch.randn(N, generator=g, device=device, dtype=torch.float64),
                          torch.randn(N, generator=g, device=device, dtype=torch.float64))
        target = torch.linalg.vector_norm(f) * 10.0 ** (-snr_db / 20.0)
        f = f + n * (target / torch.linalg.vector_norm(n))
        del n
    return f.to(dtype).contiguous(), omega, coef


def make_device_sparse_signal_direct(N: int, omega, coef, device="cuda", chunk: int = 1 << 27):
    """f[j] = sum_k coef_k (-1)^{omega_k} e^{2 pi i omega_k j / N} (the same signal as
    make_device_signal without noise), summed term by term in FP64 over chunks of j and stored as
    complex64: no length-N FFT, so any N up to 2^31 - 1 fits.  The phase index (omega_k j) mod N
    is exact in int64 (both factors are below 2^31)."""
    import torch
    f = torch.empty(N, dtype=torch.complex64, device=device)
    om = [int(w) % N for w in omega]
    cs = [complex(c) * (1.0 if int(w) % 2 == 0 else -1.0) for w, c in zip(omega, coef)]
    two_pi_n = 2.0 * np.pi / N
    for a in range(0, N, chunk):
        j = torch.arange(a, min(N, a + chunk), dtype=torch.int64, device=device)
        acc = torch.zeros(j.numel(), dtype=torch.complex128, device=device)
        for w, c in zip(om, cs):
            ang = torch.remainder(j * w, N).to(torch.float64) * two_pi_n
            acc += c * torch.polar(torch.ones_like(ang), ang)
        f[a:a + j.numel()] = acc.to(torch.complex64)
        del j, acc
    return f
