"""Noise robustness (Section 5.4): unit-magnitude, random-phase s-sparse spectra plus complex
Gaussian noise at a given SNR, the average L1 error of the coefficients over the trials whose
support is exact.

With parameters whose collision floor is low (K = 9 primes, c_p = 8), the error follows the
noise: it falls by at least 5x for every 20 dB while the noise dominates, every trial at 20 dB
and above recovers the support exactly, and at every SNR the GPU result equals the oracle's on
the same input (support, and coefficients within the FP32 path's 1e-5)."""
import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from oracle import dsft as O
from synth.signals import as_complex64, make_signal, upcast
from tests import gpu_parity_util as U

pytestmark = pytest.mark.gpu

N, S, K, CP = 2 ** 18, 16, 9, 8.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()


def _l1(snr, trials):
    errs, exact = [], 0
    for t in range(trials):
        sig = make_signal(N, S, 5400 + 31 * t + int(snr), "unit", snr)
        g = U.run_gpu(sft, N, S, as_complex64(sig.f), U.FP32, 6, K, CP, 3)
        n = g["count"]
        got = dict(zip(g["freqs"][:n].tolist(), g["coefs"][:n]))
        truth = dict(zip(sig.omega.tolist(), sig.coef))
        if set(got) == set(truth):
            exact += 1
            errs.append(sum(abs(got[w] - truth[w]) for w in truth) / S)
    return (float(np.mean(errs)) if errs else None), exact


def test_error_follows_the_noise():
    snrs = [20.0, 40.0, 60.0]
    res = {snr: _l1(snr, 5) for snr in snrs}
    for snr, (l1, exact) in res.items():
        print(f"SNR {snr:.0f} dB: average L1 error {l1:.3e} over {exact}/5 exact trials")
        assert exact == 5
    assert res[20.0][0] > 5 * res[40.0][0] > 25 * res[60.0][0]


@pytest.mark.parametrize("snr", [10.0, 30.0, 50.0])
def test_noisy_inputs_match_the_oracle(snr):
    sig = make_signal(N, S, 5500 + int(snr), "unit", snr)
    f32 = as_complex64(sig.f)
    g = U.run_gpu(sft, N, S, f32, U.FP32, 6, K, CP, 3, keep=True)
    cand = U.debug_arrays(sft, g["plan"], g["info"])[2]
    g["plan"].destroy()
    res = O.dsft(upcast(f32), U.oracle_plan(g["info"], N, S))
    U.explain_output_differences(g, res, cand, g["info"], 1e-5, log=print)
    n = g["count"]
    gmap = dict(zip(g["freqs"][:n].tolist(), g["coefs"][:n]))
    omap = dict(zip(res.freqs.tolist(), res.coefs))
    common = sorted(set(gmap) & set(omap))
    assert len(common) >= S - 1
    assert max(abs(gmap[w] - omap[w]) / abs(omap[w]) for w in common) <= 1e-5
