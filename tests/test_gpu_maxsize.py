"""The largest length the ABI accepts, N = 2^31 - 1 (a prime): an exactly s-sparse spectrum must be
recovered exactly (frequencies) and to the FP32 path's tolerance (coefficients).  At this size the
oracle cannot run the transform, so the check is the recovery property that holds at any N
(Theorem Mainthm with zero noise), on a signal synthesised term by term from its spectrum."""
import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from synth.device_signals import make_device_sparse_signal_direct
from synth.signals import draw_spectrum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()


def test_largest_length_recovers_an_exactly_sparse_spectrum():
    import torch
    N, s = 2 ** 31 - 1, 8
    omega, coef = draw_spectrum(N, s, 31, "unit")
    f = make_device_sparse_signal_direct(N, omega, coef)
    plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=4.0, seed=7))
    info = plan.info()
    assert info["N"] == N
    w, c, n = sft.execute_torch(plan, f)
    torch.cuda.synchronize()
    n = int(n.item())
    w = w.cpu().numpy()[:n]
    c = c.cpu().numpy()[:n]
    plan.destroy()
    del f
    assert n == s
    assert sorted(w.tolist()) == sorted(int(x) for x in omega)
    truth = dict(zip((int(x) for x in omega), coef))
    rel = max(abs(ci - truth[int(wi)]) / abs(truth[int(wi)]) for wi, ci in zip(w, c))
    assert rel < 1e-5
