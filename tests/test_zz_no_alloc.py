"""The batched DFT that allocates no device memory (sft_dft_noalloc) against the transform's own
measurements.

Callers that cannot call cudaMalloc (their device memory is owned by another allocator or budget)
use sft_dft_noalloc, whose tables live in a fixed array the library declares in device memory.
This test runs the sparse transform through sft_plan / sft_execute, takes the filtered samples of
one shift and prime from the plan, and checks that sft_dft_noalloc reproduces the plan's length-p
measurements of those samples, on two calls in a row with different lengths (the second call
rebuilds the tables), within the FP32 path's tolerance (1e-5 relative to the largest bin).
It is collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_dft_matches_the_plan_measurements():
    import torch

    import paper_1706_02740_gb300 as sft
    from paper_1706_02740_gb300 import build
    from synth.signals import as_complex64, make_signal

    assert torch.cuda.is_available(), "GPU test"
    build.build()
    sft.load()

    N, s = 2 ** 16, 8
    sig = make_signal(N, s, 1001, "unit", 30.0)
    plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=8.0, seed=4))
    info = plan.info()
    f = torch.from_numpy(as_complex64(sig.f)).cuda()
    sft.execute_torch(plan, f)
    torch.cuda.synchronize()
    nq, m, nsub = info["n_shifts"], info["nodes"], info["n_sub"]
    samples = sft.debug_tensor(plan, sft.BUF_SAMPLES, torch.complex64, (nq, m)).clone()
    bins = sft.debug_tensor(plan, sft.BUF_BINS, torch.complex64, (nq, m)).clone()
    torch.cuda.synchronize()
    primes = info["primes"]
    assert primes[0] != primes[1]

    for call, (qi, j) in enumerate([(0, 0), (1, 1)]):
        p = primes[j]
        off = nsub * sum(primes[:j])
        x = samples[qi, off: off + nsub * p].contiguous()       # nsub vectors of length p
        ref = bins[qi, off: off + nsub * p]
        out = torch.empty_like(x)
        sft.sft_dft_noalloc(p, nsub, x.data_ptr(), out.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        err = float((out - ref).abs().max())
        assert err <= 1e-5 * scale, (call, p, err, scale)
        # and against the definition, via numpy's DFT of the same samples
        xn = x.cpu().numpy().astype(np.complex128).reshape(nsub, p)
        exact = np.fft.fft(xn, axis=1) / p
        assert np.max(np.abs(out.cpu().numpy().reshape(nsub, p) - exact)) <= 1e-5 * scale

    with pytest.raises(sft.SftError) as e:
        sft.sft_dft_noalloc(8192, 1, x.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == sft.SFT_EINVAL and "8191" in sft.sft_last_error()
    plan.destroy()


@pytest.mark.parametrize("n", [2, 3, 64, 4096, 4097, 6000, 8191])
def test_noalloc_dft_lengths_against_numpy(n):
    """The ends of the accepted range (n = 2, and n = 8191 with its length-16384 convolution and
    one-CTA filter build), powers of two, a composite length and a prime: three vectors per call
    against numpy's DFT / n, within 1e-5 of the largest bin."""
    import torch

    import paper_1706_02740_gb300 as sft
    from paper_1706_02740_gb300 import build

    build.build()
    sft.load()
    rng = np.random.default_rng(n)
    batch = 3
    xn = (rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))).astype(np.complex64)
    x = torch.from_numpy(xn).cuda()
    out = torch.empty_like(x)
    sft.sft_dft_noalloc(n, batch, x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    exact = np.fft.fft(xn.astype(np.complex128), axis=1) / n
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(out.cpu().numpy() - exact)) <= 1e-5 * scale


def test_noalloc_dft_length_changes_on_one_stream():
    """Lengths alternating on one stream without a synchronisation between calls: each call's
    tables are rebuilt in stream order before its transforms run."""
    import torch

    import paper_1706_02740_gb300 as sft
    from paper_1706_02740_gb300 import build

    build.build()
    sft.load()
    st = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    cases = []
    with torch.cuda.stream(st):
        for n in [1531, 97, 1531, 8191, 97]:
            xn = (rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))).astype(np.complex64)
            x = torch.from_numpy(xn).to("cuda", non_blocking=False)
            out = torch.empty_like(x)
            sft.sft_dft_noalloc(n, 2, x.data_ptr(), out.data_ptr(), st.cuda_stream)
            cases.append((xn, x, out))
    st.synchronize()
    for xn, _, out in cases:
        exact = np.fft.fft(xn.astype(np.complex128), axis=1) / xn.shape[1]
        assert np.max(np.abs(out.cpu().numpy() - exact)) <= 1e-5 * np.max(np.abs(exact))
