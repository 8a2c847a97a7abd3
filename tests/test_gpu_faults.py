"""Fault recording and failure paths on the GPU, with no GPU fault involved.

* Status words: a normal execution records no fault.  A voted list whose capacity the test hook
  sft_plan_debug_limit lowers (the buffer keeps its size, so every access stays inside it) records
  SFT_FAULT_VOTED_FULL; restoring the capacity clears it and restores the result bit for bit.
* The checked build (libsft_checked.so: every gather, bin and candidate index range-checked)
  records nothing on valid plans of every kernel family (both resampling kernels, both DFT forms,
  both identification paths, both precisions, the refinement, batches) and returns the normal
  build's bits.
* Allocation failures injected on the host (sft_debug_fail_allocations) at each allocation of plan,
  batch, stream-ordered batch and server creation: the call returns SFT_ENOMEM, leaves no device
  memory behind (the server's 256 MiB arena is the one a leak would show), and the next call
  succeeds.
"""
import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from synth.signals import as_complex64, make_signal, upcast

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()
    yield
    sft.sft_debug_fail_allocations(0, 0)
    sft.use_checked(False)


def _signal(N, s, seed, c128=False):
    import torch
    f = as_complex64(make_signal(N, s, seed, "unit", 30.0).f)
    if c128:
        f = upcast(f)
    return torch.from_numpy(np.ascontiguousarray(f)).to("cuda")


def _run(N, s, f, variant, primes=None, small=None):
    """(freqs, coefs, count, faults, site) of one execution through the current library."""
    import torch
    plan = sft.sft_plan(N, s, variant, primes=primes, small_moduli=small)
    w, c, n = sft.execute_torch(plan, f)
    torch.cuda.synchronize()
    faults, site = sft.sft_plan_faults(plan)
    out = (w.cpu().numpy(), c.cpu().numpy(), int(n.item()), faults, site)
    plan.destroy()
    return out


def test_normal_execution_records_no_fault():
    f = _signal(2 ** 16, 8, 1)
    *_, faults, site = _run(2 ** 16, 8, f, sft.sft_variant_init(K=5, c_p=4.0, seed=1))
    assert (faults, site) == (0, 0)


def test_lowered_voted_capacity_is_recorded_and_restored():
    import torch
    N, s = 2 ** 16, 8
    f = _signal(N, s, 2)
    plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=4.0, seed=1))
    full = sum(plan.info()["primes"])
    w0, c0, n0 = [t.cpu().numpy() for t in sft.execute_torch(plan, f)]
    assert sft.sft_plan_faults(plan) == (0, 0)
    sft.sft_plan_debug_limit(plan, 0, 2)            # two records per shift
    w1, c1, n1 = [t.cpu().numpy() for t in sft.execute_torch(plan, f)]
    faults, site = sft.sft_plan_faults(plan)
    assert faults & sft.SFT_FAULT_VOTED_FULL and site == 0
    assert int(n1[0]) <= 2 * plan.info()["n_shifts"]
    sft.sft_plan_debug_limit(plan, 0, full)
    w2, c2, n2 = [t.cpu().numpy() for t in sft.execute_torch(plan, f)]
    torch.cuda.synchronize()
    assert sft.sft_plan_faults(plan) == (0, 0)
    assert n2[0] == n0[0] and np.array_equal(w2, w0) and np.array_equal(c2, c0)
    with pytest.raises(sft.SftError):
        sft.sft_plan_debug_limit(plan, 0, full + 1)
    plan.destroy()


CHECKED_CASES = [
    # id, N, s, variant fields, explicit primes, input complex128
    ("fp32", 2 ** 14, 6, dict(K=5, c_p=8.0, seed=11), None, False),
    ("fp64", 2 ** 14, 6, dict(K=5, c_p=8.0, seed=11, precision=1, input=1), None, True),
    ("kappa4-odd-N", 3 ** 9, 8, dict(K=5, c_p=8.0, seed=12, kappa=4), None, False),
    ("rader", 2 ** 14, 6, dict(K=5, c_p=8.0, seed=11, pool=1, dft=2), None, False),
    ("small-moduli-not-a-prefix", 2 ** 12, 3, dict(K=3, seed=3, dft=1), [11, 13, 17], False),
    ("prime-N", 100003, 12, dict(K=7, c_p=5.0, seed=14), None, False),
]


@pytest.mark.parametrize("case", CHECKED_CASES, ids=[c[0] for c in CHECKED_CASES])
def test_checked_build_records_nothing_and_returns_the_same_bits(case):
    _, N, s, fields, primes, c128 = case
    f = _signal(N, s, 7, c128)
    ref = _run(N, s, f, sft.sft_variant_init(**fields), primes)
    try:
        sft.use_checked(True)
        assert sft.checked_build()
        got = _run(N, s, f, sft.sft_variant_init(**fields), primes)
    finally:
        sft.use_checked(False)
    assert got[3:] == (0, 0), got[3:]
    assert got[2] == ref[2]
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_checked_build_wide_window_and_batch():
    """The wide-window resampling kernel (theorem-parameter mode) and a mixed batch."""
    import torch
    N, s = 2 ** 14, 8
    f = _signal(N, s, 8)
    shapes = [(2 ** 14, 6), (3 ** 9, 8), (100003, 12)]
    fs = [_signal(n_, s_, 20 + i) for i, (n_, s_) in enumerate(shapes)]

    def both():
        v = sft.sft_variant_theorem(N, 1.0, K=5, c_p=8.0, seed=1)
        one = _run(N, s, f, v)
        plans = [sft.sft_plan(n_, s_, sft.sft_variant_init(K=5, c_p=6.0, seed=2)) for n_, s_ in shapes]
        batch = sft.Batch(plans)
        outs = sft.execute_batch_torch(batch, fs)
        torch.cuda.synchronize()
        res = [tuple(t.cpu().numpy() for t in o) for o in outs]
        faults = [sft.sft_plan_faults(p) for p in plans]
        batch.destroy()
        for p in plans:
            p.destroy()
        return one, res, faults

    ref = both()
    try:
        sft.use_checked(True)
        got = both()
    finally:
        sft.use_checked(False)
    assert got[0][3:] == (0, 0) and all(x == (0, 0) for x in got[2])
    assert np.array_equal(got[0][0], ref[0][0]) and np.array_equal(got[0][1], ref[0][1])
    for a, b in zip(got[1], ref[1]):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _same_free(a, b):
    """Device memory free before and after, to the driver's 2 MiB granule (small blocks are
    sub-allocated; a leaked plan or arena is far larger)."""
    return abs(a - b) <= 2 << 20


def test_plan_creation_fails_cleanly():
    v = sft.sft_variant_init(K=5, c_p=3.0, seed=1)
    sft.sft_plan(2 ** 22, 64, v).destroy()             # warm: modules loaded, pools settled
    before = _free_bytes()
    sft.sft_debug_fail_allocations(0, 1)
    with pytest.raises(sft.SftError) as e:
        sft.sft_plan(2 ** 22, 64, v)
    assert e.value.status == sft.SFT_ENOMEM
    assert _same_free(_free_bytes(), before)
    sft.sft_plan(2 ** 22, 64, v).destroy()             # the hook has run out


def test_batch_creation_fails_cleanly_at_each_allocation():
    plans = [sft.sft_plan(2 ** 14, 6, sft.sft_variant_init(seed=i)) for i in range(3)]
    sft.Batch(plans).destroy()
    before = _free_bytes()
    for skip in (0, 1):                                 # the device array, then the pinned ring
        sft.sft_debug_fail_allocations(skip, 1)
        with pytest.raises(sft.SftError) as e:
            sft.Batch(plans)
        assert e.value.status == sft.SFT_ENOMEM, skip
        sft.sft_debug_fail_allocations(0, 0)
        assert _same_free(_free_bytes(), before), skip
    sft.Batch(plans).destroy()
    for p in plans:
        p.destroy()


def test_stream_ordered_batch_fails_cleanly():
    import torch
    shapes = [(2 ** 14, 6), (3 ** 9, 8)]
    plans = [sft.sft_plan(n_, s_, sft.sft_variant_init(seed=3)) for n_, s_ in shapes]
    fs = [_signal(n_, s_, 30 + i) for i, (n_, s_) in enumerate(shapes)]
    outs = [(torch.empty(s_, dtype=torch.int64, device="cuda"),
             torch.empty(s_, dtype=torch.complex128, device="cuda"),
             torch.zeros(1, dtype=torch.int32, device="cuda")) for _, s_ in shapes]
    ptrs = ([f.data_ptr() for f in fs], [o[0].data_ptr() for o in outs],
            [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs])
    sft.sft_debug_fail_allocations(0, 1)
    with pytest.raises(sft.SftError) as e:
        sft.sft_execute_batch(plans, *ptrs)
    assert e.value.status == sft.SFT_ENOMEM
    sft.sft_execute_batch(plans, *ptrs)
    torch.cuda.synchronize()
    assert all(int(o[2].item()) > 0 for o in outs)
    for p in plans:
        p.destroy()


def test_server_creation_fails_cleanly_at_each_allocation():
    """Allocations of sft_server_create in order: the arena, then each slot's device block and
    pinned block (two slots here)."""
    sft.Server(mem_budget=256 << 20, max_batch=8, max_inflight=2, build_threads=0).destroy()
    before = _free_bytes()
    for skip in range(5):
        sft.sft_debug_fail_allocations(skip, 1)
        with pytest.raises(sft.SftError) as e:
            sft.Server(mem_budget=256 << 20, max_batch=8, max_inflight=2, build_threads=0)
        assert e.value.status == sft.SFT_ENOMEM, skip
        sft.sft_debug_fail_allocations(0, 0)
        assert _same_free(_free_bytes(), before), skip
    sft.Server(mem_budget=256 << 20, max_batch=8, max_inflight=2, build_threads=0).destroy()
