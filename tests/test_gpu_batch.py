"""Batched execution: one launch per stage for many signals, each with its own plan.

Each signal's result from a batch must equal, bit for bit, the result of executing its plan alone
(the kernels do the same arithmetic per signal; selections do not depend on the order in which
atomics filled the lists), and agree with the oracle on a sample of the batch."""
import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from oracle import dsft as O
from synth.signals import as_complex64, make_signal, upcast
from tests import gpu_parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()


SHAPES = [(2 ** 14, 6), (65521, 12), (3 ** 10, 20), (2 ** 17, 40), (100003, 9), (2 ** 15 + 3, 30),
          (2 ** 16, 8)]


def _signals(shapes, seed0, snr=30.0):
    return [make_signal(N, s, seed0 + i, "unit" if i % 2 else "loguniform", snr)
            for i, (N, s) in enumerate(shapes)]


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_heterogeneous_batch_equals_single_executions(prec):
    import torch
    sigs = _signals(SHAPES, 500)
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(precision=prec, K=5, c_p=6.0, seed=i))
             for i, (N, s) in enumerate(SHAPES)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    singles = []
    for p, f in zip(plans, fs):
        w, c, n = sft.execute_torch(p, f)
        torch.cuda.synchronize()
        singles.append((w.cpu().numpy(), c.cpu().numpy(), int(n.item())))
    batch = sft.Batch(plans)
    for rep in range(3):                     # repeated executions through the staging ring
        outs = sft.execute_batch_torch(batch, fs)
        torch.cuda.synchronize()
        for (w, c, n), (sw, sc, sn) in zip(outs, singles):
            assert int(n.item()) == sn
            assert np.array_equal(w.cpu().numpy(), sw)
            assert np.array_equal(c.cpu().numpy(), sc)
    # and the oracle on two members
    for i in (1, 4):
        N, s = SHAPES[i]
        info = plans[i].info()
        res = O.dsft(upcast(as_complex64(sigs[i].f)), U.oracle_plan(info, N, s))
        w, c, n = singles[i]
        assert n == len(res.freqs)
        U.assert_same_output(w[:n], c[:n], res.freqs, res.coefs, 1e-5 if prec == U.FP32 else 1e-11)
    batch.destroy()
    for p in plans:
        p.destroy()


def test_one_shot_batch_equals_the_batch_object():
    """sft_execute_batch (stream-ordered: its device array is allocated and released on the
    stream) against a resident batch of the same plans: identical bits, also for a second call
    enqueued behind the first with the inputs reversed and no synchronisation between them."""
    import torch
    shapes = SHAPES[:4]
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=6.0, seed=i))
             for i, (N, s) in enumerate(shapes)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in _signals(shapes, 950)]
    batch = sft.Batch(plans)
    ref = sft.execute_batch_torch(batch, fs)
    torch.cuda.synchronize()
    batch.destroy()
    outs = [(torch.empty(s, dtype=torch.int64, device="cuda"),
             torch.empty(s, dtype=torch.complex128, device="cuda"),
             torch.empty(1, dtype=torch.int32, device="cuda")) for _, s in shapes]
    sft.sft_execute_batch(plans, [f.data_ptr() for f in fs], [o[0].data_ptr() for o in outs],
                          [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs],
                          torch.cuda.current_stream().cuda_stream)
    for (w, c, n), (rw, rc, rn) in zip(outs, ref):
        assert int(n.item()) == int(rn.item())
        assert torch.equal(w, rw) and torch.equal(c, rc)
    # two calls back to back on one stream, the second over the same plans and inputs in reverse
    # order (each plan keeps its own input and output sizes): both results stay intact
    st = torch.cuda.current_stream().cuda_stream
    rshapes, rplans, rfs = shapes[::-1], plans[::-1], fs[::-1]
    outs2 = [(torch.empty(s, dtype=torch.int64, device="cuda"),
              torch.empty(s, dtype=torch.complex128, device="cuda"),
              torch.empty(1, dtype=torch.int32, device="cuda")) for _, s in rshapes]
    batch_r = sft.Batch(rplans)
    ref_r = sft.execute_batch_torch(batch_r, rfs)
    torch.cuda.synchronize()
    batch_r.destroy()
    sft.sft_execute_batch(plans, [f.data_ptr() for f in fs], [o[0].data_ptr() for o in outs],
                          [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs], st)
    sft.sft_execute_batch(rplans, [f.data_ptr() for f in rfs], [o[0].data_ptr() for o in outs2],
                          [o[1].data_ptr() for o in outs2], [o[2].data_ptr() for o in outs2], st)
    torch.cuda.synchronize()
    for (w, c, n), (rw, rc, rn) in zip(outs, ref):
        assert int(n.item()) == int(rn.item()) and torch.equal(w, rw) and torch.equal(c, rc)
    for (w, c, n), (rw, rc, rn) in zip(outs2, ref_r):
        assert int(n.item()) == int(rn.item()) and torch.equal(w, rw) and torch.equal(c, rc)
    for p in plans:
        p.destroy()


def test_batch_of_identical_shapes_with_rotating_inputs():
    import torch
    N, s, B = 2 ** 18, 50, 6
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=4.0, seed=3)) for _ in range(B)]
    sigs = [make_signal(N, s, 900 + i, "unit", 30.0) for i in range(2 * B)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    batch = sft.Batch(plans)
    for half in (0, 1):
        outs = sft.execute_batch_torch(batch, fs[half * B:(half + 1) * B])
        torch.cuda.synchronize()
        for i, (w, c, n) in enumerate(outs):
            g = sigs[half * B + i]
            got = set(w.cpu().numpy()[: int(n.item())].tolist())
            assert len(got & set(g.omega.tolist())) >= s - 1
    batch.destroy()


def test_batch_rejects_mixed_variants_and_duplicates():
    a = sft.sft_plan(2 ** 14, 4, sft.sft_variant_init(precision=0, c_p=8.0))
    b = sft.sft_plan(2 ** 14, 4, sft.sft_variant_init(precision=1, c_p=8.0))
    c = sft.sft_plan(2 ** 14, 4, sft.sft_variant_init(kappa=4, c_p=8.0))
    for plans in ([a, b], [a, c], [a, a]):
        with pytest.raises(sft.SftError) as e:
            sft.Batch(plans)
        assert e.value.status == sft.SFT_EINVAL
    for p in (a, b, c):
        p.destroy()


def _tuning_variants(prec):
    base = sft.sft_tuning_default()
    out = []
    for rt, cap in ((128, 1), (512, 0), (64, 0), (256, 1)):
        t = dict(base, resample_threads=rt, resample_regcap=cap)
        out.append(t)
    out.append(dict(base, bin_threads=64))
    out.append(dict(base, bin_threads=512))
    out.append(dict(base, dft_per_cta=[1] * 9))
    out.append(dict(base, dft_per_cta=[max(1, g // 2) for g in base["dft_per_cta"]]))
    if prec == U.FP32:
        out.append(dict(base, dft_two_ctas=0))
    return out


def _mixed_plans(prec):
    # the last two members have p near 3000 and 3600: chirp lengths 6144 and (FP32) 8192, next to
    # the small lengths 96 .. 512 of the others, of both kinds (2^k and 3 2^k)
    shapes = SHAPES + [(2 ** 18, 1000), (2 ** 18, 1200)]
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(precision=prec, K=5,
                                                     c_p=3.0 if s >= 1000 else 6.0, seed=i))
             for i, (N, s) in enumerate(shapes)]
    sigs = _signals(shapes, 700)
    return shapes, plans, sigs


def _host(outs):
    return [(w.cpu().numpy(), c.cpu().numpy(), int(n.item())) for w, c, n in outs]


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_every_tuning_and_the_graph_give_identical_results(prec):
    import torch
    shapes, plans, sigs = _mixed_plans(prec)
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    batch = sft.Batch(plans)
    ref = _host(sft.execute_batch_torch(batch, fs))
    torch.cuda.synchronize()
    for t in _tuning_variants(prec):
        batch.set_tuning(t)
        assert batch.get_tuning() == t
        got = _host(sft.execute_batch_torch(batch, fs))
        for (w, c, n), (rw, rc, rn) in zip(got, ref):
            assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc), t
    # graph replay: captured at the first execution, replayed after
    batch.set_tuning(sft.sft_tuning_default())
    batch.graph(True)
    l0 = batch.launches
    g1 = _host(sft.execute_batch_torch(batch, fs))
    per_exec = batch.launches - l0
    assert per_exec > 0
    for (w, c, n), (rw, rc, rn) in zip(g1, ref):
        assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc)
    for rep in range(3):
        g = _host(sft.execute_batch_torch(batch, fs))
        assert batch.launches - l0 == per_exec * (rep + 2)
        for (w, c, n), (rw, rc, rn) in zip(g, ref):
            assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc)
    batch.graph(False)
    batch.destroy()
    for p in plans:
        p.destroy()


def test_graph_replay_reads_each_executions_inputs():
    import torch
    N, s, B = 2 ** 16, 20, 4
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=5.0, seed=11)) for _ in range(B)]
    sigs = [make_signal(N, s, 1200 + i, "unit", 30.0) for i in range(2 * B)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    batch = sft.Batch(plans)
    direct = [_host(sft.execute_batch_torch(batch, fs[h * B:(h + 1) * B])) for h in (0, 1)]
    batch.graph(True)
    for rep in range(2):
        for h in (0, 1):
            got = _host(sft.execute_batch_torch(batch, fs[h * B:(h + 1) * B]))
            for (w, c, n), (rw, rc, rn) in zip(got, direct[h]):
                assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc)
    batch.destroy()
    for p in plans:
        p.destroy()


def test_autotune_picks_a_valid_tuning_and_keeps_results():
    import torch
    shapes, plans, sigs = _mixed_plans(U.FP32)
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    batch = sft.Batch(plans)
    batch.profile(True)
    ref = _host(sft.execute_batch_torch(batch, fs))
    chosen = sft.autotune_batch_torch(batch, fs, reps=2)
    assert batch.get_tuning() == chosen
    got = _host(sft.execute_batch_torch(batch, fs))
    torch.cuda.synchronize()
    for (w, c, n), (rw, rc, rn) in zip(got, ref):
        assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc)
    # profiling stayed on: the execution after tuning was recorded
    _, n_exec = batch.profile_read()
    assert n_exec == 1
    batch.destroy()
    for p in plans:
        p.destroy()


def test_autotuned_geometry_is_kept_for_batches_of_the_same_class(tmp_path):
    """sft_batch_autotune stores its choice under the batch's shape class (floor(log2 N),
    floor(log2 s), kappa, precision); a new batch of that class starts from it, also after the
    table went through its file; a batch of mixed classes starts from the default."""
    import torch
    sft.tuning_table_clear()
    shapes = [(2 ** 16, 8), (2 ** 16 + 7, 9), (2 ** 17 - 1, 15), (2 ** 16, 12)]
    plans = [sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=5.0, seed=3)) for N, s in shapes]
    sigs = [make_signal(N, s, 1300 + i, "unit", 30.0) for i, (N, s) in enumerate(shapes)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    batch = sft.Batch(plans)
    assert batch.get_tuning() == sft.sft_tuning_default()
    chosen = sft.autotune_batch_torch(batch, fs, reps=2)
    assert sft.tuning_table_get(2 ** 16, 8, 6, 0) == chosen
    batch.destroy()
    again = sft.Batch(plans[::-1])
    assert again.get_tuning() == chosen
    again.destroy()
    path = str(tmp_path / "tuning.txt")
    sft.tuning_table_save(path)
    sft.tuning_table_clear()
    assert sft.Batch(plans).get_tuning() == sft.sft_tuning_default()
    sft.tuning_table_load(path)
    loaded = sft.Batch(plans)
    assert loaded.get_tuning() == chosen
    ref = _host(sft.execute_batch_torch(loaded, fs))
    loaded.destroy()
    other = sft.sft_plan(2 ** 18, 8, sft.sft_variant_init(K=5, c_p=5.0, seed=3))
    mixed = sft.Batch(plans + [other])
    assert mixed.get_tuning() == sft.sft_tuning_default()
    got = _host(sft.execute_batch_torch(mixed, fs + [fs[0][:0].new_zeros(2 ** 18)]))
    for (w, c, n), (rw, rc, rn) in zip(got[:4], ref):       # geometry never changes results
        assert n == rn and np.array_equal(w, rw) and np.array_equal(c, rc)
    mixed.destroy()
    other.destroy()
    for p in plans:
        p.destroy()
    sft.tuning_table_clear()


def test_invalid_tunings_are_rejected_and_change_nothing():
    shapes, plans, sigs = _mixed_plans(U.FP32)
    batch = sft.Batch(plans)
    base = batch.get_tuning()
    bad = [dict(base, resample_threads=100), dict(base, resample_threads=1024),
           dict(base, resample_regcap=1, resample_threads=512), dict(base, bin_threads=2048),
           dict(base, dft_per_cta=[128] + base["dft_per_cta"][1:]),
           dict(base, dft_per_cta=base["dft_per_cta"][:7] + [2, 1]), dict(base, dft_two_ctas=2)]
    for t in bad:
        with pytest.raises(sft.SftError) as e:
            batch.set_tuning(t)
        assert e.value.status == 1
        assert batch.get_tuning() == base
    batch.destroy()
    for p in plans:
        p.destroy()


def test_plan_graph_replay_equals_direct_execution():
    import torch
    N, s = 65521, 12
    sigs = [make_signal(N, s, 1300 + i, "unit", 30.0) for i in range(3)]
    fs = [torch.from_numpy(as_complex64(g.f)).cuda() for g in sigs]
    plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=5.0, seed=8))
    direct = []
    for f in fs:
        w, c, n = sft.execute_torch(plan, f)
        torch.cuda.synchronize()
        direct.append((w.cpu().numpy(), c.cpu().numpy(), int(n.item())))
    sft.sft_plan_graph(plan, True)
    l0 = sft.sft_plan_launches(plan)
    for rep in range(2):
        for f, (rw, rc, rn) in zip(fs, direct):
            w, c, n = sft.execute_torch(plan, f)          # fresh output buffers every call
            torch.cuda.synchronize()
            assert int(n.item()) == rn
            assert np.array_equal(w.cpu().numpy(), rw) and np.array_equal(c.cpu().numpy(), rc)
    per = (sft.sft_plan_launches(plan) - l0) / 6
    assert per >= 10 and per == int(per)
    sft.sft_plan_graph(plan, False)
    w, c, n = sft.execute_torch(plan, fs[0])
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), direct[0][1])
    plan.destroy()


def test_mixed_batch_sample_matches_oracle():
    """The mixed-size batched workload (N log-uniform over [2^18, 2^24], a quarter at other
    lengths including primes; s uniform over [16, 512]; unit magnitudes; SNR 20 dB; complex64):
    a seeded 64-signal sample run as one batch on the FP32 path, every member against the oracle on
    the same input.  As at the other full sizes, a frequency only one side returns must be
    explained by a residue decision without margin or by the s-th magnitude cut."""
    import torch
    from synth.device_signals import make_device_signal
    from synth.signals import draw_batch_shapes
    from tests.test_gpu_fullsize import _compare
    shapes = draw_batch_shapes(64, 4064)
    plans, fs = [], []
    for i, (N, s) in enumerate(shapes):
        f, _, _ = make_device_signal(N, s, 4064 + i, "unit", 20.0, "cuda")
        fs.append(f)
        plans.append(sft.sft_plan(N, s, sft.sft_variant_init(kappa=6, K=5, c_p=3.0, seed=i)))
    torch.backends.cuda.cufft_plan_cache[0].clear()
    batch = sft.Batch(plans)
    outs = sft.execute_batch_torch(batch, fs)
    torch.cuda.synchronize()
    worst = 0.0
    for p, f, (w, c, n), (N, s) in zip(plans, fs, outs, shapes):
        info = p.info()
        g = {"freqs": w.cpu().numpy(), "coefs": c.cpu().numpy(), "count": int(n.item()),
             "info": info}
        cand = U.debug_arrays(sft, p, info)[2]
        res = O.dsft(f.cpu().numpy().astype(np.complex128), U.oracle_plan(info, N, s))
        _, _, err = _compare(g, res, cand, 1e-5)
        worst = max(worst, err)
    assert worst <= 1e-5
    batch.destroy()
    for p in plans:
        p.destroy()
