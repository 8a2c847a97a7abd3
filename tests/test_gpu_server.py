"""Serving loop: requests of mixed N and s, admitted by device-memory budget, batched as they arrive
and run on several streams.  Every result must equal, bit for bit, what the same plan gives for
the request alone (sft_execute), whatever else it was batched or overlapped with."""
import time

import numpy as np
import pytest

import paper_1706_02740_gb300 as sft
from synth.signals import as_complex64, make_signal

pytestmark = pytest.mark.gpu

VARIANT = dict(K=5, c_p=6.0, seed=5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()


def _inputs(shapes, seed0):
    import torch
    return [torch.from_numpy(as_complex64(make_signal(N, s, seed0 + i, "unit", 30.0).f)).cuda()
            for i, (N, s) in enumerate(shapes)]


def _outputs(shapes):
    import torch
    return [(torch.full((s,), -7, dtype=torch.int64, device="cuda"),
             torch.zeros(s, dtype=torch.complex128, device="cuda"),
             torch.full((1,), -1, dtype=torch.int32, device="cuda")) for N, s in shapes]


def _alone(shapes, fs):
    import torch
    res = []
    for (N, s), f in zip(shapes, fs):
        p = sft.sft_plan(N, s, sft.sft_variant_init(**VARIANT))
        w, c, n = sft.execute_torch(p, f)
        torch.cuda.synchronize()
        res.append((w.cpu().numpy(), c.cpu().numpy(), int(n.item())))
        p.destroy()
    return res


def _submit(srv, shapes, fs, outs):
    return [srv.submit(N, s, f.data_ptr(), o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
            for (N, s), f, o in zip(shapes, fs, outs)]


def _check_equal(outs, ref, idx=None):
    for i, ((w, c, n), (rw, rc, rn)) in enumerate(zip(outs, ref)):
        if idx is not None and i not in idx:
            continue
        assert int(n.item()) == rn, i
        assert np.array_equal(w.cpu().numpy(), rw), i
        assert np.array_equal(c.cpu().numpy(), rc), i


SHAPES = [(2 ** 14, 6), (65521, 12), (2 ** 16, 8), (2 ** 14, 6), (3 ** 10, 20), (2 ** 17, 40),
          (65521, 12), (100003, 9), (2 ** 15 + 3, 30), (2 ** 14, 6), (2 ** 18, 64), (2 ** 16, 8)]


def test_each_result_is_the_same_alone_and_in_the_mix():
    fs = _inputs(SHAPES, 2000)
    ref = _alone(SHAPES, fs)
    srv = sft.Server(mem_budget=2 << 30, max_batch=3, max_inflight=2,
                     variant=sft.sft_variant_init(**VARIANT))
    outs = _outputs(SHAPES)
    ids = _submit(srv, SHAPES, fs, outs)
    for rid in ids:
        assert srv.wait(rid, 60000) == sft.SFT_OK
    _check_equal(outs, ref)
    infos = [srv.query(r) for r in ids]
    assert all(q["state"] == "done" and q["latency_ms"] >= q["queued_ms"] >= 0 for q in infos)
    assert all(q["build_ms"] > 0 for q in infos if not q["plan_reused"])
    st = srv.stats()
    assert st["completed"] == len(SHAPES) and st["failed"] == 0
    assert st["plans_built"] + st["plans_reused"] == len(SHAPES)
    assert st["max_batch_seen"] <= 3 and st["batches"] >= len(SHAPES) // 3
    assert st["kernel_launches"] > 0
    # a second pass over the same shapes reuses the resident plans
    outs2 = _outputs(SHAPES)
    ids2 = _submit(srv, SHAPES, fs, outs2)
    for rid in ids2:
        assert srv.wait(rid, 60000) == sft.SFT_OK
    _check_equal(outs2, ref)
    assert srv.stats()["plans_reused"] > st["plans_reused"]
    infos2 = [srv.query(r) for r in ids2]
    assert max(q["batch_size"] for q in infos2) >= 2         # resident plans: requests batched
    for rid in ids + ids2:
        srv.release(rid)
    with pytest.raises(sft.SftError):
        srv.query(ids[0])
    srv.destroy()


def test_requests_arriving_while_others_run_join_later_batches():
    fs = _inputs(SHAPES, 2100)
    ref = _alone(SHAPES, fs)
    srv = sft.Server(mem_budget=2 << 30, max_batch=4, max_inflight=3,
                     variant=sft.sft_variant_init(**VARIANT))
    outs = _outputs(SHAPES)
    ids = []
    for i in range(len(SHAPES)):              # a trickle: some arrive while earlier ones run
        ids += _submit(srv, SHAPES[i:i + 1], fs[i:i + 1], outs[i:i + 1])
        time.sleep(0.0005 * (i % 3))
    for rid in ids:
        assert srv.wait(rid, 60000) == sft.SFT_OK
    _check_equal(outs, ref)
    srv.destroy()


def test_small_budget_evicts_idle_plans_and_makes_requests_wait():
    shapes = [(2 ** 16, 30), (2 ** 17, 40), (3 ** 10, 20)] * 3
    sizes = []
    for N, s in set(shapes):
        p = sft.sft_plan(N, s, sft.sft_variant_init(**VARIANT))
        sizes.append(p.device_bytes)
        p.destroy()
    budget = max(1 << 20, int(1.6 * max(sizes)))     # room for one plan (or two small ones)
    fs = _inputs(shapes, 2200)
    ref = _alone(shapes, fs)
    srv = sft.Server(mem_budget=budget, max_batch=4, max_inflight=2,
                     variant=sft.sft_variant_init(**VARIANT))
    outs = _outputs(shapes)
    ids = _submit(srv, shapes, fs, outs)
    for rid in ids:
        assert srv.wait(rid, 120000) == sft.SFT_OK
    _check_equal(outs, ref)
    st = srv.stats()
    assert st["completed"] == len(shapes) and st["failed"] == 0
    assert st["plans_evicted"] > 0
    assert st["arena_peak"] <= st["arena_bytes"] <= budget
    srv.destroy()


def test_request_larger_than_the_arena_fails_and_the_server_goes_on():
    srv = sft.Server(mem_budget=1 << 20, max_batch=2, max_inflight=1,
                     variant=sft.sft_variant_init(**VARIANT))
    big, small = (2 ** 20, 200), (2 ** 12, 4)
    fs = _inputs([big, small], 2300)
    outs = _outputs([big, small])
    r_big, r_small = _submit(srv, [big, small], fs, outs)
    assert srv.wait(r_big, 60000) == sft.SFT_ENOMEM
    assert srv.query(r_big)["state"] == "failed"
    assert srv.wait(r_small, 60000) == sft.SFT_OK
    _check_equal(outs[1:], _alone([small], fs[1:]))
    assert int(outs[0][2].item()) == -1                     # untouched
    srv.destroy()


def test_invalid_requests_fail_without_stopping_the_server():
    import torch
    srv = sft.Server(mem_budget=256 << 20, max_batch=4, max_inflight=1,
                     variant=sft.sft_variant_init(**VARIANT))
    f = torch.zeros(16, dtype=torch.complex64, device="cuda")
    o = _outputs([(16, 4)])[0]
    bad = [srv.submit(1, 1, f.data_ptr(), o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr()),
           srv.submit(16, 0, f.data_ptr(), o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())]
    for rid in bad:
        assert srv.wait(rid, 60000) == sft.SFT_EINVAL
    with pytest.raises(sft.SftError):
        srv.submit(16, 4, 0, o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
    shapes = [(2 ** 14, 6)]
    fs = _inputs(shapes, 2400)
    outs = _outputs(shapes)
    rid = _submit(srv, shapes, fs, outs)[0]
    assert srv.wait(rid, 60000) == sft.SFT_OK
    _check_equal(outs, _alone(shapes, fs))
    assert srv.stats()["failed"] == 2
    srv.destroy()


def test_bursts_on_concurrent_streams_keep_every_result_exact():
    """Many requests at once: batches on three streams overlap, and each stream's launch records
    are rewritten before every batch while the other streams' kernels run."""
    import torch
    shapes = [(2 ** 14, 6), (65521, 12), (2 ** 16, 8), (3 ** 10, 20), (2 ** 17, 40),
              (100003, 9), (2 ** 15 + 3, 30), (2 ** 18, 64), (3 ** 9, 16), (2 ** 13, 4),
              (40009, 25), (2 ** 16 + 1, 33)]
    fs = _inputs(shapes, 2500)
    ref = _alone(shapes, fs)
    srv = sft.Server(mem_budget=2 << 30, max_batch=8, max_inflight=3,
                     variant=sft.sft_variant_init(**VARIANT))
    order = [i % len(shapes) for i in range(240)]
    for burst in range(2):
        outs = _outputs([shapes[i] for i in order])
        ids = _submit(srv, [shapes[i] for i in order], [fs[i] for i in order], outs)
        for rid in ids:
            assert srv.wait(rid, 60000) == sft.SFT_OK
        for (w, c, n), i in zip(outs, order):
            rw, rc, rn = ref[i]
            assert int(n.item()) == rn
            assert np.array_equal(w.cpu().numpy(), rw) and np.array_equal(c.cpu().numpy(), rc)
        assert max(srv.query(r)["batch_size"] for r in ids) >= 4
        for rid in ids:
            srv.release(rid)
    srv.destroy()


def test_poll_reports_pending_then_finished_without_blocking():
    srv = sft.Server(mem_budget=256 << 20, max_batch=4, max_inflight=1,
                     variant=sft.sft_variant_init(**VARIANT))
    shapes = [(2 ** 16, 8)]
    fs = _inputs(shapes, 2700)
    outs = _outputs(shapes)
    rid = _submit(srv, shapes, fs, outs)[0]
    done, st = srv.poll(rid)
    assert st == sft.SFT_OK                       # pending or already done, never an error here
    assert srv.wait(rid, 60000) == sft.SFT_OK
    assert srv.poll(rid) == (True, sft.SFT_OK)
    import torch
    f = torch.zeros(16, dtype=torch.complex64, device="cuda")
    o = _outputs([(16, 4)])[0]
    bad = srv.submit(16, 0, f.data_ptr(), o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr())
    srv.wait(bad, 60000)
    assert srv.poll(bad) == (True, sft.SFT_EINVAL)     # a failed request: finished, with its reason
    srv.release(rid)
    with pytest.raises(sft.SftError):
        srv.poll(rid)                                   # unknown once released
    srv.destroy()


def test_batches_that_finish_before_the_scheduler_looks_again_are_not_lost():
    """Tiny requests one at a time: each batch can complete (its callback firing) before the
    scheduler retakes its lock after launching; every completion must still be seen."""
    shapes = [(2 ** 10, 2), (3 ** 6, 2), (1021, 3)]
    fs = _inputs(shapes, 2600)
    ref = _alone(shapes, fs)
    srv = sft.Server(mem_budget=256 << 20, max_batch=4, max_inflight=3,
                     variant=sft.sft_variant_init(**VARIANT))
    for rep in range(300):
        i = rep % len(shapes)
        outs = _outputs(shapes[i:i + 1])
        rid = _submit(srv, shapes[i:i + 1], fs[i:i + 1], outs)[0]
        assert srv.wait(rid, 20000) == sft.SFT_OK
        if rep % 50 == 0:
            _check_equal(outs, ref[i:i + 1])
        srv.release(rid)
    assert srv.stats()["completed"] == 300
    srv.destroy()


@pytest.mark.parametrize("build_threads", [0, 2])
def test_a_new_length_does_not_hold_up_resident_requests(build_threads):
    """A request whose (N, s) needs a new plan, followed by requests whose plans are resident:
    with build threads the first resident one is launched while the new plan is still being built
    (it is queued for less time than that build took); without them (build_threads = 0) the
    scheduler builds inline, behind which the others wait.  Every result equals the same plan run
    alone."""
    shapes = [(2 ** 14, 6)] * 6
    # a new length and sparsity, with a seed no other test uses: its primes' tables are not in the
    # host cache yet, so its plan build does real work (the reference for it is computed after)
    fresh = (3 ** 13, 1300 + build_threads)
    fs = _inputs(shapes + [fresh], 2300)
    ref = _alone(shapes, fs[:-1])
    srv = sft.Server(mem_budget=2 << 30, max_batch=8, max_inflight=2,
                     variant=sft.sft_variant_init(**VARIANT), build_threads=build_threads)
    warm = _outputs(shapes[:1])
    for rid in _submit(srv, shapes[:1], fs[:1], warm):      # make the small plan resident
        assert srv.wait(rid, 60000) == sft.SFT_OK
    outs = _outputs([fresh] + shapes)
    ids = _submit(srv, [fresh] + shapes, [fs[-1]] + fs[:-1], outs)
    for rid in ids:
        assert srv.wait(rid, 120000) == sft.SFT_OK
    q_fresh = srv.query(ids[0])
    q_res = [srv.query(r) for r in ids[1:]]
    srv.destroy()
    ref = [_alone([fresh], fs[-1:])[0]] + ref
    _check_equal(outs, ref)
    assert not q_fresh["plan_reused"] and q_fresh["build_ms"] > 0
    print(f"build threads {build_threads}: new plan built in {q_fresh['build_ms']:.2f} ms; "
          f"first resident request queued {q_res[0]['queued_ms']:.3f} ms")
    if build_threads:
        assert q_res[0]["plan_reused"]
        assert q_res[0]["queued_ms"] < q_fresh["build_ms"], (q_res[0], q_fresh)
