"""Helpers of the GPU parity tests: run the C ABI on a signal, read the plan's intermediate
buffers, and compare every stage with the CPU oracle on the same input and the same moduli."""
from __future__ import annotations

import math

import numpy as np

from oracle import dsft as O

FP32, FP64 = 0, 1


def run_gpu(sft, N, s, f, prec=FP32, kappa=6, K=5, c_p=3.0, seed=0, primes=None, small=None,
            input_type=None, n_shifts=0, keep=False, pool=0, dft=0):
    import torch
    if input_type is None:
        input_type = 0 if f.dtype == np.complex64 else 1
    v = sft.sft_variant_init(precision=prec, kappa=kappa, K=K, c_p=c_p, seed=seed, input=input_type,
                             pool=pool, dft=dft)
    plan = sft.sft_plan(N, s, v, n_shifts=n_shifts, primes=primes, small_moduli=small)
    ft = torch.from_numpy(np.ascontiguousarray(f)).to("cuda")
    w, c, n = sft.execute_torch(plan, ft)
    torch.cuda.synchronize()
    n = int(n.item())
    out = dict(plan=plan, info=plan.info(), freqs=w.cpu().numpy(), coefs=c.cpu().numpy(), count=n)
    if not keep:
        plan.destroy()
    return out


def oracle_plan(info, N, s):
    return O.make_plan(N, s, kappa=info["kappa"], primes=info["primes"], small=info["small"],
                       n_shifts=info["n_shifts"])


def node_list(info):
    """(P, k) of every node in the library's node order: prime j, subset u, k1."""
    out = []
    nsub = info["n_sub"]
    subs = [(1, 0)]
    for t in info["small"]:
        subs += [(t, k2) for k2 in range(1, t)]
    assert len(subs) == nsub
    for p in info["primes"]:
        for (t, k2) in subs:
            k1 = np.arange(p, dtype=np.int64)
            if t == 1:
                out.append((p, k1))
            else:
                out.append((p * t, (k1 * t + k2 * p) % (p * t)))
    return out, subs


def debug_arrays(sft, plan, info):
    import torch
    nq, m = info["n_shifts"], info["nodes"]
    ctype = torch.complex128 if info["precision"] == 1 else torch.complex64
    ptot = sum(info["primes"])
    samples = sft.debug_tensor(plan, sft.BUF_SAMPLES, ctype, (nq, m)).cpu().numpy()
    bins = sft.debug_tensor(plan, sft.BUF_BINS, ctype, (nq, m)).cpu().numpy()
    cand = sft.debug_tensor(plan, sft.BUF_CAND, torch.int64, (nq, ptot)).cpu().numpy()
    nT = max(1, info["n_small"])
    resid = sft.debug_tensor(plan, sft.BUF_RESID, torch.uint8, (nq, ptot, nT)).cpu().numpy()
    return samples, bins, cand, resid


def oracle_samples(f, oplan, info):
    nodes, _ = node_list(info)
    rows = []
    for q in oplan.shifts:
        rows.append(np.concatenate([O.resample(f, oplan, P, k, q) for (P, k) in nodes]))
    return np.array(rows)


def subbins(info, bins_q, j):
    """The library's length-p_j measurements of prime j as an array [n_sub, p_j]."""
    p = info["primes"][j]
    off = info["n_sub"] * sum(info["primes"][:j])
    return bins_q[off: off + info["n_sub"] * p].reshape(info["n_sub"], p)


def folded_subbins(info, Z, l):
    """X_r[b] = (1/t) sum_{k2 < t} Z_{k2}[b] e^{-2 pi i k2 r / t} (prime-factor index map) for small
    modulus l, returned as [t, p] indexed by residue r."""
    t = info["small"][l]
    base = 1 + sum(tt - 1 for tt in info["small"][:l])
    rows = [Z[0]] + [Z[base + k2 - 1] for k2 in range(1, t)]
    Zs = np.array(rows)                                       # [t (k2), p]
    r = np.arange(t)
    E = np.exp(-2j * math.pi * np.outer(r, np.arange(t)) / t)  # [r, k2]
    return (E @ Zs) / t


def crt_band(b, residues, p, small, N):
    wt = O.crt([b] + [int(r) for r in residues], [p] + list(small))
    return O.to_band(wt, p * math.prod(small), N)


def cand_lists(cand_q, primes):
    """One shift's GPU candidate array [sum p] as the oracle's per-modulus lists (None: no
    frequency)."""
    offs = np.cumsum([0] + list(primes))
    nofreq = np.iinfo(np.int64).min
    return [[None if int(w) == nofreq else int(w) for w in cand_q[offs[j]:offs[j + 1]]]
            for j in range(len(primes))]


def oracle_vote(cand_q, primes, K):
    """The oracle's vote applied to the GPU's candidates of one shift: {w: votes}."""
    voted, votes = O.majority_vote(cand_lists(cand_q, primes), K)
    return dict(zip(voted.tolist(), votes.tolist()))


VOTED_DTYPE = np.dtype([("w", "<i8"), ("zre", "<f8"), ("zim", "<f8"), ("votes", "<i4"),
                        ("jmin", "<i4")])


def gpu_voted(sft, plan, info):
    """The GPU vote's output, per shift: {w: (votes, z)} from the plan's voted lists."""
    import torch
    nq = info["n_shifts"]
    counts = sft.debug_tensor(plan, sft.BUF_COUNTERS, torch.int32, (nq + 4,)).cpu().numpy()
    _, nbytes = sft.sft_plan_debug_buffer(plan, sft.BUF_VOTED)
    raw = sft.debug_tensor(plan, sft.BUF_VOTED, torch.uint8, (nbytes,)).cpu().numpy()
    vcap = nbytes // (nq * VOTED_DTYPE.itemsize)
    recs = raw.view(VOTED_DTYPE).reshape(nq, vcap)
    out = []
    for qi in range(nq):
        n = int(counts[qi])
        assert n <= vcap, "voted list overflowed"
        r = recs[qi, :n]
        d = {int(w): (int(v), complex(a, b)) for w, v, a, b in zip(r["w"], r["votes"], r["zre"],
                                                                   r["zim"])}
        assert len(d) == n, "a frequency was voted twice"
        out.append(d)
    return out


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def assert_same_output(gw, gc, ow, oc, tol):
    """Same frequency set; coefficients matched by frequency within tol relative; the GPU order is
    sorted by its own magnitudes (ties by frequency) and agrees with the oracle's order wherever the
    oracle's magnitudes differ by more than 2 tol (equal magnitudes may legitimately swap)."""
    gw, ow = np.asarray(gw), np.asarray(ow)
    assert sorted(gw.tolist()) == sorted(ow.tolist())
    omap = dict(zip(ow.tolist(), oc))
    ref = np.array([omap[int(w)] for w in gw])
    assert rel_err(gc, ref) <= tol, rel_err(gc, ref)
    # the library ranks by re^2 + im^2 (possibly FMA-contracted): sorted up to last-ulp ties
    mg = gc.real * gc.real + gc.imag * gc.imag
    for i in range(len(gw) - 1):
        assert mg[i] >= mg[i + 1] * (1 - 1e-14)
    mo = np.abs(ref)
    for i in range(len(gw) - 1):
        for k in range(i + 1, len(gw)):
            if mo[k] > mo[i] * (1 + 2 * tol):
                raise AssertionError(f"order differs: {gw[i]} before {gw[k]}")


def explain_output_differences(g, res, cand, info, tol, margin=1e-3, log=None):
    """Account for every frequency that only one side returns (the rule for FP decisions: integer
    stages agree given the same residues, and residues agree wherever the oracle's decision margin
    exceeds `margin`).  A frequency w returned by one side only is explained when

    * decision: at some modulus j the GPU's candidate of bin w mod p_j (shift of w's band) differs
      from the oracle's, and there the oracle's residue decision had no margin (some small modulus
      with margin <= `margin`) or the bin had no energy (< `margin` of the shift's largest bin); or
    * cut: the other side's output is full (s terms) and |c_w| is no larger than the other side's
      weakest returned coefficient, within 2 tol (the s-th magnitude decides, in the path's
      precision).

    Returns [(w, side, reason)]; raises AssertionError on a difference neither explains.  `cand` is
    the GPU's candidate array [n_shifts][sum p]."""
    n = g["count"]
    gmap = dict(zip(g["freqs"][:n].tolist(), g["coefs"][:n]))
    omap = dict(zip(res.freqs.tolist(), res.coefs))
    s = info["s"]
    primes, L = info["primes"], info["L"]
    offs = np.cumsum([0] + list(primes))
    nofreq = np.iinfo(np.int64).min
    gmin = min((abs(c) for c in gmap.values()), default=0.0)
    omin = min((abs(c) for c in omap.values()), default=0.0)
    out = []
    for w in sorted(set(gmap) ^ set(omap)):
        side = "gpu" if w in gmap else "oracle"
        c = gmap[w] if w in gmap else omap[w]
        reason = None
        qi = [i for i, q in enumerate(info["shifts"]) if q - L <= w < q + L]
        assert len(qi) == 1, (w, qi)
        sr = res.shifts[qi[0]]
        bmax = max(np.max(np.abs(y)) for y in sr.Y)
        for j, p in enumerate(primes):
            b = w % p
            oc = nofreq if sr.cand[j][b] is None else sr.cand[j][b]
            if int(cand[qi[0], offs[j] + b]) == oc:
                continue
            m = min((float(sr.margins[j][l][b]) for l in range(len(info["small"]))), default=1.0)
            e = abs(sr.Y[j][b]) / bmax
            if m <= margin or e < margin:
                reason = f"decision at p={p} bin {b}: margin {m:.2e}, energy {e:.2e}"
                break
        if reason is None:
            other_full = (len(omap) if side == "gpu" else len(gmap)) == s
            other_min = omin if side == "gpu" else gmin
            if other_full and abs(c) <= other_min * (1 + 2 * tol):
                reason = f"cut: |c| {abs(c):.6e} vs other side's weakest {other_min:.6e}"
        if reason is None:
            raise AssertionError(f"unexplained difference: w={w} only on the {side} side, |c|={abs(c):.3e}")
        out.append((w, side, reason))
        if log is not None:
            log(f"w={w} only on the {side} side: {reason}")
    return out
