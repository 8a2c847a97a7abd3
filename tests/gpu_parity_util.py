"""Helpers of the GPU parity tests: run the C ABI on a signal, read the plan's intermediate
buffers, and compare every stage with the CPU oracle on the same input and the same moduli."""
from __future__ import annotations

import math

import numpy as np

from oracle import dsft as O

FP32, FP64 = 0, 1


def run_gpu(sft, N, s, f, prec=FP32, kappa=6, K=5, c_p=3.0, seed=0, primes=None, small=None,
            input_type=None, n_shifts=0, keep=False):
    import torch
    if input_type is None:
        input_type = 0 if f.dtype == np.complex64 else 1
    v = sft.sft_variant_init(precision=prec, kappa=kappa, K=K, c_p=c_p, seed=seed, input=input_type)
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


def oracle_vote(cand_q, primes, K):
    """Apply the vote rule to a candidate array (one shift)."""
    offs = np.cumsum([0] + list(primes))
    found = {}
    for j, p in enumerate(primes):
        for b in range(p):
            w = int(cand_q[offs[j] + b])
            if w != np.iinfo(np.int64).min:
                found.setdefault(w, set()).add(j)
    need = K // 2 + 1
    return sorted(w for w, js in found.items() if len(js) >= need)


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
