"""GPU parity: the CUDA path through the C ABI against the CPU oracle, stage by stage.

Tolerances: coefficients within 1e-5 relative on the FP32 path and 1e-11 on the FP64
path; integer stages bit-exact (CRT and vote are re-run by the oracle on the GPU's own residues and
candidates); FP decisions (argmax residues) compared where the oracle's decision has margin.
"""
import math

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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1706_02740_gb300 import build
    build.build()
    sft.load()


CASES = [
    # N, s, seed, kappa, K, c_p, snr, magnitude
    (2 ** 14, 6, 11, 6, 5, 8.0, None, "unit"),
    (3 ** 9, 8, 12, 4, 5, 8.0, None, "unit"),
    (65521, 10, 13, 6, 5, 6.0, 30.0, "loguniform"),
    (2 ** 16, 8, 1000, 6, 5, 4.0, None, "unit"),           # configuration 1, trial 0
    (100003, 12, 14, 6, 7, 5.0, 40.0, "unit"),
]


@pytest.mark.parametrize("form", ["chirp", "rader"])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("case", CASES)
def test_stages_and_output_match_oracle(case, prec, form):
    """Every stage against the oracle; `form` chirp: the default prime pool and the chirp
    convolution; rader: the smooth prime pool (every p_j - 1 13-smooth) and Rader's form."""
    N, s, seed, kappa, K, c_p, snr, mag = case
    sig = make_signal(N, s, seed, mag, snr)
    f32 = as_complex64(sig.f)
    f = upcast(f32)
    kw = (dict(dft=sft.SFT_DFT_CHIRP) if form == "chirp"
          else dict(pool=sft.SFT_POOL_SMOOTH, dft=sft.SFT_DFT_RADER))
    g = U.run_gpu(sft, N, s, f32 if prec == U.FP32 else f, prec, kappa, K, c_p, seed, keep=True,
                  **kw)
    info, plan = g["info"], g["plan"]
    assert info["dft"] == (sft.SFT_DFT_CHIRP if form == "chirp" else sft.SFT_DFT_RADER)
    oplan = U.oracle_plan(info, N, s)
    assert oplan.shifts == info["shifts"] and oplan.L == info["L"]
    samples, bins, cand, resid = U.debug_arrays(sft, plan, info)
    gvoted = U.gpu_voted(sft, plan, info)
    plan.destroy()

    # (a) resampling at every node, every shift
    ref = U.oracle_samples(f, oplan, info)
    scale = np.max(np.abs(ref))
    tol_s = 2e-6 if prec == U.FP32 else 1e-13
    assert np.max(np.abs(samples - ref)) <= tol_s * scale

    res = O.dsft(f, oplan)
    primes, small = info["primes"], info["small"]
    offs = np.cumsum([0] + primes)
    for qi, sr in enumerate(res.shifts):
        bmax = max(np.max(np.abs(y)) for y in sr.Y)
        for j, p in enumerate(primes):
            Z = U.subbins(info, bins[qi], j)
            # (b) the p_j-node measurements Y_j
            tol_b = 2e-6 if prec == U.FP32 else 1e-13
            assert np.max(np.abs(Z[0] - sr.Y[j])) <= tol_b * bmax
            # (b') the folded sub-bins equal the oracle's length-(p t) measurement bins
            for l, t in enumerate(small):
                Xr = U.folded_subbins(info, Z, l)
                X = O.measure(f, oplan, sr.q, p * t)
                b = np.arange(p)
                for r in range(t):
                    u = ((r - b) * pow(p, -1, t)) % t
                    assert np.max(np.abs(Xr[r] - X[b + p * u])) <= tol_b * bmax
            # (c) residues agree wherever the oracle's decision has margin and the bin has energy
            energy = np.abs(sr.Y[j]) >= 1e-3 * bmax
            for l in range(len(small)):
                ok = (sr.margins[j][l] > 1e-3) & energy
                assert np.array_equal(resid[qi, offs[j]:offs[j + 1], l][ok], sr.residues[j][l][ok])
            # (c') CRT bit-exact on the GPU's own residues, every bin
            for b in range(p):
                w = U.crt_band(b, resid[qi, offs[j] + b, :len(small)], p, small, N)
                expect = np.iinfo(np.int64).min if w is None else w
                assert cand[qi, offs[j] + b] == expect
        # (d) the GPU's vote is the oracle's vote run on the GPU's own candidates: the same
        #     frequencies with the same counts; its medians are the oracle's within the bins'
        #     tolerance (a componentwise median moves by at most the largest input change)
        gv = U.oracle_vote(cand[qi], primes, len(primes))
        assert {w: v for w, (v, _) in gvoted[qi].items()} == gv
        for w, (_, z) in gvoted[qi].items():
            assert abs(z - O.median_estimate(sr.Y, primes, w)) <= 2 * tol_b * bmax
        # (d') against the oracle's own vote: a frequency kept (or counted) differently must have
        #      a candidate that differs at a bin whose residue decision had no margin
        ov = dict(zip(sr.voted.tolist(), sr.votes.tolist()))
        for w in set(ov) | set(gv):
            if ov.get(w) == gv.get(w):
                continue
            weak = False
            for j, p in enumerate(primes):
                b = w % p
                oc = np.iinfo(np.int64).min if sr.cand[j][b] is None else sr.cand[j][b]
                if cand[qi, offs[j] + b] != oc:
                    m = min((sr.margins[j][l][b] for l in range(len(small))), default=1.0)
                    weak |= m <= 1e-3 or abs(sr.Y[j][b]) < 1e-3 * bmax
            assert weak, (w, ov.get(w), gv.get(w))

    # final output: same support and ordering, coefficients within tolerance
    n = g["count"]
    assert n == len(res.freqs)
    tol = 1e-5 if prec == U.FP32 else 1e-11
    U.assert_same_output(g["freqs"][:n], g["coefs"][:n], res.freqs, res.coefs, tol)
    assert np.all(g["freqs"][n:] == 0) and np.all(g["coefs"][n:] == 0)


# Chirp-convolution lengths r 2^k, r = 3, 5, 7: last passes of radix 3, 6, 12 (12 then 2), 5, 10
# (10 then 2 or 4), 7, 14 (14 then 2 or 4); the largest prime of each plan is the largest below
# M/2 (the edge of the skipped first radix-2 pass), the smallest just above the next shorter length.
LENGTHS_ODD = [(96, [37, 41, 47]), (192, [67, 89]), (384, [131, 191]), (768, [257, 383]),
               (1536, [521, 761]), (3072, [1031, 1531]), (6144, [2053, 3067]),
               (12288, [4099, 6143]),
               (640, [257, 317]), (1280, [521, 631]), (2560, [1031, 1279]), (5120, [2053, 2557]),
               (10240, [4099, 5119]),
               (896, [389, 443]), (1792, [769, 887]), (3584, [1543, 1789]), (7168, [3079, 3583]),
               (14336, [6151, 7159]),
               # the longest power-of-two lengths of each path, primes up to the limits (p <= 4096
               # FP64, p <= 8192 FP32)
               (8192, [3593, 4093]), (16384, [7177, 8191])]


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("M,primes", LENGTHS_ODD)
def test_mixed_radix_lengths_match_oracle(M, primes, prec):
    if prec == U.FP64 and M > 8192:
        pytest.skip("FP64 chirp convolutions stop at length 8192")
    N, s = 2 ** 14, 4
    sig = make_signal(N, s, M, "unit", 30.0)
    f32 = as_complex64(sig.f)
    f = upcast(f32)
    g = U.run_gpu(sft, N, s, f32 if prec == U.FP32 else f, prec, 6, len(primes), 3.0, 0,
                  primes=primes, keep=True, dft=sft.SFT_DFT_CHIRP)
    info, plan = g["info"], g["plan"]
    assert info["fft_size"] == M and info["dft"] == sft.SFT_DFT_CHIRP
    oplan = U.oracle_plan(info, N, s)
    _, bins, _, _ = U.debug_arrays(sft, plan, info)
    plan.destroy()
    tol = 2e-6 if prec == U.FP32 else 1e-13
    for qi, q in enumerate(info["shifts"]):
        for j, p in enumerate(primes):
            Z = U.subbins(info, bins[qi], j)
            Y = O.measure(f, oplan, q, p)
            bmax = np.max(np.abs(Y))
            assert np.max(np.abs(Z[0] - Y)) <= tol * bmax
            for l, t in enumerate(info["small"]):
                Xr = U.folded_subbins(info, Z, l)
                X = O.measure(f, oplan, q, p * t)
                b = np.arange(p)
                for r in range(t):
                    u = ((r - b) * pow(p, -1, t)) % t
                    assert np.max(np.abs(Xr[r] - X[b + p * u])) <= tol * bmax


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_config1_recovers_truth(prec):
    """Configuration 1 (N = 2^16, s = 8, unit magnitudes, no noise), all 20 seeded trials: the
    exact support, against the brute-force DFT's best s-term approximation (here: the generating
    spectrum)."""
    for trial in range(20):
        sig = make_signal(2 ** 16, 8, 1000 + trial, "unit", None)
        f = sig.f if prec == U.FP64 else as_complex64(sig.f)
        g = U.run_gpu(sft, 2 ** 16, 8, f, prec, 6, 5, 8.0, trial)
        assert g["count"] == 8
        assert sorted(g["freqs"].tolist()) == sorted(sig.omega.tolist())


def test_input_types_and_precisions_agree():
    N, s = 2 ** 15, 7
    sig = make_signal(N, s, 5, "unit", None)
    f32 = as_complex64(sig.f)
    outs = []
    for prec, f in [(U.FP32, f32), (U.FP32, upcast(f32)), (U.FP64, f32), (U.FP64, upcast(f32))]:
        outs.append(U.run_gpu(sft, N, s, f, prec, 6, 5, 8.0, 1))
    for o in outs[1:]:
        assert sorted(o["freqs"].tolist()) == sorted(outs[0]["freqs"].tolist())
    assert np.array_equal(outs[2]["coefs"], outs[3]["coefs"])   # FP64 path: same widened input
    U.assert_same_output(outs[0]["freqs"], outs[0]["coefs"], outs[2]["freqs"], outs[2]["coefs"], 1e-5)
    assert np.array_equal(outs[0]["coefs"], outs[1]["coefs"])   # FP32 path narrows c128 exactly


@pytest.mark.parametrize("N,s,kappa,K,c_p", [(13, 1, 6, 3, 3.0), (9, 2, 4, 5, 3.0),
                                             (31, 31, 4, 3, 2.0), (1009, 1, 6, 1, 3.0),
                                             (3001, 1, 6, 3, 3100.0)])
def test_edge_cases_match_oracle(N, s, kappa, K, c_p):
    """Tiny N (window equal to N), s = N, a single modulus, and p_1 >= N (no small moduli)."""
    sig = make_signal(N, s, 7, "unit", None)
    f = sig.f
    g = U.run_gpu(sft, N, s, f, U.FP64, kappa, K, c_p, 3)
    oplan = U.oracle_plan(g["info"], N, s)
    res = O.dsft(f, oplan)
    n = g["count"]
    assert n == len(res.freqs)
    if n:
        U.assert_same_output(g["freqs"][:n], g["coefs"][:n], res.freqs, res.coefs, 1e-11)


@pytest.mark.parametrize("N,s,r", [(2 ** 14, 8, 1.0), (3 ** 9, 12, 1.0), (2 ** 14, 6, 2.0)])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_theorem_parameter_mode_matches_oracle(N, s, r, prec):
    """Theorem total_convolution_error's parameters (beta = 6 sqrt(r), half-width
    ceil(6 r ln N / (sqrt 2 pi)) + 1: 31 to 57 taps, the generic resampling kernel) on both paths."""
    import torch
    sig = make_signal(N, s, 40 + int(r), "unit", 40.0)
    f32 = as_complex64(sig.f)
    f = f32 if prec == U.FP32 else upcast(f32)
    v = sft.sft_variant_theorem(N, r, precision=prec, K=5, c_p=4.0, seed=2,
                                input=0 if prec == U.FP32 else 1)
    plan = sft.sft_plan(N, s, v)
    info = plan.info()
    assert info["kappa"] == v.kappa > 6
    w, c, n = sft.execute_torch(plan, torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    n = int(n.item())
    oplan = O.make_plan(N, s, kappa=info["kappa"], alpha=v.alpha, beta=v.beta,
                        primes=info["primes"], small=info["small"], n_shifts=info["n_shifts"])
    assert abs(oplan.c1 - info["c1"]) <= 1e-15 * oplan.c1
    # stage 1: every filtered sample against the oracle's direct per-tap sum
    got = U.debug_arrays(sft, plan, info)[0]
    ref = U.oracle_samples(upcast(f32), oplan, info)
    tol = 2e-6 if prec == U.FP32 else 1e-13
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    res = O.dsft(upcast(f32), oplan)
    assert n == len(res.freqs)
    U.assert_same_output(w.cpu().numpy()[:n], c.cpu().numpy()[:n], res.freqs, res.coefs,
                         1e-5 if prec == U.FP32 else 1e-11)
    assert set(res.freqs.tolist()) == set(sig.omega.tolist())
    plan.destroy()


@pytest.mark.parametrize("N,s,snr,prec,c128", [(100003, 12, 20.0, U.FP32, False),
                                               (2 ** 16, 8, None, U.FP32, False),
                                               (3 ** 10, 20, 20.0, U.FP64, True),
                                               (2 ** 15 + 3, 10, 30.0, U.FP32, True)])
def test_residual_energy_follows_parseval(N, s, snr, prec, c128):
    """rho = 1 - sum |c|^2 / (||f||^2 / N) against the same sums in float64 on the host."""
    import torch
    sig = make_signal(N, s, 77, "unit", snr)
    f = upcast(as_complex64(sig.f)) if c128 else as_complex64(sig.f)
    v = sft.sft_variant_init(precision=prec, K=5, c_p=5.0, seed=4, input=1 if c128 else 0)
    plan = sft.sft_plan(N, s, v)
    ft = torch.from_numpy(f).cuda()
    w, c, n = sft.execute_torch(plan, ft)
    rho = sft.residual_energy_torch(plan, ft, c, n)
    nn = int(n.item())
    fh = f.astype(np.complex128)
    ref = 1.0 - np.sum(np.abs(c.cpu().numpy()[:nn]) ** 2) / (np.sum(np.abs(fh) ** 2) / N)
    assert abs(rho - ref) <= 1e-12
    if snr is None:
        assert abs(rho) <= 1e-5                  # exactly s-sparse: the s terms carry it all
    else:
        # the noise's share of the energy, less what the estimates absorb (each bin aliases the
        # noise of ~L/p frequencies, amplified by 1/g_hat towards the band edges)
        noise = 1.0 / (1.0 + 10.0 ** (snr / 10.0))
        assert abs(rho) < 3.0 * noise
    plan.destroy()


def test_repeated_execution_is_deterministic():
    N, s = 2 ** 17, 16
    sig = make_signal(N, s, 9, "unit", 30.0)
    f32 = as_complex64(sig.f)
    import torch
    plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=6.0))
    ft = torch.from_numpy(f32).cuda()
    first = None
    for _ in range(3):
        w, c, n = sft.execute_torch(plan, ft)
        torch.cuda.synchronize()
        cur = (w.cpu().numpy().copy(), c.cpu().numpy().copy(), int(n.item()))
        if first is None:
            first = cur
        else:
            assert np.array_equal(cur[0], first[0]) and np.array_equal(cur[1], first[1])
    plan.destroy()


@pytest.mark.parametrize("N,s,c_p", [(3 ** 7, 3, 2.0), (2 ** 12, 4, 2.0), (2 ** 14, 6, 2.0)])
@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_deterministic_inner_sft_matches_oracle_and_recovers_exactly(N, s, c_p, prec):
    """The deterministic inner SFT (K = 2 (s - 1) floor(log_{p_1}(N - 1)) + 1 consecutive primes:
    13, 19 and 31 here, beyond the register path's 16) on random and adversarial spectra (all
    frequencies congruent modulo the first primes): output equal to the oracle's and to the
    generating spectrum."""
    import torch
    from synth.signals import samples_from_spectrum
    v = sft.sft_variant_init(precision=prec, c_p=c_p, deterministic=1, input=1)
    plan = sft.sft_plan(N, s, v)
    info = plan.info()
    assert info["primes"] == O.deterministic_primes(N, s, c_p)
    oplan = O.make_plan(N, s, kappa=info["kappa"], c_p=c_p, deterministic=True)
    assert oplan.primes == info["primes"] and oplan.small == info["small"]
    B = np.arange(-((N + 1) // 2) + 1, N // 2 + 1, dtype=np.int64)
    rng = np.random.default_rng(N + s)
    step = info["primes"][0] * info["primes"][1]
    step = step if step * (s - 1) < N // 2 else info["primes"][0]
    spectra = [np.array([(i - s // 2) * step for i in range(s)], dtype=np.int64),
               rng.choice(B, size=s, replace=False)]
    for w in spectra:
        coef = np.exp(2j * np.pi * rng.random(s))
        f = samples_from_spectrum(N, w, coef)
        gw, gc, gn = sft.execute_torch(plan, torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        n = int(gn.item())
        res = O.dsft(f, oplan)
        assert sorted(res.freqs.tolist()) == sorted(w.tolist())
        assert n == s
        U.assert_same_output(gw.cpu().numpy()[:n], gc.cpu().numpy()[:n], res.freqs, res.coefs,
                             1e-5 if prec == U.FP32 else 1e-11)
    plan.destroy()


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
def test_input_in_pinned_host_memory_gives_the_same_bits(prec):
    """A page-locked host input (read window by window over the host link) against the same signal
    in device memory: identical results, single execution and batch."""
    import torch
    N, s = 2 ** 18, 40
    sig = make_signal(N, s, 77, "loguniform", 30.0)
    f = as_complex64(sig.f) if prec == U.FP32 else upcast(as_complex64(sig.f))
    fd = torch.from_numpy(f).cuda()
    fh = torch.from_numpy(f).pin_memory()
    v = sft.sft_variant_init(precision=prec, K=5, c_p=4.0, seed=3, input=0 if prec == U.FP32 else 1)
    plan = sft.sft_plan(N, s, v)
    wd, cd, nd = sft.execute_torch(plan, fd)
    wh, ch, nh = sft.execute_torch(plan, fh)
    torch.cuda.synchronize()
    assert int(nd.item()) == int(nh.item()) > 0
    assert torch.equal(wd, wh) and torch.equal(cd, ch)
    batch = sft.Batch([plan])
    outs = sft.execute_batch_torch(batch, [fh])
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], wd) and torch.equal(outs[0][1], cd)
    batch.destroy()
    plan.destroy()


def test_fp32_path_without_refinement():
    """refine_fp64 = 0: the FP32 path returns its FP32 medians divided by g_hat (no re-estimation
    kernels): the same support as with refinement, coefficients within the FP32 DFTs' rounding
    (2e-6 of the largest bin, amplified by 1/g_hat at most sqrt(2 pi) e^{1/2} towards the band
    edges, i.e. below 2e-5 of the largest coefficient), three fewer launches."""
    import torch
    N, s = 2 ** 18, 24
    sig = make_signal(N, s, 31, "loguniform", 40.0)
    f = torch.from_numpy(as_complex64(sig.f)).cuda()
    outs = {}
    for refine in (1, 0):
        plan = sft.sft_plan(N, s, sft.sft_variant_init(K=5, c_p=5.0, seed=8, refine_fp64=refine))
        w, c, n = sft.execute_torch(plan, f)
        torch.cuda.synchronize()
        nn = int(n.item())
        outs[refine] = (w.cpu().numpy()[:nn], c.cpu().numpy()[:nn], sft.sft_plan_launches(plan))
        plan.destroy()
    (w1, c1, l1), (w0, c0, l0) = outs[1], outs[0]
    assert sorted(w1.tolist()) == sorted(w0.tolist())
    m1 = dict(zip(w1.tolist(), c1))
    ref = np.array([m1[int(w)] for w in w0])
    assert np.max(np.abs(c0 - ref)) <= 2e-5 * np.max(np.abs(ref))
    assert l1 - l0 == 3


# Rader's form: primes whose p - 1 exercises every radix of the pass schedule (2, 3, 4, 5, 6, 7, 8,
# 10, 11, 12, 13, 14, 16), one-pass transforms (p = 3, 5, 7, 11, 13, 17), and the largest primes
# each precision accepts (13441 - 1 = 2^7 3 5 7 for FP32, 6761 - 1 = 2^3 5 13^2 for FP64).
RADER_PRIMES = [[3, 5, 7], [11, 13, 17], [23, 29, 31], [37, 53, 67], [79, 89, 97],
                [1459, 2017, 2161], [3001, 3137, 3361], [6553, 6761], [12289, 13441]]


@pytest.mark.parametrize("prec", [U.FP32, U.FP64])
@pytest.mark.parametrize("primes", RADER_PRIMES)
def test_rader_lengths_match_oracle(primes, prec):
    if prec == U.FP64 and max(primes) > 6801:
        pytest.skip("FP64 Rader transforms stop at p = 6801")
    N, s = 2 ** 14, 2
    sig = make_signal(N, s, sum(primes), "unit", 30.0)
    f32 = as_complex64(sig.f)
    f = upcast(f32)
    g = U.run_gpu(sft, N, s, f32 if prec == U.FP32 else f, prec, 6, len(primes), 3.0, 0,
                  primes=primes, keep=True, dft=sft.SFT_DFT_RADER)
    info, plan = g["info"], g["plan"]
    assert info["dft"] == sft.SFT_DFT_RADER and info["fft_size"] == 0
    oplan = U.oracle_plan(info, N, s)
    _, bins, _, _ = U.debug_arrays(sft, plan, info)
    plan.destroy()
    tol = 2e-6 if prec == U.FP32 else 1e-13
    for qi, q in enumerate(info["shifts"]):
        for j, p in enumerate(primes):
            Z = U.subbins(info, bins[qi], j)
            Y = O.measure(f, oplan, q, p)
            bmax = np.max(np.abs(Y))
            assert np.max(np.abs(Z[0] - Y)) <= tol * bmax, (p, qi)
            for l, t in enumerate(info["small"]):
                Xr = U.folded_subbins(info, Z, l)
                X = O.measure(f, oplan, q, p * t)
                b = np.arange(p)
                for r in range(t):
                    u = ((r - b) * pow(p, -1, t)) % t
                    assert np.max(np.abs(Xr[r] - X[b + p * u])) <= tol * bmax, (p, qi, t)


def test_rader_and_chirp_forms_agree():
    """The same plan parameters in both forms: same support, coefficients within the FP32 path's
    tolerance of each other, and Rader's form at least as accurate against the oracle."""
    import torch
    N, s = 2 ** 20, 40
    sig = make_signal(N, s, 71, "loguniform", 40.0)
    f32 = as_complex64(sig.f)
    primes = O.choose_primes(s, 5, 3.0, 4, "smooth")
    outs = {}
    for form in (sft.SFT_DFT_CHIRP, sft.SFT_DFT_RADER):
        g = U.run_gpu(sft, N, s, f32, U.FP32, 6, 5, 3.0, 4, primes=primes, dft=form)
        outs[form] = g
    res = O.dsft(upcast(f32), U.oracle_plan(outs[sft.SFT_DFT_RADER]["info"], N, s))
    for form, g in outs.items():
        n = g["count"]
        U.assert_same_output(g["freqs"][:n], g["coefs"][:n], res.freqs, res.coefs, 1e-5)
