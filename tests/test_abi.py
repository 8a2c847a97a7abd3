"""CPU checks of the C ABI: the library builds, loads, exports every symbol include/sft.h declares,
and its host-only logic (argument validation, seeded moduli choice) agrees with the oracle.
No device work runs here."""
import ctypes
import os
import re

import pytest

import paper_1706_02740_gb300 as sft
from paper_1706_02740_gb300 import build as sft_build
from oracle import dsft as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sft_build.build()
    return sft.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sft.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sft_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sft_plan" in names and "sft_execute" in names and len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
        assert name in sft.EXPORTS, f"binding misses {name}"


def test_struct_sizes_match_header_layout():
    # sft_variant: 4 x int32, 3 x double, uint64, 4 x int32
    assert ctypes.sizeof(sft.sft_variant) == 64
    assert sft.SFT_MAX_K == 512
    assert ctypes.sizeof(sft.sft_plan_desc) == 8 + 6 * 4 + 512 * 8 + 12 * 4 + 32 * 8 + 8 + 8 + 8 + 16


def test_tuning_layout_and_defaults(lib):
    # sft_tuning: 13 x int32
    assert ctypes.sizeof(sft.sft_tuning) == 13 * 4
    t = sft.sft_tuning_default()
    assert t["resample_threads"] == 256 and t["resample_regcap"] == 0 and t["bin_threads"] == 256
    # transforms per CTA: a 256-thread CTA below M = 4096, one transform from there on
    assert t["dft_per_cta"] == [64, 32, 16, 8, 4, 2, 1, 1, 1]
    assert t["dft_two_ctas"] == 1


def test_server_structs_and_config_defaults(lib):
    assert ctypes.sizeof(sft.sft_server_config) == 8 + 4 + 4 + 64 + 13 * 4 + 2 * 4 + 4  # + padding
    assert ctypes.sizeof(sft.sft_request_info) == 4 * 4 + 3 * 8
    assert ctypes.sizeof(sft.sft_server_stats) == 8 * 8 + 3 * 8 + 2 * 4 + 8
    cfg = sft.sft_server_config()
    lib.sft_server_config_init(ctypes.byref(cfg))
    assert cfg.mem_budget == 8 << 30 and cfg.max_batch == 64 and cfg.max_inflight == 2
    assert cfg.build_threads == 2
    assert (cfg.variant.kappa, cfg.variant.K) == (6, 5)
    assert cfg.tune.resample_threads == 256


@pytest.mark.parametrize("field,value", [("mem_budget", 1000), ("max_batch", 0), ("max_batch", 257),
                                         ("max_inflight", 0), ("max_inflight", 9),
                                         ("build_threads", -1), ("build_threads", 17)])
def test_server_rejects_bad_configurations_without_touching_the_device(lib, field, value):
    cfg = sft.sft_server_config()
    lib.sft_server_config_init(ctypes.byref(cfg))
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.sft_server_create(ctypes.byref(h), ctypes.byref(cfg)) == sft.SFT_EINVAL
    assert not h.value


@pytest.mark.parametrize("N,r,kappa", [(2 ** 26, 1.0, 26), (2 ** 14, 1.0, 15), (3 ** 9, 2.0, 28),
                                        (2 ** 20, 1.5, 30)])
def test_theorem_variant(lib, N, r, kappa):
    # Theorem total_convolution_error: beta = 6 sqrt(r), half-width ceil(6 r ln N / (sqrt 2 pi)) + 1
    import math
    v = sft.sft_variant_theorem(N, r)
    assert v.kappa == kappa == math.ceil(6 * r * math.log(N) / (math.sqrt(2) * math.pi)) + 1
    assert abs(v.beta - 6 * math.sqrt(r)) < 1e-15 and v.alpha == v.beta
    assert (v.K, v.c_p, v.precision) == (5, 3.0, 0)


@pytest.mark.parametrize("N,r", [(2 ** 26, 2.0), (100, 3.0), (2 ** 20, 0.5)])
def test_theorem_variant_rejects_out_of_range(lib, N, r):
    v = sft.sft_variant_init()
    assert lib.sft_variant_theorem(ctypes.byref(v), N, r) == sft.SFT_EINVAL
    assert v.kappa == 6 and v.beta == 1.5


def test_variant_defaults(lib):
    v = sft.sft_variant_init()
    assert (v.kappa, v.precision, v.input, v.K) == (6, 0, 0, 5)
    assert (v.c_p, v.alpha, v.beta, v.seed, v.deterministic) == (3.0, 1.5, 1.5, 0, 0)
    assert (v.refine_fp64, v.pool, v.dft) == (1, sft.SFT_POOL_ALL, sft.SFT_DFT_AUTO)


@pytest.mark.parametrize("N,s,K,c_p,seed", [(2 ** 16, 8, 5, 4.0, 0), (2 ** 22, 64, 5, 3.0, 7),
                                            (2 ** 26, 1000, 5, 3.0, 123), (4194301, 64, 7, 8.0, 2),
                                            (1000003, 3, 3, 10.0, 2 ** 63 + 5), (97, 2, 5, 3.0, 1)])
def test_moduli_choice_matches_oracle(lib, N, s, K, c_p, seed):
    primes, small = sft.sft_choose_moduli(N, s, K, c_p, seed)
    assert primes == O.choose_primes(s, K, c_p, seed)
    assert small == O.choose_small_moduli(N, primes)


@pytest.mark.parametrize("N,s,K,c_p,seed", [(2 ** 16, 8, 5, 4.0, 0), (2 ** 26, 1000, 5, 3.0, 1),
                                            (2 ** 26, 4000, 9, 2.5, 3), (4194301, 64, 7, 3.0, 2),
                                            (1000003, 3, 3, 10.0, 2 ** 63 + 5)])
def test_smooth_pool_choice_matches_oracle(lib, N, s, K, c_p, seed):
    primes, small = sft.sft_choose_moduli_pool(N, s, K, c_p, seed, sft.SFT_POOL_SMOOTH)
    assert primes == O.choose_primes(s, K, c_p, seed, "smooth")
    assert all(O.is_smooth(p - 1) for p in primes)
    assert small == O.choose_small_moduli(N, primes)
    assert sft.sft_choose_moduli_pool(N, s, K, c_p, seed, sft.SFT_POOL_ALL) == \
        sft.sft_choose_moduli(N, s, K, c_p, seed)


def test_dft_form_limits_are_checked_on_the_host(lib):
    # Rader's form needs every p_j - 1 13-smooth: 3011 - 1 = 2 5 7 43 is refused
    with pytest.raises(sft.SftError) as e:
        sft.sft_plan(2 ** 20, 100, sft.sft_variant_init(dft=sft.SFT_DFT_RADER), primes=[3001, 3011])
    assert e.value.status == sft.SFT_EINVAL and "13" in sft.sft_last_error()
    # beyond the chirp form's 8192 only Rader's form reaches (FP32): 12289 - 1 = 2^12 3, but a chirp
    # plan of it is refused
    with pytest.raises(sft.SftError) as e:
        sft.sft_plan(2 ** 20, 100, sft.sft_variant_init(dft=sft.SFT_DFT_CHIRP), primes=[12289])
    assert e.value.status == sft.SFT_EINVAL and "8192" in sft.sft_last_error()
    with pytest.raises(sft.SftError):
        sft.sft_plan(2 ** 20, 100, sft.sft_variant_init(pool=7))
    with pytest.raises(sft.SftError):
        sft.sft_plan(2 ** 20, 100, sft.sft_variant_init(dft=9))


@pytest.mark.parametrize("kw", [dict(N=1, s=1), dict(N=100, s=0), dict(N=100, s=101),
                                dict(N=2 ** 31, s=2), dict(N=12, s=2)])
def test_plan_rejects_bad_sizes_without_touching_the_device(lib, kw):
    with pytest.raises(sft.SftError) as e:
        sft.sft_plan(kw["N"], kw["s"])
    assert e.value.status == sft.SFT_EINVAL


def test_plan_rejects_bad_moduli(lib):
    for primes, small in [([101, 101, 103], None), ([100, 103, 107], None),
                          ([101, 103, 107], [2, 4]), ([101, 103, 107], [2, 3]),
                          ([101, 103, 107], [101, 2, 3, 5, 7])]:
        with pytest.raises(sft.SftError) as e:
            sft.sft_plan(2 ** 16, 8, primes=primes, small_moduli=small)
        assert e.value.status == sft.SFT_EINVAL
    with pytest.raises(sft.SftError):
        sft.sft_plan(2 ** 16, 8, sft.sft_variant_init(kappa=0))
    with pytest.raises(sft.SftError):
        sft.sft_plan(2 ** 16, 4000, sft.sft_variant_init(precision=1))   # p_j > 4096 in FP64
    assert "4096" in sft.sft_last_error()


def test_execute_rejects_null_and_partial_outputs(lib):
    with pytest.raises(sft.SftError):
        sft.sft_execute(sft.Plan(None), 0, 0, 0, 0, 0)


def _header_enum(prefix):
    text = open(os.path.join(ROOT, "include", "sft.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"\w+)\s*=\s*(\d+)", text)}


def test_checked_build_exports_every_declared_symbol(lib):
    """The checked build (index checks compiled in) is the same ABI; each library says which it
    is."""
    import ctypes as C
    chk = C.CDLL(sft_build.LIB_CHECKED)
    for name in declared_functions():
        assert hasattr(chk, name), name
    chk.sft_checked_build.restype = C.c_int32
    assert chk.sft_checked_build() == 1
    assert lib.sft_checked_build() == 0


def test_fault_codes_match_header():
    faults = _header_enum("SFT_FAULT_")
    sites = _header_enum("SFT_SITE_")
    assert faults == {"SFT_FAULT_VOTED_FULL": 1, "SFT_FAULT_POOL_FULL": 2, "SFT_FAULT_INDEX": 4}
    for k, v in faults.items():
        assert getattr(sft, k) == v
    assert len(sites) == 6
    for k, v in sites.items():
        assert getattr(sft, k) == v


def test_fault_hooks_check_their_arguments_on_the_host(lib):
    with pytest.raises(sft.SftError) as e:
        sft.sft_debug_fail_allocations(-1, 1)
    assert e.value.status == sft.SFT_EINVAL
    sft.sft_debug_fail_allocations(0, 0)
    assert lib.sft_plan_faults(None, None, None, None) == sft.SFT_EINVAL
    assert lib.sft_plan_debug_limit(None, 0, 1) == sft.SFT_EINVAL


def test_missing_library_fails_loudly():
    """No fallback: with the compiled library absent, the first call into the module raises."""
    import subprocess
    import sys
    code = ("import paper_1706_02740_gb300 as s, paper_1706_02740_gb300.build as b\n"
            "b.LIB = '/nonexistent/libsft.so'\n"
            "try:\n"
            "    s.sft_variant_init()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "raised:" in out.stdout and "not built" in out.stdout


def test_every_entry_point_is_documented_in_the_header():
    """Each sft_* declaration of include/sft.h follows a comment block (declarations grouped under
    one comment share it), so no entry point goes without its argument, ownership and error
    description."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = open(os.path.join(root, "include", "sft.h")).read().split("\n")
    decl = re.compile(r"^(?:sft_status|void|const char\s*\*|int32_t|int64_t|size_t|double|int)"
                      r"\s+\**(sft_\w+)\s*\(")
    contin = re.compile(r"^\s{4,}\S")
    undocumented = []
    for i, ln in enumerate(lines):
        m = decl.match(ln)
        if not m:
            continue
        j = i - 1
        while j >= 0 and (decl.match(lines[j]) or contin.match(lines[j])):
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented
