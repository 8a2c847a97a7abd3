"""Python binding of the GB300 discrete sparse Fourier transform library (include/sft.h).

Argument marshalling only: every step of the transform runs in the CUDA kernels of libsft.so.
The functions keep the C names (sft_plan, sft_execute, ...).  Device buffers are passed as raw
pointers; the torch helpers below only allocate outputs and pass tensor pointers and the current
stream.  If the library has not been built, importing the package still works but every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SFT_OK, SFT_EINVAL, SFT_ENOMEM, SFT_ECUDA, SFT_ETIMEOUT, SFT_EBUSY = range(6)
SFT_DMSFT4, SFT_DMSFT6 = 4, 6
SFT_FP32, SFT_FP64 = 0, 1
SFT_IN_C64, SFT_IN_C128 = 0, 1
SFT_POOL_ALL, SFT_POOL_SMOOTH = 0, 1
SFT_DFT_AUTO, SFT_DFT_CHIRP, SFT_DFT_RADER = 0, 1, 2
SFT_MAX_K, SFT_MAX_SMALL, SFT_MAX_SHIFTS = 512, 12, 32
BUF_SAMPLES, BUF_BINS, BUF_CAND, BUF_RESID, BUF_COUNTERS, BUF_VOTED = range(6)
SFT_FAULT_VOTED_FULL, SFT_FAULT_POOL_FULL, SFT_FAULT_INDEX = 1, 2, 4
(SFT_SITE_NONE, SFT_SITE_WINDOW, SFT_SITE_DFT, SFT_SITE_SUBBIN, SFT_SITE_VOTE,
 SFT_SITE_REESTIMATE) = range(6)

_STATUS = {0: "SFT_OK", 1: "SFT_EINVAL", 2: "SFT_ENOMEM", 3: "SFT_ECUDA", 4: "SFT_ETIMEOUT",
           5: "SFT_EBUSY"}


class SftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sft_variant(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("input", ctypes.c_int32), ("K", ctypes.c_int32), ("c_p", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("deterministic", ctypes.c_int32), ("refine_fp64", ctypes.c_int32),
                ("pool", ctypes.c_int32), ("dft", ctypes.c_int32)]


class sft_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("s", ctypes.c_int32), ("kappa", ctypes.c_int32),
                ("K", ctypes.c_int32), ("n_small", ctypes.c_int32), ("n_shifts", ctypes.c_int32),
                ("n_sub", ctypes.c_int32), ("primes", ctypes.c_int64 * SFT_MAX_K),
                ("small", ctypes.c_int32 * SFT_MAX_SMALL),
                ("shifts", ctypes.c_int64 * SFT_MAX_SHIFTS), ("L", ctypes.c_int64),
                ("c1", ctypes.c_double), ("nodes", ctypes.c_int64), ("fft_size", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("input", ctypes.c_int32),
                ("dft", ctypes.c_int32)]


class sft_tuning(ctypes.Structure):
    _fields_ = [("resample_threads", ctypes.c_int32), ("resample_regcap", ctypes.c_int32),
                ("bin_threads", ctypes.c_int32), ("dft_per_cta", ctypes.c_int32 * 9),
                ("dft_two_ctas", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"resample_threads": self.resample_threads, "resample_regcap": self.resample_regcap,
                "bin_threads": self.bin_threads, "dft_per_cta": list(self.dft_per_cta),
                "dft_two_ctas": self.dft_two_ctas}

    @classmethod
    def from_dict(cls, d: dict) -> "sft_tuning":
        t = cls()
        for k, v in d.items():
            if k == "dft_per_cta":
                t.dft_per_cta = (ctypes.c_int32 * 9)(*v)
            else:
                setattr(t, k, int(v))
        return t


class sft_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("variant", sft_variant), ("tune", sft_tuning),
                ("build_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sft_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("plan_reused", ctypes.c_int32),
                ("queued_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double)]


class sft_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("plans_built", ctypes.c_int64), ("plans_reused", ctypes.c_int64),
                ("plans_evicted", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
                ("arena_peak", ctypes.c_size_t), ("resident_plans", ctypes.c_int32),
                ("max_batch_seen", ctypes.c_int32), ("build_ms_total", ctypes.c_double)]


_lib = None

EXPORTS = {
    "sft_variant_init": (ctypes.c_int, [ctypes.POINTER(sft_variant)]),
    "sft_variant_theorem": (ctypes.c_int, [ctypes.POINTER(sft_variant), ctypes.c_int64,
                                           ctypes.c_double]),
    "sft_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int32,
                                ctypes.POINTER(sft_variant), ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "sft_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sft_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sft_plan_device_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "sft_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sft_plan_desc)]),
    "sft_plan_debug_buffer": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "sft_last_error": (ctypes.c_char_p, []),
    "sft_plan_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "sft_plan_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "sft_plan_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "sft_plan_launches": (ctypes.c_int64, [ctypes.c_void_p]),
    "sft_residual_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sft_dft_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "sft_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]),
    "sft_batch_execute": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_void_p)] * 4
                          + [ctypes.c_void_p]),
    "sft_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sft_execute_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)] * 5
                          + [ctypes.c_int32, ctypes.c_void_p]),
    "sft_batch_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "sft_batch_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int32)]),
    "sft_batch_launches": (ctypes.c_int64, [ctypes.c_void_p]),
    "sft_tuning_default": (None, [ctypes.POINTER(sft_tuning)]),
    "sft_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sft_tuning)]),
    "sft_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sft_tuning)]),
    "sft_batch_autotune": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_void_p)] * 4
                           + [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(sft_tuning)]),
    "sft_batch_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "sft_server_config_init": (None, [ctypes.POINTER(sft_server_config)]),
    "sft_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(sft_server_config)]),
    "sft_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "sft_server_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.POINTER(sft_request_info)]),
    "sft_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "sft_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "sft_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "sft_server_stats_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(sft_server_stats)]),
    "sft_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "sft_batch_device_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "sft_choose_moduli_deterministic": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                                       ctypes.POINTER(ctypes.c_int64),
                                                       ctypes.POINTER(ctypes.c_int32),
                                                       ctypes.POINTER(ctypes.c_int32),
                                                       ctypes.POINTER(ctypes.c_int32)]),
    "sft_choose_moduli": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]),
    "sft_choose_moduli_pool": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32)]),
    "sft_checked_build": (ctypes.c_int32, []),
    "sft_plan_faults": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "sft_plan_debug_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "sft_debug_fail_allocations": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "sft_tuning_table_put": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.POINTER(sft_tuning)]),
    "sft_tuning_table_get": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.POINTER(sft_tuning)]),
    "sft_tuning_table_save": (ctypes.c_int, [ctypes.c_char_p]),
    "sft_tuning_table_load": (ctypes.c_int, [ctypes.c_char_p]),
    "sft_tuning_table_size": (ctypes.c_int32, []),
    "sft_tuning_table_clear": (None, []),
}


def lib_path() -> str:
    return _build.LIB


_loaded = {}


def _open(path: str):
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built ({path}); "
                           "run paper_1706_02740_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _loaded[path] = lib
    return lib


def load(path: str | None = None):
    """Load libsft.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    _lib = _loaded.get(path) or _open(path)
    return _lib


def use_checked(enable: bool = True):
    """Send every later call of this module to the checked build, libsft_checked.so (every
    gather, bin and candidate index range-checked; faults recorded in the plan's status words, see
    sft_plan_faults), or with enable=False back to libsft.so.  Plans, batches and servers belong
    to the library that made them: destroy them before switching."""
    global _lib
    path = _build.LIB_CHECKED if enable else lib_path()
    _lib = _loaded.get(path) or _open(path)
    return _lib


def _check(status: int):
    if status != SFT_OK:
        raise SftError(status, sft_last_error())


def sft_last_error() -> str:
    return load().sft_last_error().decode()


def checked_build() -> bool:
    """True when calls go to the checked build."""
    return bool(load().sft_checked_build())


def sft_plan_faults(plan: "Plan", stream: int = 0):
    """(fault bits, site of the first index fault) of the plan's last execution; waits for
    `stream`."""
    f, st = ctypes.c_int32(), ctypes.c_int32()
    _check(load().sft_plan_faults(plan.handle, stream, ctypes.byref(f), ctypes.byref(st)))
    return f.value, st.value


def sft_plan_debug_limit(plan: "Plan", which: int, value: int):
    _check(load().sft_plan_debug_limit(plan.handle, which, value))


def sft_debug_fail_allocations(skip: int, fail: int):
    _check(load().sft_debug_fail_allocations(skip, fail))


def sft_variant_init(**overrides) -> sft_variant:
    v = sft_variant()
    _check(load().sft_variant_init(ctypes.byref(v)))
    for k, val in overrides.items():
        if not hasattr(v, k):
            raise TypeError(f"unknown variant field {k}")
        setattr(v, k, val)
    return v


def sft_variant_theorem(N: int, r: float, v: sft_variant | None = None, **overrides) -> sft_variant:
    """A variant with the theorem parameters for error order N^-r (beta, kappa, alpha set)."""
    v = v if v is not None else sft_variant_init(**overrides)
    _check(load().sft_variant_theorem(ctypes.byref(v), int(N), float(r)))
    return v


class Plan:
    """Owns an sft_plan_t; destroy() (or garbage collection) releases it."""

    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self):
        if self.handle:
            load().sft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return int(load().sft_plan_device_bytes(self.handle))

    def info(self) -> dict:
        return sft_plan_info(self)


def sft_plan(N: int, s: int, variant: sft_variant | None = None, n_shifts: int = 0,
             primes=None, small_moduli=None) -> Plan:
    lib = load()
    v = variant if variant is not None else sft_variant_init()
    h = ctypes.c_void_p()
    pp, np_ = None, 0
    if primes is not None:
        pp = (ctypes.c_int64 * len(primes))(*[int(p) for p in primes])
        np_ = len(primes)
    sp, ns = None, 0
    if small_moduli is not None:
        sp = (ctypes.c_int32 * max(1, len(small_moduli)))(*[int(t) for t in small_moduli])
        ns = len(small_moduli)
    _check(lib.sft_plan(ctypes.byref(h), int(N), int(s), ctypes.byref(v), int(n_shifts),
                        pp, np_, sp, ns))
    return Plan(h.value)


def sft_execute(plan: Plan, f_dev: int, out_freqs_dev: int, out_coefs_dev: int,
                out_count_dev: int, stream: int = 0):
    _check(load().sft_execute(plan.handle, f_dev, out_freqs_dev, out_coefs_dev, out_count_dev,
                              stream))


def sft_choose_moduli(N: int, s: int, K: int = 5, c_p: float = 3.0, seed: int = 0):
    """Host-only: the (primes, small moduli) sft_plan would choose."""
    pr = (ctypes.c_int64 * K)()
    sm = (ctypes.c_int32 * SFT_MAX_SMALL)()
    ns = ctypes.c_int32()
    _check(load().sft_choose_moduli(int(N), int(s), int(K), float(c_p), int(seed) & (2**64 - 1),
                                    pr, sm, ctypes.byref(ns)))
    return list(pr), list(sm[: ns.value])


def sft_choose_moduli_pool(N: int, s: int, K: int = 5, c_p: float = 3.0, seed: int = 0,
                           pool: int = SFT_POOL_ALL):
    """Host-only: the (primes, small moduli) sft_plan would choose from the given prime pool."""
    pr = (ctypes.c_int64 * K)()
    sm = (ctypes.c_int32 * SFT_MAX_SMALL)()
    ns = ctypes.c_int32()
    _check(load().sft_choose_moduli_pool(int(N), int(s), int(K), float(c_p),
                                         int(seed) & (2**64 - 1), int(pool), pr, sm,
                                         ctypes.byref(ns)))
    return list(pr), list(sm[: ns.value])


def sft_choose_moduli_deterministic(N: int, s: int, c_p: float = 3.0):
    """Host-only: the (primes, small moduli) of the deterministic inner SFT."""
    pr = (ctypes.c_int64 * SFT_MAX_K)()
    k = ctypes.c_int32()
    sm = (ctypes.c_int32 * SFT_MAX_SMALL)()
    ns = ctypes.c_int32()
    _check(load().sft_choose_moduli_deterministic(int(N), int(s), float(c_p), pr, ctypes.byref(k),
                                                  sm, ctypes.byref(ns)))
    return list(pr[: k.value]), list(sm[: ns.value])


def sft_plan_info(plan: Plan) -> dict:
    d = sft_plan_desc()
    _check(load().sft_plan_info(plan.handle, ctypes.byref(d)))
    return {
        "N": d.N, "s": d.s, "kappa": d.kappa, "K": d.K, "n_small": d.n_small,
        "n_shifts": d.n_shifts, "n_sub": d.n_sub, "primes": list(d.primes[: d.K]),
        "small": list(d.small[: d.n_small]), "shifts": list(d.shifts[: d.n_shifts]),
        "L": d.L, "c1": d.c1, "nodes": d.nodes, "fft_size": d.fft_size,
        "precision": d.precision, "input": d.input, "dft": d.dft,
    }


STAGES = ("resample", "chirp_dft", "identify", "vote", "select", "refine")


def sft_plan_graph(plan: Plan, enable: bool = True):
    """Replay the plan's launches as a CUDA graph in later sft_execute calls."""
    _check(load().sft_plan_graph(plan.handle, 1 if enable else 0))


def sft_plan_profile(plan: Plan, enable: bool = True):
    _check(load().sft_plan_profile(plan.handle, 1 if enable else 0))


def sft_plan_profile_read(plan: Plan):
    """Summed per-stage milliseconds since the last read and the number of executions."""
    arr = (ctypes.c_double * len(STAGES))()
    n = ctypes.c_int32()
    _check(load().sft_plan_profile_read(plan.handle, arr, ctypes.byref(n)))
    return dict(zip(STAGES, list(arr))), n.value


def sft_dft_noalloc(n: int, batch: int, in_dev: int, out_dev: int, stream: int = 0):
    """Batched length-n DFT (1/n normalised) of complex64 vectors; allocates no device memory
    (its tables live in a fixed static device array of the library)."""
    _check(load().sft_dft_noalloc(int(n), int(batch), in_dev, out_dev, stream))


class Batch:
    """Owns an sft_batch_t over a list of Plans (kept alive by this object)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        _check(load().sft_batch_create(ctypes.byref(h), arr, len(self.plans)))
        self.handle = h.value

    def destroy(self):
        if self.handle:
            load().sft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def execute(self, f_ptrs, w_ptrs, c_ptrs, n_ptrs, stream: int = 0):
        n = len(self.plans)
        arrs = [(ctypes.c_void_p * n)(*[int(x) for x in ptrs])
                for ptrs in (f_ptrs, w_ptrs, c_ptrs, n_ptrs)]
        _check(load().sft_batch_execute(self.handle, *arrs, stream))

    def _ptr_arrays(self, f_ptrs, w_ptrs, c_ptrs, n_ptrs):
        n = len(self.plans)
        return [(ctypes.c_void_p * n)(*[int(x) for x in ptrs])
                for ptrs in (f_ptrs, w_ptrs, c_ptrs, n_ptrs)]

    def set_tuning(self, tuning: dict):
        t = sft_tuning.from_dict(tuning)
        _check(load().sft_batch_set_tuning(self.handle, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = sft_tuning()
        _check(load().sft_batch_get_tuning(self.handle, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, f_ptrs, w_ptrs, c_ptrs, n_ptrs, stream: int = 0, reps: int = 3) -> dict:
        t = sft_tuning()
        _check(load().sft_batch_autotune(self.handle, *self._ptr_arrays(f_ptrs, w_ptrs, c_ptrs, n_ptrs),
                                         stream, int(reps), ctypes.byref(t)))
        return t.as_dict()

    def graph(self, enable: bool = True):
        _check(load().sft_batch_graph(self.handle, 1 if enable else 0))

    def profile(self, enable: bool = True):
        _check(load().sft_batch_profile(self.handle, 1 if enable else 0))

    def profile_read(self):
        arr = (ctypes.c_double * len(STAGES))()
        n = ctypes.c_int32()
        _check(load().sft_batch_profile_read(self.handle, arr, ctypes.byref(n)))
        return dict(zip(STAGES, list(arr))), n.value

    @property
    def launches(self) -> int:
        return int(load().sft_batch_launches(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(load().sft_batch_device_bytes(self.handle))


def batch_outputs_torch(batch: Batch, device):
    """Device result tensors (freqs, coefs, count) for every plan of a batch."""
    import torch
    outs = []
    for p in batch.plans:
        s = p.info()["s"]
        outs.append((torch.empty(s, dtype=torch.int64, device=device),
                     torch.empty(s, dtype=torch.complex128, device=device),
                     torch.empty(1, dtype=torch.int32, device=device)))
    return outs


def _batch_ptrs(fs, outs):
    return ([f.data_ptr() for f in fs], [o[0].data_ptr() for o in outs],
            [o[1].data_ptr() for o in outs], [o[2].data_ptr() for o in outs])


def sft_execute_batch(plans, f_ptrs, w_ptrs, c_ptrs, n_ptrs, stream: int = 0):
    """One-shot batch over plans, enqueued on `stream` (results valid after it is synchronised)."""
    n = len(plans)
    arrs = [(ctypes.c_void_p * n)(*[int(x) for x in ptrs])
            for ptrs in ([p.handle for p in plans], f_ptrs, w_ptrs, c_ptrs, n_ptrs)]
    _check(load().sft_execute_batch(*arrs, n, stream))


def execute_batch_torch(batch: Batch, fs, stream=None, outs=None):
    """Run a batch on tensors fs (one per plan; CUDA, or pinned host memory); returns lists of
    device result tensors."""
    import torch
    dev = _cuda_device_of(fs[0])
    if outs is None:
        outs = batch_outputs_torch(batch, dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    batch.execute(*_batch_ptrs(fs, outs), st.cuda_stream)
    return outs


def autotune_batch_torch(batch: Batch, fs, reps: int = 3, stream=None) -> dict:
    """Run the autotuner of a batch on CUDA tensors fs; returns the chosen tuning."""
    import torch
    outs = batch_outputs_torch(batch, fs[0].device)
    st = stream if stream is not None else torch.cuda.current_stream(fs[0].device)
    return batch.autotune(*_batch_ptrs(fs, outs), st.cuda_stream, reps)


REQUEST_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


class Server:
    """Owns an sft_server_t (serving loop: memory-budget admission, resident plans, continuous
    batching).  Buffers passed to submit must stay alive until the request has finished."""

    def __init__(self, mem_budget: int = 8 << 30, max_batch: int = 64, max_inflight: int = 2,
                 variant: sft_variant | None = None, tuning: dict | None = None,
                 build_threads: int | None = None):
        cfg = sft_server_config()
        load().sft_server_config_init(ctypes.byref(cfg))
        cfg.mem_budget = int(mem_budget)
        cfg.max_batch = int(max_batch)
        cfg.max_inflight = int(max_inflight)
        if build_threads is not None:
            cfg.build_threads = int(build_threads)
        if variant is not None:
            cfg.variant = variant
        if tuning is not None:
            cfg.tune = sft_tuning.from_dict(tuning)
        h = ctypes.c_void_p()
        _check(load().sft_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self.handle = h.value

    def submit(self, N: int, s: int, f_ptr: int, w_ptr: int, c_ptr: int, n_ptr: int) -> int:
        rid = ctypes.c_int64()
        _check(load().sft_server_submit(self.handle, int(N), int(s), f_ptr, w_ptr, c_ptr, n_ptr,
                                        ctypes.byref(rid)))
        return rid.value

    def query(self, rid: int) -> dict:
        info = sft_request_info()
        _check(load().sft_server_query(self.handle, int(rid), ctypes.byref(info)))
        return {"state": REQUEST_STATES[info.state], "status": info.status,
                "batch_size": info.batch_size, "plan_reused": bool(info.plan_reused),
                "queued_ms": info.queued_ms, "latency_ms": info.latency_ms,
                "build_ms": info.build_ms}

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        """Waits for the request to finish; returns its status (SFT_OK when done, else why it
        failed).  Raises on timeout or an unknown handle."""
        _check(load().sft_server_wait(self.handle, int(rid), int(timeout_ms)))
        return self.query(rid)["status"]

    def poll(self, rid: int) -> tuple[bool, int]:
        """Non-blocking: (finished, status); status is SFT_OK unless the request failed."""
        done = ctypes.c_int32(0)
        st = load().sft_server_poll(self.handle, int(rid), ctypes.byref(done))
        if not done.value:
            _check(st)             # pending (SFT_OK) or an unknown handle (raises)
        return bool(done.value), int(st)

    def release(self, rid: int):
        _check(load().sft_server_release(self.handle, int(rid)))

    def stats(self) -> dict:
        st = sft_server_stats()
        _check(load().sft_server_stats_read(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in sft_server_stats._fields_}

    def destroy(self):
        if self.handle:
            load().sft_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tuning_table_put(N: int, s: int, kappa: int, precision: int, tuning: dict):
    """Store a launch geometry for the shape class of (N, s, kappa, precision)."""
    t = sft_tuning.from_dict(tuning)
    _check(load().sft_tuning_table_put(int(N), int(s), int(kappa), int(precision), ctypes.byref(t)))


def tuning_table_get(N: int, s: int, kappa: int, precision: int):
    """The stored launch geometry of that class, or None."""
    t = sft_tuning()
    st = load().sft_tuning_table_get(int(N), int(s), int(kappa), int(precision), ctypes.byref(t))
    return t.as_dict() if st == SFT_OK else None


def tuning_table_save(path: str):
    _check(load().sft_tuning_table_save(os.fsencode(path)))


def tuning_table_load(path: str):
    _check(load().sft_tuning_table_load(os.fsencode(path)))


def tuning_table_size() -> int:
    return int(load().sft_tuning_table_size())


def tuning_table_clear():
    load().sft_tuning_table_clear()


def sft_tuning_default() -> dict:
    t = sft_tuning()
    load().sft_tuning_default(ctypes.byref(t))
    return t.as_dict()


def residual_energy_torch(plan: Plan, f, coefs, count, stream=None) -> float:
    """sft_residual_energy on CUDA tensors (the input and outputs of one execution); returns rho."""
    import torch
    out = torch.empty(1, dtype=torch.float64, device=f.device)
    st = stream if stream is not None else torch.cuda.current_stream(f.device)
    _check(load().sft_residual_energy(plan.handle, f.data_ptr(), coefs.data_ptr(), count.data_ptr(),
                                      out.data_ptr(), st.cuda_stream))
    return float(out.item())


def sft_plan_launches(plan: Plan) -> int:
    return int(load().sft_plan_launches(plan.handle))


def sft_plan_debug_buffer(plan: Plan, which: int):
    ptr = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    _check(load().sft_plan_debug_buffer(plan.handle, int(which), ctypes.byref(ptr),
                                        ctypes.byref(nbytes)))
    return ptr.value, nbytes.value


# ---------------------------------------------------------------------------------------------
# torch conveniences (allocation of outputs, pointers, current stream)
# ---------------------------------------------------------------------------------------------
def _cuda_device_of(f):
    """The CUDA device a transform of tensor f runs on: f's own, or the current one when f is a
    page-locked host tensor (which the device then reads over the host link)."""
    import torch
    if f.is_cuda:
        return f.device
    if not f.is_pinned():
        raise SftError("a host input must be page-locked (pinned) memory")
    return torch.device("cuda", torch.cuda.current_device())


def execute_torch(plan: Plan, f, stream=None):
    """Run sft_execute on a tensor f (complex64 or complex128; CUDA, or pinned host memory);
    returns device tensors (freqs int64 [s], coefs complex128 [s], count int32 [1]) on the same
    stream."""
    import torch
    info = sft_plan_info(plan)
    s = info["s"]
    dev = _cuda_device_of(f)
    freqs = torch.empty(s, dtype=torch.int64, device=dev)
    coefs = torch.empty(s, dtype=torch.complex128, device=dev)
    count = torch.empty(1, dtype=torch.int32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    sft_execute(plan, f.data_ptr(), freqs.data_ptr(), coefs.data_ptr(), count.data_ptr(),
                st.cuda_stream)
    return freqs, coefs, count


class _DevArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def debug_tensor(plan: Plan, which: int, dtype, shape):
    """Zero-copy torch view of one of the plan's intermediate device buffers."""
    import torch
    ptr, nbytes = sft_plan_debug_buffer(plan, which)
    typestr = {torch.complex64: "<c8", torch.complex128: "<c16", torch.int64: "<i8",
               torch.uint8: "|u1", torch.int32: "<i4"}[dtype]
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")
