"""Regression pin: the oracle reproduces its committed fixtures (written by
tests/golden/make_golden.py from oracle/ alone)."""
import json
import os

import numpy as np

from oracle.dsft import dsft, make_plan
from synth.signals import config_signal

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_c1.json")


def test_oracle_matches_fixtures():
    with open(HERE) as fh:
        cases = json.load(fh)
    for name, c in cases.items():
        sig = config_signal(c["config"], c["trial"])
        plan = make_plan(sig.N, c["s"], kappa=c["kappa"], K=c["K"], c_p=c["c_p"], seed=c["trial"])
        assert plan.primes == c["primes"] and plan.small == c["small"] and plan.shifts == c["shifts"]
        res = dsft(sig.f, plan)
        assert res.freqs.tolist() == c["freqs"], name
        ref = np.array(c["coefs_re"]) + 1j * np.array(c["coefs_im"])
        assert np.max(np.abs(res.coefs - ref)) < 1e-12, name
        # and the support is the true one
        assert sorted(c["freqs"]) == sorted(sig.omega.tolist())
