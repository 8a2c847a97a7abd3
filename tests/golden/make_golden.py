"""Writes the oracle's regression fixtures.  Calls only oracle/ and the seeded input generator.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.dsft import dsft, make_plan          # noqa: E402
from synth.signals import config_signal          # noqa: E402

CASES = [  # (name, config, trial, kappa, K, c_p)
    ("c1_trial0_k6", 1, 0, 6, 5, 4.0),
    ("c1_trial1_k4", 1, 1, 4, 5, 4.0),
]


def main():
    out = {}
    for name, cfg, trial, kappa, K, c_p in CASES:
        sig = config_signal(cfg, trial)
        plan = make_plan(sig.N, len(sig.omega), kappa=kappa, K=K, c_p=c_p, seed=trial)
        res = dsft(sig.f, plan)
        out[name] = {
            "config": cfg, "trial": trial, "kappa": kappa, "K": K, "c_p": c_p,
            "N": sig.N, "s": len(sig.omega), "primes": plan.primes, "small": plan.small,
            "shifts": plan.shifts, "L": plan.L,
            "freqs": [int(w) for w in res.freqs],
            "coefs_re": [float(c.real) for c in res.coefs],
            "coefs_im": [float(c.imag) for c in res.coefs],
        }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c1.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
