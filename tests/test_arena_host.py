"""CPU checks of the serving arena's first-fit bookkeeping (csrc/arena.h), compiled with the host
compiler and driven with random allocate / release sequences.  Checked against properties any
first-fit allocator over one range must have: blocks are 256-byte multiples inside the range and
never overlap live ones; the returned block starts at the lowest gap that fits, and -1 means no
gap fits; `used` is the sum of the live blocks; after every release the free space is coalesced
(a fully free range is one block)."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GRAIN = 256


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_driver")
    subprocess.run([cxx, "-O1", "-std=c++17", os.path.join(HERE, "arena_driver.cpp"), "-o", exe],
                   check=True)
    return exe


def run(exe, cmds):
    out = subprocess.run([exe], input="\n".join(cmds) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    return [tuple(int(x) for x in ln.split()) for ln in out if ln.strip()]


def gaps(live, cap):
    """Free intervals (start, size) between the sorted live blocks."""
    out, pos = [], 0
    for off, n in sorted(live.items()):
        if off > pos:
            out.append((pos, off - pos))
        pos = off + n
    if pos < cap:
        out.append((pos, cap - pos))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_random_sequences_keep_first_fit_invariants(driver, seed):
    rng = random.Random(seed)
    cap = rng.choice([1 << 20, 3 * 1000 * 1000, 64 * GRAIN + 100])
    cmds, model = [f"c {cap}"], []
    live = {}
    # build the command list and the expected first-fit decisions together
    cap_r = cap // GRAIN * GRAIN
    for step in range(400):
        if live and (rng.random() < 0.45):
            off = rng.choice(sorted(live))
            cmds.append(f"f {off}")
            model.append(("f", off, live.pop(off)))
        else:
            want = rng.choice([1, 255, 256, 257, 4096, 50000, 123457, cap_r // 3])
            n = -(-want // GRAIN) * GRAIN
            fit = [g for g in gaps(live, cap_r) if g[1] >= n]
            off = fit[0][0] if fit else -1
            if off >= 0:
                live[off] = n
            cmds.append(f"a {want}")
            model.append(("a", off, n))
    res = run(driver, cmds)
    assert res[0][0] == cap_r
    live = {}
    for (kind, off, n), (r, used, largest, nfree, nlive) in zip(model, res[1:]):
        if kind == "a":
            assert r == off
            if off >= 0:
                live[off] = n
        else:
            assert r == 1
            del live[off]
        g = gaps(live, cap_r)
        assert used == sum(live.values())
        assert largest == max([x[1] for x in g], default=0)
        assert nfree == len(g)          # coalesced: one free block per gap
        assert nlive == len(live)
    # release everything: one free block spanning the range
    cmds = [f"c {cap}"]
    res = run(driver, cmds + [f"a {GRAIN * 3}", f"a {GRAIN}", f"a {GRAIN * 5}", f"f {GRAIN * 3}",
                              "f 0", f"f {GRAIN * 4}"])
    assert res[-1][1:] == (0, cap_r, 1, 0)


def test_release_of_unknown_offsets_is_refused(driver):
    res = run(driver, ["c 65536", "a 1000", "f 256", "f 12345", "f 0", "f 0"])
    assert [r[0] for r in res[1:]] == [0, 0, 0, 1, 0]
    assert res[-1][1:] == (0, 65536, 1, 0)
