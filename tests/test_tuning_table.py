"""CPU checks of the table of tuned launch geometries (sft_tuning_table_*): host-only logic, no
device call.  Classes are floor(log2 N), floor(log2 s), kappa, precision; entries are validated
as sft_batch_set_tuning validates a geometry; the text file round-trips; a bad file merges
nothing."""
import os

import pytest

import paper_1706_02740_gb300 as sft
from paper_1706_02740_gb300 import build as sft_build


@pytest.fixture(autouse=True)
def lib():
    sft_build.build()
    lib = sft.load()
    sft.tuning_table_clear()
    yield lib
    sft.tuning_table_clear()


def _tuned():
    t = sft.sft_tuning_default()
    t["bin_threads"] = 128
    t["resample_threads"] = 256
    return t


def test_entries_are_keyed_by_shape_class():
    assert sft.tuning_table_size() == 0
    assert sft.tuning_table_get(2 ** 20, 100, 6, 0) is None
    sft.tuning_table_put(2 ** 20, 100, 6, 0, _tuned())
    assert sft.tuning_table_size() == 1
    # same class: floor(log2 N) = 20, floor(log2 s) = 6
    assert sft.tuning_table_get(2 ** 21 - 1, 127, 6, 0) == _tuned()
    assert sft.tuning_table_get(2 ** 20 + 5, 64, 6, 0) == _tuned()
    # other classes
    for key in [(2 ** 21, 100, 6, 0), (2 ** 20 - 1, 100, 6, 0), (2 ** 20, 128, 6, 0),
                (2 ** 20, 63, 6, 0), (2 ** 20, 100, 4, 0), (2 ** 20, 100, 6, 1)]:
        assert sft.tuning_table_get(*key) is None, key
    sft.tuning_table_put(2 ** 20, 100, 6, 0, sft.sft_tuning_default())     # replaces
    assert sft.tuning_table_size() == 1
    assert sft.tuning_table_get(2 ** 20, 100, 6, 0) == sft.sft_tuning_default()


@pytest.mark.parametrize("field,value", [("bin_threads", 100), ("resample_threads", 32),
                                         ("resample_regcap", 2), ("dft_two_ctas", 3)])
def test_invalid_geometries_are_refused(field, value):
    t = sft.sft_tuning_default()
    t[field] = value
    with pytest.raises(sft.SftError) as e:
        sft.tuning_table_put(2 ** 20, 100, 6, 0, t)
    assert e.value.status == sft.SFT_EINVAL
    assert sft.tuning_table_size() == 0


@pytest.mark.parametrize("key", [(1, 100, 6, 0), (2 ** 20, 0, 6, 0), (2 ** 20, 100, 0, 0),
                                 (2 ** 20, 100, 49, 0), (2 ** 20, 100, 6, 2)])
def test_invalid_keys_are_refused(key):
    with pytest.raises(sft.SftError):
        sft.tuning_table_put(*key, sft.sft_tuning_default())


def test_text_file_round_trip(tmp_path):
    sft.tuning_table_put(2 ** 26, 1000, 6, 0, _tuned())
    sft.tuning_table_put(3 ** 9, 8, 4, 1, sft.sft_tuning_default())
    path = str(tmp_path / "tuning.txt")
    sft.tuning_table_save(path)
    lines = open(path).read().splitlines()
    assert lines[0].startswith("# sft tuning table")
    assert len(lines) == 3 and all(len(ln.split()) == 17 for ln in lines[1:])
    assert not os.path.exists(path + ".tmp")
    sft.tuning_table_clear()
    assert sft.tuning_table_size() == 0
    sft.tuning_table_load(path)
    assert sft.tuning_table_size() == 2
    assert sft.tuning_table_get(2 ** 26, 1000, 6, 0) == _tuned()
    assert sft.tuning_table_get(3 ** 9, 8, 4, 1) == sft.sft_tuning_default()


@pytest.mark.parametrize("body", [
    "# not a tuning table\n",
    "# sft tuning table v1\n20 6 6 0 128 0 256 64 32 16 8 4 2 1 1\n",              # 15 integers
    "# sft tuning table v1\n20 6 6 0 128 0 100 64 32 16 8 4 2 1 1 1 1\n",          # bad bin_threads
    "# sft tuning table v1\n20 6 6 0 128 0 256 64 32 16 8 4 2 1 1 1 1 7\n",        # extra field
    "# sft tuning table v1\n20 6 6 5 128 0 256 64 32 16 8 4 2 1 1 1 1\n",          # bad precision
])
def test_bad_files_merge_nothing(tmp_path, body):
    sft.tuning_table_put(2 ** 26, 1000, 6, 0, _tuned())
    good = "# sft tuning table v1\n10 3 4 0 128 0 256 64 32 16 8 4 2 1 1 1 1\n"
    path = tmp_path / "bad.txt"
    path.write_text(body if body.startswith("# not") else good + body.split("\n", 1)[1])
    with pytest.raises(sft.SftError) as e:
        sft.tuning_table_load(str(path))
    assert e.value.status == sft.SFT_EINVAL
    assert sft.tuning_table_size() == 1
    assert sft.tuning_table_get(2 ** 10, 8, 4, 0) is None
    with pytest.raises(sft.SftError):
        sft.tuning_table_load(str(tmp_path / "missing.txt"))
