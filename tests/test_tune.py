"""Host-side logic of the launch-shape tuning table (tt_tune_* in the C ABI):
key validation, entry validation, the text format, and the committed table.
No GPU needed: the calls touch no device state."""
import os

import pytest

tt = pytest.importorskip("paper_2308_01480_gb300")
N = tt._native


@pytest.fixture()
def lib():
    L = N.lib()
    yield L
    # leave the process with the committed table, as the library loads it
    if os.path.exists(N.TUNE_TABLE):
        tt.tune_load(N.TUNE_TABLE)
    else:
        tt.tune_clear()


def test_key_bucketing():
    assert tt.tune_key(N.TT_PASS_GRAM, 40, 2560000) == (3, 48, 48, 2)
    assert tt.tune_key(N.TT_PASS_GRAM, 1, 100) == (3, 16, 16, 0)
    assert tt.tune_key(N.TT_PASS_PROJECT, 40, 2560000, 20) == (2, 48, 64, 2)    # hi + lo split: N = 64
    assert tt.tune_key(N.TT_PASS_PROJECT, 800, 64000, 40) == (2, 1024, 48, 1)
    assert tt.tune_key(N.TT_PASS_PROJECT, 800, 1600, 20) == (2, 1024, 64, 0)
    assert tt.tune_key(N.TT_PASS_SKETCH, 129, 262144, 30) == (0, 256, 32, 2)
    assert tt.tune_key(N.TT_PASS_GRAMAPPLY, 7680, 100, 64) == (1, 4096, 64, 0)
    assert tt.tune_key(N.TT_PASS_SKETCH, 512, 16384, 1) == (0, 512, 16, 1)


def test_set_get_clear(lib):
    tt.tune_clear()
    assert tt.tune_entries() == 0
    k = (N.TT_PASS_GRAM, 48, 48, 1)
    assert tt.tune_get(k) is None
    tt.tune_set(k, 4, 1, kb=4)
    assert tt.tune_get(k) == (4, 1, 4, 0)
    tt.tune_set(k, 6, 2, kb=2)                      # replaces
    assert tt.tune_get(k) == (6, 2, 2, 0) and tt.tune_entries() == 1
    tt.tune_set((N.TT_PASS_PROJECT, 1024, 64, 1), 3, 2, chunk_rows=128)
    assert tt.tune_entries() == 2
    tt.tune_clear()
    assert tt.tune_entries() == 0


@pytest.mark.parametrize("key,entry", [
    ((4, 48, 48, 1), (4, 1, 0, 0)),                  # no such pass
    ((3, 256, 64, 1), (4, 1, 2, 0)),                 # the Gram has no tall rows
    ((3, 40, 48, 1), (4, 1, 2, 0)),                  # rows not a multiple of 16
    ((0, 300, 32, 1), (4, 1, 0, 0)),                 # not a row bucket
    ((0, 256, 20, 1), (4, 1, 0, 0)),                 # npad not a multiple of 16
    ((0, 256, 32, 3), (4, 1, 0, 0)),                 # n class
    ((0, 256, 32, 1), (1, 1, 0, 0)),                 # one stage
    ((0, 256, 32, 1), (9, 1, 0, 0)),                 # nine stages
    ((0, 256, 32, 1), (4, 3, 0, 0)),                 # three CTAs per SM
    ((0, 256, 32, 1), (4, 1, 2, 0)),                 # kb outside the Gram
    ((3, 48, 48, 1), (4, 1, 3, 0)),                  # kb not a power of two
    ((3, 48, 48, 1), (4, 1, 0, 0)),                  # the Gram needs kb
    ((2, 256, 64, 1), (4, 1, 0, 96)),                # chunk rows
    ((1, 256, 64, 1), (4, 1, 0, 64)),                # chunk rows outside the projection
])
def test_invalid_rejected(lib, key, entry):
    tt.tune_clear()
    assert lib.tt_tune_set(*key, *entry) == N.TT_EINVAL
    assert tt.tune_entries() == 0


def test_load_format(lib, tmp_path):
    p = tmp_path / "t.txt"
    p.write_text("# comment\n\n3 48 48 1 4 1 4 0   # gram 40 rows\n  2 1024 64 1 3 2 0 128\n")
    tt.tune_load(p)
    assert tt.tune_entries() == 2
    assert tt.tune_get((3, 48, 48, 1)) == (4, 1, 4, 0)
    assert tt.tune_get((2, 1024, 64, 1)) == (3, 2, 0, 128)


@pytest.mark.parametrize("text", ["3 48 48 1 4 1 4\n", "3 48 48 1 4 1 3 0\n", "x 48 48 1 4 1 4 0\n",
                                  "3 48 48 1 4 1 4 0\n0 256 32 1 9 1 0 0\n"])
def test_load_bad_file_leaves_table(lib, tmp_path, text):
    tt.tune_clear()
    tt.tune_set((0, 256, 32, 1), 4, 1)
    p = tmp_path / "bad.txt"
    p.write_text(text)
    assert lib.tt_tune_load(str(p).encode()) == N.TT_EINVAL
    assert tt.tune_entries() == 1 and tt.tune_get((0, 256, 32, 1)) == (4, 1, 0, 0)
    assert lib.tt_tune_load(str(tmp_path / "missing.txt").encode()) == N.TT_EINVAL
    assert tt.tune_entries() == 1


def test_committed_table_loads(lib):
    """The table the library loads parses, and its keys are the sweep's."""
    if not os.path.exists(N.TUNE_TABLE):
        pytest.skip("no committed tuning table")
    tt.tune_load(N.TUNE_TABLE)
    from paper_2308_01480_gb300 import autotune
    sweep_keys = {tt.tune_key(op, m, n, b) for op, m, n, b in autotune.SHAPES}
    n_entries = 0
    for line in open(N.TUNE_TABLE):
        s = line.strip()
        if not s or s.startswith("#"):
            continue
        v = tuple(int(x) for x in s.split()[:8])
        assert v[:4] in sweep_keys
        assert tt.tune_get(v[:4]) == v[4:]
        n_entries += 1
    assert tt.tune_entries() == n_entries
