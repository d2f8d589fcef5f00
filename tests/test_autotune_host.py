"""The autotuner's table on the host (no device): a table written by hand loads, saves back to the
same entries and reports its size; a malformed file is rejected and leaves the table as it was;
clear empties it. The table maps (kernel, double-float products, ceil(log2 nmax), ceil(log2 boxes))
to the split of the panel (kernel 0) or Schur (kernel 1) launches."""
import pytest

from paper_1407_1572_gb300 import ifmm

TABLE = """# hand-written table
0 1 7 11 2
1 1 7 11 4
1 0 6 4 16

1 1 8 2 1
"""


def _entries(text):
    return sorted(tuple(int(v) for v in l.split()) for l in text.splitlines() if l.strip() and not l.startswith("#"))


def test_table_round_trip_and_rejection(tmp_path):
    lib = ifmm.load()
    src, out = tmp_path / "t.txt", tmp_path / "out.txt"
    src.write_text(TABLE)
    try:
        ifmm.ifmm_autotune_load(str(src))
        assert ifmm.ifmm_autotune_size() == 4
        ifmm.ifmm_autotune_save(str(out))
        assert _entries(out.read_text()) == _entries(TABLE)
        for bad in ["0 1 7 11\n", "2 1 7 11 2\n", "0 2 7 11 2\n", "0 1 7 11 0\n", "0 1 7 11 65\n", "0 1 31 1 2\n",
                    "0 1 7 11 2 9\n", "x y z\n"]:
            (tmp_path / "bad.txt").write_text("0 0 1 1 1\n" + bad)
            assert lib.ifmm_autotune_load(str(tmp_path / "bad.txt").encode()) == ifmm.IFMM_ERR_INVALID_ARG, bad
            assert ifmm.ifmm_autotune_size() == 4
        assert lib.ifmm_autotune_load(str(tmp_path / "missing.txt").encode()) == ifmm.IFMM_ERR_INVALID_ARG
        assert lib.ifmm_autotune_load(None) == ifmm.IFMM_ERR_INVALID_ARG
        assert lib.ifmm_autotune(None, 1, 0) == ifmm.IFMM_ERR_INVALID_ARG
    finally:
        ifmm.ifmm_autotune_clear()
    assert ifmm.ifmm_autotune_size() == 0
