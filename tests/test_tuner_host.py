"""The batch-size tuner's table on disk (cggm_tuner_save / cggm_tuner_load; host code of
the library, no GPU): a loaded class answers cggm_tuned_batch, a save writes what was
loaded, and a malformed file is rejected whole."""
import math

import pytest

import paper_1509_04681_gb300 as cg


def cls(q, m):
    return math.ceil(math.log2(q)), math.ceil(math.log2(m))


def test_load_then_query(tmp_path):
    lq, lm = cls(5000, 10_000_000)
    f = tmp_path / "tuned.txt"
    f.write_text(f"# a comment\n\n1 {lq} {lm} 512\n0 {lq} {lm} 64\n")
    assert cg.tuner_load(f) == 2
    assert cg.tuned_batch(5000, 10_000_000, cg.CGGM_MIXED) == 512
    assert cg.tuned_batch(4097, 8_388_609, cg.CGGM_MIXED) == 512     # same class (rounded up)
    assert cg.tuned_batch(5000, 10_000_000, cg.CGGM_FP64) == 64
    assert cg.tuned_batch(5000, 100, cg.CGGM_MIXED) == 0              # another class


def test_save_and_reload(tmp_path):
    f = tmp_path / "in.txt"
    f.write_text("1 7 20 128\n")
    cg.tuner_load(f)
    out = tmp_path / "out.txt"
    n = cg.tuner_save(out)
    lines = [l for l in out.read_text().splitlines() if l and not l.startswith("#")]
    assert len(lines) == n and "1 7 20 128" in lines
    assert cg.tuner_load(out) == n


@pytest.mark.parametrize("body", ["1 7 21\n", "1 7 21 128 9\n", "2 7 21 128\n",
                                  "0 7 21 256\n", "1 7 21 100\n", "1 -1 21 128\n", "x y z w\n"])
def test_malformed_files_merge_nothing(tmp_path, body):
    f = tmp_path / "bad.txt"
    f.write_text("1 9 30 256\n" + body)                  # a good line before the bad one
    with pytest.raises(cg.CGGMError):
        cg.tuner_load(f)
    assert cg.tuned_batch(2 ** 9, 2 ** 30, cg.CGGM_MIXED) == 0


def test_missing_file(tmp_path):
    with pytest.raises(cg.CGGMError):
        cg.tuner_load(tmp_path / "nowhere.txt")
    with pytest.raises(cg.CGGMError):
        cg.tuner_save(tmp_path / "no_dir" / "t.txt")
