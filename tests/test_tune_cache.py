"""Launch-shape cache of the autotuner: text round trip through the C ABI
(no GPU needed: the cache is host data)."""
import pytest

from paper_2006_16147_gb300 import amg


def test_save_load_round_trip(tmp_path):
    amg.amg_tune_clear()
    assert amg.amg_tune_size() == 0
    src = tmp_path / "in.txt"
    src.write_text("pre/f64/n100/z500/s4/k1/sm152 152\nblock/f32/n9/z27/s3/k64/sm152 16\n\n")
    amg.amg_tune_load(str(src))
    assert amg.amg_tune_size() == 2
    out = tmp_path / "out.txt"
    amg.amg_tune_save(str(out))
    lines = out.read_text().splitlines()
    assert sorted(lines) == sorted(["pre/f64/n100/z500/s4/k1/sm152 152", "block/f32/n9/z27/s3/k64/sm152 16"])
    # a later file replaces entries with the same key
    upd = tmp_path / "upd.txt"
    upd.write_text("pre/f64/n100/z500/s4/k1/sm152 304\n")
    amg.amg_tune_load(str(upd))
    amg.amg_tune_save(str(out))
    assert "pre/f64/n100/z500/s4/k1/sm152 304" in out.read_text().splitlines()
    assert amg.amg_tune_size() == 2
    amg.amg_tune_clear()
    assert amg.amg_tune_size() == 0


def test_malformed_lines_rejected_after_valid_ones(tmp_path):
    amg.amg_tune_clear()
    f = tmp_path / "bad.txt"
    f.write_text("good/key 8\nno_value\nneg/key -3\ntoo many 1 2\nbig/key 99999999999\nalso/good 32\n")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_tune_load(str(f))
    assert e.value.status == amg.AMG_ERR_ARG
    assert "4 malformed" in str(e.value)
    assert amg.amg_tune_size() == 2
    amg.amg_tune_clear()


def test_missing_file():
    with pytest.raises(amg.AmgError):
        amg.amg_tune_load("/nonexistent/dir/cache.txt")
    with pytest.raises(amg.AmgError):
        amg.amg_tune_save("/nonexistent/dir/cache.txt")
