"""The autotuner's cache file (host logic only, no GPU): entries written by
sl_tuning_save read back by sl_tuning_load with the same values, malformed
files rejected whole, and sl_tuning_clear emptying the cache."""
import pytest

from paper_1606_06117_gb300 import _lib as sl


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1606_06117_gb300 import build
    sl.load(build.build())
    yield
    sl.sl_tuning_clear()


GOOD = """# libsl launch shapes, timed on test
64 64 64 3 0 1 32 32 0 2 0.125
100 36 23 2 0 4 32 8 0 3 1.5
48 40 7 0 0 3 32 16 8 0 0.25
"""


def test_round_trip(tmp_path):
    sl.sl_tuning_clear()
    p = tmp_path / "shapes.txt"
    p.write_text(GOOD)
    sl.sl_tuning_load(str(p))
    t = sl.sl_tuning_get([100, 36, 23], sl.BEC, sl.F32)
    assert (t.kernel, t.tile_x, t.tile_y, t.tile_z, t.ctas_per_sm) == (4, 32, 8, 0, 3)
    assert t.ms == pytest.approx(1.5)
    assert sl.sl_tuning_get([100, 36, 23], sl.FEC, sl.F32) is None   # keyed by scheme
    assert sl.sl_tuning_get([100, 36, 23], sl.BEC, sl.F64) is None   # and by dtype
    q = tmp_path / "again.txt"
    sl.sl_tuning_save(str(q))
    sl.sl_tuning_clear()
    assert sl.sl_tuning_get([64, 64, 64], sl.CEC, sl.F32) is None
    sl.sl_tuning_load(str(q))
    for dims, scheme, want in (([64, 64, 64], sl.CEC, (1, 32, 32, 0, 2)), ([48, 40, 7], sl.CIR, (3, 32, 16, 8, 0))):
        t = sl.sl_tuning_get(dims, scheme, sl.F32)
        assert (t.kernel, t.tile_x, t.tile_y, t.tile_z, t.ctas_per_sm) == want
    lines = [ln for ln in q.read_text().splitlines() if not ln.startswith("#")]
    assert len(lines) == 3


@pytest.mark.parametrize("bad", ["64 64 64 3 0 1 32 32 0 2",            # a field missing
                                 "64 64 64 5 0 1 32 32 0 2 0.1",        # unknown scheme
                                 "64 64 64 3 0 9 32 32 0 2 0.1",        # unknown kernel
                                 "64 64 64 3 0 1 32 12 0 2 0.1",        # tile height not compiled
                                 "64 64 64 3 0 1 32 32 -1 2 0.1",       # negative planes per item
                                 "64 64 64 3 0 1 32 32 0 2 0.1 x",      # trailing text
                                 "0 64 64 3 0 1 32 32 0 2 0.1"])        # empty grid
def test_malformed_file_loads_nothing(tmp_path, bad):
    sl.sl_tuning_clear()
    p = tmp_path / "bad.txt"
    p.write_text("# header\n100 36 23 2 0 4 32 8 0 3 1.5\n" + bad + "\n")
    with pytest.raises(sl.SLError) as e:
        sl.sl_tuning_load(str(p))
    assert e.value.code == -1 and "line 3" in str(e.value)
    assert sl.sl_tuning_get([100, 36, 23], sl.BEC, sl.F32) is None


def test_missing_file_is_an_argument_error(tmp_path):
    with pytest.raises(sl.SLError) as e:
        sl.sl_tuning_load(str(tmp_path / "none.txt"))
    assert e.value.code == -1
