"""The benchmark's clock record: only nvidia-smi samples taken inside the
timed region count, throttle reasons are collected from them, and a region
shorter than the sampling interval says which sample stands in for it."""
import bench


def _line(mhz, hw="Not Active", cap="Not Active"):
    return f"{mhz}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {cap}"


def _sampler(before, inside):
    c = bench.ClockSampler(0)
    c.lines = before + inside
    c.first = len(before)
    return c


def test_only_samples_inside_region():
    s = _sampler([_line(1200), _line(1300)], [_line(2070), _line(2060), _line(2070)]).summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070
    assert s["sm_max_mhz"] == 2070
    assert s["reasons"] == []
    assert "note" not in s


def test_reasons_from_inside_samples():
    s = _sampler([_line(2070, hw="Active")], [_line(1900, cap="Active")]).summary()
    assert s["reasons"] == ["sw_power_cap"]


def test_short_region_uses_last_sample_before():
    s = _sampler([_line(1500), _line(2070)], []).summary()
    assert s["samples"] == 0
    assert s["sm_mhz"] == 2070
    assert "note" in s


def test_no_sampler():
    s = _sampler([], []).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["no samples"]
