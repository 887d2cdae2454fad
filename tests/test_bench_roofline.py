"""The benchmark's roofline inputs: the host count of ao_vgl's algorithmic
work (Eq. 3 screening) equals the oracle's own count exactly, and the
roofline entries follow from the counts, the times and the peaks."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("which, walk_num, npts", [(1, None, None), (2, 1, 400), (5, 1, 150)])
def test_screen_work_matches_oracle(orc, cfg, which, walk_num, npts):
    m = cfg(which, walk_num=walk_num)
    pts = m.points if npts is None else m.points[:npts]
    assert bench.screen_work(m, pts, block=97) == orc.screen_counts(m, points=pts)


def test_alu_entry_and_bound():
    class Mol:
        point_num, ao_num, mo_num = 1000, 100, 10
    peaks = {"hbm_gbs": 1000.0, "bf16_tflops": 100.0, "sm_max_mhz": 2000.0}
    fp32, mufu = bench.alu_peaks(peaks)
    assert fp32 == pytest.approx(152 * 128 * 2 * 2e9 / 1e12)
    assert mufu == pytest.approx(152 * 16 * 2e9 / 1e12)
    work = (300, 2000, 900)
    sparsity = (10, 5000)                     # live groups, nnz
    stats = (5, 40, 0)
    r = bench.roofline("bf16x3", Mol, [1.0, 1.0], peaks, stats, sparsity, work)["ao_vgl"]
    alu = r["alu"]
    assert alu["fp32_flops"] == 10 * 2000 + 14 * 900
    assert alu["mufu_ops"] == 2000
    t = 1e-3
    assert alu["fp32"]["frac"] == pytest.approx(alu["fp32_flops"] / (fp32 * 1e12) / t)
    assert alu["mufu"]["frac"] == pytest.approx(2000 / (mufu * 1e12) / t)
    # 5 * nnz * 4 bytes over 1000 GB/s: a longer floor than the ALU's here
    assert r["bound"] == "hbm"
    assert r["frac"] == pytest.approx(5 * 5000 * 4 / 1e12 / t)
    # make the arithmetic the longer floor: exps, then Cartesian assembly
    r = bench.roofline("bf16x3", Mol, [1.0, 1.0], peaks, stats, (10, 1), (1, 10**9, 1))["ao_vgl"]
    assert r["bound"] == "alu"
    assert r["unit"] == "Tops/s" and r["frac"] == r["alu"]["mufu"]["frac"]
    r = bench.roofline("bf16x3", Mol, [1.0, 1.0], peaks, stats, (10, 1), (1, 1, 10**9))["ao_vgl"]
    assert r["bound"] == "alu"
    assert r["unit"] == "TFLOP/s" and r["frac"] == r["alu"]["fp32"]["frac"]
    # no ALU entry for the FP64 path
    r = bench.roofline("fp64", Mol, [1.0, 1.0], peaks, None, None, work)["ao_vgl"]
    assert "alu" not in r and r["bound"] == "hbm"


def test_traffic_only_while_sources_match(tmp_path, monkeypatch):
    """A kernel's ncu traffic is reported only while its source files hash
    to what was captured; any edit turns it into null."""
    import hashlib
    import json
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"k:bf16x3": {"bytes_per_launch": 1234, "source": ["k.cu"], "source_sha": sha}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k", "bf16x3") == 1234
    assert bench.traffic_for("k", "tf32") is None
    src.write_text("kernel v2\n")
    assert bench.traffic_for("k", "bf16x3") is None


def test_accuracy_and_common_bar(orc, cfg, monkeypatch):
    """The per-path accuracy entry compares each path's first rows with the
    oracle, and the speedup is stated at a bar both paths meet."""
    m = cfg(1)
    monkeypatch.setattr(bench, "CPU_SAMPLE_POINTS", 40)
    ref, size = orc.mo_vgl(m, points=m.points[:40])
    rng = np.random.default_rng(0)
    samples = {"bf16x3": (ref + 1e-6 * size * rng.uniform(-1, 1, ref.shape)).reshape(-1),
               "fp32": (ref + 1e-7 * size * rng.uniform(-1, 1, ref.shape)).reshape(-1)}
    acc = bench.accuracy(m, samples, "bf16x3")
    assert 5e-7 < acc["bf16x3"]["value"] <= 1e-6 and acc["fp32"]["value"] <= 1e-7
    assert acc["bf16x3"]["stated_bar"] == 5e-5 and acc["fp32"]["stated_bar"] == 3e-5
    res = {"accuracy": acc, "fp32_path": {"ms_per_step": 30.0}, "ms_per_step": 1.0}
    cb = bench.common_bar(res, "bf16x3")
    assert cb["bar"] == 5e-5 and cb["both_meet"] and cb["speedup"] == 30.0


def test_batch_roofline_sums_molecules():
    """The batch contraction's roofline entry: flops and bytes are the sums
    of each molecule's sparse count and its bytes, the fractions are those
    over the launch time, and the bound is the longer floor."""
    from types import SimpleNamespace
    mols = [SimpleNamespace(mo_num=100, ao_num=400, point_num=1000),
            SimpleNamespace(mo_num=50, ao_num=200, point_num=3000)]
    nnz = [20000, 90000]
    peaks = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1600.0}
    r = bench.batch_roofline(mols, nnz, 0.5, peaks)
    fl = 2 * 5 * (100 * 20000 + 50 * 90000)
    by = (20 * 20000 + 4 * 100 * 400 + 20 * 1000 * 100) + (20 * 90000 + 4 * 50 * 200 + 20 * 3000 * 50)
    assert r["algorithmic_flops"] == pytest.approx(fl)
    assert r["algorithmic_bytes"] == pytest.approx(by)
    assert r["hbm"]["frac"] == pytest.approx(by / 8e12 / 5e-4)
    assert r["tensor"]["frac"] == pytest.approx(fl / 1.6e15 / 5e-4)
    assert r["bound"] == ("hbm" if by / 8e12 >= fl / 1.6e15 else "tensor")
    assert r["frac"] == r[r["bound"]]["frac"]
