"""Host-side logic of bench.py on the CPU: the algorithmic byte count of the
path, the clock-sample summary behind the bench line's "clocks" object, and
the rule that attaches the committed DRAM traffic only while the kernel
sources are unchanged."""
import json

import bench


def kept_indices(idx):
    """Keep-last coarsening of an index list: every other index from the first,
    plus the last one when it was skipped."""
    out = idx[::2]
    if out[-1] != idx[-1]:
        out = out + [idx[-1]]
    return out


def level_sizes(shape, levels):
    sets = [list(range(n)) for n in shape]
    sizes = []
    for _ in range(levels):
        c = 1
        for s in sets:
            c *= len(s)
        sizes.append(c)
        sets = [kept_indices(s) if len(s) > 1 else s for s in sets]
    return sizes


def test_path_bytes_against_index_sets():
    for shape, levels in [((513, 513, 513), 8), ((1000, 700, 300), 8), ((65, 65, 65), 5), ((33, 20, 37), 4),
                          ((200, 150), 6), ((1025,), 9), ((2, 9, 5), 1)]:
        want = 2.0 * 8 * sum(level_sizes(shape, levels))
        assert bench.path_bytes(shape, levels, 8) == want, shape


def test_path_bytes_dyadic_ratio():
    # sum over levels of (2^k+1)^3 grids is about 8/7 of the finest grid
    n = 513 ** 3
    ratio = bench.path_bytes((513, 513, 513), 8, 1) / 2.0 / n
    assert 1.14 < ratio < 1.145


def sample(sm, mx, power, hw="Not Active", hwt="Not Active", swt="Not Active", swp="Not Active"):
    return [str(sm), str(mx), str(power), hw, hwt, swt, swp]


def test_clock_summary_timed_region():
    s = bench.ClockSampler(0)
    s.samples = [(0.5, sample(1500, 2070, 100))] + [(1.0 + 0.1 * i, sample(2070, 2070, 300 + i)) for i in range(5)]
    out = s.summary(1.0, 2.0)
    assert out["window"] == "timed region" and out["samples"] == 5
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["power_w_max"] == 304.0
    assert out["reasons"] == []


def test_clock_summary_reasons_and_fallback_window():
    s = bench.ClockSampler(0)
    s.samples = [(0.2, sample(1980, 2070, 900, swp="Active")), (0.3, sample(1800, 2070, 950, hwt="Active")),
                 (5.0, sample(2070, 2070, 400))]
    out = s.summary(1.0, 2.0)  # no sample inside the timed region
    assert out["window"].startswith("warm-up + timed region")
    assert out["samples"] == 3
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1980.0


def test_clock_summary_without_samples():
    out = bench.ClockSampler(0).summary(0.0, 1.0)
    assert out["samples"] == 0 and out["sm_mhz"] is None


def test_traffic_only_for_unchanged_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"dram_bytes_per_launch": 123456789, "source_sha1": "abc"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"level_load_dec@513x513x513:f64": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("level_load_dec", "513x513x513:f64", "abc") == 123456789
    assert bench.traffic_for("level_load_dec", "513x513x513:f64", "changed") is None
    assert bench.traffic_for("level_load_rec", "513x513x513:f64", "abc") is None
    (tmp_path / "profiles" / "traffic.json").unlink()
    assert bench.traffic_for("level_load_dec", "513x513x513:f64", "abc") is None


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


def test_reference_arm_does_not_load_the_cuda_library():
    """The reference (CPU oracle) arm imports the input generators by path, so
    neither the package nor libmgr.so enters its process."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys, json; sys.argv = ['bench.py', '--impl', 'reference', '--shape', '17,18,19', "
            "'--steps', '1', '--warmup', '0']; import bench; bench.main(); "
            "maps = open('/proc/self/maps').read(); "
            "assert 'libmgr.so' not in maps, 'libmgr.so mapped'; "
            "assert 'paper_2105_12764_gb300' not in sys.modules, 'package imported'")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["cpu_baseline"]["threads_used"] == 1
    assert line["cpu_baseline"]["host"]["host_cores"] >= 1


def test_batch_sample_covers_extremes_and_both_coordinate_kinds():
    import numpy as np

    synth = bench.synth_module()
    specs = synth.batch_field_specs(4096, seed=0)
    idx = bench.batch_sample(specs)
    assert len(idx) == 64 and len(set(idx)) == 64
    sizes = [int(np.prod(s)) for s, _ in specs]
    assert max(sizes) in [sizes[i] for i in idx]
    assert min(sizes) in [sizes[i] for i in idx]
    assert {len(specs[i][0]) for i in idx} == {2, 3}
    assert {specs[i][1] for i in idx} == {False, True}
    assert idx == bench.batch_sample(specs)  # seeded


def test_rel_linf_is_normwise():
    import numpy as np

    b = np.array([1.0, -4.0, 0.0])
    a = np.array([1.0, -4.0, 1e-3])
    assert bench.rel_linf(a, b) == 1e-3 / 4.0
    assert bench.rel_linf(np.zeros(3), np.zeros(3)) == 0.0
