"""Host logic of the benchmark that needs no GPU: roofline.traffic comes from the committed
ncu summary of the dominant kernel, scaled by coordinates, and only while the kernel sources
still hash to the version that was captured."""
import os
import shutil

import bench


def _tree_with_fresh_capture(tmp_path, monkeypatch):
    """A copy of the kernel sources and of the committed Lambda-pass summary whose recorded
    source hash is set to the copy's: the host logic is checked on a capture that is
    current by construction (the committed one goes stale whenever the kernel changes)."""
    import hashlib
    root = tmp_path / "tree"
    for rel in bench.SWEEP_SOURCES + ["profiles/lambda_sweep_kernel-q5000-bounded.md"]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    h = hashlib.sha256()
    for rel in bench.SWEEP_SOURCES:
        h.update((root / rel).read_bytes())
    prof = root / "profiles/lambda_sweep_kernel-q5000-bounded.md"
    lines = [("    source_sha256: " + h.hexdigest()) if l.strip().startswith("source_sha256:")
             else l for l in prof.read_text().splitlines()]
    prof.write_text("\n".join(lines) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    return root


def test_traffic_scales_with_coordinates(tmp_path, monkeypatch):
    _tree_with_fresh_capture(tmp_path, monkeypatch)
    t1 = bench.profiled_traffic("lambda_sweep_kernel", 1_000_000)
    t2 = bench.profiled_traffic("lambda_sweep_kernel", 2_000_000)
    assert t1 is not None and t1 > 0
    assert abs(t2 - 2 * t1) <= 1e-9 * t2
    # the committed capture: between 10 and 200 KB of DRAM traffic per coordinate
    assert 10e3 < t1 / 1e6 < 200e3


def test_traffic_is_null_for_other_kernels_and_changed_sources(tmp_path, monkeypatch):
    root = _tree_with_fresh_capture(tmp_path, monkeypatch)
    assert bench.profiled_traffic("theta_sweep_kernel", 1000) is None  # no capture there
    assert bench.profiled_traffic("lambda_sweep_kernel", 1000) is not None
    # a kernel source that differs by one byte: the capture no longer applies
    src = root / bench.SWEEP_SOURCES[0]
    src.write_bytes(src.read_bytes() + b" ")
    assert bench.profiled_traffic("lambda_sweep_kernel", 1000) is None


def test_pass_cost_counts_the_fixed_part_once():
    """A pass costing 0.3 s fixed plus 1 us per coordinate, sampled on a prefix, is
    extrapolated to 0.3 + 1e-6 m, not scaled as a whole."""
    import time as _t
    calls = []

    def run(k):
        calls.append(k)
        _t.sleep(0.3 + 1e-6 * k)

    m = 10_000_000
    t_full, t0, k, tk = bench.pass_cost(run, m, budget_s=3.0, k0=65536)
    assert calls[0] == 0 and 0.29 <= t0 <= 0.45
    assert abs(t_full - (0.3 + 1e-6 * m)) <= 0.25 * (0.3 + 1e-6 * m)


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """--impl reference times the oracle on the host cores and prints one JSON line with
    the contract's keys; run here on the small chain workload to stay quick."""
    import json
    import types
    monkeypatch.setattr(bench, "WORKLOAD", "chain-gauss-p200-q100-n100")
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=1)
    bench.run_reference(args)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-9 * d["ms_per_step"]
    c = d["config"]
    assert (c["workload"], c["p"], c["q"], c["n"]) == ("chain-gauss-p200-q100-n100", 200, 100, 100)


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    import types
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(types.SimpleNamespace(steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""


def test_clock_summary_parses_nvidia_smi_lines(tmp_path):
    """The clock record of the timed region: median SM clock, the maximum, and every
    throttle reason seen active; malformed lines are skipped; the file is removed."""
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2050, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
        f.write("0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s == {"sm_mhz": 2050.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    assert not os.path.exists(c.path)


def test_clock_summary_without_samples(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "empty.csv")
    open(c.path, "w").close()
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
