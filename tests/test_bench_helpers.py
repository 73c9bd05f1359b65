"""Host logic of the benchmark that decides whether a line is accepted: the
clock record (median SM clock under load, throttle reasons seen active) and
the DRAM record's source check."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2002, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = bench.ClockSampler.summarize(lines)
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2002.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.summarize([
        "0, 1500, 2070, 1200, 0x48, Active, Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize([]) is None


def test_dram_record_is_used_only_for_the_sources_it_was_taken_from(tmp_path, monkeypatch):
    # the DRAM bytes of profiles/traffic.json go into the bench line only while
    # the record's hash equals that of the loop kernel's sources; a stale
    # record gives null
    import hashlib
    h = hashlib.sha256()
    for f in bench.TC_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"source_sha256_16": h.hexdigest()[:16],
                               "dram_bytes_per_launch": 1234}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench._traffic_for_current_kernel() == 1234
    rec.write_text(json.dumps({"source_sha256_16": "0" * 16, "dram_bytes_per_launch": 1234}))
    assert bench._traffic_for_current_kernel() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench._traffic_for_current_kernel() is None


def test_every_workload_definition_builds_valid_parameters():
    import paper_2203_08361_gb300 as hsb
    need = {"name", "kind", "R", "sb_steps", "form", "prec", "c1", "dt", "gamma",
            "eval_every", "trace_every", "peak", "dtype"}
    for key, w in bench.OTHER.items():
        assert need <= set(w), key
        assert w["peak"] in ("fp8", "fp4", "bf16") and w["kind"] in ("single", "batch")
        p = hsb.params(w["form"], w["prec"], c1=w["c1"], dt=w["dt"], gamma=w["gamma"],
                       eval_every=w["eval_every"], trace_every=w["trace_every"],
                       **w.get("nh", {}))
        assert p.form == hsb.FORM[w["form"]] and p.prec == hsb.PREC[w["prec"]]
        if "nh" in w:
            assert p.thermostat == hsb.HSB_HEAT_NOSE_HOOVER and p.nh_M > 0
    # the headline workload is the one named by the metric
    assert bench.WORKLOAD["N"] == 2000 and bench.WORKLOAD["R"] == 1024
    assert bench.WORKLOAD["sb_steps"] == 2000 and bench.WORKLOAD["prec"] == "fp8"
