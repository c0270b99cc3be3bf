"""Host-side parts of the benchmark (no GPU): the lower-bound roofline
variant, the random-access bound, the host description, and the reference
arm's JSON line (the oracle timed on the host)."""
import os

import pytest

import bench
from workloads import keys as wk

PROBE = {"8B": {"gaccess_per_s": 40.0, "requested_gbs": 320.0},
         "32B": {"gaccess_per_s": 40.0, "requested_gbs": 1280.0},
         "128B": {"gaccess_per_s": 40.0, "requested_gbs": 5120.0},
         "rmw_line": {"gaccess_per_s": 25.0, "line_read_gbs": 3200.0}}


@pytest.mark.parametrize("scheme,unit", [("bucket", 128), ("cuckoo", 32)])
def test_lower_bound_roofline_closed_form(scheme, unit):
    fs = wk.fill_stream(40_000, 4096, 0.25, 64, seed=2)
    p = fs.n_distinct / fs.n_issued
    r_unit = 5120.0 if unit == 128 else 1280.0
    per_key_s = unit / (r_unit * 1e9) + p * 32 / 1280e9 + 9 / 6400e9
    ms = per_key_s * fs.n_issued * 1e3 * 2          # a fill taking twice the bound
    got = bench.lower_bound_roofline(scheme, fs, ms, PROBE, 6400.0)
    assert got["bytes_per_key"] == pytest.approx(unit + p * 32 + 9, abs=0.05)
    assert got["frac"] == pytest.approx(0.5, abs=1e-3)
    assert got["mops_bound"] == pytest.approx(1 / per_key_s / 1e6, rel=1e-3)
    assert bench.lower_bound_roofline(scheme, fs, ms, None, 6400.0) is None


def test_random_access_bound_bucket_counts_lines():
    # Bucket scheme: one line read per repeat at the 128-byte read rate and
    # one line claimed per new key at the claim rate.
    fs = wk.fill_stream(30_000, 4096, 0.5, 64, seed=3)
    n_rep = fs.n_issued - fs.n_distinct
    t_min = n_rep / 40e9 + fs.n_distinct / 25e9
    got = bench.random_access_roofline("bucket", fs, None, None, t_min * 1e3 * 4, PROBE)
    assert got["frac"] == pytest.approx(0.25, abs=2e-3)
    assert got["lines_claimed_per_key"] == pytest.approx(fs.n_distinct / fs.n_issued, abs=1e-3)


def test_cpu_host_names_the_cores():
    h = bench.cpu_host()
    assert h["nproc"] >= 1 and h["machine"]


def test_reference_arm_prints_the_contract_line():
    # The reference arm times the oracle on the host (no GPU): one JSON line
    # with the metric, the oracle's throughput and an e2e of no copies.
    import json
    import subprocess
    import sys
    out = subprocess.check_output(
        [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "2", "--warmup", "1",
         "--n-log2", "18", "--batch-log2", "14"], text=True, timeout=300)
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mops/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["host"]["nproc"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Mops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n_distinct"] == 1 << 18


def test_random_access_bound_cuckoo_counts_probe_cas_as_claims():
    # Cuckoo: reads are the counted probes past one per new key; claims are
    # every table atomic of the insertions -- the probe's CASes into the
    # first empty slot plus the chains' exchanges (at least one per new key).
    fs = wk.fill_stream(30_000, 4096, 0.25, 64, seed=4)
    stats = {"probes": 2 * fs.n_issued, "probe_cas": fs.n_distinct + 500, "exchanges": 1000}
    reads = 2 * fs.n_issued - fs.n_distinct
    claims = fs.n_distinct + 1500
    t_min = reads / 40e9 + claims / 25e9
    got = bench.random_access_roofline("cuckoo", fs, None, stats, t_min * 1e3 * 2, PROBE)
    assert got["frac"] == pytest.approx(0.5, abs=2e-3)
    assert got["lines_claimed_per_key"] == pytest.approx(claims / fs.n_issued, abs=1e-3)
    few = dict(stats, probe_cas=10, exchanges=10)              # never fewer claims than new keys
    got = bench.random_access_roofline("cuckoo", fs, None, few, 1.0, PROBE)
    assert got["lines_claimed_per_key"] == pytest.approx(fs.n_distinct / fs.n_issued, abs=1e-3)


def test_recorded_traffic_follows_the_sources(tmp_path, monkeypatch):
    # A record counts only while its source files hash to the recorded
    # prefix: an edited source makes it None.
    import hashlib
    src = tmp_path / "k.cu"
    src.write_text("kernel one\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text("# comment\ntraffic probe k.cu 123000000 %s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("probe") == (123000000, "k.cu")
    assert bench.recorded_traffic("insert") == (None, None)
    src.write_text("kernel two\n")
    assert bench.recorded_traffic("probe") == (None, None)


def test_only_selects_named_sections():
    assert bench.section_wanted(set(), "long", False)
    assert not bench.section_wanted(set(), "long", True)
    assert bench.section_wanted({"long", "wide"}, "long", True)
    assert not bench.section_wanted({"long"}, "replay", False)
