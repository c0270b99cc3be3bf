"""Host-side arithmetic of the benchmark line (no GPU): the lower-bound
roofline variant, the random-access bound and the host description."""
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
