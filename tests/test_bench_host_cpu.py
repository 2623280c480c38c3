"""Host-side logic of bench.py that decides whether a measurement stands: the
clock summary built from nvidia-smi samples (median SM clock under load,
throttle reasons seen under load). A fake sample file stands in for
nvidia-smi; no process is started."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

NA = "Not Active"


def _summary(lines):
    s = bench.ClockSampler(0)            # not entered: nvidia-smi is not run
    s.f.write("\n".join(lines) + "\n")
    s.f.flush()
    return s.summary()


def test_clock_summary_uses_the_samples_under_load():
    got = _summary([
        f"0, 2070, 2070, 150.0, 0x0, {NA}, {NA}, {NA}, {NA}",          # idle, before the timed region
        f"0, 1600, 2070, 1300.5, 0x4, {NA}, {NA}, {NA}, Active",
        f"0, 1800, 2070, 1250.0, 0x0, {NA}, {NA}, {NA}, {NA}",
        f"0, 1700, 2070, 1340.0, 0x4, {NA}, {NA}, {NA}, Active",
        "garbage line",
        f"0, 2070, 2070, [N/A], 0x0, Active, {NA}, {NA}, {NA}",         # no power reading: not under load
    ])
    assert got["sm_mhz"] == 1700.0 and got["sm_max_mhz"] == 2070.0
    assert got["samples"] == 3 and got["power_w_max"] == 1340.0
    assert got["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_slowdown_seen_under_load():
    got = _summary([
        f"0, 1900, 2070, 1000.0, 0x8, {NA}, Active, {NA}, {NA}",
        f"0, 1950, 2070, 1100.0, 0x0, Active, {NA}, {NA}, Active",
    ])
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 1925.0


def test_clock_summary_without_load_or_samples():
    idle = _summary([f"0, 2070, 2070, 120.0, 0x0, {NA}, {NA}, {NA}, {NA}"])
    assert idle["sm_mhz"] == 2070.0 and idle["samples"] == 1    # all samples when none is under load
    assert _summary([])["reasons"] == ["no samples"]


def test_whole_job_rate_and_rank_shards():
    assert bench.whole_job_rate(1000, 4, 3, 2.0) == 6000.0
    a, b = bench.rank_rays(32, 0), bench.rank_rays(32, 1)
    assert a.n == b.n == 32 and not (a.soa()[0] == b.soa()[0]).all()
