"""Host-side logic of bench.py that decides whether a measurement stands: the
clock summary built from nvidia-smi samples (median SM clock under load,
throttle reasons seen under load; a fake sample file stands in for
nvidia-smi, no process is started), the default command line, the per-rank
split and the bounded oracle sample of the cpu_baseline leg."""
import os
import sys

import numpy as np

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


def test_default_command_line_keeps_the_contract(monkeypatch):
    """No flags: one GPU, the full headline workload, bf16, at least 3
    warm-up steps."""
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours" and a.precision == "bf16"
    assert a.warmup >= 3 and a.steps >= 1 and a.rays == 4_194_304


def test_oracle_sample_is_bounded_spread_and_exact():
    """The cpu_baseline leg: blocks taken round-robin from every chunk of the
    query until the time budget is spent (one round at least), never more than
    the cap, with the FP64 outputs of exactly the rays it sampled."""
    from oracle import ddf_oracle as O
    from paper_2606_00817_gb300 import inputs as I
    rays = I.uniform_rays(1000, seed=9)
    blob = I.xavier_blob(I.NetShape(*bench.NET), seed=0)
    # chunks of 400, 400 and 200 rays; blocks of 50
    rate, idx, el, ref = bench.oracle_sample(rays, blob, seconds=0.0, block=50, cap=600, chunk=400)
    assert rate > 0 and el > 0
    assert sorted(set(idx // 400)) == [0, 1, 2] and idx.size == 150   # one block per chunk
    rate, idx, el, ref = bench.oracle_sample(rays, blob, seconds=1e9, block=50, cap=600, chunk=400)
    assert idx.size == 600 and ref["t"].shape == (600,) and np.unique(idx).size == 600
    for c in range(3):
        assert np.sum(idx // 400 == c) == 200                   # the same share of every chunk
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    want = O.ddf_forward(sub.origins(), sub.dirs(), blob, *bench.NET)
    # the same FP64 values up to the matrix products' summation order, which
    # depends on the batch size
    assert np.allclose(ref["t"], want["t"], rtol=1e-12, atol=1e-13)
    assert np.allclose(ref["vis"], want["vis"], rtol=1e-12, atol=1e-13)


def test_tensor_pipe_figures_come_from_the_cited_profile():
    """The tensor-pipe activity the bench line reports is copied from a
    committed ncu summary; each figure must still appear in it."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        bench.PROFILE_SOURCE)
    text = open(path).read()
    assert "sm__pipe_tensor_cycles_active" in text
    for tile in bench.PROFILED_TILES.values():
        for v in tile["active_pct_of_peak"]:
            assert f"{v} %" in text, v
        assert f"{tile['traffic_per_262144_rows'] / 1e6:.1f} MB" in text
