"""Host-side logic of bench.py that decides whether a measurement stands: the
clock summary built from nvidia-smi samples (median SM clock under load,
throttle reasons seen under load; a fake sample file stands in for
nvidia-smi, no process is started), the default command line, the per-rank
split, the bounded oracle sample of the cpu_baseline leg, the roofline
object built from fake kernel times, and a static check that every name a
bench function reads is bound."""
import os
import sys

import numpy as np
import pytest

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


def test_roofline_block_from_fake_counters():
    """The line's roofline object from the library's per-class kernel times:
    7 hidden-layer launches of 1,048,576 rows in 14 ms against a 1,707.7
    TFLOP/s peak, the profiled tile's traffic scaled by rows."""
    prof = {"gemm": (14.0, 7), "gemm_first": (0.5, 1), "head": (0.05, 1), "encode": (0.0, 0)}
    R = 1 << 20
    r = bench.roofline_block(prof, R, 1, "256x4pairstaged", "bf16", {"bf16_tflops_sustained": 1707.7})
    flops = 2.0 * R * 7 * 1280 * 1280
    assert r["achieved"] == pytest.approx(flops / 14e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1707.7)
    assert r["flops_per_launch"] == pytest.approx(flops / 7)
    assert r["avg_launch_ms"] == pytest.approx(2.0)
    assert r["traffic"] == pytest.approx(R * 1304.9e6 / 262144)
    assert r["kernel_time_share"] == pytest.approx(14.0 / 14.55)
    assert r["tensor_pipe"]["active_pct_of_peak"] == [80.9, 81.4]
    # an unprofiled tile or precision reports no traffic; no measured peak: the fallback
    r2 = bench.roofline_block(prof, R, 1, "128x4", "bf16", {})
    assert r2["traffic"] is None and r2["tensor_pipe"] is None and r2["peak"] == 1700.0


def test_bench_functions_bind_every_name_they_read():
    """Every name a function of bench.py reads is bound in it, at module
    level or as a builtin (a renamed or shadowed variable fails here instead
    of on the GPU)."""
    import ast
    import builtins
    import os
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "bench.py")).read()
    tree = ast.parse(src)
    module = set(dir(builtins))
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            module.add(n.name)
        elif isinstance(n, ast.Assign):
            module |= {x.id for t in n.targets for x in ast.walk(t) if isinstance(x, ast.Name)}
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            module |= {(a.asname or a.name).split(".")[0] for a in n.names}
    for fn in (n for n in tree.body if isinstance(n, ast.FunctionDef)):
        bound = set()
        for x in ast.walk(fn):
            if isinstance(x, ast.Name) and isinstance(x.ctx, (ast.Store, ast.Del)):
                bound.add(x.id)
            elif isinstance(x, ast.arg):
                bound.add(x.arg)
            elif isinstance(x, ast.FunctionDef):
                bound.add(x.name)
            elif isinstance(x, (ast.Import, ast.ImportFrom)):
                bound |= {(a.asname or a.name).split(".")[0] for a in x.names}
            elif isinstance(x, ast.ExceptHandler) and x.name:
                bound.add(x.name)
        used = {x.id for x in ast.walk(fn) if isinstance(x, ast.Name) and isinstance(x.ctx, ast.Load)}
        assert not (used - bound - module), (fn.name, sorted(used - bound - module))
