"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bounds (|t_gpu - t_ref| and |vis_gpu - vis_ref|, relative to max(1, |ref|)):
  * FP32 path vs the exact oracle: 1e-4 on every ray.
  * bf16 / e4m3 paths vs the oracle emulating the same roundings: the two
    differ only by FP32 accumulation order, which can move an activation across
    a rounding boundary (one bf16 ulp = 2^-8 relative, one e4m3 ulp = 2^-3);
    bounds max 2e-3 / mean 2e-4 (bf16) and max 1e-2 / mean 1e-3 (e4m3).
  * bf16 / e4m3 paths vs the exact oracle: mean |dt| <= 5e-3, max <= 5e-2
    (bf16) and mean <= 2e-2, max <= 0.2 (e4m3).
"""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMALL = (6, 128, 4)      # 78 -> 128 x4 -> 2
PAPER = (10, 1280, 8)    # 126 -> 1280 x8 -> 2
SMALL_256 = (6, 256, 3)  # 78 -> 256 x3 -> 2
LIGHT = (3.0, 3.0, 3.0)
BOUNDS = {"bf16": (2e-3, 2e-4), "fp8": (1e-2, 1e-3)}
EXACT_BOUNDS = {"bf16": (5e-2, 5e-3), "fp8": (0.2, 2e-2)}


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _dev(torch, rays):
    return [torch.from_numpy(a).cuda() for a in rays.soa()]


def _make(net, prec, blob, scales=None, chunk=None):
    from paper_2606_00817_gb300 import ddf
    m = ddf.DDF(*net, precision=prec)
    m.load(blob, scales if prec == "fp8" else None)
    if chunk:
        ddf.ddf_set_chunk_rays(m.h, chunk)
    return m


def _query(torch, m, rays):
    t, v = m.query(_dev(torch, rays))
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return np.abs(a - b) / np.maximum(1.0, np.abs(b))


def _oracle(rays, blob, net, prec, scales=None):
    return O.ddf_forward(rays.origins(), rays.dirs(), blob, *net, precision=prec, act_scales=scales)


def _check_reduced(t, v, rays, blob, net, prec, scales):
    emu = _oracle(rays, blob, net, prec, scales)
    mx, mean = BOUNDS[prec]
    for g, r in ((t, emu["t"]), (v, emu["vis"])):
        e = _rel(g, r)
        assert e.max() <= mx and e.mean() <= mean, (prec, e.max(), e.mean())
    ex = _oracle(rays, blob, net, "exact")
    dt = np.abs(t - ex["t"])
    mx, mean = EXACT_BOUNDS[prec]
    assert dt.max() <= mx and dt.mean() <= mean, (prec, dt.max(), dt.mean())


def _scales(blob, net, seed=99):
    cal = I.uniform_rays(512, seed=seed)
    return O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *net)


@pytest.mark.parametrize("n", [1, 127, 129, 16384])
def test_fp32_small_net_matches_exact_oracle(torch_cuda, n):
    blob = I.xavier_blob(I.NetShape(*SMALL))
    rays = I.uniform_rays(n, seed=1)
    t, v = _query(torch_cuda, _make(SMALL, "fp32", blob), rays)
    ex = _oracle(rays, blob, SMALL, "exact")
    assert _rel(t, ex["t"]).max() <= 1e-4
    assert _rel(v, ex["vis"]).max() <= 1e-4


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n", [1, 127, 129, 16384])
def test_reduced_small_net_matches_emulating_oracle(torch_cuda, prec, n):
    blob = I.xavier_blob(I.NetShape(*SMALL))
    sc = _scales(blob, SMALL)
    rays = I.uniform_rays(n, seed=2)
    t, v = _query(torch_cuda, _make(SMALL, prec, blob, sc), rays)
    _check_reduced(t, v, rays, blob, SMALL, prec, sc)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_paper_sized_net(torch_cuda, prec):
    blob = I.xavier_blob(I.NetShape(*PAPER))
    scene = I.random_scene(64, 0, seed=0)
    rays = I.shadow_rays(scene, 1037, LIGHT, seed=3)   # 8 full row tiles + a ragged one
    sc = _scales(blob, PAPER)
    t, v = _query(torch_cuda, _make(PAPER, prec, blob, sc), rays)
    if prec == "fp32":
        ex = _oracle(rays, blob, PAPER, "exact")
        assert _rel(t, ex["t"]).max() <= 1e-4
        assert _rel(v, ex["vis"]).max() <= 1e-4
    else:
        _check_reduced(t, v, rays, blob, PAPER, prec, sc)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_chunking_does_not_change_results(torch_cuda, prec):
    blob = I.xavier_blob(I.NetShape(*SMALL))
    rays = I.uniform_rays(1000, seed=4)
    a = _query(torch_cuda, _make(SMALL, prec, blob), rays)
    b = _query(torch_cuda, _make(SMALL, prec, blob, chunk=128), rays)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_shadow_decisions_match_oracle(torch_cuda):
    torch = torch_cuda
    blob = I.xavier_blob(I.NetShape(*SMALL))
    scene = I.random_scene(64, 0, seed=0)
    rays = I.shadow_rays(scene, 3000, LIGHT, seed=5)
    m = _make(SMALL, "bf16", blob)
    t, v, occ = m.shadow(_dev(torch, rays), LIGHT)
    torch.cuda.synchronize()
    emu = _oracle(rays, blob, SMALL, "bf16")
    ref = O.shadow(emu["t"], emu["z"][:, 1], rays.origins(), LIGHT)
    dist = np.linalg.norm(np.array(LIGHT) - rays.origins().astype(np.float64), axis=1)
    clear = (np.abs(emu["z"][:, 1]) > 1e-3) & (np.abs(emu["t"] - dist) > 1e-3)
    assert clear.mean() > 0.9
    assert np.array_equal(occ.cpu().numpy().astype(bool)[clear], ref[clear])


def test_host_buffer_query_matches_device_query(torch_cuda):
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    rays = I.uniform_rays(5000, seed=6)
    m = _make(SMALL, "bf16", blob, chunk=1024)
    t_d, v_d = _query(torch_cuda, m, rays)
    t_h, v_h = m.query_host(rays.soa())
    assert np.array_equal(t_h.astype(np.float64), t_d) and np.array_equal(v_h.astype(np.float64), v_d)
    assert ddf.ddf_check_status(m.h) == 0


def test_weights_round_trip_and_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    m = _make(SMALL, "bf16", blob)
    assert np.array_equal(ddf.ddf_get_weights(m.h, blob.size), blob)
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_load_weights(m.h, blob[:-1])
    assert e.value.status == 4
    bad = blob.copy()
    bad[5] = np.nan
    with pytest.raises(ddf.DDFError):
        ddf.ddf_load_weights(m.h, bad)
    rays = _dev(torch, I.uniform_rays(4))
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_query_rays(m.h, rays, 4, None, None)
    assert e.value.status == 1
    ddf.ddf_query_rays(m.h, rays, 0, None, None)  # empty batch: no-op
    f8 = ddf.DDF(*SMALL, precision="fp8")
    f8.load(blob)
    with pytest.raises(ddf.DDFError):
        f8.query(rays)                            # e4m3 needs activation scales
    with pytest.raises(ddf.DDFError):
        ddf.ddf_set_act_scales(f8.h, [0.3, 0.5, 0.25])   # not powers of two
    with pytest.raises(ddf.DDFError) as e:
        ddf.DDF(6, 96, 4, precision="bf16")        # tensor cores need width % 128 == 0
    assert e.value.status == 5


def test_timeout_path_gives_up_cleanly_and_recovers(torch_cuda):
    """A zero wait limit makes the pipelined kernel give up at its first wait
    that is not already satisfied: the status word reports it, nothing traps,
    and the next launch with the normal limit is correct. A wait gives up
    only once it has outlasted a tick of the global timer, so the field is
    the paper-sized one: its first accumulator takes 20 k-blocks of MMAs
    (microseconds) before the epilogue's first wait can succeed."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    rays = I.uniform_rays(65536, seed=7)
    m = _make(PAPER, "bf16", blob)
    ddf.ddf_set_timeout_ns(m.h, 0)
    m.query(_dev(torch, rays))
    assert ddf.ddf_check_status(m.h) & 1
    ddf.ddf_set_timeout_ns(m.h, 2_000_000_000)
    t, v = _query(torch, m, rays.slice(0, 512))
    assert ddf.ddf_check_status(m.h) == 0
    _check_reduced(t, v, rays.slice(0, 512), blob, PAPER, "bf16", None)


@pytest.fixture(scope="module")
def full_shadow():
    """The benchmark's input: 4,194,304 shadow rays of the 64-sphere scene
    (seed 0) toward the light, on the 8 x 1280 Xavier field."""
    scene = I.random_scene(64, 0, seed=0)
    return I.shadow_rays(scene, 4_194_304, LIGHT, seed=0), I.xavier_blob(I.NetShape(*PAPER))


CHUNK = 1 << 20          # the library's default rays per chunk
# the tiles the benchmark's autotuner picks on this field: hidden layers on the
# staged CTA-pair tile, layer 1 with the encoding fused, 4 epilogue warps each
BENCH_TILES = ((256, 4, 1, 1, 0), (256, 4, 0, 1, 1))


def _chunk_sample(n, per_chunk=256, edge=4, seed=0):
    """Row indices that cover every chunk of the query: its first and last
    `edge` rows and `per_chunk` random rows inside it."""
    rng = np.random.default_rng(seed)
    idx = []
    for lo in range(0, n, CHUNK):
        hi = min(lo + CHUNK, n)
        idx += [np.arange(lo, lo + edge), np.arange(hi - edge, hi),
                rng.choice(np.arange(lo, hi), per_chunk, replace=False)]
    return np.unique(np.concatenate(idx))


@pytest.mark.parametrize("prec,tiles", [("bf16", BENCH_TILES), ("fp8", BENCH_TILES),
                                        ("bf16", "autotune")])
def test_full_size_shadow_workload_sampled(torch_cuda, full_shadow, prec, tiles):
    """The 4,194,304-ray shadow workload on the 8x1280 field in the launch
    configuration the benchmark times: four chunks of 1,048,576 rays, hidden
    layers on the staged CTA-pair tile and layer 1 with the fused encoding (set
    explicitly, or picked by the autotuner on the first chunk as the benchmark
    does). Every chunk is sampled (its first and last rows and 256 inside it)
    against the emulating and the exact oracle, and the shadow bytes against
    the oracle's decision on rays clear of a tie."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    rays, blob = full_shadow
    sc = _scales(blob, PAPER) if prec == "fp8" else None
    m = _make(PAPER, prec, blob, sc)
    d = _dev(torch, rays)
    if tiles == "autotune":
        ddf.ddf_autotune(m.h, [r[:CHUNK] for r in d], CHUNK)
        chosen = (ddf.ddf_get_tile(m.h, 0), ddf.ddf_get_tile(m.h, 1))
        assert chosen[0][0] == 256 and chosen[1][0] == 256, chosen
    else:
        for which in (0, 1):
            ddf.ddf_set_tile(m.h, tiles[which], which)
        assert (ddf.ddf_get_tile(m.h, 0), ddf.ddf_get_tile(m.h, 1)) == tiles
    t, v, occ = m.shadow(d, LIGHT)
    torch.cuda.synchronize()
    assert ddf.ddf_check_status(m.h) == 0
    t = t.cpu().numpy().astype(np.float64)
    v = v.cpu().numpy().astype(np.float64)
    occ = occ.cpu().numpy().astype(bool)
    assert np.all(np.isfinite(t)) and np.all(np.isfinite(v))
    idx = _chunk_sample(rays.n)
    assert all(np.any((idx >= lo) & (idx < lo + CHUNK)) for lo in range(0, rays.n, CHUNK))
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    _check_reduced(t[idx], v[idx], sub, blob, PAPER, prec, sc)
    emu = _oracle(sub, blob, PAPER, prec, sc)
    ref = O.shadow(emu["t"], emu["z"][:, 1], sub.origins(), LIGHT)
    dist = np.linalg.norm(np.array(LIGHT) - sub.origins().astype(np.float64), axis=1)
    # clear of a tie by more than the parity bound can move z1 (|d vis| <= mx
    # and d vis / d z1 <= 1/4) or t (mx max(1, t)); the Xavier field puts z1
    # near 0, so at the e4m3 bound only a few percent of the rays are clear
    mx = BOUNDS[prec][0]
    clear = (np.abs(emu["z"][:, 1]) > 5 * mx) & (np.abs(emu["t"] - dist) > 2 * mx * np.maximum(1, dist))
    assert clear.sum() >= 20
    assert np.array_equal(occ[idx][clear], ref[clear])
    # every one of the 4,194,304 decisions agrees with the query's own t and
    # vis (occluded iff z1 > 0, i.e. vis > 1/2, and t below the light
    # distance), except exact ties, where float32 and float64 may differ
    o = rays.origins().astype(np.float64)
    dl = np.linalg.norm(np.array(LIGHT) - o, axis=1)
    decided = (v != 0.5) & (np.abs(t - dl) > 1e-5 * dl)
    assert decided.mean() > 0.999
    assert np.array_equal(occ[decided], ((v > 0.5) & (t < dl))[decided])


@pytest.mark.parametrize("tile", [(256, 4, 0, 0, 0), (256, 8, 0, 0, 0), (128, 4, 0, 0, 0),
                                  (128, 8, 0, 0, 0), (256, 4, 1, 0, 0), (256, 4, 1, 1, 0),
                                  (256, 8, 1, 0, 0), (256, 8, 1, 1, 0)])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_every_tile_matches_oracle(torch_cuda, tile, prec):
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    sc = _scales(blob, PAPER)
    rays = I.uniform_rays(777, seed=8)          # 3 pair row-tiles + a ragged one
    m = _make(PAPER, prec, blob, sc)
    ddf.ddf_set_tile(m.h, tile, which=0)
    ddf.ddf_set_tile(m.h, tile, which=1)
    assert ddf.ddf_get_tile(m.h, 0) == tile and ddf.ddf_get_tile(m.h, 1) == tile
    t, v = _query(torch_cuda, m, rays)
    _check_reduced(t, v, rays, blob, PAPER, prec, sc)
    assert ddf.ddf_check_status(m.h) == 0


@pytest.mark.parametrize("net,n", [(PAPER, 777), (PAPER, 300_001), (SMALL_256, 1029)])
@pytest.mark.parametrize("epi", [4, 8])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_fused_encode_layer1(torch_cuda, net, n, epi, prec):
    """Layer 1 with the encoding built in shared memory (L = 10: K = 126 in two
    64-wide slices; L = 6: K = 78, the second slice mostly padding): every
    output equals the unfused layer 1's bit for bit (same rounding of the same
    features, same epilogue), and sampled rays match the oracle. 777 rays: 7
    row blocks, the last ragged; 300,001 rays: about 15 row blocks per CTA, so
    both shared-memory A buffers are reused many times."""
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*net))
    sc = _scales(blob, net) if prec == "fp8" else None
    rays = I.uniform_rays(n, seed=11)
    m = _make(net, prec, blob, sc)
    ddf.ddf_set_tile(m.h, (256, 4, 0, 0), which=1)
    ref_t, ref_v = _query(torch_cuda, m, rays)
    ddf.ddf_set_tile(m.h, (256, epi, 0, 1, 1), which=1)
    assert ddf.ddf_get_tile(m.h, 1) == (256, epi, 0, 1, 1)
    t, v = _query(torch_cuda, m, rays)
    assert ddf.ddf_check_status(m.h) == 0
    assert np.array_equal(t, ref_t) and np.array_equal(v, ref_v)
    idx = np.unique(np.concatenate([np.arange(0, 64), np.arange(rays.n - 64, rays.n),
                                    np.random.default_rng(4).choice(rays.n, 64, replace=False)]))
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    _check_reduced(t[idx], v[idx], sub, blob, net, prec, sc)


def test_fused_encode_rejected_where_unsupported(torch_cuda):
    from paper_2606_00817_gb300 import ddf
    m = _make(PAPER, "bf16", I.xavier_blob(I.NetShape(*PAPER)))
    for tile, which in (((256, 4, 0, 1, 1), 0), ((256, 4, 1, 1, 1), 1), ((128, 4, 0, 1, 1), 1),
                        ((256, 4, 0, 0, 1), 1)):
        with pytest.raises(ddf.DDFError):
            ddf.ddf_set_tile(m.h, tile, which)
    m12 = _make((12, 256, 2), "bf16", I.xavier_blob(I.NetShape(12, 256, 2)))
    with pytest.raises(ddf.DDFError):                       # 6 + 12 x 12 = 150 > 128
        ddf.ddf_set_tile(m12.h, (256, 4, 0, 1, 1), 1)
    m1 = _make((10, 256, 1), "bf16", I.xavier_blob(I.NetShape(10, 256, 1)))
    with pytest.raises(ddf.DDFError):                       # layer 1 is also the head layer
        ddf.ddf_set_tile(m1.h, (256, 4, 0, 1, 1), 1)


def test_pair_tile_on_a_full_chunk(torch_cuda):
    """The staged CTA-pair tile over 300,001 rays (1172 pair row-tiles, more
    than one per cluster, and a ragged last tile), sampled against the oracle
    and against the default tile."""
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    rays = I.uniform_rays(300_001, seed=10)
    m = _make(PAPER, "bf16", blob)
    for which in (0, 1):
        ddf.ddf_set_tile(m.h, (256, 4, 1, 1), which)
    t, v = _query(torch_cuda, m, rays)
    assert ddf.ddf_check_status(m.h) == 0
    for which in (0, 1):
        ddf.ddf_set_tile(m.h, (256, 4, 0, 0), which)
    t1, v1 = _query(torch_cuda, m, rays)
    assert np.max(np.abs(t - t1)) <= 1e-5 and np.max(np.abs(v - v1)) <= 1e-5
    idx = np.concatenate([np.arange(0, 100), np.arange(rays.n - 100, rays.n)])
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    _check_reduced(t[idx], v[idx], sub, blob, PAPER, "bf16", None)


def test_small_width_tiles_and_autotune(torch_cuda):
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    rays = I.uniform_rays(4099, seed=9)
    m = _make(SMALL, "bf16", blob)
    with pytest.raises(ddf.DDFError):
        ddf.ddf_set_tile(m.h, (256, 4, 0, 0))  # width 128 has no 256-wide N tile
    p1, p2 = ddf.ddf_autotune(m.h, _dev(torch_cuda, rays), rays.n)
    for ms in (p1, p2):
        assert all(ms[c] is None for c in ms if c[0] == 256)
        assert ms[(128, 4, 0, 0, 0)] > 0 and ms[(128, 8, 0, 0, 0)] > 0
    assert ddf.ddf_get_tile(m.h, 0) in ((128, 4, 0, 0, 0), (128, 8, 0, 0, 0))
    assert ddf.ddf_get_tile(m.h, 1) in ((128, 4, 0, 0, 0), (128, 8, 0, 0, 0))
    t, v = _query(torch_cuda, m, rays)
    _check_reduced(t, v, rays, blob, SMALL, "bf16", None)
