"""Edge cases of every GPU path: ragged and tiny batches around the tile
sizes, empty inputs on every entry point, chunk boundaries, axis-parallel and
boundary rays, a training batch without hits, and the degenerate settings of
the sphere tracer (one step, t_max 0, rays starting inside). Bounds as in
test_gpu_parity (bf16 / e4m3 against the emulating oracle)."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMALL = (6, 128, 4)
W256 = (6, 256, 3)
PAPER = (10, 1280, 8)
BOUNDS = {"bf16": (2e-3, 2e-4), "fp8": (1e-2, 1e-3)}


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _dev(torch, arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _make(net, prec, blob, scales=None):
    from paper_2606_00817_gb300 import ddf
    m = ddf.DDF(*net, precision=prec)
    m.load(blob, scales if prec == "fp8" else None)
    return m


def _scales(blob, net):
    cal = I.uniform_rays(512, seed=99)
    return O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *net)


def _query(torch, m, rays):
    t, v = m.query(_dev(torch, rays.soa()))
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)


def _check(t, v, rays, blob, net, prec, scales):
    emu = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net, precision=prec, act_scales=scales)
    mx, mean = BOUNDS[prec]
    for g, r in ((t, emu["t"]), (v, emu["vis"])):
        e = np.abs(g - r) / np.maximum(1.0, np.abs(r))
        assert e.max() <= mx and e.mean() <= mean, (prec, e.max(), e.mean())


TILES = {"pair+fused": ((256, 4, 1, 1, 0), (256, 8, 0, 1, 1)),
         "1cta": ((128, 8, 0, 0, 0), (128, 4, 0, 0, 0))}


@pytest.mark.parametrize("n", [1, 7, 255, 257, 513])
@pytest.mark.parametrize("tiles", list(TILES))
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_ragged_batches_on_every_tile(torch_cuda, n, tiles, prec):
    """Batches smaller than one row tile, one ray either side of the 256-row
    pair tile, and a few tiles with a ragged last one."""
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*W256))
    sc = _scales(blob, W256) if prec == "fp8" else None
    m = _make(W256, prec, blob, sc)
    hidden, first = TILES[tiles]
    ddf.ddf_set_tile(m.h, hidden, 0)
    ddf.ddf_set_tile(m.h, first, 1)
    rays = I.uniform_rays(n, seed=70 + n)
    t, v = _query(torch_cuda, m, rays)
    _check(t, v, rays, blob, W256, prec, sc)
    assert ddf.ddf_check_status(m.h) == 0


@pytest.mark.parametrize("n", [1, 257])
def test_ragged_batches_paper_sized(torch_cuda, n):
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    m = _make(PAPER, "bf16", blob)
    ddf.ddf_set_tile(m.h, (256, 4, 1, 1, 0), 0)
    ddf.ddf_set_tile(m.h, (256, 4, 0, 1, 1), 1)
    rays = I.uniform_rays(n, seed=80 + n)
    t, v = _query(torch_cuda, m, rays)
    _check(t, v, rays, blob, PAPER, "bf16", None)


@pytest.mark.parametrize("n", [1023, 1024, 1025, 2049])
def test_chunk_boundaries_are_invisible(torch_cuda, n):
    """With 1024-ray chunks, every chunk split (full, one short, one over)
    gives bit-identical outputs to a single-chunk query, on the fused
    layer-1 tile and the pair tile."""
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*W256))
    rays = I.uniform_rays(n, seed=90)
    out = []
    for chunk in (1 << 20, 1024):
        m = _make(W256, "bf16", blob)
        ddf.ddf_set_tile(m.h, (256, 4, 1, 1, 0), 0)
        ddf.ddf_set_tile(m.h, (256, 4, 0, 1, 1), 1)
        ddf.ddf_set_chunk_rays(m.h, chunk)
        out.append(_query(torch_cuda, m, rays))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_empty_inputs_on_every_entry_point(torch_cuda):
    """n = 0 is a no-op everywhere: no error, no launch, status clean."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    m = _make(SMALL, "bf16", blob)
    rays = _dev(torch, I.uniform_rays(8).soa())
    out = [torch.empty(8, device="cuda") for _ in range(2)]
    occ = torch.empty(8, dtype=torch.uint8, device="cuda")
    ddf.ddf_query_rays(m.h, rays, 0, out[0], out[1])
    ddf.ddf_query_shadow(m.h, rays, 0, (3.0, 3.0, 3.0), out[0], out[1], occ)
    ddf.ddf_query_rays_noalloc(m.h, rays, 0, out[0], out[1])
    h_rays = [np.zeros(8, np.float32) for _ in range(6)]
    ddf.ddf_query_rays_host(m.h, h_rays, 0, np.zeros(8, np.float32), np.zeros(8, np.float32))
    offsets = torch.zeros(1, dtype=torch.int32, device="cuda")
    ddf.ddf_query_ao(m.h, rays, 0, offsets, 0, out[0], out[1])
    hit = torch.empty(8, dtype=torch.uint8, device="cuda")
    sph = torch.tensor([0.0, 0.0, 0.0, 0.5], device="cuda")
    ddf.ddf_cast_scene(sph, 1, None, 0, rays, 0, out[0], hit)
    pts = rays[:3]
    ddf.ddf_union_sdf(sph, 1, None, 0, pts, 0, out[0])
    s = ddf.DDF(4, 128, 3, precision="bf16", kind="sdf")
    s.load(I.xavier_blob_dims(I.sdf_layer_dims(4, 128, 3)))
    ddf.ddf_sdf_eval(s.h, pts, 0, out[0])
    steps = torch.empty(8, dtype=torch.int32, device="cuda")
    ddf.ddf_sphere_trace(s.h, rays, 0, 16, 1e-3, 4.0, out[0], hit, steps)
    torch.cuda.synchronize()
    assert ddf.ddf_check_status(m.h) == 0 and ddf.ddf_check_status(s.h) == 0


def test_axis_parallel_and_boundary_rays(torch_cuda):
    """Directions along +-x, +-y, +-z (zero components) from the corners,
    faces and centre of [-1, 1]^3: the field matches the oracle and the
    caster's closed slabs match the oracle's."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    origins = np.array([[x, y, z] for x in (-1, 0, 1) for y in (-1, 0, 1) for z in (-1, 0, 1)], float)
    o = np.repeat(origins, len(dirs), axis=0)
    d = np.tile(dirs, (len(origins), 1))
    rays = I.Rays.from_arrays(o, d)
    blob = I.xavier_blob(I.NetShape(*W256))
    m = _make(W256, "bf16", blob)
    ddf.ddf_set_tile(m.h, (256, 4, 0, 1, 1), 1)
    t, v = _query(torch, m, rays)
    _check(t, v, rays, blob, W256, "bf16", None)
    scene = I.random_scene(8, 8, seed=3)
    sph = torch.from_numpy(np.concatenate([scene.centers, scene.radii[:, None]], 1)
                           .astype(np.float32).ravel()).cuda()
    box = torch.from_numpy(np.concatenate([scene.box_lo, scene.box_hi], 1)
                           .astype(np.float32).ravel()).cuda()
    tt = torch.empty(rays.n, device="cuda")
    hit = torch.empty(rays.n, dtype=torch.uint8, device="cuda")
    ddf.ddf_cast_scene(sph, 8, box, 8, _dev(torch, rays.soa()), rays.n, tt, hit)
    torch.cuda.synchronize()
    t_ref, h_ref = O.cast_scene(scene, rays.origins(), rays.dirs())
    g_hit = hit.cpu().numpy().astype(bool)
    assert np.array_equal(g_hit, h_ref)
    g_t = tt.double().cpu().numpy()
    assert np.all(np.abs(g_t[h_ref] - t_ref[h_ref]) <= 1e-5 * np.maximum(1.0, t_ref[h_ref]))


def test_training_batch_without_hits(torch_cuda):
    """No ray hits (every target a miss): the L1 term is empty (divided by
    max(1, 0)), only the cross-entropy drives the gradient; the smallest
    batch (8 rays) and an all-miss batch of 4096 both match the oracle."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    for B in (8, 4096):
        rays = I.uniform_rays(B, seed=95)
        tt = np.full(B, np.inf, np.float32)
        y = np.zeros(B, np.uint8)
        m = _make(SMALL, "bf16", blob)
        loss = torch.zeros(1, device="cuda")
        ddf.ddf_compute_grad(m.h, _dev(torch, rays.soa()), torch.from_numpy(tt).cuda(),
                             torch.from_numpy(y).cuda(), B, loss)
        g = ddf.ddf_get_grad(m.h, blob.size).astype(np.float64)
        L_emu, g_emu = O.train_grad(rays.origins(), rays.dirs(), blob, *SMALL, tt, y,
                                    precision="bf16")
        _, g_ex = O.ddf_loss_grad(rays.origins(), rays.dirs(), blob, *SMALL, tt, y)
        assert np.isfinite(loss.item()) and abs(loss.item() - L_emu) <= 1e-4 * abs(L_emu)
        noise = np.linalg.norm(g_emu - g_ex)
        assert np.linalg.norm(g - g_emu) <= 0.4 * noise + 1e-3 * np.linalg.norm(g_emu)
        assert ddf.ddf_check_status(m.h) == 0


def test_sphere_trace_degenerate_settings(torch_cuda):
    """One step only; t_max 0 (a ray that does not hit at once is a miss
    after its first step); rays starting inside the surface (s < eps at
    t = 0: a hit at t = 0 after one evaluation). All against the oracle's
    tracer on the same affine SDF network (s = 0.5 (n.p - c))."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net = (4, 128, 3)
    dims = I.sdf_layer_dims(*net)
    n = np.array([0.36, -0.48, 0.8], np.float32)
    parts = []
    for li, (fo, fi) in enumerate(dims):
        w = np.zeros((fo, fi), np.float32)
        b = np.zeros(fo, np.float32)
        if li == 0:
            w[0, :3], b[0] = 0.5 * n, 0.0
            w[1, :3], b[1] = -0.5 * n, 0.0
        elif li < len(dims) - 1:
            w[0, 0] = w[1, 1] = 1.0
        else:
            w[0, 0], w[0, 1] = 1.0, -1.0
        parts += [w.ravel(), b]
    blob = np.concatenate(parts)                       # plane through the origin
    m = ddf.DDF(*net, precision="bf16", kind="sdf")
    m.load(blob)
    rays = I.uniform_rays(2000, seed=96)               # about half start inside
    dev = _dev(torch, rays.soa())
    sdf = lambda q: O.sdf_mlp(q, blob, *net, precision="bf16")
    for max_steps, t_max in ((1, 4.0), (64, 0.0), (64, 4.0)):
        t = torch.empty(rays.n, device="cuda")
        hit = torch.empty(rays.n, dtype=torch.uint8, device="cuda")
        steps = torch.empty(rays.n, dtype=torch.int32, device="cuda")
        ddf.ddf_sphere_trace(m.h, dev, rays.n, max_steps, 1e-3, t_max, t, hit, steps)
        torch.cuda.synchronize()
        tr, hr, sr = O.sphere_trace(sdf, rays.origins(), rays.dirs(), max_steps=max_steps,
                                    eps=1e-3, t_max=t_max)
        g_hit = hit.cpu().numpy().astype(bool)
        g_steps = steps.cpu().numpy()
        same = (g_hit == hr) & (g_steps == sr)
        assert same.mean() >= 0.99, (max_steps, t_max, same.mean())
        inside = rays.origins() @ n.astype(np.float64) < -0.01
        assert np.all(g_hit[inside]) and np.all(g_steps[inside] == 1)
        assert np.all(t.cpu().numpy()[inside] == 0.0)
        assert g_steps.max() <= max_steps
    assert ddf.ddf_check_status(m.h) == 0


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("tiles", [((256, 4, 1, 1, 0), (256, 4, 0, 1, 1)),
                                   ((256, 8, 1, 1, 0), (256, 8, 0, 1, 1)),
                                   ((256, 4, 1, 0, 0), (256, 4, 1, 0, 0))])
def test_widest_field_on_the_pair_tiles(torch_cuda, prec, tiles):
    """Width 2048, the widest field the tensor-core path takes: the staged
    pair tile then holds 5 pipeline stages, 32 KB of per-column vectors and
    the output boxes within the 227 KB of shared memory per CTA. 300 rays
    (a ragged second row tile), against the emulating oracle."""
    from paper_2606_00817_gb300 import ddf
    net = (6, 2048, 3)
    blob = I.xavier_blob(I.NetShape(*net))
    sc = _scales(blob, net) if prec == "fp8" else None
    m = _make(net, prec, blob, sc)
    ddf.ddf_set_tile(m.h, tiles[0], 0)
    ddf.ddf_set_tile(m.h, tiles[1], 1)
    rays = I.uniform_rays(300, seed=60)
    t, v = _query(torch_cuda, m, rays)
    _check(t, v, rays, blob, net, prec, sc)
    assert ddf.ddf_check_status(m.h) == 0


def test_widest_and_deepest_configurations_are_the_limits(torch_cuda):
    """The deepest field (64 hidden layers) runs and matches the oracle; one
    column or layer more is refused at creation, before any launch."""
    from paper_2606_00817_gb300 import ddf
    net = (6, 128, 64)
    blob = I.xavier_blob(I.NetShape(*net))
    m = _make(net, "bf16", blob)
    rays = I.uniform_rays(129, seed=61)
    t, v = _query(torch_cuda, m, rays)
    _check(t, v, rays, blob, net, "bf16", None)
    for bad in ((6, 2176, 2), (6, 128, 65)):
        with pytest.raises(ddf.DDFError):
            ddf.DDF(*bad, precision="bf16")
