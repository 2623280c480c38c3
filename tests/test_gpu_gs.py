"""GPU tests of the Gaussian-rendered depth (the supervision source of Sec.
3.2 studied in Sec. 4.2), the camera rays and training from a fixed pool of
supervised rays. The renderer is compared with the oracle's composite, which
evaluates every Gaussian at every pixel in float64.

Tolerance: the kernel composites in float32, so a pixel's expected distance
carries the rounding of a few hundred multiply-adds, relative 1e-4 at most.
Three float32 decisions can also land on the other side than in float64:
alpha >= 1/255, T < 1e-4 (the stop) and the depth order of nearly equal
depths. Each flip touches a pixel whose contribution sits at the threshold,
so flips are rare: at most 0.5 % of the pixels may differ beyond 1e-4."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _cam(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_deg=40.0):
    return np.array([*eye, *target, *up, np.radians(fov_deg)], np.float32)


def _render(torch, means, covs, opac, cams, W, H):
    from paper_2606_00817_gb300 import ddf
    cams = np.asarray(cams, np.float32).reshape(-1, 10)
    V = cams.shape[0]
    dm = torch.from_numpy(np.ascontiguousarray(means, np.float32)).cuda()
    dc = torch.from_numpy(np.ascontiguousarray(covs, np.float32)).cuda()
    do = torch.from_numpy(np.ascontiguousarray(opac, np.float32)).cuda()
    t = torch.empty(V * H * W, device="cuda")
    hit = torch.empty(V * H * W, dtype=torch.uint8, device="cuda")
    ddf.ddf_render_gs_depth(dm, dc, do, means.shape[0], cams, W, H, t, hit)
    torch.cuda.synchronize()
    return (t.cpu().numpy().astype(np.float64).reshape(V, H, W),
            hit.cpu().numpy().astype(bool).reshape(V, H, W))


def _oracle(means, covs, opac, cam, W, H, pixels=None):
    # the oracle reads the float32 inputs the kernel reads
    return O.gs_depth(means.astype(np.float64), O.gs_cov_matrices(covs), opac.astype(np.float64),
                      cam[0:3], cam[3:6], cam[6:9], float(cam[9]), W, H, pixels=pixels)


def _random_gaussians(n, seed, lo=-1.0, hi=1.0, smin=0.01, smax=0.2, omin=0.05, omax=1.0):
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, (n, 3))
    q, _ = np.linalg.qr(rng.normal(size=(n, 3, 3)))
    s = rng.uniform(smin, smax, (n, 3))
    cov = np.einsum("nij,nj,nkj->nik", q, s ** 2, q)
    covs = cov[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    return means.astype(np.float32), covs.astype(np.float32), rng.uniform(omin, omax, n).astype(np.float32)


def _agree(t, hit, rt, rhit, frac=0.995, rtol=1e-4):
    assert np.mean(hit == rhit) >= frac
    assert np.mean(np.isfinite(t) == np.isfinite(rt)) >= frac
    fin = np.isfinite(t) & np.isfinite(rt)
    ok = np.ones(t.shape, dtype=bool)
    ok[fin] = np.abs(t[fin] - rt[fin]) <= rtol * np.abs(rt[fin]) + 1e-6
    ok[np.isfinite(t) != np.isfinite(rt)] = False
    assert np.mean(ok) >= frac, np.mean(ok)
    return fin


def test_camera_rays_match_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    cams = I.orbit_cameras(3, seed=2)
    W, H = 37, 23
    rays = [torch.empty(3 * W * H, device="cuda") for _ in range(6)]
    ddf.ddf_camera_rays(cams, W, H, rays)
    torch.cuda.synchronize()
    got = np.stack([r.cpu().numpy() for r in rays], 1).reshape(3, H * W, 6)
    for v, cam in enumerate(cams):
        o, d = O.camera_rays(cam[0:3], cam[3:6], cam[6:9], float(cam[9]), W, H)
        assert np.allclose(got[v, :, :3], o, atol=1e-6)
        assert np.allclose(got[v, :, 3:], d, atol=2e-6)


def test_enter_box_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    rng = np.random.default_rng(7)
    n = 5000
    o = rng.uniform(-4, 4, (n, 3))
    d = rng.normal(size=(n, 3))
    d[: n // 2] = rng.uniform(-1, 1, (n // 2, 3)) - o[: n // 2]
    d[:10, 1] = 0.0                                   # axis-parallel components
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o, d = o.astype(np.float32), d.astype(np.float32)
    rays = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (*o.T, *d.T)]
    t = torch.from_numpy(np.where(np.arange(n) % 3 == 0, np.inf, 10.0).astype(np.float32)).cuda()
    t_in = torch.empty(n, device="cuda")
    ddf.ddf_enter_box(rays, t, t_in, n, 1.0)
    torch.cuda.synchronize()
    ro, re = O.enter_box(o.astype(np.float64), d.astype(np.float64))
    got = np.stack([r.cpu().numpy() for r in rays[:3]], 1)
    assert np.allclose(got, ro, atol=2e-6)
    assert np.allclose(t_in.cpu().numpy(), re, atol=2e-6)
    tt = t.cpu().numpy()
    fin = np.arange(n) % 3 != 0
    assert np.all(np.isinf(tt[~fin])) and np.allclose(tt[fin], 10.0 - re[fin], atol=2e-6)
    assert (re > 0).sum() > 1000
    with pytest.raises(ddf.DDFError):
        ddf.ddf_enter_box(rays, None, None, n, 0.0)


def test_random_gaussians_match_oracle(torch_cuda):
    """3,000 overlapping Gaussians of random shape and opacity, two views of
    48 x 40 pixels (a ragged row of tiles), every pixel against the oracle."""
    torch = torch_cuda
    means, covs, opac = _random_gaussians(3000, seed=1)
    cams = [_cam((0.5, 0.8, -3.5)), _cam((-3.0, 1.0, 1.5), fov_deg=55.0)]
    W, H = 48, 40
    t, hit = _render(torch, means, covs, opac, cams, W, H)
    for v, cam in enumerate(cams):
        rt, rhit = _oracle(means, covs, opac, cam, W, H)
        fin = _agree(t[v], hit[v], rt, rhit)
        assert fin.mean() > 0.5 and 0.1 < rhit.mean()      # the case is not trivial


def test_long_tile_lists_take_several_passes(torch_cuda):
    """6,000 faint Gaussians over one 16 x 16 tile: the list is three times
    the per-pass window, and most pixels are still open after the first
    window (every pixel gathers hundreds of contributions of alpha < 0.04)."""
    torch = torch_cuda
    rng = np.random.default_rng(3)
    W = H = 16
    cam = _cam((0.0, 0.0, -4.0))
    fp = H / (2 * np.tan(np.radians(20.0)))
    n = 6000
    z = rng.uniform(3.0, 5.0, n)                  # view depth (camera looks along +z)
    px = rng.uniform(-2, W + 1, n)
    py = rng.uniform(-2, H + 1, n)
    x = (px - (W - 1) / 2) * z / fp
    y = -(py - (H - 1) / 2) * z / fp
    means = np.stack([-x, y, z - 4.0], 1)          # right vector is -x for this camera
    sig = 1.5 * z / fp                             # 1.5 pixels
    covs = np.zeros((n, 6))
    covs[:, 0] = covs[:, 3] = covs[:, 5] = sig ** 2
    opac = np.full(n, 0.04)
    means, covs, opac = means.astype(np.float32), covs.astype(np.float32), opac.astype(np.float32)
    o_ref, d_ref = O.camera_rays(cam[0:3], cam[3:6], cam[6:9], float(cam[9]), W, H)
    mu, _, _ = O.gs_project(means.astype(np.float64), O.gs_cov_matrices(covs), cam[0:3], cam[3:6],
                            cam[6:9], float(cam[9]), W, H)
    assert np.allclose(mu[:, 0], px, atol=1e-3) and np.allclose(mu[:, 1], py, atol=1e-3)
    t, hit = _render(torch, means, covs, opac, [cam], W, H)
    rt, rhit = _oracle(means, covs, opac, cam, W, H)
    _agree(t[0], hit[0], rt, rhit)
    assert rhit.mean() > 0.9


def test_table_scene_at_full_size_sampled(torch_cuda):
    """The supervision workload's scene (60,000 surface Gaussians, four
    256 x 256 views): sampled pixels against the oracle, half of them on or
    beside the thin parts."""
    torch = torch_cuda
    scene, thin = I.table_scene()
    means, covs, opac = I.surface_gaussians(scene, 60000, seed=0)
    cams = I.orbit_cameras(4, seed=0)
    W = H = 256
    t, hit = _render(torch, means, covs, opac, cams, W, H)
    rng = np.random.default_rng(0)
    sub = I.Scene(scene.centers[:0], scene.radii[:0], scene.box_lo[thin], scene.box_hi[thin])
    for v, cam in enumerate(cams):
        o, d = O.camera_rays(cam[0:3], cam[3:6], cam[6:9], float(cam[9]), W, H)
        tt, th = O.cast_scene(sub, o, d)
        near = np.nonzero(th)[0]
        px = np.concatenate([rng.choice(near, 100), rng.choice(W * H, 100)])
        rt, rhit = _oracle(means, covs, opac, cam, W, H, pixels=px)
        _agree(t[v].ravel()[px], hit[v].ravel()[px], rt, rhit, frac=0.99)


def test_order_of_gaussians_does_not_matter(torch_cuda):
    """Permuting the Gaussians permutes only the list order before the sort,
    so the composite runs in the same order. Only Gaussians whose float32
    depths coincide exactly (a few among 2,000) can swap, which moves a
    result by a rounding at most."""
    torch = torch_cuda
    means, covs, opac = _random_gaussians(2000, seed=4)
    cams = [_cam((0.3, 0.5, -3.0))]
    t0, h0 = _render(torch, means, covs, opac, cams, 40, 40)
    p = np.random.default_rng(5).permutation(2000)
    t1, h1 = _render(torch, means[p], covs[p], opac[p], cams, 40, 40)
    assert np.array_equal(h0, h1)
    assert np.array_equal(np.isfinite(t0), np.isfinite(t1))
    fin = np.isfinite(t0)
    assert np.allclose(t0[fin], t1[fin], rtol=1e-6, atol=0)
    assert np.mean(t0[fin] == t1[fin]) > 0.99


def test_edge_cases(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    cam = _cam((0.0, 0.0, -4.0))
    W, H = 20, 18
    # no Gaussians: background everywhere
    e = np.zeros((0, 3), np.float32)
    t, hit = _render(torch, e, np.zeros((0, 6), np.float32), np.zeros(0, np.float32), [cam], W, H)
    assert np.all(np.isinf(t)) and not hit.any()
    # behind the camera, nearer than the near plane, and too faint: nothing drawn
    means = np.array([[0, 0, -5.0], [0, 0, -3.97], [0, 0, 0.0]], np.float32)
    covs = np.tile(np.array([0.04, 0, 0, 0.04, 0, 0.04], np.float32), (3, 1))
    opac = np.array([1.0, 1.0, 1.0 / 256.0], np.float32)
    t, hit = _render(torch, means, covs, opac, [cam], W, H)
    assert np.all(np.isinf(t)) and not hit.any()
    # one opaque Gaussian straight ahead: the centre pixels report its depth
    t, hit = _render(torch, means[2:], covs[2:], np.array([1.0], np.float32), [cam], W, H)
    rt, rhit = _oracle(means[2:], covs[2:], np.array([1.0], np.float32), cam, W, H)
    _agree(t[0], hit[0], rt, rhit, frac=1.0)
    assert hit[0].any()
    # bad arguments
    dt = torch.empty(W * H, device="cuda")
    dh = torch.empty(W * H, dtype=torch.uint8, device="cuda")
    dm = torch.zeros(3, device="cuda")
    with pytest.raises(ddf.DDFError):
        ddf.ddf_render_gs_depth(dm, dm, dm, -1, [cam], W, H, dt, dh)
    with pytest.raises(ddf.DDFError):
        ddf.ddf_render_gs_depth(dm, dm, dm, 1, [cam], 0, H, dt, dh)
    with pytest.raises(ddf.DDFError):
        ddf.ddf_render_gs_depth(dm, dm, dm, 1, [cam], W, H, None, dh)
    bad = cam.copy()
    bad[3:6] = bad[0:3]                                    # eye == target
    with pytest.raises(ddf.DDFError):
        ddf.ddf_render_gs_depth(dm, dm, dm, 1, [bad], W, H, dt, dh)
    bad = cam.copy()
    bad[9] = 0.0                                           # zero field of view
    with pytest.raises(ddf.DDFError):
        ddf.ddf_render_gs_depth(dm, dm, dm, 1, [bad], W, H, dt, dh)


def test_distill_from_a_pool(torch_cuda):
    """A hash-grid field trained from a fixed pool of exact camera-ray targets
    learns them (loss falls, hit flags on the pool mostly right) and the pool
    is left as it was."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    scene, thin = I.table_scene()
    sph = torch.from_numpy(np.concatenate([scene.centers, scene.radii[:, None]], 1)
                           .astype(np.float32).ravel()).cuda()
    box = torch.from_numpy(np.concatenate([scene.box_lo, scene.box_hi], 1)
                           .astype(np.float32).ravel()).cuda()
    cams = I.orbit_cameras(8, seed=1)
    W = H = 64
    n = 8 * W * H
    rays = [torch.empty(n, device="cuda") for _ in range(6)]
    ddf.ddf_camera_rays(cams, W, H, rays)
    ddf.ddf_enter_box(rays, None, None, n, 1.0)
    t = torch.empty(n, device="cuda")
    hit = torch.empty(n, dtype=torch.uint8, device="cuda")
    ddf.ddf_cast_scene(sph, len(scene.radii), box, len(scene.box_lo), rays, n, t, hit)
    snap = [r.clone() for r in rays] + [t.clone(), hit.clone()]
    m = ddf.DDF(4, 64, 2, precision="bf16", device=0, kind="hashgrid")
    m.load(I.hashgrid_blob(m.n_params, O.hashgrid_mlp_dims(), seed=0, table_scale=1e-4))
    losses = ddf.ddf_distill_pool(m.h, rays, t, hit, n, 400, 4096, 3e-3, 0.3, seed=3)
    assert np.all(np.isfinite(losses)) and losses[-50:].mean() < 0.5 * losses[:10].mean()
    for a, b in zip(snap, rays + [t, hit]):
        assert torch.equal(a, b)
    pt, pv = m.query(rays)
    torch.cuda.synchronize()
    acc = ((pv > 0.5).cpu() == (hit.cpu() > 0)).float().mean().item()
    assert acc > 0.9
    with pytest.raises(ddf.DDFError):
        ddf.ddf_distill_pool(m.h, rays, t, hit, 0, 1, 16, 3e-3)
