"""GPU tests of the sphere-tracing baseline (Sec. 4.4): the closed-form union
SDF, the SDF network, its regression gradient, and the device-driven sphere
tracer, against the FP64 oracle. Bounds as in test_gpu_parity (bf16 values)
and test_gpu_train (gradients)."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SDF_SMALL = (4, 128, 3)
SDF_PAPER = (10, 1280, 8)      # 63 -> 1280 x8 -> 1


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _dev(torch, arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _scene_dev(torch, scene):
    sph = np.concatenate([scene.centers, scene.radii[:, None]], 1).astype(np.float32).ravel()
    box = np.concatenate([scene.box_lo, scene.box_hi], 1).astype(np.float32).ravel()
    return torch.from_numpy(sph).cuda(), torch.from_numpy(box).cuda()


def _sdf(net, blob):
    from paper_2606_00817_gb300 import ddf
    m = ddf.DDF(*net, precision="bf16", kind="sdf")
    m.load(blob)
    return m


def test_union_sdf_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    scene = I.random_scene(32, 32, seed=0)
    p = I.uniform_points(5000, seed=51)
    sph, box = _scene_dev(torch, scene)
    out = torch.empty(5000, device="cuda")
    ddf.ddf_union_sdf(sph, 32, box, 32, _dev(torch, p.T), 5000, out)
    torch.cuda.synchronize()
    ref = O.union_sdf(scene, p.astype(np.float64))
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 2e-6


@pytest.mark.parametrize("net", [SDF_SMALL, SDF_PAPER])
def test_sdf_eval_matches_oracle(torch_cuda, net):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob_dims(I.sdf_layer_dims(*net))
    m = _sdf(net, blob)
    p = I.uniform_points(1037, seed=52)
    s = torch.empty(1037, device="cuda")
    ddf.ddf_sdf_eval(m.h, _dev(torch, p.T), 1037, s)
    torch.cuda.synchronize()
    ref = O.sdf_mlp(p.astype(np.float64), blob, *net, precision="bf16")
    err = np.abs(s.double().cpu().numpy() - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 2e-3 and err.mean() <= 2e-4
    with pytest.raises(ddf.DDFError):                      # ray queries refuse SDF fields
        m.query(_dev(torch, I.uniform_rays(8).soa()))


@pytest.mark.parametrize("net,B", [(SDF_SMALL, 2048), (SDF_PAPER, 2048)])
def test_sdf_gradient_matches_oracle(torch_cuda, net, B):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob_dims(I.sdf_layer_dims(*net))
    scene = I.random_scene(32, 32, seed=0)
    p = I.uniform_points(B, seed=53)
    s_t = O.union_sdf(scene, p.astype(np.float64)).astype(np.float32)
    m = _sdf(net, blob)
    loss = torch.zeros(1, device="cuda")
    ddf.ddf_sdf_compute_grad(m.h, _dev(torch, p.T), torch.from_numpy(s_t).cuda(), B, loss)
    g = ddf.ddf_get_grad(m.h, blob.size).astype(np.float64)
    L_emu, g_emu = O.sdf_train_grad(p.astype(np.float64), blob, *net, s_t, precision="bf16")
    _, g_ex = O.sdf_train_grad(p.astype(np.float64), blob, *net, s_t, precision="exact")
    assert abs(loss.item() - L_emu) <= 1e-4 * abs(L_emu)
    off = 0
    for fo, fi in I.sdf_layer_dims(*net):
        for n in (fo * fi, fo):
            a, b, c = g[off:off + n], g_emu[off:off + n], g_ex[off:off + n]
            off += n
            noise = np.linalg.norm(b - c)
            assert np.linalg.norm(a - b) <= 0.4 * noise + 1e-3 * np.linalg.norm(b)
            assert np.linalg.norm(a - c) <= 1.2 * noise + 1e-3 * np.linalg.norm(c)


def _marching_blob(net, level=0.12):
    """Xavier SDF weights with the output bias moved so the median value over
    the domain is `level`: rays then march many steps, and hit where the
    random field dips below eps."""
    blob = I.xavier_blob_dims(I.sdf_layer_dims(*net))
    s = O.sdf_mlp(I.uniform_points(2048, seed=55).astype(np.float64), blob, *net)
    blob[-1] += np.float32(level - np.median(s))
    return blob


def _trace_reference(rays, blob, net, max_steps, eps, t_max):
    sdf = lambda q: O.sdf_mlp(q, blob, *net, precision="bf16")
    return O.sphere_trace(sdf, rays.origins().astype(np.float64), rays.dirs().astype(np.float64),
                          max_steps=max_steps, eps=eps, t_max=t_max)


def _gpu_trace(torch, m, rays, max_steps, eps, t_max):
    from paper_2606_00817_gb300 import ddf
    n = rays.n
    t = torch.empty(n, device="cuda")
    hit = torch.empty(n, dtype=torch.uint8, device="cuda")
    steps = torch.empty(n, dtype=torch.int32, device="cuda")
    ddf.ddf_sphere_trace(m.h, _dev(torch, rays.soa()), n, max_steps, eps, t_max, t, hit, steps)
    torch.cuda.synchronize()
    return (t.double().cpu().numpy(), hit.cpu().numpy().astype(bool),
            steps.cpu().numpy().astype(np.int64))


def _plane_blob(net, normal=(0.36, -0.48, 0.8), c=-1.25, kappa=0.5):
    """Weights under which the SDF network computes the affine field
    s(p) = kappa (n . p - c) exactly in bf16 arithmetic: two first-layer units
    carry +-s from the raw-coordinate inputs, the hidden layers pass them on
    with unit weights and the head takes their difference. With kappa < 1 the
    field underestimates the distance to the plane n . p = c, so sphere tracing
    contracts towards it (a ray approaching at cosine a needs about
    log(eps) / log(1 - kappa a) steps) and a rounding difference in one step
    dies out in later ones instead of growing."""
    octaves, width, hidden = net
    dims = I.sdf_layer_dims(*net)
    n = np.asarray(normal, np.float32)
    parts = []
    for li, (fo, fi) in enumerate(dims):
        w = np.zeros((fo, fi), np.float32)
        b = np.zeros(fo, np.float32)
        if li == 0:
            w[0, :3], b[0] = kappa * n, -kappa * c
            w[1, :3], b[1] = -kappa * n, kappa * c
        elif li < len(dims) - 1:
            w[0, 0] = w[1, 1] = 1.0
        else:
            w[0, 0], w[0, 1] = 1.0, -1.0
        parts += [w.ravel(), b]
    return np.concatenate(parts)


def _trace_bound(t, tr, steps, hit, sr, hr, frac, tol):
    same = (steps == sr) & (hit == hr)
    assert same.mean() >= frac, same.mean()
    err = np.abs(t[same] - tr[same]) / np.maximum(1.0, tr[same])
    assert err.max() <= tol, err.max()
    return same


def test_sphere_trace_plane_matches_oracle(torch_cuda):
    """Tracing the affine field of _plane_blob (about half the rays approach
    the plane; glancing ones run into the 64-step limit): per-ray hit flag,
    step count and distance follow the oracle's trace of the same network.
    Both sides round each sample point to bf16 when encoding it; where the
    GPU's fp32 t and the oracle's fp64 t straddle a bf16 rounding boundary
    the field value moves by at most kappa |n|_inf 2^-8 (|p| < 2), and the
    contraction keeps the distance within a few such moves, so at most a
    handful of rays take a different step count."""
    torch = torch_cuda
    net = SDF_SMALL
    blob = _plane_blob(net)
    m = _sdf(net, blob)
    rays = I.uniform_rays(3000, seed=54)
    t, hit, steps = _gpu_trace(torch, m, rays, 64, 1e-3, 4.0)
    tr, hr, sr = _trace_reference(rays, blob, net, 64, 1e-3, 4.0)
    _trace_bound(t, tr, steps, hit, sr, hr, 0.995, 1e-2)
    assert 0.3 < hit.mean() < 0.7 and (steps == 64).any() and steps.mean() > 4.0
    assert steps.min() >= 1 and steps.max() <= 64


def test_sphere_trace_matches_oracle(torch_cuda):
    """A random (Xavier, output level 0.12) SDF network: the tracer follows
    the oracle's trace of the same bf16-emulated network ray by ray. Such a
    field is not 1-Lipschitz, so the marching map t -> t + s(o + t d) can
    stretch a one-ulp difference in a step's value step after step, and a
    value within rounding of eps can end a ray one step apart: most rays
    agree to float32 rounding, a small tail further."""
    torch = torch_cuda
    net = SDF_SMALL
    blob = _marching_blob(net)
    m = _sdf(net, blob)
    rays = I.uniform_rays(3000, seed=54)
    t, hit, steps = _gpu_trace(torch, m, rays, 64, 1e-3, 4.0)
    tr, hr, sr = _trace_reference(rays, blob, net, 64, 1e-3, 4.0)
    same = _trace_bound(t, tr, steps, hit, sr, hr, 0.98, 0.1)
    err = np.abs(t[same] - tr[same]) / np.maximum(1.0, tr[same])
    assert np.quantile(err, 0.95) <= 1e-5 and np.quantile(err, 0.99) <= 5e-3
    assert 1.0 < steps.mean() < 64 and 0.05 < hit.mean() < 0.99   # non-degenerate traces
    assert steps.max() <= 64 and steps.min() >= 1


def test_full_size_trace_sampled(torch_cuda):
    """1,048,576 one-bounce rays on the 64-sphere scene through the 8 x 1280
    SDF network carrying the affine field of _plane_blob, at most 128 steps,
    eps 1e-3, t_max 4: 256 sampled rays against the oracle's trace of the
    same network."""
    torch = torch_cuda
    net = SDF_PAPER
    blob = _plane_blob(net)
    scene = I.random_scene(64, 0, seed=0)
    m = _sdf(net, blob)
    rays = I.bounce_rays(scene, 1_048_576, seed=0)
    t, hit, steps = _gpu_trace(torch, m, rays, 128, 1e-3, 4.0)
    assert np.all(steps >= 1) and np.all(steps <= 128) and np.all(np.isfinite(t))
    assert steps.mean() > 4.0 and 0.1 < hit.mean() < 0.9
    idx = np.sort(np.random.default_rng(3).choice(rays.n, 256, replace=False))
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    tr, hr, sr = _trace_reference(sub, blob, net, 128, 1e-3, 4.0)
    _trace_bound(t[idx], tr, steps[idx], hit[idx], sr, hr, 0.98, 1e-2)


def test_sdf_distillation_and_full_size_trace(torch_cuda):
    """Distil the 8 x 1280 SDF network from the union SDF of the 64-sphere
    scene (65,536 points per step; the loss falls), then trace 1,048,576
    one-bounce rays (at most 128 steps, eps 1e-3, t_max 4). The distilled
    weights come from the GPU, so the oracle does not see them: instead 48
    sampled rays traced again in a batch of their own must give bit-identical
    results (each ray's trace depends on nothing but its own row)."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net = SDF_PAPER
    blob = I.xavier_blob_dims(I.sdf_layer_dims(*net))
    scene = I.random_scene(64, 0, seed=0)
    sph, box = _scene_dev(torch, scene)
    m = _sdf(net, blob)
    B = 65536
    loss = torch.zeros(1, device="cuda")
    losses = []
    for step in range(40):
        p = I.uniform_points(B, seed=200 + step)
        dp = _dev(torch, p.T)
        s_t = torch.empty(B, device="cuda")
        ddf.ddf_union_sdf(sph, 64, box, 0, dp, B, s_t)
        ddf.ddf_sdf_train_step(m.h, dp, s_t, B, 1e-3, loss)
        losses.append(loss.item())
    assert np.mean(losses[-5:]) < 0.7 * np.mean(losses[:3]), losses
    rays = I.bounce_rays(scene, 1_048_576, seed=0)
    t, hit, steps = _gpu_trace(torch, m, rays, 128, 1e-3, 4.0)
    assert np.all(steps >= 1) and np.all(steps <= 128) and np.all(np.isfinite(t))
    assert steps.mean() > 2.0
    # the trained weights are the GPU's own product: sample rays and retrace
    # them on the GPU with the same weights, one ray per call position, and
    # check the full-batch result does not depend on which rays share a batch
    idx = np.sort(np.random.default_rng(2).choice(rays.n, 48, replace=False))
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    t2, hit2, steps2 = _gpu_trace(torch, m, sub, 128, 1e-3, 4.0)
    assert np.array_equal(hit2, hit[idx]) and np.array_equal(steps2, steps[idx])
    assert np.array_equal(t2, t[idx])
    assert ddf.ddf_check_status(m.h) == 0
