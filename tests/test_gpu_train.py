"""GPU tests of the distillation step: the exact analytic caster, the
gradient, Adam, and a full-size (65,536-ray, 8 x 1280) training run.

Gradient bounds, per weight/bias block, in L2 norm. Let
  noise = |g_emu - g_exact|  (what bf16 rounding alone costs: the oracle
          emulating the step's bf16 roundings against exact float64)
Then the GPU gradient must satisfy
  |g_gpu - g_emu|   <= 0.4 noise + 1e-3 |g_emu|
  |g_gpu - g_exact| <= 1.2 noise + 1e-3 |g_exact|
i.e. it is as good as the emulated arithmetic and tracks its particular
rounding pattern. It cannot track it exactly: the tensor cores accumulate in
FP32 and the oracle in float64, so a bf16 rounding of an activation or of a
back-propagated gradient can fall the other way, and such differences
compound through the layers (measured on GB300: the ratio stays near 0.25-0.29
for 8 x 1280, and below 0.01 for 4 x 128)."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMALL = (6, 128, 4)
PAPER = (10, 1280, 8)


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


def _gpu_cast(torch, scene, rays):
    from paper_2606_00817_gb300 import ddf
    sph, box = _scene_dev(torch, scene)
    t = torch.empty(rays.n, device="cuda")
    hit = torch.empty(rays.n, dtype=torch.uint8, device="cuda")
    ddf.ddf_cast_scene(sph, len(scene.radii), box, len(scene.box_lo), _dev(torch, rays.soa()),
                       rays.n, t, hit)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64), hit.cpu().numpy().astype(bool)


def test_caster_matches_oracle(torch_cuda):
    scene = I.random_scene(32, 32, seed=0)
    rays = I.uniform_rays(20000, seed=41)
    t, hit = _gpu_cast(torch_cuda, scene, rays)
    t_ref, hit_ref = O.cast_scene(scene, rays.origins(), rays.dirs())
    assert hit_ref.mean() > 0.3
    assert np.mean(hit == hit_ref) > 0.999
    both = hit & hit_ref
    assert np.all(np.abs(t[both] - t_ref[both]) <= 1e-4 * np.maximum(1.0, t_ref[both]))
    assert np.all(np.isinf(t[~hit]))


def _blocks(g, net):
    out, off = [], 0
    for fo, fi in O.ddf_dims(*net):
        out.append(g[off:off + fo * fi])
        off += fo * fi
        out.append(g[off:off + fo])
        off += fo
    return out


def _batch(net, B, seed):
    scene = I.random_scene(32, 32, seed=0)
    rays = I.uniform_rays(B, seed=seed)
    t_ref, hit_ref = O.cast_scene(scene, rays.origins(), rays.dirs())
    return rays, t_ref.astype(np.float32), hit_ref.astype(np.uint8)


@pytest.mark.parametrize("net,B", [(SMALL, 4096), (PAPER, 4096)])
def test_gradient_matches_oracle(torch_cuda, net, B):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*net))
    rays, tt, y = _batch(net, B, seed=42)
    m = ddf.DDF(*net, precision="bf16")
    m.load(blob)
    loss = torch.zeros(1, device="cuda")
    ddf.ddf_compute_grad(m.h, _dev(torch, rays.soa()), torch.from_numpy(tt).cuda(),
                         torch.from_numpy(y).cuda(), B, loss)
    g = ddf.ddf_get_grad(m.h, blob.size).astype(np.float64)
    L_emu, g_emu = O.train_grad(rays.origins(), rays.dirs(), blob, *net, tt, y, precision="bf16")
    L_ex, g_ex = O.ddf_loss_grad(rays.origins(), rays.dirs(), blob, *net, tt, y)
    assert abs(loss.item() - L_emu) <= 1e-4 * abs(L_emu)
    for i, (a, b, c) in enumerate(zip(_blocks(g, net), _blocks(g_emu, net), _blocks(g_ex, net))):
        noise = np.linalg.norm(b - c)
        assert np.linalg.norm(a - b) <= 0.4 * noise + 1e-3 * np.linalg.norm(b), i
        assert np.linalg.norm(a - c) <= 1.2 * noise + 1e-3 * np.linalg.norm(c), i
    assert ddf.ddf_check_status(m.h) == 0


def test_adam_step_matches_oracle_update(torch_cuda):
    """First Adam step from zero moments: w1 = w0 - lr g / (|g| + eps) per
    parameter, with g the oracle's own gradient, wherever |g| is not tiny."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net, B, lr = SMALL, 4096, 1e-3
    blob = I.xavier_blob(I.NetShape(*net))
    rays, tt, y = _batch(net, B, seed=43)
    m = ddf.DDF(*net, precision="bf16")
    m.load(blob)
    ddf.ddf_train_step(m.h, _dev(torch, rays.soa()), torch.from_numpy(tt).cuda(),
                       torch.from_numpy(y).cuda(), B, lr)
    w1 = ddf.ddf_get_weights(m.h, blob.size).astype(np.float64)
    _, g = O.train_grad(rays.origins(), rays.dirs(), blob, *net, tt, y, precision="bf16")
    w_ref, _, _ = O.adam_step(blob.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    agree = np.abs(w1 - w_ref) <= 2e-6
    assert big.mean() > 0.2
    assert agree[big].mean() > 0.99
    # queries now use the updated weights
    t_after, _ = m.query(_dev(torch, rays.slice(0, 256).soa()))
    emu = O.ddf_forward(rays.origins()[:256], rays.dirs()[:256], w_ref.astype(np.float32), *net,
                        precision="bf16")
    err = np.abs(t_after.double().cpu().numpy() - emu["t"])
    assert np.median(err) < 5e-3


def test_full_size_distillation_lowers_the_loss(torch_cuda):
    """65,536 rays per batch (origins in [-1,1]^3, uniform directions), targets
    from the GPU caster on 32 spheres + 32 boxes, 8 x 1280 field, Adam 1e-3:
    20 steps lower the loss and keep every weight finite."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    scene = I.random_scene(32, 32, seed=0)
    m = ddf.DDF(*PAPER, precision="bf16")
    m.load(blob)
    B = 65536
    losses = []
    loss = torch.zeros(1, device="cuda")
    for step in range(20):
        rays = I.uniform_rays(B, seed=100 + step)
        dev = _dev(torch, rays.soa())
        sph, box = _scene_dev(torch, scene)
        tt = torch.empty(B, device="cuda")
        hit = torch.empty(B, dtype=torch.uint8, device="cuda")
        ddf.ddf_cast_scene(sph, 32, box, 32, dev, B, tt, hit)
        ddf.ddf_train_step(m.h, dev, tt, hit, B, 1e-3, loss)
        losses.append(loss.item())
    assert all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.8 * np.mean(losses[:3]), losses
    w = ddf.ddf_get_weights(m.h, blob.size)
    assert np.all(np.isfinite(w)) and not np.array_equal(w, blob)
    assert ddf.ddf_check_status(m.h) == 0
