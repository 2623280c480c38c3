"""GPU tests of the application images (Sec. 3.3): shadow and ambient
occlusion rendered with the exact caster match the oracle pixel by pixel (up
to float32 decisions at silhouettes and grazing rays), and rendered with a
distilled hash-grid field they approach the exact images (PSNR)."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CAM = (2.5, 1.8, -3.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, np.radians(50.0))
LIGHT = (3.0, 3.0, 3.0)


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _scene(torch, ns=32, nb=32):
    scene = I.random_scene(ns, nb, seed=0)
    sph = torch.from_numpy(np.concatenate([scene.centers, scene.radii[:, None]], 1)
                           .astype(np.float32).ravel()).cuda()
    box = torch.from_numpy(np.concatenate([scene.box_lo, scene.box_hi], 1)
                           .astype(np.float32).ravel()).cuda()
    return scene, sph, box


def _render(torch, ddf, h, sph, box, W, H, k, seed=5, cam=CAM):
    sh = torch.empty(H * W, device="cuda")
    ao = torch.empty(H * W, device="cuda")
    ddf.ddf_render_gi(h, sph, 32, box, 32, cam, W, H, LIGHT, k, seed, sh, ao)
    torch.cuda.synchronize()
    return sh.cpu().numpy().reshape(H, W).astype(np.float64), ao.cpu().numpy().reshape(H, W).astype(np.float64)


def test_exact_render_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    scene, sph, box = _scene(torch)
    W, H, k = 96, 72, 8
    sh, ao = _render(torch, ddf, None, sph, box, W, H, k)
    rs, ra = O.gi_images(scene, CAM[0:3], CAM[3:6], CAM[6:9], CAM[9], W, H, LIGHT, k, 5)
    fg_g, fg_r = sh >= 0, rs >= 0
    assert np.mean(fg_g == fg_r) >= 0.995 and 0.2 < fg_r.mean() < 0.95
    both = fg_g & fg_r
    assert np.mean(sh[both] == rs[both]) >= 0.99
    assert 0.05 < np.mean(rs[both] == 0) < 0.95                 # shadows exist, not everywhere
    assert np.mean(ao[both] == ra[both]) >= 0.97
    assert np.abs(ao[both] - ra[both]).mean() <= 0.01
    assert np.all(ao[~fg_g] == -1) and np.all(sh[~fg_g] == -1)


def test_render_of_empty_view_is_background(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    _, sph, box = _scene(torch)
    away = (0.0, 0.0, -3.0, 0.0, 0.0, -10.0, 0.0, 1.0, 0.0, np.radians(30.0))   # looking away
    sh, ao = _render(torch, ddf, None, sph, box, 16, 8, 4, cam=away)
    assert np.all(sh == -1) and np.all(ao == -1)


def _psnr(a, b, mask):
    mse = np.mean((a[mask] - b[mask]) ** 2)
    return 10 * np.log10(1.0 / max(mse, 1e-12))


def test_field_render_approaches_exact(torch_cuda):
    """A hash-grid field distilled for 3,000 steps (the paper's recipe)
    renders shadow and AO images whose PSNR against the exact images, over
    foreground pixels, is above 10 dB and 14.5 dB (measured on GB300 on this
    64-primitive scene with 16 AO rays: at this 128 x 96 size, with surface
    rays drawn by primitive, 11.1-11.4 and 16.2 dB at 3,000 steps and 12.3
    and 19.0 dB at 30,000; the benchmark's 512 x 512 images with surface
    rays drawn by area, 10.7-10.8 and 16.3 dB at 3,000), and its images use
    the exact primary hits (same foreground)."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    scene, sph, box = _scene(torch)
    n = ddf.ddf_param_count(ddf.make_config(4, 64, 2, kind="hashgrid"))
    m = ddf.DDF(4, 64, 2, precision="bf16", kind="hashgrid")
    m.load(I.hashgrid_blob(n, O.hashgrid_mlp_dims(), seed=0, table_scale=1e-4))
    ddf.ddf_distill(m.h, sph, 32, box, 32, 3000, 16384, 3e-3, 0.5, 0.3, seed=1)
    W, H, k = 128, 96, 16
    fs, fa = _render(torch, ddf, m.h, sph, box, W, H, k)
    es, ea = _render(torch, ddf, None, sph, box, W, H, k)
    fg = es >= 0
    assert np.array_equal(fs >= 0, fg)
    ps, pa = _psnr(fs, es, fg), _psnr(fa, ea, fg)
    assert ps > 10.0 and pa > 14.5, (ps, pa)
    assert ddf.ddf_check_status(m.h) == 0


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_field_render_matches_oracle(torch_cuda, prec):
    """The images with every secondary ray answered by a hash-grid field (a
    seeded random field, so that hits, misses and distances vary) against
    the oracle answering the same rays with the same blob
    (gi_images(field_blob=...)), pixel by pixel. Decisions within reach of
    float32 and bf16 rounding (|z1| or |t - light distance| below the
    margin) may differ; so may pixels whose primary hit is decided
    differently in float32 (silhouettes, box edges), as in the exact render."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    scene, sph, box = _scene(torch)
    m = ddf.DDF(4, 64, 2, precision=prec, kind="hashgrid")
    blob = I.hashgrid_blob(m.n_params, O.hashgrid_mlp_dims(), seed=3, table_scale=0.5)
    W, H, k = 96, 72, 6
    args = (scene, CAM[0:3], CAM[3:6], CAM[6:9], CAM[9], W, H, LIGHT, k, 5)
    fp = "exact" if prec == "fp32" else "bf16"
    # centre the visibility logit: the head bias b1 moves every z1 alike, so
    # shifting it by the median z1 of the shadow rays makes half of them hit
    _, _, det = O.gi_images(*args, field_blob=blob, field_precision=fp, detail=True)
    blob[-1] -= np.float32(np.median(det["shadow_z1"]))
    m.load(blob)
    sh, ao = _render(torch, ddf, m.h, sph, box, W, H, k)
    rs, ra, det = O.gi_images(*args, field_blob=blob, field_precision=fp, detail=True)
    margin = 1e-2 if prec == "fp32" else 5e-2
    px = det["pixels"]
    sh_g, ao_g = sh.ravel()[px], ao.ravel()[px]
    assert np.mean(sh_g >= 0) > 0.995                          # the same foreground
    clear = (np.abs(det["shadow_z1"]) > margin) & \
            (np.abs(det["shadow_t"] - det["shadow_dist"]) > margin * det["shadow_dist"])
    assert clear.mean() > 0.7
    assert 0.2 < np.mean(rs.ravel()[px] == 0) < 0.8             # the field shadows some pixels
    assert np.mean(sh_g[clear] == rs.ravel()[px][clear]) >= 0.995
    ties = np.sum(np.abs(det["ao_z1"]) <= margin, axis=1)
    ok = np.abs(ao_g - ra.ravel()[px]) <= ties / k + 1e-6
    assert np.mean(ok) >= 0.99
    assert ddf.ddf_check_status(m.h) == 0
