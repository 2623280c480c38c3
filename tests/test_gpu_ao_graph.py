"""GPU tests: FP8 activation-scale calibration, ragged ambient occlusion and
CUDA-graph replay, against the FP64 oracle (bounds as in test_gpu_parity)."""
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


def _model(net, prec, blob, scales=None):
    from paper_2606_00817_gb300 import ddf
    m = ddf.DDF(*net, precision=prec)
    m.load(blob, scales if prec == "fp8" else None)
    return m


def _oracle_amax(rays, blob, net):
    layers = O.split_blob(blob, O.ddf_dims(*net))
    _, _, acts = O.mlp_forward(O.encode(rays.origins(), rays.dirs(), net[0]), layers, keep=True)
    return np.array([np.max(a) for a in acts[1:net[2]]])


@pytest.mark.parametrize("net", [SMALL, PAPER])
def test_calibration_matches_oracle(torch_cuda, net):
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*net))
    cal = I.uniform_rays(4096, seed=31)
    m = _model(net, "fp8", blob)
    amax, sc = ddf.ddf_calibrate_fp8(m.h, _dev(torch_cuda, cal.soa()), cal.n)
    ref = _oracle_amax(cal, blob, net)
    # the calibration pass runs in bf16: amax within a few bf16 ulps of the exact one
    assert np.all(np.abs(amax - ref) <= 2e-2 * ref), (amax, ref)
    ref_sc = np.array(O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *net))
    near_edge = np.abs(np.log2(ref / 448.0) - np.round(np.log2(ref / 448.0))) < 0.03
    assert np.all((sc == ref_sc) | near_edge)
    # the handle now answers e4m3 queries with those scales
    rays = I.uniform_rays(777, seed=32)
    t, v = m.query(_dev(torch_cuda, rays.soa()))
    torch_cuda.cuda.synchronize()
    emu = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net, precision="fp8",
                        act_scales=[float(x) for x in sc])
    err = np.abs(t.double().cpu().numpy() - emu["t"]) / np.maximum(1.0, np.abs(emu["t"]))
    assert err.max() <= 1e-2 and err.mean() <= 1e-3


def _ao_reference(rays, offsets, blob, net, prec, scales):
    emu = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net, precision=prec, act_scales=scales)
    z1 = emu["z"][:, 1]
    hard, soft = O.ambient_occlusion(z1 > 0, emu["vis"], offsets)
    near = np.abs(z1) < 1e-3
    tie = np.array([near[offsets[p]:offsets[p + 1]].sum() for p in range(len(offsets) - 1)])
    cnt = np.diff(offsets)
    return hard, soft, tie / np.maximum(cnt, 1)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_ao_matches_oracle(torch_cuda, prec):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*SMALL))
    scene = I.random_scene(64, 0, seed=0)
    rays, offsets = I.ao_rays(scene, 300, seed=33)
    # splice in empty sets: points 0 and 150 get no rays
    offsets = offsets.astype(np.int64)
    cnt = np.diff(offsets)
    keep = np.ones(rays.n, bool)
    keep[offsets[0]:offsets[1]] = False
    keep[offsets[150]:offsets[151]] = False
    cnt[0] = 0
    cnt[150] = 0
    offsets = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    rays = I.Rays(*[a[keep] for a in rays.soa()])
    sc = O.calibrate_act_scales(rays.origins(), rays.dirs(), blob, *SMALL)
    m = _model(SMALL, prec, blob, sc)
    ddf.ddf_set_chunk_rays(m.h, 1024)   # ~10 chunks: outputs of every chunk land in place
    d_off = torch.from_numpy(offsets).cuda()
    hard = torch.empty(300, device="cuda")
    soft = torch.empty(300, device="cuda")
    ddf.ddf_query_ao(m.h, _dev(torch, rays.soa()), rays.n, d_off, 300, hard, soft)
    torch.cuda.synchronize()
    h_ref, s_ref, tie_frac = _ao_reference(rays, offsets, blob, SMALL, prec, sc)
    hard, soft = hard.double().cpu().numpy(), soft.double().cpu().numpy()
    assert hard[0] == 1.0 and soft[0] == 1.0 and hard[150] == 1.0
    assert np.all(np.abs(hard - h_ref) <= tie_frac + 1e-6)
    assert np.abs(soft - s_ref).max() <= (2e-3 if prec == "bf16" else 1e-2)
    assert ddf.ddf_check_status(m.h) == 0


def test_graph_mode_replays_bitwise(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    light = (3.0, 3.0, 3.0)
    r1 = I.uniform_rays(3001, seed=34)
    r2 = I.uniform_rays(3001, seed=35)
    m = _model(PAPER, "bf16", blob)
    ddf.ddf_set_chunk_rays(m.h, 1024)                    # several chunks inside one graph
    dev = _dev(torch, r1.soa())
    t, v = torch.empty(3001, device="cuda"), torch.empty(3001, device="cuda")
    occ = torch.empty(3001, dtype=torch.uint8, device="cuda")
    ddf.ddf_query_shadow(m.h, dev, 3001, light, t, v, occ)
    torch.cuda.synchronize()
    eager1 = (t.clone(), v.clone(), occ.clone())
    for a, b in zip(dev, _dev(torch, r2.soa())):
        a.copy_(b)
    ddf.ddf_query_shadow(m.h, dev, 3001, light, t, v, occ)
    torch.cuda.synchronize()
    eager2 = (t.clone(), v.clone(), occ.clone())
    ddf.ddf_set_graph_mode(m.h, True)
    for rep in range(2):                                 # capture, then replay
        for a, b in zip(dev, _dev(torch, r1.soa())):
            a.copy_(b)
        ddf.ddf_query_shadow(m.h, dev, 3001, light, t, v, occ)
        torch.cuda.synchronize()
        assert all(torch.equal(x, y) for x, y in zip((t, v, occ), eager1)), rep
        for a, b in zip(dev, _dev(torch, r2.soa())):  # same pointers, new data
            a.copy_(b)
        ddf.ddf_query_shadow(m.h, dev, 3001, light, t, v, occ)
        torch.cuda.synchronize()
        assert all(torch.equal(x, y) for x, y in zip((t, v, occ), eager2)), rep
    ddf.ddf_set_tile(m.h, (256, 4, 1, 1), 0)           # drops the cached graphs
    ddf.ddf_query_shadow(m.h, dev, 3001, light, t, v, occ)
    torch.cuda.synchronize()
    assert torch.allclose(t, eager2[0], atol=1e-5) and torch.allclose(v, eager2[1], atol=1e-5)
    assert ddf.ddf_check_status(m.h) == 0


def test_full_size_ragged_ao_fp8_graph(torch_cuda):
    """1024 x 1024 shading points, 4..64 cosine-weighted directions each
    (about 35.7M rays), e4m3 paper-sized field, one graph launch; 48 sampled
    points against the oracle, and graph replay against eager, bitwise."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*PAPER))
    scene = I.random_scene(64, 0, seed=0)
    rays, offsets = I.ao_rays(scene, 1024 * 1024, seed=0)
    assert 30e6 < rays.n < 40e6
    cal = rays.slice(0, 8192)
    sc = O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *PAPER)
    m = _model(PAPER, "fp8", blob, sc)
    dev = _dev(torch, rays.soa())
    d_off = torch.from_numpy(offsets).cuda()
    P = 1024 * 1024
    hard = torch.empty(P, device="cuda")
    soft = torch.empty(P, device="cuda")
    ddf.ddf_query_ao(m.h, dev, rays.n, d_off, P, hard, soft)
    torch.cuda.synchronize()
    eager = (hard.clone(), soft.clone())
    ddf.ddf_set_graph_mode(m.h, True)
    for _ in range(2):
        hard.fill_(-1)
        ddf.ddf_query_ao(m.h, dev, rays.n, d_off, P, hard, soft)
        torch.cuda.synchronize()
        assert torch.equal(hard, eager[0]) and torch.equal(soft, eager[1])
    pts = np.sort(np.random.default_rng(1).choice(P, 48, replace=False))
    pts[-1] = P - 1
    idx = np.concatenate([np.arange(offsets[p], offsets[p + 1]) for p in pts])
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    sub_off = np.concatenate([[0], np.cumsum(np.diff(offsets)[pts])]).astype(np.int32)
    h_ref, s_ref, tie = _ao_reference(sub, sub_off, blob, PAPER, "fp8", sc)
    g_h = hard.double().cpu().numpy()[pts]
    g_s = soft.double().cpu().numpy()[pts]
    assert np.all(np.abs(g_h - h_ref) <= tie + 1e-6)
    assert np.abs(g_s - s_ref).max() <= 1e-2
    assert ddf.ddf_check_status(m.h) == 0
