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


# ------------------------------------------- mixed shadow + ragged AO batch

def _ao_set(scene, P, seed, empty=(0,)):
    """A ragged AO batch of P points with the listed points given no rays."""
    rays, offsets = I.ao_rays(scene, P, seed=seed)
    cnt = np.diff(offsets.astype(np.int64))
    keep = np.ones(rays.n, bool)
    for p in empty:
        keep[offsets[p]:offsets[p + 1]] = False
        cnt[p] = 0
    offsets = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    return I.Rays(*[a[keep] for a in rays.soa()]), offsets


def _outs(torch, ns, P):
    return (torch.full((max(ns, 1),), -7.0, device="cuda"), torch.full((max(ns, 1),), -7.0, device="cuda"),
            torch.full((max(ns, 1),), 9, dtype=torch.uint8, device="cuda"),
            torch.full((P,), -7.0, device="cuda"), torch.full((P,), -7.0, device="cuda"))


def _separate(torch, ddf, m, sdev, ns, light, adev, na, d_off, P):
    t, v, occ, hard, soft = _outs(torch, ns, P)
    if ns:
        ddf.ddf_query_shadow(m.h, sdev, ns, light, t, v, occ)
    ddf.ddf_query_ao(m.h, adev, na, d_off, P, hard, soft)
    torch.cuda.synchronize()
    return t[:ns].clone(), v[:ns].clone(), occ[:ns].clone(), hard.clone(), soft.clone()


def _mixed(torch, ddf, m, sdev, ns, light, adev, na, d_off, P, outs):
    t, v, occ, hard, soft = outs
    for x in outs:
        x.fill_(7)
    ddf.ddf_query_mixed(m.h, sdev if ns else None, ns, light, t, v, occ, adev if na else None, na,
                        d_off, P, hard, soft)
    torch.cuda.synchronize()
    return t[:ns].clone(), v[:ns].clone(), occ[:ns].clone(), hard.clone(), soft.clone()


@pytest.mark.parametrize("net,prec,kind", [(SMALL, "bf16", "ray"), (PAPER, "fp8", "ray"),
                                           (SMALL, "fp32", "ray"), (None, "bf16", "hashgrid")])
@pytest.mark.parametrize("ns", [3001, 1024, 0])
def test_mixed_query_equals_the_separate_queries(torch_cuda, net, prec, kind, ns):
    """Shadow rays and a ragged AO batch in one query: 1024-ray chunks put the
    join inside a chunk (3001 shadow rays), on a chunk boundary (1024) or at
    the start (no shadow rays); every output equals, bit for bit, the one of
    the separate ddf_query_shadow and ddf_query_ao calls, in eager mode and in
    graph mode (one capture, then replays with new data behind the same
    pointers)."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    light = (3.0, 3.0, 3.0)
    scene = I.random_scene(64, 0, seed=0)
    P = 200
    data = []
    for k in range(3):
        sr = I.shadow_rays(scene, max(ns, 1), light, seed=36 + 2 * k)
        ar, offsets = _ao_set(scene, P, seed=37, empty=(0, 99))      # one layout of the sets
        if k:
            ar = I.Rays(*[a + np.float32(1e-3 * k) for a in ar.soa()])  # new data, same sizes
        data.append((sr, ar))
    na = data[0][1].n
    if kind == "hashgrid":
        m = ddf.DDF(4, 64, 2, precision=prec, kind="hashgrid")
        m.load(I.hashgrid_blob(m.n_params, O.hashgrid_mlp_dims(), seed=0))
    else:
        blob = I.xavier_blob(I.NetShape(*net))
        ar0 = data[0][1]
        sc = O.calibrate_act_scales(ar0.origins(), ar0.dirs(), blob, *net) if prec == "fp8" else None
        m = _model(net, prec, blob, sc)
        ddf.ddf_set_chunk_rays(m.h, 1024)
    sdev, adev = _dev(torch, data[0][0].soa()), _dev(torch, data[0][1].soa())
    d_off = torch.from_numpy(offsets).cuda()

    def load(k):
        for a, b in zip(sdev, _dev(torch, data[k][0].soa())):
            a.copy_(b)
        for a, b in zip(adev, _dev(torch, data[k][1].soa())):
            a.copy_(b)

    refs = []
    for k in range(3):
        load(k)
        refs.append(_separate(torch, ddf, m, sdev, ns, light, adev, na, d_off, P))
    outs = _outs(torch, ns, P)
    load(0)
    got = _mixed(torch, ddf, m, sdev, ns, light, adev, na, d_off, P, outs)
    assert all(torch.equal(a, b) for a, b in zip(got, refs[0]))
    assert got[3][0] == 1.0 and got[3][99] == 1.0
    if kind == "ray" and net == SMALL:
        # and directly against the oracle's shadow decision and AO
        sr, ar = data[0]
        emu_prec = "exact" if prec == "fp32" else prec
        h_ref, s_ref, tie = _ao_reference(ar, offsets, blob, net, emu_prec, sc)
        assert np.all(np.abs(got[3].double().cpu().numpy() - h_ref) <= tie + 1e-6)
        assert np.abs(got[4].double().cpu().numpy() - s_ref).max() <= 2e-3
        if ns:
            emu = O.ddf_forward(sr.origins(), sr.dirs(), blob, *net, precision=emu_prec)
            occ_ref = O.shadow(emu["t"], emu["z"][:, 1], sr.origins(), light)
            dist = np.linalg.norm(np.array(light) - sr.origins().astype(np.float64), axis=1)
            clear = (np.abs(emu["z"][:, 1]) > 1e-2) & (np.abs(emu["t"] - dist) > 1e-2)
            assert clear.mean() > 0.8
            occ = got[2].cpu().numpy().astype(bool)
            assert np.array_equal(occ[clear], occ_ref[clear])
    ddf.ddf_set_graph_mode(m.h, True)
    for k in (0, 1, 2, 1):
        load(k)
        got = _mixed(torch, ddf, m, sdev, ns, light, adev, na, d_off, P, outs)
        assert all(torch.equal(a, b) for a, b in zip(got, refs[k])), k
    assert ddf.ddf_check_status(m.h) == 0


def test_mixed_query_argument_errors(torch_cuda):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    m = _model(SMALL, "bf16", I.xavier_blob(I.NetShape(*SMALL)))
    r = [torch.zeros(8, device="cuda") for _ in range(6)]
    off = torch.tensor([0, 4, 8], dtype=torch.int32, device="cuda")
    out = torch.empty(8, device="cuda")
    occ = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(ddf.DDFError):       # shadow rays without outputs
        ddf.ddf_query_mixed(m.h, r, 8, (3, 3, 3), None, None, None, r, 8, off, 2, out, None)
    with pytest.raises(ddf.DDFError):       # AO rays without shading points
        ddf.ddf_query_mixed(m.h, r, 8, (3, 3, 3), out, out, occ, r, 8, off, 0, None, None)
    # nothing at all is a no-op; points with no rays read 1
    ddf.ddf_query_mixed(m.h, None, 0, None, None, None, None, None, 0, None, 0, None, None)
    zero = torch.zeros(3, dtype=torch.int32, device="cuda")
    hard = torch.empty(2, device="cuda")
    ddf.ddf_query_mixed(m.h, None, 0, None, None, None, None, None, 0, zero, 2, hard, None)
    torch.cuda.synchronize()
    assert hard.tolist() == [1.0, 1.0]
