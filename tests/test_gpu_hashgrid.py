"""GPU tests of the hash-grid field (Sec. 3.4, kind "hashgrid"): bf16
tensor-core and FP32 queries against the oracle's hash-grid forward (bounds
as in test_gpu_parity: bf16 against the bf16-table emulation, FP32 within
1e-4 of the exact value), the shadow and AO queries on top of it, a
full-size sampled check, graph replay, and the calls this kind refuses."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HG = (4, 64, 2)        # direction bands, width, hidden layers
BOUNDS = {"bf16": (2e-3, 2e-4), "fp32": (1e-4, 1e-5)}


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


@pytest.fixture(scope="module")
def blob():
    from paper_2606_00817_gb300 import ddf
    n = ddf.ddf_param_count(ddf.make_config(*HG, kind="hashgrid"))
    assert n == 13_058_044 + 8_130
    return I.hashgrid_blob(n, O.hashgrid_mlp_dims(), seed=0, table_scale=1.0)


def _dev(torch, arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _model(prec, blob):
    from paper_2606_00817_gb300 import ddf
    m = ddf.DDF(*HG, precision=prec, kind="hashgrid")
    m.load(blob)
    return m


def _rays(n, seed, spread=1.0):
    r = I.uniform_rays(n, seed=seed)
    if spread != 1.0:      # some origins outside the box: clamped into it
        o = r.origins() * spread
        r = I.Rays.from_arrays(o, r.dirs())
    return r


def _check(t, v, rays, blob, prec):
    ref = O.hashgrid_forward(rays.origins(), rays.dirs(), blob,
                             precision="bf16" if prec == "bf16" else "exact")
    mx, mean = BOUNDS[prec]
    for g, r in ((t, ref["t"]), (v, ref["vis"])):
        e = np.abs(g - r) / np.maximum(1.0, np.abs(r))
        assert e.max() <= mx and e.mean() <= mean, (prec, e.max(), e.mean())
    return ref


@pytest.mark.parametrize("n", [1, 127, 129, 5000])
@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_hashgrid_query_matches_oracle(torch_cuda, blob, n, prec):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    m = _model(prec, blob)
    rays = _rays(n, seed=60 + n, spread=1.3)
    t, v = m.query(_dev(torch, rays.soa()))
    torch.cuda.synchronize()
    _check(t.double().cpu().numpy(), v.double().cpu().numpy(), rays, blob, prec)
    assert ddf.ddf_check_status(m.h) == 0


def test_hashgrid_bf16_tracks_exact_field(torch_cuda, blob):
    """Against the exact (float64, unrounded table) field the bf16 query is
    off by the bf16 rounding of the table, code and activations only."""
    torch = torch_cuda
    m = _model("bf16", blob)
    rays = _rays(4096, seed=61)
    t, _ = m.query(_dev(torch, rays.soa()))
    torch.cuda.synchronize()
    ex = O.hashgrid_forward(rays.origins(), rays.dirs(), blob)
    dt = np.abs(t.double().cpu().numpy() - ex["t"])
    assert dt.max() <= 5e-2 and dt.mean() <= 5e-3


def test_hashgrid_shadow_and_ao(torch_cuda, blob):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    m = _model("bf16", blob)
    scene = I.random_scene(64, 0, seed=0)
    light = (3.0, 3.0, 3.0)
    rays = I.shadow_rays(scene, 3000, light, seed=62)
    t, v, occ = m.shadow(_dev(torch, rays.soa()), light)
    torch.cuda.synchronize()
    ref = O.hashgrid_forward(rays.origins(), rays.dirs(), blob, precision="bf16")
    occ_ref = O.shadow(ref["t"], ref["z"][:, 1], rays.origins(), light)
    near = np.abs(ref["z"][:, 1]) < 1e-3
    agree = (occ.cpu().numpy().astype(bool) == occ_ref) | near
    assert agree.mean() >= 0.999
    ao_rays, offsets = I.ao_rays(scene, 200, seed=63)
    hard = torch.empty(200, device="cuda")
    soft = torch.empty(200, device="cuda")
    ddf.ddf_query_ao(m.h, _dev(torch, ao_rays.soa()), ao_rays.n,
                     torch.from_numpy(offsets.astype(np.int32)).cuda(), 200, hard, soft)
    torch.cuda.synchronize()
    ref = O.hashgrid_forward(ao_rays.origins(), ao_rays.dirs(), blob, precision="bf16")
    h_ref, s_ref = O.ambient_occlusion(ref["z"][:, 1] > 0, ref["vis"], offsets)
    assert np.abs(soft.double().cpu().numpy() - s_ref).max() <= 1e-2
    cnt = np.diff(offsets)
    near = np.array([np.sum(np.abs(ref["z"][a:b, 1]) < 1e-3) for a, b in zip(offsets[:-1], offsets[1:])])
    assert np.all(np.abs(hard.double().cpu().numpy() - h_ref) <= near / np.maximum(cnt, 1) + 1e-6)


def test_hashgrid_full_size_sampled_and_graph(torch_cuda, blob):
    """4,194,304 shadow rays (the benchmark's workload) through the hash-grid
    field: 256 sampled rays and both ends against the oracle; graph replay
    equals the eager query bit for bit."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    m = _model("bf16", blob)
    scene = I.random_scene(64, 0, seed=0)
    rays = I.shadow_rays(scene, 4_194_304, (3.0, 3.0, 3.0), seed=0)
    dev = _dev(torch, rays.soa())
    t, v = m.query(dev)
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([[0, rays.n - 1],
                                    np.random.default_rng(5).choice(rays.n, 256, replace=False)]))
    sub = I.Rays(*[a[idx] for a in rays.soa()])
    _check(t.double().cpu().numpy()[idx], v.double().cpu().numpy()[idx], sub, blob, "bf16")
    ddf.ddf_set_graph_mode(m.h, True)
    t2 = torch.empty_like(t)
    v2 = torch.empty_like(v)
    for _ in range(2):
        ddf.ddf_query_rays(m.h, dev, rays.n, t2, v2)
    torch.cuda.synchronize()
    assert torch.equal(t, t2) and torch.equal(v, v2)
    assert ddf.ddf_check_status(m.h) == 0


def test_hashgrid_refuses_what_it_does_not_have(torch_cuda, blob):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    with pytest.raises(ddf.DDFError):
        ddf.DDF(6, 64, 2, precision="bf16", kind="hashgrid")       # bands must be 4
    with pytest.raises(ddf.DDFError):
        ddf.DDF(4, 128, 2, precision="bf16", kind="hashgrid")      # width must be 64
    with pytest.raises(ddf.DDFError):
        ddf.DDF(4, 64, 2, precision="fp8", kind="hashgrid")
    m = _model("bf16", blob)
    with pytest.raises(ddf.DDFError):
        ddf.ddf_set_tile(m.h, (256, 4, 0, 0, 0), 0)
    rays = _dev(torch, I.uniform_rays(64).soa())
    with pytest.raises(ddf.DDFError):
        ddf.ddf_compute_grad(m.h, rays, torch.zeros(64, device="cuda"),
                             torch.zeros(64, dtype=torch.uint8, device="cuda"), 64)
    w = ddf.ddf_get_weights(m.h, blob.size)
    assert np.array_equal(w, blob)
