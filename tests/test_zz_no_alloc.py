"""The allocation-free query (ddf_query_rays_noalloc) against ddf_query_rays.

ddf_query_rays_noalloc serves callers that must not have a library call
cudaMalloc mid-work (a renderer's per-frame callback, or a framework whose
memory pool owns the device); its scratch is a static device array shared by
every call. Two calls in a row, with different batches, must each agree with
the allocating entry point, and a call on a handle that has never run a query
(so owns no workspace) must succeed while every library allocation is set to
fail. This file is collected last on purpose."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 2e-3   # the bf16 parity bound used by the other GPU tests (relative to max(1, |ref|))


def _close(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))) <= TOL


@pytest.mark.parametrize("net,n1,n2", [((6, 128, 4), 3000, 1037), ((10, 1280, 8), 6000, 129)])
def test_noalloc_matches_query_rays_twice(cuda_lib, net, n1, n2):
    import torch
    from paper_2606_00817_gb300 import ddf
    blob = I.xavier_blob(I.NetShape(*net))
    m = ddf.DDF(*net, precision="bf16")
    m.load(blob)
    for seed, n in ((11, n1), (12, n2)):
        rays = I.uniform_rays(n, seed=seed)
        dev = [torch.from_numpy(a).cuda() for a in rays.soa()]
        t_ref, v_ref = m.query(dev)
        t = torch.full((n,), float("nan"), device="cuda")
        v = torch.full((n,), float("nan"), device="cuda")
        ddf.ddf_query_rays_noalloc(m.h, dev, n, t, v, torch.cuda.current_stream())
        torch.cuda.synchronize()
        _close(t, t_ref)
        _close(v, v_ref)
        emu = O.ddf_forward(rays.origins()[:64], rays.dirs()[:64], blob, *net, precision="bf16")
        err = np.abs(t.double().cpu().numpy()[:64] - emu["t"]) / np.maximum(1.0, np.abs(emu["t"]))
        assert err.max() <= TOL
    assert ddf.ddf_check_status(m.h) == 0
    m.close()


def _field(kind):
    from paper_2606_00817_gb300 import ddf
    if kind == "ray":
        net = (10, 1280, 8)
        m = ddf.DDF(*net, precision="bf16")
        m.load(I.xavier_blob(I.NetShape(*net)))
        return m, 4000
    m = ddf.DDF(4, 64, 2, precision="bf16", kind="hashgrid")
    dims = [(64, ddf.HASHGRID_CODE), (64, 64), (2, 64)]
    m.load(I.hashgrid_blob(m.n_params, dims, seed=0))
    return m, 200_000     # far above the dense-field limit: hash-grid queries need no scratch


@pytest.mark.parametrize("kind", ["ray", "hashgrid"])
def test_noalloc_on_a_fresh_handle_allocates_nothing(cuda_lib, kind):
    """With the library's allocation hook armed so that its next device
    allocation fails, the first query of a fresh handle (which owns no
    workspace yet) still succeeds through the allocation-free entry point, and
    the hook is still armed afterwards: nothing in the call allocated."""
    import torch
    from paper_2606_00817_gb300 import ddf
    m, n = _field(kind)
    rays = I.uniform_rays(n, seed=21)
    dev = [torch.from_numpy(a).cuda() for a in rays.soa()]
    outs = []
    for _ in range(2):
        t = torch.full((n,), float("nan"), device="cuda")
        v = torch.full((n,), float("nan"), device="cuda")
        torch.cuda.synchronize()
        ddf.ddf_debug_fail_allocation(0)
        try:
            ddf.ddf_query_rays_noalloc(m.h, dev, n, t, v, torch.cuda.current_stream())
            torch.cuda.synchronize()
            with pytest.raises(ddf.DDFError) as e:     # the hook is still armed
                ddf.DDF(6, 128, 4, precision="bf16")
            assert e.value.status == 3
        finally:
            ddf.ddf_debug_fail_allocation(-1)
        outs.append((t, v))
    t_ref, v_ref = m.query(dev)
    torch.cuda.synchronize()
    for t, v in outs:
        _close(t, t_ref)
        _close(v, v_ref)
    assert ddf.ddf_check_status(m.h) == 0
    m.close()


def test_noalloc_rejects_batches_beyond_the_scratch(cuda_lib):
    import torch
    from paper_2606_00817_gb300 import ddf
    net = (10, 1280, 8)
    m = ddf.DDF(*net, precision="bf16")
    m.load(I.xavier_blob(I.NetShape(*net)))
    n = 20000
    dev = [torch.zeros(n, device="cuda") for _ in range(6)]
    t = torch.empty(n, device="cuda")
    v = torch.empty(n, device="cuda")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_query_rays_noalloc(m.h, dev, n, t, v)
    assert e.value.status == 1 and "at most" in str(e.value)
    # a count whose byte size would wrap a 64-bit product is refused, not truncated
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_query_rays_noalloc(m.h, dev, 1 << 61, t, v)
    assert e.value.status == 1 and "at most" in str(e.value)
    m.close()
