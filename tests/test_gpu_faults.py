"""Out-of-memory paths without exhausting the device: the library's test
hook makes the k-th device allocation fail, for every k that a load, a
query and a training step reach. Each failing call must return
DDF_ERR_OOM. The same handle must then redo the whole sequence with results
bit for bit those of a handle that never failed. This is a host-made fault:
nothing faults, traps or hangs the GPU."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DDF_ERR_OOM = 3


@pytest.fixture(scope="module")
def torch_cuda(cuda_lib):
    import torch
    return torch


def _case(torch, kind):
    from paper_2606_00817_gb300 import ddf
    if kind == "hashgrid":
        net = (4, 64, 2)
        n = ddf.ddf_param_count(ddf.make_config(*net, kind="hashgrid"))
        blob = I.hashgrid_blob(n, O.hashgrid_mlp_dims(), seed=0)
    else:
        net = (6, 256, 3)                        # width 256: the CTA-pair training path
        blob = I.xavier_blob(I.NetShape(*net))
    rays = I.uniform_rays(1000, seed=5)
    t_ref, hit_ref = O.cast_scene(I.random_scene(8, 8, seed=0), rays.origins(), rays.dirs())
    inputs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in rays.soa()]
    tt = torch.from_numpy(np.where(hit_ref, t_ref, 0.0).astype(np.float32)).cuda()
    y = torch.from_numpy(hit_ref.astype(np.uint8)).cuda()
    return net, blob, inputs, tt, y


@pytest.mark.parametrize("kind", ["ray", "hashgrid"])
def test_every_allocation_can_fail_and_the_handle_recovers(torch_cuda, kind):
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net, blob, inputs, tt, y = _case(torch, kind)

    def run(m):
        m.load(blob)
        t, v = m.query(inputs)
        ddf.ddf_train_step(m.h, inputs, tt, y, 1000, 1e-3)
        t2, _ = m.query(inputs)
        torch.cuda.synchronize()
        return t.clone(), v.clone(), t2.clone()

    ref = ddf.DDF(*net, precision="bf16", kind=kind)
    want = run(ref)
    ref.close()
    failed = 0
    for k in range(400):
        m = ddf.DDF(*net, precision="bf16", kind=kind)
        ddf.ddf_debug_fail_allocation(k)
        try:
            run(m)
            ok = True
        except ddf.DDFError as e:
            assert e.status == DDF_ERR_OOM, (k, str(e))
            ok = False
        finally:
            ddf.ddf_debug_fail_allocation(-1)
        if ok:                                   # k is past the sequence's last allocation
            m.close()
            break
        failed += 1
        got = run(m)                             # the same handle, memory available again
        if kind == "hashgrid":                   # the table gradient sums by atomics
            assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
            assert torch.allclose(got[2], want[2], rtol=1e-4, atol=1e-5)
        else:
            for a, b in zip(got, want):
                assert torch.equal(a, b), k
        assert ddf.ddf_check_status(m.h) == 0
        m.close()
    assert failed >= 5
