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


@pytest.mark.parametrize("kind", ["ray", "hashgrid"])
def test_checkpoint_resume_and_corruption(torch_cuda, tmp_path, kind):
    """k steps, a checkpoint, a fresh handle loading it and n - k more steps
    give the weights of n steps (bit for bit for the ray field; the hash
    grid's table gradient sums by atomics). The file's CRC-32 is zlib's; a
    flipped byte, a truncated file, a foreign magic or configuration are
    refused with the handle untouched."""
    import struct
    import zlib
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net, blob, inputs, tt, y = _case(torch, kind)

    def steps(m, k):
        for _ in range(k):
            ddf.ddf_train_step(m.h, inputs, tt, y, 1000, 1e-3)
        torch.cuda.synchronize()

    a = ddf.DDF(*net, precision="bf16", kind=kind)
    a.load(blob)
    steps(a, 6)
    w_a = ddf.ddf_get_weights(a.h, blob.size)
    b = ddf.DDF(*net, precision="bf16", kind=kind)
    b.load(blob)
    steps(b, 3)
    path = tmp_path / "run.ckpt"
    ddf.ddf_save_checkpoint(b.h, path)
    raw = path.read_bytes()
    assert raw[:8] == b"DDFCKPT\0"
    version, flags = struct.unpack_from("<II", raw, 8)
    n_params, step = struct.unpack_from("<Qq", raw, 40)
    crc = struct.unpack_from("<I", raw, 56)[0]
    assert (version, flags, n_params, step) == (1, 1, blob.size, 3)
    assert len(raw) == 64 + 3 * 4 * blob.size and zlib.crc32(raw[64:]) == crc
    c = ddf.DDF(*net, precision="bf16", kind=kind)
    ddf.ddf_load_checkpoint(c.h, path)
    steps(c, 3)
    w_c = ddf.ddf_get_weights(c.h, blob.size)
    if kind == "ray":
        assert np.array_equal(w_a, w_c)
    else:
        assert np.allclose(w_a, w_c, rtol=1e-5, atol=1e-6)
    # refusals leave the handle as it was
    t0, _ = c.query(inputs)
    bad = bytearray(raw)
    bad[64 + 4 * 17] ^= 0x40
    (tmp_path / "flip.ckpt").write_bytes(bytes(bad))
    (tmp_path / "short.ckpt").write_bytes(raw[:-4])
    (tmp_path / "magic.ckpt").write_bytes(b"NOTACKPT" + raw[8:])
    for name, status in (("flip.ckpt", 4), ("short.ckpt", 4), ("magic.ckpt", 1), ("none.ckpt", 1)):
        with pytest.raises(ddf.DDFError) as e:
            ddf.ddf_load_checkpoint(c.h, tmp_path / name)
        assert e.value.status == status, name
    other = ddf.DDF(4, 64, 3, precision="bf16", kind="hashgrid") if kind == "hashgrid" \
        else ddf.DDF(6, 128, 3, precision="bf16")
    with pytest.raises(ddf.DDFError) as e:
        ddf.ddf_load_checkpoint(other.h, path)
    assert e.value.status == 1
    t1, _ = c.query(inputs)
    torch.cuda.synchronize()
    assert torch.equal(t0, t1)
    for m in (a, b, c, other):
        m.close()


def test_misaligned_device_pointers_are_refused(torch_cuda):
    """A float array that does not start on a 4-byte boundary would make the
    kernels fault: every entry point refuses it on the host, before any
    launch, and the handle stays usable."""
    torch = torch_cuda
    from paper_2606_00817_gb300 import ddf
    net = (6, 128, 3)
    blob = I.xavier_blob(I.NetShape(*net))
    m = ddf.DDF(*net, precision="bf16")
    m.load(blob)
    n = 64
    rays = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in I.uniform_rays(n, seed=1).soa()]
    raw = torch.zeros(4 * n + 16, dtype=torch.uint8, device="cuda")
    bad = raw.data_ptr() + 2                          # 2 bytes past a 16-byte boundary
    good_t = torch.empty(n, device="cuda")
    good_v = torch.empty(n, device="cuda")
    hit = torch.zeros(n, dtype=torch.uint8, device="cuda")
    calls = [
        lambda: ddf.ddf_query_rays(m.h, rays, n, bad, good_v),
        lambda: ddf.ddf_query_rays(m.h, [bad] + rays[1:], n, good_t, good_v),
        lambda: ddf.ddf_query_shadow(m.h, rays, n, (3.0, 3.0, 3.0), good_t, bad, hit),
        lambda: ddf.ddf_train_step(m.h, rays, bad, hit, n, 1e-3),
        lambda: ddf.ddf_cast_scene(good_t, 1, good_t, 0, rays, n, bad, hit),
        lambda: ddf.ddf_enter_box(rays, bad, None, n, 1.0),
        lambda: ddf.ddf_render_gs_depth(bad, good_t, good_t, 1, [[0, 0, -4, 0, 0, 0, 0, 1, 0, 0.7]],
                                        8, 8, good_t, hit),
    ]
    for i, call in enumerate(calls):
        with pytest.raises(ddf.DDFError) as e:
            call()
        assert e.value.status == 1, i
    t, v = m.query(rays)
    torch.cuda.synchronize()
    assert torch.isfinite(t).all() and ddf.ddf_check_status(m.h) == 0
