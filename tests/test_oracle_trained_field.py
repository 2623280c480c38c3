"""The oracle-trained field of tests/golden/trained_small_field.json (written
by tests/golden/make_trained_field.py from oracle functions only): it loads
in the blob layout and is a trained field, far from the constant guess and
confident on most held-out rays. CPU only; the GPU tests that use it import
its helpers from here."""
import base64
import json
import os

import numpy as np

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "trained_small_field.json")


def trained_field():
    """(net, float32 blob) of the stored field."""
    with open(GOLD) as f:
        doc = json.load(f)
    blob = np.frombuffer(base64.b64decode(doc["blob_f32_le_base64"]), dtype="<f4").astype(np.float32)
    net = (doc["octaves"], doc["width"], doc["hidden"])
    assert blob.size == I.NetShape(*net).n_params
    return net, blob


def held_out_rays(n, seed=4242):
    """Rays of the training distribution (the oracle's distillation sampler
    on the training scene) from a seed the training never used, as float32."""
    scene = I.random_scene(32, 32, seed=0)
    o, d, _ = O.distill_rays(scene, seed, 0, n, 0.5)
    o, d = o.astype(np.float32), d.astype(np.float32)
    return I.Rays(*(np.ascontiguousarray(a) for a in (o[:, 0], o[:, 1], o[:, 2], d[:, 0], d[:, 1],
                                                      d[:, 2])))


def test_trained_field_is_trained():
    net, blob = trained_field()
    assert net == (6, 128, 4) and np.all(np.isfinite(blob))
    rays = held_out_rays(4096, seed=7)
    scene = I.random_scene(32, 32, seed=0)
    t_ref, hit = O.cast_scene(scene, rays.origins(), rays.dirs())
    out = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net)
    z1 = out["z"][:, 1]
    acc = np.mean((z1 > 0) == hit)
    assert acc > max(hit.mean(), 1 - hit.mean()) + 0.04, acc
    assert np.mean(np.abs(z1) < 0.1) < 0.05
    dt = np.abs(np.minimum(out["t"], 4) - np.minimum(t_ref, 4))[hit]
    assert np.median(dt) < 0.1


def test_stored_evaluation_is_the_oracles():
    """The evaluation block the benchmark reads (exact outputs on seeded
    uniform rays, e4m3 scales) is what the oracle computes for the stored
    weights, to float32 rounding."""
    with open(GOLD) as f:
        ev = json.load(f)["evaluation"]
    net, blob = trained_field()
    dec = lambda k: np.frombuffer(base64.b64decode(ev[k]), dtype="<f4").astype(np.float64)
    t, z1 = dec("t_exact_f32_le_base64"), dec("z1_exact_f32_le_base64")
    rays = I.uniform_rays(t.size, seed=77)
    out = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net)
    assert np.allclose(t, out["t"], rtol=2 ** -23, atol=1e-30)
    assert np.allclose(z1, out["z"][:, 1], rtol=2 ** -23, atol=1e-30)
    cal = I.uniform_rays(4096, seed=78)
    assert ev["fp8_act_scales"] == O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *net)
    assert np.mean(np.abs(z1) < 0.1) < 0.05                 # a trained field: few near-ties
    # the schemes' own accuracy: the emulating oracle against the exact one
    for prec, sc in (("bf16", None), ("fp8", ev["fp8_act_scales"])):
        emu = O.ddf_forward(rays.origins(), rays.dirs(), blob, *net, precision=prec, act_scales=sc)
        want = ev["scheme"][prec]
        assert np.isclose(want["flip_rate"], np.mean((emu["z"][:, 1] > 0) != (out["z"][:, 1] > 0)))
        assert np.isclose(want["max_abs_dt"], np.abs(emu["t"] - out["t"]).max(), rtol=1e-12)
