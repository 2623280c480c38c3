"""The seeded input generators that both sides of every parity test draw
from (paper_2606_00817_gb300/inputs.py), against SplitMix64's published
outputs and against the properties each recipe states."""
import json
import os

import numpy as np

from paper_2606_00817_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_matches_the_published_outputs():
    """Seed 0, stream 0 gives key 0, so the counter form must reproduce the
    sequential generator started at state 0."""
    with open(os.path.join(GOLD, "splitmix64.json")) as f:
        want = [int(x, 16) for x in json.load(f)["outputs_from_state_0"]]
    assert [int(x) for x in I.splitmix64(0, 0, 3)] == want


def test_splitmix64_offsets_index_the_same_stream():
    full = I.splitmix64(7, 3, 100)
    assert np.array_equal(I.splitmix64(7, 3, 40, offset=60), full[60:])
    assert not np.array_equal(I.splitmix64(7, 4, 100), full)          # streams differ
    assert not np.array_equal(I.splitmix64(8, 3, 100), full)          # seeds differ


def test_uniform_gaussian_and_unit_vector_moments():
    n = 200_000
    u = I.uniform(1, 2, n, -3.0, 5.0)
    assert u.min() >= -3.0 and u.max() < 5.0 and abs(u.mean() - 1.0) < 0.03
    g = I.gaussian(1, 2, n)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.015
    v = I.unit_vectors(1, 2, n)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)
    assert np.abs(v.mean(axis=0)).max() < 0.01                           # isotropic
    assert np.allclose(v.T @ v / n, np.eye(3) / 3, atol=0.01)           # E[v v^T] = I / 3


def test_uniform_rays_are_float32_soa_with_unit_directions():
    r = I.uniform_rays(4096, seed=3)
    for a in r.soa():
        assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] and a.shape == (4096,)
    assert np.abs(r.origins()).max() <= 1.0
    assert np.allclose(np.linalg.norm(r.dirs().astype(np.float64), axis=1), 1.0, atol=1e-6)
    again = I.uniform_rays(4096, seed=3)
    assert all(np.array_equal(a, b) for a, b in zip(r.soa(), again.soa()))
    assert not np.array_equal(I.uniform_rays(4096, seed=4).ox, r.ox)


def test_xavier_blob_layout_and_bounds():
    """Xavier-uniform W in +-sqrt(6 / (fan_in + fan_out)), biases in
    +-1 / sqrt(fan_in), layers in order with W before b."""
    shape = I.NetShape(3, 64, 3)
    blob = I.xavier_blob(shape, seed=2).astype(np.float64)
    assert blob.size == shape.n_params == sum(fo * fi + fo for fo, fi in shape.layer_dims())
    off = 0
    for fo, fi in shape.layer_dims():
        w = blob[off:off + fo * fi]
        off += fo * fi
        b = blob[off:off + fo]
        off += fo
        a = np.sqrt(6.0 / (fi + fo))
        assert np.abs(w).max() <= a * (1 + 1e-7) and np.abs(w).max() > 0.9 * a
        assert np.abs(b).max() <= (1 + 1e-7) / np.sqrt(fi)
    assert shape.layer_dims()[-1] == (2, 64) and shape.d_in == 6 + 12 * 3


def test_ao_batch_is_ragged_csr_with_cosine_directions():
    scene = I.random_scene(8, 4, seed=1)
    rays, offsets = I.ao_rays(scene, 500, seed=5)
    counts = np.diff(offsets.astype(np.int64))
    assert offsets[0] == 0 and offsets[-1] == rays.n and offsets.dtype == np.int32
    assert counts.min() >= 4 and counts.max() <= 64 and len(set(counts.tolist())) > 20
    d = rays.dirs().astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)


def test_orbit_cameras_sit_on_the_stated_sphere():
    cams = I.orbit_cameras(256, radius=3.0, target=(0.0, -0.2, 0.0), elev=(10.0, 55.0), seed=4)
    eye, tg = cams[:, 0:3].astype(np.float64), cams[:, 3:6].astype(np.float64)
    rel = eye - tg
    assert np.allclose(np.linalg.norm(rel, axis=1), 3.0, atol=1e-5)
    el = np.degrees(np.arcsin(rel[:, 1] / 3.0))
    assert el.min() >= 10.0 - 1e-3 and el.max() <= 55.0 + 1e-3
    assert np.all(cams[:, 7] == 1.0) and np.allclose(cams[:, 9], np.radians(40.0))
