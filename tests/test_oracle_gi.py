"""Pins of the oracle's shadow / AO image path against values it does not
compute itself: SplitMix64's published outputs, closed forms of the pinhole
camera, normals of known surface points, the cosine-weighted distribution's
moments, and a one-sphere scene whose shadow and silhouette are closed
forms."""
import json
import os

import numpy as np

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLD, "splitmix64.json")) as f:
        want = [int(x, 16) for x in json.load(f)["outputs_from_state_0"]]
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % (1 << 64)], np.uint64)
    assert [int(v) for v in O.splitmix64(states)] == want


def test_uniforms_are_24_bit_and_uniform():
    u = O.gi_uniform(7, np.arange(200000), 3, 0)
    assert np.all((u >= 0) & (u < 1)) and np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3


def test_camera_closed_forms():
    # 3 x 3 image: the centre pixel looks exactly at the target
    o, d = O.camera_rays([0, 0, -3], [0, 0, 0], [0, 1, 0], np.pi / 2, 3, 3)
    assert np.allclose(d[4], [0, 0, 1], atol=1e-15) and np.allclose(o[4], [0, 0, -3])
    # the top-left pixel centre: sx = -(2/3) tan(45 deg), sy = +(2/3) tan(45 deg)
    # right = f x up = (0,0,1) x (0,1,0) = (-1, 0, 0)
    v = np.array([0, 0, 1]) + (-2 / 3) * np.array([-1, 0, 0]) + (2 / 3) * np.array([0, 1, 0])
    assert np.allclose(d[0], v / np.linalg.norm(v), atol=1e-15)


def test_surface_normals_of_known_points():
    sc = I.Scene(np.array([[0.0, 0.0, 0.0]]), np.array([0.5]), np.array([[1.0, -0.2, -0.2]]),
                 np.array([[1.4, 0.2, 0.2]]))
    p = np.array([[0.5, 0, 0], [0, -0.5, 0], [1.4, 0.0, 0.1], [1.2, 0.2, 0.0], [1.0, 0.05, -0.1]])
    n = O.surface_normal(sc, p)
    assert np.allclose(n, [[1, 0, 0], [0, -1, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0]])


def test_cosine_weighted_moments():
    rng = np.random.default_rng(0)
    nrm = rng.normal(size=(100000, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    d = O.cosine_dirs(nrm, rng.uniform(size=100000), rng.uniform(size=100000))
    c = np.sum(d * nrm, axis=1)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-12) and np.all(c >= -1e-12)
    assert abs(c.mean() - 2 / 3) < 3e-3              # E[cos] = 2/3 for a cosine density
    assert abs(np.mean(c ** 2) - 1 / 2) < 3e-3       # E[cos^2] = 1/2
    t1, t2 = O.onb(nrm[:1000])
    assert np.allclose(np.cross(t1, t2), nrm[:1000], atol=1e-12)


def test_one_sphere_silhouette_and_shadow():
    """A unit sphere seen from (0,0,-4) with a 60 degree camera: pixels hit
    it iff their ray passes within 1 of the centre; with the light straight
    behind the camera nothing is in shadow, and with the light straight
    behind the sphere every visible point is; AO of a lone convex sphere is
    exactly 1 (nothing to hit)."""
    sc = I.Scene(np.array([[0.0, 0.0, 0.0]]), np.array([1.0]), np.zeros((0, 3)), np.zeros((0, 3)))
    W = H = 40
    fov = np.pi / 3
    o, d = O.camera_rays([0, 0, -4], [0, 0, 0], [0, 1, 0], fov, W, H)
    closest = np.linalg.norm(np.cross(d, -o), axis=1)      # distance of the line to the centre
    sh, ao = O.gi_images(sc, [0, 0, -4], [0, 0, 0], [0, 1, 0], fov, W, H, [0, 0, -10], 4, 1)
    fg = closest < 1.0
    clear = np.abs(closest - 1.0) > 1e-9
    assert np.array_equal((sh.ravel() >= 0)[clear], fg[clear])
    assert np.all(sh.ravel()[fg] == 1.0) and np.all(ao.ravel()[fg] == 1.0)
    sh2, _ = O.gi_images(sc, [0, 0, -4], [0, 0, 0], [0, 1, 0], fov, W, H, [0, 0, 10], 2, 1)
    assert np.all(sh2.ravel()[fg] == 0.0)


def test_field_answered_images_of_constant_fields():
    """With every table entry and weight zero the field answers every ray
    with its head biases: z1 = b1 and t = softplus(b0). So the images are
    closed forms: all foreground shadowed and fully occluded when b1 > 0 and
    t is below every light distance; all lit and open when b1 < 0; lit but
    fully occluded when t exceeds every light distance."""
    scene = I.random_scene(32, 32, seed=0)
    dims = O.hashgrid_mlp_dims()
    n_tab = int(sum(O.hashgrid_table_sizes())) * 2
    n_mlp = sum(fo * fi + fo for fo, fi in dims)
    cam = ([2.5, 1.8, -3.0], [0, 0, 0], [0, 1, 0], np.radians(50.0))
    ex_s, _ = O.gi_images(scene, *cam, 24, 16, (3.0, 3.0, 3.0), 4, 5)
    fg = ex_s >= 0
    assert 0.05 < fg.mean() < 0.95

    def field(b0, b1):
        blob = np.zeros(n_tab + n_mlp, np.float32)
        blob[-2:] = [b0, b1]
        return blob

    def images(blob):
        return O.gi_images(scene, *cam, 24, 16, (3.0, 3.0, 3.0), 4, 5, field_blob=blob)

    s, a = images(field(np.log(np.expm1(0.5)), 1.0))        # t = 0.5, hit
    assert np.all(s[fg] == 0) and np.all(a[fg] == 0) and np.all(s[~fg] == -1) and np.all(a[~fg] == -1)
    s, a = images(field(0.0, -1.0))                         # misses
    assert np.all(s[fg] == 1) and np.all(a[fg] == 1)
    s, a = images(field(40.0, 1.0))                         # hits beyond the light
    assert np.all(s[fg] == 1) and np.all(a[fg] == 0)
    # detail: the shadow rays' distances to the light are those of the exact path
    s, a, det = O.gi_images(scene, *cam, 24, 16, (3.0, 3.0, 3.0), 4, 5,
                            field_blob=field(0.0, 1.0), detail=True)
    assert det["pixels"].size == fg.sum() and det["ao_z1"].shape == (fg.sum(), 4)
    assert np.allclose(det["shadow_z1"], 1.0) and np.allclose(det["shadow_t"], np.log(2.0))
