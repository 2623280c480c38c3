"""Pins of the oracle's Gaussian-rendered depth against closed forms: the
projection of a point and of an isotropic Gaussian, the alpha profile of a
single Gaussian, and the two-layer composite."""
import numpy as np

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

EYE, TGT, UP = [0.0, 0.0, -4.0], [0.0, 0.0, 0.0], [0.0, 1.0, 0.0]
FOV = np.radians(40.0)


def test_projection_matches_the_camera_rays():
    """The pixel a point projects to is the pixel whose camera ray passes
    through it."""
    W, H = 9, 7
    o, d = O.camera_rays(EYE, TGT, UP, FOV, W, H)
    pts = o + 3.0 * d                                     # points on pixel rays
    mu, S, z = O.gs_project(pts, np.zeros((W * H, 3, 3)), EYE, TGT, UP, FOV, W, H)
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.allclose(mu[:, 0], xx.ravel(), atol=1e-9) and np.allclose(mu[:, 1], yy.ravel(), atol=1e-9)
    assert np.allclose(S, O.GS_LOWPASS * np.eye(2)[None], atol=1e-12)   # zero covariance: low-pass only


def test_isotropic_gaussian_footprint():
    """An isotropic Gaussian (sigma) on the optical axis at depth zc projects
    to variance (f sigma / zc)^2 + 0.3 on each screen axis, f in pixels."""
    W = H = 64
    sigma, zc = 0.1, 4.0
    mu, S, z = O.gs_project(np.array([[0.0, 0.0, 0.0]]), (sigma ** 2 * np.eye(3))[None],
                            EYE, TGT, UP, FOV, W, H)
    fpx = H / (2 * np.tan(FOV / 2))
    assert np.allclose(mu[0], [(W - 1) / 2, (H - 1) / 2]) and abs(z[0] - zc) < 1e-12
    assert np.allclose(S[0], (fpx * sigma / zc) ** 2 * np.eye(2) + 0.3 * np.eye(2), rtol=1e-12)


def test_single_gaussian_alpha_profile_and_depth():
    """One Gaussian, opacity 0.8: every pixel it covers reports the mean's
    depth as a distance along that pixel ray, and the hit flag follows
    alpha = 0.8 exp(-q/2) > 0.5."""
    W = H = 33
    sigma = 0.15
    t, hit = O.gs_depth(np.array([[0.0, 0.0, 0.0]]), (sigma ** 2 * np.eye(3))[None], [0.8],
                        EYE, TGT, UP, FOV, W, H)
    _, d = O.camera_rays(EYE, TGT, UP, FOV, W, H)
    cosf = d[:, 2].reshape(H, W)
    cover = np.isfinite(t)
    assert np.allclose(t[cover], (4.0 / cosf)[cover], rtol=1e-12)
    fpx = H / (2 * np.tan(FOV / 2))
    var = (fpx * sigma / 4.0) ** 2 + 0.3
    yy, xx = np.mgrid[0:H, 0:W]
    q = ((xx - 16) ** 2 + (yy - 16) ** 2) / var
    assert np.array_equal(hit, 0.8 * np.exp(-q / 2) > 0.5)


def test_two_layer_composite():
    """A near Gaussian of opacity a1 in front of a far one of opacity a2 (both
    wide): at the centre pixel A = a1 + (1 - a1) a2 and the expected distance
    is (a1 t1 + (1 - a1) a2 t2) / A."""
    W = H = 5
    covs = (0.5 ** 2 * np.eye(3))[None].repeat(2, 0)
    a1, a2 = 0.3, 0.6
    t, hit = O.gs_depth(np.array([[0, 0, -1.0], [0, 0, 1.0]]), covs, [a1, a2], EYE, TGT, UP, FOV, W, H)
    q1 = 0.0      # the centre pixel sits on both means
    A = a1 + (1 - a1) * a2
    assert abs(t[2, 2] - (a1 * 3.0 + (1 - a1) * a2 * 5.0) / A) < 1e-12 and hit[2, 2] == (A > 0.5)


def test_enter_box_invariants():
    """Rays from outside that meet the box start on its surface afterwards and
    keep their line (the first hit stays at the same point); rays that start
    inside or miss are left alone."""
    rng = np.random.default_rng(0)
    n = 2000
    o = rng.uniform(-4, 4, (n, 3))
    d = rng.normal(size=(n, 3))
    d[: n // 2] = rng.uniform(-1, 1, (n // 2, 3)) - o[: n // 2]     # half aimed into the box
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o2, e = O.enter_box(o, d)
    inside = np.all(np.abs(o) <= 1, axis=1)
    assert np.all(e[inside] == 0) and np.array_equal(o2[inside], o[inside])
    moved = e > 0
    assert moved.sum() > 500 and (~moved & ~np.all(np.abs(o) <= 1, axis=1)).sum() > 500
    assert np.allclose(np.abs(o2[moved]).max(axis=1), 1.0, atol=1e-12)
    assert np.allclose(o2 - o, e[:, None] * d)
    # brute force: march each moved ray finely, the first sample inside the box
    # lies just past the entry distance
    s = np.linspace(0, 12, 120001)
    for i in np.nonzero(moved)[0][:50]:
        p = o[i] + s[:, None] * d[i]
        first = s[np.argmax(np.all(np.abs(p) <= 1, axis=1))]
        assert 0 <= first - e[i] <= 1e-4 + 1e-12
    # rays that miss: no sample of the line is inside
    miss = ~inside & ~moved
    for i in np.nonzero(miss)[0][:50]:
        p = o[i] + s[:, None] * d[i]
        assert not np.any(np.all(np.abs(p) < 1 - 1e-9, axis=1))
    # exact hits are preserved: cast before and after
    sc = I.Scene(np.zeros((1, 3)), np.array([0.5]), np.zeros((0, 3)), np.zeros((0, 3)))
    t0, h0 = O.cast_scene(sc, o, d)
    t1, h1 = O.cast_scene(sc, o2, d)
    assert np.array_equal(h0, h1) and np.allclose(t1[h0], t0[h0] - e[h0])


def test_anisotropic_and_off_axis_footprints():
    """Closed forms of the EWA screen covariance for the camera at (0, 0, -4)
    looking along +z (right = -x, up = +y, so pixel x grows with -X and pixel
    y with -Y): a Gaussian at the origin rotated in the XY plane keeps the
    sign of its XY covariance on screen, scaled by (f / 4)^2; a Gaussian at
    (X0, 0, 0) stretched only along the view axis still has a horizontal
    footprint, through the projection's depth derivative: S_xx = (f X0 / 16)^2
    c^2 + 0.3."""
    W = H = 64
    fpx = H / (2 * np.tan(FOV / 2))
    th = 0.6
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    cov = R @ np.diag([0.2 ** 2, 0.05 ** 2, 0.01 ** 2]) @ R.T
    _, S, _ = O.gs_project(np.zeros((1, 3)), cov[None], EYE, TGT, UP, FOV, W, H)
    k = (fpx / 4.0) ** 2
    assert np.allclose(S[0], k * cov[:2, :2] + 0.3 * np.eye(2), rtol=1e-12)
    assert S[0, 0, 1] > 0                                  # the sign survives
    X0, c = 0.5, 0.3
    mu, S, z = O.gs_project(np.array([[X0, 0.0, 0.0]]), np.diag([0.0, 0.0, c ** 2])[None],
                            EYE, TGT, UP, FOV, W, H)
    assert abs(mu[0, 0] - ((W - 1) / 2 - X0 / 4.0 * fpx)) < 1e-9
    assert np.allclose(S[0], np.diag([(fpx * X0 / 16.0) ** 2 * c ** 2 + 0.3, 0.3]), rtol=1e-12, atol=1e-15)
