"""Pins for the oracle's distillation schedule (Sec. 3.2 / 3.4): the training
ray sampler, the ray-march shifted points, the cosine learning rate and the
pool draw, against closed forms, invariants and an independent big-integer
evaluation of the counter-based draws. CPU only."""
import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

M64 = (1 << 64) - 1


def _mix(x):
    """SplitMix64 on Python integers (wrapping by masks), independent of the
    oracle's numpy uint64 arithmetic."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _key(seed, a, b):
    return _mix((_mix(seed ^ 0x5DEECE66D) + a) & M64) ^ ((b * 0x2545F4914F6CDD1D) & M64)


def test_uniform_draws_against_big_integers():
    for seed, step, i, m in ((0, 0, 0, 0), (7, 3, 12345, 5), (2**63 + 11, 2**40, 2**33 + 7, 7)):
        want = (_mix((_key(seed, step, i) + m) & M64) >> 40) / 2.0 ** 24
        assert float(O.distill_uniform(seed, step, i, m)) == want
    # the pool draw: top 32 bits of mix(key + 8), times n_pool, over 2^32
    for seed, step, i, n in ((1, 2, 3, 1000), (9, 0, 2**31 - 1, 2**31), (5, 17, 0, 1)):
        u32 = _mix((_key(seed, step, i) + 8) & M64) >> 32
        assert int(O.distill_pool_index(seed, step, i, n)[0]) == (u32 * n) >> 32


def test_pool_index_range_and_power_of_two():
    i = np.arange(20000)
    j = O.distill_pool_index(3, 4, i, 1 << 10)
    assert j.min() >= 0 and j.max() < 1024
    hist = np.bincount(j, minlength=1024)
    assert hist.min() > 0 and hist.max() < 60                    # about 19.5 per row
    j7 = O.distill_pool_index(3, 4, i, 7)
    assert set(np.unique(j7)) == set(range(7))


def test_learning_rate_closed_forms():
    lr0, S = 3e-3, 30000
    assert O.distill_lr(lr0, 0, S) == lr0
    assert np.isclose(O.distill_lr(lr0, S // 2, S), lr0 * (0.05 + 0.475), rtol=1e-15)
    assert np.isclose(O.distill_lr(lr0, S, S), 0.05 * lr0, rtol=1e-12)   # the limit
    k = np.arange(S)
    lr = O.distill_lr(lr0, k, S)
    assert np.all(np.diff(lr) < 0) and lr[-1] > 0.05 * lr0
    # symmetric about the midpoint: lr_k + lr_{S-k} = (0.1 + 0.95) lr0
    assert np.allclose(lr[1:] + lr[::-1][:-1], 1.05 * lr0, rtol=1e-12)


def test_uniform_sphere_dir_closed_forms_and_moments():
    e = O.uniform_sphere_dir(np.array([1.0, 0.5, 0.5, 0.0]), np.array([0.3, 0.0, 0.25, 0.0]))
    assert np.allclose(e, [[0, 0, 1], [1, 0, 0], [0, 1, 0], [0, 0, -1]], atol=1e-15)
    rng = np.random.default_rng(0)
    d = O.uniform_sphere_dir(rng.random(200000), rng.random(200000))
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-14)
    assert np.abs(d.mean(0)).max() < 0.01
    assert np.allclose(d.T @ d / d.shape[0], np.eye(3) / 3, atol=0.005)


def _surface_gap(scene, p):
    """min over primitives of |distance of p to that primitive's surface|."""
    gaps = [np.abs(np.linalg.norm(p - c, axis=1) - r) for c, r in zip(scene.centers, scene.radii)]
    for lo, hi in zip(scene.box_lo, scene.box_hi):
        q = np.abs(p - 0.5 * (lo + hi)) - 0.5 * (hi - lo)
        gaps.append(np.abs(np.linalg.norm(np.maximum(q, 0), axis=1) + np.minimum(q.max(1), 0)))
    return np.stack(gaps, 1)


def _area_counts_match(scene, o):
    """Counts of surface origins per primitive (the one whose surface the
    origin is 1e-3 off) against the closed-form area fractions, 4 pi r^2 and
    2 (ab + bc + ca), within 5 binomial sigma + 3."""
    near = np.argmin(np.abs(_surface_gap(scene, o) - 1e-3), axis=1)
    r = np.asarray(scene.radii, np.float64)
    e = np.asarray(scene.box_hi, np.float64) - np.asarray(scene.box_lo, np.float64)
    area = np.concatenate([4 * np.pi * r ** 2,
                           2 * (e[:, 0] * e[:, 1] + e[:, 1] * e[:, 2] + e[:, 2] * e[:, 0])])
    frac = area / area.sum()
    cnt = np.bincount(near, minlength=frac.size)
    want = len(o) * frac
    return bool(np.all(np.abs(cnt - want) <= 5 * np.sqrt(want * (1 - frac)) + 3))


def test_surface_weights_and_pick_by_hand():
    """A sphere of radius 0.5 and a 1 x 0.5 x 0.25 box: the weights are
    floor(A 2^24) with float32(4 pi) (1/2) (1/2) = float32(pi) =
    13176795 / 2^22 for the sphere and 0.125, 0.25, 0.5 for the box's face
    pairs across x, y and z; a uniform picks the element whose share of the
    cumulative weight it falls in."""
    sc = I.Scene(np.array([[0.0, 0.0, 0.0]]), np.array([0.5]), np.array([[2.0, 0.0, 0.0]]),
                 np.array([[3.0, 0.5, 0.25]]))
    w = O.distill_surface_weights(sc)
    assert w.tolist() == [52707180, 2097152, 2097152, 4194304, 4194304, 8388608, 8388608]
    # cumulative: 52.7M, 54.8M, 56.9M, 61.1M, 65.3M, 73.7M, 82.1M
    j, ok = O.distill_pick_surface(sc, np.array([0.0, 0.5, 0.65, 0.7, 0.85, 0.99]))
    assert ok and j.tolist() == [0, 0, 1, 3, 5, 6]
    # degenerate primitives weigh nothing; no area at all: camera rays only
    flat = I.Scene(np.zeros((1, 3)), np.array([0.0]), np.array([[0.0, 0.0, 0.0]]),
                   np.array([[1.0, 1.0, 0.0]]))
    assert O.distill_surface_weights(flat).tolist() == [0, 0, 0, 0, 0, 16777216, 16777216]
    none = I.Scene(np.zeros((1, 3)), np.array([0.0]), np.zeros((0, 3)), np.zeros((0, 3)))
    assert not np.any(O.distill_rays(none, 1, 0, 100, 1.0)[2])


def test_thin_box_caps_are_rarely_chosen():
    """A 0.04 x 0.9 x 0.04 leg: its two end caps hold 2 (0.04^2) / (2 (0.036
    + 0.0016 + 0.036)) = 2.17 % of its area, so of the surface origins about
    that fraction sits beyond its y extent."""
    leg = I.Scene(np.zeros((0, 3)), np.zeros(0), np.array([[0.0, -0.45, 0.0]]),
                  np.array([[0.04, 0.45, 0.04]]))
    o, _, surf = O.distill_rays(leg, 3, 0, 40000, 1.0)
    assert surf.all()
    cap = np.abs(o[:, 1]) > 0.45
    p = 2 * 0.04 ** 2 / (2 * (0.036 + 0.0016 + 0.036))
    assert abs(cap.mean() - p) < 4 * np.sqrt(p * (1 - p) / cap.size)


def test_planted_uniform_pick_fails_the_area_check(monkeypatch):
    """Planted in the oracle: surface elements drawn with equal weights (the
    element, not its area). The area check catches it."""
    scene = I.random_scene(32, 32, seed=0)
    monkeypatch.setattr(O, "distill_surface_weights",
                        lambda sc: np.ones(len(sc.radii) + 6 * len(sc.box_lo), np.int64))
    o, _, surf = O.distill_rays(scene, 7, 3, 40000, 0.5)
    assert not _area_counts_match(scene, o[surf])


def test_sampler_invariants():
    scene = I.random_scene(32, 32, seed=0)
    n = 40000
    o, d, surf = O.distill_rays(scene, 7, 3, n, 0.5)
    assert abs(surf.mean() - 0.5) < 0.01
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-14)
    # surface rays start 1e-3 off some primitive's surface, outside it
    g = _surface_gap(scene, o[surf][:4000])
    assert np.all(np.abs(g - 1e-3).min(1) < 1e-12)
    # each primitive is chosen in proportion to its surface area
    assert _area_counts_match(scene, o[surf])
    assert np.abs(d[surf].mean(0)).max() < 0.02                 # directions cover the sphere
    # camera rays start on a face of [-1, 1]^3 and pass through [-0.9, 0.9]^3
    oc, dc = o[~surf], d[~surf]
    ax = np.argmax(np.abs(oc), axis=1)
    assert np.all(np.abs(oc[np.arange(oc.shape[0]), ax]) == 1.0) and np.all(np.abs(oc) <= 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        a, b = (-0.9 - oc) / dc, (0.9 - oc) / dc
    tn = np.nanmax(np.minimum(a, b), axis=1)
    tf = np.nanmin(np.maximum(a, b), axis=1)
    assert np.all(tn <= tf + 1e-12) and np.all(tf > 0)
    # counter-based: another step gives other rays, the same step the same
    o2, _, _ = O.distill_rays(scene, 7, 3, 100, 0.5)
    assert np.array_equal(o2, o[:100])
    assert not np.array_equal(O.distill_rays(scene, 7, 4, 100, 0.5)[0], o[:100])
    assert not np.any(O.distill_rays(scene, 7, 3, 1000, 0.0)[2])
    assert np.all(O.distill_rays(scene, 7, 3, 1000, 1.0)[2])


def test_shift_keeps_the_first_hit():
    """A hitting ray moved forward by s along itself hits at t - s: recasting
    the shifted rays with the closed-form caster gives back the shifted
    targets; earlier rows and misses stay as they were."""
    scene = I.random_scene(32, 32, seed=0)
    n, first = 6000, 4000
    o, d, _ = O.distill_rays(scene, 9, 0, n, 0.5)
    t, hit = O.cast_scene(scene, o, d)
    o2, t2 = O.distill_shift(o, d, t, hit, first, 9, 0)
    assert np.array_equal(o2[:first], o[:first]) and np.array_equal(t2[:first], t[:first])
    miss = ~hit
    assert np.array_equal(o2[miss], o[miss])
    moved = np.zeros(n, bool)
    moved[first:] = hit[first:]
    s = t[moved] - t2[moved]
    assert np.all(s >= 0) and np.all(s < t[moved])
    assert np.allclose(np.linalg.norm(o2[moved] - o[moved], axis=1), s, rtol=1e-12, atol=1e-15)
    t3, h3 = O.cast_scene(scene, o2[moved], d[moved])
    # the shifted origin is still in front of the first surface
    assert np.mean(h3) > 0.999
    ok = h3 & (t2[moved] > 1e-9)
    assert np.allclose(t3[ok], t2[moved][ok], rtol=1e-9, atol=1e-9)
