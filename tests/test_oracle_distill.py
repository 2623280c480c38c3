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


def test_sampler_invariants():
    scene = I.random_scene(32, 32, seed=0)
    n = 40000
    o, d, surf = O.distill_rays(scene, 7, 3, n, 0.5)
    assert abs(surf.mean() - 0.5) < 0.01
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-14)
    # surface rays start 1e-3 off some primitive's surface, outside it
    g = _surface_gap(scene, o[surf][:4000])
    assert np.all(np.abs(g - 1e-3).min(1) < 1e-12)
    # every primitive is chosen about equally often (1/64 of the surface rays)
    near = np.argmin(np.abs(_surface_gap(scene, o[surf]) - 1e-3), axis=1)
    cnt = np.bincount(near, minlength=64)
    assert cnt.min() > 200 and cnt.max() < 460                  # 312.5 expected
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
