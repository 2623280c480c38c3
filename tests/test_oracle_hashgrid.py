"""Pins of the oracle's hash-grid field (Sec. 3.4) against values that do not
come from the oracle itself: the paper's layout figures, hand-computed spatial
hashes, affine fields that trilinear interpolation must reproduce exactly,
table entries at grid vertices, continuity across cell faces, clamping, and
the direction encoding's special values."""
import json
import os

import numpy as np

from oracle import ddf_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_layout_matches_the_paper():
    g = _load("hashgrid_layout.json")
    assert O.hashgrid_resolutions() == g["resolutions"]
    assert O.hashgrid_table_sizes() == g["table_sizes"]
    assert sum(O.hashgrid_table_sizes()) == g["table_entries"]
    assert 2 * g["table_entries"] == g["table_params"]
    assert sum(fo * fi + fo for fo, fi in O.hashgrid_mlp_dims()) == g["mlp_params"]
    # "about 13M parameters", "52 MB" of float32
    assert 12.5e6 < g["table_params"] < 13.5e6
    assert 51e6 < 4 * (g["table_params"] + g["mlp_params"]) < 53e6


def test_spatial_hash_hand_values():
    g = _load("hashgrid_spatial_hash.json")
    ijk = np.array([v["ijk"] for v in g["vertices"]])
    got = O.hashgrid_index(ijk, res=81, size=1 << 19)       # level 4: hashed
    assert got.tolist() == [v["hash"] for v in g["vertices"]]


def test_dense_index_is_row_major():
    res = 16
    ijk = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [16, 16, 16]])
    got = O.hashgrid_index(ijk, res, (res + 1) ** 3)
    assert got.tolist() == [0, 1, 17, 289, 17 ** 3 - 1]


def test_dense_levels_reproduce_affine_fields():
    """Trilinear interpolation reproduces any affine function of position, so
    tables holding a . v + b at every vertex v (normalised to [0, 1]^3) give
    features a . x01 + b at every point: pins the corner enumeration, the
    weights and the dense indexing together."""
    rng = np.random.default_rng(0)
    res = O.hashgrid_resolutions()[:4]
    a = rng.normal(size=(2, 3))
    b = rng.normal(size=2)
    tables = []
    for n in res:
        g = np.arange(n + 1)
        k, j, i = np.meshgrid(g, g, g, indexing="ij")          # row-major: i fastest
        v = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) / n
        tables.append(v @ a.T + b)
    x = rng.uniform(-1, 1, size=(500, 3))
    x[:4] = [[-1, -1, -1], [1, 1, 1], [1, -1, 0.3], [0, 0, 0]]   # faces and corners
    f = O.hashgrid_encode(x, tables, res)
    want = ((x + 1) / 2) @ a.T + b
    for lvl in range(4):
        assert np.abs(f[:, 2 * lvl:2 * lvl + 2] - want).max() < 1e-12


def test_hashed_level_vertices_read_their_entry():
    """A point on a grid vertex of a hashed level reads exactly the entry the
    hand-checked hash picks."""
    g = _load("hashgrid_spatial_hash.json")
    res = 81
    table = np.random.default_rng(1).normal(size=(1 << 19, 2))
    for v in g["vertices"]:
        x = (np.array(v["ijk"], float) / res) * 2 - 1
        f = O.hashgrid_encode(x[None, :], [table], [res])
        assert np.array_equal(f[0], table[v["hash"]])


def test_continuity_across_cell_faces_and_clamping():
    res = [81, 7006]
    rng = np.random.default_rng(2)
    tables = [rng.normal(size=(1 << 19, 2)) for _ in res]
    bound = 8 * np.abs(np.stack(tables)).max()   # |d feature / d x01| <= 2 N max|entry| x 4
    for n in res:
        face = (37 / n) * 2 - 1                                   # x on a cell face
        base = np.array([[face, 0.123, -0.456]])
        jumps = []
        for eps in (1e-6, 1e-9):
            lo = O.hashgrid_encode(base - [eps, 0, 0], tables, res)
            hi = O.hashgrid_encode(base + [eps, 0, 0], tables, res)
            jumps.append(np.abs(lo - hi).max())
            assert jumps[-1] <= eps * max(res) * bound      # Lipschitz, no jump at the face
        assert jumps[1] <= 2e-3 * jumps[0] + 1e-12          # shrinks with eps (linear)
    inside = rng.uniform(-1, 1, size=(50, 3))
    outside = inside.copy()
    outside[:, 0] = np.where(inside[:, 0] > 0, 3.0, -3.0)
    clamped = inside.copy()
    clamped[:, 0] = np.where(inside[:, 0] > 0, 1.0, -1.0)
    assert np.array_equal(O.hashgrid_encode(outside, tables, res),
                          O.hashgrid_encode(clamped, tables, res))


def test_direction_encoding_special_values():
    d = np.array([[1.0, 0.0, 0.5]])
    e = O.encode_dir(d, 4)
    assert e.shape == (1, 27)
    assert np.array_equal(e[0, :3], d[0])
    sx, cx = e[0, 3:11:2], e[0, 4:12:2]          # coordinate x = 1, bands 0..3
    assert np.allclose(sx, 0, atol=1e-15) and np.allclose(cx, [-1, 1, 1, 1])
    sy, cy = e[0, 11:19:2], e[0, 12:20:2]        # coordinate y = 0
    assert np.array_equal(sy, np.zeros(4)) and np.array_equal(cy, np.ones(4))
    sz = e[0, 19:27:2]                           # z = 0.5: sin(pi/2) = 1, sin(pi) = 0, ...
    assert np.allclose(sz, [1, 0, 0, 0], atol=1e-15)


def test_forward_reads_the_code_in_order():
    """An MLP that passes code entry j straight to z0 (ReLU-safe: positive
    tables and directions) returns exactly that entry: level l feature f at
    j = 2 l + f, then the direction encoding from j = 32."""
    tables_sizes = O.hashgrid_table_sizes()
    rng = np.random.default_rng(3)
    tables = [rng.uniform(0.5, 1.5, size=(t, 2)) for t in tables_sizes]
    o = rng.uniform(-1, 1, size=(20, 3))
    d = np.abs(rng.normal(size=(20, 3)))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    code = np.concatenate([O.hashgrid_encode(o, tables, O.hashgrid_resolutions()),
                           O.encode_dir(d)], axis=1)
    for j in (0, 5, 31, 32, 34):
        dims = O.hashgrid_mlp_dims()
        w1 = np.zeros(dims[0]); w1[0, j] = 1.0
        w2 = np.zeros(dims[1]); w2[0, 0] = 1.0
        wo = np.zeros(dims[2]); wo[0, 0] = 1.0
        mlp = [w1, np.zeros(64), w2, np.zeros(64), wo, np.zeros(2)]
        blob = np.concatenate([t.ravel() for t in tables] + [m.ravel() for m in mlp])
        z = O.hashgrid_forward(o, d, blob)["z"]
        assert np.allclose(z[:, 0], code[:, j], rtol=1e-13, atol=0), j


def _tiny_field(rng):
    """Two levels: a dense 3^3-vertex grid and a hashed one (res 5, 16
    entries); MLP 4 + 27 -> 6 -> 6 -> 2."""
    res = [2, 5]
    sizes = [27, 16]
    tables = [rng.normal(size=(s, 2)) for s in sizes]
    dims = [(6, 4 + 27), (6, 6), (2, 6)]
    layers = [(rng.normal(size=dims[i]) * 0.6, rng.normal(size=dims[i][0]) * 0.3)
              for i in range(3)]
    return res, tables, layers


def test_hashgrid_gradient_matches_central_differences():
    """Every table entry and every MLP parameter of a tiny field (a dense and
    a hashed level, with collisions) against central differences of the
    loss."""
    rng = np.random.default_rng(11)
    res, tables, layers = _tiny_field(rng)
    n = 40
    o = rng.uniform(-1.1, 1.1, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tt = rng.uniform(0.2, 3.0, n)
    y = rng.integers(0, 2, n)
    f = lambda tb, ly: O.hashgrid_field_loss_grad(o, d, tb, res, ly, tt, y, log2_t=4)
    L0, dtab, grads = f(tables, layers)
    h = 1e-6
    got, fd = [], []
    for l in range(2):
        for i in range(tables[l].size):
            tp = [t.copy() for t in tables]
            tm = [t.copy() for t in tables]
            tp[l].flat[i] += h
            tm[l].flat[i] -= h
            fd.append((f(tp, layers)[0] - f(tm, layers)[0]) / (2 * h))
            got.append(dtab[l].flat[i])
    for li in range(3):
        for which in range(2):
            arr = layers[li][which]
            for i in range(arr.size):
                lp = [(w.copy(), b.copy()) for w, b in layers]
                lm = [(w.copy(), b.copy()) for w, b in layers]
                lp[li][which].flat[i] += h
                lm[li][which].flat[i] -= h
                fd.append((f(tables, lp)[0] - f(tables, lm)[0]) / (2 * h))
                got.append(grads[li][which].flat[i])
    fd, got = np.array(fd), np.array(got)
    err = np.abs(fd - got) / np.maximum(1e-6, np.abs(got))
    assert np.median(err) < 1e-6
    assert np.mean(err < 1e-4) > 0.98
    assert np.count_nonzero(np.array(got[:27 * 2 + 16 * 2])) > 40   # the tables do get gradient


def test_hashgrid_table_gradient_is_a_weighted_scatter():
    """Feature gradient 1 on one point: its 8 corners of a dense level receive
    exactly their trilinear weights (which sum to 1)."""
    x = np.array([[0.1, -0.35, 0.62]])
    res = [4]
    dfeat = np.array([[1.0, 0.0]])
    g = O.hashgrid_encode_backward(x, dfeat, [125], res)[0]
    assert abs(g[:, 0].sum() - 1.0) < 1e-15 and np.count_nonzero(g[:, 0]) == 8
    assert np.all(g[:, 1] == 0)
    u = (x[0] + 1) / 2 * 4
    i0 = np.floor(u).astype(int)
    w = u - i0
    corner = g[i0[0] + 5 * (i0[1] + 5 * i0[2]), 0]       # the (0,0,0) corner
    assert abs(corner - (1 - w[0]) * (1 - w[1]) * (1 - w[2])) < 1e-15


def test_fp32_positions_round_like_float32():
    """The fp32 position mode picks the cell and in-cell coordinates from
    float32 arithmetic: u = f32(f32(f32(x) + 1) * 0.5) * f32(N). At a
    coordinate whose float32 box position rounds across a cell face, the two
    modes pick different cells; everywhere the features stay within the
    float32 position error (N x 2^-24 of a cell) of the exact ones."""
    res = [7006]
    # x such that (x + 1) / 2 * 7006 sits 1e-6 below the face at 3000 in float64
    x_exact = (3000 - 1e-6) / 7006 * 2 - 1
    x = np.array([[x_exact, 0.1, -0.2]], np.float32).astype(np.float64)
    i_ex, w_ex = O.hashgrid_cell(x, 7006, "exact")
    i_32, w_32 = O.hashgrid_cell(x, 7006, "fp32")
    f = np.float32
    u32 = f(f(f(x[0, 0]) + f(1)) * f(0.5)) * f(7006)
    assert i_32[0, 0] == int(np.floor(u32)) and w_32[0, 0] == float(u32) - int(np.floor(u32))
    rng = np.random.default_rng(4)
    table = rng.normal(size=(1 << 19, 2))
    pts = rng.uniform(-1, 1, size=(2000, 3)).astype(np.float32).astype(np.float64)
    fe = O.hashgrid_encode(pts, [table], res)
    f3 = O.hashgrid_encode(pts, [table], res, positions="fp32")
    lip = 2 * 4 * np.abs(table).max()                       # per unit of u, 4 corners per axis
    assert np.abs(fe - f3).max() <= lip * 7006 * 2.0 ** -23
    assert np.abs(fe - f3).max() > 0                        # float32 positions do move features
