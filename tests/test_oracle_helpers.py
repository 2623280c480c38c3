"""Direct pins of the oracle's helper functions, each against something that
does not come from the oracle: central differences, IEEE float32 facts,
hand-placed matrices, and the blob layout the C ABI documents (level
tables first, entry-major with the 2 features of an entry adjacent,
13,058,044 floats; then every layer as W[out][in] row-major and b[out])."""
import numpy as np

from oracle import ddf_oracle as O


def _tiny_mlp(rng, dims):
    return [(rng.normal(size=(fo, fi)) / np.sqrt(fi), rng.normal(size=fo) * 0.1) for fo, fi in dims]


def test_mlp_backward_matches_central_differences():
    """d/dtheta of sum(dz * z) for every weight, bias and input of a 5 -> 7
    -> 6 -> 2 ReLU MLP (Sec. 3.1), away from the ReLU kinks."""
    rng = np.random.default_rng(5)
    layers = _tiny_mlp(rng, [(7, 5), (6, 7), (2, 6)])
    x0 = rng.normal(size=(9, 5))
    dz = rng.normal(size=(9, 2))
    f = lambda x, ly: float(np.sum(dz * O.mlp_forward(x, ly)))
    _, pres, _ = O.mlp_forward(x0, layers, keep=True)
    assert min(np.abs(p).min() for p in pres) > 1e-4     # no pre-activation near a kink
    grads, dx = O.mlp_backward(x0, layers, dz, return_dx=True)
    h = 1e-6
    for li, (w, b) in enumerate(layers):
        for which, arr in ((0, w), (1, b)):
            for i in range(arr.size):
                lp = [(a.copy(), c.copy()) for a, c in layers]
                lm = [(a.copy(), c.copy()) for a, c in layers]
                lp[li][which].flat[i] += h
                lm[li][which].flat[i] -= h
                fd = (f(x0, lp) - f(x0, lm)) / (2 * h)
                assert abs(fd - grads[li][which].flat[i]) < 1e-7, (li, which, i)
    for i in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        assert abs((f(xp, layers) - f(xm, layers)) / (2 * h) - dx.flat[i]) < 1e-7


def test_mlp_backward_relu_derivative_at_zero_is_zero():
    """A hidden unit whose weights and bias are all zero has pre-activation
    exactly 0 on every input; with ReLU'(0) = 0 its incoming weights and
    bias get no gradient, while the other units do."""
    rng = np.random.default_rng(6)
    layers = _tiny_mlp(rng, [(4, 3), (2, 4)])
    layers[0][0][2, :] = 0.0
    layers[0][1][2] = 0.0
    grads = O.mlp_backward(rng.normal(size=(5, 3)), layers, rng.normal(size=(5, 2)))
    assert np.all(grads[0][0][2] == 0.0) and grads[0][1][2] == 0.0
    assert np.count_nonzero(grads[0][0]) > 0


def test_round_f32_follows_ieee_binary32():
    got = O.round_f32(np.array([1 / 3, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 2.0 ** -149,
                                1e-46, 3.4028234663852886e38, -0.1]))
    want = [0.3333333432674408,          # nearest binary32 to 1/3
            1.0,                         # a tie between 1 and 1 + 2^-23 goes to the even one
            1.0 + 2.0 ** -22,            # the tie between 1 + 2^-23 and 1 + 2^-22: even is 1 + 2^-22
            2.0 ** -149,                 # the smallest subnormal is exact
            0.0,                         # below half of it: zero
            3.4028234663852886e38,       # the largest finite binary32
            -0.10000000149011612]
    assert got.tolist() == want


def test_gs_cov_matrices_places_the_six_entries():
    """Rows (xx, xy, xz, yy, yz, zz) become symmetric 3 x 3 matrices, and a
    covariance R diag(s^2) R^T round-trips through its six entries."""
    got = O.gs_cov_matrices(np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0]]))
    assert got.tolist() == [[[1.0, 2.0, 3.0], [2.0, 4.0, 5.0], [3.0, 5.0, 6.0]]]
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    c = q @ np.diag([0.3, 0.02, 0.001]) ** 2 @ q.T
    six = np.array([[c[0, 0], c[0, 1], c[0, 2], c[1, 1], c[1, 2], c[2, 2]]])
    assert np.allclose(O.gs_cov_matrices(six)[0], c, rtol=0, atol=1e-15)


def test_fp8_weight_scales_per_output_channel():
    """s_n = float32(amax_n / 448) per row; an all-zero row gets 1."""
    w = np.array([[-896.0, 1.0, 2.0], [0.0, 0.0, 0.0], [448.0, 0.5, -1.0], [1.0, -0.25, 0.0]])
    s = O.fp8_weight_scales(w)
    assert s.tolist() == [2.0, 1.0, 1.0, float(np.float32(1.0 / 448.0))]
    codes, s2 = O.fp8_quantise_weights(w)
    assert np.array_equal(s, s2)
    assert np.abs(codes).max() <= 448.0 and codes[0, 0] == -448.0 and codes[2, 0] == 448.0


def test_hashgrid_split_follows_the_documented_blob_layout():
    dims = O.hashgrid_mlp_dims()
    n_tab = 13_058_044
    n = n_tab + sum(fo * fi + fo for fo, fi in dims)
    blob = np.arange(n, dtype=np.float64)
    tables, layers = O.hashgrid_split(blob)
    assert 2 * sum(t.shape[0] for t in tables) == n_tab
    off = 0
    for t in tables:                                      # entry-major, features adjacent
        assert t.shape[1] == 2 and t[0].tolist() == [off, off + 1] and t[1, 0] == off + 2
        off += t.size
    (w0, b0) = layers[0]
    assert w0.shape == (64, 59)
    assert w0[0, 0] == n_tab and w0[0, 1] == n_tab + 1 and w0[1, 0] == n_tab + 59
    assert b0[0] == n_tab + 64 * 59
    wo, bo = layers[-1]
    assert wo.shape == (2, 64) and bo[-1] == n - 1


def test_hashgrid_loss_grad_flattens_in_blob_order():
    """The flat gradient sits in blob order: central differences of the loss
    at the largest table entry and the largest MLP entry of the gradient
    match the gradient at those blob indices."""
    rng = np.random.default_rng(8)
    dims = O.hashgrid_mlp_dims()
    n_tab = 13_058_044
    blob = np.concatenate([rng.uniform(-1e-2, 1e-2, n_tab),
                           np.concatenate([np.concatenate([(rng.normal(size=(fo, fi)) / np.sqrt(fi)).ravel(),
                                                           rng.normal(size=fo) * 0.1]) for fo, fi in dims])])
    n = 6
    o = rng.uniform(-0.9, 0.9, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tt = rng.uniform(0.3, 2.0, n)
    y = np.array([1, 0, 1, 1, 0, 1])
    _, g = O.hashgrid_loss_grad(o, d, blob, tt, y)
    assert g.size == blob.size
    h = 1e-6
    for i in (int(np.argmax(np.abs(g[:n_tab]))), n_tab + int(np.argmax(np.abs(g[n_tab:])))):
        bp, bm = blob.copy(), blob.copy()
        bp[i] += h
        bm[i] -= h
        fd = (O.hashgrid_loss_grad(o, d, bp, tt, y)[0] - O.hashgrid_loss_grad(o, d, bm, tt, y)[0]) / (2 * h)
        assert g[i] != 0 and abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 1e-9, (i, fd, g[i])
