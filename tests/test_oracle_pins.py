"""Pins for the FP64 oracle: closed forms, hand-computed networks, number
format definitions, finite differences and brute force. CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ddf_oracle as O
from paper_2606_00817_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ encoding

def test_encoding_width():
    o = np.zeros((3, 3))
    d = np.zeros((3, 3))
    assert O.encode(o, d, 6).shape == (3, 78)
    assert O.encode(o, d, 10).shape == (3, 126)
    assert O.encode_points(o, 10).shape == (3, 63)


@pytest.mark.parametrize("L", [1, 6, 10])
def test_encoding_special_values(L):
    # e = 0: sin terms 0, cos terms 1
    g = O.encode(np.zeros((1, 3)), np.zeros((1, 3)), L)[0]
    assert np.all(g[6::2] == 0) and np.all(g[7::2] == 1)
    # e = 1: sin(pi 2^k) = 0, cos = -1 at k=0, +1 above
    g = O.encode(np.ones((1, 3)), np.ones((1, 3)), L)[0]
    assert np.allclose(g[6::2], 0, atol=1e-12)
    cos = g[7::2].reshape(6, L)
    assert np.allclose(cos[:, 0], -1, atol=1e-12)
    assert np.allclose(cos[:, 1:], 1, atol=1e-12)
    # e = 0.5: sin(pi/2) = 1 at k=0, 0 above; cos 0, -1, then +1
    g = O.encode(np.full((1, 3), 0.5), np.full((1, 3), 0.5), L)[0]
    s = g[6::2].reshape(6, L)
    c = g[7::2].reshape(6, L)
    assert np.allclose(s[:, 0], 1, atol=1e-12) and np.allclose(s[:, 1:], 0, atol=1e-12)
    assert np.allclose(c[:, 0], 0, atol=1e-12)
    if L > 1:
        assert np.allclose(c[:, 1], -1, atol=1e-12)
    if L > 2:
        assert np.allclose(c[:, 2:], 1, atol=1e-12)


def test_encoding_order_coordinate_major():
    # only oy = 0.25 nonzero: its block is columns 6 + 2L .. 6 + 4L
    L = 3
    o = np.array([[0.0, 0.25, 0.0]])
    g = O.encode(o, np.zeros((1, 3)), L)[0]
    blk = g[6 + 2 * L: 6 + 4 * L]
    ref = []
    for k in range(L):
        ref += [math.sin(math.pi * 0.25 * 2 ** k), math.cos(math.pi * 0.25 * 2 ** k)]
    assert np.allclose(blk, ref, atol=1e-15)
    others = np.concatenate([g[6:6 + 2 * L], g[6 + 4 * L:]])
    assert np.allclose(others[0::2], 0) and np.allclose(others[1::2], 1)
    assert g[1] == 0.25


def test_encoding_pythagoras():
    r = I.uniform_rays(257, seed=3)
    g = O.encode(r.origins(), r.dirs(), 10)
    s, c = g[:, 6::2], g[:, 7::2]
    assert np.allclose(s * s + c * c, 1.0, atol=1e-14)


# -------------------------------------------------------- number formats

def test_bf16_hand_values():
    assert O.round_bf16(1.0 + 2.0 ** -8) == 1.0                      # tie -> even
    assert O.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even (up)
    assert O.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert O.round_bf16(-3.0) == -3.0
    assert O.round_bf16(0.0) == 0.0
    assert O.round_bf16(2.0 ** -133) == 2.0 ** -133                  # smallest subnormal


def test_bf16_matches_library_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x.astype(np.float64)), ref)


def _e4m3_table():
    """All finite E4M3 values from the bit definition: sign, 4-bit exponent
    (bias 7), 3-bit mantissa; exponent field 0 is subnormal; S.1111.111 is NaN."""
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue
            v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
            vals += [v, -v]
    return np.unique(np.array(vals))


def test_e4m3_table_and_nearest():
    tab = _e4m3_table()
    assert tab.max() == 448.0 and np.min(tab[tab > 0]) == 2.0 ** -9
    assert np.array_equal(O.round_e4m3(tab), tab)                   # codes are fixed points
    rng = np.random.default_rng(1)
    x = rng.uniform(-460, 460, 50000)
    q = O.round_e4m3(x)
    # brute-force nearest value (ties are measure zero for random doubles)
    idx = np.abs(x[:, None] - tab[None, :]).argmin(axis=1)
    near = np.clip(tab[idx], -448, 448)
    assert np.array_equal(q, near)


def test_e4m3_hand_values():
    assert O.round_e4m3(448.0) == 448.0
    assert O.round_e4m3(464.0) == 448.0       # tie between 448 and (NaN-coded) 480: even -> 448
    assert O.round_e4m3(1000.0) == 448.0      # saturate
    assert O.round_e4m3(-1000.0) == -448.0
    assert O.round_e4m3(2.0 ** -10) == 0.0    # tie between 0 and 2^-9: even -> 0
    assert O.round_e4m3(3 * 2.0 ** -10) == 2.0 ** -8   # tie between 2^-9 and 2^-8 (codes 1, 2): even -> 2
    assert O.round_e4m3(1.0625) == 1.0        # tie between 1 and 1.125: even -> 1
    assert O.round_e4m3(1.1875) == 1.25       # tie between 1.125 and 1.25: even -> 1.25


def test_e4m3_matches_library_cast_in_range():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-8, 5, 20000))).astype(np.float32)
    x = np.clip(x, -448, 448)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.round_e4m3(x.astype(np.float64)), ref)


def test_pow2_scale():
    assert O.pow2_scale(448.0) == 1.0
    assert O.pow2_scale(449.0) == 2.0
    assert O.pow2_scale(1.0) == 2.0 ** -8     # 1/2^-8 = 256 <= 448 < 512
    assert O.pow2_scale(0.0) == 1.0


# ------------------------------------------------------------- heads

def test_heads_closed_forms():
    assert O.softplus(0.0) == pytest.approx(math.log(2.0), abs=1e-16)
    assert O.sigmoid(0.0) == 0.5
    assert O.softplus(50.0) == pytest.approx(50.0 + math.exp(-50.0), rel=1e-15)
    assert O.softplus(-50.0) == pytest.approx(math.exp(-50.0), rel=1e-12)
    assert O.sigmoid(40.0) == pytest.approx(1.0 - math.exp(-40.0), abs=1e-17)
    assert O.sigmoid(-40.0) == pytest.approx(math.exp(-40.0), rel=1e-12)
    z = np.linspace(-30, 30, 101)
    assert np.allclose(O.sigmoid(z) + O.sigmoid(-z), 1.0, atol=1e-15)
    assert np.allclose(O.softplus(z) - O.softplus(-z), z, atol=1e-13)


# ------------------------------------------------------ hand networks

def _hand_blob(net):
    d_in = 6 + 12 * net["octaves"]
    if "W1" in net:
        w1 = np.array(net["W1"], float)
    else:
        w1 = np.zeros((net["width"], d_in))
        for r, c, v in net["W1_sparse"]:
            w1[r, c] = v
    parts = [w1.ravel(), net["b1"]]
    if net["hidden"] == 2:
        parts += [np.ravel(net["W2"]), net["b2"]]
    parts += [np.ravel(net["Wo"]), net["bo"]]
    return np.concatenate([np.asarray(p, float) for p in parts]).astype(np.float32)


@pytest.mark.parametrize("net", _gold("hand_nets.json")["nets"], ids=lambda n: n["name"])
def test_hand_networks(net):
    blob = _hand_blob(net)
    o = np.array([r["o"] for r in net["rays"]], float)
    d = np.array([r["d"] for r in net["rays"]], float)
    out = O.ddf_forward(o, d, blob, net["octaves"], net["width"], net["hidden"])
    z = np.array([r["z"] for r in net["rays"]], float)
    assert np.allclose(out["z"], z, atol=1e-12, rtol=0)
    assert np.allclose(out["t"], np.log1p(np.exp(z[:, 0])), rtol=1e-14)
    assert np.allclose(out["vis"], 1 / (1 + np.exp(-z[:, 1])), rtol=1e-14)


def test_zero_weights_give_bias_heads():
    shape = I.NetShape(2, 8, 3)
    blob = np.zeros(shape.n_params, np.float32)
    blob[-2:] = [0.5, -1.25]
    r = I.uniform_rays(5)
    out = O.ddf_forward(r.origins(), r.dirs(), blob, 2, 8, 3)
    assert np.allclose(out["t"], math.log1p(math.exp(0.5)), rtol=1e-15)
    assert np.allclose(out["vis"], 1 / (1 + math.exp(1.25)), rtol=1e-15)


def test_positive_network_is_plain_matrix_product():
    """With non-negative weights and inputs every ReLU is the identity, so the
    trunk is a chain of affine maps; compare with explicit loops."""
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, (3, 5))
    dims = [(4, 5), (4, 4), (2, 4)]
    layers = [(rng.uniform(0, 1, d), rng.uniform(0, 1, d[0])) for d in dims]
    z = O.mlp_forward(x, layers)
    for i in range(3):
        h = list(x[i])
        for w, b in layers:
            h = [sum(w[o][k] * h[k] for k in range(len(h))) + b[o] for o in range(len(b))]
        assert np.allclose(z[i], h, rtol=1e-14)


def test_blob_layout_counts():
    assert I.NetShape(10, 1280, 8).n_params == 11_642_882
    assert I.NetShape(6, 128, 4).n_params == 78 * 128 + 128 + 3 * (128 * 128 + 128) + 2 * 128 + 2
    with pytest.raises(ValueError):
        O.split_blob(np.zeros(10), O.ddf_dims(1, 2, 1))


# ------------------------------------------------- reduced precision

def test_bf16_mode_with_representable_values_is_exact():
    """When every operand is already a bf16 value and every activation stays
    representable, the bf16 emulation equals the exact forward."""
    net = _gold("hand_nets.json")["nets"][1]
    blob = _hand_blob(net)
    o = np.array([r["o"] for r in net["rays"]], float)
    d = np.array([r["d"] for r in net["rays"]], float)
    a = O.ddf_forward(o, d, blob, 1, 2, 2, "exact")["z"]
    b = O.ddf_forward(o, d, blob, 1, 2, 2, "bf16")["z"]
    assert np.allclose(a, b, atol=1e-12)


def test_reduced_precision_error_scales_with_format():
    shape = I.NetShape(6, 128, 4)
    blob = I.xavier_blob(shape)
    r = I.uniform_rays(512)
    ex = O.ddf_forward(r.origins(), r.dirs(), blob, 6, 128, 4)["z"]
    bf = O.ddf_forward(r.origins(), r.dirs(), blob, 6, 128, 4, "bf16")["z"]
    sc = O.calibrate_act_scales(r.origins(), r.dirs(), blob, 6, 128, 4)
    f8 = O.ddf_forward(r.origins(), r.dirs(), blob, 6, 128, 4, "fp8", sc)["z"]
    e_bf = np.abs(bf - ex).max()
    e_f8 = np.abs(f8 - ex).max()
    assert 0 < e_bf < 2e-2
    assert e_bf < e_f8 < 0.2


def _reduced(name):
    """A hand-worked net of reduced_nets.json: (spec, blob, o, d)."""
    net = _gold("reduced_nets.json")[name]
    names = ["W1", "W2", "W3"][:net["hidden"]]
    parts = []
    for w in names + ["Wo"]:
        b = "bo" if w == "Wo" else "b" + w[1:]
        parts += [np.array(net[w], np.float32).ravel(), np.array(net[b], np.float32)]
    blob = np.concatenate(parts)
    o = np.array([net["ray"]["o"]], float)
    d = np.array([net["ray"]["d"]], float)
    return net, blob, o, d


def _fp8_cases_hold():
    net, blob, o, d = _reduced("fp8")
    return all(O.ddf_forward(o, d, blob, 0, 2, 3, "fp8", c["act_scales"])["z"][0].tolist() == c["z"]
               for c in net["cases"])


def test_fp8_mode_hand_worked_network():
    """e4m3 mode on a 3-layer net worked by hand (tests/golden/reduced_nets.json):
    bf16 layer 1, activation codes with each layer's own input scale (one case
    saturates at 448), weight codes that round, dequantisation by s_in s_n."""
    net, blob, o, d = _reduced("fp8")
    for c in net["cases"]:
        z = O.ddf_forward(o, d, blob, 0, 2, 3, "fp8", c["act_scales"])["z"][0]
        assert z.tolist() == c["z"], (c["act_scales"], z)
    # the scale of layer l is the one of its own input: swapping them moves z
    sw = O.ddf_forward(o, d, blob, 0, 2, 3, "fp8", net["cases"][0]["act_scales"][::-1])["z"][0]
    assert sw.tolist() != net["cases"][0]["z"]


@pytest.mark.parametrize("mistake", ["weights_unrounded", "no_saturation", "acts_unrounded",
                                     "layer1_in_e4m3"])
def test_fp8_pin_catches_planted_mistakes(monkeypatch, mistake):
    """A plausible mistake planted in the oracle makes the hand-worked e4m3
    pin fail."""
    if mistake == "weights_unrounded":
        scales = O.fp8_weight_scales
        monkeypatch.setattr(O, "fp8_quantise_weights", lambda w: (
            (np.asarray(w, np.float32) / scales(w).astype(np.float32)[:, None]).astype(float), scales(w)))
    elif mistake == "no_saturation":
        monkeypatch.setattr(O, "E4M3_MAX", np.inf)
    elif mistake == "acts_unrounded":
        orig = O.round_e4m3
        monkeypatch.setattr(O, "round_e4m3", lambda x: np.asarray(x, float) if np.ndim(x) == 2
                            and np.asarray(x).shape[0] == 1 else orig(x))
    elif mistake == "layer1_in_e4m3":
        monkeypatch.setattr(O, "round_bf16", lambda x: O.round_e4m3(x))
    assert not _fp8_cases_hold()


def test_fp8_calibration_hand_worked():
    """Calibration takes max |h_l| after the ReLU of layers 1..H-1 over the
    batch and rounds each up to a power of two: [0.125, 0.25] here, where the
    encoded input, the pre-activations or the layer after would give 1, 1 or
    0.125 (tests/golden/reduced_nets.json)."""
    net, blob, _, _ = _reduced("fp8")
    cal = net["calibration"]
    o = np.array([r["o"] for r in cal["rays"]], float)
    d = np.array([r["d"] for r in cal["rays"]], float)
    assert O.calibrate_act_scales(o, d, blob, 0, 2, 3) == cal["scales"]
    # the batch maximum: the first ray alone gives the same scales, the
    # second alone a smaller first-layer maximum
    assert O.calibrate_act_scales(o[:1], d[:1], blob, 0, 2, 3) == cal["scales"]
    assert O.calibrate_act_scales(o[1:2], d[1:2], blob, 0, 2, 3)[0] == O.pow2_scale(1.0)


def test_bf16_mode_hand_worked_network():
    """bf16 mode on a 2-layer net worked by hand: the input, a weight and a
    hidden activation (a tie, to even) round, the last hidden activation and
    the head weights do not (tests/golden/reduced_nets.json)."""
    net, blob, o, d = _reduced("bf16")
    z = O.ddf_forward(o, d, blob, 0, 2, 2, "bf16")["z"][0]
    assert z.tolist() == net["z"]
    ex = O.ddf_forward(o, d, blob, 0, 2, 2, "exact")["z"][0]
    assert ex.tolist() != net["z"]


@pytest.mark.parametrize("mistake", ["no_rounding", "round_last_activation"])
def test_bf16_pin_catches_planted_mistakes(monkeypatch, mistake):
    net, blob, o, d = _reduced("bf16")
    if mistake == "no_rounding":
        monkeypatch.setattr(O, "round_bf16", lambda x: np.asarray(x, float))
        z = O.ddf_forward(o, d, blob, 0, 2, 2, "bf16")["z"][0]
    else:
        # the last hidden activation rounded before the head (the head reads it
        # in FP32, unrounded)
        layers = O.split_blob(blob, O.ddf_dims(0, 2, 2))
        _, _, acts = O.mlp_forward(O.encode(o, d, 0), layers, "bf16", keep=True)
        wo, bo = layers[-1]
        z = (O.round_bf16(acts[-1]) @ wo.T + bo)[0]
    assert z.tolist() != net["z"]


def test_fp8_weight_quantiser():
    w = np.array([[0.5, -1.0, 0.25], [448.0 * 3, 1.0, 0.0], [0.0, 0.0, 0.0]], np.float32)
    q, s = O.fp8_quantise_weights(w)
    assert s[0] == np.float32(1.0 / 448.0) and s[1] == np.float32(3.0) and s[2] == 1.0
    assert np.max(np.abs(q)) <= 448.0
    assert q[1, 0] == 448.0 and q[0, 1] == -448.0
    rel = np.abs(q * s[:, None] - w) / np.maximum(np.abs(w), 1e-30)
    assert np.all(rel[w != 0] <= 2.0 ** -4 + 1e-7)   # half a unit in the 4th significant bit


# ------------------------------------------------------ loss / gradient

def test_loss_hand_values():
    z = np.array([[0.0, 0.0], [math.log(math.e - 1.0), 2.0], [3.0, -1.0]])
    # t_hat = [ln2, 1, softplus(3)]; targets: hit at 1.5, hit at 1.0 (exact), miss
    tt = np.array([1.5, 1.0, np.inf])
    y = np.array([1, 1, 0])
    L, dz = O.loss_and_dz(z, tt, y)
    l1 = (abs(math.log(2.0) - 1.5) + 0.0) / 2
    ce = ((math.log(2.0) - 0.0) + (O.softplus(2.0) - 2.0) + O.softplus(-1.0)) / 3
    assert L == pytest.approx(l1 + 0.3 * ce, rel=1e-14)
    assert dz[0, 0] == pytest.approx(-0.5 / 2, rel=1e-14)   # sign -1, sigmoid(0)=1/2, N_hit=2
    assert dz[1, 0] == 0.0                                  # sign(0) = 0
    assert dz[2, 0] == 0.0                                  # miss rays carry no L1 term
    assert dz[2, 1] == pytest.approx(0.3 * O.sigmoid(-1.0) / 3, rel=1e-14)
    assert dz[1, 1] == pytest.approx(0.3 * (O.sigmoid(2.0) - 1) / 3, rel=1e-14)


def test_loss_clamp_stops_gradient():
    z = np.array([[10.0, 1.0]])                    # t_hat ~ 10 > clamp 4
    L, dz = O.loss_and_dz(z, np.array([1.0]), np.array([1]))
    assert L == pytest.approx(3.0 + 0.3 * (O.softplus(1.0) - 1.0), rel=1e-12)
    assert dz[0, 0] == 0.0


def test_gradient_matches_central_differences():
    shape = I.NetShape(1, 6, 2)
    rng = np.random.default_rng(5)
    blob = (rng.standard_normal(shape.n_params) * 0.7).astype(np.float64)
    r = I.uniform_rays(16, seed=7)
    o, d = r.origins(), r.dirs()
    tt = rng.uniform(0.2, 3.0, 16)
    y = rng.integers(0, 2, 16)
    L0, g = O.ddf_loss_grad(o, d, blob, 1, 6, 2, tt, y)
    h = 1e-6
    fd = np.empty_like(blob)
    for i in range(blob.size):
        bp = blob.copy(); bp[i] += h
        bm = blob.copy(); bm[i] -= h
        fd[i] = (O.ddf_loss_grad(o, d, bp, 1, 6, 2, tt, y)[0] - O.ddf_loss_grad(o, d, bm, 1, 6, 2, tt, y)[0]) / (2 * h)
    # kinks (ReLU at 0, |.| at 0, clamp) are measure zero for these random values
    err = np.abs(fd - g) / np.maximum(1e-6, np.abs(g))
    assert np.median(err) < 1e-6
    assert np.mean(err < 1e-4) > 0.98


def test_adam_closed_forms():
    g = np.array([0.5, -2.0, 1e-3])
    w = np.zeros(3)
    w1, m1, v1 = O.adam_step(w, g, np.zeros(3), np.zeros(3), 1, 1e-3)
    assert np.allclose(w1, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    w2, _, _ = O.adam_step(w1, g, m1, v1, 2, 1e-3)
    assert np.allclose(w2 - w1, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10)
    # hand value: step 2 with gradients 1 then 0
    w1, m1, v1 = O.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, 1.0)
    w2, m2, v2 = O.adam_step(w1, np.zeros(1), m1, v1, 2, 1.0)
    mh = 0.09 / (1 - 0.81)
    vh = 0.000999 / (1 - 0.999 ** 2)
    w1_hand = -1.0 / (1.0 + 1e-8)                 # step 1: m_hat = v_hat = 1
    assert w2[0] == pytest.approx(w1_hand - mh / (math.sqrt(vh) + 1e-8), rel=1e-12)


# ------------------------------------------------------ analytic caster

def test_caster_closed_forms():
    gold = _gold("caster_closed_forms.json")
    for c in gold["spheres"]:
        t = O.cast_spheres(np.array([c["o"]], float), np.array([c["d"]], float),
                           np.array([c["c"]], float), np.array([c["r"]], float))[0]
        if c["t"] is None:
            assert np.isinf(t), c
        else:
            assert t == pytest.approx(c["t"], abs=1e-12), c
    for c in gold["boxes"]:
        t = O.cast_boxes(np.array([c["o"]], float), np.array([c["d"]], float),
                         np.array([c["lo"]], float), np.array([c["hi"]], float))[0]
        if c["t"] is None:
            assert np.isinf(t), c
        else:
            assert t == pytest.approx(c["t"], abs=1e-12), c


def _inside_each(scene, p):
    """[n, n_prims] closed-set inside flags for every primitive."""
    cols = [np.linalg.norm(p - c, axis=1) <= r for c, r in zip(scene.centers, scene.radii)]
    cols += [np.all((p >= lo) & (p <= hi), axis=1) for lo, hi in zip(scene.box_lo, scene.box_hi)]
    return np.stack(cols, axis=1)


def test_caster_against_brute_force_march():
    """March every ray in steps of 1e-4 with closed-form inside tests; the first
    step where any primitive's inside flag changes must bracket the cast t."""
    scene = I.random_scene(8, 8, seed=11)
    r = I.uniform_rays(150, seed=12)
    o, d = r.origins().astype(float), r.dirs().astype(float)
    t, hit = O.cast_scene(scene, o, d)
    step = 1e-4
    ts = np.arange(0, 4.0 + step, step)
    n_ok = 0
    for i in range(o.shape[0]):
        pts = o[i] + ts[:, None] * d[i]
        ins = _inside_each(scene, pts)
        change = np.any(ins[1:] != ins[:-1], axis=1)
        k = np.argmax(change) if change.any() else -1
        if k < 0:
            assert not (hit[i] and t[i] < 4.0 - step), i
        else:
            assert hit[i]
            assert ts[k] - 1e-9 <= t[i] <= ts[k + 1] + 1e-9, (i, t[i], ts[k])
            n_ok += 1
    assert n_ok > 20


def test_caster_hit_points_lie_on_surfaces():
    scene = I.random_scene(16, 16, seed=13)
    r = I.uniform_rays(2000, seed=14)
    o, d = r.origins().astype(float), r.dirs().astype(float)
    t, hit = O.cast_scene(scene, o, d)
    p = o[hit] + t[hit, None] * d[hit]
    ds = np.min(np.abs(np.linalg.norm(p[:, None, :] - scene.centers[None], axis=2) - scene.radii[None]), axis=1)
    q = np.abs(p[:, None, :] - 0.5 * (scene.box_lo + scene.box_hi)[None]) - 0.5 * (scene.box_hi - scene.box_lo)[None]
    on_box = np.any((np.abs(np.max(q, axis=2)) < 1e-9) & (np.max(q, axis=2) < 1e-9), axis=1)
    assert np.all((ds < 1e-9) | on_box)
    assert hit.mean() > 0.2


def test_sphere_trace_closed_form_and_caster_agreement():
    g = _gold("caster_closed_forms.json")
    c = g["sphere_trace"][0]
    sc = I.Scene(np.array([c["c"]], float), np.array([c["r"]], float), np.zeros((0, 3)), np.zeros((0, 3)))
    t, hit, steps = O.sphere_trace(lambda p: O.union_sdf(sc, p), np.array([c["o"]], float), np.array([c["d"]], float))
    assert hit[0] and t[0] == pytest.approx(c["t"], abs=1e-12) and steps[0] == c["steps"]
    for b in g["box_sdf"]:
        sb = I.Scene(np.zeros((0, 3)), np.zeros(0), np.array([b["lo"]], float), np.array([b["hi"]], float))
        assert O.union_sdf(sb, np.array([b["p"]], float))[0] == pytest.approx(b["s"], abs=1e-12)
    # random scene: rays starting outside every primitive agree with the caster
    scene = I.random_scene(8, 8, seed=21)
    r = I.uniform_rays(3000, seed=22)
    o, d = r.origins().astype(float), r.dirs().astype(float)
    outside = O.union_sdf(scene, o) > 0.01
    o, d = o[outside], d[outside]
    tc, hc = O.cast_scene(scene, o, d)
    ts, hs, st = O.sphere_trace(lambda p: O.union_sdf(scene, p), o, d, max_steps=512, eps=1e-6, t_max=4.0)
    both = hs & hc
    assert both.mean() > 0.15
    assert np.all(np.abs(ts[both] - tc[both]) < 1e-3)
    # a caster hit inside t_max is found by the tracer unless it is a near-graze
    assert np.mean(hs[hc & (tc < 3.5)]) > 0.97


# ------------------------------------------------------ queries

def test_shadow_and_ao_hand_values():
    o = np.array([[0, 0, 0], [0, 0, 0], [0, 0, 0]], float)
    light = (3.0, 4.0, 0.0)                        # distance 5
    t = np.array([4.0, 6.0, 4.0])
    z1 = np.array([1.0, 1.0, -1.0])
    assert list(O.shadow(t, z1, o, light)) == [True, False, False]
    hit = np.array([1, 0, 1, 1, 1, 0], bool)
    vis = np.array([0.9, 0.1, 0.8, 0.7, 0.6, 0.2])
    hard, soft = O.ambient_occlusion(hit, vis, [0, 2, 2, 6])
    assert np.allclose(hard, [0.5, 1.0, 0.25])
    assert np.allclose(soft, [0.5, 1.0, 1 - 2.3 / 4])


def test_train_grad_reduces_to_pinned_gradient():
    """With rounding off, the training-step gradient is the exact gradient that
    central differences pin above; with bf16 rounding it stays close."""
    shape = I.NetShape(2, 16, 3)
    rng = np.random.default_rng(8)
    blob = (rng.standard_normal(shape.n_params) * 0.5)
    r = I.uniform_rays(64, seed=9)
    tt = rng.uniform(0.2, 3.0, 64)
    y = rng.integers(0, 2, 64)
    L0, g0 = O.ddf_loss_grad(r.origins(), r.dirs(), blob, 2, 16, 3, tt, y)
    L1, g1 = O.train_grad(r.origins(), r.dirs(), blob, 2, 16, 3, tt, y, precision="exact")
    assert L1 == pytest.approx(L0, rel=1e-14)
    assert np.allclose(g1, g0, rtol=1e-12, atol=1e-15)
    L2, g2 = O.train_grad(r.origins(), r.dirs(), blob, 2, 16, 3, tt, y, precision="bf16")
    assert abs(L2 - L0) < 2e-2 * abs(L0)
    assert np.linalg.norm(g2 - g0) < 5e-2 * np.linalg.norm(g0)


def test_sdf_grad_matches_central_differences():
    L, W, H = 1, 6, 2
    n = (3 + 6 * L) * W + W + (H - 1) * (W * W + W) + W + 1
    rng = np.random.default_rng(10)
    blob = rng.standard_normal(n) * 0.6
    p = rng.uniform(-1, 1, (24, 3))
    s_t = rng.uniform(-0.5, 0.5, 24)
    L0, g = O.sdf_train_grad(p, blob, L, W, H, s_t, precision="exact")
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        bp = blob.copy(); bp[i] += h
        bm = blob.copy(); bm[i] -= h
        fd[i] = (O.sdf_train_grad(p, bp, L, W, H, s_t, "exact")[0]
                 - O.sdf_train_grad(p, bm, L, W, H, s_t, "exact")[0]) / (2 * h)
    err = np.abs(fd - g) / np.maximum(1e-6, np.abs(g))
    assert np.median(err) < 1e-6 and np.mean(err < 1e-4) > 0.97
    # the loss is the mean absolute error of the plain network
    s = O.sdf_mlp(p, blob, L, W, H)
    assert L0 == pytest.approx(np.mean(np.abs(s - s_t)), rel=1e-14)
