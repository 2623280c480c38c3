"""FP64 CPU oracle for the batched DDF query path — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The product path (the CUDA library and
its Python binding) never does, and this module never imports the product:
the two share nothing but the seeded input generators.

Every function is the plain definition, evaluated in float64 on the float32
inputs (rays, weights) promoted to double. A matrix product (numpy ``@``) is
the only library step used on the network path.

What the paper fixes and what this module reads into it:
  * Sec. 3.1, Eq. (1): f(x, d) = (t, xi); t is the distance to the first
    surface along d, xi the probability that the ray hits at all.
  * Sec. 4.3 and Table 2: the first DDF uses a sinusoidal encoding with a
    wide ReLU MLP. Reading: raw (x, d) first, then for each of the six
    coordinates, for k = 0..L-1, sin(pi 2^k e) then cos(pi 2^k e).
  * The two outputs: t = softplus(z0), xi = sigmoid(z1); a ray counts as a
    hit when z1 > 0.
  * Sec. 3.2 and 3.4: an L1 term on distance clamped at the box scale plus
    a cross-entropy term on the hit weighted 0.3, trained with Adam.
    Reading: the L1 term averages over hit rays only, the cross-entropy
    over all rays; Adam with (0.9, 0.999, 1e-8) and bias correction.
  * Sec. 3.3: a shadow ray is occluded when it hits within the light
    distance; ambient occlusion averages the hit flag over hemisphere
    directions.
  * Sec. 3.2: supervision from an exact ray cast of the geometry; here the
    geometry is a union of spheres and boxes with closed-form intersections.
  * Sec. 3.2 / 3.4: the distillation schedule (training-ray sampler, the
    ray-march shifted points, the cosine learning rate; readings in its
    section below).
  * Sec. 4.4: sphere tracing an SDF is the sequential baseline.
  * Sec. 3.4: the hash-grid field (readings in its section below).
  * Sec. 3.3 / the application: shadow and AO images (readings below).
  * Sec. 3.2 / Sec. 4.2 (the supervision study): Gaussian-rendered depth.

Reduced-precision modes emulate where the GPU path rounds (bf16 operands,
or e4m3 operands with per-output-channel weight scales and per-tensor
power-of-two activation scales) while every sum stays in float64; the
rounding functions are written from the number formats' definitions.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, hand-computed networks, finite differences, brute force, and
library casts for the rounding functions). The paper's own timing and
accuracy tables need its datasets and weights and are not reproduced.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64

# ----------------------------------------------------------------- encoding


def encode(o: np.ndarray, d: np.ndarray, octaves: int) -> np.ndarray:
    """Sinusoidal positional encoding of a ray (Sec. 4.3, Table 2).

    o, d: [n,3]. Returns [n, 6 + 12*octaves] float64: o, d, then per
    coordinate c (ox, oy, oz, dx, dy, dz) and band k: sin(pi 2^k e_c),
    cos(pi 2^k e_c).
    """
    e = np.concatenate([np.asarray(o, F64), np.asarray(d, F64)], axis=1)
    n = e.shape[0]
    out = np.empty((n, 6 + 12 * octaves), dtype=F64)
    out[:, :6] = e
    col = 6
    for c in range(6):
        for k in range(octaves):
            arg = np.pi * np.ldexp(e[:, c], k)
            out[:, col] = np.sin(arg)
            out[:, col + 1] = np.cos(arg)
            col += 2
    return out


def encode_points(p: np.ndarray, octaves: int) -> np.ndarray:
    """3D Fourier encoding of a point for the SDF baseline (Sec. 4.4):
    p, then per coordinate and band sin(pi 2^k p_c), cos(pi 2^k p_c)."""
    p = np.asarray(p, F64)
    n = p.shape[0]
    out = np.empty((n, 3 + 6 * octaves), dtype=F64)
    out[:, :3] = p
    col = 3
    for c in range(3):
        for k in range(octaves):
            arg = np.pi * np.ldexp(p[:, c], k)
            out[:, col] = np.sin(arg)
            out[:, col + 1] = np.cos(arg)
            col += 2
    return out


# ------------------------------------------------------- number formats


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significant bits, binary32 exponent
    range), ties to even. Values are returned as float64."""
    x = np.asarray(x, F64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    e = np.maximum(e, -125)                  # below 2^-126 the spacing is fixed (subnormals)
    q = np.ldexp(np.rint(np.ldexp(x, 8 - e)), e - 8)
    return np.where(x == 0, x, q)


E4M3_MAX = 448.0


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest OCP FP8 E4M3 value (4 significant bits, exponent
    bias 7, smallest normal 2^-6, subnormal spacing 2^-9, largest finite
    448), ties to even, saturating to +-448. Returned as float64."""
    x = np.asarray(x, F64)
    m, e = np.frexp(x)
    e = np.maximum(e, -5)                    # 2^-6 = 0.5 * 2^-5: subnormal range below
    q = np.ldexp(np.rint(np.ldexp(x, 4 - e)), e - 4)
    q = np.clip(q, -E4M3_MAX, E4M3_MAX)
    return np.where(x == 0, x, q)


def round_f32(x) -> np.ndarray:
    return np.asarray(x, F64).astype(np.float32).astype(F64)


# ------------------------------------------------------------- network


def softplus(z):
    z = np.asarray(z, F64)
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    z = np.asarray(z, F64)
    ez = np.exp(-np.abs(z))
    return np.where(z >= 0, 1.0 / (1.0 + ez), ez / (1.0 + ez))


def split_blob(blob, dims):
    """[(W[out,in], b[out])] from the flat blob; dims = [(out, in), ...]."""
    blob = np.asarray(blob)
    out, off = [], 0
    for fo, fi in dims:
        w = blob[off:off + fo * fi].reshape(fo, fi).astype(F64)
        off += fo * fi
        b = blob[off:off + fo].astype(F64)
        off += fo
        out.append((w, b))
    if off != blob.size:
        raise ValueError(f"blob has {blob.size} floats, layers need {off}")
    return out


def ddf_dims(octaves: int, width: int, hidden: int):
    d_in = 6 + 12 * octaves
    return [(width, d_in)] + [(width, width)] * (hidden - 1) + [(2, width)]


def fp8_weight_scales(w: np.ndarray) -> np.ndarray:
    """Per-output-channel e4m3 scale s_n = amax_n / 448, rounded to float32."""
    amax = np.max(np.abs(np.asarray(w, F64)), axis=1)
    s = round_f32(amax / E4M3_MAX)
    return np.where(s > 0, s, 1.0)


def fp8_quantise_weights(w: np.ndarray):
    """(codes, scales): codes = e4m3(float32(w / s_n)) with the division done
    in float32, as float64 values."""
    s = fp8_weight_scales(w)
    q = (np.asarray(w, np.float32) / s.astype(np.float32)[:, None]).astype(F64)
    return round_e4m3(q), s


def pow2_scale(amax: float) -> float:
    """Smallest power of two s with amax / s <= 448 (1.0 when amax is 0)."""
    if amax <= 0:
        return 1.0
    return float(2.0 ** np.ceil(np.log2(amax / E4M3_MAX)))


def mlp_forward(x0, layers, precision: str = "exact", act_scales=None, keep=False):
    """ReLU MLP trunk + linear 2-output head (Sec. 3.1), from an encoded input.

    precision:
      "exact": every operation in float64.
      "bf16":  the encoded input, hidden weights and every hidden activation
               except the last are rounded to bfloat16 before they enter a
               product; sums, bias, ReLU stay float64; the head uses float32
               weights on the unrounded last activation.
      "fp8":   layer 1 as in "bf16"; layers 2..H take e4m3 activation codes
               a_q = e4m3(h / s_l) (s_l from act_scales, one per layer input)
               and e4m3 weight codes with per-output-channel scales s_n; the
               pre-activation is (sum a_q w_q) * s_l * s_n + b.
    Returns z [n,2] (and the list of pre-activations and activations if keep).
    """
    hidden = layers[:-1]
    wo, bo = layers[-1]
    h = np.asarray(x0, F64)
    pres, acts = [], [h]
    H = len(hidden)
    for l, (w, b) in enumerate(hidden):
        if precision == "exact":
            pre = h @ w.T + b
        elif precision == "bf16" or (precision == "fp8" and l == 0):
            pre = round_bf16(h) @ round_bf16(w).T + b
        elif precision == "fp8":
            s_in = act_scales[l - 1]
            a_q = round_e4m3(h / s_in)
            w_q, s_w = fp8_quantise_weights(w)
            pre = (a_q @ w_q.T) * (s_in * s_w)[None, :] + b
        else:
            raise ValueError(precision)
        h = np.maximum(pre, 0.0)
        if precision == "bf16" and l < H - 1:
            h = round_bf16(h)
        if keep:
            pres.append(pre)
            acts.append(h)
    z = h @ wo.T + bo
    if keep:
        return z, pres, acts
    return z


def ddf_forward(o, d, blob, octaves: int, width: int, hidden: int,
                precision: str = "exact", act_scales=None):
    """DDF query f(x, d) = (t, xi) of Sec. 3.1, Eq. (1): encode, MLP, heads.

    Returns dict(t, vis, z) with t = softplus(z0), vis = sigmoid(z1)."""
    layers = split_blob(blob, ddf_dims(octaves, width, hidden))
    z = mlp_forward(encode(o, d, octaves), layers, precision, act_scales)
    return {"t": softplus(z[:, 0]), "vis": sigmoid(z[:, 1]), "z": z}


def calibrate_act_scales(o, d, blob, octaves, width, hidden):
    """Per-tensor power-of-two scales for the e4m3 inputs of layers 2..H:
    s_l = pow2_scale(max |h_l|) over a calibration batch, with h_l taken from
    the exact forward pass."""
    layers = split_blob(blob, ddf_dims(octaves, width, hidden))
    _, _, acts = mlp_forward(encode(o, d, octaves), layers, "exact", keep=True)
    return [pow2_scale(float(np.max(np.abs(a)))) for a in acts[1:hidden]]


# ------------------------------------------------------ loss / gradients

LOSS_CLAMP = 4.0
LOSS_CE_WEIGHT = 0.3


def loss_and_dz(z, t_target, hit_target, clamp=LOSS_CLAMP, lam=LOSS_CE_WEIGHT):
    """Distillation loss of Sec. 3.2/3.4 and its gradient w.r.t. z.

    L = (1/max(1,N_hit)) sum_{hit} |min(t_hat, c) - min(t*, c)|
        + lam (1/B) sum_i [softplus(z1) - y z1]
    with t_hat = softplus(z0). dL/dz0 uses d min(t,c)/dt = 1[t <= c] and
    sign(0) = 0; dL/dz1 = lam (sigmoid(z1) - y) / B.
    """
    z = np.asarray(z, F64)
    y = np.asarray(hit_target).astype(F64)
    tt = np.asarray(t_target, F64)
    B = z.shape[0]
    nh = max(1.0, float(y.sum()))
    th = softplus(z[:, 0])
    diff = np.minimum(th, clamp) - np.minimum(tt, clamp)
    l1 = np.sum(y * np.abs(diff)) / nh
    ce = np.sum(softplus(z[:, 1]) - y * z[:, 1]) / B
    L = l1 + lam * ce
    dz = np.zeros_like(z)
    dz[:, 0] = y * np.sign(diff) * (th <= clamp) * sigmoid(z[:, 0]) / nh
    dz[:, 1] = lam * (sigmoid(z[:, 1]) - y) / B
    return L, dz


def mlp_backward(x0, layers, dz, precision="exact", return_dx=False):
    """Gradient of sum(dz * z) w.r.t. every weight and bias (reverse-mode
    chain rule through the linear layers and ReLUs; ReLU'(0) = 0).
    Returns a list [(dW, db)] matching ``layers`` (and the gradient w.r.t.
    the input x0 if return_dx)."""
    z, pres, acts = mlp_forward(x0, layers, precision, keep=True)
    grads = [None] * len(layers)
    wo, _ = layers[-1]
    dz = np.asarray(dz, F64)
    grads[-1] = (dz.T @ acts[-1], dz.sum(axis=0))
    dh = dz @ wo
    for l in range(len(layers) - 2, -1, -1):
        w, _ = layers[l]
        dpre = dh * (pres[l] > 0)
        grads[l] = (dpre.T @ acts[l], dpre.sum(axis=0))
        dh = dpre @ w
    if return_dx:
        return grads, dh
    return grads


def ddf_loss_grad(o, d, blob, octaves, width, hidden, t_target, hit_target):
    """Loss and flat gradient blob (same layout as the weight blob)."""
    layers = split_blob(blob, ddf_dims(octaves, width, hidden))
    x0 = encode(o, d, octaves)
    z = mlp_forward(x0, layers)
    L, dz = loss_and_dz(z, t_target, hit_target)
    grads = mlp_backward(x0, layers, dz)
    flat = np.concatenate([np.concatenate([g.reshape(-1), gb]) for g, gb in grads])
    return L, flat


def train_grad(o, d, blob, octaves, width, hidden, t_target, hit_target, precision="bf16"):
    """Loss and flat gradient of one distillation batch (Sec. 3.2 / 3.4), with
    the roundings of the bf16 training step emulated (precision="bf16"):
    the encoding, every hidden weight matrix, every hidden activation (the last
    one too, which then feeds the FP32 head) and every back-propagated
    pre-activation gradient are rounded to bf16; sums are float64; the head,
    the loss and dL/dz stay unrounded. precision="exact" rounds nothing and
    equals ddf_loss_grad. Returns (L, flat gradient in the weight-blob layout)."""
    rnd = round_bf16 if precision == "bf16" else (lambda a: np.asarray(a, F64))
    layers = split_blob(blob, ddf_dims(octaves, width, hidden))
    hid, (wo, bo) = layers[:-1], layers[-1]
    x = rnd(encode(o, d, octaves))
    acts = [x]
    for w, b in hid:
        x = rnd(np.maximum(x @ rnd(w).T + b, 0.0))
        acts.append(x)
    z = x @ wo.T + bo
    L, dz = loss_and_dz(z, t_target, hit_target)
    grads = [None] * len(layers)
    grads[-1] = (dz.T @ acts[-1], dz.sum(axis=0))
    dpre = rnd((dz @ wo) * (acts[-1] > 0))
    for l in range(len(hid) - 1, -1, -1):
        grads[l] = (dpre.T @ acts[l], dpre.sum(axis=0))
        if l > 0:
            dpre = rnd((dpre @ rnd(hid[l][0])) * (acts[l] > 0))
    flat = np.concatenate([np.concatenate([g.reshape(-1), gb]) for g, gb in grads])
    return L, flat


def sdf_train_grad(p, blob, octaves, width, hidden, s_target, precision="bf16"):
    """SDF regression for the sphere-tracing baseline (Sec. 4.4 compares the
    DDF with tracing an SDF network): L = mean |s(p) - s*| with s the raw
    1-output network on the Fourier-encoded point. Roundings as in
    train_grad; dL/ds = sign(s - s*) / B (sign(0) = 0). Returns (L, flat
    gradient in the SDF blob layout)."""
    rnd = round_bf16 if precision == "bf16" else (lambda a: np.asarray(a, F64))
    d_in = 3 + 6 * octaves
    dims = [(width, d_in)] + [(width, width)] * (hidden - 1) + [(1, width)]
    layers = split_blob(blob, dims)
    hid, (wo, bo) = layers[:-1], layers[-1]
    x = rnd(encode_points(p, octaves))
    acts = [x]
    for w, b in hid:
        x = rnd(np.maximum(x @ rnd(w).T + b, 0.0))
        acts.append(x)
    s = (x @ wo.T + bo)[:, 0]
    B = s.shape[0]
    diff = s - np.asarray(s_target, F64)
    L = np.sum(np.abs(diff)) / B
    ds = (np.sign(diff) / B)[:, None]
    grads = [None] * len(layers)
    grads[-1] = (ds.T @ acts[-1], ds.sum(axis=0))
    dpre = rnd((ds @ wo) * (acts[-1] > 0))
    for l in range(len(hid) - 1, -1, -1):
        grads[l] = (dpre.T @ acts[l], dpre.sum(axis=0))
        if l > 0:
            dpre = rnd((dpre @ rnd(hid[l][0])) * (acts[l] > 0))
    flat = np.concatenate([np.concatenate([g.reshape(-1), gb]) for g, gb in grads])
    return L, flat


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected, no weight decay.
    step counts from 1. Returns (w, m, v)."""
    w, g, m, v = (np.asarray(a, F64) for a in (w, g, m, v))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------- analytic scene


def cast_spheres(o, d, centers, radii):
    """Nearest positive root of |o + t d - c| = r per ray and sphere, min over
    spheres; inf where none. Tangent rays (zero discriminant) hit."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    best = np.full(o.shape[0], np.inf)
    a = np.sum(d * d, axis=1)
    for c, r in zip(np.asarray(centers, F64), np.asarray(radii, F64)):
        oc = o - c
        b = np.sum(d * oc, axis=1)
        q = np.sum(oc * oc, axis=1) - r * r
        disc = b * b - a * q
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        h = -b - np.where(b >= 0, sq, -sq)          # no cancellation
        with np.errstate(divide="ignore", invalid="ignore"):
            r1 = np.where(h != 0, h / a, 0.0)
            r2 = np.where(h != 0, q / h, 0.0)
        lo = np.minimum(r1, r2)
        hi = np.maximum(r1, r2)
        t = np.where(lo > 0, lo, np.where(hi > 0, hi, np.inf))
        best = np.where(ok, np.minimum(best, t), best)
    return best


def cast_boxes(o, d, lo, hi):
    """Slab test per axis-aligned box: nearest positive crossing of the
    surface, min over boxes; inf where none."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    n = o.shape[0]
    best = np.full(n, np.inf)
    for blo, bhi in zip(np.asarray(lo, F64), np.asarray(hi, F64)):
        tn = np.full(n, -np.inf)
        tf = np.full(n, np.inf)
        miss = np.zeros(n, dtype=bool)
        for i in range(3):
            par = d[:, i] == 0
            miss |= par & ((o[:, i] < blo[i]) | (o[:, i] > bhi[i]))
            with np.errstate(divide="ignore", invalid="ignore"):
                ta = (blo[i] - o[:, i]) / d[:, i]
                tb = (bhi[i] - o[:, i]) / d[:, i]
            tn = np.where(par, tn, np.maximum(tn, np.minimum(ta, tb)))
            tf = np.where(par, tf, np.minimum(tf, np.maximum(ta, tb)))
        hit = (~miss) & (tn <= tf) & (tf > 0)
        t = np.where(tn > 0, tn, tf)
        best = np.where(hit, np.minimum(best, t), best)
    return best


def cast_scene(scene, o, d):
    """Exact first-hit distance against the union of spheres and boxes
    (the exact-cast supervision of Sec. 3.2, with analytic primitives in
    place of a mesh). Returns (t, hit) with t = inf on a miss."""
    t = np.minimum(cast_spheres(o, d, scene.centers, scene.radii),
                   cast_boxes(o, d, scene.box_lo, scene.box_hi))
    return t, np.isfinite(t)


def union_sdf(scene, p):
    """Signed distance to the union: min over spheres |p-c|-r and boxes
    (|q|_+ + min(max_i q_i, 0) with q = |p - centre| - half-extent)."""
    p = np.asarray(p, F64)
    s = np.full(p.shape[0], np.inf)
    for c, r in zip(scene.centers, scene.radii):
        s = np.minimum(s, np.linalg.norm(p - c, axis=1) - r)
    for lo, hi in zip(scene.box_lo, scene.box_hi):
        q = np.abs(p - 0.5 * (lo + hi)) - 0.5 * (hi - lo)
        out = np.linalg.norm(np.maximum(q, 0.0), axis=1)
        s = np.minimum(s, out + np.minimum(np.max(q, axis=1), 0.0))
    return s


def sphere_trace(sdf, o, d, max_steps=128, eps=1e-3, t_max=4.0):
    """Sphere tracing (Sec. 4.4): t = 0; repeat up to max_steps: s = sdf(o +
    t d); stop with a hit when s < eps, else t += s; stop with a miss when
    t > t_max. Returns (t, hit, steps) where steps counts SDF evaluations."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    n = o.shape[0]
    t = np.zeros(n)
    hit = np.zeros(n, dtype=bool)
    steps = np.zeros(n, dtype=np.int64)
    active = np.ones(n, dtype=bool)
    for _ in range(max_steps):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        s = sdf(o[idx] + t[idx, None] * d[idx])
        steps[idx] += 1
        conv = s < eps
        hit[idx[conv]] = True
        go = idx[~conv]
        t[go] += s[~conv]
        active[idx[conv]] = False
        active[go[t[go] > t_max]] = False
    return t, hit, steps


def sdf_mlp(p, blob, octaves, width, hidden, precision="exact"):
    """SDF baseline network: Fourier-encoded point -> ReLU MLP -> 1 output."""
    d_in = 3 + 6 * octaves
    dims = [(width, d_in)] + [(width, width)] * (hidden - 1) + [(1, width)]
    layers = split_blob(blob, dims)
    return mlp_forward(encode_points(p, octaves), layers, precision)[:, 0]


# ------------------------------------------- hash-grid field (Sec. 3.4)
#
# The paper's final field encodes the point x with a multiresolution hash
# grid (16 levels, 2 features per level, 2^19 entries per level, base
# resolution 16, growth 1.5, over a box bounding the object), the direction
# d with four sinusoidal bands, and reads the joined code with a two-layer
# MLP of width 64. Readings where the paper is silent:
#   * level resolution N_l = floor(16 * 1.5^l); a level is a grid of
#     (N_l + 1)^3 vertices over the box [-1, 1]^3 (x clamped into it);
#   * a level stores min(2^19, (N_l + 1)^3) entries: dense levels index a
#     vertex (i, j, k) as i + (N+1) (j + (N+1) k), hashed levels with the
#     spatial hash of the cited multiresolution-hash-encoding work,
#     (i * 1 xor j * 2654435761 xor k * 805459861) mod 2^19;
#   * trilinear interpolation of the 8 corner entries of the cell holding x
#     (cell index clamped to N - 1 at the upper face); `positions="fp32"`
#     takes the cell and in-cell coordinates from float32 arithmetic, as a
#     float32 implementation picks them (at N = 7006 a float32 box
#     coordinate moves u by up to 4e-4 of a cell, and with it every ReLU
#     decision downstream of the features);
#   * code = [level 0 features, ..., level 15 features, d, then per
#     coordinate of d and band k = 0..3: sin(pi 2^k d_c), cos(pi 2^k d_c)]
#     (59 values), MLP 59 -> 64 -> 64 -> 2 with ReLU, heads as Sec. 3.1;
#   * blob = the level tables in order (entry-major, features adjacent),
#     then the MLP as split_blob lays it out.

HG_LEVELS = 16
HG_FEATURES = 2
HG_LOG2_T = 19
HG_BASE = 16
HG_GROWTH = 1.5
HG_DIR_BANDS = 4
HG_PRIMES = (1, 2654435761, 805459861)


def hashgrid_resolutions(levels=HG_LEVELS, base=HG_BASE, growth=HG_GROWTH):
    """N_l = floor(base * growth^l) cells per axis for l = 0..levels-1."""
    return [int(np.floor(base * growth ** l)) for l in range(levels)]


def hashgrid_table_sizes(levels=HG_LEVELS, log2_t=HG_LOG2_T, base=HG_BASE, growth=HG_GROWTH):
    """Entries per level: every vertex while they fit, else 2^log2_t."""
    return [min(2 ** log2_t, (n + 1) ** 3) for n in hashgrid_resolutions(levels, base, growth)]


def hashgrid_index(ijk, res, size, log2_t=HG_LOG2_T):
    """Table row of integer vertices ijk [n, 3] on a level with res cells
    per axis and `size` entries: dense row-major index if every vertex has
    its own entry, else the spatial hash taken modulo 2^log2_t."""
    ijk = np.asarray(ijk, np.int64)
    if (res + 1) ** 3 <= size:
        return ijk[:, 0] + (res + 1) * (ijk[:, 1] + (res + 1) * ijk[:, 2])
    u = ijk.astype(np.uint64)
    h = (u[:, 0] * np.uint64(HG_PRIMES[0])) ^ (u[:, 1] * np.uint64(HG_PRIMES[1])) \
        ^ (u[:, 2] * np.uint64(HG_PRIMES[2]))
    return (h & np.uint64((1 << log2_t) - 1)).astype(np.int64)


def hashgrid_cell(x, res, positions="exact", lo=-1.0, hi=1.0):
    """Cell index i0 [n, 3] and in-cell coordinates w [n, 3] of points x on a
    level with `res` cells per axis (x clamped into the box). positions
    "fp32" takes the box coordinate (x + 1) / 2 and its product with res in
    float32, as a float32 implementation does, so that both pick the same
    cell and weights; "exact" computes in float64."""
    if positions == "fp32":
        f = np.float32
        x01 = np.clip((np.asarray(x, f) + f(1.0)) * f(0.5), f(0.0), f(1.0))
        u = (x01 * f(res)).astype(F64)
    elif positions == "exact":
        x01 = np.clip((np.asarray(x, F64) - lo) / (hi - lo), 0.0, 1.0)
        u = x01 * res
    else:
        raise ValueError(positions)
    i0 = np.minimum(np.floor(u), res - 1).astype(np.int64)
    return i0, u - i0


def hashgrid_encode(x, tables, resolutions, log2_t=HG_LOG2_T, lo=-1.0, hi=1.0,
                    positions="exact"):
    """Multiresolution hash encoding of points x [n, 3]: per level the
    trilinear interpolation of the level table ([T_l, F]) over the 8 corners
    of the cell holding x. Returns [n, levels * F] float64."""
    feats = []
    for table, res in zip(tables, resolutions):
        table = np.asarray(table, F64)
        i0, w = hashgrid_cell(x, res, positions, lo, hi)
        f = np.zeros((i0.shape[0], table.shape[1]))
        for corner in range(8):
            c = np.array([(corner >> a) & 1 for a in range(3)])
            wt = np.prod(np.where(c[None, :] == 1, w, 1.0 - w), axis=1)
            idx = hashgrid_index(i0 + c[None, :], res, table.shape[0], log2_t)
            f += wt[:, None] * table[idx]
        feats.append(f)
    return np.concatenate(feats, axis=1)


def encode_dir(d, bands=HG_DIR_BANDS):
    """Sinusoidal encoding of a direction: d, then per coordinate c and band
    k: sin(pi 2^k d_c), cos(pi 2^k d_c). Returns [n, 3 + 6 bands]."""
    d = np.asarray(d, F64)
    out = [d]
    for c in range(3):
        for k in range(bands):
            arg = np.pi * np.ldexp(d[:, c], k)
            out += [np.sin(arg)[:, None], np.cos(arg)[:, None]]
    return np.concatenate(out, axis=1)


def hashgrid_mlp_dims(width=64, hidden=2, bands=HG_DIR_BANDS):
    d_in = HG_LEVELS * HG_FEATURES + 3 + 6 * bands
    return [(width, d_in)] + [(width, width)] * (hidden - 1) + [(2, width)]


def hashgrid_split(blob, width=64, hidden=2, bands=HG_DIR_BANDS):
    """(level tables [T_l, F], MLP layers) from a hash-grid field blob."""
    blob = np.asarray(blob)
    tables, off = [], 0
    for t in hashgrid_table_sizes():
        tables.append(blob[off:off + t * HG_FEATURES].reshape(t, HG_FEATURES).astype(F64))
        off += t * HG_FEATURES
    return tables, split_blob(blob[off:], hashgrid_mlp_dims(width, hidden, bands))


def hashgrid_encode_backward(x, dfeat, table_sizes, resolutions, log2_t=HG_LOG2_T, lo=-1.0,
                             hi=1.0, positions="exact"):
    """Gradient of sum(dfeat * hashgrid_encode(x)) w.r.t. every level table:
    each of a point's 8 corner entries receives its interpolation weight
    times the point's feature gradient (summed over points sharing an entry).
    dfeat [n, levels * F]. Returns [T_l, F] arrays."""
    dfeat = np.asarray(dfeat, F64)
    out = []
    for l, (size, res) in enumerate(zip(table_sizes, resolutions)):
        g = np.zeros((size, HG_FEATURES))
        i0, w = hashgrid_cell(x, res, positions, lo, hi)
        df = dfeat[:, HG_FEATURES * l:HG_FEATURES * (l + 1)]
        for corner in range(8):
            c = np.array([(corner >> a) & 1 for a in range(3)])
            wt = np.prod(np.where(c[None, :] == 1, w, 1.0 - w), axis=1)
            idx = hashgrid_index(i0 + c[None, :], res, size, log2_t)
            np.add.at(g, idx, wt[:, None] * df)
        out.append(g)
    return out


def hashgrid_field_loss_grad(o, d, tables, resolutions, layers, t_target, hit_target,
                             bands=HG_DIR_BANDS, log2_t=HG_LOG2_T, positions="exact"):
    """Distillation loss (loss_and_dz) of a hash-grid field given as level
    tables, resolutions and MLP layers, and its gradient: the MLP by
    mlp_backward, the tables by hashgrid_encode_backward of the code
    gradient's hash-feature part. Everything in float64. Returns (L, [table
    gradients], [(dW, db)])."""
    code = np.concatenate([hashgrid_encode(o, tables, resolutions, log2_t, positions=positions),
                           encode_dir(d, bands)], axis=1)
    z = mlp_forward(code, layers)
    L, dz = loss_and_dz(z, t_target, hit_target)
    grads, dcode = mlp_backward(code, layers, dz, return_dx=True)
    nf = len(tables) * HG_FEATURES
    dtab = hashgrid_encode_backward(o, dcode[:, :nf], [t.shape[0] for t in tables], resolutions,
                                    log2_t, positions=positions)
    return L, dtab, grads


def hashgrid_loss_grad(o, d, blob, t_target, hit_target, width=64, hidden=2, bands=HG_DIR_BANDS,
                       positions="exact"):
    """hashgrid_field_loss_grad for a blob in the paper's layout; the
    gradient comes back flat in the blob layout (tables, then the MLP)."""
    tables, layers = hashgrid_split(blob, width, hidden, bands)
    L, dtab, grads = hashgrid_field_loss_grad(o, d, tables, hashgrid_resolutions(), layers,
                                              t_target, hit_target, bands, positions=positions)
    flat = [t.ravel() for t in dtab] + [np.concatenate([g.ravel(), gb]) for g, gb in grads]
    return L, np.concatenate(flat)


def hashgrid_forward(o, d, blob, width=64, hidden=2, bands=HG_DIR_BANDS, precision="exact",
                     positions="exact"):
    """Query of the hash-grid DDF: f(x, d) = (t, xi) from the joined code
    [hash features of x, encoded d]. precision "bf16" rounds the table
    entries to bfloat16 (interpolation stays float64) and runs the MLP as
    mlp_forward's bf16 mode. Returns dict(t, vis, z)."""
    tables, layers = hashgrid_split(blob, width, hidden, bands)
    if precision == "bf16":
        tables = [round_bf16(t) for t in tables]
    elif precision != "exact":
        raise ValueError(precision)
    code = np.concatenate([hashgrid_encode(o, tables, hashgrid_resolutions(), positions=positions),
                           encode_dir(d, bands)], axis=1)
    z = mlp_forward(code, layers, precision)
    return {"t": softplus(z[:, 0]), "vis": sigmoid(z[:, 1]), "z": z}


# ------------------------------------- shadow / AO images (Sec. 3.3, app.)
#
# The paper's application: per pixel of a camera image, a primary hit, then a
# shadow ray toward a point light and hemisphere rays for ambient occlusion,
# answered by the field. Readings (the paper gives no camera or sampler):
#   * pinhole camera: forward f = (target - eye)/|.|, right r = f x up /|.|,
#     u = r x f; pixel (x, y) (row 0 at the top) looks along
#     f + sx r + sy u, sx = (2 (x + 0.5)/W - 1) tan(fov/2) W/H,
#     sy = (1 - 2 (y + 0.5)/H) tan(fov/2);
#   * primary hits exact (caster); shading normal = the outward normal of the
#     primitive whose surface holds the hit point, flipped to face the eye;
#     secondary origins 1e-3 off the surface along it;
#   * shadow: occluded when the ray toward the light hits closer than the
#     light; AO: 1 - mean hit flag over k cosine-weighted directions (Malley:
#     r = sqrt(u1), phi = 2 pi u2, z = sqrt(1 - u1)) in the orthonormal basis
#     of Duff et al. (2017) around the normal;
#   * uniforms: SplitMix64 (Steele, Lea, Flood), u = (mix(key + m) >> 40) 2^-24
#     with key = mix(mix(seed xor 0x5DEECE66D) + pixel) xor (sample x
#     0x2545F4914F6CDD1D), m = 0, 1 for (u1, u2);
#   * background pixels read -1 in both images.

_U64 = np.uint64


def splitmix64(x):
    """SplitMix64 output for state x (the state is advanced by the golden
    gamma first): uint64 in, uint64 out (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, _U64) + _U64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


def gi_uniform(seed, pixel, sample, m):
    """The m-th uniform of (pixel, sample): 24-bit, exact in float32."""
    with np.errstate(over="ignore"):
        key = splitmix64(splitmix64(_U64(seed) ^ _U64(0x5DEECE66D)) + np.asarray(pixel, _U64)) \
            ^ (np.asarray(sample, _U64) * _U64(0x2545F4914F6CDD1D))
        return (splitmix64(key + _U64(m)) >> _U64(40)).astype(F64) * 2.0 ** -24


def camera_rays(eye, target, up, fov_y, width, height):
    """Pixel-centre rays of a pinhole camera, pixel index y * width + x."""
    eye = np.asarray(eye, F64)
    f = np.asarray(target, F64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, F64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = np.tan(0.5 * fov_y)
    y, x = np.mgrid[0:height, 0:width]
    sx = (2 * (x.ravel() + 0.5) / width - 1) * th * width / height
    sy = (1 - 2 * (y.ravel() + 0.5) / height) * th
    d = f[None, :] + sx[:, None] * r[None, :] + sy[:, None] * u[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.repeat(eye[None, :], width * height, axis=0), d


def surface_normal(scene, p):
    """Outward normal at points p on the scene's surfaces: of the primitive
    whose surface lies nearest p (sphere: radial; box: the nearest face)."""
    p = np.asarray(p, F64)
    cand_d, cand_n = [], []
    for c, r in zip(scene.centers, scene.radii):
        v = p - c
        dist = np.linalg.norm(v, axis=1)
        cand_d.append(np.abs(dist - r))
        cand_n.append(v / np.maximum(dist, 1e-300)[:, None])
    for lo, hi in zip(scene.box_lo, scene.box_hi):
        gaps = np.stack([np.abs(p - lo), np.abs(p - hi)], axis=2)       # [n, 3 axes, 2 sides]
        inside = np.all((p >= lo - 1e-9) & (p <= hi + 1e-9), axis=1)
        flat = gaps.reshape(p.shape[0], 6)
        k = np.argmin(flat, axis=1)
        face_gap = flat[np.arange(p.shape[0]), k]
        # distance to the box surface (off-face points are farther than the gap)
        out = np.linalg.norm(np.maximum(np.maximum(lo - p, p - hi), 0.0), axis=1)
        cand_d.append(np.where(inside, face_gap, np.maximum(out, face_gap)))
        n = np.zeros_like(p)
        n[np.arange(p.shape[0]), k // 2] = np.where(k % 2 == 1, 1.0, -1.0)
        cand_n.append(n)
    j = np.argmin(np.stack(cand_d, 1), axis=1)
    return np.stack(cand_n, 1)[np.arange(p.shape[0]), j]


def onb(n):
    """Orthonormal tangents (t1, t2) with t1 x t2 = n (Duff et al. 2017)."""
    n = np.asarray(n, F64)
    sgn = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sgn + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t1 = np.stack([1 + sgn * n[:, 0] ** 2 * a, sgn * b, -sgn * n[:, 0]], 1)
    t2 = np.stack([b, sgn + n[:, 1] ** 2 * a, -n[:, 1]], 1)
    return t1, t2


def cosine_dirs(n, u1, u2):
    """Malley's method: cosine-weighted directions about unit normals n."""
    r = np.sqrt(u1)
    phi = 2 * np.pi * u2
    z = np.sqrt(np.maximum(0.0, 1 - u1))
    t1, t2 = onb(n)
    return (r * np.cos(phi))[:, None] * t1 + (r * np.sin(phi))[:, None] * t2 + z[:, None] * n


def gi_images(scene, eye, target, up, fov_y, width, height, light, ao_samples, seed,
              field_blob=None, field_precision="exact", detail=False):
    """Shadow (1 lit, 0 shadowed) and ambient-occlusion images of the scene;
    background -1. The secondary rays are answered by exact casts, or, with
    field_blob (a hash-grid field's blob), by that field (hashgrid_forward
    in field_precision): a ray counts as a hit when z1 > 0, and a shadow ray
    occludes when it hits closer than the light. Returns (shadow, ao)
    [height, width], and with detail also, per foreground pixel (in pixel
    order), the shadow rays' t, z1 (exact casts: +-1) and light distance and
    the hemisphere rays' z1 [pixels, ao_samples]."""
    o, d = camera_rays(eye, target, up, fov_y, width, height)
    t, hit = cast_scene(scene, o, d)
    npx = width * height
    shadow = -np.ones(npx)
    ao = -np.ones(npx)
    idx = np.nonzero(hit)[0]
    p = o[idx] + t[idx, None] * d[idx]
    nrm = surface_normal(scene, p)
    nrm = np.where(np.sum(nrm * d[idx], axis=1, keepdims=True) > 0, -nrm, nrm)
    sp = p + 1e-3 * nrm

    def answer(org, dirs):
        """(t, z1) of secondary rays: exact casts or the field."""
        if field_blob is None:
            ts, hs = cast_scene(scene, org, dirs)
            return ts, np.where(hs, 1.0, -1.0)
        f = hashgrid_forward(org, dirs, field_blob, precision=field_precision)
        return f["t"], f["z"][:, 1]

    to_l = np.asarray(light, F64)[None, :] - sp
    dist = np.linalg.norm(to_l, axis=1)
    ts, zs = answer(sp, to_l / dist[:, None])
    shadow[idx] = np.where((zs > 0) & (ts < dist), 0.0, 1.0)
    hits = np.zeros(idx.size)
    z_ao = np.zeros((idx.size, ao_samples))
    for j in range(ao_samples):
        u1 = gi_uniform(seed, idx, j, 0)
        u2 = gi_uniform(seed, idx, j, 1)
        _, za = answer(sp, cosine_dirs(nrm, u1, u2))
        z_ao[:, j] = za
        hits += za > 0
    ao[idx] = 1.0 - hits / ao_samples
    images = (shadow.reshape(height, width), ao.reshape(height, width))
    if detail:
        return images + ({"pixels": idx, "shadow_t": ts, "shadow_z1": zs, "shadow_dist": dist,
                          "ao_z1": z_ao},)
    return images


# --------------------------- distillation schedule (Sec. 3.2 / Sec. 3.4)
#
# Sec. 3.2 trains on camera rays and on rays that start on the surface and
# point in all directions, adds copies of hitting rays moved forward along
# themselves (a point moved forward by s reports t - s), and Sec. 3.4 decays
# the learning rate by a cosine to 5 % of its start. The paper fixes neither
# the ray distributions nor the draws; the readings taken here:
#   * a fraction surface_frac of the rays is surface-anchored: a point
#     uniform by area over the primitives' surfaces (a surface element, a
#     sphere or one face of a box, chosen with probability proportional to
#     its area, then a point uniform on it: sphere c + r n with n uniform on
#     the sphere; box face: the two in-face coordinates uniform), the origin
#     1e-3 off the surface along the outward normal, the direction uniform on
#     the sphere; points of one primitive that lie inside another are kept;
#     the rest are camera rays: origin uniform on a face of [-1, 1]^3, aimed
#     at a point uniform in [-0.9, 0.9]^3;
#   * the element's area weight is an integer, floor(A 2^24) with A the
#     float32 product (4 pi r) r or (hi_u - lo_u)(hi_v - lo_v) clamped to
#     [0, 2^16]; the weights' prefix sums are exact integers, each rounded
#     once to float32, and the element is the first whose rounded prefix sum
#     exceeds the float32 product u W (W the rounded total), so that any
#     summation order gives the same choice;
#   * the rays from index `first` on that hit move to o + s d with s = u t,
#     u uniform in [0, 1), and report t - s; misses stay as they are;
#   * lr_k = lr0 (0.05 + 0.95 (1 + cos(pi k / steps)) / 2), k = 0..steps-1;
#   * draws: uniform m of ray i at step k is the counter-based SplitMix64
#     uniform of (seed, a = k, b = i) (the key of gi_uniform), with m = 0 the
#     surface/camera choice, 1 the surface element or camera face, 2..6 the positions and
#     directions (in the order below), 7 the shift, and for batches drawn from
#     a fixed pool the top 32 bits of mix(key + 8) pick the row;
#   * where a uniform picks one of K camera faces, the product u K is taken
#     in float32, as the GPU takes it, and floored.

DISTILL_SURFACE_OFFSET = 1e-3
DISTILL_AREA_SCALE = 2.0 ** 24   # area weights are floor(A 2^24)
DISTILL_AREA_MAX = 2.0 ** 16     # element areas are clamped to [0, 2^16]


def distill_uniform(seed, step, i, m):
    """Uniform m of ray i at distillation step `step` (24 bits, exact in
    float32)."""
    return gi_uniform(seed, step, i, m)


def _pick(u, k):
    """floor(u k) with the product rounded to float32, clamped to k - 1."""
    prod = (np.asarray(u, np.float32) * np.float32(k)).astype(F64)
    return np.minimum(np.floor(prod), k - 1).astype(np.int64)


def distill_surface_weights(scene):
    """Integer area weight of every surface element: the spheres in order,
    then the six faces of each box (face f: axis f // 2, the upper side if f
    is odd). The area is the float32 product (4 pi r) r for a sphere and
    (hi_u - lo_u)(hi_v - lo_v) over the face's two in-face axes u, v,
    clamped to [0, 2^16] (a NaN to 0); the weight is floor(A 2^24)."""
    r = np.asarray(scene.radii, np.float32).reshape(-1)
    a_s = (np.float32(4.0 * np.pi) * r) * r
    lo = np.asarray(scene.box_lo, np.float32).reshape(-1, 3)
    hi = np.asarray(scene.box_hi, np.float32).reshape(-1, 3)
    e = hi - lo
    a_f = np.zeros((lo.shape[0], 6), np.float32)
    for axis in range(3):
        u, v = (axis + 1) % 3, (axis + 2) % 3
        a_f[:, 2 * axis] = a_f[:, 2 * axis + 1] = e[:, u] * e[:, v]
    a = np.concatenate([a_s, a_f.reshape(-1)]).astype(np.float32)
    a = np.fmin(np.fmax(a, np.float32(0.0)), np.float32(DISTILL_AREA_MAX))
    return np.floor(a * np.float32(DISTILL_AREA_SCALE)).astype(np.int64)


def distill_pick_surface(scene, u):
    """The surface element each uniform u picks (readings above): the first
    element whose exact prefix sum of weights, rounded to float32, exceeds
    the float32 product u W, W the rounded total; clamped to the last
    element. Returns (element index array, W > 0)."""
    w = distill_surface_weights(scene)
    cum = np.cumsum(w)                         # exact: every sum below 2^53
    if cum.size == 0 or cum[-1] == 0:
        return np.zeros(np.shape(u), np.int64), False
    cum32 = cum.astype(F64).astype(np.float32)  # exact in float64, one rounding
    total = cum32[-1]
    x = np.asarray(u, np.float32) * total
    j = np.searchsorted(cum32, x, side="right")
    return np.minimum(j, cum.size - 1).astype(np.int64), True


def uniform_sphere_dir(a, b):
    """Unit vector uniform on the sphere from two uniforms (Archimedes:
    z = 2a - 1 uniform, azimuth 2 pi b)."""
    z = 2.0 * np.asarray(a, F64) - 1.0
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = 2.0 * np.pi * np.asarray(b, F64)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=-1)


def distill_rays(scene, seed, step, n, surface_frac):
    """The n training rays of one distillation step (readings above).
    Returns (o, d) [n, 3] float64 and the surface-anchored mask."""
    i = np.arange(n, dtype=np.int64)
    u = [distill_uniform(seed, step, i, m) for m in range(7)]
    ns = len(scene.radii)
    p, any_area = distill_pick_surface(scene, u[1])
    surf = (u[0] < np.float32(surface_frac)) & any_area
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    # surface-anchored rays
    if any_area:
        pt = np.zeros((n, 3))
        nrm = np.zeros((n, 3))
        sph = surf & (p < ns)
        if np.any(sph):
            js = p[sph]
            nv = uniform_sphere_dir(u[2][sph], u[3][sph])
            pt[sph] = np.asarray(scene.centers, F64)[js] + np.asarray(scene.radii, F64)[js, None] * nv
            nrm[sph] = nv
        r = np.nonzero(surf & (p >= ns))[0]           # box faces
        lo = np.asarray(scene.box_lo, F64)[(p[r] - ns) // 6]
        hi = np.asarray(scene.box_hi, F64)[(p[r] - ns) // 6]
        face = (p[r] - ns) % 6
        axis, plus = face // 2, face % 2 == 1
        a, c = (axis + 1) % 3, (axis + 2) % 3
        k = np.arange(r.size)
        pt[r, a] = lo[k, a] + u[3][r] * (hi[k, a] - lo[k, a])
        pt[r, c] = lo[k, c] + u[4][r] * (hi[k, c] - lo[k, c])
        pt[r, axis] = np.where(plus, hi[k, axis], lo[k, axis])
        nrm[r, axis] = np.where(plus, 1.0, -1.0)
        o[surf] = pt[surf] + DISTILL_SURFACE_OFFSET * nrm[surf]
        d[surf] = uniform_sphere_dir(u[5][surf], u[6][surf])
    # camera rays
    r = np.nonzero(~surf)[0]
    face = _pick(u[1][r], 6)
    axis, plus = face // 2, face % 2 == 1
    o[r, (axis + 1) % 3] = 2.0 * u[2][r] - 1.0
    o[r, (axis + 2) % 3] = 2.0 * u[3][r] - 1.0
    o[r, axis] = np.where(plus, 1.0, -1.0)
    cam = ~surf
    tgt = np.stack([1.8 * u[4] - 0.9, 1.8 * u[5] - 0.9, 1.8 * u[6] - 0.9], axis=1)
    v = tgt[cam] - o[cam]
    d[cam] = v / np.linalg.norm(v, axis=1, keepdims=True)
    return o, d, surf


def distill_shift(o, d, t, hit, first, seed, step):
    """Ray-march shifted points: rays i >= first that hit move to o + s d with
    s = u t (u = draw 7 of (seed, step, i)) and report t - s. Returns new
    (o, t); misses and rays before `first` are unchanged."""
    o = np.array(o, F64)
    t = np.array(t, F64)
    d = np.asarray(d, F64)
    i = np.arange(first, o.shape[0], dtype=np.int64)
    sel = i[np.asarray(hit, bool)[first:] & np.isfinite(t[first:])]
    s = distill_uniform(seed, step, sel, 7) * t[sel]
    o[sel] += s[:, None] * d[sel]
    t[sel] -= s
    return o, t


def distill_lr(lr0, k, steps):
    """Learning rate of step k of `steps`: a cosine from lr0 down to 5 % of it."""
    return lr0 * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * np.asarray(k, F64) / steps)))


def distill_pool_index(seed, step, i, n_pool):
    """Pool row of batch row i at `step`: floor(u32 n_pool / 2^32) with u32
    the top 32 bits of mix(key + 8) (integer arithmetic)."""
    with np.errstate(over="ignore"):
        key = splitmix64(splitmix64(_U64(seed) ^ _U64(0x5DEECE66D)) + _U64(step)) \
            ^ (np.asarray(i, _U64) * _U64(0x2545F4914F6CDD1D))
        u32 = splitmix64(key + _U64(8)) >> _U64(32)
    return np.array([(int(x) * int(n_pool)) >> 32 for x in np.atleast_1d(u32)], np.int64)


# ----------------------- Gaussian-rendered depth (Sec. 3.2, Sec. 4.2)
#
# The supervision source the paper finds too blurry for thin parts: depth
# rendered from the scene's 3D Gaussians. Definitions (the standard 3DGS
# depth composite, restated; the paper cites it and gives no formula):
#   * camera as camera_rays; view coordinates (x, y, z) of a point along
#     (r, u, f); pixel coordinates px = (x/z) fx + (W - 1)/2,
#     py = -(y/z) fy + (H - 1)/2 with fx = W / (2 tan(fov/2) W/H),
#     fy = H / (2 tan(fov/2)), so pixel (i, j) is looked at by camera ray
#     j W + i;
#   * screen covariance S = J V C V^T J^T + 0.3 I (EWA splatting, 3DGS's
#     low-pass), V = rows (r, u, f), J the Jacobian of (px, py) at the mean;
#   * alpha_i = min(0.99, o_i exp(-q/2)), q = dp^T S^-1 dp; contributions with
#     alpha < 1/255 are skipped; Gaussians with z <= 0.05 are culled;
#   * front to back by mean depth z (ties by index): T starts at 1; each
#     contribution adds T alpha t_i to D and T alpha to A, then T *= 1 - alpha;
#     stop once T < 1e-4; t_i = z_i / (d . f) is the mean's depth as a
#     distance along the pixel ray d;
#   * output: t = D / A where A > 0 (inf otherwise), hit = A > 0.5.

GS_LOWPASS = 0.3
GS_ALPHA_MIN = 1.0 / 255.0
GS_ALPHA_MAX = 0.99
GS_T_MIN = 1e-4
GS_NEAR = 0.05


def gs_project(means, covs, eye, target, up, fov_y, width, height):
    """Per Gaussian: pixel mean [n, 2], screen covariance [n, 2, 2], view
    depth z [n]."""
    eye = np.asarray(eye, F64)
    f = np.asarray(target, F64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, F64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    V = np.stack([r, u, f])
    th = np.tan(0.5 * fov_y)
    fx = width / (2 * th * width / height)
    fy = height / (2 * th)
    v = (np.asarray(means, F64) - eye) @ V.T
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    px = x / z * fx + (width - 1) / 2
    py = -y / z * fy + (height - 1) / 2
    J = np.zeros((v.shape[0], 2, 3))
    J[:, 0, 0] = fx / z
    J[:, 0, 2] = -fx * x / z ** 2
    J[:, 1, 1] = -fy / z
    J[:, 1, 2] = fy * y / z ** 2
    cv = np.einsum("ij,njk,lk->nil", V, np.asarray(covs, F64), V)
    S = np.einsum("nij,njk,nlk->nil", J, cv, J) + GS_LOWPASS * np.eye(2)[None]
    return np.stack([px, py], 1), S, z


def gs_depth(means, covs, opacities, eye, target, up, fov_y, width, height, pixels=None):
    """Expected distance and hit flag per pixel ([height, width] each) of a
    Gaussian scene, by the composite above, every Gaussian against every
    pixel (plain definition; small images only). covs: [n, 3, 3]. With
    `pixels` (flat indices y * width + x) only those pixels, as flat arrays."""
    mu2, S, z = gs_project(means, covs, eye, target, up, fov_y, width, height)
    _, d = camera_rays(eye, target, up, fov_y, width, height)
    f = np.asarray(target, F64) - np.asarray(eye, F64)
    f /= np.linalg.norm(f)
    yy, xx = np.mgrid[0:height, 0:width]
    pix = np.stack([xx.ravel(), yy.ravel()], 1).astype(F64)
    if pixels is not None:
        pix, d = pix[pixels], d[pixels]
    cosf = d @ f
    keep = z > GS_NEAR
    order = np.lexsort((np.arange(z.size), z))
    order = order[keep[order]]
    Sinv = np.linalg.inv(S[order])
    op = np.asarray(opacities, F64)[order]
    zz = z[order]
    npx = pix.shape[0]
    T = np.ones(npx)
    D = np.zeros(npx)
    A = np.zeros(npx)
    done = np.zeros(npx, dtype=bool)
    for g in range(order.size):
        dp = pix - mu2[order[g]]
        q = np.einsum("ni,ij,nj->n", dp, Sinv[g], dp)
        alpha = np.minimum(GS_ALPHA_MAX, op[g] * np.exp(-0.5 * q))
        use = (alpha >= GS_ALPHA_MIN) & ~done
        w = np.where(use, T * alpha, 0.0)
        D += w * (zz[g] / cosf)
        A += w
        T = np.where(use, T * (1 - alpha), T)
        done |= T < GS_T_MIN
    t = np.where(A > 0, D / np.where(A > 0, A, 1.0), np.inf)
    if pixels is not None:
        return t, A > 0.5
    return t.reshape(height, width), (A > 0.5).reshape(height, width)


def enter_box(o, d, half=1.0):
    """Entry of rays into the box [-half, half]^3 (the field's domain,
    Sec. 3.4; slab test): returns (o + e d, e) with e the distance to the
    entry point, 0 for an origin inside the box or a ray that misses it."""
    o = np.asarray(o, F64)
    d = np.asarray(d, F64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = (-half - o) / d
        b = (half - o) / d
    lo_t = np.where(d != 0, np.minimum(a, b), np.where(np.abs(o) <= half, -np.inf, np.inf))
    hi_t = np.where(d != 0, np.maximum(a, b), np.where(np.abs(o) <= half, np.inf, -np.inf))
    tn = np.maximum(lo_t.max(axis=1), 0.0)
    tf = hi_t.min(axis=1)
    e = np.where(tn <= tf, tn, 0.0)
    return o + e[:, None] * d, e


def gs_cov_matrices(covs6):
    """[n, 3, 3] covariances from rows (xx, xy, xz, yy, yz, zz)."""
    c = np.asarray(covs6, F64)
    return np.stack([c[:, [0, 1, 2]], c[:, [1, 3, 4]], c[:, [2, 4, 5]]], axis=1)


# ----------------------------------------------------------- queries


def shadow(t, z1, o, light):
    """Sec. 3.3: occluded iff the field reports a hit (z1 > 0) closer than
    the light."""
    dist = np.linalg.norm(np.asarray(light, F64)[None, :] - np.asarray(o, F64), axis=1)
    return (np.asarray(z1) > 0) & (np.asarray(t, F64) < dist)


def ambient_occlusion(hit, vis, offsets):
    """Sec. 3.3: per shading point, 1 - mean hit flag over its rays (hard),
    and 1 - mean visibility (soft). Empty sets give 1."""
    offsets = np.asarray(offsets, np.int64)
    n = offsets.size - 1
    hard = np.ones(n)
    soft = np.ones(n)
    for p in range(n):
        a, b = offsets[p], offsets[p + 1]
        if b > a:
            hard[p] = 1.0 - np.mean(np.asarray(hit[a:b], F64))
            soft[p] = 1.0 - np.mean(np.asarray(vis[a:b], F64))
    return hard, soft
