"""Writes trained_small_field.json: a 78 -> 128x4 -> 2 sinusoidal DDF (Sec. 4.3,
Table 2) distilled by the FP64 oracle alone, so that flip rates can be measured
on trained weights without any input from the GPU path.

Recipe (all oracle functions): the 32-sphere + 32-box scene (seed 0); each step
draws 4,096 training rays with the oracle's distillation sampler (half camera,
half surface-anchored rays, Sec. 3.2), takes exact targets from the oracle's
closed-form caster, moves the last 30 % by the ray-march shift, and takes one
exact-gradient Adam step (Sec. 3.2 / 3.4 loss; Adam 1e-3 with the cosine
decay to 5 %). The weights stay float64 during training and are rounded to
float32 once at the end. The file also holds the exact outputs of the
field on seeded uniform rays and its e4m3 scales (the "evaluation" block),
so that the benchmark can report flip rates on trained weights without
running the oracle.

    python tests/golden/make_trained_field.py [--steps N] [--eval-only]
"""
import argparse
import base64
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ddf_oracle as O  # noqa: E402
from paper_2606_00817_gb300 import inputs as I  # noqa: E402

NET = (6, 128, 4)
BATCH = 4096
LR0 = 1e-3
SEED = 5
SHIFT = 0.3
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "trained_small_field.json")


def held_out(scene, n=8192):
    """Held-out rays of the training distribution (another seed) and their
    exact targets."""
    o, d, _ = O.distill_rays(scene, 999, 0, n, 0.5)
    o, d = o.astype(np.float32).astype(np.float64), d.astype(np.float32).astype(np.float64)
    t, hit = O.cast_scene(scene, o, d)
    return o, d, t, hit


def train(steps):
    scene = I.random_scene(32, 32, seed=0)
    w = I.xavier_blob(I.NetShape(*NET)).astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    first = BATCH - int(round(SHIFT * BATCH))
    losses = []
    for k in range(steps):
        o, d, _ = O.distill_rays(scene, SEED, k, BATCH, 0.5)
        o, d = o.astype(np.float32).astype(np.float64), d.astype(np.float32).astype(np.float64)
        t, hit = O.cast_scene(scene, o, d)
        o, t = O.distill_shift(o, d, t, hit, first, SEED, k)
        L, g = O.ddf_loss_grad(o, d, w, *NET, t, hit)
        w, m, v = O.adam_step(w, g, m, v, k + 1, O.distill_lr(LR0, k, steps))
        losses.append(L)
    blob = w.astype(np.float32)
    o, d, t, hit = held_out(scene)
    out = O.ddf_forward(o, d, blob, *NET)
    z1 = out["z"][:, 1]
    stats = {"loss_first_10": float(np.mean(losses[:10])), "loss_last_10": float(np.mean(losses[-10:])),
             "held_out_rays": int(o.shape[0]), "held_out_hit_fraction": float(hit.mean()),
             "held_out_hit_accuracy": float(np.mean((z1 > 0) == hit)),
             "held_out_median_abs_dt_on_hits": float(np.median(np.abs(
                 np.minimum(out["t"], 4) - np.minimum(t, 4))[hit])),
             "held_out_frac_abs_z1_below_0.1": float(np.mean(np.abs(z1) < 0.1))}
    return blob, stats


EVAL_RAYS = 16384
EVAL_SEED = 77


def evaluation(blob):
    """Exact outputs of the field on EVAL_RAYS seeded uniform rays (origins
    in [-1, 1]^3, directions uniform on the sphere; the generator of the
    package's inputs module) and the e4m3 activation scales calibrated on
    4,096 of them, for a benchmark that must not run the oracle itself."""
    rays = I.uniform_rays(EVAL_RAYS, seed=EVAL_SEED)
    out = O.ddf_forward(rays.origins(), rays.dirs(), blob, *NET)
    cal = I.uniform_rays(4096, seed=EVAL_SEED + 1)
    scales = O.calibrate_act_scales(cal.origins(), cal.dirs(), blob, *NET)
    enc = lambda a: base64.b64encode(np.asarray(a, "<f4").tobytes()).decode()
    return {"rays": f"inputs.uniform_rays({EVAL_RAYS}, seed={EVAL_SEED})",
            "t_exact_f32_le_base64": enc(out["t"]), "z1_exact_f32_le_base64": enc(out["z"][:, 1]),
            "fp8_act_scales": [float(x) for x in scales],
            "fp8_scales_from": f"calibrate_act_scales on inputs.uniform_rays(4096, seed={EVAL_SEED + 1})",
            "scheme": scheme_accuracy(rays, blob, out, scales)}


def scheme_accuracy(rays, blob, exact, scales):
    """What the reduced-precision schemes themselves give on these rays: the
    oracle's float64 emulation of the bf16 and e4m3 roundings (the e4m3 one
    with the stored scales) against the exact outputs."""
    res = {}
    for prec, sc in (("bf16", None), ("fp8", scales)):
        emu = O.ddf_forward(rays.origins(), rays.dirs(), blob, *NET, precision=prec, act_scales=sc)
        dt = np.abs(emu["t"] - exact["t"])
        res[prec] = {"mean_abs_dt": float(dt.mean()), "max_abs_dt": float(dt.max()),
                     "flip_rate": float(np.mean((emu["z"][:, 1] > 0) != (exact["z"][:, 1] > 0)))}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--eval-only", action="store_true",
                    help="keep the stored weights and only (re)write the evaluation block")
    a = ap.parse_args()
    if a.eval_only:
        with open(OUT) as f:
            doc = json.load(f)
        blob = np.frombuffer(base64.b64decode(doc["blob_f32_le_base64"]), dtype="<f4").astype(np.float32)
        doc["evaluation"] = evaluation(blob)
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)
        return
    blob, stats = train(a.steps)
    doc = {
        "source": "Written by tests/golden/make_trained_field.py, which calls only the FP64 oracle "
                  "(oracle/ddf_oracle.py) and the seeded generators: a 78 -> 128x4 -> 2 sinusoidal "
                  "DDF (Sec. 4.3, Table 2; L = 6) distilled on the 32-sphere + 32-box scene with the "
                  "oracle's sampler, caster, shift, exact loss gradient (Sec. 3.2 / 3.4) and Adam "
                  "(1e-3, cosine to 5 %), batch 4,096. Weights: float32, little-endian, base64, in the "
                  "blob layout of include/ddf.h.",
        "octaves": NET[0], "width": NET[1], "hidden": NET[2], "steps": a.steps, "batch": BATCH,
        "lr0": LR0, "seed": SEED, "scene": "random_scene(32, 32, seed=0)",
        "stats": stats,
        "evaluation": evaluation(blob),
        "blob_f32_le_base64": base64.b64encode(blob.astype("<f4").tobytes()).decode(),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
