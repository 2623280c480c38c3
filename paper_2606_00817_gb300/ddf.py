"""ctypes binding of libddf.so, the C ABI in include/ddf.h.

Functions named ``ddf_*`` mirror the C entry points one to one and only
marshal arguments (torch tensors or integer addresses become pointers, numpy
arrays become host pointers). ``DDF`` is a small convenience wrapper that
allocates outputs as torch tensors. Every step of the query runs in the CUDA
library; if the library is missing this module raises instead of computing
anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddf.so")

DDF_FP32, DDF_BF16, DDF_FP8_E4M3 = 0, 1, 2
PRECISIONS = {"fp32": DDF_FP32, "bf16": DDF_BF16, "fp8": DDF_FP8_E4M3}
STATUS = {0: "DDF_OK", 1: "DDF_ERR_INVALID_ARG", 2: "DDF_ERR_CUDA", 3: "DDF_ERR_OOM",
          4: "DDF_ERR_BAD_WEIGHTS", 5: "DDF_ERR_UNSUPPORTED", 6: "DDF_ERR_TIMEOUT"}
PROFILE_CLASSES = ("encode", "gemm", "head", "gemm_first")

# every entry point of include/ddf.h: name -> (restype, argtypes)
_vp, _i32, _i64, _u64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t
_RAYS = C.POINTER(C.c_void_p)


class Tile(C.Structure):
    _fields_ = [("bn", C.c_int32), ("epi_warps", C.c_int32), ("cta_pair", C.c_int32),
                ("staged", C.c_int32), ("fused_encode", C.c_int32)]


DDF_KIND_RAY, DDF_KIND_SDF, DDF_KIND_HASHGRID = 0, 1, 2
KINDS = {"ray": DDF_KIND_RAY, "sdf": DDF_KIND_SDF, "hashgrid": DDF_KIND_HASHGRID}
# hash-grid field (Sec. 3.4): 4 direction bands, width 64; its MLP reads a
# 59-value code (16 levels x 2 features + 27 direction values)
HASHGRID_CODE = 59


class Config(C.Structure):
    _fields_ = [("octaves", C.c_int32), ("width", C.c_int32), ("hidden_layers", C.c_int32),
                ("precision", C.c_int32), ("device", C.c_int32), ("kind", C.c_int32)]


SIGNATURES = {
    "ddf_param_count": (_sz, [C.POINTER(Config)]),
    "ddf_create": (C.c_int, [C.POINTER(Config), C.POINTER(_vp)]),
    "ddf_destroy": (C.c_int, [_vp]),
    "ddf_last_error": (C.c_char_p, []),
    "ddf_load_weights": (C.c_int, [_vp, _vp, _sz]),
    "ddf_get_weights": (C.c_int, [_vp, _vp, _sz]),
    "ddf_set_act_scales": (C.c_int, [_vp, _vp, _i32]),
    "ddf_query_rays": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp]),
    "ddf_query_shadow": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp, _vp, _vp]),
    "ddf_query_rays_host": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp]),
    "ddf_query_shadow_host": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp, _vp]),
    "ddf_query_rays_noalloc": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp]),
    "ddf_query_ao": (C.c_int, [_vp, _RAYS, _i64, _vp, _i64, _vp, _vp, _vp]),
    "ddf_query_mixed": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp, _vp, _RAYS, _i64, _vp, _i64,
                                  _vp, _vp, _vp]),
    "ddf_set_graph_mode": (C.c_int, [_vp, _i32]),
    "ddf_calibrate_fp8": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp, _vp]),
    "ddf_compute_grad": (C.c_int, [_vp, _RAYS, _vp, _vp, _i64, _vp, _vp]),
    "ddf_train_step": (C.c_int, [_vp, _RAYS, _vp, _vp, _i64, C.c_float, _vp, _vp]),
    "ddf_forward_train": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp]),
    "ddf_backward": (C.c_int, [_vp, _vp, _i64, _vp]),
    "ddf_copy_grad": (C.c_int, [_vp, _vp, _sz, _vp]),
    "ddf_load_weights_device": (C.c_int, [_vp, _vp, _sz, _vp]),
    "ddf_sample_rays": (C.c_int, [_vp, _i32, _vp, _i32, _u64, _u64, _i64, C.c_float, _RAYS, _vp]),
    "ddf_shift_rays": (C.c_int, [_RAYS, _vp, _vp, _i64, _i64, _u64, _u64, _vp]),
    "ddf_distill": (C.c_int, [_vp, _vp, _i32, _vp, _i32, _i64, _i64, C.c_float, C.c_float,
                              C.c_float, _u64, _vp, _vp]),
    "ddf_render_gi": (C.c_int, [_vp, _vp, _i32, _vp, _i32, _vp, _i32, _i32, _vp, _i32, _u64, _vp,
                                _vp, _vp]),
    "ddf_render_gs_depth": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "ddf_camera_rays": (C.c_int, [_vp, _i32, _i32, _i32, _RAYS, _vp]),
    "ddf_enter_box": (C.c_int, [_RAYS, _vp, _vp, _i64, C.c_float, _vp]),
    "ddf_distill_pool": (C.c_int, [_vp, _RAYS, _vp, _vp, _i64, _i64, _i64, C.c_float, C.c_float,
                                   _u64, _vp, _vp]),
    "ddf_get_grad": (C.c_int, [_vp, _vp, _sz]),
    "ddf_reset_optimizer": (C.c_int, [_vp]),
    "ddf_set_recompute": (C.c_int, [_vp, _i32]),
    "ddf_debug_fail_allocation": (C.c_int, [_i64]),
    "ddf_save_checkpoint": (C.c_int, [_vp, C.c_char_p]),
    "ddf_load_checkpoint": (C.c_int, [_vp, C.c_char_p]),
    "ddf_get_train_activation_bytes": (C.c_int, [_vp, C.POINTER(_sz)]),
    "ddf_cast_scene": (C.c_int, [_vp, _i32, _vp, _i32, _RAYS, _i64, _vp, _vp, _vp]),
    "ddf_sdf_eval": (C.c_int, [_vp, _RAYS, _i64, _vp, _vp]),
    "ddf_sphere_trace": (C.c_int, [_vp, _RAYS, _i64, _i32, C.c_float, C.c_float, _vp, _vp, _vp,
                                   _vp]),
    "ddf_sdf_compute_grad": (C.c_int, [_vp, _RAYS, _vp, _i64, _vp, _vp]),
    "ddf_sdf_train_step": (C.c_int, [_vp, _RAYS, _vp, _i64, C.c_float, _vp, _vp]),
    "ddf_union_sdf": (C.c_int, [_vp, _i32, _vp, _i32, _RAYS, _i64, _vp, _vp]),
    "ddf_check_status": (C.c_int, [_vp, C.POINTER(C.c_uint32)]),
    "ddf_set_timeout_ns": (C.c_int, [_vp, _u64]),
    "ddf_set_chunk_rays": (C.c_int, [_vp, _i64]),
    "ddf_set_tile": (C.c_int, [_vp, _i32, C.POINTER(Tile)]),
    "ddf_get_tile": (C.c_int, [_vp, _i32, C.POINTER(Tile)]),
    "ddf_autotune": (C.c_int, [_vp, _RAYS, _i64, _vp, C.POINTER(C.c_double), _i32]),
    "ddf_profile_enable": (C.c_int, [_vp, _i32]),
    "ddf_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}

_LIB = None


class DDFError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Loads libddf.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2606_00817_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != 0:
        raise DDFError(name, st, lib().ddf_last_error().decode())


def _ptr(x):
    """Address of a torch tensor / numpy array / integer / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _rays(rays):
    if len(rays) != 6:
        raise ValueError("rays must hold 6 arrays (ox, oy, oz, dx, dy, dz)")
    arr = (C.c_void_p * 6)(*[_ptr(r) for r in rays])
    return C.cast(arr, _RAYS), arr


def _points(points):
    if len(points) != 3:
        raise ValueError("points must hold 3 arrays (x, y, z)")
    arr = (C.c_void_p * 3)(*[_ptr(p) for p in points])
    return C.cast(arr, _RAYS), arr


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_config(octaves, width, hidden_layers, precision="bf16", device=0, kind="ray") -> Config:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    return Config(int(octaves), int(width), int(hidden_layers), p, int(device), k)


# ----------------------------------------------------------- 1:1 entry points

def ddf_param_count(cfg: Config) -> int:
    return int(lib().ddf_param_count(C.byref(cfg)))


def ddf_create(cfg: Config) -> int:
    h = C.c_void_p()
    _call("ddf_create", C.byref(cfg), C.byref(h))
    _HIDDEN[h.value] = cfg.hidden_layers
    return h.value


def ddf_destroy(h) -> None:
    _call("ddf_destroy", h)


def ddf_last_error() -> str:
    return lib().ddf_last_error().decode()


def ddf_load_weights(h, blob: np.ndarray) -> None:
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    _call("ddf_load_weights", h, blob.ctypes.data, blob.size)


def ddf_get_weights(h, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _call("ddf_get_weights", h, out.ctypes.data, n)
    return out


def ddf_set_act_scales(h, scales) -> None:
    s = np.ascontiguousarray(scales, dtype=np.float32)
    _call("ddf_set_act_scales", h, s.ctypes.data if s.size else None, s.size)


def ddf_query_rays(h, rays, n, out_t, out_vis, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_query_rays", h, rp, int(n), _ptr(out_t), _ptr(out_vis), _stream(stream))


def ddf_query_shadow(h, rays, n, light, out_t, out_vis, out_occluded, stream=None) -> None:
    rp, keep = _rays(rays)
    lt = (C.c_float * 3)(*[float(v) for v in light])
    _call("ddf_query_shadow", h, rp, int(n), C.addressof(lt), _ptr(out_t), _ptr(out_vis),
          _ptr(out_occluded), _stream(stream))


def ddf_query_rays_host(h, rays, n, out_t, out_vis) -> None:
    rp, keep = _rays(rays)
    _call("ddf_query_rays_host", h, rp, int(n), _ptr(out_t), _ptr(out_vis))


def ddf_query_shadow_host(h, rays, n, light, out_t, out_vis, out_occluded) -> None:
    rp, keep = _rays(rays)
    lt = (C.c_float * 3)(*[float(v) for v in light])
    _call("ddf_query_shadow_host", h, rp, int(n), C.addressof(lt), _ptr(out_t), _ptr(out_vis),
          _ptr(out_occluded))


def ddf_query_rays_noalloc(h, rays, n, out_t, out_vis, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_query_rays_noalloc", h, rp, int(n), _ptr(out_t), _ptr(out_vis), _stream(stream))


def ddf_query_ao(h, rays, n_rays, offsets, n_points, out_hard, out_soft=None, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_query_ao", h, rp, int(n_rays), _ptr(offsets), int(n_points), _ptr(out_hard),
          _ptr(out_soft), _stream(stream))


def ddf_query_mixed(h, shadow_rays, n_shadow, light, out_t, out_vis, out_occluded, ao_rays,
                    n_ao_rays, offsets, n_points, out_hard, out_soft=None, stream=None) -> None:
    """Shadow rays and a ragged AO batch as one query; either part may be
    None (with a count of 0)."""
    sp, keep_s = _rays(shadow_rays if shadow_rays is not None else [None] * 6)
    ap, keep_a = _rays(ao_rays if ao_rays is not None else [None] * 6)
    lt = (C.c_float * 3)(*[float(v) for v in (light if light is not None else (0, 0, 0))])
    _call("ddf_query_mixed", h, sp, int(n_shadow), C.addressof(lt), _ptr(out_t), _ptr(out_vis),
          _ptr(out_occluded), ap, int(n_ao_rays), _ptr(offsets), int(n_points), _ptr(out_hard),
          _ptr(out_soft), _stream(stream))


def ddf_set_graph_mode(h, on: bool) -> None:
    _call("ddf_set_graph_mode", h, 1 if on else 0)


def ddf_calibrate_fp8(h, rays, n, stream=None):
    """Returns (amax, scales), H-1 floats each, and sets the scales."""
    rp, keep = _rays(rays)
    nl = max(0, lib_hidden_layers(h) - 1)
    amax = np.zeros(max(nl, 1), np.float32)
    sc = np.zeros(max(nl, 1), np.float32)
    _call("ddf_calibrate_fp8", h, rp, int(n), amax.ctypes.data, sc.ctypes.data, _stream(stream))
    return amax[:nl], sc[:nl]


def ddf_compute_grad(h, rays, t_target, hit_target, batch, out_loss=None, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_compute_grad", h, rp, _ptr(t_target), _ptr(hit_target), int(batch), _ptr(out_loss),
          _stream(stream))


def ddf_train_step(h, rays, t_target, hit_target, batch, lr, out_loss=None, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_train_step", h, rp, _ptr(t_target), _ptr(hit_target), int(batch), float(lr),
          _ptr(out_loss), _stream(stream))


def ddf_forward_train(h, inputs, batch, out_z, stream=None) -> None:
    """inputs: 6 ray arrays, or 3 point arrays for an SDF field."""
    ip, keep = _rays(inputs) if len(inputs) == 6 else _points(inputs)
    _call("ddf_forward_train", h, ip, int(batch), _ptr(out_z), _stream(stream))


def ddf_backward(h, dz, batch, stream=None) -> None:
    _call("ddf_backward", h, _ptr(dz), int(batch), _stream(stream))


def ddf_copy_grad(h, out, stream=None) -> None:
    _call("ddf_copy_grad", h, _ptr(out), int(out.numel()), _stream(stream))


def ddf_load_weights_device(h, blob, stream=None) -> None:
    _call("ddf_load_weights_device", h, _ptr(blob), int(blob.numel()), _stream(stream))


def ddf_sample_rays(spheres, n_spheres, boxes, n_boxes, seed, step, n, surface_frac, rays_out,
                    stream=None) -> None:
    rp, keep = _rays(rays_out)
    _call("ddf_sample_rays", _ptr(spheres), int(n_spheres), _ptr(boxes), int(n_boxes), int(seed),
          int(step), int(n), float(surface_frac), rp, _stream(stream))


def ddf_shift_rays(rays, t, hit, n, first, seed, step, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_shift_rays", rp, _ptr(t), _ptr(hit), int(n), int(first), int(seed), int(step),
          _stream(stream))


def ddf_distill(h, spheres, n_spheres, boxes, n_boxes, steps, batch, lr0, surface_frac=0.5,
                shift_frac=0.3, seed=0, stream=None) -> np.ndarray:
    """Runs the schedule; returns the per-step losses (host float32)."""
    losses = np.zeros(int(steps), np.float32)
    _call("ddf_distill", h, _ptr(spheres), int(n_spheres), _ptr(boxes), int(n_boxes), int(steps),
          int(batch), float(lr0), float(surface_frac), float(shift_frac), int(seed),
          losses.ctypes.data, _stream(stream))
    return losses


def ddf_render_gi(h, spheres, n_spheres, boxes, n_boxes, camera, width, height, light, ao_samples,
                  seed, out_shadow, out_ao, stream=None) -> None:
    """camera = (eye xyz, target xyz, up xyz, fov_y); h = None renders with
    the exact caster."""
    cam = (C.c_float * 10)(*[float(v) for v in camera])
    lt = (C.c_float * 3)(*[float(v) for v in light])
    _call("ddf_render_gi", h, _ptr(spheres), int(n_spheres), _ptr(boxes), int(n_boxes), cam,
          int(width), int(height), lt, int(ao_samples), int(seed), _ptr(out_shadow), _ptr(out_ao),
          _stream(stream))


def _cameras(cameras):
    cams = np.ascontiguousarray(np.asarray(cameras, np.float32).reshape(-1, 10))
    return cams, cams.shape[0]


def ddf_render_gs_depth(means, covs, opacities, n, cameras, width, height, out_t, out_hit,
                        stream=None) -> None:
    """cameras: [views, 10] rows (eye xyz, target xyz, up xyz, fov_y)."""
    cams, nv = _cameras(cameras)
    _call("ddf_render_gs_depth", _ptr(means), _ptr(covs), _ptr(opacities), int(n),
          cams.ctypes.data, nv, int(width), int(height), _ptr(out_t), _ptr(out_hit),
          _stream(stream))


def ddf_camera_rays(cameras, width, height, rays_out, stream=None) -> None:
    cams, nv = _cameras(cameras)
    rp, keep = _rays(rays_out)
    _call("ddf_camera_rays", cams.ctypes.data, nv, int(width), int(height), rp, _stream(stream))


def ddf_enter_box(rays, t, out_t_in, n, half_extent=1.0, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_enter_box", rp, _ptr(t), _ptr(out_t_in), int(n), float(half_extent),
          _stream(stream))


def ddf_distill_pool(h, pool, pool_t, pool_hit, n_pool, steps, batch, lr0, shift_frac=0.3, seed=0,
                     stream=None) -> np.ndarray:
    """Trains from a fixed pool of supervised rays; returns the per-step losses."""
    rp, keep = _rays(pool)
    losses = np.zeros(int(steps), np.float32)
    _call("ddf_distill_pool", h, rp, _ptr(pool_t), _ptr(pool_hit), int(n_pool), int(steps),
          int(batch), float(lr0), float(shift_frac), int(seed), losses.ctypes.data,
          _stream(stream))
    return losses


def ddf_get_grad(h, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _call("ddf_get_grad", h, out.ctypes.data, n)
    return out


def ddf_save_checkpoint(h, path) -> None:
    _call("ddf_save_checkpoint", h, os.fsencode(path))


def ddf_load_checkpoint(h, path) -> None:
    _call("ddf_load_checkpoint", h, os.fsencode(path))


def ddf_debug_fail_allocation(after: int) -> None:
    _call("ddf_debug_fail_allocation", int(after))


def ddf_set_recompute(h, segment: int) -> None:
    _call("ddf_set_recompute", h, int(segment))


def ddf_get_train_activation_bytes(h) -> int:
    out = _sz()
    _call("ddf_get_train_activation_bytes", h, C.byref(out))
    return int(out.value)


def ddf_reset_optimizer(h) -> None:
    _call("ddf_reset_optimizer", h)


def ddf_cast_scene(spheres, n_spheres, boxes, n_boxes, rays, n, out_t, out_hit, stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_cast_scene", _ptr(spheres), int(n_spheres), _ptr(boxes), int(n_boxes), rp, int(n),
          _ptr(out_t), _ptr(out_hit), _stream(stream))


def ddf_sdf_eval(h, points, n, out_s, stream=None) -> None:
    pp, keep = _points(points)
    _call("ddf_sdf_eval", h, pp, int(n), _ptr(out_s), _stream(stream))


def ddf_sphere_trace(h, rays, n, max_steps, eps, t_max, out_t, out_hit, out_steps=None,
                     stream=None) -> None:
    rp, keep = _rays(rays)
    _call("ddf_sphere_trace", h, rp, int(n), int(max_steps), float(eps), float(t_max), _ptr(out_t),
          _ptr(out_hit), _ptr(out_steps), _stream(stream))


def ddf_sdf_compute_grad(h, points, s_target, batch, out_loss=None, stream=None) -> None:
    pp, keep = _points(points)
    _call("ddf_sdf_compute_grad", h, pp, _ptr(s_target), int(batch), _ptr(out_loss), _stream(stream))


def ddf_sdf_train_step(h, points, s_target, batch, lr, out_loss=None, stream=None) -> None:
    pp, keep = _points(points)
    _call("ddf_sdf_train_step", h, pp, _ptr(s_target), int(batch), float(lr), _ptr(out_loss),
          _stream(stream))


def ddf_union_sdf(spheres, n_spheres, boxes, n_boxes, points, n, out_s, stream=None) -> None:
    pp, keep = _points(points)
    _call("ddf_union_sdf", _ptr(spheres), int(n_spheres), _ptr(boxes), int(n_boxes), pp, int(n),
          _ptr(out_s), _stream(stream))


_HIDDEN = {}


def lib_hidden_layers(h) -> int:
    return _HIDDEN[h]


def ddf_check_status(h) -> int:
    v = C.c_uint32()
    _call("ddf_check_status", h, C.byref(v))
    return int(v.value)


def ddf_set_timeout_ns(h, ns: int) -> None:
    _call("ddf_set_timeout_ns", h, int(ns))


def ddf_set_chunk_rays(h, chunk: int) -> None:
    _call("ddf_set_chunk_rays", h, int(chunk))


def ddf_set_tile(h, tile, which: int = 0) -> None:
    """tile = (bn, epi_warps, cta_pair, staged[, fused_encode]); which 0 =
    layers 2..H, 1 = layer 1."""
    _call("ddf_set_tile", h, int(which), C.byref(Tile(*[int(x) for x in tile])))


def ddf_get_tile(h, which: int = 0):
    """(bn, epi_warps, cta_pair, staged, fused_encode)"""
    t = Tile()
    _call("ddf_get_tile", h, int(which), C.byref(t))
    return (t.bn, t.epi_warps, t.cta_pair, t.staged, t.fused_encode)


# the autotuner's candidates, in its order; the last two are layer-1 only
TILE_CANDIDATES = ((256, 4, 0, 0, 0), (256, 8, 0, 0, 0), (128, 4, 0, 0, 0), (128, 8, 0, 0, 0),
                   (256, 4, 1, 0, 0), (256, 4, 1, 1, 0), (256, 8, 1, 1, 0), (256, 4, 0, 1, 1),
                   (256, 8, 0, 1, 1))


def ddf_autotune(h, rays, n, stream=None):
    """Returns ({tile: ms or None} for phase 1 (all layers), the same for
    phase 2 (layer 1 only)); leaves the fastest tiles set."""
    rp, keep = _rays(rays)
    k = len(TILE_CANDIDATES)
    ms = (C.c_double * (2 * k))()
    _call("ddf_autotune", h, rp, int(n), _stream(stream), ms, 2 * k)
    p1 = {c: (ms[i] if ms[i] >= 0 else None) for i, c in enumerate(TILE_CANDIDATES) if not c[4]}
    p2 = {c: (ms[k + i] if ms[k + i] >= 0 else None) for i, c in enumerate(TILE_CANDIDATES)}
    return p1, p2


def ddf_profile_enable(h, on: bool) -> None:
    _call("ddf_profile_enable", h, 1 if on else 0)


def ddf_profile_read(h):
    ms = (C.c_double * 4)()
    n = (C.c_int64 * 4)()
    _call("ddf_profile_read", h, ms, n)
    return {k: (ms[i], n[i]) for i, k in enumerate(PROFILE_CLASSES)}


# ----------------------------------------------------------- convenience

class DDF:
    """Owns one library handle; queries take and return torch CUDA tensors."""

    def __init__(self, octaves, width, hidden_layers, precision="bf16", device=0, kind="ray"):
        self.cfg = make_config(octaves, width, hidden_layers, precision, device, kind)
        self.device = device
        self.h = ddf_create(self.cfg)
        self.n_params = ddf_param_count(self.cfg)

    def close(self):
        if self.h:
            ddf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, blob, act_scales=None):
        ddf_load_weights(self.h, blob)
        if act_scales is not None:
            ddf_set_act_scales(self.h, act_scales)

    def _check(self, rays):
        import torch
        for r in rays:
            if not (r.is_cuda and r.dtype == torch.float32 and r.is_contiguous()):
                raise ValueError("rays must be contiguous float32 CUDA tensors")
        n = rays[0].numel()
        if any(r.numel() != n for r in rays):
            raise ValueError("ray arrays differ in length")
        return n

    def query(self, rays, stream=None):
        import torch
        n = self._check(rays)
        t = torch.empty(n, dtype=torch.float32, device=rays[0].device)
        v = torch.empty_like(t)
        ddf_query_rays(self.h, rays, n, t, v, stream or torch.cuda.current_stream(rays[0].device))
        return t, v

    def shadow(self, rays, light, stream=None):
        import torch
        n = self._check(rays)
        t = torch.empty(n, dtype=torch.float32, device=rays[0].device)
        v = torch.empty_like(t)
        occ = torch.empty(n, dtype=torch.uint8, device=rays[0].device)
        ddf_query_shadow(self.h, rays, n, light, t, v, occ,
                         stream or torch.cuda.current_stream(rays[0].device))
        return t, v, occ

    def query_host(self, rays_np, out_t=None, out_vis=None):
        n = int(rays_np[0].shape[0])
        out_t = np.empty(n, np.float32) if out_t is None else out_t
        out_vis = np.empty(n, np.float32) if out_vis is None else out_vis
        ddf_query_rays_host(self.h, rays_np, n, out_t, out_vis)
        return out_t, out_vis


def _autograd_function():
    import torch

    class DDFFunction(torch.autograd.Function):
        """z = f_theta(inputs) with theta a flat float32 CUDA tensor in the
        weight-blob layout: the head outputs before softplus / sigmoid
        (Sec. 3.1), [B, 2] for a ray field, [B] for an SDF field. Forward
        and backward are the library's (ddf_forward_train / ddf_backward:
        tensor-core layers, hand-written backward), so a loss written in
        torch on z trains the field with any torch optimiser. theta is copied
        into the handle on every forward; the activations of the latest
        forward of a handle are the ones its backward uses."""

        @staticmethod
        def forward(ctx, theta, model, inputs):
            stream = torch.cuda.current_stream(theta.device)
            B = inputs[0].numel()
            ddf_load_weights_device(model.h, theta.detach().contiguous(), stream)
            hr = 1 if model.cfg.kind == DDF_KIND_SDF else 2
            z = torch.empty((B, hr) if hr == 2 else (B,), dtype=torch.float32, device=theta.device)
            ddf_forward_train(model.h, list(inputs), B, z, stream)
            model._fwd_serial = getattr(model, "_fwd_serial", 0) + 1
            ctx.model, ctx.batch, ctx.serial, ctx.n = model, B, model._fwd_serial, theta.numel()
            return z

        @staticmethod
        def backward(ctx, dz):
            if ctx.model._fwd_serial != ctx.serial:
                raise RuntimeError("DDFFunction: another forward ran on this field since; "
                                   "its activations are gone")
            stream = torch.cuda.current_stream(dz.device)
            ddf_backward(ctx.model.h, dz.contiguous().to(torch.float32), ctx.batch, stream)
            g = torch.empty(ctx.n, dtype=torch.float32, device=dz.device)
            ddf_copy_grad(ctx.model.h, g, stream)
            return g, None, None

    return DDFFunction


def ddf_function():
    """The torch.autograd.Function over ddf_forward_train / ddf_backward
    (created on first use so that importing this module needs no torch)."""
    global _DDF_FUNCTION
    if _DDF_FUNCTION is None:
        _DDF_FUNCTION = _autograd_function()
    return _DDF_FUNCTION


_DDF_FUNCTION = None
