"""Seeded synthetic inputs for the DDF query path.

This module is shared by the FP64 oracle (``oracle/``) and by the GPU path's
tests and benchmark. It holds random numbers and workload recipes only: ray
batches, analytic scenes, surface sample points, Xavier-initialised weight
blobs and ragged ambient-occlusion direction sets. None of the DDF's own
arithmetic (encoding, MLP, heads, loss, ray casting) lives here.

Random source: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: output i of stream s is
the SplitMix64 finaliser applied to ``key(seed, s) + (i + 1) * GAMMA``, which
equals the i-th output of the sequential generator started at that key.
Uniform doubles take the top 53 bits. Everything is generated in float64 and
rounded once to float32 where the product consumes float32.

The workloads follow the paper's query kinds (Sec. 3.3: primary, shadow,
ambient-occlusion and bounce rays) at the sizes used for measurement:
  * ``uniform_rays``: origins uniform in [-1,1]^3, directions uniform on S^2.
  * ``shadow_rays``: points on an analytic sphere scene, offset along the
    normal by 1e-3, aimed at a point light.
  * ``ao_rays``: per shading point a random count in [4, 64] of
    cosine-weighted hemisphere directions, flattened with CSR offsets.

For the supervision study (Sec. 4.2), a scene with thin parts (``table_scene``)
and flat 3D Gaussians laid on its visible surfaces (``surface_gaussians``)
stand in for a trained 3DGS scene; ``orbit_cameras`` places the views.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids: one per independent random quantity
S_ORIGIN, S_DIR, S_WEIGHTS, S_SCENE, S_POINTS, S_COUNTS, S_HEMI, S_TARGET = range(1, 9)
S_TABLE = 15
S_GAUSS, S_GAUSS_OPAC, S_VIEWS = 16, 17, 18


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of SplitMix64 stream ``stream`` (uint64)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 0x1000003 + stream) & 0xFFFFFFFFFFFFFFFF],
                            dtype=np.uint64))[0]
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(key + i * GAMMA)


def uniform(seed: int, stream: int, n: int, lo=0.0, hi=1.0, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [lo, hi)."""
    u = (splitmix64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def gaussian(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    u = uniform(seed, stream, 2 * n, offset=2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def unit_vectors(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n directions uniform on S^2 (normalised Gaussian triples), float64 [n,3]."""
    g = gaussian(seed, stream, 3 * n, offset=3 * offset).reshape(n, 3)
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return g / nrm


@dataclass
class Rays:
    """Ray batch as a structure of arrays (float32, contiguous)."""
    ox: np.ndarray
    oy: np.ndarray
    oz: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray

    @property
    def n(self) -> int:
        return int(self.ox.shape[0])

    def soa(self):
        return [self.ox, self.oy, self.oz, self.dx, self.dy, self.dz]

    def origins(self) -> np.ndarray:
        return np.stack([self.ox, self.oy, self.oz], axis=1)

    def dirs(self) -> np.ndarray:
        return np.stack([self.dx, self.dy, self.dz], axis=1)

    def slice(self, a: int, b: int) -> "Rays":
        return Rays(*[x[a:b].copy() for x in self.soa()])

    @staticmethod
    def from_arrays(o: np.ndarray, d: np.ndarray) -> "Rays":
        o = np.asarray(o, dtype=np.float64)
        d = np.asarray(d, dtype=np.float64)
        f = lambda a: np.ascontiguousarray(a.astype(np.float32))
        return Rays(f(o[:, 0]), f(o[:, 1]), f(o[:, 2]), f(d[:, 0]), f(d[:, 1]), f(d[:, 2]))


def uniform_rays(n: int, seed: int = 0) -> Rays:
    """Origins uniform in [-1,1]^3, directions uniform on the sphere."""
    o = uniform(seed, S_ORIGIN, 3 * n, -1.0, 1.0).reshape(n, 3)
    d = unit_vectors(seed, S_DIR, n)
    return Rays.from_arrays(o, d)


# ---------------------------------------------------------------- networks

@dataclass
class NetShape:
    """DDF network shape: sinusoidal encoding with ``octaves`` bands per
    coordinate, ``hidden`` ReLU layers of ``width``, and a 2-output head."""
    octaves: int
    width: int
    hidden: int

    @property
    def d_in(self) -> int:
        return 6 + 12 * self.octaves

    def layer_dims(self):
        """(fan_out, fan_in) for every linear layer, the head last."""
        dims = [(self.width, self.d_in)]
        dims += [(self.width, self.width)] * (self.hidden - 1)
        dims.append((2, self.width))
        return dims

    @property
    def n_params(self) -> int:
        return sum(o * i + o for o, i in self.layer_dims())


def xavier_blob(shape: NetShape, seed: int = 0) -> np.ndarray:
    """Float32 weight blob, Xavier-uniform W and U(+-1/sqrt(fan_in)) biases.

    Layout: for each layer in order, W[out][in] row-major then b[out]; the
    2-row head comes last (row 0 drives the distance, row 1 the visibility).
    """
    parts = []
    off = 0
    for fo, fi in shape.layer_dims():
        a = np.sqrt(6.0 / (fi + fo))
        w = uniform(seed, S_WEIGHTS, fo * fi, -a, a, offset=off)
        off += fo * fi
        bb = 1.0 / np.sqrt(fi)
        b = uniform(seed, S_WEIGHTS, fo, -bb, bb, offset=off)
        off += fo
        parts += [w, b]
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def sdf_layer_dims(octaves: int, width: int, hidden: int):
    """(fan_out, fan_in) of the SDF baseline network: Fourier-encoded point
    (3 + 6 L inputs), hidden ReLU layers, a 1-output head."""
    d_in = 3 + 6 * octaves
    return [(width, d_in)] + [(width, width)] * (hidden - 1) + [(1, width)]


def xavier_blob_dims(dims, seed: int = 0) -> np.ndarray:
    """Float32 blob for arbitrary (fan_out, fan_in) layers, initialised as
    xavier_blob does."""
    parts = []
    off = 0
    for fo, fi in dims:
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(uniform(seed, S_WEIGHTS, fo * fi, -a, a, offset=off))
        off += fo * fi
        bb = 1.0 / np.sqrt(fi)
        parts.append(uniform(seed, S_WEIGHTS, fo, -bb, bb, offset=off))
        off += fo
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def hashgrid_blob(n_params: int, mlp_dims, seed: int = 0, table_scale: float = 1.0) -> np.ndarray:
    """Float32 blob of a hash-grid field: the level tables (everything before
    the MLP) uniform in +-table_scale, then Xavier MLP layers with the given
    (fan_out, fan_in) dims."""
    mlp = xavier_blob_dims(mlp_dims, seed)
    n_tab = n_params - mlp.size
    if n_tab <= 0:
        raise ValueError("n_params leaves no room for the tables")
    tab = uniform(seed, S_TABLE, n_tab, -table_scale, table_scale)
    return np.ascontiguousarray(np.concatenate([tab.astype(np.float32), mlp]))


def uniform_points(n: int, lo: float = -1.2, hi: float = 1.2, seed: int = 0) -> np.ndarray:
    """n points uniform in the cube [lo, hi]^3, float32 [n, 3]."""
    return uniform(seed, S_TARGET, 3 * n, lo, hi).reshape(n, 3).astype(np.float32)


def split_blob(shape: NetShape, blob: np.ndarray):
    """[(W[out,in], b[out]), ...] views of a weight blob, head last."""
    out = []
    off = 0
    for fo, fi in shape.layer_dims():
        w = blob[off:off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = blob[off:off + fo]
        off += fo
        out.append((w, b))
    if off != blob.size:
        raise ValueError(f"blob has {blob.size} floats, shape needs {off}")
    return out


# ---------------------------------------------------------------- scenes

@dataclass
class Scene:
    """Union of spheres (centre, radius) and axis-aligned boxes (lo, hi)."""
    centers: np.ndarray  # [S,3] float64
    radii: np.ndarray    # [S]
    box_lo: np.ndarray   # [B,3]
    box_hi: np.ndarray   # [B,3]

    def packed(self) -> np.ndarray:
        """Float32 [S*4 + B*6]: (cx,cy,cz,r) per sphere, then (lo,hi) per box."""
        s = np.concatenate([self.centers, self.radii[:, None]], axis=1).reshape(-1)
        b = np.concatenate([self.box_lo, self.box_hi], axis=1).reshape(-1)
        return np.ascontiguousarray(np.concatenate([s, b]).astype(np.float32))

    def as_float32(self) -> "Scene":
        """The scene with every number rounded to float32 (what a GPU reads)."""
        r = lambda a: a.astype(np.float32).astype(np.float64)
        return Scene(r(self.centers), r(self.radii), r(self.box_lo), r(self.box_hi))


def random_scene(n_spheres: int, n_boxes: int, seed: int = 0) -> Scene:
    """Sphere centres U[-1,1]^3, radii U[0.05,0.3]; box centres U[-1,1]^3 with
    half-extents U[0.05,0.3] per axis, clipped to [-1,1]^3."""
    u = uniform(seed, S_SCENE, 4 * n_spheres + 6 * n_boxes)
    c = -1.0 + 2.0 * u[:3 * n_spheres].reshape(n_spheres, 3)
    r = 0.05 + 0.25 * u[3 * n_spheres:4 * n_spheres]
    ub = u[4 * n_spheres:].reshape(n_boxes, 6)
    bc = -1.0 + 2.0 * ub[:, :3]
    he = 0.05 + 0.25 * ub[:, 3:]
    lo = np.clip(bc - he, -1.0, 1.0)
    hi = np.clip(bc + he, -1.0, 1.0)
    return Scene(c, r, lo, hi).as_float32()


def surface_points(scene: Scene, n: int, seed: int = 0):
    """n points uniform on the union's sphere surfaces (sphere chosen by area),
    dropping points that lie inside another sphere. Returns (p, normal), float64."""
    S = scene.radii.shape[0]
    area = scene.radii ** 2
    cdf = np.cumsum(area) / area.sum()
    got_p, got_n, have, off = [], [], 0, 0
    while have < n:
        m = int((n - have) * 1.3) + 1024
        u = uniform(seed, S_POINTS, m, offset=off)
        idx = np.minimum(np.searchsorted(cdf, u, side="right"), S - 1)
        nrm = unit_vectors(seed, S_POINTS + 100, m, offset=off)
        off += m
        p = scene.centers[idx] + scene.radii[idx, None] * nrm
        inside = np.zeros(m, dtype=bool)
        for j in range(S):
            dj = np.linalg.norm(p - scene.centers[j], axis=1)
            inside |= (dj < scene.radii[j]) & (idx != j)
        keep = ~inside
        got_p.append(p[keep])
        got_n.append(nrm[keep])
        have += int(keep.sum())
    return np.concatenate(got_p)[:n], np.concatenate(got_n)[:n]


def shadow_rays(scene: Scene, n: int, light=(3.0, 3.0, 3.0), seed: int = 0, eps: float = 1e-3) -> Rays:
    """Shadow rays: surface point offset by eps along its normal, aimed at the light."""
    p, nrm = surface_points(scene, n, seed)
    o = p + eps * nrm
    d = np.asarray(light, dtype=np.float64)[None, :] - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Rays.from_arrays(o, d)


def _frame(nrm: np.ndarray):
    """Orthonormal tangent frame (t, b) around each unit normal."""
    a = np.where(np.abs(nrm[:, :1]) > 0.9, np.array([[0.0, 1.0, 0.0]]), np.array([[1.0, 0.0, 0.0]]))
    t = np.cross(a, nrm)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    b = np.cross(nrm, t)
    return t, b


def cosine_directions(nrm: np.ndarray, seed: int, stream: int, offset: int = 0) -> np.ndarray:
    """One cosine-weighted hemisphere direction per normal (Malley's method:
    uniform disk sample lifted onto the hemisphere)."""
    m = nrm.shape[0]
    u = uniform(seed, stream, 2 * m, offset=2 * offset).reshape(m, 2)
    r = np.sqrt(u[:, 0])
    phi = 2.0 * np.pi * u[:, 1]
    x, y = r * np.cos(phi), r * np.sin(phi)
    z = np.sqrt(np.maximum(0.0, 1.0 - u[:, 0]))
    t, b = _frame(nrm)
    d = x[:, None] * t + y[:, None] * b + z[:, None] * nrm
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def bounce_rays(scene: Scene, n: int, seed: int = 0, eps: float = 1e-3) -> Rays:
    """One-bounce GI rays: surface point offset along the normal, one
    cosine-weighted direction about the normal."""
    p, nrm = surface_points(scene, n, seed)
    o = p + eps * nrm
    d = cosine_directions(nrm, seed, S_HEMI)
    return Rays.from_arrays(o, d)


def ao_rays(scene: Scene, n_points: int, seed: int = 0, lo: int = 4, hi: int = 64, eps: float = 1e-3):
    """Ragged ambient-occlusion batch. Returns (rays, offsets int32[n_points+1]).
    Point p owns rays offsets[p]..offsets[p+1]-1; counts are uniform in [lo, hi]."""
    p, nrm = surface_points(scene, n_points, seed)
    counts = lo + np.floor(uniform(seed, S_COUNTS, n_points) * (hi - lo + 1)).astype(np.int64)
    counts = np.minimum(counts, hi)
    offsets = np.zeros(n_points + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    owner = np.repeat(np.arange(n_points), counts)
    o = p[owner] + eps * nrm[owner]
    d = cosine_directions(nrm[owner], seed, S_HEMI)
    if offsets[-1] >= 2 ** 31:
        raise ValueError("ragged batch exceeds int32 offsets")
    return Rays.from_arrays(o, d), offsets.astype(np.int32)


# ------------------------------------------------- supervision-study scene

def table_scene():
    """A table on a floor slab with a ball and a mug on top (boxes in
    [-0.95, 0.95]^3): tabletop 1.4 x 0.06 x 1.0, four legs 0.04 x 0.90 x 0.04,
    two cross bars 1.2 x 0.03 x 0.03, a mug (sphere r 0.15) with a handle of
    three 0.03-thick bars, a ball (r 0.12). Returns (scene, thin) where thin
    marks the boxes that are legs, bars or handle parts: a few pixels wide in
    a 256-pixel view from 3 units away, the parts the study is about."""
    boxes, thin = [], []

    def box(lo, hi, is_thin):
        boxes.append((lo, hi))
        thin.append(is_thin)

    box((-0.95, -0.86, -0.95), (0.95, -0.80, 0.95), False)          # floor
    box((-0.70, 0.10, -0.50), (0.70, 0.16, 0.50), False)            # tabletop
    for x in (-0.64, 0.60):
        for z in (-0.44, 0.40):
            box((x, -0.80, z), (x + 0.04, 0.10, z + 0.04), True)    # legs
    for z in (-0.435, 0.405):
        box((-0.60, -0.50, z), (0.60, -0.47, z + 0.03), True)       # cross bars
    box((0.50, 0.22, -0.015), (0.53, 0.40, 0.015), True)            # handle
    box((0.43, 0.37, -0.015), (0.53, 0.40, 0.015), True)
    box((0.43, 0.22, -0.015), (0.53, 0.25, 0.015), True)
    centers = np.array([[0.30, 0.31, 0.0], [-0.30, 0.28, 0.10]])
    radii = np.array([0.15, 0.12])
    lo = np.array([b[0] for b in boxes], dtype=np.float64)
    hi = np.array([b[1] for b in boxes], dtype=np.float64)
    return Scene(centers, radii, lo, hi).as_float32(), np.array(thin)


def surface_gaussians(scene: Scene, n: int, sigma_t: float = 0.02, sigma_n: float = 0.002,
                      opacity=(0.6, 1.0), seed: int = 0, coverage: bool = True):
    """n flat 3D Gaussians on the union's outer surface, the shape a trained
    3DGS scene takes on opaque surfaces: means uniform by area over sphere
    surfaces and box faces (points strictly inside another primitive
    dropped), covariance sigma_t^2 in the tangent plane and sigma_n^2 along
    the normal, opacity uniform in the given range. With coverage, a
    Gaussian on a part narrower than itself is softened the way a fit to
    images softens it: its opacity is scaled by min(1, w / (sqrt(2 pi)
    sigma_t)), w the face's narrower side (2 r on a sphere), so that its
    alpha integrated across the part matches the part's width. Returns
    float32 means [n, 3], covs [n, 6] = (xx, xy, xz, yy, yz, zz) and
    opacities [n]."""
    S, B = scene.radii.shape[0], scene.box_lo.shape[0]
    ext = scene.box_hi - scene.box_lo
    face_area = np.stack([ext[:, 1] * ext[:, 2], ext[:, 0] * ext[:, 2], ext[:, 0] * ext[:, 1]], 1)
    area = np.concatenate([4 * np.pi * scene.radii ** 2, np.repeat(face_area, 2, axis=1).ravel()])
    cdf = np.cumsum(area) / area.sum()
    got_p, got_n, got_w, have, off = [], [], [], 0, 0
    while have < n:
        m = int((n - have) * 1.3) + 1024
        u = uniform(seed, S_GAUSS, 3 * m, offset=3 * off).reshape(m, 3)
        nrm_s = unit_vectors(seed, S_GAUSS + 100, m, offset=off)
        off += m
        k = np.minimum(np.searchsorted(cdf, u[:, 0], side="right"), area.size - 1)
        p = np.zeros((m, 3))
        nrm = np.zeros((m, 3))
        own = np.full(m, -1)
        width = np.zeros(m)
        sph = k < S
        p[sph] = scene.centers[k[sph]] + scene.radii[k[sph], None] * nrm_s[sph]
        nrm[sph] = nrm_s[sph]
        own[sph] = k[sph]
        width[sph] = 2 * scene.radii[k[sph]]
        for q in np.nonzero(~sph)[0]:
            f = k[q] - S
            b, face = f // 6, f % 6
            axis, side = face // 2, face % 2
            a1, a2 = (axis + 1) % 3, (axis + 2) % 3
            p[q, a1] = scene.box_lo[b, a1] + u[q, 1] * ext[b, a1]
            p[q, a2] = scene.box_lo[b, a2] + u[q, 2] * ext[b, a2]
            p[q, axis] = scene.box_hi[b, axis] if side else scene.box_lo[b, axis]
            nrm[q, axis] = 1.0 if side else -1.0
            own[q] = S + b
            width[q] = min(ext[b, a1], ext[b, a2])
        inside = np.zeros(m, dtype=bool)
        for j in range(S):
            inside |= (np.linalg.norm(p - scene.centers[j], axis=1) < scene.radii[j] - 1e-6) & (own != j)
        for j in range(B):
            inside |= np.all((p > scene.box_lo[j] + 1e-6) & (p < scene.box_hi[j] - 1e-6), axis=1) \
                & (own != S + j)
        got_p.append(p[~inside])
        got_n.append(nrm[~inside])
        got_w.append(width[~inside])
        have += int((~inside).sum())
    p = np.concatenate(got_p)[:n]
    nrm = np.concatenate(got_n)[:n]
    width = np.concatenate(got_w)[:n]
    t, b = _frame(nrm)
    cov = sigma_t ** 2 * (t[:, :, None] * t[:, None, :] + b[:, :, None] * b[:, None, :]) \
        + sigma_n ** 2 * nrm[:, :, None] * nrm[:, None, :]
    covs = cov[:, [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]]
    op = uniform(seed, S_GAUSS_OPAC, n, opacity[0], opacity[1])
    if coverage:
        op = op * np.minimum(1.0, width / (np.sqrt(2 * np.pi) * sigma_t))
    return tuple(np.ascontiguousarray(a, dtype=np.float32) for a in (p, covs, op))


def orbit_cameras(n: int, radius: float = 3.0, target=(0.0, -0.2, 0.0), elev=(10.0, 55.0),
                  fov_y_deg: float = 40.0, seed: int = 0, offset: int = 0) -> np.ndarray:
    """n pinhole cameras [n, 10] (eye, target, up = +y, fov_y in radians) on a
    sphere about target: azimuth uniform in [0, 360), elevation uniform in
    elev degrees."""
    u = uniform(seed, S_VIEWS, 2 * n, offset=2 * offset).reshape(n, 2)
    az = 2 * np.pi * u[:, 0]
    el = np.radians(elev[0] + (elev[1] - elev[0]) * u[:, 1])
    tg = np.asarray(target, np.float64)
    eye = tg + radius * np.stack([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)], 1)
    cams = np.zeros((n, 10))
    cams[:, 0:3] = eye
    cams[:, 3:6] = tg
    cams[:, 7] = 1.0
    cams[:, 9] = np.radians(fov_y_deg)
    return cams.astype(np.float32)
