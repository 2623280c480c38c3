// caster.cuh -- exact first hit of a ray against a union of spheres
// (cx, cy, cz, r) and axis-aligned boxes (lo xyz, hi xyz): the supervision of
// Sec. 3.2 with analytic primitives. Surfaces, not CSG: the nearest positive
// root over every primitive; tangent rays hit; slabs are closed.
#pragma once
#include <cstdint>

namespace ddf {

constexpr int kMaxPrims = 1024;

// t of the first hit (+inf on a miss); if n != nullptr also the outward
// normal of the primitive surface hit there (for a box, the normal of the
// slab the ray crosses at t).
__device__ __forceinline__ float cast_one(const float (&o)[3], const float (&d)[3],
                                          const float* sph, int ns, const float* box, int nb,
                                          float* n) {
  const float a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  float best = __int_as_float(0x7f800000);
  int kind = -1, prim = -1, axis = 0;
  float side = 0.f;
  for (int s = 0; s < ns; ++s) {
    const float oc0 = o[0] - sph[4 * s], oc1 = o[1] - sph[4 * s + 1], oc2 = o[2] - sph[4 * s + 2];
    const float r = sph[4 * s + 3];
    const float b = d[0] * oc0 + d[1] * oc1 + d[2] * oc2;
    const float q = oc0 * oc0 + oc1 * oc1 + oc2 * oc2 - r * r;
    const float disc = b * b - a * q;
    if (disc < 0.f) continue;
    const float sq = sqrtf(disc);
    const float hh = -b - (b >= 0.f ? sq : -sq);  // no cancellation
    if (hh == 0.f) continue;
    const float r1 = hh / a, r2 = q / hh;
    const float lo = fminf(r1, r2), hi = fmaxf(r1, r2);
    const float t = lo > 0.f ? lo : hi;
    if (t > 0.f && t < best) {
      best = t;
      kind = 0;
      prim = s;
    }
  }
  for (int bx = 0; bx < nb; ++bx) {
    float tn = -__int_as_float(0x7f800000), tf = __int_as_float(0x7f800000);
    int an = 0, af = 0;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = box[6 * bx + k], hi = box[6 * bx + 3 + k];
      if (d[k] == 0.f) {
        miss |= (o[k] < lo) || (o[k] > hi);
      } else {
        const float ta = (lo - o[k]) / d[k], tb = (hi - o[k]) / d[k];
        const float near = fminf(ta, tb), far = fmaxf(ta, tb);
        if (near > tn) tn = near, an = k;
        if (far < tf) tf = far, af = k;
      }
    }
    if (miss || !(tn <= tf) || !(tf > 0.f)) continue;
    const bool enter = tn > 0.f;
    const float t = enter ? tn : tf;
    if (t < best) {
      best = t;
      kind = 1;
      prim = bx;
      axis = enter ? an : af;
      // entering: the normal faces the ray; leaving from inside: along it
      side = enter ? (d[axis] > 0.f ? -1.f : 1.f) : (d[axis] > 0.f ? 1.f : -1.f);
    }
  }
  if (n != nullptr) {
    n[0] = n[1] = n[2] = 0.f;
    if (kind == 0) {
      const float* s = sph + 4 * prim;
      const float inv = 1.f / s[3];
      n[0] = (o[0] + best * d[0] - s[0]) * inv;
      n[1] = (o[1] + best * d[1] - s[1]) * inv;
      n[2] = (o[2] + best * d[2] - s[2]) * inv;
    } else if (kind == 1) {
      n[axis] = side;
    }
  }
  return best;
}

}  // namespace ddf
