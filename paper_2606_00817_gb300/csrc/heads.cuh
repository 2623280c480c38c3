// heads.cuh -- the two DDF outputs (Sec. 3.1, Eq. 1) and the shadow test of
// Sec. 3.3, shared by every kernel that finishes a query: t = softplus(z0),
// xi = sigmoid(z1), hit iff z1 > 0, occluded iff hit closer than the light.
#pragma once
#include "kernels.h"

namespace ddf {

__device__ __forceinline__ float softplus_f(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}

__device__ __forceinline__ float sigmoid_f(float z) {
  const float e = expf(-fabsf(z));
  return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

// Component c of ray `row` of a batch that may join two sets of arrays.
__device__ __forceinline__ float ray_ld(const RaySoA& r, int c, int64_t row) {
  return row < r.split ? __ldg(r.p[c] + row) : __ldg(r.q[c] + (row - r.split));
}

__device__ __forceinline__ void write_heads(const HeadOut& o, int64_t i, float z0, float z1) {
  if (i >= o.split) {  // the second part of a mixed batch: hit flag and visibility only
    const int64_t k = i - o.split;
    if (o.vis2 != nullptr) o.vis2[k] = sigmoid_f(z1);
    if (o.hit2 != nullptr) o.hit2[k] = z1 > 0.f ? 1 : 0;
    return;
  }
  const float t = softplus_f(z0);
  if (o.t != nullptr) o.t[i] = t;
  if (o.vis != nullptr) o.vis[i] = sigmoid_f(z1);
  if (o.hit != nullptr) o.hit[i] = z1 > 0.f ? 1 : 0;
  if (o.z0 != nullptr) o.z0[i] = z0;
  if (o.occluded != nullptr) {
    const float dx = o.light[0] - o.rays.p[0][i];
    const float dy = o.light[1] - o.rays.p[1][i];
    const float dz = o.light[2] - o.rays.p[2][i];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    o.occluded[i] = (z1 > 0.f && t < dist) ? 1 : 0;
  }
}

}  // namespace ddf
