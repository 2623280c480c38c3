// gi.cu -- shadow and ambient-occlusion images, the paper's application
// (Sec. 3.3): per pixel of a pinhole camera an exact primary hit, then one
// shadow ray toward a point light and k cosine-weighted hemisphere rays, the
// secondary rays answered by the field (or by the exact caster, for the
// reference image).
#include <cstdint>

#include "caster.cuh"
#include "kernels.h"
#include "rng.cuh"

namespace ddf {

namespace {

constexpr float kGiOffset = 1e-3f;  // secondary origins this far off the surface

// Primary rays: shading point (xyz, 1 on a hit / 0 on background) and the
// shading normal (outward normal of the hit primitive, facing the eye).
__global__ void gi_primary_kernel(GiCamera cam, const float* __restrict__ spheres, int ns,
                                  const float* __restrict__ boxes, int nb, int64_t npx,
                                  float4* __restrict__ sp, float* __restrict__ nrm) {
  __shared__ float s_sph[4 * kMaxPrims];
  __shared__ float s_box[6 * kMaxPrims];
  for (int i = threadIdx.x; i < 4 * ns; i += blockDim.x) s_sph[i] = spheres[i];
  for (int i = threadIdx.x; i < 6 * nb; i += blockDim.x) s_box[i] = boxes[i];
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= npx) return;
  const int x = static_cast<int>(i % cam.width), y = static_cast<int>(i / cam.width);
  const float sx = (2.f * (static_cast<float>(x) + 0.5f) / cam.width - 1.f) * cam.tan_half *
                   (static_cast<float>(cam.width) / cam.height);
  const float sy = (1.f - 2.f * (static_cast<float>(y) + 0.5f) / cam.height) * cam.tan_half;
  float d[3];
  for (int k = 0; k < 3; ++k) d[k] = cam.f[k] + sx * cam.r[k] + sy * cam.u[k];
  const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) d[k] *= inv;
  const float o[3] = {cam.eye[0], cam.eye[1], cam.eye[2]};
  float n[3];
  const float t = cast_one(o, d, s_sph, ns, s_box, nb, n);
  if (!(t < __int_as_float(0x7f800000))) {
    sp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    nrm[3 * i] = 0.f;
    nrm[3 * i + 1] = 0.f;
    nrm[3 * i + 2] = 1.f;
    return;
  }
  if (n[0] * d[0] + n[1] * d[1] + n[2] * d[2] > 0.f) {
    n[0] = -n[0];
    n[1] = -n[1];
    n[2] = -n[2];
  }
  sp[i] = make_float4(o[0] + t * d[0] + kGiOffset * n[0], o[1] + t * d[1] + kGiOffset * n[1],
                      o[2] + t * d[2] + kGiOffset * n[2], 1.f);
  nrm[3 * i] = n[0];
  nrm[3 * i + 1] = n[1];
  nrm[3 * i + 2] = n[2];
}

// Secondary rays of pixel i: ray i (1 + k) toward the light, then k
// cosine-weighted directions (Malley) in the Duff et al. basis of the normal.
__global__ void gi_rays_kernel(const float4* __restrict__ sp, const float* __restrict__ nrm,
                               int64_t npx, int k, uint64_t seed, float lx, float ly, float lz,
                               RayOut r) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t per = 1 + k;
  if (j >= npx * per) return;
  const int64_t i = j / per;
  const int s = static_cast<int>(j - i * per);
  const float4 p = sp[i];
  float d[3];
  if (s == 0) {
    d[0] = lx - p.x;
    d[1] = ly - p.y;
    d[2] = lz - p.z;
    const float inv = rsqrtf(fmaxf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], 1e-30f));
    d[0] *= inv;
    d[1] *= inv;
    d[2] *= inv;
  } else {
    const float n0 = nrm[3 * i], n1 = nrm[3 * i + 1], n2 = nrm[3 * i + 2];
    const uint64_t key = rng_key(seed, static_cast<uint64_t>(i), static_cast<uint64_t>(s - 1));
    const float u1 = rng_u01(key, 0), u2 = rng_u01(key, 1);
    const float rr = sqrtf(u1), zz = sqrtf(fmaxf(0.f, 1.f - u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    const float lx0 = rr * cs, ly0 = rr * sn;
    const float sgn = n2 >= 0.f ? 1.f : -1.f;
    const float a = -1.f / (sgn + n2);
    const float b = n0 * n1 * a;
    const float t1[3] = {1.f + sgn * n0 * n0 * a, sgn * b, -sgn * n0};
    const float t2[3] = {b, sgn + n1 * n1 * a, -n1};
    const float nn[3] = {n0, n1, n2};
    for (int c = 0; c < 3; ++c) d[c] = lx0 * t1[c] + ly0 * t2[c] + zz * nn[c];
  }
  r.p[0][j] = p.x;
  r.p[1][j] = p.y;
  r.p[2][j] = p.z;
  r.p[3][j] = d[0];
  r.p[4][j] = d[1];
  r.p[5][j] = d[2];
}

// Pixel i: shadow 0 if its light ray hits before the light, else 1; AO =
// 1 - mean hit flag of its k hemisphere rays; background -1 in both.
__global__ void gi_compose_kernel(const float4* __restrict__ sp, int64_t npx, int k, float lx,
                                  float ly, float lz, const float* __restrict__ t,
                                  const uint8_t* __restrict__ hit, float* __restrict__ shadow,
                                  float* __restrict__ ao) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= npx) return;
  const float4 p = sp[i];
  if (p.w == 0.f) {
    if (shadow != nullptr) shadow[i] = -1.f;
    if (ao != nullptr) ao[i] = -1.f;
    return;
  }
  const int64_t base = i * (1 + k);
  if (shadow != nullptr) {
    const float dx = lx - p.x, dy = ly - p.y, dz = lz - p.z;
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    shadow[i] = (hit[base] != 0 && t[base] < dist) ? 0.f : 1.f;
  }
  if (ao != nullptr) {
    int h = 0;
    for (int s = 1; s <= k; ++s) h += hit[base + s] != 0;
    ao[i] = 1.f - static_cast<float>(h) / static_cast<float>(k);
  }
}

}  // namespace

cudaError_t launch_gi_primary(const GiCamera& cam, const float* spheres, int ns, const float* boxes,
                              int nb, float4* sp, float* nrm, cudaStream_t s) {
  const int64_t npx = static_cast<int64_t>(cam.width) * cam.height;
  if (npx <= 0) return cudaSuccess;
  if (ns > kMaxPrims || nb > kMaxPrims) return cudaErrorInvalidValue;
  gi_primary_kernel<<<static_cast<unsigned>((npx + 255) / 256), 256, 0, s>>>(cam, spheres, ns, boxes,
                                                                            nb, npx, sp, nrm);
  return cudaGetLastError();
}

cudaError_t launch_gi_rays(const float4* sp, const float* nrm, int64_t npx, int k, uint64_t seed,
                           const float light[3], RayOut r, cudaStream_t s) {
  const int64_t n = npx * (1 + k);
  if (n <= 0) return cudaSuccess;
  gi_rays_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(sp, nrm, npx, k, seed, light[0],
                                                                       light[1], light[2], r);
  return cudaGetLastError();
}

cudaError_t launch_gi_compose(const float4* sp, int64_t npx, int k, const float light[3],
                              const float* t, const uint8_t* hit, float* shadow, float* ao,
                              cudaStream_t s) {
  if (npx <= 0) return cudaSuccess;
  gi_compose_kernel<<<static_cast<unsigned>((npx + 255) / 256), 256, 0, s>>>(
      sp, npx, k, light[0], light[1], light[2], t, hit, shadow, ao);
  return cudaGetLastError();
}

}  // namespace ddf
