// distill.cu -- ray sampling for the distillation schedule (Sec. 3.2 / 3.4):
// camera rays that view the object, rays anchored on its surface that point
// in all directions, and the ray-march shifted copies that keep the field
// consistent along a ray (a ray that hits at t, moved forward by s along
// itself, hits at t - s).
//
// Random numbers come from the counter-based SplitMix64 of rng.cuh: draw j of
// ray i at step k is mix(key(seed, k, i) + j), so any ray of any step can be
// regenerated alone.
#include <cstdint>

#include "kernels.h"
#include "caster.cuh"
#include "rng.cuh"

namespace ddf {

namespace {

__device__ __forceinline__ float u01(uint64_t key, int j) { return rng_u01(key, j); }

__device__ __forceinline__ uint64_t ray_key(uint64_t seed, uint64_t step, int64_t i) {
  return rng_key(seed, step, static_cast<uint64_t>(i));
}

// Unit vector uniform on the sphere from two uniforms.
__device__ __forceinline__ void sphere_dir(float a, float b, float& x, float& y, float& z) {
  z = 2.f * a - 1.f;
  const float r = sqrtf(fmaxf(0.f, 1.f - z * z));
  float s, c;
  sincospif(2.f * b, &s, &c);
  x = r * c;
  y = r * s;
}

constexpr float kSurfaceOffset = 1e-3f;  // origins sit this far off the surface
constexpr int kMaxSurfaceElems = kMaxPrims + 6 * kMaxPrims;
constexpr int kSampleThreads = 256;

// Integer area weight of surface element e (the spheres, then six faces per
// box; face f is axis f / 2, the upper side if f is odd): floor(A 2^24),
// with A the float32 product (4 pi r) r or (hi_u - lo_u)(hi_v - lo_v),
// clamped to [0, 2^16] (a NaN to 0). Rounded products, no contraction.
__device__ __forceinline__ uint64_t surface_weight(const float* spheres, int ns,
                                                   const float* boxes, int e) {
  float a;
  if (e < ns) {
    const float rad = spheres[4 * e + 3];
    a = __fmul_rn(__fmul_rn(12.566370964050293f, rad), rad);  // 4 pi rounded to float32
  } else {
    const float* b = boxes + 6 * ((e - ns) / 6);
    const int axis = ((e - ns) % 6) >> 1;
    const int u = (axis + 1) % 3, v = (axis + 2) % 3;
    a = __fmul_rn(__fsub_rn(b[u + 3], b[u]), __fsub_rn(b[v + 3], b[v]));
  }
  a = fminf(fmaxf(a, 0.f), 65536.f);
  return static_cast<uint64_t>(__fmul_rn(a, 16777216.f));
}

__global__ void __launch_bounds__(kSampleThreads)
    sample_rays_kernel(const float* __restrict__ spheres, int ns,
                       const float* __restrict__ boxes, int nb, uint64_t seed,
                       uint64_t step, int64_t n, float surface_frac, RayOut r) {
  // The block's copy of the area distribution: exact integer prefix sums of
  // the weights (each thread a contiguous run of elements, the runs' totals
  // scanned in order), each rounded once to float32, so the choice below
  // does not depend on how the sums were split.
  __shared__ float s_cum[kMaxSurfaceElems];
  __shared__ unsigned long long s_run[kSampleThreads];
  __shared__ unsigned long long s_total;
  const int E = ns + 6 * nb;
  const int per = (E + kSampleThreads - 1) / kSampleThreads;
  const int e0 = static_cast<int>(threadIdx.x) * per, e1 = min(E, e0 + per);
  unsigned long long run = 0;
  for (int e = e0; e < e1; ++e) run += surface_weight(spheres, ns, boxes, e);
  s_run[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int t = 0; t < kSampleThreads; ++t) {
      const unsigned long long v = s_run[t];
      s_run[t] = acc;
      acc += v;
    }
    s_total = acc;
  }
  __syncthreads();
  run = s_run[threadIdx.x];
  for (int e = e0; e < e1; ++e) {
    run += surface_weight(spheres, ns, boxes, e);
    s_cum[e] = __ull2float_rn(run);
  }
  __syncthreads();
  const float total = __ull2float_rn(s_total);

  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = ray_key(seed, step, i);
  float ox, oy, oz, dx, dy, dz;
  if (u01(key, 0) < surface_frac && total > 0.f) {
    // a surface point uniform by area, its normal, and a direction uniform
    // over the whole sphere; the element: the first whose rounded prefix
    // sum exceeds u W
    const float x = __fmul_rn(u01(key, 1), total);
    int lo = 0, hi = E;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_cum[mid] > x)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int p = min(lo, E - 1);
    float px, py, pz, nx, ny, nz;
    if (p < ns) {
      const float* s = spheres + 4 * p;
      sphere_dir(u01(key, 2), u01(key, 3), nx, ny, nz);
      px = s[0] + s[3] * nx;
      py = s[1] + s[3] * ny;
      pz = s[2] + s[3] * nz;
    } else {
      const float* b = boxes + 6 * ((p - ns) / 6);
      const int face = (p - ns) % 6;
      const int axis = face >> 1;
      const float sg = (face & 1) ? 1.f : -1.f;
      const float a = u01(key, 3), c = u01(key, 4);
      float q[3];
      // the two in-face coordinates take a and c; the face's own axis its side
      const int u = (axis + 1) % 3, v = (axis + 2) % 3;
      q[u] = b[u] + a * (b[u + 3] - b[u]);
      q[v] = b[v] + c * (b[v + 3] - b[v]);
      q[axis] = sg > 0.f ? b[axis + 3] : b[axis];
      float nrm[3] = {0.f, 0.f, 0.f};
      nrm[axis] = sg;
      px = q[0];
      py = q[1];
      pz = q[2];
      nx = nrm[0];
      ny = nrm[1];
      nz = nrm[2];
    }
    ox = px + kSurfaceOffset * nx;
    oy = py + kSurfaceOffset * ny;
    oz = pz + kSurfaceOffset * nz;
    sphere_dir(u01(key, 5), u01(key, 6), dx, dy, dz);
  } else {
    // a camera ray: origin uniform on a face of the box [-1, 1]^3, aimed at a
    // point uniform in the inner box [-0.9, 0.9]^3
    const int face = min(static_cast<int>(u01(key, 1) * 6.f), 5);
    const int axis = face >> 1;
    float o[3];
    o[(axis + 1) % 3] = 2.f * u01(key, 2) - 1.f;
    o[(axis + 2) % 3] = 2.f * u01(key, 3) - 1.f;
    o[axis] = (face & 1) ? 1.f : -1.f;
    const float tx = 1.8f * u01(key, 4) - 0.9f;
    const float ty = 1.8f * u01(key, 5) - 0.9f;
    const float tz = 1.8f * u01(key, 6) - 0.9f;
    ox = o[0];
    oy = o[1];
    oz = o[2];
    dx = tx - ox;
    dy = ty - oy;
    dz = tz - oz;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
  }
  r.p[0][i] = ox;
  r.p[1][i] = oy;
  r.p[2][i] = oz;
  r.p[3][i] = dx;
  r.p[4][i] = dy;
  r.p[5][i] = dz;
}

// Rays i >= first that hit move forward by s = u t along themselves; their
// target becomes t - s (the first hit along the same line is unchanged).
__global__ void shift_rays_kernel(RayOut r, float* __restrict__ t, const uint8_t* __restrict__ hit,
                                  int64_t n, int64_t first, uint64_t seed, uint64_t step) {
  const int64_t i = first + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || hit[i] == 0) return;
  const float ti = t[i];
  if (!(ti < 1e30f)) return;
  const float s = u01(ray_key(seed, step, i), 7) * ti;
  r.p[0][i] += s * r.p[3][i];
  r.p[1][i] += s * r.p[4][i];
  r.p[2][i] += s * r.p[5][i];
  t[i] = ti - s;
}

// Batch row i copies pool row floor(u n_pool), u = 32 bits of draw 8 of
// (seed, step, i) (draw 7 is the shift's).
__global__ void pool_gather_kernel(RaySoA pool, const float* __restrict__ pool_t,
                                   const uint8_t* __restrict__ pool_hit, int64_t n_pool,
                                   uint64_t seed, uint64_t step, int64_t n, RayOut r,
                                   float* __restrict__ t, uint8_t* __restrict__ hit) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t u = sm64(ray_key(seed, step, i) + 8) >> 32;
  const int64_t j = static_cast<int64_t>((u * static_cast<uint64_t>(n_pool)) >> 32);
  for (int c = 0; c < 6; ++c) r.p[c][i] = pool.p[c][j];
  t[i] = pool_t[j];
  hit[i] = pool_hit[j];
}

// Moves ray i's origin forward to where it enters the box [-h, h]^3 (slab
// test; unchanged when it starts inside or misses the box), stores that
// distance in t_in[i] and subtracts it from a finite t[i] (not below 0).
__global__ void enter_box_kernel(RayOut r, float* __restrict__ t, float* __restrict__ t_in,
                                 int64_t n, float h) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float o[3] = {r.p[0][i], r.p[1][i], r.p[2][i]};
  const float d[3] = {r.p[3][i], r.p[4][i], r.p[5][i]};
  float tn = 0.f, tf = __int_as_float(0x7f800000);
  bool miss = false;
  for (int k = 0; k < 3; ++k) {
    if (d[k] != 0.f) {
      const float a = (-h - o[k]) / d[k], b = (h - o[k]) / d[k];
      tn = fmaxf(tn, fminf(a, b));
      tf = fminf(tf, fmaxf(a, b));
    } else if (o[k] < -h || o[k] > h) {
      miss = true;
    }
  }
  const float e = (!miss && tn <= tf) ? tn : 0.f;
  if (e > 0.f)
    for (int k = 0; k < 3; ++k) r.p[k][i] = o[k] + e * d[k];
  if (t != nullptr) {
    const float ti = t[i];
    if (ti < __int_as_float(0x7f800000)) t[i] = fmaxf(ti - e, 0.f);
  }
  if (t_in != nullptr) t_in[i] = e;
}

}  // namespace

cudaError_t launch_enter_box(RayOut r, float* t, float* t_in, int64_t n, float h, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  enter_box_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(r, t, t_in, n, h);
  return cudaGetLastError();
}

cudaError_t launch_pool_gather(RaySoA pool, const float* pool_t, const uint8_t* pool_hit,
                               int64_t n_pool, uint64_t seed, uint64_t step, int64_t n,
                               RayOut r, float* t, uint8_t* hit, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pool_gather_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      pool, pool_t, pool_hit, n_pool, seed, step, n, r, t, hit);
  return cudaGetLastError();
}

cudaError_t launch_sample_rays(const float* spheres, int ns, const float* boxes, int nb,
                               uint64_t seed, uint64_t step, int64_t n, float surface_frac,
                               RayOut r, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (ns < 0 || nb < 0 || ns > kMaxPrims || nb > kMaxPrims) return cudaErrorInvalidValue;
  sample_rays_kernel<<<static_cast<unsigned>((n + kSampleThreads - 1) / kSampleThreads),
                       kSampleThreads, 0, s>>>(spheres, ns, boxes, nb, seed, step, n,
                                               surface_frac, r);
  return cudaGetLastError();
}

cudaError_t launch_shift_rays(RayOut r, float* t, const uint8_t* hit, int64_t n, int64_t first,
                              uint64_t seed, uint64_t step, cudaStream_t s) {
  if (first >= n) return cudaSuccess;
  const int64_t m = n - first;
  shift_rays_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(r, t, hit, n, first,
                                                                            seed, step);
  return cudaGetLastError();
}

}  // namespace ddf
