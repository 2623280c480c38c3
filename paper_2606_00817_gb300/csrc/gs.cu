// gs.cu -- depth rendered from 3D Gaussians, the cheap supervision source the
// paper compares with clean distances (Sec. 3.2; the study of Sec. 4.2), as a
// tile rasteriser: project every Gaussian (EWA: screen covariance J V C V^T
// J^T plus a 0.3-pixel low-pass), bin it into the 16 x 16-pixel tiles its
// alpha >= 1/255 ellipse touches, then per tile sort the list by depth in
// shared memory and composite front to back, one pixel per thread:
//   alpha = min(0.99, o exp(-q / 2)),  q = dp^T S^-1 dp,
//   D += T alpha z,  A += T alpha,  T *= 1 - alpha  (stop once T < 1e-4),
// giving per pixel the expected distance t = (D / A) / (d . f) along the
// pixel ray and the hit flag A > 0.5. Many views render in one launch each.
//
// Lists: per (view, tile) counts by atomics, one exclusive scan, then a fill
// pass that writes 64-bit keys (depth bits << 32 | Gaussian index) at atomic
// cursors. The order inside a list is arbitrary; the sort by key makes the
// result independent of it (equal depths: lower index first).
#include <cstdint>

#include "kernels.h"

namespace ddf {

namespace {

constexpr int kTile = 16;
constexpr int kTilePx = kTile * kTile;  // threads per render block, one pixel each
constexpr int kCap = 2048;              // keys composited per pass of a tile
constexpr float kLowPass = 0.3f;
constexpr float kAlphaMin = 1.f / 255.f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kNear = 0.05f;

__device__ __forceinline__ float dot3(const float* a, const float* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Per (view, Gaussian): the screen record and the rectangle of tiles it
// touches; adds 1 to the count of every tile in it.
__global__ void gs_project_kernel(const float* __restrict__ means, const float* __restrict__ covs,
                                  const float* __restrict__ opac, int64_t n,
                                  const GiCamera* __restrict__ cams, int nv, int ntx, int nty,
                                  float4* __restrict__ rec, int4* __restrict__ rect,
                                  unsigned* __restrict__ count) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n * nv) return;
  const int v = static_cast<int>(j / n);
  const int64_t g = j - static_cast<int64_t>(v) * n;
  const GiCamera& c = cams[v];
  rect[j] = make_int4(0, 0, -1, -1);
  const float m[3] = {means[3 * g] - c.eye[0], means[3 * g + 1] - c.eye[1],
                      means[3 * g + 2] - c.eye[2]};
  const float x = dot3(m, c.r), y = dot3(m, c.u), z = dot3(m, c.f);
  const float o = opac[g];
  if (!(z > kNear) || !(o >= kAlphaMin)) return;
  // square pixels: the focal length in pixels is height / (2 tan(fov_y / 2))
  const float fp = static_cast<float>(c.height) / (2.f * c.tan_half);
  const float iz = 1.f / z;
  const float px = x * iz * fp + 0.5f * static_cast<float>(c.width - 1);
  const float py = -y * iz * fp + 0.5f * static_cast<float>(c.height - 1);
  // rows of J V: d(px)/d(world) and d(py)/d(world)
  float a[3], b[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = fp * iz * (c.r[k] - x * iz * c.f[k]);
    b[k] = -fp * iz * (c.u[k] - y * iz * c.f[k]);
  }
  const float* C = covs + 6 * g;  // xx, xy, xz, yy, yz, zz
  float ca[3], cb[3];
  ca[0] = C[0] * a[0] + C[1] * a[1] + C[2] * a[2];
  ca[1] = C[1] * a[0] + C[3] * a[1] + C[4] * a[2];
  ca[2] = C[2] * a[0] + C[4] * a[1] + C[5] * a[2];
  cb[0] = C[0] * b[0] + C[1] * b[1] + C[2] * b[2];
  cb[1] = C[1] * b[0] + C[3] * b[1] + C[4] * b[2];
  cb[2] = C[2] * b[0] + C[4] * b[1] + C[5] * b[2];
  const float sxx = dot3(a, ca) + kLowPass;
  const float sxy = dot3(a, cb);
  const float syy = dot3(b, cb) + kLowPass;
  const float det = sxx * syy - sxy * sxy;
  if (!(det > 0.f)) return;
  const float id = 1.f / det;
  // alpha >= 1/255 needs q <= 2 ln(255 o): the ellipse's bounding box, one
  // pixel wider on each side for rounding
  const float kq = 2.f * logf(255.f * o);
  const float hx = sqrtf(fmaxf(kq, 0.f) * sxx) + 1.f;
  const float hy = sqrtf(fmaxf(kq, 0.f) * syy) + 1.f;
  const float fx0 = fmaxf(ceilf(px - hx), 0.f), fx1 = fminf(floorf(px + hx), c.width - 1.f);
  const float fy0 = fmaxf(ceilf(py - hy), 0.f), fy1 = fminf(floorf(py + hy), c.height - 1.f);
  if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;
  const int tx0 = static_cast<int>(fx0) / kTile, tx1 = static_cast<int>(fx1) / kTile;
  const int ty0 = static_cast<int>(fy0) / kTile, ty1 = static_cast<int>(fy1) / kTile;
  rec[2 * j] = make_float4(px, py, z, o);
  rec[2 * j + 1] = make_float4(syy * id, -sxy * id, sxx * id, 0.f);
  rect[j] = make_int4(tx0, ty0, tx1, ty1);
  unsigned* cv = count + static_cast<int64_t>(v) * ntx * nty;
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(cv + ty * ntx + tx, 1u);
}

// Exclusive scan of the tile counts (one block): off[i] = sum of count[< i],
// off[n] the total.
__global__ void gs_scan_kernel(const unsigned* __restrict__ count, int64_t n,
                               int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int64_t c = i < n ? static_cast<int64_t>(count[i]) : 0;
    part[threadIdx.x] = c;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // Hillis-Steele inclusive scan
      const int64_t add = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) off[i] = carry + part[threadIdx.x] - c;
    carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry;
}

// Writes each (view, Gaussian)'s key into the lists of its tiles.
__global__ void gs_fill_kernel(const float4* __restrict__ rec, const int4* __restrict__ rect,
                               int64_t n, int nv, int ntx, int nty,
                               const int64_t* __restrict__ off, unsigned* __restrict__ cursor,
                               unsigned long long* __restrict__ keys) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n * nv) return;
  const int4 rc = rect[j];
  if (rc.z < rc.x) return;
  const int v = static_cast<int>(j / n);
  const int64_t g = j - static_cast<int64_t>(v) * n;
  const unsigned long long key =
      (static_cast<unsigned long long>(__float_as_uint(rec[2 * j].z)) << 32) |
      static_cast<unsigned long long>(g);
  const int64_t tb = static_cast<int64_t>(v) * ntx * nty;
  for (int ty = rc.y; ty <= rc.w; ++ty)
    for (int tx = rc.x; tx <= rc.z; ++tx) {
      const int64_t t = tb + ty * ntx + tx;
      keys[off[t] + atomicAdd(cursor + t, 1u)] = key;
    }
}

// Ascending bitonic sort of s[0, p2), p2 a power of two; all threads call it.
__device__ void bitonic_sort(unsigned long long* s, int p2) {
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = s[i], b = s[l];
          if ((a > b) == ((i & k) == 0)) {
            s[i] = b;
            s[l] = a;
          }
        }
      }
      __syncthreads();
    }
}

// One block per (view, tile), one thread per pixel. A list longer than kCap
// is composited in passes: each pass keeps the kCap smallest keys not yet
// composited (merging the list chunk by chunk into a sorted window).
__global__ void __launch_bounds__(kTilePx)
gs_render_kernel(const float4* __restrict__ rec, int64_t n, const GiCamera* __restrict__ cams,
                 int ntx, int nty, const int64_t* __restrict__ off,
                 const unsigned long long* __restrict__ keys, float* __restrict__ out_t,
                 uint8_t* __restrict__ out_hit) {
  __shared__ unsigned long long s_key[2 * kCap];
  __shared__ float4 s_a[kTilePx], s_b[kTilePx];
  __shared__ int s_valid;
  const int ntiles = ntx * nty;
  const int tile = blockIdx.x;
  const int v = tile / ntiles;
  const int tt = tile - v * ntiles;
  const int tx = tt % ntx, ty = tt / ntx;
  const GiCamera& c = cams[v];
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.width && py < c.height;
  const float fx = static_cast<float>(px), fy = static_cast<float>(py);
  const int64_t beg = off[tile];
  const int64_t cnt = off[tile + 1] - beg;
  const float4* rv = rec + 2 * static_cast<int64_t>(v) * n;
  constexpr unsigned long long kEnd = ~0ull;
  float T = 1.f, D = 0.f, A = 0.f;
  bool done = !inside;
  unsigned long long lo = 0;
  bool finished = cnt == 0;
  while (!finished) {
    int wn = 0;
    int64_t valid_total = 0;
    for (int64_t base = 0; base < cnt; base += kCap) {
      const int m = static_cast<int>(cnt - base < kCap ? cnt - base : kCap);
      if (threadIdx.x == 0) s_valid = 0;
      __syncthreads();
      int mine = 0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const unsigned long long k = keys[beg + base + i];
        const bool keep = k >= lo;
        s_key[wn + i] = keep ? k : kEnd;
        mine += keep;
      }
      int p2 = 1;
      while (p2 < wn + m) p2 <<= 1;
      for (int i = wn + m + threadIdx.x; i < p2; i += blockDim.x) s_key[i] = kEnd;
      if (mine) atomicAdd(&s_valid, mine);
      __syncthreads();
      bitonic_sort(s_key, p2);
      const int got = s_valid;
      valid_total += got;
      wn = wn + got < kCap ? wn + got : kCap;
      __syncthreads();  // s_valid is rewritten by the next chunk
    }
    // composite the window front to back
    bool all_done = false;
    for (int i0 = 0; i0 < wn; i0 += kTilePx) {
      const int i = i0 + threadIdx.x;
      if (i < wn) {
        const int64_t g = static_cast<int64_t>(s_key[i] & 0xffffffffull);
        s_a[threadIdx.x] = rv[2 * g];
        s_b[threadIdx.x] = rv[2 * g + 1];
      }
      __syncthreads();
      const int nb = wn - i0 < kTilePx ? wn - i0 : kTilePx;
      if (!done) {
        for (int jj = 0; jj < nb; ++jj) {
          const float4 a = s_a[jj], b = s_b[jj];
          const float dx = fx - a.x, dy = fy - a.y;
          const float q = b.x * dx * dx + 2.f * b.y * dx * dy + b.z * dy * dy;
          const float alpha = fminf(kAlphaMax, a.w * expf(-0.5f * q));
          if (!(alpha >= kAlphaMin)) continue;
          const float w = T * alpha;
          D += w * a.z;
          A += w;
          T *= 1.f - alpha;
          if (T < kTMin) {
            done = true;
            break;
          }
        }
      }
      all_done = __syncthreads_count(!done) == 0;  // also orders the next loads
      if (all_done) break;
    }
    if (all_done || valid_total <= kCap) break;
    lo = s_key[kCap - 1] + 1;
    __syncthreads();  // everyone has read s_key before the next pass rewrites it
  }
  if (!inside) return;
  const float sx = (2.f * (fx + 0.5f) / c.width - 1.f) * c.tan_half *
                   (static_cast<float>(c.width) / c.height);
  const float sy = (1.f - 2.f * (fy + 0.5f) / c.height) * c.tan_half;
  const int64_t o = static_cast<int64_t>(v) * c.width * c.height +
                    static_cast<int64_t>(py) * c.width + px;
  out_t[o] = A > 0.f ? D / A * sqrtf(1.f + sx * sx + sy * sy) : __int_as_float(0x7f800000);
  out_hit[o] = A > 0.5f ? 1 : 0;
}

// Pixel-centre rays of each view (same model as the shadow / AO images).
__global__ void camera_rays_kernel(const GiCamera* __restrict__ cams, int nv, int64_t npx,
                                   RayOut r) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= npx * nv) return;
  const int v = static_cast<int>(j / npx);
  const GiCamera& c = cams[v];
  const int64_t i = j - static_cast<int64_t>(v) * npx;
  const int x = static_cast<int>(i % c.width), y = static_cast<int>(i / c.width);
  const float sx = (2.f * (static_cast<float>(x) + 0.5f) / c.width - 1.f) * c.tan_half *
                   (static_cast<float>(c.width) / c.height);
  const float sy = (1.f - 2.f * (static_cast<float>(y) + 0.5f) / c.height) * c.tan_half;
  float d[3];
  for (int k = 0; k < 3; ++k) d[k] = c.f[k] + sx * c.r[k] + sy * c.u[k];
  const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) {
    r.p[k][j] = c.eye[k];
    r.p[3 + k][j] = d[k] * inv;
  }
}

}  // namespace

int gs_tiles(int extent) { return (extent + kTile - 1) / kTile; }

cudaError_t launch_gs_project(const float* means, const float* covs, const float* opac, int64_t n,
                              const GiCamera* cams, int nv, int ntx, int nty, float4* rec,
                              int4* rect, unsigned* count, cudaStream_t s) {
  const int64_t m = n * nv;
  if (m <= 0) return cudaSuccess;
  gs_project_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(
      means, covs, opac, n, cams, nv, ntx, nty, rec, rect, count);
  return cudaGetLastError();
}

cudaError_t launch_gs_scan(const unsigned* count, int64_t n, int64_t* off, cudaStream_t s) {
  gs_scan_kernel<<<1, 1024, 0, s>>>(count, n, off);
  return cudaGetLastError();
}

cudaError_t launch_gs_fill(const float4* rec, const int4* rect, int64_t n, int nv, int ntx,
                           int nty, const int64_t* off, unsigned* cursor,
                           unsigned long long* keys, cudaStream_t s) {
  const int64_t m = n * nv;
  if (m <= 0) return cudaSuccess;
  gs_fill_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(rec, rect, n, nv, ntx,
                                                                         nty, off, cursor, keys);
  return cudaGetLastError();
}

cudaError_t launch_gs_render(const float4* rec, int64_t n, const GiCamera* cams, int nv, int ntx,
                             int nty, const int64_t* off, const unsigned long long* keys,
                             float* out_t, uint8_t* out_hit, cudaStream_t s) {
  const int64_t blocks = static_cast<int64_t>(nv) * ntx * nty;
  if (blocks <= 0) return cudaSuccess;
  gs_render_kernel<<<static_cast<unsigned>(blocks), kTilePx, 0, s>>>(rec, n, cams, ntx, nty, off,
                                                                     keys, out_t, out_hit);
  return cudaGetLastError();
}

cudaError_t launch_camera_rays(const GiCamera* cams, int nv, int64_t npx, RayOut r,
                               cudaStream_t s) {
  const int64_t m = npx * nv;
  if (m <= 0) return cudaSuccess;
  camera_rays_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(cams, nv, npx, r);
  return cudaGetLastError();
}

}  // namespace ddf
