// gs_api.cpp -- C entry points of the Gaussian-rendered depth (Sec. 3.2 /
// 4.2) and of pinhole camera rays: argument checks, the camera bases,
// workspace, and the launch sequence of gs.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "ddf.h"
#include "handle.h"
#include "kernels.h"

using namespace ddfi;

namespace {

ddf_status make_cameras(const float* cameras, int32_t n_views, int32_t width, int32_t height,
                        std::vector<ddf::GiCamera>* out) {
  if (cameras == nullptr) return fail(DDF_ERR_INVALID_ARG, "cameras is NULL");
  if (n_views < 1) return fail(DDF_ERR_INVALID_ARG, "n_views must be >= 1");
  if (width < 1 || height < 1 ||
      static_cast<int64_t>(width) * height * n_views > (int64_t{1} << 31))
    return fail(DDF_ERR_INVALID_ARG, "width, height >= 1 and at most 2^31 pixels over all views");
  out->resize(n_views);
  for (int v = 0; v < n_views; ++v) {
    const ddf_status s = camera_basis(cameras + 10 * v, width, height, &(*out)[v]);
    if (s != DDF_OK) return s;
  }
  return DDF_OK;
}

}  // namespace

extern "C" {

ddf_status ddf_render_gs_depth(const float* means, const float* covs, const float* opacities,
                               int64_t n, const float* cameras, int32_t n_views, int32_t width,
                               int32_t height, float* out_t, uint8_t* out_hit, void* stream) {
  if (n < 0 || n > (int64_t{1} << 31))
    return fail(DDF_ERR_INVALID_ARG, "n must be in [0, 2^31]");
  if (n > 0 && (means == nullptr || covs == nullptr || opacities == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "Gaussian arrays are NULL");
  if (out_t == nullptr || out_hit == nullptr) return fail(DDF_ERR_INVALID_ARG, "outputs are NULL");
  DDF_REQUIRE_ALIGNED(means, 4);
  DDF_REQUIRE_ALIGNED(covs, 4);
  DDF_REQUIRE_ALIGNED(opacities, 4);
  DDF_REQUIRE_ALIGNED(out_t, 4);
  std::vector<ddf::GiCamera> cams;
  ddf_status s = make_cameras(cameras, n_views, width, height, &cams);
  if (s != DDF_OK) return s;
  if (n * n_views > (int64_t{1} << 40)) return fail(DDF_ERR_INVALID_ARG, "n x n_views too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ntx = ddf::gs_tiles(width), nty = ddf::gs_tiles(height);
  const int64_t nt = static_cast<int64_t>(n_views) * ntx * nty;
  const int64_t m = n * n_views;
  // cameras, records, rectangles, counts, cursors, offsets
  const size_t cam_b = round_up(n_views * sizeof(ddf::GiCamera), 256);
  const size_t rec_b = m * 2 * sizeof(float4), rect_b = m * sizeof(int4);
  const size_t cnt_b = round_up(nt * sizeof(unsigned), 256);
  const size_t bytes = cam_b + rec_b + rect_b + 2 * cnt_b + (nt + 1) * sizeof(int64_t);
  uint8_t* buf = nullptr;
  DDF_CK(cudaMalloc(&buf, bytes));
  auto* dcam = reinterpret_cast<ddf::GiCamera*>(buf);
  auto* rec = reinterpret_cast<float4*>(buf + cam_b);
  auto* rect = reinterpret_cast<int4*>(buf + cam_b + rec_b);
  auto* count = reinterpret_cast<unsigned*>(buf + cam_b + rec_b + rect_b);
  auto* cursor = reinterpret_cast<unsigned*>(buf + cam_b + rec_b + rect_b + cnt_b);
  auto* off = reinterpret_cast<int64_t*>(buf + cam_b + rec_b + rect_b + 2 * cnt_b);
  unsigned long long* keys = nullptr;
  int64_t total = 0;
  cudaError_t e = cudaMemcpyAsync(dcam, cams.data(), n_views * sizeof(ddf::GiCamera),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, 2 * cnt_b, st);
  if (e == cudaSuccess)
    e = ddf::launch_gs_project(means, covs, opacities, n, dcam, n_views, ntx, nty, rec, rect,
                               count, st);
  if (e == cudaSuccess) e = ddf::launch_gs_scan(count, nt, off, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, off + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && total > 0) e = cudaMalloc(&keys, total * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = ddf::launch_gs_fill(rec, rect, n, n_views, ntx, nty, off, cursor, keys, st);
  if (e == cudaSuccess)
    e = ddf::launch_gs_render(rec, n, dcam, n_views, ntx, nty, off, keys, out_t, out_hit, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  cudaFree(keys);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "Gaussian depth render");
  return DDF_OK;
}

ddf_status ddf_camera_rays(const float* cameras, int32_t n_views, int32_t width, int32_t height,
                           float* const rays_out[6], void* stream) {
  if (rays_out == nullptr) return fail(DDF_ERR_INVALID_ARG, "rays_out is NULL");
  for (int c = 0; c < 6; ++c) {
    if (rays_out[c] == nullptr) return fail(DDF_ERR_INVALID_ARG, "a ray array is NULL");
    DDF_REQUIRE_ALIGNED(rays_out[c], 4);
  }
  std::vector<ddf::GiCamera> cams;
  ddf_status s = make_cameras(cameras, n_views, width, height, &cams);
  if (s != DDF_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ddf::GiCamera* dcam = nullptr;
  DDF_CK(cudaMalloc(&dcam, n_views * sizeof(ddf::GiCamera)));
  ddf::RayOut r;
  for (int c = 0; c < 6; ++c) r.p[c] = rays_out[c];
  cudaError_t e = cudaMemcpyAsync(dcam, cams.data(), n_views * sizeof(ddf::GiCamera),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = ddf::launch_camera_rays(dcam, n_views, static_cast<int64_t>(width) * height, r, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  cudaFree(dcam);
  if (e != cudaSuccess) return cuda_fail(e, "camera rays");
  return DDF_OK;
}

ddf_status ddf_enter_box(float* const rays[6], float* t, float* out_t_in, int64_t n,
                         float half_extent, void* stream) {
  if (rays == nullptr) return fail(DDF_ERR_INVALID_ARG, "rays is NULL");
  if (n < 0) return fail(DDF_ERR_INVALID_ARG, "n must be >= 0");
  if (!(half_extent > 0.f) || !std::isfinite(half_extent))
    return fail(DDF_ERR_INVALID_ARG, "half_extent must be finite and > 0");
  ddf::RayOut r;
  for (int c = 0; c < 6; ++c) {
    if (rays[c] == nullptr && n > 0) return fail(DDF_ERR_INVALID_ARG, "a ray array is NULL");
    DDF_REQUIRE_ALIGNED(rays[c], 4);
    r.p[c] = rays[c];
  }
  DDF_REQUIRE_ALIGNED(t, 4);
  DDF_REQUIRE_ALIGNED(out_t_in, 4);
  const cudaError_t e =
      ddf::launch_enter_box(r, t, out_t_in, n, half_extent, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "enter box");
  return DDF_OK;
}

}  // extern "C"
