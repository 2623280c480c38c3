// hashgrid_api.cpp -- host side of the hash-grid field (kind
// DDF_KIND_HASHGRID), the paper's final DDF (Sec. 3.4): the level layout of
// the multiresolution hash grid, weight loading (bf16 or FP32 level tables,
// swizzled MLP operand images) and the query launch. The public entry points
// (ddf_create, ddf_load_weights, the ray queries) dispatch here by kind.
#include <algorithm>
#include <cmath>

#include "handle.h"
#include "kernels.h"

namespace ddfi {

namespace {

constexpr int kLevels = 16;
constexpr int kLog2T = 19;
constexpr int kBase = 16;  // cells per axis of level 0; level l has floor(16 * 1.5^l)
constexpr int kW = 64;
constexpr int kCode = 59;

size_t mlp_params(const ddf_config& c) {
  const size_t H = c.hidden_layers;
  return kW * kCode + kW + (H - 1) * (kW * kW + kW) + 2 * kW + 2;
}

}  // namespace

ddf::HashGridParams hg_layout(int64_t* entries, bool even_offsets) {
  ddf::HashGridParams g{};
  int64_t off = 0;
  int64_t pow3 = 1;  // 3^l
  for (int l = 0; l < kLevels; ++l) {
    // floor(16 * 1.5^l) = floor(16 * 3^l / 2^l), exact in integers
    const int64_t res = (kBase * pow3) >> l;
    pow3 *= 3;
    const int64_t verts = (res + 1) * (res + 1) * (res + 1);
    const int64_t size = std::min<int64_t>(int64_t{1} << kLog2T, verts);
    g.res[l] = static_cast<int>(res);
    g.dense[l] = verts <= (int64_t{1} << kLog2T) ? 1 : 0;
    g.offset[l] = static_cast<uint32_t>(off);
    off += size;
    if (even_offsets) off += off & 1;  // the next level starts on an 8-byte pair
  }
  g.mask = (1u << kLog2T) - 1u;
  if (entries != nullptr) *entries = off;
  return g;
}

size_t hg_param_count(const ddf_config& c) {
  int64_t entries = 0;
  hg_layout(&entries, false);
  return static_cast<size_t>(entries) * 2 + mlp_params(c);
}

ddf_status hg_load(ddf_s* h, const float* host_blob) {
  const ddf_config& c = h->cfg;
  const int H = c.hidden_layers;
  const bool f32 = c.precision == DDF_FP32;
  const size_t need = hg_param_count(c);
  ddf_status s;
  void* p = nullptr;
  if (h->d_blob == nullptr) {
    // the FP32 path reads the blob's tables in place; the bf16 table starts
    // every level on an even entry (8-byte corner pairs)
    h->hg = hg_layout(&h->hg_entries, !f32);
    if ((s = dev_alloc(h, &p, need * sizeof(float))) != DDF_OK) return s;
    h->d_blob = static_cast<float*>(p);
    if (!f32) {
      if ((s = dev_alloc(h, &p, static_cast<size_t>(h->hg_entries) * 4)) != DDF_OK) return s;
      h->hg_table = p;
      if ((s = dev_alloc(h, &p, static_cast<size_t>(H) * kW * 128)) != DDF_OK) return s;
      h->hg_img = static_cast<uint8_t*>(p);
      if ((s = dev_alloc(h, &p, (static_cast<size_t>(H) * kW + 2 * kW + 2) * sizeof(float))) !=
          DDF_OK)
        return s;
      h->hg_bias = static_cast<float*>(p);
      const int per_sm = ddf::hashgrid_tc_blocks_per_sm(H);
      if (per_sm <= 0) return fail(DDF_ERR_UNSUPPORTED, "the hash-grid kernel does not fit an SM");
      h->hg_grid = per_sm * h->num_sms;
    }
  }
  DDF_CK(cudaMemcpy(h->d_blob, host_blob, need * sizeof(float), cudaMemcpyHostToDevice));
  if (!f32) {
    cudaStream_t st = nullptr;
    const float* tables = h->d_blob;
    int64_t blob_entries = 0;
    const ddf::HashGridParams dense = hg_layout(&blob_entries, false);
    uint32_t* tab = static_cast<uint32_t*>(h->hg_table);
    for (int l = 0; l < kLevels; ++l) {  // level by level into the padded layout
      const int64_t end = l + 1 < kLevels ? dense.offset[l + 1] : blob_entries;
      DDF_CK(ddf::launch_hg_pack_table(tables + 2 * static_cast<int64_t>(dense.offset[l]),
                                       end - dense.offset[l], tab + h->hg.offset[l], st));
    }
    // MLP part: W_1 [64 x 59], b_1, (W_l [64 x 64], b_l) ..., W_o [2 x 64], b_o
    const float* m = tables + 2 * blob_entries;
    int K = kCode;
    for (int l = 0; l < H; ++l) {
      DDF_CK(ddf::launch_hg_pack_image(m, K, h->hg_img + static_cast<size_t>(l) * kW * 128, st));
      DDF_CK(cudaMemcpy(h->hg_bias + l * kW, m + kW * K, kW * sizeof(float),
                        cudaMemcpyDeviceToDevice));
      m += kW * K + kW;
      K = kW;
    }
    DDF_CK(cudaMemcpy(h->hg_bias + H * kW, m, (2 * kW + 2) * sizeof(float),
                      cudaMemcpyDeviceToDevice));  // head rows then head bias
  }
  DDF_CK(cudaDeviceSynchronize());
  return DDF_OK;
}

ddf_status hg_query(ddf_s* h, ddf::RaySoA rays, int64_t n, ddf::HeadOut out, cudaStream_t st) {
  if (n <= 0) return DDF_OK;
  const int H = h->cfg.hidden_layers;
  if (h->cfg.precision == DDF_FP32) {
    ProfScope ps(h, kProfGemm, st);
    DDF_CK(ddf::launch_hashgrid_f32(h->hg, static_cast<const float2*>(static_cast<void*>(h->d_blob)),
                                    h->d_blob + 2 * h->hg_entries, H, rays, n, out, st));  // unpadded
    return DDF_OK;
  }
  ProfScope ps(h, kProfGemm, st);
  const int64_t tiles = (n + 127) / 128;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, h->hg_grid));
  const float* vecs = h->hg_bias;
  DDF_CK(ddf::launch_hashgrid_tc(h->hg, static_cast<const uint32_t*>(h->hg_table), h->hg_img, vecs,
                                 vecs + H * kW, vecs + H * kW + 2 * kW, H, rays, n, out,
                                 h->status_dev, h->timeout_ns, grid, st));
  return DDF_OK;
}

}  // namespace ddfi
