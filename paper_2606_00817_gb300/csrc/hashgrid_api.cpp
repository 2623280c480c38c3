// hashgrid_api.cpp -- host side of the hash-grid field (kind
// DDF_KIND_HASHGRID), the paper's final DDF (Sec. 3.4): the level layout of
// the multiresolution hash grid, weight loading (bf16 or FP32 level tables,
// swizzled MLP operand images), the query launch, and training (FP32
// forward and backward, the table gradient's scatter, every weight and bias
// sum in one reduction launch, Adam, the bf16 refresh). The public entry
// points (ddf_create, ddf_load_weights, the ray queries, the training calls)
// dispatch here by kind.
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

// Writes the query copies of a bf16 field (padded bf16 table, swizzled MLP
// operand images, FP32 biases and head) from the FP32 master blob, on st;
// with tables = false only those of the MLP (the training step's Adam pass
// writes the table's copy itself).
ddf_status hg_refresh(ddf_s* h, cudaStream_t st, bool tables_too) {
  const int H = h->cfg.hidden_layers;
  const float* tables = h->d_blob;
  uint32_t* tab = static_cast<uint32_t*>(h->hg_table);
  // every level into the padded layout, one launch
  if (tables_too)
    DDF_CK(ddf::launch_hg_pack_table(tables, h->hg_blob_entries, h->hg_blob, h->hg, tab, st));
  // MLP part: W_1 [64 x 59], b_1, (W_l [64 x 64], b_l) ..., W_o [2 x 64], b_o
  const float* m = tables + 2 * h->hg_blob_entries;
  int K = kCode;
  for (int l = 0; l < H; ++l) {
    DDF_CK(ddf::launch_hg_pack_image(m, K, h->hg_img + static_cast<size_t>(l) * kW * 128, st));
    DDF_CK(cudaMemcpyAsync(h->hg_bias + l * kW, m + kW * K, kW * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
    m += kW * K + kW;
    K = kW;
  }
  DDF_CK(cudaMemcpyAsync(h->hg_bias + H * kW, m, (2 * kW + 2) * sizeof(float),
                         cudaMemcpyDeviceToDevice, st));  // head rows then head bias
  return DDF_OK;
}

ddf_status hg_load(ddf_s* h, const float* host_blob) {
  const ddf_config& c = h->cfg;
  const int H = c.hidden_layers;
  const bool f32 = c.precision == DDF_FP32;
  const size_t need = hg_param_count(c);
  ddf_status s;
  void* p = nullptr;
  auto alloc_buffers = [&]() -> ddf_status {
    // the FP32 path reads the blob's tables in place; the bf16 table starts
    // every level on an even entry (8-byte corner pairs)
    h->hg = hg_layout(&h->hg_entries, !f32);
    h->hg_blob = hg_layout(&h->hg_blob_entries, false);
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
    return DDF_OK;
  };
  if (h->d_blob == nullptr && (s = alloc_buffers()) != DDF_OK) {
    // a failure half way frees everything: the next load starts from nothing
    for (void** q : {reinterpret_cast<void**>(&h->d_blob), &h->hg_table,
                     reinterpret_cast<void**>(&h->hg_img), reinterpret_cast<void**>(&h->hg_bias)}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    return s;
  }
  DDF_CK(cudaMemcpy(h->d_blob, host_blob, need * sizeof(float), cudaMemcpyHostToDevice));
  if (!f32 && (s = hg_refresh(h, nullptr)) != DDF_OK) return s;
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

// ------------------------------------------------------------ training

namespace {

constexpr int kGradSplits = 128;  // ray splits of the weight-gradient sums

struct MlpOffsets {
  int64_t w[4], b[4], wo, bo;
};

MlpOffsets mlp_offsets(int H) {
  MlpOffsets o{};
  int64_t off = 0;
  for (int l = 0; l < H; ++l) {
    const int K = l == 0 ? kCode : kW;
    o.w[l] = off;
    off += static_cast<int64_t>(kW) * K;
    o.b[l] = off;
    off += kW;
  }
  o.wo = off;
  o.bo = off + 2 * kW;
  return o;
}

}  // namespace

ddf_status hg_ensure_train(ddf_s* h, int64_t B) {
  const int H = h->cfg.hidden_layers;
  const size_t np = hg_param_count(h->cfg);
  ddf_status s;
  void* p = nullptr;
  auto alloc_state = [&]() -> ddf_status {
    for (float** q : {&h->grad, &h->adam_m, &h->adam_v}) {
      if ((s = dev_alloc(h, &p, np * sizeof(float))) != DDF_OK) return s;
      *q = static_cast<float*>(p);
    }
    DDF_CK(cudaMemset(h->adam_m, 0, np * sizeof(float)));
    DDF_CK(cudaMemset(h->adam_v, 0, np * sizeof(float)));
    h->adam_step = 0;
    // one slice of partials per weight matrix (H layers and the head), so
    // that every sum runs in one launch after the last outer product
    const size_t slices = static_cast<size_t>(H) + 1;
    if ((s = dev_alloc(h, &p, slices * kGradSplits * kW * kW * sizeof(float))) != DDF_OK) return s;
    h->tr_part = static_cast<float*>(p);
    if ((s = dev_alloc(h, &p, slices * kGradSplits * kW * sizeof(float))) != DDF_OK) return s;
    h->tr_cpart = static_cast<float*>(p);
    if ((s = dev_alloc(h, &p, sizeof(unsigned))) != DDF_OK) return s;
    h->tr_nhit = static_cast<unsigned*>(p);
    return DDF_OK;
  };
  if (h->grad == nullptr && (s = alloc_state()) != DDF_OK) {
    // a failure half way frees everything: the next call starts from nothing
    for (float** q : {&h->grad, &h->adam_m, &h->adam_v, &h->tr_part, &h->tr_cpart}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    dev_free(h, h->tr_nhit);
    h->tr_nhit = nullptr;
    return s;
  }
  if (B > h->tr_rows) {
    h->fwd_rows = 0;
    for (void** q : {reinterpret_cast<void**>(&h->hg_code), reinterpret_cast<void**>(&h->hg_acts),
                     reinterpret_cast<void**>(&h->hg_dpre), reinterpret_cast<void**>(&h->tr_z),
                     reinterpret_cast<void**>(&h->tr_dz), reinterpret_cast<void**>(&h->tr_lpart)}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    h->tr_rows = 0;
    const size_t rows = static_cast<size_t>(B);
    if ((s = dev_alloc(h, &p, rows * kW * sizeof(float))) != DDF_OK) return s;
    h->hg_code = static_cast<float*>(p);
    if ((s = dev_alloc(h, &p, static_cast<size_t>(H) * rows * kW * sizeof(float))) != DDF_OK) return s;
    h->hg_acts = static_cast<float*>(p);
    if ((s = dev_alloc(h, &p, static_cast<size_t>(H) * rows * kW * sizeof(float))) != DDF_OK) return s;
    h->hg_dpre = static_cast<float*>(p);
    if ((s = dev_alloc(h, &p, rows * sizeof(float2))) != DDF_OK) return s;
    h->tr_z = static_cast<float2*>(p);
    if ((s = dev_alloc(h, &p, rows * sizeof(float2))) != DDF_OK) return s;
    h->tr_dz = static_cast<float2*>(p);
    if ((s = dev_alloc(h, &p, ((rows + 255) / 256) * sizeof(float))) != DDF_OK) return s;
    h->tr_lpart = static_cast<float*>(p);
    h->tr_rows = B;
  }
  return DDF_OK;
}

ddf_status hg_forward_keep(ddf_s* h, ddf::RaySoA rays, int B, cudaStream_t st) {
  const float2* table = static_cast<const float2*>(static_cast<void*>(h->d_blob));
  DDF_CK(ddf::launch_hg_train_fwd(h->hg_blob, table, h->d_blob + 2 * h->hg_blob_entries,
                                  h->cfg.hidden_layers, rays, B, h->hg_code, h->hg_acts, h->tr_z,
                                  st));
  return DDF_OK;
}

ddf_status hg_backward(ddf_s* h, ddf::RaySoA rays, int B, cudaStream_t st) {
  const int H = h->cfg.hidden_layers;
  const int64_t tab = 2 * h->hg_blob_entries;
  const float* mlp = h->d_blob + tab;
  float* gmlp = h->grad + tab;
  const MlpOffsets o = mlp_offsets(H);
  const int64_t act = static_cast<int64_t>(B) * kW;
  // the table gradient is a sum of scattered contributions: start from zero
  DDF_CK(cudaMemsetAsync(h->grad, 0, tab * sizeof(float), st));
  DDF_CK(ddf::launch_hg_train_bwd(h->hg_blob, mlp, H, rays, B, h->hg_acts, h->tr_dz, h->hg_dpre,
                                  h->grad, st));
  // the split partials of weight matrix l go to slice l; the weight and bias
  // sums of all of them follow in launches of up to kRedJobs sums
  const size_t pslice = static_cast<size_t>(kGradSplits) * kW * kW;
  const size_t cslice = static_cast<size_t>(kGradSplits) * kW;
  std::vector<ddf::RedSplit> sums;
  auto add_sum = [&](const float* part, int rows, int cols, float* out) {
    ddf::RedSplit a;
    a.part = part;
    a.split_stride = static_cast<int64_t>(rows) * cols;
    a.S = kGradSplits;
    a.rows = rows;
    a.cols = cols;
    a.ldp = cols;
    a.ldo = cols;
    a.out = out;
    sums.push_back(a);
  };
  ddf::HgOuterJobs jobs{};
  for (int l = 0; l < H; ++l) {
    const float* P = h->hg_dpre + l * act;
    const float* A = l == 0 ? h->hg_code : h->hg_acts + (l - 1) * act;
    const int K = l == 0 ? kCode : kW;
    float* part = h->tr_part + l * pslice;
    float* cpart = h->tr_cpart + l * cslice;
    jobs.job[jobs.n++] = ddf::HgOuterJob{P, 1, B, kW, A, 1, B, K, part, cpart};
    add_sum(part, kW, K, gmlp + o.w[l]);
    add_sum(cpart, 1, kW, gmlp + o.b[l]);
  }
  const float* dz = reinterpret_cast<const float*>(h->tr_dz);
  float* part = h->tr_part + H * pslice;
  float* cpart = h->tr_cpart + H * cslice;
  jobs.job[jobs.n++] = ddf::HgOuterJob{dz, 2, 1, 2, h->hg_acts + (H - 1) * act, 1, B, kW, part, cpart};
  DDF_CK(ddf::launch_hg_outer_tiled(jobs, B, kGradSplits, st));  // every layer, one launch
  add_sum(part, 2, kW, gmlp + o.wo);
  add_sum(cpart, 1, 2, gmlp + o.bo);
  for (size_t j0 = 0; j0 < sums.size(); j0 += ddf::kRedJobs) {
    ddf::GradReduce g;
    g.nsplit = static_cast<int>(std::min<size_t>(ddf::kRedJobs, sums.size() - j0));
    for (int j = 0; j < g.nsplit; ++j) g.split[j] = sums[j0 + j];
    DDF_CK(ddf::launch_grad_reduce(g, st));
  }
  h->grad_valid = true;
  return DDF_OK;
}

ddf_status hg_train(ddf_s* h, ddf::RaySoA rays, const float* t_target, const uint8_t* hit_target,
                    int B, float lr, float* out_loss, cudaStream_t st) {
  ddf_status s;
  h->fwd_rows = 0;
  if ((s = hg_forward_keep(h, rays, B, st)) != DDF_OK) return s;
  DDF_CK(ddf::launch_loss(h->tr_z, t_target, hit_target, B, h->tr_nhit, kLossClamp, kLossLambda,
                          h->tr_dz, h->tr_lpart, out_loss, st));
  if ((s = hg_backward(h, rays, B, st)) != DDF_OK) return s;
  if (lr > 0.f) {
    ++h->adam_step;
    const double t = static_cast<double>(h->adam_step);
    const float bc1 = static_cast<float>(1.0 - std::pow(0.9, t));
    const float bc2 = static_cast<float>(1.0 - std::pow(0.999, t));
    const int64_t n = static_cast<int64_t>(hg_param_count(h->cfg));
    if (h->cfg.precision == DDF_FP32) {
      DDF_CK(ddf::launch_adam(h->d_blob, h->grad, h->adam_m, h->adam_v, n, lr, kAdamB1, kAdamB2,
                              kAdamEps, bc1, bc2, st));
    } else {
      // the tables' Adam and their bf16 copy in one pass, then the MLP's
      const int64_t t = 2 * h->hg_blob_entries;
      DDF_CK(ddf::launch_hg_adam_pack(h->d_blob, h->grad, h->adam_m, h->adam_v, h->hg_blob_entries,
                                      lr, kAdamB1, kAdamB2, kAdamEps, bc1, bc2, h->hg_blob, h->hg,
                                      static_cast<uint32_t*>(h->hg_table), st));
      DDF_CK(ddf::launch_adam(h->d_blob + t, h->grad + t, h->adam_m + t, h->adam_v + t, n - t, lr,
                              kAdamB1, kAdamB2, kAdamEps, bc1, bc2, st));
      if ((s = hg_refresh(h, st, false)) != DDF_OK) return s;
    }
  }
  return DDF_OK;
}

}  // namespace ddfi
