// train_api.cpp -- C ABI of the distillation step (declared in include/ddf.h).
//
// One step of Sec. 3.2 / 3.4 on a bf16 handle: forward through the encoder
// and the tensor-core layers keeping every bf16 activation, the FP32 head,
// the clamped-L1 + 0.3 x cross-entropy loss and dL/dz, then back through the
// head and every layer:
//   dW_l = dpre_l^T A_l   (tensor cores, split-K over the batch, FP32 partials
//                          reduced in a fixed order)
//   db_l = column sums of dpre_l (from 32-row sums the input-gradient
//          epilogue leaves, reduced with dW_l in the same launch)
//   dpre_{l-1} = (dpre_l W_l) masked by h_{l-1} > 0   (tensor cores, bf16)
// and, for ddf_train_step, Adam on the FP32 master weights together with the
// refresh of the bf16 copies the queries use (one pass over the blob). The exact analytic ray caster
// that produces distillation targets lives here too (ddf_cast_scene).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "handle.h"
#include "kernels.h"

using namespace ddfi;

namespace {

constexpr int kColSplits = 64;   // row splits of the column sums
constexpr int kPartSplits = 16;  // most batch splits of a weight-gradient GEMM
constexpr int kHeadSplits = 512; // row splits of the head's fused backward
constexpr float kClamp = kLossClamp;
constexpr float kLambda = kLossLambda;
constexpr float kB1 = kAdamB1, kB2 = kAdamB2, kEps = kAdamEps;

// (t, vis) head rows of a ray field; one row (the distance) for an SDF field
size_t head_rows(const ddf_s* h) { return h->cfg.kind == DDF_KIND_SDF ? 1 : 2; }

struct BlobOffsets {
  std::vector<size_t> w, b;
  size_t wo = 0, bo = 0;
};

BlobOffsets blob_offsets(const ddf_s* h) {
  BlobOffsets o;
  const size_t W = h->cfg.width;
  size_t off = 0;
  for (int l = 0; l < h->cfg.hidden_layers; ++l) {
    const size_t K = l == 0 ? h->d_in : W;
    o.w.push_back(off);
    off += W * K;
    o.b.push_back(off);
    off += W;
  }
  o.wo = off;
  o.bo = off + head_rows(h) * W;
  return o;
}

size_t n_params(const ddf_s* h) {
  if (h->cfg.kind == DDF_KIND_HASHGRID) return hg_param_count(h->cfg);
  return blob_offsets(h).bo + head_rows(h);
}

bool is_hashgrid(const ddf_s* h) { return h->cfg.kind == DDF_KIND_HASHGRID; }

// Whether layer l's output is kept through the backward (activation
// checkpointing with segment k: the outputs of layers k-1, 2k-1, ... and of
// the last layer; every output when k <= 1).
bool kept_layer(const ddf_s* h, int l) {
  const int k = h->tr_segment;
  return k <= 1 || (l + 1) % k == 0 || l == h->cfg.hidden_layers - 1;
}

ddf_status train_alloc(ddf_s* h, void** p, size_t bytes) { return dev_alloc(h, p, bytes); }

// Head partials per row the last training layer leaves (pair kernel, mode 4):
// one per 256 columns and epilogue warp of a TMEM lane quarter.
int train_head_parts(int W) { return std::max(1, W / 256) * (ddf::kTrainEpiWarps / 4); }

// Writes the bf16 query copies (W_l, and W_l^T for l >= 1), the biases and
// the head from the FP32 master blob.
ddf_status refresh_weights(ddf_s* h, cudaStream_t st) {
  const int W = h->cfg.width;
  const BlobOffsets o = blob_offsets(h);
  for (int l = 0; l < h->cfg.hidden_layers; ++l) {
    const int K = l == 0 ? h->d_in : W;
    DDF_CK(ddf::launch_pack_bf16(h->d_blob + o.w[l], W, K, l == 0 ? h->kp16 : W, h->wb[l], st));
    DDF_CK(cudaMemcpyAsync(h->bias[l], h->d_blob + o.b[l], W * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
    if (l > 0 && static_cast<int>(h->wt.size()) > l && h->wt[l] != nullptr)
      DDF_CK(ddf::launch_pack_bf16_t(h->d_blob + o.w[l], W, W, h->wt[l], st));
  }
  const size_t hr = head_rows(h);
  DDF_CK(cudaMemcpyAsync(h->head_w, h->d_blob + o.wo, hr * W * sizeof(float),
                         cudaMemcpyDeviceToDevice, st));
  DDF_CK(cudaMemcpyAsync(h->head_b, h->d_blob + o.bo, hr * sizeof(float), cudaMemcpyDeviceToDevice,
                         st));
  return DDF_OK;
}

ddf_status ensure_train(ddf_s* h, int64_t B) {
  const int W = h->cfg.width, H = h->cfg.hidden_layers;
  ddf_status s;
  void* p;
  // the optimizer state and the weight copies training needs; a failure
  // half way frees all of it, so the next call starts from nothing
  auto alloc_state = [&]() -> ddf_status {
    const size_t np = n_params(h);
    if ((s = train_alloc(h, &p, np * sizeof(float))) != DDF_OK) return s;
    h->grad = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, np * sizeof(float))) != DDF_OK) return s;
    h->adam_m = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, np * sizeof(float))) != DDF_OK) return s;
    h->adam_v = static_cast<float*>(p);
    DDF_CK(cudaMemset(h->adam_m, 0, np * sizeof(float)));
    DDF_CK(cudaMemset(h->adam_v, 0, np * sizeof(float)));
    h->adam_step = 0;
    h->wt.assign(H, nullptr);
    h->tmWT.assign(H, CUtensorMap{});
    if ((s = ensure_plain_maps(h)) != DDF_OK) return s;
    h->tr_pair = W % 256 == 0 && h->pair_clusters > 0;
    h->tmBpair.assign(H, CUtensorMap{});
    h->tmWTpair.assign(H, CUtensorMap{});
    if (h->tr_pair &&
        !make_tmap(&h->tmBpair[0], h->wb[0], false, h->kp16, W, static_cast<uint64_t>(h->kp16) * 2, 128))
      return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for a weight map");
    for (int l = 1; l < H; ++l) {
      if ((s = train_alloc(h, &p, static_cast<size_t>(W) * W * 2)) != DDF_OK) return s;
      h->wt[l] = static_cast<__nv_bfloat16*>(p);
      if (!make_tmap(&h->tmWT[l], h->wt[l], false, W, W, static_cast<uint64_t>(W) * 2, h->bn))
        return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for a weight map");
      if (h->tr_pair &&
          (!make_tmap(&h->tmWTpair[l], h->wt[l], false, W, W, static_cast<uint64_t>(W) * 2, 128) ||
           !make_tmap(&h->tmBpair[l], h->wb[l], false, W, W, static_cast<uint64_t>(W) * 2, 128)))
        return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for a weight map");
    }
    const int nmax = std::max(W, 128);
    // two sets: layer l's reduction reads set l & 1 while the GEMMs of the
    // layer below write the other
    h->tr_part_set = kPartSplits * static_cast<size_t>(W) * nmax;
    if ((s = train_alloc(h, &p, 2 * h->tr_part_set * sizeof(float))) != DDF_OK) return s;
    h->tr_part = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, kColSplits * (3 * static_cast<size_t>(W) + 4) * sizeof(float))) !=
        DDF_OK)
      return s;
    h->tr_cpart = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, kHeadSplits * (3 * static_cast<size_t>(W) + 4) * sizeof(float))) !=
        DDF_OK)
      return s;
    h->tr_hpart = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, sizeof(unsigned))) != DDF_OK) return s;
    h->tr_nhit = static_cast<unsigned*>(p);
    if ((s = train_alloc(h, &p, ddf::kRedTickets * sizeof(unsigned))) != DDF_OK) return s;
    h->tr_ticket = static_cast<unsigned*>(p);
    DDF_CK(cudaMemset(h->tr_ticket, 0, ddf::kRedTickets * sizeof(unsigned)));
    if ((s = refresh_weights(h, nullptr)) != DDF_OK) return s;
    DDF_CK(cudaDeviceSynchronize());
    return DDF_OK;
  };
  if (h->grad == nullptr && (s = alloc_state()) != DDF_OK) {
    for (__nv_bfloat16* q : h->wt) dev_free(h, q);
    h->wt.clear();
    for (float** q : {&h->grad, &h->adam_m, &h->adam_v, &h->tr_part, &h->tr_cpart, &h->tr_hpart}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    for (unsigned** q : {&h->tr_nhit, &h->tr_ticket}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    return s;
  }
  if (B > h->tr_rows) {
    h->fwd_rows = 0;
    // every freed pointer is cleared, so a failure below leaves nothing to
    // free twice on the next attempt
    for (void** q : {&h->tr_enc, &h->tr_dpre[0], &h->tr_dpre[1], reinterpret_cast<void**>(&h->tr_z),
                     reinterpret_cast<void**>(&h->tr_dz), reinterpret_cast<void**>(&h->tr_lpart),
                     reinterpret_cast<void**>(&h->tr_colpart), reinterpret_cast<void**>(&h->tr_hz)}) {
      dev_free(h, *q);
      *q = nullptr;
    }
    for (void* q : h->tr_store) dev_free(h, q);
    h->tr_store.clear();
    h->tr_h.assign(H, nullptr);
    h->tr_rows = 0;
    const size_t act = static_cast<size_t>(B) * W * 2;
    if ((s = train_alloc(h, &h->tr_enc, static_cast<size_t>(B) * h->kp16 * 2)) != DDF_OK) return s;
    // kept layers own a buffer; a dropped layer j shares scratch slot
    // (j - first layer of its run) with the dropped layers of other runs
    std::vector<void*> scratch;
    for (int l = 0; l < H; ++l) {
      if (kept_layer(h, l)) {
        if ((s = train_alloc(h, &p, act)) != DDF_OK) return s;
        h->tr_store.push_back(p);
        h->tr_h[l] = p;
        continue;
      }
      int s0 = l;
      while (s0 > 0 && !kept_layer(h, s0 - 1)) --s0;
      const size_t slot = static_cast<size_t>(l - s0);
      if (slot >= scratch.size()) {
        if ((s = train_alloc(h, &p, act)) != DDF_OK) return s;
        h->tr_store.push_back(p);
        scratch.push_back(p);
      }
      h->tr_h[l] = scratch[slot];
    }
    for (int i = 0; i < 2; ++i)
      if ((s = train_alloc(h, &h->tr_dpre[i], act)) != DDF_OK) return s;
    if ((s = train_alloc(h, &p, B * sizeof(float2))) != DDF_OK) return s;
    h->tr_z = static_cast<float2*>(p);
    if ((s = train_alloc(h, &p, B * sizeof(float2))) != DDF_OK) return s;
    h->tr_dz = static_cast<float2*>(p);
    if ((s = train_alloc(h, &p, ((B + 255) / 256) * sizeof(float))) != DDF_OK) return s;
    h->tr_lpart = static_cast<float*>(p);
    h->tr_colpart_set = static_cast<size_t>(round_up(B, 256) / 32) * W;  // two sets, as tr_part
    if ((s = train_alloc(h, &p, 2 * h->tr_colpart_set * sizeof(float))) != DDF_OK) return s;
    h->tr_colpart = static_cast<float*>(p);
    if ((s = train_alloc(h, &p, static_cast<size_t>(train_head_parts(W)) * B * sizeof(float2))) !=
        DDF_OK)
      return s;
    h->tr_hz = static_cast<float2*>(p);
    h->tr_rows = B;
  }
  return DDF_OK;
}

// One tensor-core GEMM C = A B^T with A [M x K] and B [N x K] bf16 K-major.
ddf_status tc_gemm(ddf_s* h, const void* A, int M, int K, const CUtensorMap& tmB, int bn,
                   ddf::TcGemmParams p, cudaStream_t st) {
  CUtensorMap tmA;
  if (!make_tmap(&tmA, A, false, K, M, static_cast<uint64_t>(K) * 2, 128))
    return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for an activation map");
  p.M = M;
  p.K = K;
  p.status = h->status_dev;
  p.timeout_ns = h->timeout_ns;
  const int splits = p.k_splits > 1 ? p.k_splits : 1;
  const int64_t tiles = splits * ((M + 127) / 128) * static_cast<int64_t>(p.N / bn);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, h->num_sms));
  DDF_CK(ddf::launch_tc_gemm(ddf::TcTile{bn, 4}, false, false, tmA, tmB, p, grid, st));
  return DDF_OK;
}

// The same on the CTA-pair kernel (W a multiple of 256; B-operand maps with
// 128-row boxes); staged: mode-0 outputs leave through shared memory.
ddf_status tc_gemm_pair(ddf_s* h, const void* A, int M, int K, const CUtensorMap& tmB, bool staged,
                        ddf::TcGemmParams p, cudaStream_t st) {
  CUtensorMap tmA;
  if (!make_tmap(&tmA, A, false, K, M, static_cast<uint64_t>(K) * 2, 128))
    return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for an activation map");
  p.M = M;
  p.K = K;
  p.status = h->status_dev;
  p.timeout_ns = h->timeout_ns;
  const int64_t tiles = ((M + 255) / 256) * static_cast<int64_t>(p.N / 256);
  const int clusters = static_cast<int>(std::min<int64_t>(tiles, h->pair_clusters));
  CUtensorMap tmO;  // a staged forward's output leaves shared memory by TMA stores
  const bool tma_out = staged && p.mode == 0;
  if (tma_out) {
    if (!make_tmap(&tmO, p.out, false, p.N, M, static_cast<uint64_t>(p.ldo) * 2, 32))
      return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for an output map");
    p.tma_out = 1;
  }
  DDF_CK(ddf::launch_tc_gemm_pair(false, false, staged, 4, tmA, tmB, p, clusters, st,
                                  tma_out ? &tmO : nullptr));
  return DDF_OK;
}

ddf_status check_train_args(ddf_s* h, const float* const rays[6], const float* t_target,
                            const uint8_t* hit_target, int64_t batch, int kind = DDF_KIND_RAY) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  const bool hg = h->cfg.kind == DDF_KIND_HASHGRID &&
                  (kind == DDF_KIND_RAY || kind == DDF_KIND_HASHGRID);  // a ray field too
  if (h->cfg.kind != kind && !hg)
    return fail(DDF_ERR_INVALID_ARG, kind == DDF_KIND_RAY ? "not a ray (DDF) field" : "not an SDF field");
  if (!h->loaded) return fail(DDF_ERR_BAD_WEIGHTS, "no weights loaded");
  if (h->cfg.precision != DDF_BF16 && !hg)
    return fail(DDF_ERR_UNSUPPORTED, "training runs on bf16 handles");
  if (batch < 8 || batch % 8 != 0 || batch >= (int64_t{1} << 31))
    return fail(DDF_ERR_INVALID_ARG, "batch must be a positive multiple of 8 below 2^31");
  DDF_REQUIRE_ALIGNED(t_target, 4);
  ddf_status s = check_rays(rays, batch);
  if (s != DDF_OK) return s;
  if (t_target == nullptr || (kind == DDF_KIND_RAY && hit_target == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "targets are NULL");
  return DDF_OK;
}

// Forward keeping every activation: encoding, the tensor-core layers, the
// FP32 head into h->tr_z (float2 per row; .y unused for an SDF field).
// rays: 6 SoA arrays (ray field) or 3 point arrays (SDF field, in rays[0..2]).
// Whether the last layer's epilogue computes the head (a ray field on the
// pair path: two head rows from the stored bf16 outputs); otherwise
// head_train reads the last activation back.
bool head_in_last_layer(const ddf_s* h) { return h->tr_pair && h->cfg.kind == DDF_KIND_RAY; }

// Forward of layer l over the batch: tr_h[l] = ReLU(tr_h[l-1] W_l^T + b_l)
// (layer 0 reads the encoding). The GEMMs are deterministic, so a
// recomputed layer is bitwise the first one.
ddf_status forward_layer(ddf_s* h, int l, int B, cudaStream_t st) {
  const int W = h->cfg.width, H = h->cfg.hidden_layers;
  ddf::TcGemmParams p{};
  p.N = W;
  p.bias = h->bias[l];
  p.out_scale = 1.0f;
  p.out = h->tr_h[l];
  p.ldo = W;
  p.mode = 0;
  ProfScope ps(h, l == 0 ? kProfFirst : kProfGemm, st);
  const void* A_in = l == 0 ? h->tr_enc : h->tr_h[l - 1];
  const int K = l == 0 ? h->kp16 : W;
  if (head_in_last_layer(h) && l == H - 1) {  // z's partial dot products, per 256 columns
    p.mode = 4;
    p.head_w = h->head_w;
    p.head_part = h->tr_hz;
  }
  return h->tr_pair ? tc_gemm_pair(h, A_in, B, K, h->tmBpair[l], true, p, st)
                    : tc_gemm(h, A_in, B, K, h->tmBtr[l], h->bn, p, st);
}

ddf_status forward_keep(ddf_s* h, const float* const rays[6], int B, cudaStream_t st) {
  const bool sdf = h->cfg.kind == DDF_KIND_SDF;
  const int W = h->cfg.width, H = h->cfg.hidden_layers;
  ddf::RaySoA r;
  for (int c = 0; c < 6; ++c) r.p[c] = rays[c];
  auto bf = [](void* q) { return static_cast<__nv_bfloat16*>(q); };
  {
    ProfScope ps(h, kProfEncode, st);
    if (sdf)
      DDF_CK(ddf::launch_encode_points_bf16(r.p[0], r.p[1], r.p[2], B, h->cfg.octaves, h->kp16,
                                            bf(h->tr_enc), st));
    else
      DDF_CK(ddf::launch_encode_bf16(r, B, h->cfg.octaves, h->kp16, bf(h->tr_enc), st));
  }
  for (int l = 0; l < H; ++l) {
    const ddf_status s = forward_layer(h, l, B, st);
    if (s != DDF_OK) return s;
  }
  if (head_in_last_layer(h))
    DDF_CK(ddf::launch_head_sum(h->tr_hz, train_head_parts(W), B, h->head_b, h->tr_z, st));
  else
    DDF_CK(ddf::launch_head_train(bf(h->tr_h[H - 1]), B, W, h->head_w, h->head_b, h->tr_z, st));
  return DDF_OK;
}

// The stream the layers' gradient reductions run on and its events, made on
// first use.
ddf_status ensure_reduce_stream(ddf_s* h) {
  if (h->s_red != nullptr) return DDF_OK;
  for (int b = 0; b < 2; ++b) {
    if (h->ev_gemm[b] == nullptr)
      DDF_CK(cudaEventCreateWithFlags(&h->ev_gemm[b], cudaEventDisableTiming));
    if (h->ev_red[b] == nullptr)
      DDF_CK(cudaEventCreateWithFlags(&h->ev_red[b], cudaEventDisableTiming));
  }
  if (h->ev_join == nullptr) DDF_CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  DDF_CK(cudaStreamCreateWithFlags(&h->s_red, cudaStreamNonBlocking));
  return DDF_OK;
}

ddf_status backward_layers(ddf_s* h, int B, cudaStream_t st, cudaStream_t rs);

// Backward from dL/dz in h->tr_dz through the head and every layer, using the
// activations forward_keep left; the gradient goes to h->grad.
ddf_status backward_from_dz(ddf_s* h, int B, cudaStream_t st) {
  const int hr = static_cast<int>(head_rows(h));
  const int W = h->cfg.width, H = h->cfg.hidden_layers;
  const BlobOffsets o = blob_offsets(h);
  auto bf = [](void* q) { return static_cast<__nv_bfloat16*>(q); };

  // ---- head: dW_o = dz^T h_H, db_o = sum dz, dpre_H = (dz W_o) where h_H > 0
  // and its column sums (the last layer's bias gradient), in one pass over
  // h_H; its row-split partials [dz0 h | dz1 h | dpre | dz0 | dz1 | 2 padding] reduce in
  // one deterministic launch
  const int hsplits = std::max(1, std::min(kHeadSplits, B / 64));
  DDF_CK(ddf::launch_head_back_fused(h->tr_dz, bf(h->tr_h[H - 1]), B, W, h->head_w, hsplits,
                                     bf(h->tr_dpre[0]), h->tr_hpart, st));
  {
    ddf::GradReduce g;
    ddf::RedCols& c = g.cols;
    c.X = h->tr_hpart;
    c.M = hsplits;
    c.N = 3 * W + 2;
    c.ld = 3 * W + 4;
    c.ldc = 3 * W + 4;
    c.R = kColSplits;
    c.cpart = h->tr_cpart;
    c.ticket = h->tr_ticket;
    c.nseg = 3;
    c.c0[0] = 0;          // dW_o rows (hr of them, row-major like the blob)
    c.cnt[0] = hr * W;
    c.out[0] = h->grad + o.wo;
    c.c0[1] = 2 * W;      // the last layer's bias
    c.cnt[1] = W;
    c.out[1] = h->grad + o.b[H - 1];
    c.c0[2] = 3 * W;      // db_o
    c.cnt[2] = hr;
    c.out[2] = h->grad + o.bo;
    DDF_CK(ddf::launch_grad_reduce(g, st));
  }

  // ---- layers, last to first. Each layer's reduction runs on the side
  // stream while the main stream goes on with the GEMMs below it; the
  // caller's stream waits for all of them before it returns, failed or not.
  ddf_status s = ensure_reduce_stream(h);
  if (s != DDF_OK) return s;
  DDF_CK(cudaEventRecord(h->ev_join, st));  // the head's reduction above, in order
  DDF_CK(cudaStreamWaitEvent(h->s_red, h->ev_join, 0));
  s = backward_layers(h, B, st, h->s_red);
  const cudaError_t e1 = cudaEventRecord(h->ev_join, h->s_red);
  const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(st, h->ev_join, 0) : e1;
  if (s != DDF_OK) return s;
  if (e2 != cudaSuccess) return cuda_fail(e2, "joining the reduction stream");
  h->grad_valid = true;
  return DDF_OK;
}

// The layers of the backward pass. Layer l's weight-gradient partials and
// its bias column partials live in buffer set l & 1 (tr_part, tr_colpart);
// its reduction runs on rs after the GEMM that wrote the partials, and a GEMM
// that is about to overwrite a set waits for the reduction that last read it.
ddf_status backward_layers(ddf_s* h, int B, cudaStream_t st, cudaStream_t rs) {
  const int W = h->cfg.width, H = h->cfg.hidden_layers;
  const BlobOffsets o = blob_offsets(h);
  auto part_set = [&](int l) { return h->tr_part + static_cast<size_t>(l & 1) * h->tr_part_set; };
  auto colpart_set = [&](int l) {
    return h->tr_colpart + static_cast<size_t>(l & 1) * h->tr_colpart_set;
  };
  bool pending[2] = {false, false};  // a reduction of set b was issued
  int cur = 0;
  const int num_kb = (B + 63) / 64;
  for (int l = H - 1; l >= 0; --l) {
    const int K = l == 0 ? h->d_in : W;        // columns of W_l in the blob
    const int Kst = l == 0 ? h->kp16 : W;      // stored width of the layer input
    const int N = l == 0 ? static_cast<int>(round_up(h->kp16, 128)) : W;  // GEMM N
    const int bnw = N % 256 == 0 ? 256 : 128;
    const bool pair = h->tr_pair && N % 256 == 0;
    // split the batch so that the tiles fill the GPU evenly: the number of
    // splits s minimises waves(s) / s (time per unit of work, waves = ceil(s
    // tiles / CTAs or pairs)) with 2 % per split for the partials' traffic,
    // within the partial buffer (kPartSplits W max(W, 128) floats) and at
    // least one k-block per split
    const int64_t tiles1 = pair ? static_cast<int64_t>((W + 255) / 256) * (N / 256)
                                : static_cast<int64_t>((W + 127) / 128) * (N / bnw);
    const int64_t slots = pair ? h->pair_clusters : h->num_sms;
    const int64_t cap = std::min<int64_t>(
        num_kb, (kPartSplits * static_cast<int64_t>(W) * std::max(W, 128)) / (static_cast<int64_t>(W) * N));
    int splits = 1;
    double best = 1e30;
    for (int64_t c = 1; c <= cap; ++c) {
      const double waves = static_cast<double>((c * tiles1 + slots - 1) / slots);
      const double cost = waves / static_cast<double>(c) * (1.0 + 0.02 * static_cast<double>(c));
      if (cost < best - 1e-12) {
        best = cost;
        splits = static_cast<int>(c);
      }
    }
    // with checkpointing, layer l's input may not have been kept: when it
    // is the top of a run of dropped layers, recompute the run from the kept
    // layer below it (the layers under it in the run follow in this loop)
    if (l > 0 && !kept_layer(h, l - 1) && kept_layer(h, l)) {
      int s0 = l - 1;
      while (s0 > 0 && !kept_layer(h, s0 - 1)) --s0;
      for (int j = s0; j <= l - 1; ++j) {
        const ddf_status s = forward_layer(h, j, B, st);
        if (s != DDF_OK) return s;
      }
    }
    const void* A_in = l == 0 ? h->tr_enc : h->tr_h[l - 1];
    // dW_l [W x N] = dpre^T A_in, the sum over the batch split in `splits`
    // ranges: both operands are read as stored ([B x W] and [B x Kst],
    // row-major), i.e. MN-major, so nothing is transposed
    CUtensorMap tmD, tmX;
    if (!make_tmap(&tmD, h->tr_dpre[cur], false, W, B, static_cast<uint64_t>(W) * 2, 64) ||
        !make_tmap(&tmX, A_in, false, Kst, B, static_cast<uint64_t>(Kst) * 2, 64))
      return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed for a gradient map");
    ddf::TcGemmParams p{};
    p.M = W;
    p.N = N;
    p.K = B;
    p.mode = 3;
    p.mn_major = 1;
    p.out_f32 = part_set(l);
    p.ldo = N;
    p.k_splits = splits;
    p.split_stride = static_cast<size_t>(W) * N;
    p.status = h->status_dev;
    p.timeout_ns = h->timeout_ns;
    if (pending[l & 1]) DDF_CK(cudaStreamWaitEvent(st, h->ev_red[l & 1], 0));
    {
      ProfScope ps(h, kProfGemm, st);
      const int grid = static_cast<int>(std::min<int64_t>(splits * tiles1, slots));
      if (pair)
        DDF_CK(ddf::launch_tc_gemm_pair(false, false, false, 4, tmD, tmX, p, grid, st));
      else
        DDF_CK(ddf::launch_tc_gemm(ddf::TcTile{bnw, 4}, false, false, tmD, tmX, p, grid, st));
    }
    // one launch: dW_l from the split partials, and the bias gradient, the
    // column sums of dpre_l, from the 32-row partials the pair kernel's
    // input-gradient epilogue left (below, one layer up), or read from
    // dpre_l itself without the pair kernel (the top layer's bias came with
    // the head's backward)
    {
      ddf::GradReduce g;
      g.nsplit = 1;
      ddf::RedSplit& a = g.split[0];
      a.part = part_set(l);
      a.split_stride = static_cast<int64_t>(W) * N;
      a.S = splits;
      a.rows = W;
      a.cols = K;
      a.ldp = N;
      a.ldo = K;
      a.out = h->grad + o.w[l];
      if (l < H - 1) {
        ddf::RedCols& c = g.cols;
        c.X = h->tr_pair ? static_cast<const void*>(colpart_set(l)) : h->tr_dpre[cur];
        c.x_bf16 = h->tr_pair ? 0 : 1;
        c.M = h->tr_pair ? static_cast<int>(round_up(B, 256) / 32) : B;
        c.N = W;
        c.ld = W;
        c.ldc = W;
        c.R = kColSplits;
        c.cpart = h->tr_cpart;
        c.ticket = h->tr_ticket;
        c.nseg = 1;
        c.cnt[0] = W;
        c.out[0] = h->grad + o.b[l];
      }
      DDF_CK(cudaEventRecord(h->ev_gemm[l & 1], st));
      DDF_CK(cudaStreamWaitEvent(rs, h->ev_gemm[l & 1], 0));
      DDF_CK(ddf::launch_grad_reduce(g, rs));
      DDF_CK(cudaEventRecord(h->ev_red[l & 1], rs));
      pending[l & 1] = true;
    }
    if (l == 0) break;
    // the input gradient writes set (l - 1) & 1 and dpre[cur ^ 1], which the
    // reduction of layer l + 1 read
    if (pending[(l + 1) & 1]) DDF_CK(cudaStreamWaitEvent(st, h->ev_red[(l + 1) & 1], 0));
    // dpre_{l-1} [B x W] = (dpre_l [B x W]) (W_l^T [W x W])^T masked by h_{l-1} > 0
    ddf::TcGemmParams q{};
    q.N = W;
    q.mode = 2;
    q.out = h->tr_dpre[cur ^ 1];
    q.ldo = W;
    q.mask = h->tr_h[l - 1];
    q.ldm = W;
    if (h->tr_pair) q.col_part = colpart_set(l - 1);
    {
      ProfScope ps(h, kProfGemm, st);
      ddf_status s = h->tr_pair ? tc_gemm_pair(h, h->tr_dpre[cur], B, W, h->tmWTpair[l], false, q, st)
                                : tc_gemm(h, h->tr_dpre[cur], B, W, h->tmWT[l], h->bn, q, st);
      if (s != DDF_OK) return s;
    }
    cur ^= 1;
  }
  return DDF_OK;
}

// rays: 6 SoA arrays (ray field) or 3 point arrays (SDF field, in rays[0..2]);
// t_tgt: first-hit distances (ray field) or signed distances (SDF field);
// y: hit flags (ray field only).
ddf_status compute_grad(ddf_s* h, const float* const rays[6], const float* t_tgt,
                        const uint8_t* y, int64_t B64, float* loss_out, cudaStream_t st) {
  const int B = static_cast<int>(B64);
  h->fwd_rows = 0;  // the kept activations become this batch's
  ddf_status s = forward_keep(h, rays, B, st);
  if (s != DDF_OK) return s;
  if (h->cfg.kind == DDF_KIND_SDF)
    DDF_CK(ddf::launch_sdf_loss(h->tr_z, t_tgt, B, h->tr_dz, h->tr_lpart, loss_out, st));
  else
    DDF_CK(ddf::launch_loss(h->tr_z, t_tgt, y, B, h->tr_nhit, kClamp, kLambda, h->tr_dz,
                            h->tr_lpart, loss_out, st));
  return backward_from_dz(h, B, st);
}

ddf_status train_step(ddf_s* h, const float* const rays[6], const float* t_target,
                      const uint8_t* hit_target, int64_t batch, float lr, float* out_loss,
                      cudaStream_t st);

}  // namespace

extern "C" {

ddf_status ddf_compute_grad(ddf_handle h, const float* const rays[6], const float* t_target,
                            const uint8_t* hit_target, int64_t batch, float* out_loss,
                            void* stream) {
  ddf_status s = check_train_args(h, rays, t_target, hit_target, batch);
  if (s != DDF_OK) return s;
  DDF_REQUIRE_ALIGNED(out_loss, 4);
  DeviceGuard g(h->cfg.device);
  if (is_hashgrid(h)) {
    if ((s = hg_ensure_train(h, batch)) != DDF_OK) return s;
    ddf::RaySoA r;
    for (int c = 0; c < 6; ++c) r.p[c] = rays[c];
    return hg_train(h, r, t_target, hit_target, static_cast<int>(batch), 0.f, out_loss,
                    static_cast<cudaStream_t>(stream));
  }
  if ((s = ensure_train(h, batch)) != DDF_OK) return s;
  return compute_grad(h, rays, t_target, hit_target, batch, out_loss,
                      static_cast<cudaStream_t>(stream));
}

ddf_status ddf_train_step(ddf_handle h, const float* const rays[6], const float* t_target,
                          const uint8_t* hit_target, int64_t batch, float lr, float* out_loss,
                          void* stream) {
  ddf_status s = check_train_args(h, rays, t_target, hit_target, batch);
  if (s != DDF_OK) return s;
  DDF_REQUIRE_ALIGNED(out_loss, 4);
  return train_step(h, rays, t_target, hit_target, batch, lr, out_loss,
                    static_cast<cudaStream_t>(stream));
}

ddf_status ddf_sdf_compute_grad(ddf_handle h, const float* const points[3], const float* s_target,
                                int64_t batch, float* out_loss, void* stream) {
  const float* p6[6] = {points ? points[0] : nullptr, points ? points[1] : nullptr,
                        points ? points[2] : nullptr, points ? points[0] : nullptr,
                        points ? points[1] : nullptr, points ? points[2] : nullptr};
  ddf_status s = check_train_args(h, p6, s_target, nullptr, batch, DDF_KIND_SDF);
  if (s != DDF_OK) return s;
  DeviceGuard g(h->cfg.device);
  if ((s = ensure_train(h, batch)) != DDF_OK) return s;
  return compute_grad(h, p6, s_target, nullptr, batch, out_loss, static_cast<cudaStream_t>(stream));
}

ddf_status ddf_sdf_train_step(ddf_handle h, const float* const points[3], const float* s_target,
                              int64_t batch, float lr, float* out_loss, void* stream) {
  const float* p6[6] = {points ? points[0] : nullptr, points ? points[1] : nullptr,
                        points ? points[2] : nullptr, points ? points[0] : nullptr,
                        points ? points[1] : nullptr, points ? points[2] : nullptr};
  ddf_status s = check_train_args(h, p6, s_target, nullptr, batch, DDF_KIND_SDF);
  if (s != DDF_OK) return s;
  return train_step(h, p6, s_target, nullptr, batch, lr, out_loss, static_cast<cudaStream_t>(stream));
}

ddf_status ddf_union_sdf(const float* spheres, int32_t n_spheres, const float* boxes,
                         int32_t n_boxes, const float* const points[3], int64_t n, float* out_s,
                         void* stream) {
  if (n_spheres < 0 || n_boxes < 0) return fail(DDF_ERR_INVALID_ARG, "negative primitive count");
  if ((n_spheres > 0 && spheres == nullptr) || (n_boxes > 0 && boxes == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "primitive array is NULL");
  if (n < 0) return fail(DDF_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (points == nullptr || points[0] == nullptr || points[1] == nullptr ||
                points[2] == nullptr || out_s == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "a pointer is NULL");
  if (n == 0) return DDF_OK;
  DDF_REQUIRE_ALIGNED(spheres, 4);
  DDF_REQUIRE_ALIGNED(boxes, 4);
  for (int c = 0; c < 3; ++c) DDF_REQUIRE_ALIGNED(points[c], 4);
  DDF_REQUIRE_ALIGNED(out_s, 4);
  DDF_CK(ddf::launch_union_sdf(spheres, n_spheres, boxes, n_boxes, points[0], points[1], points[2],
                               n, out_s, static_cast<cudaStream_t>(stream)));
  return DDF_OK;
}

}  // extern "C"

namespace {

// Gradient, then Adam on the FP32 master weights and a refresh of the bf16 copies.
ddf_status train_step(ddf_s* h, const float* const rays[6], const float* t_target,
                      const uint8_t* hit_target, int64_t batch, float lr, float* out_loss,
                      cudaStream_t st) {
  if (!(lr > 0.f) || !std::isfinite(lr)) return fail(DDF_ERR_INVALID_ARG, "lr must be positive");
  DeviceGuard g(h->cfg.device);
  ddf_status s;
  if (is_hashgrid(h)) {
    if ((s = hg_ensure_train(h, batch)) != DDF_OK) return s;
    ddf::RaySoA r;
    for (int c = 0; c < 6; ++c) r.p[c] = rays[c];
    return hg_train(h, r, t_target, hit_target, static_cast<int>(batch), lr, out_loss, st);
  }
  if ((s = ensure_train(h, batch)) != DDF_OK) return s;
  if ((s = compute_grad(h, rays, t_target, hit_target, batch, out_loss, st)) != DDF_OK) return s;
  ++h->adam_step;
  const double t = static_cast<double>(h->adam_step);
  const float bc1 = static_cast<float>(1.0 - std::pow(0.9, t));
  const float bc2 = static_cast<float>(1.0 - std::pow(0.999, t));
  {
    ProfScope ps(h, kProfHead, st);
    h->fwd_rows = 0;  // the weights change
    const int W = h->cfg.width, H = h->cfg.hidden_layers;
    if (2 * H + 2 > ddf::kAdamBlocks) {  // deep nets: Adam, then the copies
      DDF_CK(ddf::launch_adam(h->d_blob, h->grad, h->adam_m, h->adam_v,
                              static_cast<int64_t>(n_params(h)), lr, kB1, kB2, kEps, bc1, bc2, st));
      return refresh_weights(h, st);
    }
    // Adam and the refresh of the bf16 copies (W_l, W_l^T), biases and head
    // in one pass over the blob
    const BlobOffsets o = blob_offsets(h);
    ddf::AdamBlocks bl{};
    auto add = [&](size_t start, int rows, int cols, int ldb, __nv_bfloat16* wb,
                   __nv_bfloat16* wt, float* f32) {
      bl.b[bl.n++] = ddf::AdamBlock{static_cast<int64_t>(start), rows, cols, ldb, wb, wt, f32};
    };
    for (int l = 0; l < H; ++l) {
      const int K = l == 0 ? h->d_in : W;
      __nv_bfloat16* wt = (l > 0 && static_cast<int>(h->wt.size()) > l) ? h->wt[l] : nullptr;
      add(o.w[l], W, K, l == 0 ? h->kp16 : W, h->wb[l], wt, nullptr);
      add(o.b[l], 1, W, 0, nullptr, nullptr, h->bias[l]);
    }
    const int hr = static_cast<int>(head_rows(h));
    add(o.wo, 1, hr * W, 0, nullptr, nullptr, h->head_w);
    add(o.bo, 1, hr, 0, nullptr, nullptr, h->head_b);
    DDF_CK(ddf::launch_adam_refresh(h->d_blob, h->grad, h->adam_m, h->adam_v,
                                    static_cast<int64_t>(n_params(h)), lr, kB1, kB2, kEps, bc1, bc2,
                                    bl, st));
  }
  return DDF_OK;
}

}  // namespace

extern "C" {

ddf_status ddf_forward_train(ddf_handle h, const float* const inputs[6], int64_t batch,
                             float* out_z, void* stream) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  const bool sdf = h->cfg.kind == DDF_KIND_SDF;
  const float* p6[6] = {};
  for (int c = 0; c < 6 && inputs != nullptr; ++c) p6[c] = inputs[sdf ? c % 3 : c];
  // the target checks do not apply to a forward pass: pass a dummy target
  const float dummy = 0.f;
  const uint8_t ydummy = 0;
  ddf_status s = check_train_args(h, p6, &dummy, &ydummy, batch, h->cfg.kind);
  if (s != DDF_OK) return s;
  if (out_z == nullptr) return fail(DDF_ERR_INVALID_ARG, "out_z is NULL");
  DDF_REQUIRE_ALIGNED(out_z, 4);
  DeviceGuard g(h->cfg.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (is_hashgrid(h)) {
    if ((s = hg_ensure_train(h, batch)) != DDF_OK) return s;
    h->fwd_rows = 0;
    ddf::RaySoA r;
    for (int c = 0; c < 6; ++c) r.p[c] = p6[c];
    if ((s = hg_forward_keep(h, r, static_cast<int>(batch), st)) != DDF_OK) return s;
  } else {
    if ((s = ensure_train(h, batch)) != DDF_OK) return s;
    h->fwd_rows = 0;
    if ((s = forward_keep(h, p6, static_cast<int>(batch), st)) != DDF_OK) return s;
  }
  if (head_rows(h) == 2) {
    DDF_CK(cudaMemcpyAsync(out_z, h->tr_z, batch * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  } else {  // z0 of each float2 into a dense column
    DDF_CK(cudaMemcpy2DAsync(out_z, sizeof(float), h->tr_z, sizeof(float2), sizeof(float),
                             batch, cudaMemcpyDeviceToDevice, st));
  }
  for (int c = 0; c < 6; ++c) h->fwd_rays.p[c] = p6[c];  // the backward's table scatter re-reads them
  h->fwd_rows = batch;
  return DDF_OK;
}

ddf_status ddf_backward(ddf_handle h, const float* dz, int64_t batch, void* stream) {
  if (h == nullptr || dz == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  DDF_REQUIRE_ALIGNED(dz, 4);
  if (h->fwd_rows == 0 || h->fwd_rows != batch)
    return fail(DDF_ERR_INVALID_ARG,
                "ddf_backward needs the activations of a ddf_forward_train of the same batch, "
                "with no weight update or other training call in between");
  DeviceGuard g(h->cfg.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (head_rows(h) == 2) {
    DDF_CK(cudaMemcpyAsync(h->tr_dz, dz, batch * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  } else {  // (dz, 0) pairs: the unused second head row gets no gradient
    DDF_CK(cudaMemsetAsync(h->tr_dz, 0, batch * sizeof(float2), st));
    DDF_CK(cudaMemcpy2DAsync(h->tr_dz, sizeof(float2), dz, sizeof(float), sizeof(float), batch,
                             cudaMemcpyDeviceToDevice, st));
  }
  if (is_hashgrid(h)) return hg_backward(h, h->fwd_rays, static_cast<int>(batch), st);
  return backward_from_dz(h, static_cast<int>(batch), st);
}

ddf_status ddf_copy_grad(ddf_handle h, float* dev_grad, size_t n_floats, void* stream) {
  if (h == nullptr || dev_grad == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  DDF_REQUIRE_ALIGNED(dev_grad, 4);
  if (!h->grad_valid) return fail(DDF_ERR_INVALID_ARG, "no gradient computed yet");
  if (n_floats != n_params(h)) return fail(DDF_ERR_INVALID_ARG, "wrong blob size");
  DeviceGuard g(h->cfg.device);
  DDF_CK(cudaMemcpyAsync(dev_grad, h->grad, n_floats * sizeof(float), cudaMemcpyDeviceToDevice,
                         static_cast<cudaStream_t>(stream)));
  return DDF_OK;
}

ddf_status ddf_load_weights_device(ddf_handle h, const float* dev_blob, size_t n_floats,
                                   void* stream) {
  if (h == nullptr || dev_blob == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  DDF_REQUIRE_ALIGNED(dev_blob, 4);
  if (!h->loaded) return fail(DDF_ERR_BAD_WEIGHTS, "load weights once with ddf_load_weights first");
  if (h->cfg.precision != DDF_BF16 && !is_hashgrid(h))
    return fail(DDF_ERR_UNSUPPORTED, "device weight updates run on bf16 handles");
  if (n_floats != n_params(h)) return fail(DDF_ERR_BAD_WEIGHTS, "wrong blob size");
  DeviceGuard g(h->cfg.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->fwd_rows = 0;
  DDF_CK(cudaMemcpyAsync(h->d_blob, dev_blob, n_floats * sizeof(float), cudaMemcpyDeviceToDevice,
                         st));
  if (is_hashgrid(h)) return h->cfg.precision == DDF_FP32 ? DDF_OK : hg_refresh(h, st);
  return refresh_weights(h, st);
}

ddf_status ddf_get_grad(ddf_handle h, float* host_grad, size_t n_floats) {
  if (h == nullptr || host_grad == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  if (!h->grad_valid) return fail(DDF_ERR_INVALID_ARG, "no gradient computed yet");
  if (n_floats != n_params(h)) return fail(DDF_ERR_INVALID_ARG, "wrong blob size");
  DeviceGuard g(h->cfg.device);
  DDF_CK(cudaDeviceSynchronize());
  DDF_CK(cudaMemcpy(host_grad, h->grad, n_floats * sizeof(float), cudaMemcpyDeviceToHost));
  return DDF_OK;
}

ddf_status ddf_set_recompute(ddf_handle h, int32_t segment) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  if (segment < 1) return fail(DDF_ERR_INVALID_ARG, "segment must be >= 1");
  if (h->cfg.kind == DDF_KIND_HASHGRID)
    return fail(DDF_ERR_UNSUPPORTED, "the hash-grid field keeps its 64-wide activations");
  if (segment == h->tr_segment) return DDF_OK;
  DeviceGuard g(h->cfg.device);
  DDF_CK(cudaDeviceSynchronize());  // no launch may still use the buffers
  h->tr_segment = segment;
  h->tr_rows = 0;   // the next training call lays the activation buffers out anew
  h->fwd_rows = 0;
  return DDF_OK;
}

ddf_status ddf_get_train_activation_bytes(ddf_handle h, size_t* out) {
  if (h == nullptr || out == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  *out = h->tr_store.size() * static_cast<size_t>(h->tr_rows) * h->cfg.width * 2;
  return DDF_OK;
}

}  // extern "C"

// ---- training checkpoints -------------------------------------------------
// File: magic "DDFCKPT" + NUL, u32 version (1), u32 flags (bit 0: optimizer
// state present), the ddf_config (6 x i32), u64 parameter count, i64 Adam
// step, u32 CRC-32 of the payload, u32 zero; then the payload: the FP32
// master weights and, with bit 0, the Adam moments m and v (same layout).
// Little-endian, as every target of this library is.

namespace {

constexpr char kCkptMagic[8] = {'D', 'D', 'F', 'C', 'K', 'P', 'T', '\0'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, flags;
  ddf_config cfg;
  uint64_t n_params;
  int64_t adam_step;
  uint32_t crc, reserved;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header layout");

// CRC-32 of the ISO-HDLC / zlib definition: reflected polynomial 0xEDB88320,
// initial value and final XOR 0xFFFFFFFF.
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  static uint32_t table[256];
  static bool ready = false;
  if (!ready) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
      table[i] = c;
    }
    ready = true;
  }
  const uint8_t* b = static_cast<const uint8_t*>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ b[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

bool same_field(const ddf_config& a, const ddf_config& b) {
  return a.octaves == b.octaves && a.width == b.width && a.hidden_layers == b.hidden_layers &&
         a.precision == b.precision && a.kind == b.kind;
}

}  // namespace

extern "C" {

ddf_status ddf_save_checkpoint(ddf_handle h, const char* path) {
  if (h == nullptr || path == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  if (!h->loaded || h->d_blob == nullptr) return fail(DDF_ERR_BAD_WEIGHTS, "no weights loaded");
  DeviceGuard g(h->cfg.device);
  const size_t n = n_params(h);
  const bool opt = h->adam_m != nullptr && h->adam_v != nullptr && h->adam_step > 0;
  std::vector<float> payload(n * (opt ? 3 : 1));
  DDF_CK(cudaDeviceSynchronize());
  DDF_CK(cudaMemcpy(payload.data(), h->d_blob, n * sizeof(float), cudaMemcpyDeviceToHost));
  if (opt) {
    DDF_CK(cudaMemcpy(payload.data() + n, h->adam_m, n * sizeof(float), cudaMemcpyDeviceToHost));
    DDF_CK(cudaMemcpy(payload.data() + 2 * n, h->adam_v, n * sizeof(float), cudaMemcpyDeviceToHost));
  }
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.flags = opt ? 1u : 0u;
  hd.cfg = h->cfg;
  hd.n_params = n;
  hd.adam_step = opt ? h->adam_step : 0;
  hd.crc = crc32_update(0, payload.data(), payload.size() * sizeof(float));
  FILE* f = std::fopen(path, "wb");
  if (f == nullptr) return fail(DDF_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                  std::fwrite(payload.data(), sizeof(float), payload.size(), f) == payload.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) return fail(DDF_ERR_INVALID_ARG, std::string("cannot write ") + path);
  return DDF_OK;
}

ddf_status ddf_load_checkpoint(ddf_handle h, const char* path) {
  if (h == nullptr || path == nullptr) return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (f == nullptr) return fail(DDF_ERR_INVALID_ARG, std::string("cannot open ") + path);
  CkptHeader hd{};
  const bool got = std::fread(&hd, sizeof(hd), 1, f) == 1;
  if (!got || std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion) {
    std::fclose(f);
    return fail(DDF_ERR_INVALID_ARG, "not a checkpoint of this version");
  }
  const size_t n = n_params(h);
  if (!same_field(hd.cfg, h->cfg) || hd.n_params != n || (hd.flags & ~1u) != 0) {
    std::fclose(f);
    return fail(DDF_ERR_INVALID_ARG, "the checkpoint is of another field configuration");
  }
  const bool opt = (hd.flags & 1u) != 0;
  std::vector<float> payload(n * (opt ? 3 : 1));
  const bool full = std::fread(payload.data(), sizeof(float), payload.size(), f) == payload.size();
  const bool extra = full && std::fgetc(f) != EOF;
  std::fclose(f);
  if (!full || extra) return fail(DDF_ERR_BAD_WEIGHTS, "the checkpoint's size is wrong");
  if (crc32_update(0, payload.data(), payload.size() * sizeof(float)) != hd.crc)
    return fail(DDF_ERR_BAD_WEIGHTS, "the checkpoint's CRC-32 does not match");
  ddf_status s = ddf_load_weights(h, payload.data(), n);
  if (s != DDF_OK) return s;
  DeviceGuard g(h->cfg.device);
  if (opt) {  // the optimizer state, allocated if this handle has not trained yet
    s = h->cfg.kind == DDF_KIND_HASHGRID ? hg_ensure_train(h, 8) : ensure_train(h, 8);
    if (s != DDF_OK) return s;
    DDF_CK(cudaMemcpy(h->adam_m, payload.data() + n, n * sizeof(float), cudaMemcpyHostToDevice));
    DDF_CK(cudaMemcpy(h->adam_v, payload.data() + 2 * n, n * sizeof(float), cudaMemcpyHostToDevice));
    h->adam_step = hd.adam_step;
  } else if (h->adam_m != nullptr) {
    DDF_CK(cudaMemset(h->adam_m, 0, n * sizeof(float)));
    DDF_CK(cudaMemset(h->adam_v, 0, n * sizeof(float)));
    h->adam_step = 0;
  }
  return DDF_OK;
}

ddf_status ddf_reset_optimizer(ddf_handle h) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  if (h->adam_m == nullptr) return DDF_OK;
  DeviceGuard g(h->cfg.device);
  const size_t np = n_params(h);
  DDF_CK(cudaDeviceSynchronize());
  DDF_CK(cudaMemset(h->adam_m, 0, np * sizeof(float)));
  DDF_CK(cudaMemset(h->adam_v, 0, np * sizeof(float)));
  h->adam_step = 0;
  return DDF_OK;
}

ddf_status ddf_cast_scene(const float* spheres, int32_t n_spheres, const float* boxes,
                          int32_t n_boxes, const float* const rays[6], int64_t n, float* out_t,
                          uint8_t* out_hit, void* stream) {
  if (n_spheres < 0 || n_boxes < 0 || n_spheres > 1024 || n_boxes > 1024)
    return fail(DDF_ERR_INVALID_ARG, "0..1024 spheres and 0..1024 boxes");
  if ((n_spheres > 0 && spheres == nullptr) || (n_boxes > 0 && boxes == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "primitive array is NULL");
  ddf_status s = check_rays(rays, n);
  if (s != DDF_OK) return s;
  if (n > 0 && (out_t == nullptr || out_hit == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "output pointer is NULL");
  DDF_REQUIRE_ALIGNED(spheres, 4);
  DDF_REQUIRE_ALIGNED(boxes, 4);
  DDF_REQUIRE_ALIGNED(out_t, 4);
  ddf::RaySoA r;
  for (int c = 0; c < 6; ++c) r.p[c] = n > 0 ? rays[c] : nullptr;
  DDF_CK(ddf::launch_cast_scene(spheres, n_spheres, boxes, n_boxes, r, n, out_t, out_hit,
                                static_cast<cudaStream_t>(stream)));
  return DDF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The distillation schedule (Sec. 3.2 / 3.4) on the device.

extern "C" {

ddf_status ddf_sample_rays(const float* spheres, int32_t n_spheres, const float* boxes,
                           int32_t n_boxes, uint64_t seed, uint64_t step, int64_t n,
                           float surface_frac, float* const rays_out[6], void* stream) {
  if (n_spheres < 0 || n_boxes < 0 || n < 0) return fail(DDF_ERR_INVALID_ARG, "negative count");
  if (n_spheres > 1024 || n_boxes > 1024)
    return fail(DDF_ERR_INVALID_ARG, "at most 1024 spheres and 1024 boxes");
  if ((n_spheres > 0 && spheres == nullptr) || (n_boxes > 0 && boxes == nullptr))
    return fail(DDF_ERR_INVALID_ARG, "primitive array is NULL");
  if (!(surface_frac >= 0.f && surface_frac <= 1.f))
    return fail(DDF_ERR_INVALID_ARG, "surface_frac must be in [0, 1]");
  if (n == 0) return DDF_OK;
  if (rays_out == nullptr) return fail(DDF_ERR_INVALID_ARG, "rays_out is NULL");
  DDF_REQUIRE_ALIGNED(spheres, 4);
  DDF_REQUIRE_ALIGNED(boxes, 4);
  ddf::RayOut r;
  for (int c = 0; c < 6; ++c) {
    if (rays_out[c] == nullptr) return fail(DDF_ERR_INVALID_ARG, "a ray array is NULL");
    DDF_REQUIRE_ALIGNED(rays_out[c], 4);
    r.p[c] = rays_out[c];
  }
  DDF_CK(ddf::launch_sample_rays(spheres, n_spheres, boxes, n_boxes, seed, step, n, surface_frac, r,
                                 static_cast<cudaStream_t>(stream)));
  return DDF_OK;
}

ddf_status ddf_shift_rays(float* const rays[6], float* t, const uint8_t* hit, int64_t n,
                          int64_t first, uint64_t seed, uint64_t step, void* stream) {
  if (n < 0 || first < 0) return fail(DDF_ERR_INVALID_ARG, "negative count");
  if (first >= n) return DDF_OK;
  if (rays == nullptr || t == nullptr || hit == nullptr)
    return fail(DDF_ERR_INVALID_ARG, "NULL argument");
  DDF_REQUIRE_ALIGNED(t, 4);
  ddf::RayOut r;
  for (int c = 0; c < 6; ++c) {
    if (rays[c] == nullptr) return fail(DDF_ERR_INVALID_ARG, "a ray array is NULL");
    DDF_REQUIRE_ALIGNED(rays[c], 4);
    r.p[c] = rays[c];
  }
  DDF_CK(ddf::launch_shift_rays(r, t, hit, n, first, seed, step, static_cast<cudaStream_t>(stream)));
  return DDF_OK;
}

ddf_status ddf_distill(ddf_handle h, const float* spheres, int32_t n_spheres, const float* boxes,
                       int32_t n_boxes, int64_t steps, int64_t batch, float lr0,
                       float surface_frac, float shift_frac, uint64_t seed, float* losses,
                       void* stream) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  if (steps < 1 || !(lr0 > 0.f) || !(shift_frac >= 0.f && shift_frac <= 1.f))
    return fail(DDF_ERR_INVALID_ARG, "steps >= 1, lr0 > 0, shift_frac in [0, 1]");
  if (n_spheres > 1024 || n_boxes > 1024)
    return fail(DDF_ERR_INVALID_ARG, "at most 1024 spheres and 1024 boxes");
  DDF_REQUIRE_ALIGNED(spheres, 4);
  DDF_REQUIRE_ALIGNED(boxes, 4);
  DeviceGuard g(h->cfg.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* buf = nullptr;  // 6 ray arrays, targets, per-step losses
  uint8_t* hit = nullptr;
  DDF_CK(cudaMalloc(&buf, (7 * batch + steps) * sizeof(float)));
  if (cudaMalloc(&hit, batch) != cudaSuccess) {
    cudaFree(buf);
    return fail(DDF_ERR_OOM, "cudaMalloc of the hit flags failed");
  }
  float* rp[6];
  for (int c = 0; c < 6; ++c) rp[c] = buf + c * batch;
  float* t = buf + 6 * batch;
  float* dev_loss = buf + 7 * batch;
  const int64_t first = batch - static_cast<int64_t>(std::llround(shift_frac * batch));
  ddf_status s = DDF_OK;
  for (int64_t k = 0; k < steps && s == DDF_OK; ++k) {
    // cosine decay from lr0 to 5 % of it
    const double c = 0.5 * (1.0 + std::cos(3.14159265358979323846 * static_cast<double>(k) / steps));
    const float lr = static_cast<float>(lr0 * (0.05 + 0.95 * c));
    s = ddf_sample_rays(spheres, n_spheres, boxes, n_boxes, seed, static_cast<uint64_t>(k), batch,
                        surface_frac, rp, st);
    const float* const rc[6] = {rp[0], rp[1], rp[2], rp[3], rp[4], rp[5]};
    if (s == DDF_OK) s = ddf_cast_scene(spheres, n_spheres, boxes, n_boxes, rc, batch, t, hit, st);
    if (s == DDF_OK) s = ddf_shift_rays(rp, t, hit, batch, first, seed, static_cast<uint64_t>(k), st);
    if (s == DDF_OK) s = ddf_train_step(h, rc, t, hit, batch, lr, dev_loss + k, st);
  }
  if (s == DDF_OK && losses != nullptr) {
    const cudaError_t e = cudaMemcpyAsync(losses, dev_loss, steps * sizeof(float),
                                          cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync");
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(hit);
  if (s == DDF_OK && e != cudaSuccess) s = cuda_fail(e, "cudaStreamSynchronize");
  return s;
}

ddf_status ddf_distill_pool(ddf_handle h, const float* const pool[6], const float* pool_t,
                            const uint8_t* pool_hit, int64_t n_pool, int64_t steps,
                            int64_t batch, float lr0, float shift_frac, uint64_t seed,
                            float* losses, void* stream) {
  if (h == nullptr) return fail(DDF_ERR_INVALID_ARG, "handle is NULL");
  if (steps < 1 || !(lr0 > 0.f) || !(shift_frac >= 0.f && shift_frac <= 1.f))
    return fail(DDF_ERR_INVALID_ARG, "steps >= 1, lr0 > 0, shift_frac in [0, 1]");
  if (n_pool < 1 || n_pool > (int64_t{1} << 31))
    return fail(DDF_ERR_INVALID_ARG, "n_pool must be in [1, 2^31]");
  if (pool == nullptr || pool_t == nullptr || pool_hit == nullptr)
    return fail(DDF_ERR_INVALID_ARG, "pool arrays are NULL");
  ddf::RaySoA ps;
  for (int c = 0; c < 6; ++c) {
    if (pool[c] == nullptr) return fail(DDF_ERR_INVALID_ARG, "a pool ray array is NULL");
    DDF_REQUIRE_ALIGNED(pool[c], 4);
    ps.p[c] = pool[c];
  }
  DDF_REQUIRE_ALIGNED(pool_t, 4);
  if (batch < 1) return fail(DDF_ERR_INVALID_ARG, "batch must be >= 1");
  DeviceGuard g(h->cfg.device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* buf = nullptr;  // 6 ray arrays, targets, per-step losses
  uint8_t* hit = nullptr;
  DDF_CK(cudaMalloc(&buf, (7 * batch + steps) * sizeof(float)));
  if (cudaMalloc(&hit, batch) != cudaSuccess) {
    cudaFree(buf);
    return fail(DDF_ERR_OOM, "cudaMalloc of the hit flags failed");
  }
  ddf::RayOut ro;
  for (int c = 0; c < 6; ++c) ro.p[c] = buf + c * batch;
  float* t = buf + 6 * batch;
  float* dev_loss = buf + 7 * batch;
  const int64_t first = batch - static_cast<int64_t>(std::llround(shift_frac * batch));
  ddf_status s = DDF_OK;
  for (int64_t k = 0; k < steps && s == DDF_OK; ++k) {
    const double c = 0.5 * (1.0 + std::cos(3.14159265358979323846 * static_cast<double>(k) / steps));
    const float lr = static_cast<float>(lr0 * (0.05 + 0.95 * c));
    const cudaError_t e = ddf::launch_pool_gather(ps, pool_t, pool_hit, n_pool, seed,
                                                  static_cast<uint64_t>(k), batch, ro, t, hit, st);
    if (e != cudaSuccess) s = cuda_fail(e, "pool gather");
    const float* const rc[6] = {ro.p[0], ro.p[1], ro.p[2], ro.p[3], ro.p[4], ro.p[5]};
    if (s == DDF_OK) s = ddf_shift_rays(ro.p, t, hit, batch, first, seed, static_cast<uint64_t>(k), st);
    if (s == DDF_OK) s = ddf_train_step(h, rc, t, hit, batch, lr, dev_loss + k, st);
  }
  if (s == DDF_OK && losses != nullptr) {
    const cudaError_t e = cudaMemcpyAsync(losses, dev_loss, steps * sizeof(float),
                                          cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync");
  }
  const cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaFree(hit);
  if (s == DDF_OK && e != cudaSuccess) s = cuda_fail(e, "cudaStreamSynchronize");
  return s;
}

}  // extern "C"

