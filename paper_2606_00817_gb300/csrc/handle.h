// handle.h -- internal: the library handle (struct ddf_s) and the host-side
// helpers shared by the query runtime (ddf_api.cpp) and the training runtime
// (train_api.cpp). Not part of the public interface (include/ddf.h).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ddf.h"
#include "kernels.h"

struct ddf_s {
  ddf_config cfg{};
  // hash-grid field (kind DDF_KIND_HASHGRID): level layout, the level tables
  // (bf16x2 or float2 entries), the swizzled MLP operand images, FP32 biases
  // and head, and the query grid (CTAs) of the tensor-core kernel
  ddf::HashGridParams hg{};
  int64_t hg_entries = 0;
  void* hg_table = nullptr;
  uint8_t* hg_img = nullptr;
  float* hg_bias = nullptr;
  int hg_grid = 0;
  ddf::HashGridParams hg_blob{};  // the master blob's (unpadded) level layout
  int64_t hg_blob_entries = 0;
  float* hg_code = nullptr;   // training: [B x 64] codes
  float* hg_acts = nullptr;   // training: [H x B x 64] hidden activations
  float* hg_dpre = nullptr;   // training: [H x B x 64] dL/d(pre-activation)
  int d_in = 0;
  int kp32 = 0;  // padded encoded width, FP32 rows (multiple of 8)
  int kp16 = 0;  // padded encoded width, bf16 rows (multiple of 8 -> 16-byte rows)
  int bn = 0;    // tensor-core N tile (= tile.bn)
  ddf::TcTile tile{256, 4};        // layers 2..H
  ddf::TcTile tile_first{256, 4};  // layer 1
  int pair_clusters = 0;  // co-resident clusters of the CTA-pair kernel
  int num_sms = 0;
  bool loaded = false;
  bool scales_set = false;
  uint64_t timeout_ns = 2000000000ull;
  int64_t chunk = 1 << 20;

  std::vector<void*> owned;  // device allocations freed by ddf_destroy
  float* d_blob = nullptr;   // FP32 master weights
  std::vector<float*> wf;    // FP32: padded W per hidden layer
  std::vector<float*> bias;  // per hidden layer [W]
  std::vector<__nv_bfloat16*> wb;  // bf16 W (all layers for BF16, layer 1 for FP8)
  std::vector<uint8_t*> wq;        // FP8: e4m3 codes for layers 2..H
  std::vector<float*> wscale;      // FP8: per-output-channel scales
  std::vector<float*> colscale;    // FP8: s_{l-1} * wscale_l
  std::vector<float> act_scales;
  std::vector<CUtensorMap> tmB;
  std::vector<__nv_bfloat16*> wcal;  // FP8: bf16 copies of layers 2..H for calibration
  std::vector<CUtensorMap> tmBcal;   // FP8: maps of the bf16 weights, calibration tile

  // CUDA-graph replay of queries (ddf_set_graph_mode)
  bool graph_mode = false;
  cudaStream_t s_graph = nullptr;
  struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  float* ao_vis = nullptr;    // AO: per-ray visibility and hit flags
  uint8_t* ao_hit = nullptr;
  int64_t ao_rows = 0;
  float* head_w = nullptr;  // [2 x W]
  float* head_b = nullptr;  // [2]

  int64_t ws_rows = 0;
  void* ws_enc = nullptr;
  void* ws_act[2] = {nullptr, nullptr};
  float2* ws_part = nullptr;

  uint32_t* status_dev = nullptr;

  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;

  // host-buffer pipeline
  cudaStream_t s_copy = nullptr, s_comp = nullptr;
  float* hp_rays[2][6] = {};
  float* hp_t[2] = {};
  float* hp_v[2] = {};
  uint8_t* hp_occ[2] = {};
  int64_t hp_rows = 0;
  cudaEvent_t ev_in[2] = {}, ev_comp[2] = {};

  // distillation step (train_api.cpp)
  int64_t tr_rows = 0;
  void* tr_enc = nullptr;                 // [B x kp16] bf16
  std::vector<void*> tr_h;                // per layer [B x W] bf16 activations (views)
  std::vector<void*> tr_store;            // the activation buffers tr_h points into
  int tr_segment = 1;                     // checkpointing: keep every k-th layer (1: all)
  void* tr_dpre[2] = {nullptr, nullptr};  // [B x W] bf16 pre-activation gradients
  float* tr_part = nullptr;               // split-K partials of a weight gradient, two sets
  size_t tr_part_set = 0;                 // floats per set of tr_part
  size_t tr_colpart_set = 0;              // floats per set of tr_colpart
  cudaStream_t s_red = nullptr;           // the gradient reductions, beside the GEMMs
  cudaEvent_t ev_gemm[2] = {};            // a weight-gradient GEMM of buffer set b done
  cudaEvent_t ev_red[2] = {};             // the reduction reading buffer set b done
  cudaEvent_t ev_join = nullptr;          // every reduction of a backward pass done
  float* tr_cpart = nullptr;              // row-split partials of column sums
  float* tr_hpart = nullptr;              // [512 x (3 W + 4)] partials of the head's backward
  unsigned* tr_ticket = nullptr;          // zeroed counters of the column-sum reductions
  float2* tr_z = nullptr;
  float2* tr_dz = nullptr;
  unsigned* tr_nhit = nullptr;
  float* tr_lpart = nullptr;              // per-block loss partials
  float* tr_colpart = nullptr;            // 2 x [B / 32 x W] column sums of an input gradient
  float2* tr_hz = nullptr;                // [W / 256 x B] head partials of the last layer
  float* grad = nullptr;                  // gradient blob (weight-blob layout)
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int64_t adam_step = 0;
  bool grad_valid = false;
  // rows of the last ddf_forward_train whose activations are still kept for
  // ddf_backward (0: none; cleared by anything that changes weights or reuses
  // the training buffers)
  int64_t fwd_rows = 0;
  ddf::RaySoA fwd_rays{};  // the inputs of that forward (a hash grid's backward re-reads them)
  std::vector<__nv_bfloat16*> wt;         // layers 2..H: bf16 W^T [K x W] for input gradients
  std::vector<CUtensorMap> tmBtr;         // weight maps for the plain 1-CTA tile {bn, 4}
  std::vector<CUtensorMap> tmWT;          // maps of wt
  // CTA-pair training GEMMs (width a multiple of 256): weight maps with
  // 128-row boxes, for the forward (W_l) and the input gradients (W_l^T)
  bool tr_pair = false;
  std::vector<CUtensorMap> tmBpair, tmWTpair;

  // sphere tracing (SDF fields)
  int* trc_idx[2] = {nullptr, nullptr};   // active-ray lists
  int* trc_count = nullptr;               // [2] active counts
  int* trc_steps = nullptr;               // per-ray evaluations
  int64_t trc_rows = 0;
};

namespace ddfi {

#define DDF_CK(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

ddf_status fail(ddf_status s, const std::string& msg);
ddf_status cuda_fail(cudaError_t e, const char* what);

// A device pointer that the kernels access a bytes at a time must be a-byte
// aligned: a misaligned one would fault the GPU, so it is refused here.
#define DDF_REQUIRE_ALIGNED(ptr, a)                                                   \
  do {                                                                                \
    if ((ptr) != nullptr && reinterpret_cast<uintptr_t>(ptr) % (a) != 0)              \
      return ::ddfi::fail(DDF_ERR_INVALID_ARG, #ptr " must be " #a "-byte aligned"); \
  } while (0)

// Restores the caller's current device when it goes out of scope.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

constexpr int kProfClasses = 4;
enum ProfClass { kProfEncode = 0, kProfGemm = 1, kProfHead = 2, kProfFirst = 3 };

cudaEvent_t prof_event(ddf_s* h);

// Brackets one launch with CUDA events when the handle's profiling is on.
struct ProfScope {
  ddf_s* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(ddf_s* h_, int cls_, cudaStream_t s_) : h(h_), cls(cls_), s(s_) {
    if (h->prof && (a = prof_event(h)) != nullptr) cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (a == nullptr) return;
    cudaEvent_t b = prof_event(h);
    if (b == nullptr) return;
    cudaEventRecord(b, s);
    h->recs.push_back({cls, a, b});
  }
};

bool make_tmap(CUtensorMap* m, const void* base, bool one_byte, uint64_t inner, uint64_t rows,
               uint64_t row_bytes, uint32_t box_rows);
ddf_status dev_alloc(ddf_s* h, void** p, size_t bytes);
void dev_free(ddf_s* h, void* p);
ddf_status check_rays(const float* const rays[6], int64_t n);
ddf_status ensure_workspace(ddf_s* h, int64_t rows);
void clear_graphs(ddf_s* h);
ddf::RaySoA shift_rays(ddf::RaySoA r, int64_t off);
// Builds h->tmBtr (bf16 weight maps for the plain 1-CTA tile) once.
ddf_status ensure_plain_maps(ddf_s* h);
int64_t round_up(int64_t x, int64_t m);
// Pinhole basis of a camera given as eye[3], target[3], up[3], fov_y.
ddf_status camera_basis(const float camera[10], int32_t width, int32_t height,
                        ddf::GiCamera* cam);

// Distillation loss and optimiser constants (Sec. 3.2 / 3.4): L1 clamp at
// the box scale, cross-entropy weight 0.3, Adam (0.9, 0.999, 1e-8).
constexpr float kLossClamp = 4.0f;
constexpr float kLossLambda = 0.3f;
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;

// hash-grid field (hashgrid_api.cpp)
// Level layout; even_offsets pads each level to start on an even entry.
ddf::HashGridParams hg_layout(int64_t* entries, bool even_offsets);
size_t hg_param_count(const ddf_config& c);
ddf_status hg_load(ddf_s* h, const float* host_blob);
ddf_status hg_query(ddf_s* h, ddf::RaySoA rays, int64_t n, ddf::HeadOut out, cudaStream_t st);
// Training (FP32 on the master blob): forward keeping the code and every
// activation (z into tr_z), backward from tr_dz into h->grad, and the whole
// step (loss, gradient, optional Adam with lr > 0 and the bf16 refresh).
ddf_status hg_forward_keep(ddf_s* h, ddf::RaySoA rays, int B, cudaStream_t st);
ddf_status hg_backward(ddf_s* h, ddf::RaySoA rays, int B, cudaStream_t st);
ddf_status hg_train(ddf_s* h, ddf::RaySoA rays, const float* t_target, const uint8_t* hit_target,
                    int B, float lr, float* out_loss, cudaStream_t st);
ddf_status hg_ensure_train(ddf_s* h, int64_t B);
// Rewrites a bf16 field's query copies from the FP32 master blob (on st).
ddf_status hg_refresh(ddf_s* h, cudaStream_t st, bool tables_too = true);

}  // namespace ddfi
