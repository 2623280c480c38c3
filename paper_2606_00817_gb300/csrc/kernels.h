// kernels.h -- host-side launchers of the DDF device kernels (internal to
// libddf.so; the public interface is include/ddf.h).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ddf {

// Structure-of-arrays ray pointers (ox, oy, oz, dx, dy, dz). One batch may
// join two sets of arrays (the mixed shadow + ambient-occlusion query): rows
// below `split` read p at the row, rows from `split` on read q at row - split.
// The default split (INT64_MAX) reads p only; kernels that take rays from q
// read them through ray_ld (heads.cuh).
struct RaySoA {
  const float* p[6];
  const float* q[6] = {};
  int64_t split = INT64_MAX;
};
struct RayOut {
  float* p[6];
};

// One dense layer y = act(scale_n * (A W^T)_n + b_n) on the tcgen05 tensor cores.
// A: [M x K] activations (bf16 or e4m3 codes), W: [N x K], both K-major and
// read through TMA tensor maps. mode 0 stores ReLU(y) * out_scale as the next
// layer's activation; mode 1 (the last hidden layer) instead folds ReLU(y)
// into the 2-row FP32 head and writes one (z0, z1) partial per N-block and row.
struct TcGemmParams {
  int M, N, K;
  const float* bias;       // [N]
  const float* col_scale;  // [N] or nullptr (e4m3 inputs: s_in * s_w[n])
  float out_scale;         // multiplier before the e4m3 output cast (1/s_out)
  void* out;               // mode 0: [M x ldo] bf16 or e4m3 codes
  int ldo;                 // elements
  const float* head_w;     // mode 1: [2 x N] FP32
  float2* head_part;       // mode 1: [(N/BN) * (epi_warps/4) x M]
  int mode;
  uint32_t* status;        // device status word (timeouts)
  uint64_t timeout_ns;
  float* amax;             // mode 0, nullable: running max of the layer's outputs
                           // (rows < M), for activation-scale calibration
  // training modes:
  //   mode 2: out = bf16(acc masked by mask > 0), mask bf16 [M x ldm]
  //           (the activation whose ReLU the gradient passes back through)
  //   mode 3: out_f32[split][M x ldo] = acc, k_splits splits of the K range
  const void* mask;
  int ldm;
  int k_splits;
  size_t split_stride;     // elements between split outputs
  float* out_f32;
  // 1-CTA kernel, nullable: device int holding the number of rows to compute
  // (at most M; M remains the row stride of the head partials)
  const int* m_dev;
  // 1-CTA kernel, bf16: both operands stored MN-major, A as [K x M] and B as
  // [K x N] row-major (M / N index contiguous), their maps built with
  // 64 x 64 boxes; lets dW = dZ^T X read dZ [B x W] and X [B x K] as stored
  int mn_major;
  // training on the pair kernel: mode 4 is mode 0 for the last layer, with
  // the head partials of mode 1 taken from the stored bf16 outputs; mode 2
  // also writes per 32-row block column sums of its output into
  // col_part [ceil(M / 32) x ldo] FP32 (nullable)
  float* col_part;
  // pair kernel, staged query tile (mode 0): 1 = the outputs leave shared
  // memory by TMA tensor stores through the output map the launcher takes
  // (box 32 rows x 128 bytes), 0 = by 16-byte stores of the epilogue threads
  int tma_out;
};

// ---- sphere tracing of an SDF field (trace.cu) ----
// 3D Fourier encoding of points p [M x ld] bf16: p, then per coordinate and
// band sin(pi 2^k p_c), cos(pi 2^k p_c); zero padding to ld.
cudaError_t launch_encode_points_bf16(const float* px, const float* py, const float* pz, int64_t M,
                                      int L, int ld, __nv_bfloat16* out, cudaStream_t s);
// Same for the active rays of a trace: row j encodes o_i + t_i d_i with
// i = idx[j], for j < *count (rows up to cap written, extra rows untouched).
cudaError_t launch_trace_encode(RaySoA rays, const float* t, const int* idx, const int* count,
                                int cap, int L, int ld, __nv_bfloat16* out, cudaStream_t s);
// idx = 0..n-1, count = n, t = 0, steps = 0, hit = 0
cudaError_t launch_trace_init(int n, int* idx, int* count, float* t, int* steps, uint8_t* hit,
                              cudaStream_t s);
// One sphere-tracing step for the active rays: s = sum of nparts head
// partials [nparts x cap] + head_b[0]; steps += 1; s < eps -> hit; else
// t += s and the ray stays active (appended to idx_out / count_out) unless
// t > t_max or it has used max_steps evaluations.
cudaError_t launch_trace_update(const float2* part, int nparts, int cap, const int* count_in,
                                const int* idx_in, const float* head_b, float eps, float t_max,
                                int max_steps, float* t, int* steps, uint8_t* hit, int* idx_out,
                                int* count_out, cudaStream_t s);
// Closed-form signed distance to a union of spheres and boxes at n points.
cudaError_t launch_union_sdf(const float* spheres, int ns, const float* boxes, int nb,
                             const float* px, const float* py, const float* pz, int64_t n,
                             float* out, cudaStream_t s);
// SDF regression loss: L = mean |z0 - s*|, dz = (sign(z0 - s*) / B, 0).
cudaError_t launch_sdf_loss(const float2* z, const float* s_tgt, int64_t B, float2* dz,
                            float* part, float* loss_out, cudaStream_t s);

// Tile configuration of the tensor-core layer: N tile (128 or 256) and the
// number of epilogue warps (4, or 8 = two warps per TMEM lane quarter, each
// draining half of the columns). Mode 1 writes (N/bn) * (epi_warps/4) partials
// per row.
struct TcTile {
  int bn;
  int epi_warps;
  bool pair = false;    // 256 x 256 tile on a 2-CTA cluster (tc_gemm_pair.cu; bn 256, 4 warps)
  bool staged = false;  // pair tile, or the fused layer-1 tile: outputs staged through shared memory
  bool fused = false;   // layer 1 only: the encoding is built in shared memory (tc_layer1.cu)
};

// Layer 1 with the ray encoding computed inside the kernel (tc_layer1.cu):
// mode-0 output (bf16, or e4m3 after out_scale) of ReLU(enc(rays) W_1^T + b)
// for p.M rays, N % 256 == 0, 6 + 12 L <= 128; p.K is not used. tmO maps
// p.out [M x N] with 128-byte-swizzled boxes of 128 bytes x 32 rows.
bool tc_layer1_supported(int L, int N);
cudaError_t launch_tc_layer1(int epi_warps, bool out_fp8, const CUtensorMap& tmB,
                             const CUtensorMap& tmO, RaySoA rays, int L, const TcGemmParams& p,
                             int grid, cudaStream_t s);

// in_fp8: operands are e4m3 codes (kind::f8f6f4) instead of bf16 (kind::f16).
// out_fp8: mode-0 output is e4m3 codes instead of bf16.
cudaError_t launch_tc_gemm(const TcTile& tile, bool in_fp8, bool out_fp8, const CUtensorMap& tmA,
                           const CUtensorMap& tmB, const TcGemmParams& p, int grid,
                           cudaStream_t s);
int tc_gemm_smem_bytes(int bn, bool in_fp8);

// CTA-pair variant: clusters of 2 CTAs, 256 x 256 output tiles, persistent
// over `clusters` clusters, 4 or 8 epilogue warps per CTA (training modes
// 2-4: kTrainEpiWarps, whatever epi_warps says). Modes 1 and 4 write
// (N/256) (epi_warps/4) head partials per row; modes 2 and 3 (bf16) as the
// 1-CTA kernel, mode 2 through the staging buffers, mode 3 with K-major or
// MN-major operands.
constexpr int kTrainEpiWarps = 4;
// tmO: the output map when p.tma_out is set (the staged mode-0 tile), else
// nullptr.
cudaError_t launch_tc_gemm_pair(bool in_fp8, bool out_fp8, bool staged, int epi_warps,
                                const CUtensorMap& tmA, const CUtensorMap& tmB,
                                const TcGemmParams& p, int clusters, cudaStream_t s,
                                const CUtensorMap* tmO = nullptr);
// Clusters of the pair kernel that fit on the current device at once.
int tc_gemm_pair_max_clusters(bool in_fp8);

// Sinusoidal encoding of M rays into a row-major [M x ld] matrix (ld >= 6+12L,
// columns past 6+12L are zero).
cudaError_t launch_encode_bf16(RaySoA rays, int64_t M, int L, int ld, __nv_bfloat16* out,
                               cudaStream_t s);
cudaError_t launch_encode_f32(RaySoA rays, int64_t M, int L, int ld, float* out, cudaStream_t s);

// FP32 CUDA-core layer: C[M x N] = ReLU(A[M x K] W[N x K]^T + b), K % 8 == 0.
cudaError_t launch_sgemm_relu(const float* A, const float* W, const float* b, float* C, int M,
                              int N, int K, cudaStream_t s);

// Heads: z = Wo h + bo, t = softplus(z0), vis = sigmoid(z1), optional shadow.
struct HeadOut {
  float* t;           // nullable
  float* vis;         // nullable
  uint8_t* hit;       // nullable: 1 where z1 > 0
  float* z0;          // nullable: raw z0 (the value of an SDF field)
  uint8_t* occluded;  // nullptr unless a shadow query
  float light[3];
  RaySoA rays;        // origins for the shadow distance
  // Rows from `split` on (the ambient-occlusion part of a mixed query) write
  // only vis2 / hit2 (nullable), at row - split, instead of the outputs above.
  float* vis2 = nullptr;
  uint8_t* hit2 = nullptr;
  int64_t split = INT64_MAX;
};
// From FP32 activations H [M x W] (FP32 path).
cudaError_t launch_head_f32(const float* H, int M, int W, const float* wo, const float* bo,
                            HeadOut o, cudaStream_t s);
// From per-N-block partial dot products [nblk x M] (tensor-core path).
cudaError_t launch_finish_heads(const float2* part, int nblk, int M, const float* bo, HeadOut o,
                                cudaStream_t s);

// ---- the hash-grid field (hashgrid.cu) ----
// Level layout of the multiresolution hash grid (Sec. 3.4): per level the
// cells per axis, whether every vertex has its own entry (dense row-major
// index) or the spatial hash picks one (mod mask + 1), and the first entry.
struct HashGridParams {
  int res[16];
  int dense[16];
  uint32_t offset[16];
  uint32_t mask;
};
// Tensor-core query: table = bf16x2 entries, w_img = H swizzled 64 x 64 bf16
// operand images (layer 1 zero-padded from 59 inputs), bias [H x 64], head_w
// [2 x 64], head_b [2] FP32. grid = CTAs (each loops over 128-ray tiles).
cudaError_t launch_hashgrid_tc(const HashGridParams& g, const uint32_t* table,
                               const uint8_t* w_img, const float* bias, const float* head_w,
                               const float* head_b, int H, RaySoA rays, int64_t M, HeadOut out,
                               uint32_t* status, uint64_t timeout_ns, int grid, cudaStream_t s);
int hashgrid_tc_blocks_per_sm(int H);
int hashgrid_smem_bytes(int H);
// FP32 query: table = (f0, f1) float pairs, mlp = the blob's MLP part.
cudaError_t launch_hashgrid_f32(const HashGridParams& g, const float2* table, const float* mlp,
                                int H, RaySoA rays, int64_t M, HeadOut out, cudaStream_t s);
// FP32 table (blob layout `from`) -> bf16x2 entries in the layout `to`.
cudaError_t launch_hg_pack_table(const float* src, int64_t n_entries, const HashGridParams& from,
                                 const HashGridParams& to, uint32_t* dst, cudaStream_t s);
// Training (FP32): forward storing code [64 x B], activations [H x 64 x B]
// (feature-major) and z; backward from dz storing dL/dpre [H x 64 x B] and
// scattering the hash features' gradient into grad_table (blob layout,
// atomic adds); part[s][n][k] = sum over split s of P(r, n) A(r, k) and
// bpart[s][n] = sum of P(r, n) (n < np <= 64, k < na <= 64), with element
// (r, c) of P at P[r prs + c pcs] and of A at A[r ars + c acs].
cudaError_t launch_hg_train_fwd(const HashGridParams& g, const float2* table, const float* mlp,
                                int H, RaySoA rays, int64_t B, float* code, float* acts,
                                float2* z, cudaStream_t s);
cudaError_t launch_hg_train_bwd(const HashGridParams& g, const float* mlp, int H, RaySoA rays,
                                int64_t B, const float* acts, const float2* dz, float* dpre,
                                float* grad_table, cudaStream_t s);
struct HgOuterJob {
  const float* P;
  int64_t prs, pcs;
  int np;
  const float* A;
  int64_t ars, acs;
  int na;
  float* part;
  float* bpart;
};
constexpr int kHgOuterJobs = 5;  // up to 4 hidden layers and the head
struct HgOuterJobs {
  HgOuterJob job[kHgOuterJobs];
  int n;
};
// Every job of `jobs` in one launch (splits blocks per job).
cudaError_t launch_hg_outer_tiled(const HgOuterJobs& jobs, int64_t B, int splits, cudaStream_t s);
cudaError_t launch_hg_pack_image(const float* w, int K, uint8_t* img, cudaStream_t s);

// Ambient occlusion (Sec. 3.3): for point p with rays [offsets[p], offsets[p+1])
// hard[p] = 1 - mean(hit), soft[p] = 1 - mean(vis); empty sets give 1.
cudaError_t launch_ao_reduce(const uint8_t* hit, const float* vis, const int32_t* offsets,
                             int64_t n_points, float* hard, float* soft, cudaStream_t s);

// ---- distillation step (train.cu) ----
// z[r] = (Wo h_r + bo) from bf16 rows H [M x W]
cudaError_t launch_head_train(const __nv_bfloat16* H, int M, int W, const float* wo,
                              const float* bo, float2* z, cudaStream_t s);
// Loss of Sec. 3.2 / 3.4 and dL/dz: L1 on min(softplus(z0), clamp) against
// min(t*, clamp) over hit rays / max(1, N_hit), plus lam x BCE(z1, y) / B.
// part: ceil(B/256) floats of scratch; loss_out nullable (device scalar).
cudaError_t launch_loss(const float2* z, const float* t_tgt, const uint8_t* y, int64_t B,
                        unsigned* nhit, float clamp, float lam, float2* dz, float* part,
                        float* loss_out, cudaStream_t s);
// One pass over H [M x W]: dpre = bf16((dz wo) where H > 0), and per split
// of rows part [splits x (3 W + 4)]: partials of dz0 H, dz1 H, of dpre's
// column sums and of dz0, dz1 (each summed over the split's rows in order;
// the last two columns of a row are padding and are not written).
cudaError_t launch_head_back_fused(const float2* dz, const __nv_bfloat16* H, int M, int W,
                                  const float* wo, int splits, __nv_bfloat16* dpre, float* part,
                                  cudaStream_t s);

// Gradient reductions in one launch, every sum in a fixed order (the same
// bits whichever block finishes first).
// Split sum: out[r ldo + c] = part[0][r][c] + part[1][r][c] + ... (S terms,
// in split order), r < rows, c < cols, part[q][r][c] at q split_stride +
// r ldp + c.
struct RedSplit {
  const float* part = nullptr;
  int64_t split_stride = 0;
  int S = 0, rows = 0, cols = 0, ldp = 0, ldo = 0;
  float* out = nullptr;
  int vec = 0;  // set by the launcher: float4 loads and stores
};
// Column sums of X [M x N] (FP32, or bf16 with x_bf16), row stride ld: the
// rows split R ways ([j rps, (j + 1) rps), rps = ceil(M / R)); split j's sum
// of column c is ((S0 + S1) + S2) + S3 with S_p the sum, in row order, of
// its rows r0 + p, r0 + p + 4, ...; it goes to cpart[j ldc + c] (ldc >= N
// rounded up to 4, a multiple of 4; cpart 16-byte aligned); the column's sum
// is the same phase split over the R partials. Column c is written to
// out[k][c - c0[k]] for each segment k holding it. ticket: one counter per
// 256 columns, zero before the launch and after it. X is read 4 columns at a
// time: ld must be a multiple of 4 and at least N rounded up to 4 (the
// padding is read, never written out), X 16-byte aligned (8 for bf16).
constexpr int kRedSegs = 3;
constexpr int kRedTickets = 128;
struct RedCols {
  const void* X = nullptr;  // null: no column sum
  int x_bf16 = 0, M = 0, N = 0, ld = 0, R = 1, ldc = 0;
  float* cpart = nullptr;
  unsigned* ticket = nullptr;
  int nseg = 0;
  int c0[kRedSegs] = {}, cnt[kRedSegs] = {};
  float* out[kRedSegs] = {};
};
constexpr int kRedJobs = 8;
struct GradReduce {
  int nsplit = 0;
  RedSplit split[kRedJobs];
  RedCols cols;
  int blk0[kRedJobs + 1] = {};  // block offsets of the split jobs (set by the launcher)
};
cudaError_t launch_grad_reduce(const GradReduce& g, cudaStream_t s);
// Adam (Kingma & Ba, bias-corrected with bc1 = 1 - b1^t, bc2 = 1 - b2^t, no
// weight decay) on n parameters: m, v and w updated in place.
cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s);
// Adam over the first `entries` feature pairs of a hash-grid blob (its level
// tables, layout `from`) and their bf16x2 copy in the padded layout `to`
// (dst), in one pass; the same arithmetic as launch_adam.
cudaError_t launch_hg_adam_pack(float* w, const float* g, float* m, float* v, int64_t entries,
                                float lr, float b1, float b2, float eps, float bc1, float bc2,
                                const HashGridParams& from, const HashGridParams& to,
                                uint32_t* dst, cudaStream_t s);
// z[r] = (sum over p < nparts of part[p][r]) + bo, for the two head rows.
cudaError_t launch_head_sum(const float2* part, int nparts, int64_t M, const float* bo, float2* z,
                            cudaStream_t s);
// Adam as above, and in the same pass every copy of the updated weights the
// next step reads: block j of the blob covers [start, start + rows x cols)
// (the blocks tile [0, n) in order); a weight block also writes bf16 rows to
// wb (row stride ldb) and, when wt is set (16-byte aligned), the bf16
// transpose to wt ([cols x rows]); a vector block (rows 1) copies to f32
// (FP32). At most kAdamBlocks blocks.
constexpr int kAdamBlocks = 24;
struct AdamBlock {
  int64_t start;
  int rows, cols, ldb;
  __nv_bfloat16* wb;
  __nv_bfloat16* wt;
  float* f32;
  int cta0 = 0;  // first CTA of the block (set by the launcher)
  int vec = 0;   // set by the launcher: a weight block updated 4 columns at a time
};
struct AdamBlocks {
  int n;
  AdamBlock b[kAdamBlocks];
};
cudaError_t launch_adam_refresh(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                                float b1, float b2, float eps, float bc1, float bc2,
                                const AdamBlocks& blocks, cudaStream_t s);
// dst [K x N] = bf16(src [N x K])^T
cudaError_t launch_pack_bf16_t(const float* src, int N, int K, __nv_bfloat16* dst, cudaStream_t s);
cudaError_t launch_cast_scene(const float* spheres, int ns, const float* boxes, int nb,
                              RaySoA rays, int64_t n, float* t_out, uint8_t* hit_out,
                              cudaStream_t s);

// Weight preparation (load time).
// dst[N x ldd] = src[N x K] zero-padded to ldd columns.
cudaError_t launch_pack_f32(const float* src, int N, int K, int ldd, float* dst, cudaStream_t s);
cudaError_t launch_pack_bf16(const float* src, int N, int K, int ldd, __nv_bfloat16* dst,
                             cudaStream_t s);
// Per-output-channel e4m3: scale[n] = amax_n / 448, codes = e4m3(src / scale[n]).
cudaError_t launch_quant_e4m3(const float* src, int N, int K, int ldd, uint8_t* dst, float* scale,
                              cudaStream_t s);
// out[n] = a * v[n]
cudaError_t launch_scale_vec(const float* v, float a, int n, float* out, cudaStream_t s);

// ---- distillation sampling (distill.cu) ----
// n rays: a fraction surface_frac anchored on the scene's surface (a point
// uniform by area, 1e-3 off it along the normal, direction uniform on the
// sphere), the rest camera rays from a face of [-1,1]^3 toward a point of
// [-0.9,0.9]^3. Counter-based: (seed, step, i) fixes ray i. At most
// kMaxPrims spheres and kMaxPrims boxes.
cudaError_t launch_sample_rays(const float* spheres, int ns, const float* boxes, int nb,
                               uint64_t seed, uint64_t step, int64_t n, float surface_frac,
                               RayOut r, cudaStream_t s);
// Rays first..n-1 that hit move forward by s = u t (u uniform in [0,1)) and
// their target becomes t - s.
cudaError_t launch_shift_rays(RayOut r, float* t, const uint8_t* hit, int64_t n, int64_t first,
                              uint64_t seed, uint64_t step, cudaStream_t s);

// ---- shadow / AO images (gi.cu) ----
// Pinhole camera: eye, unit forward f, right r, up u, tan(fov_y / 2).
struct GiCamera {
  float eye[3], f[3], r[3], u[3];
  float tan_half;
  int width, height;
};
// Per pixel the exact primary hit: shading point (xyz, w = 1 hit / 0 none)
// 1e-3 off the surface along the normal, and the normal [3 per pixel] facing
// the eye.
cudaError_t launch_gi_primary(const GiCamera& cam, const float* spheres, int ns, const float* boxes,
                              int nb, float4* sp, float* nrm, cudaStream_t s);
// (1 + k) rays per pixel: toward the light, then k cosine-weighted ones.
cudaError_t launch_gi_rays(const float4* sp, const float* nrm, int64_t npx, int k, uint64_t seed,
                           const float light[3], RayOut r, cudaStream_t s);
// Images from the secondary rays' t and hit flags (background -1).
cudaError_t launch_gi_compose(const float4* sp, int64_t npx, int k, const float light[3],
                              const float* t, const uint8_t* hit, float* shadow, float* ao,
                              cudaStream_t s);

// ---- Gaussian-rendered depth (gs.cu) ----
// Tiles of 16 pixels along an image extent.
int gs_tiles(int extent);
// Per (view, Gaussian): screen record rec[2 j], rec[2 j + 1] (pixel mean,
// depth, opacity; inverse screen covariance), tile rectangle rect[j] (empty:
// z < x), and +1 on the count of each tile in it (count zeroed by the caller,
// nv x ntx x nty entries, view-major).
cudaError_t launch_gs_project(const float* means, const float* covs, const float* opac, int64_t n,
                              const GiCamera* cams, int nv, int ntx, int nty, float4* rec,
                              int4* rect, unsigned* count, cudaStream_t s);
// Exclusive scan of n counts into off[0..n], off[n] the total (one block).
cudaError_t launch_gs_scan(const unsigned* count, int64_t n, int64_t* off, cudaStream_t s);
// Writes the depth-index keys into the tile lists (cursor zeroed by the caller).
cudaError_t launch_gs_fill(const float4* rec, const int4* rect, int64_t n, int nv, int ntx,
                           int nty, const int64_t* off, unsigned* cursor,
                           unsigned long long* keys, cudaStream_t s);
// Sorts each tile's list and composites it: out_t / out_hit [nv x H x W].
cudaError_t launch_gs_render(const float4* rec, int64_t n, const GiCamera* cams, int nv, int ntx,
                             int nty, const int64_t* off, const unsigned long long* keys,
                             float* out_t, uint8_t* out_hit, cudaStream_t s);
// Pixel-centre rays of nv views of npx pixels each (cams on the device).
cudaError_t launch_camera_rays(const GiCamera* cams, int nv, int64_t npx, RayOut r, cudaStream_t s);

// Moves origins to their entry into [-h, h]^3; t (nullable) loses that
// distance, t_in (nullable) receives it.
cudaError_t launch_enter_box(RayOut r, float* t, float* t_in, int64_t n, float h, cudaStream_t s);

// ---- training from a fixed pool of supervised rays (distill.cu) ----
// Row i of the batch copies pool row floor(u n_pool), u a 32-bit uniform of
// (seed, step, i).
cudaError_t launch_pool_gather(RaySoA pool, const float* pool_t, const uint8_t* pool_hit,
                               int64_t n_pool, uint64_t seed, uint64_t step, int64_t n,
                               RayOut r, float* t, uint8_t* hit, cudaStream_t s);

}  // namespace ddf

