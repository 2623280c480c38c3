// hashgrid.cu -- kernels of the hash-grid DDF, the paper's final field
// (Sec. 3.4): the ray origin is encoded by a multiresolution hash grid, the
// direction by four sinusoidal bands, and a small MLP of width 64 maps the
// joined code to (t, xi). Queries are described below; training (FP32 on the
// master weights) has its own forward and backward with 4 threads per ray,
// the weight gradients as batch-split outer products, and the refresh of the
// bf16 table.
//
// Per ray the code costs 16 levels x 8 corner reads of the level table (the
// 26 MB bf16 table stays in the 129 MB L2), so the kernel is a gather kernel;
// the MLP is a [128 x 64] x [64 x 64] contraction per 128 rays and runs on
// the tensor cores:
//   * one CTA of 4 warps owns 128 rays at a time (thread = ray), several
//     CTAs per SM hide the gather latency of one another;
//   * each thread interpolates its levels and writes its 59-value code as
//     bf16 straight into a 128-byte-swizzled K-major shared tile;
//   * one thread issues the tcgen05.mma chain (M 128, N 64, K 4 x 16) into a
//     64-column TMEM accumulator; the threads read their row back
//     (tcgen05.ld), add bias, ReLU, and either write the next layer's tile
//     or fold the FP32 head and write t, xi (and the shadow flag).
// The FP32 kernel is the plain comparison path: same gather from an FP32
// table, FFMA layers.
#include <cuda_bf16.h>

#include "heads.cuh"
#include "kernels.h"
#include "ptx_sm103.cuh"

namespace ddf {

namespace {

constexpr int kHgRows = 128;      // rays per tile (TMEM lanes)
constexpr int kHgW = 64;          // MLP width
constexpr int kHgLevels = 16;     // levels of HashGridParams
constexpr int kHgCode = 59;       // 32 hash features + 27 direction values
constexpr int kHgImage = kHgW * 128;  // one 64 x 64 bf16 swizzled operand: 8 KB
constexpr uint32_t kPrimeY = 2654435761u;
constexpr uint32_t kPrimeZ = 805459861u;
constexpr uint64_t kHgDrainNs = 1000000000ull;

// Byte offset of element k (bf16) of row r in a 128-byte-swizzled K-major
// tile with 64 elements per row.
__device__ __forceinline__ uint32_t sw_elem(int r, int k) {
  return static_cast<uint32_t>(r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t sw_piece(int r, int q) {
  return static_cast<uint32_t>(r * 128 + ((q ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Table row of vertex (i, j, k) on level l: dense row-major index, or the
// spatial hash modulo the table size (a power of two, mask = size - 1).
__device__ __forceinline__ uint32_t hg_index(const HashGridParams& g, int l, int i, int j, int k) {
  if (g.dense[l]) {
    const uint32_t n1 = static_cast<uint32_t>(g.res[l] + 1);
    return static_cast<uint32_t>(i) + n1 * (static_cast<uint32_t>(j) + n1 * static_cast<uint32_t>(k));
  }
  return (static_cast<uint32_t>(i) ^ (static_cast<uint32_t>(j) * kPrimeY) ^
          (static_cast<uint32_t>(k) * kPrimeZ)) & g.mask;
}

// Level-l features (f0, f1) of the point with box coordinates x01 in [0,1]^3:
// trilinear interpolation of the 8 corner entries, corner bit 0 = x.
template <typename Fetch>
__device__ __forceinline__ void hg_level(const HashGridParams& g, int l, float x, float y,
                                         float z, Fetch fetch, float& f0, float& f1) {
  const int n = g.res[l];
  const float fn = static_cast<float>(n);
  const float ux = x * fn, uy = y * fn, uz = z * fn;
  const int ix = min(static_cast<int>(ux), n - 1);  // ux >= 0: truncation is floor
  const int iy = min(static_cast<int>(uy), n - 1);
  const int iz = min(static_cast<int>(uz), n - 1);
  const float wx = ux - static_cast<float>(ix);
  const float wy = uy - static_cast<float>(iy);
  const float wz = uz - static_cast<float>(iz);
  float2 v[8];
#pragma unroll
  for (int c = 0; c < 8; c += 2)  // all reads in flight before any use
    fetch(g.offset[l] + hg_index(g, l, ix, iy + ((c >> 1) & 1), iz + (c >> 2)),
          g.offset[l] + hg_index(g, l, ix + 1, iy + ((c >> 1) & 1), iz + (c >> 2)), v[c], v[c + 1]);
  f0 = 0.f;
  f1 = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = ((c & 1) ? wx : 1.f - wx) * (((c >> 1) & 1) ? wy : 1.f - wy) *
                    ((c >> 2) ? wz : 1.f - wz);
    f0 = fmaf(w, v[c].x, f0);
    f1 = fmaf(w, v[c].y, f1);
  }
}

__device__ __forceinline__ float box01(float v) { return fminf(fmaxf((v + 1.f) * 0.5f, 0.f), 1.f); }

// The 27 direction values: d, then per coordinate c and band k = 0..3
// sin(pi 2^k d_c), cos(pi 2^k d_c).
__device__ __forceinline__ void hg_dir_code(float dx, float dy, float dz, float (&out)[27]) {
  out[0] = dx;
  out[1] = dy;
  out[2] = dz;
  const float dc[3] = {dx, dy, dz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s, co;
      // pi 2^k d: the product by 2^k (exponent bits) is exact
      sincospif(dc[c] * __int_as_float((127 + k) << 23), &s, &co);
      out[3 + 8 * c + 2 * k] = s;
      out[4 + 8 * c + 2 * k] = co;
    }
  }
}

// ------------------------------------------------------------ tensor cores

struct HgSmem {
  static constexpr int A_OFF = 0;                       // [128 x 64] bf16 code / activation tile
  static constexpr int W_OFF = kHgRows * 128;           // hidden-layer operand images
  __host__ __device__ static int vec_off(int H) { return W_OFF + H * kHgImage; }
  // bias [H x 64], head rows [2 x 64], head bias [2], barrier, TMEM slot
  __host__ __device__ static int ctrl_off(int H) { return vec_off(H) + (H * kHgW + 2 * kHgW + 2) * 4; }
  __host__ __device__ static int bytes(int H) { return ((ctrl_off(H) + 16 + 15) & ~15) + 1024; }
};

__global__ void __launch_bounds__(kHgRows, 4)  // 4 CTAs per SM: 128 registers
    hashgrid_tc_kernel(const HashGridParams g, const uint32_t* __restrict__ table,
                       const uint8_t* __restrict__ w_img, const float* __restrict__ bias,
                       const float* __restrict__ head_w, const float* __restrict__ head_b, int H,
                       RaySoA rays, int64_t M, HeadOut out, uint32_t* status,
                       uint64_t timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem + HgSmem::A_OFF;
  uint8_t* sW = smem + HgSmem::W_OFF;
  float* sbias = reinterpret_cast<float*>(smem + HgSmem::vec_off(H));
  float* shw = sbias + H * kHgW;
  float* shb = shw + 2 * kHgW;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + HgSmem::ctrl_off(H));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  if (tid == 0) {
    mbar_init(smem_u32(bar), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), kHgW);
    tmem_relinquish();
  }
  // operand images (pre-swizzled at load time) and the FP32 vectors
  const uint4* src = reinterpret_cast<const uint4*>(w_img);
  uint4* dst = reinterpret_cast<uint4*>(sW);
  for (int i = tid; i < H * kHgImage / 16; i += kHgRows) dst[i] = src[i];
  for (int i = tid; i < H * kHgW; i += kHgRows) sbias[i] = bias[i];
  for (int i = tid; i < 2 * kHgW; i += kHgRows) shw[i] = head_w[i];
  if (tid < 2) shb[tid] = head_b[tid];
  fence_proxy_async_smem();  // the images are read by the MMAs (async proxy)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);  // this warp's lanes
  constexpr uint32_t idesc = mma_idesc(1u, kHgW, kHgRows);
  uint32_t phase = 0;
  bool ok = true;

  // The two x-neighbour corners of a cell: one 8-byte load when both entries
  // sit in the same aligned pair (dense levels: an even first index; hashed
  // levels: an even cell index, since x enters the hash unscrambled), else two.
  // Level offsets of this table are even, so pairs never straddle levels.
  const uint2* table2 = reinterpret_cast<const uint2*>(table);
  auto fetch = [&](uint32_t e0, uint32_t e1, float2& v0, float2& v1) {
    const uint2 a = __ldg(table2 + (e0 >> 1));
    const uint32_t w0 = (e0 & 1u) ? a.y : a.x;
    uint32_t w1;
    if ((e1 >> 1) == (e0 >> 1)) {
      w1 = (e1 & 1u) ? a.y : a.x;
    } else {
      w1 = __ldg(table + e1);
    }
    v0 = make_float2(__uint_as_float(w0 << 16), __uint_as_float(w0 & 0xFFFF0000u));
    v1 = make_float2(__uint_as_float(w1 << 16), __uint_as_float(w1 & 0xFFFF0000u));
  };

  const int64_t tiles = (M + kHgRows - 1) / kHgRows;
  for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const int64_t row = tile * kHgRows + tid;
    const bool valid = row < M;
    float ox = 0.f, oy = 0.f, oz = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
    if (valid) {
      ox = __ldg(rays.p[0] + row);
      oy = __ldg(rays.p[1] + row);
      oz = __ldg(rays.p[2] + row);
      dx = __ldg(rays.p[3] + row);
      dy = __ldg(rays.p[4] + row);
      dz = __ldg(rays.p[5] + row);
    }
    const float x = box01(ox), y = box01(oy), z = box01(oz);
    // hash features: levels 4q .. 4q+3 fill 16-byte piece q of the row
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) hg_level(g, 4 * q + j, x, y, z, fetch, f[2 * j], f[2 * j + 1]);
      *reinterpret_cast<uint4*>(sA + sw_piece(tid, q)) =
          make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    {
      float dcode[27];
      hg_dir_code(dx, dy, dz, dcode);
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = k < 27 ? dcode[k] : 0.f;  // columns 32..63
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(sA + sw_piece(tid, 4 + q)) =
            make_uint4(pack2(v[8 * q], v[8 * q + 1]), pack2(v[8 * q + 2], v[8 * q + 3]),
                       pack2(v[8 * q + 4], v[8 * q + 5]), pack2(v[8 * q + 6], v[8 * q + 7]));
    }
    for (int l = 0; l < H && ok; ++l) {
      fence_proxy_async_smem();  // this thread's tile row, for the MMAs
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA);
        const uint32_t b0 = smem_u32(sW + l * kHgImage);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          tc_mma_f16(tmem, sw128_kmajor_desc(a0 + 32u * j), sw128_kmajor_desc(b0 + 32u * j), idesc,
                     j != 0 ? 1u : 0u);
        tc_commit(smem_u32(bar));
      }
      ok = mbar_wait_bounded(smem_u32(bar), phase, nullptr, timeout_ns);
      phase ^= 1u;
      ok = __syncthreads_and(ok);
      if (!ok) break;
      tc_fence_after();
      uint32_t va[32], vb[32];
      tmem_ld32(trow, va);
      tmem_ld32(trow + 32u, vb);
      tmem_wait_ld_regs(va);
      tmem_wait_ld_regs(vb);
      const float* b = sbias + l * kHgW;
      if (l + 1 < H) {  // next layer's input: bf16(ReLU(acc + b)) into the same tile
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float h[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = 8 * q + e;
            const uint32_t bits = k < 32 ? va[k] : vb[k - 32];
            h[e] = fmaxf(__uint_as_float(bits) + b[k], 0.f);
          }
          *reinterpret_cast<uint4*>(sA + sw_piece(tid, q)) =
              make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
        }
      } else {  // the last hidden activation stays FP32 and feeds the FP32 head
        float z0 = shb[0], z1 = shb[1];
#pragma unroll
        for (int k = 0; k < kHgW; ++k) {
          const uint32_t bits = k < 32 ? va[k] : vb[k - 32];
          const float h = fmaxf(__uint_as_float(bits) + b[k], 0.f);
          z0 = fmaf(h, shw[k], z0);
          z1 = fmaf(h, shw[kHgW + k], z1);
        }
        if (valid) write_heads(out, row, z0, z1);
      }
    }
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, kStatusPipelineTimeout);
    // the chain whose wait gave up (parity phase ^ 1) must finish before its
    // TMEM is released
    mbar_wait_bounded(smem_u32(bar), phase ^ 1u, nullptr, kHgDrainNs);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kHgW);
  }
}

// ------------------------------------------------------------ FP32 path

constexpr int kHgF32Rays = 64;  // rays per block
constexpr int kHgLd = kHgW + 1; // per-thread row stride in shared memory

// Queries, thread = ray: code and activations in a per-thread shared-memory
// row, weights broadcast from shared memory, FFMA only.
__global__ void __launch_bounds__(kHgF32Rays)
    hashgrid_f32_kernel(const HashGridParams g, const float2* __restrict__ table,
                        const float* __restrict__ mlp, int H, RaySoA rays, int64_t M,
                        HeadOut out) {
  extern __shared__ float fsm[];
  const int n_mlp = kHgW * kHgCode + kHgW + (H - 1) * (kHgW * kHgW + kHgW) + 2 * kHgW + 2;
  float* sw = fsm;
  float* bufA = fsm + ((n_mlp + 3) & ~3);
  float* bufB = bufA + kHgF32Rays * kHgLd;
  for (int i = threadIdx.x; i < n_mlp; i += blockDim.x) sw[i] = mlp[i];
  __syncthreads();
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kHgF32Rays + threadIdx.x;
  if (row >= M) return;
  float* a = bufA + threadIdx.x * kHgLd;
  float* nb = bufB + threadIdx.x * kHgLd;
  const float x = box01(rays.p[0][row]), y = box01(rays.p[1][row]), z = box01(rays.p[2][row]);
  auto fetch = [&](uint32_t e0, uint32_t e1, float2& v0, float2& v1) {
    v0 = __ldg(table + e0);
    v1 = __ldg(table + e1);
  };
  for (int l = 0; l < 16; ++l) hg_level(g, l, x, y, z, fetch, a[2 * l], a[2 * l + 1]);
  float dcode[27];
  hg_dir_code(rays.p[3][row], rays.p[4][row], rays.p[5][row], dcode);
#pragma unroll
  for (int k = 0; k < 27; ++k) a[32 + k] = dcode[k];
  const float* w = sw;
  int K = kHgCode;
  for (int l = 0; l < H; ++l) {
    const float* b = w + kHgW * K;
    for (int n = 0; n < kHgW; n += 4) {  // 4 outputs at a time: 4 independent FMA chains
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      const float* w0 = w + n * K;
      for (int k = 0; k < K; ++k) {
        const float av = a[k];
        s0 = fmaf(av, w0[k], s0);
        s1 = fmaf(av, w0[K + k], s1);
        s2 = fmaf(av, w0[2 * K + k], s2);
        s3 = fmaf(av, w0[3 * K + k], s3);
      }
      nb[n] = fmaxf(s0 + b[n], 0.f);
      nb[n + 1] = fmaxf(s1 + b[n + 1], 0.f);
      nb[n + 2] = fmaxf(s2 + b[n + 2], 0.f);
      nb[n + 3] = fmaxf(s3 + b[n + 3], 0.f);
    }
    float* t = a;
    a = nb;
    nb = t;
    w = b + kHgW;
    K = kHgW;
  }
  float z0 = 0.f, z1 = 0.f;
  for (int k = 0; k < kHgW; ++k) {
    z0 = fmaf(a[k], w[k], z0);
    z1 = fmaf(a[k], w[kHgW + k], z1);
  }
  z0 += w[2 * kHgW];
  z1 += w[2 * kHgW + 1];
  write_heads(out, row, z0, z1);
}

// ---------------------------------------------------------------- training
// Training forward and backward with kHgTrainT = 4 threads per ray (64 rays,
// 256 threads per block): at the batch sizes of a distillation step (16,384
// rays) one thread per ray leaves 3-4 warps per SM, every table gather and
// atomic waiting out its full latency. Thread t of a ray takes levels t,
// t + 4, t + 8, t + 12 and outputs (or input gradients) t + 4 q; each output
// is still summed over its inputs in order, so the values are those of one
// thread per ray (8 threads per ray were measured too, and were no faster). The ray's rows live in shared memory as in the query kernel;
// __syncwarp orders the threads of a ray (same warp). Threads of rays past
// the end stay to the end (they take part in __syncwarp) and skip every
// load and store of their row.
constexpr int kHgTrainT = 4;
static_assert(kHgLevels % kHgTrainT == 0 && kHgW % kHgTrainT == 0 && 32 % kHgTrainT == 0,
              "a ray's threads share a warp and split the levels and outputs evenly");
constexpr int kHgTrainThreads = kHgF32Rays * kHgTrainT;

// Forward weight rows in shared memory: odd strides (59, 65), so that the
// 4 threads of a ray, reading rows t + 4 q of one column, hit 4 banks.
__host__ __device__ constexpr int hg_train_ldw(int l) { return l == 0 ? kHgCode : kHgW + 1; }
__host__ __device__ constexpr int hg_train_wfloats(int H) {
  return kHgW * hg_train_ldw(0) + kHgW + (H - 1) * (kHgW * hg_train_ldw(1) + kHgW) + 2 * kHgW + 2;
}

__global__ void __launch_bounds__(kHgTrainThreads)
    hg_train_fwd_kernel(const HashGridParams g, const float2* __restrict__ table,
                        const float* __restrict__ mlp, int H, RaySoA rays, int64_t M,
                        float* __restrict__ code_out, float* __restrict__ acts,
                        float2* __restrict__ z_out) {
  extern __shared__ float fsm[];
  float* sw = fsm;
  float* bufA = fsm + ((hg_train_wfloats(H) + 3) & ~3);
  float* bufB = bufA + kHgF32Rays * kHgLd;
  {  // weights: blob layout (W_l [64 x K_l], b_l, ..., W_o [2 x 64], b_o) -> padded rows
    int src = 0, dst = 0;
    for (int l = 0; l < H; ++l) {
      const int K = l == 0 ? kHgCode : kHgW, ldw = hg_train_ldw(l);
      for (int i = threadIdx.x; i < kHgW * K; i += blockDim.x)
        sw[dst + (i / K) * ldw + i % K] = mlp[src + i];
      src += kHgW * K;
      dst += kHgW * ldw;
      for (int i = threadIdx.x; i < kHgW; i += blockDim.x) sw[dst + i] = mlp[src + i];
      src += kHgW;
      dst += kHgW;
    }
    for (int i = threadIdx.x; i < 2 * kHgW + 2; i += blockDim.x) sw[dst + i] = mlp[src + i];
  }
  __syncthreads();
  const int r = threadIdx.x / kHgTrainT, t = threadIdx.x % kHgTrainT;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kHgF32Rays + r;
  const bool valid = row < M;
  float* a = bufA + r * kHgLd;
  float* nb = bufB + r * kHgLd;
  if (valid) {
    const float x = box01(rays.p[0][row]), y = box01(rays.p[1][row]), z = box01(rays.p[2][row]);
    auto fetch = [&](uint32_t e0, uint32_t e1, float2& v0, float2& v1) {
      v0 = __ldg(table + e0);
      v1 = __ldg(table + e1);
    };
#pragma unroll
    for (int j = 0; j < kHgLevels / kHgTrainT; ++j) {
      const int l = t + kHgTrainT * j;
      hg_level(g, l, x, y, z, fetch, a[2 * l], a[2 * l + 1]);
    }
    if (t == 0) {
      float dcode[27];
      hg_dir_code(rays.p[3][row], rays.p[4][row], rays.p[5][row], dcode);
#pragma unroll
      for (int k = 0; k < 27; ++k) a[32 + k] = dcode[k];
    }
  }
  __syncwarp();
  if (valid)
    for (int k = t; k < kHgW; k += kHgTrainT) code_out[k * M + row] = k < kHgCode ? a[k] : 0.f;
  const float* w = sw;
  int K = kHgCode;
  for (int l = 0; l < H; ++l) {
    const int ldw = hg_train_ldw(l);
    const float* b = w + kHgW * ldw;
    float sacc[kHgW / kHgTrainT];
#pragma unroll
    for (int q = 0; q < kHgW / kHgTrainT; ++q) sacc[q] = 0.f;
    for (int k = 0; k < K; ++k) {
      const float av = a[k];
#pragma unroll
      for (int q = 0; q < kHgW / kHgTrainT; ++q)
        sacc[q] = fmaf(av, w[(t + kHgTrainT * q) * ldw + k], sacc[q]);
    }
    float* dst = acts + static_cast<int64_t>(l) * kHgW * M + row;
#pragma unroll
    for (int q = 0; q < kHgW / kHgTrainT; ++q) {
      const int n = t + kHgTrainT * q;
      const float hv = fmaxf(sacc[q] + b[n], 0.f);
      nb[n] = hv;
      if (valid) dst[n * M] = hv;
    }
    __syncwarp();
    float* tmp = a;
    a = nb;
    nb = tmp;
    w = b + kHgW;
    K = kHgW;
  }
  if (valid && t == 0) {
    float z0 = 0.f, z1 = 0.f;
    for (int k = 0; k < kHgW; ++k) {
      z0 = fmaf(a[k], w[k], z0);
      z1 = fmaf(a[k], w[kHgW + k], z1);
    }
    z0 += w[2 * kHgW];
    z1 += w[2 * kHgW + 1];
    z_out[row] = make_float2(z0, z1);
  }
}

// Backward of the training forward above, kHgTrainT threads per ray: dL/dpre of
// every layer (feature-major, [H x 64 x B]) and the hash features' gradient
// scattered into the level tables' gradient (blob layout, 8-byte aligned):
// each corner entry receives its trilinear weight times the feature
// gradient (atomic adds; entries shared by several rays or corners sum up).
__global__ void __launch_bounds__(kHgTrainThreads)
    hg_train_bwd_kernel(const HashGridParams g, const float* __restrict__ mlp, int H, RaySoA rays,
                        int64_t M, const float* __restrict__ acts, const float2* __restrict__ dz,
                        float* __restrict__ dpre, float* __restrict__ grad_table) {
  extern __shared__ float fsm[];
  const int n_mlp = kHgW * kHgCode + kHgW + (H - 1) * (kHgW * kHgW + kHgW) + 2 * kHgW + 2;
  float* sw = fsm;
  float* bufA = fsm + ((n_mlp + 3) & ~3);
  float* bufB = bufA + kHgF32Rays * kHgLd;
  for (int i = threadIdx.x; i < n_mlp; i += blockDim.x) sw[i] = mlp[i];
  __syncthreads();
  const int r = threadIdx.x / kHgTrainT, t = threadIdx.x % kHgTrainT;
  const int64_t row = static_cast<int64_t>(blockIdx.x) * kHgF32Rays + r;
  const bool valid = row < M;
  float* dh = bufA + r * kHgLd;
  float* dn = bufB + r * kHgLd;
  // weight offsets: layer l's W [64 x K_l] and b, then the head W_o [2 x 64], b_o
  int woff[4];
  int off = 0;
  for (int l = 0; l < H; ++l) {
    woff[l] = off;
    off += kHgW * (l == 0 ? kHgCode : kHgW) + kHgW;
  }
  const float* wo = sw + off;
  const float2 d = valid ? dz[row] : make_float2(0.f, 0.f);
  for (int k = t; k < kHgW; k += kHgTrainT) dh[k] = d.x * wo[k] + d.y * wo[kHgW + k];
  __syncwarp();
  for (int l = H - 1; l >= 0; --l) {
    const float* h = acts + static_cast<int64_t>(l) * kHgW * M + row;
    float* dp = dpre + static_cast<int64_t>(l) * kHgW * M + row;
    for (int k = t; k < kHgW; k += kHgTrainT) {
      const float v = valid && h[k * M] > 0.f ? dh[k] : 0.f;
      dh[k] = v;
      if (valid) dp[k * M] = v;
    }
    __syncwarp();
    const int K = l == 0 ? 2 * 16 : kHgW;  // layer 1: only the hash features need a gradient
    const int ldw = l == 0 ? kHgCode : kHgW;
    const float* w = sw + woff[l];
    float sacc[kHgW / kHgTrainT];
#pragma unroll
    for (int q = 0; q < kHgW / kHgTrainT; ++q) sacc[q] = 0.f;
    for (int n = 0; n < kHgW; ++n) {
      const float dv = dh[n];
      const float* wr = w + n * ldw + t;
#pragma unroll
      for (int q = 0; q < kHgW / kHgTrainT; ++q)
        if (t + kHgTrainT * q < K) sacc[q] = fmaf(dv, wr[kHgTrainT * q], sacc[q]);
    }
#pragma unroll
    for (int q = 0; q < kHgW / kHgTrainT; ++q)
      if (t + kHgTrainT * q < K) dn[t + kHgTrainT * q] = sacc[q];
    __syncwarp();
    float* tmp = dh;
    dh = dn;
    dn = tmp;
  }
  if (!valid) return;
  // dh holds dL/d(hash features) [32]: this thread scatters levels t,
  // t + kHgTrainT, ...
  const float x = box01(rays.p[0][row]), y = box01(rays.p[1][row]), z = box01(rays.p[2][row]);
  for (int j = 0; j < kHgLevels / kHgTrainT; ++j) {
    const int l = t + kHgTrainT * j;
    const int n = g.res[l];
    const float fn = static_cast<float>(n);
    const float ux = x * fn, uy = y * fn, uz = z * fn;
    const int ix = min(static_cast<int>(ux), n - 1);
    const int iy = min(static_cast<int>(uy), n - 1);
    const int iz = min(static_cast<int>(uz), n - 1);
    const float wx = ux - static_cast<float>(ix);
    const float wy = uy - static_cast<float>(iy);
    const float wz = uz - static_cast<float>(iz);
    const float g0 = dh[2 * l], g1 = dh[2 * l + 1];
    for (int c = 0; c < 8; ++c) {
      const float w = ((c & 1) ? wx : 1.f - wx) * (((c >> 1) & 1) ? wy : 1.f - wy) *
                      ((c >> 2) ? wz : 1.f - wz);
      const uint32_t e = g.offset[l] + hg_index(g, l, ix + (c & 1), iy + ((c >> 1) & 1), iz + (c >> 2));
      // one 8-byte vector add for the entry's two features
      atomicAdd(reinterpret_cast<float2*>(grad_table) + e, make_float2(w * g0, w * g1));
    }
  }
}

// Weight-gradient partials dW = P^T A of the MLP layers of the hash-grid
// field, every layer in one launch (blockIdx.y = the layer's job; P =
// dL/dpre, A = the layer input; element (r, c) of P at P[r prs + c pcs], of
// A at A[r ars + c acs]): one 256-thread block per split of the rays and
// layer computes the whole [np x na] partial (np, na <= 64) from 32-ray
// slices staged in shared memory, thread (tn, tk) owning rows 4 tn .. 4 tn +
// 3 and columns 4 tk .. 4 tk + 3, and bpart[s][n] = sum of P[r][n] over the
// split (the bias gradient's partial). Every sum runs over the split's rays
// in order.
__global__ void __launch_bounds__(256)
hg_outer_tiled_kernel(const HgOuterJobs jobs, int64_t B, int64_t per_split) {
  __shared__ float sP[32][65];
  __shared__ float sA[32][65];
  const HgOuterJob& jb = jobs.job[blockIdx.y];
  const float* __restrict__ P = jb.P;
  const float* __restrict__ A = jb.A;
  const int64_t prs = jb.prs, pcs = jb.pcs, ars = jb.ars, acs = jb.acs;
  const int np = jb.np, na = jb.na;
  const int tid = threadIdx.x;
  const int tn = tid >> 4, tk = tid & 15;
  const int64_t r0 = blockIdx.x * per_split;
  const int64_t r1 = r0 + per_split < B ? r0 + per_split : B;
  float acc[4][4] = {};
  float bs[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int i = tid; i < 32 * 64; i += 256) {
      const int rr = i & 31, c = i >> 5;  // a warp reads 32 rays of one feature
      const int64_t r = rb + rr;
      const bool ok = r < r1;
      sP[rr][c] = ok && c < np ? P[r * prs + c * pcs] : 0.f;
      sA[rr][c] = ok && c < na ? A[r * ars + c * acs] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      float pv[4], av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        pv[i] = sP[rr][4 * tn + i];
        av[i] = sA[rr][4 * tk + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        bs[i] += pv[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pv[i], av[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  float* ps = jb.part + static_cast<int64_t>(blockIdx.x) * np * na;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = 4 * tn + i;
    if (n >= np) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * tk + j;
      if (k < na) ps[n * na + k] = acc[i][j];
    }
    if (tk == 0) jb.bpart[static_cast<int64_t>(blockIdx.x) * np + n] = bs[i];
  }
}

// ------------------------------------------------------------ packing

// (f0, f1) FP32 entry pairs -> bf16x2 words (f0 in the low half), every
// level in one launch: source entry i of level l (blob layout `from`) goes
// to entry i - from.offset[l] + to.offset[l] (the padded layout `to`).
__global__ void hg_pack_table_kernel(const float* __restrict__ src, int64_t n, HashGridParams from,
                                     HashGridParams to, uint32_t* __restrict__ dst) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l = 0;
#pragma unroll
  for (int k = 1; k < kHgLevels; ++k) l += i >= from.offset[k] ? 1 : 0;
  dst[i - from.offset[l] + to.offset[l]] = pack2(src[2 * i], src[2 * i + 1]);
}

// W [64 x K] FP32 (K <= 64) -> the swizzled K-major bf16 image the MMA reads,
// zero beyond K.
__global__ void hg_pack_image_kernel(const float* __restrict__ w, int K, uint8_t* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kHgW * 64) return;
  const int n = i / 64, k = i % 64;
  const float v = k < K ? w[n * K + k] : 0.f;
  *reinterpret_cast<__nv_bfloat16*>(img + sw_elem(n, k)) = __float2bfloat16_rn(v);
}

}  // namespace

int hashgrid_smem_bytes(int H) { return HgSmem::bytes(H); }

constexpr int kHgCtasPerSm = 4;  // __launch_bounds__(128, 4): 128 registers per thread

// Shared memory for the tensor-core kernel: its dynamic size, and a carveout
// just large enough for kHgCtasPerSm CTAs, so that the rest of the SM's
// unified memory stays L1 cache for the table gathers (about a third of them
// hit there).
cudaError_t hashgrid_tc_configure(int H) {
  cudaError_t e = cudaFuncSetAttribute(hashgrid_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       HgSmem::bytes(H));
  if (e != cudaSuccess) return e;
  int dev = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
      cudaSuccess)
    return e;
  const int need = kHgCtasPerSm * (HgSmem::bytes(H) + 1024);  // + the per-CTA reservation
  const int pct = static_cast<int>((100LL * need + per_sm - 1) / per_sm);
  return cudaFuncSetAttribute(hashgrid_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              pct < 100 ? pct : 100);
}

cudaError_t launch_hashgrid_tc(const HashGridParams& g, const uint32_t* table,
                               const uint8_t* w_img, const float* bias, const float* head_w,
                               const float* head_b, int H, RaySoA rays, int64_t M, HeadOut out,
                               uint32_t* status, uint64_t timeout_ns, int grid, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (H < 1 || H > 4 || grid <= 0) return cudaErrorInvalidValue;
  const int smem = HgSmem::bytes(H);
  cudaError_t e = hashgrid_tc_configure(H);
  if (e != cudaSuccess) return e;
  hashgrid_tc_kernel<<<grid, kHgRows, smem, s>>>(g, table, w_img, bias, head_w, head_b, H, rays, M,
                                                 out, status, timeout_ns);
  return cudaGetLastError();
}

int hashgrid_tc_blocks_per_sm(int H) {
  // The limits of one SM, from the kernel's own resources: registers (the
  // launch bound), shared memory, threads and TMEM (64 of 512 columns each).
  int dev = 0, smem_sm = 0, threads_sm = 0;
  cudaFuncAttributes fa{};
  if (hashgrid_tc_configure(H) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, hashgrid_tc_kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = kHgCtasPerSm;
  n = n < smem_sm / (HgSmem::bytes(H) + 1024) ? n : smem_sm / (HgSmem::bytes(H) + 1024);
  n = n < threads_sm / kHgRows ? n : threads_sm / kHgRows;
  n = n < 512 / kHgW ? n : 512 / kHgW;
  if (fa.numRegs * kHgRows * n > 65536) n = 65536 / (fa.numRegs * kHgRows);
  return n;
}

cudaError_t launch_hashgrid_f32(const HashGridParams& g, const float2* table, const float* mlp,
                                int H, RaySoA rays, int64_t M, HeadOut out, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (H < 1 || H > 4) return cudaErrorInvalidValue;
  const int n_mlp = kHgW * kHgCode + kHgW + (H - 1) * (kHgW * kHgW + kHgW) + 2 * kHgW + 2;
  const size_t smem = (((n_mlp + 3) & ~3) + 2 * kHgF32Rays * kHgLd) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(hashgrid_f32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (M + kHgF32Rays - 1) / kHgF32Rays;
  hashgrid_f32_kernel<<<static_cast<unsigned>(blocks), kHgF32Rays, smem, s>>>(
      g, table, mlp, H, rays, M, out);
  return cudaGetLastError();
}

namespace {
size_t hg_f32_smem(int H) {
  const int n_mlp = kHgW * kHgCode + kHgW + (H - 1) * (kHgW * kHgW + kHgW) + 2 * kHgW + 2;
  return (((n_mlp + 3) & ~3) + 2 * kHgF32Rays * kHgLd) * sizeof(float);
}
}  // namespace

cudaError_t launch_hg_train_fwd(const HashGridParams& g, const float2* table, const float* mlp,
                                int H, RaySoA rays, int64_t B, float* code, float* acts,
                                float2* z, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  if (H < 1 || H > 4) return cudaErrorInvalidValue;
  const size_t smem = (((hg_train_wfloats(H) + 3) & ~3) + 2 * kHgF32Rays * kHgLd) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(hg_train_fwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (B + kHgF32Rays - 1) / kHgF32Rays;
  hg_train_fwd_kernel<<<static_cast<unsigned>(blocks), kHgTrainThreads, smem, s>>>(
      g, table, mlp, H, rays, B, code, acts, z);
  return cudaGetLastError();
}

cudaError_t launch_hg_train_bwd(const HashGridParams& g, const float* mlp, int H, RaySoA rays,
                                int64_t B, const float* acts, const float2* dz, float* dpre,
                                float* grad_table, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  if (H < 1 || H > 4) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(grad_table) & 7u) != 0) return cudaErrorInvalidValue;
  const size_t smem = hg_f32_smem(H);
  cudaError_t e = cudaFuncSetAttribute(hg_train_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = (B + kHgF32Rays - 1) / kHgF32Rays;
  hg_train_bwd_kernel<<<static_cast<unsigned>(blocks), kHgTrainThreads, smem, s>>>(
      g, mlp, H, rays, B, acts, dz, dpre, grad_table);
  return cudaGetLastError();
}

cudaError_t launch_hg_pack_table(const float* src, int64_t n_entries, const HashGridParams& from,
                                 const HashGridParams& to, uint32_t* dst, cudaStream_t s) {
  if (n_entries <= 0) return cudaSuccess;
  hg_pack_table_kernel<<<static_cast<unsigned>((n_entries + 255) / 256), 256, 0, s>>>(
      src, n_entries, from, to, dst);
  return cudaGetLastError();
}

cudaError_t launch_hg_outer_tiled(const HgOuterJobs& jobs, int64_t B, int splits, cudaStream_t s) {
  if (jobs.n < 1 || jobs.n > kHgOuterJobs || splits < 1) return cudaErrorInvalidValue;
  for (int j = 0; j < jobs.n; ++j)
    if (jobs.job[j].np < 1 || jobs.job[j].np > 64 || jobs.job[j].na < 1 || jobs.job[j].na > 64)
      return cudaErrorInvalidValue;
  const int64_t per = (B + splits - 1) / splits;
  hg_outer_tiled_kernel<<<dim3(splits, jobs.n), 256, 0, s>>>(jobs, B, per);
  return cudaGetLastError();
}

cudaError_t launch_hg_pack_image(const float* w, int K, uint8_t* img, cudaStream_t s) {
  if (K < 1 || K > 64) return cudaErrorInvalidValue;
  hg_pack_image_kernel<<<(kHgW * 64 + 255) / 256, 256, 0, s>>>(w, K, img);
  return cudaGetLastError();
}

}  // namespace ddf
