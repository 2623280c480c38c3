// epilogue.cuh -- the accumulator epilogue shared by the tensor-core layer
// kernels (tc_gemm.cu, tc_gemm_pair.cu).
//
// One thread owns one row of a 128-lane TMEM accumulator. For the columns
// [32 c_begin, 32 c_end) of its tile it computes x = ReLU(acc * scale + bias)
// and either stores x (bf16, or e4m3 after out_scale) as the next layer's
// activation or folds x into the two FP32 head dot products. The per-column
// vectors are read from shared memory (staged once per CTA), and the TMEM load
// of chunk c+1 is issued before chunk c is processed so the load latency
// overlaps the arithmetic and the stores.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"
#include "ptx_sm103.cuh"

namespace ddf {

// Column vectors of one layer staged in shared memory.
struct EpiVectors {
  const float* bias;   // [N]
  const float* scale;  // [N] or nullptr
  const float* hw0;    // [N] or nullptr (mode 1)
  const float* hw1;    // [N] or nullptr (mode 1)
  float uscale;        // the scale of every column when `scale` is nullptr
};

// Widest layer whose vectors the tensor-core kernels stage (4 x 2048 floats
// fit next to 192 KB of pipeline stages within the 227 KB per CTA).
constexpr int kMaxStagedColumns = 2048;

// Bytes of shared memory the staged vectors of an N-column layer need.
__host__ __device__ constexpr int epi_vector_bytes(int n) { return 4 * n * 4; }

// Cooperative copy of the layer's vectors into shared memory (all threads).
// An e4m3 output's scale (out_scale = 1 / s_out, a power of two) is folded
// into them: ReLU(acc scale + bias) out_scale = ReLU(acc (scale out_scale) +
// bias out_scale) exactly, since multiplying by a power of two commutes with
// float32 rounding, so the epilogue saves one multiply per element.
__device__ __forceinline__ EpiVectors stage_epi_vectors(const TcGemmParams& p, float* smem) {
  const int n = p.N;
  float* sb = smem;
  float* ss = smem + n;
  float* s0 = smem + 2 * n;
  float* s1 = smem + 3 * n;
  const float os = p.out_scale;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (p.bias != nullptr) sb[i] = p.bias[i] * os;
    if (p.col_scale != nullptr) ss[i] = p.col_scale[i] * os;
    if (p.mode == 1 || p.mode == 4) {  // only a last layer folds the head
      s0[i] = p.head_w[i];
      s1[i] = p.head_w[n + i];
    }
  }
  const bool head = p.mode == 1 || p.mode == 4;
  return EpiVectors{sb, p.col_scale != nullptr ? ss : nullptr, head ? s0 : nullptr,
                    head ? s1 : nullptr, os};
}

__device__ __forceinline__ uint32_t epi_pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t epi_pack_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xFFFFu) | (hi << 16);
}

// ReLU in the conversion: max(x, 0) rounded, with lo in the low half.
__device__ __forceinline__ uint32_t epi_pack_bf16x2_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// ReLU in the conversion: four e4m3 codes of max(x, 0) (saturating at
// 448), a in the lowest byte.
__device__ __forceinline__ uint32_t epi_pack_e4m3x4_relu(float a, float b, float c, float d) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
  asm("cvt.rn.satfinite.relu.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
  return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

// One 32-byte (256-bit) global store of w[0..7] at p (32-byte aligned): a
// whole sector from one thread, so rows written by different lanes of a warp
// still reach L2 as full sectors.
__device__ __forceinline__ void st_global_256(void* p, const uint32_t* w) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]),
               "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

// Host check of what the mode-0 thread stores assume: the output and its
// row stride 32-byte aligned.
inline bool epi_out_aligned(const TcGemmParams& p, bool out_fp8) {
  if (p.mode != 0 || p.out == nullptr) return true;
  const size_t row_bytes = static_cast<size_t>(p.ldo) * (out_fp8 ? 1 : 2);
  return reinterpret_cast<uintptr_t>(p.out) % 32 == 0 && row_bytes % 32 == 0;
}

// x[j] = v[j] cs[j] + bias[j] over the chunk's 32 columns [nc, nc + 32),
// two columns per packed FP32 FMA (each lane rounds once, as fmaf does).
__device__ __forceinline__ void epi_affine32(const EpiVectors& ev, const uint32_t (&v)[32], int nc,
                                             float (&x)[32]) {
  const float4* b4 = reinterpret_cast<const float4*>(ev.bias + nc);
#pragma unroll
  for (int j4 = 0; j4 < 8; ++j4) {
    const float4 bb = b4[j4];
    float4 cs = make_float4(ev.uscale, ev.uscale, ev.uscale, ev.uscale);
    if (ev.scale != nullptr) cs = reinterpret_cast<const float4*>(ev.scale + nc)[j4];
    const float2 lo = __ffma2_rn(make_float2(__uint_as_float(v[4 * j4 + 0]), __uint_as_float(v[4 * j4 + 1])),
                                 make_float2(cs.x, cs.y), make_float2(bb.x, bb.y));
    const float2 hi = __ffma2_rn(make_float2(__uint_as_float(v[4 * j4 + 2]), __uint_as_float(v[4 * j4 + 3])),
                                 make_float2(cs.z, cs.w), make_float2(bb.z, bb.w));
    x[4 * j4 + 0] = lo.x;
    x[4 * j4 + 1] = lo.y;
    x[4 * j4 + 2] = hi.x;
    x[4 * j4 + 3] = hi.y;
  }
}

// Processes the 32 accumulator values v of columns [nc, nc + 32) of `row`.
// HEAD_ONLY: mode 1 known at compile time (no stores are compiled).
template <bool OUT_FP8, bool HEAD_ONLY = false>
__device__ __forceinline__ void epi_chunk(const TcGemmParams& p, const EpiVectors& ev,
                                          const uint32_t (&v)[32], int row, bool row_ok, int nc,
                                          float& h0, float& h1) {
  float x[32];  // before the ReLU, which the packing conversions (or the head) apply
  epi_affine32(ev, v, nc, x);
  if (!HEAD_ONLY && p.mode == 0) {
    if (p.amax != nullptr) {  // calibration: the warp's largest output of valid rows
      float m = 0.f;          // max(0, max x) = the largest output after the ReLU
      if (row_ok) {
#pragma unroll
        for (int j = 0; j < 32; ++j) m = fmaxf(m, x[j]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
      // x >= 0 after ReLU, so the float order equals the int order of its bits
      if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(p.amax), __float_as_int(m));
    }
    if (!row_ok) return;
    // 32-byte stores: the output rows start 32-byte aligned (launchers check
    // the base and the row stride) and nc is a multiple of 32
    if constexpr (OUT_FP8) {
      uint8_t* dst = static_cast<uint8_t*>(p.out) + static_cast<size_t>(row) * p.ldo + nc;
      uint32_t w[8];  // the output scale is already in the vectors
#pragma unroll
      for (int k = 0; k < 8; ++k)
        w[k] = epi_pack_e4m3x4_relu(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
      st_global_256(dst, w);
    } else {
      __nv_bfloat16* dst =
          static_cast<__nv_bfloat16*>(p.out) + static_cast<size_t>(row) * p.ldo + nc;
      uint32_t w[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) w[k] = epi_pack_bf16x2_relu(x[2 * k], x[2 * k + 1]);
      st_global_256(dst, w);
      st_global_256(dst + 16, w + 8);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = fmaxf(x[j], 0.f);
    const float4* w0 = reinterpret_cast<const float4*>(ev.hw0 + nc);
    const float4* w1 = reinterpret_cast<const float4*>(ev.hw1 + nc);
    float2 hh = make_float2(h0, h1);  // both head sums, one packed FMA per column
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
      const float4 a = w0[j4];
      const float4 bb = w1[j4];
      hh = __ffma2_rn(make_float2(x[4 * j4 + 0], x[4 * j4 + 0]), make_float2(a.x, bb.x), hh);
      hh = __ffma2_rn(make_float2(x[4 * j4 + 1], x[4 * j4 + 1]), make_float2(a.y, bb.y), hh);
      hh = __ffma2_rn(make_float2(x[4 * j4 + 2], x[4 * j4 + 2]), make_float2(a.z, bb.z), hh);
      hh = __ffma2_rn(make_float2(x[4 * j4 + 3], x[4 * j4 + 3]), make_float2(a.w, bb.w), hh);
    }
    h0 = hh.x;
    h1 = hh.y;
  }
}

// Drains chunks [c_begin, c_end) of this thread's TMEM row (tbase = lane
// quarter + accumulator column base), columns n0 + 32 c.
template <bool OUT_FP8, bool HEAD_ONLY = false>
__device__ __forceinline__ void epi_row(const TcGemmParams& p, const EpiVectors& ev,
                                        uint32_t tbase, int row, bool row_ok, int n0, int c_begin,
                                        int c_end, float& h0, float& h1) {
  uint32_t va[32], vb[32];
  tmem_ld32(tbase + 32u * c_begin, va);
  tmem_wait_ld_regs(va);
#pragma unroll 1
  for (int c = c_begin; c < c_end; c += 2) {
    const bool next = c + 1 < c_end;
    if (next) tmem_ld32(tbase + 32u * (c + 1), vb);  // in flight during chunk c
    epi_chunk<OUT_FP8, HEAD_ONLY>(p, ev, va, row, row_ok, n0 + 32 * c, h0, h1);
    if (!next) break;
    tmem_wait_ld_regs(vb);
    const bool next2 = c + 2 < c_end;
    if (next2) tmem_ld32(tbase + 32u * (c + 2), va);  // in flight during chunk c+1
    epi_chunk<OUT_FP8, HEAD_ONLY>(p, ev, vb, row, row_ok, n0 + 32 * (c + 1), h0, h1);
    if (next2) tmem_wait_ld_regs(va);
  }
}

// ---------------------------------------------------------------------------
// Training epilogues (no bias, scale or ReLU), one 32-column chunk at a time:
//   mode 2 (input gradient): x = acc where mask[row][col] > 0, else 0; bf16 to
//          p.out [M x ldo]. mask is the bf16 activation [M x ldm] whose ReLU
//          the gradient passes back through.
//   mode 3 (weight gradient, split-K): acc as FP32 to
//          p.out_f32 + split * split_stride, row-major [M x ldo].
__device__ __forceinline__ void epi_row_train(const TcGemmParams& p, uint32_t tbase, int row,
                                              bool row_ok, int n0, int c_begin, int c_end,
                                              int split) {
  uint32_t v[32];
#pragma unroll 1
  for (int c = c_begin; c < c_end; ++c) {
    tmem_ld32(tbase + 32u * c, v);
    tmem_wait_ld_regs(v);
    if (!row_ok) continue;
    const int nc = n0 + 32 * c;
    if (p.mode == 2) {
      const uint4* mk = reinterpret_cast<const uint4*>(
          static_cast<const __nv_bfloat16*>(p.mask) + static_cast<size_t>(row) * p.ldm + nc);
      uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(p.out) +
                                            static_cast<size_t>(row) * p.ldo + nc);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint4 m4 = mk[k];
        const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
        uint32_t ow[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // a bf16 activation is > 0 iff its sign bit is clear and it is not zero
          const uint32_t lo = mw[q] & 0xFFFFu, hi = mw[q] >> 16;
          const float x0 = (lo != 0 && (lo & 0x8000u) == 0) ? __uint_as_float(v[8 * k + 2 * q]) : 0.f;
          const float x1 = (hi != 0 && (hi & 0x8000u) == 0) ? __uint_as_float(v[8 * k + 2 * q + 1]) : 0.f;
          ow[q] = epi_pack_bf16x2(x0, x1);
        }
        dst[k] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
      }
    } else {
      float4* dst = reinterpret_cast<float4*>(p.out_f32 + static_cast<size_t>(split) * p.split_stride +
                                              static_cast<size_t>(row) * p.ldo + nc);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        dst[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                             __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
    }
  }
}

// ---------------------------------------------------------------------------
// Staged stores (mode 0): instead of every thread storing 16-byte pieces of
// its own row (32 rows per warp instruction, half-filled sectors), a warp
// packs 128 bytes of each of its 32 rows into a 4 KB shared buffer and then
// writes whole 128-byte lines, 4 rows per instruction. Pieces are placed at
// 16-byte slot (piece ^ (row & 7)) of their row so both the row-wise packing
// and the line-wise copy-out touch all eight bank groups.

constexpr int kStageBytesPerWarp = 32 * 128;

// Packs chunk c (32 columns) into the staging row of this lane.
template <bool OUT_FP8>
__device__ __forceinline__ void epi_chunk_stage(const TcGemmParams& p, const EpiVectors& ev,
                                                const uint32_t (&v)[32], int nc, int c,
                                                uint8_t* stage, int lane) {
  float x[32];  // before the ReLU, which the packing conversions apply
  epi_affine32(ev, v, nc, x);
  uint8_t* row = stage + lane * 128;
  const int sw = lane & 7;
  if constexpr (OUT_FP8) {
    const int piece0 = 2 * (c & 3);  // 4 chunks of 32 bytes per 128-byte row
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // the output scale is already in the vectors
      uint4 w;
      w.x = epi_pack_e4m3x4_relu(x[16 * k + 0], x[16 * k + 1], x[16 * k + 2], x[16 * k + 3]);
      w.y = epi_pack_e4m3x4_relu(x[16 * k + 4], x[16 * k + 5], x[16 * k + 6], x[16 * k + 7]);
      w.z = epi_pack_e4m3x4_relu(x[16 * k + 8], x[16 * k + 9], x[16 * k + 10], x[16 * k + 11]);
      w.w = epi_pack_e4m3x4_relu(x[16 * k + 12], x[16 * k + 13], x[16 * k + 14], x[16 * k + 15]);
      *reinterpret_cast<uint4*>(row + (((piece0 + k) ^ sw) << 4)) = w;
    }
  } else {
    const int piece0 = 4 * (c & 1);  // 2 chunks of 64 bytes per 128-byte row
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint4 w;
      w.x = epi_pack_bf16x2_relu(x[8 * k + 0], x[8 * k + 1]);
      w.y = epi_pack_bf16x2_relu(x[8 * k + 2], x[8 * k + 3]);
      w.z = epi_pack_bf16x2_relu(x[8 * k + 4], x[8 * k + 5]);
      w.w = epi_pack_bf16x2_relu(x[8 * k + 6], x[8 * k + 7]);
      *reinterpret_cast<uint4*>(row + (((piece0 + k) ^ sw) << 4)) = w;
    }
  }
}

// Writes the warp's 32 staged rows (128 bytes each) to out rows
// warp_row0 .. warp_row0 + 31 (those < M) at byte column col_bytes.
__device__ __forceinline__ void epi_flush_stage(const TcGemmParams& p, const uint8_t* stage,
                                                int warp_row0, size_t row_bytes, size_t col_bytes,
                                                int lane) {
  __syncwarp();
  const int k = lane & 7;
  uint8_t* out = static_cast<uint8_t*>(p.out) + col_bytes + (k << 4);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = 4 * i + (lane >> 3);
    const uint4 w = *reinterpret_cast<const uint4*>(stage + r * 128 + ((k ^ (r & 7)) << 4));
    const int row = warp_row0 + r;
    if (row < p.M) *reinterpret_cast<uint4*>(out + static_cast<size_t>(row) * row_bytes) = w;
  }
  __syncwarp();
}

// Mode-0 drain of chunks [c_begin, c_end) through the warp's staging buffer
// (c_begin and c_end multiples of the chunks per 128-byte row).
template <bool OUT_FP8>
__device__ __forceinline__ void epi_row_staged(const TcGemmParams& p, const EpiVectors& ev,
                                               uint32_t tbase, int warp_row0, int n0, int c_begin,
                                               int c_end, uint8_t* stage, int lane) {
  constexpr int kGroup = OUT_FP8 ? 4 : 2;  // chunks per 128 bytes of a row
  constexpr int kElem = OUT_FP8 ? 1 : 2;
  const size_t row_bytes = static_cast<size_t>(p.ldo) * kElem;
  uint32_t va[32], vb[32];
  tmem_ld32(tbase + 32u * c_begin, va);
  tmem_wait_ld_regs(va);
#pragma unroll 1
  for (int c = c_begin; c < c_end; c += 2) {
    // chunks c (in va) and c + 1 (loaded into vb meanwhile); c_end - c_begin is even
    tmem_ld32(tbase + 32u * (c + 1), vb);
    epi_chunk_stage<OUT_FP8>(p, ev, va, n0 + 32 * c, c, stage, lane);
    tmem_wait_ld_regs(vb);
    const bool next2 = c + 2 < c_end;
    if (next2) tmem_ld32(tbase + 32u * (c + 2), va);
    epi_chunk_stage<OUT_FP8>(p, ev, vb, n0 + 32 * (c + 1), c + 1, stage, lane);
    if (((c + 2 - c_begin) % kGroup) == 0) {
      const int g0 = c + 2 - kGroup;  // first chunk of the staged group
      epi_flush_stage(p, stage, warp_row0, row_bytes,
                      static_cast<size_t>(n0 + 32 * g0) * kElem, lane);
    }
    if (next2) tmem_wait_ld_regs(va);
  }
}

// Mode-0 drain by TMA stores (the fused layer 1, the staged pair tile): one
// warp's chunks [c_begin, c_end) of its TMEM rows (bias + ReLU, bf16 or e4m3), packed group by group (128 bytes of each row)
// into the warp's output boxes and written by TMA stores at
// (column n0 + 32 c, row row0). `issued` counts the warp's stores so far.
template <bool OUT_FP8, int DEPTH>
__device__ __forceinline__ void epi_tile_tma(const TcGemmParams& p, const EpiVectors& ev,
                                             const CUtensorMap* tmO, uint32_t tbase, int row0,
                                             int n0, int c_begin, int c_end, uint8_t* boxes,
                                             int lane, uint32_t& issued) {
  constexpr int kGroup = OUT_FP8 ? 4 : 2;  // 32-column chunks per 128-byte row piece
  uint32_t va[32], vb[32];
  uint8_t* box = boxes;
  tmem_ld32(tbase + 32u * c_begin, va);
  tmem_wait_ld_regs(va);
#pragma unroll 1
  for (int c = c_begin; c < c_end; c += 2) {
    if (((c - c_begin) % kGroup) == 0) {  // a new group: take the next box once it is free
      box = boxes + (issued % DEPTH) * (32 * 128);
      if (lane == 0) bulk_wait_group_read<DEPTH - 1>();
      __syncwarp();
    }
    tmem_ld32(tbase + 32u * (c + 1), vb);
    epi_chunk_stage<OUT_FP8>(p, ev, va, n0 + 32 * c, c, box, lane);
    tmem_wait_ld_regs(vb);
    const bool next2 = c + 2 < c_end;
    if (next2) tmem_ld32(tbase + 32u * (c + 2), va);
    epi_chunk_stage<OUT_FP8>(p, ev, vb, n0 + 32 * (c + 1), c + 1, box, lane);
    if (((c + 2 - c_begin) % kGroup) == 0) {
      const int g0 = c + 2 - kGroup;  // first chunk of the finished group
      fence_proxy_async_smem();       // the TMA store reads the box through the async proxy
      __syncwarp();
      if (lane == 0) {
        // element coordinates: 32 columns per chunk; e4m3 elements are bytes
        tma_store_2d(tmO, smem_u32(box), n0 + 32 * g0, row0);
        bulk_commit_group();
      }
      ++issued;
    }
    if (next2) tmem_wait_ld_regs(va);
  }
}

// Training forward of the last layer (mode 4, bf16, no column scale) through
// the warp's staging buffer, as epi_row_staged, folding the stored bf16
// outputs into the two head dot products over the thread's columns, in
// column order (h0, h1).
// One chunk (32 columns, chunk index c of the tile, half h of its 128-byte
// staging row): bias, ReLU, bf16, staged, and the head's partial sums.
__device__ __forceinline__ void epi_chunk_stage_head(const EpiVectors& ev, const uint32_t (&v)[32],
                                                     int col0, int h, uint8_t* myrow, int sw,
                                                     float& h0, float& h1) {
  const float* bias = ev.bias + col0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t ow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 8 * k + 2 * q;
      ow[q] = epi_pack_bf16x2_relu(__uint_as_float(v[j]) + bias[j],
                                   __uint_as_float(v[j + 1]) + bias[j + 1]);
      const int col = col0 + j;
      const float x0 = __uint_as_float(ow[q] << 16), x1 = __uint_as_float(ow[q] & 0xFFFF0000u);
      h0 = fmaf(x0, ev.hw0[col], h0);
      h1 = fmaf(x0, ev.hw1[col], h1);
      h0 = fmaf(x1, ev.hw0[col + 1], h0);
      h1 = fmaf(x1, ev.hw1[col + 1], h1);
    }
    *reinterpret_cast<uint4*>(myrow + (((4 * h + k) ^ sw) << 4)) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
  }
}

// The TMEM loads run one chunk ahead of the arithmetic (chunk c + 1 is in
// flight while chunk c is converted), as in epi_row_staged.
__device__ __forceinline__ void epi_row_staged_head(const TcGemmParams& p, const EpiVectors& ev,
                                                    uint32_t tbase, int warp_row0, int n0,
                                                    int c_begin, int c_end, uint8_t* stage,
                                                    int lane, float& h0, float& h1) {
  const size_t row_bytes = static_cast<size_t>(p.ldo) * 2;
  const int sw = lane & 7;
  uint8_t* myrow = stage + lane * 128;
  uint32_t va[32], vb[32];
  tmem_ld32(tbase + 32u * c_begin, va);
  tmem_wait_ld_regs(va);
#pragma unroll 1
  for (int c = c_begin; c < c_end; c += 2) {  // c_end - c_begin is even
    tmem_ld32(tbase + 32u * (c + 1), vb);
    epi_chunk_stage_head(ev, va, n0 + 32 * c, 0, myrow, sw, h0, h1);
    tmem_wait_ld_regs(vb);
    const bool next2 = c + 2 < c_end;
    if (next2) tmem_ld32(tbase + 32u * (c + 2), va);
    epi_chunk_stage_head(ev, vb, n0 + 32 * (c + 1), 1, myrow, sw, h0, h1);
    epi_flush_stage(p, stage, warp_row0, row_bytes, static_cast<size_t>(n0 + 32 * c) * 2, lane);
    if (next2) tmem_wait_ld_regs(va);
  }
}

// One chunk of the input gradient: the accumulator where the activation is
// positive, else 0, as bf16 into half h of the staging row. mk holds the
// chunk's 32 bf16 activations of this lane's row; one bf16x2 comparison
// gives the mask of both halves of a packed pair (a zero of either sign
// passes no gradient), so the result is bf16(acc) or +0.
__device__ __forceinline__ void epi_chunk_stage_masked(const uint32_t (&v)[32], const uint4* mk,
                                                       int h, uint8_t* myrow, int sw) {
  const __nv_bfloat162 zero = __float2bfloat162_rn(0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(mk + k);
    uint32_t ow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 8 * k + 2 * q;
      ow[q] = epi_pack_bf16x2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])) &
              __hgt2_mask(a[q], zero);
    }
    *reinterpret_cast<uint4*>(myrow + (((4 * h + k) ^ sw) << 4)) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
  }
}

// Input gradient (mode 2, bf16) through the warp's staging buffer: the
// accumulator where the previous layer's activation (p.mask, bf16
// [M x ldm]) is positive, else 0, leaving as 128-byte lines. With
// p.col_part, lane l also sums columns 2l and 2l + 1 of each 64-column group
// over the warp's 32 rows (the bias gradient's share of these rows) into
// col_part[warp_row0 / 32][column]. The TMEM loads of the next chunk, and
// the activations of the next two chunks, are in flight while a chunk is
// converted. c_end - c_begin is a multiple of 4.
__device__ __forceinline__ void epi_row_masked_staged(const TcGemmParams& p, uint32_t tbase,
                                                      int warp_row0, int n0, int c_begin,
                                                      int c_end, uint8_t* stage, int lane) {
  const size_t row_bytes = static_cast<size_t>(p.ldo) * 2;
  const int row = warp_row0 + lane;
  const bool row_ok = row < p.M;
  const int sw = lane & 7;
  uint8_t* myrow = stage + lane * 128;
  // 8 bf16 per uint4: chunk c of the tile starts at uint4 4 c of the row
  const uint4* mrow = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(p.mask) +
                                                     static_cast<size_t>(row_ok ? row : 0) * p.ldm + n0);
  auto load_pair = [&](int c, uint4 (&m)[8]) {  // the activations of chunks c, c + 1
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = row_ok ? __ldg(mrow + 4 * c + i) : make_uint4(0u, 0u, 0u, 0u);
  };
  uint32_t va[32], vb[32];
  // one step: chunks c and c + 1 with their activations in cur, those of
  // c + 2 and c + 3 loaded into nxt
  auto step = [&](int c, const uint4 (&cur)[8], uint4 (&nxt)[8]) {
    tmem_ld32(tbase + 32u * (c + 1), vb);
    const bool next2 = c + 2 < c_end;
    if (next2) load_pair(c + 2, nxt);
    epi_chunk_stage_masked(va, cur, 0, myrow, sw);
    tmem_wait_ld_regs(vb);
    if (next2) tmem_ld32(tbase + 32u * (c + 2), va);
    epi_chunk_stage_masked(vb, cur + 4, 1, myrow, sw);
    if (p.col_part != nullptr) {
      __syncwarp();
      // lane l: columns 2l, 2l + 1 of the group = 4-byte word (l & 3) of
      // 16-byte piece l >> 2 in every row
      float2 cs = make_float2(0.f, 0.f);  // both columns, one packed add per row
      const int piece = lane >> 2, word = lane & 3;
#pragma unroll 8
      for (int r = 0; r < 32; ++r) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(stage + r * 128 +
                                                              ((piece ^ (r & 7)) << 4) + 4 * word);
        cs = __fadd2_rn(cs, make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u)));
      }
      *reinterpret_cast<float2*>(p.col_part + static_cast<size_t>(warp_row0 / 32) * p.ldo + n0 +
                                 32 * c + 2 * lane) = cs;
    }
    epi_flush_stage(p, stage, warp_row0, row_bytes, static_cast<size_t>(n0 + 32 * c) * 2, lane);
    if (next2) tmem_wait_ld_regs(va);
  };
  uint4 m0[8], m1[8];
  load_pair(c_begin, m0);
  tmem_ld32(tbase + 32u * c_begin, va);
  tmem_wait_ld_regs(va);
#pragma unroll 1
  for (int c = c_begin; c < c_end; c += 4) {
    step(c, m0, m1);
    step(c + 2, m1, m0);
  }
}

}  // namespace ddf
