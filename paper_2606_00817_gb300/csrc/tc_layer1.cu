// tc_layer1.cu -- the ray encoding fused into the first DDF layer.
//
// Layer 1 of the DDF MLP (Sec. 3.1; the sinusoidal encoding of Sec. 4.3 /
// Table 2 feeding a wide ReLU layer) has a short reduction (K = 6 + 12 L <= 128)
// and a wide output (W columns per ray), so its cost is writing the W-wide
// activation, not the MMAs. This kernel builds the encoded A tile in shared
// memory from the ray SoA instead of reading it from an encoded copy in HBM,
// and keeps it there for all W / 256 column tiles of its 128-ray row block.
//   warp 0         TMA producer: 256 x 64 bf16 tiles of W_1 (128-byte
//                  swizzle) into a ring of 3 stages (2 with 8 epilogue warps)
//   warp 1         TMEM owner; one thread issues tcgen05.mma (M 128, N 256,
//                  K 16) into two 256-column FP32 accumulators
//   warps 2..E+1   epilogue: bias + ReLU of the accumulator; each warp packs
//                  32 rows x 128 bytes into a 128-byte-swizzled shared box
//                  (two per warp) that a TMA tensor store writes out, so no
//                  thread issues a global store
//   last 4 warps   encoder: thread = ray; raw (o, d) then sin / cos of
//                  pi 2^k e_c, written as 16-byte pieces straight into the
//                  swizzled K-major layout tcgen05 reads (two buffers, so the
//                  next row block is encoded while this one is multiplied)
// Persistent: CTA b takes row blocks b, b + grid, ... Every wait is bounded.
#include <cuda_bf16.h>

#include "kernels.h"
#include "epilogue.cuh"
#include "heads.cuh"
#include "ptx_sm103.cuh"

namespace ddf {

namespace {

constexpr uint64_t kL1DrainNs = 1000000000ull;

template <int EPI>
struct L1Shape {
  static constexpr int BM = 128;
  static constexpr int BN = 256;
  static constexpr int KB_MAX = 2;                      // K <= 128
  static constexpr int ATOM = BM * 128;                 // one 64-element K slice of A: 16 KB
  static constexpr int A_BUF = KB_MAX * ATOM;           // 32 KB
  static constexpr int B_BYTES = BN * 128;              // 32 KB
  static constexpr int STAGES = EPI == 8 ? 2 : 3;       // W_1 ring
  static constexpr int OUT_DEPTH = 2;                   // output boxes per epilogue warp
  static constexpr int OUT_BOX = 32 * 128;              // 32 rows x 128 bytes
  static constexpr int B_OFF = 2 * A_BUF;
  static constexpr int CTRL_OFF = B_OFF + STAGES * B_BYTES;
  static constexpr int NUM_BARS = 2 * STAGES + 9;
  static constexpr int CTRL_BYTES = 256;
  static constexpr int VEC_OFF = CTRL_OFF + CTRL_BYTES;  // bias [N] floats
  static constexpr int TMEM_COLS = 2 * BN;
  static_assert(NUM_BARS * 8 + 8 <= CTRL_BYTES, "control block overflow");
  // output boxes start on a 1024-byte boundary (128-byte swizzle atom)
  __host__ __device__ static constexpr int out_off(int n) { return (VEC_OFF + 4 * n + 1023) & ~1023; }
  __host__ __device__ static constexpr int smem_bytes(int n) { return out_off(n) + EPI * OUT_DEPTH * OUT_BOX + 1024; }
};

// Byte offset of 16-byte piece q (bf16 elements 8q .. 8q+7) of row r inside a
// K-major A buffer with 128-byte swizzle: 64-element slices of 16 KB, rows of
// 128 bytes, piece q mod 8 of row r stored at piece (q mod 8) ^ (r mod 8).
__device__ __forceinline__ uint32_t a_piece_offset(int r, int q) {
  return static_cast<uint32_t>((q >> 3) * (128 * 128) + r * 128 + (((q & 7) ^ (r & 7)) << 4));
}

// (sin, cos)(pi 2^k e_c) as a bf16 pair for the next (c, k) of the encoding
// order (coordinate-major, band-minor), then advances (c, k); zero once all
// six coordinates are done (padding up to the MMA's K).
__device__ __forceinline__ uint32_t next_pair(const float (&e)[6], int L, int& c, int& k) {
  if (c >= 6) return 0u;
  const float ec = c == 0 ? e[0] : c == 1 ? e[1] : c == 2 ? e[2] : c == 3 ? e[3] : c == 4 ? e[4] : e[5];
  float sn, cs;
  // pi 2^k e: the product by 2^k (built from its exponent bits; k <= 15) is
  // exact, the value ldexpf(e, k) gives, without ldexpf's general path
  sincospif(ec * __int_as_float((127 + k) << 23), &sn, &cs);
  if (++k == L) {
    k = 0;
    ++c;
  }
  return epi_pack_bf16x2(sn, cs);
}

template <bool OUT_FP8, int EPI>
__global__ void __launch_bounds__(64 + 32 * EPI + 128, 1)
    tc_layer1_kernel(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmO,
                     const RaySoA rays, const int L, const TcGemmParams p) {
  using S = L1Shape<EPI>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::B_OFF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::CTRL_OFF);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S::STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * S::STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * S::STAGES + 2 + b); };
  auto afull_bar = [&](int a) { return bar0 + 8u * (2 * S::STAGES + 4 + a); };
  auto aempty_bar = [&](int a) { return bar0 + 8u * (2 * S::STAGES + 6 + a); };
  const uint32_t mdone_bar = bar0 + 8u * (2 * S::STAGES + 8);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S::NUM_BARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto raise_abort = [&]() {
    *abort_flag = 1;
    atomicOr(p.status, kStatusPipelineTimeout);
  };

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  constexpr int kEncWarp0 = 2 + EPI;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), EPI);  // one arrival per epilogue warp
      mbar_init(afull_bar(b), 4);     // one arrival per encoder warp
      mbar_init(aempty_bar(b), 1);    // tcgen05.commit after the block's last MMA
    }
    mbar_init(mdone_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmO);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), S::TMEM_COLS);
    tmem_relinquish();
  }
  // layer 1 has no column scale and no head: only the bias is staged, with an
  // e4m3 output's scale (a power of two) folded in as stage_epi_vectors does
  float* sbias = reinterpret_cast<float*>(smem + S::VEC_OFF);
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) sbias[i] = p.bias[i] * p.out_scale;
  const EpiVectors ev{sbias, nullptr, nullptr, nullptr, p.out_scale};
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int num_m = (p.M + S::BM - 1) / S::BM;
  const int num_n = p.N / S::BN;
  const int kb_count = (6 + 12 * L + 63) / 64;  // 1 or 2 (the launcher checks)

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- W_1 producer
    int it = 0;
    bool ok = true;
    for (int mb = blockIdx.x; mb < num_m && ok; mb += gridDim.x) {
      for (int nb = 0; nb < num_n && ok; ++nb) {
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % S::STAGES;
          const uint32_t ph = (it / S::STAGES) & 1;
          if (!mbar_wait_bounded(empty_bar(s), ph ^ 1u, abort_flag, p.timeout_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(s), S::B_BYTES);
          tma_load_2d(smem_u32(sB + s * S::B_BYTES), &tmB, kb * 64, nb * S::BN, full_bar(s));
        }
      }
    }
    if (!ok) {
      raise_abort();
      const int first = it > S::STAGES ? it - S::STAGES : 0;
      for (int j = first; j < it; ++j)
        mbar_wait_bounded(full_bar(j % S::STAGES), (j / S::STAGES) & 1, nullptr, kL1DrainNs);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = mma_idesc(1u, S::BN, S::BM);
    int it = 0, local = 0, blk = 0;
    bool ok = true;
    for (int mb = blockIdx.x; mb < num_m && ok; mb += gridDim.x, ++blk) {
      const int a = blk & 1;
      if (!mbar_wait_bounded(afull_bar(a), (blk >> 1) & 1, abort_flag, p.timeout_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(sA + a * S::A_BUF);
      for (int nb = 0; nb < num_n && ok; ++nb, ++local) {
        const int b = local & 1;
        if (!mbar_wait_bounded(tempty_bar(b), ((local >> 1) & 1) ^ 1u, abort_flag, p.timeout_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(b * S::BN);
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % S::STAGES;
          if (!mbar_wait_bounded(full_bar(s), (it / S::STAGES) & 1, abort_flag, p.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = a_base + static_cast<uint32_t>(kb * S::ATOM);
          const uint32_t b0 = smem_u32(sB + s * S::B_BYTES);
#pragma unroll
          for (int j = 0; j < 4; ++j) {  // 4 x 16 elements of K per 128-byte row
            tc_mma_f16(d_tmem, sw128_kmajor_desc(a0 + 32u * j), sw128_kmajor_desc(b0 + 32u * j),
                       idesc, (kb != 0 || j != 0) ? 1u : 0u);
          }
          tc_commit(empty_bar(s));
        }
        if (!ok) break;
        tc_commit(tfull_bar(b));
      }
      if (!ok) break;
      tc_commit(aempty_bar(a));  // A buffer a is free once this block's MMAs finish
    }
    if (!ok) raise_abort();
    tc_commit(mdone_bar);
    mbar_wait_bounded(mdone_bar, 0, nullptr, kL1DrainNs);
  } else if (warp >= 2 && warp < kEncWarp0) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    constexpr int kChunks = S::BN / 32 / (EPI / 4);
    const int half = (warp - 2) / 4;
    uint8_t* boxes = smem + S::out_off(p.N) + (warp - 2) * S::OUT_DEPTH * S::OUT_BOX;
    uint32_t issued = 0;
    int local = 0;
    for (int mb = blockIdx.x; mb < num_m; mb += gridDim.x) {
      bool ok = true;
      for (int nb = 0; nb < num_n; ++nb, ++local) {
        const int b = local & 1;
        ok = mbar_wait_bounded(tfull_bar(b), (local >> 1) & 1, abort_flag, p.timeout_ns);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) raise_abort();
          break;
        }
        tc_fence_after();
        const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                               static_cast<uint32_t>(b * S::BN);
        epi_tile_tma<OUT_FP8, S::OUT_DEPTH>(p, ev, &tmO, tbase, mb * S::BM + q * 32, nb * S::BN,
                                            half * kChunks, (half + 1) * kChunks, boxes, lane,
                                            issued);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(b));
      }
      if (!ok) break;
    }
    // the boxes must stay untouched until every store has read them, and the
    // outputs be written before the kernel ends
    if (lane == 0) bulk_wait_group<0>();
    __syncwarp();
  } else if (warp >= kEncWarp0) {
    // ---------------------------------------------------------- encoder
    const int r = threadIdx.x - 32 * kEncWarp0;  // row of the 128-ray block
    const int pieces = 8 * kb_count;             // 16-byte pieces per row (8 bf16 each)
    int blk = 0;
    for (int mb = blockIdx.x; mb < num_m; mb += gridDim.x, ++blk) {
      const int a = blk & 1;
      const int64_t row = static_cast<int64_t>(mb) * S::BM + r;
      float e[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) e[c] = row < p.M ? ray_ld(rays, c, row) : 0.f;
      bool ok = mbar_wait_bounded(aempty_bar(a), ((blk >> 1) & 1) ^ 1u, abort_flag, p.timeout_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) raise_abort();
        break;
      }
      uint8_t* buf = sA + a * S::A_BUF;
      int c = 0, k = 0;
      // piece 0: the raw ray (6 values) and the first (sin, cos) pair
      uint4 pc;
      pc.x = epi_pack_bf16x2(e[0], e[1]);
      pc.y = epi_pack_bf16x2(e[2], e[3]);
      pc.z = epi_pack_bf16x2(e[4], e[5]);
      pc.w = next_pair(e, L, c, k);
      *reinterpret_cast<uint4*>(buf + a_piece_offset(r, 0)) = pc;
      for (int qp = 1; qp < pieces; ++qp) {
        pc.x = next_pair(e, L, c, k);
        pc.y = next_pair(e, L, c, k);
        pc.z = next_pair(e, L, c, k);
        pc.w = next_pair(e, L, c, k);
        *reinterpret_cast<uint4*>(buf + a_piece_offset(r, qp)) = pc;
      }
      fence_proxy_async_smem();  // the MMAs read these pieces through the async proxy
      __syncwarp();
      if (lane == 0) mbar_arrive(afull_bar(a));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, S::TMEM_COLS);
  }
}

template <bool OUT_FP8, int EPI>
cudaError_t launch_l1(const CUtensorMap& tmB, const CUtensorMap& tmO, RaySoA rays, int L,
                      const TcGemmParams& p, int grid, cudaStream_t s) {
  auto kern = tc_layer1_kernel<OUT_FP8, EPI>;
  const int smem = L1Shape<EPI>::smem_bytes(p.N);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 64 + 32 * EPI + 128, smem, s>>>(tmB, tmO, rays, L, p);
  return cudaGetLastError();
}

}  // namespace

bool tc_layer1_supported(int L, int N) {
  return L >= 1 && 6 + 12 * L <= 64 * L1Shape<4>::KB_MAX && N % L1Shape<4>::BN == 0 &&
         N <= kMaxStagedColumns && L1Shape<4>::smem_bytes(N) <= 232448 &&
         L1Shape<8>::smem_bytes(N) <= 232448;
}

cudaError_t launch_tc_layer1(int epi_warps, bool out_fp8, const CUtensorMap& tmB,
                             const CUtensorMap& tmO, RaySoA rays, int L, const TcGemmParams& p,
                             int grid, cudaStream_t s) {
  if (!tc_layer1_supported(L, p.N) || p.mode != 0 || p.amax != nullptr || p.m_dev != nullptr ||
      p.col_scale != nullptr || p.out == nullptr || p.bias == nullptr || p.M <= 0 || grid <= 0)
    return cudaErrorInvalidValue;
  if (epi_warps == 4) return out_fp8 ? launch_l1<true, 4>(tmB, tmO, rays, L, p, grid, s)
                                     : launch_l1<false, 4>(tmB, tmO, rays, L, p, grid, s);
  if (epi_warps == 8) return out_fp8 ? launch_l1<true, 8>(tmB, tmO, rays, L, p, grid, s)
                                     : launch_l1<false, 8>(tmB, tmO, rays, L, p, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace ddf
