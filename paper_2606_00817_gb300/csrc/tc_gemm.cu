// tc_gemm.cu -- one dense DDF layer on the sm_103a tensor cores.
//
// The hidden layers of the DDF MLP (Sec. 3.1 / Sec. 4.3: a wide ReLU MLP on the
// encoded ray) are the whole cost of a query at width 1280. Each layer is a
// GEMM  Y[M x N] = A[M x K] W[N x K]^T  over a chunk of M rays, followed by
// bias + ReLU. This kernel is persistent (one CTA per SM) and warp-specialised:
//   warp 0      TMA producer: 128-byte-swizzled A and W tiles into a ring of
//               shared-memory stages (mbarrier full/empty handshake)
//   warp 1      allocates TMEM; one thread issues tcgen05.mma (M=128, N=BN,
//               K=16 bf16 / 32 e4m3 per instruction) into a double-buffered
//               FP32 accumulator in TMEM, so the epilogue of tile i overlaps the
//               MMAs of tile i+1
//   warps 2-5   epilogue: tcgen05.ld of the accumulator (thread = ray row),
//               scale, bias, ReLU, then either the next layer's activation
//               (bf16 or e4m3, vectorised stores) or, for the last hidden layer,
//               the two FP32 head dot products (one partial per N-block).
// Tiles are ordered N-fastest so the N/BN CTAs that share an A row-block run
// at the same time and A is read from HBM about once. Every wait is bounded
// (globaltimer); a timeout raises a CTA abort flag and a status bit, the
// producer drains its in-flight copies and the MMA thread its in-flight MMAs
// before TMEM is released.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"
#include "epilogue.cuh"
#include "ptx_sm103.cuh"

namespace ddf {

namespace {

constexpr uint64_t kDrainTimeoutNs = 1000000000ull;  // 1 s for drains at teardown

template <int BN, bool IN_FP8>
struct TcShape {
  static constexpr int BM = 128;
  static constexpr int ROW_BYTES = 128;                 // one 128-byte swizzle row along K
  static constexpr int BK = IN_FP8 ? 128 : 64;          // K elements per stage
  static constexpr int A_BYTES = BM * ROW_BYTES;        // 16 KB
  static constexpr int B_BYTES = BN * ROW_BYTES;        // 16 or 32 KB
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (BN == 256) ? 4 : 6;
  static constexpr int TMEM_COLS = 2 * BN;              // two FP32 accumulators
  static constexpr int NUM_BARS = 2 * STAGES + 5;
  static constexpr int CTRL_BYTES = 256;  // barriers, TMEM slot, abort flag
  static constexpr int VEC_OFFSET = STAGES * STAGE_BYTES + CTRL_BYTES;
  // plus epi_vector_bytes(N) for the staged per-column vectors
  static constexpr int SMEM_BYTES = VEC_OFFSET + 1024;
  static_assert(NUM_BARS * 8 + 8 <= CTRL_BYTES, "control block overflow");
  static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation must be a power of two");
};

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, uint32_t* status) {
  *abort_flag = 1;
  atomicOr(status, kStatusPipelineTimeout);
}

template <int BN, bool IN_FP8, bool OUT_FP8, int EPI>
__global__ void __launch_bounds__(64 + 32 * EPI, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcGemmParams p) {
  using S = TcShape<BN, IN_FP8>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::STAGES * S::A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::STAGES * S::STAGE_BYTES);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S::STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * S::STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * S::STAGES + 2 + b); };
  const uint32_t mdone_bar = bar0 + 8u * (2 * S::STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S::NUM_BARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), EPI);  // one arrival per epilogue warp
    }
    mbar_init(mdone_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), S::TMEM_COLS);
    tmem_relinquish();
  }
  const EpiVectors ev = stage_epi_vectors(p, reinterpret_cast<float*>(smem + S::VEC_OFFSET));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // rows this launch computes: p.M, or fewer when a device-side count
  // (written by an earlier kernel of the stream) is given; p.M stays the row
  // stride of the head partials
  const int m_rows = p.m_dev != nullptr ? min(*p.m_dev, p.M) : p.M;
  const int num_m = (m_rows + S::BM - 1) / S::BM;
  const int num_n = p.N / BN;
  const int num_kb = (p.K + S::BK - 1) / S::BK;
  // split-K (mode 3): tile = (split, m block, n block); split s covers the
  // k-blocks [s num_kb / splits, (s+1) num_kb / splits) (the launcher makes
  // every split non-empty)
  const int splits = p.k_splits > 1 ? p.k_splits : 1;
  auto kb_lo = [&](int split) { return static_cast<int>((static_cast<int64_t>(split) * num_kb) / splits); };
  const int num_tiles = splits * num_m * num_n;
  auto decode = [&](int tile, int& split, int& m_blk, int& n_blk) {
    split = tile / (num_m * num_n);
    const int r = tile - split * num_m * num_n;
    m_blk = r / num_n;
    n_blk = r - m_blk * num_n;
  };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int split, m_blk, n_blk;
      decode(tile, split, m_blk, n_blk);
      const int m0 = m_blk * S::BM;
      const int n0 = n_blk * BN;
      for (int kb = kb_lo(split); kb < kb_lo(split + 1); ++kb, ++it) {
        const int s = it % S::STAGES;
        const uint32_t ph = (it / S::STAGES) & 1;
        if (!mbar_wait_bounded(empty_bar(s), ph ^ 1u, abort_flag, p.timeout_ns)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(full_bar(s), S::STAGE_BYTES);
        if (!IN_FP8 && p.mn_major) {
          // 64-wide boxes along M (N), each BK rows of K: 8 KB apiece
#pragma unroll
          for (int j = 0; j < S::BM / 64; ++j)
            tma_load_2d(smem_u32(sA + s * S::A_BYTES + j * 64 * S::BK * 2), &tmA, m0 + 64 * j,
                        kb * S::BK, full_bar(s));
#pragma unroll
          for (int j = 0; j < BN / 64; ++j)
            tma_load_2d(smem_u32(sB + s * S::B_BYTES + j * 64 * S::BK * 2), &tmB, n0 + 64 * j,
                        kb * S::BK, full_bar(s));
        } else {
          tma_load_2d(smem_u32(sA + s * S::A_BYTES), &tmA, kb * S::BK, m0, full_bar(s));
          tma_load_2d(smem_u32(sB + s * S::B_BYTES), &tmB, kb * S::BK, n0, full_bar(s));
        }
      }
    }
    if (!ok) {
      raise_abort(abort_flag, p.status);
      // let every copy still in flight land before the CTA may exit
      const int first = it > S::STAGES ? it - S::STAGES : 0;
      for (int j = first; j < it; ++j)
        mbar_wait_bounded(full_bar(j % S::STAGES), (j / S::STAGES) & 1, nullptr, kDrainTimeoutNs);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc_k = mma_idesc(IN_FP8 ? 0u : 1u, BN, S::BM);
    const bool mn = !IN_FP8 && p.mn_major != 0;
    const uint32_t idesc = mn ? (idesc_k | (1u << 15) | (1u << 16)) : idesc_k;
    constexpr uint32_t kBoxBytes = 64 * S::BK * 2;  // one MN-major box (bf16)
    int it = 0, local = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++local) {
      const int b = local & 1;
      const uint32_t aph = (local >> 1) & 1;
      if (!mbar_wait_bounded(tempty_bar(b), aph ^ 1u, abort_flag, p.timeout_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(b * BN);
      const int split = tile / (num_m * num_n);
      const int kb0 = kb_lo(split), kb1 = kb_lo(split + 1);
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = it % S::STAGES;
        const uint32_t ph = (it / S::STAGES) & 1;
        if (!mbar_wait_bounded(full_bar(s), ph, abort_flag, p.timeout_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + s * S::A_BYTES);
        const uint32_t b0 = smem_u32(sB + s * S::B_BYTES);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // K-major: 4 x 32 bytes of K per 128-byte row; MN-major: 4 x 16 K
          // rows of 128 bytes (two 1024-byte atoms)
          const uint64_t ad = mn ? sw128_mnmajor_desc(a0 + 2048u * j, kBoxBytes)
                                 : sw128_kmajor_desc(a0 + 32u * j);
          const uint64_t bd = mn ? sw128_mnmajor_desc(b0 + 2048u * j, kBoxBytes)
                                 : sw128_kmajor_desc(b0 + 32u * j);
          const uint32_t acc = (kb != kb0 || j != 0) ? 1u : 0u;
          if constexpr (IN_FP8)
            tc_mma_f8(d_tmem, ad, bd, idesc, acc);
          else
            tc_mma_f16(d_tmem, ad, bd, idesc, acc);
        }
        tc_commit(empty_bar(s));  // stage s is free once these MMAs finish
      }
      if (!ok) break;
      tc_commit(tfull_bar(b));  // accumulator b is complete
    }
    if (!ok) raise_abort(abort_flag, p.status);
    tc_commit(mdone_bar);  // every MMA above has finished once this arrives
    mbar_wait_bounded(mdone_bar, 0, nullptr, kDrainTimeoutNs);
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    // with 8 epilogue warps, two warps share a lane quarter and split the columns
    constexpr int kChunks = BN / 32 / (EPI / 4);
    const int half = (warp - 2) / 4;
    const int r_local = q * 32 + lane;
    int local = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++local) {
      const int b = local & 1;
      const uint32_t aph = (local >> 1) & 1;
      bool ok = mbar_wait_bounded(tfull_bar(b), aph, abort_flag, p.timeout_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) raise_abort(abort_flag, p.status);
        break;
      }
      tc_fence_after();
      int split, m_blk, n_blk;
      decode(tile, split, m_blk, n_blk);
      const int row = m_blk * S::BM + r_local;
      const bool row_ok = row < m_rows;
      const int n0 = n_blk * BN;
      const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                             static_cast<uint32_t>(b * BN);
      float h0 = 0.f, h1 = 0.f;
      if (p.mode >= 2)
        epi_row_train(p, tbase, row, row_ok, n0, half * kChunks, (half + 1) * kChunks, split);
      else
        epi_row<OUT_FP8>(p, ev, tbase, row, row_ok, n0, half * kChunks, (half + 1) * kChunks, h0,
                         h1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(b));
      if (p.mode == 1 && row_ok)
        p.head_part[(static_cast<size_t>(n_blk) * (EPI / 4) + half) * p.M + row] =
            make_float2(h0, h1);
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

template <int BN, bool IN_FP8, bool OUT_FP8, int EPI>
cudaError_t launch_one(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmParams& p,
                       int grid, cudaStream_t s) {
  using S = TcShape<BN, IN_FP8>;
  auto kern = tc_gemm_kernel<BN, IN_FP8, OUT_FP8, EPI>;
  // applies to the current device; cheap enough to repeat on every launch
  if (p.k_splits > 1 && (p.K + S::BK - 1) / S::BK < p.k_splits) return cudaErrorInvalidValue;
  if (p.mn_major && IN_FP8) return cudaErrorInvalidValue;
  const int smem = S::SMEM_BYTES + epi_vector_bytes(p.N);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 64 + 32 * EPI, smem, s>>>(tmA, tmB, p);
  return cudaGetLastError();
}

template <int BN, int EPI>
cudaError_t launch_bn(bool in_fp8, bool out_fp8, const CUtensorMap& tmA, const CUtensorMap& tmB,
                      const TcGemmParams& p, int grid, cudaStream_t s) {
  if (in_fp8) return out_fp8 ? launch_one<BN, true, true, EPI>(tmA, tmB, p, grid, s)
                             : launch_one<BN, true, false, EPI>(tmA, tmB, p, grid, s);
  return out_fp8 ? launch_one<BN, false, true, EPI>(tmA, tmB, p, grid, s)
                 : launch_one<BN, false, false, EPI>(tmA, tmB, p, grid, s);
}

}  // namespace

int tc_gemm_smem_bytes(int bn, bool in_fp8) {
  if (bn == 256) return in_fp8 ? TcShape<256, true>::SMEM_BYTES : TcShape<256, false>::SMEM_BYTES;
  return in_fp8 ? TcShape<128, true>::SMEM_BYTES : TcShape<128, false>::SMEM_BYTES;
}

cudaError_t launch_tc_gemm(const TcTile& tile, bool in_fp8, bool out_fp8, const CUtensorMap& tmA,
                           const CUtensorMap& tmB, const TcGemmParams& p, int grid,
                           cudaStream_t s) {
  if (!epi_out_aligned(p, out_fp8)) return cudaErrorInvalidValue;
  if (tile.bn == 256 && tile.epi_warps == 4) return launch_bn<256, 4>(in_fp8, out_fp8, tmA, tmB, p, grid, s);
  if (tile.bn == 256 && tile.epi_warps == 8) return launch_bn<256, 8>(in_fp8, out_fp8, tmA, tmB, p, grid, s);
  if (tile.bn == 128 && tile.epi_warps == 4) return launch_bn<128, 4>(in_fp8, out_fp8, tmA, tmB, p, grid, s);
  if (tile.bn == 128 && tile.epi_warps == 8) return launch_bn<128, 8>(in_fp8, out_fp8, tmA, tmB, p, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace ddf
