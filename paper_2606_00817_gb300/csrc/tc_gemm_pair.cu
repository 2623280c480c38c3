// tc_gemm_pair.cu -- one dense DDF layer on a pair of SMs (tcgen05 cta_group::2).
//
// Same layer as tc_gemm.cu (Y = act(A W^T * scale + b), Sec. 3.1 / Sec. 4.3,
// and the training modes: masked input gradients, split-K weight gradients
// with MN-major operands),
// but each 256 x 256 output tile is computed by a cluster of two CTAs that
// share one MMA: CTA r of the pair loads rows [128 r, 128 r + 128) of the A
// tile and rows [128 r, 128 r + 128) of the W tile into its own shared memory,
// and the leader CTA (rank 0) issues tcgen05.mma.cta_group::2 with M = 256,
// N = 256, which reads A and W from both CTAs and leaves the 128 x 256
// accumulator of each CTA's rows in that CTA's TMEM. Per SM this halves the
// shared-memory operand traffic of the 128 x 256 single-CTA tile (each SM now
// stages 32 KB instead of 48 KB per 64-wide K step for the same MMA work).
//
// Synchronisation:
//   full[s]     (leader) both CTAs' TMA copies of stage s land here; the
//               leader's producer arms it with the bytes of both halves
//   empty[s]    (each CTA) the leader's commit multicasts "stage s consumed"
//   tfull[b]    (each CTA) the leader's commit multicasts "accumulator b ready"
//   tempty[b]   (leader) every epilogue warp of both CTAs arrives (relaxed:
//               its TMEM reads are complete): "b drained"
// Every wait is bounded. A timeout raises the abort flag of both CTAs and a
// status bit. At teardown both producers publish how many stages they issued;
// after a cluster barrier the one that issued fewer copies the missing stage
// halves (in-bounds dummy loads) so that every armed barrier phase completes,
// the leader waits for those phases, and a second cluster barrier precedes
// the collective TMEM release.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"
#include "epilogue.cuh"
#include "ptx_sm103.cuh"

namespace ddf {

namespace {

constexpr uint64_t kPairDrainNs = 1000000000ull;

// STAGED: mode-0 outputs go through per-warp shared staging buffers
// (epi_row_staged); one pipeline stage fewer leaves room for them. EPI:
// epilogue warps per CTA (warps 2..), 4 (one per TMEM lane quarter) or 8
// (two per quarter, each draining half of the tile's columns).
template <bool IN_FP8, bool STAGED, int EPI = 4>
struct PairShape {
  static constexpr int BM = 256;                 // output rows per pair tile
  static constexpr int BN = 256;                 // output columns per pair tile
  static constexpr int HALF = 128;               // rows of A and of W per CTA
  static constexpr int ROW_BYTES = 128;
  static constexpr int BK = IN_FP8 ? 128 : 64;   // K elements per stage
  static constexpr int A_BYTES = HALF * ROW_BYTES;
  static constexpr int B_BYTES = HALF * ROW_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // per CTA
  static constexpr int STAGES = STAGED ? 5 : 6;
  // staged outputs: per epilogue warp OUT_DEPTH boxes of 32 rows x 128 bytes
  // (two with 4 warps, so a warp packs the next box while the TMA store of
  // the last one still reads it; one with 8)
  static constexpr int OUT_DEPTH = EPI == 4 ? 2 : 1;
  static constexpr int OUT_STAGE_BYTES = STAGED ? EPI * OUT_DEPTH * kStageBytesPerWarp : 0;
  static constexpr int EPI_WARP0 = 2;  // first epilogue warp
  static constexpr int THREADS = 32 * (EPI_WARP0 + EPI);
  static constexpr int TMEM_COLS = 512;
  static constexpr int NUM_BARS = 2 * STAGES + 5;
  static constexpr int CTRL_BYTES = 256;  // barriers, TMEM slot, abort flag, issue counts
  static constexpr int VEC_OFFSET = STAGES * STAGE_BYTES + CTRL_BYTES;
  // then epi_vector_bytes(N) for the staged per-column vectors, then the
  // output boxes on a 1024-byte boundary (the 128-byte swizzle atom)
  __host__ __device__ static constexpr int out_off(int n) {
    return (VEC_OFFSET + epi_vector_bytes(n) + 1023) & ~1023;
  }
  __host__ __device__ static constexpr int smem_bytes(int n) {
    return out_off(n) + OUT_STAGE_BYTES + 1024;  // + 1024: base alignment
  }
  static_assert(NUM_BARS * 8 + 16 <= CTRL_BYTES, "control block overflow");
};

// TM: the work the instantiation serves. 0: the query modes (0, 1) with
// thread stores; 1: mode 0 leaving by TMA stores (the staged hidden-layer
// tile); 5: mode 1 alone (the last layer's head partials, nothing stored);
// else one training mode, bf16 only (2: input gradients masked by the
// stored activation; 3: split-K weight gradients with K-major or MN-major
// operands; 4: the last layer's forward with the head partials). Each
// compiles only its own epilogue and operand paths, so no mode's loop shares
// registers or schedule with another's (one instantiation for all three
// training modes ran a plain forward epilogue 20 % slower).
template <bool IN_FP8, bool OUT_FP8, bool STAGED, int TM, int EPI = 4>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32 * (2 + EPI), 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmO, const TcGemmParams p) {
  using S = PairShape<IN_FP8, STAGED, EPI>;
  constexpr bool TRAIN = TM >= 2 && TM <= 4;
  static_assert(TM >= 0 && TM <= 5, "instantiation kind");
  static_assert(TM != 1 || STAGED, "TMA stores leave through the staging boxes");
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
  volatile uint32_t* issued = reinterpret_cast<volatile uint32_t*>(tmem_slot + 2);  // [2]

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();  // 0: leader, issues the MMAs
  const int pair = blockIdx.x >> 1;
  const int npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 2 * EPI);  // every epilogue warp of both CTAs
    }
    mbar_init(mdone_bar, 1);
    *abort_flag = 0;
    issued[0] = 0;
    issued[1] = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), S::TMEM_COLS);  // collective with the peer's warp 1
    tmem_relinquish_pair();
  }
  const EpiVectors ev = stage_epi_vectors(p, reinterpret_cast<float*>(smem + S::VEC_OFFSET));
  tc_fence_before();
  cluster_sync_all();  // barriers of both CTAs initialised, TMEM allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const uint32_t full_leader0 = map_to_cta(full_bar(0), 0);
  const uint32_t abort_peer = map_to_cta(smem_u32(const_cast<int*>(abort_flag)), rank ^ 1u);
  auto raise_abort = [&]() {
    *abort_flag = 1;
    st_cluster_u32(abort_peer, 1u);
    atomicOr(p.status, kStatusPipelineTimeout);
  };

  const int num_m = (p.M + S::BM - 1) / S::BM;
  const int num_n = p.N / S::BN;
  const int num_kb = (p.K + S::BK - 1) / S::BK;
  // split-K (mode 3): tile = (split, m block, n block); split s covers the
  // k-blocks [s num_kb / splits, (s+1) num_kb / splits)
  const int splits = (TM == 3 && p.k_splits > 1) ? p.k_splits : 1;
  auto kb_lo = [&](int split) {
    if constexpr (TM != 3) return split * num_kb;
    return static_cast<int>((static_cast<int64_t>(split) * num_kb) / splits);
  };
  const int num_tiles = splits * num_m * num_n;
  auto decode = [&](int tile, int& split, int& m_blk, int& n_blk) {
    split = tile / (num_m * num_n);
    const int r = tile - split * num_m * num_n;
    m_blk = r / num_n;
    n_blk = r - m_blk * num_n;
  };
  // MN-major operands (bf16): A as [K x M], B as [K x N] row-major, loaded as
  // 64-wide boxes of BK rows (8 KB each, two per operand half)
  const bool mn = TM == 3 && !IN_FP8 && p.mn_major != 0;
  constexpr uint32_t kBoxBytes = 64 * S::BK * 2;
  auto load_stage = [&](int s, int m0, int nb, int kb, uint32_t bar) {
    if (mn) {
#pragma unroll
      for (int j = 0; j < S::HALF / 64; ++j) {
        tma_load_2d_pair(smem_u32(sA + s * S::A_BYTES) + j * kBoxBytes, &tmA, m0 + 64 * j,
                         kb * S::BK, bar);
        tma_load_2d_pair(smem_u32(sB + s * S::B_BYTES) + j * kBoxBytes, &tmB, nb + 64 * j,
                         kb * S::BK, bar);
      }
    } else {
      tma_load_2d_pair(smem_u32(sA + s * S::A_BYTES), &tmA, kb * S::BK, m0, bar);
      tma_load_2d_pair(smem_u32(sB + s * S::B_BYTES), &tmB, kb * S::BK, nb, bar);
    }
  };

  // Roles: warp 0 lane 0 produces, warp 1 lane 0 of the leader issues the
  // MMAs, warps EPI_WARP0.. drain the accumulators.
  if (warp < S::EPI_WARP0) {
  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    uint32_t it = 0;
    bool ok = true;
    for (int tile = pair; tile < num_tiles && ok; tile += npairs) {
      int split, m_blk, n_blk;
      decode(tile, split, m_blk, n_blk);
      const int m0 = m_blk * S::BM + static_cast<int>(rank) * S::HALF;
      const int nb = n_blk * S::BN + static_cast<int>(rank) * S::HALF;
      const int kb1 = kb_lo(split + 1);
      for (int kb = kb_lo(split); kb < kb1; ++kb, ++it) {
        const int s = it % S::STAGES;
        const uint32_t ph = (it / S::STAGES) & 1;
        if (!mbar_wait_bounded(empty_bar(s), ph ^ 1u, abort_flag, p.timeout_ns)) {
          ok = false;
          break;
        }
        if (rank == 0) mbar_arrive_expect_tx(full_bar(s), 2 * S::STAGE_BYTES);
        load_stage(s, m0, nb, kb, full_leader0 + 8u * s);
      }
    }
    if (!ok) raise_abort();
    const uint32_t slot = smem_u32(const_cast<uint32_t*>(issued)) + 4u * rank;
    st_cluster_u32(map_to_cta(slot, 0), it);
    st_cluster_u32(map_to_cta(slot, 1), it);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------------------------------------------------- MMA issuer (leader)
    constexpr uint32_t idesc_k = mma_idesc(IN_FP8 ? 0u : 1u, S::BN, S::BM);
    const uint32_t idesc = mn ? (idesc_k | (1u << 15) | (1u << 16)) : idesc_k;
    int it = 0, local = 0;
    bool ok = true;
    for (int tile = pair; tile < num_tiles && ok; tile += npairs, ++local) {
      const int b = local & 1;
      const uint32_t aph = (local >> 1) & 1;
      if (!mbar_wait_bounded(tempty_bar(b), aph ^ 1u, abort_flag, p.timeout_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(b * S::BN);
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
          // rows of 128 bytes
          const uint64_t ad = mn ? sw128_mnmajor_desc(a0 + 2048u * j, kBoxBytes)
                                 : sw128_kmajor_desc(a0 + 32u * j);
          const uint64_t bd = mn ? sw128_mnmajor_desc(b0 + 2048u * j, kBoxBytes)
                                 : sw128_kmajor_desc(b0 + 32u * j);
          const uint32_t acc = (kb != kb0 || j != 0) ? 1u : 0u;
          if constexpr (IN_FP8)
            tc_mma_pair_f8(d_tmem, ad, bd, idesc, acc);
          else
            tc_mma_pair_f16(d_tmem, ad, bd, idesc, acc);
        }
        tc_commit_pair_multicast(empty_bar(s), 0x3);  // stage s free in both CTAs
      }
      if (!ok) break;
      tc_commit_pair_multicast(tfull_bar(b), 0x3);  // accumulator b ready in both CTAs
    }
    if (!ok) raise_abort();
    tc_commit_pair(mdone_bar);
    mbar_wait_bounded(mdone_bar, 0, nullptr, kPairDrainNs);
  }
  } else {
    // ---------------------------------------------------------- epilogue (both CTAs)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int half = EPI == 4 ? 0 : (warp - S::EPI_WARP0) / 4;
    constexpr int kChunks = S::BN / 32 / (EPI / 4);  // 32-column chunks per warp
    const int c0 = half * kChunks, c1 = c0 + kChunks;
    uint8_t* const stage_w =
        smem + S::out_off(p.N) + (warp - S::EPI_WARP0) * S::OUT_DEPTH * kStageBytesPerWarp;
    const int r_local = q * 32 + lane;
    const uint32_t tempty_leader0 = map_to_cta(tempty_bar(0), 0);
    uint32_t stores = 0;  // TMA stores this warp issued
    int local = 0;
    for (int tile = pair; tile < num_tiles; tile += npairs, ++local) {
      const int b = local & 1;
      const uint32_t aph = (local >> 1) & 1;
      bool ok = mbar_wait_bounded(tfull_bar(b), aph, abort_flag, p.timeout_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) raise_abort();
        break;
      }
      tc_fence_after();
      int split, m_blk, n_blk;
      decode(tile, split, m_blk, n_blk);
      const int row = m_blk * S::BM + static_cast<int>(rank) * S::HALF + r_local;
      const bool row_ok = row < p.M;
      const int n0 = n_blk * S::BN;
      const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                             static_cast<uint32_t>(b * S::BN);
      float h0 = 0.f, h1 = 0.f;
      if constexpr (TRAIN) {
        static_assert(kChunks % 4 == 0, "the masked epilogue steps over 4 chunks");
        if constexpr (TM == 4)
          epi_row_staged_head(p, ev, tbase, row - lane, n0, c0, c1, stage_w, lane, h0, h1);
        else if constexpr (TM == 2)
          epi_row_masked_staged(p, tbase, row - lane, n0, c0, c1, stage_w, lane);
        else
          epi_row_train(p, tbase, row, row_ok, n0, c0, c1, split);
      } else if constexpr (TM == 1) {
        epi_tile_tma<OUT_FP8, S::OUT_DEPTH>(p, ev, &tmO, tbase, row - lane, n0, c0, c1, stage_w,
                                            lane, stores);
      } else if constexpr (TM == 5) {
        epi_row<OUT_FP8, true>(p, ev, tbase, row, row_ok, n0, c0, c1, h0, h1);
      } else if (STAGED && p.mode == 0) {
        epi_row_staged<OUT_FP8>(p, ev, tbase, row - lane, n0, c0, c1, stage_w, lane);
      } else {
        epi_row<OUT_FP8>(p, ev, tbase, row, row_ok, n0, c0, c1, h0, h1);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty_leader0 + 8u * b);
      if ((p.mode == 1 || p.mode == 4) && row_ok)
        p.head_part[(static_cast<size_t>(n_blk) * (EPI / 4) + half) * p.M + row] =
            make_float2(h0, h1);
    }
    // the boxes must stay untouched until every store has read them, and the
    // outputs be written before the kernel ends
    if (!TRAIN && STAGED && lane == 0) bulk_wait_group<0>();
    __syncwarp();
  }

  // ---------------------------------------------------------- teardown
  tc_fence_before();
  cluster_sync_all();  // #1: no role issues anything new; issue counts published
  if (warp == 0 && lane == 0) {
    const uint32_t mine = issued[rank], other = issued[rank ^ 1u];
    // Copy this CTA's half of any stage the other producer issued and this one
    // did not (only after an abort), so every armed full[] phase can complete.
    for (uint32_t j = mine; j < other; ++j) {
      const int s = j % S::STAGES;
      if (rank == 0) mbar_arrive_expect_tx(full_bar(s), 2 * S::STAGE_BYTES);
      load_stage(s, 0, 0, 0, full_leader0 + 8u * s);
    }
    if (rank == 0) {
      const uint32_t jmax = mine > other ? mine : other;
      const uint32_t jlo = jmax > static_cast<uint32_t>(S::STAGES) ? jmax - S::STAGES : 0u;
      for (uint32_t j = jlo; j < jmax; ++j)
        mbar_wait_bounded(full_bar(j % S::STAGES), (j / S::STAGES) & 1, nullptr, kPairDrainNs);
    }
  }
  tc_fence_before();
  cluster_sync_all();  // #2: every copy landed, every MMA finished
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, S::TMEM_COLS);
  }
}

template <bool IN_FP8, bool OUT_FP8, bool STAGED, int TM = 0, int EPI = 4>
cudaError_t launch_pair_one(const CUtensorMap& tmA, const CUtensorMap& tmB, const CUtensorMap& tmO,
                            const TcGemmParams& p, int grid, cudaStream_t s) {
  using S = PairShape<IN_FP8, STAGED, EPI>;
  auto kern = tc_gemm_pair_kernel<IN_FP8, OUT_FP8, STAGED, TM, EPI>;
  const int smem = S::smem_bytes(p.N);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, S::THREADS, smem, s>>>(tmA, tmB, tmO, p);
  return cudaGetLastError();
}

template <bool IN_FP8, bool STAGED, int EPI>
int max_pairs_for() {
  using S = PairShape<IN_FP8, STAGED, EPI>;
  auto kern = tc_gemm_pair_kernel<IN_FP8, false, STAGED, 0, EPI>;
  const int smem = S::smem_bytes(kMaxStagedColumns);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2, 1, 1);
  cfg.blockDim = dim3(S::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <bool IN_FP8, bool STAGED, int EPI>
cudaError_t launch_pair_io(bool out_fp8, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const CUtensorMap& tmO, const TcGemmParams& p, int grid,
                           cudaStream_t s) {
  return out_fp8 ? launch_pair_one<IN_FP8, true, STAGED, 0, EPI>(tmA, tmB, tmO, p, grid, s)
                 : launch_pair_one<IN_FP8, false, STAGED, 0, EPI>(tmA, tmB, tmO, p, grid, s);
}

// The last layer (mode 1: head partials only): nothing is staged, so the
// unstaged layout and its deeper operand ring serve every tile.
template <int EPI>
cudaError_t launch_pair_head(bool in_fp8, const CUtensorMap& tmA, const CUtensorMap& tmB,
                             const CUtensorMap& tmO, const TcGemmParams& p, int grid,
                             cudaStream_t s) {
  return in_fp8 ? launch_pair_one<true, false, false, 5, EPI>(tmA, tmB, tmO, p, grid, s)
                : launch_pair_one<false, false, false, 5, EPI>(tmA, tmB, tmO, p, grid, s);
}

// The staged mode-0 tile whose outputs leave by TMA stores.
template <int EPI>
cudaError_t launch_pair_tma(bool in_fp8, bool out_fp8, const CUtensorMap& tmA,
                            const CUtensorMap& tmB, const CUtensorMap& tmO,
                            const TcGemmParams& p, int grid, cudaStream_t s) {
  if (in_fp8) return out_fp8 ? launch_pair_one<true, true, true, 1, EPI>(tmA, tmB, tmO, p, grid, s)
                             : launch_pair_one<true, false, true, 1, EPI>(tmA, tmB, tmO, p, grid, s);
  return out_fp8 ? launch_pair_one<false, true, true, 1, EPI>(tmA, tmB, tmO, p, grid, s)
                 : launch_pair_one<false, false, true, 1, EPI>(tmA, tmB, tmO, p, grid, s);
}

template <int EPI>
cudaError_t launch_pair_epi(bool in_fp8, bool out_fp8, bool staged, const CUtensorMap& tmA,
                            const CUtensorMap& tmB, const CUtensorMap& tmO,
                            const TcGemmParams& p, int grid, cudaStream_t s) {
  if (in_fp8) return staged ? launch_pair_io<true, true, EPI>(out_fp8, tmA, tmB, tmO, p, grid, s)
                            : launch_pair_io<true, false, EPI>(out_fp8, tmA, tmB, tmO, p, grid, s);
  return staged ? launch_pair_io<false, true, EPI>(out_fp8, tmA, tmB, tmO, p, grid, s)
                : launch_pair_io<false, false, EPI>(out_fp8, tmA, tmB, tmO, p, grid, s);
}

}  // namespace

int tc_gemm_pair_max_clusters(bool in_fp8) {
  int n = 1 << 30;
  const int v[4] = {in_fp8 ? max_pairs_for<true, false, 4>() : max_pairs_for<false, false, 4>(),
                    in_fp8 ? max_pairs_for<true, true, 4>() : max_pairs_for<false, true, 4>(),
                    in_fp8 ? max_pairs_for<true, false, 8>() : max_pairs_for<false, false, 8>(),
                    in_fp8 ? max_pairs_for<true, true, 8>() : max_pairs_for<false, true, 8>()};
  for (int x : v) n = x < n ? x : n;
  return n;
}

cudaError_t launch_tc_gemm_pair(bool in_fp8, bool out_fp8, bool staged, int epi_warps,
                                const CUtensorMap& tmA, const CUtensorMap& tmB,
                                const TcGemmParams& p, int clusters, cudaStream_t s,
                                const CUtensorMap* tmO) {
  if (p.tma_out && (tmO == nullptr || !staged || p.mode != 0 || p.amax != nullptr))
    return cudaErrorInvalidValue;  // TMA stores: the staged query tile, with its output map
  if (!p.tma_out && !epi_out_aligned(p, out_fp8)) return cudaErrorInvalidValue;
  const CUtensorMap& to = tmO != nullptr ? *tmO : tmA;  // not read unless p.tma_out
  if (p.mode == 3 && (p.k_splits > 1 ? p.k_splits : 1) > (p.K + 63) / 64)
    return cudaErrorInvalidValue;  // every split needs a k-block
  if (p.mn_major && (in_fp8 || p.mode != 3)) return cudaErrorInvalidValue;
  if (p.mode >= 2 && (in_fp8 || out_fp8)) return cudaErrorInvalidValue;
  if (p.mode == 4 && (p.head_w == nullptr || p.head_part == nullptr)) return cudaErrorInvalidValue;
  if (p.mode == 2 && (p.mask == nullptr || reinterpret_cast<uintptr_t>(p.mask) % 16 != 0 ||
                      p.ldm < p.N || p.ldm % 8 != 0))
    return cudaErrorInvalidValue;  // the activation is read as 16-byte pieces of its rows
  const int grid = 2 * clusters;
  // training modes, one instantiation each
  if (p.mode == 2) return launch_pair_one<false, false, true, 2, kTrainEpiWarps>(tmA, tmB, to, p, grid, s);
  if (p.mode == 3) return launch_pair_one<false, false, true, 3, kTrainEpiWarps>(tmA, tmB, to, p, grid, s);
  if (p.mode == 4) return launch_pair_one<false, false, true, 4, kTrainEpiWarps>(tmA, tmB, to, p, grid, s);
  if (epi_warps != 4 && epi_warps != 8) return cudaErrorInvalidValue;
  if (p.tma_out)
    return epi_warps == 8 ? launch_pair_tma<8>(in_fp8, out_fp8, tmA, tmB, to, p, grid, s)
                          : launch_pair_tma<4>(in_fp8, out_fp8, tmA, tmB, to, p, grid, s);
  if (p.mode == 1)
    return epi_warps == 8 ? launch_pair_head<8>(in_fp8, tmA, tmB, to, p, grid, s)
                          : launch_pair_head<4>(in_fp8, tmA, tmB, to, p, grid, s);
  if (epi_warps == 8) return launch_pair_epi<8>(in_fp8, out_fp8, staged, tmA, tmB, to, p, grid, s);
  return launch_pair_epi<4>(in_fp8, out_fp8, staged, tmA, tmB, to, p, grid, s);
}

}  // namespace ddf
