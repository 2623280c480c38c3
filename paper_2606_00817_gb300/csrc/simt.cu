// simt.cu -- CUDA-core kernels of the DDF query path:
//   * the sinusoidal ray encoding (Sec. 4.3) into bf16 or FP32 rows,
//   * the plain FP32 layer (FFMA, no TF32) used by the FP32 precision,
//   * the distance / visibility heads (softplus, sigmoid) and the shadow test
//     of Sec. 3.3,
//   * load-time weight packing (zero-padded FP32 / bf16 copies) and the
//     per-output-channel e4m3 quantiser.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels.h"
#include "heads.cuh"

namespace ddf {

namespace {

template <typename T>
__device__ __forceinline__ T to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// 8 consecutive floats from shared memory to 8 consecutive outputs (16-byte
// aligned destination).
__device__ __forceinline__ void store8(__nv_bfloat16* dst, const float* src) {
  uint4 w;
  __nv_bfloat162 a = __floats2bfloat162_rn(src[0], src[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(src[2], src[3]);
  __nv_bfloat162 c = __floats2bfloat162_rn(src[4], src[5]);
  __nv_bfloat162 d = __floats2bfloat162_rn(src[6], src[7]);
  w.x = *reinterpret_cast<uint32_t*>(&a);
  w.y = *reinterpret_cast<uint32_t*>(&b);
  w.z = *reinterpret_cast<uint32_t*>(&c);
  w.w = *reinterpret_cast<uint32_t*>(&d);
  *reinterpret_cast<uint4*>(dst) = w;
}
__device__ __forceinline__ void store8(float* dst, const float* src) {
  reinterpret_cast<float4*>(dst)[0] = make_float4(src[0], src[1], src[2], src[3]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(src[4], src[5], src[6], src[7]);
}

constexpr int kEncRays = 64;  // rays per block of the encoder

// One block encodes kEncRays rays: each thread builds its ray's row in shared
// memory (row stride ld+1 to spread banks), then the block writes the rows,
// which are contiguous in global memory, with consecutive threads on
// consecutive elements.
template <typename T>
__global__ void __launch_bounds__(kEncRays) encode_kernel(RaySoA rays, int64_t M, int L, int ld,
                                                          T* __restrict__ out) {
  extern __shared__ float enc_smem[];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kEncRays;
  const int rows = static_cast<int>(M - r0 < kEncRays ? M - r0 : kEncRays);
  const int sld = ld + 1;
  const int i = threadIdx.x;
  if (i < rows) {
    float* row = enc_smem + i * sld;
    float e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = ray_ld(rays, c, r0 + i);
#pragma unroll
    for (int c = 0; c < 6; ++c) row[c] = e[c];
    int col = 6;
    for (int c = 0; c < 6; ++c) {
      for (int k = 0; k < L; ++k) {
        float s, co;
        // pi 2^k e: the product by 2^k (exponent bits; k <= 15) is exact
        sincospif(e[c] * __int_as_float((127 + k) << 23), &s, &co);
        row[col] = s;
        row[col + 1] = co;
        col += 2;
      }
    }
    for (; col < ld; ++col) row[col] = 0.f;
  }
  __syncthreads();
  // The block's rows are contiguous in global memory: write them 8 elements
  // (16 bytes of bf16, 32 bytes of FP32) per thread step, consecutive threads
  // on consecutive chunks. ld is a multiple of 8.
  const int per_row = ld / 8;
  const int total = rows * per_row;
  T* dst = out + r0 * ld;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int r = idx / per_row;
    const int c = (idx - r * per_row) * 8;
    store8(dst + static_cast<int64_t>(r) * ld + c, enc_smem + r * sld + c);
  }
}

template <typename T>
cudaError_t launch_encode(RaySoA rays, int64_t M, int L, int ld, T* out, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const int64_t blocks = (M + kEncRays - 1) / kEncRays;
  const size_t smem = static_cast<size_t>(kEncRays) * (ld + 1) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(encode_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  encode_kernel<T><<<static_cast<unsigned>(blocks), kEncRays, smem, s>>>(rays, M, L, ld, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- FP32 layer
// Classic register-blocked SGEMM: 128x128 output tile per 256-thread block,
// 8x8 outputs per thread (two 4x4 quadrants 64 apart), K staged 8 at a time
// through double-buffered shared memory (operands stored k-major).
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

__global__ void __launch_bounds__(256) sgemm_relu_kernel(const float* __restrict__ A,
                                                         const float* __restrict__ W,
                                                         const float* __restrict__ bias,
                                                         float* __restrict__ C, int M, int N,
                                                         int K) {
  __shared__ __align__(16) float As[2][SG_BK][SG_BM];
  __shared__ __align__(16) float Ws[2][SG_BK][SG_BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;
  const int lr = tid >> 1, lc = (tid & 1) * 4;  // loader: row, k offset
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool a_ok = m0 + lr < M, w_ok = n0 + lr < N;
  const float* a_src = A + static_cast<size_t>(a_ok ? m0 + lr : 0) * K + lc;
  const float* w_src = W + static_cast<size_t>(w_ok ? n0 + lr : 0) * K + lc;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra = a_ok ? __ldg(reinterpret_cast<const float4*>(a_src)) : zero4;
  float4 rw = w_ok ? __ldg(reinterpret_cast<const float4*>(w_src)) : zero4;
  As[0][lc + 0][lr] = ra.x; As[0][lc + 1][lr] = ra.y; As[0][lc + 2][lr] = ra.z; As[0][lc + 3][lr] = ra.w;
  Ws[0][lc + 0][lr] = rw.x; Ws[0][lc + 1][lr] = rw.y; Ws[0][lc + 2][lr] = rw.z; Ws[0][lc + 3][lr] = rw.w;
  __syncthreads();

  const int KT = K / SG_BK;
  for (int kt = 0; kt < KT; ++kt) {
    const int cur = kt & 1;
    const bool more = kt + 1 < KT;
    if (more) {
      ra = a_ok ? __ldg(reinterpret_cast<const float4*>(a_src + (kt + 1) * SG_BK)) : zero4;
      rw = w_ok ? __ldg(reinterpret_cast<const float4*>(w_src + (kt + 1) * SG_BK)) : zero4;
    }
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Ws[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ws[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      const int nx = cur ^ 1;
      As[nx][lc + 0][lr] = ra.x; As[nx][lc + 1][lr] = ra.y; As[nx][lc + 2][lr] = ra.z; As[nx][lc + 3][lr] = ra.w;
      Ws[nx][lc + 0][lr] = rw.x; Ws[nx][lc + 1][lr] = rw.y; Ws[nx][lc + 2][lr] = rw.z; Ws[nx][lc + 3][lr] = rw.w;
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (row >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = n0 + h * 64 + tx * 4;
      if (col + 3 < N) {
        const float4 bb = __ldg(reinterpret_cast<const float4*>(bias + col));
        float4 o;
        o.x = fmaxf(acc[i][4 * h + 0] + bb.x, 0.f);
        o.y = fmaxf(acc[i][4 * h + 1] + bb.y, 0.f);
        o.z = fmaxf(acc[i][4 * h + 2] + bb.z, 0.f);
        o.w = fmaxf(acc[i][4 * h + 3] + bb.w, 0.f);
        *reinterpret_cast<float4*>(C + static_cast<size_t>(row) * N + col) = o;
      } else {
        for (int j = 0; j < 4; ++j)
          if (col + j < N)
            C[static_cast<size_t>(row) * N + col + j] = fmaxf(acc[i][4 * h + j] + bias[col + j], 0.f);
      }
    }
  }
}

// ---------------------------------------------------------------- heads

// One warp per ray: z = Wo h + bo over an FP32 activation row.
__global__ void head_f32_kernel(const float* __restrict__ H, int M, int W,
                                const float* __restrict__ wo, const float* __restrict__ bo,
                                HeadOut o) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const float* h = H + row * W;
  float s0 = 0.f, s1 = 0.f;
  for (int k = lane; k < W; k += 32) {
    const float x = h[k];
    s0 = fmaf(x, __ldg(wo + k), s0);
    s1 = fmaf(x, __ldg(wo + W + k), s1);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  if (lane == 0) write_heads(o, row, s0 + bo[0], s1 + bo[1]);
}

// One thread per ray: sum the per-N-block partial dot products in a fixed order.
__global__ void finish_heads_kernel(const float2* __restrict__ part, int nblk, int M,
                                    const float* __restrict__ bo, HeadOut o) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  float z0 = 0.f, z1 = 0.f;
  for (int b = 0; b < nblk; ++b) {
    const float2 v = part[static_cast<size_t>(b) * M + i];
    z0 += v.x;
    z1 += v.y;
  }
  write_heads(o, i, z0 + bo[0], z1 + bo[1]);
}

// ---------------------------------------------------------------- weights

template <typename T>
__global__ void pack_kernel(const float* __restrict__ src, int N, int K, int ldd, T* __restrict__ dst) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(N) * ldd) return;
  const int n = static_cast<int>(idx / ldd);
  const int k = static_cast<int>(idx - static_cast<int64_t>(n) * ldd);
  dst[idx] = to_out<T>(k < K ? src[static_cast<int64_t>(n) * K + k] : 0.f);
}

// One block per output channel: amax reduce, then e4m3 codes of src / scale.
__global__ void quant_e4m3_kernel(const float* __restrict__ src, int N, int K, int ldd,
                                  uint8_t* __restrict__ dst, float* __restrict__ scale) {
  __shared__ float red[32];
  const int n = blockIdx.x;
  const float* w = src + static_cast<int64_t>(n) * K;
  float m = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmaxf(m, fabsf(w[k]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const float amax = red[0];
  const float s = amax > 0.f ? amax / 448.f : 1.f;
  if (threadIdx.x == 0) scale[n] = s;
  for (int k = threadIdx.x; k < ldd; k += blockDim.x) {
    const float q = k < K ? w[k] / s : 0.f;
    dst[static_cast<int64_t>(n) * ldd + k] =
        static_cast<uint8_t>(__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3));
  }
}

// One warp per shading point: sums its contiguous ray segment in a fixed order.
__global__ void ao_reduce_kernel(const uint8_t* __restrict__ hit, const float* __restrict__ vis,
                                 const int32_t* __restrict__ offsets, int64_t n_points,
                                 float* __restrict__ hard, float* __restrict__ soft) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= n_points) return;
  const int32_t a = offsets[p], b = offsets[p + 1];
  int nh = 0;
  float sv = 0.f;
  for (int32_t i = a + lane; i < b; i += 32) {
    nh += hit[i];
    sv += vis[i];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    nh += __shfl_xor_sync(0xffffffffu, nh, off);
    sv += __shfl_xor_sync(0xffffffffu, sv, off);
  }
  if (lane == 0) {
    const int n = b - a;
    hard[p] = n > 0 ? 1.f - static_cast<float>(nh) / static_cast<float>(n) : 1.f;
    if (soft != nullptr) soft[p] = n > 0 ? 1.f - sv / static_cast<float>(n) : 1.f;
  }
}

__global__ void scale_vec_kernel(const float* __restrict__ v, float a, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * v[i];
}

}  // namespace

cudaError_t launch_encode_bf16(RaySoA rays, int64_t M, int L, int ld, __nv_bfloat16* out,
                               cudaStream_t s) {
  return launch_encode<__nv_bfloat16>(rays, M, L, ld, out, s);
}

cudaError_t launch_encode_f32(RaySoA rays, int64_t M, int L, int ld, float* out, cudaStream_t s) {
  return launch_encode<float>(rays, M, L, ld, out, s);
}

cudaError_t launch_sgemm_relu(const float* A, const float* W, const float* b, float* C, int M,
                              int N, int K, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (K % SG_BK != 0) return cudaErrorInvalidValue;
  dim3 grid((N + SG_BN - 1) / SG_BN, (M + SG_BM - 1) / SG_BM);
  sgemm_relu_kernel<<<grid, 256, 0, s>>>(A, W, b, C, M, N, K);
  return cudaGetLastError();
}

cudaError_t launch_head_f32(const float* H, int M, int W, const float* wo, const float* bo,
                            HeadOut o, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const int warps = 8;
  head_f32_kernel<<<(M + warps - 1) / warps, 32 * warps, 0, s>>>(H, M, W, wo, bo, o);
  return cudaGetLastError();
}

cudaError_t launch_finish_heads(const float2* part, int nblk, int M, const float* bo, HeadOut o,
                                cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  finish_heads_kernel<<<(M + 255) / 256, 256, 0, s>>>(part, nblk, M, bo, o);
  return cudaGetLastError();
}

cudaError_t launch_pack_f32(const float* src, int N, int K, int ldd, float* dst, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(N) * ldd;
  pack_kernel<float><<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(src, N, K, ldd, dst);
  return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const float* src, int N, int K, int ldd, __nv_bfloat16* dst,
                             cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(N) * ldd;
  pack_kernel<__nv_bfloat16><<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(src, N, K,
                                                                                      ldd, dst);
  return cudaGetLastError();
}

cudaError_t launch_quant_e4m3(const float* src, int N, int K, int ldd, uint8_t* dst, float* scale,
                              cudaStream_t s) {
  quant_e4m3_kernel<<<N, 256, 0, s>>>(src, N, K, ldd, dst, scale);
  return cudaGetLastError();
}

cudaError_t launch_ao_reduce(const uint8_t* hit, const float* vis, const int32_t* offsets,
                             int64_t n_points, float* hard, float* soft, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  const int warps = 8;
  const int64_t blocks = (n_points + warps - 1) / warps;
  ao_reduce_kernel<<<static_cast<unsigned>(blocks), 32 * warps, 0, s>>>(hit, vis, offsets,
                                                                       n_points, hard, soft);
  return cudaGetLastError();
}

cudaError_t launch_scale_vec(const float* v, float a, int n, float* out, cudaStream_t s) {
  scale_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(v, a, n, out);
  return cudaGetLastError();
}

}  // namespace ddf
