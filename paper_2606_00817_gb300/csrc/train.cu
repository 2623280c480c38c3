// train.cu -- CUDA-core kernels of the distillation step (Sec. 3.2 / 3.4):
// the FP32 head and its gradient, the clamped-L1 + cross-entropy loss, column
// sums and split-K reduction, Adam, transposed weight packing (the weight
// gradients themselves read their operands MN-major on the tensor cores, so
// no activation is transposed), and the exact ray caster against a union of
// spheres and boxes that supplies the distillation targets (Sec. 3.2, exact
// cast supervision with analytic primitives in place of a mesh).
#include <cuda_bf16.h>

#include "kernels.h"
#include "caster.cuh"

namespace ddf {

namespace {

__device__ __forceinline__ float softplus_t(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoid_t(float z) {
  const float e = expf(-fabsf(z));
  return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

// One warp per row: z = Wo h + bo from a bf16 activation row.
__global__ void head_train_kernel(const __nv_bfloat16* __restrict__ H, int M, int W,
                                  const float* __restrict__ wo, const float* __restrict__ bo,
                                  float2* __restrict__ z) {
  const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const __nv_bfloat16* h = H + row * W;
  float s0 = 0.f, s1 = 0.f;
  for (int k = lane; k < W; k += 32) {
    const float x = __bfloat162float(h[k]);
    s0 = fmaf(x, wo[k], s0);
    s1 = fmaf(x, wo[W + k], s1);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, off);
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
  }
  if (lane == 0) z[row] = make_float2(s0 + bo[0], s1 + bo[1]);
}

// z of each row from the last layer's head partials (in partial order).
__global__ void head_sum_kernel(const float2* __restrict__ part, int nparts, int64_t M,
                                const float* __restrict__ bo, float2* __restrict__ z) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= M) return;
  float s0 = 0.f, s1 = 0.f;
  for (int p = 0; p < nparts; ++p) {
    const float2 v = part[p * M + r];
    s0 += v.x;
    s1 += v.y;
  }
  z[r] = make_float2(s0 + bo[0], s1 + bo[1]);
}

__global__ void count_hits_kernel(const uint8_t* __restrict__ y, int64_t B, unsigned* __restrict__ n) {
  __shared__ unsigned red[32];
  unsigned c = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < B;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    c += y[i] != 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(n, t);  // integer sum: order does not matter
  }
}

// Per ray: loss terms and dL/dz (see launch_loss for the definition); one
// partial loss sum per block, summed in block order by sum_partials_kernel.
__global__ void loss_dz_kernel(const float2* __restrict__ z, const float* __restrict__ t_tgt,
                               const uint8_t* __restrict__ y, int64_t B,
                               const unsigned* __restrict__ nhit, float clamp, float lam,
                               float2* __restrict__ dz, float* __restrict__ part) {
  __shared__ float red[32];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < B) {
    const float nh = fmaxf(1.f, static_cast<float>(*nhit));
    const float2 zz = z[i];
    const bool hit = y[i] != 0;
    const float th = softplus_t(zz.x);
    float d0 = 0.f;
    if (hit) {
      const float diff = fminf(th, clamp) - fminf(t_tgt[i], clamp);
      l += fabsf(diff) / nh;
      const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
      d0 = th <= clamp ? sg * sigmoid_t(zz.x) / nh : 0.f;
    }
    const float yf = hit ? 1.f : 0.f;
    l += lam * (softplus_t(zz.y) - yf * zz.y) / static_cast<float>(B);
    dz[i] = make_float2(d0, lam * (sigmoid_t(zz.y) - yf) / static_cast<float>(B));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// SDF regression: per point |z0 - s*| / B and dz = (sign(z0 - s*) / B, 0).
__global__ void sdf_loss_kernel(const float2* __restrict__ z, const float* __restrict__ s_tgt,
                                int64_t B, float2* __restrict__ dz, float* __restrict__ part) {
  __shared__ float red[32];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < B) {
    const float diff = z[i].x - s_tgt[i];
    l = fabsf(diff) / static_cast<float>(B);
    const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
    dz[i] = make_float2(sg / static_cast<float>(B), 0.f);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(const float* __restrict__ part, int n, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t;
  }
}

// The head's backward in one pass over the last activation H [M x W] (bf16):
// per row r, dpre = bf16((dz0 wo[0] + dz1 wo[1]) where H > 0); per split s of
// rows (one block; thread t owns columns 8t .. 8t + 7) the partial sums
// part[s][0][k] = sum dz0 H[r][k], part[s][1][k] = sum dz1 H[r][k] (the head
// weights' gradient) and part[s][2][k] = sum dpre[r][k] (the last layer's
// bias gradient), in row order.
__global__ void head_back_fused_kernel(const float2* __restrict__ dz, const __nv_bfloat16* __restrict__ H,
                                       int M, int W, const float* __restrict__ wo, int rows_per_split,
                                       __nv_bfloat16* __restrict__ dpre, float* __restrict__ part) {
  const int c = 8 * threadIdx.x;
  if (c >= W) return;
  const int s = blockIdx.x;
  const int r0 = s * rows_per_split, r1 = min(M, r0 + rows_per_split);
  float w0[8], w1[8], g0[8], g1[8], cs[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    w0[j] = wo[c + j];
    w1[j] = wo[W + c + j];
    g0[j] = g1[j] = cs[j] = 0.f;
  }
#pragma unroll 4
  for (int r = r0; r < r1; ++r) {
    const float2 d = dz[r];
    const uint4 hv = *reinterpret_cast<const uint4*>(H + static_cast<int64_t>(r) * W + c);
    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
    uint32_t ow[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float h0 = __uint_as_float(hw[q] << 16), h1 = __uint_as_float(hw[q] & 0xFFFF0000u);
      const int j = 2 * q;
      const float x0 = h0 > 0.f ? d.x * w0[j] + d.y * w1[j] : 0.f;
      const float x1 = h1 > 0.f ? d.x * w0[j + 1] + d.y * w1[j + 1] : 0.f;
      const __nv_bfloat162 o = __floats2bfloat162_rn(x0, x1);
      ow[q] = *reinterpret_cast<const uint32_t*>(&o);
      cs[j] += __low2float(o);
      cs[j + 1] += __high2float(o);
      g0[j] = fmaf(d.x, h0, g0[j]);
      g1[j] = fmaf(d.y, h0, g1[j]);
      g0[j + 1] = fmaf(d.x, h1, g0[j + 1]);
      g1[j + 1] = fmaf(d.y, h1, g1[j + 1]);
    }
    *reinterpret_cast<uint4*>(dpre + static_cast<int64_t>(r) * W + c) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
  }
  float* ps = part + static_cast<size_t>(s) * 3 * W + c;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    ps[j] = g0[j];
    ps[W + j] = g1[j];
    ps[2 * W + j] = cs[j];
  }
}

// part[s][k] = sum over rows of split s of X[r][k] (bf16 or FP32 input).
template <typename T>
__device__ __forceinline__ float as_f(T v);
template <>
__device__ __forceinline__ float as_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float as_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void colsum_kernel(const T* __restrict__ X, int M, int N, int ld, int rows_per_split,
                              float* __restrict__ part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (k >= N) return;
  const int r0 = s * rows_per_split, r1 = min(M, r0 + rows_per_split);
  float a = 0.f;
  for (int r = r0; r < r1; ++r) a += as_f<T>(X[static_cast<int64_t>(r) * ld + k]);
  part[static_cast<size_t>(s) * N + k] = a;
}

// out[r * ldo + c] = sum_s part[s][r][c] (split order), c < cols_out, part row stride ldp.
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int S, int rows, int ldp,
                                     int64_t split_stride, int cols_out, float* __restrict__ out,
                                     int ldo) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(rows) * cols_out) return;
  const int r = static_cast<int>(idx / cols_out);
  const int c = static_cast<int>(idx - static_cast<int64_t>(r) * cols_out);
  float a = 0.f;
  for (int s = 0; s < S; ++s) a += part[s * split_stride + static_cast<int64_t>(r) * ldp + c];
  out[static_cast<int64_t>(r) * ldo + c] = a;
}

// Adam (Kingma & Ba): bias-corrected, no weight decay. bc1 = 1 - b1^t, bc2 = 1 - b2^t.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Adam plus the refresh of the weights' copies (see launch_adam_refresh).
// The same arithmetic as adam_kernel, element by element.
__global__ void adam_refresh_kernel(float* __restrict__ w, const float* __restrict__ g,
                                    float* __restrict__ m, float* __restrict__ v, int64_t n,
                                    float lr, float b1, float b2, float eps, float bc1, float bc2,
                                    const AdamBlocks blocks) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = wi;
  int j = 0;
  while (j + 1 < blocks.n && i >= blocks.b[j + 1].start) ++j;
  const AdamBlock& bk = blocks.b[j];
  const int64_t e = i - bk.start;
  if (e >= static_cast<int64_t>(bk.rows) * bk.cols) return;
  if (bk.f32 != nullptr) bk.f32[e] = wi;
  if (bk.wb != nullptr) {
    const int64_t r = e / bk.cols, c = e - r * bk.cols;
    const __nv_bfloat16 hb = __float2bfloat16_rn(wi);
    bk.wb[r * bk.ldb + c] = hb;
    if (bk.wt != nullptr) bk.wt[c * bk.rows + r] = hb;
  }
}

// dst[k][n] = bf16(src[n][k]): the transposed weight of a [N x K] layer.
__global__ void pack_bf16_t_kernel(const float* __restrict__ src, int N, int K,
                                   __nv_bfloat16* __restrict__ dst) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(N) * K) return;
  const int k = static_cast<int>(idx / N);
  const int n = static_cast<int>(idx - static_cast<int64_t>(k) * N);
  dst[idx] = __float2bfloat16_rn(src[static_cast<int64_t>(n) * K + k]);
}

// Exact first hit of each ray (caster.cuh), primitives staged in shared memory.
__global__ void cast_scene_kernel(const float* __restrict__ spheres, int ns,
                                  const float* __restrict__ boxes, int nb, RaySoA rays, int64_t n,
                                  float* __restrict__ t_out, uint8_t* __restrict__ hit_out) {
  __shared__ float s_sph[4 * kMaxPrims];
  __shared__ float s_box[6 * kMaxPrims];
  for (int i = threadIdx.x; i < 4 * ns; i += blockDim.x) s_sph[i] = spheres[i];
  for (int i = threadIdx.x; i < 6 * nb; i += blockDim.x) s_box[i] = boxes[i];
  __syncthreads();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float o[3] = {rays.p[0][i], rays.p[1][i], rays.p[2][i]};
  const float d[3] = {rays.p[3][i], rays.p[4][i], rays.p[5][i]};
  const float best = cast_one(o, d, s_sph, ns, s_box, nb, nullptr);
  t_out[i] = best;
  hit_out[i] = best < __int_as_float(0x7f800000) ? 1 : 0;
}

}  // namespace

cudaError_t launch_head_train(const __nv_bfloat16* H, int M, int W, const float* wo,
                              const float* bo, float2* z, cudaStream_t s) {
  head_train_kernel<<<(M + 7) / 8, 256, 0, s>>>(H, M, W, wo, bo, z);
  return cudaGetLastError();
}

cudaError_t launch_head_sum(const float2* part, int nparts, int64_t M, const float* bo, float2* z,
                            cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  head_sum_kernel<<<static_cast<unsigned>((M + 255) / 256), 256, 0, s>>>(part, nparts, M, bo, z);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float2* z, const float* t_tgt, const uint8_t* y, int64_t B,
                        unsigned* nhit, float clamp, float lam, float2* dz, float* part,
                        float* loss_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(nhit, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  count_hits_kernel<<<256, 256, 0, s>>>(y, B, nhit);
  const int blocks = static_cast<int>((B + 255) / 256);
  loss_dz_kernel<<<blocks, 256, 0, s>>>(z, t_tgt, y, B, nhit, clamp, lam, dz, part);
  if (loss_out != nullptr) sum_partials_kernel<<<1, 32, 0, s>>>(part, blocks, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_sdf_loss(const float2* z, const float* s_tgt, int64_t B, float2* dz,
                            float* part, float* loss_out, cudaStream_t s) {
  const int blocks = static_cast<int>((B + 255) / 256);
  sdf_loss_kernel<<<blocks, 256, 0, s>>>(z, s_tgt, B, dz, part);
  if (loss_out != nullptr) sum_partials_kernel<<<1, 32, 0, s>>>(part, blocks, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_head_back_fused(const float2* dz, const __nv_bfloat16* H, int M, int W,
                                  const float* wo, int splits, __nv_bfloat16* dpre, float* part,
                                  cudaStream_t s) {
  if (W % 8 != 0 || W / 8 > 1024) return cudaErrorInvalidValue;
  const int rps = (M + splits - 1) / splits;
  const int threads = ((W / 8 + 31) / 32) * 32;
  head_back_fused_kernel<<<splits, threads, 0, s>>>(dz, H, M, W, wo, rps, dpre, part);
  return cudaGetLastError();
}

cudaError_t launch_colsum_bf16(const __nv_bfloat16* X, int M, int N, int ld, int splits,
                               float* part, cudaStream_t s) {
  const int rps = (M + splits - 1) / splits;
  colsum_kernel<__nv_bfloat16><<<dim3((N + 255) / 256, splits), 256, 0, s>>>(X, M, N, ld, rps, part);
  return cudaGetLastError();
}

cudaError_t launch_colsum_f32(const float* X, int M, int N, int ld, int splits, float* part,
                              cudaStream_t s) {
  const int rps = (M + splits - 1) / splits;
  colsum_kernel<float><<<dim3((N + 255) / 256, splits), 256, 0, s>>>(X, M, N, ld, rps, part);
  return cudaGetLastError();
}

cudaError_t launch_splitk_reduce(const float* part, int S, int rows, int ldp, int64_t split_stride,
                                 int cols_out, float* out, int ldo, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(rows) * cols_out;
  splitk_reduce_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      part, S, rows, ldp, split_stride, cols_out, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_adam_refresh(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                                float b1, float b2, float eps, float bc1, float bc2,
                                const AdamBlocks& blocks, cudaStream_t s) {
  if (blocks.n < 1 || blocks.n > kAdamBlocks || blocks.b[0].start != 0) return cudaErrorInvalidValue;
  adam_refresh_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      w, g, m, v, n, lr, b1, b2, eps, bc1, bc2, blocks);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s) {
  adam_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(w, g, m, v, n, lr, b1, b2, eps,
                                                                    bc1, bc2);
  return cudaGetLastError();
}

cudaError_t launch_pack_bf16_t(const float* src, int N, int K, __nv_bfloat16* dst, cudaStream_t s) {
  const int64_t total = static_cast<int64_t>(N) * K;
  pack_bf16_t_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(src, N, K, dst);
  return cudaGetLastError();
}

cudaError_t launch_cast_scene(const float* spheres, int ns, const float* boxes, int nb,
                              RaySoA rays, int64_t n, float* t_out, uint8_t* hit_out,
                              cudaStream_t s) {
  if (ns > kMaxPrims || nb > kMaxPrims) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  cast_scene_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(spheres, ns, boxes, nb,
                                                                          rays, n, t_out, hit_out);
  return cudaGetLastError();
}

}  // namespace ddf
