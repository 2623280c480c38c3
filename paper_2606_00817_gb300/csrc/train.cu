// train.cu -- CUDA-core kernels of the distillation step (Sec. 3.2 / 3.4):
// the FP32 head and its gradient, the clamped-L1 + cross-entropy loss, the
// gradient reductions (one fixed-order launch per layer: split-K sums of the
// weight gradients and column sums for the biases), Adam (plain, and fused
// with the refresh of every weight copy, the transposed one included; the
// weight gradients themselves read their operands MN-major on the tensor
// cores, so no activation is transposed), and the exact ray caster against a
// union of spheres and boxes that supplies the distillation targets (Sec.
// 3.2, exact cast supervision with analytic primitives in place of a mesh).
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
  float zs0 = 0.f, zs1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    w0[j] = wo[c + j];
    w1[j] = wo[W + c + j];
    g0[j] = g1[j] = cs[j] = 0.f;
  }
  // rows in batches of kHeadRows, the next batch's loads in flight while a
  // batch is computed; rows are taken in order, so the sums are the same
  // bits as a plain loop over the rows
  constexpr int kHeadRows = 4;
  uint4 h0q[kHeadRows], h1q[kHeadRows];
  float2 d0q[kHeadRows], d1q[kHeadRows];
  auto load = [&](int rb, uint4 (&hq)[kHeadRows], float2 (&dq)[kHeadRows]) {
#pragma unroll
    for (int q = 0; q < kHeadRows; ++q) {
      const int r = rb + q;
      hq[q] = r < r1 ? __ldg(reinterpret_cast<const uint4*>(H + static_cast<int64_t>(r) * W + c))
                     : make_uint4(0u, 0u, 0u, 0u);
      dq[q] = r < r1 ? dz[r] : make_float2(0.f, 0.f);
    }
  };
  auto rows = [&](int rb, const uint4 (&hq)[kHeadRows], const float2 (&dq)[kHeadRows]) {
#pragma unroll
    for (int k = 0; k < kHeadRows; ++k) {
      const int r = rb + k;
      if (r >= r1) break;
      const float2 d = dq[k];
      zs0 += d.x;
      zs1 += d.y;
      const uint4 hv = hq[k];
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
  };
  load(r0, h0q, d0q);
  for (int rb = r0; rb < r1; rb += 2 * kHeadRows) {
    if (rb + kHeadRows < r1) load(rb + kHeadRows, h1q, d1q);
    rows(rb, h0q, d0q);
    if (rb + 2 * kHeadRows < r1) load(rb + 2 * kHeadRows, h0q, d0q);
    rows(rb + kHeadRows, h1q, d1q);
  }
  float* ps = part + static_cast<size_t>(s) * (3 * W + 4) + c;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    ps[j] = g0[j];
    ps[W + j] = g1[j];
    ps[2 * W + j] = cs[j];
  }
  if (c == 0) {
    ps[3 * W] = zs0;
    ps[3 * W + 1] = zs1;
  }
}

// Gradient reductions of one launch (see GradReduce). Blocks [blk0[j],
// blk0[j + 1]) do split-sum job j, four output elements per thread (one
// float4 when the job is aligned for it); the blocks after them do the
// column sum, R row splits of each 256-column block, and the last of the R
// blocks of a column block to finish (an atomic ticket) adds the R partials.
// A thread of a column block takes 4 columns and every 4th row (or partial)
// from its phase (0-3); the 4 phase sums are then added in phase order.
// Every sum runs in a fixed order, so the result does not depend on which
// block finishes when.
// Columns col .. col + 3 of one row of the column-sum input (4 aligned
// columns: the launcher checks the row stride and the base address).
__device__ __forceinline__ float4 red_cols_load4(const RedCols& cs, int64_t row_off, int col) {
  if (cs.x_bf16) {
    const uint2 u =
        *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(cs.X) + row_off + col);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
  }
  return *reinterpret_cast<const float4*>(static_cast<const float*>(cs.X) + row_off + col);
}

__device__ __forceinline__ void add4(float4& a, const float4 b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

__global__ void __launch_bounds__(256) grad_reduce_kernel(const __grid_constant__ GradReduce g) {
  const int b = blockIdx.x;
  if (b < g.blk0[g.nsplit]) {
    int j = 0;
    while (b >= g.blk0[j + 1]) ++j;
    const RedSplit& a = g.split[j];
    const int64_t e0 = 4 * (static_cast<int64_t>(b - g.blk0[j]) * blockDim.x + threadIdx.x);
    const int64_t total = static_cast<int64_t>(a.rows) * a.cols;
    if (e0 >= total) return;
    if (a.vec) {
      const int r = static_cast<int>(e0 / a.cols);
      const int c = static_cast<int>(e0 - static_cast<int64_t>(r) * a.cols);
      const float* src = a.part + static_cast<int64_t>(r) * a.ldp + c;
      float* dst = a.out + static_cast<int64_t>(r) * a.ldo + c;  // cols, ldp, ldo, split_stride multiples of 4; 16-byte aligned
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int q = 0; q < a.S; ++q) add4(acc, *reinterpret_cast<const float4*>(src + q * a.split_stride));
      *reinterpret_cast<float4*>(dst) = acc;
      return;
    }
    for (int k = 0; k < 4 && e0 + k < total; ++k) {  // the 4 elements may span rows
      const int rk = static_cast<int>((e0 + k) / a.cols);
      const int ck = static_cast<int>(e0 + k - static_cast<int64_t>(rk) * a.cols);
      const float* sk = a.part + static_cast<int64_t>(rk) * a.ldp + ck;
      float acc = 0.f;
      for (int q = 0; q < a.S; ++q) acc += sk[q * a.split_stride];
      a.out[static_cast<int64_t>(rk) * a.ldo + ck] = acc;
    }
    return;
  }
  const RedCols& cs = g.cols;
  __shared__ float4 ph_sum[4][64];
  __shared__ int last;
  const int bb = b - g.blk0[g.nsplit];
  const int ncb = (cs.N + 255) / 256;
  const int cb = bb % ncb, j = bb / ncb;
  const int quad = threadIdx.x & 63, phase = threadIdx.x >> 6;
  const int col4 = cb * 256 + 4 * quad;  // first of this thread's 4 columns
  const int col = cb * 256 + static_cast<int>(threadIdx.x);  // column of the phase sum
  {
    const int rps = (cs.M + cs.R - 1) / cs.R;
    const int r0 = j * rps, r1 = min(cs.M, r0 + rps);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (col4 < cs.N) {
#pragma unroll 4
      for (int r = r0 + phase; r < r1; r += 4)
        add4(acc, red_cols_load4(cs, static_cast<int64_t>(r) * cs.ld, col4));
    }
    ph_sum[phase][quad] = acc;
    __syncthreads();
    if (col < cs.N) {
      const float* f0 = reinterpret_cast<const float*>(ph_sum[0]);
      const float* f1 = reinterpret_cast<const float*>(ph_sum[1]);
      const float* f2 = reinterpret_cast<const float*>(ph_sum[2]);
      const float* f3 = reinterpret_cast<const float*>(ph_sum[3]);
      const int t = threadIdx.x;
      cs.cpart[static_cast<size_t>(j) * cs.ldc + col] = ((f0[t] + f1[t]) + f2[t]) + f3[t];
    }
  }
  __threadfence();  // this thread's partial is visible before the ticket is taken
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&cs.ticket[cb], 1u) == static_cast<unsigned>(cs.R - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (col4 < cs.N) {
#pragma unroll 4
    for (int q = phase; q < cs.R; q += 4)
      add4(acc, __ldcg(reinterpret_cast<const float4*>(cs.cpart + static_cast<size_t>(q) * cs.ldc + col4)));
  }
  ph_sum[phase][quad] = acc;
  __syncthreads();
  if (col < cs.N) {
    const int t = threadIdx.x;
    const float sum = ((reinterpret_cast<const float*>(ph_sum[0])[t] +
                        reinterpret_cast<const float*>(ph_sum[1])[t]) +
                       reinterpret_cast<const float*>(ph_sum[2])[t]) +
                      reinterpret_cast<const float*>(ph_sum[3])[t];
    for (int k = 0; k < cs.nseg; ++k)
      if (col >= cs.c0[k] && col < cs.c0[k] + cs.cnt[k]) cs.out[k][col - cs.c0[k]] = sum;
  }
  if (threadIdx.x == 0) cs.ticket[cb] = 0u;  // ready for the next launch
}

// One Adam update (Kingma & Ba): bias-corrected, no weight decay,
// bc1 = 1 - b1^t, bc2 = 1 - b2^t; m and v are updated in place, the new
// weight is returned. The fused multiply-adds are written out, so every
// kernel that calls this rounds the same way.
__device__ __forceinline__ float adam_elem(float w, float g, float& m, float& v, float lr, float b1,
                                           float b2, float eps, float bc1, float bc2) {
  m = fmaf(b1, m, (1.f - b1) * g);
  v = fmaf(b2, v, (1.f - b2) * g * g);
  return w - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// Adam over n parameters, 4 per thread (one float4 of each array when vec:
// all four arrays 16-byte aligned).
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, int vec) {
  const int64_t i4 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  if (i4 >= n) return;
  if (vec && i4 + 4 <= n) {
    float4 W = *reinterpret_cast<const float4*>(w + i4);
    const float4 G = *reinterpret_cast<const float4*>(g + i4);
    float4 M = *reinterpret_cast<const float4*>(m + i4);
    float4 V = *reinterpret_cast<const float4*>(v + i4);
    W.x = adam_elem(W.x, G.x, M.x, V.x, lr, b1, b2, eps, bc1, bc2);
    W.y = adam_elem(W.y, G.y, M.y, V.y, lr, b1, b2, eps, bc1, bc2);
    W.z = adam_elem(W.z, G.z, M.z, V.z, lr, b1, b2, eps, bc1, bc2);
    W.w = adam_elem(W.w, G.w, M.w, V.w, lr, b1, b2, eps, bc1, bc2);
    *reinterpret_cast<float4*>(m + i4) = M;
    *reinterpret_cast<float4*>(v + i4) = V;
    *reinterpret_cast<float4*>(w + i4) = W;
    return;
  }
  for (int64_t i = i4; i < i4 + 4 && i < n; ++i) {
    float mi = m[i], vi = v[i];
    w[i] = adam_elem(w[i], g[i], mi, vi, lr, b1, b2, eps, bc1, bc2);
    m[i] = mi;
    v[i] = vi;
  }
}

// Adam over the level tables of a hash-grid field (entry i of the blob is
// the feature pair 2 i, 2 i + 1) and, in the same pass, their bf16x2 query
// copy: source entry i of level l goes to word i - from.offset[l] +
// to.offset[l] (f0 in the low half). The arithmetic of adam_kernel, element
// by element; two entries (one float4 of each array) per thread when vec.
__global__ void hg_adam_pack_kernel(float* __restrict__ w, const float* __restrict__ g,
                                    float* __restrict__ m, float* __restrict__ v, int64_t entries,
                                    float lr, float b1, float b2, float eps, float bc1, float bc2,
                                    HashGridParams from, HashGridParams to,
                                    uint32_t* __restrict__ dst, int vec) {
  const int64_t e0 = 2 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  if (e0 >= entries) return;
  auto word = [&](int64_t e) {
    int l = 0;
#pragma unroll
    for (int k = 1; k < 16; ++k) l += e >= from.offset[k] ? 1 : 0;
    return e - from.offset[l] + to.offset[l];
  };
  auto pack = [](float lo, float hi) {
    __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&b);
  };
  const int64_t i4 = 2 * e0;
  if (vec && e0 + 2 <= entries) {
    float4 W = *reinterpret_cast<const float4*>(w + i4);
    const float4 G = *reinterpret_cast<const float4*>(g + i4);
    float4 M = *reinterpret_cast<const float4*>(m + i4);
    float4 V = *reinterpret_cast<const float4*>(v + i4);
    W.x = adam_elem(W.x, G.x, M.x, V.x, lr, b1, b2, eps, bc1, bc2);
    W.y = adam_elem(W.y, G.y, M.y, V.y, lr, b1, b2, eps, bc1, bc2);
    W.z = adam_elem(W.z, G.z, M.z, V.z, lr, b1, b2, eps, bc1, bc2);
    W.w = adam_elem(W.w, G.w, M.w, V.w, lr, b1, b2, eps, bc1, bc2);
    *reinterpret_cast<float4*>(m + i4) = M;
    *reinterpret_cast<float4*>(v + i4) = V;
    *reinterpret_cast<float4*>(w + i4) = W;
    dst[word(e0)] = pack(W.x, W.y);
    dst[word(e0 + 1)] = pack(W.z, W.w);
    return;
  }
  for (int64_t e = e0; e < e0 + 2 && e < entries; ++e) {
    float nw[2];
    for (int f = 0; f < 2; ++f) {
      const int64_t i = 2 * e + f;
      float mi = m[i], vi = v[i];
      nw[f] = adam_elem(w[i], g[i], mi, vi, lr, b1, b2, eps, bc1, bc2);
      w[i] = nw[f];
      m[i] = mi;
      v[i] = vi;
    }
    dst[word(e)] = pack(nw[0], nw[1]);
  }
}

// Adam plus the refresh of the weights' copies (see launch_adam_refresh),
// the same arithmetic as adam_kernel element by element. A CTA takes either
// 2,048 consecutive elements of a block without a transposed copy, or a
// tile of 32 rows x 64 columns of one with it: each thread updates 8
// elements of one column (rows 4 apart), the tile's bf16 values are staged
// in shared memory by column, and every thread writes 8 consecutive bf16 of
// one row of the transposed copy, so all stores are whole runs.
constexpr int kAdamTileR = 32, kAdamTileC = 64, kAdamLinear = 2048;

__device__ __forceinline__ float adam_one(float* __restrict__ w, const float* __restrict__ g,
                                          float* __restrict__ m, float* __restrict__ v, int64_t i,
                                          float lr, float b1, float b2, float eps, float bc1,
                                          float bc2) {
  float mi = m[i], vi = v[i];
  const float wi = adam_elem(w[i], g[i], mi, vi, lr, b1, b2, eps, bc1, bc2);
  m[i] = mi;
  v[i] = vi;
  w[i] = wi;
  return wi;
}

__global__ void __launch_bounds__(256) adam_refresh_kernel(float* __restrict__ w,
                                                           const float* __restrict__ g,
                                                           float* __restrict__ m,
                                                           float* __restrict__ v, float lr, float b1,
                                                           float b2, float eps, float bc1, float bc2,
                                                           const __grid_constant__ AdamBlocks blocks) {
  __shared__ __align__(16) __nv_bfloat16 tile[kAdamTileC][kAdamTileR + 8];
  int j = 0;
  while (j + 1 < blocks.n && static_cast<int>(blockIdx.x) >= blocks.b[j + 1].cta0) ++j;
  const AdamBlock& bk = blocks.b[j];
  const int u = static_cast<int>(blockIdx.x) - bk.cta0;
  const int64_t count = static_cast<int64_t>(bk.rows) * bk.cols;
  if (bk.wt == nullptr) {
    for (int k = 0; k < kAdamLinear / 256; ++k) {
      const int64_t e = static_cast<int64_t>(u) * kAdamLinear + k * 256 + threadIdx.x;
      if (e >= count) break;
      const float wi = adam_one(w, g, m, v, bk.start + e, lr, b1, b2, eps, bc1, bc2);
      if (bk.f32 != nullptr) bk.f32[e] = wi;
      if (bk.wb != nullptr) {
        const int64_t r = e / bk.cols, c = e - r * bk.cols;
        bk.wb[r * bk.ldb + c] = __float2bfloat16_rn(wi);
      }
    }
    return;
  }
  const int ntc = (bk.cols + kAdamTileC - 1) / kAdamTileC;
  const int r0 = (u / ntc) * kAdamTileR, c0 = (u % ntc) * kAdamTileC;
  if (bk.vec) {
    // four adjacent columns per thread: one float4 of each array and one
    // 8-byte piece of the bf16 rows (the launcher checked the alignment)
    const int cq = static_cast<int>(threadIdx.x) & (kAdamTileC / 4 - 1);
    const int c = c0 + 4 * cq;
#pragma unroll
    for (int k = 0; k < kAdamTileR * kAdamTileC / 4 / 256; ++k) {
      const int rl = static_cast<int>(threadIdx.x) / (kAdamTileC / 4) + (256 / (kAdamTileC / 4)) * k;
      const int r = r0 + rl;
      float4 W = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < bk.rows && c < bk.cols) {  // cols % 4 == 0: all four columns
        const int64_t e = static_cast<int64_t>(r) * bk.cols + c;
        const int64_t i = bk.start + e;
        W = *reinterpret_cast<const float4*>(w + i);
        const float4 G = *reinterpret_cast<const float4*>(g + i);
        float4 M = *reinterpret_cast<const float4*>(m + i);
        float4 V = *reinterpret_cast<const float4*>(v + i);
        W.x = adam_elem(W.x, G.x, M.x, V.x, lr, b1, b2, eps, bc1, bc2);
        W.y = adam_elem(W.y, G.y, M.y, V.y, lr, b1, b2, eps, bc1, bc2);
        W.z = adam_elem(W.z, G.z, M.z, V.z, lr, b1, b2, eps, bc1, bc2);
        W.w = adam_elem(W.w, G.w, M.w, V.w, lr, b1, b2, eps, bc1, bc2);
        *reinterpret_cast<float4*>(w + i) = W;
        *reinterpret_cast<float4*>(m + i) = M;
        *reinterpret_cast<float4*>(v + i) = V;
        if (bk.f32 != nullptr) *reinterpret_cast<float4*>(bk.f32 + e) = W;
        if (bk.wb != nullptr) {
          const __nv_bfloat162 lo = __floats2bfloat162_rn(W.x, W.y), hi = __floats2bfloat162_rn(W.z, W.w);
          uint2 pk;
          pk.x = *reinterpret_cast<const uint32_t*>(&lo);
          pk.y = *reinterpret_cast<const uint32_t*>(&hi);
          *reinterpret_cast<uint2*>(bk.wb + static_cast<int64_t>(r) * bk.ldb + c) = pk;
        }
      }
      tile[4 * cq + 0][rl] = __float2bfloat16_rn(W.x);
      tile[4 * cq + 1][rl] = __float2bfloat16_rn(W.y);
      tile[4 * cq + 2][rl] = __float2bfloat16_rn(W.z);
      tile[4 * cq + 3][rl] = __float2bfloat16_rn(W.w);
    }
  } else {
    const int cl = threadIdx.x & (kAdamTileC - 1);
    const int c = c0 + cl;
#pragma unroll
    for (int k = 0; k < kAdamTileR / 4; ++k) {
      const int rl = static_cast<int>(threadIdx.x >> 6) + 4 * k;
      const int r = r0 + rl;
      __nv_bfloat16 hb = __float2bfloat16_rn(0.f);
      if (r < bk.rows && c < bk.cols) {
        const int64_t e = static_cast<int64_t>(r) * bk.cols + c;
        const float wi = adam_one(w, g, m, v, bk.start + e, lr, b1, b2, eps, bc1, bc2);
        hb = __float2bfloat16_rn(wi);
        if (bk.f32 != nullptr) bk.f32[e] = wi;
        if (bk.wb != nullptr) bk.wb[static_cast<int64_t>(r) * bk.ldb + c] = hb;
      }
      tile[cl][rl] = hb;
    }
  }
  __syncthreads();
  // transposed copy wt [cols x rows]: thread -> column c0 + t / 4, rows
  // r0 + 8 (t % 4) .. + 7
  const int tc = c0 + static_cast<int>(threadIdx.x >> 2);
  const int q = threadIdx.x & 3;
  const int tr = r0 + 8 * q;
  if (tc < bk.cols && tr < bk.rows) {
    __nv_bfloat16* dst = bk.wt + static_cast<int64_t>(tc) * bk.rows + tr;
    const __nv_bfloat16* src = &tile[threadIdx.x >> 2][8 * q];
    if (bk.rows % 8 == 0) {  // tr + 8 <= rows, 16-byte aligned
      *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
    } else {
      for (int k = 0; k < 8 && tr + k < bk.rows; ++k) dst[k] = src[k];
    }
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

cudaError_t launch_grad_reduce(const GradReduce& g0, cudaStream_t s) {
  GradReduce g = g0;
  if (g.nsplit < 0 || g.nsplit > kRedJobs) return cudaErrorInvalidValue;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  g.blk0[0] = 0;
  for (int j = 0; j < g.nsplit; ++j) {
    RedSplit& a = g.split[j];
    if (a.part == nullptr || a.out == nullptr || a.S < 1 || a.rows < 0 || a.cols < 1 ||
        a.ldp < a.cols || a.ldo < a.cols)
      return cudaErrorInvalidValue;
    a.vec = a.cols % 4 == 0 && a.ldp % 4 == 0 && a.ldo % 4 == 0 && a.split_stride % 4 == 0 &&
            al16(a.part) && al16(a.out);
    const int64_t nb = (static_cast<int64_t>(a.rows) * a.cols + 1023) / 1024;
    if (g.blk0[j] + nb > (1ll << 30)) return cudaErrorInvalidValue;
    g.blk0[j + 1] = g.blk0[j] + static_cast<int>(nb);
  }
  for (int j = g.nsplit + 1; j <= kRedJobs; ++j) g.blk0[j] = g.blk0[g.nsplit];
  int64_t blocks = g.blk0[g.nsplit];
  RedCols& c = g.cols;
  if (c.X != nullptr) {
    const int ncb = (c.N + 255) / 256;
    const int n4 = (c.N + 3) / 4 * 4;
    if (c.N < 1 || c.M < 0 || c.R < 1 || ncb > kRedTickets || c.cpart == nullptr ||
        c.ticket == nullptr || c.nseg < 0 || c.nseg > kRedSegs || c.ldc < n4 || c.ldc % 4 != 0 ||
        !al16(c.cpart) || c.ld < c.N)
      return cudaErrorInvalidValue;
    for (int k = 0; k < c.nseg; ++k)
      if (c.out[k] == nullptr || c.c0[k] < 0 || c.cnt[k] < 0 || c.c0[k] + c.cnt[k] > c.N)
        return cudaErrorInvalidValue;
    // whole 4-column loads: rows padded to a multiple of 4 columns, aligned
    const uintptr_t xa = reinterpret_cast<uintptr_t>(c.X);
    if (c.ld % 4 != 0 || c.ld < n4 || (xa & (c.x_bf16 ? 7u : 15u)) != 0) return cudaErrorInvalidValue;
    blocks += static_cast<int64_t>(ncb) * c.R;
  }
  if (blocks == 0) return cudaSuccess;
  if (blocks > (1ll << 31) - 1) return cudaErrorInvalidValue;
  grad_reduce_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_adam_refresh(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                                float b1, float b2, float eps, float bc1, float bc2,
                                const AdamBlocks& blocks0, cudaStream_t s) {
  AdamBlocks blocks = blocks0;
  if (blocks.n < 1 || blocks.n > kAdamBlocks) return cudaErrorInvalidValue;
  // the blocks tile [0, n) in order; each gets its CTAs
  int64_t next = 0, ctas = 0;
  for (int j = 0; j < blocks.n; ++j) {
    AdamBlock& bk = blocks.b[j];
    if (bk.start != next || bk.rows < 1 || bk.cols < 1) return cudaErrorInvalidValue;
    if (bk.wt != nullptr && (reinterpret_cast<uintptr_t>(bk.wt) & 15u) != 0) return cudaErrorInvalidValue;
    auto al = [](const void* q, uintptr_t a) { return (reinterpret_cast<uintptr_t>(q) & (a - 1)) == 0; };
    bk.vec = bk.wt != nullptr && bk.cols % 4 == 0 && bk.start % 4 == 0 && al(w, 16) && al(g, 16) &&
             al(m, 16) && al(v, 16) && (bk.f32 == nullptr || al(bk.f32, 16)) &&
             (bk.wb == nullptr || (al(bk.wb, 8) && bk.ldb % 4 == 0));
    const int64_t count = static_cast<int64_t>(bk.rows) * bk.cols;
    next += count;
    bk.cta0 = static_cast<int>(ctas);
    ctas += bk.wt != nullptr ? static_cast<int64_t>((bk.rows + kAdamTileR - 1) / kAdamTileR) *
                                   ((bk.cols + kAdamTileC - 1) / kAdamTileC)
                             : (count + kAdamLinear - 1) / kAdamLinear;
    if (ctas > (1ll << 30)) return cudaErrorInvalidValue;
  }
  if (next != n) return cudaErrorInvalidValue;
  adam_refresh_kernel<<<static_cast<unsigned>(ctas), 256, 0, s>>>(w, g, m, v, lr, b1, b2, eps, bc1,
                                                                   bc2, blocks);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr,
                        float b1, float b2, float eps, float bc1, float bc2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const uintptr_t a = reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(g) |
                      reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
  const int64_t threads = (n + 3) / 4;
  adam_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(
      w, g, m, v, n, lr, b1, b2, eps, bc1, bc2, (a & 15u) == 0 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_hg_adam_pack(float* w, const float* g, float* m, float* v, int64_t entries,
                                float lr, float b1, float b2, float eps, float bc1, float bc2,
                                const HashGridParams& from, const HashGridParams& to,
                                uint32_t* dst, cudaStream_t s) {
  if (entries <= 0) return cudaSuccess;
  const uintptr_t a = reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(g) |
                      reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
  const int64_t threads = (entries + 1) / 2;
  hg_adam_pack_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(
      w, g, m, v, entries, lr, b1, b2, eps, bc1, bc2, from, to, dst, (a & 15u) == 0 ? 1 : 0);
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
