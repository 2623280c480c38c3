// trace.cu -- kernels of the sphere-tracing baseline (Sec. 4.4: tracing an
// SDF takes one full network evaluation per step, the DDF one in total).
//   * 3D Fourier encoding of points, or of the current points o + t d of the
//     rays still being traced (rows taken from an active-ray list),
//   * the per-step state update with stream compaction of the active rays,
//   * the closed-form signed distance to a union of spheres and boxes (the
//     regression target that distils the SDF network).
#include <cuda_bf16.h>

#include "kernels.h"

namespace ddf {

namespace {

constexpr int kPtRows = 64;  // points per block of the encoder

// Encodes kPtRows points per block through shared memory (row stride ld+1),
// then writes the rows with 16-byte stores. mode 0: point r = (px, py, pz)[r];
// mode 1: row j < *count is o_i + t_i d_i with i = idx[j].
__global__ void __launch_bounds__(kPtRows)
    encode_points_kernel(const float* __restrict__ px, const float* __restrict__ py,
                         const float* __restrict__ pz, RaySoA rays, const float* __restrict__ t,
                         const int* __restrict__ idx, const int* __restrict__ count, int64_t M,
                         int L, int ld, __nv_bfloat16* __restrict__ out) {
  extern __shared__ float pt_smem[];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kPtRows;
  int64_t limit = M;
  if (count != nullptr && *count < limit) limit = *count;
  if (r0 >= limit) return;
  const int rows = static_cast<int>(limit - r0 < kPtRows ? limit - r0 : kPtRows);
  const int sld = ld + 1;
  const int j = threadIdx.x;
  if (j < rows) {
    float e[3];
    if (idx == nullptr) {
      e[0] = px[r0 + j];
      e[1] = py[r0 + j];
      e[2] = pz[r0 + j];
    } else {
      const int i = idx[r0 + j];
      const float ti = t[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) e[c] = fmaf(ti, rays.p[3 + c][i], rays.p[c][i]);
    }
    float* row = pt_smem + j * sld;
    row[0] = e[0];
    row[1] = e[1];
    row[2] = e[2];
    int col = 3;
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < L; ++k) {
        float s, co;
        sincospif(e[c] * __int_as_float((127 + k) << 23), &s, &co);  // 2^k exactly
        row[col] = s;
        row[col + 1] = co;
        col += 2;
      }
    for (; col < ld; ++col) row[col] = 0.f;
  }
  __syncthreads();
  const int per_row = ld / 8;
  for (int q = threadIdx.x; q < rows * per_row; q += blockDim.x) {
    const int r = q / per_row;
    const int c = (q - r * per_row) * 8;
    const float* src = pt_smem + r * sld + c;
    uint4 w;
    __nv_bfloat162 a = __floats2bfloat162_rn(src[0], src[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(src[2], src[3]);
    __nv_bfloat162 cc = __floats2bfloat162_rn(src[4], src[5]);
    __nv_bfloat162 d = __floats2bfloat162_rn(src[6], src[7]);
    w.x = *reinterpret_cast<uint32_t*>(&a);
    w.y = *reinterpret_cast<uint32_t*>(&b);
    w.z = *reinterpret_cast<uint32_t*>(&cc);
    w.w = *reinterpret_cast<uint32_t*>(&d);
    *reinterpret_cast<uint4*>(out + (r0 + r) * ld + c) = w;
  }
}

__global__ void trace_init_kernel(int n, int* __restrict__ idx, int* __restrict__ count,
                                  float* __restrict__ t, int* __restrict__ steps,
                                  uint8_t* __restrict__ hit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *count = n;
  if (i >= n) return;
  idx[i] = i;
  t[i] = 0.f;
  steps[i] = 0;
  hit[i] = 0;
}

// One step for active slot j (the whole warp takes part in the compaction).
__global__ void trace_update_kernel(const float2* __restrict__ part, int nparts, int cap,
                                    const int* __restrict__ count_in, const int* __restrict__ idx_in,
                                    const float* __restrict__ head_b, float eps, float t_max,
                                    int max_steps, float* __restrict__ t, int* __restrict__ steps,
                                    uint8_t* __restrict__ hit, int* __restrict__ idx_out,
                                    int* __restrict__ count_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int cnt = *count_in;
  bool keep = false;
  int i = 0;
  if (j < cnt) {
    i = idx_in[j];
    float s = head_b[0];
    for (int b = 0; b < nparts; ++b) s += part[static_cast<size_t>(b) * cap + j].x;
    const int st = steps[i] + 1;
    steps[i] = st;
    if (s < eps) {
      hit[i] = 1;
    } else {
      const float tn = t[i] + s;
      t[i] = tn;
      keep = !(tn > t_max) && st < max_steps;
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  int base = 0;
  if (lane == 0 && m != 0u) base = atomicAdd(count_out, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (keep) idx_out[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// min over spheres |p - c| - r and boxes |max(q, 0)| + min(max_i q_i, 0),
// q = |p - centre| - half extent.
__global__ void union_sdf_kernel(const float* __restrict__ spheres, int ns,
                                 const float* __restrict__ boxes, int nb,
                                 const float* __restrict__ px, const float* __restrict__ py,
                                 const float* __restrict__ pz, int64_t n, float* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float p[3] = {px[i], py[i], pz[i]};
  float best = __int_as_float(0x7f800000);
  for (int s = 0; s < ns; ++s) {
    const float dx = p[0] - spheres[4 * s], dy = p[1] - spheres[4 * s + 1],
                dz = p[2] - spheres[4 * s + 2];
    best = fminf(best, sqrtf(dx * dx + dy * dy + dz * dz) - spheres[4 * s + 3]);
  }
  for (int b = 0; b < nb; ++b) {
    float q[3], out2 = 0.f, qmax = -__int_as_float(0x7f800000);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = boxes[6 * b + k], hi = boxes[6 * b + 3 + k];
      q[k] = fabsf(p[k] - 0.5f * (lo + hi)) - 0.5f * (hi - lo);
      const float qp = fmaxf(q[k], 0.f);
      out2 += qp * qp;
      qmax = fmaxf(qmax, q[k]);
    }
    best = fminf(best, sqrtf(out2) + fminf(qmax, 0.f));
  }
  out[i] = best;
}

}  // namespace

cudaError_t launch_encode_points_bf16(const float* px, const float* py, const float* pz, int64_t M,
                                      int L, int ld, __nv_bfloat16* out, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  const size_t smem = static_cast<size_t>(kPtRows) * (ld + 1) * sizeof(float);
  RaySoA none{};
  encode_points_kernel<<<static_cast<unsigned>((M + kPtRows - 1) / kPtRows), kPtRows, smem, s>>>(
      px, py, pz, none, nullptr, nullptr, nullptr, M, L, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_trace_encode(RaySoA rays, const float* t, const int* idx, const int* count,
                                int cap, int L, int ld, __nv_bfloat16* out, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  const size_t smem = static_cast<size_t>(kPtRows) * (ld + 1) * sizeof(float);
  encode_points_kernel<<<(cap + kPtRows - 1) / kPtRows, kPtRows, smem, s>>>(
      nullptr, nullptr, nullptr, rays, t, idx, count, cap, L, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_trace_init(int n, int* idx, int* count, float* t, int* steps, uint8_t* hit,
                              cudaStream_t s) {
  trace_init_kernel<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, s>>>(n, idx, count, t,
                                                                           steps, hit);
  return cudaGetLastError();
}

cudaError_t launch_trace_update(const float2* part, int nparts, int cap, const int* count_in,
                                const int* idx_in, const float* head_b, float eps, float t_max,
                                int max_steps, float* t, int* steps, uint8_t* hit, int* idx_out,
                                int* count_out, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  trace_update_kernel<<<(cap + 255) / 256, 256, 0, s>>>(part, nparts, cap, count_in, idx_in, head_b,
                                                       eps, t_max, max_steps, t, steps, hit,
                                                       idx_out, count_out);
  return cudaGetLastError();
}

cudaError_t launch_union_sdf(const float* spheres, int ns, const float* boxes, int nb,
                             const float* px, const float* py, const float* pz, int64_t n,
                             float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  union_sdf_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(spheres, ns, boxes, nb,
                                                                          px, py, pz, n, out);
  return cudaGetLastError();
}

}  // namespace ddf
