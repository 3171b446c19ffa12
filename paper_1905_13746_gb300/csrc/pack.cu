// Storage packing kernels (supporting; run once when data is stored, not
// inside a timed score):
//   U16 counts -> U8 plane + overflow list (column, count - 255) for counts
//                 above 255, row by row in column order;
//   U16 / F32  -> BF16, round to nearest even;
//   U16 / F32  -> FP8 E4M3 with a per-row power-of-two scale 2^e,
//                 e = max(0, ceil(log2(max_row / 448))), round to nearest even.
#include <cub/device/device_scan.cuh>
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.cuh"

namespace nbg {

__global__ void k_pack_u8_count(const uint16_t* X, int64_t n, int F, int64_t ld, int64_t* cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    int c = 0;
    for (int j = lane; j < F; j += 32) c += X[i * ld + j] > 255;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
    if (lane == 0) cnt[i + 1] = c;
    if (i == 0 && lane == 0) cnt[0] = 0;
  }
}

__global__ void k_pack_u8_fill(const uint16_t* X, int64_t n, int F, int64_t ld, uint8_t* plane,
                               int64_t ld_out, const int64_t* ptr, uint16_t* col, uint16_t* add) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    int64_t pos = ptr[i];
    for (int j0 = 0; j0 < F; j0 += 32) {
      const int j = j0 + lane;
      const uint32_t v = j < F ? X[i * ld + j] : 0u;
      if (j < F) plane[i * ld_out + j] = (uint8_t)(v > 255 ? 255 : v);
      const bool big = v > 255;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, big);
      if (big) {
        const int64_t k = pos + __popc(m & ((1u << lane) - 1u));
        col[k] = (uint16_t)j;
        add[k] = (uint16_t)(v - 255);
      }
      pos += __popc(m);
    }
  }
}

__device__ __forceinline__ float src_val(const void* X, int src, int64_t idx) {
  return src == NB_U16 ? (float)static_cast<const uint16_t*>(X)[idx]
                       : static_cast<const float*>(X)[idx];
}

__global__ void k_pack_bf16(const void* X, int src, int64_t n, int F, int64_t ld, uint16_t* out,
                            int64_t ld_out) {
  const int64_t total = n * F;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / F;
    const int j = (int)(t % F);
    const __nv_bfloat16 b = __float2bfloat16_rn(src_val(X, src, i * ld + j));
    out[i * ld_out + j] = *reinterpret_cast<const uint16_t*>(&b);
  }
}

__global__ void k_pack_fp8(const void* X, int src, int64_t n, int F, int64_t ld, uint8_t* out,
                           int64_t ld_out, int8_t* row_exp) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
    float mx = 0.f;
    for (int j = lane; j < F; j += 32) mx = fmaxf(mx, src_val(X, src, i * ld + j));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    int e = 0;
    while (e < 127 && mx > 448.f * exp2f((float)e)) ++e;
    const float inv = exp2f((float)-e);
    if (lane == 0) row_exp[i] = (int8_t)e;
    for (int j = lane; j < F; j += 32) {
      const float v = src_val(X, src, i * ld + j) * inv;
      uint16_t pair;
      asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(pair) : "f"(0.f), "f"(v));
      out[i * ld_out + j] = (uint8_t)(pair & 0xFFu);
    }
  }
}

static unsigned grid_for(int64_t items, int per_block) {
  int64_t b = (items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace nbg

using namespace nbg;

extern "C" nb_status nb_pack_u8_count(const uint16_t* X, int64_t n, int32_t F, int64_t ld,
                                      int64_t* ovf_ptr, int64_t* host_total, void* cuda_stream) {
  if (n < 0 || F < 1 || ld < F || !ovf_ptr || (n > 0 && !X)) {
    set_error("nb_pack_u8_count: bad arguments");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (n == 0) {
    NB_TRY_CUDA(cudaMemsetAsync(ovf_ptr, 0, sizeof(int64_t), st), "memset");
    if (host_total) *host_total = 0;
    return NB_OK;
  }
  count_launch();
  k_pack_u8_count<<<grid_for(n, 8), 256, 0, st>>>(X, n, F, ld, ovf_ptr);
  NB_TRY_CUDA(cudaGetLastError(), "k_pack_u8_count");
  size_t tmp_bytes = 0;
  NB_TRY_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tmp_bytes, ovf_ptr, ovf_ptr, n + 1, st),
              "scan size");
  void* tmp = nullptr;
  NB_TRY_CUDA(cudaMallocAsync(&tmp, tmp_bytes, st), "cudaMallocAsync(scan)");
  cudaError_t e = cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, ovf_ptr, ovf_ptr, n + 1, st);
  cudaFreeAsync(tmp, st);
  NB_TRY_CUDA(e, "scan");
  if (host_total) {
    NB_TRY_CUDA(cudaMemcpyAsync(host_total, ovf_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                st),
                "memcpy total");
    NB_TRY_CUDA(cudaStreamSynchronize(st), "sync");
  }
  return NB_OK;
}

extern "C" nb_status nb_pack_u8_fill(const uint16_t* X, int64_t n, int32_t F, int64_t ld,
                                     uint8_t* plane, int64_t ld_out, const int64_t* ovf_ptr,
                                     uint16_t* ovf_col, uint16_t* ovf_add, void* cuda_stream) {
  if (n < 0 || F < 1 || ld < F || ld_out < F || !ovf_ptr || (n > 0 && (!X || !plane))) {
    set_error("nb_pack_u8_fill: bad arguments");
    return NB_EINVAL;
  }
  if (n == 0) return NB_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  count_launch();
  k_pack_u8_fill<<<grid_for(n, 8), 256, 0, st>>>(X, n, F, ld, plane, ld_out, ovf_ptr, ovf_col,
                                                  ovf_add);
  NB_TRY_CUDA(cudaGetLastError(), "k_pack_u8_fill");
  return NB_OK;
}

extern "C" nb_status nb_pack_bf16(const void* X, nb_dtype src, int64_t n, int32_t F, int64_t ld,
                                  uint16_t* out, int64_t ld_out, void* cuda_stream) {
  if (n < 0 || F < 1 || ld < F || ld_out < F || (src != NB_U16 && src != NB_F32) ||
      (n > 0 && (!X || !out))) {
    set_error("nb_pack_bf16: bad arguments");
    return NB_EINVAL;
  }
  if (n == 0) return NB_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  count_launch();
  k_pack_bf16<<<grid_for(n * F, 256), 256, 0, st>>>(X, src, n, F, ld, out, ld_out);
  NB_TRY_CUDA(cudaGetLastError(), "k_pack_bf16");
  return NB_OK;
}

extern "C" nb_status nb_pack_fp8(const void* X, nb_dtype src, int64_t n, int32_t F, int64_t ld,
                                 uint8_t* out, int64_t ld_out, int8_t* row_exp,
                                 void* cuda_stream) {
  if (n < 0 || F < 1 || ld < F || ld_out < F || (src != NB_U16 && src != NB_F32) ||
      (n > 0 && (!X || !out || !row_exp))) {
    set_error("nb_pack_fp8: bad arguments");
    return NB_EINVAL;
  }
  if (n == 0) return NB_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  count_launch();
  k_pack_fp8<<<grid_for(n, 8), 256, 0, st>>>(X, src, n, F, ld, out, ld_out, row_exp);
  NB_TRY_CUDA(cudaGetLastError(), "k_pack_fp8");
  return NB_OK;
}
