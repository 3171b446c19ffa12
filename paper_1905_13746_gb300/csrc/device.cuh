// Device-side helpers shared by the nbgpu kernels: streaming loads, integer
// dot products, byte -> float decoding, and the bulk-copy (TMA) staging of
// parameter tables into shared memory behind an mbarrier with a bounded wait.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nbg {

// Programmatic dependent launch: a kernel launched with launch_pdl() may start
// while the previous kernel on its stream drains; it calls pdl_wait() before it
// reads anything that kernel wrote (the wait returns at once when there is no
// such kernel).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 16-byte streaming load: read once, do not keep in L1.
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// sum_k a.byte[k] (unsigned) * b.byte[k] (signed) + c
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// sum_k a.byte[k] (unsigned) * b.byte[k] (unsigned) + c
__device__ __forceinline__ uint32_t dp4a_uu(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// c + a.half0 * b.byte0 + a.half1 * b.byte1 (a: two unsigned 16-bit values,
// b: four signed bytes); the .hi form takes bytes 2 and 3 of b
__device__ __forceinline__ int dp2a_lo_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Exact conversion of an unsigned 8- or 16-bit field to float: place the
// field in the low significand bits of 2^23 and subtract 2^23.
__device__ __forceinline__ float u_field_to_f32(uint32_t w, uint32_t sel) {
  return __int_as_float(__byte_perm(w, 0x4B000000u, sel)) - 8388608.0f;
}
// selector for __byte_perm(w, 0x4B000000, sel) giving bytes [w.k, 0, 0, 0x4B]
__device__ __forceinline__ constexpr uint32_t sel_u8(int k) { return 0x7440u | (uint32_t)k; }
constexpr uint32_t kSelU16Lo = 0x7410u;   // [w.0, w.1, 0, 0x4B]
constexpr uint32_t kSelU16Hi = 0x7432u;   // [w.2, w.3, 0, 0x4B]

// two E4M3 values (low 16 bits of w = first two bytes) -> float2
__device__ __forceinline__ float2 e4m3x2_to_f32(uint16_t w) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(w));
  __half2 h = *reinterpret_cast<__half2*>(&h2);
  return __half22float2(h);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (non-tensor TMA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, letting the hardware suspend the thread for up to
// `hint_ns` nanoseconds while the phase is incomplete (no busy polling).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity,
                                                    uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after ~`budget` clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget = 4000000000LL) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Stage `bytes` (multiple of 16, both addresses 16-byte aligned) of a global
// table into shared memory with bulk copies.  All threads of the block call
// it; returns false (and raises `timeout_bit` in *status) if the copy did not
// land within the wait budget.
__device__ __forceinline__ bool stage_table(void* smem_dst, const void* gsrc, uint32_t bytes,
                                            uint64_t* bar, int* status, int timeout_bit) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, bytes);
    constexpr uint32_t kChunk = 32768;
    for (uint32_t off = 0; off < bytes; off += kChunk) {
      uint32_t len = bytes - off < kChunk ? bytes - off : kChunk;
      bulk_g2s(static_cast<char*>(smem_dst) + off, static_cast<const char*>(gsrc) + off, len,
               bar);
    }
  }
  __syncthreads();
  bool ok = mbar_wait_bounded(bar, 0);
  if (!ok && status) atomicOr(status, timeout_bit);
  return __syncthreads_and(ok) != 0;
}

}  // namespace nbg
