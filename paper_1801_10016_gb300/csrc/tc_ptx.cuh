// PTX wrappers for the tcgen05 / TMA / mbarrier kernels (sm_103a): bounded mbarrier
// waits, 2-D TMA tile loads, shared-memory matrix descriptors, tcgen05.mma issue and
// commit, TMEM loads, and operand rounding.
#pragma once

#include <cuda.h>

#include "gsp2_internal.cuh"

namespace gsp2 {
constexpr uint64_t kWaitNs = 200ull * 1000ull * 1000ull;  // 200 ms; normal waits take microseconds
constexpr uint32_t kTileBytes = 128 * 128;  // 128 rows x 128 bytes

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait: gives up after kWaitNs nanoseconds, or at once when another block
// has already given up (the shared abort flag), and then raises the flag itself.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int32_t* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255u) == 0u) {
      if (*(volatile int32_t*)abort_flag != 0 || global_ns() - t0 > kWaitNs) {
        *(volatile int32_t*)abort_flag = 1;
        return false;
      }
    }
  }
}

// Bounded wait on this thread's own time limit only, for the drains of an aborting CTA:
// the copies and MMAs it has issued still complete whatever other blocks do, so the
// shared abort flag must not cut this wait short (a CTA may not exit, nor free its
// TMEM, while they are in flight).
__device__ __forceinline__ bool mbar_wait_own(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255u) == 0u && global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte swizzle,
// 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// The same for K-major tiles with rows of ROW bytes (32 or 64) and the swizzle of that
// width: 8-row groups 8 ROW bytes apart.
template <int ROW>
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr) {
  static_assert(ROW == 32 || ROW == 64, "32- or 64-byte rows");
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;         // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * ROW) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)(ROW == 32 ? 6 : 4) << 61;  // 32- or 64-byte swizzle
  return d;
}

// MN-major tile of 16-bit elements with 128-byte swizzle: atoms of 64 MN-consecutive
// elements x 8 K values (1 KB); `lbo` bytes between the atoms along MN, 1 KB between the
// groups of 8 K values.
__device__ __forceinline__ uint64_t smem_desc_mn128(uint32_t addr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // leading byte offset: next 64 MN elements
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: next 8 K values
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Operand kinds of the low-precision tensor-core steps: 0 BF16, 1 TF32, 2 FP16 of x 2^14.
// Element bytes, K per MMA, the A/B format code of the instruction descriptor (kind::f16:
// F16 0, BF16 1; kind::tf32: TF32 2) and the factor that scales a product sum back.
template <int KIND>
struct Kind {
  static constexpr int ES = KIND == 1 ? 4 : 2;
  static constexpr int KMMA = KIND == 1 ? 8 : 16;
  static constexpr uint32_t FMT = KIND == 0 ? 1u : (KIND == 1 ? 2u : 0u);
  static constexpr float YSCALE = KIND == 2 ? 3.7252902984619141e-09f : 1.0f;  // 2^-28 = (2^-14)^2
};

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (KIND != 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

// MMA that keeps its A operand in the tensor core's collector buffer for the next MMAs
// with the same A: op 1 reads A from shared memory and keeps it (fill), 2 reuses the kept
// A (use), 3 reuses it for the last time (lastuse); 0 reads A and does not keep it.
// Consecutive MMAs that share A then read it from shared memory once.
#define GSP2_MMA_COL(KINDSTR, OPSTR)                                                                  \
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"                                       \
               " tcgen05.mma.cta_group::1.kind::" KINDSTR ".collector::a::" OPSTR " [%0], %1, %2, %3, p;\n}\n" ::"r"( \
                   tmem),                                                                           \
               "l"(a), "l"(b), "r"(idesc), "r"(acc))
template <int KIND>
__device__ __forceinline__ void mma_col(int op, uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (op == 0) {
    mma<KIND>(tmem, a, b, idesc, acc);
  } else if (KIND != 1) {
    if (op == 1) GSP2_MMA_COL("f16", "fill");
    else if (op == 2) GSP2_MMA_COL("f16", "use");
    else GSP2_MMA_COL("f16", "lastuse");
  } else {
    if (op == 1) GSP2_MMA_COL("tf32", "fill");
    else if (op == 2) GSP2_MMA_COL("tf32", "use");
    else GSP2_MMA_COL("tf32", "lastuse");
  }
}
#undef GSP2_MMA_COL
__device__ __forceinline__ void mma_f16_col(int op, uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  mma_col<0>(op, tmem, a, b, idesc, acc);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// 16 columns of 32 lanes into TMEM (one word per thread and column); tmem_wait_st orders
// them before later TMEM reads of the same thread
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// operand rounding: BF16 round-to-nearest-even, TF32 round-to-nearest (ties away), FP16
// round-to-nearest-even of x 2^14
template <int KIND>
struct Operand;
template <>
struct Operand<0> {
  static __device__ __forceinline__ uint16_t bits(float x) {
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;\n" : "=h"(h) : "f"(x));
    return h;
  }
  static __device__ __forceinline__ float value(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
};
template <>
struct Operand<1> {
  // TF32 (10 fraction bits), round to nearest with ties away from zero, in two integer
  // instructions: adding half of the 13 dropped bits to the sign-magnitude pattern and
  // clearing them rounds the magnitude up exactly when the dropped part is at least half.
  // Non-finite values pass unchanged.
  static __device__ __forceinline__ uint32_t bits(float x) {
    const uint32_t u = __float_as_uint(x);
    if ((u & 0x7F800000u) == 0x7F800000u) return u;
    return (u + 0x1000u) & 0xFFFFE000u;
  }
  static __device__ __forceinline__ float value(uint32_t b) { return __uint_as_float(b); }
};
template <>
struct Operand<2> {
  // |x| <= 1 (the spectrum of X lies in [0, 1]) keeps x 2^14 inside FP16's range, and the
  // scale moves entries down to 2^-28 into FP16's normal range (absolute spacing 2^-38
  // below that); the scalings by powers of two are exact
  static constexpr float kScale = 16384.0f;
  static __device__ __forceinline__ uint16_t bits(float x) {
    uint16_t h;
    asm("cvt.rn.f16.f32 %0, %1;\n" : "=h"(h) : "f"(x * kScale));
    return h;
  }
  static __device__ __forceinline__ float value(uint16_t h) {
    float f;
    asm("cvt.f32.f16 %0, %1;\n" : "=f"(f) : "h"(h));
    return f * (1.0f / kScale);
  }
};


__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

}  // namespace gsp2
