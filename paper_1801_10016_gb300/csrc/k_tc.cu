// Low-precision purification steps on the tcgen05 tensor cores (sm_103a).
//
// One launch = one SP2 step (Eq. 2) for every part.  Work item = one upper-triangular
// 128x128 output tile (ti <= tj) of one part.  Operands are the previous iterate in
// BF16 or TF32 (pre-rounded, in their own arena); X is symmetric, so both the A tile
// (rows I) and the B tile (rows J) are K-major slices of columns of X and stream with
// the same per-part TMA tensor map (128-byte swizzle).  Accumulation is FP32 in TMEM.
// With NPROD = 3 the operand is split X = hi + lo and Y = hi hi + hi lo + lo hi.
//
// Roles (256 threads): warp 0 lane 0 issues TMA loads into a ring of stages, warp 1
// allocates TMEM and its lane 0 issues tcgen05.mma, then all eight warps drain TMEM
// (warp w owns rows 32 (w % 4) .. + 31 and column half w / 4), form X_new = Y or 2X - Y against the FP32 master
// copy, write X_new (master and next operands) to (I, J) and mirrored to (J, I), and
// add the core-diagonal traces of Y and X_new in FP64.  The last block runs the same
// FP64 trace/branch/stopping bookkeeping as the FP64 path.
//
// Every mbarrier wait is bounded; a wait that gives up sets the device timeout flag,
// lets the block finish without further waits, frees its TMEM and returns.
#include <cuda.h>

#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"
#include "tc_ptx.cuh"

namespace gsp2 {

// Store the operand(s) of x at element index e of the operand arena(s).
template <int KIND, int NPROD>
__device__ __forceinline__ void store_operands(void* hi, void* lo, int64_t e, float x) {
  if (KIND != 1) {
    const uint16_t h = Operand<KIND>::bits(x);
    reinterpret_cast<uint16_t*>(hi)[e] = h;
    if (NPROD == 3) reinterpret_cast<uint16_t*>(lo)[e] = Operand<KIND>::bits(x - Operand<KIND>::value(h));
  } else {
    const uint32_t h = Operand<1>::bits(x);
    reinterpret_cast<uint32_t*>(hi)[e] = h;
    if (NPROD == 3) reinterpret_cast<uint32_t*>(lo)[e] = Operand<1>::bits(x - Operand<1>::value(h));
  }
}

// Store the operand(s) of N consecutive elements x[0..N-1] (N a multiple of 8) starting at
// element e (16-byte aligned) with vector stores.
template <int KIND, int NPROD, int N>
__device__ __forceinline__ void store_operand_row(void* hi, void* lo, int64_t e, const float (&x)[N]) {
  static_assert(N % 8 == 0, "whole 16-byte vectors");
  if (KIND != 1) {
    uint32_t hw[N / 2], lw[N / 2];
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const uint16_t h0 = Operand<KIND>::bits(x[2 * q]), h1 = Operand<KIND>::bits(x[2 * q + 1]);
      hw[q] = (uint32_t)h0 | ((uint32_t)h1 << 16);
      if (NPROD == 3) {
        const uint16_t l0 = Operand<KIND>::bits(x[2 * q] - Operand<KIND>::value(h0));
        const uint16_t l1 = Operand<KIND>::bits(x[2 * q + 1] - Operand<KIND>::value(h1));
        lw[q] = (uint32_t)l0 | ((uint32_t)l1 << 16);
      }
    }
    uint4* dh = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(hi) + e);
#pragma unroll
    for (int q = 0; q < N / 8; ++q) dh[q] = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
    if (NPROD == 3) {
      uint4* dl = reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(lo) + e);
#pragma unroll
      for (int q = 0; q < N / 8; ++q) dl[q] = make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
    }
  } else {
    uint4* dh = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(hi) + e);
    uint4* dl = reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(lo) + e);
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        h[u] = Operand<1>::bits(x[4 * q + u]);
        if (NPROD == 3) l[u] = Operand<1>::bits(x[4 * q + u] - Operand<1>::value(h[u]));
      }
      dh[q] = make_uint4(h[0], h[1], h[2], h[3]);
      if (NPROD == 3) dl[q] = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

template <int KIND, int NPROD>
__global__ void __launch_bounds__(256, 2) square_tc_kernel(TcStepArgs a) {
  constexpr int NOPS = NPROD == 3 ? 4 : 2;
  constexpr int STAGES = NPROD == 3 ? 2 : 3;
  constexpr uint32_t STAGE_B = NOPS * kTileBytes;
  constexpr int ES = Kind<KIND>::ES;  // operand element bytes
  constexpr int BKE = 128 / ES;          // K elements per stage (one 128-byte swizzle row)
  constexpr int KMMA = Kind<KIND>::KMMA;
  constexpr int NMMA = BKE / KMMA;       // MMAs per stage and product (4)
  // instruction descriptor: FP32 accumulate, A/B format, K-major A and B, N = 128, M = 128
  constexpr uint32_t FMT = Kind<KIND>::FMT;
  constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

  int step = a.step;
  if (a.tail) {
    const int32_t stt = *(volatile int32_t*)&a.ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&a.ctl.st->steps + 1;
  } else if (*(volatile int32_t*)&a.ctl.st->stopped) {
    return;
  }
  const int bi = (step - 1) & 1, bo = step & 1;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_B;  // full[s], empty[s], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 1));
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t done = bars + 8u * (2 * STAGES);
  auto tile_addr = [&](int s, int op) { return base + (uint32_t)s * STAGE_B + (uint32_t)op * kTileBytes; };

  int32_t* abort_flag = &a.ctl.st->timeout;
  const Tile t = a.tiles[blockIdx.x];
  const PartDesc p = a.parts[t.part];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = t.ti * 128, c0 = t.tj * 128;
  const int nk = (p.s + BKE - 1) / BKE;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    const CUtensorMap* mhi = reinterpret_cast<const CUtensorMap*>(a.map_hi[bi]) + t.part;
    const CUtensorMap* mlo = reinterpret_cast<const CUtensorMap*>(a.map_lo[bi]) + t.part;
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty(s), ((kb / STAGES) - 1) & 1, abort_flag)) {
        *s_err = 1;
        break;
      }
      mbar_expect_tx(full(s), STAGE_B);
      const int k0 = kb * BKE;
      tma_load_2d(tile_addr(s, 0), mhi, k0, r0, full(s));
      tma_load_2d(tile_addr(s, 1), mhi, k0, c0, full(s));
      if (NPROD == 3) {
        tma_load_2d(tile_addr(s, 2), mlo, k0, r0, full(s));
        tma_load_2d(tile_addr(s, 3), mlo, k0, c0, full(s));
      }
      issued = kb + 1;
    }
    // do not leave while copies are in flight: wait (bounded) for the last stages issued
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb) {
      if (!mbar_wait_own(full(kb % STAGES), (kb / STAGES) & 1)) *s_err = 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool bad = false;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full(s), (kb / STAGES) & 1, abort_flag)) {
        *s_err = 1;
        bad = true;
        break;
      }
      tc_fence_after();
      const uint64_t ah = smem_desc(tile_addr(s, 0)), bh = smem_desc(tile_addr(s, 1));
      const uint64_t al = smem_desc(tile_addr(s, 2)), bl = smem_desc(tile_addr(s, 3));
#pragma unroll
      for (int kk = 0; kk < NMMA; ++kk) {
        const uint64_t adv = (uint64_t)((kk * KMMA * ES) >> 4);
        // hi x hi and hi x lo share their A operand (collector buffer)
        mma_col<KIND>(NPROD == 3 ? 1 : 0, tmem, ah + adv, bh + adv, IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
        if (NPROD == 3) {
          mma_col<KIND>(3, tmem, ah + adv, bl + adv, IDESC, 1u);
          mma<KIND>(tmem, al + adv, bh + adv, IDESC, 1u);
        }
      }
      mma_commit(empty(s));
    }
    mma_commit(done);
    // after an abort the epilogue no longer waits for `done`: the MMAs issued must still
    // finish before the block frees its TMEM
    if (bad) (void)mbar_wait_own(done, 0);
  }
  __syncwarp();

  // epilogue: 8 warps; warp w drains TMEM lanes 32 (w % 4) .. + 31 (its rows) and the
  // column half w / 4, in chunks of 32 columns
  // warp-uniform outcome: tcgen05.ld is a warp-collective instruction
  const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, abort_flag));
  if (!ok) *s_err = 1;
  tc_fence_after();
  int8_t al;
  if (a.tail == 1) al = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
  else if (a.tail == 2) al = (int8_t)(-a.ctl.alpha[step - 1]);
  else al = a.ctl.alpha[step];
  const float* Xi = a.master[bi] + p.off;
  float* Xo = a.master[bo] + p.off;
  void* ohi = a.op_hi[bo];
  void* olo = a.op_lo[bo];
  const int64_t ld = p.ld;
  const int quarter = warp & 3, half = warp >> 2;
  const int m = quarter * 32 + lane;
  const int r = r0 + m;
  const bool diag = t.slot >= 0;
  double tY = 0.0, tN = 0.0;
  if (ok) {
#pragma unroll 1
    for (int cc = 0; cc < 2; ++cc) {
      const int cb = half * 2 + cc;
      const int cbase = c0 + cb * 32;
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cb * 32), v);
      float x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = Xi[(int64_t)(cbase + j) * ld + r];
      // the one diagonal entry of this row segment, if any, picked out in FP32 and added in
      // FP64 once (an FP64 add in the unrolled loop would be issued for every element)
      float yd = 0.0f, zd = 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float y = __uint_as_float(v[j]) * Kind<KIND>::YSCALE;
        const float z = (al > 0) ? (2.0f * x[j] - y) : y;
        yd = (cbase + j == r) ? y : yd;
        zd = (cbase + j == r) ? z : zd;
        x[j] = z;
      }
      if (diag && r >= cbase && r < cbase + 32 && r < p.c) {
        tY += (double)yd;
        tN += (double)zd;
      }
#pragma unroll
      // diagonal tiles: keep the upper triangle (c >= r) and mirror it, so X stays exactly
      // symmetric whatever order the tensor cores sum the split products in
      for (int j = 0; j < 32; ++j) {
        if (t.ti == t.tj && cbase + j < r) continue;
        const int64_t e = (int64_t)(cbase + j) * ld + r;
        Xo[e] = x[j];
        store_operands<KIND, NPROD>(ohi, olo, p.off + e, x[j]);
      }
      if (t.ti == t.tj && cbase <= r) {
        for (int j = 0; j < 32; ++j) {
          if (cbase + j <= r) continue;
          const int64_t e = (int64_t)r * ld + cbase + j;
          Xo[e] = x[j];
          store_operands<KIND, NPROD>(ohi, olo, p.off + e, x[j]);
        }
      } else {
        const int64_t e0 = (int64_t)r * ld + cbase;
        float4* dst = reinterpret_cast<float4*>(Xo + e0);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        store_operand_row<KIND, NPROD, 32>(ohi, olo, p.off + e0, x);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem));
  if (threadIdx.x == 0 && *s_err) a.ctl.st->timeout = 1;

  if (diag) {
    const double2 sum = block_sum2(tY, tN);
    if (threadIdx.x == 0) a.slots[t.slot] = sum;
  }
  if (last_block_ticket(&a.ctl.st->counter)) {
    double u = 0.0, w = 0.0;
    for (int k = threadIdx.x; k < a.nslots; k += blockDim.x) {
      u += ld_cg(&a.slots[k].x);
      w += ld_cg(&a.slots[k].y);
    }
    const double2 sum = block_sum2(u, w);
    if (threadIdx.x == 0) {
      if (a.ctl.st->timeout) {
        a.ctl.st->status = ST_TIMEOUT;
        a.ctl.st->stopped = 1;
      } else if (a.tail) {
        a.ctl.alpha[step] = al;
        finish_tail(a.ctl, step, sum.y, sum.x, false);
      } else {
        finish_step(a.ctl, step, sum.y, sum.x);
      }
      a.ctl.st->counter = 0;
    }
  }
}

// Persistent variant: one CTA per SM walks the tiles (largest parts first): blockIdx.x,
// then the ones its producer claims from a counter (steps and reverse steps), or
// blockIdx.x + gridDim.x, ... in the static deal.  Two TMEM accumulators let the epilogue of one tile run
// while the tensor cores work on the next.  20 warps: warp 0 lane 0 issues TMA loads,
// warp 1 owns TMEM and its lane 0 issues tcgen05.mma, warps 4..19 drain TMEM (four per
// lane quarter, so that the epilogue, which writes the master and operand copies of the
// tile and its mirror, keeps up with the tensor cores).  Same arithmetic and the same
// bookkeeping as square_tc_kernel, bitwise; the MMAs of a part's last column block cover
// only its columns, and the epilogue leaves the padding beyond them alone.
//
// MODE 1 rebuilds iterate X_step of the FP32 adjoint from explicit buffers with the
// recorded branch; MODE 2 is a reverse step of that adjoint: an upper tile (I, J) of
// Xbar X + X Xbar is one product over K = 2s, rows I of [Xbar | X] times rows J of
// [X | Xbar] (both symmetric and stored whole), and Xbar_new = that or 2 Xbar minus it.
// The adjoint runs on FP16 hi + lo operands (KIND 2); Xbar's carry a per-part scale.
// Neither mode keeps traces or runs the step bookkeeping.

// 2^e as FP32 for -126 <= e <= 127 (built from the exponent bits).
__device__ __forceinline__ float pow2i(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Columns of tile column block tj that an MMA must cover: those inside the part, rounded up
// to 16 (N of an M = 128 MMA is a multiple of 16); the rest of the block is zero padding.
__host__ __device__ constexpr int tc_tile_cols(int s, int tj) {
  return s - tj * 128 >= 128 ? 128 : ((s - tj * 128 + 15) & ~15);
}

constexpr int TC_EPI_WARPS = 16;  // 4 per TMEM lane quarter, 32 columns each
constexpr int TC_RING = 4;        // dynamic schedule: tiles claimed ahead of the MMA and epilogue warps
constexpr int TC_THREADS = 32 * (4 + TC_EPI_WARPS);
enum : int { TC_STEP = 0, TC_REBUILD = 1, TC_ADJOINT = 2 };

template <int KIND, int NPROD, int MODE = TC_STEP>
__global__ void __launch_bounds__(TC_THREADS, 1) square_tc_persistent_kernel(TcStepArgs a) {
  constexpr int NOPS = NPROD == 3 ? 4 : 2;
  constexpr int STAGES = NPROD == 3 ? 3 : 4;
  constexpr uint32_t STAGE_B = NOPS * kTileBytes;
  constexpr int ES = Kind<KIND>::ES;
  constexpr int BKE = 128 / ES;
  constexpr int KMMA = Kind<KIND>::KMMA;
  constexpr int NMMA = BKE / KMMA;
  constexpr uint32_t FMT = Kind<KIND>::FMT;
  // instruction descriptor without N (set per tile: the last column block of a part covers
  // only the part's columns, rounded up to 16)
  constexpr uint32_t IDESC0 = (1u << 4) | (FMT << 7) | (FMT << 10) | ((128u >> 4) << 24);
  static_assert(MODE == TC_STEP || (KIND == 2 && NPROD == 3), "the FP32 adjoint runs on FP16 hi + lo operands");
  // the FP16 adjoint's reverse step: Xbar's operands carry a per-part scale (read at one,
  // written at the next) and the step records each part's largest |Xbar_new|
  constexpr bool XBAR16 = MODE == TC_ADJOINT && KIND == 2;
  // 16-bit kinds keep only the tiles on or above the diagonal (diagonal tiles whole): an
  // operand slice in a K block right of the tile's own block is read MN-major from the
  // upper tile (two boxes of 64 rows, 8 KB apart, 128-byte swizzle, transpose bit)
  constexpr bool UPPER = KIND != 1;

  int step = a.step;
  int n = 0;
  if (MODE != TC_STEP) {
    // steps <= 0 count back from n (the tail steps); loop steps end at n - adj_tail, and
    // the sweep never reads the loop's last iterate from a rebuild
    n = *(volatile int32_t*)&a.ctl.st->steps;
    if (step <= 0) {
      step += n;
      if (step < 1) return;
    } else if (step > n - a.adj_tail || (MODE == TC_REBUILD && step == n - a.adj_tail)) {
      return;
    }
  } else if (a.tail) {
    const int32_t stt = *(volatile int32_t*)&a.ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&a.ctl.st->steps + 1;
  } else if (*(volatile int32_t*)&a.ctl.st->stopped) {
    return;
  }
  // iterate buffers read / written; the adjoint's Xbar: in (n - step) & 1, out the other
  const int bi = MODE == TC_ADJOINT ? (n - step) & 1 : (step - 1) & 1;
  const int bo = MODE == TC_ADJOINT ? bi ^ 1 : step & 1;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_B;  // full[S], empty[S], tfull[2], tempty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 4));
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  double2* red = reinterpret_cast<double2*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 4) + 16);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  auto tfull = [&](int b) { return bars + 8u * (2 * STAGES + b); };
  auto tempty = [&](int b) { return bars + 8u * (2 * STAGES + 2 + b); };
  auto tile_addr = [&](int s, int op) { return base + (uint32_t)s * STAGE_B + (uint32_t)op * kTileBytes; };
  int32_t* abort_flag = &a.ctl.st->timeout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // dynamic schedule (steps and reverse steps; the rebuilt iterates, which may run beside
  // reverse steps and have no last block, keep the static deal): the producer claims each
  // next tile from a counter in global memory and passes it to the MMA thread and the
  // epilogue warps through a ring in shared memory (full: claimed; empty: read by all of
  // them); -1 ends the walk
  const bool dyn = a.tile_ctr != nullptr && MODE != TC_REBUILD;
  const uint32_t ring_bars = smem_u32(red + TC_EPI_WARPS);
  int* s_items = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(red + TC_EPI_WARPS) + 8 * 2 * TC_RING);
  auto item_full = [&](int q) { return ring_bars + 8u * q; };
  auto item_empty = [&](int q) { return ring_bars + 8u * (TC_RING + q); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), TC_EPI_WARPS);
    }
    for (int q = 0; q < TC_RING; ++q) {
      mbar_init(item_full(q), 1);
      mbar_init(item_empty(q), 1 + TC_EPI_WARPS);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: one ring of stages across all tiles of this CTA
    uint32_t g = 0;
    bool bad = false;
    // dynamic: the first item is blockIdx.x, the next ones gridDim.x + the counter's count,
    // each claimed one item ahead so that the atomic's latency hides behind an item's loads
    int nxt = dyn && (int)blockIdx.x < a.ntiles ? (int)gridDim.x + (int)atomicAdd(a.tile_ctr, 1u) : a.ntiles;
    for (int v = 0, ti = blockIdx.x; !bad; ++v, ti += gridDim.x) {
      if (dyn) {
        if (v > 0) {
          ti = nxt;
          if (ti < a.ntiles) nxt = (int)gridDim.x + (int)atomicAdd(a.tile_ctr, 1u);
        }
        const int q = v % TC_RING;
        if (v >= TC_RING && !mbar_wait(item_empty(q), ((v / TC_RING) - 1) & 1, abort_flag)) {
          bad = true;
          break;
        }
        s_items[q] = ti < a.ntiles ? ti : -1;
        mbar_arrive(item_full(q));
      }
      if (ti >= a.ntiles) break;
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      // operand maps: the step's input iterate (MODE 0: by parity; 1 and 2: the rebuilt X)
      const CUtensorMap* mhi =
          reinterpret_cast<const CUtensorMap*>(MODE == TC_STEP ? a.map_hi[bi] : a.xmap_hi) + t.part;
      const CUtensorMap* mlo =
          reinterpret_cast<const CUtensorMap*>(MODE == TC_STEP ? a.map_lo[bi] : a.xmap_lo) + t.part;
      const CUtensorMap* bhi =  // Xbar (adjoint)
          MODE == TC_ADJOINT ? reinterpret_cast<const CUtensorMap*>(a.map_hi[bi]) + t.part : nullptr;
      const CUtensorMap* blo = MODE == TC_ADJOINT ? reinterpret_cast<const CUtensorMap*>(a.map_lo[bi]) + t.part : nullptr;
      // the same arenas through MN-major boxes (16-bit kinds)
      const CUtensorMap* mhi_mn =
          UPPER ? reinterpret_cast<const CUtensorMap*>(MODE == TC_STEP ? a.map_mn_hi[bi] : a.xmap_mn_hi) + t.part
                : nullptr;
      const CUtensorMap* mlo_mn =
          UPPER ? reinterpret_cast<const CUtensorMap*>(MODE == TC_STEP ? a.map_mn_lo[bi] : a.xmap_mn_lo) + t.part
                : nullptr;
      const CUtensorMap* bhi_mn =
          (UPPER && MODE == TC_ADJOINT) ? reinterpret_cast<const CUtensorMap*>(a.map_mn_hi[bi]) + t.part : nullptr;
      const CUtensorMap* blo_mn =
          (UPPER && MODE == TC_ADJOINT) ? reinterpret_cast<const CUtensorMap*>(a.map_mn_lo[bi]) + t.part : nullptr;
      // a diagonal tile of X X needs rows I only (B = A): two K blocks per stage
      const bool dg = MODE != TC_ADJOINT && t.ti == t.tj;
      const int sub = dg ? 2 : 1;
      const int nk = (p.s + sub * BKE - 1) / (sub * BKE);
      for (int kb = 0; kb < (MODE == TC_ADJOINT ? 2 * nk : nk); ++kb, ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(empty(s), ((g / STAGES) - 1) & 1, abort_flag)) {
          bad = true;
          break;
        }
        mbar_expect_tx(full(s), STAGE_B);
        // rows `blk` of the K block at k0: K-major from the tile (k block, blk) where it is on
        // or above the diagonal, else (16-bit kinds) MN-major from the upper tile (blk, k block)
        auto load = [&](uint32_t dst, const CUtensorMap* mk, const CUtensorMap* mm, int k0, int blk) {
          if (UPPER && k0 / 128 > blk) {
            tma_load_2d(dst, mm, blk * 128, k0, full(s));
            tma_load_2d(dst + kTileBytes / 2, mm, blk * 128 + 64, k0, full(s));
          } else {
            tma_load_2d(dst, mk, k0, blk * 128, full(s));
          }
        };
        if (MODE == TC_ADJOINT) {
          // first nk blocks: Xbar (rows I) times X (rows J); then X (rows I) times Xbar (rows J)
          const bool h2 = kb >= nk;
          const int k0 = (h2 ? kb - nk : kb) * BKE;
          load(tile_addr(s, 0), h2 ? mhi : bhi, h2 ? mhi_mn : bhi_mn, k0, t.ti);
          load(tile_addr(s, 1), h2 ? bhi : mhi, h2 ? bhi_mn : mhi_mn, k0, t.tj);
          load(tile_addr(s, 2), h2 ? mlo : blo, h2 ? mlo_mn : blo_mn, k0, t.ti);
          load(tile_addr(s, 3), h2 ? blo : mlo, h2 ? blo_mn : mlo_mn, k0, t.tj);
        } else if (dg) {
          for (int u = 0; u < 2; ++u) {
            const int k0 = (2 * kb + u) * BKE;
            load(tile_addr(s, u * (NOPS / 2)), mhi, mhi_mn, k0, t.ti);
            if (NPROD == 3) load(tile_addr(s, u * 2 + 1), mlo, mlo_mn, k0, t.ti);
          }
        } else {
          const int k0 = kb * BKE;
          load(tile_addr(s, 0), mhi, mhi_mn, k0, t.ti);
          load(tile_addr(s, 1), mhi, mhi_mn, k0, t.tj);
          if (NPROD == 3) {
            load(tile_addr(s, 2), mlo, mlo_mn, k0, t.ti);
            load(tile_addr(s, 3), mlo, mlo_mn, k0, t.tj);
          }
        }
      }
    }
    if (bad) {
      *s_err = 1;
      // do not leave while copies are in flight: bounded wait for the last stages issued
      const uint32_t first = g > STAGES ? g - STAGES : 0;
      for (uint32_t q = first; q < g; ++q) (void)mbar_wait_own(full(q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: tile i accumulates in TMEM columns [128 (i & 1), + 128)
    uint32_t g = 0;
    int i = 0;
    bool bad = false;
    for (int ti = blockIdx.x; !bad; ti += gridDim.x, ++i) {
      if (dyn) {
        const int q = i % TC_RING;
        if (!mbar_wait(item_full(q), (i / TC_RING) & 1, abort_flag)) {
          bad = true;
          break;
        }
        ti = s_items[q];
        mbar_arrive(item_empty(q));
        if (ti < 0) break;
      }
      if (ti >= a.ntiles) break;
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const bool dg = MODE != TC_ADJOINT && t.ti == t.tj;
      const int nk = (MODE == TC_ADJOINT ? 2 : 1) * ((p.s + (dg ? 2 : 1) * BKE - 1) / ((dg ? 2 : 1) * BKE));
      const int b = i & 1, u = i >> 1;
      if (u >= 1 && !mbar_wait(tempty(b), (u - 1) & 1, abort_flag)) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * 128);
      const uint32_t IDESC = IDESC0 | ((uint32_t)(tc_tile_cols(p.s, t.tj) >> 3) << 17);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        if (!mbar_wait(full(s), (g / STAGES) & 1, abort_flag)) {
          bad = true;
          break;
        }
        tc_fence_after();
        for (int v = 0; v < (dg ? 2 : 1); ++v) {  // K blocks of the stage, in K order
          // the K block and how each operand came in (MN-major right of the tile's block)
          const int kq = dg ? 2 * kb + v : (MODE == TC_ADJOINT && kb >= nk / 2 ? kb - nk / 2 : kb);
          const int kt = kq * BKE / 128;
          const bool amn = UPPER && kt > t.ti, bmn = UPPER && kt > t.tj;
          auto desc = [&](uint32_t addr, bool mn) {
            return mn ? smem_desc_mn128(addr, kTileBytes / 2) : smem_desc(addr);
          };
          uint64_t ah, bh, al, bl;
          if (dg) {
            ah = bh = desc(tile_addr(s, v * (NOPS / 2)), amn);
            al = bl = desc(tile_addr(s, v * 2 + 1), amn);
          } else {
            ah = desc(tile_addr(s, 0), amn);
            bh = desc(tile_addr(s, 1), bmn);
            al = desc(tile_addr(s, 2), amn);
            bl = desc(tile_addr(s, 3), bmn);
          }
          // a K = KMMA step advances KMMA elements along a K-major row, KMMA rows of 128 B
          // (64 MN elements) in an MN-major box
          const uint32_t adv_a = amn ? (uint32_t)(KMMA * 128) >> 4 : (uint32_t)(KMMA * ES) >> 4;
          const uint32_t adv_b = (dg ? amn : bmn) ? (uint32_t)(KMMA * 128) >> 4 : (uint32_t)(KMMA * ES) >> 4;
          const uint32_t idesc = IDESC | ((amn ? 1u : 0u) << 15) | (((dg ? amn : bmn) ? 1u : 0u) << 16);
#pragma unroll
          for (int kk = 0; kk < NMMA; ++kk) {
            const uint64_t aa = (uint64_t)(adv_a * kk), ab = (uint64_t)(adv_b * kk);
            // hi x hi and hi x lo share their A operand (collector buffer)
            mma_col<KIND>(NPROD == 3 ? 1 : 0, d, ah + aa, bh + ab, idesc, (kb > 0 || v > 0 || kk > 0) ? 1u : 0u);
            if (NPROD == 3) {
              mma_col<KIND>(3, d, ah + aa, bl + ab, idesc, 1u);
              mma<KIND>(d, al + aa, bh + ab, idesc, 1u);
            }
          }
        }
        mma_commit(empty(s));
      }
      mma_commit(tfull(b));
    }
    if (bad) {
      *s_err = 1;
      // MMAs already issued keep reading shared memory and writing TMEM: wait (on this
      // thread's own limit) for the last commit, which covers all of them
      if (g > 0) (void)mbar_wait_own(empty((g - 1) % STAGES), ((g - 1) / STAGES) & 1);
    }
  } else if (warp >= 4) {
    // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31, columns 32 ((w - 4) / 4) .. + 31,
    // in two halves of 16
    const int quarter = warp & 3, colq = (warp - 4) >> 2;
    const int m = quarter * 32 + lane;
    int i = 0;
    for (int ti = blockIdx.x;; ti += gridDim.x, ++i) {
      if (dyn) {
        const int q = i % TC_RING;
        const bool got = __all_sync(0xffffffffu, mbar_wait(item_full(q), (i / TC_RING) & 1, abort_flag));
        if (!got) {
          *s_err = 1;
          break;
        }
        ti = s_items[q];
        __syncwarp();
        if (lane == 0) mbar_arrive(item_empty(q));
        if (ti < 0) break;
      }
      if (ti >= a.ntiles) break;
      const int b = i & 1, u = i >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull(b), u & 1, abort_flag));
      tc_fence_after();
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      int8_t alf;
      if (MODE != TC_STEP) alf = a.ctl.alpha[step];  // the recorded branch
      else if (a.tail == 1) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
      else if (a.tail == 2) alf = (int8_t)(-a.ctl.alpha[step - 1]);
      else alf = a.ctl.alpha[step];
      const float* Xi = (MODE == TC_REBUILD ? a.xin : a.master[bi]) + p.off;
      float* Xo = (MODE == TC_REBUILD ? a.xout : a.master[bo]) + p.off;
      void* ohi = MODE == TC_REBUILD ? a.xo_hi : a.op_hi[bo];
      void* olo = MODE == TC_REBUILD ? a.xo_lo : a.op_lo[bo];
      const int64_t ld = p.ld;
      const int r0 = t.ti * 128, c0 = t.tj * 128;
      const int r = r0 + m;
      const bool diag = t.slot >= 0;
      // sums back to the unscaled product: 2^-28 for FP16 operands of X 2^14 on both sides,
      // 2^(sig - 28) where the Xbar side is FP16 of Xbar 2^(14 - sig)
      const float ysc = XBAR16 ? pow2i(a.xb_sig[t.part] - 28) : Kind<KIND>::YSCALE;
      const float osc = XBAR16 ? pow2i(-a.xb_sig[a.nparts + t.part]) : 1.0f;  // Xbar_new's operand scale
      uint32_t amax = 0;  // FP16 adjoint: largest |Xbar_new| of the thread's entries (FP32 bits)
      double tY = 0.0, tN = 0.0;
      if (ok) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int cl = colq * 32 + h * 16;
          // 16-column chunks beyond the MMAs' columns lie in the part's zero padding, which
          // no step writes (the iterate and operand arenas are zeroed when the workspace is
          // bound); on a diagonal tile a chunk wholly left of the warp's first row holds only
          // entries below the diagonal, which the mirror of the upper triangle writes
          if (cl >= tc_tile_cols(p.s, t.tj) || (t.ti == t.tj && cl + 16 <= quarter * 32)) continue;
          const int cbase = c0 + cl;
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 128 + cl), v);
          float x[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) x[j] = Xi[(int64_t)(cbase + j) * ld + r];
          // the one diagonal entry of this half row, if any, picked out in FP32 and added in
          // FP64 once (an FP64 add in the unrolled loop would be issued for every element)
          float yd = 0.0f, zd = 0.0f;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float y = __uint_as_float(v[j]) * ysc;
            const float z = (alf > 0) ? (2.0f * x[j] - y) : y;
            yd = (cbase + j == r) ? y : yd;
            zd = (cbase + j == r) ? z : zd;
            x[j] = z;
            if (XBAR16) amax = max(amax, __float_as_uint(z) & 0x7FFFFFFFu);  // NaN bits exceed Inf
          }
          if (MODE == TC_STEP && diag && r >= cbase && r < cbase + 16 && r < p.c) {
            tY += (double)yd;
            tN += (double)zd;
          }
          // diagonal tiles: keep the upper triangle (c >= r) and mirror it, so X stays exactly
          // symmetric whatever order the tensor cores sum the split products in
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (t.ti == t.tj && cbase + j < r) continue;
            const int64_t e = (int64_t)(cbase + j) * ld + r;
            Xo[e] = x[j];
            store_operands<KIND, NPROD>(ohi, olo, p.off + e, XBAR16 ? x[j] * osc : x[j]);
          }
          if (t.ti == t.tj && cbase <= r) {
            // the 16 x 16 blocks of a diagonal tile that straddle the diagonal: element stores
            for (int j = 0; j < 16; ++j) {
              if (cbase + j <= r) continue;
              const int64_t e = (int64_t)r * ld + cbase + j;
              Xo[e] = x[j];
              store_operands<KIND, NPROD>(ohi, olo, p.off + e, XBAR16 ? x[j] * osc : x[j]);
            }
          } else if (!UPPER || t.ti == t.tj) {
            // the mirrored row segment (all of it right of the diagonal): vector stores (the
            // 16-bit kinds keep off-diagonal tiles upper only and mirror diagonal tiles only)
            const int64_t e0 = (int64_t)r * ld + cbase;
            float4* dst = reinterpret_cast<float4*>(Xo + e0);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            if (XBAR16) {
              float xs[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) xs[j] = x[j] * osc;
              store_operand_row<KIND, NPROD, 16>(ohi, olo, p.off + e0, xs);
            } else {
              store_operand_row<KIND, NPROD, 16>(ohi, olo, p.off + e0, x);
            }
          }
        }
      } else {
        *s_err = 1;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
      if (XBAR16) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if (lane == 0 && amax != 0) atomicMax(&a.xb_max[t.part], amax);
      }
      if (MODE == TC_STEP && diag) {
        // fixed-order reduction over the epilogue warps (named barrier 1)
        tY = warp_sum(tY);
        tN = warp_sum(tN);
        if (lane == 0) red[warp - 4] = make_double2(tY, tN);
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * TC_EPI_WARPS) : "memory");
        if (warp == 4 && lane == 0) {
          double2 acc = make_double2(0.0, 0.0);
          for (int w = 0; w < TC_EPI_WARPS; ++w) {
            acc.x += red[w].x;
            acc.y += red[w].y;
          }
          a.slots[t.slot] = acc;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * TC_EPI_WARPS) : "memory");
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
  if (threadIdx.x == 0 && *s_err) {
    a.ctl.st->timeout = 1;
    if (MODE != TC_STEP) a.ctl.st->status = ST_TIMEOUT;  // no step bookkeeping follows
  }
  if (XBAR16 && last_block_ticket(&a.ctl.st->counter)) {
    // the scales move on: the next step reads the operands written at xb_sig[nparts + k] and
    // writes at 2^e (the smallest power of two above max |Xbar_new|; e = 0 for a zero or a
    // non-finite Xbar, whose operands carry the NaN or Inf on) times the headroom, clamped to
    // the range the FP32 scalings stay exact in; the maxima are cleared for the next step
    for (int k = threadIdx.x; k < a.nparts; k += blockDim.x) {
      const uint32_t mb = __ldcg(&a.xb_max[k]);
      a.xb_max[k] = 0u;
      int e = 0;
      if (mb != 0u && mb < 0x7F800000u) (void)frexpf(__uint_as_float(mb), &e);
      e += a.xb_headroom;
      a.xb_sig[k] = a.xb_sig[a.nparts + k];
      a.xb_sig[a.nparts + k] = e < TC_SIG_MIN ? TC_SIG_MIN : (e > TC_SIG_MAX ? TC_SIG_MAX : e);
    }
    if (threadIdx.x == 0) {
      a.ctl.st->counter = 0;
      if (dyn) *a.tile_ctr = 0u;  // every CTA has claimed its last tile
    }
  }
  if (MODE != TC_STEP) return;

  if (last_block_ticket(&a.ctl.st->counter)) {
    double u = 0.0, w = 0.0;
    for (int k = threadIdx.x; k < a.nslots; k += blockDim.x) {
      u += ld_cg(&a.slots[k].x);
      w += ld_cg(&a.slots[k].y);
    }
    const double2 sum = block_sum2(u, w);
    if (threadIdx.x == 0) {
      if (a.ctl.st->timeout) {
        a.ctl.st->status = ST_TIMEOUT;
        a.ctl.st->stopped = 1;
      } else if (a.tail) {
        int8_t alf;
        if (a.tail == 1) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
        else alf = (int8_t)(-a.ctl.alpha[step - 1]);
        a.ctl.alpha[step] = alf;
        finish_tail(a.ctl, step, sum.y, sum.x, false);
      } else {
        finish_step(a.ctl, step, sum.y, sum.x);
      }
      a.ctl.st->counter = 0;
      if (dyn) *a.tile_ctr = 0u;  // every CTA has claimed its last tile: ready for the next launch
    }
  }
}

// Wide variant (tile_shape 1): each work item covers one or two 128-column blocks of a row
// block of upper tiles (two tiles per MMA, N = 256), so every A tile feeds twice the MMA
// work; two 256-column TMEM accumulators.  Stage: A hi (16 KB), A lo, then B hi and B lo of
// up to 256 rows (32 KB each); a diagonal item takes its A from the first rows of B.  The
// arithmetic of every output element is that of the 128 x 128 kernels.
template <int NPROD>
struct TcWideStage {
  static constexpr uint32_t A_HI = 0, A_LO = kTileBytes;
  static constexpr uint32_t B_HI = (NPROD == 3 ? 2 : 1) * kTileBytes;
  static constexpr uint32_t B_LO = B_HI + 2 * kTileBytes;
  static constexpr uint32_t BYTES = (NPROD == 3 ? 6 : 3) * kTileBytes;
  static constexpr int STAGES = NPROD == 3 ? 2 : 4;
};

template <int KIND, int NPROD>
__global__ void __launch_bounds__(TC_THREADS, 1) square_tc_wide_kernel(TcStepArgs a) {
  using SL = TcWideStage<NPROD>;
  constexpr int STAGES = SL::STAGES;
  constexpr uint32_t STAGE_B = SL::BYTES;
  constexpr int ES = Kind<KIND>::ES;
  constexpr int BKE = 128 / ES;
  constexpr int KMMA = Kind<KIND>::KMMA;
  constexpr int NMMA = BKE / KMMA;
  constexpr uint32_t FMT = Kind<KIND>::FMT;
  constexpr uint32_t IDESC0 = (1u << 4) | (FMT << 7) | (FMT << 10) | ((128u >> 4) << 24);  // N set per item

  int step = a.step;
  if (a.tail) {
    const int32_t stt = *(volatile int32_t*)&a.ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&a.ctl.st->steps + 1;
  } else if (*(volatile int32_t*)&a.ctl.st->stopped) {
    return;
  }
  const int bi = (step - 1) & 1, bo = step & 1;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_B;  // full[S], empty[S], tfull[2], tempty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 4));
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  double2* red = reinterpret_cast<double2*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 4) + 16);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  auto tfull = [&](int b) { return bars + 8u * (2 * STAGES + b); };
  auto tempty = [&](int b) { return bars + 8u * (2 * STAGES + 2 + b); };
  auto sa = [&](int s, uint32_t off) { return base + (uint32_t)s * STAGE_B + off; };
  int32_t* abort_flag = &a.ctl.st->timeout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), TC_EPI_WARPS);
    }
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    uint32_t g = 0;
    bool bad = false;
    for (int ti = blockIdx.x; ti < a.ntiles && !bad; ti += gridDim.x) {
      const Tile t = a.tiles[ti];
      const int nb = a.nb[ti];
      const PartDesc p = a.parts[t.part];
      const CUtensorMap* mhi = reinterpret_cast<const CUtensorMap*>(a.map_hi[bi]) + t.part;
      const CUtensorMap* mlo = reinterpret_cast<const CUtensorMap*>(a.map_lo[bi]) + t.part;
      const bool dg = t.ti == t.tj;  // rows I are the first rows of B
      const uint32_t per = (uint32_t)(NPROD == 3 ? 2 : 1) * kTileBytes;  // one 128-row block, hi (+ lo)
      const uint32_t bytes = (uint32_t)(nb + (dg ? 0 : 1)) * per;
      const int nk = (p.s + BKE - 1) / BKE;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !mbar_wait(empty(s), ((g / STAGES) - 1) & 1, abort_flag)) {
          bad = true;
          break;
        }
        mbar_expect_tx(full(s), bytes);
        const int k0 = kb * BKE;
        if (!dg) {
          tma_load_2d(sa(s, SL::A_HI), mhi, k0, t.ti * 128, full(s));
          if (NPROD == 3) tma_load_2d(sa(s, SL::A_LO), mlo, k0, t.ti * 128, full(s));
        }
        for (int q = 0; q < nb; ++q) {
          tma_load_2d(sa(s, SL::B_HI + q * kTileBytes), mhi, k0, (t.tj + q) * 128, full(s));
          if (NPROD == 3) tma_load_2d(sa(s, SL::B_LO + q * kTileBytes), mlo, k0, (t.tj + q) * 128, full(s));
        }
      }
    }
    if (bad) {
      *s_err = 1;
      const uint32_t first = g > STAGES ? g - STAGES : 0;
      for (uint32_t q = first; q < g; ++q) (void)mbar_wait_own(full(q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: item i accumulates in TMEM columns [256 (i & 1), + 128 nb)
    uint32_t g = 0;
    int i = 0;
    bool bad = false;
    for (int ti = blockIdx.x; ti < a.ntiles && !bad; ti += gridDim.x, ++i) {
      const Tile t = a.tiles[ti];
      const int nb = a.nb[ti];
      const PartDesc p = a.parts[t.part];
      const bool dg = t.ti == t.tj;
      const int nk = (p.s + BKE - 1) / BKE;
      const uint32_t idesc = IDESC0 | ((uint32_t)(128 * nb) >> 3) << 17;
      const int b = i & 1, u = i >> 1;
      if (u >= 1 && !mbar_wait(tempty(b), (u - 1) & 1, abort_flag)) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * 256);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % STAGES;
        if (!mbar_wait(full(s), (g / STAGES) & 1, abort_flag)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint64_t bh = smem_desc(sa(s, SL::B_HI)), bl = smem_desc(sa(s, SL::B_LO));
        const uint64_t ah = dg ? bh : smem_desc(sa(s, SL::A_HI)), al = dg ? bl : smem_desc(sa(s, SL::A_LO));
#pragma unroll
        for (int kk = 0; kk < NMMA; ++kk) {
          const uint64_t adv = (uint64_t)((kk * KMMA * ES) >> 4);
          // hi x hi and hi x lo share their A operand (collector buffer)
          mma_col<KIND>(NPROD == 3 ? 1 : 0, d, ah + adv, bh + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          if (NPROD == 3) {
            mma_col<KIND>(3, d, ah + adv, bl + adv, idesc, 1u);
            mma<KIND>(d, al + adv, bh + adv, idesc, 1u);
          }
        }
        mma_commit(empty(s));
      }
      mma_commit(tfull(b));
    }
    if (bad) {
      *s_err = 1;
      // MMAs already issued keep reading shared memory and writing TMEM: wait (on this
      // thread's own limit) for the last commit, which covers all of them
      if (g > 0) (void)mbar_wait_own(empty((g - 1) % STAGES), ((g - 1) / STAGES) & 1);
    }
  } else if (warp >= 4) {
    // epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 and 32 nb columns, in 16-column
    // pieces
    const int quarter = warp & 3, colq = (warp - 4) >> 2;
    const int m = quarter * 32 + lane;
    int i = 0;
    for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x, ++i) {
      const int b = i & 1, u = i >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull(b), u & 1, abort_flag));
      tc_fence_after();
      const Tile t = a.tiles[ti];
      const int nb = a.nb[ti];
      const PartDesc p = a.parts[t.part];
      int8_t alf;
      if (a.tail == 1) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
      else if (a.tail == 2) alf = (int8_t)(-a.ctl.alpha[step - 1]);
      else alf = a.ctl.alpha[step];
      const float* Xi = a.master[bi] + p.off;
      float* Xo = a.master[bo] + p.off;
      void* ohi = a.op_hi[bo];
      void* olo = a.op_lo[bo];
      const int64_t ld = p.ld;
      const int r0 = t.ti * 128, c0 = t.tj * 128;
      const int r = r0 + m;
      const bool diag = t.slot >= 0;
      double tY = 0.0, tN = 0.0;
      if (ok) {
#pragma unroll 1
        for (int h = 0; h < 2 * nb; ++h) {
          // columns colq * 32 nb + 16 h .. + 15 of the item; block 0 of a diagonal item is
          // the diagonal tile
          const int cl = colq * 32 * nb + h * 16;
          const int cbase = c0 + cl;
          const bool dblk = diag && cl < 128;
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cl), v);
          float x[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) x[j] = Xi[(int64_t)(cbase + j) * ld + r];
          float yd = 0.0f, zd = 0.0f;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float y = __uint_as_float(v[j]) * Kind<KIND>::YSCALE;
            const float z = (alf > 0) ? (2.0f * x[j] - y) : y;
            yd = (cbase + j == r) ? y : yd;
            zd = (cbase + j == r) ? z : zd;
            x[j] = z;
          }
          if (dblk && r >= cbase && r < cbase + 16 && r < p.c) {
            tY += (double)yd;
            tN += (double)zd;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (dblk && cbase + j < r) continue;
            const int64_t e = (int64_t)(cbase + j) * ld + r;
            Xo[e] = x[j];
            store_operands<KIND, NPROD>(ohi, olo, p.off + e, x[j]);
          }
          if (dblk && cbase <= r) {
            for (int j = 0; j < 16; ++j) {
              if (cbase + j <= r) continue;
              const int64_t e = (int64_t)r * ld + cbase + j;
              Xo[e] = x[j];
              store_operands<KIND, NPROD>(ohi, olo, p.off + e, x[j]);
            }
          } else {
            const int64_t e0 = (int64_t)r * ld + cbase;
            float4* dst = reinterpret_cast<float4*>(Xo + e0);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            store_operand_row<KIND, NPROD, 16>(ohi, olo, p.off + e0, x);
          }
        }
      } else {
        *s_err = 1;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
      if (diag) {
        tY = warp_sum(tY);
        tN = warp_sum(tN);
        if (lane == 0) red[warp - 4] = make_double2(tY, tN);
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * TC_EPI_WARPS) : "memory");
        if (warp == 4 && lane == 0) {
          double2 acc = make_double2(0.0, 0.0);
          for (int w = 0; w < TC_EPI_WARPS; ++w) {
            acc.x += red[w].x;
            acc.y += red[w].y;
          }
          a.slots[t.slot] = acc;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * TC_EPI_WARPS) : "memory");
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  if (threadIdx.x == 0 && *s_err) a.ctl.st->timeout = 1;

  if (last_block_ticket(&a.ctl.st->counter)) {
    double u = 0.0, w = 0.0;
    for (int k = threadIdx.x; k < a.nslots; k += blockDim.x) {
      u += ld_cg(&a.slots[k].x);
      w += ld_cg(&a.slots[k].y);
    }
    const double2 sum = block_sum2(u, w);
    if (threadIdx.x == 0) {
      if (a.ctl.st->timeout) {
        a.ctl.st->status = ST_TIMEOUT;
        a.ctl.st->stopped = 1;
      } else if (a.tail) {
        int8_t alf;
        if (a.tail == 1) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
        else alf = (int8_t)(-a.ctl.alpha[step - 1]);
        a.ctl.alpha[step] = alf;
        finish_tail(a.ctl, step, sum.y, sum.x, false);
      } else {
        finish_step(a.ctl, step, sum.y, sum.x);
      }
      a.ctl.st->counter = 0;
    }
  }
}

template <int KIND, int NPROD>
static cudaError_t launch_tc_wide(const TcStepArgs& a, int grid, cudaStream_t s) {
  constexpr int STAGES = TcWideStage<NPROD>::STAGES;
  const int smem = STAGES * (int)TcWideStage<NPROD>::BYTES + 1024 + 8 * (2 * STAGES + 4) + 16 + 16 * TC_EPI_WARPS;
  cudaError_t e = cudaFuncSetAttribute(square_tc_wide_kernel<KIND, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  square_tc_wide_kernel<KIND, NPROD><<<grid, TC_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int KIND, int NPROD, int MODE = TC_STEP>
static cudaError_t launch_tc_persistent(const TcStepArgs& a, int grid, cudaStream_t s) {
  constexpr int NOPS = NPROD == 3 ? 4 : 2;
  constexpr int STAGES = NPROD == 3 ? 3 : 4;
  const int smem =
      STAGES * NOPS * (int)kTileBytes + 1024 + 8 * (2 * STAGES + 4) + 16 + 16 * TC_EPI_WARPS + 8 * 2 * TC_RING + 4 * TC_RING;
  cudaError_t e = cudaFuncSetAttribute(square_tc_persistent_kernel<KIND, NPROD, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  square_tc_persistent_kernel<KIND, NPROD, MODE><<<grid, TC_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tc_adjoint(const TcStepArgs& a, int grid, bool rebuild, cudaStream_t s) {
  const int g = grid < a.ntiles ? grid : a.ntiles;
  return rebuild ? launch_tc_persistent<2, 3, TC_REBUILD>(a, g, s) : launch_tc_persistent<2, 3, TC_ADJOINT>(a, g, s);
}

// FP16 hi + lo operands of an FP32 arena, one warp per column up to ld: of x 2^-sig[part]
// (the FP16 adjoint's seed Xbar; sig NULL: of x, an iterate).  Skipped where need > n - tail
// (a checkpoint the reverse sweep does not reach).
__global__ void __launch_bounds__(256) split_f16_kernel(const PartDesc* __restrict__ parts,
                                                        const ColBlock* __restrict__ blocks, const float* x,
                                                        uint16_t* hi, uint16_t* lo, const int32_t* __restrict__ sig,
                                                        int need, int tail, const DevState* st) {
  if (need > *(volatile const int32_t*)&st->steps - tail) return;
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.ld) return;
  const float f = sig ? pow2i(-sig[b.part]) : 1.0f;
  const int64_t cbase = p.off + (int64_t)j * p.ld;
  for (int r = lane; r < p.ld; r += 32) store_operands<2, 3>(hi, lo, cbase + r, x[cbase + r] * f);
}

// Scales of the seed Xbar's FP16 operands: each part's largest |x| into xb_max (one warp
// per column), then, in the last block, the exponent its operands are written at
// (xb_sig[k]) and the one the first reverse step writes at (xb_sig[nparts + k], with the
// headroom); maxima cleared.
__global__ void __launch_bounds__(256) xbar_seed_scale_kernel(const PartDesc* __restrict__ parts,
                                                              const ColBlock* __restrict__ blocks, const float* x,
                                                              uint32_t* xb_max, int32_t* xb_sig, int nparts,
                                                              int headroom, DevState* st) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  uint32_t m = 0;
  if (j < p.s)
    for (int r = lane; r < p.s; r += 32) m = max(m, __float_as_uint(x[p.off + (int64_t)j * p.ld + r]) & 0x7FFFFFFFu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && m != 0) atomicMax(&xb_max[b.part], m);
  if (last_block_ticket(&st->counter)) {
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
      const uint32_t mb = __ldcg(&xb_max[k]);
      xb_max[k] = 0u;
      int e = 0;
      if (mb != 0u && mb < 0x7F800000u) (void)frexpf(__uint_as_float(mb), &e);
      const int e2 = e + headroom;
      xb_sig[k] = e < TC_SIG_MIN ? TC_SIG_MIN : (e > TC_SIG_MAX ? TC_SIG_MAX : e);
      xb_sig[nparts + k] = e2 < TC_SIG_MIN ? TC_SIG_MIN : (e2 > TC_SIG_MAX ? TC_SIG_MAX : e2);
    }
    if (threadIdx.x == 0) st->counter = 0;
  }
}

cudaError_t launch_split_f16(const PartDesc* parts, const ColBlock* blocks, int nblocks, const float* x, void* hi,
                             void* lo, const int32_t* sig, int need, int tail, const DevState* st, cudaStream_t s) {
  split_f16_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, x, (uint16_t*)hi, (uint16_t*)lo, sig, need,
                                                            tail, st);
  return cudaGetLastError();
}

cudaError_t launch_xbar_seed_scale(const PartDesc* parts, const ColBlock* blocks, int nblocks, const float* x,
                                   uint32_t* xb_max, int32_t* xb_sig, int nparts, int headroom, DevState* st,
                                   cudaStream_t s) {
  xbar_seed_scale_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, x, xb_max, xb_sig, nparts, headroom,
                                                                  st);
  return cudaGetLastError();
}


template <int KIND, int NPROD>
static cudaError_t launch_tc(const TcStepArgs& a, int ntiles, cudaStream_t s) {
  constexpr int NOPS = NPROD == 3 ? 4 : 2;
  constexpr int STAGES = NPROD == 3 ? 2 : 3;
  const int smem = STAGES * NOPS * (int)kTileBytes + 1024 + 8 * (2 * STAGES + 1) + 16;
  cudaError_t e = cudaFuncSetAttribute(square_tc_kernel<KIND, NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  square_tc_kernel<KIND, NPROD><<<ntiles, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_square_tc(int kind, int nprod, const TcStepArgs& a, int ntiles, int persistent_grid,
                             cudaStream_t s) {
  if (persistent_grid > 0 && a.nb) {  // 128 x 256 work items
    const int g = persistent_grid < ntiles ? persistent_grid : ntiles;
    if (kind == 0 && nprod == 1) return launch_tc_wide<0, 1>(a, g, s);
    if (kind == 0 && nprod == 3) return launch_tc_wide<0, 3>(a, g, s);
    if (kind == 1 && nprod == 1) return launch_tc_wide<1, 1>(a, g, s);
    if (kind == 1 && nprod == 3) return launch_tc_wide<1, 3>(a, g, s);
    if (kind == 2 && nprod == 3) return launch_tc_wide<2, 3>(a, g, s);
    return cudaErrorInvalidValue;
  }
  if (persistent_grid > 0) {
    const int g = persistent_grid < ntiles ? persistent_grid : ntiles;
    if (kind == 0 && nprod == 1) return launch_tc_persistent<0, 1>(a, g, s);
    if (kind == 0 && nprod == 3) return launch_tc_persistent<0, 3>(a, g, s);
    if (kind == 1 && nprod == 1) return launch_tc_persistent<1, 1>(a, g, s);
    if (kind == 1 && nprod == 3) return launch_tc_persistent<1, 3>(a, g, s);
    if (kind == 2 && nprod == 3) return launch_tc_persistent<2, 3>(a, g, s);
    return cudaErrorInvalidValue;
  }
  if (kind == 0 && nprod == 1) return launch_tc<0, 1>(a, ntiles, s);
  if (kind == 0 && nprod == 3) return launch_tc<0, 3>(a, ntiles, s);
  if (kind == 1 && nprod == 1) return launch_tc<1, 1>(a, ntiles, s);
  if (kind == 1 && nprod == 3) return launch_tc<1, 3>(a, ntiles, s);
  if (kind == 2 && nprod == 3) return launch_tc<2, 3>(a, ntiles, s);
  return cudaErrorInvalidValue;
}

// Gather + Eq. 1 for the low-precision paths: like the FP64 gather, but X0 is stored
// as the FP32 master copy and, for the tensor-core kinds, as the rounded operand(s): the
// warp assembles its column of the master (zeros, then the stored entries), then writes the
// operands from it, coalesced.  Every column of the padded part (up to ld) is written, all
// its rows, or with `upper_rows` only those on or above its diagonal block (the upper-only
// 16-bit steps read no others).  T_0 is summed in FP64 from the stored FP32 values.
// KIND = -1: FP32 master only (CUDA-core FP32 path).
template <int KIND, int NPROD>
__global__ void __launch_bounds__(256) gather_lp_kernel(const PartDesc* __restrict__ parts,
                                                        const ColBlock* __restrict__ blocks,
                                                        const int32_t* __restrict__ Sall,
                                                        const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ loc,
                                                        const int64_t* __restrict__ locptr,
                                                        const double* __restrict__ x0, float* __restrict__ master,
                                                        void* op_hi, void* op_lo, double* __restrict__ slots,
                                                        StepCtl ctl, int upper_rows) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  const int32_t* S = Sall + p.soff;
  double tr = 0.0;
  if (j < p.ld) {
    const int64_t cbase = p.off + (int64_t)j * p.ld;
    const int rend = upper_rows ? min(p.ld, (j / 128 + 1) * 128) : p.ld;
    float* col = master + cbase;
    for (int r = lane; r < rend; r += 32) col[r] = 0.0f;
    __syncwarp();
    if (j < p.s) {
      const int32_t g = S[j];
      const int64_t q0 = rowptr[g], nq = rowptr[g + 1] - q0;
      const int32_t* lj = loc + locptr[p.soff + j];
      for (int64_t t = lane; t < nq; t += 32) {
        const int a = lj[t];
        const int64_t q = q0 + t;
        if (a >= 0 && a < rend) {
          const double x = x0[q];
          const float xf = (float)x;
          col[a] = xf;
          if (a == j && j < p.c) tr = (double)xf;
        }
      }
    }
    if (KIND >= 0) {
      __syncwarp();  // the lanes' stores to the column are visible to the whole warp
      for (int r = lane; r < rend; r += 32)
        store_operands<(KIND < 0 ? 0 : KIND), NPROD>(op_hi, op_lo, cbase + r, col[r]);
    }
  }
  const double2 t = block_sum2(tr, 0.0);
  if (threadIdx.x == 0) slots[blockIdx.x] = t.x;
  if (last_block_ticket(&ctl.st->counter)) {
    double acc = 0.0;
    for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) acc += ld_cg(&slots[k]);
    const double2 sum = block_sum2(acc, 0.0);
    if (threadIdx.x == 0) {
      if (ctl.st->nonfinite) ctl.st->status = ST_NONFINITE;
      finish_step(ctl, 0, sum.x, 0.0);
      ctl.st->counter = 0;
    }
  }
}

cudaError_t launch_gather_lp(int kind, int nprod, const PartDesc* parts, const ColBlock* blocks, int nblocks,
                             const int32_t* Sall, const int64_t* rowptr, const int32_t* loc, const int64_t* locptr,
                             const double* x0, float* master, void* op_hi, void* op_lo, double* slots,
                             const StepCtl& ctl, cudaStream_t s, int upper_rows) {
  const dim3 g(nblocks), b(32 * COLS_PER_BLOCK);
  if (kind < 0)
    gather_lp_kernel<-1, 1><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                            slots, ctl, upper_rows);
  else if (kind == 0 && nprod == 1)
    gather_lp_kernel<0, 1><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                           slots, ctl, upper_rows);
  else if (kind == 0 && nprod == 3)
    gather_lp_kernel<0, 3><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                           slots, ctl, upper_rows);
  else if (kind == 1 && nprod == 1)
    gather_lp_kernel<1, 1><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                           slots, ctl, upper_rows);
  else if (kind == 1 && nprod == 3)
    gather_lp_kernel<1, 3><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                           slots, ctl, upper_rows);
  else if (kind == 2 && nprod == 3)
    gather_lp_kernel<2, 3><<<g, b, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, master, op_hi, op_lo,
                                           slots, ctl, upper_rows);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// FP32 master of the last low-precision iterate -> FP64 arena for the tail steps.
__global__ void convert_kernel(const float* const* __restrict__ master_of_step, double* __restrict__ out, int64_t n,
                               const DevState* st) {
  const float* in = master_of_step[st->steps];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

cudaError_t launch_convert(const float* const* master_of_step, double* out, int64_t n, const DevState* st,
                           cudaStream_t s) {
  convert_kernel<<<152 * 8, 256, 0, s>>>(master_of_step, out, n, st);
  return cudaGetLastError();
}

// Adjoint of a low-precision run: copy the FP32 iterate n - back (n = steps applied,
// found on the device) out of the per-step table, the start of the tail's recomputation.
__global__ void copy_iterate_kernel(const float* const* __restrict__ master_of_step, float* __restrict__ out,
                                    int64_t n, const DevState* st, int back) {
  const int i = st->steps - back;
  const float* in = master_of_step[i < 0 ? 0 : i];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = in[e];
}

cudaError_t launch_copy_iterate(const float* const* master_of_step, float* out, int64_t n, const DevState* st,
                                int back, cudaStream_t s) {
  copy_iterate_kernel<<<152 * 8, 256, 0, s>>>(master_of_step, out, n, st, back);
  return cudaGetLastError();
}

// Encode one tensor map per part over an operand arena: 2-D, inner dimension = rows
// of a column (contiguous), outer = columns, box = 128 bytes x 128 columns, 128-byte
// swizzle.  `enc` is cuTensorMapEncodeTiled obtained from the driver.
// One 2-D tensor map per part over an arena (x = row within a column, y = column), box
// box_bytes x box_cols columns with the swizzle of the box's width (128, 64 or 32 bytes).
int encode_part_maps(void* enc_fn, void* out_maps, const PartDesc* parts, int nparts, void* arena, int kind,
                     int box_bytes, int box_cols) {
  CUtensorMap* out = reinterpret_cast<CUtensorMap*>(out_maps);
  using Enc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                           const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                           CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Enc enc = reinterpret_cast<Enc>(enc_fn);
  const int es = kind == 1 ? 4 : 2;
  const CUtensorMapDataType dt = kind == 0   ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  for (int k = 0; k < nparts; ++k) {
    const PartDesc& p = parts[k];
    cuuint64_t dims[2] = {(cuuint64_t)p.ld, (cuuint64_t)p.ld};
    cuuint64_t strides[1] = {(cuuint64_t)p.ld * es};
    cuuint32_t box[2] = {(cuuint32_t)(box_bytes / es), (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1u, 1u};
    void* addr = (char*)arena + (size_t)p.off * es;
    CUresult r = enc(&out[k], dt, 2, addr,
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     box_bytes == 32   ? CU_TENSOR_MAP_SWIZZLE_32B
                     : box_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                       : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return (int)r;
  }
  return 0;
}

// Maps over the ndig consecutive BF16 digit arenas of the emulated step (digit t at
// arena0 + t dstride bytes) whose boxes take `nbox` digits at once, so that one request
// fills nbox consecutive 128 x box_k digit tiles of a stage.  K-major: (column, row, digit),
// strides 2 ld B and dstride B, box box_k x 128 x nbox, 64-byte rows and swizzle.  MN-major:
// (64 consecutive rows, column, 64-row block, digit), strides 2 ld B, 128 B and dstride B,
// box 64 x box_k x 2 x nbox: each tile lands as two 128-byte-swizzled 64-row atoms back to
// back, as the MN-major matrix descriptors expect them.
int encode_part_maps_digits(void* enc_fn, void* out_k, void* out_mn, const PartDesc* parts, int nparts, void* arena0,
                            size_t dstride, int ndig, int nbox, int box_k) {
  CUtensorMap* ok = reinterpret_cast<CUtensorMap*>(out_k);
  CUtensorMap* om = reinterpret_cast<CUtensorMap*>(out_mn);
  using Enc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                           const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                           CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Enc enc = reinterpret_cast<Enc>(enc_fn);
  for (int k = 0; k < nparts; ++k) {
    const PartDesc& p = parts[k];
    void* addr = (char*)arena0 + (size_t)p.off * 2;
    const cuuint64_t ld = (cuuint64_t)p.ld;
    {
      cuuint64_t dims[3] = {ld, ld, (cuuint64_t)ndig};
      cuuint64_t strides[2] = {ld * 2, (cuuint64_t)dstride};
      cuuint32_t box[3] = {(cuuint32_t)box_k, 128, (cuuint32_t)nbox};
      cuuint32_t estr[3] = {1u, 1u, 1u};
      CUresult r = enc(&ok[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, addr, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, box_k * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                       : CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return (int)r;
    }
    {
      cuuint64_t dims[4] = {64, ld, ld / 64, (cuuint64_t)ndig};
      cuuint64_t strides[3] = {ld * 2, 128, (cuuint64_t)dstride};
      cuuint32_t box[4] = {64, (cuuint32_t)box_k, 2, (cuuint32_t)nbox};
      cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
      CUresult r = enc(&om[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, addr, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return (int)r;
    }
  }
  return 0;
}

}  // namespace gsp2
