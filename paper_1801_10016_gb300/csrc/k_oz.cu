// FP64-accurate purification steps on the BF16 tensor cores (sm_103a).
//
// GB300 runs FP64 at 1/1800 of its BF16 rate, so the FP64 product X X is rebuilt from
// exact BF16 products, in the spirit of the Ozaki splitting (Ozaki, Ogita, Oishi and
// Rump, 2012).  With T = OZ_SLICES digits:
//
//   every entry of X (|x| <= 1: the spectrum of X stays in [0, 1]) is written in base 2^7
//   with rounded signed digits, x = sum_{t<T} S_t 2^{-7(t+1)} + r, |S_0| <= 2^7 + 1,
//   |S_t| <= 2^6 (t >= 1), |r| <= 2^{-7T-1} (+ 2^-57 from the fixed point); every S_t is an
//   integer exact in BF16;
//
//   X X = sum_{d<T} 2^{-7(d+2)} G_d + (terms below 2^{-7(T+2)}), G_d = sum_{a+b=d} S_a S_b.
//
// Each G_d is a sum of integer products accumulated in FP32 in TMEM.  Because ||X||_2 <= 1,
// sum_k |x_ik x_kj| <= 1, which keeps the leading groups (d <= 4) below 2^24 at the sizes
// here, so they are exact; later groups carry a rounding of 2^-24 relative on a value
// scaled by 2^{-49} or less.  The groups are added as integers into a 64-bit fixed-point
// accumulator (resolution 2^-56), and a final elementwise pass forms X_new = Y or 2X - Y on
// that grid (kept as FP64 master copy), the core traces in FP64, and the digits of X_new for
// the next step by integer arithmetic.  With T = 7 (28 BF16
// products per tile) the digits hold x to 2^-49 and the dropped products are of order
// 2^-63 K 2^12; the error of Y is about 1e-13, far below the 1e-10 parity of the FP64 path.
#include <cuda.h>

#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"
#include "tc_ptx.cuh"

namespace gsp2 {

// Digits of a value held in 64-bit fixed point v = x 2^56 (|x| <= 1 + small): rounded to
// w = x 2^{7T}, then balanced base-2^7 digits from the least significant up, S_t in
// [-64, 63] for t >= 1 and the rest in S_0, so that w = sum_t S_t 2^{7(T-1-t)} exactly;
// written as BF16 to the digit arenas (digit t weighs 2^{-7(t+1)}).
__device__ __forceinline__ void store_digits(uint16_t* const* slices, int64_t e, long long v) {
  constexpr int drop = 56 - 7 * OZ_SLICES;
  long long w = drop > 0 ? ((v + (1ll << (drop - 1))) >> drop) : v;
#pragma unroll
  for (int t = OZ_SLICES - 1; t >= 0; --t) {
    long long dgt;
    if (t > 0) {
      dgt = ((w + 64) & 127) - 64;
      w = (w - dgt) >> 7;
    } else {
      dgt = w;
    }
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;\n" : "=h"(h) : "f"((float)dgt));
    slices[t][e] = h;
  }
}

// Conversions between FP64 and the 2^-56 fixed point done with integer instructions (the
// FP64 pipe of GB300 is 64x slower than its integer pipe), rounding to nearest even.
__device__ __forceinline__ long long to_fixed(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;                                    // zero and subnormals (< 2^-1022)
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1023 - 52 + 56;                       // value * 2^56 = m * 2^sh
  unsigned long long a;
  if (sh >= 0) {
    a = m << sh;                                            // |x| < 2^7 keeps this below 2^63
  } else if (sh > -64) {
    const int k = -sh;
    const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
    a = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  } else {
    a = 0;
  }
  return (b >> 63) ? -(long long)a : (long long)a;
}

__device__ __forceinline__ double from_fixed(long long v) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(a);
  const unsigned long long m = a << lz;                     // top bit at 63
  unsigned long long mant = m >> 11;                        // 53 bits with the leading one
  const unsigned long long rem = m & 0x7FFull;
  int e = 63 - lz - 56;                                     // value = 1.f x 2^e
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    mant += 1;
    if (mant >> 53) {
      mant >>= 1;
      e += 1;
    }
  }
  const unsigned long long bits = sgn | ((unsigned long long)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Digits of an FP64 arena (X0 after the gather): one warp per column up to ld.
__global__ void __launch_bounds__(256) oz_slice_kernel(const PartDesc* __restrict__ parts,
                                                       const ColBlock* __restrict__ blocks, const double* __restrict__ X,
                                                       OzSlices sl) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.ld) return;
  const int64_t cbase = p.off + (int64_t)j * p.ld;
  for (int r = lane; r < p.ld; r += 32) store_digits(sl.s, cbase + r, to_fixed(X[cbase + r]));
}

// One group G_d for every upper 128x128 tile of every part, persistent (one CTA per SM,
// tiles blockIdx.x, blockIdx.x + gridDim.x, ...).  Work items are (K block, pair) with the
// pairs (a, d - a); each item loads the A tile from slice a (rows I) and the B tile from
// slice d - a (rows J) by TMA and issues four K = 16 MMAs into the tile's TMEM accumulator
// (two accumulators alternate between tiles).  The epilogue converts the integer-valued
// FP32 sums to 64-bit integers scaled to 2^-56 and adds them (group 0 stores) at (I, J) and
// mirrored at (J, I).
__global__ void __launch_bounds__(384, 1) oz_group_kernel(OzGroupArgs a) {
  constexpr int STAGES = 4;
  constexpr uint32_t STAGE_B = 2 * kTileBytes;
  constexpr int BKE = 64;  // BF16 K elements per 128-byte row
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

  if (a.mode == SQ_FORWARD) {
    if (*(volatile int32_t*)&a.st->stopped) return;
  } else {
    const int32_t stt = *(volatile int32_t*)&a.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
  }
  const int d = a.group;
  const int npairs = d + 1 < OZ_SLICES ? d + 1 : OZ_SLICES;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_B;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + STAGES * STAGE_B + 8 * (2 * STAGES + 4));
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
  auto tfull = [&](int b) { return bars + 8u * (2 * STAGES + b); };
  auto tempty = [&](int b) { return bars + 8u * (2 * STAGES + 2 + b); };
  auto tile_addr = [&](int s, int op) { return base + (uint32_t)s * STAGE_B + (uint32_t)op * kTileBytes; };
  int32_t* abort_flag = &a.st->timeout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), 8);
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
  // pair p of group d: A from slice d - p... choose a = p, b = d - p, both < OZ_SLICES
  const int a_lo = d - (OZ_SLICES - 1) > 0 ? d - (OZ_SLICES - 1) : 0;

  if (warp == 0 && lane == 0) {
    uint32_t g = 0;
    bool bad = false;
    for (int ti = blockIdx.x; ti < a.ntiles && !bad; ti += gridDim.x) {
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const int nk = (p.s + BKE - 1) / BKE;
      for (int kb = 0; kb < nk && !bad; ++kb) {
        for (int q = 0; q < npairs; ++q, ++g) {
          const int sa = a_lo + q, sbb = d - sa;
          const int s = g % STAGES;
          if (g >= STAGES && !mbar_wait(empty(s), ((g / STAGES) - 1) & 1, abort_flag)) {
            bad = true;
            break;
          }
          mbar_expect_tx(full(s), STAGE_B);
          const CUtensorMap* ma = reinterpret_cast<const CUtensorMap*>(a.maps) + (size_t)sa * a.nparts + t.part;
          const CUtensorMap* mb = reinterpret_cast<const CUtensorMap*>(a.maps) + (size_t)sbb * a.nparts + t.part;
          tma_load_2d(tile_addr(s, 0), ma, kb * BKE, t.ti * 128, full(s));
          tma_load_2d(tile_addr(s, 1), mb, kb * BKE, t.tj * 128, full(s));
        }
      }
    }
    if (bad) {
      *s_err = 1;
      const uint32_t first = g > STAGES ? g - STAGES : 0;
      for (uint32_t q = first; q < g; ++q) (void)mbar_wait(full(q % STAGES), (q / STAGES) & 1, abort_flag);
    }
  } else if (warp == 1 && lane == 0) {
    uint32_t g = 0;
    int i = 0;
    bool bad = false;
    for (int ti = blockIdx.x; ti < a.ntiles && !bad; ti += gridDim.x, ++i) {
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const int nk = (p.s + BKE - 1) / BKE;
      const int b = i & 1, u = i >> 1;
      if (u >= 1 && !mbar_wait(tempty(b), (u - 1) & 1, abort_flag)) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint32_t dt = tmem + (uint32_t)(b * 128);
      bool first = true;
      for (int kb = 0; kb < nk && !bad; ++kb) {
        for (int q = 0; q < npairs; ++q, ++g) {
          const int s = g % STAGES;
          if (!mbar_wait(full(s), (g / STAGES) & 1, abort_flag)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint64_t ad = smem_desc(tile_addr(s, 0)), bd = smem_desc(tile_addr(s, 1));
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adv = (uint64_t)((kk * 16 * 2) >> 4);
            mma<0>(dt, ad + adv, bd + adv, IDESC, first ? 0u : 1u);
            first = false;
          }
          mma_commit(empty(s));
        }
      }
      mma_commit(tfull(b));
    }
    if (bad) *s_err = 1;
  } else if (warp >= 4) {
    const int quarter = warp & 3, half = (warp - 4) >> 2;
    const int m = quarter * 32 + lane;
    // fixed point 2^-56: group d carries 2^{-7(d+2)}, i.e. a shift of 7 (6 - d)
    const int shift = 7 * (6 - d);
    int i = 0;
    for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x, ++i) {
      const int b = i & 1, u = i >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull(b), u & 1, abort_flag));
      tc_fence_after();
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      long long* Y = a.acc + p.off;
      const int64_t ld = p.ld;
      const int r = t.ti * 128 + m, c0 = t.tj * 128;
      if (ok) {
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
          const int cb = half * 2 + cc;
          const int cbase = c0 + cb * 32;
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 128 + cb * 32), v);
          long long z[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float f = __uint_as_float(v[j]);
            z[j] = shift >= 0 ? __float2ll_rn(f) * (1ll << shift) : __float2ll_rn(f * 0.0078125f);
          }
          // diagonal tiles: upper triangle (c >= r) mirrored, so the sum stays exactly symmetric
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (t.ti == t.tj && cbase + j < r) continue;
            long long* y = Y + (int64_t)(cbase + j) * ld + r;
            *y = a.first ? z[j] : *y + z[j];
          }
          if (t.ti == t.tj) {
            for (int j = 0; j < 32; ++j) {
              if (cbase + j <= r) continue;
              long long* y = Y + (int64_t)r * ld + cbase + j;
              *y = a.first ? z[j] : *y + z[j];
            }
          } else {
            longlong2* ym = reinterpret_cast<longlong2*>(Y + (int64_t)r * ld + cbase);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              longlong2 o = a.first ? make_longlong2(0, 0) : ym[q];
              o.x += z[2 * q];
              o.y += z[2 * q + 1];
              ym[q] = o;
            }
          }
        }
      } else {
        *s_err = 1;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
  if (threadIdx.x == 0 && *s_err) {
    a.st->timeout = 1;
    a.st->status = ST_TIMEOUT;
    a.st->stopped = 1;
  }
}

// Y = acc 2^-56; X_new = Y (alpha = -1) or 2 X - Y (alpha = +1) in FP64; digits of X_new
// for the next step; core traces of Y and X_new per block; the last block runs the
// step bookkeeping.  One warp per column (all columns up to ld).
__global__ void __launch_bounds__(256) oz_finalize_kernel(const PartDesc* __restrict__ parts,
                                                          const ColBlock* __restrict__ blocks,
                                                          const long long* __restrict__ acc, const double* __restrict__ xin,
                                                          double* __restrict__ xout, OzSlices sl,
                                                          double2* __restrict__ slots, StepCtl ctl, int step, int mode) {
  if (mode == SQ_FORWARD) {
    if (*(volatile int32_t*)&ctl.st->stopped) return;
  } else {
    const int32_t stt = *(volatile int32_t*)&ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&ctl.st->steps + 1;
  }
  int8_t al;
  if (mode == SQ_TAIL_FIRST) al = (ctl.traces[step - 1] <= (double)ctl.nocc) ? (int8_t)1 : (int8_t)-1;
  else if (mode == SQ_TAIL_NEXT) al = (int8_t)(-ctl.alpha[step - 1]);
  else al = ctl.alpha[step];
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  double tY = 0.0, tN = 0.0;
  if (j < p.ld) {
    const int64_t cbase = p.off + (int64_t)j * p.ld;
    for (int r = lane; r < p.ld; r += 32) {
      const int64_t e = cbase + r;
      const long long yf = acc[e];
      const long long xf = (al > 0) ? 2 * to_fixed(xin[e]) - yf : yf;
      const double xn = from_fixed(xf);
      xout[e] = xn;
      store_digits(sl.s, e, xf);
      if (r == j && j < p.c) {
        tY += from_fixed(yf);
        tN += xn;
      }
    }
  }
  const double2 sum = block_sum2(tY, tN);
  if (threadIdx.x == 0) slots[blockIdx.x] = sum;
  if (last_block_ticket(&ctl.st->counter)) {
    double u = 0.0, w = 0.0;
    for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
      u += ld_cg(&slots[k].x);
      w += ld_cg(&slots[k].y);
    }
    const double2 s2 = block_sum2(u, w);
    if (threadIdx.x == 0) {
      if (ctl.st->timeout) {
        ctl.st->status = ST_TIMEOUT;
        ctl.st->stopped = 1;
      } else if (mode == SQ_FORWARD) {
        finish_step(ctl, step, s2.y, s2.x);
      } else {
        ctl.alpha[step] = al;
        finish_tail(ctl, step, s2.y, s2.x, true);
      }
      ctl.st->counter = 0;
    }
  }
}

cudaError_t launch_oz_slice(const PartDesc* parts, const ColBlock* blocks, int nblocks, const double* X,
                            const OzSlices& sl, cudaStream_t s) {
  oz_slice_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, X, sl);
  return cudaGetLastError();
}

cudaError_t launch_oz_step(const OzGroupArgs& g0, int grid, const ColBlock* blocks, int nblocks, const double* xin,
                           double* xout, const OzSlices& sl, double2* slots, const StepCtl& ctl, int step, int mode,
                           cudaStream_t s) {
  constexpr int STAGES = 4;
  const int smem = STAGES * 2 * (int)kTileBytes + 1024 + 8 * (2 * STAGES + 4) + 16;
  cudaError_t e = cudaFuncSetAttribute(oz_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int gr = grid < g0.ntiles ? grid : g0.ntiles;
  for (int d = 0; d < OZ_SLICES; ++d) {
    OzGroupArgs a = g0;
    a.group = d;
    a.first = d == 0 ? 1 : 0;
    a.mode = mode;
    oz_group_kernel<<<gr, 384, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  oz_finalize_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(g0.parts, blocks, g0.acc, xin, xout, sl, slots, ctl,
                                                            step, mode);
  return cudaGetLastError();
}

}  // namespace gsp2
