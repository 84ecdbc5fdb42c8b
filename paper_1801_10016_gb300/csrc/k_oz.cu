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
__device__ __forceinline__ void digits_of(long long v, uint16_t (&dg)[OZ_SLICES]) {
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
    asm("cvt.rn.bf16.f32 %0, %1;\n" : "=h"(dg[t]) : "f"((float)dgt));
  }
}

__device__ __forceinline__ void store_digits(uint16_t* const* slices, int64_t e, long long v) {
  uint16_t dg[OZ_SLICES];
  digits_of(v, dg);
#pragma unroll
  for (int t = 0; t < OZ_SLICES; ++t) slices[t][e] = dg[t];
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

// An integer-valued FP32 number (|f| < 2^31) times 2^shift as a 64-bit integer, with integer
// instructions only (a 64-bit conversion would run on the FP64 pipe).
__device__ __forceinline__ long long fint_shl(float f, int shift) {
  const uint32_t b = __float_as_uint(f);
  const int ex = (int)((b >> 23) & 0xFF) - 127;  // f = 1.m 2^ex
  if (ex < 0) return 0;                          // f == 0 (|f| >= 1 otherwise)
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 23 + shift;
  const long long a = sh >= 0 ? (m << sh) : (m >> (-sh));  // exact: f is an integer, shift >= 0
  return (b >> 31) ? -a : a;
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

// Digits of an FP64 arena (X0 after the gather, or the converted iterate before an FP64
// tail): one warp per column up to ld.
// The digits go to the buffer of the current step count's parity (the buffer the next
// step reads).
__global__ void __launch_bounds__(256) oz_slice_kernel(const PartDesc* __restrict__ parts,
                                                       const ColBlock* __restrict__ blocks, const double* __restrict__ X,
                                                       OzSlices d0, OzSlices d1, const DevState* st) {
  const OzSlices& sl = (st->steps & 1) ? d1 : d0;
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.ld) return;
  const int64_t cbase = p.off + (int64_t)j * p.ld;
  for (int r = lane; r < p.ld; r += 32) store_digits(sl.s, cbase + r, to_fixed(X[cbase + r]));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// One FP64-accurate purification step for every part, in one persistent launch (one CTA
// per SM walks the upper 128x128 tiles blockIdx.x, blockIdx.x + gridDim.x, ...).
//
// For each tile, the digit groups d = 0 .. T-1 are computed one after the other; a unit
// (tile, d) is the K loop over the pairs (a, d - a), each item loading the A tile from digit
// a (rows I) and the B tile from digit d - a (rows J) by TMA into a ring of stages, with
// four K = 16 BF16 MMAs per item into one of two FP32 TMEM accumulators (columns 0-255,
// alternating between units so the drain of one unit overlaps the next unit's MMAs).  The
// epilogue warps turn each unit's integer-valued sums into 64-bit fixed point (2^-56) and
// add them into a 64-bit accumulator that lives in TMEM columns 256-511 (low and high
// words).  After the last group they form X_new = Y or 2X - Y, write the FP64 master copy
// and the digits of X_new (into the other digit buffer) at (I, J) and mirrored at (J, I)
// (diagonal tiles from their upper triangle), and add the core traces; the last block runs
// the step bookkeeping.
//
// 12 warps: warp 0 lane 0 TMA, warp 1 TMEM owner and MMA issuer, warps 4..11 epilogue
// (warp w: TMEM lanes 32 (w % 4) .. + 31, column half (w - 4) / 4).
__global__ void __launch_bounds__(384, 1) oz_step_kernel(OzStepArgs a) {
  constexpr int STAGES = 6;
  constexpr uint32_t STAGE_B = 2 * kTileBytes;
  constexpr int BKE = 64;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
  constexpr int T = OZ_SLICES;
  constexpr uint32_t ACC_LO = 256, ACC_HI = 384;  // TMEM columns of the 64-bit accumulator

  int step = a.step;
  if (a.mode == SQ_FORWARD) {
    if (*(volatile int32_t*)&a.ctl.st->stopped) return;
  } else {
    const int32_t stt = *(volatile int32_t*)&a.ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&a.ctl.st->steps + 1;
  }
  const int dbi = (step - 1) & 1, dbo = step & 1;  // digit buffers read / written

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + STAGES * STAGE_B;
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
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(a.maps) + (size_t)dbi * T * a.nparts;

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
      const PartDesc p = a.parts[t.part];
      const int nk = (p.s + BKE - 1) / BKE;
      for (int d = 0; d < T && !bad; ++d) {
        for (int kb = 0; kb < nk && !bad; ++kb) {
          for (int q = 0; q <= d; ++q, ++g) {
            const int s = g % STAGES;
            if (g >= STAGES && !mbar_wait(empty(s), ((g / STAGES) - 1) & 1, abort_flag)) {
              bad = true;
              break;
            }
            mbar_expect_tx(full(s), STAGE_B);
            tma_load_2d(tile_addr(s, 0), maps + (size_t)q * a.nparts + t.part, kb * BKE, t.ti * 128, full(s));
            tma_load_2d(tile_addr(s, 1), maps + (size_t)(d - q) * a.nparts + t.part, kb * BKE, t.tj * 128, full(s));
          }
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
    int i = 0;  // unit counter (tile, group)
    bool bad = false;
    for (int ti = blockIdx.x; ti < a.ntiles && !bad; ti += gridDim.x) {
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const int nk = (p.s + BKE - 1) / BKE;
      for (int d = 0; d < T && !bad; ++d, ++i) {
        const int b = i & 1, u = i >> 1;
        if (u >= 1 && !mbar_wait(tempty(b), (u - 1) & 1, abort_flag)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * 128);
        bool first = true;
        for (int kb = 0; kb < nk && !bad; ++kb) {
          for (int q = 0; q <= d; ++q, ++g) {
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
    }
    if (bad) *s_err = 1;
  } else if (warp >= 4) {
    const int quarter = warp & 3, half = (warp - 4) >> 2;
    const int m = quarter * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    int8_t alf;
    if (a.mode == SQ_TAIL_FIRST) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
    else if (a.mode == SQ_TAIL_NEXT) alf = (int8_t)(-a.ctl.alpha[step - 1]);
    else alf = a.ctl.alpha[step];
    int i = 0;
    for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const int64_t ld = p.ld;
      const int r = t.ti * 128 + m, c0 = t.tj * 128;
      const bool diag = t.slot >= 0;
      double tY = 0.0, tN = 0.0;
      bool okall = true;
      for (int d = 0; d < T; ++d, ++i) {
        const int b = i & 1, u = i >> 1;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull(b), u & 1, abort_flag));
        tc_fence_after();
        okall = okall && ok;
        const int shift = 7 * (6 - d) + 7 * (7 - T);  // 2^{-7(d+2)} in units of 2^-56
#pragma unroll 1
        for (int cc = 0; cc < 2 && ok; ++cc) {
          const int cb = half * 2 + cc;
          uint32_t v[32], lo[32], hi[32];
          tmem_ld32(tmem + lane_off + (uint32_t)(b * 128 + cb * 32), v);
          if (d > 0) {
            tmem_ld32(tmem + lane_off + ACC_LO + (uint32_t)(cb * 32), lo);
            tmem_ld32(tmem + lane_off + ACC_HI + (uint32_t)(cb * 32), hi);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            long long z = fint_shl(__uint_as_float(v[j]), shift);
            if (d > 0) z += (long long)(((unsigned long long)hi[j] << 32) | lo[j]);
            lo[j] = (uint32_t)((unsigned long long)z & 0xFFFFFFFFull);
            hi[j] = (uint32_t)((unsigned long long)z >> 32);
          }
          if (d < T - 1) {
            tmem_st32(tmem + lane_off + ACC_LO + (uint32_t)(cb * 32), lo);
            tmem_st32(tmem + lane_off + ACC_HI + (uint32_t)(cb * 32), hi);
          } else {
            // final pass of the tile: X_new on the 2^-56 grid, FP64 master, digits, traces;
            // column writes are coalesced across the warp, the mirrored row segment of each
            // thread goes out in groups of 8 as 16-byte vectors
            const int cbase = c0 + cb * 32;
            const bool offd = t.ti != t.tj;
#pragma unroll
            for (int sub = 0; sub < 4; ++sub) {
              double xn8[8];
              uint16_t dg8[8][OZ_SLICES];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int j = sub * 8 + u;
                const int c = cbase + j;
                const long long yf = (long long)(((unsigned long long)hi[j] << 32) | lo[j]);
                const int64_t e = (int64_t)c * ld + r;
                const bool upper = offd || c >= r;  // diagonal tiles: upper triangle only
                const long long xf = (alf > 0 && upper) ? 2 * to_fixed(a.xin[p.off + e]) - yf : yf;
                xn8[u] = from_fixed(xf);
                digits_of(xf, dg8[u]);
                if (upper) {
                  a.xout[p.off + e] = xn8[u];
#pragma unroll
                  for (int q = 0; q < OZ_SLICES; ++q) a.digits[dbo].s[q][p.off + e] = dg8[u][q];
                  if (c == r && diag && r < p.c) {
                    tY += from_fixed(yf);
                    tN += xn8[u];
                  }
                }
              }
              const int64_t em = p.off + (int64_t)r * ld + cbase + sub * 8;
              if (offd) {
                double2* xm = reinterpret_cast<double2*>(a.xout + em);
#pragma unroll
                for (int u = 0; u < 4; ++u) xm[u] = make_double2(xn8[2 * u], xn8[2 * u + 1]);
#pragma unroll
                for (int q = 0; q < OZ_SLICES; ++q) {
                  uint4 pk;
                  pk.x = (uint32_t)dg8[0][q] | ((uint32_t)dg8[1][q] << 16);
                  pk.y = (uint32_t)dg8[2][q] | ((uint32_t)dg8[3][q] << 16);
                  pk.z = (uint32_t)dg8[4][q] | ((uint32_t)dg8[5][q] << 16);
                  pk.w = (uint32_t)dg8[6][q] | ((uint32_t)dg8[7][q] << 16);
                  *reinterpret_cast<uint4*>(a.digits[dbo].s[q] + em) = pk;
                }
              } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  if (cbase + sub * 8 + u <= r) continue;
                  a.xout[em + u] = xn8[u];
#pragma unroll
                  for (int q = 0; q < OZ_SLICES; ++q) a.digits[dbo].s[q][em + u] = dg8[u][q];
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty(b));
      }
      if (!okall) *s_err = 1;
      if (diag) {
        tY = warp_sum(tY);
        tN = warp_sum(tN);
        if (lane == 0) red[warp - 4] = make_double2(tY, tN);
        asm volatile("bar.sync 1, 256;\n" ::: "memory");
        if (warp == 4 && lane == 0) {
          double2 acc = make_double2(0.0, 0.0);
          for (int w = 0; w < 8; ++w) {
            acc.x += red[w].x;
            acc.y += red[w].y;
          }
          a.slots[t.slot] = acc;
        }
        asm volatile("bar.sync 1, 256;\n" ::: "memory");
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
      } else if (a.mode == SQ_FORWARD) {
        finish_step(a.ctl, step, sum.y, sum.x);
      } else {
        int8_t alf;
        if (a.mode == SQ_TAIL_FIRST) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
        else alf = (int8_t)(-a.ctl.alpha[step - 1]);
        a.ctl.alpha[step] = alf;
        finish_tail(a.ctl, step, sum.y, sum.x, true);
      }
      a.ctl.st->counter = 0;
    }
  }
}

cudaError_t launch_oz_slice(const PartDesc* parts, const ColBlock* blocks, int nblocks, const double* X,
                            const OzSlices* digits, const DevState* st, cudaStream_t s) {
  oz_slice_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, X, digits[0], digits[1], st);
  return cudaGetLastError();
}

cudaError_t launch_oz_step(const OzStepArgs& a, int grid, cudaStream_t s) {
  constexpr int STAGES = 6;
  const int smem = STAGES * 2 * (int)kTileBytes + 1024 + 8 * (2 * STAGES + 4) + 16 + 8 * 16;
  cudaError_t e = cudaFuncSetAttribute(oz_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int gr = grid < a.ntiles ? grid : a.ntiles;
  oz_step_kernel<<<gr, 384, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gsp2
