// FP64-accurate purification steps on the BF16 tensor cores (sm_103a).
//
// GB300 runs FP64 at 1/1800 of its BF16 rate, so the FP64 product X X is rebuilt from
// exact BF16 products, in the spirit of the Ozaki splitting (Ozaki, Ogita, Oishi and
// Rump, 2012).  With T = OZ_SLICES digits:
//
//   every entry of X (|x| <= 1: the spectrum of X stays in [0, 1]) is written in base 2^7
//   with rounded signed digits, x = sum_{t<T} S_t 2^{-7(t+1)} + r, |S_0| <= 2^7 |x| + 1,
//   |S_t| <= 2^6 (t >= 1), |r| <= 2^{-7T-1} (+ 2^-57 from the fixed point); every S_t is an
//   integer of at most 8 bits, stored in BF16 as S_t 2^{-7t} (still exact) so that the
//   product of digits a and b carries the factor 2^{-7(a+b)} of its group;
//
//   X X = sum_{d<T} 2^{-7(d+2)} G_d + (terms below 2^{-7(T+2)}), G_d = sum_{a+b=d} S_a S_b.
//
// Each 2^{-7d} G_d is a sum of such products accumulated in FP32 in TMEM.  Because
// ||X||_2 <= 1, sum_k |x_ik x_kj| <= 1 bounds G_0; the groups up to d = 4 add products of
// lower digits, which behave like independent values except on the diagonal (sums of
// squares, about K 2^10.4), and stay below 2^24 (in units of their own scale) for K up to
// 4096, so they are exact; later groups carry a rounding of 2^-24 relative on a value
// scaled by 2^{-49} or less.  G_0 and G_1 share one
// accumulator, G_0 + 2^-7 G_1: its terms are multiples of 2^-7 whose magnitudes sum to at
// most 2^14 + 3 2^7 (sum_k |x_ik| + |x_kj|) / 2 + 2 K (with sum_k |x_ik| <= sqrt(K)), below
// 2^16 for K <= 4096, so it is exact as well.  The groups are added as integers into a
// 64-bit fixed-point accumulator (resolution 2^-56), and a final elementwise pass forms
// X_new = Y or 2X - Y on that grid (the master copy of the iterate stays in this fixed
// point), the core traces in FP64, and the digits of X_new for the next step by integer
// arithmetic.  With T = 7 (28 BF16 products per tile) the digits hold x to 2^-49 and the
// dropped products are of order 2^-63 K 2^12; the error of Y is about 1e-13, far below the
// 1e-10 parity of the FP64 path.
//
// The adjoint step Xbar <- Xbar X + X Xbar (or 2 Xbar minus that) runs on the same
// machinery: an upper tile (I, J) of Xbar X + X Xbar is one product over K = 2s, rows I of
// [Xbar | X] times columns J of [X ; Xbar], both symmetric and kept as upper tiles.  Xbar
// has no a-priori bound, so its digits hold Xbar / 2^sig with one power-of-two scale per
// part, chosen from the largest row 2-norm of Xbar so that every row of Xbar / 2^sig has
// 2-norm <= 1/2.  With ||X||_2 <= 1, Cauchy-Schwarz gives
// sum_k |xbar_ik x_kj| + |x_ik xbar_kj| <= 1/2 + 1/2, the bound the forward step rests on,
// so the digit groups stay exact in the same way and the result carries an error of
// order 2^-49 2^sig.
#include <cuda.h>

#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"
#include "tc_ptx.cuh"

namespace gsp2 {

// Digits of a value held in 64-bit fixed point v = x 2^56 (|x| < 1.5): rounded to
// w = x 2^{7T}, then written as balanced base-2^7 digits, S_t in [-64, 63] for t >= 1 and
// the rest in S_0 (|S_0| <= 2^7 + 1 for |x| <= 1), w = sum_t S_t 2^{7(T-1-t)} exactly.
// The balanced digits of w are the plain base-2^7 digits of w + 64 (1 + 2^7 + ... +
// 2^{7(T-2)}) less 64, so each is one shift-and-mask; the small integer becomes exact BF16
// bits through the FP32 magic-number form.  Digit t is stored as S_t 2^{-7t} (exact: a
// power-of-two scale of an integer of at most 8 bits): the float 2^{23-7t} + u 2^{-7t}
// less (2^23 + 64) 2^{-7t}, one OR and one exact subtraction, so that the product of digits
// a and b lands at 2^{-7(a+b)} and groups can share an accumulator at their own scale.
// Returned are the FP32 bit patterns whose upper halves are the BF16 digits (S_t weighs
// 2^{-7(t+1)} in x, so every stored digit S_t 2^{-7t} weighs 2^-7).
__device__ __forceinline__ void digit_words(long long v, uint32_t (&fw)[OZ_SLICES]) {
  constexpr int drop = 56 - 7 * OZ_SLICES;
  constexpr long long bias = 64ll * (((1ll << (7 * (OZ_SLICES - 1))) - 1) / 127);
  const long long w = (drop > 0 ? ((v + (1ll << (drop - 1))) >> drop) : v) + bias;
#pragma unroll
  for (int t = OZ_SLICES - 1; t >= 1; --t) {
    const uint32_t u = (uint32_t)(w >> (7 * (OZ_SLICES - 1 - t))) & 127u;
    const uint32_t e = (uint32_t)(150 - 7 * t) << 23;  // exponent field of 2^{23-7t}
    fw[t] = __float_as_uint(__fsub_rn(__uint_as_float(e | u), __uint_as_float(e | 64u)));  // (2^23 + 64) 2^{-7t}
  }
  const int s0 = (int)(w >> (7 * (OZ_SLICES - 1)));  // |s0| < 256
  fw[0] = __float_as_uint(__fsub_rn(__uint_as_float(0x4B000000u | (uint32_t)(s0 + 256)), 8388864.0f));
}

// The digits of four consecutive elements e .. e + 3 (e a multiple of 4), one 8-byte store
// per digit array (a warp's lanes on consecutive groups of four write 256 B per store).
__device__ __forceinline__ void store_digits4(uint16_t* const* slices, int64_t e, const long long (&v)[4]) {
  uint32_t fw[4][OZ_SLICES];
#pragma unroll
  for (int i = 0; i < 4; ++i) digit_words(v[i], fw[i]);
#pragma unroll
  for (int t = 0; t < OZ_SLICES; ++t) {
    uint2 pk;  // upper halves of two words per 32 bits
    pk.x = __byte_perm(fw[0][t], fw[1][t], 0x7632);
    pk.y = __byte_perm(fw[2][t], fw[3][t], 0x7632);
    *reinterpret_cast<uint2*>(slices[t] + e) = pk;
  }
}

// Start of the emulated FP64 tail of a low-precision run: the last FP32 iterate (found on the
// device from the step count) converted to the fixed-point master and written as digits, in one pass
// over the rows on or above each column's diagonal block, the only ones the emulated steps
// read (and the scatter, which reads the upper tiles).  One warp per column up to ld.
__global__ void __launch_bounds__(256) oz_convert_slice_kernel(const PartDesc* __restrict__ parts,
                                                               const ColBlock* __restrict__ blocks,
                                                               const float* const* __restrict__ master_of_step,
                                                               double* __restrict__ X, OzSlices d0, OzSlices d1,
                                                               const DevState* st) {
  long long* __restrict__ xq = reinterpret_cast<long long*>(X);
  const int n = st->steps;
  const OzSlices& sl = (n & 1) ? d1 : d0;
  const float* __restrict__ in = master_of_step[n];
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.ld) return;
  const int rows = min(p.ld, (j / 128 + 1) * 128);
  const int64_t cbase = p.off + (int64_t)j * p.ld;
  for (int r = 4 * lane; r < rows; r += 128) {  // rows and cbase are multiples of 128
    const float4 f = *reinterpret_cast<const float4*>(in + cbase + r);
    const double x[4] = {(double)f.x, (double)f.y, (double)f.z, (double)f.w};
    long long v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = to_fixed(x[i]);
    longlong2* xo = reinterpret_cast<longlong2*>(xq + cbase + r);
    xo[0] = make_longlong2(v[0], v[1]);
    xo[1] = make_longlong2(v[2], v[3]);
    store_digits4(sl.s, cbase + r, v);
  }
}

// Gather of the emulated path: Eq. 1 and the digits of X0 in one pass.  One warp per column
// j < ld assembles the rows of column j of X0 on or above its diagonal block, the only ones
// the emulated steps read (zeros, then the stored entries of row S_j of H that fall there,
// at the local indices of the plan's table (locate_kernel), with the values of Eq. 1 from
// x0_values_kernel, each stored in the 64-bit
// fixed point x 2^56 of the emulated steps' master), then reads them back from L1/L2 and
// writes their digits, coalesced (rows outside the part are zero).  Blocks store
// the core-diagonal sum of their columns; the last block forms T_0 and takes the first
// branch.
__global__ void __launch_bounds__(32 * COLS_PER_BLOCK) oz_gather_kernel(
    const PartDesc* __restrict__ parts, const ColBlock* __restrict__ blocks, const int32_t* __restrict__ Sall,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ loc, const int64_t* __restrict__ locptr,
    const double* __restrict__ x0, double* __restrict__ arena, OzSlices dig, double* __restrict__ slots,
    StepCtl ctl) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = b.j0 + w;
  const int32_t* S = Sall + p.soff;
  long long* col = reinterpret_cast<long long*>(arena) + p.off + (int64_t)j * p.ld;
  double tr = 0.0;
  if (j < p.ld) {
    const int rend = min(p.ld, (j / 128 + 1) * 128);
    for (int r = lane; r < rend; r += 32) col[r] = 0ll;
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
          col[a] = to_fixed(x);
          if (a == j && j < p.c) tr = x;
        }
      }
    }
    __syncwarp();  // the lanes' stores to the column are visible to the whole warp
    const int64_t cbase = p.off + (int64_t)j * p.ld;
    for (int r = 4 * lane; r < rend; r += 128) {  // rend and cbase are multiples of 128
      long long v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = col[r + i];
      store_digits4(dig.s, cbase + r, v);
    }
  }
  const double2 t = block_sum2(tr, 0.0);
  if (threadIdx.x == 0) slots[blockIdx.x] = t.x;
  if (last_block_ticket(&ctl.st->counter)) {
    double a = 0.0;
    for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) a += ld_cg(&slots[k]);
    const double2 acc = block_sum2(a, 0.0);
    if (threadIdx.x == 0) {
      if (ctl.st->nonfinite) ctl.st->status = ST_NONFINITE;
      finish_step(ctl, 0, acc.x, 0.0);
      ctl.st->counter = 0;
    }
  }
}

// The adjoint's operands.  `after` names the reverse step just run (0: the seed), whose
// Xbar lies in buffer (n - after + 1) & 1 of the pair (x0, x1); kernels for a step that was
// not run (after > n: the forward stopped earlier) return at once.

// Squared row 2-norms of the symmetric Xbar held in its upper 128-tiles (the seed; the
// reverse steps sum theirs in their epilogue), FP64, added into
// norm[soff + r] for rows r < s: the column sums of an upper tile (I, J) give the entries
// of rows J within block I (a diagonal tile holds its whole block), and the row sums of an
// off-diagonal tile the entries of rows I within block J.  One CTA per tile.
__global__ void __launch_bounds__(256) oz_norm_kernel(const PartDesc* __restrict__ parts,
                                                      const Tile* __restrict__ tiles, const double* xb0,
                                                      const double* xb1, int after, double* __restrict__ norm,
                                                      const DevState* st) {
  const int n = *(volatile const int32_t*)&st->steps;
  if (after > n) return;
  const double* X = (after > 0 && ((n - after + 1) & 1)) ? xb1 : xb0;
  const Tile t = tiles[blockIdx.x];
  const PartDesc p = parts[t.part];
  const double* x = X + p.off;
  const int64_t ld = p.ld;
  const int r0 = t.ti * 128, c0 = t.tj * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < 16; ++q) {  // warp w: columns c0 + 16 w .. + 15, lanes over the rows
    const int c = c0 + warp * 16 + q;
    if (c >= p.s) break;
    double v = 0.0;
    for (int i = lane; i < 128; i += 32) {
      const int r = r0 + i;
      if (r < p.s) {
        const double d = x[(int64_t)c * ld + r];
        v = fma(d, d, v);
      }
    }
    v = warp_sum(v);
    if (lane == 0) atomicAdd(&norm[p.soff + c], v);
  }
  if (t.ti != t.tj) {  // thread: row r0 + (tid % 128), half of the tile's columns
    const int r = r0 + (threadIdx.x & 127), h = threadIdx.x >> 7;
    if (r < p.s) {
      double v = 0.0;
      for (int q = 0; q < 64; ++q) {
        const int c = c0 + h * 64 + q;
        if (c >= p.s) break;
        const double d = x[(int64_t)c * ld + r];
        v = fma(d, d, v);
      }
      atomicAdd(&norm[p.soff + r], v);
    }
  }
}

// Scale of each part's Xbar digits: the smallest sig with 2^sig >= 2 max_r ||xbar_r||_2
// (with a relative margin of 2^-20 over the rounding of the FP64 sums), 0 for a zero Xbar,
// OZ_SIG_NONFINITE where a row norm is NaN or Inf.  Clears the norms for the next step.
// One CTA per part.
__global__ void __launch_bounds__(256) oz_scale_kernel(const PartDesc* __restrict__ parts, int after,
                                                       double* __restrict__ norm, int32_t* __restrict__ sig,
                                                       const DevState* st) {
  const int n = *(volatile const int32_t*)&st->steps;
  if (after > n) return;
  const PartDesc p = parts[blockIdx.x];
  __shared__ double smax[8];
  double m = 0.0;
  int bad = 0;
  for (int r = threadIdx.x; r < p.s; r += blockDim.x) {
    const double v = norm[p.soff + r];
    norm[p.soff + r] = 0.0;
    if (!(v <= 1.7976931348623157e308)) bad = 1;  // NaN or Inf
    else m = fmax(m, v);
  }
  bad = __syncthreads_or(bad);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, smax[w]);
    int e = 0;
    if (bad) e = OZ_SIG_NONFINITE;
    else if (m > 0.0) (void)frexp(2.0 * sqrt(m) * (1.0 + 9.5367431640625e-07), &e);  // 2^(e-1) <= v < 2^e
    sig[blockIdx.x] = e;
  }
}

// Digits of the upper 128-tiles of a symmetric arena, of x / 2^sig[part] from FP64 (an
// adjoint's Xbar), or, with sig NULL, of a forward iterate held in the 64-bit fixed point
// x 2^56, into `out`; entries outside the part (rows or columns >= s) get zero digits.
// One warp per column up to ld.  Skipped where need > n (an iterate the adjoint does not
// reach) or where `after` names a reverse step that was not run.
__global__ void __launch_bounds__(256) oz_digits_kernel(const PartDesc* __restrict__ parts,
                                                        const ColBlock* __restrict__ blocks, const double* x0,
                                                        const double* x1, int after, int need, OzSlices out,
                                                        const int32_t* __restrict__ sig, const DevState* st) {
  const int n = *(volatile const int32_t*)&st->steps;
  if (need > n || after > n) return;
  const double* X = (after > 0 && ((n - after + 1) & 1)) ? x1 : x0;
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.ld) return;
  const int sg = sig ? sig[b.part] : 0;
  const int rend = min(p.ld, (j / 128 + 1) * 128);
  const int64_t cbase = p.off + (int64_t)j * p.ld;
  for (int r = 4 * lane; r < rend; r += 128) {  // rend and cbase are multiples of 128
    long long v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      v[i] = (r + i >= p.s || j >= p.s || sg == OZ_SIG_NONFINITE) ? 0ll
             : sig ? to_fixed(X[cbase + r + i], sg)
                   : reinterpret_cast<const long long*>(X)[cbase + r + i];
    store_digits4(out.s, cbase + r, v);
  }
}

// One FP64-accurate purification step for every part, in one persistent launch (one CTA
// per SM walks the upper 128x128 tiles: blockIdx.x, then the ones it claims from a counter,
// or blockIdx.x + gridDim.x, ... in the static deal).
//
// The T(T+1)/2 digit products of a tile need an FP32 accumulator per group d = a + b
// (128 TMEM columns each; G_0 and G_1 share one), more than the 512 columns of an SM, so a
// tile takes two passes over K: first the high groups d >= OZ_SPLIT (all seven digits; 22
// of the 28 products, columns 0-511), then the low groups d < OZ_SPLIT (digits below
// OZ_SPLIT, columns 0-255).  A stage of the TMA ring holds one K = OZ_BK slice of every
// digit the pass needs, for rows I (A) and rows J (B; diagonal tiles reuse A), so each
// distinct digit tile is loaded once per slice and feeds all its products (one K = 16 BF16
// MMA each).  The epilogue warps turn the high groups' sums into 64-bit fixed point (2^-56)
// and park them in TMEM columns 256-511, which the low pass leaves alone; after the low
// pass they add the low groups, hand all 512 columns back and keep the tile's sums in a
// per-CTA scratch tile (L2-resident) for the final pass, which forms X_new = Y or 2X - Y,
// writes the master copy (64-bit fixed point) and the digits of X_new (into the other
// digit buffer) at (I, J) and mirrored at (J, I) (diagonal tiles from their upper
// triangle), and adds the core traces, while the MMAs of the next tile's high pass run.  The new
// iterate is written with evict-first stores: the next step reads it after this launch,
// and keeping it out of L2 leaves room for the digit panels the running tiles share.  The last block
// runs the step bookkeeping.
//
// 20 warps: warp 0 lane 0 TMA, warp 1 TMEM owner and MMA issuer, warps 4..19 epilogue
// (warp w: TMEM lanes 32 (w % 4) .. + 31, columns 32 ((w - 4) / 4) .. + 31 of each group,
// in two chunks of 16), sized so that four epilogue warps per scheduler hide latency.
constexpr int OZ_STAGES = 2;
constexpr uint32_t OZ_DTILE = 128u * OZ_BK * 2u;                 // one digit tile: 128 rows x 64 B
constexpr uint32_t OZ_STAGE_B = 2u * OZ_SLICES * OZ_DTILE;       // all A and B digit tiles
constexpr int OZ_EPI_WARPS = 16;                                 // 4 per TMEM lane quarter
constexpr int OZ_THREADS = 32 * (4 + OZ_EPI_WARPS);
constexpr int OZ_RING = 4;  // dynamic schedule: tiles claimed ahead of the MMA and epilogue warps
constexpr int OZ_SMEM = OZ_STAGES * (int)OZ_STAGE_B + 1024 + 8 * (2 * OZ_STAGES + 4) + 16 + 16 * OZ_EPI_WARPS +
                        8 * 2 * OZ_RING + 4 * OZ_RING;
static_assert(OZ_SLICES - OZ_SPLIT <= 4 && OZ_SPLIT <= 4, "groups of one pass must fit in 512 TMEM columns");
static_assert(OZ_SMEM <= 232448, "shared memory of the emulated step");

// K slices per stage: as many as the stage's 2 T tile slots hold (a slice needs nd digit tiles
// of A, and as many of B unless the tile is diagonal), at most one 128-block of K, a power of 2
// so that the slices of a stage never cross a 128-block.
__host__ __device__ constexpr int oz_slices_per_stage(int nd, bool diag) {
  const int fit = (2 * OZ_SLICES) / ((diag ? 1 : 2) * nd), cap = 128 / OZ_BK;
  const int m = fit < cap ? fit : cap;
  return m >= 4 ? 4 : (m >= 2 ? 2 : 1);
}
static_assert(oz_slices_per_stage(OZ_SLICES, false) >= 1, "a high-pass slice fits a stage");

// Columns of tile column block tj that an MMA must cover: those inside the part, rounded up
// to 16 (N of an M = 128 MMA is a multiple of 16); the rest of the block is zero padding.
__host__ __device__ constexpr int oz_tile_cols(int s, int tj) {
  return s - tj * 128 >= 128 ? 128 : ((s - tj * 128 + 15) & ~15);
}

// Accumulator of group d: the high pass's groups 5, 6, 3, 4 in columns 0-127, 128-255,
// 256-383, 384-511; the low pass's G_0 + 2^-7 G_1 in columns 0-127 and G_2 in 128-255, so the
// low pass can start once groups 5 and 6 are read, and columns 256-511 hold the high pass's
// 64-bit sums (low and high words) until the low pass is drained.
static_assert(OZ_SPLIT == 3 && OZ_SLICES - OZ_SPLIT == 4, "the TMEM plan of the emulated step");
constexpr uint32_t OZ_PARK_LO = 256, OZ_PARK_HI = 384;
__host__ __device__ constexpr uint32_t oz_group_col(int d) {
  return (uint32_t)(d >= OZ_SPLIT ? (d >= 5 ? 128 * (d - 5) : 256 + 128 * (d - 3)) : (d <= 1 ? 0 : 128));
}

// The MMAs of one stage for the groups d0 <= d < d1, fully unrolled: every pair (q, d - q)
// of a group into the group's accumulator, descriptors formed by adding compile-time
// offsets to the stage's base descriptors (the 14-bit address field cannot carry: shared
// addresses stay below 2^18).  The products are issued A digit by A digit: the products of
// A digit q (one per group d >= q) follow one another and share their A operand through the
// collector buffer, so each A digit tile is read from shared memory once per K = 16 slice
// instead of once per product (the MMAs' shared-memory reads, A and B, set the pace of the
// tensor pipe otherwise).  Every accumulator's first product is the one with q = 0 (for the
// shared G_0 + 2^-7 G_1, the product (0, 0)).
template <int D0, int D1>
__device__ __forceinline__ void oz_issue_stage(uint32_t tmem, uint64_t da, uint64_t db, uint32_t adv_a,
                                               uint32_t adv_b, uint32_t idesc, bool first_k) {
  constexpr uint64_t step = OZ_DTILE >> 4;
#pragma unroll
  for (int kk = 0; kk < OZ_BK / 16; ++kk) {  // K = 16 slices of the stage
#pragma unroll
    for (int q = 0; q < D1; ++q) {
      const int dlo = q > D0 ? q : D0;  // groups holding a product of A digit q
#pragma unroll
      for (int d = dlo; d < D1; ++d) {
        const int op = (D1 - dlo == 1) ? 0 : (d == dlo ? 1 : (d == D1 - 1 ? 3 : 2));
        // the first product into each accumulator is (0, d) of its lowest group
        const bool opens = q == 0 && !(D0 == 0 && d == 1);
        mma_f16_col(op, tmem + oz_group_col(d), da + (uint64_t)q * step + (uint64_t)(adv_a * kk),
                    db + (uint64_t)(d - q) * step + (uint64_t)(adv_b * kk), idesc,
                    (!opens || kk > 0 || !first_k) ? 1u : 0u);
      }
    }
  }
}

// z[j] += u[j] 2^SHIFT for one accumulator of one 16-column chunk, where u = v 2^M is the
// integer its FP32 sums v hold at the scale 2^-M: the groups d >= 3 alone (M = 7 d, SHIFT =
// 56 - 7 (d + 2)), G_2 (M = 14, SHIFT = 28), G_0 + 2^-7 G_1 (M = 7, SHIFT = 35: u = 2^7 G_0 +
// G_1).  A chunk whose integers all lie below 2^22 in magnitude is converted without the
// conversion unit: v + 1.5 2^(23 - M) is a float in [2^(23 - M), 2^(24 - M)) with spacing 2^-M,
// whose bit pattern less that of 1.5 2^(23 - M) is u, and a 32 x 32 -> 64-bit multiply-add
// (by the power of two, or on the upper word for shifts of 32 and more) accumulates it; any
// other chunk goes through the exact rounding conversion of v 2^M (|u| < 2^31).
template <int M, int SHIFT>
__device__ __forceinline__ void oz_drain_slot(uint32_t taddr, long long (&z)[16]) {
  uint32_t v[16];
  tmem_ld16(taddr, v);
  const float magic = __uint_as_float(((uint32_t)(150 - M) << 23) | 0x400000u);  // 1.5 2^(23 - M)
  const float lim = __uint_as_float((uint32_t)(149 - M) << 23);                   // 2^(22 - M)
  float mx = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fabsf(__uint_as_float(v[j])));
  if (__all_sync(0xffffffffu, mx < lim)) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int32_t g = (int32_t)(__float_as_uint(__fadd_rn(__uint_as_float(v[j]), magic)) - __float_as_uint(magic));
      if constexpr (SHIFT < 32) {
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(z[j]) : "r"(g), "r"(1 << SHIFT));
      } else {
        z[j] += (long long)((unsigned long long)((uint32_t)g << (SHIFT - 32)) << 32);
      }
    }
  } else {
    const float scale = __uint_as_float((uint32_t)(127 + M) << 23);  // 2^M
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long g = (long long)__float2int_rn(__fmul_rn(__uint_as_float(v[j]), scale));
      z[j] += (long long)((unsigned long long)g << SHIFT);
    }
  }
}

// The high pass of one chunk, in two halves: groups 5 and 6 (the columns the low pass
// reuses), then groups 3 and 4 (the columns that then hold the sums), into z.
__device__ __forceinline__ void oz_drain_high56(uint32_t taddr, long long (&z)[16]) {
  oz_drain_slot<35, 7>(taddr + oz_group_col(5), z);
  oz_drain_slot<42, 0>(taddr + oz_group_col(6), z);
}
__device__ __forceinline__ void oz_drain_high34(uint32_t taddr, long long (&z)[16]) {
  oz_drain_slot<21, 21>(taddr + oz_group_col(3), z);
  oz_drain_slot<28, 14>(taddr + oz_group_col(4), z);
}

// The low pass of one chunk: G_0 + 2^-7 G_1 and G_2 into z.
__device__ __forceinline__ void oz_drain_low(uint32_t taddr, long long (&z)[16]) {
  oz_drain_slot<7, 35>(taddr + oz_group_col(0), z);
  oz_drain_slot<14, 28>(taddr + oz_group_col(2), z);
}

// |v| 2^-56 as FP32 (integer instructions, truncated: at most 2^-23 below), for the row
// norms of the adjoint's new Xbar on its fixed-point grid.
__device__ __forceinline__ float fixed_to_f32_abs(long long v) {
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  if (a == 0) return 0.0f;
  const int lz = __clzll(a);
  const uint32_t mant = (uint32_t)((a << lz) >> 40) & 0x7FFFFFu;  // 23 bits below the leading one
  return __uint_as_float(((uint32_t)(63 - lz - 56 + 127) << 23) | mant);
}

// Sum of v[j] (j < 16) over the 32 lanes of a warp in 16 shuffles (each step exchanges half
// of the remaining columns with the partner lane); lanes 2q and 2q + 1 end with the sum of
// column `col` = 8 b4 + 4 b3 + 2 b2 + b1 (b the lane's bits).
__device__ __forceinline__ float warp_colsum16(const float (&v)[16], int lane, int& col) {
  float a8[8], a4[4], a2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    a8[j] = (h16 ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, h16 ? v[j] : v[j + 8], 16);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    a4[j] = (h8 ? a8[j + 4] : a8[j]) + __shfl_xor_sync(0xffffffffu, h8 ? a8[j] : a8[j + 4], 8);
#pragma unroll
  for (int j = 0; j < 2; ++j)
    a2[j] = (h4 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, h4 ? a4[j] : a4[j + 2], 4);
  float a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? a2[0] : a2[1], 2);
  a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  col = (h16 ? 8 : 0) + (h8 ? 4 : 0) + (h4 ? 2 : 0) + (h2 ? 1 : 0);
  return a1;
}

// ADJ: the adjoint step (see the top of the file): K runs over [Xbar | X] x [X ; Xbar],
// diagonal tiles load both operands, the epilogue forms Xbar_new in FP64 without digits
// or traces and adds its squared row norms (FP32, on the grid of the input scale); the last
// block turns them into each part's new scale.
template <bool ADJ>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_step_kernel(OzStepArgs a) {
  constexpr int T = OZ_SLICES;
  // instruction descriptor without N (bits 17..22, N / 8): FP32 accumulate, BF16 A and B, M = 128
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);

  int step = a.step;
  const bool rec = !ADJ && a.mode == SQ_RECOMPUTE;
  int n = 0;
  if (ADJ || rec) {
    // reverse step `step` exists iff step <= n; a rebuilt X_step is read iff step < n
    n = *(volatile int32_t*)&a.ctl.st->steps;
    if (ADJ ? step > n : step >= n) return;
  } else if (a.mode == SQ_FORWARD) {
    if (*(volatile int32_t*)&a.ctl.st->stopped) return;
  } else {
    const int32_t stt = *(volatile int32_t*)&a.ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&a.ctl.st->steps + 1;
  }
  // digit buffers read / written (the adjoint's sets are passed explicitly)
  const int dbi = (ADJ || rec) ? 0 : (step - 1) & 1, dbo = (ADJ || rec) ? 0 : step & 1;

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* sb = smem_raw + (base - raw);
  const uint32_t bars = base + OZ_STAGES * OZ_STAGE_B;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + OZ_STAGES * OZ_STAGE_B + 8 * (2 * OZ_STAGES + 4));
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  int* s_half = reinterpret_cast<int*>(tmem_slot + 2);  // split adjoint: halves of the tile done before
  double2* red = reinterpret_cast<double2*>(sb + OZ_STAGES * OZ_STAGE_B + 8 * (2 * OZ_STAGES + 4) + 16);
  // dynamic schedule: the producer claims each next tile from a counter in global memory and
  // passes it on through a ring (full: claimed; empty: read by the MMA thread and every
  // epilogue warp); -1 ends the walk
  const uint32_t ring_bars = smem_u32(red + OZ_EPI_WARPS);
  int* s_items = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(red + OZ_EPI_WARPS) + 8 * 2 * OZ_RING);
  auto item_full = [&](int q) { return ring_bars + 8u * q; };
  auto item_empty = [&](int q) { return ring_bars + 8u * (OZ_RING + q); };
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (OZ_STAGES + s); };
  // accumulator barriers: [0] high groups, [1] low groups
  auto afull = [&](int pass) { return bars + 8u * (2 * OZ_STAGES + pass); };
  auto aempty = [&](int pass) { return bars + 8u * (2 * OZ_STAGES + 2 + pass); };
  auto tileA = [&](int s, int q) { return base + (uint32_t)s * OZ_STAGE_B + (uint32_t)q * OZ_DTILE; };
  auto tileB = [&](int s, int q) { return base + (uint32_t)s * OZ_STAGE_B + (uint32_t)(OZ_SLICES + q) * OZ_DTILE; };
  int32_t* abort_flag = &a.ctl.st->timeout;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(a.maps) + (size_t)dbi * T * a.nparts;
  const CUtensorMap* maps_mn = reinterpret_cast<const CUtensorMap*>(a.maps_mn) + (size_t)dbi * T * a.nparts;
  const CUtensorMap* maps_b = reinterpret_cast<const CUtensorMap*>(a.maps_b);
  const CUtensorMap* maps_mn_b = reinterpret_cast<const CUtensorMap*>(a.maps_mn_b);
  // work items: the upper tiles, or (split K) each tile's two K halves
  const bool split = a.split != 0;
  const int nitems = split ? 2 * a.ntiles : a.ntiles;
  // items claimed at run time (forward, tail and reverse steps; the list order) or dealt in turn
  // (the rebuilt iterates, which may run beside reverse steps and have no last block)
  const bool dyn = a.tile_ctr != nullptr && !rec;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(afull(q), 1);
      mbar_init(aempty(q), OZ_EPI_WARPS);
    }
    for (int q = 0; q < OZ_RING; ++q) {
      mbar_init(item_full(q), 1);
      mbar_init(item_empty(q), 1 + OZ_EPI_WARPS);
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
    // dynamic: the first item is blockIdx.x, the next ones gridDim.x + the counter's count,
    // each claimed one item ahead so that the atomic's latency hides behind an item's loads
    int nxt = dyn && (int)blockIdx.x < nitems ? (int)gridDim.x + (int)atomicAdd(a.tile_ctr, 1u) : nitems;
    for (int v = 0, it = blockIdx.x; !bad; ++v, it += gridDim.x) {
      if (dyn) {
        if (v > 0) {
          it = nxt;
          if (it < nitems) nxt = (int)gridDim.x + (int)atomicAdd(a.tile_ctr, 1u);
        }
        const int q = v % OZ_RING;
        if (v >= OZ_RING && !mbar_wait(item_empty(q), ((v / OZ_RING) - 1) & 1, abort_flag)) {
          bad = true;
          break;
        }
        s_items[q] = it < nitems ? it : -1;
        mbar_arrive(item_full(q));
      }
      if (it >= nitems) break;
      const int code = split ? a.split_items[it] : it;
      const int ti = split ? code >> 1 : it, half = split ? code & 1 : -1;
      const Tile t = a.tiles[ti];
      const int sz = a.parts[t.part].s;
      const bool dg = !ADJ && t.ti == t.tj;  // X X on a diagonal tile: B is A
      for (int pass = 0; pass < 2 && !bad; ++pass) {
        const int nd = pass == 0 ? T : OZ_SPLIT;  // digits the pass multiplies
        const int sub = oz_slices_per_stage(nd, dg);
        const int nk = (sz + sub * OZ_BK - 1) / (sub * OZ_BK);
        // K stages of the item: the adjoint's halves are Xbar X and X Xbar, the forward's the
        // two halves of the stages of the pass
        const int kb0 = half < 1 ? 0 : (ADJ ? nk : (nk + 1) / 2);
        const int kb1 = ADJ ? (half == 0 ? nk : 2 * nk) : (half == 0 ? (nk + 1) / 2 : nk);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          // the adjoint's first nk stages multiply Xbar (rows I) by X (rows J), the rest X by Xbar
          const bool h2 = ADJ && kb >= nk;
          const int kq = h2 ? kb - nk : kb;
          const CUtensorMap* const mA = (ADJ && !h2) ? maps_b : maps;
          const CUtensorMap* const mmA = (ADJ && !h2) ? maps_mn_b : maps_mn;
          const CUtensorMap* const mB = h2 ? maps_b : maps;
          const CUtensorMap* const mmB = h2 ? maps_mn_b : maps_mn;
          const int s = g % OZ_STAGES;
          if (g >= OZ_STAGES && !mbar_wait(empty(s), ((g / OZ_STAGES) - 1) & 1, abort_flag)) {
            bad = true;
            break;
          }
          mbar_expect_tx(full(s), (uint32_t)(sub * (dg ? nd : 2 * nd)) * OZ_DTILE);
          // rows I over the K slice: K-major from columns I of the tiles on or above the
          // diagonal (slice block <= I's block), else MN-major from rows I of tile (I, slice);
          // the slices of one stage lie in one 128-block of K.  One request per slice and
          // operand brings all nd digit tiles (slots u nd .. u nd + nd - 1): the maps of the
          // high pass take OZ_SLICES digits per box, those of the low pass OZ_SPLIT
          const size_t at = (size_t)(nd == T ? 0 : 1) * a.nparts + t.part;
          for (int u = 0; u < sub; ++u) {
            const int k0 = (kq * sub + u) * OZ_BK;
            const int kt = k0 / 128;
            const int slot = u * nd;
            if (kt <= t.ti) {
              tma_load_3d(tileA(s, slot), mA + at, k0, t.ti * 128, 0, full(s));
            } else {
              tma_load_4d(tileA(s, slot), mmA + at, 0, k0, 2 * t.ti, 0, full(s));  // 64-row atoms x digits
            }
            if (dg) continue;
            if (kt <= t.tj) {
              tma_load_3d(tileB(s, slot), mB + at, k0, t.tj * 128, 0, full(s));
            } else {
              tma_load_4d(tileB(s, slot), mmB + at, 0, k0, 2 * t.tj, 0, full(s));
            }
          }
        }
      }
    }
    if (bad) {
      *s_err = 1;
      const uint32_t first = g > OZ_STAGES ? g - OZ_STAGES : 0;
      for (uint32_t q = first; q < g; ++q) (void)mbar_wait_own(full(q % OZ_STAGES), (q / OZ_STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    uint32_t g = 0;
    int u = 0;  // items done by this CTA
    bool bad = false;
    for (int it = blockIdx.x; !bad; it += gridDim.x, ++u) {
      if (dyn) {
        const int q = u % OZ_RING;
        if (!mbar_wait(item_full(q), (u / OZ_RING) & 1, abort_flag)) {
          bad = true;
          break;
        }
        it = s_items[q];
        mbar_arrive(item_empty(q));
        if (it < 0) break;
      }
      if (it >= nitems) break;
      const int code = split ? a.split_items[it] : it;
      const int ti = split ? code >> 1 : it, half = split ? code & 1 : -1;
      const Tile t = a.tiles[ti];
      const int sz = a.parts[t.part].s;
      const bool dg = !ADJ && t.ti == t.tj;
      for (int pass = 0; pass < 2 && !bad; ++pass) {
        const int nd = pass == 0 ? T : OZ_SPLIT;
        const int sub = oz_slices_per_stage(nd, dg);
        const int nk = (sz + sub * OZ_BK - 1) / (sub * OZ_BK);
        // K stages of the item: the adjoint's halves are Xbar X and X Xbar, the forward's the
        // two halves of the stages of the pass
        const int kb0 = half < 1 ? 0 : (ADJ ? nk : (nk + 1) / 2);
        const int kb1 = ADJ ? (half == 0 ? nk : 2 * nk) : (half == 0 ? (nk + 1) / 2 : nk);
        // the high pass reuses the columns of the previous tile's low groups, the low pass
        // those of this tile's high groups: wait until the epilogue has read them
        const bool ready = pass == 0 ? (u == 0 || mbar_wait(aempty(1), (u - 1) & 1, abort_flag))
                                     : mbar_wait(aempty(0), u & 1, abort_flag);
        if (!ready) {
          bad = true;
          break;
        }
        tc_fence_after();
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int kq = (ADJ && kb >= nk) ? kb - nk : kb;
          const int s = g % OZ_STAGES;
          if (!mbar_wait(full(s), (g / OZ_STAGES) & 1, abort_flag)) {
            bad = true;
            break;
          }
          tc_fence_after();
          // pairs (q, d - q) of every group of the pass; both digits are < d1 <= T.  Operands
          // right of the tile's own block came in MN-major (transpose bits 15 / 16); a K = 16
          // step advances 32 B in a K-major row, 2 KB (16 K values) in an MN-major tile
          const int kt = kq * sub * OZ_BK / 128;
          const bool amn = kt > t.ti, bmn = kt > t.tj;
          const uint64_t da = amn ? smem_desc_mn128(tileA(s, 0), OZ_DTILE / 2) : smem_desc_sw<2 * OZ_BK>(tileA(s, 0));
          const uint64_t db = dg ? da
                                 : (bmn ? smem_desc_mn128(tileB(s, 0), OZ_DTILE / 2)
                                        : smem_desc_sw<2 * OZ_BK>(tileB(s, 0)));
          const uint32_t adv_a = amn ? (2048u >> 4) : (32u >> 4), adv_b = bmn ? (2048u >> 4) : (32u >> 4);
          const uint32_t idesc =
              IDESC | ((uint32_t)(oz_tile_cols(sz, t.tj) >> 3) << 17) | ((amn ? 1u : 0u) << 15) | ((bmn ? 1u : 0u) << 16);
          for (int u = 0; u < sub; ++u) {  // the stage's K slices, nd tiles apart
            const uint64_t off = (uint64_t)(u * nd) * (OZ_DTILE >> 4);
            if (pass == 0) oz_issue_stage<OZ_SPLIT, T>(tmem, da + off, db + off, adv_a, adv_b, idesc, kb == kb0 && u == 0);
            else oz_issue_stage<0, OZ_SPLIT>(tmem, da + off, db + off, adv_a, adv_b, idesc, kb == kb0 && u == 0);
          }
          mma_commit(empty(s));
        }
        if (!bad) mma_commit(afull(pass));
      }
    }
    if (bad) {
      *s_err = 1;
      // MMAs already issued keep reading shared memory and writing TMEM: wait (on this
      // thread's own limit) for the last commit, which covers all of them
      if (g > 0) (void)mbar_wait_own(empty((g - 1) % OZ_STAGES), ((g - 1) / OZ_STAGES) & 1);
    }
  } else if (warp >= 4) {
    const int quarter = warp & 3, colq = (warp - 4) >> 2;
    const int m = quarter * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    long long* const cta_acc = a.acc + (size_t)blockIdx.x * (128 * 128);
    int8_t alf;
    if (ADJ || rec) alf = a.ctl.alpha[step];  // the recorded branch of step `step`
    else if (a.mode == SQ_TAIL_FIRST) alf = (a.ctl.traces[step - 1] <= (double)a.ctl.nocc) ? (int8_t)1 : (int8_t)-1;
    else if (a.mode == SQ_TAIL_NEXT) alf = (int8_t)(-a.ctl.alpha[step - 1]);
    else alf = a.ctl.alpha[step];
    // the adjoint's Xbar ping-pong: in = buffer (n - step) & 1, out = the other
    const double* xin = a.xin;
    double* xout = a.xout;
    if (ADJ && ((n - step) & 1)) {
      xin = a.xout;
      xout = const_cast<double*>(a.xin);
    }
    long long* const xq = reinterpret_cast<long long*>(xout);
    int u = 0;
    for (int it = blockIdx.x;; it += gridDim.x, ++u) {
      if (dyn) {
        const int q = u % OZ_RING;
        const bool got = __all_sync(0xffffffffu, mbar_wait(item_full(q), (u / OZ_RING) & 1, abort_flag));
        if (!got) {
          *s_err = 1;
          break;
        }
        it = s_items[q];
        __syncwarp();
        if (lane == 0) mbar_arrive(item_empty(q));
        if (it < 0) break;
      }
      if (it >= nitems) break;
      const int code = split ? a.split_items[it] : it;
      const int ti = split ? code >> 1 : it;
      // a split item's 64-bit partial goes to its own tile of split_acc, which the item that
      // finishes the tile reads; otherwise the sums wait in this CTA's scratch tile
      long long* const acc = split ? a.split_acc + (size_t)code * (128 * 128) : cta_acc;
      const Tile t = a.tiles[ti];
      const PartDesc p = a.parts[t.part];
      const int64_t ld = p.ld;
      const int r = t.ti * 128 + m, c0 = t.tj * 128;
      const bool diag = t.slot >= 0;
      const int sg = ADJ ? a.sig[t.part] : 0;  // the adjoint's sums hold (Xbar X + X Xbar) / 2^sg
      // columns the MMAs covered; the 16-column chunks beyond them lie in the part's zero
      // padding, which no step writes (the arenas are zeroed when the workspace is bound)
      const int ncols = oz_tile_cols(p.s, t.tj);
      // a diagonal tile keeps its upper triangle and mirrors it: a chunk wholly left of the
      // warp's first row (all its entries below the diagonal) is neither drained nor formed
      const int cskip = (t.ti == t.tj) ? quarter * 32 : 0;
      double tY = 0.0, tN = 0.0;
      bool ok = true;
      // the two passes: read the groups' sums (integers at their groups' scales, held
      // exactly in FP32) and add them as 64-bit integers, parked in TMEM between the passes
      // and then in the scratch tile (thread-private entries: column cl, row m); each pass
      // hands its columns back
      for (int pass = 0; pass < 2; ++pass) {
        ok = __all_sync(0xffffffffu, mbar_wait(afull(pass), u & 1, abort_flag)) && ok;
        tc_fence_after();
        // the high pass hands its columns back as soon as the warp's last chunk has read
        // groups 5 and 6, which the low pass reuses (-1: no chunk, hand back at the end)
        const int clast = (colq * 32 + 16 < ncols && colq * 32 + 32 > cskip) ? 1
                          : (colq * 32 < ncols && colq * 32 + 16 > cskip)   ? 0
                                                                            : -1;
        bool released = false;
#pragma unroll 1
        for (int cc = 0; cc < 2 && ok; ++cc) {
          const int cl = colq * 32 + cc * 16;
          if (cl >= ncols || cl + 16 <= cskip) continue;
          const uint32_t tc = tmem + lane_off + (uint32_t)cl;
          long long z[16];
          uint32_t w[16];
          if (pass == 0) {
            // the high groups' sum waits in the columns this warp has just drained (its own
            // columns of groups 3 and 4), which the low pass leaves alone
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = 0ll;
            oz_drain_high56(tc, z);
            if (cc == clast) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(aempty(0));
              released = true;
            }
            oz_drain_high34(tc, z);
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = (uint32_t)(unsigned long long)z[j];
            tmem_st16(tc + OZ_PARK_LO, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = (uint32_t)((unsigned long long)z[j] >> 32);
            tmem_st16(tc + OZ_PARK_HI, w);
          } else {
            tmem_ld16(tc + OZ_PARK_LO, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = (long long)(unsigned long long)w[j];
            tmem_ld16(tc + OZ_PARK_HI, w);
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] += (long long)((unsigned long long)w[j] << 32);
            oz_drain_low(tc, z);
            long long* zp = acc + (size_t)cl * 128 + m;
#pragma unroll
            for (int j = 0; j < 16; ++j) zp[(size_t)j * 128] = z[j];
          }
        }
        if (pass == 0) tmem_wait_st();
        if (!released) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(aempty(pass));
        }
      }
      if (!ok) *s_err = 1;
      // split K: the first half to finish leaves its partial; the second adds the first's
      // (64-bit integers: exact, so which one finishes first does not matter) and forms the tile
      const long long* other = nullptr;
      if (split) {
        __threadfence();
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * OZ_EPI_WARPS) : "memory");
        if (warp == 4 && lane == 0) {
          const unsigned int before = atomicAdd(&a.split_cnt[ti], 1u);
          if (before == 1u) a.split_cnt[ti] = 0u;  // both halves in: clear for the next launch
          *s_half = (int)before;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * OZ_EPI_WARPS) : "memory");
        if (*s_half == 0) continue;
        __threadfence();
        other = a.split_acc + (size_t)(code ^ 1) * (128 * 128);
      }
      // final pass of the tile: X_new on the 2^-56 grid, fixed-point master, digits, traces (the
      // adjoint: Xbar_new, FP64 only); column writes are coalesced across the warp.  Only
      // tiles on or above the diagonal are kept (the next step reads the rest MN-major from
      // them); a diagonal tile mirrors its upper triangle, each thread's row segment in
      // groups of 4 as 32-byte (FP64) and 8-byte (digit) vectors
      const bool offd = t.ti != t.tj;
      float rown = 0.0f;  // adjoint: squared norm of row r over this thread's upper entries
#pragma unroll 1
      for (int cc = 0; cc < 2 && ok; ++cc) {
        const int cl = colq * 32 + cc * 16;
        if (cl >= ncols || cl + 16 <= cskip) continue;
        const int cbase = c0 + cl;
        const long long* zp = acc + (size_t)cl * 128 + m;
        const long long* zo = other ? other + (size_t)cl * 128 + m : nullptr;
        float coln[16];  // adjoint: squares of the entries (r, c) for the norms of rows c
#pragma unroll
        for (int j = 0; j < 16; ++j) coln[j] = 0.0f;
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {
          // loads of the group first (xin is not written by this launch), so that they are
          // in flight together rather than each behind the previous group's stores
          // the forward iterates are kept in the fixed point itself; the adjoint's Xbar in FP64
          long long yv[4], xv[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int j = sub * 4 + w;
            yv[w] = zp[(size_t)j * 128] + (zo ? __ldcg(zo + (size_t)j * 128) : 0ll);
            xv[w] = alf > 0 ? __ldg(reinterpret_cast<const long long*>(xin) + p.off + (int64_t)(cbase + j) * ld + r)
                            : 0ll;
          }
          long long xn4[4];  // the words stored: fixed point (forward) or FP64 bits (adjoint)
          uint32_t dw4[4][OZ_SLICES];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int c = cbase + sub * 4 + w;
            const long long yf = yv[w];
            const int64_t e = (int64_t)c * ld + r;
            const bool upper = offd || c >= r;  // diagonal tiles: upper triangle only
            const long long xi = ADJ ? to_fixed(__longlong_as_double(xv[w]), sg) : xv[w];
            const long long xf = (alf > 0 && upper) ? 2 * xi - yf : yf;
            if (ADJ)
              xn4[w] = sg == OZ_SIG_NONFINITE ? 0x7FF8000000000000ll : __double_as_longlong(from_fixed(xf, sg));
            else
              xn4[w] = xf;
            if (!ADJ) digit_words(xf, dw4[w]);
            if (ADJ && upper && r < p.s && c < p.s) {
              // every stored entry (r, c) adds to the norm of row r, and of row c unless c = r
              const float f = fixed_to_f32_abs(xf);
              rown = fmaf(f, f, rown);
              if (c != r) coln[sub * 4 + w] = f * f;
            }
            if (upper) {
              __stcs(xq + p.off + e, xn4[w]);
              if (!ADJ) {
#pragma unroll
                for (int q = 0; q < OZ_SLICES; ++q)
                  __stcs(a.digits[dbo].s[q] + p.off + e, (unsigned short)(dw4[w][q] >> 16));
              }
              if (!ADJ && !rec && c == r && diag && r < p.c) {
                tY += from_fixed(yf);
                tN += from_fixed(xf);
              }
            }
          }
          const int64_t em = p.off + (int64_t)r * ld + cbase + sub * 4;
          if (!offd && cbase + sub * 4 > r) {
            // the four mirrored elements are contiguous in column r: vector stores whenever
            // all four lie right of the diagonal
            longlong2* xm = reinterpret_cast<longlong2*>(xq + em);
            __stcs(xm, make_longlong2(xn4[0], xn4[1]));
            __stcs(xm + 1, make_longlong2(xn4[2], xn4[3]));
            if (!ADJ) {
#pragma unroll
              for (int q = 0; q < OZ_SLICES; ++q) {
                uint2 pk;  // upper halves of two words per 32 bits
                pk.x = __byte_perm(dw4[0][q], dw4[1][q], 0x7632);
                pk.y = __byte_perm(dw4[2][q], dw4[3][q], 0x7632);
                __stcs(reinterpret_cast<uint2*>(a.digits[dbo].s[q] + em), pk);
              }
            }
          } else if (!offd) {
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              if (cbase + sub * 4 + w <= r) continue;
              __stcs(xq + em + w, xn4[w]);
              if (!ADJ) {
#pragma unroll
                for (int q = 0; q < OZ_SLICES; ++q)
                  __stcs(a.digits[dbo].s[q] + em + w, (unsigned short)(dw4[w][q] >> 16));
              }
            }
          }
        }
        if (ADJ) {
          int col;
          const float cs = warp_colsum16(coln, lane, col);
          if (!(lane & 1) && cbase + col < p.s && cs != 0.0f) atomicAdd(&a.normf[p.soff + cbase + col], cs);
        }
      }
      if (ADJ && ok && r < p.s && rown != 0.0f) atomicAdd(&a.normf[p.soff + r], rown);
      if (!ADJ && !rec && diag) {
        tY = warp_sum(tY);
        tN = warp_sum(tN);
        if (lane == 0) red[warp - 4] = make_double2(tY, tN);
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * OZ_EPI_WARPS) : "memory");
        if (warp == 4 && lane == 0) {
          double2 sum = make_double2(0.0, 0.0);
          for (int w = 0; w < OZ_EPI_WARPS; ++w) {
            sum.x += red[w].x;
            sum.y += red[w].y;
          }
          a.slots[t.slot] = sum;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * OZ_EPI_WARPS) : "memory");
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  if (threadIdx.x == 0 && *s_err) {
    a.ctl.st->timeout = 1;
    if (ADJ || rec) a.ctl.st->status = ST_TIMEOUT;  // no step bookkeeping follows
  }
  if (rec) return;
  if (ADJ) {
    // the last block: each part's new scale from the largest squared row norm m (on the grid
    // of the old scale sg): the smallest e with 2^e >= 2 sqrt(m) (1 + 2^-10), the margin
    // covering the truncated squares and the FP32 sums; the norms are cleared for the next step
    if (last_block_ticket(&a.ctl.st->counter)) {
      for (int k = warp; k < a.nparts; k += OZ_THREADS / 32) {
        const PartDesc p = a.parts[k];
        float mx = 0.0f;
        for (int rr = lane; rr < p.s; rr += 32) {
          float* q = a.normf + p.soff + rr;
          mx = fmaxf(mx, __ldcg(q));
          *q = 0.0f;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
          const int sg = a.sig[k];
          int e = 0;
          if (sg != OZ_SIG_NONFINITE && mx > 0.0f) {
            (void)frexpf(2.0f * sqrtf(mx) * (1.0f + 0.0009765625f), &e);
            a.sig[k] = sg + e;
          }
        }
      }
      if (threadIdx.x == 0) {
        a.ctl.st->counter = 0;
        if (dyn) *a.tile_ctr = 0u;  // every CTA has claimed its last item
      }
    }
    return;
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
      if (dyn) *a.tile_ctr = 0u;  // every CTA has claimed its last tile: ready for the next launch
    }
  }
}

cudaError_t launch_oz_convert_slice(const PartDesc* parts, const ColBlock* blocks, int nblocks,
                                    const float* const* master_of_step, double* X, const OzSlices* digits,
                                    const DevState* st, cudaStream_t s) {
  oz_convert_slice_kernel<<<nblocks, 256, 0, s>>>(parts, blocks, master_of_step, X, digits[0], digits[1], st);
  return cudaGetLastError();
}

cudaError_t launch_oz_step(const OzStepArgs& a, int grid, cudaStream_t s, bool adjoint) {
  auto kern = adjoint ? oz_step_kernel<true> : oz_step_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  if (e != cudaSuccess) return e;
  const int nitems = a.split ? 2 * a.ntiles : a.ntiles;
  int gr = grid < nitems ? grid : nitems;
  if (gr > OZ_MAX_GRID) gr = OZ_MAX_GRID;  // one scratch tile per CTA
  kern<<<gr, OZ_THREADS, OZ_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_oz_gather(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                             const int64_t* rowptr, const int32_t* loc, const int64_t* locptr, const double* x0,
                             double* arena, const OzSlices& dig, double* slots, const StepCtl& ctl, cudaStream_t s) {
  oz_gather_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, arena, dig,
                                                            slots, ctl);
  return cudaGetLastError();
}

cudaError_t launch_oz_adj_scale(const PartDesc* parts, int nparts, const Tile* tiles, int ntiles, const double* xb0,
                                const double* xb1, int after, double* norm, int32_t* sig, const DevState* st,
                                cudaStream_t s) {
  if (ntiles > 0) oz_norm_kernel<<<ntiles, 256, 0, s>>>(parts, tiles, xb0, xb1, after, norm, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_scale_kernel<<<nparts, 256, 0, s>>>(parts, after, norm, sig, st);
  return cudaGetLastError();
}

cudaError_t launch_oz_digits(const PartDesc* parts, const ColBlock* blocks, int nblocks, const double* x0,
                             const double* x1, int after, int need, const OzSlices& out, const int32_t* sig,
                             const DevState* st, cudaStream_t s) {
  oz_digits_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, x0, x1, after, need, out, sig, st);
  return cudaGetLastError();
}

}  // namespace gsp2
