// Internal data structures shared by the G-SP2 kernels and the host plan code.
//
// Layout in device memory (all inside the caller's workspace):
//   * one "arena" per buffer holds every part's dense s_k x s_k matrix, column-major,
//     padded to ld_k = roundup(s_k, LD_PAD) rows and columns, at element offset off_k;
//     rows/columns in [s_k, ld_k) are zero so padded products stay exact;
//   * part descriptors, the per-part vertex lists S_k (cores ascending, then halo
//     ascending), the scatter permutation, the work lists and the per-step state.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gsp2 {

constexpr int LD_PAD = 128;      // ld_k multiple (tile edge of every square kernel)
constexpr int SQ_TILE = 64;      // FP64 square tile edge
constexpr int TC_TILE = 128;     // tensor-core square tile edge
constexpr int COLS_PER_BLOCK = 8;  // gather/scatter: one warp per column, 8 warps

struct PartDesc {
  int64_t off;   // arena element offset of X_k
  int64_t soff;  // offset of S_k in the vertex-list table
  int32_t s;     // core + halo size
  int32_t c;     // core count
  int32_t ld;    // padded leading dimension
  int32_t nt;    // FP64 square tiles per edge: ceil(s / SQ_TILE)
};

struct Tile {  // one upper-triangular output tile of one part
  int32_t part, ti, tj, slot;  // slot: diagonal-tile trace slot, -1 otherwise
};

struct ColBlock {  // COLS_PER_BLOCK consecutive local columns of one part
  int32_t part, j0;
};

// Per-call device state.  `counter` is the ticket of the last-block-done
// reductions; the block that finishes a reduction sets it back to zero.
struct DevState {
  double eps_min, eps_max;
  double idem_fro;     // idempotency report of the final P (core columns), -1 if not run
  unsigned int counter;
  int32_t stopped;     // 1: no further purification steps this call
  int32_t steps;       // purification steps applied so far
  int32_t status;      // gsp2_status detected on the device
  int32_t nonfinite;   // set by any block that meets NaN/Inf
  int32_t fp64_steps;
  int32_t timeout;     // a bounded device wait gave up
  int32_t tail_left;   // FP64 path: alternating tail steps still to run (0: none)
  int32_t pad[4];
};

enum : int32_t { ST_OK = 0, ST_NOT_CONVERGED = 5, ST_TRACE = 6, ST_NONFINITE = 7, ST_TIMEOUT = 9 };
enum : int32_t { MODE_RECORD = 0, MODE_REPLAY = 1 };
enum : int32_t { SQ_FORWARD = 0, SQ_RECOMPUTE = 1, SQ_TAIL_FIRST = 2, SQ_TAIL_NEXT = 3, SQ_RESIDUAL = 4 };

// Exchange slot of a shard plan (a plan over a subset of the parts, one per GPU): the
// last block of a step leaves its partial core traces here instead of deciding, and the
// decision is taken by a separate launch once every shard's partials are summed.
struct ShardSlot {
  double t;      // partial Tr_core[X_step] over this shard's parts
  double y;      // partial Tr_core[X_{step-1}^2]
  int32_t step;  // the step the partials belong to
  int32_t pad;
};

// Which bookkeeping an exchange of a shard plan completes: the gather of X0, a step of
// the purification loop, an alternating tail step in the low precision, an FP64 tail step.
enum : int32_t { SHARD_GATHER = 0, SHARD_LOOP = 1, SHARD_TAIL_LP = 2, SHARD_TAIL_FP64 = 3 };

// Arguments of the per-step trace bookkeeping done by the last block of a step.
struct StepCtl {
  DevState* st;
  int8_t* alpha;     // alpha[i] = branch of step i (1-based), int8
  double* traces;    // traces[i] = T_i (core trace of X_i)
  double* idem;      // idem[i] = e_i = T_i - Tr_core[X_i^2]
  int64_t nocc;
  double idem_tol;
  double trace_tol;
  int32_t mode;
  int32_t last_step;  // max_steps (RECORD) or nsteps (REPLAY)
  int32_t stop_lag;   // stopping test compares e_{i-1} with e_{i-1-stop_lag}
  int32_t tail_steps; // RECORD: alternating steps after the stopping test (last_step includes them)
  ShardSlot* xchg;    // shard plans: export the partial traces here instead of deciding (else NULL)
};

// Arguments of one tensor-core purification step (k_tc.cu).
// Buffers alternate with the step parity: X_{step-1} is read from buffer (step-1)&1 and
// X_step written to buffer step&1.
struct TcStepArgs {
  const PartDesc* parts;
  const Tile* tiles;       // upper tiles: 128x128, or 128 x 128 nb[t] for the wide persistent kernel
  const int8_t* nb;        // wide tiles: 128-column blocks of each tile (1 or 2); NULL: 128x128 tiles
  const void* map_hi[2];   // CUtensorMap[nparts] over each operand arena (hi part)
  const void* map_lo[2];   // CUtensorMap[nparts] over each lo arena (split mode)
  // 16-bit kinds: the persistent kernel keeps only the tiles on or above the diagonal and
  // reads the operand panels right of a tile's block MN-major from them (boxes of 64 rows
  // by one K block), through these maps over the same arenas
  const void* map_mn_hi[2];
  const void* map_mn_lo[2];
  float* master[2];        // FP32 master copies of X
  void* op_hi[2];          // operand arenas
  void* op_lo[2];
  double2* slots;
  int nslots;
  int ntiles;
  StepCtl ctl;
  int step;                // ignored in tail mode (step = steps applied + 1)
  int tail;                // 0: loop step; 1: first alternating tail step; 2: further ones
  // FP32 adjoint of the low-precision plans (FP16 hi + lo operands, explicit buffers):
  // the rebuilt iterate X_step reads the operands of X_{step-1} (xmap_*) and its master
  // xin and writes master xout and operands xo_*; the reverse step `step` reads the
  // operands of X_{step-1} (xmap_*) and Xbar's ping-pong (map_*, master, op_* [2], the
  // roles chosen on the device by step parity).  `step` <= 0 names step n + step (the
  // FP64 tail steps, counted back from the device's step count n); loop steps above
  // n - adj_tail are skipped.
  const void* xmap_hi;
  const void* xmap_lo;
  const void* xmap_mn_hi;
  const void* xmap_mn_lo;
  const float* xin;
  float* xout;
  void* xo_hi;
  void* xo_lo;
  int adj_tail;
  // FP16 operands (KIND 2) of the adjoint: Xbar's are FP16 of Xbar 2^(14 - sig) with one
  // scale exponent per part: xb_sig[k] that of the operands a reverse step reads,
  // xb_sig[nparts + k] that of the operands it writes, chosen before the step from the
  // largest |Xbar| so far plus xb_headroom bits (one step multiplies the largest entry by
  // at most 2 + 2 sqrt(s), Cauchy-Schwarz with ||X||_2 <= 1).  The step records the largest
  // |Xbar_new| of each part (FP32 bits, xb_max) and its last block moves the scales on
  int32_t* xb_sig;
  uint32_t* xb_max;
  int nparts;
  int xb_headroom;
  // the persistent 128x128 kernel's steps and reverse steps: each CTA claims its next tile
  // from this counter (zero between launches; the last block resets it); NULL: static deal
  uint32_t* tile_ctr;
};
constexpr int TC_SIG_MIN = -98, TC_SIG_MAX = 126;  // range of the FP16 adjoint's scale exponents

// FP64 products rebuilt from BF16 digits (k_oz.cu)
constexpr int OZ_SLICES = 7;  // base-2^7 digits per entry
constexpr int OZ_SPLIT = 3;   // digit groups d < OZ_SPLIT form the second pass of a tile
constexpr int OZ_MAX_GRID = 256;  // CTAs of the emulated step (one 128x128 int64 scratch each)
constexpr int OZ_BK = 32;         // K per pipeline stage of the emulated step (64-byte rows)

struct OzSlices {
  uint16_t* s[OZ_SLICES];  // BF16 digit arenas (same element indexing as the arenas)
};

// One emulated step: digits of X_{step-1} are read from buffer (step-1)&1 and the digits
// of X_step written to buffer step&1 (SQ_FORWARD and the tail modes).  SQ_RECOMPUTE (the
// adjoint's rebuilt iterates) reads the digit set `maps` points at and writes digits[0],
// with the recorded branch and no bookkeeping.  The adjoint instantiation reads the digits
// of X (`maps`) and of Xbar / 2^sig (`maps_b`) and writes Xbar's FP64 ping-pong pair
// (xin = Xbar buffer 0, xout = buffer 1, the roles swapped on the device by step parity).
struct OzStepArgs {
  const PartDesc* parts;
  const Tile* tiles;   // 128x128 upper tiles
  int ntiles;
  const void* maps;    // per digit buffer (OZ_SLICES x nparts maps apart): CUtensorMap[2][nparts], K-major
                       // boxes of all OZ_SLICES digits ([0]) or the first OZ_SPLIT ([1]) of a tile slice
  const void* maps_mn; // the same with MN-major boxes (each tile 128 rows x OZ_BK columns as two 64-row atoms,
                       // 128-byte swizzle)
  const void* maps_b;    // adjoint: the same two K-major map arrays over the digits of Xbar / 2^sig
  const void* maps_mn_b; // the same, MN-major
  int32_t* sig;          // adjoint: per-part scale exponent of Xbar's digits (OZ_SIG_NONFINITE: NaN),
                         // replaced by the new Xbar's scale by the last block of the step
  float* normf;          // adjoint: squared row norms of the new Xbar / 2^sig (zero between steps)
  int nparts;
  OzSlices digits[2];
  const double* xin;   // master of X_{step-1}: 64-bit fixed point x 2^56 (the adjoint's Xbar: FP64)
  double* xout;        // master of X_step, the same form
  double2* slots;      // diagonal-tile trace slots
  int nslots;
  long long* acc;      // OZ_MAX_GRID x 128 x 128 fixed-point partial sums, one tile per CTA
  StepCtl ctl;
  int step;            // ignored in tail modes (step = steps applied + 1)
  int mode;            // SQ_FORWARD, SQ_RECOMPUTE, SQ_TAIL_FIRST or SQ_TAIL_NEXT
  // split K: the work item of code 2 t + h is the half h of upper tile t's product (adjoint:
  // h = 0 Xbar X, h = 1 X Xbar; forward: the two halves of each pass's K stages); each writes
  // its 64-bit partial tile to split_acc[2 t + h] and the second of the two to finish
  // (split_cnt[t], left at zero) adds both and forms the tile (X_new, digits, traces)
  int split;
  long long* split_acc;  // [2 ntiles][128 x 128], indexed by item code 2 t + h
  uint32_t* split_cnt;   // [ntiles]
  const int32_t* split_items;  // [2 ntiles]: item codes in the order the CTAs take them
  // forward, tail and reverse steps: when set, each CTA claims its next item from this
  // counter (the items are then taken in list order by whichever CTA is free); the step's
  // last block sets it back to zero.  NULL (and the rebuilt iterates): CTA b takes items b,
  // b + gridDim.x, ...
  uint32_t* tile_ctr;
};
constexpr int32_t OZ_SIG_NONFINITE = 0x7FFF;  // scale of a part whose Xbar holds NaN or Inf

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 16-byte asynchronous global->shared copies (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Local index of global vertex g in S_k (cores [0, c) ascending, halo [c, s)
// ascending), or -1.
__device__ __forceinline__ int find_local(const int32_t* __restrict__ S, int c, int s, int32_t g) {
  int lo = 0, hi = c;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (S[m] < g) lo = m + 1; else hi = m;
  }
  if (lo < c && S[lo] == g) return lo;
  lo = c; hi = s;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (S[m] < g) lo = m + 1; else hi = m;
  }
  if (lo < s && S[lo] == g) return lo;
  return -1;
}

// Last-block-done ticket.  Every block calls it once, after its partial results are
// stored; returns true in exactly one block (the last), which may then read all
// partials.  All threads of the block must call it.
__device__ __forceinline__ bool last_block_ticket(unsigned int* counter) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Deterministic block-wide sum of two doubles per thread (fixed tree).  Result valid
// in thread 0.  blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double2 red[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = make_double2(a, b);
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) { r.x += red[i].x; r.y += red[i].y; }
  }
  return r;
}

// Bookkeeping of step `step` (0 = the initial guess X0), run by one thread of the
// last block once the global sums are known:
//   tN = Tr_core[X_step], tY = Tr_core[X_{step-1}^2] (unused for step 0).
// Records T_step and e_{step-1}, applies the stopping test, and in RECORD mode
// chooses the branch of the next step: alpha = +1 iff T_step <= Nocc.
// Stopping test (RECORD): |e| <= idem_tol and (e < 0 or e >= e_{step-1-stop_lag});
// e >= 0 in exact arithmetic and falls once all eigenvalues are near 0 or 1, so a
// small e that is negative or no longer falls leaves only rounding (or the G-SP2
// drift of a core trace that cannot reach Nocc) to iterate on.  Every path uses lag 1
// (the field is kept for experiments with longer lags).
__device__ __forceinline__ void finish_step(const StepCtl& c, int step, double tN, double tY) {
  if (c.xchg) {  // shard plan: the sums over all shards decide, in a later launch
    c.xchg->t = tN;
    c.xchg->y = tY;
    c.xchg->step = step;
    return;
  }
  DevState* st = c.st;
  c.traces[step] = tN;
  st->steps = step;
  bool stop = false, fire = false;
  if (step > 0) {
    const double e = c.traces[step - 1] - tY;
    c.idem[step - 1] = e;
    if (c.mode == MODE_RECORD && step >= 1 + c.stop_lag && fabs(e) <= c.idem_tol &&
        (e < 0.0 || e >= c.idem[step - 1 - c.stop_lag]))
      fire = true;
    if (!isfinite(e)) st->nonfinite = 1;
  }
  if (!isfinite(tN)) st->nonfinite = 1;
  if (st->nonfinite) {
    st->status = ST_NONFINITE;
    st->stopped = 1;
    return;
  }
  if (c.mode == MODE_RECORD && st->tail_left > 0) {
    // this step was one of the alternating tail steps
    st->tail_left -= 1;
    if (st->tail_left == 0) {
      st->stopped = 1;
    } else {
      c.alpha[step + 1] = (int8_t)(-c.alpha[step]);
    }
    return;
  }
  const bool cap = step >= c.last_step - (c.mode == MODE_RECORD ? c.tail_steps : 0);
  if (fire) stop = true;
  if (!stop && cap) {
    stop = true;
    if (c.mode == MODE_RECORD && step > 0 && !(fabs(c.idem[step - 1]) <= c.idem_tol)) st->status = ST_NOT_CONVERGED;
  }
  if (stop && c.mode == MODE_RECORD && c.tail_steps > 0) {
    // start the tail: first branch from the trace rule, then alternating
    st->tail_left = c.tail_steps;
    c.alpha[step + 1] = (tN <= (double)c.nocc) ? (int8_t)1 : (int8_t)-1;
    return;
  }
  if (stop) {
    st->stopped = 1;
    if (c.mode == MODE_REPLAY && st->status == ST_OK) {
      const double d = tN - (double)c.nocc;
      if (!(fabs(d) <= c.trace_tol)) st->status = ST_TRACE;
    }
  } else if (c.mode == MODE_RECORD) {
    c.alpha[step + 1] = (tN <= (double)c.nocc) ? (int8_t)1 : (int8_t)-1;
  }
}

// Bookkeeping of a tail step of a low-precision run (FP64, or alternating steps in the
// low precision): records T_step, e_{step-1} and the step count; no stopping test and
// no branch choice.
__device__ __forceinline__ void finish_tail(const StepCtl& c, int step, double tN, double tY, bool fp64) {
  if (c.xchg) {
    c.xchg->t = tN;
    c.xchg->y = tY;
    c.xchg->step = step;
    return;
  }
  DevState* st = c.st;
  c.traces[step] = tN;
  c.idem[step - 1] = c.traces[step - 1] - tY;
  st->steps = step;
  if (fp64) st->fp64_steps += 1;
  if (!isfinite(tN) || !isfinite(c.idem[step - 1])) {
    st->nonfinite = 1;
    st->status = ST_NONFINITE;
  }
}

// Conversions between FP64 and the 2^-56 fixed point of x / 2^sig done with integer
// instructions (the FP64 pipe of GB300 is 64x slower than its integer pipe), rounding to
// nearest even.  |x| / 2^sig < 2^7; larger inputs saturate, results below 2^-1022 flush to 0.
__device__ __forceinline__ long long to_fixed(double x, int sig = 0) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;                                    // zero and subnormals (< 2^-1022)
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1023 - 52 + 56 - sig;                 // (x / 2^sig) * 2^56 = m * 2^sh
  unsigned long long a;
  if (sh > 10) {
    a = 1ull << 62;                                         // out of range: saturate
  } else if (sh >= 0) {
    a = m << sh;
  } else if (sh > -64) {
    const int k = -sh;
    const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
    a = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  } else {
    a = 0;
  }
  return (b >> 63) ? -(long long)a : (long long)a;
}

__device__ __forceinline__ double from_fixed(long long v, int sig = 0) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(a);
  const unsigned long long m = a << lz;                     // top bit at 63
  unsigned long long mant = m >> 11;                        // 53 bits with the leading one
  const unsigned long long rem = m & 0x7FFull;
  int e = 63 - lz - 56 + sig;                               // value = 1.f x 2^e
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    mant += 1;
    if (mant >> 53) {
      mant >>= 1;
      e += 1;
    }
  }
  if (e < -1022) return __longlong_as_double((long long)sgn);
  const unsigned long long bits = sgn | ((unsigned long long)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

}  // namespace gsp2
