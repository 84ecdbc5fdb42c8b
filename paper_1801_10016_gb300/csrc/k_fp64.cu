// FP64 kernels of the G-SP2 forward pass: Gershgorin bounds, submatrix gather with
// the initial guess, grouped symmetric squaring with the fused branch/trace epilogue,
// and the core-column scatter into P.
#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"

namespace gsp2 {

// ------------------------------------------------------------------------------------
// Gershgorin bounds (Section 2.1): eps_min = min_i (H_ii - R_i), eps_max = max_i (H_ii
// + R_i), R_i = sum_{j != i} |H_ij|.  One warp per row; block min/max into a slot; the
// last block reduces the slots and resets the per-call state.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bounds_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colind,
                                                     const double* __restrict__ vals,
                                                     double2* __restrict__ slots, DevState* st) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double lo = INFINITY, hi = -INFINITY;
  int bad = 0;
  for (int64_t i = warp; i < n; i += nwarps) {
    double rad = 0.0, dia = 0.0;
    for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
      const double v = vals[p];
      if (!isfinite(v)) bad = 1;
      if (colind[p] == i) dia = v; else rad += fabs(v);
    }
    rad = warp_sum(rad);
    dia = warp_sum(dia);  // exactly one lane holds the diagonal
    lo = fmin(lo, dia - rad);
    hi = fmax(hi, dia + rad);
  }
  __shared__ double s_lo[8], s_hi[8];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (bad) s_bad = 1;
  if (lane == 0) { s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = fmin(lo, s_lo[w]); hi = fmax(hi, s_hi[w]); }
    slots[blockIdx.x] = make_double2(lo, hi);
    if (s_bad) st->nonfinite = 1;
  }
  if (last_block_ticket(&st->counter)) {
    if (threadIdx.x == 0) {
      double a = INFINITY, b = -INFINITY;
      for (unsigned int k = 0; k < gridDim.x; ++k) {
        a = fmin(a, ld_cg(&slots[k].x));
        b = fmax(b, ld_cg(&slots[k].y));
      }
      st->eps_min = a;
      st->eps_max = b;
      if (!isfinite(a) || !isfinite(b) || !(b > a)) st->nonfinite = 1;
      st->counter = 0;
    }
  }
}

// Resets the per-call state; must run before bounds_kernel on the same stream.
__global__ void reset_kernel(DevState* st, int8_t* alpha, const int8_t* alpha_in, int n_in, int n_alpha) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->stopped = 0;
    st->steps = 0;
    st->status = ST_OK;
    st->nonfinite = 0;
    st->fp64_steps = 0;
    st->timeout = 0;
    st->tail_left = 0;
    st->idem_fro = -1.0;
    st->counter = 0;
  }
  for (int i = threadIdx.x; i < n_alpha; i += blockDim.x)
    alpha[i] = (alpha_in != nullptr && i >= 1 && i <= n_in) ? alpha_in[i - 1] : (int8_t)0;
}

// ------------------------------------------------------------------------------------
// Eq. 1 on the stored entries of H, once per P-build: x0[q] = (eps_max [col = row] - H_q) /
// (eps_max - eps_min).  Every entry lies in several parts (each of which gathers it), so
// dividing once here keeps the divisions, which run on GB300's slow FP64 pipe, out of the
// gathers.  One warp per row.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) x0_values_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ colind,
                                                        const double* __restrict__ vals, const DevState* st,
                                                        double* __restrict__ x0) {
  const double emax = st->eps_max, emin = st->eps_min;
  const double den = emax - emin;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w0; g < n; g += nw)
    for (int64_t q = rowptr[g] + lane; q < rowptr[g + 1]; q += 32)
      x0[q] = (colind[q] == g) ? (emax - vals[q]) / den : (0.0 - vals[q]) / den;
}

// ------------------------------------------------------------------------------------
// Local indices of the stored entries of H that the gathers place (Section 2.2: the rows
// S_k[j] of H restricted to the columns S_k): for the stored entry t of row S_k[j],
// loc[locptr[soff_k + j] + t] = a with S_k[a] its column, or -1 when that column is not in
// S_k.  Found by binary search in the ascending core (S_k[0, c)) and halo (S_k[c, s)) lists,
// once per bound workspace: the pattern of H and the parts are fixed by the plan, so every
// gather then reads one index per entry.  One warp per local column j < s_k.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) locate_kernel(const PartDesc* __restrict__ parts,
                                                     const ColBlock* __restrict__ blocks,
                                                     const int32_t* __restrict__ Sall,
                                                     const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colind,
                                                     const int64_t* __restrict__ locptr, int32_t* __restrict__ loc) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.s) return;
  const int32_t* S = Sall + p.soff;
  const int32_t g = S[j];
  const int64_t q0 = rowptr[g], nq = rowptr[g + 1] - q0;
  int32_t* lj = loc + locptr[p.soff + j];
  for (int64_t t = lane; t < nq; t += 32) lj[t] = find_local(S, p.c, p.s, colind[q0 + t]);
}

// ------------------------------------------------------------------------------------
// Gather + Eq. 1: X0_k[a, j] = (eps_max [a == j] - H[S_k[j], S_k[a]]) / (eps_max - eps_min)
// for a, j < s_k; zero in the padding.  One warp per local column j; the row S_k[j]
// of H is walked once, each stored entry's value taken from x0_values_kernel and its
// local index a from the plan's table (locate_kernel, once per bound workspace).  The
// diagonal entry must be stored.
// Blocks store the core-diagonal sum of their columns; the last block forms T_0 and
// chooses the first branch.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gather_kernel(const PartDesc* __restrict__ parts,
                                                     const ColBlock* __restrict__ blocks,
                                                     const int32_t* __restrict__ Sall,
                                                     const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ loc,
                                                     const int64_t* __restrict__ locptr,
                                                     const double* __restrict__ x0, double* __restrict__ arena,
                                                     double* __restrict__ slots, StepCtl ctl) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int lane = threadIdx.x & 31;
  const int j = b.j0 + (threadIdx.x >> 5);
  const int32_t* S = Sall + p.soff;
  double tr = 0.0;
  // columns [s, ld) are zero padding: the squares read it up to the tile edge, and the
  // emulated steps up to ld (their K slices are packed within 128-blocks)
  if (j < p.ld) {
    double* col = arena + p.off + (int64_t)j * p.ld;
    for (int r = lane; r < p.ld; r += 32) col[r] = 0.0;
    __syncwarp();
    if (j < p.s) {
      const int32_t g = S[j];
      const int64_t q0 = rowptr[g], nq = rowptr[g + 1] - q0;
      const int32_t* lj = loc + locptr[p.soff + j];
      for (int64_t t = lane; t < nq; t += 32) {
        const int a = lj[t];
        const int64_t q = q0 + t;
        if (a >= 0) {
          const double x = x0[q];
          col[a] = x;
          if (a == j && j < p.c) tr = x;
        }
      }
    }
  }
  const double2 t = block_sum2(tr, 0.0);
  if (threadIdx.x == 0) slots[blockIdx.x] = t.x;
  if (last_block_ticket(&ctl.st->counter)) {
    double2 acc = make_double2(0.0, 0.0);
    double a = 0.0;
    for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) a += ld_cg(&slots[k]);
    acc = block_sum2(a, 0.0);
    if (threadIdx.x == 0) {
      if (ctl.st->nonfinite) ctl.st->status = ST_NONFINITE;
      finish_step(ctl, 0, acc.x, 0.0);
      ctl.st->counter = 0;
    }
  }
}

// ------------------------------------------------------------------------------------
// One purification step for every part (Eq. 2) on the CUDA cores, T = double (FP64
// path and the FP64 tail of the low-precision paths) or float (FP32 path).
//
// Work item = one upper-triangular 64x64 output tile (ti <= tj) of one part.  X is
// symmetric, so both operands of Y = X X stream from columns of X: the A slice
// X[I, k] is column k rows I, and the B slice X[k, J] = X[J, k] is column k rows J.
// Each of the 256 threads owns a 4x4 block of the tile; 16-wide K slices are double
// buffered in shared memory with cp.async.
// Epilogue: X_new = Y (alpha = -1) or 2 X - Y (alpha = +1), written to (I, J) and
// mirrored to (J, I); diagonal tiles add Tr_core[Y] and Tr_core[X_new] (FP64) to their
// slot.  The last block sums the slots in a fixed order and runs the bookkeeping.
//
// mode: SQ_FORWARD   - step `step`; nothing to do once the loop has stopped;
//       SQ_RECOMPUTE - FP64 adjoint: rebuild X_step from X_{step-1} with the recorded
//                      branch if step < steps applied; no bookkeeping;
//       SQ_TAIL_FIRST/SQ_TAIL_NEXT - FP64 tail of a low-precision run: step = steps+1;
//                      the first tail step takes its branch from the trace rule, each
//                      further one the opposite of the previous, so that eigenvalues
//                      near 0 and near 1 are both purified.
// ------------------------------------------------------------------------------------
constexpr int BK = 16;

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using V = double2;
};
template <>
struct Vec2<float> {
  using V = float2;
};

//
// SQ_RESIDUAL - idempotency report of the final iterate X (from `xin_table[steps]` when
//               given, else `xin`): no write; the block adds sum (X^2 - X)_ij^2 over the
//               core columns j of its tile (and of the mirrored tile) to rslots, and the
//               last block stores sqrt(sum / N) in the state.
template <typename T>
__global__ void __launch_bounds__(256, 2) square_simt_kernel(const PartDesc* __restrict__ parts,
                                                             const Tile* __restrict__ tiles,
                                                             const T* __restrict__ xin, T* __restrict__ xout,
                                                             double2* __restrict__ slots, int nslots, StepCtl ctl,
                                                             int step, int mode, const T* const* xin_table,
                                                             double* __restrict__ rslots, int64_t n) {
  using V2 = typename Vec2<T>::V;
  if (mode == SQ_RECOMPUTE) {
    if (step >= *(volatile int32_t*)&ctl.st->steps) return;  // the sweep never reads X_n
  } else if (mode == SQ_FORWARD) {
    if (*(volatile int32_t*)&ctl.st->stopped) return;
  } else {
    const int32_t stt = *(volatile int32_t*)&ctl.st->status;
    if (stt == ST_NONFINITE || stt == ST_TIMEOUT) return;
    step = *(volatile int32_t*)&ctl.st->steps + 1;
  }
  __shared__ __align__(16) T As[2][BK][SQ_TILE];
  __shared__ __align__(16) T Bs[2][BK][SQ_TILE];
  const Tile t = tiles[blockIdx.x];
  const PartDesc p = parts[t.part];
  const T* xbase = (mode == SQ_RESIDUAL && xin_table) ? xin_table[step - 1] : xin;
  const T* X = xbase + p.off;
  const int64_t ld = p.ld;
  const int r0 = t.ti * SQ_TILE, c0 = t.tj * SQ_TILE;
  const int kend = (p.s + BK - 1) / BK * BK;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  constexpr int EPC = 16 / sizeof(T);             // elements per 16-byte chunk
  constexpr int CPR = SQ_TILE / EPC;              // chunks per slice row
  constexpr int CHUNKS = BK * CPR;                // chunks per operand slice

  auto load_slice = [&](int buf, int k0) {
#pragma unroll
    for (int q = tid; q < CHUNKS; q += 256) {
      const int kr = q / CPR, c2 = (q % CPR) * EPC;
      const T* col = X + (int64_t)(k0 + kr) * ld;
      cp_async16(&As[buf][kr][c2], col + r0 + c2);
      cp_async16(&Bs[buf][kr][c2], col + c0 + c2);
    }
    cp_async_commit();
  };

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);

  const int nk = kend / BK;
  load_slice(0, 0);
  for (int it = 0; it < nk; ++it) {
    const int buf = it & 1;
    if (it + 1 < nk) {
      load_slice(buf ^ 1, (it + 1) * BK);
      cp_async_wait_1();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const V2 a01 = *reinterpret_cast<const V2*>(&As[buf][kk][tx * 4]);
      const V2 a23 = *reinterpret_cast<const V2*>(&As[buf][kk][tx * 4 + 2]);
      const V2 b01 = *reinterpret_cast<const V2*>(&Bs[buf][kk][ty * 4]);
      const V2 b23 = *reinterpret_cast<const V2*>(&Bs[buf][kk][ty * 4 + 2]);
      const T a[4] = {a01.x, a01.y, a23.x, a23.y};
      const T b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
    }
    __syncthreads();
  }

  if (mode == SQ_RESIDUAL) {
    double res = 0.0;
    const int rb = r0 + tx * 4, cb = c0 + ty * 4;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int c = cb + jj;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = rb + i;
        const double d = (double)acc[i][jj] - (double)X[(int64_t)c * ld + r];
        if (c < p.c) res += d * d;
        if (t.ti != t.tj && r < p.c) res += d * d;
      }
    }
    const double2 sr = block_sum2(res, 0.0);
    if (tid == 0) rslots[blockIdx.x] = sr.x;
    if (last_block_ticket(&ctl.st->counter)) {
      double a = 0.0;
      for (unsigned int k = tid; k < gridDim.x; k += blockDim.x) a += ld_cg(&rslots[k]);
      const double2 sum = block_sum2(a, 0.0);
      if (tid == 0) {
        ctl.st->idem_fro = sqrt(sum.x / (double)n);
        ctl.st->counter = 0;
      }
    }
    return;
  }

  // branch of this step
  int8_t al;
  if (mode == SQ_TAIL_FIRST) al = (ctl.traces[step - 1] <= (double)ctl.nocc) ? (int8_t)1 : (int8_t)-1;
  else if (mode == SQ_TAIL_NEXT) al = (int8_t)(-ctl.alpha[step - 1]);
  else al = ctl.alpha[step];
  const bool book = mode != SQ_RECOMPUTE;

  T* Y = xout + p.off;
  double tY = 0.0, tN = 0.0;
  const int rb = r0 + tx * 4, cb = c0 + ty * 4;
  // rb and cb are multiples of 4: a thread's block meets the diagonal only when rb == cb,
  // at (i, i); its entries are added in FP64 outside the unrolled loop
  T yd[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) yd[i] = acc[i][i];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int c = cb + jj;
    const V2 x01 = *reinterpret_cast<const V2*>(X + (int64_t)c * ld + rb);
    const V2 x23 = *reinterpret_cast<const V2*>(X + (int64_t)c * ld + rb + 2);
    const T xv[4] = {x01.x, x01.y, x23.x, x23.y};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T y = acc[i][jj];
      const T xn = (al > 0) ? (T(2) * xv[i] - y) : y;
      acc[i][jj] = xn;
    }
    V2 v;
    v.x = acc[0][jj]; v.y = acc[1][jj];
    *reinterpret_cast<V2*>(Y + (int64_t)c * ld + rb) = v;
    v.x = acc[2][jj]; v.y = acc[3][jj];
    *reinterpret_cast<V2*>(Y + (int64_t)c * ld + rb + 2) = v;
  }
  if (book && t.slot >= 0 && rb == cb) {
    for (int i = 0; i < 4; ++i) {
      if (cb + i >= p.c) break;
      tY += (double)yd[i];
      tN += (double)acc[i][i];
    }
  }
  if (t.ti != t.tj) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + i;
      V2 v;
      v.x = acc[i][0]; v.y = acc[i][1];
      *reinterpret_cast<V2*>(Y + (int64_t)r * ld + cb) = v;
      v.x = acc[i][2]; v.y = acc[i][3];
      *reinterpret_cast<V2*>(Y + (int64_t)r * ld + cb + 2) = v;
    }
  }
  if (!book) return;
  if (t.slot >= 0) {
    const double2 s = block_sum2(tY, tN);
    if (tid == 0) slots[t.slot] = s;
  }
  if (last_block_ticket(&ctl.st->counter)) {
    double a = 0.0, b = 0.0;
    for (int k = tid; k < nslots; k += blockDim.x) {
      a += ld_cg(&slots[k].x);
      b += ld_cg(&slots[k].y);
    }
    const double2 s = block_sum2(a, b);
    if (tid == 0) {
      if (mode == SQ_FORWARD) {
        finish_step(ctl, step, s.y, s.x);
      } else {
        ctl.alpha[step] = al;
        finish_tail(ctl, step, s.y, s.x, true);
      }
      ctl.st->counter = 0;
    }
  }
}

// ------------------------------------------------------------------------------------
// Scatter of core columns (Section 1.1, Fig. 1): for core j of part k with global
// index g = S_k[j], P[:, g] on rows sorted(S_k) = X_k[perm_k[t], j].  The final
// iterate X_steps sits in the arena arena_of_step[steps].
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) scatter_kernel(const PartDesc* __restrict__ parts,
                                                      const ColBlock* __restrict__ blocks,
                                                      const int32_t* __restrict__ Sall,
                                                      const int32_t* __restrict__ perm,
                                                      const int64_t* __restrict__ pcolptr,
                                                      const double* const* __restrict__ arena_of_step,
                                                      const double* __restrict__ fixed_arena,
                                                      double* __restrict__ pvals, const DevState* st,
                                                      int upper_block, int fx) {
  const ColBlock b = blocks[blockIdx.x];
  const PartDesc p = parts[b.part];
  const int j = b.j0 + (threadIdx.x >> 5);
  if (j >= p.c) return;
  const int lane = threadIdx.x & 31;
  const double* A = (fixed_arena ? fixed_arena : arena_of_step[st->steps]) + p.off;
  const double* X = A + (int64_t)j * p.ld;
  const int32_t g = Sall[p.soff + j];
  const int32_t* pm = perm + p.soff;
  double* out = pvals + pcolptr[g];
  // upper_block > 0: only the tiles of that edge on or above the diagonal are stored (the
  // matrix is symmetric), so X[a, j] below them is read as X[j, a]
  const int jb = upper_block > 0 ? j / upper_block : 0;
  // fx: the arena holds 64-bit fixed point (x 2^56), as the emulated FP64 steps keep it
  for (int t = lane; t < p.s; t += 32) {
    const int a = pm[t];
    const double* v = (upper_block > 0 && a / upper_block > jb) ? A + (int64_t)a * p.ld + j : X + a;
    out[t] = fx ? from_fixed(*reinterpret_cast<const long long*>(v)) : *v;
  }
}

// An arena of 64-bit fixed point (x 2^56) turned into FP64 in place, for the FP64 consumers
// of the final iterate (the idempotency report).
__global__ void __launch_bounds__(256) fixed_to_fp64_kernel(const double* const* __restrict__ arena_of_step,
                                                            double* arena, const DevState* st, int64_t n) {
  double* a = arena ? arena : const_cast<double*>(arena_of_step[st->steps]);
  long long* v = reinterpret_cast<long long*>(a);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = from_fixed(v[i]);
}

// Fill the lower tiles of arenas that hold only the upper 128-tiles (emulated FP64 steps
// without mirrored writes), for consumers that read whole columns: one block per upper
// off-diagonal tile, 32 x 32 blocks transposed through shared memory.
__global__ void __launch_bounds__(256) symmetrize_kernel(const PartDesc* __restrict__ parts,
                                                         const Tile* __restrict__ tiles,
                                                         const double* const* __restrict__ arena_of_step,
                                                         double* __restrict__ fixed_arena, const DevState* st) {
  const Tile t = tiles[blockIdx.x];
  if (t.ti == t.tj) return;
  const PartDesc p = parts[t.part];
  double* A = (fixed_arena ? fixed_arena : const_cast<double*>(arena_of_step[st->steps])) + p.off;
  __shared__ double buf[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int bi = 0; bi < 4; ++bi)
    for (int bj = 0; bj < 4; ++bj) {
      const int r0 = t.ti * 128 + bi * 32, c0 = t.tj * 128 + bj * 32;
      for (int y = ty; y < 32; y += 8) buf[y][tx] = A[(int64_t)(c0 + y) * p.ld + r0 + tx];  // column c0+y
      __syncthreads();
      for (int y = ty; y < 32; y += 8) A[(int64_t)(r0 + y) * p.ld + c0 + tx] = buf[tx][y];   // column r0+y
      __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// launch wrappers
// ------------------------------------------------------------------------------------
cudaError_t launch_reset(DevState* st, int8_t* alpha, const int8_t* alpha_in, int n_in, int n_alpha,
                         cudaStream_t s) {
  reset_kernel<<<1, 256, 0, s>>>(st, alpha, alpha_in, n_in, n_alpha);
  return cudaGetLastError();
}

cudaError_t launch_bounds(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                          double2* slots, int nblocks, DevState* st, cudaStream_t s) {
  bounds_kernel<<<nblocks, 256, 0, s>>>(n, rowptr, colind, vals, slots, st);
  return cudaGetLastError();
}

cudaError_t launch_gather(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                          const int64_t* rowptr, const int32_t* loc, const int64_t* locptr, const double* x0,
                          double* arena, double* slots, const StepCtl& ctl, cudaStream_t s) {
  gather_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, Sall, rowptr, loc, locptr, x0, arena,
                                                       slots, ctl);
  return cudaGetLastError();
}

cudaError_t launch_x0_values(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                             const DevState* st, double* x0, int nsm, cudaStream_t s) {
  x0_values_kernel<<<8 * nsm, 256, 0, s>>>(n, rowptr, colind, vals, st, x0);
  return cudaGetLastError();
}

cudaError_t launch_locate(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                          const int64_t* rowptr, const int32_t* colind, const int64_t* locptr, int32_t* loc,
                          cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  locate_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, Sall, rowptr, colind, locptr, loc);
  return cudaGetLastError();
}

cudaError_t launch_square_fp64(const PartDesc* parts, const Tile* tiles, int ntiles, const double* xin,
                               double* xout, double2* slots, int nslots, const StepCtl& ctl, int step, int mode,
                               cudaStream_t s) {
  square_simt_kernel<double><<<ntiles, 256, 0, s>>>(parts, tiles, xin, xout, slots, nslots, ctl, step, mode,
                                                    nullptr, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_residual_fp64(const PartDesc* parts, const Tile* tiles, int ntiles, const double* x,
                                 const double* const* x_of_step, double* rslots, int64_t n, const StepCtl& ctl,
                                 cudaStream_t s) {
  square_simt_kernel<double><<<ntiles, 256, 0, s>>>(parts, tiles, x, nullptr, nullptr, 0, ctl, 0, SQ_RESIDUAL,
                                                    x_of_step, rslots, n);
  return cudaGetLastError();
}

cudaError_t launch_square_fp32(const PartDesc* parts, const Tile* tiles, int ntiles, const float* xin, float* xout,
                               double2* slots, int nslots, const StepCtl& ctl, int step, cudaStream_t s) {
  square_simt_kernel<float><<<ntiles, 256, 0, s>>>(parts, tiles, xin, xout, slots, nslots, ctl, step, SQ_FORWARD,
                                                   nullptr, nullptr, 0);
  return cudaGetLastError();
}

// |P_e| > tau over the stored values of P (graph refresh of Section 2.2).
__global__ void threshold_kernel(const double* __restrict__ p, int64_t n, double tau, uint8_t* __restrict__ mask) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    mask[e] = fabs(p[e]) > tau ? 1 : 0;
}

cudaError_t launch_threshold(const double* p, int64_t n, double tau, uint8_t* mask, cudaStream_t s) {
  threshold_kernel<<<152 * 8, 256, 0, s>>>(p, n, tau, mask);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                           const int32_t* perm, const int64_t* pcolptr, const double* const* arena_of_step,
                           const double* fixed_arena, double* pvals, const DevState* st, cudaStream_t s, int upper_block,
                           int fx) {
  scatter_kernel<<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, Sall, perm, pcolptr, arena_of_step,
                                                        fixed_arena, pvals, st, upper_block, fx);
  return cudaGetLastError();
}

cudaError_t launch_fixed_to_fp64(const double* const* arena_of_step, double* arena, const DevState* st, int64_t n,
                                 int nsm, cudaStream_t s) {
  fixed_to_fp64_kernel<<<4 * nsm, 256, 0, s>>>(arena_of_step, arena, st, n);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(const PartDesc* parts, const Tile* tiles, int ntiles, const double* const* arena_of_step,
                              double* fixed_arena, const DevState* st, cudaStream_t s) {
  symmetrize_kernel<<<ntiles, 256, 0, s>>>(parts, tiles, arena_of_step, fixed_arena, st);
  return cudaGetLastError();
}

}  // namespace gsp2
