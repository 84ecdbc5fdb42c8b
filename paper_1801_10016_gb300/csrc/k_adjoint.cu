// Adjoint of the G-SP2 density matrix: seed (FP64, or FP32 for the low-precision plans),
// the reverse purification steps of the native FP64 plans on the CUDA cores, and the
// scatter-add onto the pattern of H.  (The emulated FP64 plans and the low-precision plans
// run their reverse steps on the tensor cores: k_oz.cu, k_tc.cu.)
//
// With L = sum Pbar .* P and the branch sequence alpha_1..alpha_n fixed:
//   seed:   Xbar_n = sym(M_k), M_k[:, j] = Pbar[S_k, g_j] for core j, 0 for halo columns
//           (X_k is a symmetric function of a symmetric argument);
//   step i: alpha_i = -1 (X_i = X^2):      Xbar <- Xbar X + X Xbar
//           alpha_i = +1 (X_i = 2X - X^2): Xbar <- 2 Xbar - Xbar X - X Xbar
//           with X = X_{i-1};
//   Eq. 1:  dL/dH[S_k, S_k] = -Xbar_0 / (eps_max - eps_min), summed over the parts
//           that hold both indices; the bounds are held fixed.
#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"

namespace gsp2 {

// Seed: one warp per local column b (including the zero padding up to nt*TILE).
template <typename T>
__global__ void __launch_bounds__(256) adj_seed_kernel(const PartDesc* __restrict__ parts,
                                                       const ColBlock* __restrict__ blocks,
                                                       const int32_t* __restrict__ Sall,
                                                       const int32_t* __restrict__ invperm,
                                                       const int64_t* __restrict__ pcolptr,
                                                       const double* __restrict__ pbar, T* __restrict__ xbar) {
  const ColBlock bl = blocks[blockIdx.x];
  const PartDesc p = parts[bl.part];
  const int lane = threadIdx.x & 31;
  const int b = bl.j0 + (threadIdx.x >> 5);
  if (b >= p.nt * SQ_TILE) return;
  const int32_t* S = Sall + p.soff;
  const int32_t* ip = invperm + p.soff;
  T* col = xbar + p.off + (int64_t)b * p.ld;
  const bool bin = b < p.s;
  const int64_t colb = (bin && b < p.c) ? pcolptr[S[b]] : -1;  // column g_b of P if b is a core
  const int ipb = bin ? ip[b] : 0;
  for (int a = lane; a < p.ld; a += 32) {
    double v = 0.0;
    if (bin && a < p.s) {
      const double mab = (colb >= 0) ? pbar[colb + ip[a]] : 0.0;             // M(a, b)
      const double mba = (a < p.c) ? pbar[pcolptr[S[a]] + ipb] : 0.0;       // M(b, a)
      v = 0.5 * (mab + mba);
    }
    col[a] = (T)v;
  }
}

// One reverse step for every part.  Work item = one upper tile (ti <= tj);
// Z_IJ = sum_k Xbar[I,k] X[k,J] + X[I,k] Xbar[k,J] with all four slices streamed from
// columns k of the symmetric Xbar and X.  Result mirrored to (J, I).
// The Xbar buffers alternate with (n - step) so that skipped steps keep the parity: input
// xb[(n - step) & 1], output xb[(n - step + 1) & 1], n the steps applied by the forward;
// steps above n are skipped.
// Four consecutive elements (16-byte aligned for FP32, 32 for FP64) in vector stores.
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}
__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <typename T>
struct AdjBK {
  static constexpr int v = 64 / (int)sizeof(T);  // K slice: 8 (FP64) or 16 (FP32) = 16 B per thread
};

template <typename T>
__global__ void __launch_bounds__(256, 2) adj_step_kernel(const PartDesc* __restrict__ parts,
                                                          const Tile* __restrict__ tiles, const T* __restrict__ Xall,
                                                          T* __restrict__ xb0, T* __restrict__ xb1,
                                                          const int8_t* __restrict__ alpha, const DevState* st,
                                                          int step) {
  constexpr int ABK = AdjBK<T>::v;
  const int n = *(volatile const int32_t*)&st->steps;
  if (step > n) return;
  const T* XBin = ((n - step) & 1) ? xb1 : xb0;
  T* XBout = ((n - step) & 1) ? xb0 : xb1;
  __shared__ __align__(16) T S1[2][ABK][SQ_TILE];  // Xbar rows I
  __shared__ __align__(16) T S2[2][ABK][SQ_TILE];  // X    rows J
  __shared__ __align__(16) T S3[2][ABK][SQ_TILE];  // X    rows I
  __shared__ __align__(16) T S4[2][ABK][SQ_TILE];  // Xbar rows J
  const Tile t = tiles[blockIdx.x];
  const PartDesc p = parts[t.part];
  const T* X = Xall + p.off;
  const T* B = XBin + p.off;
  const int64_t ld = p.ld;
  const int r0 = t.ti * SQ_TILE, c0 = t.tj * SQ_TILE;
  const int kend = (p.s + ABK - 1) / ABK * ABK;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  auto load_slice = [&](int buf, int k0) {
    // ABK x 64 elements per operand = 256 16-byte chunks: one per thread per operand
    constexpr int EPC = 16 / (int)sizeof(T);
    const int kr = tid / (SQ_TILE / EPC), c2 = (tid % (SQ_TILE / EPC)) * EPC;
    const int64_t co = (int64_t)(k0 + kr) * ld;
    cp_async16(&S1[buf][kr][c2], B + co + r0 + c2);
    cp_async16(&S2[buf][kr][c2], X + co + c0 + c2);
    cp_async16(&S3[buf][kr][c2], X + co + r0 + c2);
    cp_async16(&S4[buf][kr][c2], B + co + c0 + c2);
    cp_async_commit();
  };

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  const int nk = kend / ABK;
  load_slice(0, 0);
  for (int it = 0; it < nk; ++it) {
    const int buf = it & 1;
    if (it + 1 < nk) {
      load_slice(buf ^ 1, (it + 1) * ABK);
      cp_async_wait_1();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < ABK; ++kk) {
      T a1[4], b1[4], a2[4], b2[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a1[q] = S1[buf][kk][tx * 4 + q];
        b1[q] = S2[buf][kk][ty * 4 + q];
        a2[q] = S3[buf][kk][tx * 4 + q];
        b2[q] = S4[buf][kk][ty * 4 + q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a2[i], b2[j], fma(a1[i], b1[j], acc[i][j]));
    }
    __syncthreads();
  }

  const int8_t al = alpha[step];
  T* O = XBout + p.off;
  const int rb = r0 + tx * 4, cb = c0 + ty * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cb + j;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const T z = acc[i][j];
      acc[i][j] = (al > 0) ? (T(2) * B[(int64_t)c * ld + rb + i] - z) : z;
    }
    store4(O + (int64_t)c * ld + rb, acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
  }
  if (t.ti != t.tj) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + i;
      store4(O + (int64_t)r * ld + cb, acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
  }
}

// dL/dH on the CSR pattern: for every stored (r, col), the sum over the parts k that
// hold r (membership list of r) and col of -Xbar0_k[col, r] / (eps_max - eps_min), in
// the fixed membership order (ascending part id).  One warp per row, lanes over the row's entries.  With
// upper_block > 0 only the tiles of that edge on or above the diagonal hold Xbar0 (the
// emulated adjoint); the symmetric entry is read from there.
template <typename T>
__global__ void __launch_bounds__(256) adj_hbar_kernel(int64_t n, const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colind,
                                                       const int64_t* __restrict__ memptr,
                                                       const int32_t* __restrict__ mempart,
                                                       const int32_t* __restrict__ memloc,
                                                       const PartDesc* __restrict__ parts,
                                                       const int32_t* __restrict__ Sall,
                                                       const T* __restrict__ xb0, const T* __restrict__ xb1,
                                                       double* __restrict__ hbar, const DevState* st,
                                                       int upper_block) {
  const int nsteps = st->steps;
  const T* XB = (nsteps & 1) ? xb1 : xb0;
  const double scale = -1.0 / (st->eps_max - st->eps_min);
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = warp; r < n; r += nwarps) {
    const int64_t m0 = memptr[r], m1 = memptr[r + 1];
    for (int64_t q = rowptr[r] + lane; q < rowptr[r + 1]; q += 32) {
      const int32_t col = colind[q];
      // the parts holding both r and col: the intersection of their membership lists, both
      // in ascending part order, walked as a merge (the same parts in the same order as a
      // search of col in every S_k of r's list, so the same sum)
      int64_t mc = memptr[col];
      const int64_t mc1 = memptr[col + 1];
      double sum = 0.0;
      for (int64_t m = m0; m < m1 && mc < mc1; ++m) {
        const int32_t k = mempart[m];
        while (mc < mc1 && mempart[mc] < k) ++mc;
        if (mc == mc1 || mempart[mc] != k) continue;
        const PartDesc p = parts[k];
        const int lc = memloc[mc], lr = memloc[m];
        const bool swap = upper_block > 0 && lc / upper_block > lr / upper_block;
        sum += (double)XB[p.off + (swap ? (int64_t)lc * p.ld + lr : (int64_t)lr * p.ld + lc)];
      }
      hbar[q] = scale * sum;
    }
  }
}

template <typename T>
cudaError_t launch_adj_seed(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                            const int32_t* invperm, const int64_t* pcolptr, const double* pbar, T* xbar,
                            cudaStream_t s) {
  adj_seed_kernel<T><<<nblocks, 32 * COLS_PER_BLOCK, 0, s>>>(parts, blocks, Sall, invperm, pcolptr, pbar, xbar);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_step(const PartDesc* parts, const Tile* tiles, int ntiles, const T* X, T* xb0, T* xb1,
                            const int8_t* alpha, const DevState* st, int step, cudaStream_t s) {
  adj_step_kernel<T><<<ntiles, 256, 0, s>>>(parts, tiles, X, xb0, xb1, alpha, st, step);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_hbar(int64_t n, const int64_t* rowptr, const int32_t* colind, const int64_t* memptr,
                            const int32_t* mempart, const int32_t* memloc, const PartDesc* parts,
                            const int32_t* Sall, const T* xb0, const T* xb1, double* hbar, const DevState* st,
                            cudaStream_t s, int upper_block) {
  adj_hbar_kernel<T><<<608, 256, 0, s>>>(n, rowptr, colind, memptr, mempart, memloc, parts, Sall, xb0, xb1, hbar, st,
                                         upper_block);
  return cudaGetLastError();
}

#define GSP2_ADJ_INSTANTIATE(T)                                                                                     \
  template cudaError_t launch_adj_seed<T>(const PartDesc*, const ColBlock*, int, const int32_t*, const int32_t*,   \
                                          const int64_t*, const double*, T*, cudaStream_t);                        \
  template cudaError_t launch_adj_hbar<T>(int64_t, const int64_t*, const int32_t*, const int64_t*, const int32_t*, \
                                          const int32_t*, const PartDesc*, const int32_t*, const T*, const T*,     \
                                          double*, const DevState*, cudaStream_t, int);
GSP2_ADJ_INSTANTIATE(double)
GSP2_ADJ_INSTANTIATE(float)
template cudaError_t launch_adj_step<double>(const PartDesc*, const Tile*, int, const double*, double*, double*,
                                             const int8_t*, const DevState*, int, cudaStream_t);

}  // namespace gsp2
