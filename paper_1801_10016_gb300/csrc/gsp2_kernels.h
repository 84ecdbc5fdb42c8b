// Launch wrappers of the G-SP2 kernels (host-callable, internal to the library).
#pragma once

#include "gsp2_internal.cuh"

namespace gsp2 {

cudaError_t launch_reset(DevState* st, int8_t* alpha, const int8_t* alpha_in, int n_in, int n_alpha,
                         cudaStream_t s);
cudaError_t launch_bounds(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                          double2* slots, int nblocks, DevState* st, cudaStream_t s);
cudaError_t launch_gather(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                          const int64_t* rowptr, const int32_t* loc, const int64_t* locptr, const double* x0,
                          double* arena, double* slots, const StepCtl& ctl, cudaStream_t s);
// Eq. 1 on the stored entries of H (the gathers' values)
cudaError_t launch_x0_values(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                             const DevState* st, double* x0, int nsm, cudaStream_t s);
// the gathers' table of local indices (once per bound workspace)
cudaError_t launch_locate(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                          const int64_t* rowptr, const int32_t* colind, const int64_t* locptr, int32_t* loc,
                          cudaStream_t s);
cudaError_t launch_square_fp64(const PartDesc* parts, const Tile* tiles, int ntiles, const double* xin,
                               double* xout, double2* slots, int nslots, const StepCtl& ctl, int step, int mode,
                               cudaStream_t s);
cudaError_t launch_residual_fp64(const PartDesc* parts, const Tile* tiles, int ntiles, const double* x,
                                 const double* const* x_of_step, double* rslots, int64_t n, const StepCtl& ctl,
                                 cudaStream_t s);
cudaError_t launch_threshold(const double* p, int64_t n, double tau, uint8_t* mask, cudaStream_t s);
cudaError_t launch_square_fp32(const PartDesc* parts, const Tile* tiles, int ntiles, const float* xin, float* xout,
                               double2* slots, int nslots, const StepCtl& ctl, int step, cudaStream_t s);
cudaError_t launch_scatter(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                           const int32_t* perm, const int64_t* pcolptr, const double* const* arena_of_step,
                           const double* fixed_arena, double* pvals, const DevState* st, cudaStream_t s,
                           int upper_block = 0, int fx = 0);
// an arena of 64-bit fixed point (x 2^56) to FP64 in place (arena, or arena_of_step[steps])
cudaError_t launch_fixed_to_fp64(const double* const* arena_of_step, double* arena, const DevState* st, int64_t n,
                                 int nsm, cudaStream_t s);
cudaError_t launch_symmetrize(const PartDesc* parts, const Tile* tiles, int ntiles, const double* const* arena_of_step,
                              double* fixed_arena, const DevState* st, cudaStream_t s);

// low-precision paths (k_tc.cu)
cudaError_t launch_square_tc(int kind, int nprod, const TcStepArgs& a, int ntiles, int persistent_grid,
                             cudaStream_t s);
cudaError_t launch_gather_lp(int kind, int nprod, const PartDesc* parts, const ColBlock* blocks, int nblocks,
                             const int32_t* Sall, const int64_t* rowptr, const int32_t* loc, const int64_t* locptr,
                             const double* x0, float* master, void* op_hi, void* op_lo, double* slots,
                             const StepCtl& ctl, cudaStream_t s, int upper_rows = 0);
// FP32 adjoint of the low-precision plans on the tensor cores (FP16 hi + lo operands)
cudaError_t launch_tc_adjoint(const TcStepArgs& a, int grid, bool rebuild, cudaStream_t s);
cudaError_t launch_split_f16(const PartDesc* parts, const ColBlock* blocks, int nblocks, const float* x, void* hi,
                             void* lo, const int32_t* sig, int need, int tail, const DevState* st, cudaStream_t s);
cudaError_t launch_xbar_seed_scale(const PartDesc* parts, const ColBlock* blocks, int nblocks, const float* x,
                                   uint32_t* xb_max, int32_t* xb_sig, int nparts, int headroom, DevState* st,
                                   cudaStream_t s);
cudaError_t launch_copy_iterate(const float* const* master_of_step, float* out, int64_t n, const DevState* st,
                                int back, cudaStream_t s);
cudaError_t launch_convert(const float* const* master_of_step, double* out, int64_t n, const DevState* st,
                           cudaStream_t s);
// FP64 products from BF16 digits (k_oz.cu)
cudaError_t launch_oz_step(const OzStepArgs& a, int grid, cudaStream_t s, bool adjoint = false);
// the last FP32 iterate of a low-precision run as fixed-point master and digits (upper rows only)
cudaError_t launch_oz_convert_slice(const PartDesc* parts, const ColBlock* blocks, int nblocks,
                                    const float* const* master_of_step, double* X, const OzSlices* digits,
                                    const DevState* st, cudaStream_t s);
// gather with Eq. 1 and the digits of X0 in one pass (emulated path)
cudaError_t launch_oz_gather(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                             const int64_t* rowptr, const int32_t* loc, const int64_t* locptr, const double* x0,
                             double* arena, const OzSlices& dig, double* slots, const StepCtl& ctl, cudaStream_t s);
// the emulated adjoint's Xbar digits: row norms and per-part scales, then the digits
cudaError_t launch_oz_adj_scale(const PartDesc* parts, int nparts, const Tile* tiles, int ntiles, const double* xb0,
                                const double* xb1, int after, double* norm, int32_t* sig, const DevState* st,
                                cudaStream_t s);
cudaError_t launch_oz_digits(const PartDesc* parts, const ColBlock* blocks, int nblocks, const double* x0,
                             const double* x1, int after, int need, const OzSlices& out, const int32_t* sig,
                             const DevState* st, cudaStream_t s);
int encode_part_maps(void* enc_fn, void* out_maps, const PartDesc* parts, int nparts, void* arena, int kind,
                     int box_bytes = 128, int box_cols = 128);
int encode_part_maps_digits(void* enc_fn, void* out_k, void* out_mn, const PartDesc* parts, int nparts, void* arena0,
                            size_t dstride, int ndig, int nbox, int box_k);

// shard plans (k_shard.cu): this shard's partial traces out, the summed decision in
cudaError_t launch_shard_partial(const DevState* st, const ShardSlot* slot, double* send, cudaStream_t s);
cudaError_t launch_shard_decide(const StepCtl& c, const double* recv, int nranks, int kind, cudaStream_t s);

// adjoint (k_adjoint.cu)
template <typename T>
cudaError_t launch_adj_seed(const PartDesc* parts, const ColBlock* blocks, int nblocks, const int32_t* Sall,
                            const int32_t* invperm, const int64_t* pcolptr, const double* pbar, T* xbar,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_adj_step(const PartDesc* parts, const Tile* tiles, int ntiles, const T* X, T* xb0, T* xb1,
                            const int8_t* alpha, const DevState* st, int step, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_hbar(int64_t n, const int64_t* rowptr, const int32_t* colind, const int64_t* memptr,
                            const int32_t* mempart, const int32_t* memloc, const PartDesc* parts,
                            const int32_t* Sall, const T* xb0, const T* xb1, double* hbar, const DevState* st,
                            cudaStream_t s, int upper_block = 0);

}  // namespace gsp2
