// Shard plans: the parts of one G-SP2 problem split over several GPUs (one shard each).
//
// Parts are independent except through the branch of every step, which Section 2.1 takes
// from the trace of the whole iterate: in G-SP2 the sum over all parts of their core
// diagonals (Section 2.2).  A shard's step kernels therefore leave their partial sums
// (core trace of the new iterate and core trace of the square) in a slot instead of
// deciding; the caller gathers every shard's 16-byte partial (an all-gather across
// GPUs); and the decide kernel below adds them in rank order, so that every shard sums
// the same numbers in the same order and takes bitwise the same branch, then does the
// bookkeeping the fused step would have done (trace and idempotency history, stopping
// test, branch of the next step, tail steps).
#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"

namespace gsp2 {

// This shard's partial of the last bookkeeping launch, copied out for the exchange.  A
// shard that met a NaN/Inf or a timed-out wait sends NaN, so that every shard's sum turns
// non-finite and all of them stop together.
__global__ void shard_partial_kernel(const DevState* __restrict__ st, const ShardSlot* __restrict__ slot,
                                     double* __restrict__ send) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int32_t stt = st->status;
  const bool bad = st->nonfinite || stt == ST_NONFINITE || stt == ST_TIMEOUT;
  send[0] = bad ? __longlong_as_double(0x7FF8000000000000ll) : slot->t;
  send[1] = bad ? __longlong_as_double(0x7FF8000000000000ll) : slot->y;
}

// Bookkeeping of one exchange from the gathered partials recv[r] = (t_r, y_r), r in rank
// order.  `kind` names the launch the partials came from, and the skip rule is that
// launch's own: a loop step does nothing once the loop has stopped, a tail step nothing
// after a NaN/Inf or a timeout; the gather always runs.
__global__ void shard_decide_kernel(StepCtl c, const double* __restrict__ recv, int nranks, int kind) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  DevState* st = c.st;
  const int32_t stt = *(volatile int32_t*)&st->status;
  if (kind == SHARD_LOOP && *(volatile int32_t*)&st->stopped) return;
  if ((kind == SHARD_TAIL_LP || kind == SHARD_TAIL_FP64) && (stt == ST_NONFINITE || stt == ST_TIMEOUT)) return;
  if (st->timeout) {
    // this shard's step gave up on a wait (it has already stopped itself)
    st->status = ST_TIMEOUT;
    st->stopped = 1;
    return;
  }
  double t = 0.0, y = 0.0;
  for (int r = 0; r < nranks; ++r) {
    t += recv[2 * r];
    y += recv[2 * r + 1];
  }
  const int step = c.xchg->step;
  StepCtl d = c;
  d.xchg = nullptr;
  if (kind == SHARD_GATHER) finish_step(d, 0, t, 0.0);
  else if (kind == SHARD_LOOP) finish_step(d, step, t, y);
  else finish_tail(d, step, t, y, kind == SHARD_TAIL_FP64);
}

cudaError_t launch_shard_partial(const DevState* st, const ShardSlot* slot, double* send, cudaStream_t s) {
  shard_partial_kernel<<<1, 32, 0, s>>>(st, slot, send);
  return cudaGetLastError();
}

cudaError_t launch_shard_decide(const StepCtl& c, const double* recv, int nranks, int kind, cudaStream_t s) {
  shard_decide_kernel<<<1, 32, 0, s>>>(c, recv, nranks, kind);
  return cudaGetLastError();
}

}  // namespace gsp2
