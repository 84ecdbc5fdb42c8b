/*
 * gsp2.h -- C ABI of the GB300 graph-partitioned SP2 (G-SP2) density-matrix library.
 *
 * The library computes the density matrix P of a sparse symmetric Hamiltonian H by
 * the data-parallel G-SP2 method (Ghale et al., "Task-based Parallel Computation of
 * the Density Matrix in Quantum-based Molecular Dynamics using Graph Partitioning"):
 *
 *   1. a graph G_tau over the orbitals is partitioned into parts; part k owns its
 *      core vertices and sees as halo every vertex adjacent to a core (Section 2.2);
 *   2. each part's dense core+halo submatrix H[S_k, S_k] is gathered and mapped to
 *      X0 = (eps_max I - H)/(eps_max - eps_min) with Gershgorin bounds (Eq. 1);
 *   3. all parts are purified together, X <- X^2 or X <- 2X - X^2 (Eq. 2), with one
 *      branch per step chosen from the global sum of core traces (Section 2.1);
 *   4. core columns are scattered back into P (Section 1.1, Fig. 1).
 *
 * Everything after gsp2_bind_workspace runs on the GPU in hand-written sm_103a
 * kernels; there is no CPU fallback.  The library never allocates device memory:
 * the caller passes one device workspace of the size gsp2_workspace_bytes reports.
 *
 * Conventions for every call:
 *  - "host" pointers are ordinary CPU memory, read during the call and not kept;
 *  - "device" pointers are CUDA global memory on the current device, owned by the
 *    caller, which must keep them alive until the work queued on the stream ends;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *  - a call returns GSP2_OK or an error code; on error gsp2_last_error(h) gives a
 *    one-line reason, nothing is queued, and the handle stays usable;
 *  - a handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef GSP2_H
#define GSP2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsp2_plan* gsp2_handle;

typedef enum {
  GSP2_OK = 0,
  GSP2_E_ARG = 1,            /* invalid argument: bad CSR, part map, size, pointer */
  GSP2_E_OOM = 2,            /* host allocation failed */
  GSP2_E_STATE = 3,          /* call out of order (no workspace, no forward pass) */
  GSP2_E_CUDA = 4,           /* a CUDA runtime call failed (see gsp2_last_error) */
  GSP2_E_NOT_CONVERGED = 5,  /* device: max_steps reached before the stopping test */
  GSP2_E_TRACE = 6,          /* device: replayed sequence ended with |Tr P - Nocc| > trace_tol */
  GSP2_E_NONFINITE = 7,      /* device: NaN/Inf met in H, the bounds or a trace */
  GSP2_E_WORKSPACE = 8,      /* workspace too small or misaligned (256 bytes) */
  GSP2_E_TIMEOUT = 9         /* device: a bounded wait inside a kernel gave up */
} gsp2_status;

/* Arithmetic of the purification steps.  Traces, bounds and branch decisions are
 * always FP64.  The low-precision modes keep an FP32 master copy of every X_k, run
 * the squarings in that precision (TF32/BF16: tcgen05 tensor cores, FP32 accumulation
 * in TMEM; FP32: CUDA cores), stop when |e| <= max(idem_tol, 16 N u) (u: unit roundoff
 * of one product) and e < 0 or e no longer falls, and finish with
 * `fp64_tail_steps` FP64 steps: the first takes its branch from the trace rule, each
 * further one the opposite branch, so eigenvalues near 0 and near 1 are both purified.
 * The low-precision modes support RECORD only; their adjoint runs in FP32 (see ckpt_every). */
typedef enum {
  GSP2_PREC_FP64 = 0,
  GSP2_PREC_FP32 = 1,   /* FP32 CUDA-core squarings (no tensor cores) */
  GSP2_PREC_TF32 = 2,
  GSP2_PREC_BF16 = 3,
  GSP2_PREC_BF16X3 = 4, /* split operands hi+lo in BF16, three products, FP32 accumulate */
  GSP2_PREC_TF32X3 = 5, /* split operands hi+lo in TF32, three products, FP32 accumulate */
  GSP2_PREC_FP64_EMU = 6, /* FP64 results; every product X X rebuilt from 7 base-2^7 digits of X
                             held in BF16 (28 exact BF16 tensor-core products per tile, groups
                             summed as 64-bit fixed point), master copy in that fixed point */
  GSP2_PREC_FP16X3 = 7  /* split operands hi+lo in FP16 of X 2^14 (22 bits like TF32X3, entries
                           down to 2^-28 in FP16's normal range), three products at the
                           16-bit tensor rate, FP32 accumulate, sums scaled back by 2^-28 */
} gsp2_precision;

typedef enum {
  GSP2_MODE_RECORD = 0, /* choose each branch on the device from the global trace */
  GSP2_MODE_REPLAY = 1  /* apply a given branch sequence (Section 2.1, sequence reuse) */
} gsp2_mode;

typedef struct {
  int32_t max_steps;       /* cap on purification steps (default 45), 1..1024 */
  double idem_tol;         /* stopping gate on e = Tr X - Tr X^2 (default 1e-3): after step i
                              the loop stops when |e_{i-1}| <= idem_tol and e_{i-1} < 0 or
                              e_{i-1} >= e_{i-2} (idempotency no longer improves) */
  double trace_tol;        /* replay check on |Tr P - Nocc| (default 1e-2) */
  int32_t precision;       /* gsp2_precision (default FP64) */
  int32_t fp64_tail_steps; /* FP64 steps after the stopping test, -1..8 (default -1: 0 for the
                              FP64 precision, 2 for the low-precision modes); their first
                              branch follows the trace rule, each further one the opposite */
  int32_t ckpt_every;      /* adjoint: keep every k-th iterate; 0 = no adjoint; -1 (default) =
                              8 for FP64 and FP64_EMU, 0 for the low-precision modes, whose
                              adjoint (k > 0, lp_tail_steps = 0) runs in FP32 from FP32
                              checkpoints, products as FP16 hi + lo on the tensor cores, the
                              FP64 tail steps reversed in FP32 too */
  int32_t use_graph;       /* 1 (default): capture the whole step sequence in a CUDA graph, one
                              per (H, P, alpha, mode, nsteps) of a density call, the two most
                              recently used kept (two alternating buffer pairs replay theirs) */
  int32_t time_steps;      /* 1: record CUDA events around every purification-step launch
                              (read with gsp2_step_times); default 0 */
  int32_t lp_tail_steps;   /* tensor-core precisions: alternating steps in that precision
                              after its loop stops, before the FP64 tail (default 0);
                              lp_tail_steps + fp64_tail_steps <= 8 */
  int32_t tc_schedule;     /* tensor-core steps: 0 (default) persistent, one CTA per SM with two
                              TMEM accumulators so the epilogue of one tile overlaps the
                              next tile's MMAs; 1 = one CTA per tile */
  int32_t report_idem;     /* 1: after each density call, one extra FP64 pass over the final
                              iterates computes the idempotency report idem_fro (default 0) */
  int32_t fp64_tail_emulated; /* low-precision modes: 1 (default) runs the FP64 tail steps with
                                 the products rebuilt from BF16 digits (as GSP2_PREC_FP64_EMU),
                                 0 on the FP64 units */
  int32_t tile_order;      /* order of the 128x128 tiles walked by the persistent kernels
                              (tensor-core steps with tc_schedule = 0, FP64_EMU steps): 0 = parts
                              by descending size, tile t to CTA t mod (number of SMs); 1 (default)
                              = the same list reversed in every other round of SMs, so that
                              each SM's share of the uneven tiles evens out (with few tiles per
                              SM, the CTA that took the largest tile of one round takes the
                              smallest of the next); 2 = that order with the tiles of the last
                              four rounds re-dealt, largest first, to the least loaded CTA of a
                              cost model (columns x padded K), so that the CTAs finish together;
                              set by gsp2_autotune */
  int32_t tile_shape;      /* output tiles of the persistent tensor-core steps: 0 (default)
                              128 x 128; 1 = 128 x 256 (two upper tiles of a row block per
                              MMA, N = 256, halving the loads of the A operand); set by
                              gsp2_autotune */
  int32_t split_k;         /* FP64_EMU steps: 1 = each upper tile's product as two work items, one
                              per half of its K (forward and rebuilt steps: the two halves of the
                              K stages; adjoint reverse steps: Xbar X and X Xbar), their 64-bit
                              partial sums added by the second to finish (more, shorter items for
                              small problems); 0 = one item per tile; -1 (default) = 1 when the
                              plan has at most 512 upper 128-tiles.  Needs every part above 128
                              orbitals (else 0) and 2 x 128 KB of workspace per tile; gsp2_autotune
                              may turn it off.  The 64-bit sums are exact; the group sums of each
                              half are rounded in FP32 like the whole K's, so results agree to the
                              last bits only */
  int32_t tile_claim;      /* persistent 128 x 128 steps (tensor-core steps and reverse steps, FP64_EMU
                              forward and reverse steps): 1 (default) = each CTA takes its first
                              tile by its index and claims every next one from a counter in the
                              workspace, one tile ahead, walking the list of tile_order, so that
                              CTAs that run faster take more tiles; 0 = the static deal (tile t
                              to CTA t mod the number of SMs).  The rebuilt iterates of the
                              adjoint (which may run beside reverse steps), the 128 x 256 tiles
                              and the one-CTA-per-tile schedule keep the static deal.  Set by
                              gsp2_autotune */
} gsp2_options;

/* Per-call report, read back by gsp2_sync_status. */
typedef struct {
  int32_t status;       /* gsp2_status detected on the device for the last density call */
  int32_t steps;        /* purification steps applied */
  int32_t stopped;      /* 1 if the stopping test ended the loop */
  int32_t fp64_steps;   /* of which FP64 steps (low-precision modes) */
  double eps_min;       /* Gershgorin bounds (Section 2.1) */
  double eps_max;
  double trace;         /* Tr P = sum of core diagonal entries of the final iterates */
  double idem;          /* last idempotency error e computed */
  double idem_fro;      /* report_idem = 1: sqrt(sum_k ||(X_k^2 - X_k)[:, cores of k]||_F^2 / N),
                           the idempotency of P column by column (Eq. 3's check); else -1 */
} gsp2_report;

/* Plan sizes, for accounting (flops from the real part sizes). */
typedef struct {
  int64_t n;            /* orbitals */
  int64_t nocc;
  int32_t nparts;
  int32_t max_s;        /* largest core+halo size */
  int64_t sum_s;        /* sum_k s_k */
  double sum_s2;        /* sum_k s_k^2  (elements of one arena) */
  double sum_s3;        /* sum_k s_k^3  (Eq. 5 cost) */
  int64_t nnz_h;
  int64_t nnz_p;        /* sum_k c_k s_k */
  int64_t arena_elems;  /* sum_k ld_k^2 (padded) */
  int64_t ntiles;       /* upper-triangular square tiles per step */
  int32_t tile;         /* square tile edge */
  int32_t ld_pad;       /* padding multiple of ld_k */
  int32_t step_launches;   /* purification-step launches per density call (the loop's) */
  int32_t fp64_tail_steps; /* resolved value of the option */
  int32_t tc_schedule;     /* schedule, tile order and tile shape in use (options, or gsp2_autotune's choice) */
  int32_t tile_order;
  int32_t tile_shape;
  int32_t split_k;         /* 1 if the emulated steps split K into two work items (in use now) */
  int32_t tile_claim;      /* 1 if the persistent steps claim their tiles from a counter */
} gsp2_plan_info;

/* Fill `opt` with the defaults listed above. */
void gsp2_default_options(gsp2_options* opt);

/*
 * Build a plan from the sparsity pattern of H, the partition and the graph G_tau
 * (Section 2.2).  Host-only: validates, builds halos, the per-part vertex lists
 * S_k (cores ascending, then halo ascending), the padded dense layout, the tile work
 * list and the pattern of P.  Allocates host memory only.
 *
 *  n                 orbitals, 1..2^31-1
 *  rowptr, colind    host CSR of H (full symmetric pattern, both triangles), int64
 *                    rowptr[n+1], int32 colind[nnz], columns strictly ascending per
 *                    row, every diagonal entry present, pattern symmetric
 *  nocc              occupied orbitals (N_el = 2 nocc), 0..n
 *  part              host int32[n], part id of each orbital, in [0, nparts)
 *  nparts            number of parts, >= 1, no part may be empty
 *  g_rowptr/g_colind host CSR of G_tau (same format; self loops ignored; must be
 *                    symmetric); both NULL = use the pattern of H
 *  opt               options (NULL = defaults)
 *  out               receives the handle (NULL on error)
 * Errors: GSP2_E_ARG, GSP2_E_OOM; the reason is gsp2_last_error(NULL).
 */
gsp2_status gsp2_create(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t nocc,
                        const int32_t* part, int32_t nparts, const int64_t* g_rowptr,
                        const int32_t* g_colind, const gsp2_options* opt, gsp2_handle* out);

/* Device workspace bytes the plan needs (arenas, tables, checkpoints). */
gsp2_status gsp2_workspace_bytes(gsp2_handle h, size_t* bytes);

/* Attach a caller-owned device workspace of at least gsp2_workspace_bytes bytes,
 * 256-byte aligned, on the current device, and upload the plan tables into it
 * (queued on `stream`).  May be called again to move the plan to another buffer. */
gsp2_status gsp2_bind_workspace(gsp2_handle h, void* d_workspace, size_t bytes, void* stream);

/* Pattern of P in core-column CSC form (host output): column g holds the rows
 * S_{part(g)} in ascending order.  colptr: int64[n+1]; rowind: int32[nnz_p].
 * Either array may be NULL to query only nnz_p. */
gsp2_status gsp2_p_pattern(gsp2_handle h, int64_t* colptr, int32_t* rowind, int64_t* nnz_p);

/* Sizes of the plan; s and c (host int32[nparts], may be NULL) receive s_k and c_k. */
gsp2_status gsp2_plan_query(gsp2_handle h, gsp2_plan_info* info, int32_t* s, int32_t* c);

/*
 * Density matrix P(H) (Sections 1.1, 2.1, 2.2; Eqs. 1-3).  Asynchronous on `stream`.
 *
 *  d_hvals  device double[nnz_h]: values of H on the pattern given to gsp2_create
 *           (symmetric values expected; a new SCF/MD H reuses the plan, Section 1.1)
 *  d_pvals  device double[nnz_p]: output, P on the pattern of gsp2_p_pattern
 *  d_alpha  device int8[max_steps + 8] or NULL.  RECORD: receives the branch sequence
 *           (+1: 2X - X^2, -1: X^2) of the applied steps (tail steps included), zeros
 *           after the last.  REPLAY: the sequence to apply; its length is `nsteps`.
 *  mode     gsp2_mode
 *  nsteps   REPLAY: number of steps to apply (1..max_steps + fp64_tail_steps); RECORD: ignored
 * Host-visible errors are argument/state errors only; numerical outcomes
 * (convergence, trace check, non-finite values) are read with gsp2_sync_status.
 */
gsp2_status gsp2_density(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha,
                         int32_t mode, int32_t nsteps, void* stream);

/* Wait for the last density call and return its device status (GSP2_OK or one of
 * GSP2_E_NOT_CONVERGED / GSP2_E_TRACE / GSP2_E_NONFINITE); `r` may be NULL. */
gsp2_status gsp2_sync_status(gsp2_handle h, gsp2_report* r);

/* Per-step history of the last density call, copied to host after a sync:
 * traces[0..steps] (core traces T_i of X_i), idem[0..steps-1] (e_i), alpha[0..steps-1].
 * `cap` bounds each array; any pointer may be NULL. */
gsp2_status gsp2_history(gsp2_handle h, double* traces, double* idem, int8_t* alpha, int32_t cap);

/* Device time of each purification-step launch of the last density call, in
 * milliseconds, ms[i-1] for step i (1..max_steps); needs time_steps = 1.  Steps after
 * the stopping test return at once and show a few microseconds.  Waits for the call. */
gsp2_status gsp2_step_times(gsp2_handle h, float* ms, int32_t cap);

/*
 * Density for the next H of a sequence (SCF iterations or MD steps): Section 2.1 reuses the
 * recorded sequence of multiplications as long as it still gives the right trace.  With
 * *nsteps > 0 the call replays d_alpha[0 .. *nsteps) (GSP2_MODE_REPLAY) and checks Tr P; when
 * the replayed sequence gives the wrong trace (|Tr P - Nocc| > trace_tol) or *nsteps == 0, it
 * runs GSP2_MODE_RECORD, which chooses the branches afresh and writes them to d_alpha, and
 * sets *nsteps to the steps applied and *recomputed to 1 (else 0).
 *  d_alpha   device int8[max_steps + 8], the sequence carried from call to call
 *  nsteps    in/out, host; 0 on the first call
 * FP64 and FP64_EMU plans only (the branch replay of the low-precision modes is not
 * available).  Synchronises `stream`; returns the device status of the call that produced P.
 */
gsp2_status gsp2_density_reuse(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha,
                               int32_t* nsteps, void* stream, int32_t* recomputed);

/*
 * Dependency graph G_tau from a density matrix (Section 2.2: vertices i and j are adjacent
 * when |P_ij| > tau), for re-planning between SCF or MD steps: the pattern of `d_pvals`
 * (the core-column layout of gsp2_p_pattern) thresholded on the device, symmetrised (an
 * edge when either of P_ij, P_ji is stored and above tau), with every diagonal entry, as a
 * CSR graph with sorted columns that gsp2_create accepts.
 *  g_rowptr  host int64[n + 1], always written
 *  g_colind  host int32[cap]; written when cap >= the number of entries, which is returned
 *            in *nnz either way (call once with cap = 0 to size the buffer)
 * Synchronises `stream`.  Errors: GSP2_E_ARG (tau < 0, NULL outputs), GSP2_E_STATE, GSP2_E_CUDA.
 */
gsp2_status gsp2_threshold_graph(gsp2_handle h, const double* d_pvals, double tau, void* stream, int64_t* g_rowptr,
                                 int32_t* g_colind, int64_t cap, int64_t* nnz);

/* Outcome of gsp2_autotune: the candidates tried and their times. */
typedef struct {
  int32_t ncand;        /* candidates timed (1 when the precision has no choice) */
  int32_t chosen;       /* index of the fastest, now in use */
  int32_t tc_schedule[8];
  int32_t tile_order[8];
  int32_t tile_shape[8];
  double ms[8];         /* median device time of one density call, milliseconds */
  int32_t split_k[8];   /* FP64_EMU: 1 if the candidate splits each tile's K into two work items */
  int32_t tile_claim[8]; /* 1 if the candidate's persistent 128 x 128 steps claim their tiles */
} gsp2_tune_report;

/*
 * Autotuner of the step schedule (batching of uneven parts, not in the paper): times whole
 * density calls (RECORD mode, `trials` >= 1 each after one untimed call) with every candidate
 * that applies to the plan's precision -- tensor-core steps: persistent 128 x 128 tiles in
 * tile orders 0 and 1, each with claimed tiles and with the static deal, 128 x 256 tiles in
 * either order, and one CTA per tile; FP64_EMU steps: the three tile orders with claimed
 * tiles, tile order 2 with the static deal, and for small plans split-K work items;
 * FP64 and FP32: the only schedule -- and keeps the fastest in the plan (gsp2_plan_query
 * reports it).  Every candidate without split-K work items computes bitwise the same P (a
 * tile's arithmetic does not depend on the CTA that runs it); split-K agrees to the last
 * bits.
 *  d_hvals, d_pvals  as for gsp2_density; d_pvals is overwritten
 *  rep               optional output
 * Synchronises `stream`.  Errors: GSP2_E_ARG, GSP2_E_STATE (no workspace), GSP2_E_CUDA, or
 * the device status of a timed call (the plan then keeps the candidate that failed).
 */
gsp2_status gsp2_autotune(gsp2_handle h, const double* d_hvals, double* d_pvals, int32_t trials, void* stream,
                          gsp2_tune_report* rep);

/*
 * Adjoint of P(H): given Pbar = dL/dP on the pattern of P, write Hbar = dL/dH on the
 * pattern of H, through the branch sequence of the last density call (its bounds
 * held fixed).  X^2 steps map Xbar -> Xbar X + X Xbar, 2X - X^2 steps map
 * Xbar -> 2 Xbar - Xbar X - X Xbar; dX0/dH = -1/(eps_max - eps_min) (Eq. 1).
 * Iterates are recomputed from checkpoints kept every `ckpt_every` steps.  FP64 plans
 * run it on the FP64 pipe, FP64_EMU plans from BF16 digit products (Xbar's digits scaled
 * by a power of two per part taken from its row norms), the low-precision plans in FP32
 * with FP16 hi + lo products (Xbar's operands scaled by a power of two per part).
 *  d_pbar  device double[nnz_p]
 *  d_hbar  device double[nnz_h], overwritten; symmetric for a symmetric problem
 * Requires ckpt_every > 0 at create and a completed density call (GSP2_E_STATE).  The sweep
 * covers max_steps (launches for steps the forward did not apply return at once) unless
 * gsp2_sync_status has been called after the density call: then it covers exactly the steps
 * applied, with bitwise the same result.
 */
gsp2_status gsp2_backward(gsp2_handle h, const double* d_pbar, double* d_hbar, void* stream);

/* ---------------------------------------------------------------- re-partitioning
 *
 * Between SCF or MD steps the graph G_tau is refreshed from the new P (Section 1.1, Fig. 1;
 * gsp2_threshold_graph) and may be re-partitioned before the next plan is built.  The cost
 * Section 2.2 gives to a partition is Eq. 5, C = sum_i (c_i + h_i)^3 (core plus halo of
 * every part: the dense work of one squaring).  Host only; no device memory. */
typedef enum {
  GSP2_PARTITION_AUTO = -1,       /* every method that applies; the smallest Eq. 5 cost wins
                                     (ties: the lower method) */
  GSP2_PARTITION_BLOCK = 0,       /* Section 2.3: consecutive indices, sizes differing by at
                                     most one, the larger parts first */
  GSP2_PARTITION_GRAPH_ORDER = 1, /* the same blocks over a breadth-first order of G_tau (each
                                     component from a far vertex, neighbours ascending) */
  GSP2_PARTITION_RCB = 2          /* recursive coordinate bisection over `coords` (longest
                                     extent, count-proportional split, ties by index) */
} gsp2_partition_method;

/* Eq. 5 cost of a partition of G_tau (CSR as for gsp2_create; self loops ignored).
 *  part     host int32[n] in [0, nparts)
 *  cost     output, sum_i (c_i + h_i)^3
 *  sizes    host int32[nparts] or NULL: c_i + h_i
 * GSP2_E_ARG for a bad graph or part id. */
gsp2_status gsp2_partition_cost(int64_t n, const int64_t* g_rowptr, const int32_t* g_colind, const int32_t* part,
                                int32_t nparts, double* cost, int32_t* sizes);

/* A partition of G_tau into nparts non-empty parts (1 <= nparts <= n) by `method`
 * (gsp2_partition_method).  coords: host double[3 n] (x, y, z per vertex) or NULL; needed
 * by GSP2_PARTITION_RCB, used by AUTO when given.  part: host int32[n], output; chosen and
 * cost (may be NULL): the method used and its Eq. 5 cost.  Deterministic. */
gsp2_status gsp2_partition(int64_t n, const int64_t* g_rowptr, const int32_t* g_colind, int32_t nparts,
                           int32_t method, const double* coords, int32_t* part, int32_t* chosen, double* cost);

/* ---------------------------------------------------------------- shard plans
 *
 * One problem's parts split over several GPUs, one process (and plan) per GPU.  Parts are
 * independent except through the branch of every step, which Section 2.1 takes from the
 * trace of the whole iterate, in G-SP2 the sum of all parts' core diagonals (Section 2.2).
 * A shard plan holds the parts of one rank; each of its bookkeeping launches (the gather
 * of X0, every purification step) leaves this rank's partial sums -- core trace of the new
 * iterate and core trace of the square of the old one, 16 bytes -- for the caller to
 * all-gather, and a decide launch adds every rank's partials in rank order and takes the
 * branch, the stopping test and the history exactly as the fused step does.  Every rank
 * sums the same numbers in the same order, so all take bitwise the same branches; with one
 * rank the result is bitwise that of gsp2_density.  A call is:
 *
 *   gsp2_shard_exchanges(h, mode, nsteps, &count);
 *   gsp2_shard_begin(h, H, P, alpha, mode, nsteps, send, s);     exchange 0 queued
 *   for x in 0 .. count-1:
 *     all-gather send (double[2]) of every rank into recv (double[nranks][2]), on s;
 *     gsp2_shard_decide(h, x, recv, nranks, s);
 *     if x + 1 < count: gsp2_shard_step(h, x + 1, send, s);
 *   gsp2_shard_end(h, s);                                        scatter of this rank's P
 *
 * P of a shard plan holds the core columns of its parts (gsp2_p_pattern: the other columns
 * are empty); the ranks' columns are disjoint and together are P.  gsp2_backward gives this
 * rank's share of dL/dH (the parts it holds); the sum over ranks is dL/dH.  gsp2_density,
 * gsp2_density_reuse and gsp2_autotune return GSP2_E_STATE on a shard plan.
 */

/* Parts to ranks by longest processing time first on the Eq. 5 cost s_k^3 (Section 2.2):
 * parts in descending size (ties: lower id first), each to the rank with the least cost so
 * far (ties: lower rank).  Host only, deterministic: every rank computes the same map.
 *  sizes      host int32[nparts], s_k of every part (gsp2_plan_query of a plain plan), >= 1
 *  nranks     1 .. nparts (every rank gets at least one part)
 *  part_rank  host int32[nparts], output
 *  rank_cost  host double[nranks] or NULL: sum of s_k^3 per rank */
gsp2_status gsp2_assign_parts(const int32_t* sizes, int32_t nparts, int32_t nranks, int32_t* part_rank,
                              double* rank_cost);

/* A shard plan: as gsp2_create (same arguments, validation and halos from the whole
 * problem), holding only the parts with part_rank[k] == rank (host int32[nparts], >= 0;
 * the rank must own at least one part), numbered in ascending global order. */
gsp2_status gsp2_create_shard(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t nocc,
                              const int32_t* part, int32_t nparts, const int64_t* g_rowptr, const int32_t* g_colind,
                              const int32_t* part_rank, int32_t rank, const gsp2_options* opt, gsp2_handle* out);

/* Rank of a shard plan (0 for a plain one), the problem's part count, and the global id
 * of each part the plan holds (host int32[gsp2_plan_info.nparts]); pointers may be NULL. */
gsp2_status gsp2_shard_info(gsp2_handle h, int32_t* rank, int32_t* nparts_global, int32_t* part_ids);

/* Number of exchanges of a shard density call: 1 (X0) + the step launches (RECORD: the
 * loop's max_steps plus tail steps; REPLAY: nsteps, FP64 precisions only). */
gsp2_status gsp2_shard_exchanges(gsp2_handle h, int32_t mode, int32_t nsteps, int32_t* count);

/* Opens a shard density call (arguments as gsp2_density; the buffers must stay valid until
 * gsp2_shard_end) and queues the bounds and the gather of X0; d_send (device double[2])
 * receives this rank's partial of exchange 0.  A rank whose launches met NaN/Inf or a
 * timed-out wait sends NaN, so that every rank's sum is non-finite and all stop. */
gsp2_status gsp2_shard_begin(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha, int32_t mode,
                             int32_t nsteps, double* d_send, void* stream);

/* Bookkeeping of exchange x (0 .. count-1) from d_recv (device double[nranks][2], the
 * partials of ranks 0 .. nranks-1 in order), summed in rank order.  Must follow
 * gsp2_shard_begin (x = 0) or gsp2_shard_step(x); GSP2_E_STATE otherwise. */
gsp2_status gsp2_shard_decide(gsp2_handle h, int32_t x, const double* d_recv, int32_t nranks, void* stream);

/* Queues the launches up to the bookkeeping of exchange x (1 .. count-1), the purification
 * step x and what prepares it; d_send receives this rank's partial.  Must follow
 * gsp2_shard_decide(x - 1). */
gsp2_status gsp2_shard_step(gsp2_handle h, int32_t x, double* d_send, void* stream);

/* Closes the call after gsp2_shard_decide(count - 1): scatter of this rank's core columns
 * into d_pvals, the branch sequence into d_alpha (RECORD).  Then gsp2_sync_status,
 * gsp2_history and gsp2_backward apply as after gsp2_density. */
gsp2_status gsp2_shard_end(gsp2_handle h, void* stream);

/*
 * Allocation-free Gershgorin bounds (the paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory, such as code running in
 * another framework's memory pool or a plugin barred from growing the process's
 * device footprint).  Computes d_bounds[0] = min_i (A_ii - sum_{j!=i} |A_ij|) and
 * d_bounds[1] = max_i (A_ii + sum_{j!=i} |A_ij|) of a CSR matrix, the same bounds
 * gsp2_density uses, with no cudaMalloc/cudaFree and no allocating library call.
 *
 *  n         rows, 1 .. 1,048,576 (4096 blocks of 256 rows); larger n -> GSP2_E_ARG
 *  d_rowptr  device int64[n+1]; d_colind device int32[nnz]; d_vals device double[nnz]
 *            (each row's diagonal entry stored once; rows may be in any column order)
 *  d_bounds  device double[2], output
 *  stream    cudaStream_t as void*; the call is asynchronous
 * Returns GSP2_E_ARG for a bad size or a NULL pointer, GSP2_E_CUDA if a CUDA call fails
 * (no message is stored).  A NaN anywhere in d_vals, or an Inf - Inf radius, gives NaN
 * bounds; an infinite value otherwise gives infinite bounds.
 *
 * Its scratch (one 16-byte partial per block and a counter, about 64 KB) is a fixed
 * device array inside the library, held on every GPU that loads the library until
 * the process exits.  All calls on a device share that array: calls that can overlap
 * on the GPU (different streams without ordering) race and must not be issued.  Every
 * call made outside a CUDA stream capture looks the array's device address up afresh
 * (so a context re-created by cudaDeviceReset is followed); a call inside a capture uses
 * the address an earlier call on the same device found, so make the first call on each
 * device outside any capture.
 */
gsp2_status gsp2_bounds_noalloc(int64_t n, const int64_t* d_rowptr, const int32_t* d_colind,
                                const double* d_vals, double* d_bounds, void* stream);

/* Last error message of the handle; with h == NULL, the reason the last failed
 * gsp2_create on the calling thread gave. */
const char* gsp2_last_error(gsp2_handle h);

/* Release the plan (host memory and CUDA graphs; the workspace stays the caller's). */
void gsp2_destroy(gsp2_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GSP2_H */
