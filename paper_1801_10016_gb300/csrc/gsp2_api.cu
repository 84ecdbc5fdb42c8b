// C ABI of the G-SP2 library: plan construction on the host (validation, halos,
// padded layout, work lists, pattern of P), workspace binding, and the queued step
// sequence of a density call, captured once into a CUDA graph and replayed.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/gsp2.h"
#include "gsp2_internal.cuh"
#include "gsp2_kernels.h"

using namespace gsp2;

namespace {

constexpr int BOUNDS_BLOCKS = 608;  // 152 SMs x 4

struct WsLayout {
  size_t parts, S, perm, invperm, tiles, tc_tiles, tc_wide, tc_wide_nb, gblocks, gblocks_ld, sblocks, pcolptr, rowptr,
      colind;
  size_t locptr, loc;  // the gathers' local indices of the stored entries of the rows S_k[j]
  size_t x0;           // Eq. 1 on the stored entries of H (FP64, per P-build)
  size_t memptr, mempart, memloc;
  // low-precision paths
  size_t mf[2];        // FP32 master copies of X (ping-pong)
  size_t op_hi[2];     // operand arenas (BF16 or TF32), ping-pong
  size_t op_lo[2];     // split-mode low parts
  size_t maps;         // CUtensorMap[2 buffers][hi, lo][nparts]
  size_t maps_mn;      // 16-bit kinds: the same with MN-major boxes (upper tiles only kept)
  size_t master_of_step;
  size_t d[2];         // FP64 arenas of the tail steps
  // FP64 products from BF16 digits
  size_t oz_slice[2][OZ_SLICES];  // BF16 digit arenas, two buffers (read / written by a step)
  size_t oz_maps;                 // CUtensorMap[2][OZ_SLICES][nparts], K-major boxes
  size_t oz_maps_mn;              // the same, MN-major boxes
  size_t oz_acc;                  // int64[OZ_MAX_GRID][128 * 128] partial sums of the emulated step
  // emulated FP64 adjoint: digit sets 0..k-1 hold X_{c0+j} of a checkpoint segment, set k
  // holds Xbar / 2^sig; their tensor maps; row norms and per-part scales of Xbar
  std::vector<size_t> adj_dig;    // adj_dig[set * OZ_SLICES + t]
  size_t adj_maps, adj_maps_mn;   // CUtensorMap[k + 1][OZ_SLICES][nparts]
  size_t adj_norm, adj_sig;       // double[sum of s] (the seed's row norms), int32[nparts]
  size_t adj_normf;               // float[sum of s]: the reverse steps' row norms on their grid
  size_t split_acc, split_cnt;    // split-K reverse steps: int64[2 tiles][128 x 128], uint32[tiles]
  size_t split_items;             // int32[2 tiles]: the order in which the CTAs take the items
  size_t tile_ctr;                // uint32: next tile of the emulated forward steps' dynamic schedule
  // FP32 adjoint of the low-precision plans: FP16 (hi, lo) operand arenas aop[2 set + lo],
  // sets 0..S-1 for rebuilt iterates, S and S + 1 for Xbar's ping-pong (in the FP64 tail
  // arenas d[0], d[1], which the backward does not need); their tensor maps; Xbar's
  // per-part scale exponents and maxima
  std::vector<size_t> aop;
  size_t aop_maps;                // CUtensorMap[2 (S + 2)][nparts]
  size_t aop_maps_mn;             // the same, MN-major boxes
  size_t xb_sig, xb_max;          // int32[2][nparts] (scales read, written), uint32[nparts]
  size_t mask;                    // uint8[nnz_p]: |P| > tau flags of gsp2_threshold_graph
  std::vector<size_t> tailf;      // low-precision adjoint: FP32 iterates of the FP64 tail, recomputed
  size_t slots, rslots, state, alpha, traces, idem, step_arena;
  size_t xchg;                 // ShardSlot of a shard plan's exchanges
  size_t arena0, arena1;       // ping-pong iterates
  std::vector<size_t> ckpt;    // X_0, X_k, X_2k, ... (adjoint checkpoints)
  std::vector<size_t> seg;     // seg[j] = X_{c0+j}, j = 1..k-1, recomputed in the adjoint
  std::vector<size_t> seg2;    // the same for the other checkpoint segment (overlapped adjoint)
  size_t oz_acc2;              // the side stream's per-CTA scratch tiles (overlapped adjoint)
  size_t xb0, xb1;             // adjoint Xbar ping-pong
  size_t total;
};

struct GraphKey {
  const void* h;
  void* p;
  void* a;
  int mode, nsteps;
  bool operator==(const GraphKey& o) const {
    return h == o.h && p == o.p && a == o.a && mode == o.mode && nsteps == o.nsteps;
  }
};

}  // namespace

struct gsp2_plan {
  int64_t n = 0, nocc = 0, nnz_h = 0;
  int32_t nparts = 0;
  gsp2_options opt{};
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<PartDesc> parts;
  std::vector<int32_t> S, perm, invperm;
  std::vector<int64_t> memptr;           // vertex -> parts holding it (CSR)
  std::vector<int64_t> locptr;           // per entry of S: its row's first slot in the local-index table
  int64_t nloc = 0;                      // slots of that table (stored entries of all rows S_k[j])
  std::vector<int32_t> mempart, memloc;  // part id, local index in S_part
  std::vector<Tile> tiles;                 // 64x64 upper tiles (CUDA-core steps)
  std::vector<Tile> tc_tiles;              // 128x128 upper tiles (tensor-core steps)
  std::vector<Tile> tc_order;              // tc_tiles in the order of opt.tile_order (uploaded)
  std::vector<Tile> tc_wide;               // tile_shape 1: one or two column blocks per tile
  std::vector<int8_t> tc_wide_nb;
  std::vector<Tile> tcw_order;             // tc_wide / tc_wide_nb in the order of opt.tile_order
  std::vector<int8_t> tcw_nb_order;
  std::vector<int32_t> split_items;        // split reverse steps: item codes 2 i + half (i into tc_order)
  std::vector<size_t> mf_of_step;          // low precision: FP32 arena of iterate i (checkpoints or ping-pong)
  std::vector<ColBlock> gblocks, sblocks;  // gather (to nt*64) and scatter (cores) columns
  std::vector<ColBlock> gblocks_ld;        // low-precision gather: every column up to ld
  int32_t nslots_tc = 0;
  int32_t total_steps = 0;  // FP64 path: max_steps + tail steps (static launches of a call)
  bool use_oz = false;      // FP64 products from BF16 digits (fp64e steps or emulated tail steps)
  bool split_ok = false;    // emulated steps: buffers for split-K work items are in the workspace
  bool split_on = false;    // emulated steps split each tile's K into two work items
  std::vector<int64_t> pcolptr;
  std::vector<int32_t> prowind;
  int32_t nslots = 0, max_s = 0, min_s = 0;
  int64_t arena_elems = 0, sum_s = 0;
  double sum_s2 = 0, sum_s3 = 0;
  WsLayout L{};
  char* ws = nullptr;
  size_t ws_size = 0;
  int device = -1;
  int num_sms = 0;
  cudaStream_t cap_stream = nullptr;
  // emulated adjoint of small plans: the iterates of the next checkpoint segment are rebuilt
  // on a side stream while the reverse steps of the current one run (two digit-set buffers)
  bool adj_overlap = false;
  cudaStream_t side_stream = nullptr;
  std::vector<cudaEvent_t> bev;  // fork, per segment: rebuilt, reversed
  // forward graphs, one per (H, P, alpha, mode, nsteps) key, the two most recent kept (a
  // caller alternating two buffer pairs, e.g. to overlap copies with compute, replays both)
  struct ForwardGraph {
    GraphKey key{};
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
  } fg[2];
  uint64_t fg_clock = 0;
  cudaGraphExec_t bexec = nullptr;  // adjoint graph
  const void* bkey_pbar = nullptr;
  void* bkey_hbar = nullptr;
  std::vector<size_t> step_arena_off;  // workspace offset of the arena holding X_i
  std::vector<cudaEvent_t> ev;  // 2 per step when time_steps is set
  bool have_forward = false;
  // steps the last density call applied, once gsp2_sync_status has read them (-1: unknown);
  // the adjoint then schedules exactly those steps instead of max_steps
  int32_t known_steps = -1;
  int32_t bkey_m = -1;
  // shard plans (gsp2_create_shard): the plan holds the parts one rank owns, numbered in
  // ascending global order; part_global maps them back.  A plain plan owns every part.
  bool shard = false;
  int32_t shard_rank = 0, nparts_global = 0;
  std::vector<int32_t> part_global;
  // exchange sequence of the shard density call in progress: its buffers, and the next
  // call expected (begin, then decide 0, step 1, decide 1, ..., end)
  struct ShardCall {
    const double* hv = nullptr;
    double* pv = nullptr;
    int8_t* alpha = nullptr;
    int mode = 0, nsteps = 0, count = 0;
    int next = -1;  // -1: no call open; 2x: decide x expected; 2x + 1: step x + 1 (or end)
  } sx;
  std::string err;
};

// reason of the last failed gsp2_create on this thread (read with gsp2_last_error(NULL))
static thread_local std::string t_create_err = "invalid handle";

static gsp2_status fail(gsp2_plan* h, gsp2_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

static gsp2_status cuda_fail(gsp2_plan* h, cudaError_t e, const char* where) {
  return fail(h, GSP2_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CU(h, call)                                     \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// history slots beyond max_steps: the FP64 tail steps of the low-precision paths
constexpr int HIST_EXTRA = 16;
constexpr int MAX_TAIL = 8;

// FP64 results: native FP64 steps or FP64 products rebuilt from BF16 digits
static bool fp64_like(int prec) { return prec == GSP2_PREC_FP64 || prec == GSP2_PREC_FP64_EMU; }

// tensor-core operand kind (-1: FP32 CUDA cores, 0: BF16, 1: TF32, 2: FP16 of x 2^14) and
// products per tile
static int prec_kind(int prec) {
  if (prec == GSP2_PREC_FP32) return -1;
  if (prec == GSP2_PREC_BF16 || prec == GSP2_PREC_BF16X3) return 0;
  return prec == GSP2_PREC_FP16X3 ? 2 : 1;
}
static int prec_nprod(int prec) {
  return (prec == GSP2_PREC_BF16X3 || prec == GSP2_PREC_TF32X3 || prec == GSP2_PREC_FP16X3) ? 3 : 1;
}
// unit roundoff of one product of the low-precision phase
static double prec_unit(int prec) {
  switch (prec) {
    case GSP2_PREC_FP32: return 0x1p-24;
    case GSP2_PREC_TF32: return 0x1p-11;
    case GSP2_PREC_BF16: return 0x1p-8;
    case GSP2_PREC_BF16X3: return 0x1p-16;
    case GSP2_PREC_TF32X3: return 0x1p-22;
    case GSP2_PREC_FP16X3: return 0x1p-22;
    default: return 0x1p-53;
  }
}

static std::string check_csr(int64_t n, const int64_t* rowptr, const int32_t* colind, bool need_diag,
                             const char* what) {
  if (!rowptr) return std::string(what) + ": rowptr is NULL";
  if (rowptr[0] != 0) return std::string(what) + ": rowptr[0] != 0";
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return std::string(what) + ": rowptr not monotone at row " + std::to_string(i);
  }
  if (rowptr[n] > 0 && !colind) return std::string(what) + ": colind is NULL";
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int32_t c = colind[p];
      if (c < 0 || c >= n) return std::string(what) + ": column index out of range in row " + std::to_string(i);
      if (p > rowptr[i] && colind[p - 1] >= c)
        return std::string(what) + ": columns not strictly ascending in row " + std::to_string(i);
      if (c == i) diag = true;
    }
    if (need_diag && !diag) return std::string(what) + ": diagonal entry missing in row " + std::to_string(i);
  }
  return "";
}

static bool has_entry(const int64_t* rowptr, const int32_t* colind, int64_t i, int32_t j) {
  const int32_t* b = colind + rowptr[i];
  const int32_t* e = colind + rowptr[i + 1];
  const int32_t* q = std::lower_bound(b, e, j);
  return q != e && *q == j;
}

extern "C" void gsp2_default_options(gsp2_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->max_steps = 45;
  o->idem_tol = 1e-3;
  o->trace_tol = 1e-2;
  o->precision = GSP2_PREC_FP64;
  o->fp64_tail_steps = -1;
  o->ckpt_every = -1;
  o->use_graph = 1;
  o->fp64_tail_emulated = 1;
  o->tile_order = 1;
  o->split_k = -1;
  o->tile_claim = 1;
}

extern "C" const char* gsp2_last_error(gsp2_handle h) { return h ? h->err.c_str() : t_create_err.c_str(); }

static void build_layout(gsp2_plan* h) {
  WsLayout& L = h->L;
  h->use_oz = h->opt.precision == GSP2_PREC_FP64_EMU ||
              (!fp64_like(h->opt.precision) && h->opt.fp64_tail_steps > 0 && h->opt.fp64_tail_emulated);
  h->total_steps = h->opt.max_steps + (fp64_like(h->opt.precision) ? h->opt.fp64_tail_steps : 0);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.parts = take(h->parts.size() * sizeof(PartDesc));
  L.S = take(h->S.size() * sizeof(int32_t));
  L.perm = take(h->perm.size() * sizeof(int32_t));
  L.invperm = take(h->invperm.size() * sizeof(int32_t));
  L.memptr = take(h->memptr.size() * sizeof(int64_t));
  L.mempart = take(h->mempart.size() * sizeof(int32_t));
  L.memloc = take(h->memloc.size() * sizeof(int32_t));
  L.tiles = take(h->tiles.size() * sizeof(Tile));
  L.tc_tiles = take(h->tc_tiles.size() * sizeof(Tile));
  L.tc_wide = take(h->tc_wide.size() * sizeof(Tile));
  L.tc_wide_nb = take(h->tc_wide_nb.size());
  L.gblocks = take(h->gblocks.size() * sizeof(ColBlock));
  L.gblocks_ld = take(h->gblocks_ld.size() * sizeof(ColBlock));
  L.sblocks = take(h->sblocks.size() * sizeof(ColBlock));
  L.pcolptr = take(h->pcolptr.size() * sizeof(int64_t));
  L.rowptr = take(h->rowptr.size() * sizeof(int64_t));
  L.colind = take(h->colind.size() * sizeof(int32_t));
  h->locptr.resize(h->S.size());
  h->nloc = 0;
  for (size_t q = 0; q < h->S.size(); ++q) {
    h->locptr[q] = h->nloc;
    h->nloc += h->rowptr[(size_t)h->S[q] + 1] - h->rowptr[(size_t)h->S[q]];
  }
  L.locptr = take(h->locptr.size() * sizeof(int64_t));
  L.loc = take((size_t)h->nloc * sizeof(int32_t));
  L.x0 = take(h->colind.size() * sizeof(double));
  const size_t nsl = std::max<size_t>({(size_t)h->nslots, (size_t)h->nslots_tc, h->gblocks.size(),
                                        h->gblocks_ld.size(), (size_t)BOUNDS_BLOCKS, 1});
  L.slots = take(nsl * sizeof(double2));
  L.rslots = take(std::max<size_t>(h->tiles.size(), 1) * sizeof(double));
  L.state = take(sizeof(DevState));
  L.tile_ctr = take(sizeof(uint32_t));
  L.xchg = take(sizeof(ShardSlot));
  L.alpha = take((size_t)h->opt.max_steps + HIST_EXTRA);
  L.traces = take(((size_t)h->opt.max_steps + HIST_EXTRA) * sizeof(double));
  L.idem = take(((size_t)h->opt.max_steps + HIST_EXTRA) * sizeof(double));
  L.step_arena = take(((size_t)h->total_steps + 1) * sizeof(double*));
  L.master_of_step = take(((size_t)h->opt.max_steps + 1 + MAX_TAIL) * sizeof(float*));
  L.mask = take((size_t)h->pcolptr[(size_t)h->n]);
  const size_t ab = (size_t)h->arena_elems * sizeof(double);
  const int prec = h->opt.precision;
  if (!fp64_like(prec)) {
    // low precision: FP32 masters, operands, tensor maps, FP64 tail arenas; for the FP32
    // adjoint, FP32 checkpoints every k steps, k - 1 segment arenas, two Xbar arenas and the
    // recomputed tail iterates
    const size_t af = (size_t)h->arena_elems * sizeof(float);
    L.mf[0] = take(af);
    L.mf[1] = take(af);
    const int k = h->opt.ckpt_every;
    L.ckpt.clear();
    L.seg.clear();
    L.seg2.clear();
    L.tailf.clear();
    L.aop.clear();
    L.xb0 = L.xb1 = L.aop_maps = L.aop_maps_mn = L.xb_sig = L.xb_max = 0;
    // small plans rebuild the next checkpoint segment on a side stream during the reverse
    // steps of the current one: a second buffer of k operand sets and k - 1 segment arenas
    h->adj_overlap = k > 1 && h->tc_tiles.size() <= 512;
    if (k > 0) {
      for (int c = 0; c <= h->opt.max_steps / k; ++c) L.ckpt.push_back(take(af));
      for (int j = 1; j < k; ++j) L.seg.push_back(take(af));
      if (h->adj_overlap)
        for (int j = 1; j < k; ++j) L.seg2.push_back(take(af));
      L.xb0 = take(af);
      L.xb1 = take(af);
      for (int t = 0; t < h->opt.fp64_tail_steps; ++t) L.tailf.push_back(take(af));
      const int nsets = std::max(k, h->opt.fp64_tail_steps) + (h->adj_overlap ? k : 0);
      for (int q = 0; q < 2 * nsets; ++q) L.aop.push_back(take((size_t)h->arena_elems * 2));
      L.aop_maps = take((size_t)2 * (nsets + 2) * h->parts.size() * 128);
      L.aop_maps_mn = take((size_t)2 * (nsets + 2) * h->parts.size() * 128);
      L.xb_sig = take(2 * h->parts.size() * sizeof(int32_t));
      L.xb_max = take(h->parts.size() * sizeof(uint32_t));
    }
    h->mf_of_step.assign((size_t)h->opt.max_steps + 1 + MAX_TAIL, 0);
    for (size_t i = 0; i < h->mf_of_step.size(); ++i)
      h->mf_of_step[i] = (k > 0 && (int)i <= h->opt.max_steps && i % (size_t)k == 0) ? L.ckpt[i / k] : L.mf[i & 1];
    const int kind = prec_kind(prec), nprod = prec_nprod(prec);
    const size_t es = kind == 1 ? 4 : 2;
    L.op_hi[0] = L.op_hi[1] = L.op_lo[0] = L.op_lo[1] = 0;
    if (kind >= 0) {
      L.op_hi[0] = take((size_t)h->arena_elems * es);
      L.op_hi[1] = take((size_t)h->arena_elems * es);
      if (nprod == 3) {
        L.op_lo[0] = take((size_t)h->arena_elems * es);
        L.op_lo[1] = take((size_t)h->arena_elems * es);
      }
      L.maps = take(4 * h->parts.size() * 128);
      L.maps_mn = kind == 1 ? 0 : take(4 * h->parts.size() * 128);
    }
    L.d[0] = take(ab);
    L.d[1] = take(ab);
    if (k > 0)
      for (int b = 0; b < 2; ++b) {
        L.aop.push_back(L.d[b]);
        L.aop.push_back(L.d[b] + (size_t)h->arena_elems * 2);
      }
    if (h->use_oz) {
      for (int b = 0; b < 2; ++b)
        for (int t = 0; t < OZ_SLICES; ++t) L.oz_slice[b][t] = take((size_t)h->arena_elems * 2);
      L.oz_maps = take((size_t)2 * OZ_SLICES * h->parts.size() * 128);
      L.oz_maps_mn = take((size_t)2 * OZ_SLICES * h->parts.size() * 128);
      L.oz_acc = take((size_t)OZ_MAX_GRID * 128 * 128 * 8);
    }
    L.arena0 = L.d[0];
    L.arena1 = L.d[1];
    L.total = o;
    h->step_arena_off.assign((size_t)h->opt.max_steps + 1, L.d[0]);
    return;
  }
  L.arena0 = take(ab);
  L.arena1 = take(ab);
  const int k = h->opt.ckpt_every;
  L.ckpt.clear();
  L.seg.clear();
  L.xb0 = L.xb1 = 0;
  if (k > 0) {
    for (int c = 0; c <= h->total_steps / k; ++c) L.ckpt.push_back(take(ab));
    for (int j = 1; j < k; ++j) L.seg.push_back(take(ab));
    L.xb0 = take(ab);
    L.xb1 = take(ab);
  }
  if (h->use_oz) {
    for (int b = 0; b < 2; ++b)
      for (int t = 0; t < OZ_SLICES; ++t) L.oz_slice[b][t] = take((size_t)h->arena_elems * 2);
    L.oz_maps = take((size_t)2 * OZ_SLICES * h->parts.size() * 128);
    L.oz_maps_mn = take((size_t)2 * OZ_SLICES * h->parts.size() * 128);
    L.oz_acc = take((size_t)OZ_MAX_GRID * 128 * 128 * 8);
  }
  L.adj_dig.clear();
  L.adj_maps = L.adj_maps_mn = L.adj_norm = L.adj_sig = L.adj_normf = 0;
  L.split_acc = L.split_cnt = L.split_items = 0;
  L.seg2.clear();
  L.oz_acc2 = 0;
  h->adj_overlap = h->opt.precision == GSP2_PREC_FP64_EMU && k > 1 && h->tc_tiles.size() <= 512;
  // split-K work items: FP64_EMU plans whose parts all exceed 128 orbitals (so that both K
  // halves of every pass hold at least one stage)
  h->split_ok = h->opt.precision == GSP2_PREC_FP64_EMU && h->min_s > 128 &&
                (h->opt.split_k == 1 || (h->opt.split_k < 0 && h->tc_tiles.size() <= 512));
  h->split_on = h->split_ok;
  if (h->split_ok) {
    L.split_acc = take(2 * h->tc_tiles.size() * 128 * 128 * sizeof(long long));
    L.split_cnt = take(h->tc_tiles.size() * sizeof(uint32_t));
    L.split_items = take(2 * h->tc_tiles.size() * sizeof(int32_t));
  }
  if (h->use_oz && k > 0) {
    // digit sets: the iterates of a checkpoint segment (k sets; two buffers of k when the
    // rebuilds overlap the reverse steps), then Xbar / 2^sig
    const int nsets = (h->adj_overlap ? 2 * k : k) + 1;
    for (int set = 0; set < nsets; ++set)
      for (int t = 0; t < OZ_SLICES; ++t) L.adj_dig.push_back(take((size_t)h->arena_elems * 2));
    L.adj_maps = take((size_t)nsets * OZ_SLICES * h->parts.size() * 128);
    L.adj_maps_mn = take((size_t)nsets * OZ_SLICES * h->parts.size() * 128);
    if (h->adj_overlap) {
      for (int j = 1; j < k; ++j) L.seg2.push_back(take(ab));
      L.oz_acc2 = take((size_t)OZ_MAX_GRID * 128 * 128 * 8);
    }
    L.adj_norm = take(h->S.size() * sizeof(double));
    L.adj_normf = take(h->S.size() * sizeof(float));
    L.adj_sig = take(h->parts.size() * sizeof(int32_t));
  }
  L.total = o;
  // arena of each iterate X_i: checkpoints where i is a multiple of k, else ping-pong
  h->step_arena_off.assign((size_t)h->total_steps + 1, 0);
  for (int i = 0; i <= h->total_steps; ++i) {
    if (k > 0 && i % k == 0) h->step_arena_off[i] = L.ckpt[i / k];
    else h->step_arena_off[i] = (i & 1) ? L.arena1 : L.arena0;
  }
}

// Plan over the parts that `part_rank` assigns to `rank` (every part when part_rank is NULL).
static gsp2_status create_plan(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t nocc,
                               const int32_t* part, int32_t nparts, const int64_t* g_rowptr, const int32_t* g_colind,
                               const int32_t* part_rank, int32_t rank, const gsp2_options* opt, gsp2_handle* out) {
  if (!out) return GSP2_E_ARG;
  *out = nullptr;
  gsp2_plan* h = new (std::nothrow) gsp2_plan();
  if (!h) return GSP2_E_OOM;
  auto bail = [&](gsp2_status s, const std::string& m) {
    t_create_err = m;
    delete h;
    return s;
  };
  try {
    if (opt) h->opt = *opt; else gsp2_default_options(&h->opt);
    const gsp2_options& o = h->opt;
    if (n < 1 || n > INT32_MAX) return bail(GSP2_E_ARG, "n out of range");
    if (nocc < 0 || nocc > n) return bail(GSP2_E_ARG, "nocc must be in [0, n]");
    if (nparts < 1 || nparts > n) return bail(GSP2_E_ARG, "nparts must be in [1, n]");
    if (!part) return bail(GSP2_E_ARG, "part is NULL");
    if (o.max_steps < 1 || o.max_steps > 1024) return bail(GSP2_E_ARG, "max_steps must be in [1, 1024]");
    if (!(o.idem_tol >= 0.0) || !(o.trace_tol >= 0.0)) return bail(GSP2_E_ARG, "tolerances must be >= 0");
    if (o.precision < GSP2_PREC_FP64 || o.precision > GSP2_PREC_FP16X3) return bail(GSP2_E_ARG, "unknown precision");
    if (o.fp64_tail_steps < -1 || o.fp64_tail_steps > MAX_TAIL)
      return bail(GSP2_E_ARG, "fp64_tail_steps must be in [-1, 8]");
    if (h->opt.fp64_tail_steps < 0) h->opt.fp64_tail_steps = fp64_like(o.precision) ? 0 : 2;
    if (o.lp_tail_steps < 0 || o.fp64_tail_steps + o.lp_tail_steps > MAX_TAIL)
      return bail(GSP2_E_ARG, "lp_tail_steps must be >= 0 with lp_tail_steps + fp64_tail_steps <= 8");
    if (o.tc_schedule < 0 || o.tc_schedule > 1) return bail(GSP2_E_ARG, "tc_schedule must be 0 or 1");
    if (o.tile_order < 0 || o.tile_order > 2) return bail(GSP2_E_ARG, "tile_order must be 0, 1 or 2");
    if (o.tile_shape < 0 || o.tile_shape > 1) return bail(GSP2_E_ARG, "tile_shape must be 0 or 1");
    if (o.split_k < -1 || o.split_k > 1) return bail(GSP2_E_ARG, "split_k must be -1, 0 or 1");
    if (o.tile_claim < 0 || o.tile_claim > 1) return bail(GSP2_E_ARG, "tile_claim must be 0 or 1");
    if (o.lp_tail_steps > 0 && (fp64_like(o.precision) || o.precision == GSP2_PREC_FP32))
      return bail(GSP2_E_ARG, "lp_tail_steps needs a tensor-core precision");
    if (o.ckpt_every < -1) return bail(GSP2_E_ARG, "ckpt_every must be >= -1");
    if (h->opt.ckpt_every < 0) h->opt.ckpt_every = fp64_like(o.precision) ? 8 : 0;
    if (!fp64_like(o.precision) && o.ckpt_every > 0 && o.lp_tail_steps > 0)
      return bail(GSP2_E_ARG, "the low-precision adjoint (ckpt_every > 0) needs lp_tail_steps = 0");
    if ((g_rowptr == nullptr) != (g_colind == nullptr)) return bail(GSP2_E_ARG, "graph: give both arrays or neither");
    std::string m = check_csr(n, rowptr, colind, true, "H");
    if (!m.empty()) return bail(GSP2_E_ARG, m);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (!has_entry(rowptr, colind, colind[p], (int32_t)i))
          return bail(GSP2_E_ARG, "H pattern is not symmetric at (" + std::to_string(i) + ", " +
                                      std::to_string(colind[p]) + ")");
    const int64_t* grp = g_rowptr ? g_rowptr : rowptr;
    const int32_t* gci = g_rowptr ? g_colind : colind;
    if (g_rowptr) {
      m = check_csr(n, g_rowptr, g_colind, false, "graph");
      if (!m.empty()) return bail(GSP2_E_ARG, m);
    }
    h->n = n;
    h->nocc = nocc;
    h->nparts = nparts;
    h->nnz_h = rowptr[n];
    h->rowptr.assign(rowptr, rowptr + n + 1);
    h->colind.assign(colind, colind + rowptr[n]);

    // cores per part (ascending by construction)
    std::vector<std::vector<int32_t>> core(nparts), halo(nparts);
    for (int64_t i = 0; i < n; ++i) {
      const int32_t k = part[i];
      if (k < 0 || k >= nparts) return bail(GSP2_E_ARG, "part id out of range at vertex " + std::to_string(i));
      core[k].push_back((int32_t)i);
    }
    for (int32_t k = 0; k < nparts; ++k)
      if (core[k].empty()) return bail(GSP2_E_ARG, "part " + std::to_string(k) + " is empty");
    // the parts this plan holds: all, or those of `rank` (local index = rank of the global id)
    std::vector<int32_t> local(nparts, -1);
    if (part_rank) {
      for (int32_t k = 0; k < nparts; ++k) {
        if (part_rank[k] < 0) return bail(GSP2_E_ARG, "part_rank[" + std::to_string(k) + "] is negative");
        if (part_rank[k] == rank) {
          local[k] = (int32_t)h->part_global.size();
          h->part_global.push_back(k);
        }
      }
      if (h->part_global.empty()) return bail(GSP2_E_ARG, "rank " + std::to_string(rank) + " owns no part");
      h->shard = true;
      h->shard_rank = rank;
    } else {
      for (int32_t k = 0; k < nparts; ++k) {
        local[k] = k;
        h->part_global.push_back(k);
      }
    }
    h->nparts_global = nparts;
    const int32_t nloc = (int32_t)h->part_global.size();
    // halo: vertices outside part k adjacent (out-edges of G_tau) to a core of k
    std::vector<int32_t> stamp(n, -1);
    for (int32_t k : h->part_global) {
      for (int32_t u : core[k])
        for (int64_t p = grp[u]; p < grp[u + 1]; ++p) {
          const int32_t v = gci[p];
          if (part[v] != k && stamp[v] != k) {
            stamp[v] = k;
            halo[k].push_back(v);
          }
        }
      std::sort(halo[k].begin(), halo[k].end());
    }
    // layout
    h->nparts = nloc;
    h->parts.resize(nloc);
    int64_t off = 0, soff = 0;
    for (int32_t kl = 0; kl < nloc; ++kl) {
      const int32_t k = h->part_global[kl];
      PartDesc& d = h->parts[kl];
      d.c = (int32_t)core[k].size();
      d.s = d.c + (int32_t)halo[k].size();
      d.ld = (d.s + LD_PAD - 1) / LD_PAD * LD_PAD;
      d.nt = (d.s + SQ_TILE - 1) / SQ_TILE;
      d.off = off;
      d.soff = soff;
      off += (int64_t)d.ld * d.ld;
      soff += d.s;
      h->max_s = std::max(h->max_s, d.s);
      h->min_s = kl == 0 ? d.s : std::min(h->min_s, d.s);
      h->sum_s2 += (double)d.s * d.s;
      h->sum_s3 += (double)d.s * d.s * d.s;
      h->S.insert(h->S.end(), core[k].begin(), core[k].end());
      h->S.insert(h->S.end(), halo[k].begin(), halo[k].end());
    }
    h->arena_elems = off;
    h->sum_s = soff;
    // scatter permutation and the pattern of P (rows of column g = sorted S_part(g))
    h->perm.resize(soff);
    for (int32_t k = 0; k < nloc; ++k) {
      const PartDesc& d = h->parts[k];
      int32_t* pk = h->perm.data() + d.soff;
      std::iota(pk, pk + d.s, 0);
      const int32_t* Sk = h->S.data() + d.soff;
      std::sort(pk, pk + d.s, [&](int32_t a, int32_t b) { return Sk[a] < Sk[b]; });
    }
    h->invperm.resize(soff);
    for (int32_t k = 0; k < nloc; ++k) {
      const PartDesc& d = h->parts[k];
      for (int32_t t = 0; t < d.s; ++t) h->invperm[d.soff + h->perm[d.soff + t]] = t;
    }
    // memberships: for every vertex, the parts whose S_k hold it, in part order
    h->memptr.assign(n + 1, 0);
    for (size_t q = 0; q < h->S.size(); ++q) h->memptr[h->S[q] + 1]++;
    for (int64_t v = 0; v < n; ++v) h->memptr[v + 1] += h->memptr[v];
    h->mempart.resize(soff);
    h->memloc.resize(soff);
    {
      std::vector<int64_t> fill(h->memptr.begin(), h->memptr.end() - 1);
      for (int32_t k = 0; k < nloc; ++k) {
        const PartDesc& d = h->parts[k];
        for (int32_t a = 0; a < d.s; ++a) {
          const int32_t v = h->S[d.soff + a];
          h->mempart[fill[v]] = k;
          h->memloc[fill[v]] = a;
          fill[v]++;
        }
      }
    }
    // columns of parts held elsewhere (shard plans) are empty
    h->pcolptr.assign(n + 1, 0);
    for (int64_t g = 0; g < n; ++g)
      h->pcolptr[g + 1] = h->pcolptr[g] + (local[part[g]] >= 0 ? h->parts[local[part[g]]].s : 0);
    h->prowind.resize(h->pcolptr[n]);
    for (int64_t g = 0; g < n; ++g) {
      if (local[part[g]] < 0) continue;
      const PartDesc& d = h->parts[local[part[g]]];
      const int32_t* Sk = h->S.data() + d.soff;
      const int32_t* pk = h->perm.data() + d.soff;
      int32_t* r = h->prowind.data() + h->pcolptr[g];
      for (int32_t t = 0; t < d.s; ++t) r[t] = Sk[pk[t]];
    }
    // work lists: parts in descending size, so the longest tiles start first
    std::vector<int32_t> order(nloc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return h->parts[a].s > h->parts[b].s; });
    int32_t slot = 0;
    for (int32_t k : order) {
      const PartDesc& d = h->parts[k];
      for (int32_t ti = 0; ti < d.nt; ++ti)
        for (int32_t tj = ti; tj < d.nt; ++tj) h->tiles.push_back(Tile{k, ti, tj, ti == tj ? slot++ : -1});
      for (int32_t j = 0; j < d.nt * SQ_TILE; j += COLS_PER_BLOCK) h->gblocks.push_back(ColBlock{k, j});
      for (int32_t j = 0; j < d.ld; j += COLS_PER_BLOCK) h->gblocks_ld.push_back(ColBlock{k, j});
      const int32_t nt128 = (d.s + TC_TILE - 1) / TC_TILE;
      const int32_t slot0 = h->nslots_tc;  // diagonal tiles take slots slot0 + ti in both lists
      for (int32_t ti = 0; ti < nt128; ++ti)
        for (int32_t tj = ti; tj < nt128; ++tj)
          h->tc_tiles.push_back(Tile{k, ti, tj, ti == tj ? h->nslots_tc++ : -1});
      // the same upper tiles two column blocks at a time along each row block (the last
      // one alone when the row has an odd number)
      for (int32_t ti = 0; ti < nt128; ++ti)
        for (int32_t tj = ti; tj < nt128; tj += 2) {
          h->tc_wide.push_back(Tile{k, ti, tj, ti == tj ? slot0 + ti : -1});
          h->tc_wide_nb.push_back((int8_t)(tj + 1 < nt128 ? 2 : 1));
        }
      for (int32_t j = 0; j < d.c; j += COLS_PER_BLOCK) h->sblocks.push_back(ColBlock{k, j});
    }
    h->nslots = slot;
    if (h->tiles.size() > (size_t)INT32_MAX || h->gblocks.size() > (size_t)INT32_MAX)
      return bail(GSP2_E_ARG, "problem too large for one launch");
    build_layout(h);
  } catch (const std::bad_alloc&) {
    t_create_err = "host allocation failed";
    delete h;
    return GSP2_E_OOM;
  }
  *out = h;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_create(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t nocc,
                                   const int32_t* part, int32_t nparts, const int64_t* g_rowptr,
                                   const int32_t* g_colind, const gsp2_options* opt, gsp2_handle* out) {
  return create_plan(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, nullptr, 0, opt, out);
}

extern "C" gsp2_status gsp2_create_shard(int64_t n, const int64_t* rowptr, const int32_t* colind, int64_t nocc,
                                         const int32_t* part, int32_t nparts, const int64_t* g_rowptr,
                                         const int32_t* g_colind, const int32_t* part_rank, int32_t rank,
                                         const gsp2_options* opt, gsp2_handle* out) {
  if (!part_rank) {
    t_create_err = "part_rank is NULL";
    if (out) *out = nullptr;
    return GSP2_E_ARG;
  }
  return create_plan(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, part_rank, rank, opt, out);
}

// Longest processing time first over the Eq. 5 cost s_k^3: parts in descending cost (ties by
// id), each to the rank with the least cost so far (ties to the lowest rank).  Deterministic,
// so every rank computes the same assignment from the same sizes.
extern "C" gsp2_status gsp2_assign_parts(const int32_t* sizes, int32_t nparts, int32_t nranks, int32_t* part_rank,
                                         double* rank_cost) {
  if (!sizes || !part_rank || nparts < 1 || nranks < 1 || nranks > nparts) return GSP2_E_ARG;
  for (int32_t k = 0; k < nparts; ++k)
    if (sizes[k] < 1) return GSP2_E_ARG;
  std::vector<int32_t> order(nparts);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return sizes[a] > sizes[b]; });
  std::vector<double> load(nranks, 0.0);
  for (int32_t k : order) {
    int32_t r = 0;
    for (int32_t q = 1; q < nranks; ++q)
      if (load[q] < load[r]) r = q;
    part_rank[k] = r;
    load[r] += (double)sizes[k] * sizes[k] * sizes[k];
  }
  if (rank_cost)
    for (int32_t r = 0; r < nranks; ++r) rank_cost[r] = load[r];
  return GSP2_OK;
}

static bool usable(gsp2_plan* h) { return h && !h->parts.empty(); }

extern "C" gsp2_status gsp2_workspace_bytes(gsp2_handle h, size_t* bytes) {
  if (!usable(h) || !bytes) return fail(h, GSP2_E_ARG, "invalid handle or NULL output");
  *bytes = h->L.total;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_plan_query(gsp2_handle h, gsp2_plan_info* info, int32_t* s, int32_t* c) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (info) {
    info->n = h->n;
    info->nocc = h->nocc;
    info->nparts = h->nparts;
    info->max_s = h->max_s;
    info->sum_s = h->sum_s;
    info->sum_s2 = h->sum_s2;
    info->sum_s3 = h->sum_s3;
    info->nnz_h = h->nnz_h;
    info->nnz_p = h->pcolptr[h->n];
    info->arena_elems = h->arena_elems;
    info->ntiles = (int64_t)h->tiles.size();
    info->tile = SQ_TILE;
    info->ld_pad = LD_PAD;
    info->step_launches = (int32_t)(h->ev.empty() ? std::max(h->total_steps, h->opt.max_steps) : h->ev.size() / 2);
    info->fp64_tail_steps = h->opt.fp64_tail_steps;
    info->tc_schedule = h->opt.tc_schedule;
    info->tile_order = h->opt.tile_order;
    info->tile_shape = h->opt.tile_shape;
    info->split_k = h->split_on ? 1 : 0;
    info->tile_claim = h->opt.tile_claim;
  }
  for (int32_t k = 0; k < h->nparts; ++k) {
    if (s) s[k] = h->parts[k].s;
    if (c) c[k] = h->parts[k].c;
  }
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_p_pattern(gsp2_handle h, int64_t* colptr, int32_t* rowind, int64_t* nnz_p) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (nnz_p) *nnz_p = h->pcolptr[h->n];
  if (colptr) std::memcpy(colptr, h->pcolptr.data(), h->pcolptr.size() * sizeof(int64_t));
  if (rowind) std::memcpy(rowind, h->prowind.data(), h->prowind.size() * sizeof(int32_t));
  return GSP2_OK;
}

static void drop_graph(gsp2_plan* h) {
  for (auto& f : h->fg) {
    if (f.exec) cudaGraphExecDestroy(f.exec);
    f = gsp2_plan::ForwardGraph{};
  }
  if (h->bexec) cudaGraphExecDestroy(h->bexec);
  h->bexec = nullptr;
  h->bkey_pbar = nullptr;
  h->bkey_hbar = nullptr;
}

// The 128x128 tile list in the order of opt.tile_order for a grid of `grid` persistent CTAs
// (CTA b takes entries b, b + grid, ...): 0 keeps parts by descending size; 1 reverses every
// other round of `grid` entries, so that the CTA that took the largest tile of one round
// takes the smallest of the next.
static void order_tc_tiles(gsp2_plan* h, int grid) {
  h->tc_order = h->tc_tiles;
  h->tcw_order = h->tc_wide;
  h->tcw_nb_order = h->tc_wide_nb;
  if (h->opt.tile_order == 0 || grid < 2) return;
  const size_t g = (size_t)grid;
  auto serpentine = [g](auto& v) {
    for (size_t r = 0; r * g < v.size(); ++r)
      if (r & 1) {
        const size_t b = r * g, e = std::min(b + g, v.size());
        std::reverse(v.begin() + b, v.begin() + e);
      }
  };
  serpentine(h->tc_order);
  serpentine(h->tcw_order);
  serpentine(h->tcw_nb_order);
  if (h->opt.tile_order != 2) return;
  // tile_order 2: the serpentine deal, then the tiles of the last rounds re-dealt so that the
  // CTAs finish together.  Each CTA's load up to the last rounds is summed from a cost model
  // (the tile's columns times K, K padded to the stage and a fixed part for fill and epilogue);
  // the remaining tiles, largest first, go to the least loaded CTA that still has a place in
  // those rounds (its positions stay b, b + grid, ...: only the list order changes).
  const size_t nt = h->tc_order.size();
  const size_t rounds = (nt + g - 1) / g, tail = std::min<size_t>(4, rounds);
  if (tail < 2) return;
  const size_t first = (rounds - tail) * g;  // positions from here on are re-dealt
  auto cost = [&](const Tile& t) {
    const int32_t s = h->parts[t.part].s;
    const int32_t cols = std::min(128, ((s - t.tj * 128) + 15) & ~15);
    return (double)cols * (double)(((s + 31) & ~31) + 192);
  };
  std::vector<double> load(g, 0.0);
  for (size_t p = 0; p < first; ++p) load[p % g] += cost(h->tc_order[p]);
  std::vector<Tile> rest(h->tc_order.begin() + (long)first, h->tc_order.end());
  std::stable_sort(rest.begin(), rest.end(), [&](const Tile& a, const Tile& b) { return cost(a) > cost(b); });
  std::vector<size_t> next(g);  // next free position of each CTA
  for (size_t b = 0; b < g; ++b) next[b] = first + b;
  for (const Tile& tl : rest) {
    size_t best = g;
    for (size_t b = 0; b < g; ++b)
      if (next[b] < nt && (best == g || load[b] < load[best])) best = b;
    h->tc_order[next[best]] = tl;
    next[best] += g;
    load[best] += cost(tl);
  }
}

// Work items of the split reverse steps (both K halves of every upper tile, codes 2 i + half
// with i indexing tc_order): by descending cost (the tile's K = 2 s_k times its columns), in
// rounds of `grid` items dealt like the tiles (tile_order 1: every other round reversed).
static void order_split_items(gsp2_plan* h, int grid) {
  const size_t nt = h->tc_order.size();
  std::vector<int32_t> idx(nt);
  std::iota(idx.begin(), idx.end(), 0);
  auto cost = [&](int32_t i) {
    const Tile& t = h->tc_order[i];
    const int32_t s = h->parts[t.part].s;
    return (double)s * (double)std::min(128, s - t.tj * 128);
  };
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return cost(a) > cost(b); });
  h->split_items.clear();
  for (int32_t i : idx) {
    h->split_items.push_back(2 * i);
    h->split_items.push_back(2 * i + 1);
  }
  if (h->opt.tile_order >= 1 && grid >= 2) {
    const size_t g = (size_t)grid;
    for (size_t r = 0; r * g < h->split_items.size(); ++r)
      if (r & 1) {
        const size_t b = r * g, e = std::min(b + g, h->split_items.size());
        std::reverse(h->split_items.begin() + b, h->split_items.begin() + e);
      }
  }
}

extern "C" gsp2_status gsp2_bind_workspace(gsp2_handle h, void* d_ws, size_t bytes, void* stream) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!d_ws || ((uintptr_t)d_ws & 255)) return fail(h, GSP2_E_WORKSPACE, "workspace NULL or not 256-byte aligned");
  if (bytes < h->L.total) return fail(h, GSP2_E_WORKSPACE, "workspace smaller than gsp2_workspace_bytes");
  cudaPointerAttributes at{};
  CU(h, cudaPointerGetAttributes(&at, d_ws));
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(h, GSP2_E_WORKSPACE, "workspace is not device memory");
  int dev = 0;
  CU(h, cudaGetDevice(&dev));
  CU(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  drop_graph(h);
  h->ws = (char*)d_ws;
  h->ws_size = bytes;
  h->device = dev;
  h->have_forward = false;
  if (!h->cap_stream) CU(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (h->adj_overlap && !h->side_stream) {
    CU(h, cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    h->bev.resize(1 + 2 * (size_t)(h->total_steps / h->opt.ckpt_every + 1));
    for (auto& e : h->bev) CU(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (h->opt.time_steps && h->ev.empty()) {
    h->ev.resize(2 * (size_t)std::max(h->total_steps, h->opt.max_steps));
    for (auto& e : h->ev) CU(h, cudaEventCreate(&e));
  }
  const WsLayout& L = h->L;
  auto up = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(h->ws + off, src, n, cudaMemcpyHostToDevice, s);
  };
  CU(h, up(L.parts, h->parts.data(), h->parts.size() * sizeof(PartDesc)));
  CU(h, up(L.S, h->S.data(), h->S.size() * sizeof(int32_t)));
  CU(h, up(L.perm, h->perm.data(), h->perm.size() * sizeof(int32_t)));
  CU(h, up(L.invperm, h->invperm.data(), h->invperm.size() * sizeof(int32_t)));
  CU(h, up(L.memptr, h->memptr.data(), h->memptr.size() * sizeof(int64_t)));
  CU(h, up(L.mempart, h->mempart.data(), h->mempart.size() * sizeof(int32_t)));
  CU(h, up(L.memloc, h->memloc.data(), h->memloc.size() * sizeof(int32_t)));
  std::vector<const double*> tab(h->step_arena_off.size());
  for (size_t i = 0; i < tab.size(); ++i) tab[i] = (const double*)(h->ws + h->step_arena_off[i]);
  CU(h, up(L.step_arena, tab.data(), tab.size() * sizeof(double*)));
  CU(h, up(L.tiles, h->tiles.data(), h->tiles.size() * sizeof(Tile)));
  order_tc_tiles(h, h->num_sms);
  CU(h, up(L.tc_tiles, h->tc_order.data(), h->tc_order.size() * sizeof(Tile)));
  CU(h, up(L.tc_wide, h->tcw_order.data(), h->tcw_order.size() * sizeof(Tile)));
  CU(h, up(L.tc_wide_nb, h->tcw_nb_order.data(), h->tcw_nb_order.size()));
  if (L.split_items) {
    order_split_items(h, h->num_sms);
    CU(h, up(L.split_items, h->split_items.data(), h->split_items.size() * sizeof(int32_t)));
    // the per-tile counters of split items start at zero (every launch leaves them so)
    CU(h, cudaMemsetAsync(h->ws + L.split_cnt, 0, h->tc_tiles.size() * sizeof(uint32_t), s));
  }
  CU(h, up(L.gblocks_ld, h->gblocks_ld.data(), h->gblocks_ld.size() * sizeof(ColBlock)));
  if (h->use_oz) {
    void* enc = nullptr;
    cudaDriverEntryPointQueryResult q{};
    CU(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &enc, 12000, cudaEnableDefault, &q));
    if (!enc || q != cudaDriverEntryPointSuccess)
      return fail(h, GSP2_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
    const size_t np = h->parts.size();
    // per digit set, K-major and MN-major maps whose boxes take all OZ_SLICES digits (the
    // high pass) or the first OZ_SPLIT (the low pass) of a tile slice in one request; a set's
    // digit arenas lie one arena apart (consecutive equal allocations)
    const size_t dstride = (size_t)h->arena_elems * 2;
    auto encode_set = [&](unsigned char* mk, unsigned char* mm, const size_t* dig) -> int {
      for (int t = 1; t < OZ_SLICES; ++t)
        if (dig[t] != dig[0] + (size_t)t * dstride) return -1;
      int r = encode_part_maps_digits(enc, mk, mm, h->parts.data(), (int)np, h->ws + dig[0], dstride, OZ_SLICES,
                                      OZ_SLICES, OZ_BK);
      if (r == 0)
        r = encode_part_maps_digits(enc, mk + np * 128, mm + np * 128, h->parts.data(), (int)np, h->ws + dig[0],
                                    dstride, OZ_SLICES, OZ_SPLIT, OZ_BK);
      return r;
    };
    std::vector<unsigned char> maps((size_t)2 * OZ_SLICES * np * 128, 0), maps_mn(maps.size(), 0);
    for (int b = 0; b < 2; ++b) {
      const size_t at = (size_t)b * OZ_SLICES * np * 128;
      const int r = encode_set(maps.data() + at, maps_mn.data() + at, L.oz_slice[b]);
      if (r != 0) return fail(h, GSP2_E_CUDA, "digit tensor maps failed: " + std::to_string(r));
    }
    CU(h, up(L.oz_maps, maps.data(), maps.size()));
    CU(h, up(L.oz_maps_mn, maps_mn.data(), maps_mn.size()));
    // the emulated steps never write the 16-column chunks of a part's padding: every arena
    // and digit buffer they write starts zeroed here
    {
      const size_t ab = (size_t)h->arena_elems * sizeof(double), dbytes = (size_t)h->arena_elems * 2;
      std::vector<size_t> fp64_arenas{L.arena0, L.arena1};
      if (fp64_like(h->opt.precision)) {
        fp64_arenas.insert(fp64_arenas.end(), L.ckpt.begin(), L.ckpt.end());
        fp64_arenas.insert(fp64_arenas.end(), L.seg.begin(), L.seg.end());
        fp64_arenas.insert(fp64_arenas.end(), L.seg2.begin(), L.seg2.end());
      }
      for (size_t off : fp64_arenas) CU(h, cudaMemsetAsync(h->ws + off, 0, ab, s));
      for (int b = 0; b < 2; ++b)
        for (int t = 0; t < OZ_SLICES; ++t) CU(h, cudaMemsetAsync(h->ws + L.oz_slice[b][t], 0, dbytes, s));
      for (size_t off : L.adj_dig) CU(h, cudaMemsetAsync(h->ws + off, 0, dbytes, s));
    }
    if (!L.adj_dig.empty()) {
      std::vector<unsigned char> amaps(L.adj_dig.size() * np * 128, 0), amaps_mn(amaps.size(), 0);
      for (size_t i = 0; i < L.adj_dig.size(); i += OZ_SLICES) {
        const int r = encode_set(amaps.data() + i * np * 128, amaps_mn.data() + i * np * 128, &L.adj_dig[i]);
        if (r != 0) return fail(h, GSP2_E_CUDA, "digit tensor maps failed: " + std::to_string(r));
      }
      CU(h, up(L.adj_maps, amaps.data(), amaps.size()));
      CU(h, up(L.adj_maps_mn, amaps_mn.data(), amaps_mn.size()));
      // Xbar's arenas start zeroed, so that padding the seed does not write stays zero
      CU(h, cudaMemsetAsync(h->ws + L.xb0, 0, (size_t)h->arena_elems * sizeof(double), s));
      CU(h, cudaMemsetAsync(h->ws + L.xb1, 0, (size_t)h->arena_elems * sizeof(double), s));
    }
  }
  if (!fp64_like(h->opt.precision)) {
    std::vector<const float*> mt(h->mf_of_step.size());
    for (size_t i = 0; i < mt.size(); ++i) mt[i] = (const float*)(h->ws + h->mf_of_step[i]);
    CU(h, up(L.master_of_step, mt.data(), mt.size() * sizeof(float*)));
    const int kind = prec_kind(h->opt.precision), nprod = prec_nprod(h->opt.precision);
    if (kind >= 0) {
      void* enc = nullptr;
      cudaDriverEntryPointQueryResult q{};
      CU(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &enc, 12000, cudaEnableDefault, &q));
      if (!enc || q != cudaDriverEntryPointSuccess)
        return fail(h, GSP2_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
      const size_t np = h->parts.size();
      std::vector<unsigned char> maps(4 * np * 128, 0), maps_mn(maps.size(), 0);
      // K-major boxes (one 128-byte row of K by 128 rows); for the 16-bit kinds also MN-major
      // boxes (64 rows of 128 bytes by one K block of 64 elements)
      for (int b = 0; b < 2; ++b)
        for (int q = 0; q < (nprod == 3 ? 2 : 1); ++q) {
          void* arena = h->ws + (q ? L.op_lo[b] : L.op_hi[b]);
          const size_t at = (size_t)(2 * b + q) * np * 128;
          int r = encode_part_maps(enc, maps.data() + at, h->parts.data(), (int)np, arena, kind);
          if (r == 0 && L.maps_mn) r = encode_part_maps(enc, maps_mn.data() + at, h->parts.data(), (int)np, arena, kind,
                                                        128, 64);
          if (r != 0) return fail(h, GSP2_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(r));
        }
      CU(h, up(L.maps, maps.data(), maps.size()));
      if (L.maps_mn) CU(h, up(L.maps_mn, maps_mn.data(), maps_mn.size()));
    }
    {
      // every iterate and operand arena starts zeroed, so that the padding no step writes
      // stays zero for the steps and conversions that read whole 128-column blocks: the
      // CUDA-core steps work in 64-column tiles up to roundup(s, 64), the tensor-core steps
      // skip the 16-column chunks beyond roundup(s, 16)
      const size_t af = (size_t)h->arena_elems * sizeof(float);
      const size_t ab = (size_t)h->arena_elems * sizeof(double);
      const size_t es = kind == 1 ? 4 : 2;
      std::vector<std::pair<size_t, size_t>> zero{{L.mf[0], af}, {L.mf[1], af}, {L.d[0], ab}, {L.d[1], ab}};
      for (size_t off : L.ckpt) zero.push_back({off, af});
      for (size_t off : L.seg) zero.push_back({off, af});
      for (size_t off : L.seg2) zero.push_back({off, af});
      for (size_t off : L.tailf) zero.push_back({off, af});
      for (size_t off : L.aop) zero.push_back({off, (size_t)h->arena_elems * 2});
      if (L.xb_max) zero.push_back({L.xb_max, h->parts.size() * sizeof(uint32_t)});
      if (L.xb0) zero.push_back({L.xb0, af});
      if (L.xb1) zero.push_back({L.xb1, af});
      for (int b = 0; b < 2; ++b) {
        if (L.op_hi[b]) zero.push_back({L.op_hi[b], (size_t)h->arena_elems * es});
        if (L.op_lo[b]) zero.push_back({L.op_lo[b], (size_t)h->arena_elems * es});
      }
      for (const auto& z : zero) CU(h, cudaMemsetAsync(h->ws + z.first, 0, z.second, s));
    }
    if (!L.aop.empty()) {
      // the FP32 adjoint: maps over its FP16 operand arenas
      void* enc = nullptr;
      cudaDriverEntryPointQueryResult q{};
      CU(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &enc, 12000, cudaEnableDefault, &q));
      if (!enc || q != cudaDriverEntryPointSuccess)
        return fail(h, GSP2_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
      const size_t np = h->parts.size();
      std::vector<unsigned char> amaps(L.aop.size() * np * 128, 0), amaps_mn(amaps.size(), 0);
      for (size_t i = 0; i < L.aop.size(); ++i) {
        int r = encode_part_maps(enc, amaps.data() + i * np * 128, h->parts.data(), (int)np, h->ws + L.aop[i], 2);
        if (r == 0)
          r = encode_part_maps(enc, amaps_mn.data() + i * np * 128, h->parts.data(), (int)np, h->ws + L.aop[i], 2, 128,
                               64);
        if (r != 0) return fail(h, GSP2_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(r));
      }
      CU(h, up(L.aop_maps, amaps.data(), amaps.size()));
      CU(h, up(L.aop_maps_mn, amaps_mn.data(), amaps_mn.size()));
    }
  }
  CU(h, up(L.gblocks, h->gblocks.data(), h->gblocks.size() * sizeof(ColBlock)));
  CU(h, up(L.sblocks, h->sblocks.data(), h->sblocks.size() * sizeof(ColBlock)));
  CU(h, up(L.pcolptr, h->pcolptr.data(), h->pcolptr.size() * sizeof(int64_t)));
  CU(h, up(L.rowptr, h->rowptr.data(), h->rowptr.size() * sizeof(int64_t)));
  CU(h, up(L.colind, h->colind.data(), h->colind.size() * sizeof(int32_t)));
  CU(h, up(L.locptr, h->locptr.data(), h->locptr.size() * sizeof(int64_t)));
  CU(h, launch_locate((const PartDesc*)(h->ws + L.parts), (const ColBlock*)(h->ws + L.gblocks_ld),
                      (int)h->gblocks_ld.size(), (const int32_t*)(h->ws + L.S), (const int64_t*)(h->ws + L.rowptr),
                      (const int32_t*)(h->ws + L.colind), (const int64_t*)(h->ws + L.locptr),
                      (int32_t*)(h->ws + L.loc), s));
  CU(h, cudaMemsetAsync(h->ws + L.state, 0, sizeof(DevState), s));
  CU(h, cudaMemsetAsync(h->ws + L.tile_ctr, 0, sizeof(uint32_t), s));
  CU(h, cudaMemsetAsync(h->ws + L.alpha, 0, (size_t)h->opt.max_steps + HIST_EXTRA, s));
  // the uploads read pageable host vectors; finish them before the call returns
  CU(h, cudaStreamSynchronize(s));
  return GSP2_OK;
}

// Arguments of the emulated FP64 step common to all its launches of a call.
static OzStepArgs oz_args(gsp2_plan* h, const StepCtl& ctl) {
  const WsLayout& L = h->L;
  char* w = h->ws;
  OzStepArgs a{};
  if (!h->use_oz) return a;
  a.parts = (const PartDesc*)(w + L.parts);
  a.tiles = (const Tile*)(w + L.tc_tiles);
  a.ntiles = (int)h->tc_tiles.size();
  a.maps = w + L.oz_maps;
  a.maps_mn = w + L.oz_maps_mn;
  a.nparts = (int)h->parts.size();
  for (int b = 0; b < 2; ++b)
    for (int t = 0; t < OZ_SLICES; ++t) a.digits[b].s[t] = (uint16_t*)(w + L.oz_slice[b][t]);
  a.slots = (double2*)(w + L.slots);
  a.nslots = h->nslots_tc;
  a.acc = (long long*)(w + L.oz_acc);
  a.ctl = ctl;
  a.tile_ctr = h->opt.tile_claim ? (uint32_t*)(w + L.tile_ctr) : nullptr;
  if (h->split_on) {
    a.split = 1;
    a.split_acc = (long long*)(w + L.split_acc);
    a.split_cnt = (uint32_t*)(w + L.split_cnt);
    a.split_items = (const int32_t*)(w + L.split_items);
  }
  return a;
}

// Bookkeeping arguments of a forward call: `ctl` for the FP64 steps, and for the
// low-precision loop the same with its stopping test gated at max(idem_tol, 16 N u).
static StepCtl forward_ctl(gsp2_plan* h, int mode, int nsteps) {
  const WsLayout& L = h->L;
  char* w = h->ws;
  const bool fp64 = fp64_like(h->opt.precision);
  StepCtl ctl{(DevState*)(w + L.state),
              (int8_t*)(w + L.alpha),
              (double*)(w + L.traces),
              (double*)(w + L.idem),
              h->nocc,
              h->opt.idem_tol,
              h->opt.trace_tol,
              mode,
              mode == MODE_REPLAY ? nsteps : (fp64 ? h->total_steps : h->opt.max_steps),
              1,
              (mode == MODE_RECORD && fp64) ? h->opt.fp64_tail_steps : 0,
              h->shard ? (ShardSlot*)(w + L.xchg) : nullptr};
  return ctl;
}
static StepCtl lowprec_ctl(gsp2_plan* h, const StepCtl& ctl) {
  StepCtl lp = ctl;
  lp.idem_tol = std::max(h->opt.idem_tol, 16.0 * (double)h->n * prec_unit(h->opt.precision));
  lp.stop_lag = 1;
  return lp;
}

// The forward pass is a sequence of segments.  Segment 0 resets the call state, takes the
// bounds and gathers X0; every further segment ends with one purification-step launch (and
// holds the launches that prepare it); each of those launches ends with the step's trace
// bookkeeping in its last block.  The last segment (index = exchanges) scatters P and
// writes the reports.  The number of bookkeeping launches, segments 0 .. exchanges - 1:
static int forward_exchanges(gsp2_plan* h, int mode, int nsteps) {
  if (fp64_like(h->opt.precision)) return 1 + (mode == MODE_REPLAY ? nsteps : h->total_steps);
  return 1 + h->opt.max_steps + h->opt.lp_tail_steps + h->opt.fp64_tail_steps;
}
// The bookkeeping that exchange x completes (SHARD_*), and its arguments.
static int exchange_kind(gsp2_plan* h, int x, int mode, int nsteps, StepCtl* c) {
  const StepCtl ctl = forward_ctl(h, mode, nsteps);
  if (fp64_like(h->opt.precision)) {
    *c = ctl;
    return x == 0 ? SHARD_GATHER : SHARD_LOOP;
  }
  const StepCtl lp = lowprec_ctl(h, ctl);
  if (x == 0) { *c = lp; return SHARD_GATHER; }
  if (x <= h->opt.max_steps) { *c = lp; return SHARD_LOOP; }
  if (x <= h->opt.max_steps + h->opt.lp_tail_steps) { *c = lp; return SHARD_TAIL_LP; }
  *c = ctl;
  return SHARD_TAIL_FP64;
}

// Queue segments seg_lo .. seg_hi of the forward pass on `s` (the whole pass: 0 .. INT_MAX).
static gsp2_status enqueue_forward(gsp2_plan* h, const double* hv, double* pv, int8_t* alpha_user, int mode,
                                   int nsteps, cudaStream_t s, int seg_lo = 0, int seg_hi = INT_MAX) {
  const WsLayout& L = h->L;
  char* w = h->ws;
  auto parts = (const PartDesc*)(w + L.parts);
  auto Sall = (const int32_t*)(w + L.S);
  auto perm = (const int32_t*)(w + L.perm);
  auto tiles = (const Tile*)(w + L.tiles);
  auto gbl = (const ColBlock*)(w + L.gblocks_ld);  // every column up to ld, padding zeroed
  auto sbl = (const ColBlock*)(w + L.sblocks);
  auto pcol = (const int64_t*)(w + L.pcolptr);
  auto rp = (const int64_t*)(w + L.rowptr);
  auto ci = (const int32_t*)(w + L.colind);
  auto loc = (const int32_t*)(w + L.loc);
  auto locp = (const int64_t*)(w + L.locptr);
  auto x0 = (double*)(w + L.x0);
  auto slots = (double2*)(w + L.slots);
  auto st = (DevState*)(w + L.state);
  auto alpha = (int8_t*)(w + L.alpha);
  auto A = [&](int i) { return (double*)(w + h->step_arena_off[i]); };
  const StepCtl ctl = forward_ctl(h, mode, nsteps);
  int seg = 0;  // segment of the next launch; a bookkeeping launch closes it
  auto on = [&]() { return seg >= seg_lo && seg <= seg_hi; };
  if (on()) {
    CU(h, launch_reset(st, alpha, mode == MODE_REPLAY ? alpha_user : nullptr, nsteps, h->opt.max_steps + HIST_EXTRA,
                       s));
    CU(h, launch_bounds(h->n, rp, ci, hv, slots, BOUNDS_BLOCKS, st, s));
    CU(h, launch_x0_values(h->n, rp, ci, hv, st, x0, h->num_sms, s));
  }
  const int prec = h->opt.precision;
  if (!fp64_like(prec)) {
    // low-precision phase, stopping test gated at max(idem_tol, 16 N u)
    const int kind = prec_kind(prec), nprod = prec_nprod(prec);
    const StepCtl lp = lowprec_ctl(h, ctl);
    float* mf[2] = {(float*)(w + L.mf[0]), (float*)(w + L.mf[1])};
    // FP32 iterate i of the loop: a checkpoint arena when the adjoint keeps it, else ping-pong
    auto mfs = [&](int i) { return (float*)(w + h->mf_of_step[(size_t)i]); };
    void* oh[2] = {w + L.op_hi[0], w + L.op_hi[1]};
    void* ol[2] = {w + L.op_lo[0], w + L.op_lo[1]};
    const size_t np = h->parts.size();
    // tensor-core schedule: persistent (one CTA per SM, overlapped epilogue) or one CTA per tile
    const int pgrid = h->opt.tc_schedule == 0 ? h->num_sms : 0;
    TcStepArgs tc_args{};
    const bool wide = pgrid > 0 && h->opt.tile_shape == 1;
    // the persistent 128x128 steps of the 16-bit kinds read the upper tiles only; the other
    // schedules read whole columns
    const bool upper_rows = (kind == 0 || kind == 2) && pgrid > 0 && !wide;
    if (on())
      CU(h, launch_gather_lp(kind, nprod, parts, (const ColBlock*)(w + L.gblocks_ld), (int)h->gblocks_ld.size(), Sall,
                             rp, loc, locp, x0, mfs(0), kind >= 0 ? oh[0] : nullptr, nprod == 3 ? ol[0] : nullptr,
                             (double*)slots, lp, s, upper_rows ? 1 : 0));
    ++seg;
    if (kind >= 0) {
      tc_args.parts = parts;
      tc_args.tiles = (const Tile*)(w + (wide ? L.tc_wide : L.tc_tiles));
      tc_args.nb = wide ? (const int8_t*)(w + L.tc_wide_nb) : nullptr;
      for (int b = 0; b < 2; ++b) {
        tc_args.map_hi[b] = w + L.maps + (size_t)(2 * b + 0) * np * 128;
        tc_args.map_lo[b] = w + L.maps + (size_t)(2 * b + 1) * np * 128;
        if (L.maps_mn) {
          tc_args.map_mn_hi[b] = w + L.maps_mn + (size_t)(2 * b + 0) * np * 128;
          tc_args.map_mn_lo[b] = w + L.maps_mn + (size_t)(2 * b + 1) * np * 128;
        }
        tc_args.master[b] = mf[b];
        tc_args.op_hi[b] = oh[b];
        tc_args.op_lo[b] = nprod == 3 ? ol[b] : nullptr;
      }
      tc_args.slots = slots;
      tc_args.nslots = h->nslots_tc;
      tc_args.ntiles = (int)(wide ? h->tc_wide.size() : h->tc_tiles.size());
      tc_args.ctl = lp;
      tc_args.tail = 0;
      tc_args.tile_ctr = h->opt.tile_claim ? (uint32_t*)(w + L.tile_ctr) : nullptr;
    }
    for (int i = 1; i <= lp.last_step; ++i, ++seg) {
      if (!on()) continue;
      const int bi = (i - 1) & 1, bo = i & 1;
      if (!h->ev.empty()) CU(h, cudaEventRecordWithFlags(h->ev[2 * (i - 1)], s, cudaEventRecordExternal));
      if (kind < 0) {
        CU(h, launch_square_fp32(parts, tiles, (int)h->tiles.size(), mfs(i - 1), mfs(i), slots, h->nslots, lp, i, s));
      } else {
        TcStepArgs a = tc_args;
        a.step = i;
        a.master[bi] = mfs(i - 1);
        a.master[bo] = mfs(i);
        CU(h, launch_square_tc(kind, nprod, a, a.ntiles, pgrid, s));
      }
      if (!h->ev.empty()) CU(h, cudaEventRecordWithFlags(h->ev[2 * (i - 1) + 1], s, cudaEventRecordExternal));
    }
    // alternating tail steps in the low precision
    for (int t = 0; t < h->opt.lp_tail_steps; ++t, ++seg) {
      if (!on()) continue;
      TcStepArgs a = tc_args;
      a.tail = t == 0 ? 1 : 2;
      CU(h, launch_square_tc(kind, nprod, a, a.ntiles, pgrid, s));
    }
    // FP64 tail: convert the last FP32 iterate, then purification steps in FP64 (native, or
    // with the products rebuilt from BF16 digits); the conversions open the segment of the
    // first tail step (or the last segment when there is no tail)
    double* d[2] = {(double*)(w + L.d[0]), (double*)(w + L.d[1])};
    const int T = h->opt.fp64_tail_steps;
    // the persistent kernel of the 16-bit kinds keeps upper tiles only: the native FP64 tail
    // reads whole 64-tiles, so it gets the lower ones first
    const bool lp_upper = kind == 0 || kind == 2;
    OzStepArgs toz = oz_args(h, ctl);
    if (on()) {
      if (h->use_oz) {
        // the emulated tail reads the rows on or above each diagonal block: conversion and
        // digits of those rows in one pass
        CU(h, launch_oz_convert_slice(parts, (const ColBlock*)(w + L.gblocks_ld), (int)h->gblocks_ld.size(),
                                      (const float* const*)(w + L.master_of_step), d[0], toz.digits, st, s));
      } else {
        CU(h, launch_convert((const float* const*)(w + L.master_of_step), d[0], h->arena_elems, st, s));
        if (lp_upper && T > 0)
          CU(h, launch_symmetrize(parts, (const Tile*)(w + L.tc_tiles), (int)h->tc_tiles.size(), nullptr, d[0], st,
                                  s));
      }
    }
    for (int t = 0; t < T; ++t, ++seg) {
      if (!on()) continue;
      const int tmode = (t == 0 && h->opt.lp_tail_steps == 0) ? SQ_TAIL_FIRST : SQ_TAIL_NEXT;
      if (h->use_oz) {
        OzStepArgs a = toz;
        a.xin = d[t & 1];
        a.xout = d[(t + 1) & 1];
        a.mode = tmode;
        CU(h, launch_oz_step(a, h->num_sms, s));
      } else
        CU(h, launch_square_fp64(parts, tiles, (int)h->tiles.size(), d[t & 1], d[(t + 1) & 1], slots, h->nslots, ctl,
                                 0, tmode, s));
    }
    if (!on()) return GSP2_OK;
    // emulated tail steps, and the 16-bit steps without a tail, leave the upper 128-tiles only
    const int ub = ((h->use_oz && T > 0) || (lp_upper && T == 0)) ? TC_TILE : 0;
    CU(h, launch_scatter(parts, sbl, (int)h->sblocks.size(), Sall, perm, pcol, nullptr, d[T & 1], pv, st, s, ub,
                         h->use_oz));
    if (h->opt.report_idem) {
      // the emulated tail keeps the iterate in 64-bit fixed point: FP64 for the residual
      if (h->use_oz)
        CU(h, launch_fixed_to_fp64(nullptr, d[T & 1], st, h->arena_elems, h->num_sms, s));
      if (ub) CU(h, launch_symmetrize(parts, (const Tile*)(w + L.tc_tiles), (int)h->tc_tiles.size(), nullptr, d[T & 1],
                                      st, s));
      CU(h, launch_residual_fp64(parts, tiles, (int)h->tiles.size(), d[T & 1], nullptr, (double*)(w + L.rslots),
                                 h->n, ctl, s));
    }
    if (alpha_user)
      CU(h, cudaMemcpyAsync(alpha_user, alpha + 1, (size_t)h->opt.max_steps + MAX_TAIL, cudaMemcpyDeviceToDevice, s));
    return GSP2_OK;
  }
  const bool emu = prec == GSP2_PREC_FP64_EMU;
  OzStepArgs oz{};
  if (emu) oz = oz_args(h, ctl);
  if (on()) {
    if (emu) {
      // X0 and its digits in one pass (the digits to buffer 0, read by step 1)
      CU(h, launch_oz_gather(parts, gbl, (int)h->gblocks_ld.size(), Sall, rp, loc, locp, x0, A(0), oz.digits[0],
                             (double*)slots, ctl, s));
    } else {
      CU(h, launch_gather(parts, gbl, (int)h->gblocks_ld.size(), Sall, rp, loc, locp, x0, A(0), (double*)slots, ctl,
                          s));
    }
  }
  ++seg;
  for (int i = 1; i <= ctl.last_step; ++i, ++seg) {
    if (!on()) continue;
    const double* xin = A(i - 1);
    double* xout = A(i);
    if (!h->ev.empty()) CU(h, cudaEventRecordWithFlags(h->ev[2 * (i - 1)], s, cudaEventRecordExternal));
    if (emu) {
      OzStepArgs a = oz;
      a.xin = xin;
      a.xout = xout;
      a.step = i;
      a.mode = SQ_FORWARD;
      CU(h, launch_oz_step(a, h->num_sms, s));
    } else
      CU(h, launch_square_fp64(parts, tiles, (int)h->tiles.size(), xin, xout, slots, h->nslots, ctl, i, SQ_FORWARD,
                               s));
    if (!h->ev.empty()) CU(h, cudaEventRecordWithFlags(h->ev[2 * (i - 1) + 1], s, cudaEventRecordExternal));
  }
  if (!on()) return GSP2_OK;
  CU(h, launch_scatter(parts, sbl, (int)h->sblocks.size(), Sall, perm, pcol, (const double* const*)(w + L.step_arena),
                       nullptr, pv, st, s, emu ? TC_TILE : 0, emu));
  if (h->opt.report_idem) {
    if (emu) {
      // the emulated steps keep the iterate in 64-bit fixed point: FP64 for the residual
      // (the backward never reads the last iterate)
      CU(h, launch_fixed_to_fp64((const double* const*)(w + L.step_arena), nullptr, st, h->arena_elems,
                                 h->num_sms, s));
      CU(h, launch_symmetrize(parts, (const Tile*)(w + L.tc_tiles), (int)h->tc_tiles.size(),
                              (const double* const*)(w + L.step_arena), nullptr, st, s));
    }
    CU(h, launch_residual_fp64(parts, tiles, (int)h->tiles.size(), nullptr, (const double* const*)(w + L.step_arena),
                               (double*)(w + L.rslots), h->n, ctl, s));
  }
  if (mode == MODE_RECORD && alpha_user)
    CU(h, cudaMemcpyAsync(alpha_user, alpha + 1, (size_t)h->opt.max_steps + MAX_TAIL, cudaMemcpyDeviceToDevice, s));
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_density(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha,
                                    int32_t mode, int32_t nsteps, void* stream) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!h->ws) return fail(h, GSP2_E_STATE, "no workspace bound");
  if (!d_hvals || !d_pvals) return fail(h, GSP2_E_ARG, "NULL H or P buffer");
  if (mode != MODE_RECORD && mode != MODE_REPLAY) return fail(h, GSP2_E_ARG, "mode must be RECORD or REPLAY");
  if (mode == MODE_REPLAY && (!d_alpha || nsteps < 1 || nsteps > h->total_steps))
    return fail(h, GSP2_E_ARG, "REPLAY needs d_alpha and 1 <= nsteps <= max_steps + fp64_tail_steps");
  if (mode == MODE_REPLAY && !fp64_like(h->opt.precision))
    return fail(h, GSP2_E_ARG, "REPLAY is available for the FP64 precision only");
  if (mode == MODE_RECORD) nsteps = 0;
  if (h->shard) return fail(h, GSP2_E_STATE, "a shard plan computes P with the gsp2_shard_* calls");
  int dev = 0;
  CU(h, cudaGetDevice(&dev));
  if (dev != h->device) return fail(h, GSP2_E_STATE, "current device differs from the workspace's device");
  cudaStream_t s = (cudaStream_t)stream;
  if (h->opt.use_graph) {
    GraphKey k{d_hvals, d_pvals, d_alpha, mode, nsteps};
    gsp2_plan::ForwardGraph* f = nullptr;
    for (auto& c : h->fg)
      if (c.exec && c.key == k) f = &c;
    if (!f) {
      // replace the empty or least recently used entry
      f = (!h->fg[0].exec || (h->fg[1].exec && h->fg[0].used <= h->fg[1].used)) ? &h->fg[0] : &h->fg[1];
      if (f->exec) cudaGraphExecDestroy(f->exec);
      *f = gsp2_plan::ForwardGraph{};
      cudaGraph_t g = nullptr;
      CU(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      gsp2_status st = enqueue_forward(h, d_hvals, d_pvals, d_alpha, mode, nsteps, h->cap_stream);
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
      if (st != GSP2_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&f->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        f->exec = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
      }
      f->key = k;
    }
    f->used = ++h->fg_clock;
    CU(h, cudaGraphLaunch(f->exec, s));
  } else {
    gsp2_status st = enqueue_forward(h, d_hvals, d_pvals, d_alpha, mode, nsteps, s);
    if (st != GSP2_OK) return st;
  }
  h->have_forward = true;
  h->known_steps = -1;
  return GSP2_OK;
}

// ------------------------------------------------------------------ shard plans

extern "C" gsp2_status gsp2_shard_info(gsp2_handle h, int32_t* rank, int32_t* nparts_global, int32_t* part_ids) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (rank) *rank = h->shard ? h->shard_rank : 0;
  if (nparts_global) *nparts_global = h->nparts_global;
  if (part_ids) std::memcpy(part_ids, h->part_global.data(), h->part_global.size() * sizeof(int32_t));
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_shard_exchanges(gsp2_handle h, int32_t mode, int32_t nsteps, int32_t* count) {
  if (!usable(h) || !count) return fail(h, GSP2_E_ARG, "invalid handle or NULL output");
  if (mode != MODE_RECORD && mode != MODE_REPLAY) return fail(h, GSP2_E_ARG, "mode must be RECORD or REPLAY");
  if (mode == MODE_REPLAY && (nsteps < 1 || nsteps > h->total_steps || !fp64_like(h->opt.precision)))
    return fail(h, GSP2_E_ARG, "REPLAY needs the FP64 precision and 1 <= nsteps <= max_steps + fp64_tail_steps");
  *count = forward_exchanges(h, mode, mode == MODE_REPLAY ? nsteps : 0);
  return GSP2_OK;
}

static gsp2_status shard_ready(gsp2_plan* h) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!h->shard) return fail(h, GSP2_E_STATE, "not a shard plan (gsp2_create_shard)");
  if (!h->ws) return fail(h, GSP2_E_STATE, "no workspace bound");
  int dev = 0;
  CU(h, cudaGetDevice(&dev));
  if (dev != h->device) return fail(h, GSP2_E_STATE, "current device differs from the workspace's device");
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_shard_begin(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha,
                                        int32_t mode, int32_t nsteps, double* d_send, void* stream) {
  gsp2_status r = shard_ready(h);
  if (r != GSP2_OK) return r;
  if (!d_hvals || !d_pvals || !d_send) return fail(h, GSP2_E_ARG, "NULL H, P or send buffer");
  if (mode != MODE_RECORD && mode != MODE_REPLAY) return fail(h, GSP2_E_ARG, "mode must be RECORD or REPLAY");
  if (mode == MODE_REPLAY && (!d_alpha || nsteps < 1 || nsteps > h->total_steps))
    return fail(h, GSP2_E_ARG, "REPLAY needs d_alpha and 1 <= nsteps <= max_steps + fp64_tail_steps");
  if (mode == MODE_REPLAY && !fp64_like(h->opt.precision))
    return fail(h, GSP2_E_ARG, "REPLAY is available for the FP64 precision only");
  if (mode == MODE_RECORD) nsteps = 0;
  cudaStream_t s = (cudaStream_t)stream;
  h->sx = gsp2_plan::ShardCall{};
  h->have_forward = false;
  h->known_steps = -1;
  r = enqueue_forward(h, d_hvals, d_pvals, d_alpha, mode, nsteps, s, 0, 0);
  if (r != GSP2_OK) return r;
  CU(h, launch_shard_partial((const DevState*)(h->ws + h->L.state), (const ShardSlot*)(h->ws + h->L.xchg), d_send, s));
  h->sx.hv = d_hvals;
  h->sx.pv = d_pvals;
  h->sx.alpha = d_alpha;
  h->sx.mode = mode;
  h->sx.nsteps = nsteps;
  h->sx.count = forward_exchanges(h, mode, nsteps);
  h->sx.next = 0;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_shard_decide(gsp2_handle h, int32_t x, const double* d_recv, int32_t nranks,
                                         void* stream) {
  gsp2_status r = shard_ready(h);
  if (r != GSP2_OK) return r;
  if (!d_recv || nranks < 1) return fail(h, GSP2_E_ARG, "NULL receive buffer or nranks < 1");
  if (h->sx.next != 2 * x) return fail(h, GSP2_E_STATE, "gsp2_shard_decide out of order");
  StepCtl c{};
  const int kind = exchange_kind(h, x, h->sx.mode, h->sx.nsteps, &c);
  CU(h, launch_shard_decide(c, d_recv, nranks, kind, (cudaStream_t)stream));
  h->sx.next = 2 * x + 1;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_shard_step(gsp2_handle h, int32_t x, double* d_send, void* stream) {
  gsp2_status r = shard_ready(h);
  if (r != GSP2_OK) return r;
  if (!d_send) return fail(h, GSP2_E_ARG, "NULL send buffer");
  if (x < 1 || x >= h->sx.count || h->sx.next != 2 * x - 1) return fail(h, GSP2_E_STATE, "gsp2_shard_step out of order");
  cudaStream_t s = (cudaStream_t)stream;
  r = enqueue_forward(h, h->sx.hv, h->sx.pv, h->sx.alpha, h->sx.mode, h->sx.nsteps, s, x, x);
  if (r != GSP2_OK) return r;
  CU(h, launch_shard_partial((const DevState*)(h->ws + h->L.state), (const ShardSlot*)(h->ws + h->L.xchg), d_send, s));
  h->sx.next = 2 * x;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_shard_end(gsp2_handle h, void* stream) {
  gsp2_status r = shard_ready(h);
  if (r != GSP2_OK) return r;
  if (h->sx.count < 1 || h->sx.next != 2 * h->sx.count - 1) return fail(h, GSP2_E_STATE, "gsp2_shard_end out of order");
  const int last = h->sx.count;
  r = enqueue_forward(h, h->sx.hv, h->sx.pv, h->sx.alpha, h->sx.mode, h->sx.nsteps, (cudaStream_t)stream, last, last);
  if (r != GSP2_OK) return r;
  h->sx.next = -1;
  h->have_forward = true;
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_autotune(gsp2_handle h, const double* d_hvals, double* d_pvals, int32_t trials,
                                     void* stream, gsp2_tune_report* rep) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!h->ws) return fail(h, GSP2_E_STATE, "no workspace bound");
  if (!d_hvals || !d_pvals || trials < 1 || trials > 100) return fail(h, GSP2_E_ARG, "NULL buffer or trials not in 1..100");
  cudaStream_t s = (cudaStream_t)stream;
  // candidates (tc_schedule, tile_order) that change something for this precision
  struct Cand {
    int sched, order, shape, split, claim;
  };
  std::vector<Cand> cand;
  const int prec = h->opt.precision;
  const int sp = h->split_on ? 1 : 0;
  if (!fp64_like(prec) && prec_kind(prec) >= 0)
    cand = {{0, 0, 0, 0, 1}, {0, 1, 0, 0, 1}, {0, 0, 0, 0, 0}, {0, 1, 0, 0, 0},
            {0, 0, 1, 0, 0}, {0, 1, 1, 0, 0}, {1, 0, 0, 0, 0}};
  else if (prec == GSP2_PREC_FP64_EMU && h->split_ok)
    cand = {{0, 0, 0, 0, 1}, {0, 1, 0, 0, 1}, {0, 2, 0, 0, 1}, {0, 0, 0, 1, 1}, {0, 1, 0, 1, 1}, {0, 2, 0, 0, 0}};
  else if (prec == GSP2_PREC_FP64_EMU) cand = {{0, 0, 0, 0, 1}, {0, 1, 0, 0, 1}, {0, 2, 0, 0, 1}, {0, 2, 0, 0, 0}};
  else cand = {{h->opt.tc_schedule, h->opt.tile_order, h->opt.tile_shape, sp, h->opt.tile_claim}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  auto apply = [&](const Cand& c) -> cudaError_t {
    // schedule and shape are part of the captured launches; the order only of the tile lists
    // (the claim counter's pointer is one of the launches' arguments)
    if (c.sched != h->opt.tc_schedule || c.shape != h->opt.tile_shape || (c.split != 0) != h->split_on ||
        c.claim != h->opt.tile_claim)
      drop_graph(h);
    h->opt.tile_claim = c.claim;
    h->opt.tc_schedule = c.sched;
    h->opt.tile_order = c.order;
    h->opt.tile_shape = c.shape;
    h->split_on = c.split != 0 && h->split_ok;
    order_tc_tiles(h, h->num_sms);
    if (h->tc_order.empty()) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(h->ws + h->L.tc_tiles, h->tc_order.data(), h->tc_order.size() * sizeof(Tile),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ws + h->L.tc_wide, h->tcw_order.data(), h->tcw_order.size() * sizeof(Tile),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->ws + h->L.tc_wide_nb, h->tcw_nb_order.data(), h->tcw_nb_order.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h->L.split_items) {
      order_split_items(h, h->num_sms);
      e = cudaMemcpyAsync(h->ws + h->L.split_items, h->split_items.data(), h->split_items.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s);
    }
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);  // the host vectors may change next round
  };
  std::vector<double> med(cand.size(), 0.0);
  gsp2_status out = GSP2_OK;
  for (size_t c = 0; c < cand.size() && out == GSP2_OK; ++c) {
    cudaError_t e = apply(cand[c]);
    if (e != cudaSuccess) {
      out = cuda_fail(h, e, "autotune: tile list upload");
      break;
    }
    std::vector<float> t;
    for (int k = 0; k <= trials && out == GSP2_OK; ++k) {
      if (k > 0 && (e = cudaEventRecord(e0, s)) != cudaSuccess) out = cuda_fail(h, e, "cudaEventRecord");
      if (out == GSP2_OK) out = gsp2_density(h, d_hvals, d_pvals, nullptr, MODE_RECORD, 0, stream);
      if (out == GSP2_OK && k > 0) {
        float ms = 0.f;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
          out = cuda_fail(h, e, "autotune timing");
        t.push_back(ms);
      }
      if (out == GSP2_OK) {
        gsp2_report r{};
        const gsp2_status st = gsp2_sync_status(h, &r);
        if (st != GSP2_OK && st != GSP2_E_NOT_CONVERGED) out = st;
      }
    }
    if (out == GSP2_OK) {
      std::sort(t.begin(), t.end());
      med[c] = t[t.size() / 2];
    }
  }
  size_t best = 0;
  if (out == GSP2_OK) {
    for (size_t c = 1; c < cand.size(); ++c)
      if (med[c] < med[best]) best = c;
    const cudaError_t e = apply(cand[best]);
    if (e != cudaSuccess) out = cuda_fail(h, e, "autotune: tile list upload");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->ncand = (int32_t)cand.size();
    rep->chosen = (int32_t)best;
    for (size_t c = 0; c < cand.size(); ++c) {
      rep->tc_schedule[c] = cand[c].sched;
      rep->tile_order[c] = cand[c].order;
      rep->tile_shape[c] = cand[c].shape;
      rep->split_k[c] = cand[c].split;
      rep->tile_claim[c] = cand[c].claim;
      rep->ms[c] = med[c];
    }
  }
  return out;
}

extern "C" gsp2_status gsp2_density_reuse(gsp2_handle h, const double* d_hvals, double* d_pvals, int8_t* d_alpha,
                                          int32_t* nsteps, void* stream, int32_t* recomputed) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!nsteps || !d_alpha || *nsteps < 0) return fail(h, GSP2_E_ARG, "NULL d_alpha or nsteps, or nsteps < 0");
  if (!fp64_like(h->opt.precision)) return fail(h, GSP2_E_STATE, "sequence reuse needs an FP64 or FP64_EMU plan");
  if (recomputed) *recomputed = 0;
  gsp2_report r{};
  if (*nsteps > 0) {
    gsp2_status st = gsp2_density(h, d_hvals, d_pvals, d_alpha, MODE_REPLAY, *nsteps, stream);
    if (st != GSP2_OK) return st;
    st = gsp2_sync_status(h, &r);
    if (st != GSP2_E_TRACE) return st;  // the sequence still holds (or another outcome to report)
  }
  gsp2_status st = gsp2_density(h, d_hvals, d_pvals, d_alpha, MODE_RECORD, 0, stream);
  if (st != GSP2_OK) return st;
  st = gsp2_sync_status(h, &r);
  *nsteps = r.steps;
  if (recomputed) *recomputed = 1;
  return st;
}

extern "C" gsp2_status gsp2_threshold_graph(gsp2_handle h, const double* d_pvals, double tau, void* stream,
                                            int64_t* g_rowptr, int32_t* g_colind, int64_t cap, int64_t* nnz) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!d_pvals || !g_rowptr || !nnz || !(tau >= 0.0) || cap < 0) return fail(h, GSP2_E_ARG, "NULL argument or tau < 0");
  if (!h->ws) return fail(h, GSP2_E_STATE, "no workspace bound");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t np = h->pcolptr[h->n];
  std::vector<uint8_t> mask((size_t)np);
  uint8_t* dmask = (uint8_t*)(h->ws + h->L.mask);
  CU(h, launch_threshold(d_pvals, np, tau, dmask, s));
  CU(h, cudaMemcpyAsync(mask.data(), dmask, (size_t)np, cudaMemcpyDeviceToHost, s));
  CU(h, cudaStreamSynchronize(s));
  const int64_t n = h->n;
  // edges (r, g) and (g, r) for every stored P_rg above tau, plus the diagonal
  std::vector<int64_t> deg((size_t)n + 1, 0);
  for (int64_t g = 0; g < n; ++g) {
    ++deg[(size_t)g];
    for (int64_t e = h->pcolptr[g]; e < h->pcolptr[g + 1]; ++e) {
      const int32_t r = h->prowind[(size_t)e];
      if (mask[(size_t)e] && r != g) {
        ++deg[(size_t)r];
        ++deg[(size_t)g];
      }
    }
  }
  std::vector<int64_t> rp((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) rp[(size_t)i + 1] = rp[(size_t)i] + deg[(size_t)i];
  std::vector<int32_t> ci((size_t)rp[(size_t)n]);
  std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
  for (int64_t g = 0; g < n; ++g) {
    ci[(size_t)fill[(size_t)g]++] = (int32_t)g;
    for (int64_t e = h->pcolptr[g]; e < h->pcolptr[g + 1]; ++e) {
      const int32_t r = h->prowind[(size_t)e];
      if (mask[(size_t)e] && r != g) {
        ci[(size_t)fill[(size_t)r]++] = (int32_t)g;
        ci[(size_t)fill[(size_t)g]++] = r;
      }
    }
  }
  // sort and deduplicate every row (an edge can come from both P_rg and P_gr), compacting
  // the rows to the front of ci
  int64_t out = 0;
  g_rowptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    auto b = ci.begin() + rp[(size_t)i], e = ci.begin() + rp[(size_t)i + 1];
    std::sort(b, e);
    const int64_t m = std::unique(b, e) - b;
    if (ci.begin() + out != b) std::copy(b, b + m, ci.begin() + out);  // out < rp[i]: moves left
    out += m;
    g_rowptr[i + 1] = out;
  }
  *nnz = out;
  if (!g_colind) return GSP2_OK;
  if (cap < out) return fail(h, GSP2_E_ARG, "g_colind smaller than the graph (see *nnz)");
  std::copy(ci.begin(), ci.begin() + out, g_colind);
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_sync_status(gsp2_handle h, gsp2_report* r) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!h->ws || !h->have_forward) return fail(h, GSP2_E_STATE, "no density call to report on");
  CU(h, cudaDeviceSynchronize());
  DevState st{};
  CU(h, cudaMemcpy(&st, h->ws + h->L.state, sizeof(DevState), cudaMemcpyDeviceToHost));
  double tr = 0.0, e = 0.0;
  CU(h, cudaMemcpy(&tr, h->ws + h->L.traces + sizeof(double) * st.steps, sizeof(double), cudaMemcpyDeviceToHost));
  if (st.steps > 0)
    CU(h, cudaMemcpy(&e, h->ws + h->L.idem + sizeof(double) * (st.steps - 1), sizeof(double),
                     cudaMemcpyDeviceToHost));
  // a finished call's step count lets the adjoint schedule exactly the applied steps
  h->known_steps = (st.status == ST_OK || st.status == ST_NOT_CONVERGED || st.status == ST_TRACE) ? st.steps : -1;
  if (r) {
    r->status = st.status;
    r->steps = st.steps;
    r->stopped = st.stopped;
    r->fp64_steps = st.fp64_steps;
    r->eps_min = st.eps_min;
    r->eps_max = st.eps_max;
    r->trace = tr;
    r->idem = e;
    r->idem_fro = st.idem_fro;
  }
  if (st.status != 0) {
    const char* what = st.status == ST_NOT_CONVERGED ? "not converged within max_steps"
                       : st.status == ST_TRACE       ? "replayed sequence gave the wrong trace"
                       : st.status == ST_NONFINITE   ? "non-finite value in H, bounds or traces"
                       : st.status == ST_TIMEOUT     ? "a bounded device wait gave up"
                                                     : "device error";
    h->err = what;
  }
  return (gsp2_status)st.status;
}

extern "C" gsp2_status gsp2_history(gsp2_handle h, double* traces, double* idem, int8_t* alpha, int32_t cap) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (!h->ws || !h->have_forward) return fail(h, GSP2_E_STATE, "no density call");
  if (cap < 0) return fail(h, GSP2_E_ARG, "cap < 0");
  CU(h, cudaDeviceSynchronize());
  const size_t m = (size_t)std::min<int32_t>(cap, h->opt.max_steps + MAX_TAIL + 1);
  if (traces) CU(h, cudaMemcpy(traces, h->ws + h->L.traces, m * sizeof(double), cudaMemcpyDeviceToHost));
  if (idem) CU(h, cudaMemcpy(idem, h->ws + h->L.idem, m * sizeof(double), cudaMemcpyDeviceToHost));
  if (alpha) CU(h, cudaMemcpy(alpha, h->ws + h->L.alpha + 1, m, cudaMemcpyDeviceToHost));
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_step_times(gsp2_handle h, float* ms, int32_t cap) {
  if (!usable(h) || !ms) return fail(h, GSP2_E_ARG, "invalid handle or NULL output");
  if (h->ev.empty() || !h->have_forward) return fail(h, GSP2_E_STATE, "time_steps not set or no density call");
  CU(h, cudaDeviceSynchronize());
  const int32_t m = std::min<int32_t>(cap, (int32_t)(h->ev.size() / 2));
  for (int32_t i = 0; i < m; ++i) {
    ms[i] = 0.0f;
    cudaError_t e = cudaEventElapsedTime(&ms[i], h->ev[2 * i], h->ev[2 * i + 1]);
    if (e == cudaErrorNotReady || e == cudaErrorInvalidResourceHandle) {
      (void)cudaGetLastError();
      ms[i] = 0.0f;
    } else if (e != cudaSuccess) {
      return cuda_fail(h, e, "cudaEventElapsedTime");
    }
  }
  return GSP2_OK;
}

// Queue the adjoint on `s`: seed, then per checkpoint segment (last first) the
// recomputed iterates and the reverse steps, then the scatter-add onto H.  The
// schedule covers max_steps; kernels for steps beyond the applied count return at once.
// Adjoint of an emulated-FP64 plan on the BF16 tensor cores.  For each checkpoint segment
// the iterates X_{c0} .. X_{c0+k-1} are rebuilt as digit sets (digits of the checkpoint,
// then emulated steps with the recorded branches); every reverse step multiplies the
// digits of X_{i-1} with those of Xbar / 2^sig and leaves the new Xbar's per-part scales
// (from its row norms, summed in the step's epilogue), and the new digits follow.  The
// seed's scales come from a separate norm pass.  Xbar is kept in its upper 128-tiles like
// the forward iterates.
// Steps the adjoint schedules (launches for steps the forward did not apply return at once):
// max_steps (FP64 plans: plus their tail steps), or the applied count once gsp2_sync_status
// has read it (the loop's steps for the low-precision plans, whose FP64 tail steps are
// reversed apart)
static int backward_steps(gsp2_plan* h) {
  if (fp64_like(h->opt.precision))
    return h->known_steps >= 0 ? std::min(h->known_steps, h->total_steps) : h->total_steps;
  const int T = h->opt.fp64_tail_steps;
  return h->known_steps >= T ? std::min(h->known_steps - T, h->opt.max_steps) : h->opt.max_steps;
}

static gsp2_status enqueue_backward_emu(gsp2_plan* h, const double* pbar, double* hbar, cudaStream_t s) {
  const WsLayout& L = h->L;
  char* w = h->ws;
  auto parts = (const PartDesc*)(w + L.parts);
  auto Sall = (const int32_t*)(w + L.S);
  auto gbl = (const ColBlock*)(w + L.gblocks);
  auto gbl_ld = (const ColBlock*)(w + L.gblocks_ld);
  const int ngb = (int)h->gblocks_ld.size();
  auto tct = (const Tile*)(w + L.tc_tiles);
  const int ntc = (int)h->tc_tiles.size();
  auto st = (DevState*)(w + L.state);
  auto alpha = (int8_t*)(w + L.alpha);
  double* xb0 = (double*)(w + L.xb0);
  double* xb1 = (double*)(w + L.xb1);
  double* norm = (double*)(w + L.adj_norm);
  float* normf = (float*)(w + L.adj_normf);
  int32_t* sig = (int32_t*)(w + L.adj_sig);
  const int k = h->opt.ckpt_every, M = backward_steps(h);
  const int np = (int)h->parts.size();
  StepCtl ctl{st, alpha, (double*)(w + L.traces), (double*)(w + L.idem), h->nocc, h->opt.idem_tol,
              h->opt.trace_tol, MODE_REPLAY, M, 1, 0};
  // digit set j of buffer b (the iterates X_{c0+j} of a checkpoint segment), and Xbar's set
  const int xset = h->adj_overlap ? 2 * k : k;
  auto sidx = [&](int b, int j) { return (h->adj_overlap ? b * k : 0) + j; };
  auto dset = [&](int idx) {
    OzSlices o{};
    for (int t = 0; t < OZ_SLICES; ++t) o.s[t] = (uint16_t*)(w + L.adj_dig[(size_t)idx * OZ_SLICES + t]);
    return o;
  };
  auto smaps = [&](size_t base, int idx) { return (const void*)(w + base + (size_t)idx * OZ_SLICES * np * 128); };
  auto seg = [&](int b, int j) { return (double*)(w + (b ? L.seg2[(size_t)j] : L.seg[(size_t)j])); };
  const OzStepArgs base = oz_args(h, ctl);
  // segment q covers the steps c0 + 1 .. c0 + k, c0 = q k; its buffer alternates when overlapped
  auto rebuild = [&](int q, cudaStream_t ss) -> gsp2_status {
    const int c0 = q * k, b = h->adj_overlap ? (q & 1) : 0;
    const double* ck = (const double*)(w + L.ckpt[(size_t)q]);
    CU(h, launch_oz_digits(parts, gbl_ld, ngb, ck, ck, 0, c0 + 1, dset(sidx(b, 0)), nullptr, st, ss));
    for (int j = 1; j < k && c0 + j < M; ++j) {
      OzStepArgs a = base;
      a.maps = smaps(L.adj_maps, sidx(b, j - 1));
      a.maps_mn = smaps(L.adj_maps_mn, sidx(b, j - 1));
      a.digits[0] = a.digits[1] = dset(sidx(b, j));
      a.xin = (j == 1) ? ck : seg(b, j - 2);
      a.xout = seg(b, j - 1);
      a.step = c0 + j;
      a.mode = SQ_RECOMPUTE;
      if (h->adj_overlap) {
        // beside the reverse steps: its own scratch tiles, no split items (their buffers are the
        // reverse steps')
        a.acc = (long long*)(w + L.oz_acc2);
        a.split = 0;
      }
      CU(h, launch_oz_step(a, h->num_sms, ss));
    }
    return GSP2_OK;
  };
  auto reverse = [&](int q, cudaStream_t ss) -> gsp2_status {
    const int c0 = q * k, b = h->adj_overlap ? (q & 1) : 0;
    for (int i = std::min(c0 + k, M); i >= c0 + 1; --i) {
      OzStepArgs a = base;
      a.maps = smaps(L.adj_maps, sidx(b, i - 1 - c0));
      a.maps_mn = smaps(L.adj_maps_mn, sidx(b, i - 1 - c0));
      a.maps_b = smaps(L.adj_maps, xset);
      a.maps_mn_b = smaps(L.adj_maps_mn, xset);
      a.sig = sig;
      a.normf = normf;
      a.xin = xb0;
      a.xout = xb1;
      a.step = i;
      CU(h, launch_oz_step(a, h->num_sms, ss, true));  // also leaves the new Xbar's scales in sig
      if (i > 1) CU(h, launch_oz_digits(parts, gbl_ld, ngb, xb0, xb1, i, 0, dset(xset), sig, st, ss));
    }
    return GSP2_OK;
  };
  auto seed = [&]() -> gsp2_status {
    CU(h, cudaMemsetAsync(norm, 0, h->S.size() * sizeof(double), s));
    CU(h, cudaMemsetAsync(normf, 0, h->S.size() * sizeof(float), s));
    CU(h, launch_adj_seed<double>(parts, gbl, (int)h->gblocks.size(), Sall, (const int32_t*)(w + L.invperm),
                                  (const int64_t*)(w + L.pcolptr), pbar, xb0, s));
    CU(h, launch_oz_adj_scale(parts, np, tct, ntc, xb0, xb1, 0, norm, sig, st, s));
    CU(h, launch_oz_digits(parts, gbl_ld, ngb, xb0, xb1, 0, 0, dset(xset), sig, st, s));
    return GSP2_OK;
  };
  const int Q = M / k;  // the last segment
  gsp2_status r;
  if (!h->adj_overlap) {
    if ((r = seed()) != GSP2_OK) return r;
    for (int q = Q; q >= 0; --q) {
      if ((r = rebuild(q, s)) != GSP2_OK) return r;
      if ((r = reverse(q, s)) != GSP2_OK) return r;
    }
  } else {
    // the side stream rebuilds segment q while the main stream reverses segment q + 1; the
    // rebuild of q waits for the reverse of q + 2, which read the same buffer
    cudaStream_t s2 = h->side_stream;
    cudaEvent_t* ev_b = h->bev.data() + 1;            // segment q rebuilt
    cudaEvent_t* ev_r = h->bev.data() + 1 + (Q + 1);  // segment q reversed
    CU(h, cudaEventRecord(h->bev[0], s));
    CU(h, cudaStreamWaitEvent(s2, h->bev[0], 0));
    for (int q = Q; q >= std::max(0, Q - 1); --q) {
      if ((r = rebuild(q, s2)) != GSP2_OK) return r;
      CU(h, cudaEventRecord(ev_b[q], s2));
    }
    if ((r = seed()) != GSP2_OK) return r;
    for (int q = Q; q >= 0; --q) {
      CU(h, cudaStreamWaitEvent(s, ev_b[q], 0));
      if ((r = reverse(q, s)) != GSP2_OK) return r;
      CU(h, cudaEventRecord(ev_r[q], s));
      if (q - 2 >= 0) {
        CU(h, cudaStreamWaitEvent(s2, ev_r[q], 0));
        if ((r = rebuild(q - 2, s2)) != GSP2_OK) return r;
        CU(h, cudaEventRecord(ev_b[q - 2], s2));
      }
    }
  }
  CU(h, launch_adj_hbar<double>(h->n, (const int64_t*)(w + L.rowptr), (const int32_t*)(w + L.colind),
                                (const int64_t*)(w + L.memptr), (const int32_t*)(w + L.mempart),
                                (const int32_t*)(w + L.memloc), parts, Sall, xb0, xb1, hbar, st, s, TC_TILE));
  return GSP2_OK;
}

static gsp2_status enqueue_backward(gsp2_plan* h, const double* pbar, double* hbar, cudaStream_t s) {
  if (h->opt.precision == GSP2_PREC_FP64_EMU) return enqueue_backward_emu(h, pbar, hbar, s);
  const WsLayout& L = h->L;
  char* w = h->ws;
  auto parts = (const PartDesc*)(w + L.parts);
  auto Sall = (const int32_t*)(w + L.S);
  auto tiles = (const Tile*)(w + L.tiles);
  auto gbl = (const ColBlock*)(w + L.gblocks);
  auto st = (DevState*)(w + L.state);
  auto alpha = (int8_t*)(w + L.alpha);
  double* xb0 = (double*)(w + L.xb0);
  double* xb1 = (double*)(w + L.xb1);
  const int k = h->opt.ckpt_every, M = backward_steps(h);
  const int nt = (int)h->tiles.size();
  StepCtl ctl{st, alpha, (double*)(w + L.traces), (double*)(w + L.idem), h->nocc, h->opt.idem_tol,
              h->opt.trace_tol, MODE_REPLAY, M, 1, 0};
  CU(h, launch_adj_seed<double>(parts, gbl, (int)h->gblocks.size(), Sall, (const int32_t*)(w + L.invperm),
                                (const int64_t*)(w + L.pcolptr), pbar, xb0, s));
  for (int c0 = (M / k) * k; c0 >= 0; c0 -= k) {
    const double* ck = (const double*)(w + L.ckpt[c0 / k]);
    for (int j = 1; j < k && c0 + j < M; ++j) {
      const double* xin = (j == 1) ? ck : (const double*)(w + L.seg[j - 2]);
      double* xout = (double*)(w + L.seg[j - 1]);
      CU(h, launch_square_fp64(parts, tiles, nt, xin, xout, nullptr, 0, ctl, c0 + j, SQ_RECOMPUTE, s));
    }
    for (int i = std::min(c0 + k, M); i >= c0 + 1; --i) {
      const double* X = (i - 1 == c0) ? ck : (const double*)(w + L.seg[i - 1 - c0 - 1]);
      CU(h, launch_adj_step<double>(parts, tiles, nt, X, xb0, xb1, alpha, st, i, s));
    }
  }
  CU(h, launch_adj_hbar<double>(h->n, (const int64_t*)(w + L.rowptr), (const int32_t*)(w + L.colind),
                                (const int64_t*)(w + L.memptr), (const int32_t*)(w + L.mempart),
                                (const int32_t*)(w + L.memloc), parts, Sall, xb0, xb1, hbar, st, s));
  return GSP2_OK;
}

// Adjoint of a low-precision plan, in FP32 with FP16 hi + lo products on the tensor cores
// (three products per K step, as the fp16x3 squaring): the T FP64 tail steps came last, so
// they are reversed first, on FP32 iterates rebuilt from the loop's last iterate X_L
// (L = n - T is known only on the device: these launches count back from n); then the
// loop's steps, from the FP32 checkpoints the forward kept every k steps.  Every FP32
// iterate the sweep reads gets its FP16 operand copies of X 2^14 (a split of a stored
// iterate, or the rebuild's own output).  Xbar keeps its FP32 master and its operands,
// FP16 of Xbar 2^(14 - sig) with one power-of-two scale per part, in a ping-pong pair: the
// seed's scale from a scan, each reverse step's output written at a scale fixed before the
// step from the largest |Xbar| so far and the growth bound of one step.
static gsp2_status enqueue_backward_lp(gsp2_plan* h, const double* pbar, double* hbar, cudaStream_t s) {
  const WsLayout& L = h->L;
  char* w = h->ws;
  auto parts = (const PartDesc*)(w + L.parts);
  auto Sall = (const int32_t*)(w + L.S);
  auto gbl = (const ColBlock*)(w + L.gblocks);
  auto gbl_ld = (const ColBlock*)(w + L.gblocks_ld);
  const int ngb = (int)h->gblocks_ld.size();
  auto st = (DevState*)(w + L.state);
  auto alpha = (int8_t*)(w + L.alpha);
  float* xb0 = (float*)(w + L.xb0);
  float* xb1 = (float*)(w + L.xb1);
  int32_t* xb_sig = (int32_t*)(w + L.xb_sig);
  uint32_t* xb_max = (uint32_t*)(w + L.xb_max);
  const int k = h->opt.ckpt_every, M = backward_steps(h), T = h->opt.fp64_tail_steps;
  const int64_t ne = h->arena_elems;
  const size_t np = h->parts.size();
  const int nsets = (int)L.aop.size() / 2 - 2;  // operand sets of rebuilt iterates (both buffers)
  const int set1 = std::max(k, T);                // first set of the second buffer (overlap)
  StepCtl ctl{st, alpha, (double*)(w + L.traces), (double*)(w + L.idem), h->nocc, h->opt.idem_tol,
              h->opt.trace_tol, MODE_REPLAY, M, 1, T};
  auto tf = [&](int t) { return (float*)(w + L.tailf[(size_t)t]); };
  auto aop = [&](int set, int lo) { return (void*)(w + L.aop[(size_t)(2 * set + lo)]); };
  auto amap = [&](int set, int lo) { return (const void*)(w + L.aop_maps + (size_t)(2 * set + lo) * np * 128); };
  auto amap_mn = [&](int set, int lo) {
    return (const void*)(w + L.aop_maps_mn + (size_t)(2 * set + lo) * np * 128);
  };
  TcStepArgs base{};
  base.parts = parts;
  base.tiles = (const Tile*)(w + L.tc_tiles);
  base.ntiles = (int)h->tc_tiles.size();
  base.ctl = ctl;
  base.adj_tail = T;
  base.xb_sig = xb_sig;
  base.xb_max = xb_max;
  base.nparts = (int)np;
  // headroom of the written scale: one reverse step multiplies the largest |Xbar| by at most
  // 2 + 2 sqrt(s) (Cauchy-Schwarz, ||X||_2 <= 1), one bit more for the rounding of X
  int smax = 1;
  for (const PartDesc& d : h->parts) smax = std::max(smax, (int)d.s);
  base.xb_headroom = (int)std::ceil(std::log2(2.0 + 2.0 * std::sqrt((double)smax))) + 1;
  base.tile_ctr = h->opt.tile_claim ? (uint32_t*)(w + L.tile_ctr) : nullptr;
  for (int b = 0; b < 2; ++b) {
    base.map_hi[b] = amap(nsets + b, 0);
    base.map_lo[b] = amap(nsets + b, 1);
    base.map_mn_hi[b] = amap_mn(nsets + b, 0);
    base.map_mn_lo[b] = amap_mn(nsets + b, 1);
    base.master[b] = b ? xb1 : xb0;
    base.op_hi[b] = aop(nsets + b, 0);
    base.op_lo[b] = aop(nsets + b, 1);
  }
  // operands of a stored iterate into set `set` (skipped where need > n - T)
  auto split_x = [&](const float* x, int set, int need, cudaStream_t ss) {
    return launch_split_f16(parts, gbl_ld, ngb, x, aop(set, 0), aop(set, 1), nullptr, need, T, st, ss);
  };
  // X_step rebuilt from X_{step-1} (operand set `in`, master xin) into set `out`, master xout
  auto rebuild = [&](int in, const float* xin, int out, float* xout, int step, cudaStream_t ss) {
    TcStepArgs a = base;
    a.xmap_hi = amap(in, 0);
    a.xmap_lo = amap(in, 1);
    a.xmap_mn_hi = amap_mn(in, 0);
    a.xmap_mn_lo = amap_mn(in, 1);
    a.xin = xin;
    a.xout = xout;
    a.xo_hi = aop(out, 0);
    a.xo_lo = aop(out, 1);
    a.step = step;
    return launch_tc_adjoint(a, h->num_sms, true, ss);
  };
  // reverse step `step` with X_{step-1} in operand set `x`
  auto reverse = [&](int x, int step) {
    TcStepArgs a = base;
    a.xmap_hi = amap(x, 0);
    a.xmap_lo = amap(x, 1);
    a.xmap_mn_hi = amap_mn(x, 0);
    a.xmap_mn_lo = amap_mn(x, 1);
    a.step = step;
    return launch_tc_adjoint(a, h->num_sms, false, s);
  };
  // Xbar's operands live in the FP64 tail arenas: zeroed first, so that the padding the
  // reverse steps do not write reads as zero, and again at the end, so that the next
  // forward's FP64 tail finds its padding zero
  const size_t ab = (size_t)ne * sizeof(double);
  CU(h, cudaMemsetAsync(w + L.d[0], 0, ab, s));
  CU(h, cudaMemsetAsync(w + L.d[1], 0, ab, s));
  CU(h, launch_adj_seed<float>(parts, gbl, (int)h->gblocks.size(), Sall, (const int32_t*)(w + L.invperm),
                               (const int64_t*)(w + L.pcolptr), pbar, xb0, s));
  CU(h, launch_xbar_seed_scale(parts, gbl_ld, ngb, xb0, xb_max, xb_sig, (int)np, base.xb_headroom, st, s));
  CU(h, launch_split_f16(parts, gbl_ld, ngb, xb0, aop(nsets, 0), aop(nsets, 1), xb_sig, 0, 0, st, s));
  if (T > 0) {
    CU(h, launch_copy_iterate((const float* const*)(w + L.master_of_step), tf(0), ne, st, T, s));
    CU(h, split_x(tf(0), 0, 0, s));
    for (int t = 1; t < T; ++t) CU(h, rebuild(t - 1, tf(t - 1), t, tf(t), t - T, s));
    for (int t = T; t >= 1; --t) CU(h, reverse(t - 1, t - T));
  }
  // segment q (steps c0 + 1 .. c0 + k, c0 = q k): its iterates' operands in buffer b (sets
  // b set1 + j), masters in the segment arenas of b
  auto segm = [&](int b, int j) { return (float*)(w + (b ? L.seg2[(size_t)j] : L.seg[(size_t)j])); };
  auto build_segment = [&](int q, cudaStream_t ss) -> gsp2_status {
    const int c0 = q * k, b = h->adj_overlap ? (q & 1) : 0, o = b * set1;
    const float* ck = (const float*)(w + L.ckpt[(size_t)q]);
    CU(h, split_x(ck, o, c0 + 1, ss));
    for (int j = 1; j < k && c0 + j < M; ++j)
      CU(h, rebuild(o + j - 1, (j == 1) ? ck : segm(b, j - 2), o + j, segm(b, j - 1), c0 + j, ss));
    return GSP2_OK;
  };
  auto reverse_segment = [&](int q) -> gsp2_status {
    const int c0 = q * k, o = (h->adj_overlap ? (q & 1) : 0) * set1;
    for (int i = std::min(c0 + k, M); i >= c0 + 1; --i) CU(h, reverse(o + i - 1 - c0, i));
    return GSP2_OK;
  };
  const int Q = M / k;
  gsp2_status r;
  if (!h->adj_overlap) {
    for (int q = Q; q >= 0; --q) {
      if ((r = build_segment(q, s)) != GSP2_OK) return r;
      if ((r = reverse_segment(q)) != GSP2_OK) return r;
    }
  } else {
    // the side stream rebuilds segment q while the main stream reverses segment q + 1; the
    // rebuild of q waits for the reverse of q + 2, which read the same buffer (forked after
    // the FP64 tail, which uses the first buffer's sets)
    cudaStream_t s2 = h->side_stream;
    cudaEvent_t* ev_b = h->bev.data() + 1;
    cudaEvent_t* ev_r = h->bev.data() + 1 + (Q + 1);
    CU(h, cudaEventRecord(h->bev[0], s));
    CU(h, cudaStreamWaitEvent(s2, h->bev[0], 0));
    for (int q = Q; q >= std::max(0, Q - 1); --q) {
      if ((r = build_segment(q, s2)) != GSP2_OK) return r;
      CU(h, cudaEventRecord(ev_b[q], s2));
    }
    for (int q = Q; q >= 0; --q) {
      CU(h, cudaStreamWaitEvent(s, ev_b[q], 0));
      if ((r = reverse_segment(q)) != GSP2_OK) return r;
      CU(h, cudaEventRecord(ev_r[q], s));
      if (q - 2 >= 0) {
        CU(h, cudaStreamWaitEvent(s2, ev_r[q], 0));
        if ((r = build_segment(q - 2, s2)) != GSP2_OK) return r;
        CU(h, cudaEventRecord(ev_b[q - 2], s2));
      }
    }
  }
  CU(h, launch_adj_hbar<float>(h->n, (const int64_t*)(w + L.rowptr), (const int32_t*)(w + L.colind),
                               (const int64_t*)(w + L.memptr), (const int32_t*)(w + L.mempart),
                               (const int32_t*)(w + L.memloc), parts, Sall, xb0, xb1, hbar, st, s, TC_TILE));
  CU(h, cudaMemsetAsync(w + L.d[0], 0, ab, s));
  CU(h, cudaMemsetAsync(w + L.d[1], 0, ab, s));
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_backward(gsp2_handle h, const double* d_pbar, double* d_hbar, void* stream) {
  if (!usable(h)) return fail(h, GSP2_E_ARG, "invalid handle");
  if (h->opt.ckpt_every <= 0) return fail(h, GSP2_E_STATE, "the adjoint needs a plan built with ckpt_every > 0");
  if (!h->ws || !h->have_forward) return fail(h, GSP2_E_STATE, "gsp2_backward needs a completed density call");
  if (!d_pbar || !d_hbar) return fail(h, GSP2_E_ARG, "NULL Pbar or Hbar buffer");
  int dev = 0;
  CU(h, cudaGetDevice(&dev));
  if (dev != h->device) return fail(h, GSP2_E_STATE, "current device differs from the workspace's device");
  cudaStream_t s = (cudaStream_t)stream;
  if (h->opt.use_graph) {
    if (!h->bexec || h->bkey_pbar != d_pbar || h->bkey_hbar != d_hbar || h->bkey_m != backward_steps(h)) {
      if (h->bexec) cudaGraphExecDestroy(h->bexec);
      h->bexec = nullptr;
      cudaGraph_t g = nullptr;
      CU(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      gsp2_status st = fp64_like(h->opt.precision) ? enqueue_backward(h, d_pbar, d_hbar, h->cap_stream)
                                                   : enqueue_backward_lp(h, d_pbar, d_hbar, h->cap_stream);
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
      if (st != GSP2_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->bexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        h->bexec = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
      }
      h->bkey_pbar = d_pbar;
      h->bkey_hbar = d_hbar;
      h->bkey_m = backward_steps(h);
    }
    CU(h, cudaGraphLaunch(h->bexec, s));
    return GSP2_OK;
  }
  return fp64_like(h->opt.precision) ? enqueue_backward(h, d_pbar, d_hbar, s) : enqueue_backward_lp(h, d_pbar, d_hbar, s);
}

extern "C" void gsp2_destroy(gsp2_handle h) {
  if (!h) return;
  drop_graph(h);
  for (auto& e : h->ev) cudaEventDestroy(e);
  for (auto& e : h->bev) cudaEventDestroy(e);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}
