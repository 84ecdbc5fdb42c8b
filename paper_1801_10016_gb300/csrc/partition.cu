// Host-side partitioning of the dependency graph G_tau for re-planning (Section 2.2,
// Eq. 5; Section 2.3): the CH cost of a partition, and three partitions to choose from by
// that cost when the graph is refreshed between SCF or MD steps (Section 1.1, Fig. 1):
//
//  * block: consecutive vertex indices, part sizes differing by at most one, the larger
//    parts first (the block partitioning of Section 2.3);
//  * graph order: the same blocks over a breadth-first order of G_tau (started from a
//    far vertex of each connected component), so that consecutive vertices are graph
//    neighbours and a block's halo stays small without coordinates;
//  * recursive coordinate bisection over caller-given vertex coordinates.
//
// The graph-partitioning packages the paper uses (METIS and others) are not part of this
// library; these are the partitions it offers.  No device memory is touched.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/gsp2.h"

namespace {

// Eq. 5: sum over parts of (c_i + h_i)^3, h_i the vertices outside part i adjacent in G to
// a core of part i (self loops ignored).
bool ch_sizes(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* part, int32_t nparts,
              std::vector<int64_t>& size) {
  size.assign(nparts, 0);
  for (int64_t v = 0; v < n; ++v) {
    if (part[v] < 0 || part[v] >= nparts) return false;
    size[part[v]]++;
  }
  // halo count of part k: distinct v with part[v] != k adjacent to a core of k; stamp by k
  std::vector<std::vector<int32_t>> cores(nparts);
  for (int64_t v = 0; v < n; ++v) cores[part[v]].push_back((int32_t)v);
  std::vector<int32_t> stamp(n, -1);
  for (int32_t k = 0; k < nparts; ++k)
    for (int32_t u : cores[k])
      for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
        const int32_t v = colind[p];
        if (part[v] != k && stamp[v] != k) {
          stamp[v] = k;
          size[k]++;
        }
      }
  return true;
}

double cost_of(const std::vector<int64_t>& size) {
  double c = 0.0;
  for (int64_t s : size) c += (double)s * (double)s * (double)s;
  return c;
}

// Block partition of the sequence `order` (vertex order[i] takes block(i)).
void blocks_over(const std::vector<int32_t>& order, int32_t nparts, int32_t* part) {
  const int64_t n = (int64_t)order.size();
  const int64_t base = n / nparts, extra = n % nparts;
  int64_t i = 0;
  for (int32_t k = 0; k < nparts; ++k) {
    const int64_t len = base + (k < extra ? 1 : 0);
    for (int64_t q = 0; q < len; ++q) part[order[i++]] = k;
  }
}

// Breadth-first order of every connected component, neighbours in ascending index; each
// component starts at the last vertex a first search from its lowest vertex reaches (a
// far vertex, so that the levels of the second search are long and thin).
std::vector<int32_t> graph_order(int64_t n, const int64_t* rowptr, const int32_t* colind) {
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<uint8_t> seen(n, 0);
  std::vector<int32_t> mark(n, -1), queue;
  queue.reserve(n);
  for (int64_t root = 0; root < n; ++root) {
    if (seen[root]) continue;
    // first search: the last vertex reached from `root`
    queue.clear();
    queue.push_back((int32_t)root);
    mark[root] = (int32_t)root;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int32_t u = queue[h];
      for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
        const int32_t v = colind[p];
        if (mark[v] != (int32_t)root) {
          mark[v] = (int32_t)root;
          queue.push_back(v);
        }
      }
    }
    const int32_t start = queue.back();
    // second search from there gives the order of this component
    const size_t first = order.size();
    order.push_back(start);
    seen[start] = 1;
    for (size_t h = first; h < order.size(); ++h) {
      const int32_t u = order[h];
      for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
        const int32_t v = colind[p];
        if (!seen[v]) {
          seen[v] = 1;
          order.push_back(v);
        }
      }
    }
  }
  return order;
}

// Recursive coordinate bisection: split along the longest extent, the left side taking
// round(count * left parts / parts) vertices ordered by (coordinate, index).
void rcb(int64_t n, const double* xyz, int32_t nparts, int32_t* part) {
  struct Job {
    std::vector<int32_t> idx;
    int32_t p0, np;
  };
  std::vector<Job> stack;
  Job all;
  all.idx.resize(n);
  std::iota(all.idx.begin(), all.idx.end(), 0);
  all.p0 = 0;
  all.np = nparts;
  stack.push_back(std::move(all));
  while (!stack.empty()) {
    Job j = std::move(stack.back());
    stack.pop_back();
    if (j.np == 1) {
      for (int32_t v : j.idx) part[v] = j.p0;
      continue;
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t v : j.idx)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * (int64_t)v + d]);
        hi[d] = std::max(hi[d], xyz[3 * (int64_t)v + d]);
      }
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    std::sort(j.idx.begin(), j.idx.end(), [&](int32_t a, int32_t b) {
      const double ca = xyz[3 * (int64_t)a + ax], cb = xyz[3 * (int64_t)b + ax];
      return ca < cb || (ca == cb && a < b);
    });
    const int32_t nl = j.np / 2;
    const int64_t cnt = (int64_t)j.idx.size();
    int64_t nleft = (int64_t)std::llround((double)cnt * nl / j.np);
    nleft = std::min(std::max(nleft, (int64_t)nl), cnt - (j.np - nl));
    Job a, b;
    a.idx.assign(j.idx.begin(), j.idx.begin() + nleft);
    b.idx.assign(j.idx.begin() + nleft, j.idx.end());
    a.p0 = j.p0;
    a.np = nl;
    b.p0 = j.p0 + nl;
    b.np = j.np - nl;
    stack.push_back(std::move(b));
    stack.push_back(std::move(a));
  }
}

bool valid_graph(int64_t n, const int64_t* rowptr, const int32_t* colind) {
  if (!rowptr || rowptr[0] != 0) return false;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return false;
  if (rowptr[n] > 0 && !colind) return false;
  for (int64_t p = 0; p < rowptr[n]; ++p)
    if (colind[p] < 0 || colind[p] >= n) return false;
  return true;
}

}  // namespace

extern "C" gsp2_status gsp2_partition_cost(int64_t n, const int64_t* g_rowptr, const int32_t* g_colind,
                                           const int32_t* part, int32_t nparts, double* cost, int32_t* sizes) {
  if (n < 1 || n > INT32_MAX || nparts < 1 || !part || !cost || !valid_graph(n, g_rowptr, g_colind))
    return GSP2_E_ARG;
  try {
    std::vector<int64_t> size;
    if (!ch_sizes(n, g_rowptr, g_colind, part, nparts, size)) return GSP2_E_ARG;
    *cost = cost_of(size);
    if (sizes)
      for (int32_t k = 0; k < nparts; ++k) sizes[k] = (int32_t)size[k];
  } catch (const std::bad_alloc&) {
    return GSP2_E_OOM;
  }
  return GSP2_OK;
}

extern "C" gsp2_status gsp2_partition(int64_t n, const int64_t* g_rowptr, const int32_t* g_colind, int32_t nparts,
                                      int32_t method, const double* coords, int32_t* part, int32_t* chosen,
                                      double* cost) {
  if (n < 1 || n > INT32_MAX || nparts < 1 || nparts > n || !part || !valid_graph(n, g_rowptr, g_colind))
    return GSP2_E_ARG;
  if (method < GSP2_PARTITION_AUTO || method > GSP2_PARTITION_RCB) return GSP2_E_ARG;
  if (method == GSP2_PARTITION_RCB && !coords) return GSP2_E_ARG;
  if (coords)
    for (int64_t q = 0; q < 3 * n; ++q)
      if (!std::isfinite(coords[q])) return GSP2_E_ARG;
  try {
    std::vector<int32_t> cand(n);
    double best = INFINITY;
    int32_t best_m = -1;
    std::vector<int64_t> size;
    for (int32_t m = GSP2_PARTITION_BLOCK; m <= GSP2_PARTITION_RCB; ++m) {
      if (method != GSP2_PARTITION_AUTO && m != method) continue;
      if (m == GSP2_PARTITION_RCB && !coords) continue;
      if (m == GSP2_PARTITION_BLOCK) {
        std::vector<int32_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        blocks_over(order, nparts, cand.data());
      } else if (m == GSP2_PARTITION_GRAPH_ORDER) {
        blocks_over(graph_order(n, g_rowptr, g_colind), nparts, cand.data());
      } else {
        rcb(n, coords, nparts, cand.data());
      }
      ch_sizes(n, g_rowptr, g_colind, cand.data(), nparts, size);
      const double c = cost_of(size);
      if (c < best) {  // ties keep the lower method
        best = c;
        best_m = m;
        std::memcpy(part, cand.data(), (size_t)n * sizeof(int32_t));
      }
    }
    if (chosen) *chosen = best_m;
    if (cost) *cost = best;
  } catch (const std::bad_alloc&) {
    return GSP2_E_OOM;
  }
  return GSP2_OK;
}
