// Host-side mesh decomposition and renumbering of the sparse-solver module (Sec. 3.2.1):
// recursive bisection of the cell graph along breadth-first level structures, then a
// Cuthill-McKee numbering of every subdomain with a stable sort on dependency levels.
//
// The paper partitions with SCOTCH's multilevel recursive bisection; this file uses the
// single-level form of graph bisection (George & Liu, "Computer Solution of Large Sparse
// Positive Definite Systems", 1981: level structures rooted at pseudo-peripheral nodes),
// which needs no external library and cuts a mesh along breadth-first fronts.
//
// Subtrees of the bisection and the subdomains of the renumbering are processed by several
// host threads. A cell belongs to exactly one subgraph at a time and each thread writes only
// its own cells; the label of a neighbouring cell, which another thread may be rewriting, is
// read and written with relaxed atomics. Results do not depend on the thread count.
#include "../../include/df_solver.h"

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

namespace dfgb {
df_status fail(df_state* s, df_status code, const char* fmt, ...);
}

namespace {

struct Graph {
  int64_t n = 0;
  std::vector<int64_t> ptr;   // [n + 1]
  std::vector<int32_t> adj;   // neighbours of each cell, in face order
};

Graph build_graph(int64_t n, int64_t nf, const int32_t* owner, const int32_t* neighbour) {
  Graph g;
  g.n = n;
  g.ptr.assign(n + 1, 0);
  for (int64_t f = 0; f < nf; ++f) {
    ++g.ptr[owner[f] + 1];
    ++g.ptr[neighbour[f] + 1];
  }
  for (int64_t c = 0; c < n; ++c) g.ptr[c + 1] += g.ptr[c];
  g.adj.resize(2 * nf);
  std::vector<int64_t> pos(g.ptr.begin(), g.ptr.end() - 1);
  for (int64_t f = 0; f < nf; ++f) {
    g.adj[pos[owner[f]]++] = neighbour[f];
    g.adj[pos[neighbour[f]]++] = owner[f];
  }
  return g;
}

inline int32_t ld(const int32_t* a, int64_t i) { return __atomic_load_n(a + i, __ATOMIC_RELAXED); }
inline void st(int32_t* a, int64_t i, int32_t v) { __atomic_store_n(a + i, v, __ATOMIC_RELAXED); }

struct Ctx {
  const Graph* g;
  int32_t* label;                 // current subgraph of every cell
  int32_t* stamp;                 // breadth-first visit marks (own cells only)
  std::atomic<int32_t> next_label{1};
  std::atomic<int32_t> next_stamp{1};
  int32_t* part_of;
  std::atomic<int> threads_left{0};
};

int64_t degree(const Graph& g, int32_t c) { return g.ptr[c + 1] - g.ptr[c]; }

// Breadth-first order of the cells labelled L reachable from `root`, appended to `out`.
// Neighbours are taken in ascending (degree, index) order when `by_degree` (Cuthill-McKee),
// in adjacency order otherwise. Returns the number of levels; `last` gets the index in `out`
// where the last level begins.
int bfs(Ctx& cx, int32_t L, int32_t root, int32_t mark, bool by_degree, std::vector<int32_t>& out,
        size_t& last) {
  const Graph& g = *cx.g;
  size_t head = out.size();
  out.push_back(root);
  cx.stamp[root] = mark;
  int levels = 0;
  std::vector<int32_t> nb;
  while (head < out.size()) {
    const size_t level_end = out.size();
    last = head;
    ++levels;
    for (; head < level_end; ++head) {
      const int32_t c = out[head];
      nb.clear();
      for (int64_t e = g.ptr[c]; e < g.ptr[c + 1]; ++e) {
        const int32_t v = g.adj[e];
        if (ld(cx.label, v) != L || cx.stamp[v] == mark) continue;
        cx.stamp[v] = mark;
        nb.push_back(v);
      }
      if (by_degree)
        std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
          const int64_t da = degree(g, a), db = degree(g, b);
          return da != db ? da < db : a < b;
        });
      out.insert(out.end(), nb.begin(), nb.end());
    }
  }
  return levels;
}

// Pseudo-peripheral cell of the component of `start` (George & Liu): breadth-first searches
// from the lowest-degree cell of the last level while the eccentricity grows (at most three
// moves). `order` receives the breadth-first order (adjacency order) from the returned cell.
int32_t pseudo_peripheral(Ctx& cx, int32_t L, int32_t start, std::vector<int32_t>& order) {
  const Graph& g = *cx.g;
  int32_t r = start;
  size_t last = 0;
  order.clear();
  int ecc = bfs(cx, L, r, cx.next_stamp++, false, order, last);
  std::vector<int32_t> cand;
  for (int it = 0; it < 3; ++it) {
    int32_t best = order[last];
    for (size_t k = last; k < order.size(); ++k) {
      const int32_t c = order[k];
      if (degree(g, c) < degree(g, best) || (degree(g, c) == degree(g, best) && c < best)) best = c;
    }
    if (best == r) break;
    cand.clear();
    size_t cand_last = 0;
    const int e = bfs(cx, L, best, cx.next_stamp++, false, cand, cand_last);
    if (e <= ecc) break;
    ecc = e;
    r = best;
    order.swap(cand);
    last = cand_last;
  }
  return r;
}

// Breadth-first order of all cells of subgraph L (listed in `cells`, ascending), component by
// component, each grown from a pseudo-peripheral cell: in adjacency order for the bisection,
// in Cuthill-McKee order (neighbours by ascending degree) when `by_degree`.
std::vector<int32_t> level_order(Ctx& cx, int32_t L, const std::vector<int32_t>& cells,
                                 bool by_degree) {
  const Graph& g = *cx.g;
  std::vector<int32_t> out, comp;
  out.reserve(cells.size());
  const int32_t mark = cx.next_stamp++;
  size_t scan = 0;
  while (out.size() < cells.size()) {
    // lowest-degree unvisited cell starts the next component
    int32_t seed = -1;
    for (size_t k = scan; k < cells.size(); ++k) {
      const int32_t c = cells[k];
      if (cx.stamp[c] == mark) continue;
      if (seed < 0 || degree(g, c) < degree(g, seed)) seed = c;
    }
    while (scan < cells.size() && cx.stamp[cells[scan]] == mark) ++scan;
    const int32_t root = pseudo_peripheral(cx, L, seed, comp);
    if (by_degree) {
      // the searches inside pseudo_peripheral used other marks; cells of earlier components
      // keep `mark`, so this search covers exactly the new component
      size_t last = 0;
      bfs(cx, L, root, mark, true, out, last);
    } else {
      for (int32_t c : comp) cx.stamp[c] = mark;
      out.insert(out.end(), comp.begin(), comp.end());
    }
  }
  return out;
}

void bisect(Ctx& cx, std::vector<int32_t> cells, int32_t L, int nparts, int part_base) {
  if (nparts == 1) {
    for (int32_t c : cells) cx.part_of[c] = part_base;
    return;
  }
  std::vector<int32_t> order = level_order(cx, L, cells, false);
  const int ta = nparts / 2, tb = nparts - ta;
  const int64_t m = (int64_t)order.size();
  const int64_t ma = (m * ta + nparts / 2) / nparts;
  const int32_t La = cx.next_label++, Lb = cx.next_label++;
  std::vector<int32_t> A(order.begin(), order.begin() + ma), B(order.begin() + ma, order.end());
  std::sort(A.begin(), A.end());
  std::sort(B.begin(), B.end());
  for (int32_t c : A) st(cx.label, c, La);
  for (int32_t c : B) st(cx.label, c, Lb);
  order.clear();
  order.shrink_to_fit();
  cells.clear();
  cells.shrink_to_fit();
  // one more host thread for the first half of a large subgraph while the budget lasts
  const bool spawn = m > 200000 && cx.threads_left.fetch_sub(1) > 0;
  if (spawn) {
    std::thread th([&cx, A = std::move(A), La, ta, part_base]() mutable {
      bisect(cx, std::move(A), La, ta, part_base);
    });
    bisect(cx, std::move(B), Lb, tb, part_base + ta);
    th.join();
  } else {
    bisect(cx, std::move(A), La, ta, part_base);
    bisect(cx, std::move(B), Lb, tb, part_base + ta);
  }
}

int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::min(32u, std::max(1u, h));
}

}  // namespace

extern "C" {

df_status df_mesh_decompose(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                            const int32_t* neighbour, int32_t n_parts, int32_t* new_of_old,
                            int64_t* part_ptr) {
  using dfgb::fail;
  if (n_cells <= 0 || n_cells >= (int64_t(1) << 31) || n_faces < 0 || n_faces >= (int64_t(1) << 30))
    return fail(nullptr, DF_ERR_INVALID_ARG, "n_cells must be in 1..2^31-1, n_faces in 0..2^30-1");
  if (n_faces > 0 && (!owner || !neighbour))
    return fail(nullptr, DF_ERR_INVALID_ARG, "NULL face array");
  if (!new_of_old || !part_ptr) return fail(nullptr, DF_ERR_INVALID_ARG, "NULL output array");
  if (n_parts < 1 || n_parts > n_cells)
    return fail(nullptr, DF_ERR_INVALID_ARG, "n_parts must be in 1..n_cells");
  for (int64_t f = 0; f < n_faces; ++f) {
    const int32_t a = owner[f], b = neighbour[f];
    if (a < 0 || b < 0 || a >= n_cells || b >= n_cells || a == b)
      return fail(nullptr, DF_ERR_INVALID_ARG, "face %lld joins cells %d and %d", (long long)f, a, b);
  }
  const Graph g = build_graph(n_cells, n_faces, owner, neighbour);
  std::vector<int32_t> label(n_cells, 0), stamp(n_cells, 0), part_of(n_cells, 0);
  Ctx cx;
  cx.g = &g;
  cx.label = label.data();
  cx.stamp = stamp.data();
  cx.part_of = part_of.data();
  cx.threads_left = host_threads() - 1;
  {
    std::vector<int32_t> all(n_cells);
    for (int64_t c = 0; c < n_cells; ++c) all[c] = (int32_t)c;
    bisect(cx, std::move(all), 0, n_parts, 0);
  }

  // subdomain sizes and member lists (ascending cell index)
  std::vector<int64_t> ptr(n_parts + 1, 0);
  for (int64_t c = 0; c < n_cells; ++c) ++ptr[part_of[c] + 1];
  for (int p = 0; p < n_parts; ++p) ptr[p + 1] += ptr[p];
  std::vector<int32_t> members(n_cells);
  {
    std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
    for (int64_t c = 0; c < n_cells; ++c) members[pos[part_of[c]]++] = (int32_t)c;
  }
  // labels = subdomain index (+1, so that 0 never matches), read-only from here on
  for (int64_t c = 0; c < n_cells; ++c) label[c] = part_of[c] + 1;

  // Cuthill-McKee inside every subdomain, then the stable sort on dependency levels
  std::vector<int32_t> cm_pos(n_cells, 0), level(n_cells, 0);
  std::atomic<int> next_part{0};
  auto worker = [&]() {
    for (int p = next_part++; p < n_parts; p = next_part++) {
      const std::vector<int32_t> cells(members.begin() + ptr[p], members.begin() + ptr[p + 1]);
      const std::vector<int32_t> cm = level_order(cx, p + 1, cells, true);
      for (size_t k = 0; k < cm.size(); ++k) cm_pos[cm[k]] = (int32_t)k;
      int32_t max_level = 0;
      for (size_t k = 0; k < cm.size(); ++k) {
        const int32_t c = cm[k];
        int32_t lv = 0;
        for (int64_t e = g.ptr[c]; e < g.ptr[c + 1]; ++e) {
          const int32_t v = g.adj[e];
          if (label[v] == p + 1 && cm_pos[v] < (int32_t)k) lv = std::max(lv, level[v] + 1);
        }
        level[c] = lv;
        max_level = std::max(max_level, lv);
      }
      std::vector<int64_t> cnt(max_level + 2, 0);
      for (int32_t c : cm) ++cnt[level[c] + 1];
      for (int32_t l = 0; l <= max_level; ++l) cnt[l + 1] += cnt[l];
      for (int32_t c : cm) new_of_old[c] = (int32_t)(ptr[p] + cnt[level[c]]++);
    }
  };
  {
    const int nt = std::min(host_threads(), n_parts);
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
  }
  for (int p = 0; p <= n_parts; ++p) part_ptr[p] = ptr[p];
  return DF_OK;
}

df_status df_mesh_renumber(int64_t n_cells, int64_t n_faces, const int32_t* owner,
                           const int32_t* neighbour, const int32_t* new_of_old,
                           int32_t* owner_out, int32_t* neighbour_out, int64_t* face_old,
                           uint8_t* face_flip) {
  using dfgb::fail;
  if (n_cells <= 0 || n_cells >= (int64_t(1) << 31) || n_faces < 0)
    return fail(nullptr, DF_ERR_INVALID_ARG, "bad sizes");
  if (!new_of_old || (n_faces > 0 && (!owner || !neighbour || !owner_out || !neighbour_out || !face_old)))
    return fail(nullptr, DF_ERR_INVALID_ARG, "NULL array");
  std::vector<uint8_t> seen(n_cells, 0);
  for (int64_t c = 0; c < n_cells; ++c) {
    const int32_t v = new_of_old[c];
    if (v < 0 || v >= n_cells || seen[v]) return fail(nullptr, DF_ERR_INVALID_ARG, "new_of_old is not a permutation");
    seen[v] = 1;
  }
  std::vector<int64_t> bucket(n_cells + 1, 0);
  for (int64_t f = 0; f < n_faces; ++f) {
    const int32_t a0 = owner[f], b0 = neighbour[f];
    if (a0 < 0 || b0 < 0 || a0 >= n_cells || b0 >= n_cells || a0 == b0)
      return fail(nullptr, DF_ERR_INVALID_ARG, "face %lld joins cells %d and %d", (long long)f, a0, b0);
    ++bucket[std::min(new_of_old[a0], new_of_old[b0]) + 1];
  }
  for (int64_t c = 0; c < n_cells; ++c) bucket[c + 1] += bucket[c];
  std::vector<int64_t> slot(bucket.begin(), bucket.end() - 1);
  for (int64_t f = 0; f < n_faces; ++f) {
    const int32_t a = new_of_old[owner[f]], b = new_of_old[neighbour[f]];
    face_old[slot[std::min(a, b)]++] = f;
  }
  for (int64_t c = 0; c < n_cells; ++c) {
    std::sort(face_old + bucket[c], face_old + bucket[c + 1], [&](int64_t x, int64_t y) {
      const int32_t nx = std::max(new_of_old[owner[x]], new_of_old[neighbour[x]]);
      const int32_t ny = std::max(new_of_old[owner[y]], new_of_old[neighbour[y]]);
      return nx != ny ? nx < ny : x < y;
    });
  }
  for (int64_t k = 0; k < n_faces; ++k) {
    const int64_t f = face_old[k];
    const int32_t a = new_of_old[owner[f]], b = new_of_old[neighbour[f]];
    owner_out[k] = std::min(a, b);
    neighbour_out[k] = std::max(a, b);
    if (face_flip) face_flip[k] = a > b ? 1 : 0;
  }
  return DF_OK;
}

}  // extern "C"
