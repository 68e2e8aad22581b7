// Host side of libnsi_assemble: mesh preparation at create time (validation,
// CSR pattern, row-gather map, element colouring, packed coordinates), handle
// lifetime and error reporting.  The per-call kernels live in nsi_kernels.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "nsi_internal.cuh"

namespace nsi {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

nsi_status fail(nsi_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

nsi_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? NSI_ERR_OOM : NSI_ERR_CUDA;
}

// run fn(lo, hi) over [0, n) on up to hardware_concurrency threads
static void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, n / 65536));
  if (nt <= 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo < hi) th.emplace_back(fn, lo, hi);
  }
  for (auto& x : th) x.join();
}

template <typename T>
static nsi_status dev_upload(NsiHandle* h, T** dst, const T* src, size_t count, cudaStream_t s) {
  size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  NSI_CUDA(cudaMalloc((void**)dst, bytes));
  h->device_bytes += (int64_t)bytes;
  if (count) NSI_CUDA(cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return NSI_OK;
}

static void free_handle(NsiHandle* h) {
  if (!h) return;
  cudaFree(h->row_ptr);
  cudaFree(h->col_idx);
  cudaFree(h->lnods);
  cudaFree(h->color_elems);
  cudaFree(h->walk_ptr);
  cudaFree(h->walk);
  cudaFree(h->diag_pos);
  cudaFree(h->elem_pos);
  cudaFree(h->exact_list);
  cudaFree(h->long_list);
  cudaFree(h->bad_list);
  cudaFree(h->bad_mask);
  cudaFree(h->long_ptr);
  cudaFree(h->long_inc);
  cudaFree(h->exact_ptr);
  cudaFree(h->exact_inc);
  cudaFree(h->star_word);
  cudaFree(h->star_task);
  cudaFree(h->fan);
  cudaFree(h->fan_blk);
  cudaFree(h->xyz64);
  cudaFree(h->xyz_hi);
  cudaFree(h->xyz_lo);
  cudaFree(h->err);
  cudaFree(h->rec);
  cudaFree(h->stage);
  for (cudaEvent_t e : h->chunk_ev)
    if (e) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
}

// Mesh preparation ---------------------------------------------------------
// The element walk of one row: the order in which the row-gather kernel visits
// the elements of the star of node i, and the one-byte steps that drive it.
// Every element of the star is a triangle of row positions (the face opposite
// i, listed so that (i, a, b, c) has the element's orientation).  Two
// triangles that share two positions are neighbours; the walk follows paths of
// that neighbour graph, so consecutive elements share an edge and each step
// brings one new node into a window of two (the kernel keeps the window in
// registers and reads one node's data per element instead of three).  A path
// starts with two steps that only fill the window; a later path first flushes
// the window with two steps on the diagonal position dp, whose slot stays
// zero until the kernel writes the diagonal.  The kernel prefetches the next
// step's node while the current element is evaluated, so a step never brings
// in a node held by the previous step (dp excepted); the encoder checks this.
struct WalkWork {  // per-thread buffers of encode_walk
  std::vector<std::pair<int, int>> ed;
  std::vector<int> adj, nadj, cand, ncand, idx, path, best;
  std::vector<char> used;
};

static bool encode_walk(const uint16_t* tri, int m, int dp, std::vector<uint8_t>& out, WalkWork& ws) {
  constexpr int MAXN = 8;  // neighbours kept per triangle (3 in a manifold link)
  auto P = [&](int t, int c) { return (int)((tri[t] >> (STAR_BITS * c)) & (STAR_MAX_ROW - 1)); };
  auto has = [&](int t, int v) { return P(t, 0) == v || P(t, 1) == v || P(t, 2) == v; };
  // (a, b) consecutive in t's cyclic order: (a, b, third) is an even permutation
  auto even = [&](int t, int a, int b) {
    for (int c = 0; c < 3; ++c)
      if (P(t, c) == a && P(t, (c + 1) % 3) == b) return true;
    return false;
  };
  // neighbours through shared edges (sorted edge records)
  auto& ed = ws.ed;
  ed.clear();
  for (int t = 0; t < m; ++t)
    for (int c = 0; c < 3; ++c) {
      const int a = P(t, c), b = P(t, (c + 1) % 3);
      ed.push_back({std::min(a, b) * STAR_MAX_ROW + std::max(a, b), t});
    }
  std::sort(ed.begin(), ed.end());
  ws.adj.assign((size_t)m * MAXN, -1);
  ws.nadj.assign(m, 0);
  for (size_t x = 0; x < ed.size();) {
    size_t y = x;
    while (y < ed.size() && ed[y].first == ed[x].first) ++y;
    for (size_t a = x; a < y; ++a)
      for (size_t b = x; b < y; ++b) {
        const int ta = ed[a].second, tb = ed[b].second;
        if (ta == tb || ws.nadj[ta] == MAXN) continue;
        bool dup = false;
        for (int k = 0; k < ws.nadj[ta]; ++k) dup |= ws.adj[ta * MAXN + k] == tb;
        if (!dup) ws.adj[ta * MAXN + ws.nadj[ta]++] = tb;
      }
    x = y;
  }
  // path cover: depth-first search for a long path, neighbours with the fewest
  // unvisited neighbours first, with bounded work per path
  auto& used = ws.used;  // 0 free, 1 emitted, 2 on the current path
  used.assign(m, 0);
  auto deg = [&](int t) {
    int d = 0;
    for (int k = 0; k < ws.nadj[t]; ++k) d += used[ws.adj[t * MAXN + k]] == 0;
    return d;
  };
  auto by_deg = [&](int* a, int n) {  // insertion sort, n <= MAXN
    for (int x = 1; x < n; ++x)
      for (int y = x; y > 0 && deg(a[y]) < deg(a[y - 1]); --y) std::swap(a[y], a[y - 1]);
  };
  ws.cand.assign((size_t)m * MAXN, 0);
  ws.ncand.assign(m, 0);
  ws.idx.assign(m, 0);
  std::vector<std::vector<int>> paths;
  int left = m;
  while (left > 0) {
    auto& best = ws.best;
    auto& path = ws.path;
    best.clear();
    int starts[3], nst = 0;
    {  // up to three free triangles with the fewest free neighbours
      int dbest[3];
      for (int t = 0; t < m; ++t) {
        if (used[t]) continue;
        const int d = deg(t);
        int x = nst < 3 ? nst++ : 3;
        while (x > 0 && dbest[x - 1] > d) {
          if (x < 3) {
            starts[x] = starts[x - 1];
            dbest[x] = dbest[x - 1];
          }
          --x;
        }
        if (x < 3) {
          starts[x] = t;
          dbest[x] = d;
        }
      }
    }
    int work = 0;
    const int budget = 64 * m + 256;
    for (int k = 0; k < nst && (int)best.size() < left; ++k) {
      path.assign(1, starts[k]);
      used[starts[k]] = 2;
      ws.idx[0] = -1;  // candidates of this depth not listed yet
      while (!path.empty()) {
        if (path.size() > best.size()) best = path;
        if ((int)best.size() == left || work > budget) break;
        const int d = (int)path.size() - 1;
        int* cd = &ws.cand[(size_t)d * MAXN];
        if (ws.idx[d] < 0) {
          const int t = path[d];
          int nc = 0;
          for (int a = 0; a < ws.nadj[t]; ++a)
            if (!used[ws.adj[t * MAXN + a]]) cd[nc++] = ws.adj[t * MAXN + a];
          by_deg(cd, nc);
          ws.ncand[d] = nc;
          ws.idx[d] = 0;
        }
        if (ws.idx[d] < ws.ncand[d]) {
          const int u = cd[ws.idx[d]++];
          if (used[u]) continue;
          ++work;
          used[u] = 2;
          path.push_back(u);
          ws.idx[d + 1] = -1;
        } else {
          used[path.back()] = 0;
          path.pop_back();
        }
      }
      for (int t : path) used[t] = 0;
    }
    for (int t : best) used[t] = 1;
    left -= (int)best.size();
    paths.push_back(best);
  }
  // emission, simulating the kernel's window (wp, wq) and the nodes held by
  // the previous step (r0, r1, r2)
  int wp = dp, wq = dp, r0 = dp, r1 = dp, r2 = dp;
  auto emit = [&](int c, bool elem, bool neg, bool evq) {
    if (c != dp && (c == r0 || c == r1 || c == r2)) return false;
    out.push_back((uint8_t)(c | (elem ? WALK_ELEM : 0u) | (neg ? WALK_NEG : 0u) | (evq ? WALK_EVQ : 0u)));
    r0 = wp;
    r1 = wq;
    r2 = c;
    if (!evq) wp = wq;  // p leaves: q's node moves to p
    wq = c;             // the newest node is always q
    return true;
  };
  for (size_t pi = 0; pi < paths.size(); ++pi) {
    std::vector<int> path = paths[pi];
    if (pi > 0) {  // flush: dp into both window registers
      emit(dp, false, false, false);
      emit(dp, false, false, false);
    }
    // first element (x, y, z) in its own order, z on the edge shared with the
    // next element; x must not be a node the flush still holds
    const int t0 = path[0];
    int x = -1, y = -1, z = -1;
    for (int c = 0; c < 3 && x < 0; ++c) {
      const int zc = P(t0, c);
      if (path.size() > 1 && !has(path[1], zc)) continue;
      const int xc = P(t0, (c + 1) % 3);
      if (xc != dp && (xc == r0 || xc == r1 || xc == r2)) continue;
      x = xc;
      y = P(t0, (c + 2) % 3);
      z = zc;
    }
    if (x < 0 || !emit(x, false, false, false) || !emit(y, false, false, false)) return false;  // window (x, y)
    for (size_t k = 0; k < path.size(); ++k) {
      const int t = path[k];
      if (!has(t, wp) || !has(t, wq)) return false;
      const int c = k == 0 ? z : P(t, 0) ^ P(t, 1) ^ P(t, 2) ^ wp ^ wq;
      bool evq = false;
      bool split = false;
      if (k + 1 < path.size()) {
        const int nx = path[k + 1];
        if (has(nx, c) && has(nx, wq))
          evq = false;
        else if (has(nx, c) && has(nx, wp))
          evq = true;
        else
          split = true;  // the next element shares the window's own edge
      }
      if (!emit(c, true, !even(t, wp, wq), evq)) return false;
      if (split) {
        paths.push_back(std::vector<int>(path.begin() + k + 1, path.end()));
        break;
      }
    }
  }
  return true;
}

static nsi_status build(NsiHandle* h, const NsiMesh* m, cudaStream_t s) {
  const int64_t n = h->n, E = h->E;
  std::vector<int32_t> ln(4 * E);
  std::vector<double> X(n), Y(n), Z(n);
  if (E) NSI_CUDA(cudaMemcpy(ln.data(), m->lnods, sizeof(int32_t) * 4 * E, cudaMemcpyDeviceToHost));
  NSI_CUDA(cudaMemcpy(X.data(), m->x, sizeof(double) * n, cudaMemcpyDeviceToHost));
  NSI_CUDA(cudaMemcpy(Y.data(), m->y, sizeof(double) * n, cudaMemcpyDeviceToHost));
  NSI_CUDA(cudaMemcpy(Z.data(), m->z, sizeof(double) * n, cudaMemcpyDeviceToHost));

  // 1. validate indices and orientation (det J > 0, in double)
  std::atomic<int64_t> bad_index{-1}, bad_det{-1};
  parallel_for(E, [&](int64_t lo, int64_t hi) {
    for (int64_t e = lo; e < hi; ++e) {
      const int32_t* v = &ln[4 * e];
      bool ok = true;
      for (int a = 0; a < 4; ++a) ok &= (v[a] >= 0 && v[a] < n);
      if (!ok) {
        int64_t exp = -1;
        bad_index.compare_exchange_strong(exp, e);
        continue;
      }
      V3<double> x0{X[v[0]], Y[v[0]], Z[v[0]]};
      V3<double> d1 = sub(V3<double>{X[v[1]], Y[v[1]], Z[v[1]]}, x0);
      V3<double> d2 = sub(V3<double>{X[v[2]], Y[v[2]], Z[v[2]]}, x0);
      V3<double> d3 = sub(V3<double>{X[v[3]], Y[v[3]], Z[v[3]]}, x0);
      double det = dot(d1, cross(d2, d3));
      if (!(det > 0.0)) {
        int64_t exp = -1;
        bad_det.compare_exchange_strong(exp, e);
      }
    }
  });
  if (bad_index.load() >= 0)
    return fail(NSI_ERR_BAD_MESH, "element " + std::to_string(bad_index.load()) + " has a node index outside [0, n_nodes)");
  if (bad_det.load() >= 0)
    return fail(NSI_ERR_BAD_MESH, "element " + std::to_string(bad_det.load()) + " is inverted or degenerate (det J <= 0)");

  // 2. node -> element incidence (elements ascending per node)
  std::vector<int64_t> inc_ptr(n + 1, 0);
  for (int64_t t = 0; t < 4 * E; ++t) inc_ptr[ln[t] + 1]++;
  for (int64_t i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
  std::vector<int64_t> inc(4 * E);  // e * 4 + a
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 4; ++a) inc[fill[ln[4 * e + a]]++] = e * 4 + a;
  }

  // 3. CSR pattern: row i = sorted set of nodes sharing an element with i
  //    (node i itself included; a node in no element has an empty row)
  std::vector<int64_t> row_len(n);
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    std::vector<int32_t> buf;
    for (int64_t i = lo; i < hi; ++i) {
      buf.clear();
      for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
        int64_t e = inc[t] >> 2;
        for (int a = 0; a < 4; ++a) buf.push_back(ln[4 * e + a]);
      }
      std::sort(buf.begin(), buf.end());
      row_len[i] = std::unique(buf.begin(), buf.end()) - buf.begin();
    }
  });
  std::vector<int64_t> rp64(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) rp64[i + 1] = rp64[i] + row_len[i];
  const int64_t nnz = rp64[n];
  if (nnz > INT32_MAX) return fail(NSI_ERR_UNSUPPORTED, "nnz exceeds int32 CSR indices");
  h->nnz = nnz;
  std::vector<int32_t> row_ptr(n + 1), col(nnz);
  for (int64_t i = 0; i <= n; ++i) row_ptr[i] = (int32_t)rp64[i];
  int64_t max_row = 0;
  for (int64_t i = 0; i < n; ++i) max_row = std::max(max_row, row_len[i]);
  h->max_row = (int)max_row;
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    std::vector<int32_t> buf;
    for (int64_t i = lo; i < hi; ++i) {
      buf.clear();
      for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
        int64_t e = inc[t] >> 2;
        for (int a = 0; a < 4; ++a) buf.push_back(ln[4 * e + a]);
      }
      std::sort(buf.begin(), buf.end());
      int64_t k = std::unique(buf.begin(), buf.end()) - buf.begin();
      std::copy(buf.begin(), buf.begin() + k, col.begin() + rp64[i]);
    }
  });

  // 4. row-gather map (positions of the other three nodes in the row).  Rows
  //    of more than 32 entries (five bits of row position) are "long rows":
  //    the row gather leaves them out and long_rows_kernel computes them.
  h->gather_ok = inc_ptr[n] <= INT32_MAX;
  std::vector<uint16_t> star;
  std::vector<uint8_t> diag(n, 0);
  std::vector<uint8_t> is_long(n, 0);
  for (int64_t i = 0; i < n; ++i) is_long[i] = row_len[i] > STAR_MAX_ROW;
  if (h->gather_ok) {
    star.resize(inc_ptr[n]);
    // even permutations of (0,1,2,3) that bring vertex a to the front
    static const int EVEN[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
    parallel_for(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        const int32_t* c = &col[rp64[i]];
        int64_t len = row_len[i];
        if (is_long[i]) {
          diag[i] = DIAG_LONG;
          continue;
        }
        auto pos = [&](int32_t j) { return (int)(std::lower_bound(c, c + len, j) - c); };
        diag[i] = len ? (uint8_t)pos((int32_t)i) : 0;
        for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
          int64_t e = inc[t] >> 2;
          int a = (int)(inc[t] & 3);
          unsigned w = 0;
          for (int m2 = 0; m2 < 3; ++m2) w |= (unsigned)pos(ln[4 * e + EVEN[a][m2]]) << (STAR_BITS * m2);
          star[t] = (uint16_t)w;
        }
      }
    });
  }

  // 4.5 element-position map for the element-centric kernels (colouring,
  //     atomics): the row position of every other node of each element
  const bool pos_ok = max_row <= STAR_MAX_ROW;
  std::vector<unsigned long long> elem_pos;
  if (pos_ok) {
    elem_pos.assign(E, 0ull);
    parallel_for(E, [&](int64_t lo, int64_t hi) {
      for (int64_t e = lo; e < hi; ++e) {
        const int32_t* v = &ln[4 * e];
        unsigned long long w = 0;
        for (int a = 0; a < 4; ++a) {
          const int32_t* c = &col[rp64[v[a]]];
          const int64_t len = row_len[v[a]];
          for (int b = 0; b < 4; ++b) {
            if (b == a) continue;
            const unsigned long long q = (unsigned long long)(std::lower_bound(c, c + len, v[b]) - c);
            w |= q << (ELEM_POS_BITS * elem_pos_slot(a, b));
          }
        }
        elem_pos[e] = w;
      }
    });
  }

  // 4a. every row's element walk (the order and steps of the kernel's element loop)
  std::vector<int32_t> walk_ptr;
  std::vector<uint8_t> walk;
  if (h->gather_ok) {
    std::vector<int32_t> wlen(n, 0);
    std::vector<std::pair<int64_t, std::vector<uint8_t>>> parts;
    std::mutex mu;
    std::atomic<bool> bad{false};
    parallel_for(n, [&](int64_t lo, int64_t hi) {
      std::vector<uint8_t> buf;
      WalkWork ws;
      for (int64_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); ++i) {
        const size_t before = buf.size();
        if (!is_long[i] && !encode_walk(&star[inc_ptr[i]], (int)(inc_ptr[i + 1] - inc_ptr[i]), diag[i], buf, ws)) {
          // a star the encoder cannot walk: the row becomes a long row
          buf.resize(before);
          is_long[i] = 1;
          diag[i] = DIAG_LONG;
        }
        wlen[i] = (int32_t)(buf.size() - before);
      }
      std::lock_guard<std::mutex> g(mu);
      parts.emplace_back(lo, std::move(buf));
    });
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += wlen[i];
    if (bad.load() || total > INT32_MAX - 64) {
      h->gather_ok = false;
    } else {
      walk_ptr.assign(n + 1, 0);
      for (int64_t i = 0; i < n; ++i) walk_ptr[i + 1] = walk_ptr[i] + wlen[i];
      std::sort(parts.begin(), parts.end(),
                [](const std::pair<int64_t, std::vector<uint8_t>>& a, const std::pair<int64_t, std::vector<uint8_t>>& b) {
                  return a.first < b.first;
                });
      walk.reserve(total + 8);
      for (auto& pr : parts) walk.insert(walk.end(), pr.second.begin(), pr.second.end());
      walk.resize(total + 8, 0);  // the kernel copies whole aligned words
    }
  }

  // 4b. edge-fan map: per off-diagonal entry (i, j) the ring of nodes around the edge
  std::vector<uint32_t> fan;
  std::vector<int32_t> fan_blk;
  h->fan_ok = h->gather_ok && max_row <= FAN_MAX_ROW &&
              std::find(is_long.begin(), is_long.end(), (uint8_t)1) == is_long.end();
  if (h->fan_ok) {
    fan.assign(nnz, 0u);
    std::atomic<bool> bad{false};
    parallel_for(n, [&](int64_t lo, int64_t hi) {
      int nxt[FAN_MAX_ROW], prv[FAN_MAX_ROW];
      for (int64_t i = lo; i < hi && !bad.load(std::memory_order_relaxed); ++i) {
        const int len = (int)row_len[i];
        const int dp = diag[i];
        for (int q = 0; q < len; ++q) {
          if (q == dp) continue;
          for (int v = 0; v < len; ++v) nxt[v] = prv[v] = -1;
          int edges = 0;
          bool ok = true;
          // every element of the star holding q: (i, q, k, l) as an even permutation
          for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) {
            const unsigned w = star[t];
            const int p1 = w & 31, p2 = (w >> 5) & 31, p3 = (w >> 10) & 31;
            int k, l;
            if (p1 == q) { k = p2; l = p3; }
            else if (p2 == q) { k = p3; l = p1; }
            else if (p3 == q) { k = p1; l = p2; }
            else continue;
            if (nxt[k] != -1 || prv[l] != -1) { ok = false; break; }
            nxt[k] = l;
            prv[l] = k;
            ++edges;
          }
          if (!ok || edges == 0) { bad = true; break; }
          // chain: start at a node without predecessor (open fan) or anywhere (closed)
          int start = -1, nodes = 0;
          for (int v = 0; v < len; ++v)
            if (nxt[v] != -1 && prv[v] == -1) start = v;
          const bool closed = start == -1;
          if (closed)
            for (int v = 0; v < len && start == -1; ++v)
              if (nxt[v] != -1) start = v;
          uint32_t word = 0;
          int v = start;
          while (v != -1 && nodes <= FAN_MAX_RING) {
            if (nodes < FAN_MAX_RING) word |= (uint32_t)v << (4 * nodes);
            ++nodes;
            v = nxt[v];
            if (v == start) break;
          }
          if (nodes > FAN_MAX_RING || edges != (closed ? nodes : nodes - 1)) { bad = true; break; }
          word |= (uint32_t)nodes << 24;
          if (closed) word |= 1u << 27;
          fan[rp64[i] + q] = word;
        }
      }
    });
    if (bad.load()) {
      h->fan_ok = false;
      fan.clear();
    }
  }
  if (h->fan_ok) {
    // blocks of whole rows holding at most FAN_BLOCK entries
    fan_blk.push_back(0);
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (acc + row_len[i] > FAN_BLOCK) {
        fan_blk.push_back((int32_t)i);
        acc = 0;
      }
      acc += row_len[i];
    }
    fan_blk.push_back((int32_t)n);
    h->fan_blocks = (int64_t)fan_blk.size() - 1;
  }

  // 5. greedy element colouring: no two elements of one colour share a node
  std::vector<int32_t> color(E);
  {
    std::vector<uint64_t> used;  // per node, 64 colours per word, grown on demand
    int words = 1;
    used.assign(n, 0);
    std::vector<std::vector<uint64_t>> extra;  // colours >= 64 (rare)
    int ncol = 0;
    for (int64_t e = 0; e < E; ++e) {
      const int32_t* v = &ln[4 * e];
      uint64_t m0 = used[v[0]] | used[v[1]] | used[v[2]] | used[v[3]];
      int c = -1;
      if (~m0) c = __builtin_ctzll(~m0);
      else {
        for (int w = 0; w < (int)extra.size() && c < 0; ++w) {
          uint64_t mw = extra[w][v[0]] | extra[w][v[1]] | extra[w][v[2]] | extra[w][v[3]];
          if (~mw) c = 64 * (w + 1) + __builtin_ctzll(~mw);
        }
        if (c < 0) {
          extra.emplace_back(n, 0);
          c = 64 * (int)extra.size();
          words++;
        }
      }
      color[e] = c;
      ncol = std::max(ncol, c + 1);
      for (int a = 0; a < 4; ++a) {
        if (c < 64) used[v[a]] |= 1ull << c;
        else extra[c / 64 - 1][v[a]] |= 1ull << (c % 64);
      }
    }
    (void)words;
    h->n_colors = ncol;
  }
  std::vector<int32_t> color_elems(E);
  h->color_off.assign(h->n_colors + 1, 0);
  for (int64_t e = 0; e < E; ++e) h->color_off[color[e] + 1]++;
  for (int c = 0; c < h->n_colors; ++c) h->color_off[c + 1] += h->color_off[c];
  {
    std::vector<int64_t> fill(h->color_off.begin(), h->color_off.end() - 1);
    for (int64_t e = 0; e < E; ++e) color_elems[fill[color[e]]++] = (int32_t)e;
  }

  // 6. packed coordinates
  std::vector<D4> xyz64;
  std::vector<float4> xhi, xlo;
  if (h->precision == NSI_FP64) {
    xyz64.resize(n);
    for (int64_t i = 0; i < n; ++i) xyz64[i] = D4{X[i], Y[i], Z[i], 0.0};
  } else {
    xhi.resize(n);
    xlo.resize(n);
    for (int64_t i = 0; i < n; ++i) {
      float hx = (float)X[i], hy = (float)Y[i], hz = (float)Z[i];
      xhi[i] = make_float4(hx, hy, hz, 0.0f);
      xlo[i] = make_float4((float)(X[i] - hx), (float)(Y[i] - hy), (float)(Z[i] - hz), 0.0f);
    }
  }

  // 7. gather launch plan: largest rows-per-block whose entries fit the budget
  {
    // rows per block chosen for the most resident warps per SM (shared memory
    // of the block's layout, the kernel's registers, 2048 threads per SM); on
    // a tie the smallest block, whose barriers hold fewer warps
    const size_t smem_sm = 228 * 1024, smem_max = 200 * 1024;
    const int regs = std::max(32, gather_kernel_regs(h->precision));
    int64_t short_max = 0;
    for (int64_t i = 0; i < n; ++i)
      if (!is_long[i]) short_max = std::max(short_max, row_len[i]);
    int chosen = 0, best_warps = 0;
    for (int R : {32, 64, 96, 128}) {
      if (!h->gather_ok) break;
      int64_t mL = 0, mS = 0;
      for (int64_t r0 = 0; r0 < n; r0 += R) {
        const int64_t r1 = std::min(n, r0 + R);
        mL = std::max<int64_t>(mL, rp64[r1] - rp64[r0]);
        mS = std::max<int64_t>(mS, walk_ptr[r1] - walk_ptr[r0]);
      }
      // slots per row: the longest row the kernel takes, or more where a
      // block's long rows would not leave room for its entries in R * w
      const int W = (int)std::max<int64_t>({1, short_max, (mL + R - 1) / R});
      const GatherSmem g = gather_smem(h->precision, R, W, (int)mL, (int)mS);
      const size_t sm = g.total();
      if (sm > smem_max || !g.stage_fits()) continue;
      int blocks = (int)std::min<size_t>({smem_sm / (sm + 1024), (size_t)32, (size_t)(2048 / R),
                                          (size_t)(65536 / (R * regs))});
      const int warps = blocks * R / 32;
      GatherPlan cand;
      cand.rows_per_block = R;
      cand.max_block_entries = (int)mL;
      cand.max_block_steps = (int)mS;
      cand.w = W;
      cand.n_blocks = (n + R - 1) / R;
      h->plans[h->n_plans++] = cand;
      if (warps > best_warps) {
        best_warps = warps;
        chosen = h->n_plans - 1;
      }
    }
    if (best_warps == 0) h->gather_ok = false;
    else h->plan = h->plans[chosen];
    // the persistent grid (next block's phase 0 under the current block's
    // write-out) measured faster for the mixed modes: mixed64 0.280 against
    // 0.302 ms, mixed32 0.228 against 0.239 ms at the 100^3 cube; it slowed
    // FP64 (4.23 against 3.29 ms, on an earlier kernel)
    h->persistent = h->precision != NSI_FP64;
  }

  // 7b. badly shaped elements (mixed modes): a float determinant of an
  // element with |d1||d2||d3| > EXACT_RATIO |det| (edge vectors from any of its
  // nodes) would carry about that ratio times the float rounding of the edge
  // vectors.  The rows of all four nodes of such an element are listed; after
  // the assembly they are recomputed in double (exact_rows_kernel).
  std::vector<int32_t> exact_list, exact_ptr, bad_list;
  std::vector<uint32_t> exact_inc;
  if (h->precision != NSI_FP64) {
    std::vector<uint8_t> flag(n, 0);
    for (int64_t e = 0; e < E; ++e) {
      const int32_t* v = &ln[4 * e];
      double worst = 0.0;
      for (int a = 0; a < 4; ++a) {
        const V3<double> x0{X[v[a]], Y[v[a]], Z[v[a]]};
        V3<double> d[3];
        for (int b = 0, c = 0; b < 4; ++b)
          if (b != a) d[c++] = sub(V3<double>{X[v[b]], Y[v[b]], Z[v[b]]}, x0);
        const double det = std::fabs(dot(d[0], cross(d[1], d[2])));
        const double had = std::sqrt(dot(d[0], d[0]) * dot(d[1], d[1]) * dot(d[2], d[2]));
        worst = std::max(worst, had / det);
      }
      if (worst > EXACT_RATIO) {
        for (int a = 0; a < 4; ++a) flag[v[a]] = 1;
        bad_list.push_back((int32_t)e);
      }
    }
    for (int64_t i = 0; i < n; ++i)
      if (flag[i] && row_len[i] <= STAR_MAX_ROW) exact_list.push_back((int32_t)i);
    h->exact_rows = (int64_t)exact_list.size();
    // every listed row's incident elements (element * 4 + local index of the node)
    exact_ptr.assign(exact_list.size() + 1, 0);
    for (size_t r = 0; r < exact_list.size(); ++r) {
      const int64_t i = exact_list[r];
      for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) exact_inc.push_back((uint32_t)inc[t]);
      exact_ptr[r + 1] = (int32_t)exact_inc.size();
    }
    if (E > (int64_t)(UINT32_MAX >> 2)) h->exact_rows = 0;  // not encodable: keep the float results
  }

  // 7c. long rows: every incident element of each (element * 4 + local index)
  std::vector<int32_t> long_list, long_ptr;
  std::vector<uint32_t> long_inc;
  if (h->gather_ok) {
    for (int64_t i = 0; i < n; ++i)
      if (is_long[i]) long_list.push_back((int32_t)i);
    long_ptr.assign(long_list.size() + 1, 0);
    for (size_t r = 0; r < long_list.size(); ++r) {
      const int64_t i = long_list[r];
      for (int64_t t = inc_ptr[i]; t < inc_ptr[i + 1]; ++t) long_inc.push_back((uint32_t)inc[t]);
      long_ptr[r + 1] = (int32_t)long_inc.size();
    }
    if (!long_list.empty() && (E > (int64_t)(UINT32_MAX >> 2) || long_inc.size() > (size_t)INT32_MAX))
      h->gather_ok = false;
    h->long_rows = h->gather_ok ? (int64_t)long_list.size() : 0;
  }

  // 8. upload
  nsi_status st;
  if ((st = dev_upload(h, &h->row_ptr, row_ptr.data(), n + 1, s))) return st;
  h->row_ptr_host = row_ptr;
  if ((st = dev_upload(h, &h->col_idx, col.data(), nnz, s))) return st;
  if ((st = dev_upload(h, &h->lnods, reinterpret_cast<const int4*>(ln.data()), E, s))) return st;
  if ((st = dev_upload(h, &h->color_elems, color_elems.data(), E, s))) return st;
  if (h->fan_ok) {
    // available to the autotuner / nsi_set_launch; the per-row star kernel stays
    // the default (each element is evaluated 3 times per row in the fan kernel,
    // which costs more than the shared-memory accumulation it saves on GB300)
    if ((st = dev_upload(h, &h->fan, fan.data(), fan.size(), s))) return st;
    if ((st = dev_upload(h, &h->fan_blk, fan_blk.data(), fan_blk.size(), s))) return st;
  }
  if (h->gather_ok) {
    if ((st = dev_upload(h, &h->walk_ptr, walk_ptr.data(), n + 1, s))) return st;
    if ((st = dev_upload(h, &h->walk, walk.data(), walk.size(), s))) return st;
  }
  if (pos_ok || h->gather_ok) {
    if ((st = dev_upload(h, &h->diag_pos, diag.data(), n, s))) return st;
  }
  if (pos_ok) {
    if ((st = dev_upload(h, &h->elem_pos, elem_pos.data(), E, s))) return st;
  }
  if (h->long_rows > 0) {
    if ((st = dev_upload(h, &h->long_list, long_list.data(), long_list.size(), s))) return st;
    if ((st = dev_upload(h, &h->long_ptr, long_ptr.data(), long_ptr.size(), s))) return st;
    if ((st = dev_upload(h, &h->long_inc, long_inc.data(), long_inc.size(), s))) return st;
  }
  if (!bad_list.empty() && E <= (int64_t)INT32_MAX) {
    std::vector<uint32_t> mask((size_t)(E + 31) / 32, 0u);
    for (int32_t e : bad_list) mask[e >> 5] |= 1u << (e & 31);
    h->n_bad = (int64_t)bad_list.size();
    if ((st = dev_upload(h, &h->bad_list, bad_list.data(), bad_list.size(), s))) return st;
    if ((st = dev_upload(h, &h->bad_mask, mask.data(), mask.size(), s))) return st;
  }
  if (h->exact_rows > 0) {
    if ((st = dev_upload(h, &h->exact_list, exact_list.data(), exact_list.size(), s))) return st;
    if ((st = dev_upload(h, &h->exact_ptr, exact_ptr.data(), exact_ptr.size(), s))) return st;
    if ((st = dev_upload(h, &h->exact_inc, exact_inc.data(), exact_inc.size(), s))) return st;
  }
  // the stabilised block's row kernel: star words and warp tasks of one row
  // (up to 32 entries, or a long row, which the kernel skips) or two
  // consecutive rows of at most 16 entries each
  std::vector<int4> star_task;
  if (h->gather_ok) {
    for (int64_t i = 0; i < n;) {
      const bool pair = i + 1 < n && !is_long[i] && !is_long[i + 1] && row_len[i] <= 16 && row_len[i + 1] <= 16;
      const int64_t e = i + (pair ? 2 : 1);
      const int d0 = is_long[i] ? 0 : diag[i], d1 = pair ? diag[i + 1] : 0;
      star_task.push_back(int4{(int)i, (int)rp64[i], (int)rp64[i + 1], (int)rp64[e]});
      star_task.push_back(int4{(int)inc_ptr[i], (int)inc_ptr[i + 1], (int)inc_ptr[e],
                               d0 | (d1 << 8) | ((int)(e - i) << 16) | ((is_long[i] ? 1 : 0) << 24)});
      i = e;
    }
    h->n_star_tasks = (int64_t)star_task.size() / 2;
    if ((st = dev_upload(h, &h->star_word, star.data(), star.size(), s))) return st;
    if ((st = dev_upload(h, &h->star_task, star_task.data(), star_task.size(), s))) return st;
  }
  if (h->precision == NSI_FP64) {
    if ((st = dev_upload(h, &h->xyz64, xyz64.data(), n, s))) return st;
  } else {
    if ((st = dev_upload(h, &h->xyz_hi, xhi.data(), n, s))) return st;
    if ((st = dev_upload(h, &h->xyz_lo, xlo.data(), n, s))) return st;
  }
  if (h->gather_ok) {
    h->rec_bytes = h->precision == NSI_FP64 ? 64 : 32;
    NSI_CUDA(cudaMalloc(&h->rec, (size_t)h->rec_bytes * n));
    h->device_bytes += (int64_t)h->rec_bytes * n;
  }
  NSI_CUDA(cudaMalloc((void**)&h->err, sizeof(unsigned)));
  NSI_CUDA(cudaMemsetAsync(h->err, 0, sizeof(unsigned), s));
  NSI_CUDA(cudaStreamSynchronize(s));  // host vectors die at return
  return NSI_OK;
}

}  // namespace nsi

using namespace nsi;

extern "C" {

int32_t nsi_abi_version(void) { return NSI_ABI_VERSION; }

const char* nsi_last_error(void) { return g_last_error.c_str(); }

nsi_status nsi_assemble_create(const NsiMesh* mesh, const NsiOptions* opts, void* stream, NsiHandle** out) {
  if (!out) return fail(NSI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !opts) return fail(NSI_ERR_INVALID_ARG, "mesh or opts is NULL");
  if (mesh->n_nodes <= 0 || mesh->n_elems < 0) return fail(NSI_ERR_INVALID_ARG, "n_nodes must be > 0 and n_elems >= 0");
  if (mesh->n_nodes > INT32_MAX || mesh->n_elems > INT32_MAX)
    return fail(NSI_ERR_UNSUPPORTED, "more than 2^31-1 nodes or elements");
  if (!mesh->x || !mesh->y || !mesh->z || (mesh->n_elems > 0 && !mesh->lnods))
    return fail(NSI_ERR_INVALID_ARG, "mesh array pointer is NULL");
  if (opts->precision < NSI_FP64 || opts->precision > NSI_MIXED_F32_ACC32)
    return fail(NSI_ERR_INVALID_ARG, "unknown precision");
  if (opts->scatter < NSI_SCATTER_AUTO || opts->scatter > NSI_SCATTER_GATHER)
    return fail(NSI_ERR_INVALID_ARG, "unknown scatter mode");
  if (opts->block < 0 || opts->block > 1024 || (opts->block % 32) != 0)
    return fail(NSI_ERR_INVALID_ARG, "block must be 0 or a multiple of 32 up to 1024");
  for (int r : opts->reserved)
    if (r != 0) return fail(NSI_ERR_INVALID_ARG, "reserved option fields must be 0");

  NsiHandle* h = new (std::nothrow) NsiHandle();
  if (!h) return fail(NSI_ERR_OOM, "host allocation failed");
  cudaGetDevice(&h->device);
  h->n = mesh->n_nodes;
  h->E = mesh->n_elems;
  h->precision = opts->precision;
  h->scatter = opts->scatter;
  h->block = opts->block ? opts->block : 256;
  h->debug = opts->debug_checks != 0;
  nsi_status st;
  try {
    st = build(h, mesh, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    st = fail(NSI_ERR_OOM, "host allocation failed while building the mesh maps");
  } catch (const std::exception& ex) {
    st = fail(NSI_ERR_CUDA, std::string("unexpected error: ") + ex.what());
  }
  if (st == NSI_OK && h->scatter == NSI_SCATTER_GATHER && !h->gather_ok) {
    st = fail(NSI_ERR_UNSUPPORTED, "row-gather mode needs rows of at most 32 entries");
  }
  // the default mode: row gather where the mesh allows it (rows <= 32 entries)
  if (st == NSI_OK && h->scatter == NSI_SCATTER_AUTO)
    h->scatter = h->gather_ok ? NSI_SCATTER_GATHER : NSI_SCATTER_ATOMIC;
  if (st != NSI_OK) {
    free_handle(h);
    return st;
  }
  *out = h;
  return NSI_OK;
}

nsi_status nsi_assemble_destroy(NsiHandle* h) {
  if (!h) return NSI_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_handle(h);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize in destroy");
  return NSI_OK;
}

nsi_status nsi_csr_pattern(const NsiHandle* h, const int32_t** row_ptr, const int32_t** col_idx, int64_t* nnz) {
  if (!h) return fail(NSI_ERR_INVALID_ARG, "handle is NULL");
  if (row_ptr) *row_ptr = h->row_ptr;
  if (col_idx) *col_idx = h->col_idx;
  if (nnz) *nnz = h->nnz;
  return NSI_OK;
}

nsi_status nsi_csr_pattern_copy(const NsiHandle* h, int32_t* row_ptr, int32_t* col_idx, void* stream) {
  if (!h) return fail(NSI_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (row_ptr) NSI_CUDA(cudaMemcpyAsync(row_ptr, h->row_ptr, sizeof(int32_t) * (h->n + 1), cudaMemcpyDefault, s));
  if (col_idx) NSI_CUDA(cudaMemcpyAsync(col_idx, h->col_idx, sizeof(int32_t) * h->nnz, cudaMemcpyDefault, s));
  NSI_CUDA(cudaStreamSynchronize(s));
  return NSI_OK;
}

nsi_status nsi_info(const NsiHandle* h, NsiInfo* info) {
  if (!h || !info) return fail(NSI_ERR_INVALID_ARG, "handle or info is NULL");
  info->n_nodes = h->n;
  info->n_elems = h->E;
  info->nnz = h->nnz;
  info->n_colors = h->n_colors;
  info->max_row = h->max_row;
  info->precision = h->precision;
  info->scatter = h->scatter;
  info->device_bytes = h->device_bytes;
  info->rows_per_block = h->use_fan ? -1 : h->plan.rows_per_block;
  info->n_plans = h->n_plans;
  info->persistent = h->persistent && !h->use_fan ? 1 : 0;
  info->exact_rows = (int32_t)std::min<int64_t>(h->exact_rows, INT32_MAX);
  info->long_rows = (int32_t)std::min<int64_t>(h->long_rows, INT32_MAX);
  info->fan_ok = h->fan_ok ? 1 : 0;
  return NSI_OK;
}

nsi_status nsi_set_launch(NsiHandle* h, int32_t scatter, int32_t rows_per_block) {
  if (!h) return fail(NSI_ERR_INVALID_ARG, "handle is NULL");
  if (scatter < NSI_SCATTER_AUTO || scatter > NSI_SCATTER_GATHER) return fail(NSI_ERR_INVALID_ARG, "unknown scatter mode");
  if (scatter == NSI_SCATTER_GATHER && !h->gather_ok) return fail(NSI_ERR_UNSUPPORTED, "row-gather mode not available for this mesh");
  if (scatter == NSI_SCATTER_ATOMIC) {
    // the atomic kernel: 1 warp-aggregated, 2 one atomic per value, 0 unchanged
    if (rows_per_block < 0 || rows_per_block > 2)
      return fail(NSI_ERR_INVALID_ARG, "for the atomic mode, rows_per_block is 0, 1 or 2");
    if (rows_per_block) h->atomic_agg = rows_per_block == 1;
  } else if (rows_per_block == -1) {
    if (!h->fan_ok) return fail(NSI_ERR_UNSUPPORTED, "no edge-fan map for this mesh");
    h->use_fan = true;
  } else if (rows_per_block != 0) {
    int k = 0;
    while (k < h->n_plans && h->plans[k].rows_per_block != rows_per_block) ++k;
    if (k == h->n_plans) return fail(NSI_ERR_UNSUPPORTED, "no launch plan with that many rows per block");
    h->plan = h->plans[k];
    h->use_fan = false;
  }
  if (scatter != NSI_SCATTER_AUTO) h->scatter = scatter;
  return NSI_OK;
}

nsi_status nsi_set_timing_events(NsiHandle* h, void* start, void* stop) {
  if (!h) return fail(NSI_ERR_INVALID_ARG, "handle is NULL");
  if ((start == nullptr) != (stop == nullptr)) return fail(NSI_ERR_INVALID_ARG, "give both events or neither");
  h->ev_start = static_cast<cudaEvent_t>(start);
  h->ev_stop = static_cast<cudaEvent_t>(stop);
  return NSI_OK;
}

nsi_status nsi_device_status(NsiHandle* h, void* stream) {
  if (!h) return fail(NSI_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned word = 0;
  NSI_CUDA(cudaMemcpyAsync(&word, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  NSI_CUDA(cudaStreamSynchronize(s));
  if (word) {
    NSI_CUDA(cudaMemsetAsync(h->err, 0, sizeof(unsigned), s));
    NSI_CUDA(cudaStreamSynchronize(s));
    char buf[96];
    snprintf(buf, sizeof buf, "device bounds check fired (error word 0x%x)", word);
    return fail(NSI_ERR_DEVICE_CHECK, buf);
  }
  return NSI_OK;
}

}  // extern "C"
