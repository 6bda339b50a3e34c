// Seeded synthetic graph generators (host C++, OpenMP).
//
// This module only makes inputs: it holds none of the BFS arithmetic, and it
// is the one piece of code that both the oracle-side tests and the GPU path's
// tests and benchmark use.  Every random draw comes from a counter-based
// generator (SplitMix64's finaliser applied to (seed, stream, index)), so the
// output depends only on the arguments, never on the thread count or the
// machine.  All graphs come out as symmetric CSR (every undirected edge stored
// in both directions), without self-loops or duplicate entries, with each
// adjacency row sorted ascending.
//
// Families (the shapes of the paper's evaluation suite, Section 3 / Table 1,
// which names a Kronecker graph and a uniform random graph):
//   * R-MAT (recursive matrix) edge lists with quadrant probabilities a,b,c,d,
//     vertex ids permuted by a seeded Fisher-Yates shuffle;
//   * Erdos-Renyi style uniform random pairs;
//   * 2-D 4-neighbour grids (large diameter);
//   * random geometric graphs in the unit square (large diameter);
//   * sets of many small uniform random graphs;
//   * BFS sources drawn uniformly among vertices of nonzero degree.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// SplitMix64 finaliser (Steele, Lea, Flood 2014; constants as published by Vigna).
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Draw number `idx` of stream `stream` under `seed`.
inline uint64_t rand64(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t key = mix64(seed ^ mix64(stream + kGolden));
  return mix64(key + (idx + 1) * kGolden);
}

// The same draws as rand64 with the per-(seed, stream) key computed once.
struct StreamGen {
  uint64_t key;
  StreamGen(uint64_t seed, uint64_t stream) : key(mix64(seed ^ mix64(stream + kGolden))) {}
  uint64_t operator()(uint64_t idx) const { return mix64(key + (idx + 1) * kGolden); }
};

// Uniform double in [0, 1) from the top 53 bits.
inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

// Uniform integer in [0, bound) by the multiply-high method.
inline uint64_t bounded(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)bound) >> 64);
}

// Streams (one per purpose, so that families never share draws).
enum : uint64_t {
  kStreamRmat = 0,
  kStreamPerm = 1,
  kStreamEr = 2,
  kStreamRgg = 3,
  kStreamSrc = 4,
  kStreamSetSize = 5,
  kStreamSetSeed = 6,
};

}  // namespace

struct gg_csr {
  int64_t n = 0;
  // Rows after sort+unique live in tmp[off[v] .. off[v] + deg[v]), or, when
  // `packed`, in the low 32 bits of arcs[off[v] .. off[v] + deg[v]).
  std::vector<int64_t> off;
  std::vector<int64_t> deg;
  std::vector<int32_t> tmp;
  std::vector<uint64_t> arcs;
  bool packed = false;
  int64_t m = 0;  // sum of deg
};

namespace {

int num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Exclusive prefix sum of a[0..n) into out[0..n], out[n] = total.
void exclusive_scan(const int64_t* a, int64_t n, int64_t* out) {
  int64_t acc = 0;
  for (int64_t i = 0; i < n; ++i) {
    out[i] = acc;
    acc += a[i];
  }
  out[n] = acc;
}

// Sort and de-duplicate every row of g (rows are independent).
void sort_unique_rows(gg_csr* g) {
  const int64_t n = g->n;
  g->deg.assign(n, 0);
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : total)
  for (int64_t v = 0; v < n; ++v) {
    int32_t* b = g->tmp.data() + g->off[v];
    int32_t* e = g->tmp.data() + g->off[v + 1];
    std::sort(b, e);
    int64_t d = std::unique(b, e) - b;
    g->deg[v] = d;
    total += d;
  }
  g->m = total;
}

// Parallel build: arcs (u,v) and (v,u) of every pair are radix-partitioned by
// the high bits of their first vertex into thread-private runs, then every
// bucket is sorted and de-duplicated on its own.  Same CSR as the serial path.
gg_csr* build_bucketed(int64_t n, int64_t npairs, const uint32_t* pu, const uint32_t* pv) {
  int bits = 0;
  while (((int64_t)1 << bits) < n) ++bits;
  const int bbits = bits > 12 ? 12 : bits;
  const int shift = bits - bbits;
  const int64_t nb = (int64_t)1 << bbits;
  const int T = num_threads();
  std::vector<int64_t> hist((size_t)T * (size_t)nb, 0);
  gg_csr* g = new gg_csr();
  g->n = n;
  g->packed = true;
#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num();
#else
    const int t = 0;
#endif
    const int64_t lo = npairs * t / T, hi = npairs * (t + 1) / T;
    int64_t* h = hist.data() + (size_t)t * (size_t)nb;
    for (int64_t k = lo; k < hi; ++k) {
      if (pu[k] == pv[k]) continue;
      h[pu[k] >> shift]++;
      h[pv[k] >> shift]++;
    }
  }
  std::vector<int64_t> bstart(nb + 1, 0);
  int64_t acc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    bstart[b] = acc;
    for (int t = 0; t < T; ++t) {
      int64_t c = hist[(size_t)t * (size_t)nb + b];
      hist[(size_t)t * (size_t)nb + b] = acc;
      acc += c;
    }
  }
  bstart[nb] = acc;
  g->arcs.resize((size_t)acc);
  uint64_t* arcs = g->arcs.data();
#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num();
#else
    const int t = 0;
#endif
    const int64_t lo = npairs * t / T, hi = npairs * (t + 1) / T;
    int64_t* h = hist.data() + (size_t)t * (size_t)nb;
    for (int64_t k = lo; k < hi; ++k) {
      const uint64_t a = pu[k], b = pv[k];
      if (a == b) continue;
      arcs[h[a >> shift]++] = (a << 32) | b;
      arcs[h[b >> shift]++] = (b << 32) | a;
    }
  }
  g->off.assign(n + 1, 0);
  g->deg.assign(n, 0);
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
  for (int64_t b = 0; b < nb; ++b) {
    uint64_t* s0 = arcs + bstart[b];
    uint64_t* e0 = arcs + bstart[b + 1];
    std::sort(s0, e0);
    uint64_t* e1 = std::unique(s0, e0);
    const int64_t base = bstart[b];
    for (uint64_t* p = s0; p < e1; ++p) {
      const int64_t u = (int64_t)(*p >> 32);
      if (g->deg[u] == 0) g->off[u] = base + (p - s0);
      g->deg[u]++;
    }
    total += e1 - s0;
  }
  g->m = total;
  return g;
}

// Build a symmetric CSR from a list of undirected pairs (u[k], v[k]); self
// loops are dropped, duplicates removed, rows sorted.
gg_csr* build_from_pairs(int64_t n, int64_t npairs, const uint32_t* pu, const uint32_t* pv,
                         bool serial) {
  if (!serial && npairs >= ((int64_t)1 << 20)) return build_bucketed(n, npairs, pu, pv);
  gg_csr* g = new gg_csr();
  g->n = n;
  std::vector<int64_t> cnt(n, 0);
  if (serial) {
    for (int64_t k = 0; k < npairs; ++k) {
      if (pu[k] == pv[k]) continue;
      cnt[pu[k]]++;
      cnt[pv[k]]++;
    }
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; ++k) {
      if (pu[k] == pv[k]) continue;
      __atomic_fetch_add(&cnt[pu[k]], 1, __ATOMIC_RELAXED);
      __atomic_fetch_add(&cnt[pv[k]], 1, __ATOMIC_RELAXED);
    }
  }
  g->off.assign(n + 1, 0);
  exclusive_scan(cnt.data(), n, g->off.data());
  g->tmp.assign((size_t)g->off[n], 0);
  std::vector<int64_t>& cur = cnt;  // reuse as cursor
  for (int64_t v = 0; v < n; ++v) cur[v] = g->off[v];
  if (serial) {
    for (int64_t k = 0; k < npairs; ++k) {
      uint32_t a = pu[k], b = pv[k];
      if (a == b) continue;
      g->tmp[cur[a]++] = (int32_t)b;
      g->tmp[cur[b]++] = (int32_t)a;
    }
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; ++k) {
      uint32_t a = pu[k], b = pv[k];
      if (a == b) continue;
      int64_t pa = __atomic_fetch_add(&cur[a], 1, __ATOMIC_RELAXED);
      int64_t pb = __atomic_fetch_add(&cur[b], 1, __ATOMIC_RELAXED);
      g->tmp[pa] = (int32_t)b;
      g->tmp[pb] = (int32_t)a;
    }
  }
  if (serial) {
    g->deg.assign(n, 0);
    int64_t total = 0;
    for (int64_t v = 0; v < n; ++v) {
      int32_t* b = g->tmp.data() + g->off[v];
      int32_t* e = g->tmp.data() + g->off[v + 1];
      std::sort(b, e);
      g->deg[v] = std::unique(b, e) - b;
      total += g->deg[v];
    }
    g->m = total;
  } else {
    sort_unique_rows(g);
  }
  return g;
}

std::vector<uint32_t> fisher_yates(int64_t n, uint64_t seed) {
  std::vector<uint32_t> p(n);
  for (int64_t i = 0; i < n; ++i) p[i] = (uint32_t)i;
  for (int64_t i = n - 1; i >= 1; --i) {
    uint64_t j = bounded(rand64(seed, kStreamPerm, (uint64_t)i), (uint64_t)i + 1);
    std::swap(p[i], p[j]);
  }
  return p;
}

gg_csr* er_impl(int64_t n, double avg_deg, uint64_t seed, bool serial) {
  int64_t npairs = (int64_t)std::llround((double)n * avg_deg / 2.0);
  std::vector<uint32_t> pu(npairs), pv(npairs);
  if (serial) {
    for (int64_t k = 0; k < npairs; ++k) {
      pu[k] = (uint32_t)bounded(rand64(seed, kStreamEr, 2 * (uint64_t)k), (uint64_t)n);
      pv[k] = (uint32_t)bounded(rand64(seed, kStreamEr, 2 * (uint64_t)k + 1), (uint64_t)n);
    }
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; ++k) {
      pu[k] = (uint32_t)bounded(rand64(seed, kStreamEr, 2 * (uint64_t)k), (uint64_t)n);
      pv[k] = (uint32_t)bounded(rand64(seed, kStreamEr, 2 * (uint64_t)k + 1), (uint64_t)n);
    }
  }
  return build_from_pairs(n, npairs, pu.data(), pv.data(), serial);
}

void copy_out(const gg_csr* g, int64_t* row_ptr, int32_t* col) {
  const int64_t n = g->n;
  std::vector<int64_t> rp(n + 1);
  exclusive_scan(g->deg.data(), n, rp.data());
  if (g->packed) {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
      const uint64_t* a = g->arcs.data() + g->off[v];
      int32_t* c = col + rp[v];
      for (int64_t i = 0; i < g->deg[v]; ++i) c[i] = (int32_t)(uint32_t)(a[i] & 0xffffffffull);
    }
  } else {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
      std::memcpy(col + rp[v], g->tmp.data() + g->off[v], sizeof(int32_t) * (size_t)g->deg[v]);
    }
  }
  std::memcpy(row_ptr, rp.data(), sizeof(int64_t) * (size_t)(n + 1));
}

}  // namespace

extern "C" {

uint64_t gg_rand64(uint64_t seed, uint64_t stream, uint64_t idx) { return rand64(seed, stream, idx); }

int gg_threads(void) { return num_threads(); }

// R-MAT with 2^scale vertices and edgefactor * 2^scale generated pairs.  For
// pair k, bit `lvl` (0 = most significant) of the row/column ids picks one of
// the four quadrants with one uniform draw u = U(seed, stream 0, k*scale+lvl):
// u < a -> (0,0); u < a+b -> (0,1); u < a+b+c -> (1,0); else (1,1).  Both ids
// are then mapped through a Fisher-Yates permutation drawn from perm_seed.
gg_csr* gg_rmat(int scale, int edgefactor, double a, double b, double c, uint64_t seed,
                uint64_t perm_seed) {
  if (scale < 1 || scale > 30 || edgefactor < 1) return nullptr;
  const int64_t n = (int64_t)1 << scale;
  const int64_t npairs = (int64_t)edgefactor * n;
  const double ab = a + b, abc = a + b + c;
  std::vector<uint32_t> perm = fisher_yates(n, perm_seed);
  std::vector<uint32_t> pu(npairs), pv(npairs);
  // u01(r) < t  <=>  (r >> 11) < ceil(t * 2^53): the same comparisons in integers.
  const double two53 = 9007199254740992.0;
  const uint64_t t1 = (uint64_t)std::ceil(a * two53), t2 = (uint64_t)std::ceil(ab * two53),
                 t3 = (uint64_t)std::ceil(abc * two53);
  const StreamGen rng(seed, kStreamRmat);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < npairs; ++k) {
    uint64_t row = 0, col = 0;
    const uint64_t base = (uint64_t)k * (uint64_t)scale;
    for (int lvl = 0; lvl < scale; ++lvl) {
      const uint64_t x = rng(base + (uint64_t)lvl) >> 11;
      const uint64_t rb = x >= t2, cb = (x >= t1) & ((x < t2) | (x >= t3));
      row = (row << 1) | rb;
      col = (col << 1) | cb;
    }
    pu[k] = perm[row];
    pv[k] = perm[col];
  }
  return build_from_pairs(n, npairs, pu.data(), pv.data(), false);
}

// Uniform random graph: round(n*avg_deg/2) pairs, each endpoint uniform in
// [0, n) from stream 2 (draws 2k and 2k+1 for pair k).
gg_csr* gg_er(int64_t n, double avg_deg, uint64_t seed) {
  if (n < 1 || n > ((int64_t)1 << 31) - 1 || avg_deg < 0) return nullptr;
  return er_impl(n, avg_deg, seed, false);
}

// rows x cols 4-neighbour grid without wrap-around; vertex (r, c) has id r*cols + c.
gg_csr* gg_grid(int64_t rows, int64_t cols) {
  if (rows < 1 || cols < 1 || rows * cols > ((int64_t)1 << 31) - 1) return nullptr;
  gg_csr* g = new gg_csr();
  const int64_t n = rows * cols;
  g->n = n;
  g->off.assign(n + 1, 0);
  g->deg.assign(n, 0);
  for (int64_t v = 0; v < n; ++v) {
    int64_t r = v / cols, c = v % cols;
    g->deg[v] = (r > 0) + (c > 0) + (c + 1 < cols) + (r + 1 < rows);
  }
  exclusive_scan(g->deg.data(), n, g->off.data());
  g->tmp.assign((size_t)g->off[n], 0);
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int64_t r = v / cols, c = v % cols, p = g->off[v];
    if (r > 0) g->tmp[p++] = (int32_t)(v - cols);
    if (c > 0) g->tmp[p++] = (int32_t)(v - 1);
    if (c + 1 < cols) g->tmp[p++] = (int32_t)(v + 1);
    if (r + 1 < rows) g->tmp[p++] = (int32_t)(v + cols);
  }
  g->m = g->off[n];
  return g;
}

// Random geometric graph: point i is (U(seed,3,2i), U(seed,3,2i+1)) in the
// unit square (no wrap-around); i and j are adjacent when their squared
// distance, computed in double precision, is <= radius^2.
gg_csr* gg_rgg(int64_t n, double radius, uint64_t seed) {
  if (n < 1 || n > ((int64_t)1 << 31) - 1 || !(radius > 0.0)) return nullptr;
  std::vector<double> x(n), y(n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    x[i] = u01(rand64(seed, kStreamRgg, 2 * (uint64_t)i));
    y[i] = u01(rand64(seed, kStreamRgg, 2 * (uint64_t)i + 1));
  }
  int64_t cells = (int64_t)std::floor(1.0 / radius);
  if (cells < 1) cells = 1;
  if (cells > 65536) cells = 65536;
  const int64_t nc = cells * cells;
  auto cell_of = [&](int64_t i) {
    int64_t cx = std::min<int64_t>((int64_t)(x[i] * (double)cells), cells - 1);
    int64_t cy = std::min<int64_t>((int64_t)(y[i] * (double)cells), cells - 1);
    return cy * cells + cx;
  };
  std::vector<int64_t> ccount(nc + 1, 0), cstart(nc + 1, 0);
  std::vector<int64_t> pcell(n);
  for (int64_t i = 0; i < n; ++i) {
    pcell[i] = cell_of(i);
    ccount[pcell[i]]++;
  }
  exclusive_scan(ccount.data(), nc, cstart.data());
  std::vector<int32_t> bucket(n);
  {
    std::vector<int64_t> cur(cstart.begin(), cstart.end() - 1);
    for (int64_t i = 0; i < n; ++i) bucket[cur[pcell[i]]++] = (int32_t)i;
  }
  const double r2 = radius * radius;
  gg_csr* g = new gg_csr();
  g->n = n;
  g->deg.assign(n, 0);
  auto visit = [&](int64_t i, auto&& fn) {
    int64_t cx = pcell[i] % cells, cy = pcell[i] / cells;
    for (int64_t dy = -1; dy <= 1; ++dy) {
      int64_t yy = cy + dy;
      if (yy < 0 || yy >= cells) continue;
      for (int64_t dx = -1; dx <= 1; ++dx) {
        int64_t xx = cx + dx;
        if (xx < 0 || xx >= cells) continue;
        int64_t cid = yy * cells + xx;
        for (int64_t t = cstart[cid]; t < cstart[cid + 1]; ++t) {
          int64_t j = bucket[t];
          if (j == i) continue;
          double ddx = x[i] - x[j], ddy = y[i] - y[j];
          if (ddx * ddx + ddy * ddy <= r2) fn(j);
        }
      }
    }
  };
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = 0;
    visit(i, [&](int64_t) { ++d; });
    g->deg[i] = d;
  }
  g->off.assign(n + 1, 0);
  exclusive_scan(g->deg.data(), n, g->off.data());
  g->tmp.assign((size_t)g->off[n], 0);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = g->off[i];
    visit(i, [&](int64_t j) { g->tmp[p++] = (int32_t)j; });
    std::sort(g->tmp.data() + g->off[i], g->tmp.data() + g->off[i + 1]);
  }
  g->m = g->off[n];
  return g;
}

int64_t gg_n(const gg_csr* g) { return g ? g->n : -1; }
int64_t gg_m(const gg_csr* g) { return g ? g->m : -1; }

// Write the CSR into caller buffers: row_ptr[n+1] (int64), col[m] (int32).
void gg_copy(const gg_csr* g, int64_t* row_ptr, int32_t* col) { copy_out(g, row_ptr, col); }

void gg_free(gg_csr* g) { delete g; }

// k BFS sources, uniform among vertices of nonzero degree: draw t of stream 4
// proposes bounded(r, n) and is rejected while that vertex has degree 0.
// Returns k, or -1 when the graph has no edge.
int64_t gg_sources(const int64_t* row_ptr, int64_t n, uint64_t seed, int64_t k, int32_t* out) {
  bool any = false;
  for (int64_t v = 0; v < n && !any; ++v) any = row_ptr[v + 1] > row_ptr[v];
  if (!any) return -1;
  uint64_t t = 0;
  for (int64_t i = 0; i < k; ++i) {
    for (;;) {
      uint64_t v = bounded(rand64(seed, kStreamSrc, t++), (uint64_t)n);
      if (row_ptr[v + 1] > row_ptr[v]) {
        out[i] = (int32_t)v;
        break;
      }
    }
  }
  return k;
}

// U[0,1) draws start..start+count-1 of (seed, stream), for host-side helpers
// such as Poisson arrival times.
void gg_uniform(uint64_t seed, uint64_t stream, uint64_t start, int64_t count, double* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = u01(rand64(seed, stream, start + (uint64_t)i));
}

// A set of `count` uniform random graphs.  Graph i has
// n_i = floor(exp(ln(nmin) + U(seed,5,i) * (ln(nmax) - ln(nmin)))) vertices
// (log-uniform), average degree avg_deg, its own seed rand64(seed, 6, i), and
// one source drawn by gg_sources(seed_i).  Output sizes are queried with
// sizes_only=1 (fills nv_out[0] = total vertices, ne_out[0] = total entries);
// the second call fills:
//   voff[count+1]  first vertex of each graph in the concatenated order,
//   eoff[count+1]  first col entry of each graph,
//   row_ptr[total_vertices + count]  per-graph local row pointers (graph i's
//                  n_i+1 entries start at voff[i] + i), int64,
//   col[total_entries]  local (0-based) neighbour ids,
//   src[count]     local source id per graph.
int gg_graphset(int64_t count, int64_t nmin, int64_t nmax, double avg_deg, uint64_t seed,
                int sizes_only, int64_t* nv_out, int64_t* ne_out, int64_t* voff, int64_t* eoff,
                int64_t* row_ptr, int32_t* col, int32_t* src) {
  if (count < 1 || nmin < 1 || nmax < nmin) return -1;
  std::vector<gg_csr*> gs(count, nullptr);
  const double lo = std::log((double)nmin), hi = std::log((double)nmax);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < count; ++i) {
    double u = u01(rand64(seed, kStreamSetSize, (uint64_t)i));
    int64_t ni = (int64_t)std::floor(std::exp(lo + u * (hi - lo)));
    if (ni < nmin) ni = nmin;
    if (ni > nmax) ni = nmax;
    gs[i] = er_impl(ni, avg_deg, rand64(seed, kStreamSetSeed, (uint64_t)i), true);
  }
  int64_t tv = 0, te = 0;
  for (int64_t i = 0; i < count; ++i) {
    tv += gs[i]->n;
    te += gs[i]->m;
  }
  nv_out[0] = tv;
  ne_out[0] = te;
  int rc = 0;
  if (!sizes_only) {
    voff[0] = 0;
    eoff[0] = 0;
    for (int64_t i = 0; i < count; ++i) {
      voff[i + 1] = voff[i] + gs[i]->n;
      eoff[i + 1] = eoff[i] + gs[i]->m;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < count; ++i) {
      gg_csr* g = gs[i];
      int64_t* rp = row_ptr + voff[i] + i;
      int32_t* cl = col + eoff[i];
      int64_t acc = 0;
      for (int64_t v = 0; v < g->n; ++v) {
        rp[v] = acc;
        std::memcpy(cl + acc, g->tmp.data() + g->off[v], sizeof(int32_t) * (size_t)g->deg[v]);
        acc += g->deg[v];
      }
      rp[g->n] = acc;
      int32_t s = 0;
      if (gg_sources(rp, g->n, rand64(seed, kStreamSetSeed, (uint64_t)i), 1, &s) < 0) s = 0;
      src[i] = s;
    }
  }
  for (int64_t i = 0; i < count; ++i) delete gs[i];
  return rc;
}

}  // extern "C"
