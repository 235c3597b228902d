// Host part of the hierarchical clustering (Sec. 3.3, Algorithm 3): the
// max-heap of candidate pairs and the union-find merge, then the cluster
// order.  Readings of the points the paper leaves open:
//  * the loop runs until the heap is empty;
//  * two popped roots are merged only if the merged cluster has at most
//    max_cluster rows; the smaller root id becomes the root;
//  * otherwise both rows are replaced by their roots; unless they are in one
//    cluster or the pair was ever a candidate, the Jaccard score of the two
//    root rows is computed and the pair pushed (and recorded) if above jacc_th;
//  * heap order: higher score first (exact, cross-multiplied), then smaller i,
//    then smaller j; pairs are stored once with i < j;
//  * clusters are ordered by their smallest row (the root), rows ascending.
#include <parallel/algorithm>

#include <algorithm>
#include <cstdint>
#include <queue>
#include <unordered_set>
#include <vector>

namespace sgc {

namespace {

struct HPair {
  int64_t c, u;
  int32_t i, j;
};

struct Lower {  // true if a has lower priority than b
  bool operator()(const HPair& a, const HPair& b) const {
    const int64_t l = a.c * b.u, r = b.c * a.u;
    if (l != r) return l < r;
    if (a.i != b.i) return a.i > b.i;
    return a.j > b.j;
  }
};

int32_t find_root(std::vector<int32_t>& parent, int32_t x) {
  int32_t r = x;
  while (parent[r] != r) r = parent[r];
  while (parent[x] != r) {  // path compression (does not change any root)
    const int32_t nx = parent[x];
    parent[x] = r;
    x = nx;
  }
  return r;
}

void overlap(const int64_t* rp, const int32_t* col, int32_t a, int32_t b, int64_t* inter, int64_t* uni) {
  int64_t p = rp[a], pe = rp[a + 1], q = rp[b], qe = rp[b + 1];
  int64_t c = 0;
  while (p < pe && q < qe) {
    if (col[p] < col[q]) ++p;
    else if (col[p] > col[q]) ++q;
    else { ++c; ++p; ++q; }
  }
  *inter = c;
  *uni = (rp[a + 1] - rp[a]) + (rp[b + 1] - rp[b]) - c;
}

inline uint64_t pkey(int32_t i, int32_t j) { return ((uint64_t)(uint32_t)i << 32) | (uint32_t)j; }

}  // namespace

// Unique candidate pairs (i < j) of the per-row lists, in the heap's priority
// order (score descending, then i, then j): u[e], v[e] for rank e; returns the count.
int64_t hc_rank_edges(int64_t n, const int32_t* cj, const int32_t* cc, const int32_t* cu, int topk, int32_t* u,
                      int32_t* v) {
  auto in_list = [&](int64_t row, int32_t x) {
    const int32_t* L = cj + row * topk;
    for (int s = 0; s < topk && L[s] >= 0; ++s)
      if (L[s] == x) return true;
    return false;
  };
  std::vector<int64_t> start((size_t)n + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int s = 0; s < topk; ++s) {
      const int32_t j = cj[i * topk + s];
      if (j < 0) break;
      c += (i < j || !in_list(j, (int32_t)i)) ? 1 : 0;
    }
    start[(size_t)i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) start[(size_t)i + 1] += start[(size_t)i];
  std::vector<HPair> pairs((size_t)start[(size_t)n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = start[(size_t)i];
    for (int s = 0; s < topk; ++s) {
      const int32_t j = cj[i * topk + s];
      if (j < 0) break;
      if (i < j || !in_list(j, (int32_t)i))
        pairs[(size_t)o++] = HPair{cc[i * topk + s], cu[i * topk + s], (int32_t)std::min<int64_t>(i, j),
                                   (int32_t)std::max<int64_t>(i, j)};
    }
  }
  const Lower lower;
  __gnu_parallel::sort(pairs.begin(), pairs.end(), [&](const HPair& x, const HPair& y) { return lower(y, x); });
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < (int64_t)pairs.size(); ++e) {
    u[e] = pairs[(size_t)e].i;
    v[e] = pairs[(size_t)e].j;
  }
  return (int64_t)pairs.size();
}

// Clusters from a root per row (root = smallest row of its cluster): ordered by
// root, rows ascending.  Returns ncl.
int64_t hc_order_by_root(int64_t n, const int32_t* root, int32_t* perm, int64_t* cluster_ptr) {
  std::vector<int64_t> cnt((size_t)n + 1, 0);
  for (int64_t r = 0; r < n; ++r) ++cnt[(size_t)root[r] + 1];
  for (int64_t r = 0; r < n; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t r = 0; r < n; ++r) perm[fill[(size_t)root[r]]++] = (int32_t)r;
  int64_t ncl = 0;
  cluster_ptr[0] = 0;
  for (int64_t r = 0; r < n; ++r)
    if (root[r] == r) cluster_ptr[++ncl] = cnt[(size_t)r + 1];
  return ncl;
}

// n rows; rp/col: host copy of A's pattern; cand arrays: n*topk (j = -1: none).
// Writes perm[n] and cluster_ptr[ncl+1]; returns ncl.
//
// The candidate pairs are popped in priority order from two sources: the
// original candidates, sorted once (in parallel), and a heap that holds only
// the pairs re-scored during the merge.  "Was (a, b) ever a candidate" is a
// scan of the two rows' candidate lists plus a set of the re-scored pairs.
int64_t hc_merge_host(int64_t n, const int64_t* rp, const int32_t* col, const int32_t* cj, const int32_t* cc,
                      const int32_t* cu, int topk, double th, int max_cluster, int32_t* perm, int64_t* cluster_ptr) {
  auto in_list = [&](int64_t row, int32_t x) {
    const int32_t* L = cj + row * topk;
    for (int s = 0; s < topk && L[s] >= 0; ++s)
      if (L[s] == x) return true;
    return false;
  };
  // unique candidate pairs (i < j): a pair in both rows' lists is taken from the smaller row
  std::vector<int64_t> start((size_t)n + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int s = 0; s < topk; ++s) {
      const int32_t j = cj[i * topk + s];
      if (j < 0) break;
      c += (i < j || !in_list(j, (int32_t)i)) ? 1 : 0;
    }
    start[(size_t)i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) start[(size_t)i + 1] += start[(size_t)i];
  std::vector<HPair> pairs((size_t)start[(size_t)n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = start[(size_t)i];
    for (int s = 0; s < topk; ++s) {
      const int32_t j = cj[i * topk + s];
      if (j < 0) break;
      if (i < j || !in_list(j, (int32_t)i))
        pairs[(size_t)o++] = HPair{cc[i * topk + s], cu[i * topk + s], (int32_t)std::min<int64_t>(i, j),
                                   (int32_t)std::max<int64_t>(i, j)};
    }
  }
  const Lower lower;
  // highest priority first
  __gnu_parallel::sort(pairs.begin(), pairs.end(), [&](const HPair& x, const HPair& y) { return lower(y, x); });
  std::unordered_set<uint64_t> added;
  auto is_cand = [&](int32_t a, int32_t b) {
    return in_list(a, b) || in_list(b, a) || added.count(pkey(a, b)) != 0;
  };
  std::priority_queue<HPair, std::vector<HPair>, Lower> heap;  // re-scored pairs only
  size_t next = 0;
  std::vector<int32_t> parent((size_t)n), size((size_t)n, 1);
  for (int64_t r = 0; r < n; ++r) parent[(size_t)r] = (int32_t)r;
  constexpr size_t AHEAD = 48;  // pairs whose union-find and candidate-list entries are fetched ahead
  while (next < pairs.size() || !heap.empty()) {
    if (next + AHEAD < pairs.size()) {
      const HPair& f = pairs[next + AHEAD];
      __builtin_prefetch(&parent[(size_t)f.i]);
      __builtin_prefetch(&parent[(size_t)f.j]);
      __builtin_prefetch(cj + (int64_t)f.i * topk);
      __builtin_prefetch(cj + (int64_t)f.j * topk);
    }
    HPair t;
    if (!heap.empty() && (next == pairs.size() || lower(pairs[next], heap.top()))) {
      t = heap.top();
      heap.pop();
    } else {
      t = pairs[next++];
    }
    if (parent[t.i] == t.i && parent[t.j] == t.j) {
      if (size[t.i] + size[t.j] <= max_cluster) {
        const int32_t lo = std::min(t.i, t.j), hi = std::max(t.i, t.j);
        parent[hi] = lo;
        size[lo] += size[hi];
      }
      continue;
    }
    const int32_t ri = find_root(parent, t.i), rj = find_root(parent, t.j);
    if (ri == rj) continue;
    const int32_t a = std::min(ri, rj), b = std::max(ri, rj);
    // roots whose clusters can never merge (sizes only grow): scoring them could only
    // push pairs that are popped without effect, so the clustering is the same
    if (size[a] + size[b] > max_cluster) continue;
    if (is_cand(a, b)) continue;
    int64_t inter, uni;
    overlap(rp, col, a, b, &inter, &uni);
    if ((double)inter > th * (double)uni) {
      added.insert(pkey(a, b));
      heap.push(HPair{inter, uni, a, b});
    }
  }
  // clusters by root (= smallest row), rows ascending
  std::vector<int64_t> cnt((size_t)n + 1, 0);
  std::vector<int32_t> root((size_t)n);
  for (int64_t r = 0; r < n; ++r) {
    root[(size_t)r] = find_root(parent, (int32_t)r);
    ++cnt[(size_t)root[(size_t)r] + 1];
  }
  for (int64_t r = 0; r < n; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t r = 0; r < n; ++r) perm[fill[(size_t)root[(size_t)r]]++] = (int32_t)r;
  int64_t ncl = 0;
  cluster_ptr[0] = 0;
  for (int64_t r = 0; r < n; ++r)
    if (root[(size_t)r] == r) cluster_ptr[++ncl] = cnt[(size_t)r + 1];
  return ncl;
}

}  // namespace sgc
