/*
 * CPU oracle for cover-edge triangle counting (CETC).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the GPU library
 * never does, and the two share no code, header or table.
 *
 * Paper: D. A. Bader et al., "Cover Edge-Based Novel Triangle Counting"
 * (arXiv 2403.02997).  Each function names the section / algorithm it follows.
 *
 * Conventions
 *   - vertices are uint32 ids 0..n-1; the graph is undirected and simple
 *     (Section "Notations and Definitions"): a self-loop (u, u) is dropped and
 *     repeated pairs collapse to one edge;
 *   - CSR: row_ptr[n+1] (int64), col[row_ptr[n]] (uint32), every row sorted
 *     ascending without repeats, each undirected edge stored in both rows;
 *   - level[v] is an int32 BFS distance, -1 while unvisited.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Graph construction (Section "Notations and Definitions": N(v) is the set of
 * neighbours; the input is read as an undirected simple graph).
 *
 * For every input pair (u, v) with u != v, v joins N(u) and u joins N(v).  Each
 * row is then sorted (qsort) and repeats are removed.  `col` must hold 2*E
 * entries (the bound before de-duplication).  Returns the number of stored
 * entries 2m, or -1 if some id is >= n (nothing is written in that case).
 */
int64_t orc_build_csr(uint32_t n, uint64_t E, const uint32_t* src, const uint32_t* dst,
                      int64_t* row_ptr, uint32_t* col) {
  for (uint64_t i = 0; i < E; ++i)
    if (src[i] >= n || dst[i] >= n) return -1;
  int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (uint32_t v = 0; v <= n; ++v) row_ptr[v] = 0;
  for (uint64_t i = 0; i < E; ++i) {
    if (src[i] == dst[i]) continue;
    row_ptr[src[i] + 1]++;
    row_ptr[dst[i] + 1]++;
  }
  for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
  for (uint32_t v = 0; v < n; ++v) fill[v] = row_ptr[v];
  for (uint64_t i = 0; i < E; ++i) {
    uint32_t u = src[i], v = dst[i];
    if (u == v) continue;
    col[fill[u]++] = v;
    col[fill[v]++] = u;
  }
  /* sort each row, drop repeats, and pack the rows to the front */
  int64_t out = 0;
  for (uint32_t v = 0; v < n; ++v) {
    int64_t b = row_ptr[v], e = row_ptr[v + 1];
    if (e > b) qsort(col + b, (size_t)(e - b), sizeof(uint32_t), cmp_u32);
    int64_t start = out;
    for (int64_t j = b; j < e; ++j)
      if (j == b || col[j] != col[j - 1]) col[out++] = col[j];
    row_ptr[v] = start;
  }
  row_ptr[n] = out;
  free(fill);
  return out;
}

/*
 * BFS levels (Definition "BFS-Edge": L(v) is the shortest distance from the
 * root) with the restart rule of Algorithm CETC-Seq ("for all v: if v is
 * unvisited, BFS(G, v)").
 *
 * A FIFO-queue BFS from `root` runs first; afterwards the vertices are scanned in
 * ascending id order and a new BFS (levels restarting at 0) starts from every
 * vertex still unvisited.  Every vertex therefore ends with level >= 0 and an
 * isolated vertex gets level 0.  `root` >= n skips the first search (plain
 * Algorithm CETC-Seq order).
 */
void orc_bfs_levels(uint32_t n, const int64_t* row_ptr, const uint32_t* col, uint32_t root,
                    int32_t* level) {
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  for (uint32_t v = 0; v < n; ++v) level[v] = -1;
  for (uint64_t s = 0; s <= (uint64_t)n; ++s) {
    uint32_t start;
    if (s == 0) {
      if (root >= n) continue;
      start = root;
    } else {
      start = (uint32_t)(s - 1);
    }
    if (level[start] != -1) continue;
    uint64_t head = 0, tail = 0;
    level[start] = 0;
    queue[tail++] = start;
    while (head < tail) {
      uint32_t x = queue[head++];
      for (int64_t j = row_ptr[x]; j < row_ptr[x + 1]; ++j) {
        uint32_t y = col[j];
        if (level[y] == -1) {
          level[y] = level[x] + 1;
          queue[tail++] = y;
        }
      }
    }
  }
  free(queue);
}

/*
 * Statistics filled by orc_cetc.  Index meaning:
 *   [0] T      triangle count (Algorithm CETC-Seq rule)
 *   [1] c1     apexes on another level        (Algorithm CETC-SM)
 *   [2] c2     apexes on the same level       (Algorithm CETC-SM)
 *   [3] |S|    number of horizontal (cover) edges u < v
 *   [4] sum over S of d(u) + d(v)
 *   [5] sum over S of min(d(u), d(v))
 *   [6] number of common neighbours found (c1 + c2)
 *   [7] number of cover edges actually intersected (|S| / stride, rounded up)
 */
enum { ST_T, ST_C1, ST_C2, ST_S, ST_SUMDEG, ST_SUMMIN, ST_MATCH, ST_DONE, ST_N };

/*
 * Two-pointer intersection of N(u) and N(v) (the merge of Algorithm EMP),
 * applying the counting rule of Algorithm CETC-Seq to every common neighbour w:
 * count it when L(u) != L(w), or when L(u) == L(w) and v < w.  Returns the
 * per-edge count; adds the CETC-SM split (c1, c2) and the match total to st.
 */
static uint64_t cover_edge(const int64_t* row_ptr, const uint32_t* col, const int32_t* level,
                           uint32_t u, uint32_t v, uint64_t* c1, uint64_t* c2) {
  int64_t x = row_ptr[u], xe = row_ptr[u + 1];
  int64_t y = row_ptr[v], ye = row_ptr[v + 1];
  uint64_t t = 0;
  while (x < xe && y < ye) {
    uint32_t a = col[x], b = col[y];
    if (a == b) {
      uint32_t w = a;
      if (level[w] != level[u]) {
        ++t;
        ++*c1;
      } else {
        ++*c2;
        if (v < w) ++t;
      }
      ++x;
      ++y;
    } else if (a < b) {
      ++x;
    } else {
      ++y;
    }
  }
  return t;
}

/*
 * Algorithm CETC-Seq, its edge loop taken literally: for every stored edge (u, v)
 * with L(u) == L(v) and u < v (a horizontal edge, taken once), intersect
 * N(u) and N(v) and count each common neighbour under the rule above.  The
 * c1 / c2 split of Algorithm CETC-SM is accumulated beside it; the caller checks
 * T == c1 + c2 / 3.
 *
 * `stride` > 1 intersects only every stride-th cover edge (in loop order) so a
 * bounded sample can be timed; stride == 1 is the full algorithm.  When
 * cover_u / cover_v are non-NULL they receive S in loop order, which is
 * lexicographic (u, v) order.
 */
void orc_cetc(uint32_t n, const int64_t* row_ptr, const uint32_t* col, const int32_t* level,
              uint64_t stride, uint64_t* st, uint32_t* cover_u, uint32_t* cover_v) {
  for (int k = 0; k < ST_N; ++k) st[k] = 0;
  if (stride == 0) stride = 1;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      uint32_t v = col[j];
      if (!(level[u] == level[v] && u < v)) continue;
      uint64_t idx = st[ST_S]++;
      if (cover_u) cover_u[idx] = u;
      if (cover_v) cover_v[idx] = v;
      uint64_t du = (uint64_t)(row_ptr[u + 1] - row_ptr[u]);
      uint64_t dv = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
      st[ST_SUMDEG] += du + dv;
      st[ST_SUMMIN] += du < dv ? du : dv;
      if (idx % stride != 0) continue;
      uint64_t c1 = 0, c2 = 0;
      st[ST_T] += cover_edge(row_ptr, col, level, u, v, &c1, &c2);
      st[ST_C1] += c1;
      st[ST_C2] += c2;
      st[ST_MATCH] += c1 + c2;
      st[ST_DONE]++;
    }
  }
}

/*
 * Algorithm CETC-SM (shared-memory parallel form): the same loop over
 * horizontal edges, run in parallel over u with OpenMP, accumulating only
 * c1 (apex on another level) and c2 (apex on the same level); returns
 * T = c1 + c2 / 3.  Sampling by `stride` as in orc_cetc, counted per row
 * (every stride-th cover edge of each row, starting with the first).
 * out[0] = c1, out[1] = c2, out[2] = cover edges intersected.
 */
uint64_t orc_cetc_sm(uint32_t n, const int64_t* row_ptr, const uint32_t* col,
                     const int32_t* level, uint64_t stride, uint64_t* out) {
  uint64_t c1 = 0, c2 = 0, done = 0;
  if (stride == 0) stride = 1;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : c1, c2, done)
  for (int64_t uu = 0; uu < (int64_t)n; ++uu) {
    uint32_t u = (uint32_t)uu;
    uint64_t k = 0;
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      uint32_t v = col[j];
      if (!(level[u] == level[v] && u < v)) continue;
      if ((k++) % stride != 0) continue;
      cover_edge(row_ptr, col, level, u, v, &c1, &c2);
      ++done;
    }
  }
  out[0] = c1;
  out[1] = c2;
  out[2] = done;
  return c1 + c2 / 3;
}

/* Number of host threads orc_cetc_sm uses. */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Algorithm CETC-Seq's count restricted to a given list of k horizontal edges
 * (us[i] < vs[i]): the sum of their per-edge counts, with the CETC-SM split.
 * out[0] = T, out[1] = c1, out[2] = c2.  Used to time a sample of the edge
 * loop; over all of S it equals orc_cetc.
 */
void orc_cetc_edges(const int64_t* row_ptr, const uint32_t* col, const int32_t* level,
                    uint64_t k, const uint32_t* us, const uint32_t* vs, uint64_t* out) {
  uint64_t t = 0, c1 = 0, c2 = 0;
  for (uint64_t i = 0; i < k; ++i) t += cover_edge(row_ptr, col, level, us[i], vs[i], &c1, &c2);
  out[0] = t;
  out[1] = c1;
  out[2] = c2;
}

/*
 * orc_cetc_edges run as Algorithm CETC-SM runs its cover-edge loop: the k
 * given horizontal edges split over the host's OpenMP threads (dynamic
 * schedule), per-edge counts summed.  Same outputs as orc_cetc_edges; used to
 * time a sample of the parallel edge loop on all host cores.
 */
void orc_cetc_sm_edges(const int64_t* row_ptr, const uint32_t* col, const int32_t* level,
                       uint64_t k, const uint32_t* us, const uint32_t* vs, uint64_t* out) {
  uint64_t t = 0, c1 = 0, c2 = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : t, c1, c2)
  for (int64_t i = 0; i < (int64_t)k; ++i) {
    uint64_t a = 0, b = 0;
    t += cover_edge(row_ptr, col, level, us[i], vs[i], &a, &b);
    c1 += a;
    c2 += b;
  }
  out[0] = t;
  out[1] = c1;
  out[2] = c2;
}

/*
 * The per-edge count of Algorithm CETC-Seq for one horizontal edge (u, v),
 * u < v: the number of w in N(u) ∩ N(v) with L(u) != L(w), or L(u) == L(w)
 * and v < w.
 */
uint64_t orc_edge_count(const int64_t* row_ptr, const uint32_t* col, const int32_t* level,
                        uint32_t u, uint32_t v) {
  uint64_t c1 = 0, c2 = 0;
  return cover_edge(row_ptr, col, level, u, v, &c1, &c2);
}

/*
 * Algorithm Triples (brute force): over all ordered triples (u, v, w) of
 * vertices, count those whose three pairs are all edges, and divide by 6.
 * `adj` is the n x n 0/1 adjacency matrix (row-major, zero diagonal).
 */
uint64_t orc_triples(uint32_t n, const uint8_t* adj) {
  uint64_t t = 0;
  for (uint32_t u = 0; u < n; ++u)
    for (uint32_t v = 0; v < n; ++v)
      for (uint32_t w = 0; w < n; ++w)
        if (adj[(uint64_t)u * n + v] && adj[(uint64_t)v * n + w] && adj[(uint64_t)u * n + w])
          ++t;
  return t / 6;
}

/*
 * Algorithm Forward (Schank and Wagner), after relabelling the vertices in
 * decreasing order of degree (ties: smaller id first), as the paper's
 * "reorder by decreasing degree" pre-processing describes.
 *
 * In the new ids, edges {u, v} with u < v are taken in increasing u (then v);
 * for each, |A(u) ∩ A(v)| is added to T and u is appended to A(v).  Appends
 * arrive in increasing u, so every A() stays sorted and a merge intersects
 * them.  Shares nothing with the cover-edge method: no BFS, no levels.
 */
uint64_t orc_forward(uint32_t n, const int64_t* row_ptr, const uint32_t* col) {
  if (n == 0) return 0;
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * n);  /* new id -> old id */
  uint32_t* rank = (uint32_t*)malloc(sizeof(uint32_t) * n);   /* old id -> new id */
  int64_t maxd = 0;
  for (uint32_t v = 0; v < n; ++v) {
    int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (d > maxd) maxd = d;
  }
  /* counting sort by decreasing degree, stable in id */
  int64_t* cnt = (int64_t*)calloc((size_t)maxd + 2, sizeof(int64_t));
  for (uint32_t v = 0; v < n; ++v) cnt[maxd - (row_ptr[v + 1] - row_ptr[v]) + 1]++;
  for (int64_t d = 0; d <= maxd; ++d) cnt[d + 1] += cnt[d];
  for (uint32_t v = 0; v < n; ++v) {
    int64_t key = maxd - (row_ptr[v + 1] - row_ptr[v]);
    order[cnt[key]++] = v;
  }
  for (uint32_t i = 0; i < n; ++i) rank[order[i]] = i;
  free(cnt);

  /* relabelled adjacency, rows sorted */
  int64_t nnz = row_ptr[n];
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  uint32_t* cl = (uint32_t*)malloc(sizeof(uint32_t) * (nnz ? (size_t)nnz : 1));
  rp[0] = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t v = order[i];
    int64_t d = row_ptr[v + 1] - row_ptr[v];
    for (int64_t j = 0; j < d; ++j) cl[rp[i] + j] = rank[col[row_ptr[v] + j]];
    if (d) qsort(cl + rp[i], (size_t)d, sizeof(uint32_t), cmp_u32);
    rp[i + 1] = rp[i] + d;
  }
  /* A(v) storage: at most the number of neighbours of v with a smaller new id */
  int64_t* abase = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int64_t* alen = (int64_t*)calloc(n, sizeof(int64_t));
  abase[0] = 0;
  for (uint32_t i = 0; i < n; ++i) {
    int64_t lower = 0;
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
      if (cl[j] < i) ++lower;
    abase[i + 1] = abase[i] + lower;
  }
  uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * (abase[n] ? (size_t)abase[n] : 1));
  uint64_t T = 0;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t j = rp[u]; j < rp[u + 1]; ++j) {
      uint32_t v = cl[j];
      if (!(u < v)) continue;
      const uint32_t* a = A + abase[u];
      const uint32_t* b = A + abase[v];
      int64_t x = 0, y = 0, xe = alen[u], ye = alen[v];
      while (x < xe && y < ye) {
        if (a[x] == b[y]) {
          ++T;
          ++x;
          ++y;
        } else if (a[x] < b[y]) {
          ++x;
        } else {
          ++y;
        }
      }
      A[abase[v] + alen[v]++] = u;
    }
  }
  free(order);
  free(rank);
  free(rp);
  free(cl);
  free(abase);
  free(alen);
  free(A);
  return T;
}

/*
 * Algorithm CETC-Seq-S (Section "CETC Split Triangle Counting"), given the
 * levels.  The edges split into E0, the horizontal edges (L(u) == L(v)), and
 * E1, the edges between levels; G0 = (V, E0) and G1 = (V, E1).
 *
 *   T0 = the triangles of G0, by Algorithm forward-hashed (Section "Related
 *        Work"): edges {u, v} of G0 with u < v are taken in increasing u, then
 *        v; the vertices of A(u) are marked in a boolean hash array, the
 *        marked vertices of A(v) are counted, the marks are cleared, and u
 *        joins A(v).
 *   T1 = for every u: mark N_G1(u); for every v in N_G0(u) with u < v, count
 *        the marked w in N_G1(v); clear the marks.
 *
 * out[0] = T0 (triangles with three horizontal edges), out[1] = T1
 * (triangles whose apex is on another level than their horizontal edge).
 * Returns T0 + T1.
 */
uint64_t orc_cetc_split(uint32_t n, const int64_t* row_ptr, const uint32_t* col,
                        const int32_t* level, uint64_t* out) {
  uint64_t t0 = 0, t1 = 0;
  if (n == 0) {
    out[0] = out[1] = 0;
    return 0;
  }
  uint8_t* hash = (uint8_t*)calloc(n, 1);
  /* A(v): room for every lower G0 neighbour of v */
  int64_t* abase = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int64_t* alen = (int64_t*)calloc(n, sizeof(int64_t));
  abase[0] = 0;
  for (uint32_t v = 0; v < n; ++v) {
    int64_t lower = 0;
    for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j)
      if (col[j] < v && level[col[j]] == level[v]) ++lower;
    abase[v + 1] = abase[v] + lower;
  }
  uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * (abase[n] ? (size_t)abase[n] : 1));
  /* T0: forward-hashed on G0 */
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      const uint32_t v = col[j];
      if (!(u < v && level[u] == level[v])) continue;
      for (int64_t k = 0; k < alen[u]; ++k) hash[A[abase[u] + k]] = 1;
      for (int64_t k = 0; k < alen[v]; ++k) t0 += hash[A[abase[v] + k]];
      for (int64_t k = 0; k < alen[u]; ++k) hash[A[abase[u] + k]] = 0;
      A[abase[v] + alen[v]++] = u;
    }
  }
  /* T1: hashed intersections of G1 rows over the edges of G0 */
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j)
      if (level[col[j]] != level[u]) hash[col[j]] = 1;
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      const uint32_t v = col[j];
      if (!(u < v && level[u] == level[v])) continue;
      for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        const uint32_t w = col[k];
        if (level[w] != level[v] && hash[w]) ++t1;
      }
    }
    for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) hash[col[j]] = 0;
  }
  free(hash);
  free(abase);
  free(alen);
  free(A);
  out[0] = t0;
  out[1] = t1;
  return t0 + t1;
}

/*
 * Triangle listing (Section "Introduction": listing and per-vertex counts feed
 * k-truss and clustering coefficients).  Every triangle {a, b, c}, a < b < c,
 * exactly once: for each a, each b in N(a) above a, each c in N(a) ∩ N(b)
 * above b (two-pointer merge).  Writes up to `cap` triples (a, b, c) to `out`
 * in increasing (a, b, c) order and adds, for every triangle, 1 to vcount[a],
 * vcount[b] and vcount[c] (vcount may be NULL).  Returns the number of
 * triangles.
 */
uint64_t orc_list_triangles(uint32_t n, const int64_t* row_ptr, const uint32_t* col,
                            uint32_t* out, uint64_t cap, uint64_t* vcount) {
  uint64_t t = 0;
  for (uint32_t a = 0; a < n; ++a) {
    for (int64_t j = row_ptr[a]; j < row_ptr[a + 1]; ++j) {
      const uint32_t b = col[j];
      if (b <= a) continue;
      int64_t x = row_ptr[a], y = row_ptr[b];
      while (x < row_ptr[a + 1] && y < row_ptr[b + 1]) {
        if (col[x] < col[y]) {
          ++x;
        } else if (col[x] > col[y]) {
          ++y;
        } else {
          const uint32_t c = col[x];
          if (c > b) {
            if (out && t < cap) {
              out[3 * t] = a;
              out[3 * t + 1] = b;
              out[3 * t + 2] = c;
            }
            if (vcount) {
              ++vcount[a];
              ++vcount[b];
              ++vcount[c];
            }
            ++t;
          }
          ++x;
          ++y;
        }
      }
    }
  }
  return t;
}
