/*
 * Seeded, counter-based synthetic graph generators.
 *
 * These produce the undirected edge lists (as uint32 (src, dst) pairs, with
 * self-loops and duplicates left in, exactly as drawn) that feed both the CUDA
 * counting path and the CPU oracle.  Nothing here knows about BFS levels,
 * cover edges or triangle counting: it is input generation only.
 *
 * Every random number is a pure function of (seed, stream, index):
 *
 *     h(seed, stream, i) = sm64( sm64( sm64(seed) + stream ) + i )
 *
 * where sm64 is the SplitMix64 output function (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014).  Because the
 * draws depend only on their counter, the generators give the same bytes on
 * any machine, for any thread count.
 *
 * Streams: 1 = Erdos-Renyi draws, 2 = R-MAT quadrant draws, 3 = R-MAT vertex
 * permutation, 4 = mesh diagonals.
 *
 * Workload shapes follow the paper's experimental section: Graph500 R-MAT
 * graphs with (a, b, c, d) = (0.57, 0.19, 0.19, 0.05) and edge factor 16, and
 * low-degree, long-diameter road-like graphs (here a 2D mesh with random
 * anti-diagonals).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

uint64_t gg_hash(uint64_t seed, uint64_t stream, uint64_t i) {
  return sm64(sm64(sm64(seed) + stream) + i);
}

/* Uniform integer in [0, n) from 32 random bits (multiply-shift). */
static inline uint32_t below(uint32_t r32, uint32_t n) {
  return (uint32_t)(((uint64_t)r32 * (uint64_t)n) >> 32);
}

/*
 * Erdos-Renyi G(n, m) draws: m ordered pairs (u, v), each coordinate uniform on
 * [0, n), i.i.d. from stream 1.  Self-loops and repeats are kept: removing them
 * is the job of graph construction.
 */
void gg_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)m; ++i) {
    uint64_t h = gg_hash(seed, 1, (uint64_t)i);
    src[i] = below((uint32_t)h, n);
    dst[i] = below((uint32_t)(h >> 32), n);
  }
}

/*
 * Uniform random permutation of [0, n) by Fisher-Yates, driven by stream 3.
 */
void gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  for (uint32_t i = n; i > 1; --i) {
    uint32_t k = i - 1;
    uint32_t j = below((uint32_t)(gg_hash(seed, 3, k) >> 32), i);
    uint32_t t = perm[k];
    perm[k] = perm[j];
    perm[j] = t;
  }
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004) without noise: each of the m draws
 * descends `scale` levels of the adjacency matrix; at each level one 32-bit
 * uniform r picks quadrant (0,0) if r < t_a, (0,1) if r < t_ab, (1,0) if
 * r < t_abc, else (1,1).  The thresholds are the cumulative probabilities
 * scaled by 2^32 (so a = 0.57, b = 0.19, c = 0.19 give 2448131359,
 * 3264175145, 4080218931).  Level k (k = 0 first) sets bit (scale-1-k).
 * Draw i uses 32-bit halves of h(seed, 2, i*ceil(scale/2) + k/2).
 * If `permute` is set, vertex ids are relabelled by gg_permutation(seed).
 */
void gg_rmat(uint32_t scale, uint64_t m, uint64_t seed, uint32_t t_a, uint32_t t_ab,
             uint32_t t_abc, int permute, uint32_t* src, uint32_t* dst) {
  const uint64_t words = (scale + 1) / 2;
  uint32_t* perm = NULL;
  if (permute) {
    perm = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)1 << scale));
    gg_permutation((uint32_t)1 << scale, seed, perm);
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)m; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t h = 0;
    for (uint32_t k = 0; k < scale; ++k) {
      if ((k & 1) == 0) h = gg_hash(seed, 2, (uint64_t)i * words + k / 2);
      uint32_t r = (k & 1) ? (uint32_t)(h >> 32) : (uint32_t)h;
      uint32_t bit = 1u << (scale - 1 - k);
      if (r < t_a) {
      } else if (r < t_ab) {
        v |= bit;
      } else if (r < t_abc) {
        u |= bit;
      } else {
        u |= bit;
        v |= bit;
      }
    }
    if (perm) {
      u = perm[u];
      v = perm[v];
    }
    src[i] = u;
    dst[i] = v;
  }
  free(perm);
}

/*
 * Anti-diagonal flags of a rows x cols mesh: cell (i, j), 0 <= i < rows-1,
 * 0 <= j < cols-1, holds the diagonal {(i+1, j), (i, j+1)} when the low 32 bits
 * of h(seed, 4, i*(cols-1) + j) are below `thresh` (thresh = p * 2^32; a value
 * of 2^32 or more keeps every diagonal).  Returns the number of diagonals.
 */
uint64_t gg_mesh_diagonals(uint32_t rows, uint32_t cols, uint64_t thresh, uint64_t seed,
                           uint8_t* flags) {
  if (rows < 2 || cols < 2) return 0;
  const uint64_t cells = (uint64_t)(rows - 1) * (cols - 1);
  uint64_t d = 0;
#pragma omp parallel for schedule(static) reduction(+ : d)
  for (int64_t c = 0; c < (int64_t)cells; ++c) {
    uint64_t r = gg_hash(seed, 4, (uint64_t)c) & 0xffffffffull;
    flags[c] = (uint8_t)(r < thresh);
    d += flags[c];
  }
  return d;
}

/*
 * Mesh edge list: vertex (i, j) has id i*cols + j.  Emits, in this order, all
 * horizontal edges {(i,j),(i,j+1)} row-major, all vertical edges
 * {(i,j),(i+1,j)} row-major, then the present anti-diagonals
 * {(i+1,j),(i,j+1)} in cell order.  `flags` is the output of
 * gg_mesh_diagonals.  Returns the number of edges written.
 */
uint64_t gg_mesh_edges(uint32_t rows, uint32_t cols, const uint8_t* flags, uint32_t* src,
                       uint32_t* dst) {
  uint64_t e = 0;
  const uint64_t h = (uint64_t)rows * (cols > 0 ? cols - 1 : 0);
  const uint64_t vv = (uint64_t)(rows > 0 ? rows - 1 : 0) * cols;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)h; ++k) {
    uint64_t i = (uint64_t)k / (cols - 1), j = (uint64_t)k % (cols - 1);
    src[k] = (uint32_t)(i * cols + j);
    dst[k] = (uint32_t)(i * cols + j + 1);
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < (int64_t)vv; ++k) {
    uint64_t i = (uint64_t)k / cols, j = (uint64_t)k % cols;
    src[h + k] = (uint32_t)(i * cols + j);
    dst[h + k] = (uint32_t)((i + 1) * cols + j);
  }
  e = h + vv;
  if (rows >= 2 && cols >= 2) {
    const uint64_t cells = (uint64_t)(rows - 1) * (cols - 1);
    for (uint64_t c = 0; c < cells; ++c) {
      if (!flags[c]) continue;
      uint64_t i = c / (cols - 1), j = c % (cols - 1);
      src[e] = (uint32_t)((i + 1) * cols + j);
      dst[e] = (uint32_t)(i * cols + j + 1);
      ++e;
    }
  }
  return e;
}
