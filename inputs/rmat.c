/*
 * Seeded synthetic inputs: directed R-MAT graphs in CSR form and uniform
 * query sources.
 *
 * This module is shared by the CPU oracle and by the CUDA path.  It holds
 * none of the query method's arithmetic (no push, no walk, no estimate):
 * it only produces graphs and source lists, the stand-ins for the social
 * graphs of the paper's experiments (Section 8, Table "Datasets"), which
 * generates its own synthetic graphs with the R-MAT model
 * (Chakrabarti, Zhan, Faloutsos 2004).
 *
 * Recipe (one directed edge per draw, duplicates and self-loops kept):
 *   - edge e picks its (src, dst) cell by `scale` recursive quadrant choices,
 *     most significant bit first, with probabilities (a, b, c, 1-a-b-c) for
 *     quadrants (0,0), (0,1), (1,0), (1,1); each choice uses 16 random bits;
 *   - the node ids are relabelled by a seeded uniform permutation so that
 *     hubs are not clustered at low ids;
 *   - every node left with no out-edge gets one edge to a uniform node
 *     (the random-walk definition of Section 2.1 needs d_out >= 1);
 *   - CSR: rows by source id, each row's targets sorted ascending.
 *
 * Randomness: splitmix64 used as a counter-based generator,
 *   word(seed, stream, i) = mix64(base(seed, stream) + (i + 1) * GOLDEN),
 * so that every edge depends on its index only and the result does not
 * depend on the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

enum { STREAM_EDGES = 1, STREAM_PERM = 2, STREAM_DANGLING = 3, STREAM_SOURCES = 4 };

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(seed * 0xD1B54A32D192ED03ULL + stream * GOLDEN);
}

static inline uint64_t word(uint64_t base, uint64_t i) {
  return mix64(base + (i + 1) * GOLDEN);
}

/* uniform integer in [0, bound) from a 64-bit word (multiply-high). */
static inline uint64_t bounded(uint64_t w, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)w * bound) >> 64);
}

typedef struct {
  int scale;
  uint64_t e_begin, e_end;
  uint64_t base;
  uint32_t qa, qab, qabc; /* cumulative 16-bit thresholds */
  uint32_t *src, *dst;
} edge_job;

static void *edge_worker(void *p) {
  edge_job *j = (edge_job *)p;
  for (uint64_t e = j->e_begin; e < j->e_end; ++e) {
    uint32_t s = 0, d = 0;
    uint64_t w = 0;
    for (int l = 0; l < j->scale; ++l) {
      if ((l & 3) == 0) w = word(j->base, e * 8 + (uint64_t)(l >> 2));
      uint32_t q = (uint32_t)(w & 0xFFFF);
      w >>= 16;
      uint32_t sb, db;
      if (q < j->qa) { sb = 0; db = 0; }
      else if (q < j->qab) { sb = 0; db = 1; }
      else if (q < j->qabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      s = (s << 1) | sb;
      d = (d << 1) | db;
    }
    j->src[e] = s;
    j->dst[e] = d;
  }
  return NULL;
}

/*
 * Generate an R-MAT graph with n = 2^scale nodes and n*avg_deg raw edges,
 * then apply the id permutation and the dangling fix and build the CSR.
 *
 * On success returns 0 and sets *row_ptr_out (n+1 int64) and *col_out
 * (m int32) to malloc'ed arrays owned by the caller (free with
 * rmat_free); *m_out is the final edge count (raw edges + dangling-fix
 * edges).  Returns -1 on bad arguments, -2 on allocation failure.
 */
int rmat_generate(int scale, double avg_deg, double a, double b, double c,
                  uint64_t seed, int nthreads, int64_t **row_ptr_out,
                  int32_t **col_out, int64_t *m_out) {
  if (scale < 1 || scale > 30 || avg_deg <= 0.0 || a < 0 || b < 0 || c < 0 ||
      a + b + c > 1.0 || nthreads < 1)
    return -1;
  const uint64_t n = 1ULL << scale;
  const uint64_t m_raw = (uint64_t)(avg_deg * (double)n + 0.5);
  if (m_raw + n >= (1ULL << 32)) return -1;

  uint32_t *src = (uint32_t *)malloc((m_raw + n) * sizeof(uint32_t));
  uint32_t *dst = (uint32_t *)malloc((m_raw + n) * sizeof(uint32_t));
  uint32_t *perm = (uint32_t *)malloc(n * sizeof(uint32_t));
  int64_t *deg = (int64_t *)calloc(n + 1, sizeof(int64_t));
  if (!src || !dst || !perm || !deg) {
    free(src); free(dst); free(perm); free(deg);
    return -2;
  }

  /* 1. raw edges, in parallel by index ranges */
  edge_job *jobs = (edge_job *)malloc(sizeof(edge_job) * (size_t)nthreads);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  const uint64_t base = stream_base(seed, STREAM_EDGES);
  const uint32_t qa = (uint32_t)(a * 65536.0 + 0.5);
  const uint32_t qab = (uint32_t)((a + b) * 65536.0 + 0.5);
  const uint32_t qabc = (uint32_t)((a + b + c) * 65536.0 + 0.5);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].scale = scale;
    jobs[t].e_begin = m_raw * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].e_end = m_raw * (uint64_t)(t + 1) / (uint64_t)nthreads;
    jobs[t].base = base;
    jobs[t].qa = qa; jobs[t].qab = qab; jobs[t].qabc = qabc;
    jobs[t].src = src; jobs[t].dst = dst;
  }
  int started = 0;
  for (int t = 1; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, edge_worker, &jobs[t]) == 0) started = t;
    else { edge_worker(&jobs[t]); }
  edge_worker(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);

  /* 2. seeded uniform relabelling (Fisher-Yates) */
  const uint64_t pbase = stream_base(seed, STREAM_PERM);
  for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
  for (uint64_t i = n - 1; i > 0; --i) {
    uint64_t j = bounded(word(pbase, i), i + 1);
    uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  for (uint64_t e = 0; e < m_raw; ++e) {
    src[e] = perm[src[e]];
    dst[e] = perm[dst[e]];
  }
  free(perm);

  /* 3. dangling fix: one edge to a uniform node for every node with d_out = 0 */
  for (uint64_t e = 0; e < m_raw; ++e) deg[src[e]]++;
  uint64_t m = m_raw;
  const uint64_t dbase = stream_base(seed, STREAM_DANGLING);
  for (uint64_t v = 0; v < n; ++v) {
    if (deg[v] == 0) {
      src[m] = (uint32_t)v;
      dst[m] = (uint32_t)bounded(word(dbase, v), n);
      deg[v] = 1;
      ++m;
    }
  }

  /* 4. CSR with sorted rows: stable counting sort by dst, then by src */
  uint32_t *s2 = (uint32_t *)malloc(m * sizeof(uint32_t));
  uint32_t *d2 = (uint32_t *)malloc(m * sizeof(uint32_t));
  int64_t *cnt = (int64_t *)calloc(n + 1, sizeof(int64_t));
  int64_t *row_ptr = (int64_t *)malloc((n + 1) * sizeof(int64_t));
  int32_t *col = (int32_t *)malloc(m * sizeof(int32_t));
  if (!s2 || !d2 || !cnt || !row_ptr || !col) {
    free(src); free(dst); free(deg); free(s2); free(d2); free(cnt);
    free(row_ptr); free(col);
    return -2;
  }
  for (uint64_t e = 0; e < m; ++e) cnt[dst[e] + 1]++;
  for (uint64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  for (uint64_t e = 0; e < m; ++e) {
    int64_t p = cnt[dst[e]]++;
    s2[p] = src[e];
    d2[p] = dst[e];
  }
  free(src);
  free(dst);
  row_ptr[0] = 0;
  for (uint64_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + deg[v];
  memcpy(cnt, row_ptr, n * sizeof(int64_t));
  for (uint64_t e = 0; e < m; ++e) col[cnt[s2[e]]++] = (int32_t)d2[e];
  free(s2);
  free(d2);
  free(cnt);
  free(deg);

  *row_ptr_out = row_ptr;
  *col_out = col;
  *m_out = (int64_t)m;
  return 0;
}

void rmat_free(void *p) { free(p); }

/* `count` query sources drawn uniformly (with replacement) from [0, n). */
int uniform_sources(int64_t n, int64_t count, uint64_t seed, int32_t *out) {
  if (n <= 0 || n > 0x7FFFFFFF || count < 0) return -1;
  const uint64_t base = stream_base(seed, STREAM_SOURCES);
  for (int64_t i = 0; i < count; ++i)
    out[i] = (int32_t)bounded(word(base, (uint64_t)i), (uint64_t)n);
  return 0;
}
