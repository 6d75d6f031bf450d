/*
 * CPU oracle for the index-free FORA single-source PPR query
 * (Wang et al., "Efficient Algorithms for Approximate Single-Source
 * Personalized PageRank Queries", TODS 2019).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It is plain, slow, FP64 C that
 * follows the paper's steps in the paper's order; it shares no code with the
 * CUDA path.
 *
 * Steps and the passages they follow:
 *   - parameters: omega = r_sum * (2eps/3 + 2) * log(2/p_f) / (eps^2 delta)
 *     (Alg. 2) and the r_max rule (Eq. rmax, Section 3.2, with its
 *     Case 2 fallback when m * r_max > 1);
 *   - Forward Push (Alg. 1), run as synchronous rounds: round t takes the set
 *     F_t of every v with r(v)/d_out(v) > r_max (Section 2.2 takes all nodes
 *     above the threshold at once), first moves alpha*r(v) to the reserve
 *     and zeroes r(v) for all of F_t, then spreads (1-alpha)*r(v)/d_out(v) to
 *     every out-neighbour; residue arriving at a node of F_t during round t
 *     waits for round t+1.  The test is written r(v) > r_max * d_out(v);
 *   - random walks (Alg. 2): for every v with r(v) > 0,
 *     omega_v = ceil(r(v) * omega / r_sum) walks, each adding
 *     a_v * r_sum / omega = r(v) / omega_v to the estimate of its end node.
 *     omega / r_sum is the constant C = (2eps/3+2) log(2/p_f) / (eps^2 delta),
 *     so omega_v = ceil(r(v) * C).  Each walk stops with probability alpha at
 *     every node, else moves to a uniform out-neighbour (Section 2.1);
 *   - estimate pi_hat(t) = reserve(t) + sum of walk weights ending at t;
 *   - top-k by (pi_hat descending, id ascending) (Section 2.1: the query
 *     returns the k nodes with the highest PPR values);
 *   - the FORA+ walk index (Section 3.3, Eq. index-rwnum): omega_max(v) stored
 *     walk ends per node, and the walk phase that takes the first omega_v of
 *     them (oracle_walk_index, oracle_walk_phase_indexed).
 *
 * Readings where the paper is silent (the same ones the CUDA path takes):
 *   - log is the natural logarithm;
 *   - the random stream of walk j from node v for source s is Philox4x32-10
 *     (Salmon et al., SC'11) with counter (c, j, v, s), c = 0, 1, ..., and
 *     key (seed low 32 bits, seed high 32 bits); the walk consumes the four
 *     output words of block c, then of block c+1, and so on;
 *   - at every node the walk takes one word u and stops if u < T_alpha with
 *     T_alpha = floor(alpha * 2^32); otherwise it picks the neighbour index in
 *     [0, d) by Lemire's multiply-and-reject method (unbiased), consuming one
 *     word per try;
 *   - the per-walk weight r(v)/omega_v is accumulated as an unsigned 64-bit
 *     fixed-point number with 63 fractional bits, W_v = rint(w_v * 2^63), so
 *     the sum does not depend on the order of the walks; pi_hat(t) =
 *     reserve(t) + acc(t) * 2^-63;
 *   - a walk longer than ORACLE_WALK_CAP steps is an error (probability
 *     (1-alpha)^cap).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_BAD_ARG (-1)
#define ORACLE_ERR_DANGLING (-2)
#define ORACLE_ERR_OOM (-3)
#define ORACLE_ERR_WALK_OVERFLOW (-4)
#define ORACLE_ERR_PUSH_NOT_CONVERGED (-5)
#define ORACLE_ERR_WALK_CAP (-6)

#define ORACLE_WALK_CAP 16384
#define ORACLE_ROUND_CAP 1000000

typedef struct {
  int64_t rounds;       /* push rounds executed */
  int64_t pushes;       /* node pushes (|F_0| + |F_1| + ...) */
  int64_t edge_pushes;  /* sum of d_out over pushed nodes */
  double rsum;          /* sum of residues after the push */
} oracle_push_stats;

typedef struct {
  int64_t residual_nodes; /* nodes with r(v) > 0 */
  int64_t walks;          /* sum of omega_v */
  int64_t walk_steps;     /* total moves over all walks */
} oracle_walk_stats;

/* ---------------------------------------------------------------- params */

/* C = omega / r_sum = (2eps/3 + 2) * log(2/p_f) / (eps^2 * delta)  (Alg. 2). */
double oracle_walk_scale(double eps, double delta, double pf) {
  return ((2.0 * eps / 3.0 + 2.0) * log(2.0 / pf)) / (eps * eps * delta);
}

/* r_max by Eq. (rmax) of Section 3.2; if m * r_max > 1 (Case 2) use
 * eps^2 delta / ((2eps/3 + 2) log(2/p_f)). */
double oracle_rmax_rule(double eps, double delta, double pf, double m) {
  double rmax = (eps / sqrt(m)) * sqrt(delta / ((2.0 * eps / 3.0 + 2.0) * log(2.0 / pf)));
  if (m * rmax > 1.0)
    rmax = (eps * eps * delta) / ((2.0 * eps / 3.0 + 2.0) * log(2.0 / pf));
  return rmax;
}

/* Stop test threshold: a walk stops when its 32-bit word is < floor(alpha * 2^32). */
uint32_t oracle_alpha_threshold(double alpha) {
  return (uint32_t)floor(alpha * 4294967296.0);
}

/* --------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11, Section 3). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------ helpers */

static int check_graph(int64_t n, const int64_t *row_ptr, const int32_t *col) {
  if (n <= 0 || n > 0x7FFFFFFF || !row_ptr || !col) return ORACLE_ERR_BAD_ARG;
  if (row_ptr[0] != 0) return ORACLE_ERR_BAD_ARG;
  for (int64_t v = 0; v < n; ++v) {
    if (row_ptr[v + 1] < row_ptr[v]) return ORACLE_ERR_BAD_ARG;
    if (row_ptr[v + 1] == row_ptr[v]) return ORACLE_ERR_DANGLING;
  }
  for (int64_t e = 0; e < row_ptr[n]; ++e)
    if (col[e] < 0 || col[e] >= n) return ORACLE_ERR_BAD_ARG;
  return ORACLE_OK;
}

/* ------------------------------------------------------- Forward Push */

/*
 * Forward Push (Alg. 1) from source s in synchronous rounds.
 * Writes reserve[n] and residue[n] (caller-allocated).
 */
int oracle_forward_push(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                        double alpha, double rmax, double *reserve, double *residue,
                        oracle_push_stats *st) {
  int rc = check_graph(n, row_ptr, col);
  if (rc) return rc;
  if (s < 0 || s >= n || !(alpha > 0.0 && alpha < 1.0) || !(rmax > 0.0)) return ORACLE_ERR_BAD_ARG;

  int32_t *frontier = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *taken = (double *)malloc(sizeof(double) * (size_t)n);
  if (!frontier || !taken) {
    free(frontier); free(taken);
    return ORACLE_ERR_OOM;
  }
  oracle_push_stats local = {0, 0, 0, 0.0};

  /* Alg. 1 */
  for (int64_t v = 0; v < n; ++v) { reserve[v] = 0.0; residue[v] = 0.0; }
  residue[s] = 1.0;

  for (;;) {
    /* the set of nodes with r(v)/d_out(v) > r_max, in ascending id */
    int64_t nf = 0;
    for (int64_t v = 0; v < n; ++v) {
      double d = (double)(row_ptr[v + 1] - row_ptr[v]);
      if (residue[v] > rmax * d) frontier[nf++] = (int32_t)v;
    }
    if (nf == 0) break;
    if (local.rounds >= ORACLE_ROUND_CAP) {
      free(frontier); free(taken);
      return ORACLE_ERR_PUSH_NOT_CONVERGED;
    }
    local.rounds++;
    local.pushes += nf;

    /* reserve(v) += alpha * r(v); r(v) = 0, for every v of the round */
    for (int64_t i = 0; i < nf; ++i) {
      int32_t v = frontier[i];
      taken[i] = residue[v];
      reserve[v] += alpha * taken[i];
      residue[v] = 0.0;
    }
    /* r(u) += (1 - alpha) * r(v) / d_out(v) for every out-neighbour u */
    for (int64_t i = 0; i < nf; ++i) {
      int32_t v = frontier[i];
      int64_t d = row_ptr[v + 1] - row_ptr[v];
      double inc = ((1.0 - alpha) * taken[i]) / (double)d;
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) residue[col[e]] += inc;
      local.edge_pushes += d;
    }
  }
  for (int64_t v = 0; v < n; ++v) local.rsum += residue[v];
  free(frontier);
  free(taken);
  if (st) *st = local;
  return ORACLE_OK;
}

/*
 * Forward Push with push/walk balancing (Section 4.2, Alg. 3), in synchronous rounds.
 * Alg. 3 keeps pushing while some node is above the threshold and the push cost so far,
 * FC, is below the estimated cost of the walks that would follow, omega * rc, where
 * omega = r_sum * C' (C' = C, or (1 - alpha) C with zero-hop pruning) and rc is the cost
 * of one walk; it starts from r_max = 1.  Read here: the threshold theta starts at 1 and
 * is halved whenever no node is above it (with theta = 1 nothing can be, since r <= 1 <=
 * d_out), so the threshold falls until the cost rule stops the push.  Costs are counted,
 * not timed: FC = cost_edge * (edge pushes) + cost_push * (node pushes), and
 * r_sum = 1 - (sum of the alpha r(v) moved to reserves), as the mass is conserved.
 * Each loop step: stop if FC >= (r_sum * C') * cost_walk; else take the set of nodes
 * with r(v) > theta * d_out(v) (ascending id) and push it as one round (as
 * oracle_forward_push does), or halve theta if the set is empty.
 * Writes reserve[n], residue[n], the statistics and the final theta.
 */
int oracle_forward_push_balanced(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                 int32_t s, double alpha, double walk_scale, double cost_edge,
                                 double cost_push, double cost_walk, double *reserve,
                                 double *residue, oracle_push_stats *st, double *theta_out) {
  int rc = check_graph(n, row_ptr, col);
  if (rc) return rc;
  if (s < 0 || s >= n || !(alpha > 0.0 && alpha < 1.0) || !(walk_scale > 0.0) ||
      !(cost_edge >= 0.0) || !(cost_push >= 0.0) || !(cost_walk >= 0.0))
    return ORACLE_ERR_BAD_ARG;
  int32_t *frontier = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *taken = (double *)malloc(sizeof(double) * (size_t)n);
  if (!frontier || !taken) {
    free(frontier); free(taken);
    return ORACLE_ERR_OOM;
  }
  oracle_push_stats local = {0, 0, 0, 0.0};
  for (int64_t v = 0; v < n; ++v) { reserve[v] = 0.0; residue[v] = 0.0; }
  residue[s] = 1.0;
  double theta = 1.0;
  double moved = 0.0;  /* sum of alpha * r(v) over all pushes */
  int64_t steps = 0;
  for (;;) {
    const double fc = cost_edge * (double)local.edge_pushes + cost_push * (double)local.pushes;
    const double walk_cost = ((1.0 - moved) * walk_scale) * cost_walk;
    if (fc >= walk_cost) break;
    if (steps++ >= ORACLE_ROUND_CAP) {
      free(frontier); free(taken);
      return ORACLE_ERR_PUSH_NOT_CONVERGED;
    }
    int64_t nf = 0;
    for (int64_t v = 0; v < n; ++v) {
      double d = (double)(row_ptr[v + 1] - row_ptr[v]);
      if (residue[v] > theta * d) frontier[nf++] = (int32_t)v;
    }
    if (nf == 0) {
      theta = 0.5 * theta;
      continue;
    }
    local.rounds++;
    local.pushes += nf;
    for (int64_t i = 0; i < nf; ++i) {
      int32_t v = frontier[i];
      taken[i] = residue[v];
      reserve[v] += alpha * taken[i];
      moved += alpha * taken[i];
      residue[v] = 0.0;
    }
    for (int64_t i = 0; i < nf; ++i) {
      int32_t v = frontier[i];
      int64_t d = row_ptr[v + 1] - row_ptr[v];
      double inc = ((1.0 - alpha) * taken[i]) / (double)d;
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) residue[col[e]] += inc;
      local.edge_pushes += d;
    }
  }
  for (int64_t v = 0; v < n; ++v) local.rsum += residue[v];
  free(frontier);
  free(taken);
  if (st) *st = local;
  if (theta_out) *theta_out = theta;
  return ORACLE_OK;
}

/* ---------------------------------------------------------- walk phase */

typedef struct {
  uint32_t ctr[4];
  uint32_t key[2];
  uint32_t buf[4];
  int pos;
  int64_t words;
} walk_stream;

static void stream_init(walk_stream *w, uint32_t j, uint32_t v, uint32_t s, uint64_t seed) {
  w->ctr[0] = 0; w->ctr[1] = j; w->ctr[2] = v; w->ctr[3] = s;
  w->key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  w->key[1] = (uint32_t)(seed >> 32);
  w->pos = 4;
  w->words = 0;
}

static uint32_t stream_next(walk_stream *w) {
  if (w->pos == 4) {
    oracle_philox4x32_10(w->ctr, w->key, w->buf);
    w->ctr[0] += 1;
    w->pos = 0;
  }
  w->words++;
  return w->buf[w->pos++];
}

/* uniform index in [0, d) by Lemire's multiply-and-reject method. */
static uint32_t uniform_index(walk_stream *w, uint32_t d) {
  uint64_t m = (uint64_t)stream_next(w) * d;
  uint32_t low = (uint32_t)m;
  if (low < d) {
    uint32_t reject_below = (0u - d) % d; /* 2^32 mod d */
    while (low < reject_below) {
      m = (uint64_t)stream_next(w) * d;
      low = (uint32_t)m;
    }
  }
  return (uint32_t)(m >> 32);
}

/* One alpha-terminating random walk (Section 2.1) from v; returns its end node or -1 on cap. */
static int64_t random_walk(const int64_t *row_ptr, const int32_t *col, uint32_t t_alpha,
                           walk_stream *w, int32_t v, int64_t *steps) {
  int64_t x = v;
  for (int64_t step = 0; step < ORACLE_WALK_CAP; ++step) {
    uint32_t u = stream_next(w);
    if (u < t_alpha) return x;
    uint32_t d = (uint32_t)(row_ptr[x + 1] - row_ptr[x]);
    uint32_t idx = uniform_index(w, d);
    x = col[row_ptr[x] + idx];
    (*steps)++;
  }
  return -1;
}

/*
 * Random-walk phase of Alg. 2 on a given residue vector:
 * omega_v = ceil(r(v) * C) walks from every v with r(v) > 0, each adding
 * W_v = rint((r(v)/omega_v) * 2^63) to acc[end] and 1 to count[end].
 * count[n] and acc[n] are caller-allocated and overwritten.
 */
int oracle_walk_phase(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                      double alpha, double walk_scale, uint64_t seed, const double *residue,
                      uint32_t *count, uint64_t *acc, oracle_walk_stats *st) {
  int rc = check_graph(n, row_ptr, col);
  if (rc) return rc;
  if (s < 0 || s >= n || !(alpha > 0.0 && alpha < 1.0) || !(walk_scale > 0.0))
    return ORACLE_ERR_BAD_ARG;
  const uint32_t t_alpha = oracle_alpha_threshold(alpha);
  oracle_walk_stats local = {0, 0, 0};
  for (int64_t t = 0; t < n; ++t) { count[t] = 0; acc[t] = 0; }

  /* total walk budget first: per source the walk count must fit in 32 bits */
  for (int64_t v = 0; v < n; ++v) {
    if (residue[v] > 0.0) {
      double omega_v = ceil(residue[v] * walk_scale);
      local.residual_nodes++;
      if (omega_v > 4294967295.0) return ORACLE_ERR_WALK_OVERFLOW;
      local.walks += (int64_t)omega_v;
    } else if (residue[v] < 0.0) {
      return ORACLE_ERR_BAD_ARG;
    }
  }
  if (local.walks > 4294967295LL) return ORACLE_ERR_WALK_OVERFLOW;

  for (int64_t v = 0; v < n; ++v) {
    if (!(residue[v] > 0.0)) continue;
    const double omega_v = ceil(residue[v] * walk_scale);
    const double weight = residue[v] / omega_v;              /* a_v * r_sum / omega */
    const uint64_t fixed = (uint64_t)nearbyint(ldexp(weight, 63));
    const uint32_t nw = (uint32_t)omega_v;
    for (uint32_t j = 0; j < nw; ++j) {
      walk_stream w;
      stream_init(&w, j, (uint32_t)v, (uint32_t)s, seed);
      int64_t end = random_walk(row_ptr, col, t_alpha, &w, (int32_t)v, &local.walk_steps);
      if (end < 0) return ORACLE_ERR_WALK_CAP;
      count[end] += 1;
      acc[end] += fixed;
    }
  }
  if (st) *st = local;
  return ORACLE_OK;
}

/*
 * Walk phase with zero-hop pruning (Section 4.1).  A walk from v stops at v at once
 * with probability alpha, so that part of r(v) goes straight to the estimate
 * (alpha r(v), added by oracle_estimate_zero_hop) and only r'(v) = (1 - alpha) r(v)
 * is sampled: omega_v = ceil(r'(v) * C) walks from v, each of which first moves to a
 * uniform out-neighbour u of v (no stop test at v) and then runs the alpha-terminating
 * walk from u; each adds r'(v) / omega_v at its end.  This applies (1 - alpha) once,
 * as the derivation of Section 4.1 does (Alg. 3 applies it twice, a typo).
 * The walk's word stream is the same as in oracle_walk_phase: the forced first move
 * draws its neighbour index first.
 */
int oracle_walk_phase_zero_hop(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                               double alpha, double walk_scale, uint64_t seed,
                               const double *residue, uint32_t *count, uint64_t *acc,
                               oracle_walk_stats *st) {
  int rc = check_graph(n, row_ptr, col);
  if (rc) return rc;
  if (s < 0 || s >= n || !(alpha > 0.0 && alpha < 1.0) || !(walk_scale > 0.0))
    return ORACLE_ERR_BAD_ARG;
  const uint32_t t_alpha = oracle_alpha_threshold(alpha);
  oracle_walk_stats local = {0, 0, 0};
  for (int64_t t = 0; t < n; ++t) { count[t] = 0; acc[t] = 0; }
  for (int64_t v = 0; v < n; ++v) {
    if (residue[v] > 0.0) {
      const double omega_v = ceil(((1.0 - alpha) * residue[v]) * walk_scale);
      local.residual_nodes++;
      if (omega_v > 4294967295.0) return ORACLE_ERR_WALK_OVERFLOW;
      local.walks += (int64_t)omega_v;
    } else if (residue[v] < 0.0) {
      return ORACLE_ERR_BAD_ARG;
    }
  }
  if (local.walks > 4294967295LL) return ORACLE_ERR_WALK_OVERFLOW;
  for (int64_t v = 0; v < n; ++v) {
    if (!(residue[v] > 0.0)) continue;
    const double r_kept = (1.0 - alpha) * residue[v];
    const double omega_v = ceil(r_kept * walk_scale);
    const double weight = r_kept / omega_v;
    const uint64_t fixed = (uint64_t)nearbyint(ldexp(weight, 63));
    const uint32_t nw = (uint32_t)omega_v;
    const uint32_t dv = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
    for (uint32_t j = 0; j < nw; ++j) {
      walk_stream w;
      stream_init(&w, j, (uint32_t)v, (uint32_t)s, seed);
      const uint32_t idx = uniform_index(&w, dv); /* the forced first move */
      const int32_t u = col[row_ptr[v] + idx];
      local.walk_steps += 1;
      int64_t end = random_walk(row_ptr, col, t_alpha, &w, u, &local.walk_steps);
      if (end < 0) return ORACLE_ERR_WALK_CAP;
      count[end] += 1;
      acc[end] += fixed;
    }
  }
  if (st) *st = local;
  return ORACLE_OK;
}

/*
 * FORA+ walk index (Section 3.3).  After the push every residue satisfies
 * r(v) <= RN(r_max * d(v)), so a query needs at most
 *     omega_max(v) = ceil(RN(RN(r_max * d(v)) * C))
 * walks from v (Eq. index-rwnum with the same FP64 operations as omega_v, so that
 * omega_v <= omega_max(v) holds exactly).  The index stores, for every v, the end
 * nodes of walks j = 0 .. omega_max(v) - 1 from v, walk j reading the Philox stream
 * with counter (c, j, v, s_index), the same walk definition as oracle_walk_phase.
 * With zero_hop the stored walks are those of oracle_walk_phase_zero_hop (a forced
 * first move, Section 4.1) and omega_max(v) = ceil(RN(RN((1 - alpha) RN(r_max d(v))) C)),
 * the bound of that phase's omega_v (the index is then smaller by about alpha).
 * off[n + 1] is the exclusive prefix of omega_max; dest[off[v] + j] is the end of walk
 * j from v.  Returns the total number of walks (off[n]) when it is <= cap and dest is
 * filled; with cap smaller than that it fills off only and returns the total, negated
 * error codes otherwise.
 */
int64_t oracle_walk_index(int64_t n, const int64_t *row_ptr, const int32_t *col, double alpha,
                          double walk_scale, double rmax, uint64_t seed, uint32_t s_index,
                          int zero_hop, int64_t *off, int32_t *dest, int64_t cap) {
  int rc = check_graph(n, row_ptr, col);
  if (rc) return rc;
  if (!(alpha > 0.0 && alpha < 1.0) || !(walk_scale > 0.0) || !(rmax > 0.0))
    return ORACLE_ERR_BAD_ARG;
  off[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    const double d = (double)(row_ptr[v + 1] - row_ptr[v]);
    const double r_bound = rmax * d;
    const double omega_max = zero_hop ? ceil(((1.0 - alpha) * r_bound) * walk_scale)
                                      : ceil(r_bound * walk_scale);
    if (omega_max > 4294967295.0) return ORACLE_ERR_WALK_OVERFLOW;
    off[v + 1] = off[v] + (int64_t)omega_max;
  }
  const int64_t total = off[n];
  if (total > cap) return total;
  const uint32_t t_alpha = oracle_alpha_threshold(alpha);
  int64_t steps = 0;
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t j = 0; j < off[v + 1] - off[v]; ++j) {
      walk_stream w;
      stream_init(&w, (uint32_t)j, (uint32_t)v, s_index, seed);
      int32_t start = (int32_t)v;
      if (zero_hop) { /* the forced first move */
        const uint32_t dv = (uint32_t)(row_ptr[v + 1] - row_ptr[v]);
        start = col[row_ptr[v] + uniform_index(&w, dv)];
        steps += 1;
      }
      const int64_t end = random_walk(row_ptr, col, t_alpha, &w, start, &steps);
      if (end < 0) return ORACLE_ERR_WALK_CAP;
      dest[off[v] + j] = (int32_t)end;
    }
  }
  return total;
}

/*
 * Walk phase of Alg. 2 served from a FORA+ index (Section 3.3): for every v with
 * r(v) > 0, the ends of the first omega_v = ceil(r(v) * C) walks stored for v, each
 * adding W_v = rint((r(v)/omega_v) * 2^63) to acc[end] and 1 to count[end].  An
 * omega_v above the index's omega_max(v) is an error (the residue exceeds the index's
 * r_max).  st->walk_steps stays 0 (no walk is simulated).  With zero_hop (an index of
 * zero-hop walks) the residue sampled is (1 - alpha) r(v), as in
 * oracle_walk_phase_zero_hop; alpha r(v) goes to the estimate there.
 */
int oracle_walk_phase_indexed(int64_t n, double alpha, double walk_scale, const double *residue,
                              const int64_t *off, const int32_t *dest, int zero_hop,
                              uint32_t *count, uint64_t *acc, oracle_walk_stats *st) {
  if (n < 1 || !(walk_scale > 0.0) || !(alpha > 0.0 && alpha < 1.0)) return ORACLE_ERR_BAD_ARG;
  oracle_walk_stats local = {0, 0, 0};
  for (int64_t t = 0; t < n; ++t) { count[t] = 0; acc[t] = 0; }
  for (int64_t v = 0; v < n; ++v) {
    if (residue[v] < 0.0) return ORACLE_ERR_BAD_ARG;
    if (!(residue[v] > 0.0)) continue;
    const double r_sampled = zero_hop ? (1.0 - alpha) * residue[v] : residue[v];
    const double omega_v = ceil(r_sampled * walk_scale);
    if (omega_v > (double)(off[v + 1] - off[v])) return ORACLE_ERR_BAD_ARG;
    const double weight = r_sampled / omega_v;
    const uint64_t fixed = (uint64_t)nearbyint(ldexp(weight, 63));
    local.residual_nodes++;
    local.walks += (int64_t)omega_v;
    for (int64_t j = 0; j < (int64_t)omega_v; ++j) {
      const int32_t end = dest[off[v] + j];
      count[end] += 1;
      acc[end] += fixed;
    }
  }
  if (st) *st = local;
  return ORACLE_OK;
}

/* Zero-hop estimate: pi_hat(t) = (reserve(t) + alpha * r(t)) + acc(t) * 2^-63 */
void oracle_estimate_zero_hop(int64_t n, const double *reserve, const double *residue,
                              const uint64_t *acc, double alpha, double *est) {
  for (int64_t t = 0; t < n; ++t)
    est[t] = (reserve[t] + alpha * residue[t]) + ldexp((double)acc[t], -63);
}

/* pi_hat(t) = reserve(t) + acc(t) * 2^-63 */
void oracle_estimate(int64_t n, const double *reserve, const uint64_t *acc, double *est) {
  for (int64_t t = 0; t < n; ++t) est[t] = reserve[t] + ldexp((double)acc[t], -63);
}

/* --------------------------------------------------------------- top-k */

static const double *g_sort_est; /* qsort has no context argument in C11 */

static int by_estimate_then_id(const void *pa, const void *pb) {
  int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
  double ea = g_sort_est[a], eb = g_sort_est[b];
  if (ea > eb) return -1;
  if (ea < eb) return 1;
  return (a > b) - (a < b);
}

/* The k nodes with the largest estimates, ties by ascending id (full sort). */
int oracle_topk(int64_t n, const double *est, int64_t k, int32_t *ids, double *vals) {
  if (n <= 0 || k < 0 || k > n) return ORACLE_ERR_BAD_ARG;
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!order) return ORACLE_ERR_OOM;
  for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
  g_sort_est = est;
  qsort(order, (size_t)n, sizeof(int32_t), by_estimate_then_id);
  for (int64_t i = 0; i < k; ++i) {
    ids[i] = order[i];
    vals[i] = est[order[i]];
  }
  free(order);
  return ORACLE_OK;
}

/* ----------------------------------------------------- whole query */

/*
 * One whole query (Alg. 2 then top-k).  rmax <= 0 selects the r_max rule.
 * reserve/residue/count/acc/est are caller-allocated [n] work arrays whose
 * final contents are the query's intermediate results.
 */
int oracle_ssppr(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                 double alpha, double eps, double delta, double pf, double rmax,
                 uint64_t seed, int64_t k, double *reserve, double *residue, uint32_t *count,
                 uint64_t *acc, double *est, int32_t *ids, double *vals,
                 oracle_push_stats *pst, oracle_walk_stats *wst) {
  if (!(eps > 0.0) || !(delta > 0.0) || !(pf > 0.0 && pf < 1.0)) return ORACLE_ERR_BAD_ARG;
  if (!(rmax > 0.0)) rmax = oracle_rmax_rule(eps, delta, pf, (double)row_ptr[n]);
  int rc = oracle_forward_push(n, row_ptr, col, s, alpha, rmax, reserve, residue, pst);
  if (rc) return rc;
  rc = oracle_walk_phase(n, row_ptr, col, s, alpha, oracle_walk_scale(eps, delta, pf), seed,
                         residue, count, acc, wst);
  if (rc) return rc;
  oracle_estimate(n, reserve, acc, est);
  return oracle_topk(n, est, k, ids, vals);
}

/* The whole query with zero-hop pruning (Section 4.1) in the walk phase. */
int oracle_ssppr_zero_hop(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                          double alpha, double eps, double delta, double pf, double rmax,
                          uint64_t seed, int64_t k, double *reserve, double *residue,
                          uint32_t *count, uint64_t *acc, double *est, int32_t *ids,
                          double *vals, oracle_push_stats *pst, oracle_walk_stats *wst) {
  if (!(eps > 0.0) || !(delta > 0.0) || !(pf > 0.0 && pf < 1.0)) return ORACLE_ERR_BAD_ARG;
  if (!(rmax > 0.0)) rmax = oracle_rmax_rule(eps, delta, pf, (double)row_ptr[n]);
  int rc = oracle_forward_push(n, row_ptr, col, s, alpha, rmax, reserve, residue, pst);
  if (rc) return rc;
  rc = oracle_walk_phase_zero_hop(n, row_ptr, col, s, alpha, oracle_walk_scale(eps, delta, pf),
                                  seed, residue, count, acc, wst);
  if (rc) return rc;
  oracle_estimate_zero_hop(n, reserve, residue, acc, alpha, est);
  return oracle_topk(n, est, k, ids, vals);
}

/* ------------------------------------------------------ top-k FORA (Alg. 5) */

/*
 * Top-k FORA (Alg. 5, Section 5.2).  For delta = 1/k, 1/(2k), 1/(4k), ... and finally
 * 1/n, run Alg. 2 with eps' = eps/2, failure probability p_f' = p_f / (n log2(n/k))
 * and r_max by Eq. (rmax) for these parameters (or the given rmax > 0); stop as soon
 * as the k-th largest estimate is >= (1 + eps) delta and return that round's top-k.
 * Readings: iteration i < I = ceil(log2(n/k)) uses delta_i = 1/(k 2^i), the last one
 * delta_I = 1/n; log2(n/k) is taken as at least 1; round i draws its walks with key
 * seed + i.  *iterations and *final_delta report where it stopped.
 */
int oracle_topk_fora(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
                     double alpha, double eps, double pf, double rmax, uint64_t seed,
                     int64_t k, double *reserve, double *residue, uint32_t *count,
                     uint64_t *acc, double *est, int32_t *ids, double *vals,
                     int32_t *iterations, double *final_delta) {
  if (k < 1 || k > n || !(eps > 0.0) || !(pf > 0.0 && pf < 1.0)) return ORACLE_ERR_BAD_ARG;
  int32_t rounds_total = 0;
  while ((double)k * ldexp(1.0, rounds_total) < (double)n) ++rounds_total; /* I */
  double lg = log2((double)n / (double)k);
  if (lg < 1.0) lg = 1.0;
  const double pf_round = pf / ((double)n * lg);
  for (int32_t i = 0; i <= rounds_total; ++i) {
    const double delta = i < rounds_total ? 1.0 / ((double)k * ldexp(1.0, i)) : 1.0 / (double)n;
    int rc = oracle_ssppr(n, row_ptr, col, s, alpha, eps / 2.0, delta, pf_round, rmax,
                          seed + (uint64_t)i, k, reserve, residue, count, acc, est, ids, vals,
                          NULL, NULL);
    if (rc) return rc;
    if (vals[k - 1] >= (1.0 + eps) * delta || i == rounds_total) {
      if (iterations) *iterations = i + 1;
      if (final_delta) *final_delta = delta;
      return ORACLE_OK;
    }
  }
  return ORACLE_OK; /* not reached */
}
