/*
 * Oracle: plain, serial, FP64 Dykstra's method for the regularized
 * correlation-clustering LP (and a threaded form of the same sweep, below).  TEST INFRASTRUCTURE ONLY: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may load
 * this code.  It shares nothing with the CUDA path.
 *
 * Problem (Sec. II-A, Eq. mn1): variables x_ij (distances) and f_ij (slacks)
 * for every pair i<j; minimize sum_{i<j} w_ij f_ij subject to
 *     x_ij <= x_ik + x_jk   for every triplet and each choice of the
 *                           "hypotenuse" pair (three rows per triplet),
 *     x_ij - d_ij <= f_ij,  d_ij - x_ij <= f_ij   for every pair.
 * Regularized form (Sec. II-B, Eq. qp): min c^T v + (eps/2) v^T W v, Av <= b,
 * with v = (x, f), c = (0, w) and W = diag(w, w) (the weights on both blocks).
 *
 * Method (Algorithm 1): y := 0, v := -(1/eps) W^{-1} c, then visit the rows
 * of A cyclically; for row a_i:
 *     correction  v := v + y_i (1/eps) W^{-1} a_i
 *     theta       := eps * max(a_i^T v - b_i, 0) / (a_i^T W^{-1} a_i)
 *     projection  v := v - theta (1/eps) W^{-1} a_i
 *     dual        y_i := theta.
 * A metric row has three nonzeros (+1 on the hypotenuse, -1 on the two legs),
 * so every update touches three entries (Sec. II-B, localized projections).
 *
 * Visiting order ("schedules", Sec. III-B): a sweep visits every triplet once
 * and, for each triplet, its three rows in the order hypotenuse = ij, ik, jk;
 * after all triplets it visits every pair's two rows (x - f <= d first).
 *   0: the paper's diagonal schedule (Sec. III-B): the set S_{i,k} holds
 *      the triplets (i, j, k), i < j < k, of one outer pair (i, k); two sets
 *      on one anti-diagonal i + k = s of the (i, k) grid share no pair, so a
 *      diagonal is a phase.  With 1-based indices the phases are s = n+1 down
 *      to 4, then s = n+2 up to 2n-2 (2n-5 phases, every (i, k) with
 *      k >= i+2 on exactly one of them); inside a phase the sets come by
 *      ascending i, inside a set the triplets by ascending middle index j.
 *   1: triplets grouped by (i+j+k) mod n; phase s = 0..n-1, inside a phase in
 *      ascending (i, j).  Two triplets of one phase that share two indices
 *      share the third, so a phase touches every pair at most once (the
 *      two-triplet lemma of Sec. III-A at triplet granularity).
 *   2: tiled (the b x b tiling idea of Sec. III-C): indices cut into blocks
 *      of B; block triples I<=J<=K grouped by (I+J+K) mod Nb (Nb = ceil(n/B)),
 *      inside a block triple sub-phases t = 0..B-1 over local offsets
 *      (a, b, c) with (a+b+c) mod B == t, then ascending (a, b).
 *
 * Storage: pairs packed row-major, p(i,j) = i*n - i(i+1)/2 + (j-i-1) for
 * i<j (0-based; the paper is 1-based).  Triangle duals y in canonical order:
 * lexicographic rank of (i<j<k), times 3, plus the row (0: hyp ij, 1: hyp ik,
 * 2: hyp jk).  Pair duals: 2 per pair, (x - f <= d, d - x <= f).
 *
 * Build with -ffp-contract=off: every product and sum is rounded on its own,
 * in the order written.
 *
 * Threaded sweeps (ora_sweep_threads, ora_sweep_l2_threads): the units of a
 * phase (a set S_{i,k} in schedule 0, a first index i in schedule 1, a block
 * triple in schedule 2) touch pairwise disjoint pairs and duals (Sec. III-A,
 * III-C), so they are dealt round-robin to T threads that wait for each other
 * at the end of every phase; every row is then computed from the same values
 * as in the serial walk, and the result is the same bit for bit.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <math.h>
#include <pthread.h>

static inline int64_t pidx(int64_t n, int64_t i, int64_t j) {
  return i * n - i * (i + 1) / 2 + (j - i - 1);
}
static inline int64_t ch2(int64_t m) { return m < 2 ? 0 : m * (m - 1) / 2; }
static inline int64_t ch3(int64_t m) { return m < 3 ? 0 : m * (m - 1) * (m - 2) / 6; }

/* lexicographic rank of i<j<k among all triplets of {0..n-1} */
int64_t ora_trank(int64_t n, int64_t i, int64_t j, int64_t k) {
  return (ch3(n) - ch3(n - i)) + (ch2(n - 1 - i) - ch2(n - j)) + (k - j - 1);
}

int64_t ora_pidx(int64_t n, int64_t i, int64_t j) { return pidx(n, i, j); }

/* Algorithm 1's initialisation: y = 0, v = -(1/eps) W^{-1} c with c = (0, w). */
void ora_init(int64_t n, double eps, const double* w, double* winv, double* x,
              double* f, double* ytri, double* ypair) {
  int64_t P = ch2(n), T = ch3(n);
  for (int64_t p = 0; p < P; ++p) {
    winv[p] = 1.0 / w[p];                 /* diagonal of W^{-1} (both blocks) */
    x[p] = 0.0;                           /* c is 0 on the x block */
    f[p] = -(1.0 / eps) * (w[p] / w[p]);  /* c is w on the f block */
    ypair[2 * p] = 0.0;
    ypair[2 * p + 1] = 0.0;
  }
  for (int64_t t = 0; t < 3 * T; ++t) ytri[t] = 0.0;
}

/* One row of Algorithm 1 for the metric constraint x_h - x_a - x_b <= 0
 * (b_i = 0; a_i = +1 at h, -1 at a and b). */
static void visit_metric_row(double eps, double* xh, double* xa, double* xb,
                             double wh, double wa, double wb, double* y) {
  double corr = *y / eps;                /* y_i (1/eps) */
  *xh = *xh + corr * wh;                 /* correction: + y_i/eps W^{-1} a_i */
  *xa = *xa - corr * wa;
  *xb = *xb - corr * wb;
  double delta = *xh - *xa - *xb;        /* a_i^T v - b_i */
  double aWa = wh + wa + wb;             /* a_i^T W^{-1} a_i */
  double theta = eps * fmax(delta, 0.0) / aWa;
  double step = theta / eps;             /* theta (1/eps) */
  *xh = *xh - step * wh;                 /* projection: - theta/eps W^{-1} a_i */
  *xa = *xa + step * wa;
  *xb = *xb + step * wb;
  *y = theta;                            /* dual update */
}

/* The three metric rows of triplet i<j<k, in the order hyp = ij, ik, jk;
 * only the first `rows` of them (1..3). */
static void visit_triplet(int64_t n, double eps, const double* winv, double* x,
                          double* ytri, int64_t i, int64_t j, int64_t k, int rows) {
  int64_t pij = pidx(n, i, j), pik = pidx(n, i, k), pjk = pidx(n, j, k);
  double* y = ytri + 3 * ora_trank(n, i, j, k);
  visit_metric_row(eps, &x[pij], &x[pik], &x[pjk], winv[pij], winv[pik], winv[pjk], &y[0]);
  if (rows < 2) return;
  visit_metric_row(eps, &x[pik], &x[pij], &x[pjk], winv[pik], winv[pij], winv[pjk], &y[1]);
  if (rows < 3) return;
  visit_metric_row(eps, &x[pjk], &x[pij], &x[pik], winv[pjk], winv[pij], winv[pik], &y[2]);
}

void ora_visit_triplet(int64_t n, double eps, const double* winv, double* x,
                       double* ytri, int64_t i, int64_t j, int64_t k, int rows) {
  visit_triplet(n, eps, winv, x, ytri, i, j, k, rows);
}

/* The two rows of pair p: x - f <= d (a = (+1, -1), b = d), then
 * d - x <= f, i.e. -x - f <= -d (a = (-1, -1), b = -d).  a^T W^{-1} a = 2/w. */
static void visit_pair(double eps, double d, double wv, double* x, double* f,
                       double* y, int rows) {
  double corr = y[0] / eps;
  *x = *x + corr * wv;
  *f = *f - corr * wv;
  double delta = *x - *f - d;
  double theta = eps * fmax(delta, 0.0) / (wv + wv);
  double step = theta / eps;
  *x = *x - step * wv;
  *f = *f + step * wv;
  y[0] = theta;
  if (rows < 2) return;
  corr = y[1] / eps;
  *x = *x - corr * wv;
  *f = *f - corr * wv;
  delta = -*x - *f + d;
  theta = eps * fmax(delta, 0.0) / (wv + wv);
  step = theta / eps;
  *x = *x + step * wv;
  *f = *f + step * wv;
  y[1] = theta;
}

void ora_visit_pair(int64_t n, double eps, const double* d, const double* winv,
                    double* x, double* f, double* ypair, int64_t p, int rows) {
  (void)n;
  visit_pair(eps, d[p], winv[p], &x[p], &f[p], &ypair[2 * p], rows);
}

/* ---- walking a schedule ------------------------------------------------ */

typedef struct {
  int64_t n;
  double eps;
  const double* winv;
  double* x;
  double* ytri;
  int64_t rows_left;  /* metric rows still allowed; < 0: no limit */
  int32_t* rec;       /* when non-NULL: record (phase, i, j, k) instead */
  int64_t rec_cap;
  int64_t count;      /* triplets reached so far */
  int64_t phase;
  /* threaded walks (all zero in a serial walk) */
  int nthr, tid;      /* this thread visits the units u with u mod nthr == tid */
  int64_t unit;       /* units started so far */
  int skip;           /* the current unit belongs to another thread */
  int64_t stop_after; /* > 0: stop after this many phases */
  pthread_barrier_t* bar;
} walk_t;

/* Start of a unit of the current phase (units of one phase are disjoint). */
static void unit_begin(walk_t* w) {
  if (w->nthr > 1) w->skip = (w->unit % w->nthr) != w->tid;
  w->unit++;
}

/* End of a phase: all threads wait here.  Returns 0 when the walk must stop. */
static int end_phase(walk_t* w) {
  w->phase++;
  if (w->bar) pthread_barrier_wait(w->bar);
  return !(w->stop_after > 0 && w->phase >= w->stop_after);
}

/* returns 0 when the walk must stop */
static int walk_step(walk_t* w, int64_t i, int64_t j, int64_t k) {
  if (w->skip) return 1;
  if (w->rec) {
    if (w->count < w->rec_cap) {
      int32_t* r = w->rec + 4 * w->count;
      r[0] = (int32_t)w->phase; r[1] = (int32_t)i; r[2] = (int32_t)j; r[3] = (int32_t)k;
    }
    w->count++;
    return 1;
  }
  int rows = 3;
  if (w->rows_left >= 0) {
    if (w->rows_left == 0) return 0;
    if (w->rows_left < 3) rows = (int)w->rows_left;
    w->rows_left -= rows;
  }
  visit_triplet(w->n, w->eps, w->winv, w->x, w->ytri, i, j, k, rows);
  w->count++;
  return 1;
}

/* Schedule 0, one phase: the sets S_{i,k} on the anti-diagonal i + k = s
 * (1-based), i.e. every i with 1 <= i, k = s - i <= n and k - i >= 2, by
 * ascending i; each set is a serial chain over j = i+1 .. k-1. */
static int walk_diagonal(walk_t* w, int64_t s) {
  const int64_t n = w->n;
  for (int64_t i = (s - n > 1 ? s - n : 1); s - i - i >= 2; ++i) {
    const int64_t k = s - i;
    unit_begin(w);
    for (int64_t j = i + 1; j < k; ++j)
      if (!walk_step(w, i - 1, j - 1, k - 1)) return 0;   /* stored 0-based */
  }
  return end_phase(w);
}

/* Schedule 0: the diagonals s = n+1, n, ..., 4, then s = n+2, ..., 2n-2. */
static int walk_sched0(walk_t* w) {
  const int64_t n = w->n;
  for (int64_t s = n + 1; s >= 4; --s)
    if (!walk_diagonal(w, s)) return 0;
  for (int64_t s = n + 2; s <= 2 * n - 2; ++s)
    if (!walk_diagonal(w, s)) return 0;
  return 1;
}

/* Schedule 1: phase s holds the triplets with (i+j+k) mod n == s. */
static int walk_sched1(walk_t* w) {
  int64_t n = w->n;
  for (int64_t s = 0; s < n; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      unit_begin(w);
      for (int64_t j = i + 1; j < n; ++j) {
        int64_t k = ((s - i - j) % n + n) % n;   /* the one k of this phase */
        if (k > j)
          if (!walk_step(w, i, j, k)) return 0;
      }
    }
    if (!end_phase(w)) return 0;
  }
  return 1;
}

/* Schedule 2: tiled, block size B. */
static int walk_sched2(walk_t* w, int64_t B) {
  int64_t n = w->n;
  int64_t nb = (n + B - 1) / B;
  for (int64_t g = 0; g < nb; ++g) {
    for (int64_t I = 0; I < nb; ++I)
      for (int64_t J = I; J < nb; ++J)
        for (int64_t K = J; K < nb; ++K) {
          if ((I + J + K) % nb != g) continue;
          unit_begin(w);
          for (int64_t t = 0; t < B; ++t)
            for (int64_t a = 0; a < B; ++a)
              for (int64_t b = 0; b < B; ++b) {
                int64_t c = ((t - a - b) % B + B) % B;
                int64_t i = I * B + a, j = J * B + b, k = K * B + c;
                if (i < j && j < k && k < n)
                  if (!walk_step(w, i, j, k)) return 0;
              }
        }
    if (!end_phase(w)) return 0;
  }
  return 1;
}

static int walk_schedule(walk_t* w, int sched, int64_t B) {
  if (sched == 0) return walk_sched0(w);
  if (sched == 1) return walk_sched1(w);
  return walk_sched2(w, B);
}

/* Record the visiting order: rec[4*t .. 4*t+3] = (phase, i, j, k) for the
 * t-th triplet visited.  Returns the number of triplets in one sweep. */
int64_t ora_order(int64_t n, int sched, int64_t B, int32_t* rec, int64_t cap) {
  walk_t w = {n, 0.0, NULL, NULL, NULL, -1, rec, cap, 0, 0};
  walk_schedule(&w, sched, B);
  return w.count;
}

/* Number of phases of a schedule. */
int64_t ora_num_phases(int64_t n, int sched, int64_t B) {
  int32_t dummy[4];
  walk_t w = {n, 0.0, NULL, NULL, NULL, -1, dummy, 0, 0, 0};
  walk_schedule(&w, sched, B);
  return w.phase;
}

/* One sweep: every triplet in schedule order, then every pair.  With
 * max_rows >= 0 the sweep stops after that many rows (metric rows first, then
 * pair rows), for step-by-step checks.  Returns the rows visited. */
int64_t ora_sweep(int64_t n, int sched, int64_t B, double eps, const double* d,
                  const double* winv, double* x, double* f, double* ytri,
                  double* ypair, int64_t max_rows) {
  walk_t w = {n, eps, winv, x, ytri, max_rows, NULL, 0, 0, 0};
  int64_t rows = 0;
  if (!walk_schedule(&w, sched, B)) return max_rows;
  rows = max_rows >= 0 ? max_rows - w.rows_left : 3 * w.count;
  int64_t P = ch2(n);
  for (int64_t p = 0; p < P; ++p) {
    int r = 2;
    if (max_rows >= 0) {
      int64_t left = max_rows - rows;
      if (left <= 0) break;
      if (left < 2) r = (int)left;
    }
    visit_pair(eps, d[p], winv[p], &x[p], &f[p], &ypair[2 * p], r);
    rows += r;
  }
  return rows;
}

/* Largest violation of a metric row on the current x: max over triplets and
 * hypotenuse choices of max(0, x_h - x_a - x_b). */
double ora_max_violation(int64_t n, const double* x) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      for (int64_t k = j + 1; k < n; ++k) {
        double xij = x[pidx(n, i, j)], xik = x[pidx(n, i, k)], xjk = x[pidx(n, j, k)];
        double v0 = xij - xik - xjk, v1 = xik - xij - xjk, v2 = xjk - xij - xik;
        if (v0 > m) m = v0;
        if (v1 > m) m = v1;
        if (v2 > m) m = v2;
      }
  return m;
}

/* out[0] = LP objective sum w|x - d|   (Eq. mn1 at f = |x - d|)
 * out[1] = QP primal  sum w f + (eps/2) sum w (x^2 + f^2)   (Eq. qp)
 * out[2] = dual objective -b^T y - (eps/2) v^T W v with b^T y = sum d (y+ - y-)
 * out[3] = largest pair-row violation max(0, x - f - d, d - x - f)
 * out[4] = sum w f (the LP objective at the current slacks) */
void ora_objectives(int64_t n, double eps, const double* d, const double* w,
                    const double* x, const double* f, const double* ypair,
                    double* out) {
  int64_t P = ch2(n);
  double lp = 0.0, wf = 0.0, quad = 0.0, by = 0.0, pv = 0.0;
  for (int64_t p = 0; p < P; ++p) {
    lp += w[p] * fabs(x[p] - d[p]);
    wf += w[p] * f[p];
    quad += w[p] * (x[p] * x[p] + f[p] * f[p]);
    by += d[p] * (ypair[2 * p] - ypair[2 * p + 1]);
    double v0 = x[p] - f[p] - d[p], v1 = d[p] - x[p] - f[p];
    if (v0 > pv) pv = v0;
    if (v1 > pv) pv = v1;
  }
  out[0] = lp;
  out[1] = wf + 0.5 * eps * quad;
  out[2] = -by - 0.5 * eps * quad;
  out[3] = pv;
  out[4] = wf;
}

/* ---- l2 metric nearness (Sec. II-A, Eq. metricnear with p = 2) -----------
 * min sum_{i<j} w_ij (x_ij - d_ij)^2 subject to the metric rows only (for
 * n >= 3 they imply x >= 0).  As an instance of Eq. qp: v = x, W = diag(w),
 * eps = 1, c = -W d, b = 0, so Algorithm 1 starts from
 * x = -(1/eps) W^{-1} c = d with y = 0 and visits only metric rows; its dual
 * y is the multiplier of (1/2) sum w (x - d)^2. */

/* Algorithm 1's initialisation for this instance of Eq. qp. */
void ora_init_l2(int64_t n, const double* d, const double* w, double* winv, double* x,
                 double* ytri) {
  int64_t P = ch2(n), T = ch3(n);
  for (int64_t p = 0; p < P; ++p) {
    winv[p] = 1.0 / w[p];
    x[p] = d[p];                          /* -(1/eps) W^{-1} c = W^{-1} W d = d */
  }
  for (int64_t t = 0; t < 3 * T; ++t) ytri[t] = 0.0;
}

/* One sweep over the metric rows only (every triplet in schedule order, its
 * three rows as in ora_sweep); eps = 1.  Returns the rows visited. */
int64_t ora_sweep_l2(int64_t n, int sched, int64_t B, const double* winv, double* x,
                     double* ytri, int64_t max_rows) {
  walk_t w = {n, 1.0, winv, x, ytri, max_rows, NULL, 0, 0, 0};
  if (!walk_schedule(&w, sched, B)) return max_rows;
  return max_rows >= 0 ? max_rows - w.rows_left : 3 * w.count;
}

/* out[0] = objective of Eq. metricnear squared, sum w (x - d)^2
 * out[1] = QP primal (1/2) sum w (x - d)^2
 * out[2] = dual objective y^T A d - (1/2) y^T A W^{-1} A^T y, evaluated through
 *          A^T y = W (d - x) (the identity Algorithm 1 maintains):
 *          sum w d (d - x) - (1/2) sum w (d - x)^2
 * out[3] = out[4] = 0 (no pair rows) */
void ora_objectives_l2(int64_t n, const double* d, const double* w, const double* x,
                       double* out) {
  int64_t P = ch2(n);
  double sq = 0.0, dd = 0.0;
  for (int64_t p = 0; p < P; ++p) {
    double r = x[p] - d[p];
    sq += w[p] * (r * r);
    dd += w[p] * (d[p] * (d[p] - x[p]));
  }
  out[0] = sq;
  out[1] = 0.5 * sq;
  out[2] = dd - 0.5 * sq;
  out[3] = 0.0;
  out[4] = 0.0;
}

/* ---- threaded sweeps ----------------------------------------------------
 * The same sweep as ora_sweep / ora_sweep_l2, the units of each phase dealt
 * to nthr threads (see the header).  With max_phases > 0 only the first
 * max_phases phases of metric rows are visited (no pair rows), otherwise the
 * whole sweep.  Returns the rows visited, or -1 when the threads could not be
 * started (then nothing is visited). */

typedef struct {
  pthread_mutex_t mu;
  pthread_cond_t cv;
  int state;         /* 0: wait, 1: run, 2: give up */
} start_gate;

typedef struct {
  walk_t w;
  int sched;
  int64_t B;
  const double* d;   /* pair rows when pairs != 0 */
  double *f, *ypair;
  int pairs;
  start_gate* gate;
} thread_job;

static void* thread_main(void* arg) {
  thread_job* t = (thread_job*)arg;
  pthread_mutex_lock(&t->gate->mu);            /* wait until every thread exists */
  while (t->gate->state == 0) pthread_cond_wait(&t->gate->cv, &t->gate->mu);
  int run = t->gate->state == 1;
  pthread_mutex_unlock(&t->gate->mu);
  if (!run) return NULL;
  walk_schedule(&t->w, t->sched, t->B);
  if (t->pairs) {                              /* every pair is its own unit */
    int64_t P = ch2(t->w.n);
    for (int64_t p = t->w.tid; p < P; p += t->w.nthr)
      visit_pair(t->w.eps, t->d[p], t->w.winv[p], &t->w.x[p], &t->f[p], &t->ypair[2 * p], 2);
  }
  return NULL;
}

static int64_t sweep_threads(int64_t n, int sched, int64_t B, double eps, const double* d,
                             const double* winv, double* x, double* f, double* ytri,
                             double* ypair, int nthr, int64_t max_phases) {
  if (nthr < 1) nthr = 1;
  thread_job* jobs = (thread_job*)calloc((size_t)nthr, sizeof(thread_job));
  pthread_t* ids = (pthread_t*)calloc((size_t)nthr, sizeof(pthread_t));
  if (!jobs || !ids) {
    free(jobs);
    free(ids);
    return -1;
  }
  pthread_barrier_t bar;
  start_gate gate = {PTHREAD_MUTEX_INITIALIZER, PTHREAD_COND_INITIALIZER, 0};
  if (pthread_barrier_init(&bar, NULL, (unsigned)nthr) != 0) {
    free(jobs);
    free(ids);
    return -1;
  }
  for (int t = 0; t < nthr; ++t) {
    walk_t w = {n, eps, winv, x, ytri, -1, NULL, 0, 0, 0};
    w.nthr = nthr;
    w.tid = t;
    w.stop_after = max_phases > 0 ? max_phases : 0;
    w.bar = &bar;
    thread_job* j = &jobs[t];
    j->w = w;
    j->sched = sched;
    j->B = B;
    j->d = d;
    j->f = f;
    j->ypair = ypair;
    j->pairs = d != NULL && max_phases <= 0;
    j->gate = &gate;
  }
  int made = 1;                                /* thread 0 is this one */
  while (made < nthr && pthread_create(&ids[made], NULL, thread_main, &jobs[made]) == 0) ++made;
  pthread_mutex_lock(&gate.mu);
  gate.state = made == nthr ? 1 : 2;
  pthread_cond_broadcast(&gate.cv);
  pthread_mutex_unlock(&gate.mu);
  if (made == nthr) thread_main(&jobs[0]);
  for (int t = 1; t < made; ++t) pthread_join(ids[t], NULL);
  pthread_barrier_destroy(&bar);
  int64_t rows = -1;
  if (made == nthr) {
    rows = 0;
    for (int t = 0; t < nthr; ++t) rows += 3 * jobs[t].w.count;
    if (d != NULL && max_phases <= 0) rows += 2 * ch2(n);
  }
  free(jobs);
  free(ids);
  return rows;
}

int64_t ora_sweep_threads(int64_t n, int sched, int64_t B, double eps, const double* d,
                          const double* winv, double* x, double* f, double* ytri,
                          double* ypair, int nthr, int64_t max_phases) {
  return sweep_threads(n, sched, B, eps, d, winv, x, f, ytri, ypair, nthr, max_phases);
}

int64_t ora_sweep_l2_threads(int64_t n, int sched, int64_t B, const double* winv, double* x,
                             double* ytri, int nthr, int64_t max_phases) {
  return sweep_threads(n, sched, B, 1.0, NULL, winv, x, NULL, ytri, NULL, nthr, max_phases);
}

/* ---- threaded largest violation -------------------------------------------
 * ora_max_violation with the first indices i dealt round-robin to nthr
 * threads, each keeping its own maximum; a maximum does not depend on the
 * order it is taken in, so the result equals the serial one exactly. */
typedef struct {
  int64_t n;
  const double* x;
  int nthr, tid;
  double m;
} maxv_job;

static void* maxv_main(void* arg) {
  maxv_job* t = (maxv_job*)arg;
  const int64_t n = t->n;
  const double* x = t->x;
  double m = 0.0;
  for (int64_t i = t->tid; i < n; i += t->nthr)
    for (int64_t j = i + 1; j < n; ++j)
      for (int64_t k = j + 1; k < n; ++k) {
        double xij = x[pidx(n, i, j)], xik = x[pidx(n, i, k)], xjk = x[pidx(n, j, k)];
        double v0 = xij - xik - xjk, v1 = xik - xij - xjk, v2 = xjk - xij - xik;
        if (v0 > m) m = v0;
        if (v1 > m) m = v1;
        if (v2 > m) m = v2;
      }
  t->m = m;
  return NULL;
}

/* Returns -1 when the threads could not be started. */
double ora_max_violation_threads(int64_t n, const double* x, int nthr) {
  if (nthr < 1) nthr = 1;
  maxv_job* jobs = (maxv_job*)calloc((size_t)nthr, sizeof(maxv_job));
  pthread_t* ids = (pthread_t*)calloc((size_t)nthr, sizeof(pthread_t));
  if (!jobs || !ids) {
    free(jobs);
    free(ids);
    return -1.0;
  }
  for (int t = 0; t < nthr; ++t) {
    jobs[t].n = n;
    jobs[t].x = x;
    jobs[t].nthr = nthr;
    jobs[t].tid = t;
  }
  int made = 1, ok = 1;
  for (; made < nthr; ++made)
    if (pthread_create(&ids[made], NULL, maxv_main, &jobs[made]) != 0) {
      ok = 0;
      break;
    }
  maxv_main(&jobs[0]);
  for (int t = 1; t < made; ++t) pthread_join(ids[t], NULL);
  double m = 0.0;
  for (int t = 0; t < nthr && ok; ++t)
    if (jobs[t].m > m) m = jobs[t].m;
  free(jobs);
  free(ids);
  return ok ? m : -1.0;
}
