/*
 * Plain FP64 CPU oracle for the HNTL batched query path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it (through oracle/hntl_oracle.py). It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Every distance is formed in FP64 from the stored (FP32 / BF16 / FP8-decoded)
 * values in direct difference form, sum over t of (a_t - b_t)^2, in index
 * order. Selections are total orders on (distance, id) ascending; routing on
 * (distance, grain) ascending. OpenMP runs independent queries or points in
 * parallel; it never changes the arithmetic of one result.
 *
 * Paper passages followed (HNTL technical report):
 *   sec. 2.1 step 1 and sec. 2.3 item 1  - centroid routing to the nprobe nearest grains
 *   Eq. 1 (centering), Eq. 2 (projection), Eq. 3 (residual), Eq. 4 (squared residual norm)
 *   Eq. 6                                  - approximate distance ||z_q - z_i||^2 + r_q + r_i
 *   sec. 2.1 step 3, sec. 2.3 item 2       - scan of every row of each probed grain
 *   Table 1 "Pool C"                       - candidate pool of the C best approximate distances
 *   sec. 2.1 step 4, Mode B                - exact float L2 re-ranking of the pool to the top k
 *   sec. 1 / in-situ filters               - attribute predicate checked inside the scan loop
 * Grain partitioning is not specified by the paper; the oracle uses k-means++
 * seeding (Arthur and Vassilvitskii, 2007) followed by Lloyd iterations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double sq_diff_f32(const float* a, const float* b, int64_t d) {
  double s = 0.0;
  for (int64_t t = 0; t < d; ++t) {
    double x = (double)a[t] - (double)b[t];
    s += x * x;
  }
  return s;
}

static double sq_diff_f32_f64(const float* a, const double* b, int64_t d) {
  double s = 0.0;
  for (int64_t t = 0; t < d; ++t) {
    double x = (double)a[t] - b[t];
    s += x * x;
  }
  return s;
}

/* (dist, key) pair ordered lexicographically */
typedef struct {
  double dist;
  int64_t key;
} pair_t;

static int pair_less(pair_t a, pair_t b) {
  return a.dist < b.dist || (a.dist == b.dist && a.key < b.key);
}

static int pair_cmp(const void* pa, const void* pb) {
  pair_t a = *(const pair_t*)pa, b = *(const pair_t*)pb;
  if (pair_less(a, b)) return -1;
  if (pair_less(b, a)) return 1;
  return 0;
}

/* Bounded max-heap that keeps the `cap` smallest pairs seen. */
typedef struct {
  pair_t* v;
  int64_t n, cap;
} heap_t;

static void heap_sift_down(heap_t* h, int64_t i) {
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->n && pair_less(h->v[m], h->v[l])) m = l;
    if (r < h->n && pair_less(h->v[m], h->v[r])) m = r;
    if (m == i) return;
    pair_t t = h->v[i];
    h->v[i] = h->v[m];
    h->v[m] = t;
    i = m;
  }
}

static void heap_push(heap_t* h, pair_t p) {
  if (h->cap <= 0) return;
  if (h->n < h->cap) {
    int64_t i = h->n++;
    h->v[i] = p;
    while (i > 0) {
      int64_t par = (i - 1) / 2;
      if (!pair_less(h->v[par], h->v[i])) break;
      pair_t t = h->v[i];
      h->v[i] = h->v[par];
      h->v[par] = t;
      i = par;
    }
  } else if (pair_less(p, h->v[0])) {
    h->v[0] = p;
    heap_sift_down(h, 0);
  }
}

/* ------------------------------------------------------------------ */
/* brute force exact kNN                                               */
/* ------------------------------------------------------------------ */

/* Exact k nearest rows of X [n x d] to each query (FP64 direct form), sorted
 * by (dist, id). Also returns the (k+1)-th distance (or +inf) so callers can
 * apply a gap rule. When ranges != NULL, only rows whose attr lies in the
 * query's inclusive [lo, hi] range are considered. */
void or_bruteforce(const float* X, int64_t n, int64_t d, const float* Q, int64_t nq, int64_t k,
                   const int64_t* attr, const int64_t* ranges, int64_t* out_id, double* out_d,
                   double* out_next) {
#pragma omp parallel
  {
    heap_t h;
    h.cap = k + 1;
    h.v = (pair_t*)malloc(sizeof(pair_t) * (size_t)(k + 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t qi = 0; qi < nq; ++qi) {
      const float* q = Q + qi * d;
      h.n = 0;
      for (int64_t i = 0; i < n; ++i) {
        if (ranges) {
          int64_t a = attr[i];
          if (a < ranges[2 * qi] || a > ranges[2 * qi + 1]) continue;
        }
        pair_t p = {sq_diff_f32(q, X + i * d, d), i};
        heap_push(&h, p);
      }
      qsort(h.v, (size_t)h.n, sizeof(pair_t), pair_cmp);
      for (int64_t j = 0; j < k; ++j) {
        out_id[qi * k + j] = j < h.n ? h.v[j].key : -1;
        out_d[qi * k + j] = j < h.n ? h.v[j].dist : INFINITY;
      }
      out_next[qi] = k < h.n ? h.v[k].dist : INFINITY;
    }
    free(h.v);
  }
}

/* ------------------------------------------------------------------ */
/* grain partitioning: k-means++ seeding and Lloyd iterations          */
/* ------------------------------------------------------------------ */

/* k-means++ seeding. The first centre is row floor(u[0] * n); centre c > 0 is
 * the smallest row i whose running sum of D(x)^2 exceeds u[c] * total, where
 * D(x) is the distance from x to its nearest chosen centre. The uniforms u
 * are inputs. Returns the chosen row indices. */
void or_kmeanspp(const float* X, int64_t n, int64_t d, int64_t G, const double* u, int64_t* chosen) {
  double* dmin = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t first = (int64_t)floor(u[0] * (double)n);
  if (first >= n) first = n - 1;
  chosen[0] = first;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) dmin[i] = sq_diff_f32(X + i * d, X + first * d, d);
  for (int64_t c = 1; c < G; ++c) {
    double total = 0.0;
    for (int64_t i = 0; i < n; ++i) total += dmin[i];
    int64_t pick = n - 1;
    if (total > 0.0) {
      double target = u[c] * total, run = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        run += dmin[i];
        if (run > target) {
          pick = i;
          break;
        }
      }
    } else {
      pick = (int64_t)floor(u[c] * (double)n);
      if (pick >= n) pick = n - 1;
    }
    chosen[c] = pick;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double dd = sq_diff_f32(X + i * d, X + pick * d, d);
      if (dd < dmin[i]) dmin[i] = dd;
    }
  }
  free(dmin);
}

/* Nearest centre of every row (ties to the lower grain id); FP64 centres. */
void or_assign(const float* X, int64_t n, int64_t d, const double* M, int64_t G, int32_t* assign,
               double* dist) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double best = INFINITY;
    int32_t bg = 0;
    for (int64_t g = 0; g < G; ++g) {
      double dd = sq_diff_f32_f64(X + i * d, M + g * d, d);
      if (dd < best) {
        best = dd;
        bg = (int32_t)g;
      }
    }
    assign[i] = bg;
    if (dist) dist[i] = best;
  }
}

/* FP64 mean of each grain's members. Returns the number of empty grains;
 * empty grains keep their previous centre. */
int64_t or_means(const float* X, int64_t n, int64_t d, const int32_t* assign, int64_t G, double* M,
                 int64_t* count) {
  double* acc = (double*)calloc((size_t)(G * d), sizeof(double));
  for (int64_t g = 0; g < G; ++g) count[g] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = assign[i];
    count[g]++;
    for (int64_t t = 0; t < d; ++t) acc[g * d + t] += (double)X[i * d + t];
  }
  int64_t empty = 0;
  for (int64_t g = 0; g < G; ++g) {
    if (count[g] == 0) {
      empty++;
      continue;
    }
    for (int64_t t = 0; t < d; ++t) M[g * d + t] = acc[g * d + t] / (double)count[g];
  }
  free(acc);
  return empty;
}

/* Lloyd iterations from the centres in M (in/out). Each iteration assigns
 * every row to its nearest centre, stops if no assignment changed, and
 * otherwise moves each centre to the FP64 mean of its members. A grain left
 * empty is re-seeded with the row farthest from its own centre (ties to the
 * lower row index; each such row is used once). Returns the iterations run. */
int64_t or_lloyd(const float* X, int64_t n, int64_t d, int64_t G, double* M, int64_t max_iter,
                 int32_t* assign) {
  double* dist = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* prev = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* count = (int64_t*)malloc(sizeof(int64_t) * (size_t)G);
  char* used = (char*)calloc((size_t)n, 1);
  int64_t it = 0;
  for (int64_t i = 0; i < n; ++i) prev[i] = -1;
  for (it = 0; it < max_iter; ++it) {
    or_assign(X, n, d, M, G, assign, dist);
    int64_t changed = 0;
    for (int64_t i = 0; i < n; ++i) changed += assign[i] != prev[i];
    if (changed == 0) break;
    memcpy(prev, assign, sizeof(int32_t) * (size_t)n);
    or_means(X, n, d, assign, G, M, count);
    memset(used, 0, (size_t)n);
    for (int64_t g = 0; g < G; ++g) {
      if (count[g] != 0) continue;
      int64_t far = -1;
      for (int64_t i = 0; i < n; ++i) {
        if (used[i]) continue;
        if (far < 0 || dist[i] > dist[far]) far = i;
      }
      if (far < 0) break;
      used[far] = 1;
      for (int64_t t = 0; t < d; ++t) M[g * d + t] = (double)X[far * d + t];
    }
  }
  free(dist);
  free(prev);
  free(count);
  free(used);
  return it;
}

/* ------------------------------------------------------------------ */
/* capacity-bounded grains: deferred acceptance                        */
/* ------------------------------------------------------------------ */

/* Grains of at most cap rows (the paper leaves the partition open, sec. 2.2;
 * bounded grain sizes are this build's reading for balanced work). Deferred
 * acceptance with rows proposing (Gale and Shapley, 1962): every row ranks
 * the centres by (squared distance, grain) and every centre ranks rows by
 * (squared distance, row); a free row proposes to its best centre that has
 * not yet refused it; a centre holding cap rows keeps the cap it ranks best
 * among them and the proposer and refuses the other. The result is the
 * row-optimal stable assignment, which does not depend on the order in which
 * free rows propose. Requires cap * G >= n. Distances in FP64 (FP64 centres). */
typedef struct {
  double dist;
  int64_t row;
} held_t;

static int held_worse(held_t a, held_t b) { /* a ranks below b for the centre */
  return a.dist > b.dist || (a.dist == b.dist && a.row > b.row);
}

void or_balanced_assign(const float* X, int64_t n, int64_t d, const double* M, int64_t G, int64_t cap,
                        int32_t* assign) {
  int32_t* pref = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * G));
  double* dist = (double*)malloc(sizeof(double) * (size_t)(n * G));
#pragma omp parallel
  {
    pair_t* tmp = (pair_t*)malloc(sizeof(pair_t) * (size_t)G);
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t g = 0; g < G; ++g) {
        tmp[g].dist = sq_diff_f32_f64(X + i * d, M + g * d, d);
        tmp[g].key = g;
        dist[i * G + g] = tmp[g].dist;
      }
      qsort(tmp, (size_t)G, sizeof(pair_t), pair_cmp);
      for (int64_t g = 0; g < G; ++g) pref[i * G + g] = (int32_t)tmp[g].key;
    }
    free(tmp);
  }
  /* per centre a max-heap (worst held row on top) of at most cap rows */
  held_t* heap = (held_t*)malloc(sizeof(held_t) * (size_t)(G * cap));
  int64_t* hn = (int64_t*)calloc((size_t)G, sizeof(int64_t));
  int64_t* next = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t top = 0;
  for (int64_t i = n - 1; i >= 0; --i) stack[top++] = i;
  while (top > 0) {
    const int64_t i = stack[--top];
    if (next[i] >= G) continue; /* cannot happen when cap * G >= n */
    const int64_t g = pref[i * G + next[i]++];
    held_t* h = heap + g * cap;
    held_t me = {dist[i * G + g], i};
    if (hn[g] < cap) {
      int64_t k = hn[g]++;
      h[k] = me;
      while (k > 0) {
        const int64_t p = (k - 1) / 2;
        if (!held_worse(h[k], h[p])) break;
        held_t t = h[k];
        h[k] = h[p];
        h[p] = t;
        k = p;
      }
      assign[i] = (int32_t)g;
    } else if (held_worse(h[0], me)) {
      const int64_t out = h[0].row;
      h[0] = me;
      int64_t k = 0;
      for (;;) {
        const int64_t l = 2 * k + 1, r = l + 1;
        int64_t m = k;
        if (l < cap && held_worse(h[l], h[m])) m = l;
        if (r < cap && held_worse(h[r], h[m])) m = r;
        if (m == k) break;
        held_t t = h[k];
        h[k] = h[m];
        h[m] = t;
        k = m;
      }
      assign[i] = (int32_t)g;
      assign[out] = -1;
      stack[top++] = out;
    } else {
      stack[top++] = i; /* refused: propose to the next centre */
    }
  }
  free(pref);
  free(dist);
  free(heap);
  free(hn);
  free(next);
  free(stack);
}

/* ------------------------------------------------------------------ */
/* Mode B search                                                       */
/* ------------------------------------------------------------------ */

/*
 * Index, in grain order (the layout the oracle writes):
 *   M [G x d] f32 centres, U [G x r x d] f32 bases (rows orthonormal),
 *   grain_off [G+1] row offsets, ids [N] original ids, Z [N x r] coordinates
 *   (as stored: FP32, or FP8 codes already decoded and scaled by the caller),
 *   rho [N] residual norms; X [N x d] raw rows in original id order
 *   (FP32, or BF16 widened by the caller); attr [N] in original id order.
 *
 * Qp (may be NULL) is the query as routed and projected (the precision form
 * rounds it to BF16); the rerank always uses Q.
 *
 * probe_in (may be NULL): nq x nprobe grain ids that replace step 1 (a
 * router's probes); each is used in the given order with its distance
 * ||q - mu_g||^2, and the (nprobe+1)-th routing distance is reported as +inf
 * (there is no routing boundary).
 *
 * Per query:
 *   1. routing: ||q - mu_g||^2 for every g, the nprobe smallest by (dist, g);
 *   2. per probed grain: v' = q - mu_g, z_q = U_g v', rho_q = ||v' - U_g^T z_q||^2;
 *   3. per row i of the grain (passing the filter): D = ||z_q - z_i||^2 + rho_q + rho_i;
 *   4. pool: the C smallest (D, id);
 *   5. rerank: exact ||q - x_id||^2 of the pool, the k smallest (dist, id);
 *      with Xl (may be NULL; [N x d], the rows' second BF16 parts widened, in
 *      original id order) the kref smallest (dist, id) of that rerank are
 *      ranked again by ||q - (x_id + xl_id)||^2 and the k smallest kept.
 * Outputs: probe [nq x nprobe] grain ids, probe_d [nq x (nprobe+1)] routing
 * distances (the (nprobe+1)-th, or +inf, last); cand_id [nq x C] (0xFFFFFFFF
 * pad), cand_d [nq x (C+1)] (+inf pad; the (C+1)-th last); out_id [nq x k]
 * (-1 pad), out_d [nq x (k+1)] (+inf pad; the (k+1)-th pool distance last).
 */
void or_search(const float* M, const float* U, int64_t G, int64_t d, int64_t r, const int64_t* grain_off,
               const uint32_t* ids, const float* Z, const float* rho, const float* X, const int64_t* attr,
               const float* Q, const float* Qp, int64_t nq, int64_t k, int64_t C, int64_t nprobe,
               const int64_t* ranges, int32_t* probe, double* probe_d, uint32_t* cand_id, double* cand_d,
               int64_t* out_id, double* out_d, int64_t mode, const int64_t* pos_of_id,
               const int32_t* grain_of_pos, const double* qdelta, const double* qdres,
               const int32_t* probe_in, const int16_t* Zc, int64_t i16_flags, const int16_t* qc_in,
               const int32_t* qr_in, const float* pz_in, const float* prho_in, const float* Xl, int64_t kref) {
#pragma omp parallel
  {
    pair_t* route = (pair_t*)malloc(sizeof(pair_t) * (size_t)G);
    double* v = (double*)malloc(sizeof(double) * (size_t)d);
    double* e = (double*)malloc(sizeof(double) * (size_t)d);
    double* zq = (double*)malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    int64_t* qc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(r > 0 ? r : 1));
    heap_t pool;
    pool.cap = C + 1;
    pool.v = (pair_t*)malloc(sizeof(pair_t) * (size_t)(C + 1));
    pair_t* rr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(C + 1));
    double* xh = (double*)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
      const float* q = Q + qi * d;
      const float* qp = Qp ? Qp + qi * d : q; /* query as routed and projected */
      /* 1. centroid routing, or the given probes */
      if (probe_in) {
        for (int64_t p = 0; p < nprobe; ++p) {
          const int64_t g = probe_in[qi * nprobe + p];
          route[p].dist = sq_diff_f32(qp, M + g * d, d);
          route[p].key = g;
        }
      } else {
        for (int64_t g = 0; g < G; ++g) {
          route[g].dist = sq_diff_f32(qp, M + g * d, d);
          route[g].key = g;
        }
        qsort(route, (size_t)G, sizeof(pair_t), pair_cmp);
      }
      for (int64_t p = 0; p < nprobe; ++p) {
        probe[qi * nprobe + p] = (int32_t)route[p].key;
        probe_d[qi * (nprobe + 1) + p] = route[p].dist;
      }
      probe_d[qi * (nprobe + 1) + nprobe] = (nprobe < G && !probe_in) ? route[nprobe].dist : INFINITY;
      /* 2-4. projection, scan, pool */
      pool.n = 0;
      for (int64_t p = 0; p < nprobe; ++p) {
        int64_t g = route[p].key;
        const float* mu = M + g * d;
        const float* Ug = U + g * r * d;
        for (int64_t t = 0; t < d; ++t) v[t] = (double)qp[t] - (double)mu[t];
        for (int64_t j = 0; j < r; ++j) {
          double s = 0.0;
          for (int64_t t = 0; t < d; ++t) s += (double)Ug[j * d + t] * v[t];
          zq[j] = s;
        }
        for (int64_t t = 0; t < d; ++t) e[t] = v[t];
        for (int64_t j = 0; j < r; ++j)
          for (int64_t t = 0; t < d; ++t) e[t] -= zq[j] * (double)Ug[j * d + t];
        double rho_q = 0.0;
        for (int64_t t = 0; t < d; ++t) rho_q += e[t] * e[t];
        if (pz_in) {
          /* the projection step taken elsewhere (pz_in [nq][nprobe][r], prho_in
           * [nq][nprobe]): the scan, pool and rerank run on those values */
          for (int64_t j = 0; j < r; ++j) zq[j] = (double)pz_in[(qi * nprobe + p) * r + j];
          rho_q = (double)prho_in[qi * nprobe + p];
        }
        float dl = 0.f, rq16 = 0.f;
        if (qdelta) {
          /* 16-bit form (Eq. 5): the query's coordinates and residual norm are
           * put on the grain's grids in IEEE single precision, code =
           * rint(fl32(fl32(value) / step)) (round half to even). A coordinate
           * code beyond the signed 16-bit range saturates at +-32767 and is
           * counted; the residual code is clipped at the unsigned 16-bit
           * maximum 65535. The grain is left out when more than a quarter of
           * the coordinates saturate (Quantization Envelope Filter, sec. 2.3);
           * with i16_flags bit 0 (the build's own option, not the paper's) it
           * is also left out when the residual code would exceed 65535.
           * Given codes (qc_in, qr_in: the same quantisation taken elsewhere;
           * qr_in < 0 marks a pair left out) replace this step. */
          dl = (float)qdelta[g];
          const float dr = (float)qdres[g];
          float tr;
          if (qc_in) {
            const int64_t base = (qi * nprobe + p) * r;
            if (qr_in[qi * nprobe + p] < 0) continue;
            for (int64_t j = 0; j < r; ++j) qc[j] = qc_in[base + j];
            tr = (float)qr_in[qi * nprobe + p];
          } else {
            int64_t sat = 0;
            for (int64_t j = 0; j < r; ++j) {
              float t = rintf((float)zq[j] / dl);
              if (fabsf(t) > 32767.f) {
                ++sat;
                t = t > 0 ? 32767.f : -32767.f;
              }
              qc[j] = (int64_t)t;
            }
            if (4 * sat > r) continue;
            tr = rintf((float)rho_q / dr);
            if (tr > 65535.f) {
              if (i16_flags & 1) continue;
              tr = 65535.f;
            }
          }
          rq16 = tr * dr; /* the query's residual on the grain's grid, fl32 */
        }
        for (int64_t i = grain_off[g]; i < grain_off[g + 1]; ++i) {
          uint32_t id = ids[i];
          if (ranges) {
            int64_t a = attr[id];
            if (a < ranges[2 * qi] || a > ranges[2 * qi + 1]) continue;
          }
          double dist;
          if (qdelta) {
            /* Eq. 6 on the 16-bit representations: the exact integer
             * S = sum_j (zq_j - z_ij)^2 of the codes, scaled back in IEEE
             * single precision as fl32(fl32(delta^2) * fl32(S)) plus
             * fl32(rho_q + rho_i) of the grid residuals */
            int64_t S = 0;
            for (int64_t j = 0; j < r; ++j) {
              const int64_t t = qc[j] - (int64_t)Zc[i * r + j];
              S += t * t;
            }
            const float dl2 = dl * dl;
            const float a = dl2 * (float)S;
            const float b = rq16 + rho[i];
            dist = (double)(float)(a + b);
          } else {
            double s = 0.0;
            for (int64_t j = 0; j < r; ++j) {
              double t = zq[j] - (double)Z[i * r + j];
              s += t * t;
            }
            dist = s + rho_q + (double)rho[i];
          }
          pair_t cand = {dist, (int64_t)id};
          heap_push(&pool, cand);
        }
      }
      qsort(pool.v, (size_t)pool.n, sizeof(pair_t), pair_cmp);
      for (int64_t j = 0; j < C; ++j) {
        cand_id[qi * C + j] = j < pool.n ? (uint32_t)pool.v[j].key : 0xFFFFFFFFu;
        cand_d[qi * (C + 1) + j] = j < pool.n ? pool.v[j].dist : INFINITY;
      }
      cand_d[qi * (C + 1) + C] = C < pool.n ? pool.v[C].dist : INFINITY;
      /* 5. rerank of the pool: Mode B, exact L2 to the raw row (sec. 2.1 step 4);
       * Mode A, L2 to the row's reconstruction mu_g + W_g z_i from its grain's
       * centre and basis and its stored coordinates, against the query as routed
       * and projected (sec. 2.1 step 4, sec. 1) */
      int64_t m = pool.n < C ? pool.n : C;
      for (int64_t j = 0; j < m; ++j) {
        rr[j].key = pool.v[j].key;
        if (mode == 1) {
          const int64_t i = pos_of_id[rr[j].key];
          const int64_t g = grain_of_pos[i];
          const float* mu = M + g * d;
          const float* Ug = U + g * r * d;
          for (int64_t t = 0; t < d; ++t) xh[t] = (double)mu[t];
          for (int64_t a = 0; a < r; ++a)
            for (int64_t t = 0; t < d; ++t) xh[t] += (double)Ug[a * d + t] * (double)Z[i * r + a];
          double s = 0.0;
          for (int64_t t = 0; t < d; ++t) {
            const double df = (double)qp[t] - xh[t];
            s += df * df;
          }
          rr[j].dist = s;
        } else {
          rr[j].dist = sq_diff_f32(q, X + rr[j].key * d, d);
        }
      }
      qsort(rr, (size_t)m, sizeof(pair_t), pair_cmp);
      if (Xl && mode == 0) {
        /* second stage: the first kref again, on both parts of each row */
        m = m < kref ? m : kref;
        for (int64_t j = 0; j < m; ++j) {
          const float* x = X + rr[j].key * d;
          const float* xl = Xl + rr[j].key * d;
          double s = 0.0;
          for (int64_t t = 0; t < d; ++t) {
            const double df = (double)q[t] - ((double)x[t] + (double)xl[t]);
            s += df * df;
          }
          rr[j].dist = s;
        }
        qsort(rr, (size_t)m, sizeof(pair_t), pair_cmp);
      }
      for (int64_t j = 0; j < k; ++j) {
        out_id[qi * k + j] = j < m ? rr[j].key : -1;
        out_d[qi * (k + 1) + j] = j < m ? rr[j].dist : INFINITY;
      }
      out_d[qi * (k + 1) + k] = k < m ? rr[k].dist : INFINITY;
    }
    free(route);
    free(v);
    free(e);
    free(zq);
    free(qc);
    free(pool.v);
    free(rr);
    free(xh);
  }
}

/* Number of OpenMP threads the oracle runs with. */
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
