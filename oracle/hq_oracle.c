/*
 * hq_oracle.c -- CPU oracle for the spatial hypercube queue with heterogeneous
 * service rates (Hua, Luo, Swersey & Wen, "A Geometrically Convergent Solution to
 * Spatial Hypercube Queueing Models", arXiv 2603.03019).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Everything is IEEE double (FP64) except the birth-death products, which use
 * long double.  States live in natural binary order ("y-order", Section 4.2,
 * y(B_m) = sum_i b_{m,i} 2^{i-1}): bit i of the index is unit i (0-based) busy.
 *
 * What it computes, in the paper's order and notation:
 *   - transition rates lambda_{lm} by the first-idle-unit rule of Eq. (3)
 *     (the reading that the product runs over the units ranked strictly before
 *     unit i_{lm}, all busy, with i_{lm} idle in B_l; the sentence after Eq. (3)
 *     states exactly this);
 *   - Algorithm 1 (Conditional Probability Update): initial p_n = 1/C(N,n),
 *     outer sweeps k over layers n = 1..N-1 in ascending order, and in each layer
 *     the inner loop r of Eq. (12)/(14) run until the change is <= delta, then
 *     Eq. (13).  The inner loop is run literally (do-while); the two inflow sums
 *     of Eq. (12) do not depend on r, so they are formed once per layer;
 *   - p(n) from Eq. (10), Proposition 2 (finite buffer C) and the Remark
 *     (infinite buffer), by plain products;
 *   - P{B_m} = p(w(B_m)) p_{w(B_m)}(B_m), per-unit utilisation, the response
 *     pattern (probability a call from node j is served by unit i), workload,
 *     and the global balance residual of Eq. (1).
 *
 * Threads: built plainly this file is single-threaded.  Built with -fopenmp, the
 * loops over the states of one layer (and over states or nodes in the outputs) run
 * on all host threads, which is the within-layer parallelism of Algorithm 2 (states
 * of a layer are independent given layers n-1 and n+1); only the order in which the
 * sums and maxima over a layer are added changes.
 *
 * Parity pins for this file (tests, CPU only): dense direct solve of Eq. (1)-(2),
 * Erlang-B / M/M/N/N+C / Erlang-C closed forms in the homogeneous case, an N=2
 * hand-derived closed form, the single-unit-first-choice M/M/1/1 marginal, the
 * normalisation property of Lemma 1 and the contraction bound of the Corollary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LOSS 0
#define OR_FINITE 1
#define OR_INFINITE 2

typedef struct {
  int N, J, mode, C;
  double lam;     /* lambda = sum_j lambda_j (region-wide arrival rate) */
  double nu_sum;  /* sum_i nu_i = mu(N) */
  double* lam_j;  /* J: per-node arrival rate lambda f_j */
  double* nu;     /* N: service rates nu_i */
  int32_t* pref;  /* J x N: pref[j*N + h] = zeta_j(h+1), 0-based unit ids */
  int64_t S;      /* 2^N */
  int64_t* off;   /* N+2: layer n holds lst[off[n] .. off[n+1]) */
  uint32_t* lst;  /* S: states grouped by layer, ascending y inside a layer */
  int32_t* pos;   /* S: pos[y] = index of y inside its layer */
  double* mu_m;   /* S (y-indexed): mu_m = sum_{i busy} nu_i */
  double** up;    /* up[n]: rows of layer n, up[n][k*N+u] = rate B -> B+u */
  double* p;      /* S (y-indexed): conditional probability p_{w(B)}(B) */
  double* lam_n;  /* N+1: lambda(n) */
  double* mu_n;   /* N+1: mu(n) */
  double* work;   /* scratch, size of the largest layer */
  double* upsum;  /* scratch: per-state up-inflow sum of Eq. (12) */
  double* dnsum;  /* scratch: per-state down-inflow sum of Eq. (12) */
  long inner_total;
} or_ctx;

static int popc(uint64_t x) {
  int c = 0;
  while (x) {
    x &= x - 1;
    c++;
  }
  return c;
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
  return floor(r + 0.5);
}

/* lambda_m of Section 2.1: every arrival leaves a non-full state; in the loss
 * system the all-busy state has no upward transition.  In the queued systems an
 * arrival to the all-busy state joins the queue, so lambda_m = lambda there. */
static double lambda_m(const or_ctx* c, uint64_t B) {
  if (B == (uint64_t)(c->S - 1)) return c->mode == OR_LOSS ? 0.0 : c->lam;
  return c->lam;
}

/* First idle unit of node j's preference list in state B (-1 if all busy):
 * the unit to which Eq. (3) sends a call from node j. */
int or_first_idle(int N, const int32_t* pref_row, uint64_t B) {
  for (int h = 0; h < N; h++) {
    int u = pref_row[h];
    if (!((B >> u) & 1ULL)) return u;
  }
  return -1;
}

/* lambda_{lm} for l = src, m = src + unit u (u idle in src): Eq. (3). */
double or_dispatch_rate(int N, int J, const double* lam_j, const int32_t* pref,
                        uint64_t src, int u) {
  if ((src >> u) & 1ULL) return 0.0;
  double s = 0.0;
  for (int j = 0; j < J; j++)
    if (or_first_idle(N, pref + (size_t)j * N, src) == u) s += lam_j[j];
  return s;
}

void or_dispatch_rates_batch(int N, int J, const double* lam_j, const int32_t* pref,
                             int64_t count, const uint64_t* src, const int32_t* u,
                             double* out) {
  for (int64_t k = 0; k < count; k++)
    out[k] = or_dispatch_rate(N, J, lam_j, pref, src[k], u[k]);
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->lam_j);
  free(c->nu);
  free(c->pref);
  free(c->off);
  free(c->lst);
  free(c->pos);
  free(c->mu_m);
  if (c->up) {
    for (int n = 0; n <= c->N; n++) free(c->up[n]);
    free(c->up);
  }
  free(c->p);
  free(c->lam_n);
  free(c->mu_n);
  free(c->work);
  free(c->upsum);
  free(c->dnsum);
  free(c);
}

/* Build the instance.  Returns NULL on invalid input. */
or_ctx* or_create(int N, int J, const double* lam_j, const double* nu,
                  const int32_t* pref, int mode, int C) {
  if (N < 1 || N > 30 || J < 1) return NULL;
  if (mode < 0 || mode > 2 || (mode == OR_FINITE && C < 1)) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->N = N;
  c->J = J;
  c->mode = mode;
  c->C = mode == OR_FINITE ? C : 0;
  c->S = (int64_t)1 << N;
  c->lam_j = (double*)malloc(sizeof(double) * J);
  c->nu = (double*)malloc(sizeof(double) * N);
  c->pref = (int32_t*)malloc(sizeof(int32_t) * (size_t)J * N);
  memcpy(c->lam_j, lam_j, sizeof(double) * J);
  memcpy(c->nu, nu, sizeof(double) * N);
  memcpy(c->pref, pref, sizeof(int32_t) * (size_t)J * N);
  c->lam = 0.0;
  for (int j = 0; j < J; j++) c->lam += lam_j[j];
  c->nu_sum = 0.0;
  for (int i = 0; i < N; i++) c->nu_sum += nu[i];
  int bad = c->lam <= 0.0;
  for (int i = 0; i < N; i++) bad |= !(nu[i] > 0.0);
  for (int j = 0; j < J && !bad; j++) {
    bad |= lam_j[j] < 0.0;
    uint64_t seen = 0;
    for (int h = 0; h < N; h++) {
      int u = pref[(size_t)j * N + h];
      if (u < 0 || u >= N || ((seen >> u) & 1ULL)) bad = 1;
      else seen |= 1ULL << u;
    }
  }
  if (mode == OR_INFINITE && c->lam >= c->nu_sum) bad = 1;
  if (bad) {
    or_destroy(c);
    return NULL;
  }
  /* layers C_n (Section 2.2), states in ascending y */
  c->off = (int64_t*)calloc(N + 2, sizeof(int64_t));
  for (int n = 0; n <= N; n++) c->off[n + 1] = c->off[n] + (int64_t)binom(N, n);
  c->lst = (uint32_t*)malloc(sizeof(uint32_t) * c->S);
  c->pos = (int32_t*)malloc(sizeof(int32_t) * c->S);
  int64_t* fill = (int64_t*)calloc(N + 1, sizeof(int64_t));
  for (int64_t y = 0; y < c->S; y++) {
    int n = popc((uint64_t)y);
    c->pos[y] = (int32_t)fill[n];
    c->lst[c->off[n] + fill[n]] = (uint32_t)y;
    fill[n]++;
  }
  free(fill);
  c->mu_m = (double*)malloc(sizeof(double) * c->S);
  for (int64_t y = 0; y < c->S; y++) {
    double s = 0.0;
    for (int i = 0; i < N; i++)
      if ((y >> i) & 1) s += nu[i];
    c->mu_m[y] = s;
  }
  c->up = (double**)calloc(N + 1, sizeof(double*));
  c->p = (double*)calloc(c->S, sizeof(double));
  c->lam_n = (double*)calloc(N + 1, sizeof(double));
  c->mu_n = (double*)calloc(N + 1, sizeof(double));
  int64_t maxl = 0;
  for (int n = 0; n <= N; n++)
    if (c->off[n + 1] - c->off[n] > maxl) maxl = c->off[n + 1] - c->off[n];
  c->work = (double*)malloc(sizeof(double) * maxl);
  c->upsum = (double*)malloc(sizeof(double) * maxl);
  c->dnsum = (double*)malloc(sizeof(double) * maxl);
  return c;
}

int64_t or_layer_size(const or_ctx* c, int n) { return c->off[n + 1] - c->off[n]; }
void or_layer_states(const or_ctx* c, int n, uint32_t* out) {
  memcpy(out, c->lst + c->off[n], sizeof(uint32_t) * or_layer_size(c, n));
}

/* Upward transition rates out of every state of source layers n_lo..n_hi:
 * for each state B and node j, the call goes to the first idle unit u on
 * zeta_j and adds lambda f_j to the rate B -> B+u (Eq. 3). */
int or_build_up(or_ctx* c, int n_lo, int n_hi) {
  int N = c->N;
  if (n_lo < 0) n_lo = 0;
  if (n_hi > N - 1) n_hi = N - 1;
  for (int n = n_lo; n <= n_hi; n++) {
    int64_t L = or_layer_size(c, n);
    free(c->up[n]);
    c->up[n] = (double*)calloc((size_t)L * N, sizeof(double));
    if (!c->up[n]) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L; k++) {
      uint64_t B = c->lst[c->off[n] + k];
      for (int j = 0; j < c->J; j++) {
        int u = or_first_idle(N, c->pref + (size_t)j * N, B);
        if (u >= 0) c->up[n][k * N + u] += c->lam_j[j];
      }
    }
  }
  return 0;
}

/* rate of the upward transition (B - u) -> B, read from the stored rows */
static double up_rate_into(const or_ctx* c, uint64_t B, int u) {
  uint64_t src = B & ~(1ULL << u);
  int n = popc(src);
  return c->up[n][(int64_t)c->pos[src] * c->N + u];
}

void or_get_up_rows(const or_ctx* c, int n, double* out) {
  memcpy(out, c->up[n], sizeof(double) * or_layer_size(c, n) * c->N);
}

/* Eq. (6)-(7): lambda(n) = sum_m p_n(B_m) lambda_m, mu(n) = sum_m p_n(B_m) mu_m */
void or_layer_rates(or_ctx* c, double* lam_n, double* mu_n) {
  for (int n = 0; n <= c->N; n++) {
    double sl = 0.0, sm = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sl, sm)
    for (int64_t k = c->off[n]; k < c->off[n + 1]; k++) {
      uint64_t B = c->lst[k];
      sl += c->p[B] * lambda_m(c, B);
      sm += c->p[B] * c->mu_m[B];
    }
    lam_n[n] = sl;
    mu_n[n] = sm;
  }
}

/* Algorithm 1, step 2: p_n^1(B_m) = 1/C(N,n), or a caller-given start
 * (conditional probabilities in y-order).  lambda(n), mu(n) follow Eq. (6)-(7). */
void or_init(or_ctx* c, const double* p0) {
  for (int n = 0; n <= c->N; n++) {
    double v = 1.0 / (double)or_layer_size(c, n);
#pragma omp parallel for schedule(static)
    for (int64_t k = c->off[n]; k < c->off[n + 1]; k++) {
      uint64_t B = c->lst[k];
      c->p[B] = p0 ? p0[B] : v;
    }
  }
  or_layer_rates(c, c->lam_n, c->mu_n);
  c->inner_total = 0;
}

void or_set_p(or_ctx* c, const double* p) { memcpy(c->p, p, sizeof(double) * c->S); }
void or_get_p(const or_ctx* c, double* out) { memcpy(out, c->p, sizeof(double) * c->S); }
void or_get_layer_scalars(const or_ctx* c, double* lam_n, double* mu_n) {
  memcpy(lam_n, c->lam_n, sizeof(double) * (c->N + 1));
  memcpy(mu_n, c->mu_n, sizeof(double) * (c->N + 1));
}
long or_inner_total(const or_ctx* c) { return c->inner_total; }

/* One layer of one outer iteration k of Algorithm 1 (Eq. 12-14), in place.
 * Layer n-1 already holds iteration k (updated earlier in this sweep); layer n+1
 * still holds iteration k-1.  lam_n[n-1] is lambda^k(n-1); lam_n[n] and
 * mu_n[n+1] are still lambda^{k-1}(n) and mu^{k-1}(n+1); mu_n[n] starts as
 * mu^{k,0}(n) = mu^{k-1}(n).  Returns the number of inner updates r; writes
 * max_m |p_n^k - p_n^{k-1}| and sum_m |p_n^k - p_n^{k-1}|. */
int or_update_layer(or_ctx* c, int n, double delta, int max_inner, double* maxdiff,
                    double* l1diff) {
  int N = c->N;
  int64_t L = or_layer_size(c, n);
  const uint32_t* st = c->lst + c->off[n];
  double mu_np1 = (n + 1 == N) ? c->nu_sum : c->mu_n[n + 1];
  /* r-independent parts of Eq. (12) */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < L; k++) {
    uint64_t B = st[k];
    double us = 0.0, ds = 0.0;
    for (int u = 0; u < N; u++) {
      if ((B >> u) & 1ULL) {
        uint64_t l = B & ~(1ULL << u); /* l in C_{n-1} */
        us += c->p[l] * up_rate_into(c, B, u);
      } else {
        uint64_t l = B | (1ULL << u); /* l in C^m_{n+1}, mu_{lm} = nu_u */
        ds += c->p[l] * c->nu[u];
      }
    }
    c->upsum[k] = us;
    c->dnsum[k] = ds;
    c->work[k] = c->p[B]; /* p^{k,0} = p^{k-1} */
  }
  double lam_nm1 = c->lam_n[n - 1];
  double down_coef = c->lam_n[n] / mu_np1; /* lambda^{k-1}(n) / mu^{k-1}(n+1) */
  int r = 0;
  double md;
  do {
    r++;
    double mu_prev = c->mu_n[n]; /* mu^{k,r-1}(n) */
    md = 0.0;
    double mu_new = 0.0;
#pragma omp parallel for schedule(static) reduction(max : md) reduction(+ : mu_new)
    for (int64_t k = 0; k < L; k++) {
      uint64_t B = st[k];
      double denom = lambda_m(c, B) + c->mu_m[B];
      double v = c->upsum[k] * (mu_prev / lam_nm1) / denom + c->dnsum[k] * down_coef / denom;
      double d = fabs(v - c->work[k]);
      if (d > md) md = d;
      c->work[k] = v;
      mu_new += c->mu_m[B] * v; /* Eq. (14) */
    }
    c->mu_n[n] = mu_new;
  } while (md > delta && r < max_inner);
  c->inner_total += r;
  double lam_new = 0.0, mx = 0.0, l1 = 0.0;
#pragma omp parallel for schedule(static) reduction(max : mx) reduction(+ : l1, lam_new)
  for (int64_t k = 0; k < L; k++) {
    uint64_t B = st[k];
    double d = fabs(c->work[k] - c->p[B]);
    if (d > mx) mx = d;
    l1 += d;
    c->p[B] = c->work[k];
    lam_new += c->p[B] * lambda_m(c, B); /* Eq. (13) */
  }
  c->lam_n[n] = lam_new;
  if (maxdiff) *maxdiff = mx;
  if (l1diff) *l1diff = l1;
  return r;
}

/* One outer iteration k of Algorithm 1 (layers 1..N-1 ascending).  Returns
 * max_{n,m} |p^k - p^{k-1}|; *l1sup = max_n sum_m |p_n^k - p_n^{k-1}| (the M_k
 * of the convergence proof). */
double or_sweep(or_ctx* c, double delta, int max_inner, double* l1sup) {
  double mx = 0.0, l1s = 0.0;
  for (int n = 1; n <= c->N - 1; n++) {
    double md, l1;
    or_update_layer(c, n, delta, max_inner, &md, &l1);
    if (md > mx) mx = md;
    if (l1 > l1s) l1s = l1;
  }
  if (l1sup) *l1sup = l1s;
  return mx;
}

/* Algorithm 1 main loop: sweep until max |p^k - p^{k-1}| <= eps, at most
 * max_sweeps times.  eps < 0 runs exactly max_sweeps sweeps.  trace_* (nullable,
 * max_sweeps entries) record the step of every sweep.  Returns the number of
 * sweeps; *converged = 1 if the step test passed. */
int or_solve(or_ctx* c, double eps, double delta, int max_sweeps, int max_inner,
             double* trace_linf, double* trace_l1, int* converged) {
  int k = 0;
  int conv = 0;
  while (k < max_sweeps) {
    double l1;
    double step = or_sweep(c, delta, max_inner, &l1);
    if (trace_linf) trace_linf[k] = step;
    if (trace_l1) trace_l1[k] = l1;
    k++;
    if (eps >= 0.0 && step <= eps) {
      conv = 1;
      break;
    }
  }
  if (converged) *converged = conv;
  return k;
}

/* p(n) of the birth-death process: Eq. (10) (loss), Proposition 2 (finite C)
 * and the Remark after it (infinite C).  lam_n, mu_n hold lambda(n), mu(n) for
 * n = 0..N.  Writes pn[0..N] (loss, infinite) or pn[0..N+C] (finite).  For the
 * infinite system *tail = sum_{c>=1} P~{c} (the queued-state mass).  Plain
 * products in long double. */
void or_birth_death(int N, int mode, int C, double lam, double nu_sum, const double* lam_n,
                    const double* mu_n, double* pn, double* tail) {
  int top = mode == OR_FINITE ? N + C : N;
  long double* G = (long double*)malloc(sizeof(long double) * (top + 1));
  G[0] = 1.0L;
  for (int n = 1; n <= top; n++) {
    /* lambda(n-1) and mu(n) of Proposition 2: for n > N, lambda(n-1) = lambda
     * and mu(n) = sum_i nu_i (the reading of G(n) for n > N that makes it the
     * birth-death product) */
    long double ln1 = n - 1 <= N ? (long double)lam_n[n - 1] : (long double)lam;
    long double mn = n <= N ? (long double)mu_n[n] : (long double)nu_sum;
    if (mode != OR_LOSS && n - 1 == N) ln1 = (long double)lam;
    G[n] = G[n - 1] * ln1 / mn;
  }
  long double Z = 0.0L;
  long double extra = 0.0L;
  if (mode == OR_INFINITE) {
    /* Remark: p(0) = [1 + sum_{n<N} G(n) + G(N) / (1 - lambda/mu(N))]^{-1},
     * with G(N) = prod lambda(s-1)/mu(s) (= lambda^N/(mu(1)..mu(N)) because
     * lambda(s) = lambda sum_m p_s(B_m) = lambda for s < N) */
    long double rho = (long double)lam / (long double)nu_sum;
    for (int n = 0; n < N; n++) Z += G[n];
    Z += G[N] / (1.0L - rho);
    extra = G[N] * rho / (1.0L - rho);
  } else {
    for (int n = 0; n <= top; n++) Z += G[n];
  }
  for (int n = 0; n <= top; n++) pn[n] = (double)(G[n] / Z);
  if (tail) *tail = (double)(extra / Z);
  free(G);
}

/* P{B_m} = p(w(B_m)) * p_{w(B_m)}(B_m)  (Proposition 1) */
void or_stationary(const or_ctx* c, const double* pn, double* P) {
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < c->S; y++) P[y] = pn[popc((uint64_t)y)] * c->p[y];
}

/* Per-unit utilisation rho_i = P(unit i busy) (queued states: all busy),
 * response pattern R[j*N+i] = P(a call from node j is served by unit i) and
 * workload W[i*J+j] = lambda_j R_ji / nu_i (fraction of time unit i serves node
 * j).  P is the y-order stationary vector, q_busy the queued-state mass
 * sum_{c>=1} P~{c}, q_wait the probability that an arrival waits (joins the
 * queue): sum_{c=0}^{C-1} P~{c} (finite) or sum_{c>=0} P~{c} (infinite), with
 * P~{0} = P{all busy}.  A waiting call is taken by the unit that frees first,
 * which is unit i with probability nu_i / sum nu (exponential services).
 * Writes rho[N], R[J*N], W[N*J] (nullable) and returns the throughput
 * sum_i nu_i rho_i. */
double or_outputs(const or_ctx* c, const double* P, double q_busy, double q_wait,
                  double* rho, double* R, double* W) {
  int N = c->N, J = c->J;
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t y = 0; y < c->S; y++)
      if ((y >> i) & 1) s += P[y];
    rho[i] = s + q_busy;
  }
  if (R) {
    for (int64_t k = 0; k < (int64_t)J * N; k++) R[k] = 0.0;
    /* node by node (each R[j][.] is added in increasing y, as state by state would) */
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < J; j++) {
      for (int64_t y = 0; y < c->S; y++) {
        int u = or_first_idle(N, c->pref + (size_t)j * N, (uint64_t)y);
        if (u >= 0) R[(size_t)j * N + u] += P[y];
      }
    }
    if (c->mode != OR_LOSS)
      for (int j = 0; j < J; j++)
        for (int i = 0; i < N; i++) R[(size_t)j * N + i] += q_wait * c->nu[i] / c->nu_sum;
  }
  if (W && R)
    for (int i = 0; i < N; i++)
      for (int j = 0; j < J; j++) W[(size_t)i * J + j] = c->lam_j[j] * R[(size_t)j * N + i] / c->nu[i];
  double thr = 0.0;
  for (int i = 0; i < N; i++) thr += c->nu[i] * rho[i];
  return thr;
}

/* Global balance of Eq. (1) at state B, from its definition: outflow
 * P{B}(lambda_m + mu_m) and inflow from the N neighbours (plus, for the all-busy
 * state of a queued system, the service completion out of one waiting call at
 * rate sum nu with probability pq1 = P~{1}).  Uses the stored upward rates. */
void or_state_balance(const or_ctx* c, const double* P, double pq1, uint64_t B, double* out,
                      double* in) {
  double o = P[B] * (lambda_m(c, B) + c->mu_m[B]);
  double s = 0.0;
  for (int u = 0; u < c->N; u++) {
    if ((B >> u) & 1ULL) s += P[B & ~(1ULL << u)] * up_rate_into(c, B, u);
    else s += P[B | (1ULL << u)] * c->nu[u];
  }
  if (B == (uint64_t)(c->S - 1) && c->mode != OR_LOSS) s += pq1 * c->nu_sum;
  *out = o;
  *in = s;
}

/* Relative global-balance residual max_m |out_m - in_m| / max_m out_m over the
 * 2^N hypercube states (the queued states satisfy their birth-death balance by
 * construction and are not included). */
double or_residual(const or_ctx* c, const double* P, double pq1) {
  double mr = 0.0, mo = 0.0;
#pragma omp parallel for schedule(static) reduction(max : mr, mo)
  for (int64_t y = 0; y < c->S; y++) {
    double o, i;
    or_state_balance(c, P, pq1, (uint64_t)y, &o, &i);
    double d = fabs(o - i);
    if (d > mr) mr = d;
    if (o > mo) mo = o;
  }
  return mr / mo;
}

/* Same balance at sampled states with caller-given neighbour probabilities and
 * the dispatch rule evaluated on the spot (no stored rates): for very large N,
 * where the full rate table does not fit the test budget.  Pnb[k*N + u] is P of
 * the neighbour of B_k that differs in unit u; Pself[k] = P{B_k}. */
/* host threads of the OpenMP build (1 in the plain build); n < 1 keeps the default */
int or_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void or_sampled_balance(int N, int J, const double* lam_j, const double* nu,
                        const int32_t* pref, int mode, int64_t count, const uint64_t* B,
                        const double* Pself, const double* Pnb, double pq1, double* out,
                        double* in) {
  double lam = 0.0, nu_sum = 0.0;
  for (int j = 0; j < J; j++) lam += lam_j[j];
  for (int i = 0; i < N; i++) nu_sum += nu[i];
  uint64_t full = (N == 64) ? ~0ULL : ((1ULL << N) - 1);
  for (int64_t k = 0; k < count; k++) {
    uint64_t b = B[k];
    double mu = 0.0;
    for (int i = 0; i < N; i++)
      if ((b >> i) & 1ULL) mu += nu[i];
    double lm = (b == full && mode == OR_LOSS) ? 0.0 : lam;
    double s = 0.0;
    for (int u = 0; u < N; u++) {
      if ((b >> u) & 1ULL)
        s += Pnb[k * N + u] * or_dispatch_rate(N, J, lam_j, pref, b & ~(1ULL << u), u);
      else
        s += Pnb[k * N + u] * nu[u];
    }
    if (b == full && mode != OR_LOSS) s += pq1 * nu_sum;
    out[k] = Pself[k] * (lm + mu);
    in[k] = s;
  }
}
