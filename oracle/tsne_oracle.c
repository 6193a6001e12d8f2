/*
 * tsne_oracle.c -- plain, slow, FP64 CPU reference of exact t-SNE.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the test-suite, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes.  The CudaMon paper (Sec. 3-4, Table 1 step 7 "Umap + t-sne")
 * runs t-SNE on PCA scores but never states the method, so every function below
 * follows the textbook exact t-SNE: van der Maaten & Hinton (2008) for the
 * Student-t similarities, the KL objective and its gradient, and the
 * optimiser with early exaggeration, momentum and gains; van der Maaten (2014)
 * for the k-nearest-neighbour sparse input affinities.  Each function names the
 * definition it writes out.  Readings of points the papers leave open:
 *   - neighbours ordered by (squared distance, index), self excluded by index;
 *   - entropy in nats, perplexity = exp(H);
 *   - rows whose target entropy is unreachable (>= perplexity tied minimum
 *     distances, e.g. all k distances equal) get the beta -> infinity limit:
 *     uniform weight on the tied minimum set; they are flagged;
 *   - P = (P_cond + P_cond^T) / (2N), so sum(P) = 1;
 *   - w_ij = 1 / (1 + |y_i - y_j|^2) (one degree of freedom), Z = sum_{i!=j} w_ij;
 *   - gradient constant 4; exaggeration alpha multiplies P in the gradient;
 *   - KL_alpha = sum p log p + alpha sum p log(1 + d^2) + log Z, whose gradient
 *     is exactly the exaggerated gradient (equals KL(P||Q) at alpha = 1 when
 *     sum(P) = 1);
 *   - gains: +0.2 where g*u < 0 strictly, else *0.8, floored at min_gain;
 *     u <- mu*u - eta*gain*g ; Y <- Y + u ; no re-centring of Y.
 * Pins (tests/test_oracle.py): brute-force kNN by full sort, entropy and Gibbs
 * form of each calibrated row, the k = 2 closed form, dense symmetrisation,
 * KL against its direct definition sum p log(p/q), central finite differences,
 * the N = 2 closed form, P = Q stationarity, rigid-motion invariances and a
 * hand-worked two-point optimiser trajectory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

ORACLE_API int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* kNN: for each query row q, the k points j != q with the smallest squared
 * Euclidean distance sum_c (x_qc - x_jc)^2, computed directly (no norm
 * expansion), ordered by (d2, j).  A bounded insertion list keeps the first k
 * of that order while j is scanned in increasing order.                      */
ORACLE_API void oracle_knn_rows(const double* X, int64_t n, int d, int k,
                                const int64_t* rows, int64_t n_rows,
                                int32_t* idx, double* d2) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < n_rows; r++) {
    const int64_t q = rows ? rows[r] : r;
    const double* xq = X + q * d;
    int32_t* oi = idx + r * k;
    double* od = d2 + r * k;
    int filled = 0;
    for (int64_t j = 0; j < n; j++) {
      if (j == q) continue;
      const double* xj = X + j * d;
      double s = 0.0;
      for (int c = 0; c < d; c++) {
        double t = xq[c] - xj[c];
        s += t * t;
      }
      /* j is larger than every index already held, so (s, j) goes after all
       * entries with distance <= s. */
      if (filled == k && !(s < od[k - 1])) continue;
      int pos = (filled < k) ? filled : k - 1;
      while (pos > 0 && od[pos - 1] > s) {
        od[pos] = od[pos - 1];
        oi[pos] = oi[pos - 1];
        pos--;
      }
      od[pos] = s;
      oi[pos] = (int32_t)j;
      if (filled < k) filled++;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Perplexity calibration of one row (van der Maaten & Hinton 2008, Sec. 2):
 * p_{j|i} = exp(-beta d_j) / sum_l exp(-beta d_l) over the k neighbours, with
 * beta chosen so that H = -sum_j p_j log p_j equals log(perplexity).  With
 * s_j = d_j - min d, S = sum exp(-beta s_j): H(beta) = log S + beta sum p_j s_j,
 * strictly decreasing in beta from log k (beta = 0) to log(#ties at the min)
 * (beta -> inf).  Bracket by doubling / halving from beta = 1, then bisect.
 * Returns 0 when converged, 1 when the target is unreachable (limit used),
 * 2 when max_iter ran out.                                                   */
static double row_entropy(const double* s, int k, double beta, double* p) {
  double S = 0.0;
  for (int j = 0; j < k; j++) { p[j] = exp(-beta * s[j]); S += p[j]; }
  double m = 0.0;
  for (int j = 0; j < k; j++) { p[j] /= S; m += p[j] * s[j]; }
  return log(S) + beta * m;
}

static int calibrate_row(const double* dist, int k, double perp, double tol,
                         int max_iter, double* p, double* beta_out) {
  double* s = (double*)malloc(sizeof(double) * k);
  double dmin = dist[0];
  for (int j = 1; j < k; j++) if (dist[j] < dmin) dmin = dist[j];
  int ties = 0;
  for (int j = 0; j < k; j++) { s[j] = dist[j] - dmin; if (s[j] == 0.0) ties++; }
  const double target = log(perp);
  if ((double)ties >= perp) {
    for (int j = 0; j < k; j++) p[j] = (s[j] == 0.0) ? 1.0 / ties : 0.0;
    *beta_out = INFINITY;
    free(s);
    return 1;
  }
  /* beta = 0 is always a lower bracket: H(0) = log k > log(perplexity). */
  double beta = 1.0, lo = 0.0, hi = INFINITY;
  int status = 2;
  for (int it = 0; it < max_iter; it++) {
    double H = row_entropy(s, k, beta, p);
    if (fabs(H - target) <= tol) { status = 0; break; }
    if (H > target) lo = beta; else hi = beta;     /* H decreases with beta */
    beta = isinf(hi) ? 2.0 * beta : 0.5 * (lo + hi);
  }
  if (status != 0) row_entropy(s, k, beta, p);
  *beta_out = beta;
  free(s);
  return status;
}

ORACLE_API int64_t oracle_calibrate(const double* d2, int64_t n, int k, double perp,
                                    double tol, int max_iter, double* pcond,
                                    double* beta, int8_t* flag) {
  int64_t n_bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : n_bad)
  for (int64_t i = 0; i < n; i++) {
    int st = calibrate_row(d2 + i * k, k, perp, tol, max_iter, pcond + i * k, beta + i);
    flag[i] = (int8_t)st;
    if (st != 0) n_bad++;
  }
  return n_bad;
}

/* The Gibbs distribution of a row at a given beta (beta = +inf: uniform on
 * the minimum-distance set): p_j = exp(-beta (d_j - min d)) / sum_l (...).   */
ORACLE_API void oracle_cond_at_beta(const double* d2, int64_t n, int k, const double* beta,
                                    double* pcond) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    const double* d = d2 + i * k;
    double* p = pcond + i * k;
    double dmin = d[0];
    for (int j = 1; j < k; j++) if (d[j] < dmin) dmin = d[j];
    double S = 0.0;
    for (int j = 0; j < k; j++) {
      p[j] = isinf(beta[i]) ? (d[j] == dmin ? 1.0 : 0.0) : exp(-beta[i] * (d[j] - dmin));
      S += p[j];
    }
    for (int j = 0; j < k; j++) p[j] /= S;
  }
}

/* ------------------------------------------------------------------------- */
/* Symmetrisation: p_ij = (p_{j|i} + p_{i|j}) / (2N) on the union of the two
 * kNN graphs, as CSR with ascending columns.  Written as: emit both (i,j) and
 * (j,i) copies of every conditional entry scaled by 1/(2N), sort the triplets
 * by (row, col), and add equal keys.                                          */
typedef struct { int64_t r; int64_t c; double v; } trip;

static int trip_cmp(const void* a, const void* b) {
  const trip* x = (const trip*)a;
  const trip* y = (const trip*)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

/* Writes row_ptr[n+1]; col/val must hold 2nk entries; returns nnz.          */
ORACLE_API int64_t oracle_symmetrize(const int32_t* idx, const double* pcond, int64_t n,
                                     int k, int64_t* row_ptr, int32_t* col, double* val) {
  const int64_t m = 2 * n * (int64_t)k;
  trip* t = (trip*)malloc(sizeof(trip) * (size_t)m);
  const double scale = 1.0 / (2.0 * (double)n);
  int64_t e = 0;
  for (int64_t i = 0; i < n; i++)
    for (int a = 0; a < k; a++) {
      int64_t j = idx[i * k + a];
      double v = pcond[i * k + a] * scale;
      t[e].r = i; t[e].c = j; t[e].v = v; e++;
      t[e].r = j; t[e].c = i; t[e].v = v; e++;
    }
  qsort(t, (size_t)m, sizeof(trip), trip_cmp);
  int64_t nnz = 0;
  for (int64_t i = 0; i <= n; i++) row_ptr[i] = 0;
  for (int64_t a = 0; a < m; a++) {
    if (nnz > 0 && t[a].r == t[a - 1].r && t[a].c == t[a - 1].c) {
      val[nnz - 1] += t[a].v;
    } else {
      col[nnz] = (int32_t)t[a].c;
      val[nnz] = t[a].v;
      row_ptr[t[a].r + 1]++;
      nnz++;
    }
  }
  for (int64_t i = 0; i < n; i++) row_ptr[i + 1] += row_ptr[i];
  free(t);
  return nnz;
}

/* ------------------------------------------------------------------------- */
/* Normaliser Z = sum_{i != j} 1 / (1 + |y_i - y_j|^2) over all ordered pairs
 * of the n points (Y row-major n x 2).                                       */
ORACLE_API double oracle_Z(const double* Y, int64_t n) {
  double Z = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : Z)
  for (int64_t i = 0; i < n; i++) {
    double zi = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
      zi += 1.0 / (1.0 + dx * dx + dy * dy);
    }
    Z += zi;
  }
  return Z;
}

/* Exact gradient (van der Maaten & Hinton 2008, Eq. 5 with exaggeration):
 *   dC/dy_i = 4 sum_{j != i} (alpha p_ij - q_ij) w_ij (y_i - y_j),  q_ij = w_ij / Z.
 * p_ij is read from the CSR row (ascending columns, no diagonal) while j runs
 * over all points.  Returns Z.                                               */
ORACLE_API double oracle_grad(const int64_t* row_ptr, const int32_t* col, const double* val,
                              const double* Y, int64_t n, double alpha, double* grad) {
  const double Z = oracle_Z(Y, n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) {
    int64_t e = row_ptr[i], end = row_ptr[i + 1];
    double gx = 0.0, gy = 0.0;
    for (int64_t j = 0; j < n; j++) {
      double p = 0.0;
      if (e < end && col[e] == j) p = val[e++];
      if (j == i) continue;
      double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
      double w = 1.0 / (1.0 + dx * dx + dy * dy);
      double c = (alpha * p - w / Z) * w;
      gx += c * dx;
      gy += c * dy;
    }
    grad[2 * i] = 4.0 * gx;
    grad[2 * i + 1] = 4.0 * gy;
  }
  return Z;
}

/* The two halves of the gradient for selected rows, for per-term checks:
 *   Fa_i = sum_j p_ij w_ij (y_i - y_j)          (attraction, over the CSR row)
 *   Fr_i = sum_{j != i} w_ij^2 (y_i - y_j)      (repulsion, over all points)
 *   Z_i  = sum_{j != i} w_ij
 * so that dC/dy_i = 4 (alpha Fa_i - Fr_i / Z) with Z = sum_i Z_i.
 * Optionally (Aa, Ar non-null) the sums of the terms' magnitudes,
 *   Aa_i = sum_j p_ij w_ij |y_i - y_j|,   Ar_i = sum_{j != i} w_ij^2 |y_i - y_j|,
 * the scale against which the rounding error of a floating-point evaluation
 * of each row's sum is bounded (|Fa_i| <= Aa_i, |Fr_i| <= Ar_i).             */
ORACLE_API void oracle_forces_rows(const int64_t* row_ptr, const int32_t* col, const double* val,
                                   const double* Y, int64_t n, const int64_t* rows, int64_t n_rows,
                                   double* Fa, double* Fr, double* Zi, double* Aa, double* Ar) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < n_rows; r++) {
    const int64_t i = rows ? rows[r] : r;
    double ax = 0.0, ay = 0.0, aa = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      int64_t j = col[e];
      double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
      double w = 1.0 / (1.0 + dx * dx + dy * dy);
      ax += val[e] * w * dx;
      ay += val[e] * w * dy;
      if (Aa) aa += fabs(val[e]) * w * sqrt(dx * dx + dy * dy);
    }
    double rx = 0.0, ry = 0.0, z = 0.0, ar = 0.0;
    for (int64_t j = 0; j < n; j++) {
      if (j == i) continue;
      double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
      double w = 1.0 / (1.0 + dx * dx + dy * dy);
      rx += w * w * dx;
      ry += w * w * dy;
      z += w;
      if (Ar) ar += w * w * sqrt(dx * dx + dy * dy);
    }
    Fa[2 * r] = ax; Fa[2 * r + 1] = ay;
    Fr[2 * r] = rx; Fr[2 * r + 1] = ry;
    Zi[r] = z;
    if (Aa) Aa[r] = aa;
    if (Ar) Ar[r] = ar;
  }
}

/* KL_alpha(Y) = sum_ij p_ij log p_ij + alpha sum_ij p_ij log(1 + d_ij^2) + log Z.
 * At alpha = 1 and sum(P) = 1 this is KL(P || Q) = sum p log(p / q).         */
ORACLE_API double oracle_kl(const int64_t* row_ptr, const int32_t* col, const double* val,
                            const double* Y, int64_t n, double alpha, double Z) {
  double a = 0.0, b = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : a, b)
  for (int64_t i = 0; i < n; i++)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
      int64_t j = col[e];
      double p = val[e];
      if (p <= 0.0) continue;
      double dx = Y[2 * i] - Y[2 * j], dy = Y[2 * i + 1] - Y[2 * j + 1];
      a += p * log(p);
      b += p * log(1.0 + dx * dx + dy * dy);
    }
  if (!(Z > 0.0)) Z = oracle_Z(Y, n);
  return a + alpha * b + log(Z);
}

/* ------------------------------------------------------------------------- */
/* Gradient descent of van der Maaten & Hinton (2008), Sec. 3.4, with the
 * delta-bar-delta gains of the reference implementations: for t = 0..T-1
 *   alpha = ee if t < ee_iters else 1 ;  mu = mom0 if t < mom_switch else mom1
 *   g = grad(Y, alpha)
 *   gain = (g*u < 0) ? gain + 0.2 : gain * 0.8 ; gain = max(gain, min_gain)
 *   u = mu*u - eta*gain*g ; Y = Y + u
 * kl_trace[m] (if non-null) = KL at alpha = 1 of the Y whose gradient is taken
 * at iterations t with (t+1) % kl_every == 0.                                */
ORACLE_API void oracle_run(const int64_t* row_ptr, const int32_t* col, const double* val,
                           int64_t n, double* Y, double* U, double* gains, int n_iter,
                           int ee_iters, double ee, int mom_switch, double mom0, double mom1,
                           double eta, double min_gain, int kl_every, double* kl_trace) {
  double* g = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  int m = 0;
  for (int t = 0; t < n_iter; t++) {
    const double alpha = (t < ee_iters) ? ee : 1.0;
    const double mu = (t < mom_switch) ? mom0 : mom1;
    const double Z = oracle_grad(row_ptr, col, val, Y, n, alpha, g);
    if (kl_trace && kl_every > 0 && (t + 1) % kl_every == 0)
      kl_trace[m++] = oracle_kl(row_ptr, col, val, Y, n, 1.0, Z);
    for (int64_t a = 0; a < 2 * n; a++) {
      double gain = (g[a] * U[a] < 0.0) ? gains[a] + 0.2 : gains[a] * 0.8;
      if (gain < min_gain) gain = min_gain;
      gains[a] = gain;
      U[a] = mu * U[a] - eta * gain * g[a];
      Y[a] += U[a];
    }
  }
  free(g);
}
