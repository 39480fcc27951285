/*
 * oracle/tdc_oracle.c -- plain, slow, FP64 CPU oracle for the structured
 * divide-and-conquer tridiagonal eigensolver of Liao, Li, Lu and Roman
 * ("A parallel structured divide-and-conquer algorithm for symmetric
 * tridiagonal eigenvalue problems", IEEE TPDS 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path never links, calls or imports it, and shares no code with it.
 *
 * Every routine follows the paper's steps in the paper's order with no
 * blocking, fusion or reordering beyond what the definitions state:
 *   - Algorithm 1 (classical DC): leaf solve, split, two recursive calls,
 *     rank-one eigenproblem, Q = diag(Q1,Q2) * Qhat.
 *   - Eq. (T2)/(T3)/(rankone): T = diag(T1,T2) + b_k v v^T,
 *     u = diag(Q1,Q2)^T v, M = D + b_k u u^T.
 *   - Eq. (secular): f(lambda) = 1 + rho * sum_i z_i^2/(d_i - lambda)
 *     (the paper's printed form drops the sum; the sum is the reading used).
 *   - Eq. (eigenvector)/(Q_Cauchy): Qhat_ij = zhat_i s_j / (d_i - lambda_j).
 *   - Section 3.2, Eq. (T3-def)/(evect): deflation of small z_i (type 1) and
 *     of nearly equal poles by a plane rotation (type 2).
 *   - Remark after Algorithm 3, Eq. (d-lambda): every d_i - lambda_j is formed
 *     from the pole differences and the root offset, never from lambda_j.
 *   - zhat is recomputed from (d, lambda) (Loewner / Gu-Eisenstat formula, the
 *     construction the paper relies on through its references for the
 *     orthogonality of Qhat).
 *   - Section 2.1 (SRRSC): Schur-complement low-rank approximation of a
 *     Cauchy-like matrix from its generators, Theorem 1, Corollary 1,
 *     Theorem 2, Eq. (sid)/(geneZ).
 *
 * Readings of points the paper leaves open (also listed in the design notes):
 *   - the tree has a uniform depth t, the smallest t with ceil(n/2^t) <= leaf
 *     (leaf >= 2, so that no node of the tree is empty),
 *     and node boundaries at floor(i n / 2^l) on level l (so the top split is
 *     k = floor(n/2) and sibling sizes differ by at most one);
 *   - corner modification d_{k-1} -= |b|, d_k -= |b|, rho = 2|b| >= 0 and
 *     z = [last row of Q1, sign(b) * first row of Q2]/sqrt(2), so ||z|| = 1;
 *   - deflation tolerance tol = 8 eps max(max|d_i|, max|z_i|);
 *     type 1: rho |z_i| <= tol;  type 2: |(d_i - d_j) c s| <= tol for the
 *     last kept pole j and candidate i;
 *   - secular root j lies in (d_j, d_{j+1}); its origin is d_j if
 *     f((d_j+d_{j+1})/2) >= 0 else d_{j+1}; the last root uses d_K;
 *   - leaf solver: implicit symmetric tridiagonal QR with Wilkinson shift
 *     (the paper says "QR algorithm");
 *   - final eigenvalues sorted ascending (stable over [roots, deflated]);
 *     every column is signed so that its entry of largest magnitude is
 *     positive (lowest index on exact ties).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EPS DBL_EPSILON /* 2^-52 */
#define ORC_MAX_LEVELS 48

typedef struct {
  int levels;                      /* number of merge levels (tree depth) */
  int64_t n_merges[ORC_MAX_LEVELS];
  int64_t sum_n[ORC_MAX_LEVELS];   /* sum of merge sizes at the level */
  int64_t sum_K[ORC_MAX_LEVELS];   /* sum of non-deflated sizes */
  int64_t max_K[ORC_MAX_LEVELS];
  int64_t type1[ORC_MAX_LEVELS];
  int64_t type2[ORC_MAX_LEVELS];
  int64_t secular_iter_max;
  int64_t secular_iter_sum;
  int64_t secular_roots;
  int64_t secular_noconv;
  int64_t leaf_noconv;
} orc_stats;

/* ------------------------------------------------------------------ */
/* threads                                                            */
/* ------------------------------------------------------------------ */
static int g_threads = 1;

void orc_set_threads(int t) {
  g_threads = t < 1 ? 1 : t;
#ifdef _OPENMP
  omp_set_num_threads(g_threads);
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* tree depth: the smallest t >= 0 with ceil(n / 2^t) <= leaf          */
/* ------------------------------------------------------------------ */
int orc_tree_depth(int64_t n, int64_t leaf) {
  int t = 0;
  if (leaf < 1) leaf = 1;
  while (((n + ((int64_t)1 << t) - 1) >> t) > leaf) ++t;
  return t;
}

/* ------------------------------------------------------------------ */
/* Leaf: implicit symmetric tridiagonal QR with Wilkinson shift        */
/* (Algorithm 1, "apply the QR algorithm").  d[n] (in/out eigenvalues), */
/* e[n-1] (destroyed), Q n x n column-major (ldq) receives the         */
/* eigenvectors.  Eigenvalues are sorted ascending on return.          */
/* Returns 0, or 1 when the iteration cap was hit.                     */
/* ------------------------------------------------------------------ */
int orc_leaf_qr(int n, double* d, double* e, double* Q, int64_t ldq) {
  int status = 0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
  if (n <= 1) return 0;
  int q = n - 1;
  long iter = 0, max_iter = 30L * n;
  while (q > 0) {
    /* neglect negligible off-diagonal entries */
    for (int k = 0; k < q; ++k)
      if (fabs(e[k]) <= ORC_EPS * (fabs(d[k]) + fabs(d[k + 1]))) e[k] = 0.0;
    while (q > 0 && e[q - 1] == 0.0) --q;
    if (q == 0) break;
    int p = q - 1;
    while (p > 0 && e[p - 1] != 0.0) --p;
    if (++iter > max_iter) { status = 1; break; }
    /* Wilkinson shift from the trailing 2x2 block of [p..q] */
    double dd = 0.5 * (d[q - 1] - d[q]);
    double b = e[q - 1];
    double h = hypot(dd, b);
    double mu = d[q] - b * b / (dd + (dd >= 0.0 ? h : -h));
    double x = d[p] - mu, z = e[p];
    for (int k = p; k < q; ++k) {
      double r = hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) { c = x / r; s = z / r; }
      if (k > p) e[k - 1] = r;
      double ak = d[k], ak1 = d[k + 1], bk = e[k];
      d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      if (k < q - 1) {
        z = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      /* accumulate V <- V R^T on columns k, k+1 */
      double* vk = Q + (int64_t)k * ldq;
      double* vk1 = Q + (int64_t)(k + 1) * ldq;
      for (int i = 0; i < n; ++i) {
        double a0 = vk[i], a1 = vk1[i];
        vk[i] = c * a0 + s * a1;
        vk1[i] = -s * a0 + c * a1;
      }
    }
  }
  /* selection sort, ascending */
  for (int i = 0; i < n - 1; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (d[j] < d[m]) m = j;
    if (m != i) {
      double t = d[i]; d[i] = d[m]; d[m] = t;
      for (int r = 0; r < n; ++r) {
        double u = Q[r + (int64_t)i * ldq];
        Q[r + (int64_t)i * ldq] = Q[r + (int64_t)m * ldq];
        Q[r + (int64_t)m * ldq] = u;
      }
    }
  }
  return status;
}

/* ------------------------------------------------------------------ */
/* Secular equation, Eq. (secular) with the sum restored:              */
/*   f(lambda) = 1 + rho sum_i z_i^2 / (d_i - lambda),                 */
/* solved for root j of K in shifted coordinates lambda = d_org + tau  */
/* (Remark, Eq. (d-lambda)): delta_i = d_i - d_org, and                */
/*   g(tau) = 1/rho + sum_i z_i^2 / (delta_i - tau)                    */
/* has the sign of f and increases with tau.  Newton steps safeguarded */
/* by bisection on the bracket until the bracket or the step reaches    */
/* rounding level: a Newton step is taken only if it stays inside the   */
/* bracket and is at most half the step before last, otherwise the      */
/* bracket is halved, so the bracket at least halves every second step  */
/* (once g is rounding noise, Newton steps alone can shrink it by tiny  */
/* amounts for thousands of steps).  D ascending, rho > 0, z_i != 0.    */
/* Returns the iteration count (negative when the cap was hit).        */
/* ------------------------------------------------------------------ */
static void secular_eval(int K, const double* D, const double* z, double rho, int org, double tau,
                         double* g, double* dg, double* gabs) {
  double s = 1.0 / rho, ds = 0.0, sa = 1.0 / rho;
  for (int i = 0; i < K; ++i) {
    double del = (D[i] - D[org]) - tau;
    double t = z[i] * z[i] / del;
    s += t;
    sa += fabs(t);
    ds += t / del;
  }
  *g = s;
  *dg = ds;
  *gabs = sa;
}

int orc_secular_root(int K, const double* D, const double* z, double rho, int j, int max_iter,
                     int* org_out, double* tau_out) {
  int org;
  double lo, hi;
  if (j < K - 1) {
    double gap = D[j + 1] - D[j];
    double g, dg, ga;
    secular_eval(K, D, z, rho, j, 0.5 * gap, &g, &dg, &ga);
    if (g >= 0.0) { org = j; lo = 0.0; hi = 0.5 * gap; }
    else { org = j + 1; lo = -0.5 * gap; hi = 0.0; }
  } else {
    double zz = 0.0;
    for (int i = 0; i < K; ++i) zz += z[i] * z[i];
    org = K - 1; lo = 0.0; hi = rho * zz;
  }
  double tau = 0.5 * (lo + hi);
  double prev = hi - lo, last = hi - lo; /* the two previous step lengths */
  int it;
  for (it = 1; it <= max_iter; ++it) {
    double g, dg, ga;
    secular_eval(K, D, z, rho, org, tau, &g, &dg, &ga);
    if (g == 0.0) break;
    if (g < 0.0) lo = tau; else hi = tau;
    double step = g / dg;
    double tn = tau - step;
    if (!(tn > lo && tn < hi) || fabs(step) > 0.5 * prev) tn = 0.5 * (lo + hi);
    prev = last;
    last = fabs(tn - tau);
    double w = hi - lo;
    if (w <= 2.0 * ORC_EPS * fmax(fabs(lo), fabs(hi))) { tau = tn; break; }
    if (fabs(tn - tau) <= ORC_EPS * fabs(tau)) { tau = tn; break; }
    tau = tn;
  }
  *org_out = org;
  *tau_out = tau;
  return it > max_iter ? -max_iter : it;
}

/* all K roots; returns the max iteration count, negative if any root hit the cap */
int orc_secular(int K, const double* D, const double* z, double rho, int max_iter, int* org, double* tau,
                int64_t* iter_sum) {
  int maxit = 0, bad = 0;
  int64_t sum = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : maxit) reduction(+ : sum, bad)
  for (int j = 0; j < K; ++j) {
    int it = orc_secular_root(K, D, z, rho, j, max_iter, &org[j], &tau[j]);
    if (it < 0) { bad += 1; it = -it; }
    if (it > maxit) maxit = it;
    sum += it;
  }
  if (iter_sum) *iter_sum = sum;
  return bad ? -maxit : maxit;
}

/* ------------------------------------------------------------------ */
/* Loewner recomputation of zhat from (d, lambda):                     */
/*   zhat_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j!=i} (d_j - d_i)) */
/* evaluated as the product of the ratios                              */
/*   (lambda_j - d_i)/(d_j - d_i)      j < i                           */
/*   (lambda_j - d_i)/(d_{j+1} - d_i)  i <= j < K-1                    */
/*   (lambda_{K-1} - d_i)/rho                                          */
/* with lambda_j - d_i = (d_org(j) - d_i) + tau_j (Eq. (d-lambda)).    */
/* The sign of zhat_i is that of z_i.                                  */
/* ------------------------------------------------------------------ */
void orc_lowner(int K, const double* D, const double* z, double rho, const int* org, const double* tau,
                double* zhat) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < K; ++i) {
    double p = ((D[org[K - 1]] - D[i]) + tau[K - 1]) / rho;
    for (int j = 0; j < i; ++j) p *= ((D[org[j]] - D[i]) + tau[j]) / (D[j] - D[i]);
    for (int j = i; j < K - 1; ++j) p *= ((D[org[j]] - D[i]) + tau[j]) / (D[j + 1] - D[i]);
    zhat[i] = copysign(sqrt(p), z[i]);
  }
}

/* column normalisers s_j = 1/sqrt(sum_i zhat_i^2/delta_ij^2), delta_ij = d_i - lambda_j */
void orc_colnorm(int K, const double* D, const int* org, const double* tau, const double* zhat, double* s) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int j = 0; j < K; ++j) {
    double acc = 0.0;
    for (int i = 0; i < K; ++i) {
      double del = (D[i] - D[org[j]]) - tau[j];
      double t = zhat[i] / del;
      acc += t * t;
    }
    s[j] = 1.0 / sqrt(acc);
  }
}

/* dense Qhat (K x K, column-major, ldu): Qhat_ij = zhat_i s_j / delta_ij  (Eq. (Q_Cauchy)) */
void orc_qhat(int K, const double* D, const int* org, const double* tau, const double* zhat, const double* s,
              double* U, int64_t ldu) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < K; ++j)
    for (int i = 0; i < K; ++i) {
      double del = (D[i] - D[org[j]]) - tau[j];
      U[i + (int64_t)j * ldu] = zhat[i] * s[j] / del;
    }
}

/* ------------------------------------------------------------------ */
/* Deflation (Section 3.2, Eq. (T3-def)).                              */
/* Input: D[n], z[n] in merge-column order, the stable ascending order  */
/* perm[n] of D, rho.  Rotations are applied to the columns of Q       */
/* (n rows, ldq) and to D and z.  Output: kept[K] (column indices in    */
/* ascending pole order), defl[n-K] (column indices in scan order),    */
/* counts of type-1 and type-2 deflations.  Returns K.                 */
/* ------------------------------------------------------------------ */
int orc_deflate(int n, double* D, double* z, const int* perm, double rho, double* Q, int64_t ldq, int* kept,
                int* defl, int* n_type1, int* n_type2) {
  double dmax = 0.0, zmax = 0.0;
  for (int i = 0; i < n; ++i) {
    if (fabs(D[i]) > dmax) dmax = fabs(D[i]);
    if (fabs(z[i]) > zmax) zmax = fabs(z[i]);
  }
  double tol = 8.0 * ORC_EPS * fmax(dmax, zmax);
  int K = 0, nd = 0, t1 = 0, t2 = 0;
  int pj = -1;
  for (int q = 0; q < n; ++q) {
    int i = perm[q];
    if (rho * fabs(z[i]) <= tol) { /* type 1 */
      defl[nd++] = i;
      ++t1;
      continue;
    }
    if (pj < 0) { pj = i; continue; }
    double zs = z[pj], zc = z[i];
    double tau = hypot(zc, zs);
    double c = zc / tau, s = -zs / tau;
    double t = D[i] - D[pj];
    if (fabs(t * c * s) <= tol) { /* type 2: rotate the pair so that z[pj] = 0 */
      z[i] = tau;
      z[pj] = 0.0;
      double dp = D[pj], di = D[i];
      D[pj] = dp * c * c + di * s * s;
      D[i] = dp * s * s + di * c * c;
      double* qp = Q + (int64_t)pj * ldq;
      double* qi = Q + (int64_t)i * ldq;
      for (int r = 0; r < n; ++r) {
        double a = qp[r], b = qi[r];
        qp[r] = c * a + s * b;
        qi[r] = -s * a + c * b;
      }
      defl[nd++] = pj;
      ++t2;
      pj = i;
    } else {
      kept[K++] = pj;
      pj = i;
    }
  }
  if (pj >= 0) kept[K++] = pj;
  if (n_type1) *n_type1 = t1;
  if (n_type2) *n_type2 = t2;
  return K;
}

/* ------------------------------------------------------------------ */
/* One merge (Algorithm 1, lines "form M", "find eigenvalues", "compute */
/* the eigenvectors"; Section 3.2 for deflation).                      */
/* lam[n]: children's eigenvalues (each half ascending); Q: the n x n  */
/* block with Q1 and Q2 on its diagonal (off-diagonal blocks zero).    */
/* b = the coupling off-diagonal entry e_{n1-1}.                       */
/* ------------------------------------------------------------------ */
static int cmp_idx_val(const double* v, int a, int b) {
  if (v[a] < v[b]) return -1;
  if (v[a] > v[b]) return 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}

static void stable_sort_idx(int n, const double* v, int* idx) {
  /* insertion-merge sort (bottom-up merge sort) on indices, stable */
  int* tmp = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int w = 1; w < n; w *= 2) {
    for (int lo = 0; lo < n; lo += 2 * w) {
      int mid = lo + w < n ? lo + w : n, hi = lo + 2 * w < n ? lo + 2 * w : n;
      int a = lo, b = mid, o = lo;
      while (a < mid && b < hi) tmp[o++] = (cmp_idx_val(v, idx[b], idx[a]) < 0) ? idx[b++] : idx[a++];
      while (a < mid) tmp[o++] = idx[a++];
      while (b < hi) tmp[o++] = idx[b++];
    }
    memcpy(idx, tmp, sizeof(int) * (size_t)n);
  }
  free(tmp);
}

int orc_merge(int n, int n1, double b, double* lam, double* Q, int64_t ldq, int max_iter, orc_stats* st,
              int level) {
  const double rs2 = 1.0 / sqrt(2.0);
  double rho = 2.0 * fabs(b);
  double sg = b < 0.0 ? -1.0 : 1.0;
  double* D = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  int* perm = (int*)malloc(sizeof(int) * (size_t)n);
  int* kept = (int*)malloc(sizeof(int) * (size_t)n);
  int* defl = (int*)malloc(sizeof(int) * (size_t)n);
  int status = 0;
  /* Eq. (T3): u = [last row of Q1; first row of Q2] (sign of b folded in), z = u/sqrt(2) */
  for (int i = 0; i < n; ++i) D[i] = lam[i];
  for (int i = 0; i < n1; ++i) z[i] = Q[(n1 - 1) + (int64_t)i * ldq] * rs2;
  for (int i = n1; i < n; ++i) z[i] = sg * Q[n1 + (int64_t)i * ldq] * rs2;
  for (int i = 0; i < n; ++i) perm[i] = i;
  stable_sort_idx(n, D, perm);
  int t1 = 0, t2 = 0;
  int K = orc_deflate(n, D, z, perm, rho, Q, ldq, kept, defl, &t1, &t2);
  int nd = n - K;
  if (st && level < ORC_MAX_LEVELS) {
    st->n_merges[level] += 1;
    st->sum_n[level] += n;
    st->sum_K[level] += K;
    if (K > st->max_K[level]) st->max_K[level] = K;
    st->type1[level] += t1;
    st->type2[level] += t2;
  }
  double* Dk = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* zk = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  int* org = (int*)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
  double* tau = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* zh = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  double* sn = (double*)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
  for (int j = 0; j < K; ++j) { Dk[j] = D[kept[j]]; zk[j] = z[kept[j]]; }
  if (K > 0) {
    int64_t isum = 0;
    int mi = orc_secular(K, Dk, zk, rho, max_iter, org, tau, &isum);
    if (mi < 0) { status = 2; mi = -mi; if (st) st->secular_noconv += 1; }
    if (st) {
      if (mi > st->secular_iter_max) st->secular_iter_max = mi;
      st->secular_iter_sum += isum;
      st->secular_roots += K;
    }
    orc_lowner(K, Dk, zk, rho, org, tau, zh);
    orc_colnorm(K, Dk, org, tau, zh, sn);
  }
  /* eigenpairs: roots first (ascending), deflated after (scan order) */
  double* val = (double*)malloc(sizeof(double) * (size_t)n);
  int* ord = (int*)malloc(sizeof(int) * (size_t)n);
  for (int j = 0; j < K; ++j) val[j] = Dk[org[j]] + tau[j];
  for (int q = 0; q < nd; ++q) val[K + q] = D[defl[q]];
  for (int i = 0; i < n; ++i) ord[i] = i;
  stable_sort_idx(n, val, ord);
  /* new eigenvector columns, Eq. (evect): [diag(Q1,Q2) G P] diag(Qhat, I) */
  double* C = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < K; ++j) {
    double* c = C + (int64_t)j * n;
    for (int r = 0; r < n; ++r) c[r] = 0.0;
    for (int i = 0; i < K; ++i) {
      double del = (Dk[i] - Dk[org[j]]) - tau[j];
      double u = zh[i] * sn[j] / del;
      const double* qc = Q + (int64_t)kept[i] * ldq;
      for (int r = 0; r < n; ++r) c[r] += qc[r] * u;
    }
  }
  for (int q = 0; q < nd; ++q) {
    double* c = C + (int64_t)(K + q) * n;
    const double* qc = Q + (int64_t)defl[q] * ldq;
    for (int r = 0; r < n; ++r) c[r] = qc[r];
  }
  for (int p = 0; p < n; ++p) {
    lam[p] = val[ord[p]];
    const double* c = C + (int64_t)ord[p] * n;
    double* qo = Q + (int64_t)p * ldq;
    for (int r = 0; r < n; ++r) qo[r] = c[r];
  }
  free(C); free(val); free(ord);
  free(Dk); free(zk); free(org); free(tau); free(zh); free(sn);
  free(D); free(z); free(perm); free(kept); free(defl);
  return status;
}

/* ------------------------------------------------------------------ */
/* Recursive DC (Algorithm 1) on the node [lo, hi) of depth `level`,   */
/* index `idx` within its level; the tree of order n and depth t has   */
/* its node boundaries at floor(i n / 2^level), so the node splits at  */
/* mid = floor((2 idx + 1) n / 2^(level+1)).  d is a private copy that */
/* receives the corner modifications.                                  */
/* ------------------------------------------------------------------ */
static int dc_rec(int64_t ntot, int64_t lo, int64_t hi, int level, int64_t idx, int t, double* d, const double* e,
                  double* lam, double* Q, int64_t ldq, int max_iter, orc_stats* st) {
  int n = (int)(hi - lo);
  double* Qb = Q + lo + lo * ldq;
  if (level == t || n <= 1) {
    double* ee = (double*)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
    for (int i = 0; i < n - 1; ++i) ee[i] = e[lo + i];
    for (int i = 0; i < n; ++i) lam[lo + i] = d[lo + i];
    int s = orc_leaf_qr(n, lam + lo, ee, Qb, ldq);
    free(ee);
    if (s && st) st->leaf_noconv += 1;
    return s ? 3 : 0;
  }
  int64_t mid = ((2 * idx + 1) * ntot) >> (level + 1);
  int n1 = (int)(mid - lo);
  double b = e[mid - 1];
  /* Eq. (T2): T = diag(T1, T2) + |b| v v^T, v = e_{mid-1} + sign(b) e_{mid} */
  d[mid - 1] -= fabs(b);
  d[mid] -= fabs(b);
  for (int j = 0; j < n1; ++j)
    for (int i = n1; i < n; ++i) Qb[i + (int64_t)j * ldq] = 0.0;
  for (int j = n1; j < n; ++j)
    for (int i = 0; i < n1; ++i) Qb[i + (int64_t)j * ldq] = 0.0;
  int s1 = dc_rec(ntot, lo, mid, level + 1, 2 * idx, t, d, e, lam, Q, ldq, max_iter, st);
  int s2 = dc_rec(ntot, mid, hi, level + 1, 2 * idx + 1, t, d, e, lam, Q, ldq, max_iter, st);
  int s3 = orc_merge(n, n1, b, lam + lo, Qb, ldq, max_iter, st, level);
  return s1 ? s1 : (s2 ? s2 : s3);
}

/* sign convention: the entry of largest magnitude in each column is positive */
void orc_sign_normalise(int n, double* Q, int64_t ldq) {
  for (int j = 0; j < n; ++j) {
    double* q = Q + (int64_t)j * ldq;
    int im = 0;
    for (int i = 1; i < n; ++i)
      if (fabs(q[i]) > fabs(q[im])) im = i;
    if (q[im] < 0.0)
      for (int i = 0; i < n; ++i) q[i] = -q[i];
  }
}

/* Full eigensolve: T = Q diag(lam) Q^T, lam ascending.  Returns 0 on success,
 * 2 when a secular root hit the iteration cap, 3 when a leaf did not converge. */
int orc_eig(int n, const double* d, const double* e, int leaf, int max_iter, double* lam, double* Q,
            int64_t ldq, orc_stats* st) {
  if (st) memset(st, 0, sizeof(*st));
  if (n <= 0) return 0;
  double* dc = (double*)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; ++i) dc[i] = d[i];
  int depth = orc_tree_depth(n, leaf);
  if (st) st->levels = depth;
  int s = dc_rec(n, 0, n, 0, 0, depth, dc, e, lam, Q, ldq, max_iter, st);
  orc_sign_normalise(n, Q, ldq);
  free(dc);
  return s;
}

/* ------------------------------------------------------------------ */
/* Plain dense product C = A * B (column-major), the reference for the  */
/* Q*U products (Eq. (updateV)).  A m x k (lda), B k x n (ldb).        */
/* ------------------------------------------------------------------ */
void orc_gemm(int m, int n, int k, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
              int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j) {
    double* c = C + (int64_t)j * ldc;
    for (int i = 0; i < m; ++i) c[i] = 0.0;
    for (int p = 0; p < k; ++p) {
      double bpj = B[p + (int64_t)j * ldb];
      const double* a = A + (int64_t)p * lda;
      for (int i = 0; i < m; ++i) c[i] += a[i] * bpj;
    }
  }
}
