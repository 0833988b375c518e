/*
 * spid_oracle.c -- plain FP64 CPU restatement of the sketched column
 * interpolative decomposition (SPID with a Gaussian sketch).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is written for a reader who checks it against the paper
 * (arXiv 2103.01380, Pacella, Dunton, Doostan, Iaccarino):
 *   - data matrix A is m x n, rows = grid points x QoIs, columns = time
 *     snapshots, 0-based (Section 2, notation table);
 *   - column ID  A ~ A(:,I) C  with C = [I_k | R11^+ R12] Z^T from a
 *     column-pivoted QR  A Z = Q R  (Section 2, Eqs. for AZ = QR and C,
 *     Algorithm 1);
 *   - ID from a sketch B = Omega A with Omega l x m i.i.d. N(0,1)
 *     (Section 2, the random-projection paragraph; Algorithm 2 output form
 *     A(:,I_B) C_B);
 *   - pivoted QR by modified Gram-Schmidt ("mgsqr", Section 2 / Algorithm 1);
 *   - adaptive rank (Remark 2.1), relative Frobenius error (Section 5.1),
 *     compression factor CF = mn / (k(m+n)) (Section 2, Eq. for CF).
 *
 * Readings where the paper is silent:
 *   - Omega(i, r) = Box-Muller of Philox4x32-10 (Salmon et al., SC'11) words,
 *     key = (seed lo32, seed hi32), counter = (r, i/4, 0, 0); words (x0,x1)
 *     give rows 4g, 4g+1 and (x2,x3) give rows 4g+2, 4g+3 of group g = i/4;
 *     u = (x + 0.5) 2^-32, g0 = sqrt(-2 ln u_a) cos(2 pi u_b),
 *     g1 = sqrt(-2 ln u_a) sin(2 pi u_b).
 *   - the sketch sums rows in ascending order.
 *   - pivot = largest residual column norm, recomputed from scratch at every
 *     step; ties go to the lowest original column index.
 *   - adaptive stop: smallest k with ||R22^(k)||_F <= tol ||Y||_F, k <= kmax.
 *   - rank guard: keep the leading pivots with |R_jj| > 2 u_mode |R_00|.
 *
 * All arrays are column-major with explicit leading dimensions unless noted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11, Section 3 (Philox S-box: two 32x32->64       */
/* multiplications per round, Weyl-sequence key schedule).                  */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  /* multipliers and Weyl increments as published for Philox4x32 */
  const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
  const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(PHILOX_M0, c0, &hi0, &lo0);
    mulhilo32(PHILOX_M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller on a pair of 32-bit words, in FP64. */
static void box_muller(uint32_t xa, uint32_t xb, double* g0, double* g1) {
  const double two_m32 = 2.3283064365386963e-10; /* 2^-32 */
  const double two_pi = 6.283185307179586476925286766559;
  double ua = ((double)xa + 0.5) * two_m32;
  double ub = ((double)xb + 0.5) * two_m32;
  double rad = sqrt(-2.0 * log(ua));
  *g0 = rad * cos(two_pi * ub);
  *g1 = rad * sin(two_pi * ub);
}

/* One entry of the Gaussian test matrix Omega (l x m), Section 2 random
 * projection B = Omega A.  Omega does not depend on the subdomain. */
double orc_omega_entry(uint64_t seed, int64_t i, int64_t r) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(i / 4), 0u, 0u};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  double g0, g1;
  int w = (int)(i % 4);
  if (w < 2) box_muller(x[0], x[1], &g0, &g1);
  else       box_muller(x[2], x[3], &g0, &g1);
  return (w % 2 == 0) ? g0 : g1;
}

/* Omega(:, r0 : r0+nrows) into out, column-major l x nrows (ld = l). */
void orc_omega(uint64_t seed, int64_t r0, int64_t nrows, int32_t l, double* out) {
  for (int64_t r = 0; r < nrows; ++r)
    for (int32_t i = 0; i < l; ++i)
      out[i + (int64_t)l * r] = orc_omega_entry(seed, i, r0 + r);
}

/* Sketch Y = Omega A (Section 2, B = Omega A).  A: m x n (ld), Y: l x n
 * (ld = l).  Each Y(i,j) sums over rows r = 0..m-1 in ascending order. */
void orc_sketch(const double* A, int64_t m, int64_t n, int64_t ld, int32_t l,
                uint64_t seed, double* Y) {
  double* Om = (double*)malloc(sizeof(double) * (size_t)l * (size_t)(m > 0 ? m : 1));
  orc_omega(seed, 0, m, l, Om);
  for (int64_t j = 0; j < n; ++j) {
    double* y = Y + (int64_t)l * j;
    for (int32_t i = 0; i < l; ++i) y[i] = 0.0;
    const double* a = A + ld * j;
    for (int64_t r = 0; r < m; ++r) {
      const double arj = a[r];
      const double* om = Om + (int64_t)l * r;
      for (int32_t i = 0; i < l; ++i) y[i] += om[i] * arj;
    }
  }
  free(Om);
}

/* ------------------------------------------------------------------------ */
/* Column-pivoted QR by modified Gram-Schmidt ("mgsqr", Section 2,           */
/* Algorithm 1 step 3), with the adaptive stop of Remark 2.1.               */
/*                                                                          */
/* Input W: l x n (ld = l), overwritten with the residual columns.          */
/* Output: J[0..k-1] pivots in pivot order, R (kmax x n, row-major:         */
/* R[j*n + c] = R(j, column c in ORIGINAL numbering)), the number of steps  */
/* k, and ||Y||_F^2.  R(j, J[j]) = R_jj >= 0; R(j, J[p]) for p > j is R11's */
/* upper part; R(j, c) for non-pivoted c is R12.                            */
/* tol <= 0 means fixed rank kmax.                                          */
/* ------------------------------------------------------------------------ */
int orc_qrcp_mgs(double* W, int32_t l, int64_t n, int32_t kmax, double tol,
                 int32_t* J, double* R, double* normY2_out) {
  char* active = (char*)malloc((size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)l);
  for (int64_t c = 0; c < n; ++c) active[c] = 1;
  for (int64_t x = 0; x < (int64_t)kmax * n; ++x) R[x] = 0.0;
  double normY2 = 0.0;
  for (int64_t c = 0; c < n; ++c)
    for (int32_t i = 0; i < l; ++i) normY2 += W[i + (int64_t)l * c] * W[i + (int64_t)l * c];
  if (normY2_out) *normY2_out = normY2;
  int32_t kcap = kmax;
  if (kcap > l) kcap = l;
  if (kcap > n) kcap = (int32_t)n;
  int32_t k = 0;
  for (int32_t j = 0; j < kcap; ++j) {
    /* residual norms, from scratch */
    double rest = 0.0, best = -1.0;
    int64_t piv = -1;
    for (int64_t c = 0; c < n; ++c) {
      if (!active[c]) continue;
      double nu = 0.0;
      for (int32_t i = 0; i < l; ++i) nu += W[i + (int64_t)l * c] * W[i + (int64_t)l * c];
      rest += nu;
      if (nu > best) { best = nu; piv = c; }   /* strict '>' keeps the lowest index on ties */
    }
    if (tol > 0.0 && rest <= tol * tol * normY2) break;
    if (piv < 0 || best <= 0.0) break;         /* nothing left to pivot on */
    double rjj = sqrt(best);
    R[(int64_t)j * n + piv] = rjj;
    for (int32_t i = 0; i < l; ++i) q[i] = W[i + (int64_t)l * piv] / rjj;
    active[piv] = 0;
    J[j] = (int32_t)piv;
    for (int32_t i = 0; i < l; ++i) W[i + (int64_t)l * piv] = 0.0;
    /* modified Gram-Schmidt: remove q_j from every remaining column now */
    for (int64_t c = 0; c < n; ++c) {
      if (!active[c]) continue;
      double* w = W + (int64_t)l * c;
      double rjc = 0.0;
      for (int32_t i = 0; i < l; ++i) rjc += q[i] * w[i];
      R[(int64_t)j * n + c] = rjc;
      for (int32_t i = 0; i < l; ++i) w[i] -= rjc * q[i];
    }
    /* entries R(j, J[p]) for pivots p < j were set when those columns were
     * still active; R(j, J[p]) for p > j are set here through 'active'. */
    k = j + 1;
  }
  free(active);
  free(q);
  return k;
}

/* Householder QR with column pivoting (Golub & Van Loan, Alg. 5.4.1), norms
 * recomputed from scratch at every step.  Cross-check for orc_qrcp_mgs: the
 * same pivots in exact arithmetic, R equal up to the sign of each row.
 * Same argument conventions as orc_qrcp_mgs. */
int orc_qrcp_householder(double* W, int32_t l, int64_t n, int32_t kmax, double tol,
                         int32_t* J, double* R, double* normY2_out) {
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)l);
  for (int64_t c = 0; c < n; ++c) perm[c] = c;
  for (int64_t x = 0; x < (int64_t)kmax * n; ++x) R[x] = 0.0;
  double normY2 = 0.0;
  for (int64_t c = 0; c < n; ++c)
    for (int32_t i = 0; i < l; ++i) normY2 += W[i + (int64_t)l * c] * W[i + (int64_t)l * c];
  if (normY2_out) *normY2_out = normY2;
  int32_t kcap = kmax;
  if (kcap > l) kcap = l;
  if (kcap > n) kcap = (int32_t)n;
  int32_t k = 0;
  for (int32_t j = 0; j < kcap; ++j) {
    double rest = 0.0, best = -1.0;
    int64_t pivpos = -1;
    for (int64_t pc = j; pc < n; ++pc) {
      double* w = W + (int64_t)l * pc;
      double nu = 0.0;
      for (int32_t i = j; i < l; ++i) nu += w[i] * w[i];
      rest += nu;
      if (nu > best || (nu == best && perm[pc] < perm[pivpos])) { best = nu; pivpos = pc; }
    }
    if (tol > 0.0 && rest <= tol * tol * normY2) break;
    if (pivpos < 0 || best <= 0.0) break;
    /* swap storage columns j and pivpos */
    if (pivpos != j) {
      for (int32_t i = 0; i < l; ++i) {
        double t = W[i + (int64_t)l * j];
        W[i + (int64_t)l * j] = W[i + (int64_t)l * pivpos];
        W[i + (int64_t)l * pivpos] = t;
      }
      int64_t tp = perm[j]; perm[j] = perm[pivpos]; perm[pivpos] = tp;
    }
    double* x = W + (int64_t)l * j;
    double norm = sqrt(best);
    double alpha = (x[j] >= 0.0) ? -norm : norm;   /* sign avoids cancellation */
    for (int32_t i = 0; i < l; ++i) v[i] = (i < j) ? 0.0 : x[i];
    v[j] -= alpha;
    double vtv = 0.0;
    for (int32_t i = j; i < l; ++i) vtv += v[i] * v[i];
    x[j] = alpha;
    for (int32_t i = j + 1; i < l; ++i) x[i] = 0.0;
    for (int64_t pc = j + 1; pc < n; ++pc) {
      double* w = W + (int64_t)l * pc;
      double s = 0.0;
      for (int32_t i = j; i < l; ++i) s += v[i] * w[i];
      double f = (vtv > 0.0) ? 2.0 * s / vtv : 0.0;
      for (int32_t i = j; i < l; ++i) w[i] -= f * v[i];
    }
    J[j] = (int32_t)perm[j];
    k = j + 1;
  }
  /* scatter the first k rows of the triangular factor to original numbering */
  for (int32_t j = 0; j < k; ++j)
    for (int64_t pc = j; pc < n; ++pc)
      R[(int64_t)j * n + perm[pc]] = W[j + (int64_t)l * pc];
  free(perm);
  free(v);
  return k;
}

/* Rank guard: number of leading pivots with |R_jj| > 2 u_mode |R_00|. */
int orc_rank_guard(const double* R, int64_t n, const int32_t* J, int32_t k, double u_mode) {
  if (k <= 0) return 0;
  double r00 = fabs(R[J[0]]);
  if (!(r00 > 0.0)) return 0;
  int32_t keff = 0;
  for (int32_t j = 0; j < k; ++j) {
    if (fabs(R[(int64_t)j * n + J[j]]) > 2.0 * u_mode * r00) keff = j + 1;
    else break;
  }
  return keff;
}

/* Coefficient matrix C = [I_k | R11^+ R12] Z^T (Section 2, Eq. for C;
 * Algorithm 1 steps 4-6), k x n row-major: C[p*n + c].
 * R11(i, p) = R(i, J[p]); for every non-pivoted column c, C(:, c) solves
 * R11 t = R(0:k, c) by back-substitution; C(:, J[p]) = e_p exactly. */
void orc_coefficients(const double* R, int64_t n, const int32_t* J, int32_t k, double* C) {
  char* piv = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  double* t = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  for (int32_t p = 0; p < k; ++p) piv[J[p]] = 1;
  for (int64_t c = 0; c < n; ++c) {
    if (piv[c]) continue;
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = R[(int64_t)i * n + c];
      for (int32_t p = i + 1; p < k; ++p) s -= R[(int64_t)i * n + J[p]] * t[p];
      t[i] = s / R[(int64_t)i * n + J[i]];
    }
    for (int32_t p = 0; p < k; ++p) C[(int64_t)p * n + c] = t[p];
  }
  for (int32_t p = 0; p < k; ++p)
    for (int32_t q = 0; q < k; ++q) C[(int64_t)p * n + J[q]] = (p == q) ? 1.0 : 0.0;
  free(piv);
  free(t);
}

/* Neumaier (improved Kahan) compensated accumulation. */
static void neu_add(double* s, double* comp, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *comp += (*s - t) + x;
  else *comp += (x - t) + *s;
  *s = t;
}

/* Reconstruction A_hat = A(:, J) C and the squared Frobenius norms of the
 * error A - A_hat and of A (Section 5.1, relative Frobenius error).
 * Ahat may be NULL.  C is k x n row-major as produced above. */
void orc_reconstruct_error(const double* A, int64_t m, int64_t n, int64_t ld,
                           const int32_t* J, int32_t k, const double* C,
                           double* Ahat, int64_t ldh, double* e2, double* a2) {
  double se = 0.0, ce = 0.0, sa = 0.0, ca = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t r = 0; r < m; ++r) {
      double ah = 0.0;
      for (int32_t p = 0; p < k; ++p) ah += A[r + ld * J[p]] * C[(int64_t)p * n + j];
      double a = A[r + ld * j];
      double e = a - ah;
      if (Ahat) Ahat[r + ldh * j] = ah;
      neu_add(&se, &ce, e * e);
      neu_add(&sa, &ca, a * a);
    }
  }
  *e2 = se + ce;
  *a2 = sa + ca;
}

/* Per-QoI errors of one subdomain (Section 5.1 reports the relative error of
 * each quantity of interest separately; Section 5.3 compresses each QoI of a
 * sub-domain on its own).  The rows of a box are ordered with the QoI
 * slowest, r = ((q ez + z) ey + y) ex + x, so QoI q is the row block
 * [q m / nq, (q + 1) m / nq) (m a multiple of nq).  e2[q] and a2[q] receive
 * ||A_q - A_hat_q||_F^2 and ||A_q||_F^2 of that block, with A_hat = A(:, J) C
 * formed exactly as in orc_reconstruct_error (Neumaier sums, columns outer). */
void orc_error_per_qoi(const double* A, int64_t m, int64_t n, int64_t ld, const int32_t* J,
                       int32_t k, const double* C, int32_t nq, double* e2, double* a2) {
  const int64_t mq = m / nq;
  for (int32_t q = 0; q < nq; ++q) {
    double se = 0.0, ce = 0.0, sa = 0.0, ca = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      for (int64_t r = q * mq; r < (q + 1) * mq; ++r) {
        double ah = 0.0;
        for (int32_t p = 0; p < k; ++p) ah += A[r + ld * J[p]] * C[(int64_t)p * n + j];
        double a = A[r + ld * j];
        double e = a - ah;
        neu_add(&se, &ce, e * e);
        neu_add(&sa, &ca, a * a);
      }
    }
    e2[q] = se + ce;
    a2[q] = sa + ca;
  }
}

/* Per-QoI totals over a batch whose subdomains each hold one QoI of a box
 * (Section 5.3: each QoI of each sub-domain compressed on its own):
 * ge2[g] = sum of e2[s] and ga2[g] = sum of a2[s] over the subdomains s with
 * qoi[s] == g, in subdomain order.  The relative error of QoI g over the
 * whole domain is sqrt(ge2[g] / ga2[g]) (Section 5.1). */
void orc_qoi_totals(int32_t num, const int32_t* qoi, const double* e2, const double* a2,
                    int32_t nqoi, double* ge2, double* ga2) {
  for (int32_t g = 0; g < nqoi; ++g) {
    ge2[g] = 0.0;
    ga2[g] = 0.0;
  }
  for (int32_t s = 0; s < num; ++s) {
    ge2[qoi[s]] += e2[s];
    ga2[qoi[s]] += a2[s];
  }
}

/* Compression factor, aggregated over subdomains (Section 2 Eq. for CF;
 * Section 3.2 aggregate over partitions): sum m_i n_i / sum k_i (s_i + n_i),
 * where s_i is the number of rows stored for part i (s = NULL: s_i = m_i;
 * a coarse-grid skeleton stores m_c rows, Section 5.2 subsampling). */
double orc_compression_factor(int32_t num, const int64_t* m, const int64_t* s_rows,
                              const int64_t* n, const int32_t* k) {
  double num_ = 0.0, den = 0.0;
  for (int32_t s = 0; s < num; ++s) {
    double stored = s_rows ? (double)s_rows[s] : (double)m[s];
    num_ += (double)m[s] * (double)n[s];
    den += (double)k[s] * (stored + (double)n[s]);
  }
  return den > 0.0 ? num_ / den : INFINITY;
}

int orc_spid_kqr(const double* A, int64_t m, int64_t n, int64_t ld, int32_t l, int32_t kmax,
                 double tol, double u_mode, uint64_t seed, double* Y, int32_t* J, int32_t* k_out,
                 int32_t* kqr_out, double* R, double* C, double* e2, double* a2);

/* Whole SPID on one subdomain: sketch, mgsqr with pivoting, rank guard,
 * coefficients, reconstruction error.  Outputs may be NULL except J, k_out,
 * C.  Y: l x n, R: kmax x n row-major, C: kmax x n row-major (rows >= k are
 * zero), J: kmax (entries >= k are -1). */
int orc_spid(const double* A, int64_t m, int64_t n, int64_t ld, int32_t l, int32_t kmax,
             double tol, double u_mode, uint64_t seed, double* Y, int32_t* J, int32_t* k_out,
             double* R, double* C, double* e2, double* a2) {
  return orc_spid_kqr(A, m, n, ld, l, kmax, tol, u_mode, seed, Y, J, k_out, NULL, R, C, e2, a2);
}

/* As orc_spid, and kqr_out (may be NULL) receives the number of pivots the
 * QR produced before the rank guard: the guard cut the rank (an informational
 * outcome of the rank guard) exactly when *k_out < *kqr_out. */
int orc_spid_kqr(const double* A, int64_t m, int64_t n, int64_t ld, int32_t l, int32_t kmax,
                 double tol, double u_mode, uint64_t seed, double* Y, int32_t* J, int32_t* k_out,
                 int32_t* kqr_out, double* R, double* C, double* e2, double* a2) {
  double* Yw = (double*)malloc(sizeof(double) * (size_t)l * (size_t)(n > 0 ? n : 1));
  double* Rw = (double*)malloc(sizeof(double) * (size_t)kmax * (size_t)(n > 0 ? n : 1));
  orc_sketch(A, m, n, ld, l, seed, Yw);
  if (Y) memcpy(Y, Yw, sizeof(double) * (size_t)l * (size_t)n);
  for (int32_t p = 0; p < kmax; ++p) J[p] = -1;
  double normY2 = 0.0;
  int32_t k = orc_qrcp_mgs(Yw, l, n, kmax, tol, J, Rw, &normY2);
  int32_t keff = orc_rank_guard(Rw, n, J, k, u_mode);
  for (int32_t p = keff; p < kmax; ++p) J[p] = -1;
  for (int64_t x = 0; x < (int64_t)kmax * n; ++x) C[x] = 0.0;
  orc_coefficients(Rw, n, J, keff, C);
  if (R) memcpy(R, Rw, sizeof(double) * (size_t)kmax * (size_t)n);
  if (e2 && a2) orc_reconstruct_error(A, m, n, ld, J, keff, C, NULL, 0, e2, a2);
  *k_out = keff;
  if (kqr_out) *kqr_out = k;
  free(Yw);
  free(Rw);
  return 0;
}

/* SPID over a batch of subdomains stored in one FP64 window: subdomain s is
 * the m[s] x n[s] column-major block at window + off[s] with leading
 * dimension ld[s].  Outputs are packed per subdomain: J at s*kmax, k at s,
 * C at kmax * coff[s] where coff[s] = sum_{s'<s} n[s'], Y (optional) at
 * l * coff[s], e2/a2 at s.  Subdomains are independent (Section 3.2) and run
 * in parallel over OpenMP threads. */
int orc_spid_batch(const double* window, int32_t num, const int64_t* m, const int64_t* n,
                   const int64_t* off, const int64_t* ld, int32_t l, int32_t kmax, double tol,
                   double u_mode, uint64_t seed, double* Y, int32_t* J, int32_t* k,
                   int32_t* kqr, double* C, double* e2, double* a2) {
  int64_t* coff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(num + 1));
  coff[0] = 0;
  for (int32_t s = 0; s < num; ++s) coff[s + 1] = coff[s] + n[s];
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t s = 0; s < num; ++s) {
    orc_spid_kqr(window + off[s], m[s], n[s], ld[s], l, kmax, tol, u_mode, seed,
                 Y ? Y + (int64_t)l * coff[s] : NULL, J + (int64_t)kmax * s, k + s,
                 kqr ? kqr + s : NULL, NULL, C + (int64_t)kmax * coff[s], e2 ? e2 + s : NULL,
                 a2 ? a2 + s : NULL);
  }
  free(coff);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Subsampled ID and single-pass ID on a coarse grid (Section 2, SubID and  */
/* SPID paragraphs, Algorithms 2 and 3; Section 5.2 subsampling study).     */
/* A subdomain is a box of nq QoIs x ez x ey x ex points whose rows are     */
/* ordered r = ((q ez + z) ey + y) ex + x.  B = A(J,:) keeps the points of a */
/* coarse grid with interval s along each axis; M interpolates the coarse   */
/* grid back onto the box (trilinear, Section 5.2).                         */
/* ------------------------------------------------------------------------ */

/* Coarse indices along one axis of e points with interval s >= 1:
 * 0, s, 2s, ... < e, and e - 1 appended when it is not one of them (reading:
 * the 64-point runs of Section 5.2 with intervals 3, 7 and 9 keep both ends
 * because 63 is a multiple of each; appending the end keeps that property for
 * every size, so M never extrapolates).  Returns the count; idx may be NULL. */
int orc_coarse_axis(int32_t e, int32_t s, int32_t* idx) {
  int32_t c = 0;
  for (int32_t x = 0; x < e; x += s) {
    if (idx) idx[c] = x;
    ++c;
  }
  if (e > 0 && (e - 1) % s != 0) {
    if (idx) idx[c] = e - 1;
    ++c;
  }
  return c;
}

/* Rows of the coarse matrix: nq * cz * cy * cx. */
int64_t orc_coarse_rows(const int32_t box[4], const int32_t stride[3]) {
  return (int64_t)box[0] * orc_coarse_axis(box[1], stride[0], NULL) *
         orc_coarse_axis(box[2], stride[1], NULL) * orc_coarse_axis(box[3], stride[2], NULL);
}

/* B = A(J, :): B is mc x n column-major (leading dimension mc), its rows in
 * (q, cz, cy, cx) order with cx fastest.  box = (nq, ez, ey, ex),
 * stride = (sz, sy, sx). */
void orc_subsample(const double* A, int64_t ld, int64_t n, const int32_t box[4],
                   const int32_t stride[3], double* B) {
  const int32_t nq = box[0], ez = box[1], ey = box[2], ex = box[3];
  int32_t* iz = (int32_t*)malloc(sizeof(int32_t) * (size_t)ez);
  int32_t* iy = (int32_t*)malloc(sizeof(int32_t) * (size_t)ey);
  int32_t* ix = (int32_t*)malloc(sizeof(int32_t) * (size_t)ex);
  const int32_t cz = orc_coarse_axis(ez, stride[0], iz);
  const int32_t cy = orc_coarse_axis(ey, stride[1], iy);
  const int32_t cx = orc_coarse_axis(ex, stride[2], ix);
  const int64_t mc = (int64_t)nq * cz * cy * cx;
  for (int64_t j = 0; j < n; ++j) {
    int64_t cr = 0;
    for (int32_t q = 0; q < nq; ++q)
      for (int32_t a = 0; a < cz; ++a)
        for (int32_t b = 0; b < cy; ++b)
          for (int32_t c = 0; c < cx; ++c, ++cr) {
            const int64_t r = (((int64_t)q * ez + iz[a]) * ey + iy[b]) * ex + ix[c];
            B[cr + mc * j] = A[r + ld * j];
          }
  }
  free(iz);
  free(iy);
  free(ix);
}

/* Coarse cell of fine coordinate x on one axis: lower coarse index position
 * a (idx[a] <= x, and a + 1 < count unless count == 1) and the weight of the
 * upper node, w = (x - idx[a]) / (idx[a+1] - idx[a]). */
static void coarse_cell(const int32_t* idx, int32_t count, int32_t x, int32_t* a, double* w) {
  if (count == 1) { *a = 0; *w = 0.0; return; }
  int32_t lo = 0;
  while (lo + 2 < count && idx[lo + 1] <= x) ++lo;
  *a = lo;
  *w = (double)(x - idx[lo]) / (double)(idx[lo + 1] - idx[lo]);
}

/* F = M G: trilinear interpolation of the coarse matrix G (mc x n, leading
 * dimension mc, rows as orc_subsample) onto the box (F m x n, leading
 * dimension ldf).  Per axis the fine point lies in coarse cell [X_a, X_a+1]
 * with upper weight w; the value is the sum over the 8 cell corners of
 * prod((1 - w) or w) times the corner value.  A fine point on a coarse node
 * gets that node's value. */
void orc_trilinear(const double* G, int64_t n, const int32_t box[4], const int32_t stride[3],
                   double* F, int64_t ldf) {
  const int32_t nq = box[0], ez = box[1], ey = box[2], ex = box[3];
  int32_t* iz = (int32_t*)malloc(sizeof(int32_t) * (size_t)ez);
  int32_t* iy = (int32_t*)malloc(sizeof(int32_t) * (size_t)ey);
  int32_t* ix = (int32_t*)malloc(sizeof(int32_t) * (size_t)ex);
  const int32_t cz = orc_coarse_axis(ez, stride[0], iz);
  const int32_t cy = orc_coarse_axis(ey, stride[1], iy);
  const int32_t cx = orc_coarse_axis(ex, stride[2], ix);
  const int64_t mc = (int64_t)nq * cz * cy * cx;
  for (int64_t j = 0; j < n; ++j) {
    const double* g = G + mc * j;
    for (int32_t q = 0; q < nq; ++q)
      for (int32_t z = 0; z < ez; ++z)
        for (int32_t y = 0; y < ey; ++y)
          for (int32_t x = 0; x < ex; ++x) {
            int32_t a, b, c;
            double wz, wy, wx;
            coarse_cell(iz, cz, z, &a, &wz);
            coarse_cell(iy, cy, y, &b, &wy);
            coarse_cell(ix, cx, x, &c, &wx);
            double v = 0.0;
            for (int32_t dz = 0; dz < 2; ++dz)
              for (int32_t dy = 0; dy < 2; ++dy)
                for (int32_t dx = 0; dx < 2; ++dx) {
                  const double w = (dz ? wz : 1.0 - wz) * (dy ? wy : 1.0 - wy) *
                                   (dx ? wx : 1.0 - wx);
                  if (w == 0.0) continue;   /* also keeps single-node axes in range */
                  const int64_t cr = (((int64_t)q * cz + a + dz) * cy + b + dy) * cx + c + dx;
                  v += w * g[cr];
                }
            const int64_t r = (((int64_t)q * ez + z) * ey + y) * ex + x;
            F[r + ldf * j] = v;
          }
  }
  free(iz);
  free(iy);
  free(ix);
}

/* SubID and SPID on one box (Algorithms 2 and 3): B = A(J,:); pivoted MGS QR
 * of B (orc_qrcp_mgs: norms from scratch, ties to the lowest index, adaptive
 * stop when tol > 0), rank guard with u_mode, C_B = [I | R11^-1 R12] Z^T.
 * Outputs: J (kmax, -1 past k), C (kmax x n row-major, zero rows past k),
 * Bskel = B(:, I_B) (mc x kmax column-major, may be NULL), and
 * err[0] = ||A - A(:,I_B) C_B||_F^2 (SubID), err[1] = ||A - M B(:,I_B) C_B||_F^2
 * (SPID), err[2] = ||A||_F^2, err[3] = mc.  Ahat (m x n, ld m, may be NULL)
 * receives the SPID reconstruction.  Returns k. */
int orc_subid(const double* A, int64_t ld, int64_t n, const int32_t box[4],
              const int32_t stride[3], int32_t kmax, double tol, double u_mode, int32_t* J,
              double* C, double* Bskel, double* err, double* Ahat) {
  const int64_t m = (int64_t)box[0] * box[1] * box[2] * box[3];
  const int64_t mc = orc_coarse_rows(box, stride);
  const int64_t nn = n > 0 ? n : 1;
  double* B = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  double* W = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  double* R = (double*)malloc(sizeof(double) * (size_t)kmax * (size_t)nn);
  orc_subsample(A, ld, n, box, stride, B);
  memcpy(W, B, sizeof(double) * (size_t)(mc * n));
  for (int32_t p = 0; p < kmax; ++p) J[p] = -1;
  double normB2 = 0.0;
  const int32_t k0 = orc_qrcp_mgs(W, (int32_t)mc, n, kmax, tol, J, R, &normB2);
  const int32_t k = orc_rank_guard(R, n, J, k0, u_mode);
  for (int32_t p = k; p < kmax; ++p) J[p] = -1;
  for (int64_t x = 0; x < (int64_t)kmax * n; ++x) C[x] = 0.0;
  orc_coefficients(R, n, J, k, C);
  if (Bskel)
    for (int32_t p = 0; p < kmax; ++p)
      for (int64_t cr = 0; cr < mc; ++cr) Bskel[cr + mc * p] = (p < k) ? B[cr + mc * J[p]] : 0.0;
  /* SubID: A(:, I_B) C_B */
  double e2s = 0.0, a2 = 0.0;
  orc_reconstruct_error(A, m, n, ld, J, k, C, NULL, 0, &e2s, &a2);
  /* SPID: M (B(:, I_B) C_B) -- interpolate the coarse reconstruction */
  double* G = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t cr = 0; cr < mc; ++cr) {
      double v = 0.0;
      for (int32_t p = 0; p < k; ++p) v += B[cr + mc * J[p]] * C[(int64_t)p * n + j];
      G[cr + mc * j] = v;
    }
  double* F = Ahat ? Ahat : (double*)malloc(sizeof(double) * (size_t)(m * nn));
  orc_trilinear(G, n, box, stride, F, m);
  double se = 0.0, ce = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      const double e = A[r + ld * j] - F[r + m * j];
      neu_add(&se, &ce, e * e);
    }
  err[0] = e2s;
  err[1] = se + ce;
  err[2] = a2;
  err[3] = (double)mc;
  if (!Ahat) free(F);
  free(G);
  free(B);
  free(W);
  free(R);
  return k;
}

/* SubID and SPID on an arbitrary point set (Section 2: rows of A in any
 * order, e.g. a flattened unstructured grid; Section 5.1's random points).
 * The coarse matrix keeps the listed rows, B = A(crow, :) (mc x n, row i =
 * A row crow[i]); M is given as a stencil of t (index, weight) pairs per fine
 * row: (M G)(r, j) = sum_q w[r t + q] G(idx[r t + q], j).  Otherwise as
 * orc_subid: pivoted MGS of B, rank guard, C_B, Bskel = B(:, I_B), err[0] =
 * ||A - A(:,I_B) C_B||^2, err[1] = ||A - M (B(:,I_B) C_B)||^2, err[2] =
 * ||A||^2, err[3] = mc; Ahat (m x n, may be NULL) the SPID reconstruction.
 * Returns k. */
int orc_subid_points(const double* A, int64_t m, int64_t ld, int64_t n, const int32_t* crow,
                     int64_t mc, int32_t t, const int32_t* idx, const double* w, int32_t kmax,
                     double tol, double u_mode, int32_t* J, double* C, double* Bskel,
                     double* err, double* Ahat) {
  const int64_t nn = n > 0 ? n : 1;
  double* B = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  double* W = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  double* R = (double*)malloc(sizeof(double) * (size_t)kmax * (size_t)nn);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < mc; ++i) B[i + mc * j] = A[crow[i] + ld * j];
  memcpy(W, B, sizeof(double) * (size_t)(mc * n));
  for (int32_t p = 0; p < kmax; ++p) J[p] = -1;
  double normB2 = 0.0;
  const int32_t k0 = orc_qrcp_mgs(W, (int32_t)mc, n, kmax, tol, J, R, &normB2);
  const int32_t k = orc_rank_guard(R, n, J, k0, u_mode);
  for (int32_t p = k; p < kmax; ++p) J[p] = -1;
  for (int64_t x = 0; x < (int64_t)kmax * n; ++x) C[x] = 0.0;
  orc_coefficients(R, n, J, k, C);
  if (Bskel)
    for (int32_t p = 0; p < kmax; ++p)
      for (int64_t i = 0; i < mc; ++i) Bskel[i + mc * p] = (p < k) ? B[i + mc * J[p]] : 0.0;
  double e2s = 0.0, a2 = 0.0;
  orc_reconstruct_error(A, m, n, ld, J, k, C, NULL, 0, &e2s, &a2);
  /* SPID: M (B(:, I_B) C_B) */
  double* G = (double*)malloc(sizeof(double) * (size_t)(mc * nn));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < mc; ++i) {
      double v = 0.0;
      for (int32_t p = 0; p < k; ++p) v += B[i + mc * J[p]] * C[(int64_t)p * n + j];
      G[i + mc * j] = v;
    }
  double se = 0.0, ce = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      double v = 0.0;
      for (int32_t q = 0; q < t; ++q) v += w[r * t + q] * G[idx[r * t + q] + mc * j];
      if (Ahat) Ahat[r + m * j] = v;
      const double e = A[r + ld * j] - v;
      neu_add(&se, &ce, e * e);
    }
  err[0] = e2s;
  err[1] = se + ce;
  err[2] = a2;
  err[3] = (double)mc;
  free(G);
  free(B);
  free(W);
  free(R);
  return k;
}

/* ------------------------------------------------------------------------ */
/* Modified (two-stage) SPID, Section 3.3.2 and Algorithm 6.                */
/* Stage 1: the n columns are cut into N blocks of nb = n / N; block b gets */
/* the sketched ID with target rank k (orc_spid, tol = 0): A_b ~ A_b(:,I_b) */
/* C_b.  Stage 2: A0' = [A_0(:,I_0) .. A_{N-1}(:,I_{N-1})] gets the         */
/* sketched ID with tolerance tol2 (rank cap k2max): A0' ~ A0'(:,J2) C1.    */
/* Final: C1' = C1 C0', C0' = blockdiag(C_0, .., C_{N-1}) (kN x n; the      */
/* printed size k(N-1) x N is read as kN x n, the size the product needs),  */
/* and J = I_U(J2), the window column of A0' column q = b k + p being       */
/* b nb + I_b(p).  A0' keeps k slots per block; a block whose rank guard    */
/* kept k_b < k pads with zero columns (never picked, C rows zero).         */
/* Outputs: J (k2max, -1 past k2), C (k2max x n row-major, zero rows past   */
/* k2), optional stage-1 Jb (N x k) / kb (N) / Cb (N x k x nb), stage-2 J2   */
/* (k2max) / C1 (k2max x N k); err = {e2, a2}.  Returns k2.                 */
/* ------------------------------------------------------------------------ */
int orc_two_stage(const double* A, int64_t m, int64_t n, int64_t ld, int32_t N, int32_t k,
                  int32_t p, int32_t k2max, double tol2, double u_mode, uint64_t seed,
                  int32_t* J, double* C, int32_t* Jb, int32_t* kb, double* Cb, int32_t* J2,
                  double* C1, double* err) {
  const int64_t nb = n / N;
  const int64_t n2 = (int64_t)N * k;
  int32_t* Jbw = (int32_t*)malloc(sizeof(int32_t) * (size_t)n2);
  int32_t* kbw = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  double* Cbw = (double*)malloc(sizeof(double) * (size_t)n2 * (size_t)nb);
  double* A0 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n2);
  int32_t* J2w = (int32_t*)malloc(sizeof(int32_t) * (size_t)k2max);
  double* C1w = (double*)malloc(sizeof(double) * (size_t)k2max * (size_t)n2);
  /* stage 1, block by block */
  for (int32_t b = 0; b < N; ++b) {
    orc_spid(A + ld * (b * nb), m, nb, ld, k + p, k, 0.0, u_mode, seed, NULL, Jbw + (int64_t)b * k,
             kbw + b, NULL, Cbw + (int64_t)b * k * nb, NULL, NULL);
  }
  /* A0': k slots per block, zero past k_b */
  for (int32_t b = 0; b < N; ++b)
    for (int32_t q = 0; q < k; ++q) {
      double* dst = A0 + m * ((int64_t)b * k + q);
      if (q < kbw[b]) {
        const double* src = A + ld * (b * nb + Jbw[(int64_t)b * k + q]);
        for (int64_t r = 0; r < m; ++r) dst[r] = src[r];
      } else {
        for (int64_t r = 0; r < m; ++r) dst[r] = 0.0;
      }
    }
  /* stage 2 with the tolerance */
  int32_t k2 = 0;
  orc_spid(A0, m, n2, m, k2max + p, k2max, tol2, u_mode, seed, NULL, J2w, &k2, NULL, C1w, NULL,
           NULL);
  /* composition C1' = C1 C0' and J = I_U(J2) */
  for (int32_t i = 0; i < k2max; ++i) {
    for (int64_t t = 0; t < n; ++t) {
      const int64_t b = t / nb, tt = t - b * nb;
      double acc = 0.0;
      if (i < k2)
        for (int32_t q = 0; q < k; ++q)
          acc += C1w[(int64_t)i * n2 + b * k + q] * Cbw[((int64_t)b * k + q) * nb + tt];
      C[(int64_t)i * n + t] = acc;
    }
    if (i < k2) {
      const int32_t q = J2w[i];
      J[i] = (int32_t)((q / k) * nb + Jbw[q]);
    } else {
      J[i] = -1;
    }
  }
  if (err) orc_reconstruct_error(A, m, n, ld, J, k2, C, NULL, 0, err, err + 1);
  if (Jb) memcpy(Jb, Jbw, sizeof(int32_t) * (size_t)n2);
  if (kb) memcpy(kb, kbw, sizeof(int32_t) * (size_t)N);
  if (Cb) memcpy(Cb, Cbw, sizeof(double) * (size_t)n2 * (size_t)nb);
  if (J2) memcpy(J2, J2w, sizeof(int32_t) * (size_t)k2max);
  if (C1) memcpy(C1, C1w, sizeof(double) * (size_t)k2max * (size_t)n2);
  free(Jbw);
  free(kbw);
  free(Cbw);
  free(A0);
  free(J2w);
  free(C1w);
  return k2;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
