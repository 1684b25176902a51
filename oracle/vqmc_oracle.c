/*
 * vqmc_oracle.c -- plain, slow, FP64 CPU oracle for the VQMC hot path of
 * "Overcoming barriers to scalability in variational quantum Monte Carlo"
 * (Zhao, Stokes, Veerapaneni et al., arXiv 2106.13308).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it.  The CUDA library never calls it
 * and shares no code, header, table or constant generator with it.
 *
 * Every function states the passage it follows.  Notation is the paper's:
 *   n spins, h hidden units, spins s_i in {-1,+1} (Algorithm 1 draws y_i in
 *   {+-1}), MADE layer (Sec. 2.3):
 *       g1 = act((M1 . W1) s + b1),   W1: h x n   (row k = hidden unit k)
 *       z  = (M2 . W2) g1 + b2,       W2: n x h   (row i = output i)
 *       pi(s) = prod_i pi_i(s_i | s_<i),  pi_i(+1 | s_<i) = sigma(z_i).
 *   The paper's hidden activation is the rectifier; the logistic sigmoid is
 *   the alternative activation selected with act = 1.
 *
 * Reduced precision.  The paper states no arithmetic precision; reduced
 * precision is an option of the library under test, not a step of the
 * paper's method.  The library's BF16 model is defined here as: weights
 * rounded to bfloat16, each hidden activation g1_k rounded to bfloat16 before
 * the output layer, everything else exact.  The library's samplers and its
 * log-prob/adjoint GEMMs all evaluate this one model, so the score-function
 * estimator stays unbiased for the distribution that is actually sampled.
 * act | VO_HIDDEN_BF16 selects the rounding of g1; the weights are rounded by
 * the caller.  How far this model lies from the exact model of the FP32
 * master weights (the quantisation error) is measured by the tests against
 * the exact model (act without VO_HIDDEN_BF16), not assumed.
 *
 * Masks (the paper only asks for "appropriate binary masks", Sec. 2.3; the
 * reading used here is the standard MADE degree rule with sorted degrees):
 *   hidden unit k (0-based) has degree m(k) = 1 + floor(k (n-1) / h);
 *   M1[k][j] = 1 iff m(k) >= j  (1-based input j),
 *   M2[i][k] = 1 iff i > m(k)   (1-based output i).
 *
 * Diagonal Ising energy (the diagonal of Eq. (hamiltonian), with the Max-Cut
 * weights placed directly on the couplings so that minimising E maximises
 * the cut):  E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.
 *
 * Floating point is IEEE double throughout; compile without -ffast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- degrees */

/* Degree of hidden unit k: m(k) = 1 + floor(k (n-1) / h)  (MADE, Sec. 2.3). */
long vo_degree(long k, long n, long h) { return 1 + (k * (n - 1)) / h; }

int vo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------- Philox4x32 */

/* Philox4x32-10 counter-based generator, from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11, Sec. 4.2): each round computes the two 32x32->64 products of
 * (c0, c2) with the round multipliers and permutes/xors the halves with the
 * remaining words and the round key; the key advances by the Weyl constants
 * between rounds. */
void vo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The i.i.d. uniforms that Algorithm 1 transforms into a sample (Sec. 4: exact
 * samples are obtained "by transforming i.i.d. samples").  The uniform for
 * spin i of sample b in iteration `iter` is word (i mod 4) of
 * Philox4x32-10(counter = (floor(i/4), b, iter_lo, iter_hi), key = seed),
 * mapped to [0,1) as (x >> 8) * 2^-24. */
void vo_uniforms(int B, int n, uint64_t seed, uint64_t iter, float* u) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    for (int i = 0; i < n; ++i) {
      uint32_t ctr[4] = {(uint32_t)(i / 4), (uint32_t)b, (uint32_t)iter, (uint32_t)(iter >> 32)};
      uint32_t out[4];
      vo_philox4x32_10(ctr, key, out);
      u[(size_t)b * n + i] = (float)((double)(out[i % 4] >> 8) * (1.0 / 16777216.0));
    }
  }
}

/* ------------------------------------------------------------ primitives */

static double sigmoid(double t) { return 1.0 / (1.0 + exp(-t)); }

/* log sigma(t), evaluated without overflow. */
static double log_sigmoid(double t) {
  if (t >= 0) return -log1p(exp(-t));
  return t - log1p(exp(t));
}

#define VO_HIDDEN_BF16 2

/* x rounded to the nearest bfloat16 value (IEEE binary32 exponent range, 8
 * significant bits, ties to even; subnormals keep the fixed spacing 2^-133).
 * rint rounds ties to even in the default rounding mode. */
double vo_round_bf16(double x) {
  if (x == 0.0 || isnan(x) || isinf(x)) return x;
  int e;
  frexp(x, &e);          /* |x| = f 2^e, f in [0.5, 1) */
  int q = e - 8;         /* spacing of 8-bit significands at this binade */
  if (q < -133) q = -133;
  return ldexp(rint(ldexp(x, -q)), q);
}

static double act_f(int act, double a) {
  double g = (act & 1) == 0 ? (a > 0 ? a : 0.0) : sigmoid(a);
  return (act & VO_HIDDEN_BF16) ? vo_round_bf16(g) : g;
}

/* derivative of the activation at pre-activation a (ReLU'(0) = 0); the
 * bfloat16 rounding of g1 is not differentiated (it is the identity up to
 * rounding). */
static double act_d(int act, double a) {
  if ((act & 1) == 0) return a > 0 ? 1.0 : 0.0;
  double g = sigmoid(a);
  return g * (1.0 - g);
}

/* ------------------------------------------------------------ MADE forward */

/* One MADE forward pass (Sec. 2.3): a = (M1 . W1) s + b1, g1 = act(a),
 * z = (M2 . W2) g1 + b2.  Writes the pre-activations a (h, may be NULL) and
 * the logits z (n).  pi_i(+1 | s_<i) = sigma(z_i). */
void vo_forward(int n, int h, int act, const double* W1, const double* b1, const double* W2,
                const double* b2, const int8_t* s, double* a_out, double* z_out) {
  double* g = (double*)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
  for (int k = 0; k < h; ++k) {
    long mk = vo_degree(k, n, h);
    double a = b1[k];
    for (int j = 1; j <= n; ++j)
      if (mk >= j) a += W1[(size_t)k * n + (j - 1)] * (double)s[j - 1];
    if (a_out) a_out[k] = a;
    g[k] = act_f(act, a);
  }
  for (int i = 1; i <= n; ++i) {
    double z = b2[i - 1];
    for (int k = 0; k < h; ++k)
      if (i > vo_degree(k, n, h)) z += W2[(size_t)(i - 1) * h + k] * g[k];
    z_out[i - 1] = z;
  }
  free(g);
}

/* log pi(s) = sum_i log pi_i(s_i | s_<i) = sum_i log sigma(s_i z_i)
 * (autoregressive factorisation, Sec. 2.3), for a batch of B samples. */
void vo_logprob(int B, int n, int h, int act, const double* W1, const double* b1, const double* W2,
                const double* b2, const int8_t* S, double* logp) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    const int8_t* s = S + (size_t)b * n;
    vo_forward(n, h, act, W1, b1, W2, b2, s, NULL, z);
    double lp = 0.0;
    for (int i = 0; i < n; ++i) lp += log_sigmoid((double)s[i] * z[i]);
    logp[b] = lp;
    free(z);
  }
}

/* All n logits z_i(s) of each sample (one forward pass each). */
void vo_logits(int B, int n, int h, int act, const double* W1, const double* b1, const double* W2,
               const double* b2, const int8_t* S, double* Z) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b)
    vo_forward(n, h, act, W1, b1, W2, b2, S + (size_t)b * n, NULL, Z + (size_t)b * n);
}

/* ---------------------------------------------------------------- sampling */

/* Algorithm 1 (autoregressive sampling), taken literally: for i = 1..n run a
 * full forward pass on the current state x^{i-1} (x^0 = all +1; the masks make
 * the unset entries irrelevant), read pi_i(+1 | x_<i) = sigma(z_i), draw
 * y_i = +1 iff u_{b,i} < sigma(z_i) (else -1) and set x_i = y_i.
 * Cost O(h n^2) per sample.  Also returns log pi(x*) accumulated on the way. */
void vo_sample_literal(int B, int n, int h, int act, const double* W1, const double* b1,
                       const double* W2, const double* b2, const float* U, int8_t* S, double* logp) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    int8_t* x = S + (size_t)b * n;
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) x[i] = 1;
    double lp = 0.0;
    for (int i = 1; i <= n; ++i) {
      vo_forward(n, h, act, W1, b1, W2, b2, x, NULL, z);
      double p = sigmoid(z[i - 1]);
      double u = (double)U[(size_t)b * n + (i - 1)];
      int8_t y = (u < p) ? 1 : -1;
      x[i - 1] = y;
      lp += log_sigmoid((double)y * z[i - 1]);
    }
    if (logp) logp[b] = lp;
    free(z);
  }
}

/* Algorithm 1 with each forward pass restricted to what step i reads.  Only
 * hidden units with m(k) < i feed z_i, and those units' inputs j <= m(k) are
 * all drawn already, so the pre-activations a_k = b1_k + sum_{j<=m(k)} W1_kj s_j
 * can be kept and extended by one term as each spin is drawn:
 *   z_i = b2_i + sum_{k: m(k) < i} W2_ik act(a_k);  draw s_i;
 *   a_k += W1_{k i} s_i  for every k with m(k) >= i.
 * Same conditionals as vo_sample_literal, cost O(h n) per sample. */
void vo_sample_incremental(int B, int n, int h, int act, const double* W1, const double* b1,
                           const double* W2, const double* b2, const float* U, int8_t* S,
                           double* logp) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    int8_t* x = S + (size_t)b * n;
    double* a = (double*)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    long* m = (long*)malloc(sizeof(long) * (size_t)(h > 0 ? h : 1));
    for (int k = 0; k < h; ++k) {
      a[k] = b1[k];
      m[k] = vo_degree(k, n, h);
    }
    double lp = 0.0;
    for (int i = 1; i <= n; ++i) {
      double z = b2[i - 1];
      for (int k = 0; k < h; ++k)
        if (m[k] < i) z += W2[(size_t)(i - 1) * h + k] * act_f(act, a[k]);
      double p = sigmoid(z);
      double u = (double)U[(size_t)b * n + (i - 1)];
      int8_t y = (u < p) ? 1 : -1;
      x[i - 1] = y;
      lp += log_sigmoid((double)y * z);
      for (int k = 0; k < h; ++k)
        if (m[k] >= i) a[k] += W1[(size_t)k * n + (i - 1)] * (double)y;
    }
    if (logp) logp[b] = lp;
    free(a);
    free(m);
  }
}

/* ---------------------------------------------------------- local energies */

/* Diagonal local energy l(s) = (H psi)(s)/psi(s) = H_ss for a diagonal H
 * (Sec. 2.1 and Eq. (e:tim) with alpha = 0):
 *   E(s) = sum_{(i,j) in E, i<j} J_ij s_i s_j + sum_i h_i s_i.
 * The couplings are given as the strict upper triangle in CSR form: row i
 * lists its neighbours j > i.  field may be NULL (h = 0). */
void vo_energy_sparse(int B, int n, const int* row_ptr, const int* col, const double* w,
                      const double* field, const int8_t* S, double* E) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    const int8_t* s = S + (size_t)b * n;
    double e = 0.0;
    for (int i = 0; i < n; ++i)
      for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) e += w[p] * (double)s[i] * (double)s[col[p]];
    if (field)
      for (int i = 0; i < n; ++i) e += field[i] * (double)s[i];
    E[b] = e;
  }
}

/* Same energy with a dense symmetric coupling matrix J (n x n, zero diagonal):
 * E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i. */
void vo_energy_dense(int B, int n, const double* J, const double* field, const int8_t* S, double* E) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    const int8_t* s = S + (size_t)b * n;
    double e = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) e += J[(size_t)i * n + j] * (double)s[i] * (double)s[j];
    if (field)
      for (int i = 0; i < n; ++i) e += field[i] * (double)s[i];
    E[b] = e;
  }
}

/* Off-diagonal part of the local energy of the transverse-field Ising model,
 * Eq. (hamiltonian): the term -sum_i alpha_i X_i joins x to the n states x^(i)
 * that differ from x in spin i only (matrix entries, Eq. (e:tim):
 * H_{x, x^(i)} = -alpha_i).  With the wave function psi = sqrt(pi) of the
 * autoregressive model (Sec. 2.1), the local energy sum_y H_xy psi(y)/psi(x)
 * gets from these entries
 *     E_off(x) = -sum_i alpha_i sqrt(pi(x^(i)) / pi(x))
 *              = -sum_i alpha_i exp((log pi(x^(i)) - log pi(x)) / 2),
 * each log pi(x^(i)) one more full forward pass (n + 1 per sample).  The
 * diagonal part (-beta_i Z_i, -beta_ij Z_i Z_j) is an Ising energy as above,
 * with J_ij = -beta_ij and h_i = -beta_i. */
static double logprob_one(int n, int h, int act, const double* W1, const double* b1, const double* W2,
                          const double* b2, const int8_t* s, double* z) {
  vo_forward(n, h, act, W1, b1, W2, b2, s, NULL, z);
  double lp = 0.0;
  for (int i = 0; i < n; ++i) lp += log_sigmoid((double)s[i] * z[i]);
  return lp;
}

void vo_energy_tim_offdiag(int B, int n, int h, int act, const double* W1, const double* b1, const double* W2,
                           const double* b2, const double* alpha, const int8_t* S, double* E) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int8_t* t = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
    memcpy(t, S + (size_t)b * n, (size_t)n);
    const double lp0 = logprob_one(n, h, act, W1, b1, W2, b2, t, z);
    double e = 0.0;
    for (int i = 0; i < n; ++i) {
      t[i] = (int8_t)(-t[i]);
      const double lpi = logprob_one(n, h, act, W1, b1, W2, b2, t, z);
      t[i] = (int8_t)(-t[i]);
      e -= alpha[i] * exp(0.5 * (lpi - lp0));
    }
    E[b] = e;
    free(t);
    free(z);
  }
}

/* Cut value of the partition given by s: sum over edges of w_ij [s_i != s_j]
 * (Max-Cut, Sec. 2.4), counted directly from the edge list. */
void vo_cut(int B, int n, const int* row_ptr, const int* col, const double* w, const int8_t* S,
            double* cut) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < B; ++b) {
    const int8_t* s = S + (size_t)b * n;
    double c = 0.0;
    for (int i = 0; i < n; ++i)
      for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
        if (s[i] != s[col[p]]) c += w[p];
    cut[b] = c;
  }
}

/* Largest cut over all 2^n partitions (n <= 30), by enumeration with s_n
 * fixed to +1 (cut(s) = cut(-s)). */
double vo_maxcut_bruteforce(int n, const int* row_ptr, const int* col, const double* w) {
  if (n <= 1) return 0.0;
  long long total = 1LL << (n - 1);
  double best = -1e300;
#pragma omp parallel
  {
    double local = -1e300;
    int8_t* s = (int8_t*)malloc((size_t)n);
#pragma omp for schedule(static)
    for (long long x = 0; x < total; ++x) {
      for (int i = 0; i < n - 1; ++i) s[i] = ((x >> i) & 1) ? -1 : 1;
      s[n - 1] = 1;
      double c = 0.0;
      for (int i = 0; i < n; ++i)
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
          if (s[i] != s[col[p]]) c += w[p];
      if (c > local) local = c;
    }
#pragma omp critical
    if (local > best) best = local;
    free(s);
  }
  return best;
}

/* ------------------------------------------------------------- statistics */

/* Batch statistics of the local energies (Eq. (e:vmc) and Eq.
 * (eq:stochastic_variance) estimated on the batch): mean L = sum E_b / B,
 * var = sum (E_b - L)^2 / B, min, max; and the per-sample coefficients of the
 * score-function estimator c_b = (E_b - L) / B (baseline = batch mean).
 * out4 = {mean, var, min, max}; coef may be NULL. */
void vo_stats(int B, const double* E, double* out4, double* coef) {
  double sum = 0.0, mn = 1e300, mx = -1e300;
  for (int b = 0; b < B; ++b) {
    sum += E[b];
    if (E[b] < mn) mn = E[b];
    if (E[b] > mx) mx = E[b];
  }
  double mean = B > 0 ? sum / B : 0.0;
  double ss = 0.0;
  for (int b = 0; b < B; ++b) ss += (E[b] - mean) * (E[b] - mean);
  out4[0] = mean;
  out4[1] = B > 0 ? ss / B : 0.0;
  out4[2] = mn;
  out4[3] = mx;
  if (coef)
    for (int b = 0; b < B; ++b) coef[b] = (E[b] - mean) / B;
}

/* --------------------------------------------------------------- gradient */

/* Accumulates sum_b coef_b * grad_theta log pi(s_b) into (dW1, db1, dW2, db2)
 * for one sample, by the chain rule through the MADE layer of Sec. 2.3:
 *   d log pi / d z_i = s_i sigma(-s_i z_i)
 *   dW2_ik += dz_i g1_k M2_ik,   db2_i += dz_i
 *   dg1_k   = sum_i M2_ik W2_ik dz_i,   da_k = dg1_k act'(a_k)
 *   dW1_kj += da_k s_j M1_kj,    db1_k += da_k. */
static void grad_one(int n, int h, int act, const double* W1, const double* b1, const double* W2,
                     const double* b2, const int8_t* s, double c, double* dW1, double* db1,
                     double* dW2, double* db2, double* a, double* z, double* dz) {
  vo_forward(n, h, act, W1, b1, W2, b2, s, a, z);
  for (int i = 1; i <= n; ++i) {
    double si = (double)s[i - 1];
    dz[i - 1] = c * si * sigmoid(-si * z[i - 1]);
  }
  for (int i = 1; i <= n; ++i) {
    db2[i - 1] += dz[i - 1];
    for (int k = 0; k < h; ++k)
      if (i > vo_degree(k, n, h)) dW2[(size_t)(i - 1) * h + k] += dz[i - 1] * act_f(act, a[k]);
  }
  for (int k = 0; k < h; ++k) {
    long mk = vo_degree(k, n, h);
    double dg = 0.0;
    for (int i = 1; i <= n; ++i)
      if (i > mk) dg += W2[(size_t)(i - 1) * h + k] * dz[i - 1];
    double da = dg * act_d(act, a[k]);
    db1[k] += da;
    for (int j = 1; j <= n; ++j)
      if (mk >= j) dW1[(size_t)k * n + (j - 1)] += da * (double)s[j - 1];
  }
}

/* g = sum_b coef_b grad_theta log pi(s_b).  With coef_b = (E_b - L)/B this is
 * the batch estimate of grad L = E[(l - L) grad log pi] (Sec. 2.1: grad L =
 * 2 E[(l - L) grad log|psi|] with psi = sqrt(pi), Sec. 2.3).  Samples are
 * split into one fixed contiguous chunk per thread and the per-chunk sums are
 * added in chunk order, so the result depends only on the thread count. */
void vo_logprob_grad(int B, int n, int h, int act, const double* W1, const double* b1,
                     const double* W2, const double* b2, const int8_t* S, const double* coef,
                     double* dW1, double* db1, double* dW2, double* db2) {
  size_t nW1 = (size_t)h * n, nW2 = (size_t)n * h;
  memset(dW1, 0, sizeof(double) * nW1);
  memset(db1, 0, sizeof(double) * (size_t)h);
  memset(dW2, 0, sizeof(double) * nW2);
  memset(db2, 0, sizeof(double) * (size_t)n);
  int T = vo_num_threads();
  if (T > B) T = B > 0 ? B : 1;
  size_t per = nW1 + (size_t)h + nW2 + (size_t)n;
  double* acc = (double*)calloc((size_t)T * per, sizeof(double));
#pragma omp parallel for schedule(static, 1) num_threads(T)
  for (int t = 0; t < T; ++t) {
    double* g = acc + (size_t)t * per;
    double* a = (double*)malloc(sizeof(double) * (size_t)(h > 0 ? h : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* dz = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int b0 = (int)((long long)B * t / T), b1e = (int)((long long)B * (t + 1) / T);
    for (int b = b0; b < b1e; ++b)
      grad_one(n, h, act, W1, b1, W2, b2, S + (size_t)b * n, coef[b], g, g + nW1, g + nW1 + h,
               g + nW1 + h + nW2, a, z, dz);
    free(a);
    free(z);
    free(dz);
  }
  for (int t = 0; t < T; ++t) {
    const double* g = acc + (size_t)t * per;
    for (size_t q = 0; q < nW1; ++q) dW1[q] += g[q];
    for (int q = 0; q < h; ++q) db1[q] += g[nW1 + q];
    for (size_t q = 0; q < nW2; ++q) dW2[q] += g[nW1 + h + q];
    for (int q = 0; q < n; ++q) db2[q] += g[nW1 + h + nW2 + q];
  }
  free(acc);
}

/* ------------------------------------------------------------------- Adam */

/* One Adam step (the paper's default optimiser, Sec. 5.1, lr 0.01), with the
 * usual bias correction at step t >= 1 and no weight decay:
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 *   theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void vo_adam(long d, double* theta, double* m, double* v, const double* g, int t, double lr,
             double beta1, double beta2, double eps) {
  double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
  for (long q = 0; q < d; ++q) {
    m[q] = beta1 * m[q] + (1.0 - beta1) * g[q];
    v[q] = beta2 * v[q] + (1.0 - beta2) * g[q] * g[q];
    double mh = m[q] / bc1, vh = v[q] / bc2;
    theta[q] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------ enumeration */

/* Exact expectations by summing over all 2^n states (n <= 24): with
 * p(s) = exp(log pi(s)),
 *   out[0] = sum_s p(s)                  (= 1 by normalisation, Sec. 2.3)
 *   out[1] = L = sum_s p(s) E(s)         (Eq. (e:vmc))
 *   out[2] = var = sum_s p(s) (E(s) - L)^2   (Eq. (eq:stochastic_variance))
 * and, when grads is non-NULL, the exact gradient
 *   grad L = sum_s p(s) (E(s) - L) grad log pi(s)     (Sec. 2.1)
 * written as (dW1 | db1 | dW2 | db2).  State x maps to s_i = 1 - 2 x_i with
 * x_i the bit i-1 of x.  The energy is the sparse form (J in CSR). */
void vo_enumerate(int n, int h, int act, const double* W1, const double* b1, const double* W2,
                  const double* b2, const int* row_ptr, const int* col, const double* w,
                  const double* field, double* out, double* grads) {
  long long N = 1LL << n;
  double* lp = (double*)malloc(sizeof(double) * (size_t)N);
  double* E = (double*)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel
  {
    int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(static)
    for (long long x = 0; x < N; ++x) {
      for (int i = 0; i < n; ++i) s[i] = (int8_t)(1 - 2 * ((x >> i) & 1));
      vo_forward(n, h, act, W1, b1, W2, b2, s, NULL, z);
      double l = 0.0;
      for (int i = 0; i < n; ++i) l += log_sigmoid((double)s[i] * z[i]);
      lp[x] = l;
      double e = 0.0;
      for (int i = 0; i < n; ++i)
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) e += w[p] * (double)s[i] * (double)s[col[p]];
      if (field)
        for (int i = 0; i < n; ++i) e += field[i] * (double)s[i];
      E[x] = e;
    }
    free(s);
    free(z);
  }
  double Z = 0.0, L = 0.0;
  for (long long x = 0; x < N; ++x) {
    double p = exp(lp[x]);
    Z += p;
    L += p * E[x];
  }
  double var = 0.0;
  for (long long x = 0; x < N; ++x) var += exp(lp[x]) * (E[x] - L) * (E[x] - L);
  out[0] = Z;
  out[1] = L;
  out[2] = var;
  if (grads) {
    int8_t* S = (int8_t*)malloc((size_t)N * (size_t)n);
    double* c = (double*)malloc(sizeof(double) * (size_t)N);
    for (long long x = 0; x < N; ++x) {
      for (int i = 0; i < n; ++i) S[(size_t)x * n + i] = (int8_t)(1 - 2 * ((x >> i) & 1));
      c[x] = exp(lp[x]) * (E[x] - L);
    }
    size_t nW1 = (size_t)h * n;
    vo_logprob_grad((int)N, n, h, act, W1, b1, W2, b2, S, c, grads, grads + nW1, grads + nW1 + h,
                    grads + nW1 + h + (size_t)n * h);
    free(S);
    free(c);
  }
  free(lp);
  free(E);
}
