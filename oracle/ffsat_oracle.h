/*
 * FP64 CPU oracle for the FastFourierSAT hot path — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The product path (the CUDA C-ABI library) never
 * calls it, shares no code with it, and fails when its own extension is
 * missing.
 *
 * Conventions (Preliminaries, "Walsh Expansions"): -1 is True, +1 is False.
 * A constraint c over L literals with values y_i = sigma_i * x_{v_i} is
 * symmetric: its truth depends only on s = number of True literals, written
 * v(s) in {-1 (satisfied), +1 (violated)}.  FE_c is its Walsh (multilinear)
 * expansion (Thm. "Walsh Transform"), F = sum_c w_c FE_c (Def. "Objective").
 *
 * Every routine is plain double precision and follows a definition from the
 * paper or from textbook mathematics; see each function's comment.
 */
#ifndef FFSAT_ORACLE_H
#define FFSAT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OR = 0, ORC_XOR = 1, ORC_ATLEAST = 2 };

/* v(s): constraint truth with s True literals (-1 satisfied, +1 violated). */
int orc_value(int type, int param, int L, int s);

/* Walsh coefficient f^(S) of Thm. "Walsh Transform" for the subset S given as a
 * bit mask over L <= 20 literals, by the 2^L corner sum of that theorem. */
double orc_walsh_subset(int type, int param, int L, uint32_t mask);

/* Walsh coefficients by subset size, a[m] = f^(S) for |S| = m (Eq. effi_eval:
 * WE_c = sum_m a_m e_m).  Computed by grouping the corner sum of Thm. "Walsh
 * Transform" by the number of True coordinates inside and outside S
 * (Krawtchouk form); exact integer binomials, valid for L <= 60. */
void orc_walsh_by_size(int type, int param, int L, double *a);

/* FE and dFE/dy_i by the Walsh expansion itself: sum over all 2^L subsets S of
 * f^(S) prod_{i in S} y_i, with f^(S) from the corner sum (L <= 12). */
double orc_fe_walsh_bruteforce(int type, int param, int L, const double *y, double *dy);

/* FE and gradient as the expectation over the 2^L cube corners z of
 * v(#True(z)) prod_i (1 + y_i z_i)/2 -- the multilinear extension written as
 * an expectation under independent rounding (L <= 20). */
double orc_fe_corners(int type, int param, int L, const double *y, double *dy);

/* Elementary symmetric polynomials e_0..e_L of y (Def. ESP), by the recurrence
 * e_m <- e_m + y_i e_{m-1}. */
void orc_esp(int L, const double *y, double *e);

/* FE = sum_m a_m e_m(y) (Eq. effi_eval) and dFE/dy_i = sum_m a_m e_{m-1}(y without i).
 * Accurate only for short constraints in FP64 (cancellation grows with L). */
double orc_fe_esp(int type, int param, int L, const double *y, double *dy);

/* Alg. 2 ("Forward Evaluation with FFT method") in complex double, N = L+1,
 * omega = exp(-2 pi i / N): gamma_i[j] = omega^j + y_i (Eq. forward),
 * gamma[j] = prod_i gamma_i[j] (Eq. reduction), WE = ftilde . gamma with
 * ftilde = fhat W^{-1}, fhat ordered [e_L .. e_0] (Eq. inverse).  The gradient
 * follows the chain rule of Prop. "Chain rule" / Eq. chain:
 * dWE/dy_i = sum_j ftilde_j prod_{l != i} gamma_l[j].  Short L only. */
double orc_fe_paper(int type, int param, int L, const double *y, double *dy);
/* ftilde of Eq. inverse (real and imaginary parts, N = L+1 entries). */
void orc_paper_ftilde(int type, int param, int L, double *re, double *im);

/* FE = sum_s v(s) P(S = s) for S = number of True literals under independent
 * rounding with P(literal True) = (1 - y_i)/2 (the probability reading of the
 * expansion, App. A.2), by the O(L^2) Poisson-binomial recurrence; gradient
 * dFE/dy_i = 1/2 sum_t P_{-i}(t) (v(t) - v(t+1)) through backward messages.
 * All forward terms are non-negative: stable for any L. */
double orc_fe_dp(int type, int param, int L, const double *y, double *dy);

/* Closed forms: a clause is -1 + 2 prod_i (1+y_i)/2 (footnote of App. B);
 * an XOR of parity p is (-1)^(p+1) prod_i y_i (App. B, Cor. "Reduction"). */
double orc_fe_or(int L, const double *y, double *dy);
double orc_fe_xor(int param, int L, const double *y, double *dy);

/* Dispatcher used for instance evaluation: closed forms for OR and XOR, the
 * stable recurrence for ATLEAST. */
double orc_fe(int type, int param, int L, const double *y, double *dy);

/* F(x_b) = sum_c w_c FE_c and g_b = grad F(x_b) for B points x [B, n] (row major).
 * lits are DIMACS signed 1-based.  nthreads <= 0 uses all OpenMP threads.
 * route: 0 = dispatcher (orc_fe), 1 = DP for every type, 2 = ESP, 3 = paper Alg. 2.
 * Returns 0, or -1 on bad input (variable out of range, NaN in x). */
int orc_eval_grad(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                  const uint8_t *type, const int32_t *param, const double *w,
                  int32_t B, const double *x, double *f, double *g, int nthreads, int route);

/* Condition scales of the sums above, used for tolerances: sf[b] = sum_c w_c |FE_c(x_b)|
 * and A[b, v] = sum_{c contains v} w_c max(|dFE_c/dy_v|, floor_c), where floor_c =
 * floor for constraints whose type bit is set in floor_types (bit t for type t)
 * and 0 otherwise.  Returns 0 or -1. */
int orc_eval_scale(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                   const uint8_t *type, const int32_t *param, const double *w,
                   int32_t B, const double *x, double *sf, double *A, double floor, int floor_types,
                   int nthreads);

/* Exact checker twin (Alg. 1, line 5, read as an exact test): z = sgn(x) with
 * sgn(x) = -1 iff x < 0 (so +-0 -> +1); every constraint is evaluated on z with
 * integer counting; n_unsat[b] = number of violated constraints, sat[b] = (n_unsat == 0).
 * Returns 0, or -1 if any x is NaN. */
int orc_check(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
              const uint8_t *type, const int32_t *param,
              int32_t B, const double *x, uint8_t *sat, int32_t *n_unsat, int nthreads);

/* U[c] = number of the B points whose sign vector violates constraint c (the
 * unsatisfaction count of the weighting heuristic, Sec. "Weighting Heuristics"). */
int orc_unsat_counts(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                     const uint8_t *type, const int32_t *param, int32_t B, const double *x, int32_t *U);

/* Prop. "Adaptive weight": r_c = U_c / max_c U_c (0 when every U_c is 0),
 * w_c <- (1 - alpha) w_c + alpha r_c, in place. */
void orc_erwa(int32_t m, const int32_t *U, double alpha, double *w);

/* splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then the
 * published output mix.  Returns the output for the given pre-increment state. */
uint64_t orc_splitmix64(uint64_t state);
/* Uniform restart draw for (seed, epoch, point b, variable v), with
 * S(t) = orc_splitmix64(t):  h = S(S(S(S(seed) ^ epoch) ^ b) ^ v);
 * value = ((h >> 40) - 2^23) / 2^23, a 24-bit grid on [-1, 1) that is exact
 * in both float and double. */
double orc_uniform(uint64_t seed, uint64_t epoch, uint64_t b, uint64_t v);

/* One outer round of Alg. 1 with the paper's projected-gradient fixed-point
 * update (App. A.3, Alg. "PGFP") and a FISTA line search (Beck and Teboulle,
 * backtracking variant), per point:
 *   y_1 = x_0, t_1 = 1, eta = eta0; for k = 1..T:
 *     g = grad F(y_k); find eta <- eta * beta^i (i >= 0, at most maxls trials,
 *       the last trial accepted if none passes) with
 *       F(p) <= F(y_k) + <g, p - y_k> + ||p - y_k||^2 / (2 eta) + slack,
 *       p = clip(y_k - eta g, -1, 1);
 *     x_k = p; t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
 *     y_{k+1} = clip(x_k + (t_k - 1) / t_{k+1} (x_k - x_{k-1}), -1, 1);
 *     stop once eta < eta_min (the paper's 1e-12).
 * x holds x_0 on entry and the last iterate on return; then the exact check and
 * the uniform restart as in orc_step.  iters[b] (optional) receives the
 * iterations taken and eta_out[b] (optional) the final step size.  Returns 0,
 * or -1 on bad input or parameters. */
int orc_step_pgfp(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                  const uint8_t *type, const int32_t *param, const double *w,
                  int32_t B, double *x, int32_t T, double eta0, double beta, int32_t maxls,
                  double eta_min, double slack,
                  uint64_t seed, uint64_t epoch, uint64_t b_offset, int restart,
                  uint8_t *solved, int32_t *n_unsat, int32_t *iters, double *eta_out, int nthreads);

/* Rephasing (Sec. "Rephasing Heuristics"): every point b with solved == NULL or
 * solved[b] == 0 takes phase 0 = original (x_b kept), 1 = flipped (x_b = -x_b)
 * or 2 = random (x_b[v] = orc_uniform(seed, epoch, b_offset + b, v)).
 * Returns 0, or -1 for an unknown phase. */
int orc_rephase(int32_t n, int32_t B, double *x, int phase, const uint8_t *solved,
                uint64_t seed, uint64_t epoch, uint64_t b_offset);

/* One outer round of Alg. 1 with fixed-step projected gradient descent
 * (App. A.3, Alg. "PGFP" without the line search): T times
 * x <- clip(x - lr * grad F(x), -1, 1); then the exact check; solved points keep
 * x, unsolved points restart at orc_uniform(seed, epoch, b_offset + b, v).
 * Returns 0 or -1 on bad input. */
int orc_step(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
             const uint8_t *type, const int32_t *param, const double *w,
             int32_t B, double *x, int32_t T, double lr,
             uint64_t seed, uint64_t epoch, uint64_t b_offset, int restart,
             uint8_t *solved, int32_t *n_unsat, int nthreads);

/* Number of OpenMP threads the library would use for nthreads <= 0. */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
