/*
 * FP64 CPU oracle for the FastFourierSAT hot path — TEST INFRASTRUCTURE ONLY.
 * See ffsat_oracle.h for what each routine computes and which passage of the
 * paper it follows.  Nothing here is shared with the CUDA library.
 */
#include "ffsat_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Constraint truth table v(s)                                              */
/* ------------------------------------------------------------------------ */

int orc_value(int type, int param, int L, int s) {
    (void)L;
    switch (type) {
    case ORC_OR: /* clause: True as soon as one literal is True */
        return s >= 1 ? -1 : 1;
    case ORC_XOR: /* parity constraint: True iff #True = param (mod 2) */
        return ((s & 1) == (param & 1)) ? -1 : 1;
    case ORC_ATLEAST: /* cardinality: True iff #True >= param */
        return s >= param ? -1 : 1;
    default:
        return 1;
    }
}

static int popcount32(uint32_t v) {
    int c = 0;
    while (v) {
        v &= v - 1;
        ++c;
    }
    return c;
}

/* ------------------------------------------------------------------------ */
/* Thm. "Walsh Transform": f^(S) = 2^-L sum_x f(x) prod_{i in S} x_i         */
/* A corner is a bit pattern z; bit i set means x_i = -1 (True).             */
/* ------------------------------------------------------------------------ */

double orc_walsh_subset(int type, int param, int L, uint32_t mask) {
    double acc = 0.0;
    uint32_t ncorner = 1u << L;
    for (uint32_t z = 0; z < ncorner; ++z) {
        int fz = orc_value(type, param, L, popcount32(z));
        int chi = (popcount32(z & mask) & 1) ? -1 : 1; /* prod_{i in S} x_i */
        acc += (double)(fz * chi);
    }
    return acc / (double)ncorner;
}

/* Pascal triangle in exact unsigned 64-bit integers, rows 0..62. */
static uint64_t binom_tab[63][63];

__attribute__((constructor)) static void binom_init(void) {
    for (int a = 0; a < 63; ++a) {
        binom_tab[a][0] = 1;
        for (int b = 1; b <= a; ++b)
            binom_tab[a][b] = binom_tab[a - 1][b - 1] + (b <= a - 1 ? binom_tab[a - 1][b] : 0);
        for (int b = a + 1; b < 63; ++b) binom_tab[a][b] = 0;
    }
}

static uint64_t binom_u64(int n, int k) {
    if (k < 0 || k > n || n < 0 || n > 62) return 0;
    return binom_tab[n][k];
}

void orc_walsh_by_size(int type, int param, int L, double *a) {
    /* Group the corner sum of the theorem for a fixed S with |S| = m by
     * s = #True coordinates and t = #True coordinates inside S:
     * there are C(m,t) C(L-m, s-t) such corners, each with prod_{S} x = (-1)^t. */
    for (int m = 0; m <= L; ++m) {
        int64_t total = 0;
        for (int s = 0; s <= L; ++s) {
            int64_t kraw = 0;
            for (int t = 0; t <= m && t <= s; ++t) {
                int64_t term = (int64_t)(binom_u64(m, t) * binom_u64(L - m, s - t));
                kraw += (t & 1) ? -term : term;
            }
            total += (int64_t)orc_value(type, param, L, s) * kraw;
        }
        a[m] = ldexp((double)total, -L);
    }
}

double orc_fe_walsh_bruteforce(int type, int param, int L, const double *y, double *dy) {
    uint32_t nsub = 1u << L;
    double fe = 0.0;
    if (dy)
        for (int i = 0; i < L; ++i) dy[i] = 0.0;
    for (uint32_t S = 0; S < nsub; ++S) {
        double coef = orc_walsh_subset(type, param, L, S);
        if (coef == 0.0) continue;
        double mono = 1.0;
        for (int i = 0; i < L; ++i)
            if (S & (1u << i)) mono *= y[i];
        fe += coef * mono;
        if (dy) {
            for (int i = 0; i < L; ++i) {
                if (!(S & (1u << i))) continue;
                double d = 1.0;
                for (int l = 0; l < L; ++l)
                    if (l != i && (S & (1u << l))) d *= y[l];
                dy[i] += coef * d;
            }
        }
    }
    return fe;
}

double orc_fe_corners(int type, int param, int L, const double *y, double *dy) {
    uint32_t ncorner = 1u << L;
    double fe = 0.0;
    if (dy)
        for (int i = 0; i < L; ++i) dy[i] = 0.0;
    for (uint32_t z = 0; z < ncorner; ++z) {
        double fz = (double)orc_value(type, param, L, popcount32(z));
        double prob = 1.0;
        for (int i = 0; i < L; ++i) {
            double zi = (z & (1u << i)) ? -1.0 : 1.0;
            prob *= 0.5 * (1.0 + y[i] * zi);
        }
        fe += fz * prob;
        if (dy) {
            for (int i = 0; i < L; ++i) {
                double zi = (z & (1u << i)) ? -1.0 : 1.0;
                double rest = 1.0;
                for (int l = 0; l < L; ++l) {
                    if (l == i) continue;
                    double zl = (z & (1u << l)) ? -1.0 : 1.0;
                    rest *= 0.5 * (1.0 + y[l] * zl);
                }
                dy[i] += fz * 0.5 * zi * rest;
            }
        }
    }
    return fe;
}

/* ------------------------------------------------------------------------ */
/* Def. ESP and Eq. effi_eval                                               */
/* ------------------------------------------------------------------------ */

void orc_esp(int L, const double *y, double *e) {
    e[0] = 1.0;
    for (int m = 1; m <= L; ++m) e[m] = 0.0;
    for (int i = 0; i < L; ++i)
        for (int m = i + 1; m >= 1; --m) e[m] += y[i] * e[m - 1];
}

double orc_fe_esp(int type, int param, int L, const double *y, double *dy) {
    double *a = (double *)malloc(sizeof(double) * (size_t)(L + 1));
    double *e = (double *)malloc(sizeof(double) * (size_t)(L + 1));
    double *yy = (double *)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
    orc_walsh_by_size(type, param, L, a);
    orc_esp(L, y, e);
    double fe = 0.0;
    for (int m = 0; m <= L; ++m) fe += a[m] * e[m];
    if (dy) {
        for (int i = 0; i < L; ++i) {
            int k = 0;
            for (int l = 0; l < L; ++l)
                if (l != i) yy[k++] = y[l];
            orc_esp(L - 1, yy, e); /* e_{m-1} of the other literals */
            double d = 0.0;
            for (int m = 1; m <= L; ++m) d += a[m] * e[m - 1];
            dy[i] = d;
        }
    }
    free(a);
    free(e);
    free(yy);
    return fe;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (forward with FFT) and Eq. chain (backward), complex double        */
/* ------------------------------------------------------------------------ */

void orc_paper_ftilde(int type, int param, int L, double *re, double *im) {
    int N = L + 1;
    double *a = (double *)malloc(sizeof(double) * (size_t)N);
    orc_walsh_by_size(type, param, L, a);
    for (int j = 0; j < N; ++j) {
        double complex acc = 0.0;
        for (int t = 0; t < N; ++t) {
            double fhat_t = a[L - t]; /* fhat ordered [e_L, ..., e_0] */
            /* W^{-1}[t, j] = omega^{-t j} / N with omega = exp(-2 pi i / N) */
            double ang = 2.0 * M_PI * (double)(((long long)t * j) % N) / (double)N;
            acc += fhat_t * cexp(I * ang);
        }
        acc /= (double)N;
        re[j] = creal(acc);
        im[j] = cimag(acc);
    }
    free(a);
}

double orc_fe_paper(int type, int param, int L, const double *y, double *dy) {
    int N = L + 1;
    double *fr = (double *)malloc(sizeof(double) * (size_t)N);
    double *fi = (double *)malloc(sizeof(double) * (size_t)N);
    orc_paper_ftilde(type, param, L, fr, fi);
    double complex we = 0.0;
    for (int j = 0; j < N; ++j) {
        double ang = -2.0 * M_PI * (double)j / (double)N;
        double complex wj = cexp(I * ang); /* omega^j */
        double complex gam = 1.0;        /* gamma_{1:k}[j] */
        for (int i = 0; i < L; ++i) gam *= (wj + y[i]);
        we += (fr[j] + I * fi[j]) * gam;
    }
    if (dy) {
        for (int i = 0; i < L; ++i) {
            double complex d = 0.0;
            for (int j = 0; j < N; ++j) {
                double ang = -2.0 * M_PI * (double)j / (double)N;
                double complex wj = cexp(I * ang);
                double complex rest = 1.0;
                for (int l = 0; l < L; ++l)
                    if (l != i) rest *= (wj + y[l]);
                d += (fr[j] + I * fi[j]) * rest;
            }
            dy[i] = creal(d);
        }
    }
    free(fr);
    free(fi);
    return creal(we);
}

/* ------------------------------------------------------------------------ */
/* Probability reading: Poisson-binomial recurrence                          */
/* ------------------------------------------------------------------------ */

static _Thread_local double *tl_buf = NULL;
static _Thread_local size_t tl_cap = 0;

static double *scratch(size_t count) {
    if (count > tl_cap) {
        free(tl_buf);
        tl_cap = count + count / 2 + 64;
        tl_buf = (double *)malloc(sizeof(double) * tl_cap);
    }
    return tl_buf;
}

double orc_fe_dp(int type, int param, int L, const double *y, double *dy) {
    size_t W = (size_t)L + 2;
    /* layout: pi[W] | h[(L+1) * W] (h_k for k = 0..L) */
    double *buf = scratch(W + (size_t)(L + 1) * W);
    double *pi = buf;
    double *h = buf + W;

    /* forward: distribution of S over all literals */
    for (size_t s = 0; s < W; ++s) pi[s] = 0.0;
    pi[0] = 1.0;
    for (int i = 0; i < L; ++i) {
        double p = 0.5 * (1.0 - y[i]); /* P(literal True) */
        double q = 0.5 * (1.0 + y[i]); /* P(literal False) */
        for (int s = i + 1; s >= 1; --s) pi[s] = pi[s] * q + pi[s - 1] * p;
        pi[0] *= q;
    }
    double fe = 0.0;
    for (int s = 0; s <= L; ++s) fe += (double)orc_value(type, param, L, s) * pi[s];

    if (dy) {
        /* h_L(u) = v(u) - v(u+1); h_k(u) = q_k h_{k+1}(u) + p_k h_{k+1}(u+1) */
        double *hL = h + (size_t)L * W;
        for (int u = 0; u < L; ++u)
            hL[u] = (double)(orc_value(type, param, L, u) - orc_value(type, param, L, u + 1));
        hL[L] = 0.0;
        for (int k = L - 1; k >= 1; --k) {
            double p = 0.5 * (1.0 - y[k]);
            double q = 0.5 * (1.0 + y[k]);
            double *hk = h + (size_t)k * W;
            double *hn = h + (size_t)(k + 1) * W;
            for (int u = 0; u < k; ++u) hk[u] = q * hn[u] + p * hn[u + 1];
            hk[k] = 0.0;
        }
        /* dFE/dy_i = 1/2 sum_u pre_i(u) h_{i+1}(u); pre_i = distribution of literals 0..i-1 */
        for (size_t s = 0; s < W; ++s) pi[s] = 0.0;
        pi[0] = 1.0;
        for (int i = 0; i < L; ++i) {
            double *hn = h + (size_t)(i + 1) * W;
            double d = 0.0;
            for (int u = 0; u <= i; ++u) d += pi[u] * hn[u];
            dy[i] = 0.5 * d;
            double p = 0.5 * (1.0 - y[i]);
            double q = 0.5 * (1.0 + y[i]);
            for (int s = i + 1; s >= 1; --s) pi[s] = pi[s] * q + pi[s - 1] * p;
            pi[0] *= q;
        }
    }
    return fe;
}

/* ------------------------------------------------------------------------ */
/* Closed forms                                                             */
/* ------------------------------------------------------------------------ */

double orc_fe_or(int L, const double *y, double *dy) {
    double prod = 1.0;
    for (int i = 0; i < L; ++i) prod *= 0.5 * (1.0 + y[i]);
    if (dy) {
        for (int i = 0; i < L; ++i) {
            double rest = 1.0;
            for (int l = 0; l < L; ++l)
                if (l != i) rest *= 0.5 * (1.0 + y[l]);
            dy[i] = rest; /* d/dy_i of 2 prod_l (1+y_l)/2 */
        }
    }
    return -1.0 + 2.0 * prod;
}

double orc_fe_xor(int param, int L, const double *y, double *dy) {
    double sgn = (param & 1) ? 1.0 : -1.0;
    double prod = 1.0;
    for (int i = 0; i < L; ++i) prod *= y[i];
    if (dy) {
        for (int i = 0; i < L; ++i) {
            double rest = 1.0;
            for (int l = 0; l < L; ++l)
                if (l != i) rest *= y[l];
            dy[i] = sgn * rest;
        }
    }
    return sgn * prod;
}

double orc_fe(int type, int param, int L, const double *y, double *dy) {
    switch (type) {
    case ORC_OR:
        return orc_fe_or(L, y, dy);
    case ORC_XOR:
        return orc_fe_xor(param, L, y, dy);
    default:
        return orc_fe_dp(type, param, L, y, dy);
    }
}

static double fe_route(int route, int type, int param, int L, const double *y, double *dy) {
    switch (route) {
    case 1:
        return orc_fe_dp(type, param, L, y, dy);
    case 2:
        return orc_fe_esp(type, param, L, y, dy);
    case 3:
        return orc_fe_paper(type, param, L, y, dy);
    default:
        return orc_fe(type, param, L, y, dy);
    }
}

/* ------------------------------------------------------------------------ */
/* Instance evaluation (Def. "Objective") and its gradient                  */
/* ------------------------------------------------------------------------ */

static int resolve_threads(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_max_threads(void) { return resolve_threads(0); }

static int max_len(int32_t m, const int64_t *row_ptr) {
    int64_t mx = 0;
    for (int32_t c = 0; c < m; ++c) {
        int64_t l = row_ptr[c + 1] - row_ptr[c];
        if (l > mx) mx = l;
    }
    return (int)mx;
}

/* F and grad F at one point x (length n); g must hold n entries. */
static int eval_point(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                      const uint8_t *type, const int32_t *param, const double *w,
                      const double *x, double *f, double *g, double *y, double *dy, int route) {
    for (int32_t v = 0; v < n; ++v) {
        if (isnan(x[v])) return -1;
        g[v] = 0.0;
    }
    double acc = 0.0;
    for (int32_t c = 0; c < m; ++c) {
        int64_t a = row_ptr[c];
        int L = (int)(row_ptr[c + 1] - a);
        for (int i = 0; i < L; ++i) {
            int32_t lit = lits[a + i];
            int32_t v = (lit > 0 ? lit : -lit) - 1;
            if (v < 0 || v >= n) return -1;
            y[i] = lit > 0 ? x[v] : -x[v];
        }
        double wc = w ? w[c] : 1.0;
        double fe = fe_route(route, type[c], param[c], L, y, dy);
        acc += wc * fe;
        for (int i = 0; i < L; ++i) {
            int32_t lit = lits[a + i];
            int32_t v = (lit > 0 ? lit : -lit) - 1;
            g[v] += wc * (lit > 0 ? dy[i] : -dy[i]);
        }
    }
    *f = acc;
    return 0;
}

int orc_eval_grad(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                  const uint8_t *type, const int32_t *param, const double *w,
                  int32_t B, const double *x, double *f, double *g, int nthreads, int route) {
    int nt = resolve_threads(nthreads);
    int L = max_len(m, row_ptr);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        double *y = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        double *dy = (double *)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int32_t b = 0; b < B; ++b) {
            int rc = eval_point(n, m, row_ptr, lits, type, param, w, x + (size_t)b * n, f + b,
                                g + (size_t)b * n, y, dy, route);
            if (rc) {
#pragma omp atomic write
                status = rc;
            }
        }
        free(y);
        free(dy);
    }
    return status;
}

int orc_eval_scale(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                   const uint8_t *type, const int32_t *param, const double *w,
                   int32_t B, const double *x, double *sf, double *A, double floor, int floor_types,
                   int nthreads) {
    int nt = resolve_threads(nthreads);
    int L = max_len(m, row_ptr);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        double *y = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        double *dy = (double *)malloc(sizeof(double) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int32_t b = 0; b < B; ++b) {
            const double *xb = x + (size_t)b * n;
            double *Ab = A + (size_t)b * n;
            for (int32_t v = 0; v < n; ++v) Ab[v] = 0.0;
            double acc = 0.0;
            for (int32_t c = 0; c < m; ++c) {
                int64_t a = row_ptr[c];
                int Lc = (int)(row_ptr[c + 1] - a);
                int bad = 0;
                for (int i = 0; i < Lc; ++i) {
                    int32_t lit = lits[a + i];
                    int32_t v = (lit > 0 ? lit : -lit) - 1;
                    if (v < 0 || v >= n) bad = 1;
                    else y[i] = lit > 0 ? xb[v] : -xb[v];
                }
                if (bad) {
#pragma omp atomic write
                    status = -1;
                    continue;
                }
                double wc = w ? w[c] : 1.0;
                double fe = orc_fe(type[c], param[c], Lc, y, dy);
                acc += wc * fabs(fe);
                double fl = ((floor_types >> type[c]) & 1) ? floor : 0.0;
                for (int i = 0; i < Lc; ++i) {
                    int32_t lit = lits[a + i];
                    int32_t v = (lit > 0 ? lit : -lit) - 1;
                    double d = fabs(dy[i]);
                    Ab[v] += wc * (d > fl ? d : fl);
                }
            }
            sf[b] = acc;
        }
        free(y);
        free(dy);
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* Exact checker twin                                                       */
/* ------------------------------------------------------------------------ */

static int32_t check_point(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                           const uint8_t *type, const int32_t *param, const double *x, int *bad) {
    int32_t unsat = 0;
    for (int32_t c = 0; c < m; ++c) {
        int64_t a = row_ptr[c];
        int L = (int)(row_ptr[c + 1] - a);
        int s = 0;
        for (int i = 0; i < L; ++i) {
            int32_t lit = lits[a + i];
            int32_t v = (lit > 0 ? lit : -lit) - 1;
            if (v < 0 || v >= n || isnan(x[v])) {
                *bad = 1;
                return 0;
            }
            int var_true = x[v] < 0.0; /* sgn(x) = -1 encodes True */
            int lit_true = lit > 0 ? var_true : !var_true;
            s += lit_true;
        }
        if (orc_value(type[c], param[c], L, s) > 0) ++unsat;
    }
    return unsat;
}

int orc_check(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
              const uint8_t *type, const int32_t *param,
              int32_t B, const double *x, uint8_t *sat, int32_t *n_unsat, int nthreads) {
    int nt = resolve_threads(nthreads);
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int32_t b = 0; b < B; ++b) {
        int bad = 0;
        int32_t u = check_point(n, m, row_ptr, lits, type, param, x + (size_t)b * n, &bad);
        if (bad) {
#pragma omp atomic write
            status = -1;
        }
        n_unsat[b] = u;
        sat[b] = (uint8_t)(u == 0 && !bad);
    }
    return status;
}

int orc_unsat_counts(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                     const uint8_t *type, const int32_t *param, int32_t B, const double *x, int32_t *U) {
    for (int32_t c = 0; c < m; ++c) U[c] = 0;
    for (int32_t b = 0; b < B; ++b) {
        const double *xb = x + (size_t)b * n;
        for (int32_t c = 0; c < m; ++c) {
            int64_t a = row_ptr[c];
            int L = (int)(row_ptr[c + 1] - a);
            int s = 0;
            for (int i = 0; i < L; ++i) {
                int32_t lit = lits[a + i];
                int32_t v = (lit > 0 ? lit : -lit) - 1;
                if (v < 0 || v >= n || isnan(xb[v])) return -1;
                int var_true = xb[v] < 0.0;
                s += lit > 0 ? var_true : !var_true;
            }
            if (orc_value(type[c], param[c], L, s) > 0) U[c] += 1;
        }
    }
    return 0;
}

void orc_erwa(int32_t m, const int32_t *U, double alpha, double *w) {
    int32_t umax = 0;
    for (int32_t c = 0; c < m; ++c)
        if (U[c] > umax) umax = U[c];
    for (int32_t c = 0; c < m; ++c) {
        double r = umax > 0 ? (double)U[c] / (double)umax : 0.0;
        w[c] = (1.0 - alpha) * w[c] + alpha * r;
    }
}

/* ------------------------------------------------------------------------ */
/* Counter-based restart draws and one CLS round                            */
/* ------------------------------------------------------------------------ */

uint64_t orc_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t epoch, uint64_t b, uint64_t v) {
    uint64_t h = orc_splitmix64(orc_splitmix64(orc_splitmix64(orc_splitmix64(seed) ^ epoch) ^ b) ^ v);
    int64_t u = (int64_t)(h >> 40) - (int64_t)(1 << 23);
    return ldexp((double)u, -23);
}

int orc_step_pgfp(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
                  const uint8_t *type, const int32_t *param, const double *w,
                  int32_t B, double *x, int32_t T, double eta0, double beta, int32_t maxls,
                  double eta_min, double slack,
                  uint64_t seed, uint64_t epoch, uint64_t b_offset, int restart,
                  uint8_t *solved, int32_t *n_unsat, int32_t *iters, double *eta_out, int nthreads) {
    if (!(eta0 > 0.0) || !(beta > 0.0 && beta < 1.0) || maxls < 1) return -1;
    int nt = resolve_threads(nthreads);
    int L = max_len(m, row_ptr);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        double *ybuf = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        double *dy = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        size_t nn = (size_t)(n > 0 ? n : 1);
        double *g = (double *)malloc(sizeof(double) * nn);
        double *gp = (double *)malloc(sizeof(double) * nn);
        double *yk = (double *)malloc(sizeof(double) * nn);   /* extrapolated point y_k */
        double *pk = (double *)malloc(sizeof(double) * nn);   /* trial point p */
#pragma omp for schedule(dynamic, 1)
        for (int32_t b = 0; b < B; ++b) {
            double *xb = x + (size_t)b * n; /* the iterate x_k (x_0 on entry) */
            double eta = eta0, t = 1.0, fy, fp;
            int rc = 0;
            int32_t it = 0;
            for (int32_t v = 0; v < n; ++v) yk[v] = xb[v];
            while (it < T && rc == 0) {
                ++it;
                rc = eval_point(n, m, row_ptr, lits, type, param, w, yk, &fy, g, ybuf, dy, 0);
                if (rc) break;
                /* backtracking on the sufficient-decrease condition of the proximal
                   (projected) gradient step */
                for (int32_t ls = 0; ls < maxls; ++ls) {
                    double d = 0.0, q = 0.0;
                    for (int32_t v = 0; v < n; ++v) {
                        double z = yk[v] - eta * g[v];
                        z = z < -1.0 ? -1.0 : (z > 1.0 ? 1.0 : z);
                        pk[v] = z;
                        d += g[v] * (z - yk[v]);
                        q += (z - yk[v]) * (z - yk[v]);
                    }
                    rc = eval_point(n, m, row_ptr, lits, type, param, w, pk, &fp, gp, ybuf, dy, 0);
                    if (rc) break;
                    if (fp <= fy + d + q / (2.0 * eta) + slack) break;
                    if (ls + 1 < maxls) eta *= beta;
                }
                if (rc) break;
                /* momentum: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, y = Pi(x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1})) */
                double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
                double mom = (t - 1.0) / tn;
                t = tn;
                for (int32_t v = 0; v < n; ++v) {
                    double xn = pk[v];
                    double z = xn + mom * (xn - xb[v]);
                    yk[v] = z < -1.0 ? -1.0 : (z > 1.0 ? 1.0 : z);
                    xb[v] = xn;
                }
                if (eta < eta_min) break;
            }
            if (iters) iters[b] = it;
            if (eta_out) eta_out[b] = eta;
            int bad = rc != 0;
            int32_t u = bad ? 0 : check_point(n, m, row_ptr, lits, type, param, xb, &bad);
            n_unsat[b] = u;
            solved[b] = (uint8_t)(!bad && u == 0);
            if (bad) {
#pragma omp atomic write
                status = -1;
            } else if (u != 0 && restart) {
                for (int32_t v = 0; v < n; ++v) xb[v] = orc_uniform(seed, epoch, b_offset + (uint64_t)b, (uint64_t)v);
            }
        }
        free(ybuf);
        free(dy);
        free(g);
        free(gp);
        free(yk);
        free(pk);
    }
    return status;
}

int orc_rephase(int32_t n, int32_t B, double *x, int phase, const uint8_t *solved,
                uint64_t seed, uint64_t epoch, uint64_t b_offset) {
    if (phase < 0 || phase > 2) return -1;
    for (int32_t b = 0; b < B; ++b) {
        if (solved && solved[b]) continue;
        double *xb = x + (size_t)b * (size_t)n;
        for (int32_t v = 0; v < n; ++v) {
            if (phase == 1)
                xb[v] = -xb[v];
            else if (phase == 2)
                xb[v] = orc_uniform(seed, epoch, b_offset + (uint64_t)b, (uint64_t)v);
        }
    }
    return 0;
}

int orc_step(int32_t n, int32_t m, const int64_t *row_ptr, const int32_t *lits,
             const uint8_t *type, const int32_t *param, const double *w,
             int32_t B, double *x, int32_t T, double lr,
             uint64_t seed, uint64_t epoch, uint64_t b_offset, int restart,
             uint8_t *solved, int32_t *n_unsat, int nthreads) {
    int nt = resolve_threads(nthreads);
    int L = max_len(m, row_ptr);
    int status = 0;
#pragma omp parallel num_threads(nt)
    {
        double *y = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        double *dy = (double *)malloc(sizeof(double) * (size_t)(L + 1));
        double *g = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (int32_t b = 0; b < B; ++b) {
            double *xb = x + (size_t)b * n;
            double fval;
            int rc = 0;
            for (int32_t it = 0; it < T && rc == 0; ++it) {
                rc = eval_point(n, m, row_ptr, lits, type, param, w, xb, &fval, g, y, dy, 0);
                for (int32_t v = 0; v < n && rc == 0; ++v) {
                    double z = xb[v] - lr * g[v];
                    xb[v] = z < -1.0 ? -1.0 : (z > 1.0 ? 1.0 : z);
                }
            }
            int bad = rc != 0;
            int32_t u = bad ? 0 : check_point(n, m, row_ptr, lits, type, param, xb, &bad);
            n_unsat[b] = u;
            solved[b] = (uint8_t)(!bad && u == 0);
            if (bad) {
#pragma omp atomic write
                status = -1;
            } else if (u != 0 && restart) {
                for (int32_t v = 0; v < n; ++v) xb[v] = orc_uniform(seed, epoch, b_offset + (uint64_t)b, (uint64_t)v);
            }
        }
        free(y);
        free(dy);
        free(g);
    }
    return status;
}
