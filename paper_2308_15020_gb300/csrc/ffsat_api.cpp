// Host side of libffsat: validation, FP64 preprocessing of the node tables,
// length bucketing, device upload and the C ABI declared in include/ffsat.h.
#include <algorithm>
#include <array>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ffsat.h"
#include "cluster_launch.h"
#include "ffsat_internal.h"
#include "heuristics.h"

using namespace ffsat;

namespace {

thread_local std::string t_err;
thread_local int32_t t_launches = 0;
thread_local int32_t t_cluster = 0;
thread_local int32_t t_pairs = 0;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(FFSAT_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kMaxLen = FFSAT_MAX_LEN;
constexpr int kPaperMaxLen = 60;

enum ConsClass : int8_t { CLS_CLAUSE3 = 0, CLS_PRODUCT = 1, CLS_NODE = 2, CLS_CONST = 3, CLS_XOR2 = 4 };

// v(s) of a symmetric constraint: -1 if s True literals satisfy it, +1 otherwise.
inline int truth_value(int type, int param, int s) {
    if (type == FFSAT_OR) return s >= 1 ? -1 : 1;
    if (type == FFSAT_XOR) return ((s & 1) == (param & 1)) ? -1 : 1;
    return s >= param ? -1 : 1;
}

inline int pow2_at_least(int v) {
    int g = 1;
    while (g < v) g <<= 1;
    return g;
}

// Walsh coefficients a_m (coefficient of e_m in the expansion, Eq. effi_eval)
// of a symmetric constraint with L <= 60 literals.  Setting every literal to
// the same value t turns the expansion into sum_m a_m C(L,m) t^m, while the
// probability reading gives 2^-L sum_s v(s) C(L,s) (1-t)^s (1+t)^(L-s); the
// coefficients of the latter polynomial are computed in exact 128-bit integers.
void walsh_coefficients(int type, int param, int L, std::vector<double> &a) {
    std::vector<std::vector<__int128>> C(L + 1, std::vector<__int128>(L + 1, 0));
    for (int i = 0; i <= L; ++i) {
        C[i][0] = 1;
        for (int k = 1; k <= i; ++k) C[i][k] = C[i - 1][k - 1] + (k < i ? C[i - 1][k] : 0);
    }
    std::vector<__int128> Q(L + 1, 0);
    std::vector<__int128> poly(L + 1);
    for (int s = 0; s <= L; ++s) {
        // poly = (1 - t)^s (1 + t)^(L - s)
        std::fill(poly.begin(), poly.end(), 0);
        poly[0] = 1;
        int deg = 0;
        for (int k = 0; k < L; ++k) {
            const __int128 sg = k < s ? -1 : 1;
            for (int d = deg + 1; d >= 1; --d) poly[d] += sg * poly[d - 1];
            ++deg;
        }
        const __int128 scale = C[L][s] * (__int128)truth_value(type, param, s);
        for (int d = 0; d <= L; ++d) Q[d] += scale * poly[d];
    }
    a.assign(L + 1, 0.0);
    for (int m = 0; m <= L; ++m)
        a[m] = std::ldexp((double)Q[m] / (double)C[L][m], -L);
}

// Split alpha_re + beta_re = 1 so that the rounded pair still sums to exactly 1
// (then the padding value y = +1 gives a factor of exactly 1 + 0i).
template <typename R>
void split_unit(double alpha, R &a, R &b) {
    if (alpha >= 0.5) {
        a = (R)alpha;
        b = R(1) - a;
    } else {
        b = (R)(1.0 - alpha);
        a = R(1) - b;
    }
}

struct Arena {
    std::vector<unsigned char> host;
    template <typename T>
    size_t put(const std::vector<T> &v) {
        size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + std::max<size_t>(v.size() * sizeof(T), 16));
        if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

struct TaskSet {
    std::vector<int4> tasks;
    int node_r = 0;
};

// Tile choices of one resident image: the defaults, or what the autotuner
// measured fastest for the instance.
struct Knobs {
    int32_t shape = 0;        // node segment shape: 0 cost model, 1 fewest lanes, 2 fewest literal slots
    int32_t clause_k = 0;     // clause groups of 32 per clause task: 0 automatic, else 1, 2 or 4
    int32_t pts_per_cta = 1;  // points per CTA of the fused kernel (grid = ceil(B / pts_per_cta))
    bool operator==(const Knobs &o) const {
        return shape == o.shape && clause_k == o.clause_k && pts_per_cta == o.pts_per_cta;
    }
};

}  // namespace

struct ffsat_instance {
    int device = 0;
    int32_t n = 0, m = 0;
    int64_t nnz = 0;
    ffsat_options opt{};
    int num_sms = 0;
    int max_smem = 0;
    // per constraint
    std::vector<int8_t> cls;
    std::vector<int32_t> slot;
    std::vector<double> w;
    std::vector<uint8_t> type;
    std::vector<int32_t> param, len;
    // host copies of the weight-carrying arrays
    std::vector<int4> clauses;   // {l0, l1, l2, FP32 weight bits}, bank-ordered, padded
    std::vector<int4> seg_info;  // canonical {offset into seg_lits, length, aux, FP32 weight bits}
    std::vector<int32_t> seg_lits;
    int n_node_seg = 0;
    int32_t pad_node = 0;        // padding literal of node segments (dummy n or n + 1)
    int nr[2] = {0, 0};          // node R family of each image (16: 16/12/8 per segment, 8, or 0)
    std::vector<double> clause_wd;
    std::vector<double> seg_wd;
    std::vector<double> cons_wd;
    double f_const = 0.0;        // constants of the fused kernel's f (see fill_weights)
    double f_const_plain = 0.0;  // sum of w FE over constant constraints
    float fix_s1 = 1.0f, fix_s2 = 1.0f, fix_i1 = 1.0f, fix_i12 = 1.0f;
    int32_t fix_two = 1;
    double fix64_s = 1.0, fix64_i = 1.0;
    int32_t fix64_l = 0;
    bool fix64_ok = false;  // the cluster step's fixed point resolves 2^-44 or finer
    std::vector<int64_t> row_ptr;  // host copy of the CSR (fixed-point scales)
    std::vector<int32_t> lits_in;
    // resident images (index 0: FP32 task list, 1: FP64 task list), each with the
    // tile choices it was built with and its own device allocation
    int n_images = 2;
    std::vector<int4> tasks[2];
    std::vector<int4> image[2];
    Knobs knobs[2];
    int32_t img_off[2][4] = {{0}};  // tasks, clauses, segmeta, seg_lits (int4 units)
    int4 *d_img[2] = {nullptr, nullptr};
    // what the task lists are built from (kept for the autotuner's rebuilds)
    std::vector<int32_t> seg_len;
    int n_clause_pad = 0, n_xor2_pad = 0, max_node_len = 0;
    // device
    unsigned char *d_arena = nullptr;
    size_t arena_bytes = 0;
    size_t off_clause_wd = 0, off_seg_wd = 0, off_cons_wd = 0;
    size_t off_f_const = 0, off_cls = 0, off_slot = 0, off_umax = 0;
    int32_t *d_status = nullptr;
    int32_t *d_node_ids = nullptr, *d_closed_ids = nullptr;
    int32_t n_node_ids = 0, n_closed_ids = 0;
    DevView V32{}, V64{};
    int nr32 = 0, nr64 = 0;
    int smem_mode32 = SMEM_FULL, smem_mode64 = SMEM_FULL;
    size_t smem32 = 0, smem64 = 0;
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    void *d_yscratch = nullptr;  // extrapolated points of ffsat_step_pgfp
    size_t yscratch_bytes = 0;
    ffsat_info info{};
    // resident clusters of the FP64 cluster step for CL = 2, 4, 8 (-1: not asked yet)
    int cluster_active[3] = {-1, -1, -1};
    std::mutex cluster_mu;  // guards the lazy fill of cluster_active (steps may run on several host threads)
    // learned-proposal graph data (built on first use)
    unsigned char *d_graph = nullptr;
    GraphView graph{};
};

namespace {

int validate(int32_t n, int32_t m, const int64_t *rp, const int32_t *lits, const uint8_t *type,
             const int32_t *param, const double *w, const ffsat_options &o) {
    if (n <= 0) return fail(FFSAT_ERR_ARG, "n_vars must be positive (got %d)", n);
    if (m < 0) return fail(FFSAT_ERR_ARG, "n_cons must be >= 0 (got %d)", m);
    if (o.form != FFSAT_FORM_STABLE && o.form != FFSAT_FORM_PAPER) return fail(FFSAT_ERR_ARG, "bad form %d", o.form);
    if (o.node_r != 0 && o.node_r != 8 && o.node_r != 16) return fail(FFSAT_ERR_ARG, "node_r must be 0, 8 or 16");
    if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8)
        return fail(FFSAT_ERR_ARG, "cluster must be 0, 1, 2, 4 or 8");
    if (!rp) return fail(FFSAT_ERR_ARG, "row_ptr is NULL");
    if (m > 0 && (!type || !param)) return fail(FFSAT_ERR_ARG, "type/param is NULL");
    if (rp[0] != 0) return fail(FFSAT_ERR_PARAM, "row_ptr[0] must be 0");
    const int64_t nnz = rp[m];
    if (nnz < 0 || nnz >= (int64_t(1) << 31) - 1) return fail(FFSAT_ERR_ARG, "literal count out of range");
    if (nnz > 0 && !lits) return fail(FFSAT_ERR_ARG, "lits is NULL");
    std::vector<int32_t> stamp((size_t)n, -1);
    for (int32_t c = 0; c < m; ++c) {
        const int64_t a = rp[c], e = rp[c + 1];
        if (e < a || e > nnz) return fail(FFSAT_ERR_PARAM, "row_ptr not non-decreasing at constraint %d", c);
        const int64_t L = e - a;
        if (L == 0) return fail(FFSAT_ERR_EMPTY, "constraint %d has no literals", c);
        if (L > kMaxLen) return fail(FFSAT_ERR_TOOLONG, "constraint %d has %lld literals (max %d)", c, (long long)L, kMaxLen);
        const int t = type[c];
        if (t != FFSAT_OR && t != FFSAT_XOR && t != FFSAT_ATLEAST) return fail(FFSAT_ERR_PARAM, "constraint %d: unknown type %d", c, t);
        if (t == FFSAT_XOR && param[c] != 0 && param[c] != 1) return fail(FFSAT_ERR_PARAM, "constraint %d: XOR parity must be 0 or 1", c);
        if (t == FFSAT_ATLEAST && param[c] < 0) return fail(FFSAT_ERR_PARAM, "constraint %d: K must be >= 0", c);
        if (w && !(std::isfinite(w[c]) && w[c] >= 0.0)) return fail(FFSAT_ERR_WEIGHT, "constraint %d: weight must be finite and >= 0", c);
        for (int64_t i = a; i < e; ++i) {
            const int32_t l = lits[i];
            if (l == 0 || l == INT32_MIN) return fail(FFSAT_ERR_VAR_RANGE, "constraint %d: literal %d", c, l);
            const int32_t v = (l > 0 ? l : -l) - 1;
            if (v >= n) return fail(FFSAT_ERR_VAR_RANGE, "constraint %d: variable %d > n_vars", c, v + 1);
            if (stamp[v] == c) return fail(FFSAT_ERR_DUPVAR, "constraint %d: variable %d occurs twice", c, v + 1);
            stamp[v] = c;
        }
    }
    return FFSAT_OK;
}

// Packed literal: variable index | (negated << 31).
inline int32_t pack_lit(int32_t l) {
    const uint32_t v = (uint32_t)((l > 0 ? l : -l) - 1);
    return (int32_t)(v | (l < 0 ? 0x80000000u : 0u));
}

// Lanes per constraint segment: the smallest power of two G with G * R >= L.
inline int seg_lanes(int L, int R) { return std::max(1, pow2_at_least((L + R - 1) / R)); }

// Literals per lane of a node segment.  A kernel built for node R = 16 also
// runs 12 and 8 literals per lane, and in FP32 with the imaginary-node form 14
// and 10 (read as 8-byte pairs); per segment the host picks the shape with
// the smallest modelled issue cost per node, G * (7 NR + 58 + 8 log2 G) lane
// instructions for the imaginary-node task (7 per literal slot; per node the
// normalisation, division and scales, and per butterfly level three shuffles,
// an exponent add and a complex product), G * (14 NR + 12 + 10 log2 G) for the
// generic one.
// The autotuner may replace the model by another segment shape: the fewest
// lanes per segment (shape 1; ties to fewer literal slots) or the fewest literal
// slots G * NR (shape 2; ties to fewer lanes).
inline int node_nr(int L, int nr_max, bool imag, int shape = 0, bool f32 = true) {
    if (nr_max < 16) return nr_max;
    auto cost = [&](int nr) {
        const int G = seg_lanes(L, nr);
        if (G > 32) return 1e30;
        const double lg = std::log2((double)G);
        if (shape == 1) return (double)G * 1024.0 + (double)(G * nr);
        if (shape == 2) return (double)(G * nr) * 64.0 + (double)G;
        return imag ? (double)G * (7.0 * nr + 58.0 + 8.0 * lg) : (double)G * (14.0 * nr + 12.0 + 10.0 * lg);
    };
    int best = 16;
    for (int nr : {14, 12, 10, 8}) {
        // the generic node task, and the FP64 kernels, run 16, 12 and 8
        if ((nr == 14 || nr == 10) && !(imag && f32)) continue;
        if (cost(nr) < cost(best)) best = nr;
    }
    return best;
}

// Per-constraint FE of constant constraints (cardinality with K <= 0 or K > L).
inline bool constant_value(int type, int param, int L, double &fe) {
    if (type != FFSAT_ATLEAST) return false;
    if (param <= 0) {
        fe = -1.0;
        return true;
    }
    if (param > L) {
        fe = 1.0;
        return true;
    }
    return false;
}

// Append the node table of one (type, L, param) key: J = floor((L+1)/2) + 1
// nodes of the N = L + 1 roots of unity, conjugate-symmetric half with the
// multiplicity folded into c_j and d_j.
void build_table(int type, int param, int L, int form, std::vector<float> &tf, std::vector<double> &td) {
    const int N = L + 1;
    const int J = N / 2 + 1;
    std::vector<double> coef(L + 1);
    if (form == FFSAT_FORM_PAPER) {
        walsh_coefficients(type, param, L, coef);  // coefficient of e_m
    } else {
        for (int s = 0; s <= L; ++s) coef[s] = (double)truth_value(type, param, s);  // v(s)
    }
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int j = 0; j < J; ++j) {
        const double mult = (j == 0 || 2 * j == N) ? 1.0 : 2.0;
        const double th = -two_pi * (double)j / (double)N;  // omega^j = exp(i th)
        const double wr = std::cos(th), wi = std::sin(th);
        double ar, ai, br, bi;
        if (form == FFSAT_FORM_PAPER) {
            ar = 1.0;
            ai = 0.0;
            br = wr;
            bi = wi;
        } else {
            ar = 0.5 * (1.0 + wr);
            ai = 0.5 * wi;
            br = 0.5 * (1.0 - wr);
            bi = -0.5 * wi;
        }
        // c_j = (mult / N) sum_k coef[k] omega^{-j k}: the powers come from a
        // rotation recurrence, re-anchored on exact values every 32 terms
        double cr = 0.0, ci = 0.0;
        const double rot_r = std::cos(two_pi * (double)j / (double)N), rot_i = std::sin(two_pi * (double)j / (double)N);
        double zr = 1.0, zi = 0.0;
        for (int k = 0; k <= L; ++k) {
            if ((k & 31) == 0) {
                const long long jk = ((long long)j * k) % N;
                const double ph = two_pi * (double)jk / (double)N;
                zr = std::cos(ph);
                zi = std::sin(ph);
            }
            cr += coef[k] * zr;
            ci += coef[k] * zi;
            const double nr = zr * rot_r - zi * rot_i;
            zi = zr * rot_i + zi * rot_r;
            zr = nr;
        }
        cr *= mult / N;
        ci *= mult / N;
        const double dr = cr * br - ci * bi, di = cr * bi + ci * br;
        // FP32 entry
        float far, fbr;
        if (form == FFSAT_FORM_PAPER) {
            far = 1.0f;
            fbr = (float)br;
        } else {
            split_unit<float>(ar, far, fbr);
        }
        const float fai = (float)ai;
        const float fbi = form == FFSAT_FORM_PAPER ? (float)bi : -fai;
        const float ft[8] = {far, fai, fbr, fbi, (float)dr, (float)di, (float)cr, (float)ci};
        tf.insert(tf.end(), ft, ft + 8);
        double dar, dbr;
        if (form == FFSAT_FORM_PAPER) {
            dar = 1.0;
            dbr = br;
        } else {
            split_unit<double>(ar, dar, dbr);
        }
        const double dbi = form == FFSAT_FORM_PAPER ? bi : -ai;
        const double dt[8] = {dar, ai, dbr, dbi, dr, di, cr, ci};
        td.insert(td.end(), dt, dt + 8);
    }
}

// Mantissa and exponent of a complex number: (re, im) = (mr, mi) 2^e with the
// larger of |mr|, |mi| in [1/2, 1); zero gives (0, 0, 0).  The number is given
// as 2^lg (cos ph, sin ph), so magnitudes far outside the FP64 range are fine.
void split_exp(double lg, double ph, double &mr, double &mi, int &e) {
    const double cr = std::cos(ph), ci = std::sin(ph);
    const double mx = std::max(std::fabs(cr), std::fabs(ci));
    const double l2 = lg + std::log2(mx);
    e = (int)std::floor(l2) + 1;
    const double s = std::exp2(l2 - e) / mx;
    mr = cr * s;
    mi = ci * s;
}

// Append the imaginary-node table of one (type, L, param) key: N = L + 1 or
// L + 2, whichever is odd, nodes j = 0 .. (N - 1) / 2 of the conjugate-symmetric
// half.  With w = e^{-2 pi i / N}: c_j = (m_j / N) sum_s v(s) w^{-j s} (the
// stable form's coefficients, m_j = 1 for j = 0 and 2 otherwise), alpha_j =
// (1 + w^j) / 2 = cos(pi j / N) e^{-i pi j / N}, t_j = tan(pi j / N),
// C_j = c_j alpha_j^L (the kernels form D_j = i t_j C_j).  All in FP64 on the host; the
// magnitude of alpha_j^L is carried as a base-2 logarithm, cos(pi j / N) taken
// as sin(pi (N - 2j) / 2N) to keep its relative accuracy near j = N / 2.
void build_table_im(int type, int param, int L, std::vector<float> &tf, std::vector<double> &td) {
    const int N = (L % 2 == 0) ? L + 1 : L + 2;
    const int J = (N - 1) / 2 + 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> cosk(N), sink(N);  // cos, sin of 2 pi k / N
    for (int k = 0; k < N; ++k) {
        cosk[k] = std::cos(2.0 * pi * (double)k / (double)N);
        sink[k] = std::sin(2.0 * pi * (double)k / (double)N);
    }
    for (int j = 0; j < J; ++j) {
        const double mult = j == 0 ? 1.0 : 2.0;
        double cr = 0.0, ci = 0.0;
        for (int s = 0; s <= L; ++s) {
            const int k = (int)(((long long)j * s) % N);
            const double v = (double)truth_value(type, param, s);
            cr += v * cosk[k];
            ci += v * sink[k];
        }
        cr *= mult / N;
        ci *= mult / N;
        const double sn = std::sin(pi * (double)j / (double)N);
        const double cs = std::sin(pi * (double)(N - 2 * j) / (2.0 * (double)N));  // cos(pi j / N) > 0
        const double t = sn / cs;
        double Cr = 0.0, Ci = 0.0;
        int ec = 0;
        const double cabs = std::hypot(cr, ci);
        if (cabs > 0.0) {
            const double lg = std::log2(cabs) + (double)L * std::log2(cs);
            const double ph = std::atan2(ci, cr) - pi * (double)(((long long)L * j) % (2LL * N)) / (double)N;
            split_exp(lg, ph, Cr, Ci, ec);
        }
        int32_t eci = ec;
        float fec;
        std::memcpy(&fec, &eci, 4);
        const float ft[4] = {(float)t, (float)Cr, (float)Ci, fec};
        tf.insert(tf.end(), ft, ft + 4);
        const double dt[4] = {t, Cr, Ci, (double)ec};
        td.insert(td.end(), dt, dt + 4);
    }
}

// Warp tasks for one node R: node tasks (longest first), then product tasks,
// then clause tasks.  Segments are node constraints followed by product
// constraints, each group sorted by length, descending.
// Clause groups (32 clauses) per clause task for a kernel with `warps` warps:
// the choice that minimises (rounds of tasks over the warps) x (task length),
// counting one group per clause task step plus a fixed task overhead and each
// other task as one group.
int clause_groups_per_task(int groups, int other_tasks, int warps) {
    double best = 1e300;
    int pick = kClausePerLane;
    for (int k = kClausePerLane; k >= 1; k >>= 1) {
        const int tasks = (groups + k - 1) / k + other_tasks;
        const double t = (double)((tasks + warps - 1) / warps) * (k + 0.3);
        if (t < best - 1e-9) {
            best = t;
            pick = k;
        }
    }
    return pick;
}

void build_tasks(const std::vector<int32_t> &seg_len, int n_node_seg, int n_clause, int n_xor2, int node_r,
                 int warps, bool imag, const Knobs &kn, TaskSet &ts, bool f32) {
    ts.tasks.clear();
    ts.node_r = node_r;
    auto group = [&](int first, int count, int kind, int R) {
        int i = first;
        const int end = first + count;
        while (i < end) {
            const int L = seg_len[i];
            const int nr = kind == TASK_NODE ? node_nr(L, R, imag, kn.shape, f32) : R;
            const int G = seg_lanes(L, nr);
            const int S = 32 / G;
            int k = 0;
            while (k < S && i + k < end) {
                const int Lk = seg_len[i + k];
                const int nk = kind == TASK_NODE ? node_nr(Lk, R, imag, kn.shape, f32) : R;
                if (nk != nr || seg_lanes(Lk, nk) != G) break;
                ++k;
            }
            const int J = kind == TASK_NODE ? (L + 1) / 2 + 1 : 0;
            ts.tasks.push_back(make_int4(kind | (G << 8) | (nr << 16), i, k, J));
            i += k;
        }
    };
    if (n_node_seg > 0) group(0, n_node_seg, TASK_NODE, node_r);
    group(n_node_seg, (int)seg_len.size() - n_node_seg, TASK_PROD, kProdR);
    // the clause list is padded to whole groups of 32; a task covers 1..kClausePerLane groups
    // (1, 2 or 4 groups: the kernel has one unrolled body for each; a tail that is not
    // a whole task is split into smaller powers of two)
    // records [0, n_clause) are clauses, [n_clause, n_clause + n_xor2) short XORs
    const int k = kn.clause_k ? kn.clause_k : clause_groups_per_task((n_clause + n_xor2) / 32, (int)ts.tasks.size(), warps);
    for (int part = 0; part < 2; ++part) {
        const int kind = part == 0 ? TASK_CLAUSE : TASK_XOR2;
        const int end = part == 0 ? n_clause : n_clause + n_xor2;
        int c = part == 0 ? 0 : n_clause;
        for (int kk = k; kk >= 1; kk >>= 1)
            for (; c + 32 * kk <= end; c += 32 * kk) ts.tasks.push_back(make_int4(kind, c, 32 * kk, 0));
    }
    // node tasks first (the longest), then product tasks spread evenly among the
    // first quarter of the clause tasks: their long dependent chains overlap
    // with clause work in other warps instead of all warps starting on them at
    // once, and the end of every iteration is left to short clause tasks
    // (CNF-XOR step, two points per CTA: over the first three quarters 1.516 ms,
    // a half 1.473, a quarter 1.474; one point per CTA, 152 points: 0.972 and,
    // over a quarter, 0.950 ms)
    {
        std::vector<int4> node, prod, rest;
        for (const int4 &t : ts.tasks) {
            const int kd = t.x & 0xff;
            (kd == TASK_NODE ? node : (kd == TASK_PROD ? prod : rest)).push_back(t);
        }
        std::vector<int4> out = node;
        const size_t np = prod.size(), nc = rest.size();
        const size_t nc_mix = nc / 4;
        size_t ip = 0, ic = 0;
        while (ip < np || ic < nc) {
            // keep the product share of the emitted tasks at np / (np + nc_mix)
            if (ip < np && (ic >= nc_mix || (ip + 1) * (np + nc_mix) <= (ip + ic + 1) * np)) out.push_back(prod[ip++]);
            else out.push_back(rest[ic++]);
        }
        ts.tasks.swap(out);
    }
}

int smem_mode_for(int n, size_t elem, size_t image_bytes, int max_smem, size_t &bytes) {
    const size_t npad = ((size_t)n + 2 + 3) & ~size_t(3);  // two dummy variables, rounded to 4
    const size_t budget = max_smem > 2048 ? (size_t)max_smem - 1024 : 0;
    // FP32 resident mode keeps the gradient as two int32 words and one FP32 word per
    // variable; FP64 keeps two int32 fixed-point words and one FP64 product word
    const size_t xg = elem == 4 ? 2 * npad * 4 : 3 * npad * 8;
    const size_t res_xg = elem == 4 ? 4 * npad * 4 : xg;
    if (res_xg + image_bytes <= budget) {
        bytes = res_xg + image_bytes;
        return SMEM_RES;
    }
    if (xg <= budget) {
        bytes = xg;
        return SMEM_FULL;
    }
    if (npad * elem <= budget) {
        bytes = npad * elem;
        return SMEM_X;
    }
    bytes = 0;
    return SMEM_NONE;
}

using FusedFn = cudaError_t (*)(const DevView &, int, const FusedArgs &, size_t, int, cudaStream_t, bool);

FusedFn launcher_for(bool f64, int nr) {
    if (f64) return nr == 0 ? fused_f64_r0 : (nr == 8 ? fused_f64_r8 : fused_f64_r16);
    return nr == 0 ? fused_f32_r0 : (nr == 8 ? fused_f32_r8 : fused_f32_r16);
}

// Scales of the two-word fixed-point accumulator: a contribution is bounded by
// its weight (|dFE/dy| <= 1, with a margin for rounding).  Each weight is
// bounded by b_c = max(w_c, 1), which also bounds every later ERWA weight
// ((1 - a) w + a r <= b_c for r in [0, 1]); with wmax and Dmax taken over b_c, S1 =
// min(21 - ceil(log2 wmax), 30 - ceil(log2 Dmax)) the hi word is rounded
// exactly (|c 2^S1| < 2^22) and never exceeds 2^30 in sum (Dmax = largest
// weighted variable degree); the residual lies in [-1/2, 1/2], so with
// S2 = min(22, 30 - ceil(log2 degmax)) the lo word is exact and bounded too
// (the kernel adds the lo word only where S1 + floor(log2 bmin) < 20, bmin the
// smallest b_c of a positive weight).
// The FP64 cluster step rounds each contribution to an integer V = c 2^S64
// and adds it as two 32-bit words, lo = V mod 2^L and hi = floor(V / 2^L):
// L = 32 - ceil(log2(degmax + 1)) keeps the lo sums below 2^32, and
// S64 = min(30 + L - e_d, 50 - e_w) keeps the hi sums below 2^31 and |V| below
// 2^51 (the range of the kernel's one-FMA rounding).  At unit weights that is
// 2^-50 per contribution, near FP64's own rounding of the sums it replaces;
// coarser than 2^-44 (very high degrees or weights) the library keeps one CTA
// per point.
void fixed_point_scales(ffsat_instance *I) {
    std::vector<double> D((size_t)I->n, 0.0);
    std::vector<int32_t> deg((size_t)I->n, 0);
    double wmax = 0.0, wmin = 0.0;  // over b_c = max(w_c, 1) of the weighted constraints
    for (int32_t c = 0; c < I->m; ++c) {
        if (I->cls[c] == CLS_CONST) continue;
        const double bc = std::max(I->w[c], 1.0);
        wmax = std::max(wmax, bc);
        if (I->w[c] > 0.0 && (wmin == 0.0 || bc < wmin)) wmin = bc;
        for (int64_t i = I->row_ptr[c]; i < I->row_ptr[c + 1]; ++i) {
            const int32_t l = I->lits_in[i];
            const int32_t v = (l > 0 ? l : -l) - 1;
            D[v] += bc;
            deg[v] += 1;
        }
    }
    double dmax = 0.0;
    int32_t gmax = 1;
    for (int32_t v = 0; v < I->n; ++v) {
        dmax = std::max(dmax, D[v]);
        gmax = std::max(gmax, deg[v]);
    }
    if (wmax <= 0.0) wmax = 1.0;
    if (dmax <= 0.0) dmax = 1.0;
    const int e_w = (int)std::ceil(std::log2(wmax * 1.0625));
    const int e_d = (int)std::ceil(std::log2(dmax * 1.0625 + 1.0));
    const int S1 = std::min(21 - e_w, 30 - e_d);
    const int S2 = std::min(22, 30 - (int)std::ceil(std::log2((double)gmax + 1.0)));
    I->fix_s1 = std::ldexp(1.0f, S1);
    I->fix_s2 = std::ldexp(1.0f, S2);
    I->fix_i1 = std::ldexp(1.0f, -S1);
    I->fix_i12 = std::ldexp(1.0f, -(S1 + S2));
    // the hi word alone rounds each contribution to 2^-S1, 2^-(S1 + log2 bmin)
    // of the smallest bound b_c = max(w_c, 1): enough (FP32 itself rounds sums
    // to 2^-24) from 2^-20 on.  b_c, not w_c, so that ERWA's weights (which
    // stay below b_c) keep the choice, and a resumed search with the same bits
    I->fix_two = (wmin == 0.0 || S1 + (int)std::floor(std::log2(wmin)) >= 20) ? 0 : 1;
    const int L = 32 - (int)std::ceil(std::log2((double)gmax + 1.0));
    const int S64 = std::min(30 + L - e_d, 50 - e_w);
    I->fix64_s = std::ldexp(1.0, S64);
    I->fix64_i = std::ldexp(1.0, -S64);
    I->fix64_l = L;
    I->fix64_ok = S64 >= 44 && L >= 1;
}

void fill_weights(ffsat_instance *I) {
    fixed_point_scales(I);
    I->f_const = 0.0;
    I->f_const_plain = 0.0;
    for (int32_t c = 0; c < I->m; ++c) {
        const double wc = I->w[c];
        I->cons_wd[c] = wc;
        const int s = I->slot[c];
        switch (I->cls[c]) {
        case CLS_CLAUSE3: {
            const float wf = (float)wc;
            std::memcpy(&I->clauses[s].w, &wf, 4);
            I->clause_wd[s] = wc;
            I->f_const -= wc;  // the kernel accumulates 2 w prod q; FE = 2 prod q - 1
            break;
        }
        case CLS_XOR2: {  // FE = w prod y: no constant part
            const float wf = (float)wc;
            std::memcpy(&I->clauses[s].w, &wf, 4);
            I->clause_wd[s] = wc;
            break;
        }
        case CLS_PRODUCT:
        case CLS_NODE: {
            const float wf = (float)wc;
            std::memcpy(&I->seg_info[s].w, &wf, 4);
            I->seg_wd[s] = wc;
            break;
        }
        default: {
            double fe = 0.0;
            constant_value(I->type[c], I->param[c], I->len[c], fe);
            I->f_const += wc * fe;
            I->f_const_plain += wc * fe;
        }
        }
    }
}

// Literal placement of one product-path warp task (32 lanes; segment j of the
// task owns lanes [j G, j G + G), each lane kProdR slots starting at the
// segment's offset).  Position r of every lane is one gather and one
// scatter-add instruction of the warp, so we fill the task position by
// position with a maximum bipartite matching of lanes to shared-memory banks
// (bank = variable mod 32): a lane may take any literal still left in its
// segment (the product is order-free), a segment places at least as many
// literals at each position as its remaining slots require, and lanes that
// need not place a literal get the padding literal.  Literals that cannot be
// placed without a conflict are placed anyway.
void bank_place_products(std::vector<int32_t> &lits, const std::vector<int4> &meta, int4 task, int32_t pad) {
    constexpr int RL = kProdR;
    const int G = (task.x >> 8) & 0xff;
    const int nseg = task.z;
    const int lanes = nseg * G;
    std::vector<std::vector<int32_t>> pool(nseg);
    std::vector<int32_t> base(nseg);
    for (int j = 0; j < nseg; ++j) {
        const int4 m = meta[task.y + j];
        base[j] = m.x;
        for (int t = 0; t < G * RL; ++t) {
            const int32_t l = lits[(size_t)m.x + t];
            if (l != pad) pool[j].push_back(l);
        }
    }
    std::vector<int32_t> out((size_t)lanes * RL, pad);
    for (int r = 0; r < RL; ++r) {
        int owner[32];
        std::fill(owner, owner + 32, -1);
        std::vector<int32_t> pick(lanes, -1);  // index into the segment's pool
        std::function<bool(int, uint32_t &)> augment = [&](int l, uint32_t &seen) -> bool {
            const auto &P = pool[l / G];
            for (size_t t = 0; t < P.size(); ++t) {
                const int bk = (int)((uint32_t)P[t] & 31u);
                if (seen & (1u << bk)) continue;
                seen |= 1u << bk;
                if (owner[bk] < 0 || augment(owner[bk], seen)) {
                    owner[bk] = l;
                    pick[l] = (int32_t)t;
                    return true;
                }
            }
            return false;
        };
        // lanes that must place a literal first, then the optional ones
        std::vector<int> need(nseg);
        for (int j = 0; j < nseg; ++j) need[j] = std::max(0, (int)pool[j].size() - G * (RL - 1 - r));
        for (int pass = 0; pass < 2; ++pass)
            for (int l = 0; l < lanes; ++l) {
                const int j = l / G, sl = l % G;
                const bool required = sl < need[j];
                if (required != (pass == 0) || pool[j].empty() || sl >= (int)pool[j].size()) continue;
                uint32_t seen = 0;
                augment(l, seen);
            }
        // take the matched literals out of the pools (largest pool index first per segment)
        std::vector<std::vector<std::pair<int32_t, int>>> taken(nseg);
        for (int bk = 0; bk < 32; ++bk)
            if (owner[bk] >= 0) taken[owner[bk] / G].push_back({pick[owner[bk]], owner[bk]});
        for (int j = 0; j < nseg; ++j) {
            auto &T = taken[j];
            std::sort(T.begin(), T.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
            for (const auto &pr : T) {
                out[(size_t)pr.second * RL + r] = pool[j][pr.first];
                pool[j].erase(pool[j].begin() + pr.first);
            }
            // required lanes left unmatched take the literal whose bank is least used
            int placed = (int)T.size();
            for (int sl = 0; sl < G && placed < need[j]; ++sl) {
                const int l = j * G + sl;
                if (out[(size_t)l * RL + r] != pad || pool[j].empty()) continue;
                int load[32] = {0};
                for (int ll = 0; ll < lanes; ++ll) {
                    const int32_t v = out[(size_t)ll * RL + r];
                    if (v != pad) load[(uint32_t)v & 31u]++;
                }
                size_t best = 0;
                for (size_t t = 1; t < pool[j].size(); ++t)
                    if (load[(uint32_t)pool[j][t] & 31u] < load[(uint32_t)pool[j][best] & 31u]) best = t;
                out[(size_t)l * RL + r] = pool[j][best];
                pool[j].erase(pool[j].begin() + best);
                ++placed;
            }
        }
    }
    for (int j = 0; j < nseg; ++j)
        std::memcpy(lits.data() + base[j], out.data() + (size_t)j * G * RL, (size_t)G * RL * sizeof(int32_t));
}

// Image k = {tasks | clauses | segmeta | segment literals}, each part 16-byte
// aligned.  Segment s of length L on lanes G = seg_lanes(L, R) occupies G * R
// literal slots; lane sl reads slots [sl R, sl R + R).  Unused slots hold the
// padding literal (dummy variable n, or n + 1 for paper-form node factors).
void build_image(ffsat_instance *I, int k) {
    const int nr = I->nr[k];
    std::vector<int4> meta(I->seg_info.size());
    std::vector<int32_t> lits;
    for (size_t s = 0; s < I->seg_info.size(); ++s) {
        const int4 si = I->seg_info[s];
        const bool node = (int)s < I->n_node_seg;
        const int R = node ? node_nr(si.y, nr, I->opt.form == FFSAT_FORM_STABLE, I->knobs[k].shape, k == 0) : kProdR;
        const int G = seg_lanes(si.y, R);
        const int32_t pad = node ? I->pad_node : I->n;
        const int32_t off = (int32_t)lits.size();
        lits.insert(lits.end(), I->seg_lits.begin() + si.x, I->seg_lits.begin() + si.x + si.y);
        // every segment starts on a 16-byte boundary (lanes of 10 or 14 literals
        // leave odd pairs at the end of one-lane segments)
        lits.resize(((size_t)off + (size_t)G * R + 3) & ~size_t(3), pad);
        meta[s] = make_int4(off, si.y, si.z, si.w);
    }
    for (const int4 &t : I->tasks[k])
        if ((t.x & 0xff) == TASK_PROD) bank_place_products(lits, meta, t, I->n);
    std::vector<int4> &img = I->image[k];
    img.clear();
    I->img_off[k][0] = (int32_t)img.size();
    img.insert(img.end(), I->tasks[k].begin(), I->tasks[k].end());
    I->img_off[k][1] = (int32_t)img.size();
    img.insert(img.end(), I->clauses.begin(), I->clauses.end());
    I->img_off[k][2] = (int32_t)img.size();
    img.insert(img.end(), meta.begin(), meta.end());
    I->img_off[k][3] = (int32_t)img.size();
    const size_t nl = lits.size();
    const size_t base = img.size();
    img.resize(base + (nl + 3) / 4, make_int4(I->n, I->n, I->n, I->n));
    if (nl) std::memcpy(reinterpret_cast<int32_t *>(img.data() + base), lits.data(), nl * sizeof(int32_t));
}

// Order clauses in groups of 32 (one per warp instruction) so that, literal
// position by literal position, the 32 variables of a group fall into distinct
// shared-memory banks (bank = variable mod 32).  A group is conflict-free iff
// every bank occurs exactly 3 times among its 96 literals: its clause-bank
// incidence graph is then 3-regular bipartite and splits into 3 perfect
// matchings (one per literal position).  Packing: best fit of each clause into
// the fullest group that still has capacity 3 per bank, leftovers where they
// exceed the capacity least; positions: one maximum matching per position.
void bank_order(std::vector<int4> &cls, std::vector<int32_t> &cid) {
    const size_t m = cls.size();
    if (m == 0) return;
    const size_t G = (m + 31) / 32;
    std::vector<std::array<uint8_t, 32>> cap(G);
    for (auto &c : cap) c.fill(3);
    std::vector<int> size(G, 0);
    std::vector<std::vector<int32_t>> members(G);
    auto banks = [&](size_t i) {
        const int4 &c = cls[i];
        return std::array<int, 3>{(int)((uint32_t)c.x & 31u), (int)((uint32_t)c.y & 31u), (int)((uint32_t)c.z & 31u)};
    };
    // groups with free slots, kept ordered by size (fullest first) through buckets
    std::vector<std::vector<int32_t>> by_size(33);
    for (size_t g = 0; g < G; ++g) by_size[0].push_back((int32_t)g);
    std::vector<int32_t> where(G, 0);  // index of g inside by_size[size[g]]
    for (size_t g = 0; g < G; ++g) where[g] = (int32_t)g;
    auto move_group = [&](int32_t g, int from, int to) {
        auto &vf = by_size[from];
        const int32_t last = vf.back();
        vf[where[g]] = last;
        where[last] = where[g];
        vf.pop_back();
        where[g] = (int32_t)by_size[to].size();
        by_size[to].push_back(g);
    };
    std::vector<int32_t> left;
    for (size_t i = 0; i < m; ++i) {
        const auto b = banks(i);
        int found = -1;
        int probes = 0;
        constexpr int kMaxProbe = 256;  // groups examined per clause (fullest first)
        for (int sz = 31; sz >= 0 && found < 0 && probes < kMaxProbe; --sz) {
            for (int32_t g : by_size[sz]) {
                if (++probes > kMaxProbe) break;
                uint8_t need[32] = {0};
                bool ok = true;
                for (int q = 0; q < 3 && ok; ++q) ok = cap[g][b[q]] > need[b[q]]++;
                if (ok) {
                    found = g;
                    break;
                }
            }
        }
        if (found < 0) {
            left.push_back((int32_t)i);
            continue;
        }
        for (int q = 0; q < 3; ++q) cap[found][b[q]]--;
        members[found].push_back((int32_t)i);
        move_group(found, size[found], size[found] + 1);
        size[found]++;
    }
    for (int32_t i : left) {
        const auto b = banks(i);
        int best = -1, best_cost = 1 << 30;
        for (size_t g = 0; g < G && best_cost > 0; ++g) {
            if (size[g] >= 32) continue;
            int cost = 0;
            uint8_t need[32] = {0};
            for (int q = 0; q < 3; ++q) cost += cap[g][b[q]] > need[b[q]]++ ? 0 : 1;
            if (cost < best_cost) {
                best_cost = cost;
                best = (int)g;
            }
        }
        for (int q = 0; q < 3; ++q) cap[best][b[q]] = cap[best][b[q]] ? cap[best][b[q]] - 1 : 0;
        members[best].push_back(i);
        size[best]++;
    }
    // literal positions by maximum bipartite matching (clauses x banks), position by position
    std::vector<int4> out;
    std::vector<int32_t> out_id;
    out.reserve(G * 32);
    out_id.reserve(G * 32);
    for (size_t g = 0; g < G; ++g) {
        const auto &mem = members[g];
        const int k = (int)mem.size();
        std::vector<std::array<int32_t, 3>> lit(k);
        std::vector<std::array<bool, 3>> used(k);
        std::vector<std::array<int32_t, 3>> pos(k);
        for (int c = 0; c < k; ++c) {
            const int4 &r = cls[mem[c]];
            lit[c] = {r.x, r.y, r.z};
            used[c] = {false, false, false};
        }
        for (int q = 0; q < 3; ++q) {
            int owner_c[32], owner_k[32];
            std::fill(owner_c, owner_c + 32, -1);
            std::function<bool(int, uint32_t &)> augment = [&](int c, uint32_t &seen) -> bool {
                for (int t = 0; t < 3; ++t) {
                    if (used[c][t]) continue;
                    const int bk = (int)((uint32_t)lit[c][t] & 31u);
                    if (seen & (1u << bk)) continue;
                    seen |= 1u << bk;
                    if (owner_c[bk] < 0 || augment(owner_c[bk], seen)) {
                        owner_c[bk] = c;
                        owner_k[bk] = t;
                        return true;
                    }
                }
                return false;
            };
            for (int c = 0; c < k; ++c) {
                uint32_t seen = 0;
                augment(c, seen);
            }
            std::vector<int> chosen(k, -1);
            for (int bk = 0; bk < 32; ++bk)
                if (owner_c[bk] >= 0) chosen[owner_c[bk]] = owner_k[bk];
            for (int c = 0; c < k; ++c) {
                int t = chosen[c];
                if (t < 0)
                    for (t = 0; used[c][t]; ++t) {
                    }
                used[c][t] = true;
                pos[c][q] = lit[c][t];
            }
        }
        for (int c = 0; c < k; ++c) {
            out.push_back(make_int4(pos[c][0], pos[c][1], pos[c][2], cls[mem[c]].w));
            out_id.push_back(cid[mem[c]]);
        }
    }
    cls.swap(out);
    cid.swap(out_id);
}

// DevView of image k on top of the shared part V.
DevView view_for_image(ffsat_instance *P, const DevView &V, int k) {
    DevView W = V;
    const int4 *img = P->d_img[k];
    W.res_image = img;
    W.res_int4 = (int32_t)P->image[k].size();
    W.res_off_tasks = P->img_off[k][0];
    W.res_off_clauses = P->img_off[k][1];
    W.res_off_segmeta = P->img_off[k][2];
    W.res_off_lits = P->img_off[k][3];
    W.tasks = img + W.res_off_tasks;
    W.clauses = img + W.res_off_clauses;
    W.segmeta = img + W.res_off_segmeta;
    W.seg_lits = reinterpret_cast<const int32_t *>(img + W.res_off_lits);
    W.n_task = (int32_t)P->tasks[k].size();
    return W;
}

// Warp tasks and resident image k (0: FP32, 1: FP64) from the instance's node R
// family nr[k] and tile choices knobs[k].
void rebuild_image(ffsat_instance *P, int k) {
    TaskSet ts;
    build_tasks(P->seg_len, P->n_node_seg, P->n_clause_pad, P->n_xor2_pad, P->nr[k],
                fused_threads(k == 1, P->nr[k]) / 32, P->opt.form == FFSAT_FORM_STABLE, P->knobs[k], ts, k == 0);
    P->tasks[k] = ts.tasks;
    build_image(P, k);
}

// Every literal the kernels will index must name a variable or one of the two dummies.
int check_image(const ffsat_instance *P, int k) {
    const int32_t *w = reinterpret_cast<const int32_t *>(P->image[k].data());
    for (size_t i = (size_t)P->img_off[k][1] * 4; i < (size_t)P->img_off[k][2] * 4; ++i)
        if ((i & 3) != 3 && ((uint32_t)w[i] & 0x7fffffffu) > (uint32_t)P->n + 1)
            return fail(FFSAT_ERR_PARAM, "internal: clause record %zu out of range", i / 4);
    for (size_t i = (size_t)P->img_off[k][3] * 4; i < P->image[k].size() * 4; ++i)
        if (((uint32_t)w[i] & 0x7fffffffu) > (uint32_t)P->n + 1)
            return fail(FFSAT_ERR_PARAM, "internal: segment literal %zu out of range", i);
    return FFSAT_OK;
}

// (Re)allocate and upload resident image k (the device must be current).
int upload_image(ffsat_instance *P, int k) {
    if (P->d_img[k]) CUDA_TRY(cudaFree(P->d_img[k]));
    P->d_img[k] = nullptr;
    const size_t bytes = P->image[k].size() * sizeof(int4);
    CUDA_TRY(cudaMalloc(&P->d_img[k], std::max<size_t>(bytes, 16)));
    CUDA_TRY(cudaMemcpy(P->d_img[k], P->image[k].data(), bytes, cudaMemcpyHostToDevice));
    return FFSAT_OK;
}

// FP64 shared-memory mode: the gradient in shared memory is the two-word fixed
// point (Fix64Acc); where its resolution would be coarser than 2^-44 (very high
// degrees or weights) the instance keeps the gradient in a global row instead
// (SMEM_X, native FP64 global atomics).
void fp64_mode(ffsat_instance *P) {
    P->smem_mode64 = smem_mode_for(P->n, sizeof(double), P->image[1].size() * sizeof(int4), P->max_smem, P->smem64);
    if (!P->fix64_ok && (P->smem_mode64 == SMEM_FULL || P->smem_mode64 == SMEM_RES)) {
        P->smem_mode64 = SMEM_X;
        P->smem64 = (((size_t)P->n + 2 + 3) & ~size_t(3)) * sizeof(double);
    }
    P->info.smem_mode_f64 = P->smem_mode64;
    P->info.smem_bytes_f64 = (int64_t)P->smem64;
}

// Tile choices found by earlier loads, keyed by the instance's shape (sizes,
// path counts, longest node constraint, node work, form): an instance of the
// same shape reuses them without timing.
using TuneKey = std::array<int64_t, 10>;
struct TuneChoice {
    int nr;
    Knobs kn;
    float default_us, best_us;
    int candidates;
};
std::mutex &tune_mutex() {
    static std::mutex mu;
    return mu;
}
std::map<TuneKey, TuneChoice> &tune_cache() {
    static std::map<TuneKey, TuneChoice> cache;
    return cache;
}
TuneKey tune_key(const ffsat_instance *P) {
    int64_t node_work = 0;
    for (int s = 0; s < P->n_node_seg; ++s) node_work += (int64_t)((P->seg_len[s] + 1) / 2 + 1) * P->seg_len[s];
    return {P->n, P->m, P->nnz, P->n_node_seg, (int64_t)P->seg_len.size() - P->n_node_seg, P->n_clause_pad,
            P->n_xor2_pad, P->max_node_len, node_work, P->opt.form};
}

// The FP32 autotuner.  It times one evaluation of F and grad F
// (min over three launches after a warm-up) on a probe batch of two points per
// SM, for each candidate image in a coordinate search, and keeps the fastest:
//   1. node literals per lane: the 16/12/8 family with the cost-model segment
//      shape (default), the fewest lanes per segment or the fewest literal slots,
//      and the 8-literal family (constraints of at most 256 literals);
//   2. clause groups of 32 per clause task: automatic (default), 1, 2 or 4;
//   3. points per CTA: one (default) or two, which halves the copies of a
//      shared-memory-resident image.
// A candidate replaces the best only when at least 1% faster.  The choice is
// cached by instance shape.
int autotune(ffsat_instance *P, const DevView &V) {
    const TuneKey key = tune_key(P);
    {
        std::lock_guard<std::mutex> lock(tune_mutex());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            const TuneChoice &c = it->second;
            if (c.nr != P->nr[0] || !(c.kn == P->knobs[0])) {
                P->nr[0] = c.nr;
                P->knobs[0] = c.kn;
                rebuild_image(P, 0);
                int rc = check_image(P, 0);
                if (rc != FFSAT_OK) return rc;
                rc = upload_image(P, 0);
                if (rc != FFSAT_OK) return rc;
            }
            P->info.autotune_us[0] = c.default_us;
            P->info.autotune_us[1] = c.best_us;
            P->info.tune_candidates = 0;
            P->info.tune_cached = 1;
            goto apply;
        }
    }
    {
        const int B = 2 * P->num_sms;
        const size_t elems = (size_t)B * (size_t)P->n;
        std::vector<float> hx(elems);
        uint64_t st = 0x9E3779B97F4A7C15ull;
        for (size_t i = 0; i < elems; ++i) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            hx[i] = (float)((double)(st >> 40) / (double)(1ull << 23) - 1.0);
        }
        float *dx = nullptr, *dg = nullptr;
        double *df = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int rc = FFSAT_OK;
        int tried = 0;
        auto cleanup = [&]() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            cudaFree(dx);
            cudaFree(dg);
            cudaFree(df);
        };
        // time the image currently in slot 0 with points-per-CTA pts
        auto time_image = [&](int pts, float &us) -> int {
            size_t smem = 0;
            const int mode = smem_mode_for(P->n, sizeof(float), P->image[0].size() * sizeof(int4), P->max_smem, smem);
            const DevView W = view_for_image(P, V, 0);
            FusedArgs a{};
            a.B = B;
            a.mode = MODE_EVAL;
            a.x_in = dx;
            a.f = df;
            a.g = dg;
            const FusedFn fn = launcher_for(false, P->nr[0]);
            const int grid = (B + pts - 1) / pts;
            CUDA_TRY(fn(W, mode, a, smem, 0, 0, true));
            CUDA_TRY(fn(W, mode, a, smem, grid, 0, false));
            us = 1e30f;
            for (int r = 0; r < 3; ++r) {
                CUDA_TRY(cudaEventRecord(e0, 0));
                CUDA_TRY(fn(W, mode, a, smem, grid, 0, false));
                CUDA_TRY(cudaEventRecord(e1, 0));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                us = std::min(us, 1000.f * ms);
            }
            ++tried;
            return FFSAT_OK;
        };
        // build, upload and time candidate (nr, kn); keep it as the best if faster
        int best_nr = P->nr[0];
        Knobs best = P->knobs[0];
        float best_us = 0.f, default_us = 0.f;
        std::vector<int4> best_tasks = P->tasks[0];
        auto try_candidate = [&](int nr, const Knobs &kn) -> int {
            P->nr[0] = nr;
            P->knobs[0] = kn;
            rebuild_image(P, 0);
            if (P->tasks[0].size() == best_tasks.size() &&
                std::memcmp(P->tasks[0].data(), best_tasks.data(), best_tasks.size() * sizeof(int4)) == 0 &&
                kn.pts_per_cta == best.pts_per_cta)
                return FFSAT_OK;  // the same image as the best so far
            int r = check_image(P, 0);
            if (r == FFSAT_OK) r = upload_image(P, 0);
            float us = 0.f;
            if (r == FFSAT_OK) r = time_image(kn.pts_per_cta, us);
            if (r != FFSAT_OK) return r;
            if (us < 0.99f * best_us) {
                best_us = us;
                best_nr = nr;
                best = kn;
                best_tasks = P->tasks[0];
            }
            return FFSAT_OK;
        };
        if (cudaMalloc(&dx, elems * sizeof(float)) != cudaSuccess || cudaMalloc(&dg, elems * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&df, (size_t)B * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess ||
            cudaMemcpy(dx, hx.data(), elems * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cleanup();
            return fail(FFSAT_ERR_CUDA, "autotune: allocation or upload of the probe batch failed");
        }
        rc = time_image(best.pts_per_cta, default_us);
        best_us = default_us;
        // 1. node literals per lane
        if (rc == FFSAT_OK && P->n_node_seg > 0 && P->opt.node_r == 0) {
            for (int shape : {1, 2}) {
                if (rc != FFSAT_OK) break;
                Knobs kn = best;
                kn.shape = shape;
                rc = try_candidate(16, kn);
            }
            if (rc == FFSAT_OK && P->max_node_len <= 8 * 32) {
                Knobs kn = best;
                kn.shape = 0;
                rc = try_candidate(8, kn);
            }
        }
        // 2. clause groups per clause task
        if (rc == FFSAT_OK && P->n_clause_pad + P->n_xor2_pad >= 64) {
            for (int ck : {1, 2, 4}) {
                if (rc != FFSAT_OK) break;
                Knobs kn = best;
                kn.clause_k = ck;
                rc = try_candidate(best_nr, kn);
            }
        }
        // 3. points per CTA
        if (rc == FFSAT_OK) {
            Knobs kn = best;
            kn.pts_per_cta = 2;
            rc = try_candidate(best_nr, kn);
        }
        cleanup();
        if (rc != FFSAT_OK) return rc;
        // slot 0 holds the last candidate: rebuild the best
        P->nr[0] = best_nr;
        P->knobs[0] = best;
        rebuild_image(P, 0);
        rc = check_image(P, 0);
        if (rc == FFSAT_OK) rc = upload_image(P, 0);
        if (rc != FFSAT_OK) return rc;
        P->info.autotune_us[0] = default_us;
        P->info.autotune_us[1] = best_us;
        P->info.tune_candidates = tried;
        P->info.tune_cached = 0;
        std::lock_guard<std::mutex> lock(tune_mutex());
        tune_cache()[key] = TuneChoice{best_nr, best, default_us, best_us, tried};
    }
apply:
    P->V32 = view_for_image(P, V, 0);
    P->nr32 = P->nr[0];
    P->smem_mode32 = smem_mode_for(P->n, sizeof(float), P->image[0].size() * sizeof(int4), P->max_smem, P->smem32);
    CUDA_TRY(launcher_for(false, P->nr32)(P->V32, P->smem_mode32, FusedArgs{}, P->smem32, 0, 0, true));
    CUDA_TRY(cudaMemset(P->d_status, 0, sizeof(int32_t)));
    P->info.autotuned = 1;
    return FFSAT_OK;
}

}  // namespace

extern "C" {

void ffsat_default_options(ffsat_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->form = FFSAT_FORM_STABLE;
    opt->node_all = 0;
    opt->node_r = 0;
    opt->autotune = 0;
    opt->device = -1;
    opt->cluster = 0;
}

const char *ffsat_last_error(void) { return t_err.c_str(); }

int32_t ffsat_last_launch_count(void) { return t_launches; }

int32_t ffsat_last_cluster_size(void) { return t_cluster; }

int32_t ffsat_last_points_per_cta(void) { return t_pairs; }

int ffsat_load_instance(int32_t n_vars, int32_t n_cons, const int64_t *row_ptr, const int32_t *lits,
                        const uint8_t *type, const int32_t *param, const double *weights,
                        const ffsat_options *opt_in, ffsat_instance **out) {
    t_err.clear();
    if (!out) return fail(FFSAT_ERR_ARG, "out is NULL");
    *out = nullptr;
    ffsat_options opt;
    ffsat_default_options(&opt);
    if (opt_in) opt = *opt_in;
    int rc = validate(n_vars, n_cons, row_ptr, lits, type, param, weights, opt);
    if (rc != FFSAT_OK) return rc;

    std::unique_ptr<ffsat_instance> I(new ffsat_instance());
    ffsat_instance *P = I.get();
    P->n = n_vars;
    P->m = n_cons;
    P->nnz = row_ptr[n_cons];
    P->opt = opt;
    P->cls.resize(n_cons);
    P->slot.resize(n_cons);
    P->w.resize(n_cons);
    P->type.assign(type, type + n_cons);
    P->param.assign(param, param + n_cons);
    P->len.resize(n_cons);
    P->cons_wd.resize(n_cons);
    P->row_ptr.assign(row_ptr, row_ptr + n_cons + 1);
    P->lits_in.assign(lits, lits + P->nnz);

    // ---- classify ----
    std::vector<int32_t> node_c, prod_c, clause_c, const_c, xor2_c;
    for (int32_t c = 0; c < n_cons; ++c) {
        const int L = (int)(row_ptr[c + 1] - row_ptr[c]);
        P->len[c] = L;
        P->w[c] = weights ? weights[c] : 1.0;
        const int t = type[c];
        double fe;
        if (constant_value(t, param[c], L, fe)) {
            P->cls[c] = CLS_CONST;
            const_c.push_back(c);
        } else if (!opt.node_all && t == FFSAT_OR && L <= 3) {
            P->cls[c] = CLS_CLAUSE3;
            clause_c.push_back(c);
        } else if (!opt.node_all && t == FFSAT_XOR && L <= 2) {
            P->cls[c] = CLS_XOR2;
            xor2_c.push_back(c);
        } else if (!opt.node_all && t != FFSAT_ATLEAST && L <= 32 * kProdR) {
            P->cls[c] = CLS_PRODUCT;
            prod_c.push_back(c);
        } else {
            if (opt.form == FFSAT_FORM_PAPER && L > kPaperMaxLen)
                return fail(FFSAT_ERR_TOOLONG, "paper form supports constraints of <= %d literals (constraint %d has %d)",
                            kPaperMaxLen, c, L);
            P->cls[c] = CLS_NODE;
            node_c.push_back(c);
        }
    }
    auto by_len_desc = [&](int32_t a, int32_t b) { return P->len[a] > P->len[b] || (P->len[a] == P->len[b] && a < b); };
    std::stable_sort(node_c.begin(), node_c.end(), by_len_desc);
    std::stable_sort(prod_c.begin(), prod_c.end(), by_len_desc);

    // ---- node tables (one per distinct key), FP64 preprocessing ----
    std::map<std::tuple<int, int, int>, int32_t> tab_index;
    std::vector<float> tab_f;
    std::vector<double> tab_d;
    // the imaginary-node tables serve the stable form's node tasks, the generic
    // tables the paper form's and the plain FP64 comparator
    const bool node_imag = opt.form == FFSAT_FORM_STABLE;
    // entry 0 is an all-zero node (t = 0, C = D = 0): the node tasks read it past
    // the end of a segment that is shorter than the longest one of its task
    std::map<std::tuple<int, int, int>, int32_t> tab_im_index;
    std::vector<float> tab_im_f(4, 0.0f);
    std::vector<double> tab_im_d(4, 0.0);
    std::vector<int32_t> cons_tab(n_cons, -1), seg_tab(n_cons, -1);
    int max_node_len = 0;
    for (int32_t c : node_c) {
        const int L = P->len[c];
        const int t = type[c];
        const int p = t == FFSAT_OR ? 0 : (t == FFSAT_XOR ? (param[c] & 1) : param[c]);
        auto key = std::make_tuple(t, L, p);
        auto it = tab_index.find(key);
        if (it == tab_index.end()) {
            const int32_t off = (int32_t)(tab_f.size() / 8);
            build_table(t, p, L, opt.form, tab_f, tab_d);
            it = tab_index.emplace(key, off).first;
        }
        cons_tab[c] = it->second;
        seg_tab[c] = it->second;
        if (node_imag) {
            auto jt = tab_im_index.find(key);
            if (jt == tab_im_index.end()) {
                const int32_t off = (int32_t)(tab_im_f.size() / 4);
                build_table_im(t, p, L, tab_im_f, tab_im_d);
                jt = tab_im_index.emplace(key, off).first;
            }
            seg_tab[c] = jt->second;
        }
        max_node_len = std::max(max_node_len, L);
    }

    // ---- segments, clauses, CSR ----
    std::vector<int32_t> seg_len;
    std::vector<int32_t> &seg_lits = P->seg_lits;
    auto add_seg = [&](int32_t c, int32_t aux) {
        P->slot[c] = (int32_t)seg_len.size();
        P->seg_info.push_back(make_int4((int32_t)seg_lits.size(), P->len[c], aux, 0));
        seg_len.push_back(P->len[c]);
        for (int64_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) seg_lits.push_back(pack_lit(lits[i]));
    };
    for (int32_t c : node_c) add_seg(c, seg_tab[c]);
    for (int32_t c : prod_c) {
        const int t = type[c];
        add_seg(c, t == FFSAT_OR ? PROD_OR : ((param[c] & 1) ? PROD_XOR_ODD : PROD_XOR_EVEN));
    }
    P->n_node_seg = (int)node_c.size();
    P->pad_node = n_vars + 1;  // x = 0: a factor of exactly 1 in both node forms
    P->seg_wd.assign(seg_len.size(), 0.0);
    // clauses of <= 3 literals: bank-ordered, then padded to whole tasks with
    // zero-weight clauses on the dummy variable
    std::vector<int32_t> clause_ids = clause_c;
    P->clauses.resize(clause_c.size());
    for (size_t k = 0; k < clause_c.size(); ++k) {
        const int32_t c = clause_c[k];
        int32_t l3[3] = {n_vars, n_vars, n_vars};
        for (int64_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) l3[i - row_ptr[c]] = pack_lit(lits[i]);
        P->clauses[k] = make_int4(l3[0], l3[1], l3[2], 0);
    }
    bank_order(P->clauses, clause_ids);
    const size_t n_clause_pad = (clause_ids.size() + 31) / 32 * 32;
    P->clauses.resize(n_clause_pad, make_int4(n_vars, n_vars, n_vars, 0));
    clause_ids.resize(n_clause_pad, -1);
    // XOR constraints of <= 2 literals: records {l0, l1, dummy, w} after the
    // clauses, the dummy negated for even parity (FE = w y0 y1 y2), bank-ordered
    // and padded like the clauses
    std::vector<int4> x2(xor2_c.size());
    std::vector<int32_t> x2_ids = xor2_c;
    for (size_t k = 0; k < xor2_c.size(); ++k) {
        const int32_t c = xor2_c[k];
        int32_t l2[2] = {n_vars, n_vars};
        for (int64_t i = row_ptr[c]; i < row_ptr[c + 1]; ++i) l2[i - row_ptr[c]] = pack_lit(lits[i]);
        const int32_t dummy = (param[c] & 1) ? n_vars : (int32_t)((uint32_t)n_vars | 0x80000000u);
        x2[k] = make_int4(l2[0], l2[1], dummy, 0);
    }
    bank_order(x2, x2_ids);
    const size_t n_xor2_pad = (x2_ids.size() + 31) / 32 * 32;
    x2.resize(n_xor2_pad, make_int4(n_vars, n_vars, n_vars, 0));
    x2_ids.resize(n_xor2_pad, -1);
    P->clauses.insert(P->clauses.end(), x2.begin(), x2.end());
    clause_ids.insert(clause_ids.end(), x2_ids.begin(), x2_ids.end());
    const size_t n_rec = n_clause_pad + n_xor2_pad;
    P->clause_wd.assign(n_rec, 0.0);
    for (size_t k = 0; k < clause_ids.size(); ++k)
        if (clause_ids[k] >= 0) P->slot[clause_ids[k]] = (int32_t)k;
    for (int32_t c : const_c) P->slot[c] = -1;
    fill_weights(P);

    std::vector<int32_t> rp32(n_cons + 1), lp32((size_t)P->nnz);
    for (int32_t c = 0; c <= n_cons; ++c) rp32[c] = (int32_t)row_ptr[c];
    for (int64_t i = 0; i < P->nnz; ++i) lp32[i] = pack_lit(lits[i]);
    std::vector<int32_t> par32(param, param + n_cons);
    std::vector<int32_t> closed_ids;
    closed_ids.insert(closed_ids.end(), clause_c.begin(), clause_c.end());
    closed_ids.insert(closed_ids.end(), prod_c.begin(), prod_c.end());
    closed_ids.insert(closed_ids.end(), xor2_c.begin(), xor2_c.end());

    // ---- node R and task lists ----
    int nr32 = 0, nr64 = 0;
    if (!node_c.empty()) {
        nr32 = opt.node_r ? opt.node_r : 16;
        if (nr32 * 32 < max_node_len) nr32 = 16;
        nr64 = max_node_len <= 8 * 32 ? 8 : 16;
    }
    P->nr[0] = nr32;
    P->nr[1] = nr64;
    // FP64 steps on few points spread each point over a cluster of CTAs that
    // split the warp tasks: one clause group of 32 per task keeps every warp of
    // the cluster busy with a short task
    P->knobs[1].clause_k = 1;
    P->seg_len = seg_len;
    P->n_clause_pad = (int)n_clause_pad;
    P->n_xor2_pad = (int)n_xor2_pad;
    P->max_node_len = max_node_len;
    for (int k = 0; k < 2; ++k) {
        rebuild_image(P, k);
        rc = check_image(P, k);
        if (rc != FFSAT_OK) return rc;
    }

    // ---- device ----
    int dev = opt.device;
    if (dev < 0) CUDA_TRY(cudaGetDevice(&dev));
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(dev));
    P->device = dev;
    CUDA_TRY(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&P->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

    Arena A;
    P->off_clause_wd = A.put(P->clause_wd);
    P->off_seg_wd = A.put(P->seg_wd);
    const size_t o_tf = A.put(tab_f), o_td = A.put(tab_d);
    const size_t o_tif = A.put(tab_im_f), o_tid = A.put(tab_im_d);
    const size_t o_rp = A.put(rp32), o_lits = A.put(lp32), o_type = A.put(P->type), o_par = A.put(par32);
    const size_t o_ctab = A.put(cons_tab);
    P->off_cons_wd = A.put(P->cons_wd);
    P->off_f_const = A.put(std::vector<double>{P->f_const, P->f_const_plain});
    P->off_cls = A.put(P->cls);
    P->off_slot = A.put(P->slot);
    P->off_umax = A.put(std::vector<int32_t>{0});
    const size_t o_nid = A.put(node_c), o_cid = A.put(closed_ids);
    // start values of the FP32 fixed-point gradient words (see FixAcc): every
    // clause-record literal and every node-segment literal on a real variable
    // adds one raw magic-offset value per evaluation
    std::vector<int32_t> fix_bias(((size_t)n_vars + 2 + 3) & ~size_t(3), 0);
    {
        std::vector<uint32_t> deg((size_t)n_vars, 0);
        auto count = [&](int32_t lp) {
            const uint32_t v = (uint32_t)lp & 0x7fffffffu;
            if (v < (uint32_t)n_vars) deg[v]++;
        };
        for (const int4 &r : P->clauses) {
            count(r.x);
            count(r.y);
            count(r.z);
        }
        for (int s = 0; s < P->n_node_seg; ++s) {
            const int4 si = P->seg_info[s];
            for (int i = 0; i < si.y; ++i) count(P->seg_lits[(size_t)si.x + i]);
        }
        for (int32_t v = 0; v < n_vars; ++v) fix_bias[v] = (int32_t)(0u - deg[v] * 0x4B400000u);
    }
    const size_t o_bias = A.put(fix_bias);
    P->arena_bytes = A.host.size();
    CUDA_TRY(cudaMalloc(&P->d_arena, P->arena_bytes));
    CUDA_TRY(cudaMemcpy(P->d_arena, A.host.data(), P->arena_bytes, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(&P->d_status, sizeof(int32_t)));
    CUDA_TRY(cudaMemset(P->d_status, 0, sizeof(int32_t)));
    for (int k = 0; k < 2; ++k) {
        rc = upload_image(P, k);
        if (rc != FFSAT_OK) return rc;
    }

    unsigned char *base = P->d_arena;
    DevView V{};
    V.n = n_vars;
    V.m = n_cons;
    V.n_seg = (int32_t)seg_len.size();
    V.n_clause = (int32_t)n_rec;
    V.clause_wd = reinterpret_cast<const double *>(base + P->off_clause_wd);
    V.seg_wd = reinterpret_cast<const double *>(base + P->off_seg_wd);
    V.tab_f = reinterpret_cast<const float4 *>(base + o_tf);
    V.tab_d = reinterpret_cast<const double *>(base + o_td);
    V.tab_im_f = reinterpret_cast<const float4 *>(base + o_tif);
    V.tab_im_d = reinterpret_cast<const double *>(base + o_tid);
    V.node_form = node_imag ? NODE_FORM_IMAG : NODE_FORM_GENERIC;
    V.f_const = reinterpret_cast<const double *>(base + P->off_f_const);
    V.fix_s1 = P->fix_s1;
    V.fix_s2 = P->fix_s2;
    V.fix_i1 = P->fix_i1;
    V.fix_i12 = P->fix_i12;
    V.fix_two = P->fix_two;
    V.fix64_s = P->fix64_s;
    V.fix64_i = P->fix64_i;
    V.fix64_l = P->fix64_l;
    V.has_prod = (int32_t)seg_len.size() > P->n_node_seg ? 1 : 0;
    V.row_ptr = reinterpret_cast<const int32_t *>(base + o_rp);
    V.lits = reinterpret_cast<const int32_t *>(base + o_lits);
    V.type = reinterpret_cast<const uint8_t *>(base + o_type);
    V.param = reinterpret_cast<const int32_t *>(base + o_par);
    V.cons_tab = reinterpret_cast<const int32_t *>(base + o_ctab);
    V.cons_wd = reinterpret_cast<const double *>(base + P->off_cons_wd);
    V.fix_bias = reinterpret_cast<const int32_t *>(base + o_bias);
    V.status = P->d_status;
    P->V32 = view_for_image(P, V, 0);
    P->V64 = view_for_image(P, V, 1);
    P->d_node_ids = reinterpret_cast<int32_t *>(base + o_nid);
    P->d_closed_ids = reinterpret_cast<int32_t *>(base + o_cid);
    P->n_node_ids = (int32_t)node_c.size();
    P->n_closed_ids = (int32_t)closed_ids.size();
    P->nr32 = nr32;
    P->nr64 = nr64;

    P->smem_mode32 = smem_mode_for(n_vars, sizeof(float), P->image[0].size() * sizeof(int4), P->max_smem, P->smem32);
    fp64_mode(P);
    FusedArgs dummy{};
    CUDA_TRY(launcher_for(false, nr32)(P->V32, P->smem_mode32, dummy, P->smem32, 0, 0, true));
    CUDA_TRY(launcher_for(true, nr64)(P->V64, P->smem_mode64, dummy, P->smem64, 0, 0, true));
    if (opt.autotune) {
        rc = autotune(P, V);
        if (rc != FFSAT_OK) return rc;
        nr32 = P->nr32;
    }

    ffsat_info &inf = P->info;
    inf.n = n_vars;
    inf.m = n_cons;
    inf.nnz = P->nnz;
    inf.n_clause3 = (int32_t)clause_c.size();
    inf.n_xor2 = (int32_t)xor2_c.size();
    inf.smem_bytes_f32 = (int64_t)P->smem32;
    inf.smem_bytes_f64 = (int64_t)P->smem64;
    inf.n_product = (int32_t)prod_c.size();
    inf.n_node = (int32_t)node_c.size();
    inf.n_const = (int32_t)const_c.size();
    inf.n_tables = (int32_t)tab_index.size();
    inf.n_tasks = (int32_t)P->tasks[0].size();
    inf.node_r = nr32;
    inf.tune_shape = P->knobs[0].shape;
    inf.tune_clause_k = P->knobs[0].clause_k;
    inf.tune_pts_per_cta = P->knobs[0].pts_per_cta;
    inf.fix_words_f32 = P->fix_two ? 2 : 1;
    inf.smem_mode_f32 = P->smem_mode32;
    inf.smem_mode_f64 = P->smem_mode64;
    inf.threads_f32 = fused_threads(false, nr32);
    int64_t lane_work = 0;
    for (const int4 &t : P->tasks[0])
        if ((t.x & 0xff) == TASK_NODE) lane_work += (int64_t)t.w * 32 * ((t.x >> 16) & 0xff);
    inf.node_lane_work = lane_work;
    inf.device_bytes = (int64_t)P->arena_bytes;

    *out = I.release();
    return FFSAT_OK;
}

int ffsat_set_weights(ffsat_instance *I, const double *weights) {
    t_err.clear();
    if (!I || !weights) return fail(FFSAT_ERR_ARG, "NULL argument");
    for (int32_t c = 0; c < I->m; ++c)
        if (!(std::isfinite(weights[c]) && weights[c] >= 0.0)) return fail(FFSAT_ERR_WEIGHT, "constraint %d: bad weight", c);
    I->w.assign(weights, weights + I->m);
    fill_weights(I);
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    unsigned char *base = I->d_arena;
    for (int k = 0; k < I->n_images; ++k) {
        build_image(I, k);  // same tasks and tile choices: the same size
        CUDA_TRY(cudaMemcpy(I->d_img[k], I->image[k].data(), I->image[k].size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(base + I->off_clause_wd, I->clause_wd.data(), I->clause_wd.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(base + I->off_seg_wd, I->seg_wd.data(), I->seg_wd.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(base + I->off_cons_wd, I->cons_wd.data(), I->cons_wd.size() * sizeof(double), cudaMemcpyHostToDevice));
    const double fc[2] = {I->f_const, I->f_const_plain};
    CUDA_TRY(cudaMemcpy(base + I->off_f_const, fc, sizeof(fc), cudaMemcpyHostToDevice));
    for (DevView *W : {&I->V32, &I->V64}) {
        W->fix_s1 = I->fix_s1;
        W->fix_s2 = I->fix_s2;
        W->fix_i1 = I->fix_i1;
        W->fix_i12 = I->fix_i12;
        W->fix_two = I->fix_two;
        W->fix64_s = I->fix64_s;
        W->fix64_i = I->fix64_i;
        W->fix64_l = I->fix64_l;
    }
    I->info.fix_words_f32 = I->fix_two ? 2 : 1;
    fp64_mode(I);  // the fixed point's resolution follows the weights
    return FFSAT_OK;
}

static int check_dtype(int32_t dtype) {
    if (dtype != FFSAT_F32 && dtype != FFSAT_F64) return fail(FFSAT_ERR_ARG, "dtype must be FFSAT_F32 or FFSAT_F64");
    return FFSAT_OK;
}

// CTAs of a fused-kernel launch on B points: each CTA runs pts_per_cta points in
// turn (the image's tile choice; one by default).
static inline int grid_for(const ffsat_instance *I, bool f64, int32_t B) {
    const int k = std::max(1, I->knobs[f64 ? 1 : 0].pts_per_cta);
    return (B + k - 1) / k;
}

using ClusterFn = cudaError_t (*)(const DevView &, int, const FusedArgs &, size_t, size_t, int, int, cudaStream_t,
                                  int *);

static ClusterFn cluster_launcher(int nr) {
    return nr == 0 ? cluster_f64_r0 : (nr == 8 ? cluster_f64_r8 : cluster_f64_r16);
}

// CTAs per point for an FP64 fixed-step call on B points (ffsat_options.cluster):
// 1 for the one-CTA kernel, else the cluster size, with the cluster kernel's
// dynamic shared memory and the offset of its second gradient buffer.
static int step_cluster_size(ffsat_instance *I, int32_t B, int mode, size_t &smem, size_t &g1_off, int &cmode) {
    const int opt = I->opt.cluster;
    if (opt == 1 || (mode != SMEM_FULL && mode != SMEM_RES) || !I->fix64_ok) return 1;
    const size_t npad = ((size_t)I->n + 2 + 3) & ~size_t(3);
    // the one-CTA layout, then the second fixed-point and FP64 product words; a
    // resident image that leaves no room for them stays in global memory
    auto layout = [&](int m) {
        g1_off = ((m == SMEM_RES ? I->smem64 : 3 * npad * sizeof(double)) + 15) & ~size_t(15);
        smem = g1_off + 2 * npad * sizeof(double);
    };
    cmode = mode;
    layout(cmode);
    if (smem + 1024 > (size_t)I->max_smem && cmode == SMEM_RES) layout(cmode = SMEM_FULL);
    if (smem + 1024 > (size_t)I->max_smem) return 1;
    // more than half of an SM's shared memory: one CTA per SM, so that the CTAs of
    // the clusters do not share an SM's FP64 pipe while other SMs idle
    smem = std::max(smem, (size_t)I->max_smem / 2 + 1024);
    static const int sizes[3] = {2, 4, 8};
    for (int k = 2; k >= 0; --k) {
        const int cl = sizes[k];
        if (opt != 0 && cl != opt) continue;
        if (opt == 0 && ((int64_t)B * cl > I->num_sms || I->V64.n_task < cl)) continue;
        std::lock_guard<std::mutex> lock(I->cluster_mu);
        if (I->cluster_active[k] < 0) {
            int active = 0;
            if (cluster_launcher(I->nr64)(I->V64, cmode, FusedArgs{}, smem, g1_off, 1, cl, nullptr, &active) !=
                cudaSuccess) {
                (void)cudaGetLastError();
                active = 0;
            }
            I->cluster_active[k] = active;
        }
        if (I->cluster_active[k] >= (opt == 0 ? B : 1)) return cl;
    }
    return 1;
}

// Dynamic shared memory of the two-points-per-CTA step: the one-point layout
// (x | hi | lo | gf | image) plus the second point's x | hi | gf.
static size_t pair_smem(const ffsat_instance *I) {
    const size_t npad = ((size_t)I->n + 2 + 3) & ~size_t(3);
    return I->smem32 + 3 * npad * 4;
}

// Two points per CTA for an FP32 fixed step on the resident image with one
// fixed-point word, where the points would otherwise need more than one wave
// of one CTA per SM and the second point's words fit beside the image: each
// warp task then serves both points with one load of its records.
static bool step_pairs(const ffsat_instance *I, bool f64, int mode, const FusedArgs &a, int32_t B) {
    return !f64 && mode == SMEM_RES && !I->fix_two && a.mode == MODE_STEP && B > I->num_sms &&
           std::max(1, I->knobs[0].pts_per_cta) == 1 && pair_smem(I) + 1024 <= (size_t)I->max_smem;
}

// The fused step launch of ffsat_step and ffsat_step_noalloc.
static int launch_step(ffsat_instance *I, bool f64, int mode, const FusedArgs &a, int32_t B, void *stream) {
    const DevView &V = f64 ? I->V64 : I->V32;
    size_t csmem = 0, g1_off = 0;
    int cmode = mode;
    const int cl = f64 ? step_cluster_size(I, B, mode, csmem, g1_off, cmode) : 1;
    bool pairs = false;
    if (cl > 1) {
        CUDA_TRY(cluster_launcher(I->nr64)(V, cmode, a, csmem, g1_off, B, cl, static_cast<cudaStream_t>(stream),
                                           nullptr));
    } else if ((pairs = step_pairs(I, f64, mode, a, B))) {
        // two points per CTA: the second point's x and gradient words after the image
        FusedArgs ap = a;
        ap.pairs = 1;
        CUDA_TRY(launcher_for(false, I->nr32)(V, mode, ap, pair_smem(I), (B + 1) / 2, static_cast<cudaStream_t>(stream),
                                              false));
    } else {
        CUDA_TRY(launcher_for(f64, f64 ? I->nr64 : I->nr32)(V, mode, a, f64 ? I->smem64 : I->smem32, grid_for(I, f64, B),
                                                              static_cast<cudaStream_t>(stream), false));
    }
    t_cluster = cl;
    t_pairs = pairs ? 2 : 1;
    t_launches = 1;
    return FFSAT_OK;
}

int ffsat_eval_grad(ffsat_instance *I, int32_t B, const void *x, int32_t dtype, double *f, void *g, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (B < 0) return fail(FFSAT_ERR_ARG, "B must be >= 0");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    const bool f64 = dtype == FFSAT_F64;
    FusedArgs a{};
    a.B = B;
    a.mode = MODE_EVAL;
    a.x_in = x;
    a.x_out = nullptr;
    a.f = f;
    a.g = g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const DevView &V = f64 ? I->V64 : I->V32;
    CUDA_TRY(launcher_for(f64, f64 ? I->nr64 : I->nr32)(V, f64 ? I->smem_mode64 : I->smem_mode32, a,
                                                          f64 ? I->smem64 : I->smem32, grid_for(I, f64, B), s, false));
    t_launches = 1;
    return FFSAT_OK;
}

int ffsat_eval_grad_plain64(ffsat_instance *I, int32_t B, const double *x, double *f, double *g, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (B < 0) return fail(FFSAT_ERR_ARG, "B must be >= 0");
    if (B == 0) return FFSAT_OK;
    if (!x || !f || !g) return fail(FFSAT_ERR_ARG, "x, f and g are required");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    int nl = 0;
    CUDA_TRY(launch_plain64(I->V64, B, x, f, g, I->n_node_ids, I->d_node_ids, I->n_closed_ids, I->d_closed_ids,
                            static_cast<cudaStream_t>(stream), &nl));
    t_launches = nl;
    return FFSAT_OK;
}

int ffsat_step(ffsat_instance *I, int32_t B, void *x, int32_t dtype, const ffsat_step_args *args, uint8_t *solved,
               int32_t *n_unsat, void *stream) {
    t_err.clear();
    t_launches = 0;
    t_cluster = 1;
    t_pairs = 1;
    if (!I || !args) return fail(FFSAT_ERR_ARG, "NULL argument");
    if (B < 0 || args->T < 0) return fail(FFSAT_ERR_ARG, "B and T must be >= 0");
    if (!std::isfinite(args->lr)) return fail(FFSAT_ERR_ARG, "lr must be finite");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    const bool f64 = dtype == FFSAT_F64;
    const int mode = f64 ? I->smem_mode64 : I->smem_mode32;
    const size_t elem = f64 ? sizeof(double) : sizeof(float);
    FusedArgs a{};
    a.B = B;
    a.mode = MODE_STEP;
    a.x_in = x;
    a.x_out = x;
    a.solved = solved;
    a.n_unsat = n_unsat;
    a.sp.T = args->T;
    a.sp.restart = args->restart;
    a.sp.lr = args->lr;
    a.sp.seed = args->seed;
    a.sp.epoch = args->epoch;
    a.sp.b_offset = args->b_offset;
    a.unsat_counts = args->unsat_counts;
    // the gradient lives in shared memory in modes SMEM_FULL and SMEM_RES; the
    // other two accumulate it in a [B, n] scratch
    if (mode == SMEM_X || mode == SMEM_NONE) {
        const size_t need = (size_t)B * (size_t)I->n * elem;
        if (need > I->scratch_bytes) {
            if (I->d_scratch) CUDA_TRY(cudaFree(I->d_scratch));
            I->d_scratch = nullptr;
            I->scratch_bytes = 0;
            CUDA_TRY(cudaMalloc(&I->d_scratch, need));
            I->scratch_bytes = need;
        }
        a.g_scratch = I->d_scratch;
    }
    return launch_step(I, f64, mode, a, B, stream);
}

int ffsat_step_noalloc(ffsat_instance *I, int32_t B, void *x, int32_t dtype, const ffsat_step_args *args,
                       uint8_t *solved, int32_t *n_unsat, void *stream) {
    t_err.clear();
    t_launches = 0;
    t_cluster = 1;
    t_pairs = 1;
    if (!I || !args) return fail(FFSAT_ERR_ARG, "NULL argument");
    if (B < 0 || args->T < 0) return fail(FFSAT_ERR_ARG, "B and T must be >= 0");
    if (!std::isfinite(args->lr)) return fail(FFSAT_ERR_ARG, "lr must be finite");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    const bool f64 = dtype == FFSAT_F64;
    const int mode = f64 ? I->smem_mode64 : I->smem_mode32;
    const size_t elem = f64 ? sizeof(double) : sizeof(float);
    FusedArgs a{};
    a.B = B;
    a.mode = MODE_STEP;
    a.x_in = x;
    a.x_out = x;
    a.solved = solved;
    a.n_unsat = n_unsat;
    a.sp.T = args->T;
    a.sp.restart = args->restart;
    a.sp.lr = args->lr;
    a.sp.seed = args->seed;
    a.sp.epoch = args->epoch;
    a.sp.b_offset = args->b_offset;
    a.unsat_counts = args->unsat_counts;
    if (mode != SMEM_FULL && mode != SMEM_RES) {
        const size_t need = (size_t)B * (size_t)I->n * elem;
        if (need > (size_t)FFSAT_STATIC_SCRATCH_BYTES)
            return fail(FFSAT_ERR_ARG, "B * n * %zu = %zu bytes of gradient scratch exceed the static %u bytes",
                        elem, need, (unsigned)FFSAT_STATIC_SCRATCH_BYTES);
        void *p = nullptr;
        CUDA_TRY(static_scratch(I->device, &p));
        a.g_scratch = p;
    }
    return launch_step(I, f64, mode, a, B, stream);
}

static int grow_scratch(void **p, size_t *have, size_t need) {
    if (need <= *have) return FFSAT_OK;
    if (*p) CUDA_TRY(cudaFree(*p));
    *p = nullptr;
    *have = 0;
    CUDA_TRY(cudaMalloc(p, need));
    *have = need;
    return FFSAT_OK;
}

int ffsat_step_pgfp(ffsat_instance *I, int32_t B, void *x, int32_t dtype, const ffsat_pgfp_args *args,
                    uint8_t *solved, int32_t *n_unsat, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I || !args) return fail(FFSAT_ERR_ARG, "NULL argument");
    if (B < 0 || args->T < 0) return fail(FFSAT_ERR_ARG, "B and T must be >= 0");
    if (!(args->eta0 > 0.0) || !std::isfinite(args->eta0)) return fail(FFSAT_ERR_ARG, "eta0 must be positive");
    if (!(args->beta > 0.0 && args->beta < 1.0)) return fail(FFSAT_ERR_ARG, "beta must lie in (0, 1)");
    if (args->maxls < 1) return fail(FFSAT_ERR_ARG, "maxls must be >= 1");
    if (!(args->eta_min >= 0.0) || !(args->slack >= 0.0) || !std::isfinite(args->slack))
        return fail(FFSAT_ERR_ARG, "eta_min and slack must be >= 0");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    const bool f64 = dtype == FFSAT_F64;
    const int mode = f64 ? I->smem_mode64 : I->smem_mode32;
    if (mode == SMEM_NONE)
        return fail(FFSAT_ERR_ARG, "the line-search step needs x in shared memory (n = %d is too large)", I->n);
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    const size_t elem = f64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)B * (size_t)I->n * elem;
    FusedArgs a{};
    a.B = B;
    a.mode = MODE_PGFP;
    a.x_in = x;
    a.x_out = x;
    a.solved = solved;
    a.n_unsat = n_unsat;
    a.sp.T = args->T;
    a.sp.restart = args->restart;
    a.sp.lr = args->eta0;
    a.sp.seed = args->seed;
    a.sp.epoch = args->epoch;
    a.sp.b_offset = args->b_offset;
    a.unsat_counts = args->unsat_counts;
    a.beta = args->beta;
    a.eta_min = args->eta_min;
    a.slack = args->slack;
    a.maxls = args->maxls;
    a.iters = args->iters;
    a.eta_out = args->eta_out;
    if (mode != SMEM_FULL && mode != SMEM_RES) {
        rc = grow_scratch(&I->d_scratch, &I->scratch_bytes, need);
        if (rc) return rc;
        a.g_scratch = I->d_scratch;
    }
    rc = grow_scratch(&I->d_yscratch, &I->yscratch_bytes, need);
    if (rc) return rc;
    a.y_scratch = I->d_yscratch;
    const DevView &V = f64 ? I->V64 : I->V32;
    CUDA_TRY(launcher_for(f64, f64 ? I->nr64 : I->nr32)(V, mode, a, f64 ? I->smem64 : I->smem32, grid_for(I, f64, B),
                                                          static_cast<cudaStream_t>(stream), false));
    t_launches = 1;
    return FFSAT_OK;
}

int ffsat_check(ffsat_instance *I, int32_t B, const void *x, int32_t dtype, uint8_t *sat, int32_t *n_unsat,
                void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (B < 0) return fail(FFSAT_ERR_ARG, "B must be >= 0");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    CUDA_TRY(launch_check(I->V32, dtype == FFSAT_F64, B, x, sat, n_unsat, nullptr, static_cast<cudaStream_t>(stream)));
    t_launches = 1;
    return FFSAT_OK;
}

int ffsat_unsat_counts(ffsat_instance *I, int32_t B, const void *x, int32_t dtype, int32_t *U, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (B < 0) return fail(FFSAT_ERR_ARG, "B must be >= 0");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (I->m == 0) return FFSAT_OK;
    if (!U) return fail(FFSAT_ERR_ARG, "U is NULL");
    if (B > 0 && !x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(U, 0, (size_t)I->m * sizeof(int32_t), s));
    CUDA_TRY(launch_check(I->V32, dtype == FFSAT_F64, B, x, nullptr, nullptr, U, s));
    t_launches = B > 0 ? 1 : 0;
    return FFSAT_OK;
}

int ffsat_erwa_update(ffsat_instance *I, const int32_t *U, double alpha, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(FFSAT_ERR_ARG, "alpha must lie in [0, 1]");
    if (I->m == 0) return FFSAT_OK;
    if (!U) return fail(FFSAT_ERR_ARG, "U is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    unsigned char *base = I->d_arena;
    WeightSites W{};
    W.m = I->m;
    W.n_images = I->n_images;
    for (int k = 0; k < I->n_images; ++k) {
        int4 *img = I->d_img[k];
        W.clauses[k] = img + I->img_off[k][1];
        W.segmeta[k] = img + I->img_off[k][2];
    }
    W.clause_wd = reinterpret_cast<double *>(base + I->off_clause_wd);
    W.seg_wd = reinterpret_cast<double *>(base + I->off_seg_wd);
    W.cons_wd = reinterpret_cast<double *>(base + I->off_cons_wd);
    W.cls = reinterpret_cast<const int8_t *>(base + I->off_cls);
    W.slot = reinterpret_cast<const int32_t *>(base + I->off_slot);
    W.row_ptr = I->V64.row_ptr;
    W.param = I->V64.param;
    int nl = 0;
    CUDA_TRY(launch_erwa(W, U, reinterpret_cast<int32_t *>(base + I->off_umax), alpha,
                         reinterpret_cast<double *>(base + I->off_f_const), static_cast<cudaStream_t>(stream), &nl));
    t_launches = nl;
    return FFSAT_OK;
}

static int rephase_impl(ffsat_instance *I, int32_t B, void *x, int32_t dtype, int32_t phase, const uint8_t *solved,
                        uint64_t seed, uint64_t epoch, const uint64_t *epoch_dev, uint64_t b_offset, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    if (B < 0) return fail(FFSAT_ERR_ARG, "B must be >= 0");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    if (phase != FFSAT_PHASE_ORIGINAL && phase != FFSAT_PHASE_FLIPPED && phase != FFSAT_PHASE_RANDOM)
        return fail(FFSAT_ERR_ARG, "phase must be FFSAT_PHASE_ORIGINAL, _FLIPPED or _RANDOM");
    if (B == 0) return FFSAT_OK;
    if (!x) return fail(FFSAT_ERR_ARG, "x is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    int nl = 0;
    CUDA_TRY(launch_rephase(dtype == FFSAT_F64, x, B, I->n, phase, solved, seed, epoch, b_offset, epoch_dev,
                            static_cast<cudaStream_t>(stream), &nl));
    t_launches = nl;
    return FFSAT_OK;
}

int ffsat_rephase(ffsat_instance *I, int32_t B, void *x, int32_t dtype, int32_t phase, const uint8_t *solved,
                  uint64_t seed, uint64_t epoch, uint64_t b_offset, void *stream) {
    return rephase_impl(I, B, x, dtype, phase, solved, seed, epoch, nullptr, b_offset, stream);
}

int ffsat_rephase_at(ffsat_instance *I, int32_t B, void *x, int32_t dtype, int32_t phase, const uint8_t *solved,
                     uint64_t seed, const uint64_t *epoch_dev, uint64_t b_offset, void *stream) {
    if (!epoch_dev) return fail(FFSAT_ERR_ARG, "epoch_dev is NULL");
    return rephase_impl(I, B, x, dtype, phase, solved, seed, 0, epoch_dev, b_offset, stream);
}

int ffsat_get_weights(ffsat_instance *I, double *weights) {
    t_err.clear();
    if (!I || !weights) return fail(FFSAT_ERR_ARG, "NULL argument");
    if (I->m == 0) return FFSAT_OK;
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(weights, I->d_arena + I->off_cons_wd, (size_t)I->m * sizeof(double), cudaMemcpyDeviceToHost));
    return FFSAT_OK;
}

}  // extern "C"

namespace ffsat {

// Variable features: 1, clause occurrences (positive, negative) over the mean
// degree, their signed balance, XOR occurrences, the signed balance of
// cardinality occurrences, the total degree over the mean, 0.  Constraint
// features: 1, type one-hot (OR, XOR, ATLEAST), length / 10, XOR parity as
// +-1, K / length, 0.
int instance_graph(ffsat_instance *I, GraphView *out) {
    if (I->d_graph) {
        *out = I->graph;
        return FFSAT_OK;
    }
    const int n = I->n, m = I->m;
    std::vector<int32_t> var_ptr(n + 1, 0);
    std::vector<float> pos(n, 0.f), neg(n, 0.f), nx(n, 0.f), cpos(n, 0.f), cneg(n, 0.f);
    for (int64_t i = 0; i < I->nnz; ++i) {
        const int32_t l = I->lits_in[i];
        var_ptr[(l > 0 ? l : -l)] += 1;
    }
    for (int v = 0; v < n; ++v) var_ptr[v + 1] += var_ptr[v];
    std::vector<uint32_t> occ((size_t)std::max<int64_t>(I->nnz, 1));
    std::vector<int32_t> fill(var_ptr.begin(), var_ptr.end() - 1);
    std::vector<float> fc((size_t)m * 8, 0.f), inv_len(std::max(m, 1), 0.f);
    for (int32_t c = 0; c < m; ++c) {
        const int64_t a = I->row_ptr[c], e = I->row_ptr[c + 1];
        const int L = (int)(e - a);
        const int t = I->type[c];
        for (int64_t i = a; i < e; ++i) {
            const int32_t l = I->lits_in[i];
            const int32_t v = (l > 0 ? l : -l) - 1;
            occ[fill[v]++] = (uint32_t)c | (l < 0 ? 0x80000000u : 0u);
            if (t == FFSAT_OR) (l > 0 ? pos : neg)[v] += 1.f;
            else if (t == FFSAT_XOR) nx[v] += 1.f;
            else (l > 0 ? cpos : cneg)[v] += 1.f;
        }
        float *f = &fc[(size_t)c * 8];
        f[0] = 1.f;
        f[1] = t == FFSAT_OR;
        f[2] = t == FFSAT_XOR;
        f[3] = t == FFSAT_ATLEAST;
        f[4] = (float)L / 10.f;
        f[5] = t == FFSAT_XOR ? ((I->param[c] & 1) ? 1.f : -1.f) : 0.f;
        f[6] = t == FFSAT_ATLEAST ? (float)I->param[c] / (float)L : 0.f;
        inv_len[c] = 1.f / (float)L;
    }
    const float mean_deg = n > 0 ? (float)I->nnz / (float)n : 1.f;
    std::vector<float> fv((size_t)n * 8, 0.f), inv_deg(std::max(n, 1), 0.f);
    for (int v = 0; v < n; ++v) {
        const float d = (float)(var_ptr[v + 1] - var_ptr[v]);
        float *f = &fv[(size_t)v * 8];
        f[0] = 1.f;
        f[1] = pos[v] / mean_deg;
        f[2] = neg[v] / mean_deg;
        f[3] = (pos[v] - neg[v]) / (pos[v] + neg[v] + 1.f);
        f[4] = nx[v] / mean_deg;
        f[5] = (cpos[v] - cneg[v]) / (cpos[v] + cneg[v] + 1.f);
        f[6] = d / mean_deg;
        inv_deg[v] = d > 0 ? 1.f / d : 0.f;
    }
    std::vector<int32_t> rp32(m + 1);
    for (int c = 0; c <= m; ++c) rp32[c] = (int32_t)I->row_ptr[c];
    std::vector<uint32_t> lp((size_t)std::max<int64_t>(I->nnz, 1));
    for (int64_t i = 0; i < I->nnz; ++i) lp[i] = (uint32_t)pack_lit(I->lits_in[i]);
    Arena A;
    const size_t o_rp = A.put(rp32), o_l = A.put(lp), o_vp = A.put(var_ptr), o_vo = A.put(occ), o_fv = A.put(fv),
                 o_fc = A.put(fc), o_id = A.put(inv_deg), o_il = A.put(inv_len);
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    CUDA_TRY(cudaMalloc(&I->d_graph, A.host.size()));
    CUDA_TRY(cudaMemcpy(I->d_graph, A.host.data(), A.host.size(), cudaMemcpyHostToDevice));
    GraphView &g = I->graph;
    g.device = I->device;
    g.n = n;
    g.m = m;
    g.row_ptr = reinterpret_cast<const int32_t *>(I->d_graph + o_rp);
    g.lits = reinterpret_cast<const uint32_t *>(I->d_graph + o_l);
    g.var_ptr = reinterpret_cast<const int32_t *>(I->d_graph + o_vp);
    g.var_occ = reinterpret_cast<const uint32_t *>(I->d_graph + o_vo);
    g.fv = reinterpret_cast<const float *>(I->d_graph + o_fv);
    g.fc = reinterpret_cast<const float *>(I->d_graph + o_fc);
    g.inv_deg = reinterpret_cast<const float *>(I->d_graph + o_id);
    g.inv_len = reinterpret_cast<const float *>(I->d_graph + o_il);
    *out = g;
    return FFSAT_OK;
}

// ffsat_last_error for code outside this file.
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace ffsat

struct ffsat_batch {
    int device = 0;
    int num_sms = 0;
    std::vector<ffsat_instance *> insts;
    int node_r[2] = {0, 0};      // batch-kernel variant per real type (0 or 16)
    int threads[2] = {0, 0};     // CTA width per real type
    float tune_us[2] = {0.f, 0.f};  // FP32 probe evaluation at 384 / 512 threads (0: not timed)
    size_t smem[2] = {0, 0};
    int grid[2] = {0, 0};
    std::vector<BatchInst> h_insts;  // last table uploaded (per real type: re-uploaded when it changes)
    int h_insts_dtype = -1;
    BatchInst *d_insts = nullptr;
    int *d_counter = nullptr;
    int2 *d_items = nullptr;
    size_t items_cap = 0;
    int n_items = 0;
    std::vector<int32_t> items_B;  // B per instance of the cached item list
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
};

namespace {

// Items (instance, point), longest first by a per-point cost estimate; cached
// while the per-instance point counts stay the same.
int batch_items(ffsat_batch *bt, const ffsat_batch_io *io, cudaStream_t s) {
    const int K = (int)bt->insts.size();
    std::vector<int32_t> Bs(K);
    for (int k = 0; k < K; ++k) Bs[k] = io[k].B;
    if (Bs == bt->items_B && bt->d_items) return FFSAT_OK;
    std::vector<std::pair<double, int>> order(K);
    for (int k = 0; k < K; ++k) {
        const ffsat_info &inf = bt->insts[k]->info;
        const double cost = (double)inf.node_lane_work * 12.0 / 32.0 + (double)inf.nnz * 2.0 + (double)inf.n;
        order[k] = {-cost, k};
    }
    std::sort(order.begin(), order.end());
    std::vector<int2> items;
    for (const auto &o : order)
        for (int b = 0; b < Bs[o.second]; ++b) items.push_back(make_int2(o.second, b));
    CUDA_TRY(cudaStreamSynchronize(s));  // earlier launches may still read the old list
    if (items.size() > bt->items_cap) {
        if (bt->d_items) CUDA_TRY(cudaFree(bt->d_items));
        bt->d_items = nullptr;
        bt->items_cap = 0;
        CUDA_TRY(cudaMalloc(&bt->d_items, std::max<size_t>(items.size(), 1) * sizeof(int2)));
        bt->items_cap = std::max<size_t>(items.size(), 1);
    }
    if (!items.empty())
        CUDA_TRY(cudaMemcpyAsync(bt->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // items is a host temporary
    bt->n_items = (int)items.size();
    bt->items_B = Bs;
    return FFSAT_OK;
}

int batch_launch(ffsat_batch *bt, const ffsat_batch_io *io, int32_t dtype, int mode, const ffsat_step_args *args,
                 cudaStream_t s) {
    const bool f64 = dtype == FFSAT_F64;
    const int K = (int)bt->insts.size();
    const size_t elem = f64 ? sizeof(double) : sizeof(float);
    for (int k = 0; k < K; ++k) {
        if (io[k].B < 0) return fail(FFSAT_ERR_ARG, "io[%d].B must be >= 0", k);
        if (io[k].B > 0 && !io[k].x) return fail(FFSAT_ERR_ARG, "io[%d].x is NULL", k);
    }
    // gradient scratch for step on instances without the gradient in shared memory
    size_t need = 0;
    std::vector<size_t> scr_off(K, 0);
    if (mode == MODE_STEP) {
        for (int k = 0; k < K; ++k) {
            const int m = f64 ? bt->insts[k]->smem_mode64 : bt->insts[k]->smem_mode32;
            if (m == SMEM_X || m == SMEM_NONE) {
                scr_off[k] = need;
                need += ((size_t)io[k].B * (size_t)bt->insts[k]->n * elem + 255) & ~size_t(255);
            }
        }
        if (need > bt->scratch_bytes) {
            if (bt->d_scratch) CUDA_TRY(cudaFree(bt->d_scratch));
            bt->d_scratch = nullptr;
            bt->scratch_bytes = 0;
            CUDA_TRY(cudaMalloc(&bt->d_scratch, need));
            bt->scratch_bytes = need;
        }
    }
    int rc = batch_items(bt, io, s);
    if (rc) return rc;
    if (bt->n_items == 0) return FFSAT_OK;
    // per-instance table (views, buffers, shared-memory modes); step parameters go
    // by value so that a loop over fixed buffers enqueues only a memset and a launch
    std::vector<BatchInst> tab(K);
    std::memset(tab.data(), 0, tab.size() * sizeof(BatchInst));
    for (int k = 0; k < K; ++k) {
        ffsat_instance *I = bt->insts[k];
        BatchInst &bi = tab[k];
        bi.V = f64 ? I->V64 : I->V32;
        bi.mode = f64 ? I->smem_mode64 : I->smem_mode32;
        FusedArgs &a = bi.A;
        a.B = io[k].B;
        a.mode = mode;
        a.x_in = io[k].x;
        if (mode == MODE_STEP) {
            a.x_out = io[k].x;
            a.solved = io[k].solved;
            a.n_unsat = io[k].n_unsat;
            a.sp.b_offset = io[k].b_offset;
            if (bi.mode == SMEM_X || bi.mode == SMEM_NONE)
                a.g_scratch = static_cast<unsigned char *>(bt->d_scratch) + scr_off[k];
        } else {
            a.f = io[k].f;
            a.g = io[k].g;
        }
    }
    if (bt->h_insts_dtype != dtype || bt->h_insts.size() != tab.size() ||
        std::memcmp(bt->h_insts.data(), tab.data(), tab.size() * sizeof(BatchInst)) != 0) {
        CUDA_TRY(cudaStreamSynchronize(s));
        CUDA_TRY(cudaMemcpy(bt->d_insts, tab.data(), tab.size() * sizeof(BatchInst), cudaMemcpyHostToDevice));
        bt->h_insts.swap(tab);
        bt->h_insts_dtype = dtype;
    }
    StepParams sp{};
    if (mode == MODE_STEP) {
        sp.T = args->T;
        sp.restart = args->restart;
        sp.lr = args->lr;
        sp.seed = args->seed;
        sp.epoch = args->epoch;
    }
    CUDA_TRY(cudaMemsetAsync(bt->d_counter, 0, sizeof(int), s));
    const int v = f64 ? 1 : 0;
    CUDA_TRY(launch_batch(f64, bt->node_r[v], bt->threads[v], bt->d_insts, bt->d_items, bt->n_items, bt->d_counter, sp, bt->smem[v],
                          bt->grid[v], s, false, nullptr));
    t_launches = 1;
    return FFSAT_OK;
}


// CTA width `threads` for real type v, and the persistent grid it allows.
int batch_set_threads(ffsat_batch *bt, int v, int threads) {
    int per_sm = 0;
    const StepParams none{};
    CUDA_TRY(launch_batch(v == 1, bt->node_r[v], threads, nullptr, nullptr, 0, nullptr, none, bt->smem[v], 0, 0, true,
                          &per_sm));
    bt->threads[v] = threads;
    bt->grid[v] = std::max(1, per_sm) * bt->num_sms;
    return FFSAT_OK;
}

// Time one FP32 batch evaluation (two points per instance, min over three
// launches after a warm-up) at 384 and at 512 threads per CTA and keep the
// faster width (512 unless 384 is at least 1% faster).
int batch_tune_threads(ffsat_batch *bt) {
    const int K = (int)bt->insts.size();
    const int P = 2;
    size_t xs = 0;
    for (ffsat_instance *I : bt->insts) xs += (size_t)P * (size_t)I->n;
    std::vector<float> hx(xs);
    uint64_t st = 0xD1B54A32D192ED03ull;
    for (size_t i = 0; i < xs; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        hx[i] = (float)((double)(st >> 40) / (double)(1ull << 23) - 1.0);
    }
    float *dx = nullptr, *dg = nullptr;
    double *df = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = FFSAT_OK;
    if (cudaMalloc(&dx, xs * sizeof(float)) != cudaSuccess || cudaMalloc(&dg, xs * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&df, (size_t)K * P * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemcpy(dx, hx.data(), xs * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = fail(FFSAT_ERR_CUDA, "batch tuning: allocation or upload of the probe batch failed");
    std::vector<ffsat_batch_io> io(K);
    size_t off = 0;
    for (int k = 0; k < K; ++k) {
        std::memset(&io[k], 0, sizeof(io[k]));
        io[k].B = P;
        io[k].x = dx + off;
        io[k].g = dg + off;
        io[k].f = df + (size_t)k * P;
        off += (size_t)P * (size_t)bt->insts[k]->n;
    }
    const int widths[2] = {384, 512};
    for (int c = 0; c < 2 && rc == FFSAT_OK; ++c) {
        rc = batch_set_threads(bt, 0, widths[c]);
        if (rc == FFSAT_OK) rc = batch_launch(bt, io.data(), FFSAT_F32, MODE_EVAL, nullptr, 0);
        float best = 1e30f;
        for (int r = 0; r < 3 && rc == FFSAT_OK; ++r) {
            float ms = 0.f;
            if (cudaEventRecord(e0, 0) != cudaSuccess) rc = fail(FFSAT_ERR_CUDA, "batch tuning: event record failed");
            if (rc == FFSAT_OK) rc = batch_launch(bt, io.data(), FFSAT_F32, MODE_EVAL, nullptr, 0);
            if (rc == FFSAT_OK && (cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                   cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = fail(FFSAT_ERR_CUDA, "batch tuning: timing failed");
            best = std::min(best, 1000.f * ms);
        }
        bt->tune_us[c] = best;
    }
    if (rc == FFSAT_OK) rc = batch_set_threads(bt, 0, bt->tune_us[0] < 0.99f * bt->tune_us[1] ? 384 : 512);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dx);
    cudaFree(dg);
    cudaFree(df);
    for (ffsat_instance *I : bt->insts) cudaMemset(I->d_status, 0, sizeof(int32_t));
    return rc;
}

}  // namespace

extern "C" {

int ffsat_batch_create(ffsat_instance *const *insts, int32_t count, ffsat_batch **out) {
    t_err.clear();
    if (!out || !insts || count <= 0) return fail(FFSAT_ERR_ARG, "insts, count > 0 and out are required");
    *out = nullptr;
    std::unique_ptr<ffsat_batch> bt(new ffsat_batch());
    for (int k = 0; k < count; ++k) {
        if (!insts[k]) return fail(FFSAT_ERR_ARG, "insts[%d] is NULL", k);
        if (insts[k]->device != insts[0]->device) return fail(FFSAT_ERR_ARG, "instances live on different devices");
        bt->insts.push_back(insts[k]);
    }
    bt->device = insts[0]->device;
    bt->num_sms = insts[0]->num_sms;
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(bt->device));
    for (int v = 0; v < 2; ++v) {
        size_t smem = 0;
        int nr = 0;
        for (ffsat_instance *I : bt->insts) {
            smem = std::max(smem, v ? I->smem64 : I->smem32);
            if ((v ? I->nr64 : I->nr32) > 0) nr = 16;
        }
        bt->smem[v] = smem;
        bt->node_r[v] = nr;
        int rc = batch_set_threads(bt.get(), v, batch_threads_default(v == 1, nr));
        if (rc != FFSAT_OK) return rc;
    }
    CUDA_TRY(cudaMalloc(&bt->d_insts, (size_t)count * sizeof(BatchInst)));
    CUDA_TRY(cudaMalloc(&bt->d_counter, sizeof(int)));
    // FP32 node-path batches of autotuned instances also choose the CTA width
    bool tuned = bt->node_r[0] > 0;
    for (ffsat_instance *I : bt->insts) tuned = tuned && I->opt.autotune;
    if (tuned) {
        int rc = batch_tune_threads(bt.get());
        if (rc != FFSAT_OK) return rc;
    }
    *out = bt.release();
    return FFSAT_OK;
}

int ffsat_batch_threads(const ffsat_batch *bt, int32_t dtype, int32_t *threads, float *us384, float *us512) {
    t_err.clear();
    if (!bt || !threads) return fail(FFSAT_ERR_ARG, "NULL argument");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    const int v = dtype == FFSAT_F64 ? 1 : 0;
    *threads = bt->threads[v];
    if (us384) *us384 = v == 0 ? bt->tune_us[0] : 0.f;
    if (us512) *us512 = v == 0 ? bt->tune_us[1] : 0.f;
    return FFSAT_OK;
}

int ffsat_batch_eval_grad(ffsat_batch *bt, const ffsat_batch_io *io, int32_t dtype, void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!bt || !io) return fail(FFSAT_ERR_ARG, "NULL argument");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(bt->device));
    return batch_launch(bt, io, dtype, MODE_EVAL, nullptr, static_cast<cudaStream_t>(stream));
}

int ffsat_batch_step(ffsat_batch *bt, const ffsat_batch_io *io, int32_t dtype, const ffsat_step_args *args,
                     void *stream) {
    t_err.clear();
    t_launches = 0;
    if (!bt || !io || !args) return fail(FFSAT_ERR_ARG, "NULL argument");
    if (args->T < 0) return fail(FFSAT_ERR_ARG, "T must be >= 0");
    if (!std::isfinite(args->lr)) return fail(FFSAT_ERR_ARG, "lr must be finite");
    int rc = check_dtype(dtype);
    if (rc) return rc;
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(bt->device));
    return batch_launch(bt, io, dtype, MODE_STEP, args, static_cast<cudaStream_t>(stream));
}

void ffsat_batch_free(ffsat_batch *bt) {
    if (!bt) return;
    DeviceGuard dev_guard;
    dev_guard.set(bt->device);
    if (bt->d_insts) cudaFree(bt->d_insts);
    if (bt->d_counter) cudaFree(bt->d_counter);
    if (bt->d_items) cudaFree(bt->d_items);
    if (bt->d_scratch) cudaFree(bt->d_scratch);
    delete bt;
}

int ffsat_sync_status(ffsat_instance *I, void *stream) {
    t_err.clear();
    if (!I) return fail(FFSAT_ERR_ARG, "instance is NULL");
    DeviceGuard dev_guard;
    CUDA_TRY(dev_guard.set(I->device));
    CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int32_t st = 0;
    CUDA_TRY(cudaMemcpy(&st, I->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(I->d_status, 0, sizeof(int32_t)));
    if (st & STATUS_NAN) return fail(FFSAT_ERR_NAN, "NaN found in x");
    if (st) return fail(FFSAT_ERR_DEVICE, "device status 0x%x", st);
    return FFSAT_OK;
}

int ffsat_instance_info(const ffsat_instance *I, ffsat_info *info) {
    if (!I || !info) return fail(FFSAT_ERR_ARG, "NULL argument");
    *info = I->info;
    return FFSAT_OK;
}

void ffsat_free(ffsat_instance *I) {
    if (!I) return;
    DeviceGuard dev_guard;
    dev_guard.set(I->device);
    if (I->d_graph) cudaFree(I->d_graph);
    for (int k = 0; k < 2; ++k)
        if (I->d_img[k]) cudaFree(I->d_img[k]);
    if (I->d_arena) cudaFree(I->d_arena);
    if (I->d_status) cudaFree(I->d_status);
    if (I->d_scratch) cudaFree(I->d_scratch);
    if (I->d_yscratch) cudaFree(I->d_yscratch);
    delete I;
}

}  // extern "C"
