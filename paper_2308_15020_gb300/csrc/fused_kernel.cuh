// Fused per-point kernel of the FastFourierSAT hot path.
//
// One CTA owns one restart point b (thread-level parallelism p_t of the paper's
// "Acceleration with GPU" section maps to CTAs).  The point's x row and its
// gradient accumulator live in shared memory when they fit, and so does the
// instance's constraint data when it fits beside them; every constraint is
// evaluated against them by warp tasks pulled from a shared-memory counter
// (instruction-level parallelism p_i: constraints), and the literals of one
// long constraint are spread over a segment of G lanes (data-level
// parallelism p_d).
//
// Three constraint paths:
//  * clause3: one thread per clause of <= 3 literals, FE = -1 + 2 q1 q2 q3 with
//    q = (1+y)/2 and dFE/dy_i = prod_{l != i} q_l (footnote of App. B).
//  * product: OR / XOR of any length <= 256, FE = c0 + c1 prod_i (a + b y_i)
//    (App. B "Transform-Free", Cor. "Reduction"): an O(L) product with the
//    all-but-one products formed by in-lane suffix/prefix products and a
//    butterfly over the segment's lanes.
//  * node: the DFT evaluation of Alg. 2 with conjugate symmetry.  For node j of
//    N roots of unity the factor of literal i is alpha_j + beta_j y_i (Eq.
//    forward), the node value is the product over literals (Eq. reduction),
//    FE = Re sum_j c_j prod_i(.) (Eq. inverse with the preprocessed
//    coefficients) and dFE/dy_i = Re sum_j d_j prod_{l != i}(.) (Eq. chain),
//    d_j = c_j beta_j.  The stable form runs it as the paper's E(z) =
//    prod (1 + y_i z) at the imaginary nodes z_j = i tan(pi j / N) with the
//    per-node scale carried as an exponent (node_task_im); the paper form runs
//    the generic factors (node_task).  The all-but-one products come from
//    in-lane suffix products, a product over the segment lanes and an in-lane
//    prefix pass.
// Projected gradient descent (App. A.3 with a fixed step), the exact sign check
// (Thm. "SAT Certificate", evaluated on integers) and the uniform restart of
// Alg. 1 run in the same launch.
//
// Literals are packed as variable | (negated << 31).  Padding literals name two
// dummy variables that follow the n real ones in shared memory: x[n] = +1 and
// x[n+1] = 0, which make a clause or product factor (resp. a node factor of
// either form) exactly 1; their gradients land in dummy accumulator slots.  When x or g live in global memory, accesses to the dummy
// variables are resolved without touching memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ffsat_internal.h"

namespace ffsat {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kVarMask = 0x7fffffffu;
constexpr uint32_t kSignBit = 0x80000000u;

template <typename R>
struct C2 {
    R re, im;
};

template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

template <typename R>
struct Node {
    C2<R> a, b, d, c;
};

__device__ __forceinline__ Node<float> load_node(const DevView &V, float, int idx) {
    const float4 p = __ldg(&V.tab_f[2 * idx]);
    const float4 q = __ldg(&V.tab_f[2 * idx + 1]);
    return {{p.x, p.y}, {p.z, p.w}, {q.x, q.y}, {q.z, q.w}};
}

__device__ __forceinline__ Node<double> load_node(const DevView &V, double, int idx) {
    const double2 *t = reinterpret_cast<const double2 *>(V.tab_d) + 4 * idx;
    const double2 p = __ldg(t), q = __ldg(t + 1), r = __ldg(t + 2), s = __ldg(t + 3);
    return {{p.x, p.y}, {q.x, q.y}, {r.x, r.y}, {s.x, s.y}};
}

// Node of the imaginary-node form: t = tan(pi j / N) and the coefficient
// C_j = c_j alpha_j^L as a mantissa (largest component in [1/2, 1)) times 2^ec;
// D_j = i t_j C_j is formed from them.
template <typename R>
struct NodeIm {
    R t;
    C2<R> c;
    int ec;
};

__device__ __forceinline__ NodeIm<float> load_node_im(const DevView &V, float, int idx) {
    const float4 p = __ldg(&V.tab_im_f[idx]);
    return {p.x, {p.y, p.z}, __float_as_int(p.w)};
}

__device__ __forceinline__ NodeIm<double> load_node_im(const DevView &V, double, int idx) {
    const double2 *t = reinterpret_cast<const double2 *>(V.tab_im_d) + 2 * idx;
    const double2 p = __ldg(t), q = __ldg(t + 1);
    return {p.x, {p.y, q.x}, (int)q.y};
}

// e such that max(|a|, |b|) 2^-e lies in [1/2, 1) (a, b finite, not both zero;
// integer operations on the exponent field only).
__device__ __forceinline__ int frexp_max(float a, float b) {
    const int ia = __float_as_int(a) & 0x7fffffff, ib = __float_as_int(b) & 0x7fffffff;
    return (max(ia, ib) >> 23) - 126;
}
__device__ __forceinline__ int frexp_max(double a, double b) {
    const long long ia = __double_as_longlong(a) & 0x7fffffffffffffffll;
    const long long ib = __double_as_longlong(b) & 0x7fffffffffffffffll;
    return (int)(max(ia, ib) >> 52) - 1022;
}
// 2^k built from its exponent field; 0 below the normal range (such terms are
// below 2^-126 of the result), clamped at the top (reached only when the
// coefficient it scales is zero).
__device__ __forceinline__ float exp2i(float, int k) {
    k = min(max(k, -127), 127);
    return __int_as_float((k + 127) << 23);
}
__device__ __forceinline__ double exp2i(double, int k) {
    k = min(max(k, -1023), 1023);
    return __longlong_as_double((long long)(k + 1023) << 52);
}
// s = 2^-e with e = frexp_max(a, b), built from the exponent field of the larger
// of |a|, |b| (a, b finite, the larger normal and below 2^126).
__device__ __forceinline__ float norm_scale(float a, float b, int &e) {
    const int m = max(__float_as_int(a) & 0x7fffffff, __float_as_int(b) & 0x7fffffff) & 0x7f800000;
    e = (m >> 23) - 126;
    return __int_as_float(0x7e800000 - m);
}
__device__ __forceinline__ double norm_scale(double a, double b, int &e) {
    e = frexp_max(a, b);
    return exp2i(0.0, -e);
}
// Bring the cache line of node table entry idx into L1 ahead of its use.
__device__ __forceinline__ void prefetch_node_im(const DevView &V, float, int idx) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(V.tab_im_f + idx));
}
__device__ __forceinline__ void prefetch_node_im(const DevView &V, double, int idx) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(V.tab_im_d + 4 * idx));
}
// 1/a for the node task's division by a lane product of modulus in [1/2, 2)
// (FP32: the hardware's approximate reciprocal, within about an ulp).
__device__ __forceinline__ float recip(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double recip(double a) { return __drcp_rn(a); }

// Where the warp tasks read the constraint data from: global memory, or the
// CTA's shared-memory copy of the resident image.
struct Src {
    const int4 *tasks;
    const int4 *clauses;
    const int4 *segmeta;
    const int32_t *seg_lits;
};

template <typename R>
__device__ __forceinline__ R seg_weight(const DevView &V, int4 meta, int c);
template <>
__device__ __forceinline__ float seg_weight<float>(const DevView &, int4 meta, int) { return __int_as_float(meta.w); }
template <>
__device__ __forceinline__ double seg_weight<double>(const DevView &V, int4, int c) { return __ldg(&V.seg_wd[c]); }

template <typename R>
__device__ __forceinline__ R clause_weight(const DevView &V, int4 cl, int idx);
template <>
__device__ __forceinline__ float clause_weight<float>(const DevView &, int4 cl, int) { return __int_as_float(cl.w); }
template <>
__device__ __forceinline__ double clause_weight<double>(const DevView &V, int4, int idx) {
    return __ldg(&V.clause_wd[idx]);
}

// Multiply by -1 when the sign bit of the packed literal is set.
__device__ __forceinline__ float flip(float x, uint32_t lp) {
    return __int_as_float(__float_as_int(x) ^ (int)(lp & kSignBit));
}
__device__ __forceinline__ double flip(double x, uint32_t lp) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(lp & kSignBit) << 32));
}

// y = sigma x[v].  XG: where x lives (dummy variables n, n+1 exist in shared memory).
template <typename R, int XG>
__device__ __forceinline__ R gather(const R *xrow, uint32_t lp, int n) {
    const uint32_t v = lp & kVarMask;
    R xv;
    if constexpr (XG == SMEM_NONE)
        xv = v < (uint32_t)n ? xrow[v] : (v == (uint32_t)n ? R(1) : R(0));
    else
        xv = xrow[v];
    return flip(xv, lp);
}

// Gradient accumulators.  Plain: one real per variable updated with atomicAdd
// (shared or global memory).  Fixed: two int32 words per variable in shared
// memory updated with the native integer reduction; a contribution c is split
// into hi = round(c 2^S1) and lo = round((c 2^S1 - hi) 2^S2), both rounded by
// adding 1.5 * 2^23 (exact round-to-nearest for |t| < 2^22, which the host's
// choice of S1, S2 guarantees).  Padding literals (dummy variables) are
// skipped: many lanes of a warp share the dummy and same-address updates
// serialise.
template <typename R>
struct PlainAcc {
    static constexpr bool kDummySlots = false;
    R *g;
    __device__ __forceinline__ void add(uint32_t v, R c) const { atomicAdd(&g[v], c); }
    __device__ __forceinline__ void addf(uint32_t v, R c) const { atomicAdd(&g[v], c); }
    __device__ __forceinline__ R get(int v) const { return g[v]; }
    __device__ __forceinline__ void zero(int v) const { g[v] = R(0); }
};

// Fixed point of the FP64 cluster step: each contribution c is rounded to the
// integer V = c 2^S64, split into lo = V mod 2^L and hi = floor(V / 2^L), and
// the two words are added with native 32-bit shared-memory reductions (a
// 64-bit shared-memory add would be a compare-and-swap loop).  Integer sums are
// the same in any order, so the step is bit-reproducible; the host's choice of
// S64 and L keeps |V| below 2^51, every lo sum below 2^32 and every hi sum
// below 2^31.  The rounding is one FMA: for |a b| < 2^51, fma(a, b, 1.5 2^52)
// lies in [2^52, 2^53), where the spacing of doubles is 1, so it equals
// 1.5 2^52 + round(a b) and its bit pattern minus that of 1.5 2^52 is the
// integer.
struct Fix64Acc {
    static constexpr bool kDummySlots = true;  // npad >= n + 2 words
    static constexpr double kRound = 6755399441055744.0;  // 1.5 * 2^52
    uint2 *g;    // {lo, hi} per variable
    double *gf;  // product contributions (FP64 atomics; see addf)
    double s, inv;  // 2^S64 and 2^-S64
    int l;
    // m = fma(a, b, kRound): adds round(a b) to variable v
    __device__ __forceinline__ void put(uint32_t v, double m) const {
        const long long V = __double_as_longlong(m) - __double_as_longlong(kRound);
        const unsigned lo = (unsigned)V & ((1u << l) - 1u);
        const int hi = (int)(V >> l);
        const unsigned a = (unsigned)__cvta_generic_to_shared(&g[v]);
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(lo) : "memory");
        asm volatile("red.shared.add.s32 [%0+4], %1;" ::"r"(a), "r"(hi) : "memory");
    }
    __device__ __forceinline__ void add(uint32_t v, double c) const { put(v, fma(c, s, kRound)); }
    // Product contributions (XORs and long clauses: products of many factors)
    // can lie far below the fixed point's resolution, as in the FP32
    // accumulator: they go to an FP64 word with atomicAdd, keeping their
    // relative precision (and the order of these additions is not fixed).
    __device__ __forceinline__ void addf(uint32_t v, double c) const { atomicAdd(&gf[v], c); }
    // g = (hi 2^L + lo) 2^-S64 + gf
    __device__ __forceinline__ double fixed(uint2 w) const {
        const long long G = (long long)((unsigned long long)(long long)(int)w.y << l) + (long long)w.x;
        return (double)G * inv;
    }
    __device__ __forceinline__ double get(int v) const { return fixed(g[v]) + gf[v]; }
    __device__ __forceinline__ void zero(int v) const {
        g[v] = make_uint2(0u, 0u);
        gf[v] = 0.0;
    }
};

// Clause and node contributions (bounded by their weight) go to the fixed-point
// words; product contributions (XOR and long clauses, whose gradients are
// products of many factors and can be far below the fixed-point resolution)
// go to an FP32 word updated with atomicAdd.  The words are added the raw bits
// of the rounded values, 0x4B400000 + h (the magic constant's bits plus the
// integer); every variable receives the same number deg_v of fixed-point
// contributions in every evaluation, so each word starts the evaluation at
// bias_v = -deg_v * 0x4B400000 (mod 2^32) and ends it holding the exact sum of
// the integers (two's-complement sums are exact modulo 2^32).  The lo word
// (the residual at 2^-(S1+S2)) is used only where the instance needs it: with
// unit weights and degrees up to about 2^10 the hi word alone resolves 2^-20,
// within FP32 rounding of the sums (one shared reduction per contribution).
// FW = 1: hi only; FW = 2: hi and lo.
template <int FW>
struct FixAcc {
    static constexpr bool kDummySlots = true;  // npad >= n + 2 words per array
    int *hi;
    int *lo;
    float *gf;
    const int32_t *bias;
    float s1, s2, i1, i12;
    __device__ __forceinline__ void add(uint32_t v, float c) const {
        constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
        const float m1 = __fmaf_rn(c, s1, kMagic);  // c 2^S1 is exact; one rounding to an integer
        const int h = __float_as_int(m1);           // 0x4B400000 + round(c 2^S1)
        const unsigned a = (unsigned)__cvta_generic_to_shared(hi + v);
        asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(h) : "memory");
        if constexpr (FW == 2) {
            const float r = __fmaf_rn(c, s1, __fsub_rn(kMagic, m1));  // exact residual in [-1/2, 1/2]
            const float m2 = __fmaf_rn(r, s2, kMagic);
            const unsigned b = (unsigned)__cvta_generic_to_shared(lo + v);
            asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(b), "r"(__float_as_int(m2)) : "memory");
        }
    }
    __device__ __forceinline__ void addf(uint32_t v, float c) const { atomicAdd(&gf[v], c); }
    __device__ __forceinline__ float get(int v) const {
        const float g1 = __fmaf_rn((float)hi[v], i1, gf[v]);
        if constexpr (FW == 2) return __fmaf_rn((float)lo[v], i12, g1);
        return g1;
    }
    __device__ __forceinline__ void zero(int v) const {
        const int b = bias[v];
        hi[v] = b;
        if constexpr (FW == 2) lo[v] = b;
        gf[v] = 0.0f;
    }
};

// Accumulators whose dummy variables n and n + 1 have words of their own (reset
// with the others, never read) take the contributions of padding literals
// there instead of branching around them.
template <typename R, typename Acc>
__device__ __forceinline__ void scatter(const Acc &acc, uint32_t lp, R val, int n) {
    const uint32_t v = lp & kVarMask;
    if constexpr (Acc::kDummySlots)
        acc.add(v, flip(val, lp));
    else if (v < (uint32_t)n)
        acc.add(v, flip(val, lp));
}

template <typename R, typename Acc>
__device__ __forceinline__ void scatter_f(const Acc &acc, uint32_t lp, R val, int n) {
    const uint32_t v = lp & kVarMask;
    if (v < (uint32_t)n) acc.addf(v, flip(val, lp));
}

// R consecutive packed literals of this lane (R a multiple of 4, 16-byte aligned).
// (R a multiple of 4: 16-byte loads from a 16-byte aligned lane start; R = 10
// or 14: 8-byte loads from an 8-byte aligned one.)
template <int RL>
__device__ __forceinline__ void load_lits(const int32_t *p, uint32_t (&lp)[RL]) {
    if constexpr (RL % 4 == 0) {
        const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
        for (int k = 0; k < RL / 4; ++k) {
            const int4 t = q[k];
            lp[4 * k + 0] = (uint32_t)t.x;
            lp[4 * k + 1] = (uint32_t)t.y;
            lp[4 * k + 2] = (uint32_t)t.z;
            lp[4 * k + 3] = (uint32_t)t.w;
        }
    } else {
        static_assert(RL % 2 == 0, "literals per lane must be even");
        const int2 *q = reinterpret_cast<const int2 *>(p);
#pragma unroll
        for (int k = 0; k < RL / 2; ++k) {
            const int2 t = q[k];
            lp[2 * k + 0] = (uint32_t)t.x;
            lp[2 * k + 1] = (uint32_t)t.y;
        }
    }
}

// ---------------------------------------------------------------------------
// clause3 path: task.z = 32 CPL clauses, CPL in {1, 2, 4} (whole groups of 32)
// ---------------------------------------------------------------------------
// FE = 2 w q0 q1 q2 - w; the constant -w is folded into f_const on the host,
// so facc collects 2 w q0 q1 q2 only.
// XOR: the record is a short XOR, FE = w y0 y1 y2 where one of the three is the
// dummy (+1, or -1 when negated: even parity; the bank ordering may put it in
// any position, and its scatter is skipped like every dummy's).
template <typename R, int XG, int CPL, bool XOR, typename Acc>
__device__ __forceinline__ void clause_task(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                            const Acc &acc, bool want_g, R &facc) {
    const int n = V.n;
    int4 cl[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) cl[k] = S.clauses[task.y + k * 32 + lane];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const R w = clause_weight<R>(V, cl[k], task.y + k * 32 + lane);
        const R y0 = gather<R, XG>(xrow, (uint32_t)cl[k].x, n);
        const R y1 = gather<R, XG>(xrow, (uint32_t)cl[k].y, n);
        const R y2 = gather<R, XG>(xrow, (uint32_t)cl[k].z, n);
        if constexpr (XOR) {
            const R wy2 = w * y2;
            const R y01 = y0 * y1;
            facc += wy2 * y01;
            if (want_g) {
                scatter<R>(acc, (uint32_t)cl[k].x, wy2 * y1, n);
                scatter<R>(acc, (uint32_t)cl[k].y, wy2 * y0, n);
                scatter<R>(acc, (uint32_t)cl[k].z, w * y01, n);
            }
            continue;
        }
        const R q0 = R(0.5) + R(0.5) * y0;
        const R q1 = R(0.5) + R(0.5) * y1;
        const R q2 = R(0.5) + R(0.5) * y2;
        const R wq12 = w * (q1 * q2);
        facc += wq12 * (R(1) + y0);  // 2 w q0 q1 q2
        if (want_g) {
            const R wq0 = w * q0;
            scatter<R>(acc, (uint32_t)cl[k].x, wq12, n);
            scatter<R>(acc, (uint32_t)cl[k].y, wq0 * q2, n);
            scatter<R>(acc, (uint32_t)cl[k].z, wq0 * q1, n);
        }
    }
}

// ---------------------------------------------------------------------------
// product path (closed forms), kProdR literals per lane, G lanes per constraint
// ---------------------------------------------------------------------------
template <typename R, int XG, typename Acc>
__device__ __forceinline__ void prod_task(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                          const Acc &acc, bool want_g, R &facc) {
    constexpr int RL = kProdR;
    const int n = V.n;
    const int G = (task.x >> 8) & 0xff;
    const int seg = lane >> (__ffs(G) - 1);
    const int sl = lane & (G - 1);
    const int c = task.y + seg;
    const bool valid = seg < task.z;
    uint32_t lp[RL];
    int kind = PROD_OR;
    R w = R(0);
    if (valid) {
        const int4 meta = S.segmeta[c];
        kind = meta.z;
        w = seg_weight<R>(V, meta, c);
        load_lits<RL>(S.seg_lits + meta.x + sl * RL, lp);
    } else {
#pragma unroll
        for (int r = 0; r < RL; ++r) lp[r] = (uint32_t)n;
    }
    const R a = kind == PROD_OR ? R(0.5) : R(0);
    const R bco = kind == PROD_OR ? R(0.5) : R(1);
    const R c0 = kind == PROD_OR ? R(-1) : R(0);
    const R c1 = kind == PROD_OR ? R(2) : (kind == PROD_XOR_ODD ? R(1) : R(-1));
    R u[RL];
#pragma unroll
    for (int r = 0; r < RL; ++r) u[r] = a + bco * gather<R, XG>(xrow, lp[r], n);  // padding: y = +1, u = 1
    R suf[RL];
    suf[RL - 1] = R(1);
#pragma unroll
    for (int r = RL - 1; r >= 1; --r) suf[r - 1] = suf[r] * u[r];
    R P = u[0] * suf[0];
    R X = R(1);
    for (int s = 1; s < G; s <<= 1) {
        const R Pp = __shfl_xor_sync(kFull, P, s);
        X *= Pp;
        P *= Pp;
    }
    if (sl == 0) facc += w * (c0 + c1 * P);
    if (want_g) {
        R pre = w * c1 * bco * X;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            scatter_f<R>(acc, lp[r], pre * suf[r], n);
            pre *= u[r];
        }
    }
}

// ---------------------------------------------------------------------------
// node path (DFT evaluation), NR literals per lane, G lanes per constraint,
// NI nodes per iteration; SF: keep the factors of a node in registers between
// the suffix and the prefix pass (else recompute them)
// ---------------------------------------------------------------------------
template <typename R, int NR, int NI, bool SF, int XG, typename Acc>
__device__ __forceinline__ void node_task(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                          const Acc &acc, bool want_g, R &facc) {
    const int n = V.n;
    const int G = (task.x >> 8) & 0xff;
    const int seg = lane >> (__ffs(G) - 1);
    const int sl = lane & (G - 1);
    const int c = task.y + seg;
    const bool valid = seg < task.z;
    int L = 0, toff = 0;
    const int32_t *lits = nullptr;
    R w = R(0);
    R y[NR];
    if (valid) {
        const int4 meta = S.segmeta[c];
        L = meta.y;
        toff = meta.z;
        w = seg_weight<R>(V, meta, c);
        lits = S.seg_lits + meta.x + sl * NR;
        uint32_t lp[NR];
        load_lits<NR>(lits, lp);
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r] = gather<R, XG>(xrow, lp[r], n);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r] = R(0);
    }
    const int Jc = valid ? (L + 1) / 2 + 1 : 0;  // nodes j = 0 .. floor(N/2), N = L + 1
    R gacc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) gacc[r] = R(0);
    R fe = R(0);
    const int J = task.w;
    const Node<R> zero = {{R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}};
    Node<R> nd[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) nd[q] = q < Jc ? load_node(V, R(0), toff + q) : zero;
    for (int j0 = 0; j0 < J; j0 += NI) {
        Node<R> nx[NI];
#pragma unroll
        for (int q = 0; q < NI; ++q) nx[q] = (j0 + NI + q < Jc) ? load_node(V, R(0), toff + j0 + NI + q) : zero;
        // factors f_r = alpha_j + beta_j y_r (Eq. forward)
        C2<R> fac[NI][SF ? NR : 1];
        if constexpr (SF) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int q = 0; q < NI; ++q)
                    fac[q][r] = {nd[q].a.re + nd[q].b.re * y[r], nd[q].a.im + nd[q].b.im * y[r]};
        }
        auto factor = [&](int q, int r) -> C2<R> {
            if constexpr (SF)
                return fac[q][r];
            else
                return {nd[q].a.re + nd[q].b.re * y[r], nd[q].a.im + nd[q].b.im * y[r]};
        };
        // in-lane suffix products suf[r] = prod_{k > r} f_k
        C2<R> suf[NI][NR];
#pragma unroll
        for (int q = 0; q < NI; ++q) suf[q][NR - 1] = {R(1), R(0)};
#pragma unroll
        for (int r = NR - 1; r >= 1; --r) {
#pragma unroll
            for (int q = 0; q < NI; ++q) suf[q][r - 1] = cmul(suf[q][r], factor(q, r));
        }
        C2<R> P[NI], X[NI];
#pragma unroll
        for (int q = 0; q < NI; ++q) {
            P[q] = cmul(factor(q, 0), suf[q][0]);  // this lane's product
            X[q] = {R(1), R(0)};                   // product of the other lanes of the segment
        }
        for (int s = 1; s < G; s <<= 1) {
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                const C2<R> Pp = {__shfl_xor_sync(kFull, P[q].re, s), __shfl_xor_sync(kFull, P[q].im, s)};
                X[q] = cmul(X[q], Pp);
                P[q] = cmul(P[q], Pp);
            }
        }
        C2<R> pre[NI];
#pragma unroll
        for (int q = 0; q < NI; ++q) {
            fe += nd[q].c.re * P[q].re - nd[q].c.im * P[q].im;  // Re(c_j Q_j)
            pre[q] = cmul(nd[q].d, X[q]);                      // d_j prod(other lanes)
        }
        // prefix pass: pre = d_j X prod_{k < r} f_k
#pragma unroll
        for (int r = 0; r < NR; ++r) {
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                gacc[r] += pre[q].re * suf[q][r].re - pre[q].im * suf[q][r].im;
                if (r + 1 < NR) pre[q] = cmul(pre[q], factor(q, r));
            }
        }
#pragma unroll
        for (int q = 0; q < NI; ++q) nd[q] = nx[q];
    }
    if (valid && sl == 0) facc += w * fe;
    if (want_g && valid) {
        uint32_t lp[NR];
        load_lits<NR>(lits, lp);
#pragma unroll
        for (int r = 0; r < NR; ++r) scatter<R>(acc, lp[r], w * gacc[r], n);
    }
}

// ---------------------------------------------------------------------------
// node path, imaginary-node form (the stable form's default)
// ---------------------------------------------------------------------------
// The stable node factor alpha_j + beta_j y equals alpha_j (1 + z_j y) with
// z_j = beta_j / alpha_j = (1 - w^j) / (1 + w^j) = i t_j, t_j = tan(pi j / N):
// the paper's E(z) = prod_i (1 + y_i z) (Eq. forward / Eq. reduction) at the
// images of the roots of unity, with the per-node scale alpha_j^L folded into
// the coefficients C_j = c_j alpha_j^L and D_j = i t_j C_j (Eq. inverse, Eq.
// chain).  N is odd (L + 1 or L + 2), so no node sits at w^j = -1 and t_j is
// finite.  Every factor 1 + i u (u = t_j y) has real part 1, so a complex
// product by it is two FMAs instead of four, and its modulus is at least 1, so
// the all-but-one product of the other lanes is the segment's product divided
// by this lane's (a well-conditioned division).  Magnitudes are tracked as
// integer exponents (the per-constraint log-magnitude scaling): each lane's
// product is normalised before the cross-lane product, and the terms get their
// scale back through exponent-field arithmetic.  Per (node, literal): u (1
// FMUL), suffix product (2 FFMA), prefix product (2 FFMA), Re(pre suf) (2
// FFMA).
template <typename R, int NR>
struct NodeImConst {
    // a lane's product of NR factors stays below 2^120 (FP32) when
    // t <= 2^(120/NR); above it the suffix product is renormalised once, in the
    // middle of the lane (only for NR = 16 segments longer than 337 literals)
    static constexpr bool kMaySplit = sizeof(R) == 4 && NR >= 16;
    static constexpr float kSplitT = 181.0f;
    // exponent offset of the prefix values (FP32): keeps them in the normal
    // range when the suffix products are large; removed from the result
    static constexpr int kOff = sizeof(R) == 4 ? 64 : 0;
};

// In-lane state of one segment lane: its NR literal values y, the suffix
// products of the current node and the gradient sums over the nodes.  (Packed
// f32x2 FFMA2/FMUL2 for u and the gradient sums were measured slower on the
// cardinality workload: fewer instructions, but more FMA-pipe throttling.)
template <typename R, int NR>
struct LaneIm {
    using K = NodeImConst<R, NR>;
    static constexpr int M = NR / 2;
    R y[NR], u[NR], gacc[NR];
    C2<R> suf[NR];
    __device__ __forceinline__ void set_y(int r, R v) { y[r] = v; }
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int r = 0; r < NR; ++r) gacc[r] = R(0);
    }
    __device__ __forceinline__ R grad(int r) const { return gacc[r]; }
    // suffix products suf[r] = prod_{k > r} (1 + i u_k), u = t y; returns this
    // lane's product (renormalised by 2^-emid in the middle when split)
    __device__ __forceinline__ C2<R> suffix(R t, bool split, int &emid) {
#pragma unroll
        for (int r = 0; r < NR; ++r) u[r] = t * y[r];
        suf[NR - 1] = {R(1), R(0)};
#pragma unroll
        for (int r = NR - 1; r >= 1; --r) {
            suf[r - 1] = {fma(-suf[r].im, u[r], suf[r].re), fma(suf[r].re, u[r], suf[r].im)};
            if (K::kMaySplit && r - 1 == M && split) {
                emid = frexp_max(suf[M].re, suf[M].im);
                const R s = exp2i(R(0), -emid);
                suf[M].re *= s;
                suf[M].im *= s;
            }
        }
        return {fma(-suf[0].im, u[0], suf[0].re), fma(suf[0].re, u[0], suf[0].im)};
    }
    // gacc[r] += Re(pre_r suf[r]) with pre_r = pre prod_{k < r} (1 + i u_k)
    __device__ __forceinline__ void prefix(C2<R> pre, bool split, int emid) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (K::kMaySplit && r == M + 1 && split) {
                const R s = exp2i(R(0), -emid);
                pre.re *= s;
                pre.im *= s;
            }
            gacc[r] = fma(pre.re, suf[r].re, gacc[r]);
            gacc[r] = fma(-pre.im, suf[r].im, gacc[r]);
            if (r + 1 < NR) pre = {fma(-pre.im, u[r], pre.re), fma(pre.re, u[r], pre.im)};
        }
    }
};

template <typename R, int NR, bool FULL, int XG, typename Acc>
__device__ __forceinline__ void node_task_im(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                             const Acc &acc, bool want_g, R &facc, bool want_f) {
    using K = NodeImConst<R, NR>;
    const int n = V.n;
    const int G = (task.x >> 8) & 0xff;
    const int seg = lane >> (__ffs(G) - 1);
    const int sl = lane & (G - 1);
    const int c = task.y + seg;
    const bool valid = seg < task.z;
    int L = 0, toff = 0;
    const int32_t *lits = nullptr;
    R w = R(0);
    LaneIm<R, NR> ln;
    if (valid) {
        const int4 meta = S.segmeta[c];
        L = meta.y;
        toff = meta.z;
        w = seg_weight<R>(V, meta, c);
        lits = S.seg_lits + meta.x + sl * NR;
        uint32_t lp[NR];
        load_lits<NR>(lits, lp);
#pragma unroll
        for (int r = 0; r < NR; ++r) ln.set_y(r, gather<R, XG>(xrow, lp[r], n));  // padding: y = 0, factor 1
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) ln.set_y(r, R(0));
    }
    // nodes j = 0 .. (N - 1) / 2 of this segment; past them (a shorter segment
    // of the same task) the table's entry 0, an all-zero node, is read
    const int Jc = valid ? (L + 1) / 2 + 1 : 0;
    ln.clear();
    // node 0: t = 0, every factor is 1; FE gets C_0, the gradient nothing
    R fe = R(0);
    if (valid) {
        const NodeIm<R> n0 = load_node_im(V, R(0), toff);
        fe = n0.c.re * exp2i(R(0), n0.ec);
    }
    const int J = task.w;
    NodeIm<R> nd = load_node_im(V, R(0), 1 < Jc ? toff + 1 : 0);
    for (int j = 1; j < J; ++j) {
        const NodeIm<R> nx = load_node_im(V, R(0), j + 1 < Jc ? toff + j + 1 : 0);
        // the table is read in order: fetch 256 bytes ahead into L1
        constexpr int kAhead = 256 / (4 * (int)sizeof(R));
        if (j + kAhead < Jc) prefetch_node_im(V, R(0), toff + j + kAhead);
        const bool split = K::kMaySplit && nd.t > R(K::kSplitT);
        int emid = 0;
        C2<R> P = ln.suffix(nd.t, split, emid);
        // this lane's product, normalised: P 2^eown
        int e0;
        {
            const R s = norm_scale(P.re, P.im, e0);
            P.re *= s;
            P.im *= s;
        }
        const int eown = e0 + emid;
        // product over the segment's lanes: A 2^EA.  A full warp (FULL: G = 32)
        // runs the five butterfly levels unconditionally and sums the exponents
        // with one warp reduction; narrower segments take the levels below G
        // (G is the same for the whole warp)
        C2<R> A = P;
        int EA;
        if constexpr (FULL) {
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const C2<R> Ap = {__shfl_xor_sync(kFull, A.re, s), __shfl_xor_sync(kFull, A.im, s)};
                A = cmul(A, Ap);
            }
            EA = __reduce_add_sync(kFull, eown);
        } else {
            EA = eown;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                if (s < G) {
                    const C2<R> Ap = {__shfl_xor_sync(kFull, A.re, s), __shfl_xor_sync(kFull, A.im, s)};
                    EA += __shfl_xor_sync(kFull, EA, s);
                    A = cmul(A, Ap);
                }
            }
        }
        if (want_f) fe = fma(fma(nd.c.re, A.re, -nd.c.im * A.im), exp2i(R(0), nd.ec + EA), fe);  // Re(C_j Q_j)
        // product of the other lanes X = A / P = A conj(P) / |P|^2 (|P| >= 1/2);
        // pre = D_j X, scaled by 2^kOff (and by 2^emid while it meets
        // renormalised suffix products)
        const R sc = recip(fma(P.re, P.re, P.im * P.im)) * exp2i(R(0), nd.ec + EA - eown + K::kOff + emid);
        const C2<R> AP = {fma(A.re, P.re, A.im * P.im), fma(A.im, P.re, -A.re * P.im)};
        const C2<R> D = {-nd.t * nd.c.im, nd.t * nd.c.re};  // D_j = i t_j C_j
        C2<R> pre = cmul(D, AP);
        pre.re *= sc;
        pre.im *= sc;
        ln.prefix(pre, split, emid);
        nd = nx;
    }
    if (valid && sl == 0) facc += w * fe;
    if (want_g && valid) {
        const R wg = w * exp2i(R(0), -K::kOff);
        uint32_t lp[NR];
        load_lits<NR>(lits, lp);
#pragma unroll
        for (int r = 0; r < NR; ++r) scatter<R>(acc, lp[r], wg * ln.grad(r), n);
    }
}

// A node task of either form, nr literals per lane (task bits 16..23): a kernel
// built for NR = 16 also runs 12 and 8 (both forms) and, in FP32, 14 and 10
// (imaginary form); one built for NR = 8 runs 8.
template <typename R, int NR, int NI, bool SF, int XG, typename Acc>
__device__ __forceinline__ void node_dispatch(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                              const Acc &acc, bool want_g, R &facc, bool want_f = true) {
    const int nr = (task.x >> 16) & 0xff;
    if (V.node_form == NODE_FORM_IMAG) {
        const bool full = ((task.x >> 8) & 0xff) == 32;
        if constexpr (NR >= 16) {
            // 14 and 10 literals per lane: FP32 images only (the host never builds them for FP64)
            constexpr bool kOdd = sizeof(R) == 4;
            if (kOdd && nr == 14) {
                if constexpr (kOdd) {
                    if (full) node_task_im<R, 14, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                    else node_task_im<R, 14, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                }
            } else if (nr == 12) {
                if (full) node_task_im<R, 12, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                else node_task_im<R, 12, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
            } else if (kOdd && nr == 10) {
                if constexpr (kOdd) {
                    if (full) node_task_im<R, 10, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                    else node_task_im<R, 10, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                }
            } else if (nr == 8) {
                if (full) node_task_im<R, 8, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                else node_task_im<R, 8, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
            } else {
                if (full) node_task_im<R, 16, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
                else node_task_im<R, 16, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
            }
        } else if constexpr (NR > 0) {
            if (full) node_task_im<R, NR, true, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
            else node_task_im<R, NR, false, XG>(V, S, task, lane, xrow, acc, want_g, facc, want_f);
        }
    } else {
        if constexpr (NR >= 16) {
            if (nr == 12)
                node_task<R, 12, NI, SF, XG>(V, S, task, lane, xrow, acc, want_g, facc);
            else if (nr == 8)
                node_task<R, 8, NI, SF, XG>(V, S, task, lane, xrow, acc, want_g, facc);
            else
                node_task<R, 16, NI, SF, XG>(V, S, task, lane, xrow, acc, want_g, facc);
        } else if constexpr (NR > 0) {
            node_task<R, NR, NI, SF, XG>(V, S, task, lane, xrow, acc, want_g, facc);
        }
    }
}

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.  Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T t = T(0);
    if (wid == 0) {
        t = lane < nw ? red[lane] : T(0);
        t = warp_sum(t);
    }
    return t;
}

// Exact check of sgn(xrow): number of violated constraints (valid in thread 0).
// With U set, also adds one to U[c] for every violated constraint c.
template <typename R>
__device__ __forceinline__ int block_unsat(const DevView &V, const R *xrow, int *ired, int32_t *U) {
    int cnt = 0;
    for (int c = threadIdx.x; c < V.m; c += blockDim.x) {
        const int a = __ldg(&V.row_ptr[c]), e = __ldg(&V.row_ptr[c + 1]);
        int s = 0;
        for (int i = a; i < e; ++i) {
            const uint32_t lp = (uint32_t)__ldg(&V.lits[i]);
            const int var_true = xrow[lp & kVarMask] < R(0);  // sgn(x) = -1 encodes True
            s += var_true ^ (int)(lp >> 31);
        }
        const int t = __ldg(&V.type[c]), p = __ldg(&V.param[c]);
        const bool ok = t == 0 ? s >= 1 : (t == 1 ? ((s & 1) == (p & 1)) : s >= p);
        cnt += ok ? 0 : 1;
        if (!ok && U) atomicAdd(&U[c], 1);
    }
    return block_sum(cnt, ired);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform restart value on the 24-bit grid of [-1, 1).
template <typename R>
__device__ __forceinline__ R restart_value(uint64_t key_b, uint64_t v) {
    const uint64_t h = splitmix64(key_b ^ v);
    const int u = (int)(h >> 40) - (1 << 23);
    return R(u) * R(1.0 / 8388608.0);
}

// ---------------------------------------------------------------------------
// the per-point body (shared by the single-instance and the batch kernels)
// ---------------------------------------------------------------------------
// Shared-memory layout: x | gradient words | resident image (SMEM_RES); the
// image part is set up by the caller (make_src).
template <typename R, int SM>
__device__ __forceinline__ size_t image_offset(int n) {
    const int npad = (n + 2 + 3) & ~3;
    constexpr bool FIX = SM == SMEM_RES && sizeof(R) == 4;
    // FP32 resident: x | hi | lo | gf; FP64: x | fixed-point words | FP64 product word
    return FIX ? 4 * (size_t)npad * 4 : (sizeof(R) == 8 ? 3 : 2) * (size_t)npad * sizeof(R);
}

// Constraint-data view for the point loop; SMEM_RES copies the image into shared
// memory first (skipped when copy is false: the same instance's image is there).
template <typename R, int SM, int THREADS>
__device__ __forceinline__ Src make_src(const DevView &V, unsigned char *smem_raw, bool copy) {
    Src S;
    if constexpr (SM == SMEM_RES) {
        int4 *img = reinterpret_cast<int4 *>(smem_raw + image_offset<R, SM>(V.n));
        if (copy)
            for (int i = threadIdx.x; i < V.res_int4; i += THREADS) img[i] = __ldg(&V.res_image[i]);
        S.tasks = img + V.res_off_tasks;
        S.clauses = img + V.res_off_clauses;
        S.segmeta = img + V.res_off_segmeta;
        S.seg_lits = reinterpret_cast<const int32_t *>(img + V.res_off_lits);
    } else {
        S.tasks = V.tasks;
        S.clauses = V.clauses;
        S.segmeta = V.segmeta;
        S.seg_lits = V.seg_lits;
    }
    return S;
}

struct BlockShared {
    int ctr;
    double red[32];
    int ired[32];
};

// One evaluation of every warp task at the point xrow: this thread's share of
// sum_c w FE_c (up to the constants) is returned; with want_g the gradient
// contributions are added to G.  Starts and ends with a CTA barrier.
template <typename R, int NR, int NI, bool SF, int XG, typename Acc>
__device__ __forceinline__ R eval_tasks(const DevView &V, const Src &S, const R *xrow, const Acc &G, bool want_g,
                                        int &s_ctr, bool want_f = true) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_ctr = 0;
    __syncthreads();
    R facc = R(0);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&s_ctr, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= V.n_task) break;
        const int4 task = S.tasks[t];
        const int kind = task.x & 0xff;
        if (kind == TASK_CLAUSE) {
            if (task.z == 128)
                clause_task<R, XG, 4, false>(V, S, task, lane, xrow, G, want_g, facc);
            else if (task.z == 64)
                clause_task<R, XG, 2, false>(V, S, task, lane, xrow, G, want_g, facc);
            else
                clause_task<R, XG, 1, false>(V, S, task, lane, xrow, G, want_g, facc);
        } else if (kind == TASK_XOR2) {
            if (task.z == 128)
                clause_task<R, XG, 4, true>(V, S, task, lane, xrow, G, want_g, facc);
            else if (task.z == 64)
                clause_task<R, XG, 2, true>(V, S, task, lane, xrow, G, want_g, facc);
            else
                clause_task<R, XG, 1, true>(V, S, task, lane, xrow, G, want_g, facc);
        } else if (kind == TASK_PROD) {
            prod_task<R, XG>(V, S, task, lane, xrow, G, want_g, facc);
        } else {
            // node tasks carry their literals per lane in bits 16..23 (the batch
            // kernel also meets images built with 8 literals per lane)
            node_dispatch<R, NR, NI, SF, XG>(V, S, task, lane, xrow, G, want_g, facc, want_f);
        }
    }
    __syncthreads();
    return facc;
}

// Correctly rounded multiply and add (no contraction), as the FP64 reference computes.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename R>
__device__ __forceinline__ R clip1(R z) {
    return z < R(-1) ? R(-1) : (z > R(1) ? R(1) : z);
}

// Sum over the CTA, result in every thread (uses sh.red; contains barriers).
__device__ __forceinline__ double block_sum_all(double v, BlockShared &sh) {
    const double t = block_sum(v, sh.red);
    if (threadIdx.x == 0) sh.red[0] = t;
    __syncthreads();
    const double r = sh.red[0];
    __syncthreads();
    return r;
}

// One point b of one instance: stage x, T projected-GD iterations (or one
// evaluation), exact check and restart.  All threads of the CTA take part.
// FW: words of the FP32 fixed-point gradient in the shared-memory-resident mode
// (1 where the instance's range allows it, else 2; see FixAcc).
template <typename R, int NR, int NI, int SM, int THREADS, int FW = 2>
__device__ __forceinline__ void run_point(const DevView &V, const FusedArgs &A, int b, unsigned char *smem_raw,
                                          const Src &S, BlockShared &sh) {
    // FP32 node factors: kept in registers between the suffix and the prefix pass,
    // except for 16 literals per lane at 512 threads per CTA (the single-instance
    // kernel), which recomputes them to fit the registers (measured 2.6% faster on
    // the cardinality workload than 384 threads with stored factors; the batch
    // kernel keeps 384 threads and stored factors, 4% faster on the uneven set)
    constexpr bool SF = sizeof(R) == 4 && !(NR >= 16 && THREADS > 384);
    // SMEM_RES keeps x and g in shared memory like SMEM_FULL and adds the resident image.
    constexpr bool RES = SM == SMEM_RES;
    constexpr int XG = RES ? SMEM_FULL : SM;
    // FP32 shared-resident mode: x | g hi words | g lo words | g FP32 words | image;
    // otherwise x | g | image.
    constexpr bool FIX = RES && sizeof(R) == 4;
    // FP64 with the gradient in shared memory: two-word fixed point (Fix64Acc;
    // the host keeps such instances out of these modes where its resolution
    // would be coarser than 2^-44)
    constexpr bool FIX64 = sizeof(R) == 8 && XG == SMEM_FULL;
    using Acc = typename std::conditional<FIX, FixAcc<FW>,
                                          typename std::conditional<FIX64, Fix64Acc, PlainAcc<R>>::type>::type;
    int &s_ctr = sh.ctr;
    double *s_red = sh.red;
    int *s_ired = sh.ired;

    const int n = V.n;
    const int npad = (n + 2 + 3) & ~3;  // n variables + 2 dummies, rounded to 4
    const int tid = threadIdx.x;
    R *xs = reinterpret_cast<R *>(smem_raw);
    R *gs = xs + npad;
    const bool pgfp = A.mode == MODE_PGFP;
    const bool step = A.mode == MODE_STEP || pgfp;
    const R *x_in = static_cast<const R *>(A.x_in);
    R *x_out = static_cast<R *>(A.x_out);
    R *g_out = static_cast<R *>(A.g);
    R *g_scr = static_cast<R *>(A.g_scratch);
    const R lr = R(A.sp.lr);

    const size_t rowoff = (size_t)b * (size_t)n;
    // ---- stage x ----
    const R *xrow;
    if constexpr (XG != SMEM_NONE) {
        bool bad = false;
        for (int v = tid; v < n; v += THREADS) {
            const R xv = x_in[rowoff + v];
            bad |= isnan(xv);
            xs[v] = xv;
        }
        if (tid == 0) {
            xs[n] = R(1);
            xs[n + 1] = R(0);
        }
        if (bad) atomicOr(V.status, STATUS_NAN);
        xrow = xs;
    } else {
        if (step && x_out != x_in) {
            for (int v = tid; v < n; v += THREADS) x_out[rowoff + v] = x_in[rowoff + v];
            __syncthreads();
        }
        xrow = step ? x_out + rowoff : x_in + rowoff;
        bool bad = false;
        for (int v = tid; v < n; v += THREADS) bad |= isnan(xrow[v]);
        if (bad) atomicOr(V.status, STATUS_NAN);
    }
    Acc G;
    bool want_g;
    int glen;
    if constexpr (FIX) {
        G.hi = reinterpret_cast<int *>(smem_raw + (size_t)npad * 4);
        G.lo = G.hi + npad;
        G.gf = reinterpret_cast<float *>(G.lo + npad);
        G.bias = V.fix_bias;
        G.s1 = V.fix_s1;
        G.s2 = V.fix_s2;
        G.i1 = V.fix_i1;
        G.i12 = V.fix_i12;
        want_g = step || g_out != nullptr;
        glen = npad;
    } else if constexpr (FIX64) {
        G.g = reinterpret_cast<uint2 *>(gs);
        G.gf = gs + npad;
        G.s = V.fix64_s;
        G.inv = V.fix64_i;
        G.l = V.fix64_l;
        want_g = step || g_out != nullptr;
        glen = npad;
    } else if constexpr (XG == SMEM_FULL) {
        G.g = gs;
        want_g = step || g_out != nullptr;
        glen = npad;
    } else {
        G.g = step ? g_scr + rowoff : (g_out ? g_out + rowoff : nullptr);
        want_g = G.g != nullptr;
        glen = n;
    }
    if (want_g)
        for (int v = tid; v < glen; v += THREADS) G.zero(v);

    if constexpr (XG != SMEM_NONE) {
        if (pgfp) {
            // App. A.3, Alg. PGFP with a FISTA line search (Beck-Teboulle backtracking):
            // xs holds the point being evaluated (y_k or a trial p), the iterate x_k
            // lives in the output row and y_k in the caller's scratch row.
            R *xk = x_out + rowoff;
            R *ys = static_cast<R *>(A.y_scratch) + rowoff;
            for (int v = tid; v < n; v += THREADS) {
                ys[v] = xs[v];
                xk[v] = xs[v];
            }
            double eta = A.sp.lr, tk = 1.0;
            int it = 0;
            while (it < A.sp.T) {
                ++it;
                const double fy = block_sum_all((double)eval_tasks<R, NR, NI, SF, XG>(V, S, xs, G, true, s_ctr), sh);
                for (int ls = 0; ls < A.maxls; ++ls) {
                    double d = 0.0, q = 0.0;
                    const R er = R(eta);
                    for (int v = tid; v < n; v += THREADS) {
                        const R y = ys[v];
                        const R gv = R(G.get(v));
                        const R p = clip1(add_rn(y, -mul_rn(er, gv)));
                        const R dz = add_rn(p, -y);
                        xs[v] = p;
                        d += (double)gv * (double)dz;
                        q += (double)dz * (double)dz;
                    }
                    d = block_sum_all(d, sh);
                    q = block_sum_all(q, sh);
                    const double fp =
                        block_sum_all((double)eval_tasks<R, NR, NI, SF, XG>(V, S, xs, G, false, s_ctr), sh);
                    // same value in every thread; a trial equal to y (q = 0: every
                    // coordinate clipped) meets the test with equality and is taken
                    // without comparing two evaluations of the same point
                    if (q == 0.0 || fp <= fy + d + q / (2.0 * eta) + A.slack) break;
                    if (ls + 1 < A.maxls) eta *= A.beta;
                }
                const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
                const R mom = R((tk - 1.0) / tn);
                tk = tn;
                for (int v = tid; v < n; v += THREADS) {
                    const R xn = xs[v];
                    const R z = clip1(add_rn(xn, mul_rn(mom, add_rn(xn, -xk[v]))));
                    xk[v] = xn;
                    ys[v] = z;
                    xs[v] = z;
                    G.zero(v);
                }
                __syncthreads();
                if (eta < A.eta_min) break;
            }
            for (int v = tid; v < n; v += THREADS) xs[v] = xk[v];
            if (tid == 0) {
                if (A.iters) A.iters[b] = it;
                if (A.eta_out) A.eta_out[b] = eta;
            }
            __syncthreads();
        }
    }
    const int iters = pgfp ? 0 : (step ? A.sp.T : 1);
    for (int it = 0; it < iters; ++it) {
        // a fixed step needs the gradient only; the objective is skipped on the node path
        R facc = eval_tasks<R, NR, NI, SF, XG>(V, S, xrow, G, want_g, s_ctr, !step);
        if (!step) {
            if (A.f) {
                const double tot = block_sum((double)facc, s_red);
                if (tid == 0) A.f[b] = tot + V.f_const[0];
            }
            if constexpr (XG == SMEM_FULL) {
                if (g_out)
                    for (int v = tid; v < n; v += THREADS) g_out[rowoff + v] = G.get(v);
            }
        } else {
            // projected gradient step x <- clip(x - lr g, -1, 1); reset the accumulator
            R *xw = (XG != SMEM_NONE) ? xs : (x_out + rowoff);
            for (int v = tid; v < n; v += THREADS) {
                R z = xw[v] - lr * G.get(v);
                z = z < R(-1) ? R(-1) : (z > R(1) ? R(1) : z);
                xw[v] = z;
                G.zero(v);
            }
            __syncthreads();
        }
    }
    if (step) {
        __syncthreads();  // the staged x (T = 0) or the last update is complete
        const R *xc = (XG != SMEM_NONE) ? xs : (x_out + rowoff);
        const int unsat = block_unsat<R>(V, xc, s_ired, A.unsat_counts);
        if (tid == 0) s_ired[0] = unsat;
        __syncthreads();
        const int u = s_ired[0];
        if (tid == 0) {
            if (A.solved) A.solved[b] = (uint8_t)(u == 0);
            if (A.n_unsat) A.n_unsat[b] = u;
        }
        R *xw = (XG != SMEM_NONE) ? xs : (x_out + rowoff);
        if (u != 0 && A.sp.restart) {
            const uint64_t kb =
                splitmix64(splitmix64(splitmix64(A.sp.seed) ^ A.sp.epoch) ^ (A.sp.b_offset + (uint64_t)b));
            for (int v = tid; v < n; v += THREADS) xw[v] = restart_value<R>(kb, (uint64_t)v);
        }
        if constexpr (XG != SMEM_NONE) {
            for (int v = tid; v < n; v += THREADS) x_out[rowoff + v] = xs[v];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Two points per CTA (fixed step, FP32, shared-memory-resident image, one
// fixed-point word): every warp task is evaluated at both points after one
// load of its clause records, which shares the record loads and the task
// overhead and gives each warp two independent dependency chains.  Point 0
// keeps the one-point layout (x | hi | lo (unused) | gf | image); point 1 has
// its own x | hi | gf block after the image.  Each point's arithmetic is the
// one-point kernel's, term for term, and its fixed-point sums do not depend on
// the order of the reductions, so both points end with the one-point results
// bit for bit where every contribution is fixed point (XOR products add with
// FP32 atomics, whose order may differ).
// ---------------------------------------------------------------------------
template <int CPL, bool XOR>
__device__ __forceinline__ void clause_task2(const DevView &V, const Src &S, int4 task, int lane, const float *x0,
                                             const float *x1, const FixAcc<1> &G0, const FixAcc<1> &G1) {
    const int n = V.n;
    int4 cl[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) cl[k] = S.clauses[task.y + k * 32 + lane];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const float w = clause_weight<float>(V, cl[k], task.y + k * 32 + lane);
        const uint32_t l0 = (uint32_t)cl[k].x, l1 = (uint32_t)cl[k].y, l2 = (uint32_t)cl[k].z;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float *xr = p ? x1 : x0;
            const FixAcc<1> &G = p ? G1 : G0;
            const float y0 = gather<float, SMEM_FULL>(xr, l0, n);
            const float y1 = gather<float, SMEM_FULL>(xr, l1, n);
            const float y2 = gather<float, SMEM_FULL>(xr, l2, n);
            if constexpr (XOR) {
                const float wy2 = w * y2;
                const float y01 = y0 * y1;
                scatter<float>(G, l0, wy2 * y1, n);
                scatter<float>(G, l1, wy2 * y0, n);
                scatter<float>(G, l2, w * y01, n);
            } else {
                const float q0 = 0.5f + 0.5f * y0;
                const float q1 = 0.5f + 0.5f * y1;
                const float q2 = 0.5f + 0.5f * y2;
                const float wq12 = w * (q1 * q2);
                const float wq0 = w * q0;
                scatter<float>(G, l0, wq12, n);
                scatter<float>(G, l1, wq0 * q2, n);
                scatter<float>(G, l2, wq0 * q1, n);
            }
        }
    }
}

// One evaluation (gradients only) of every warp task at both points; starts and
// ends with a CTA barrier.
template <int NR, int NI, bool SF>
__device__ __forceinline__ void eval_tasks2(const DevView &V, const Src &S, const float *x0, const float *x1,
                                            const FixAcc<1> &G0, const FixAcc<1> &G1, int &s_ctr) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_ctr = 0;
    __syncthreads();
    float facc = 0.0f;  // the objective is not needed by a fixed step
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&s_ctr, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= V.n_task) break;
        const int4 task = S.tasks[t];
        const int kind = task.x & 0xff;
        if (kind == TASK_CLAUSE || kind == TASK_XOR2) {
            const bool xr = kind == TASK_XOR2;
            if (task.z == 128) {
                if (xr) clause_task2<4, true>(V, S, task, lane, x0, x1, G0, G1);
                else clause_task2<4, false>(V, S, task, lane, x0, x1, G0, G1);
            } else if (task.z == 64) {
                if (xr) clause_task2<2, true>(V, S, task, lane, x0, x1, G0, G1);
                else clause_task2<2, false>(V, S, task, lane, x0, x1, G0, G1);
            } else {
                if (xr) clause_task2<1, true>(V, S, task, lane, x0, x1, G0, G1);
                else clause_task2<1, false>(V, S, task, lane, x0, x1, G0, G1);
            }
        } else if (kind == TASK_PROD) {
            prod_task<float, SMEM_FULL>(V, S, task, lane, x0, G0, true, facc);
            prod_task<float, SMEM_FULL>(V, S, task, lane, x1, G1, true, facc);
        } else {
            node_dispatch<float, NR, NI, SF, SMEM_FULL>(V, S, task, lane, x0, G0, true, facc, false);
            node_dispatch<float, NR, NI, SF, SMEM_FULL>(V, S, task, lane, x1, G1, true, facc, false);
        }
    }
    __syncthreads();
}

// Points b and b + 1 through T fixed-step iterations, the exact check, the
// violation counts, the restart and the write-back, as run_point does for one.
template <int NR, int NI, int THREADS>
__device__ __forceinline__ void run_pair(const DevView &V, const FusedArgs &A, int b, unsigned char *smem_raw,
                                         const Src &S, BlockShared &sh) {
    constexpr bool SF = !(NR >= 16 && THREADS > 384);  // as run_point for FP32
    const int n = V.n;
    const int npad = (n + 2 + 3) & ~3;
    const int tid = threadIdx.x;
    unsigned char *blk1 = smem_raw + image_offset<float, SMEM_RES>(n) + (size_t)V.res_int4 * 16;
    float *xs[2] = {reinterpret_cast<float *>(smem_raw), reinterpret_cast<float *>(blk1)};
    FixAcc<1> G[2];
    G[0].hi = reinterpret_cast<int *>(smem_raw + (size_t)npad * 4);
    G[0].lo = G[0].hi + npad;
    G[0].gf = reinterpret_cast<float *>(G[0].lo + npad);
    G[1].hi = reinterpret_cast<int *>(blk1 + (size_t)npad * 4);
    G[1].lo = nullptr;
    G[1].gf = reinterpret_cast<float *>(G[1].hi + npad);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        G[p].bias = V.fix_bias;
        G[p].s1 = V.fix_s1;
        G[p].s2 = V.fix_s2;
        G[p].i1 = V.fix_i1;
        G[p].i12 = V.fix_i12;
    }
    const float *x_in = static_cast<const float *>(A.x_in);
    float *x_out = static_cast<float *>(A.x_out);
    const float lr = float(A.sp.lr);
    bool bad = false;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const size_t rowoff = (size_t)(b + p) * (size_t)n;
        for (int v = tid; v < n; v += THREADS) {
            const float xv = x_in[rowoff + v];
            bad |= isnan(xv);
            xs[p][v] = xv;
        }
        if (tid == 0) {
            xs[p][n] = 1.0f;
            xs[p][n + 1] = 0.0f;
        }
        for (int v = tid; v < npad; v += THREADS) G[p].zero(v);
    }
    if (bad) atomicOr(V.status, STATUS_NAN);
    for (int it = 0; it < A.sp.T; ++it) {
        eval_tasks2<NR, NI, SF>(V, S, xs[0], xs[1], G[0], G[1], sh.ctr);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            for (int v = tid; v < n; v += THREADS) {
                float z = xs[p][v] - lr * G[p].get(v);
                z = z < -1.0f ? -1.0f : (z > 1.0f ? 1.0f : z);
                xs[p][v] = z;
                G[p].zero(v);
            }
        }
        __syncthreads();
    }
    __syncthreads();  // the staged points (T = 0) are complete
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int unsat = block_unsat<float>(V, xs[p], sh.ired, A.unsat_counts);
        if (tid == 0) sh.ired[0] = unsat;
        __syncthreads();
        const int u = sh.ired[0];
        __syncthreads();  // every thread has read u before the next check writes sh.ired
        if (tid == 0) {
            if (A.solved) A.solved[b + p] = (uint8_t)(u == 0);
            if (A.n_unsat) A.n_unsat[b + p] = u;
        }
        if (u != 0 && A.sp.restart) {
            const uint64_t kb = splitmix64(splitmix64(splitmix64(A.sp.seed) ^ A.sp.epoch) ^
                                           (A.sp.b_offset + (uint64_t)(b + p)));
            for (int v = tid; v < n; v += THREADS) xs[p][v] = restart_value<float>(kb, (uint64_t)v);
        }
        const size_t rowoff = (size_t)(b + p) * (size_t)n;
        for (int v = tid; v < n; v += THREADS) x_out[rowoff + v] = xs[p][v];
    }
    __syncthreads();
}

// Nodes per iteration of the node loop (independent multiply chains): one.  Two
// interleaved nodes at 16 literals per lane need about 170 registers and were
// measured slower on the cardinality workload (fewer warps per SM).
template <typename R, int NR>
constexpr int node_interleave() {
    return 1;
}

// ---------------------------------------------------------------------------
// the fused kernel: one instance, points b = blockIdx.x, blockIdx.x + gridDim.x, ...
// ---------------------------------------------------------------------------
// PP = 2: two points per CTA (fixed step, FP32, SMEM_RES, FW = 1; run_pair),
// the last point of an odd B alone.
template <typename R, int NR, int NI, int SM, int THREADS, int FW = 2, int PP = 1>
__global__ void __launch_bounds__(THREADS, 1) fused_kernel(const DevView V, const FusedArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockShared sh;
    const Src S = make_src<R, SM, THREADS>(V, smem_raw, true);
    if constexpr (PP == 2) {
        static_assert(sizeof(R) == 4 && SM == SMEM_RES && FW == 1, "two points per CTA: FP32, resident, one word");
        for (int b = 2 * blockIdx.x; b < A.B; b += 2 * gridDim.x) {
            if (b + 1 < A.B) run_pair<NR, NI, THREADS>(V, A, b, smem_raw, S, sh);
            else run_point<R, NR, NI, SM, THREADS, FW>(V, A, b, smem_raw, S, sh);
        }
    } else {
        for (int b = blockIdx.x; b < A.B; b += gridDim.x)
            run_point<R, NR, NI, SM, THREADS, FW>(V, A, b, smem_raw, S, sh);
    }
}

// ---------------------------------------------------------------------------
// the batch kernel: several instances of uneven size in one persistent launch.
// Each CTA pulls (instance, point) items, ordered by decreasing estimated cost,
// from a global counter; no CTA ever waits on another.
// ---------------------------------------------------------------------------
template <typename R, int NR, int NI, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) batch_kernel(const BatchInst *__restrict__ insts,
                                                           const int2 *__restrict__ items, int n_items,
                                                           int *counter, const StepParams sp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockShared sh;
    __shared__ int s_item;
    int cur = -1;  // instance whose resident image is in shared memory
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 item = items[it];
        const BatchInst &BI = insts[item.x];
        // the call's step parameters; the restart key offset stays per instance
        FusedArgs A = BI.A;
        const uint64_t b_offset = A.sp.b_offset;
        A.sp = sp;
        A.sp.b_offset = b_offset;
        switch (BI.mode) {
        case SMEM_RES: {
            const Src S = make_src<R, SMEM_RES, THREADS>(BI.V, smem_raw, item.x != cur);
            cur = item.x;
            run_point<R, NR, NI, SMEM_RES, THREADS>(BI.V, A, item.y, smem_raw, S, sh);
            break;
        }
        case SMEM_FULL:
            cur = -1;
            run_point<R, NR, NI, SMEM_FULL, THREADS>(BI.V, A, item.y, smem_raw,
                                                     make_src<R, SMEM_FULL, THREADS>(BI.V, smem_raw, false), sh);
            break;
        case SMEM_X:
            cur = -1;
            run_point<R, NR, NI, SMEM_X, THREADS>(BI.V, A, item.y, smem_raw,
                                                  make_src<R, SMEM_X, THREADS>(BI.V, smem_raw, false), sh);
            break;
        default:
            cur = -1;
            run_point<R, NR, NI, SMEM_NONE, THREADS>(BI.V, A, item.y, smem_raw,
                                                     make_src<R, SMEM_NONE, THREADS>(BI.V, smem_raw, false), sh);
        }
    }
}

}  // namespace dev
}  // namespace ffsat
