// Exact checker kernel and the plain FP64 comparator.
#include "ffsat.h"
#include "fused_kernel.cuh"

namespace ffsat {
namespace dev {

// ---------------------------------------------------------------------------
// exact checker: one CTA per point, x read straight from global memory
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) check_kernel(const DevView V, int B, const R *__restrict__ x, uint8_t *sat,
                                                    int32_t *n_unsat, int32_t *U) {
    __shared__ int s_ired[32];
    const int n = V.n;
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const R *xrow = x + (size_t)b * (size_t)n;
        bool bad = false;
        for (int v = threadIdx.x; v < n; v += blockDim.x) bad |= isnan(xrow[v]);
        if (bad) atomicOr(V.status, STATUS_NAN);
        const int u = block_unsat<R>(V, xrow, s_ired, U);
        if (threadIdx.x == 0) {
            if (sat) sat[b] = (uint8_t)(u == 0);
            if (n_unsat) n_unsat[b] = u;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// plain FP64 comparator: naive mapping, one thread per (constraint, point)
// ---------------------------------------------------------------------------
__global__ void plain64_init(int B, int n, double *f, double *g, const double *f_const) {
    const size_t tot = (size_t)B * (size_t)n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
        g[i] = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B; i += (size_t)gridDim.x * blockDim.x)
        f[i] = f_const[1];
}

// Clauses and XOR constraints by their closed forms, all-but-one products by
// direct O(L^2) loops.
__global__ void plain64_closed(const DevView V, int B, const double *x, double *f, double *g, int n_ids,
                               const int32_t *ids) {
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_ids * (size_t)B) return;
    const int c = ids[idx % n_ids];
    const int b = (int)(idx / n_ids);
    const double *xb = x + (size_t)b * V.n;
    double *gb = g + (size_t)b * V.n;
    const int a = V.row_ptr[c], e = V.row_ptr[c + 1];
    const int t = V.type[c], p = V.param[c];
    const double w = V.cons_wd[c];
    const bool is_or = t == 0;
    double prod = 1.0;
    for (int i = a; i < e; ++i) {
        const double y = gather<double, SMEM_FULL>(xb, (uint32_t)V.lits[i], V.n);
        prod *= is_or ? 0.5 * (1.0 + y) : y;
    }
    const double c1 = is_or ? 2.0 : ((p & 1) ? 1.0 : -1.0);
    const double c0 = is_or ? -1.0 : 0.0;
    const double bco = is_or ? 0.5 : 1.0;
    atomicAdd(&f[b], w * (c0 + c1 * prod));
    for (int i = a; i < e; ++i) {
        double rest = 1.0;
        for (int l = a; l < e; ++l) {
            if (l == i) continue;
            const double y = gather<double, SMEM_FULL>(xb, (uint32_t)V.lits[l], V.n);
            rest *= is_or ? 0.5 * (1.0 + y) : y;
        }
        scatter<double>(PlainAcc<double>{gb}, (uint32_t)V.lits[i], w * c1 * bco * rest, V.n);
    }
}

// Node (DFT) constraints: per node, prefix products in a local array, then a
// backward sweep with a running suffix product.
__global__ void __launch_bounds__(128) plain64_node(const DevView V, int B, const double *x, double *f, double *g,
                                                    int n_ids, const int32_t *ids) {
    const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)n_ids * (size_t)B) return;
    const int c = ids[idx % n_ids];
    const int b = (int)(idx / n_ids);
    const double *xb = x + (size_t)b * V.n;
    double *gb = g + (size_t)b * V.n;
    const int a = V.row_ptr[c], e = V.row_ptr[c + 1];
    const int L = e - a;
    const int toff = V.cons_tab[c];
    const double w = V.cons_wd[c];
    double yv[FFSAT_MAX_LEN], gr[FFSAT_MAX_LEN];
    double pre_re[FFSAT_MAX_LEN], pre_im[FFSAT_MAX_LEN];
    for (int i = 0; i < L; ++i) {
        yv[i] = gather<double, SMEM_FULL>(xb, (uint32_t)V.lits[a + i], V.n);
        gr[i] = 0.0;
    }
    const int J = (L + 1) / 2 + 1;
    double fe = 0.0;
    for (int j = 0; j < J; ++j) {
        const double *t = V.tab_d + 8 * (size_t)(toff + j);
        const double ar = t[0], ai = t[1], br = t[2], bi = t[3], dr = t[4], di = t[5], cr = t[6], ci = t[7];
        double pr = 1.0, pi = 0.0;
        for (int i = 0; i < L; ++i) {
            pre_re[i] = pr;
            pre_im[i] = pi;
            const double fr = ar + br * yv[i], fi = ai + bi * yv[i];
            const double nr = pr * fr - pi * fi, ni = pr * fi + pi * fr;
            pr = nr;
            pi = ni;
        }
        fe += cr * pr - ci * pi;
        double sr = 1.0, si = 0.0;
        for (int i = L - 1; i >= 0; --i) {
            // d * pre * suf
            const double qr = pre_re[i] * sr - pre_im[i] * si, qi = pre_re[i] * si + pre_im[i] * sr;
            gr[i] += dr * qr - di * qi;
            const double fr = ar + br * yv[i], fi = ai + bi * yv[i];
            const double nr = sr * fr - si * fi, ni = sr * fi + si * fr;
            sr = nr;
            si = ni;
        }
    }
    atomicAdd(&f[b], w * fe);
    for (int i = 0; i < L; ++i) scatter<double>(PlainAcc<double>{gb}, (uint32_t)V.lits[a + i], w * gr[i], V.n);
}

}  // namespace dev

cudaError_t launch_check(const DevView &V, bool f64, int B, const void *x, uint8_t *sat, int32_t *n_unsat,
                         int32_t *U, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const int grid = B < 65535 * 32 ? B : 65535 * 32;
    if (f64)
        dev::check_kernel<double><<<grid, 256, 0, s>>>(V, B, static_cast<const double *>(x), sat, n_unsat, U);
    else
        dev::check_kernel<float><<<grid, 256, 0, s>>>(V, B, static_cast<const float *>(x), sat, n_unsat, U);
    return cudaGetLastError();
}

cudaError_t launch_plain64(const DevView &V, int B, const double *x, double *f, double *g, int32_t n_node,
                           const int32_t *node_ids, int32_t n_closed, const int32_t *closed_ids,
                           cudaStream_t s, int *launches) {
    int nl = 0;
    if (B > 0) {
        dev::plain64_init<<<1024, 256, 0, s>>>(B, V.n, f, g, V.f_const);
        ++nl;
        if (n_closed > 0) {
            const size_t tot = (size_t)n_closed * (size_t)B;
            dev::plain64_closed<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(V, B, x, f, g, n_closed, closed_ids);
            ++nl;
        }
        if (n_node > 0) {
            const size_t tot = (size_t)n_node * (size_t)B;
            dev::plain64_node<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(V, B, x, f, g, n_node, node_ids);
            ++nl;
        }
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace ffsat
