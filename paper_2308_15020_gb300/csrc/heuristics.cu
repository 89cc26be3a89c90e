// Restart heuristics of the continuous local search: the ERWA update of the
// constraint weights (Sec. 5, Prop. "Adaptive weight") and the rephasing of
// restart points (Sec. 5, "Rephasing Heuristics": original, flipped or random
// phase).  The unsatisfaction counts U_c come from the exact checker (the
// check kernel, or the check that ends a fused step), which adds one per point
// that violates c.
#include <algorithm>

#include "fused_kernel.cuh"
#include "heuristics.h"

namespace ffsat {
namespace dev {

__global__ void umax_kernel(const int32_t *__restrict__ U, int m, int32_t *umax) {
    int best = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) best = max(best, U[c]);
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(umax, best);
}

// w_c <- (1 - alpha) w_c + alpha r_c with r_c = U_c / max U (0 when no point
// violates anything), written to every device copy of the weight.  Rounded
// operation by operation (no contraction), as the FP64 reference does.
__global__ void erwa_kernel(const WeightSites W, const int32_t *__restrict__ U, const int32_t *umax, double alpha) {
    const int32_t um = *umax;
    const double keep = __dadd_rn(1.0, -alpha);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W.m; c += gridDim.x * blockDim.x) {
        const double r = um > 0 ? __ddiv_rn((double)max(U[c], 0), (double)um) : 0.0;
        const double w = __dadd_rn(__dmul_rn(keep, W.cons_wd[c]), __dmul_rn(alpha, r));
        W.cons_wd[c] = w;
        const int s = W.slot[c];
        const int wbits = __float_as_int((float)w);
        if (W.cls[c] == 0 || W.cls[c] == 4) {
            W.clause_wd[s] = w;
            for (int k = 0; k < W.n_images; ++k) W.clauses[k][s].w = wbits;
        } else if (W.cls[c] == 1 || W.cls[c] == 2) {
            W.seg_wd[s] = w;
            for (int k = 0; k < W.n_images; ++k) W.segmeta[k][s].w = wbits;
        }
    }
}

// Constants of f under the current weights, summed in a fixed order by one CTA:
// f_const[0] = sum over clauses of -w (the fused kernel accumulates 2 w prod q)
// plus sum over constant constraints of w FE; f_const[1] = the latter alone.
__global__ void __launch_bounds__(512) f_const_kernel(const WeightSites W, double *f_const) {
    __shared__ double s_red[32];
    double a = 0.0, b = 0.0;
    for (int c = threadIdx.x; c < W.m; c += blockDim.x) {
        const int k = W.cls[c];
        const double w = W.cons_wd[c];
        if (k == 0) {
            a -= w;
        } else if (k == 3) {
            const int L = W.row_ptr[c + 1] - W.row_ptr[c];
            const double fe = W.param[c] <= 0 ? -1.0 : (W.param[c] > L ? 1.0 : 0.0);
            a += w * fe;
            b += w * fe;
        }
    }
    const double ta = block_sum(a, s_red);
    const double tb = block_sum(b, s_red);
    if (threadIdx.x == 0) {
        f_const[0] = ta;
        f_const[1] = tb;
    }
}

// Rephasing of every point b with solved[b] == 0 (all points if solved is
// NULL): phase 0 keeps x (original), 1 negates it (flipped), 2 draws it
// uniformly from [-1, 1)^n with the restart generator keyed by (seed, epoch,
// b_offset + b) (random).
// With epoch_dev set, the epoch is read from device memory (a counter that a
// captured CUDA graph advances between replays).
template <typename R>
__global__ void rephase_kernel(R *__restrict__ x, int B, int n, int phase, const uint8_t *__restrict__ solved,
                               uint64_t seed, uint64_t epoch, uint64_t b_offset, const uint64_t *epoch_dev) {
    if (epoch_dev) epoch = *epoch_dev;
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        if (solved && solved[b]) continue;
        R *xb = x + (size_t)b * (size_t)n;
        if (phase == 1) {
            for (int v = threadIdx.x; v < n; v += blockDim.x) xb[v] = -xb[v];
        } else {
            const uint64_t kb = splitmix64(splitmix64(splitmix64(seed) ^ epoch) ^ (b_offset + (uint64_t)b));
            for (int v = threadIdx.x; v < n; v += blockDim.x) xb[v] = restart_value<R>(kb, (uint64_t)v);
        }
    }
}

}  // namespace dev

cudaError_t launch_erwa(const WeightSites &W, const int32_t *U, int32_t *umax, double alpha, double *f_const,
                        cudaStream_t s, int *launches) {
    int nl = 0;
    cudaError_t e = cudaMemsetAsync(umax, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (W.m > 0) {
        const int blocks = std::min((W.m + 255) / 256, 2048);
        dev::umax_kernel<<<blocks, 256, 0, s>>>(U, W.m, umax);
        dev::erwa_kernel<<<blocks, 256, 0, s>>>(W, U, umax, alpha);
        dev::f_const_kernel<<<1, 512, 0, s>>>(W, f_const);
        nl = 3;
    }
    if (launches) *launches = nl;
    return cudaGetLastError();
}

cudaError_t launch_rephase(bool f64, void *x, int B, int n, int phase, const uint8_t *solved, uint64_t seed,
                           uint64_t epoch, uint64_t b_offset, const uint64_t *epoch_dev, cudaStream_t s,
                           int *launches) {
    if (launches) *launches = 0;
    if (B <= 0 || phase == 0) return cudaSuccess;
    const int grid = std::min(B, 1 << 20);
    if (f64)
        dev::rephase_kernel<double><<<grid, 256, 0, s>>>(static_cast<double *>(x), B, n, phase, solved, seed, epoch,
                                                         b_offset, epoch_dev);
    else
        dev::rephase_kernel<float><<<grid, 256, 0, s>>>(static_cast<float *>(x), B, n, phase, solved, seed, epoch,
                                                        b_offset, epoch_dev);
    if (launches) *launches = 1;
    return cudaGetLastError();
}

}  // namespace ffsat
