// FP64 projected-GD step with one thread-block cluster per point.
//
// GB300 executes FP64 far below its FP32 rate, so an FP64 step whose points
// occupy only a few SMs is bound by the FP64 pipes of those SMs.  This kernel
// gives each point a cluster of CL CTAs on CL SMs (CL = 2, 4 or 8):
//
//   * every CTA holds the point's x in its shared memory and evaluates the warp
//     tasks r, r + CL, r + 2 CL, ... (r = its rank in the cluster) into its own
//     gradient buffer: clause and node contributions in fixed point (Fix64Acc:
//     two native 32-bit shared-memory reductions each, no compare-and-swap
//     loops), product contributions in an FP64 word per variable (atomicAdd);
//   * the cluster barrier (release / acquire) makes the CL partial gradients
//     visible to the whole cluster;
//   * every CTA sums the CL partials of each variable through distributed
//     shared memory and takes the same step x <- clip(x - lr g, -1, 1) on its
//     own copy, so the copies stay identical.  Integer sums do not depend on
//     the order of the additions: without product constraints the step is
//     bit-reproducible.
//
// Two gradient buffers alternate between iterations: the buffer a CTA clears
// after the barrier of iteration k was last read by its peers before that
// barrier, so one cluster barrier per iteration suffices.  After the last
// iteration a final cluster barrier ends all remote reads; rank 0 alone then
// runs the exact check, the violation counts, the restart and the write-back.
// Fixed-step mode only (the line search needs F on every trial).
#pragma once
#include "fused_launch.cuh"

namespace ffsat {
namespace dev {

__device__ __forceinline__ int cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_index() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return (int)r;
}

// Every thread of every CTA of the cluster; shared-memory writes before it are
// visible to distributed shared-memory reads after it.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Element v of the shared array `local` as held by CTA `rank` of the cluster.
__device__ __forceinline__ double ld_peer(const double *local, int v, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local + v);
    uint32_t ra;
    double x;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(x) : "r"(ra) : "memory");
    return x;
}
__device__ __forceinline__ uint2 ld_peer(const uint2 *local, int v, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local + v);
    uint32_t ra;
    uint2 x;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(x.x), "=r"(x.y) : "r"(ra) : "memory");
    return x;
}

// Clause task of the cluster step (clause3 path, see clause_task): the weight
// is scaled by 2^S64 once, and the last multiplication of every contribution
// is the fixed-point rounding FMA, so a contribution costs no FP64 operation
// beyond its own product.  Negated literals flip the sign of the first factor.
template <int CPL, bool XOR>
__device__ __forceinline__ void clause_task_fix(const DevView &V, const Src &S, int4 task, int lane,
                                                const double *xrow, const Fix64Acc &acc) {
    constexpr double M = Fix64Acc::kRound;
    const int n = V.n;
    int4 cl[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) cl[k] = S.clauses[task.y + k * 32 + lane];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const double ws = __ldg(&V.clause_wd[task.y + k * 32 + lane]) * acc.s;
        const uint32_t l0 = (uint32_t)cl[k].x, l1 = (uint32_t)cl[k].y, l2 = (uint32_t)cl[k].z;
        const double y0 = gather<double, SMEM_FULL>(xrow, l0, n);
        const double y1 = gather<double, SMEM_FULL>(xrow, l1, n);
        const double y2 = gather<double, SMEM_FULL>(xrow, l2, n);
        double m0, m1, m2;
        if constexpr (XOR) {  // FE = w y0 y1 y2 (one of them the dummy)
            const double wy2 = ws * y2;
            m0 = fma(flip(wy2, l0), y1, M);
            m1 = fma(flip(wy2, l1), y0, M);
            m2 = fma(flip(ws, l2), y0 * y1, M);
        } else {  // FE = 2 w q0 q1 q2 - w, q = (1 + y) / 2
            const double q0 = 0.5 + 0.5 * y0;
            const double q1 = 0.5 + 0.5 * y1;
            const double q2 = 0.5 + 0.5 * y2;
            const double wq0 = ws * q0;
            m0 = fma(flip(ws, l0), q1 * q2, M);
            m1 = fma(flip(wq0, l1), q2, M);
            m2 = fma(flip(wq0, l2), q1, M);
        }
        // padding literals add into the words of the dummy variables n and n + 1
        // (both buffers hold npad >= n + 2 words; those words are never read)
        acc.put(l0 & kVarMask, m0);
        acc.put(l1 & kVarMask, m1);
        acc.put(l2 & kVarMask, m2);
    }
}

// One warp task of the cluster step.
template <typename R, int NR, int NI, int XG>
__device__ __forceinline__ void cluster_task(const DevView &V, const Src &S, int4 task, int lane, const R *xrow,
                                             const Fix64Acc &G) {
    constexpr bool SF = false;  // FP64 node factors are recomputed in the prefix pass
    R facc = R(0);              // the objective is not needed by a fixed-step call
    const int kind = task.x & 0xff;
    const bool xr = kind == TASK_XOR2;
    if (kind == TASK_CLAUSE || xr) {
        if (task.z == 128) {
            if (xr) clause_task_fix<4, true>(V, S, task, lane, xrow, G);
            else clause_task_fix<4, false>(V, S, task, lane, xrow, G);
        } else if (task.z == 64) {
            if (xr) clause_task_fix<2, true>(V, S, task, lane, xrow, G);
            else clause_task_fix<2, false>(V, S, task, lane, xrow, G);
        } else {
            if (xr) clause_task_fix<1, true>(V, S, task, lane, xrow, G);
            else clause_task_fix<1, false>(V, S, task, lane, xrow, G);
        }
    } else if (kind == TASK_PROD) {
        prod_task<R, XG>(V, S, task, lane, xrow, G, true, facc);
    } else {
        node_dispatch<R, NR, NI, SF, XG>(V, S, task, lane, xrow, G, true, facc);
    }
}

// The warp tasks t with t mod CL = rank into G.  At most one task per warp:
// warp w takes local task w (no counter).  Otherwise the tasks are pulled in
// order from the CTA's counter, which is never reset: every warp pulls until
// its first pull past this CTA's n_local tasks, so an iteration makes exactly
// n_local + (warps per CTA) pulls and iteration `it` owns the pulls from
// it * (n_local + warps) on.  The caller separates iterations by barriers (the
// cluster barrier after the evaluation, a CTA barrier after the update) and
// zeroes the counter before the first.
template <typename R, int NR, int NI, int XG>
__device__ __forceinline__ void eval_tasks_strided(const DevView &V, const Src &S, const R *xrow, const Fix64Acc &G,
                                                   int &s_ctr, int rank, int CL, int it) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)(blockDim.x >> 5);
    const int n_local = (V.n_task - rank + CL - 1) / CL;
    if (n_local <= warps) {
        const int tl = (int)(threadIdx.x >> 5);
        if (tl < n_local) cluster_task<R, NR, NI, XG>(V, S, S.tasks[tl * CL + rank], lane, xrow, G);
        return;
    }
    // unsigned: the counter and the base wrap together for any T
    const unsigned base = (unsigned)it * (unsigned)(n_local + warps);
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(reinterpret_cast<unsigned *>(&s_ctr), 1u);
        const int tl = (int)(__shfl_sync(kFull, t, 0) - base);
        if (tl >= n_local) break;
        cluster_task<R, NR, NI, XG>(V, S, S.tasks[tl * CL + rank], lane, xrow, G);
    }
}

// Shared memory: x | gradient buffer 0 | resident image (SMEM_RES) as in the
// one-CTA kernel, and gradient buffer 1 at byte offset g1_off.
template <typename R, int NR, int NI, int SM, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) fused_cluster_kernel(const DevView V, const FusedArgs A,
                                                                   unsigned g1_off) {
    static_assert(sizeof(R) == 8 && (SM == SMEM_FULL || SM == SMEM_RES), "FP64, x and gradient in shared memory");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockShared sh;
    const Src S = make_src<R, SM, THREADS>(V, smem_raw, true);
    const int CL = cluster_count(), rank = cluster_rank(), b = cluster_index();
    if (b >= A.B) return;  // the whole cluster leaves together
    const int n = V.n;
    const int npad = (n + 2 + 3) & ~3;
    const int tid = threadIdx.x;
    R *xs = reinterpret_cast<R *>(smem_raw);
    using U = uint2;
    // fixed-point words, then the FP64 product words (Fix64Acc::addf)
    U *const g0 = reinterpret_cast<U *>(xs + npad);
    U *const g1 = reinterpret_cast<U *>(smem_raw + g1_off);
    R *const gf0 = reinterpret_cast<R *>(g0 + npad);
    R *const gf1 = reinterpret_cast<R *>(g1 + npad);
    const bool prods = V.has_prod != 0;  // only product tasks add to the FP64 words
    const R *x_in = static_cast<const R *>(A.x_in);
    R *x_out = static_cast<R *>(A.x_out);
    const size_t rowoff = (size_t)b * (size_t)n;
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
    if (bad && rank == 0) atomicOr(V.status, STATUS_NAN);
    for (int v = tid; v < npad; v += THREADS) {
        g0[v] = make_uint2(0u, 0u);
        g1[v] = make_uint2(0u, 0u);
        gf0[v] = R(0);
        gf1[v] = R(0);
    }
    if (tid == 0) sh.ctr = 0;
    __syncthreads();
    // x - lr g with g = (hi 2^L + lo) 2^-S64: lr 2^-S64 is exact (a power-of-two scaling)
    const R lrs = R(A.sp.lr) * V.fix64_i;
    const int fl = V.fix64_l;
    Fix64Acc G;
    G.s = V.fix64_s;
    G.inv = V.fix64_i;
    G.l = fl;
    for (int it = 0; it < A.sp.T; ++it) {
        U *const gw = (it & 1) ? g1 : g0;
        U *const gz = (it & 1) ? g0 : g1;
        R *const gfw = (it & 1) ? gf1 : gf0;
        R *const gfz = (it & 1) ? gf0 : gf1;
        G.g = gw;
        G.gf = gfw;
        eval_tasks_strided<R, NR, NI, SMEM_FULL>(V, S, xs, G, sh.ctr, rank, CL, it);
        cluster_barrier();  // also ends the evaluation of this CTA's warps
        for (int v = tid; v < n; v += THREADS) {
            long long hs = 0;
            unsigned long long ls = 0;
            for (int q = 0; q < CL; ++q) {
                const uint2 p = ld_peer(gw, v, q);
                ls += p.x;
                hs += (int)p.y;
            }
            const long long gi = (long long)((unsigned long long)hs << fl) + (long long)ls;
            R z = fma(-lrs, R(gi), xs[v]);
            if (prods) {  // the same for every thread
                R gp = ld_peer(gfw, v, 0);
                for (int q = 1; q < CL; ++q) gp += ld_peer(gfw, v, q);
                z = fma(-R(A.sp.lr), gp, z);
                gfz[v] = R(0);
            }
            // clip to [-1, 1] on the integer pipes: |z| > 1 becomes sign(z) 1
            long long zb = __double_as_longlong(z);
            if ((zb & 0x7fffffffffffffffll) > 0x3ff0000000000000ll) zb = (zb & (long long)0x8000000000000000ull) | 0x3ff0000000000000ll;
            xs[v] = __longlong_as_double(zb);
            gz[v] = make_uint2(0u, 0u);
        }
        __syncthreads();  // x and the cleared buffer before the next evaluation
    }
    cluster_barrier();  // no peer reads this CTA's buffers after this point
    if (rank != 0) return;
    __syncthreads();
    const int unsat = block_unsat<R>(V, xs, sh.ired, A.unsat_counts);
    if (tid == 0) sh.ired[0] = unsat;
    __syncthreads();
    const int u = sh.ired[0];
    if (tid == 0) {
        if (A.solved) A.solved[b] = (uint8_t)(u == 0);
        if (A.n_unsat) A.n_unsat[b] = u;
    }
    if (u != 0 && A.sp.restart) {
        const uint64_t kb = splitmix64(splitmix64(splitmix64(A.sp.seed) ^ A.sp.epoch) ^ (A.sp.b_offset + (uint64_t)b));
        for (int v = tid; v < n; v += THREADS) xs[v] = restart_value<R>(kb, (uint64_t)v);
    }
    for (int v = tid; v < n; v += THREADS) x_out[rowoff + v] = xs[v];
}

template <typename R, int NR, int SM>
cudaError_t cluster_launch_mode(const DevView &V, const FusedArgs &a, size_t smem, size_t g1_off, int B, int CL,
                                cudaStream_t s, int *max_active) {
    constexpr int TH = fused_threads(true, NR);
    auto k = fused_cluster_kernel<R, NR, node_interleave<R, NR>(), SM, TH>;
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)B * (unsigned)CL);
    cfg.blockDim = dim3(TH);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (max_active) return cudaOccupancyMaxActiveClusters(max_active, k, &cfg);
    e = cudaLaunchKernelEx(&cfg, k, V, a, (unsigned)g1_off);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename R, int NR>
cudaError_t cluster_launch(const DevView &V, int smem_mode, const FusedArgs &a, size_t smem, size_t g1_off, int B,
                           int CL, cudaStream_t s, int *max_active) {
    if (smem_mode == SMEM_RES) return cluster_launch_mode<R, NR, SMEM_RES>(V, a, smem, g1_off, B, CL, s, max_active);
    return cluster_launch_mode<R, NR, SMEM_FULL>(V, a, smem, g1_off, B, CL, s, max_active);
}

}  // namespace dev
}  // namespace ffsat

#define FFSAT_DEFINE_CLUSTER(name, NR)                                                                       \
    namespace ffsat {                                                                                        \
    FFSAT_CLUSTER_LAUNCHER(name) { return dev::cluster_launch<double, NR>(V, smem_mode, a, smem, g1_off, B, CL, s, max_active); } \
    }
