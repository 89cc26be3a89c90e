// Learned restart proposal: a message-passing network over the
// variable-constraint graph of an instance (no counterpart in the paper).
//
// Architecture (hidden width H = 64, L layers):
//   h_v^0 = relu(Wv0 f_v + bv0),  h_c^0 = relu(Wc0 f_c + bc0)
//   layer l:  t_v = A_l h_v^{l-1}
//             m_c = (1/|c|) sum_{(c,v)} s_cv t_v
//             h_c^l = relu(Uc_l [h_c^{l-1}; m_c] + buc_l)
//             t_c = B_l h_c^l
//             m_v = (1/deg v) sum_{(c,v)} s_cv t_c
//             h_v^l = relu(Uv_l [h_v^{l-1}; m_v] + buv_l)
//   z_v = wo . h_v^L + bo,   proposal x0_v = tanh(z_v)
// s_cv = +1 for a positive literal, -1 for a negated one.  Loss for sign targets
// t in {-1,+1}: mean_v softplus(-t_v z_v).
//
// Weights are kept in FP32 (master copy, Adam state) and used by the dense
// layers as BF16; the dense layers run on the tensor cores (tcgen05) with their
// inputs rounded to BF16 and FP32 accumulation.  Every aggregation is a
// deterministic gather over a CSR structure (constraint -> literals, or the
// transposed variable -> occurrences); only the weight-gradient reduction over
// row tiles uses FP32 atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "ffsat.h"
#include "ffsat_internal.h"
#include "fused_kernel.cuh"
#include "mpnn_tc.cuh"

namespace ffsat {
namespace mp {

constexpr int H = 64;
constexpr int FV = 8;  // variable features (padded)
constexpr int FC = 8;  // constraint features (padded)
static_assert(H % 4 == 0 && FV % 4 == 0 && FC % 4 == 0, "dense kernels move float4 groups");
constexpr uint32_t kSign = 0x80000000u;
constexpr uint32_t kIdx = 0x7fffffffu;

// ---------------------------------------------------------------------------
// Dense layers on the tensor cores (mpnn_tc.cuh): one CTA of four warps per
// 128-row tile, BF16 operands (inputs rounded to nearest even, weights stored in
// BF16), FP32 accumulation in TMEM.  Input widths K1 + K2 are multiples of 8
// (8, 64 or 128) and padded with zeros to a multiple of 16 (the K of one MMA).
//   forward:  Y = act([X1, X2] W^T + b)        A = [X1, X2] rows, B = W (H x K)
//   dX:       [dX1, dX2] = dY W                A = dY rows, B = W^T (K x H)
//   dW:       dW += dY^T [X1, X2], db += sum dY   A = [X1, X2]^T (K x rows), B = dY^T
// Each output element is one FP32 tensor-core sum over its K terms (the bias is
// added after it); dW and db add each CTA's sum with one FP32 atomic.
// ---------------------------------------------------------------------------
constexpr int TCR = tc::kRows;
constexpr int TCT = tc::kThreads;
// dynamic shared memory of every dense launch: at most four CTAs per SM, so
// that four TMEM allocations of at most 128 columns never exceed the SM's 512
constexpr size_t kDenseSmem = 56 * 1024;

__device__ __forceinline__ const float *concat_row(const float *__restrict__ X1, int K1, const float *__restrict__ X2,
                                                   int K2, int r, int k) {
    return k < K1 ? X1 + (size_t)r * K1 + k : X2 + (size_t)r * K2 + (k - K1);
}

__device__ __forceinline__ void load8(const float *p, float *v) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p + 4));
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}

// TMEM allocation and mbarrier set-up at the start of a dense kernel; the
// caller's barrier (with the tcgen05 fences) publishes both.
__device__ __forceinline__ void tc_setup(uint32_t *holder, uint64_t *bar, uint32_t ncols) {
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(holder, ncols);
    if (threadIdx.x == 0) tc::mbar_init(bar, 1);
}

// Operands staged: publish them to the tensor core and the TMEM address to all threads.
__device__ __forceinline__ uint32_t tc_publish(const uint32_t *holder) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *holder;
}

// End of a dense kernel: every TMEM read done, warp 0 frees the columns.
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t ncols) {
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, ncols);
    }
}

// One thread issues the Kp / 16 MMAs of a tile (A and B K-major, kc8 = Kp / 8
// column groups each) and commits them to bar.
__device__ __forceinline__ void tc_issue(uint32_t tmem, const unsigned char *As, const unsigned char *Bs, int kc8,
                                         int ksteps, uint32_t idesc, bool acc_first, uint64_t *bar) {
    const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs), sbo = (uint32_t)kc8 * 128u;
    for (int j = 0; j < ksteps; ++j)
        tc::mma_bf16(tmem, tc::smem_desc(a0 + 256u * j, 128u, sbo), tc::smem_desc(b0 + 256u * j, 128u, sbo), idesc,
                     acc_first || j > 0);
    tc::mma_commit(bar);
}

template <bool RELU>
__global__ void __launch_bounds__(TCT) tc_dense_fwd(const float *__restrict__ X1, int K1,
                                                    const float *__restrict__ X2, int K2,
                                                    const __nv_bfloat16 *__restrict__ W,
                                                    const float *__restrict__ b, float *__restrict__ Y, int R,
                                                    int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t holder;
    const int K = K1 + K2, Kp = (K + 15) & ~15, kc8 = Kp / 8;
    unsigned char *As = smem, *Bs = smem + (size_t)TCR * Kp * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * TCR;
    tc_setup(&holder, &bar, H);
    // A: 128 rows of [X1, X2], eight chunks per thread in flight
    for (int base = tid; base < TCR * kc8; base += 8 * TCT) {
        float v[8][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * TCT;
            const int r8 = i & 7, c = (i >> 3) % kc8, g = (i >> 3) / kc8;
            const int r = r0 + g * 8 + r8, k = c * 8;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[u][e] = 0.f;
            if (i < TCR * kc8 && r < R && k < K) load8(concat_row(X1, K1, X2, K2, r, k), v[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * TCT;
            if (i < TCR * kc8) tc::st_chunk(As, (i >> 3) / kc8, (i >> 3) % kc8, kc8, i & 7, tc::pack8(v[u]));
        }
    }
    for (int i = tid; i < H * kc8; i += TCT) {  // B: W, H rows of K
        const int n8 = i & 7, c = (i >> 3) % kc8, g = (i >> 3) / kc8;
        const int n = g * 8 + n8, k = c * 8;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (k < K) w = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)n * K + k));
        tc::st_chunk(Bs, g, c, kc8, n8, w);
    }
    const uint32_t tmem = tc_publish(&holder);
    if (tid == 0) tc_issue(tmem, As, Bs, kc8, Kp / 16, tc::idesc_bf16(TCR, H), false, &bar);
    const bool ok = tc::mbar_wait(&bar, 0);
    tc::fence_after_sync();
    const int r = r0 + warp * 32 + lane;
#pragma unroll
    for (int h = 0; h < H / 32; ++h) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 32), v);
        if (r < R) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 o;
                o.x = v[j] + (b ? __ldg(b + h * 32 + j) : 0.f);
                o.y = v[j + 1] + (b ? __ldg(b + h * 32 + j + 1) : 0.f);
                o.z = v[j + 2] + (b ? __ldg(b + h * 32 + j + 2) : 0.f);
                o.w = v[j + 3] + (b ? __ldg(b + h * 32 + j + 3) : 0.f);
                if (RELU) o = make_float4(fmaxf(o.x, 0.f), fmaxf(o.y, 0.f), fmaxf(o.z, 0.f), fmaxf(o.w, 0.f));
                if (!ok) o = make_float4(__int_as_float(0x7fc00000), o.y, o.z, o.w);
                *reinterpret_cast<float4 *>(Y + (size_t)r * H + h * 32 + j) = o;
            }
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, 1);
        (void)tc::mbar_wait(&bar, 0);
    }
    tc_teardown(tmem, H);
}

// [dX1, dX2] = dY W for one 128-row tile: N = K1 + K2 (64 or 128) TMEM columns.
__global__ void __launch_bounds__(TCT) tc_dense_bwd_x(const float *__restrict__ dY,
                                                      const __nv_bfloat16 *__restrict__ W, int K1, int K2,
                                                      float *__restrict__ dX1, float *__restrict__ dX2, int R,
                                                      int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t holder;
    constexpr int kc8 = H / 8;
    const int N = K1 + K2;
    unsigned char *As = smem, *Bs = smem + (size_t)TCR * H * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * TCR;
    tc_setup(&holder, &bar, (uint32_t)N);
    // A: 128 rows of dY, eight chunks per thread in flight
    static_assert(TCR * kc8 == 8 * TCT, "one pass of eight chunks per thread");
    {
        float v[8][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = tid + u * TCT;
            const int r8 = i & 7, c = (i >> 3) % kc8, g = (i >> 3) / kc8;
            const int r = r0 + g * 8 + r8;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[u][e] = 0.f;
            if (r < R) load8(dY + (size_t)r * H + c * 8, v[u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = tid + u * TCT;
            tc::st_chunk(As, (i >> 3) / kc8, (i >> 3) % kc8, kc8, i & 7, tc::pack8(v[u]));
        }
    }
    for (int i = tid; i < N * kc8; i += TCT) {  // B: W^T, N rows of H (a column of W each)
        const int n8 = i & 7, c = (i >> 3) % kc8, g = (i >> 3) / kc8;
        const int j = g * 8 + n8;
        uint4 w;
        uint16_t *e = reinterpret_cast<uint16_t *>(&w);
#pragma unroll
        for (int t = 0; t < 8; ++t) e[t] = __ldg(reinterpret_cast<const unsigned short *>(W) + (size_t)(c * 8 + t) * N + j);
        tc::st_chunk(Bs, g, c, kc8, n8, w);
    }
    const uint32_t tmem = tc_publish(&holder);
    if (tid == 0) tc_issue(tmem, As, Bs, kc8, H / 16, tc::idesc_bf16(TCR, N), false, &bar);
    const bool ok = tc::mbar_wait(&bar, 0);
    tc::fence_after_sync();
    const int r = r0 + warp * 32 + lane;
    for (int h = 0; h < N / 32; ++h) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 32), v);
        const int j0 = h * 32;
        float *dst = j0 < K1 ? dX1 : dX2;
        if (r < R && dst) {
            const int pitch = j0 < K1 ? K1 : K2, jj = j0 < K1 ? j0 : j0 - K1;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                if (!ok) o.x = __int_as_float(0x7fc00000);
                *reinterpret_cast<float4 *>(dst + (size_t)r * pitch + jj + j) = o;
            }
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, 1);
        (void)tc::mbar_wait(&bar, 0);
    }
    tc_teardown(tmem, (uint32_t)N);
}

// dW += dY^T [X1, X2] (dW is H x K, K = K1 + K2 <= 128) and db += sum_r dY: the
// CTA walks the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ..., adding
// D[k][o] = sum_r X[r][k] dY[r][o] (M = 128 >= K rows of the transposed input,
// N = H) in TMEM over its tiles, then adds D and its column sums of dY to dW
// and db with FP32 atomics.  Rows past K of A stay zero.
__global__ void __launch_bounds__(TCT) tc_dense_bwd_w(const float *__restrict__ dY, const float *__restrict__ X1,
                                                      int K1, const float *__restrict__ X2, int K2,
                                                      float *__restrict__ dW, float *__restrict__ db, int R,
                                                      int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t holder;
    constexpr int kc8 = TCR / 8;  // the K of these MMAs is the tile's 128 rows
    const int K = K1 + K2;
    unsigned char *As = smem, *Bs = smem + (size_t)TCR * TCR * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    tc_setup(&holder, &bar, H);
    // the zero rows k >= K of A, written once
    for (int i = tid; i < TCR * kc8; i += TCT) {
        const int k = (i >> 3) / kc8 * 8 + (i & 7);
        if (k >= K) tc::st_chunk(As, (i >> 3) / kc8, (i >> 3) % kc8, kc8, i & 7, make_uint4(0u, 0u, 0u, 0u));
    }
    // Staging: a task reads 8 consecutive rows x 4 consecutive columns (eight
    // float4 loads, the lanes of a warp covering consecutive columns of the same
    // rows) and writes the four transposed chunks (one column, 8 rows each).
    // B tasks: thread t owns columns o = 4 (t % 16) .. + 3 of dY in every tile.
    float bsum[4] = {0.f, 0.f, 0.f, 0.f};
    const int tiles = (R + TCR - 1) / TCR;
    const int K4 = K / 4;
    uint32_t tmem = 0;
    bool ok = true;
    int done = 0;
    auto stage4 = [&](unsigned char *base, const float *const *rows, int col, int kcol, int rc, float *sum) {
        float v[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (rows[t]) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(rows[t] + col));
                v[t][0] = q.x, v[t][1] = q.y, v[t][2] = q.z, v[t][3] = q.w;
            } else {
                v[t][0] = v[t][1] = v[t][2] = v[t][3] = 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float w[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) w[t] = v[t][c];
            if (sum)
#pragma unroll
                for (int t = 0; t < 8; ++t) sum[c] += w[t];
            const int k = kcol + c;
            tc::st_chunk(base, k >> 3, rc, kc8, k & 7, tc::pack8(w));
        }
    };
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++done) {
        const int r0 = tile * TCR;
        if (done > 0) ok &= tc::mbar_wait(&bar, (uint32_t)(done - 1) & 1u);  // the MMAs have read the buffers
        for (int i = tid; i < K4 * kc8; i += TCT) {  // A[k][r] = X[r][k]
            const int j = i % K4, rc = i / K4, k = 4 * j;
            const float *rows[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int r = r0 + rc * 8 + t;
                rows[t] = r < R ? (k < K1 ? X1 + (size_t)r * K1 : X2 + (size_t)r * K2) : nullptr;
            }
            stage4(As, rows, k < K1 ? k : k - K1, k, rc, nullptr);
        }
        for (int i = tid; i < (H / 4) * kc8; i += TCT) {  // B[o][r] = dY[r][o]
            const int j = i % (H / 4), rc = i / (H / 4);
            const float *rows[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int r = r0 + rc * 8 + t;
                rows[t] = r < R ? dY + (size_t)r * H : nullptr;
            }
            stage4(Bs, rows, 4 * j, 4 * j, rc, bsum);
        }
        const uint32_t t_addr = tc_publish(&holder);
        tmem = t_addr;
        if (tid == 0) tc_issue(tmem, As, Bs, kc8, TCR / 16, tc::idesc_bf16(TCR, H), done > 0, &bar);
    }
    if (done > 0) ok &= tc::mbar_wait(&bar, (uint32_t)(done - 1) & 1u);
    else tmem = tc_publish(&holder);
    tc::fence_after_sync();
    const int k = warp * 32 + lane;
    if (done > 0) {
#pragma unroll
        for (int h = 0; h < H / 32; ++h) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 32), v);
            if (k < K)
#pragma unroll
                for (int j = 0; j < 32; ++j) atomicAdd(dW + (size_t)(h * 32 + j) * K + k, ok ? v[j] : __int_as_float(0x7fc00000));
        }
    }
    if (db) {
        // lanes l and l + 16 hold the same columns: fold them, then one atomic per column
        static_assert(TCT % (H / 4) == 0 && H / 4 == 16, "thread t owns the columns 4 (t % 16) .. + 3");
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float s = bsum[c];
            s += __shfl_xor_sync(0xffffffffu, s, 16);
            if (lane < 16) atomicAdd(db + 4 * lane + c, s);
        }
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    tc_teardown(tmem, H);
}

// out[r, :] = (norm ? 1/cnt_r : 1) * sum_{e in row r} sign_e * scale[src_e] * src[src_e, :]
// (scale may be NULL).  One warp per row, two features per lane.
__global__ void gather_sum(const float *__restrict__ src, const int32_t *__restrict__ ptr,
                           const uint32_t *__restrict__ idx, const float *__restrict__ scale, int R, bool norm,
                           float *__restrict__ out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= R) return;
    const int a = ptr[warp], e = ptr[warp + 1];
    float s0 = 0.f, s1 = 0.f;
    for (int i = a; i < e; ++i) {
        const uint32_t ix = idx[i];
        const uint32_t j = ix & kIdx;
        float w = (ix & kSign) ? -1.f : 1.f;
        if (scale) w *= scale[j];
        const float2 v = reinterpret_cast<const float2 *>(src + (size_t)j * H)[lane];
        s0 = fmaf(w, v.x, s0);
        s1 = fmaf(w, v.y, s1);
    }
    const float f = (norm && e > a) ? 1.f / (float)(e - a) : 1.f;
    reinterpret_cast<float2 *>(out + (size_t)warp * H)[lane] = make_float2(s0 * f, s1 * f);
}

__global__ void relu_mask(float *__restrict__ d, const float *__restrict__ y, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        if (!(y[i] > 0.f)) d[i] = 0.f;
}

__global__ void add_inplace(float *__restrict__ a, const float *__restrict__ b, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

// z = H wo + bo, x0 = tanh z; optional loss mean softplus(-t z) and dz = -t sigmoid(-t z) / n.
__global__ void output_head(const float *__restrict__ Hv, const __nv_bfloat16 *__restrict__ wo, const float *bo,
                            int n, float *__restrict__ x0, const float *__restrict__ target, float *__restrict__ dz,
                            float *__restrict__ loss) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float2 h = reinterpret_cast<const float2 *>(Hv + (size_t)warp * H)[lane];
    float z = __bfloat162float(wo[2 * lane]) * h.x + __bfloat162float(wo[2 * lane + 1]) * h.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    z += bo[0];
    if (lane == 0) {
        if (x0) x0[warp] = tanhf(z);
        if (target) {
            const float t = target[warp];
            const float u = -t * z;
            const float sp = u > 20.f ? u : log1pf(expf(u));  // softplus(u)
            atomicAdd(loss, sp / (float)n);
            dz[warp] = -t / (1.f + expf(-u)) / (float)n;  // d softplus(u)/dz = sigmoid(u) * (-t)
        }
    }
}

// dH = dz wo^T; dwo += dz^T H; dbo += sum dz
__global__ void output_head_bwd(const float *__restrict__ Hv, const __nv_bfloat16 *__restrict__ wo,
                                const float *__restrict__ dz, int n, float *__restrict__ dH, float *__restrict__ dwo,
                                float *__restrict__ dbo) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float d = dz[warp];
    const float2 h = reinterpret_cast<const float2 *>(Hv + (size_t)warp * H)[lane];
    reinterpret_cast<float2 *>(dH + (size_t)warp * H)[lane] =
        make_float2(d * __bfloat162float(wo[2 * lane]), d * __bfloat162float(wo[2 * lane + 1]));
    atomicAdd(&dwo[2 * lane], d * h.x);
    atomicAdd(&dwo[2 * lane + 1], d * h.y);
    if (lane == 0) atomicAdd(dbo, d);
}

// Adam on the FP32 master weights; refreshes the BF16 copy.
__global__ void adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                     __nv_bfloat16 *__restrict__ pb, int count, float lr, float b1, float b2, float eps, float c1,
                     float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16(pi);
    }
}

__global__ void to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16(p[i]);
}

// Restart from a proposal: unsolved points get x = clip(p + noise * u, -1, 1),
// u uniform on [-1, 1) from the same counter-based draws as the uniform restart.
template <typename R>
__global__ void proposal_restart(R *__restrict__ x, int B, int n, const float *__restrict__ prop, float noise,
                                 const uint8_t *__restrict__ solved, uint64_t seed, uint64_t epoch,
                                 uint64_t b_offset) {
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        if (solved && solved[b]) continue;
        const uint64_t kb = dev::splitmix64(dev::splitmix64(dev::splitmix64(seed) ^ epoch) ^ (b_offset + (uint64_t)b));
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const float u = dev::restart_value<float>(kb, (uint64_t)v);
            const float z = fminf(fmaxf(prop[v] + noise * u, -1.f), 1.f);
            x[(size_t)b * n + v] = (R)z;
        }
    }
}

}  // namespace mp
}  // namespace ffsat

// ===========================================================================
// host side
// ===========================================================================

struct ffsat_mpnn {
    int device = 0;
    int L = 3;
    int n_params = 0;
    // parameter offsets (floats)
    int o_wv0, o_bv0, o_wc0, o_bc0, o_wo, o_bo;
    std::vector<int> o_A, o_Uc, o_buc, o_B, o_Uv, o_buv;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *pb = nullptr;
    int adam_t = 0;
    // activations and gradients, sized for cap_n variables and cap_m constraints
    size_t cap_n = 0, cap_m = 0;
    std::vector<float *> Hv, Hc, Mc, Mv;
    float *T1 = nullptr, *T2 = nullptr;
    float *dHv = nullptr, *dHv2 = nullptr, *dHvx = nullptr, *dMv = nullptr, *dT1 = nullptr;
    float *dHc = nullptr, *dHc2 = nullptr, *dHcx = nullptr, *dMc = nullptr, *dT2 = nullptr;
    float *dz = nullptr, *x0 = nullptr;
    int *d_err = nullptr;  // set by a dense kernel whose tensor-core wait gave up
    std::vector<void *> allocs;
};

namespace {

using namespace ffsat;
using namespace ffsat::mp;

#define MP_TRY(expr)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            std::string m_ = std::string(#expr) + ": " + cudaGetErrorString(e_);        \
            return set_error(FFSAT_ERR_CUDA, m_.c_str());                                \
        }                                                                                \
    } while (0)

uint64_t sm64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int ensure_capacity(ffsat_mpnn *M, size_t n, size_t m) {
    if (n <= M->cap_n && m <= M->cap_m) return FFSAT_OK;
    for (void *a : M->allocs) cudaFree(a);
    M->allocs.clear();
    n = std::max(n, M->cap_n);
    m = std::max(m, M->cap_m);
    auto get = [&](size_t rows, float **out) -> int {
        void *ptr = nullptr;
        MP_TRY(cudaMalloc(&ptr, std::max<size_t>(rows, 1) * H * sizeof(float)));
        M->allocs.push_back(ptr);
        *out = static_cast<float *>(ptr);
        return FFSAT_OK;
    };
    M->Hv.assign(M->L + 1, nullptr);
    M->Hc.assign(M->L + 1, nullptr);
    M->Mc.assign(M->L + 1, nullptr);
    M->Mv.assign(M->L + 1, nullptr);
    int rc = 0;
    for (int l = 0; l <= M->L; ++l) {
        if ((rc = get(n, &M->Hv[l])) || (rc = get(m, &M->Hc[l])) || (rc = get(m, &M->Mc[l])) || (rc = get(n, &M->Mv[l])))
            return rc;
    }
    float *dzx = nullptr;
    if ((rc = get(n, &M->T1)) || (rc = get(m, &M->T2)) || (rc = get(n, &M->dHv)) || (rc = get(n, &M->dHv2)) ||
        (rc = get(n, &M->dHvx)) || (rc = get(n, &M->dMv)) || (rc = get(n, &M->dT1)) || (rc = get(m, &M->dHc)) ||
        (rc = get(m, &M->dHc2)) || (rc = get(m, &M->dHcx)) || (rc = get(m, &M->dMc)) || (rc = get(m, &M->dT2)) ||
        (rc = get(n, &dzx)))
        return rc;
    M->dz = dzx;           // [n]
    M->x0 = dzx + n;       // [n] (the buffer has n * H floats)
    M->cap_n = n;
    M->cap_m = m;
    return FFSAT_OK;
}

inline unsigned blocks_for(size_t threads, unsigned per) { return (unsigned)((threads + per - 1) / per); }

// Raise the dynamic shared-memory limit of the dense kernels once per device.
void dense_smem_limits() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(mu);
    if (!done.insert(dev).second) return;
    cudaFuncSetAttribute(tc_dense_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem);
    cudaFuncSetAttribute(tc_dense_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem);
    cudaFuncSetAttribute(tc_dense_bwd_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem);
    cudaFuncSetAttribute(tc_dense_bwd_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDenseSmem);
}

void dense(cudaStream_t s, bool relu, const float *X1, int K1, const float *X2, int K2, const __nv_bfloat16 *W,
           const float *b, float *Y, int R, int *err) {
    if (R <= 0) return;
    dense_smem_limits();
    if (relu)
        tc_dense_fwd<true><<<blocks_for(R, TCR), TCT, kDenseSmem, s>>>(X1, K1, X2, K2, W, b, Y, R, err);
    else
        tc_dense_fwd<false><<<blocks_for(R, TCR), TCT, kDenseSmem, s>>>(X1, K1, X2, K2, W, b, Y, R, err);
}

void gather(cudaStream_t s, const float *src, const int32_t *ptr, const uint32_t *idx, const float *scale, int R,
            bool norm, float *out) {
    if (R <= 0) return;
    gather_sum<<<blocks_for((size_t)R * 32, 256), 256, 0, s>>>(src, ptr, idx, scale, R, norm, out);
}

int sm_count() {
    static int count = 0;
    if (!count) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            count = 1;
    }
    return count;
}

// Weight gradient: at most half the SMs' worth of CTAs, each summing its row
// tiles in TMEM, so that the FP32 atomics into dW stay few.
void dW(cudaStream_t s, const float *dY, const float *X1, int K1, const float *X2, int K2, float *gW, float *gb,
        int R, int *err) {
    if (R <= 0) return;
    dense_smem_limits();
    const unsigned grid = std::min<unsigned>(blocks_for(R, TCR), (unsigned)std::max(1, sm_count() / 2));
    tc_dense_bwd_w<<<grid, TCT, kDenseSmem, s>>>(dY, X1, K1, X2, K2, gW, gb, R, err);
}

void dX(cudaStream_t s, const float *dY, const __nv_bfloat16 *W, int K1, int K2, float *dX1, float *dX2, int R,
        int *err) {
    if (R <= 0) return;
    dense_smem_limits();
    tc_dense_bwd_x<<<blocks_for(R, TCR), TCT, kDenseSmem, s>>>(dY, W, K1, K2, dX1, dX2, R, err);
}

void mask(cudaStream_t s, float *d, const float *y, size_t count) {
    if (count) relu_mask<<<std::min<size_t>(blocks_for(count, 256), 4096), 256, 0, s>>>(d, y, count);
}

// Forward pass; with target != NULL also the loss, its gradient and the
// backward pass into M->g (zeroed first).
int run(ffsat_mpnn *M, const GraphView &G, const float *target, float *loss, float *x0_out, cudaStream_t s) {
    const int n = G.n, m = G.m, L = M->L;
    int rc = ensure_capacity(M, n, m);
    if (rc) return rc;
    const __nv_bfloat16 *P = M->pb;
    // forward
    dense(s, true, G.fv, FV, nullptr, 0, P + M->o_wv0, M->p + M->o_bv0, M->Hv[0], n, M->d_err);
    dense(s, true, G.fc, FC, nullptr, 0, P + M->o_wc0, M->p + M->o_bc0, M->Hc[0], m, M->d_err);
    for (int l = 1; l <= L; ++l) {
        dense(s, false, M->Hv[l - 1], H, nullptr, 0, P + M->o_A[l - 1], nullptr, M->T1, n, M->d_err);
        gather(s, M->T1, G.row_ptr, G.lits, nullptr, m, true, M->Mc[l]);
        dense(s, true, M->Hc[l - 1], H, M->Mc[l], H, P + M->o_Uc[l - 1], M->p + M->o_buc[l - 1], M->Hc[l], m, M->d_err);
        dense(s, false, M->Hc[l], H, nullptr, 0, P + M->o_B[l - 1], nullptr, M->T2, m, M->d_err);
        gather(s, M->T2, G.var_ptr, G.var_occ, nullptr, n, true, M->Mv[l]);
        dense(s, true, M->Hv[l - 1], H, M->Mv[l], H, P + M->o_Uv[l - 1], M->p + M->o_buv[l - 1], M->Hv[l], n, M->d_err);
    }
    float *x0 = x0_out ? x0_out : M->x0;
    if (target) MP_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
    output_head<<<blocks_for((size_t)n * 32, 256), 256, 0, s>>>(M->Hv[L], P + M->o_wo, M->p + M->o_bo, n, x0, target,
                                                                M->dz, loss);
    MP_TRY(cudaGetLastError());
    if (!target) return FFSAT_OK;
    // backward
    MP_TRY(cudaMemsetAsync(M->g, 0, (size_t)M->n_params * sizeof(float), s));
    MP_TRY(cudaMemsetAsync(M->dHc, 0, (size_t)std::max(m, 1) * H * sizeof(float), s));
    output_head_bwd<<<blocks_for((size_t)n * 32, 256), 256, 0, s>>>(M->Hv[L], P + M->o_wo, M->dz, n, M->dHv,
                                                                    M->g + M->o_wo, M->g + M->o_bo);
    float *dHv = M->dHv, *dHv2 = M->dHv2, *dHc = M->dHc, *dHc2 = M->dHc2;
    for (int l = L; l >= 1; --l) {
        // h_v^l = relu(Uv [h_v^{l-1}; m_v] + buv)
        mask(s, dHv, M->Hv[l], (size_t)n * H);
        dW(s, dHv, M->Hv[l - 1], H, M->Mv[l], H, M->g + M->o_Uv[l - 1], M->g + M->o_buv[l - 1], n, M->d_err);
        dX(s, dHv, P + M->o_Uv[l - 1], H, H, dHv2, M->dMv, n, M->d_err);
        // m_v = (1/deg v) sum s t_c  ->  dt_c = sum_{v in c} s dm_v / deg v
        gather(s, M->dMv, G.row_ptr, G.lits, G.inv_deg, m, false, M->dT2);
        // t_c = B h_c^l
        dW(s, M->dT2, M->Hc[l], H, nullptr, 0, M->g + M->o_B[l - 1], nullptr, m, M->d_err);
        dX(s, M->dT2, P + M->o_B[l - 1], H, 0, M->dHcx, nullptr, m, M->d_err);
        add_inplace<<<std::min<unsigned>(blocks_for((size_t)m * H, 256), 4096), 256, 0, s>>>(dHc, M->dHcx,
                                                                                           (size_t)m * H);
        // h_c^l = relu(Uc [h_c^{l-1}; m_c] + buc)
        mask(s, dHc, M->Hc[l], (size_t)m * H);
        dW(s, dHc, M->Hc[l - 1], H, M->Mc[l], H, M->g + M->o_Uc[l - 1], M->g + M->o_buc[l - 1], m, M->d_err);
        dX(s, dHc, P + M->o_Uc[l - 1], H, H, dHc2, M->dMc, m, M->d_err);
        // m_c = (1/|c|) sum s t_v  ->  dt_v = sum_{c ni v} s dm_c / |c|
        gather(s, M->dMc, G.var_ptr, G.var_occ, G.inv_len, n, false, M->dT1);
        // t_v = A h_v^{l-1}
        dW(s, M->dT1, M->Hv[l - 1], H, nullptr, 0, M->g + M->o_A[l - 1], nullptr, n, M->d_err);
        dX(s, M->dT1, P + M->o_A[l - 1], H, 0, M->dHvx, nullptr, n, M->d_err);
        add_inplace<<<std::min<unsigned>(blocks_for((size_t)n * H, 256), 4096), 256, 0, s>>>(dHv2, M->dHvx,
                                                                                           (size_t)n * H);
        std::swap(dHv, dHv2);
        std::swap(dHc, dHc2);
    }
    mask(s, dHv, M->Hv[0], (size_t)n * H);
    dW(s, dHv, G.fv, FV, nullptr, 0, M->g + M->o_wv0, M->g + M->o_bv0, n, M->d_err);
    mask(s, dHc, M->Hc[0], (size_t)m * H);
    dW(s, dHc, G.fc, FC, nullptr, 0, M->g + M->o_wc0, M->g + M->o_bc0, m, M->d_err);
    MP_TRY(cudaGetLastError());
    return FFSAT_OK;
}

}  // namespace

extern "C" {

int ffsat_mpnn_create(int32_t layers, uint64_t seed, ffsat_mpnn **out) {
    if (!out || layers < 1 || layers > 8) return set_error(FFSAT_ERR_ARG, "layers must be in 1..8 and out non-NULL");
    *out = nullptr;
    ffsat_mpnn *M = new ffsat_mpnn();
    M->L = layers;
    int off = 0;
    auto take = [&](int count) {
        const int o = off;
        off += count;
        return o;
    };
    M->o_wv0 = take(H * FV);
    M->o_bv0 = take(H);
    M->o_wc0 = take(H * FC);
    M->o_bc0 = take(H);
    for (int l = 0; l < layers; ++l) {
        M->o_A.push_back(take(H * H));
        M->o_Uc.push_back(take(H * 2 * H));
        M->o_buc.push_back(take(H));
        M->o_B.push_back(take(H * H));
        M->o_Uv.push_back(take(H * 2 * H));
        M->o_buv.push_back(take(H));
    }
    M->o_wo = take(H);
    M->o_bo = take(1);
    M->n_params = off;
    // the dense kernels read weight rows as 16-byte groups of eight BF16 values
    bool aligned = M->o_wv0 % 8 == 0 && M->o_wc0 % 8 == 0;
    for (int l = 0; l < layers; ++l)
        aligned = aligned && M->o_A[l] % 8 == 0 && M->o_Uc[l] % 8 == 0 && M->o_B[l] % 8 == 0 && M->o_Uv[l] % 8 == 0;
    if (!aligned) {
        delete M;
        return set_error(FFSAT_ERR_ARG, "internal: weight offsets not 16-byte aligned");
    }
    // Glorot-uniform weights from splitmix64, zero biases
    std::vector<float> hp(off, 0.f);
    uint64_t st = seed;
    auto init = [&](int o, int rows, int cols) {
        const double a = std::sqrt(6.0 / (double)(rows + cols));
        for (int i = 0; i < rows * cols; ++i) {
            const double u = (double)(sm64(st) >> 11) / 9007199254740992.0;
            hp[o + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    init(M->o_wv0, H, FV);
    init(M->o_wc0, H, FC);
    for (int l = 0; l < layers; ++l) {
        init(M->o_A[l], H, H);
        init(M->o_Uc[l], H, 2 * H);
        init(M->o_B[l], H, H);
        init(M->o_Uv[l], H, 2 * H);
    }
    init(M->o_wo, 1, H);
    cudaError_t e = cudaGetDevice(&M->device);
    if (e == cudaSuccess) e = cudaMalloc(&M->p, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->g, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->m1, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->m2, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&M->pb, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&M->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(M->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(M->p, hp.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m1, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(M->m2, 0, off * sizeof(float));
    if (e == cudaSuccess) {
        to_bf16<<<blocks_for(off, 256), 256>>>(M->p, M->pb, off);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        std::string msg = std::string("ffsat_mpnn_create: ") + cudaGetErrorString(e);
        ffsat_mpnn_free(M);
        return set_error(FFSAT_ERR_CUDA, msg.c_str());
    }
    *out = M;
    return FFSAT_OK;
}

int32_t ffsat_mpnn_num_params(const ffsat_mpnn *M) { return M ? M->n_params : 0; }

int ffsat_mpnn_get_params(const ffsat_mpnn *M, float *host) {
    if (!M || !host) return set_error(FFSAT_ERR_ARG, "NULL argument");
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(M->device));
    MP_TRY(cudaMemcpy(host, M->p, M->n_params * sizeof(float), cudaMemcpyDeviceToHost));
    return FFSAT_OK;
}

int ffsat_mpnn_set_params(ffsat_mpnn *M, const float *host) {
    if (!M || !host) return set_error(FFSAT_ERR_ARG, "NULL argument");
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(M->device));
    MP_TRY(cudaMemcpy(M->p, host, M->n_params * sizeof(float), cudaMemcpyHostToDevice));
    to_bf16<<<blocks_for(M->n_params, 256), 256>>>(M->p, M->pb, M->n_params);
    MP_TRY(cudaDeviceSynchronize());
    return FFSAT_OK;
}

int ffsat_mpnn_forward(ffsat_mpnn *M, ffsat_instance *inst, float *x0, void *stream) {
    if (!M || !inst || !x0) return set_error(FFSAT_ERR_ARG, "NULL argument");
    GraphView G;
    int rc = instance_graph(inst, &G);
    if (rc) return rc;
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(M->device));
    return run(M, G, nullptr, nullptr, x0, static_cast<cudaStream_t>(stream));
}

int ffsat_mpnn_loss_grad(ffsat_mpnn *M, ffsat_instance *inst, const float *target, float *loss, float *x0,
                         float *grad_host, void *stream) {
    if (!M || !inst || !target || !loss) return set_error(FFSAT_ERR_ARG, "NULL argument");
    GraphView G;
    int rc = instance_graph(inst, &G);
    if (rc) return rc;
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(M->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = run(M, G, target, loss, x0, s);
    if (rc) return rc;
    if (grad_host) {
        MP_TRY(cudaMemcpyAsync(grad_host, M->g, M->n_params * sizeof(float), cudaMemcpyDeviceToHost, s));
        MP_TRY(cudaStreamSynchronize(s));
    }
    return FFSAT_OK;
}

int ffsat_mpnn_adam_step(ffsat_mpnn *M, float lr, void *stream) {
    if (!M || !(lr >= 0.f)) return set_error(FFSAT_ERR_ARG, "bad argument");
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(M->device));
    M->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->adam_t), c2 = 1.f - std::pow(b2, (float)M->adam_t);
    adam<<<blocks_for(M->n_params, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        M->p, M->g, M->m1, M->m2, M->pb, M->n_params, lr, b1, b2, 1e-8f, c1, c2);
    MP_TRY(cudaGetLastError());
    return FFSAT_OK;
}

int ffsat_restart_from_proposal(ffsat_instance *inst, int32_t B, void *x, int32_t dtype, const float *proposal,
                                float noise, const uint8_t *solved, uint64_t seed, uint64_t epoch, uint64_t b_offset,
                                void *stream) {
    if (!inst || (B > 0 && (!x || !proposal))) return set_error(FFSAT_ERR_ARG, "NULL argument");
    if (B < 0 || !(noise >= 0.f)) return set_error(FFSAT_ERR_ARG, "B >= 0 and noise >= 0 required");
    if (dtype != FFSAT_F32 && dtype != FFSAT_F64) return set_error(FFSAT_ERR_ARG, "bad dtype");
    if (B == 0) return FFSAT_OK;
    ffsat_info info;
    int rc = ffsat_instance_info(inst, &info);
    if (rc) return rc;
    GraphView G;
    rc = instance_graph(inst, &G);
    if (rc) return rc;
    ffsat::DeviceGuard dev_guard;
    MP_TRY(dev_guard.set(G.device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)std::min(B, 65535 * 16);
    if (dtype == FFSAT_F32)
        proposal_restart<float><<<grid, 256, 0, s>>>(static_cast<float *>(x), B, info.n, proposal, noise, solved, seed,
                                                      epoch, b_offset);
    else
        proposal_restart<double><<<grid, 256, 0, s>>>(static_cast<double *>(x), B, info.n, proposal, noise, solved,
                                                       seed, epoch, b_offset);
    MP_TRY(cudaGetLastError());
    return FFSAT_OK;
}

void ffsat_mpnn_free(ffsat_mpnn *M) {
    if (!M) return;
    ffsat::DeviceGuard dev_guard;
    dev_guard.set(M->device);
    for (void *a : M->allocs) cudaFree(a);
    if (M->p) cudaFree(M->p);
    if (M->g) cudaFree(M->g);
    if (M->m1) cudaFree(M->m1);
    if (M->m2) cudaFree(M->m2);
    if (M->pb) cudaFree(M->pb);
    if (M->d_err) cudaFree(M->d_err);
    delete M;
}

}  // extern "C"
