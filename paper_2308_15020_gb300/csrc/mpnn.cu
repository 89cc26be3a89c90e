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
// Weights are kept in FP32 (master copy, Adam state) and used by the forward and
// backward kernels as BF16, with FP32 accumulation.  Every aggregation is a
// deterministic gather over a CSR structure (constraint -> literals, or the
// transposed variable -> occurrences); only the weight-gradient reduction over
// rows uses FP32 atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ffsat.h"
#include "ffsat_internal.h"
#include "fused_kernel.cuh"

namespace ffsat {
namespace mp {

constexpr int H = 64;
constexpr int FV = 8;  // variable features (padded)
constexpr int FC = 8;  // constraint features (padded)
static_assert(H % 4 == 0 && FV % 4 == 0 && FC % 4 == 0, "dense kernels move float4 groups");
constexpr uint32_t kSign = 0x80000000u;
constexpr uint32_t kIdx = 0x7fffffffu;

// ---------------------------------------------------------------------------
// dense layer: Y[r, :] = act(W [X1[r, :]; X2[r, :]] + b), W is N x (K1 + K2), N = H.
// Register-tiled FP32 SIMT GEMMs: a CTA owns TR rows, each thread a 4 x 4 block of
// the output; operands are staged in shared memory in 64-column chunks of the
// concatenated input, W transposed to [k][o] so that lanes read consecutive
// banks.  K1 and K2 are multiples of 4, K1 + K2 <= 2H.  Every output element
// sums its terms in the order bias, k = 0 .. K-1 (fwd) and o = 0 .. H-1 (dX).
// ---------------------------------------------------------------------------
constexpr int TR = 32;       // rows per CTA tile
constexpr int KC = 64;       // input columns per shared-memory chunk
constexpr int XP = KC + 4;   // padded row pitch of the staged inputs (keeps float4 alignment)
constexpr int FWD_THREADS = (TR / 4) * (H / 4);  // 128

__device__ __forceinline__ float concat_at(const float *__restrict__ X1, int K1, const float *__restrict__ X2, int K2,
                                           int r, int k) {
    return k < K1 ? X1[(size_t)r * K1 + k] : X2[(size_t)r * K2 + (k - K1)];
}

template <bool RELU>
__global__ void __launch_bounds__(FWD_THREADS) dense_fwd(const float *__restrict__ X1, int K1,
                                                         const float *__restrict__ X2, int K2,
                                                         const __nv_bfloat16 *__restrict__ W,
                                                         const float *__restrict__ b, float *__restrict__ Y, int R) {
    __shared__ __align__(16) float wt[KC][H];  // wt[k][o] = W[o][c0 + k]
    __shared__ __align__(16) float xs[TR][XP];
    const int K = K1 + K2;
    const int t = threadIdx.x, tx = t % (H / 4), ty = t / (H / 4);
    const int r0 = blockIdx.x * TR;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float bj = b ? b[tx * 4 + j] : 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
    for (int c0 = 0; c0 < K; c0 += KC) {
        const int kc = min(KC, K - c0);  // a multiple of 4
        __syncthreads();
        for (int i = t; i < H * kc; i += FWD_THREADS) {
            const int o = i % H, k = i / H;
            wt[k][o] = __bfloat162float(W[(size_t)o * K + c0 + k]);
        }
        for (int i = t; i < TR * kc; i += FWD_THREADS) {
            const int rr = i / kc, k = i % kc, r = r0 + rr;
            xs[rr][k] = r < R ? concat_at(X1, K1, X2, K2, r, c0 + k) : 0.f;
        }
        __syncthreads();
        for (int k = 0; k < kc; k += 4) {
            float4 xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) xv[i] = *reinterpret_cast<const float4 *>(&xs[ty * 4 + i][k]);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float4 wv = *reinterpret_cast<const float4 *>(&wt[k + kk][tx * 4]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float xi = kk == 0 ? xv[i].x : kk == 1 ? xv[i].y : kk == 2 ? xv[i].z : xv[i].w;
                    acc[i][0] = fmaf(wv.x, xi, acc[i][0]);
                    acc[i][1] = fmaf(wv.y, xi, acc[i][1]);
                    acc[i][2] = fmaf(wv.z, xi, acc[i][2]);
                    acc[i][3] = fmaf(wv.w, xi, acc[i][3]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= R) break;
        float4 v = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        if (RELU) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
        *reinterpret_cast<float4 *>(Y + (size_t)r * H + tx * 4) = v;
    }
}

// dX = dY W, split into the two input blocks; dY already includes the activation
// mask.  K = K1 + K2 in {4, 8, .., 2H}; the CTA has (K / 4) * (TR / 4) threads.
__global__ void __launch_bounds__(2 * H / 4 * (TR / 4)) dense_bwd_x(const float *__restrict__ dY,
                                                                   const __nv_bfloat16 *__restrict__ W, int K1, int K2,
                                                                   float *__restrict__ dX1, float *__restrict__ dX2,
                                                                   int R) {
    __shared__ __align__(16) float ws[H][2 * H];  // ws[o][k] = W[o][k]
    __shared__ __align__(16) float ds[TR][H + 4];
    const int K = K1 + K2, K4 = K / 4, nt = K4 * (TR / 4);
    const int t = threadIdx.x, tx = t % K4, ty = t / K4;
    const int r0 = blockIdx.x * TR;
    for (int i = t; i < H * K; i += nt) ws[i / K][i % K] = __bfloat162float(W[i]);
    for (int i = t; i < TR * H; i += nt) {
        const int rr = i / H, o = i % H, r = r0 + rr;
        ds[rr][o] = r < R ? dY[(size_t)r * H + o] : 0.f;
    }
    __syncthreads();
    float acc[4][4] = {};
    for (int o = 0; o < H; o += 4) {
        float4 dv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) dv[i] = *reinterpret_cast<const float4 *>(&ds[ty * 4 + i][o]);
#pragma unroll
        for (int oo = 0; oo < 4; ++oo) {
            const float4 wv = *reinterpret_cast<const float4 *>(&ws[o + oo][tx * 4]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float di = oo == 0 ? dv[i].x : oo == 1 ? dv[i].y : oo == 2 ? dv[i].z : dv[i].w;
                acc[i][0] = fmaf(di, wv.x, acc[i][0]);
                acc[i][1] = fmaf(di, wv.y, acc[i][1]);
                acc[i][2] = fmaf(di, wv.z, acc[i][2]);
                acc[i][3] = fmaf(di, wv.w, acc[i][3]);
            }
        }
    }
    const int k = tx * 4;
    float *dst = k < K1 ? dX1 : dX2;
    if (!dst) return;
    const int pitch = k < K1 ? K1 : K2, kk = k < K1 ? k : k - K1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= R) break;
        *reinterpret_cast<float4 *>(dst + (size_t)r * pitch + kk) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
}

// dW += dY^T [X1, X2], db += sum_r dY.  A grid of at most a few CTAs per SM walks
// the TR-row tiles; each thread keeps the 4 x 4 blocks (o, k) it owns in registers
// across tiles and adds them to dW with one FP32 atomic per element at the end.
constexpr int BW_THREADS = 256;
template <int NB>  // 4 x 4 blocks per thread: 16 * K / 4 <= NB * BW_THREADS
__global__ void __launch_bounds__(BW_THREADS) dense_bwd_w(const float *__restrict__ dY, const float *__restrict__ X1,
                                                          int K1, const float *__restrict__ X2, int K2,
                                                          float *__restrict__ dW, float *__restrict__ db, int R) {
    __shared__ __align__(16) float ds[TR][H];
    __shared__ __align__(16) float xs[TR][2 * H];
    const int K = K1 + K2, K4 = K / 4, nblk = (H / 4) * K4;
    const int t = threadIdx.x;
    float acc[NB][4][4] = {};
    float bacc = 0.f;
    const int tiles = (R + TR - 1) / TR;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int r0 = tile * TR;
        __syncthreads();
        for (int i = t; i < TR * H; i += BW_THREADS) {
            const int rr = i / H, o = i % H, r = r0 + rr;
            ds[rr][o] = r < R ? dY[(size_t)r * H + o] : 0.f;
        }
        for (int i = t; i < TR * K; i += BW_THREADS) {
            const int rr = i / K, k = i % K, r = r0 + rr;
            xs[rr][k] = r < R ? concat_at(X1, K1, X2, K2, r, k) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int blk = t + q * BW_THREADS;
            if (blk >= nblk) break;
            const int o = (blk / K4) * 4, k = (blk % K4) * 4;
            for (int rr = 0; rr < TR; ++rr) {
                const float4 dv = *reinterpret_cast<const float4 *>(&ds[rr][o]);
                const float4 xv = *reinterpret_cast<const float4 *>(&xs[rr][k]);
                const float d[4] = {dv.x, dv.y, dv.z, dv.w}, x[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][a][c] = fmaf(d[a], x[c], acc[q][a][c]);
            }
        }
        if (db && t < H)
            for (int rr = 0; rr < TR; ++rr) bacc += ds[rr][t];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int blk = t + q * BW_THREADS;
        if (blk >= nblk) break;
        const int o = (blk / K4) * 4, k = (blk % K4) * 4;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) atomicAdd(&dW[(size_t)(o + a) * K + k + c], acc[q][a][c]);
    }
    if (db && t < H) atomicAdd(&db[t], bacc);
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

void dense(cudaStream_t s, bool relu, const float *X1, int K1, const float *X2, int K2, const __nv_bfloat16 *W,
           const float *b, float *Y, int R) {
    if (R <= 0) return;
    if (relu)
        dense_fwd<true><<<blocks_for(R, TR), FWD_THREADS, 0, s>>>(X1, K1, X2, K2, W, b, Y, R);
    else
        dense_fwd<false><<<blocks_for(R, TR), FWD_THREADS, 0, s>>>(X1, K1, X2, K2, W, b, Y, R);
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

void dW(cudaStream_t s, const float *dY, const float *X1, int K1, const float *X2, int K2, float *gW, float *gb,
        int R) {
    if (R <= 0) return;
    const unsigned grid = std::min<unsigned>(blocks_for(R, TR), (unsigned)sm_count());
    if (4 * (K1 + K2) <= BW_THREADS)
        dense_bwd_w<1><<<grid, BW_THREADS, 0, s>>>(dY, X1, K1, X2, K2, gW, gb, R);
    else
        dense_bwd_w<2><<<grid, BW_THREADS, 0, s>>>(dY, X1, K1, X2, K2, gW, gb, R);
}

void dX(cudaStream_t s, const float *dY, const __nv_bfloat16 *W, int K1, int K2, float *dX1, float *dX2, int R) {
    if (R <= 0) return;
    dense_bwd_x<<<blocks_for(R, TR), (K1 + K2) / 4 * (TR / 4), 0, s>>>(dY, W, K1, K2, dX1, dX2, R);
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
    dense(s, true, G.fv, FV, nullptr, 0, P + M->o_wv0, M->p + M->o_bv0, M->Hv[0], n);
    dense(s, true, G.fc, FC, nullptr, 0, P + M->o_wc0, M->p + M->o_bc0, M->Hc[0], m);
    for (int l = 1; l <= L; ++l) {
        dense(s, false, M->Hv[l - 1], H, nullptr, 0, P + M->o_A[l - 1], nullptr, M->T1, n);
        gather(s, M->T1, G.row_ptr, G.lits, nullptr, m, true, M->Mc[l]);
        dense(s, true, M->Hc[l - 1], H, M->Mc[l], H, P + M->o_Uc[l - 1], M->p + M->o_buc[l - 1], M->Hc[l], m);
        dense(s, false, M->Hc[l], H, nullptr, 0, P + M->o_B[l - 1], nullptr, M->T2, m);
        gather(s, M->T2, G.var_ptr, G.var_occ, nullptr, n, true, M->Mv[l]);
        dense(s, true, M->Hv[l - 1], H, M->Mv[l], H, P + M->o_Uv[l - 1], M->p + M->o_buv[l - 1], M->Hv[l], n);
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
        dW(s, dHv, M->Hv[l - 1], H, M->Mv[l], H, M->g + M->o_Uv[l - 1], M->g + M->o_buv[l - 1], n);
        dX(s, dHv, P + M->o_Uv[l - 1], H, H, dHv2, M->dMv, n);
        // m_v = (1/deg v) sum s t_c  ->  dt_c = sum_{v in c} s dm_v / deg v
        gather(s, M->dMv, G.row_ptr, G.lits, G.inv_deg, m, false, M->dT2);
        // t_c = B h_c^l
        dW(s, M->dT2, M->Hc[l], H, nullptr, 0, M->g + M->o_B[l - 1], nullptr, m);
        dX(s, M->dT2, P + M->o_B[l - 1], H, 0, M->dHcx, nullptr, m);
        add_inplace<<<std::min<unsigned>(blocks_for((size_t)m * H, 256), 4096), 256, 0, s>>>(dHc, M->dHcx,
                                                                                           (size_t)m * H);
        // h_c^l = relu(Uc [h_c^{l-1}; m_c] + buc)
        mask(s, dHc, M->Hc[l], (size_t)m * H);
        dW(s, dHc, M->Hc[l - 1], H, M->Mc[l], H, M->g + M->o_Uc[l - 1], M->g + M->o_buc[l - 1], m);
        dX(s, dHc, P + M->o_Uc[l - 1], H, H, dHc2, M->dMc, m);
        // m_c = (1/|c|) sum s t_v  ->  dt_v = sum_{c ni v} s dm_c / |c|
        gather(s, M->dMc, G.var_ptr, G.var_occ, G.inv_len, n, false, M->dT1);
        // t_v = A h_v^{l-1}
        dW(s, M->dT1, M->Hv[l - 1], H, nullptr, 0, M->g + M->o_A[l - 1], nullptr, n);
        dX(s, M->dT1, P + M->o_A[l - 1], H, 0, M->dHvx, nullptr, n);
        add_inplace<<<std::min<unsigned>(blocks_for((size_t)n * H, 256), 4096), 256, 0, s>>>(dHv2, M->dHvx,
                                                                                           (size_t)n * H);
        std::swap(dHv, dHv2);
        std::swap(dHc, dHc2);
    }
    mask(s, dHv, M->Hv[0], (size_t)n * H);
    dW(s, dHv, G.fv, FV, nullptr, 0, M->g + M->o_wv0, M->g + M->o_bv0, n);
    mask(s, dHc, M->Hc[0], (size_t)m * H);
    dW(s, dHc, G.fc, FC, nullptr, 0, M->g + M->o_wc0, M->g + M->o_bc0, m);
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
    delete M;
}

}  // extern "C"
