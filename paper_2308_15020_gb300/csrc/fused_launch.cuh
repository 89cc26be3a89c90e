// Launcher body shared by the per-variant translation units.
#pragma once
#include "fused_kernel.cuh"

namespace ffsat {
namespace dev {

// Nodes per iteration of the node loop: two independent multiply chains in
// FP32, one in FP64 (register budget).
template <typename R, int NR>
constexpr int node_interleave() {
    return (sizeof(R) == 4 && NR > 0) ? 2 : 1;
}

template <typename R, int NR, int SM>
cudaError_t fused_launch_mode(const DevView &V, const FusedArgs &a, size_t smem, int grid, cudaStream_t s,
                              bool prepare_only) {
    constexpr int TH = fused_threads(sizeof(R) == 8, NR);
    auto k = fused_kernel<R, NR, node_interleave<R, NR>(), SM, TH>;
    if (prepare_only) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, TH, smem, s>>>(V, a);
    return cudaGetLastError();
}

template <typename R, int NR>
cudaError_t fused_launch(const DevView &V, int smem_mode, const FusedArgs &a, size_t smem, int grid,
                         cudaStream_t s, bool prepare_only) {
    switch (smem_mode) {
    case SMEM_FULL:
        return fused_launch_mode<R, NR, SMEM_FULL>(V, a, smem, grid, s, prepare_only);
    case SMEM_RES:
        return fused_launch_mode<R, NR, SMEM_RES>(V, a, smem, grid, s, prepare_only);
    case SMEM_X:
        return fused_launch_mode<R, NR, SMEM_X>(V, a, smem, grid, s, prepare_only);
    default:
        return fused_launch_mode<R, NR, SMEM_NONE>(V, a, smem, grid, s, prepare_only);
    }
}

}  // namespace dev
}  // namespace ffsat

#define FFSAT_DEFINE_FUSED(name, R, NR)                                                               \
    namespace ffsat {                                                                                 \
    FFSAT_FUSED_LAUNCHER(name) { return dev::fused_launch<R, NR>(V, smem_mode, a, smem, grid, s, prepare_only); } \
    }
