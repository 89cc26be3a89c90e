// Launcher body shared by the per-variant translation units.
#pragma once
#include <map>
#include <mutex>
#include <utility>

#include "fused_kernel.cuh"

namespace ffsat {
namespace dev {

// Raise a kernel's dynamic shared-memory limit to at least `smem` on the
// current device.  The limit belongs to the kernel in one device's context, not
// to an instance, so it only ever grows per (device, kernel): a later, smaller
// instance must not lower it below what an earlier one launches with, and an
// instance on another device sets it there too.  The first request on a device
// always sets the attribute: the default limit is 48 KB less the kernel's static
// shared memory, not 48 KB.
inline std::mutex &smem_limit_mutex() {
    static std::mutex mu;
    return mu;
}
inline std::map<std::pair<int, const void *>, size_t> &smem_limits() {
    static std::map<std::pair<int, const void *>, size_t> limits;
    return limits;
}

template <typename Kernel>
cudaError_t raise_smem_limit(Kernel k, size_t smem) {
    std::lock_guard<std::mutex> lock(smem_limit_mutex());
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return ge;
    size_t &current = smem_limits()[{dev, reinterpret_cast<const void *>(k)}];
    if (current != 0 && smem <= current) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) current = smem;
    return e;
}

template <typename R, int NR, int SM, int FW = 2, int PP = 1>
cudaError_t fused_launch_mode(const DevView &V, const FusedArgs &a, size_t smem, int grid, cudaStream_t s,
                              bool prepare_only) {
    constexpr int TH = fused_threads(sizeof(R) == 8, NR);
    auto k = fused_kernel<R, NR, node_interleave<R, NR>(), SM, TH, FW, PP>;
    // (cached per device and kernel; a weight update can switch an instance to
    // the other fixed-point variant after its preparation)
    const cudaError_t e = raise_smem_limit(k, smem);
    if (prepare_only || e != cudaSuccess) return e;
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
        // FP32: one fixed-point word where the instance's range allows it
        if constexpr (sizeof(R) == 4) {
            // two points per CTA where the caller asks for them (smem and grid sized for it)
            if (!V.fix_two && a.pairs)
                return fused_launch_mode<R, NR, SMEM_RES, 1, 2>(V, a, smem, grid, s, prepare_only);
            if (!V.fix_two) return fused_launch_mode<R, NR, SMEM_RES, 1>(V, a, smem, grid, s, prepare_only);
        }
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
