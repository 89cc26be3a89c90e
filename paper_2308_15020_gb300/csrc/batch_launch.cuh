// Launcher body of the batch kernel, shared by the per-variant translation units
// (one kernel instantiation each, so that nvcc compiles them in parallel).
#pragma once
#include "fused_launch.cuh"

namespace ffsat {
namespace dev {

template <typename R, int NR, int TH>
cudaError_t batch_one(const BatchInst *insts, const int2 *items, int n_items, int *counter, const StepParams &sp,
                      size_t smem, int grid, cudaStream_t s, bool prepare_only, int *blocks_per_sm) {
    auto k = batch_kernel<R, NR, node_interleave<R, NR>(), TH>;
    if (prepare_only) {
        cudaError_t e = raise_smem_limit(k, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, TH, smem);
    }
    k<<<grid, TH, smem, s>>>(insts, items, n_items, counter, sp);
    return cudaGetLastError();
}

}  // namespace dev
}  // namespace ffsat

#define FFSAT_DEFINE_BATCH(name, R, NR, TH)                                                      \
    namespace ffsat {                                                                            \
    FFSAT_BATCH_LAUNCHER(name) {                                                                 \
        return dev::batch_one<R, NR, TH>(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, \
                                         blocks_per_sm);                                         \
    }                                                                                            \
    }
