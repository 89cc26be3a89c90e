// Batch-kernel instances: several instances of uneven size in one launch.
#include "fused_launch.cuh"

namespace ffsat {

namespace {
template <typename R, int NR>
cudaError_t batch_one(const BatchInst *insts, const int2 *items, int n_items, int *counter, const StepParams &sp,
                      size_t smem, int grid, cudaStream_t s, bool prepare_only, int *blocks_per_sm) {
    constexpr int TH = batch_threads_for(sizeof(R) == 8, NR);
    auto k = dev::batch_kernel<R, NR, dev::node_interleave<R, NR>(), TH>;
    if (prepare_only) {
        cudaError_t e = dev::raise_smem_limit(k, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, TH, smem);
    }
    k<<<grid, TH, smem, s>>>(insts, items, n_items, counter, sp);
    return cudaGetLastError();
}
}  // namespace

int batch_threads(bool f64, int node_r) { return batch_threads_for(f64, node_r > 0 ? 16 : 0); }

cudaError_t launch_batch(bool f64, int node_r, const BatchInst *insts, const int2 *items, int n_items, int *counter,
                         const StepParams &sp, size_t smem, int grid, cudaStream_t s, bool prepare_only,
                         int *blocks_per_sm) {
    if (f64)
        return node_r > 0 ? batch_one<double, 16>(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm)
                          : batch_one<double, 0>(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm);
    return node_r > 0 ? batch_one<float, 16>(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm)
                      : batch_one<float, 0>(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm);
}

}  // namespace ffsat
