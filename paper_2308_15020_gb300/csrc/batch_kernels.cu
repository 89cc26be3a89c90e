// Batch-kernel dispatch: several instances of uneven size in one launch.  The
// kernel instances live in batch_*.cu; FP32 node-path batches come in two CTA
// widths (384 and 512 threads) between which the batch's tuner chooses.
#include "ffsat_internal.h"

namespace ffsat {

cudaError_t launch_batch(bool f64, int node_r, int threads, const BatchInst *insts, const int2 *items, int n_items,
                         int *counter, const StepParams &sp, size_t smem, int grid, cudaStream_t s, bool prepare_only,
                         int *blocks_per_sm) {
    if (f64)
        return node_r > 0 ? batch_f64_r16(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm)
                          : batch_f64_r0(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm);
    if (node_r == 0) return batch_f32_r0(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm);
    return threads == 384
               ? batch_f32_r16_t384(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm)
               : batch_f32_r16_t512(insts, items, n_items, counter, sp, smem, grid, s, prepare_only, blocks_per_sm);
}

}  // namespace ffsat
