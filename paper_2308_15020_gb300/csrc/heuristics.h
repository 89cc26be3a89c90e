// Device-side restart heuristics (internal): ERWA weights and rephasing.
#pragma once
#include "ffsat_internal.h"

namespace ffsat {

// Every device location that holds a constraint's weight.
struct WeightSites {
    int32_t m;
    int32_t n_images;
    int4 *clauses[3];   // clause records of each resident image (FP32 weight bits in .w)
    int4 *segmeta[3];   // segment metadata of each resident image (FP32 weight bits in .w)
    double *clause_wd;  // FP64 weight by clause slot
    double *seg_wd;     // FP64 weight by segment slot
    double *cons_wd;    // FP64 weight by constraint (the master copy)
    const int8_t *cls;  // 0 clause of <= 3 literals, 1 product, 2 node, 3 constant, 4 XOR of <= 2 literals
    const int32_t *slot;
    const int32_t *row_ptr;
    const int32_t *param;
};

// umax: one device int32 of scratch; f_const: the instance's two device constants.
cudaError_t launch_erwa(const WeightSites &W, const int32_t *U, int32_t *umax, double alpha, double *f_const,
                        cudaStream_t s, int *launches);
cudaError_t launch_rephase(bool f64, void *x, int B, int n, int phase, const uint8_t *solved, uint64_t seed,
                           uint64_t epoch, uint64_t b_offset, const uint64_t *epoch_dev, cudaStream_t s,
                           int *launches);

}  // namespace ffsat
