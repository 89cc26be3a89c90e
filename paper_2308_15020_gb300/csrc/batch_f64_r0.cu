// Batch-kernel instance: double, node R 0, 256 threads per CTA.
#include "batch_launch.cuh"
FFSAT_DEFINE_BATCH(batch_f64_r0, double, 0, 256)
