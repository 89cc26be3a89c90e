// Batch-kernel instance: double, node R 16, 128 threads per CTA.
#include "batch_launch.cuh"
FFSAT_DEFINE_BATCH(batch_f64_r16, double, 16, 128)
