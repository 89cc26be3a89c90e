// Batch-kernel instance: float, node R 0, 1024 threads per CTA.
#include "batch_launch.cuh"
FFSAT_DEFINE_BATCH(batch_f32_r0, float, 0, 1024)
