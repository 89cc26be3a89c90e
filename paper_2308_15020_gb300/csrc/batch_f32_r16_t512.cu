// Batch-kernel instance: float, node R 16, 512 threads per CTA.
#include "batch_launch.cuh"
FFSAT_DEFINE_BATCH(batch_f32_r16_t512, float, 16, 512)
