// Fused kernel instances: float, node R = 0.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f32_r0, float, 0)
