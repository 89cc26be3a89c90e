// Fused kernel instances: float, node R = 8.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f32_r8, float, 8)
