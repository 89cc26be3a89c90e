// Fused kernel instances: float, node R = 16.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f32_r16, float, 16)
