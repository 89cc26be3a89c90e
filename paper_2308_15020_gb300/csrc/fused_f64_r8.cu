// Fused kernel instances: double, node R = 8.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f64_r8, double, 8)
