// Fused kernel instances: double, node R = 0.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f64_r0, double, 0)
