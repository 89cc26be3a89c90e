// Fused kernel instances: double, node R = 16.
#include "fused_launch.cuh"
FFSAT_DEFINE_FUSED(fused_f64_r16, double, 16)
