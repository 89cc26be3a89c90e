// One-cluster-per-point FP64 step kernels, node R = 0.
#include "cluster_launch.h"
#include "cluster_step.cuh"
FFSAT_DEFINE_CLUSTER(cluster_f64_r0, 0)
