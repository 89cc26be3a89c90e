// One-cluster-per-point FP64 step kernels, node R = 8.
#include "cluster_launch.h"
#include "cluster_step.cuh"
FFSAT_DEFINE_CLUSTER(cluster_f64_r8, 8)
