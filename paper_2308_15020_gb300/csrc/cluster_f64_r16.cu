// One-cluster-per-point FP64 step kernels, node R = 16.
#include "cluster_launch.h"
#include "cluster_step.cuh"
FFSAT_DEFINE_CLUSTER(cluster_f64_r16, 16)
