// Launchers of the FP64 one-cluster-per-point step kernel (cluster_step.cuh),
// one per node R; each handles the SMEM_FULL and SMEM_RES layouts.  The grid is
// B clusters of CL CTAs; smem is the dynamic shared memory per CTA, g1_off the
// byte offset of its second gradient buffer.  With max_active set the launcher
// raises the kernel's shared-memory limit, stores the number of such clusters
// that can be resident at once and launches nothing.
#pragma once
#include <cuda_runtime.h>

#include "ffsat_internal.h"

namespace ffsat {

#define FFSAT_CLUSTER_LAUNCHER(name)                                                                     \
    cudaError_t name(const DevView &V, int smem_mode, const FusedArgs &a, size_t smem, size_t g1_off, int B, \
                     int CL, cudaStream_t s, int *max_active)
FFSAT_CLUSTER_LAUNCHER(cluster_f64_r0);
FFSAT_CLUSTER_LAUNCHER(cluster_f64_r8);
FFSAT_CLUSTER_LAUNCHER(cluster_f64_r16);

}  // namespace ffsat
