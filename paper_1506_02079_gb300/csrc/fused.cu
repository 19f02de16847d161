// Fused wavefront multigrid kernels (filled in below).
#include "emfuse_common.cuh"
