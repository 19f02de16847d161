// FP64 wavefront kernels with 6 and 8 half-sweeps per leg (nu = 3, 4; kernels in fused_impl.cuh,
// launchers in fused_launch.cuh), in a translation unit of their own so that they compile in
// parallel with the others.
#include "fused_launch.cuh"

namespace emfuse {
namespace fused_detail {
template int launch_wave_s<double, 6>(const WaveArgs<double>&, bool, bool, cudaStream_t);
template int launch_wave_s<double, 8>(const WaveArgs<double>&, bool, bool, cudaStream_t);
}  // namespace fused_detail
}  // namespace emfuse
