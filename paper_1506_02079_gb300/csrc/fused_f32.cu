// FP32 instantiation of the fused multigrid schedule (kernels in fused_impl.cuh, launchers in
// fused_launch.cuh).
#include "fused_launch.cuh"

namespace emfuse {
namespace fused_detail {
// nu = 3, 4: instantiated in fused_f32_s68.cu
extern template int launch_wave_s<float, 6>(const WaveArgs<float>&, bool, bool, cudaStream_t);
extern template int launch_wave_s<float, 8>(const WaveArgs<float>&, bool, bool, cudaStream_t);
}  // namespace fused_detail

template <>
int launch_wave<float>(const WaveArgs<float>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    return launch_wave_impl<float>(a, S, zero_init, up, st, bytes);
}
template <>
int launch_tail<float>(const TailArgs<float>& a, cudaStream_t st, double bytes) {
    return launch_tail_impl<float>(a, st, bytes);
}

}  // namespace emfuse
