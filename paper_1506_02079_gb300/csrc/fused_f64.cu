// FP64 instantiation of the fused multigrid schedule (kernels in fused_impl.cuh, launchers in
// fused_launch.cuh).
#include "fused_launch.cuh"

namespace emfuse {
namespace fused_detail {
// nu = 3, 4: instantiated in fused_f64_s68.cu
extern template int launch_wave_s<double, 6>(const WaveArgs<double>&, bool, bool, cudaStream_t);
extern template int launch_wave_s<double, 8>(const WaveArgs<double>&, bool, bool, cudaStream_t);
}  // namespace fused_detail

template <>
int launch_wave<double>(const WaveArgs<double>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    return launch_wave_impl<double>(a, S, zero_init, up, st, bytes);
}
template <>
int launch_tail<double>(const TailArgs<double>& a, cudaStream_t st, double bytes) {
    return launch_tail_impl<double>(a, st, bytes);
}

}  // namespace emfuse
