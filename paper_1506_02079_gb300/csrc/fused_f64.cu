// FP64 instantiation of the fused multigrid schedule (kernels in fused_impl.cuh, launchers in
// fused_launch.cuh).
#include "fused_launch.cuh"

namespace emfuse {

template <>
int launch_wave<double>(const WaveArgs<double>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    return launch_wave_impl<double>(a, S, zero_init, up, st, bytes);
}
template <>
int launch_tail<double>(const TailArgs<double>& a, cudaStream_t st, double bytes) {
    return launch_tail_impl<double>(a, st, bytes);
}

}  // namespace emfuse
