// FP64 instantiations of the fused multigrid schedule (kernels in fused_impl.cuh).
#include <algorithm>

#include "fused_impl.cuh"

namespace emfuse {
using fused_detail::kWaveWarps;

template <class T>
static int launch_wave_impl(const WaveArgs<T>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    if (a.nitems == 0) return EMFUSE_OK;
    int sms = 0, dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    EMF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    static const char* const kUp[] = {"wave_up_l0", "wave_up_l1", "wave_up_l2", "wave_up_l3", "wave_up_l4",
                                      "wave_up_l5+"};
    static const char* const kDown[] = {"wave_down_l0", "wave_down_l1", "wave_down_l2", "wave_down_l3",
                                        "wave_down_l4", "wave_down_l5+"};
    const char* name = up ? kUp[a.k < 5 ? a.k : 5] : kDown[a.k < 5 ? a.k : 5];
    KernelScope ks(name, st, bytes);
    // persistent warps: as many CTAs as fit on the GPU at once (items are fetched dynamically)
#define EMF_WAVE_ONE(KERNEL, SMEM)                                                           \
    do {                                                                                     \
        const int smem = SMEM;                                                               \
        static int per_sm = 0;                                                               \
        EMF_CUDA(cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)); \
        if (per_sm == 0) {                                                                   \
            int nb = 0;                                                                      \
            EMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, KERNEL, kWaveWarps * 32, smem)); \
            per_sm = nb < 1 ? 1 : nb;                                                        \
        }                                                                                    \
        const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(a.nitems, kWaveWarps), (int64_t)sms * per_sm); \
        KERNEL<<<grid, kWaveWarps * 32, smem, st>>>(a);                                      \
    } while (0)
#define EMF_WAVE(SS)                                                                         \
    do {                                                                                     \
        if (up) EMF_WAVE_ONE((fused_detail::k_wave<T, SS, false, true>),                     \
                             (fused_detail::wave_smem_bytes<T, SS, false, true>()));         \
        else if (zero_init) EMF_WAVE_ONE((fused_detail::k_wave<T, SS, true, false>),         \
                                         (fused_detail::wave_smem_bytes<T, SS, true, false>())); \
        else EMF_WAVE_ONE((fused_detail::k_wave<T, SS, false, false>),                       \
                          (fused_detail::wave_smem_bytes<T, SS, false, false>()));           \
    } while (0)
    switch (S) {
        case 2: EMF_WAVE(2); break;
        case 4: EMF_WAVE(4); break;
        default: set_error("wavefront kernel: unsupported sweep count"); return EMFUSE_EINVAL;
    }
#undef EMF_WAVE
#undef EMF_WAVE_ONE
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

template <class T>
static int launch_tail_impl(const TailArgs<T>& a, cudaStream_t st, double bytes) {
    if (a.nslices == 0) return EMFUSE_OK;
    KernelScope ks("coarse_tail", st, bytes);
    fused_detail::k_tail<T><<<(unsigned)a.nslices, 512, 0, st>>>(a);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

template <>
int launch_wave<double>(const WaveArgs<double>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    return launch_wave_impl<double>(a, S, zero_init, up, st, bytes);
}
template <>
int launch_tail<double>(const TailArgs<double>& a, cudaStream_t st, double bytes) {
    return launch_tail_impl<double>(a, st, bytes);
}

}  // namespace emfuse
