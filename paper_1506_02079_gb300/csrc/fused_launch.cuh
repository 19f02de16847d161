// Host-side launchers of the fused multigrid schedule (kernels in fused_impl.cuh), one template
// for both iterate types.  fused_f32.cu and fused_f64.cu instantiate it for their type with 2 and
// 4 half-sweeps (nu = 1, 2); fused_f32_s68.cu and fused_f64_s68.cu the kernels with 6 and 8
// (nu = 3, 4), so that the four sets compile in parallel.
#pragma once
#include <algorithm>
#include <mutex>

#include "fused_impl.cuh"

namespace emfuse {
namespace fused_detail {

// Per-device launch data of one kernel instantiation: its dynamic shared-memory attribute is
// set once per device, and its resident CTAs per SM (occupancy query) cached.  One cache per
// instantiation <T, S, ZERO, UP> (the kernels share one function type).
struct WaveLaunchCache {
    std::mutex mu;
    int per_sm[64] = {0};
    int sms[64] = {0};
};

template <class T, int S, bool ZERO, bool UP, class K>
int wave_launch_info(K* kernel, int smem, int& per_sm, int& sms) {
    static WaveLaunchCache cache;
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("wavefront kernel: device ordinal out of range");
        return EMFUSE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(cache.mu);
    if (cache.per_sm[dev] == 0) {
        EMF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int nb = 0;
        EMF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kWaveWarps * 32, smem));
        EMF_CUDA(cudaDeviceGetAttribute(&cache.sms[dev], cudaDevAttrMultiProcessorCount, dev));
        cache.per_sm[dev] = nb < 1 ? 1 : nb;
    }
    per_sm = cache.per_sm[dev];
    sms = cache.sms[dev];
    return EMFUSE_OK;
}

// Persistent warps: as many CTAs as fit on the GPU at once (items are fetched dynamically).
template <class T, int S, bool ZERO, bool UP>
int launch_wave_one(const WaveArgs<T>& a, cudaStream_t st) {
    auto* kernel = k_wave<T, S, ZERO, UP>;
    const int smem = wave_smem_bytes<T, S, ZERO, UP>();
    int per_sm = 0, sms = 0;
    EMF_TRY((wave_launch_info<T, S, ZERO, UP>(kernel, smem, per_sm, sms)));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(a.nitems, kWaveWarps), (int64_t)sms * per_sm);
    kernel<<<grid, kWaveWarps * 32, smem, st>>>(a);
    return EMFUSE_OK;
}

template <class T, int S>
int launch_wave_s(const WaveArgs<T>& a, bool zero_init, bool up, cudaStream_t st) {
    if (up) return launch_wave_one<T, S, false, true>(a, st);
    if constexpr (S + 1 > kWaveHalo) {  // the DOWN leg's residual needs S + 1 <= the strip halo
        set_error("wavefront kernel: the DOWN leg supports at most 3 sweeps");
        return EMFUSE_EINVAL;
    } else {
        if (zero_init) return launch_wave_one<T, S, true, false>(a, st);
        return launch_wave_one<T, S, false, false>(a, st);
    }
}

}  // namespace fused_detail

template <class T>
int launch_wave_impl(const WaveArgs<T>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes) {
    if (a.nitems == 0) return EMFUSE_OK;
    static const char* const kUp[] = {"wave_up_l0", "wave_up_l1", "wave_up_l2", "wave_up_l3", "wave_up_l4",
                                      "wave_up_l5+"};
    static const char* const kDown[] = {"wave_down_l0", "wave_down_l1", "wave_down_l2", "wave_down_l3",
                                        "wave_down_l4", "wave_down_l5+"};
    const char* name = up ? kUp[a.k < 5 ? a.k : 5] : kDown[a.k < 5 ? a.k : 5];
    KernelScope ks(name, st, bytes);
    switch (S) {
        case 2: EMF_TRY((fused_detail::launch_wave_s<T, 2>(a, zero_init, up, st))); break;
        case 4: EMF_TRY((fused_detail::launch_wave_s<T, 4>(a, zero_init, up, st))); break;
        case 6: EMF_TRY((fused_detail::launch_wave_s<T, 6>(a, zero_init, up, st))); break;
        case 8: EMF_TRY((fused_detail::launch_wave_s<T, 8>(a, zero_init, up, st))); break;
        default: set_error("wavefront kernel: unsupported sweep count"); return EMFUSE_EINVAL;
    }
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

template <class T>
int launch_tail_impl(const TailArgs<T>& a, cudaStream_t st, double bytes) {
    if (a.nslices == 0) return EMFUSE_OK;
    static std::mutex mu;
    static int attr_set[64] = {0};  // the shared-memory limit set per device
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(mu);
        if (attr_set[dev] < a.smem_bytes) {
            EMF_CUDA(cudaFuncSetAttribute(fused_detail::k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          a.smem_bytes));
            attr_set[dev] = a.smem_bytes;
        }
    }
    KernelScope ks("coarse_tail", st, bytes);
    fused_detail::k_tail<T><<<(unsigned)a.nslices, 512, (size_t)a.smem_bytes, st>>>(a);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

}  // namespace emfuse
