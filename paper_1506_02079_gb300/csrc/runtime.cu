// Launch accounting and optional per-kernel CUDA-event timing (the instrumentation entry
// points of include/emfuse.h).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "emfuse_common.cuh"
#include "fpconv.cuh"
#include "tma.cuh"

namespace emfuse {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}
}  // namespace

int encode_tensor_map_2d(CUtensorMap* out, const void* base, int elem_bytes, int64_t nx, int64_t ny,
                         int64_t pitch, int box_x, int box_y) {
    auto fn = tensor_map_encoder();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the CUDA driver");
        return EMFUSE_ECUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[1] = {(cuuint64_t)(pitch * elem_bytes)};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(out, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                          const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return EMFUSE_ECUDA;
    }
    return EMFUSE_OK;
}

int encode_tensor_map_3d(CUtensorMap* out, const void* base, int elem_bytes, int64_t nx, int64_t ny,
                         int64_t nz, int64_t pitch, int box_x, int box_y) {
    auto fn = tensor_map_encoder();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the CUDA driver");
        return EMFUSE_ECUDA;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * elem_bytes), (cuuint64_t)(pitch * ny * elem_bytes)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(out, elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (3-D) failed with CUresult " + std::to_string((int)r));
        return EMFUSE_ECUDA;
    }
    return EMFUSE_OK;
}

namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_profiling{false};
std::mutex g_mu;
struct Rec {
    const char* name;
    cudaEvent_t a, b;
    double bytes;
    double flops;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

bool profiling_active() { return g_profiling.load(std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(int64_t n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

KernelScope::KernelScope(const char* name, cudaStream_t s, double bytes, double fp64_flops)
    : name_(name), s_(s), bytes_(bytes), flops_(fp64_flops) {
    if (g_profiling.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        a_ = take_event();
        b_ = take_event();
        if (a_ && b_) cudaEventRecord(a_, s_);
    }
}

KernelScope::~KernelScope() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (a_ && b_) {
        cudaEventRecord(b_, s_);
        std::lock_guard<std::mutex> lk(g_mu);
        g_recs.push_back(Rec{name_, a_, b_, bytes_, flops_});
    }
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {nullptr};
bool g_pool_failed[64] = {false};
}  // namespace

cudaMemPool_t library_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev] && !g_pool_failed[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            g_pool_failed[dev] = true;
            return nullptr;
        }
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = p;
    }
    return g_pools[dev];
}

size_t library_pool_idle_bytes() {
    cudaMemPool_t p = library_pool();
    if (!p) return 0;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return reserved > used ? (size_t)(reserved - used) : 0;
}

void trim_library_pools() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int d = 0; d < 64; ++d)
        if (g_pools[d]) cudaMemPoolTrimTo(g_pools[d], 0);
}

// One int per device, allocated on first use and kept for the life of the process: kernels
// whose bounded waits give up set it; solves read and clear it when they synchronise.
int* device_error_flag() {
    static std::mutex mu;
    static int* flags[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!flags[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        flags[dev] = p;
    }
    return flags[dev];
}

// ---------------------------------------------------------------- bounded-wait self-test
namespace {

// The bounded wait of tma.cuh (mbar_wait_warp) with a poll limit given at run time.
__device__ __forceinline__ bool wait_warp_polls(uint32_t bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it)
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    return false;
}

// One warp waits, with at most `limit` polls, for phase 0 of an mbarrier that nothing arrives
// on: the wait runs out, and the kernel records that in the device error word and returns,
// as every bounded wait of the library does when a copy never lands.
__global__ void k_wait_timeout(int* err, int limit) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_init_fence();
    }
    __syncwarp();
    if (!wait_warp_polls(b, 0, limit) && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace

// ---------------------------------------------------------------- conversion self-test
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    // SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014)
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ bool same_double(double a, double b) {
    return (a != a) ? (b != b) : __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_float(float a, float b) {
    return (a != a) ? (b != b) : __float_as_uint(a) == __float_as_uint(b);
}

// Every binary32 bit pattern u: f2d_ieee against the hardware widening; d2f_ieee against the
// hardware rounding on the widened value with the 29 bits below binary32 precision set to
// rounding-critical patterns (just above zero, just below / at / just above the half, all
// ones, a quarter), and on one SplitMix64 bit pattern per u (every binary64 exponent,
// including the ranges that underflow to subnormals or overflow).
__global__ void k_selftest_fpconv(unsigned long long* bad) {
    unsigned long long nf = 0, nd = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const float f = __uint_as_float((uint32_t)i);
        const double w = f2d_ieee(f);
        nf += !same_double(w, (double)f);
        const uint32_t hi = (uint32_t)__double2hiint(w), lo = (uint32_t)__double2loint(w);
        const uint32_t lows[6] = {1u, 0x0fffffffu, 0x10000000u, 0x10000001u, 0x1fffffffu, 0x08000000u};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double x = __hiloint2double((int)hi, (int)((lo & 0xe0000000u) | lows[k]));
            nd += !same_float(d2f_ieee(x), (float)x);
        }
        const double r = __longlong_as_double((long long)splitmix64(i));
        nd += !same_float(d2f_ieee(r), (float)r);
    }
    if (nf) atomicAdd(&bad[0], nf);
    if (nd) atomicAdd(&bad[1], nd);
}

}  // namespace

// ---------------------------------------------------------------- FP64 rate probe
namespace {

constexpr int kRateChains = 8;  // independent DFMA chains per thread (covers the pipe latency)

// Every thread runs kRateChains independent chains x <- x * a + b for `iters` steps (a, b keep
// x bounded); the sums are written only if they match an impossible sentinel, so that the
// chains stay live without a store per thread.
__global__ void __launch_bounds__(256) k_fp64_rate(double* sink, int iters, double a, double b) {
    double x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
#pragma unroll 1
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kRateChains; ++i) x[i] = __fma_rn(x[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) s += x[i];
    if (sink && s == -1.25e300) sink[0] = s;
}

}  // namespace

}  // namespace emfuse

using namespace emfuse;

extern "C" {

uint64_t emfuse_kernel_launches(void) { return g_launches.load(); }

void emfuse_profile_begin(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_profiling.store(true);
}

int emfuse_profile_end(emfuse_kernel_profile* out, int max_entries) {
    g_profiling.store(false);
    std::lock_guard<std::mutex> lk(g_mu);
    struct Acc { int64_t n = 0; double ms = 0, bytes = 0, flops = 0; };
    std::map<std::string, Acc> acc;
    int rc = 0;
    for (auto& r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) { rc = -1; continue; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) { rc = -1; continue; }
        Acc& x = acc[r.name];
        x.n += 1;
        x.ms += ms;
        x.bytes += r.bytes;
        x.flops += r.flops;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    if (rc < 0) {
        set_error("emfuse_profile_end: a CUDA event could not be read");
        return -1;
    }
    std::vector<std::pair<std::string, Acc>> v(acc.begin(), acc.end());
    std::sort(v.begin(), v.end(), [](auto& p, auto& q) { return p.second.ms > q.second.ms; });
    for (int i = 0; i < (int)v.size() && i < max_entries && out; ++i) {
        std::memset(&out[i], 0, sizeof(out[i]));
        std::strncpy(out[i].name, v[i].first.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = v[i].second.n;
        out[i].total_ms = v[i].second.ms;
        out[i].bytes = v[i].second.bytes;
        out[i].fp64_flops = v[i].second.flops;
    }
    return (int)v.size();
}

int emfuse_selftest_wait_timeout(int limit, void* stream) {
    set_error("");
    if (limit < 1 || limit > kWaitLimit) {
        set_error("emfuse_selftest_wait_timeout: limit must be in [1, 2^20]");
        return EMFUSE_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    int* err = device_error_flag();
    if (!err) {
        set_error("emfuse_selftest_wait_timeout: could not allocate the device error word");
        return EMFUSE_ENOMEM;
    }
    k_wait_timeout<<<1, 32, 0, st>>>(err, limit);
    EMF_CHECK_LAUNCH();
    int flag = 0;
    EMF_CUDA(cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EMF_CUDA(cudaStreamSynchronize(st));
    if (flag) {
        EMF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        EMF_CUDA(cudaStreamSynchronize(st));
        set_error("emfuse_selftest_wait_timeout: the bounded wait ran out (expected)");
        return EMFUSE_ETIMEOUT;
    }
    return EMFUSE_OK;
}

int emfuse_kernel_binary_version(int* binary_version) {
    set_error("");
    if (!binary_version) {
        set_error("emfuse_kernel_binary_version: null pointer");
        return EMFUSE_EINVAL;
    }
    cudaFuncAttributes attr;
    EMF_CUDA(cudaFuncGetAttributes(&attr, k_wait_timeout));
    *binary_version = attr.binaryVersion;
    return EMFUSE_OK;
}

int emfuse_probe_fp64_fma_rate(double* tflops, void* stream) {
    set_error("");
    if (!tflops) {
        set_error("emfuse_probe_fp64_fma_rate: null pointer");
        return EMFUSE_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    EMF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t a = nullptr, b = nullptr;
    EMF_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        set_error("emfuse_probe_fp64_fma_rate: cudaEventCreate failed");
        return EMFUSE_ECUDA;
    }
    float best = 0.f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
        cudaEventRecord(a, st);
        {
            KernelScope ks("fp64_rate_probe", st, 0.0, 2.0 * kRateChains * (double)iters * blocks * threads);
            k_fp64_rate<<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999, 1e-7);
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess || !(best > 0.f)) {
        set_error(std::string("emfuse_probe_fp64_fma_rate: ") + cudaGetErrorString(e));
        return EMFUSE_ECUDA;
    }
    *tflops = 2.0 * kRateChains * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    return EMFUSE_OK;
}

int emfuse_selftest_fpconv(int64_t* f2d_mismatches, int64_t* d2f_mismatches) {
    set_error("");
    if (!f2d_mismatches || !d2f_mismatches) {
        set_error("emfuse_selftest_fpconv: null pointer");
        return EMFUSE_EINVAL;
    }
    unsigned long long* bad = nullptr;
    EMF_CUDA(cudaMalloc(&bad, 2 * sizeof(unsigned long long)));
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemset(bad, 0, sizeof(h));
    if (e == cudaSuccess) {
        k_selftest_fpconv<<<kNumSMs * 8, 256>>>(bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (e != cudaSuccess) {
        set_error(std::string("emfuse_selftest_fpconv: ") + cudaGetErrorString(e));
        return EMFUSE_ECUDA;
    }
    *f2d_mismatches = (int64_t)h[0];
    *d2f_mismatches = (int64_t)h[1];
    return EMFUSE_OK;
}

}  // extern "C"
