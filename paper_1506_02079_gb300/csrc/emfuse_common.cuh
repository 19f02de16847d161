// Shared device/host helpers of libemfuse (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "emfuse.h"  // from include/ (-I)

namespace emfuse {

// ---------------------------------------------------------------- error plumbing (host)
void set_error(const std::string& msg);
const char* last_error();

struct Status {
    int code = EMFUSE_OK;
    bool ok() const { return code == EMFUSE_OK; }
};

#define EMF_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::emfuse::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));       \
            return (e_ == cudaErrorMemoryAllocation) ? EMFUSE_ENOMEM : EMFUSE_ECUDA;       \
        }                                                                                  \
    } while (0)

#define EMF_CHECK_LAUNCH()                                                                 \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess) {                                                           \
            ::emfuse::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));  \
            return EMFUSE_ECUDA;                                                           \
        }                                                                                  \
    } while (0)

#define EMF_TRY(expr)                                                                      \
    do {                                                                                   \
        int rc_ = (expr);                                                                  \
        if (rc_ != EMFUSE_OK) return rc_;                                                  \
    } while (0)

// Counts one kernel launch and, while profiling is on, brackets it with CUDA events on `s`.
// Construct immediately before the launch; the scope's end records the stop event.
class KernelScope {
  public:
    KernelScope(const char* name, cudaStream_t s, double bytes, double fp64_flops = 0.0);
    ~KernelScope();
    KernelScope(const KernelScope&) = delete;
    KernelScope& operator=(const KernelScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    double bytes_;
    double flops_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (grids are sized from the device query)

// Instrumentation state (runtime.cu): whether per-launch event timing is on, and the count
// of kernel launches (a replayed CUDA graph adds the kernels it holds).
bool profiling_active();
uint64_t launch_count();
void add_launches(int64_t n);

// ---------------------------------------------------------------- device-memory scratch
// The library's memory pool on the current device (runtime.cu): created on first use with no
// release threshold, so pages freed by one call stay mapped for the next instead of going back
// to the driver at every synchronisation; trim_library_pools() returns them.  nullptr if the
// pool cannot be created (the device's default pool is used then).
cudaMemPool_t library_pool();
void trim_library_pools();
// bytes the pool of the current device holds without any allocation using them
size_t library_pool_idle_bytes();

// Stream-ordered allocation from the library's pool; freed stream-ordered at scope exit.
class DeviceBuffer {
  public:
    DeviceBuffer() = default;
    DeviceBuffer(const DeviceBuffer&) = delete;
    DeviceBuffer& operator=(const DeviceBuffer&) = delete;
    ~DeviceBuffer() { release(); }
    int alloc(size_t bytes, cudaStream_t s) {
        release();
        stream_ = s;
        if (bytes == 0) return EMFUSE_OK;
        cudaMemPool_t pool = library_pool();
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&ptr_, bytes, pool, s) : cudaMallocAsync(&ptr_, bytes, s);
        if (e != cudaSuccess) {
            ptr_ = nullptr;
            set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) +
                      " bytes): " + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? EMFUSE_ENOMEM : EMFUSE_ECUDA;
        }
        bytes_ = bytes;
        return EMFUSE_OK;
    }
    // Allocation kept across calls (solver plans): plain cudaMalloc / cudaFree, so it is not
    // tied to the lifetime of the caller's stream.
    int alloc_persistent(size_t bytes) {
        release();
        persistent_ = true;
        if (bytes == 0) return EMFUSE_OK;
        cudaError_t e = cudaMalloc(&ptr_, bytes);
        if (e != cudaSuccess) {
            ptr_ = nullptr;
            set_error(std::string("cudaMalloc(") + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? EMFUSE_ENOMEM : EMFUSE_ECUDA;
        }
        bytes_ = bytes;
        return EMFUSE_OK;
    }
    void release() {
        if (ptr_) {
            if (persistent_) cudaFree(ptr_);
            else cudaFreeAsync(ptr_, stream_);
        }
        ptr_ = nullptr;
        bytes_ = 0;
        persistent_ = false;
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(ptr_); }
    size_t bytes() const { return bytes_; }

  private:
    void* ptr_ = nullptr;
    size_t bytes_ = 0;
    cudaStream_t stream_ = nullptr;
    bool persistent_ = false;
};

// ---------------------------------------------------------------- multigrid geometry
// Level k of a slice with fine size n0 (per axis) has n_k = ceil(n0 / 2^k) cells; cell I
// covers fine pixels [I 2^k, min((I+1) 2^k, n0)).  Only the last cell can be partial.
// The coarse operator is the finite-volume rediscretisation on those true cells (see
// multigrid.cu), which keeps the V-cycle contraction independent of odd sizes.
__host__ __device__ inline int level_size(int n0, int k) { return ((n0 - 1) >> k) + 1; }

// Width of cell I at level k in units of a full level-k cell: 1, or (0,1) for a partial last
// cell.
template <class T>
__host__ __device__ inline T cell_width(int I, int n0, int k) {
    const int full = 1 << k;
    const int rem = n0 - (I << k);
    return rem >= full ? T(1) : T(rem) / T(full);
}

// Face coefficient 2 / (w_I + w_{I+1}) between cells I and I+1 (0 outside: Neumann).
template <class T>
__host__ __device__ inline T face_coeff(int I, int n, int n0, int k) {
    if (I < 0 || I + 1 >= n) return T(0);
    return T(2) / (cell_width<T>(I, n0, k) + cell_width<T>(I + 1, n0, k));
}

}  // namespace emfuse
