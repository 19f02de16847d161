// Internal (non-exported) interfaces between the translation units of libemfuse.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "emfuse_common.cuh"

namespace emfuse {

// ---- device error word set by kernels whose bounded waits expire (runtime.cu)
int* device_error_flag();

// ---- smoothing (smooth.cu)
int support_radius(float sigma);
std::vector<float> gaussian_taps(float sigma, int R);
std::vector<float> inverse_norms(const std::vector<float>& w, int n);
// force_path: 0 = automatic, 1 = three 1-D passes; kappa > 0: robust z-averaging (samples
// beyond kappa weighted standard deviations of the window's weighted mean left out)
int smooth_stack(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                 int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                 cudaStream_t st, int force_path, float kappa = 0.f);
int smooth_transpose(const float* g, float* out, int64_t nx, int64_t ny, int64_t nz,
                     float sigma_xy, float sigma_z, cudaStream_t st);
int smooth_dsigma_z(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                    float sigma_xy, float sigma_z, cudaStream_t st);

// ---- multigrid screened-Poisson solve (multigrid.cu)
struct SolveRequest {
    const float* s = nullptr;   // value constraints (I1), packed ragged batch
    const void* o = nullptr;    // gradient constraints (I0), packed, dtype o_dtype
    int o_dtype = EMFUSE_F32;
    const float* rhs = nullptr; // if non-null: solve A x = rhs instead (adjoint); s, o unused
    float* out = nullptr;       // solution, packed
    int64_t nslices = 0;
    const int64_t* nx = nullptr;       // host
    const int64_t* ny = nullptr;       // host
    const int64_t* offsets = nullptr;  // host, elements
    double alpha = 0.0;
    emfuse_solve_opts opts{};
    emfuse_slice_stats* stats = nullptr;  // host, may be null
};
int solve_batch(const SolveRequest& req, cudaStream_t st);
// candidates timed by the last autotuning solve on this host thread, the chosen one first
const std::vector<emfuse_tune_entry>& last_autotune();
void release_plans();
// after a synchronisation of `st`: EMFUSE_ETIMEOUT (and the error word cleared) if a bounded wait
// of the last solve of the plan of (current device, st, precision) expired, else EMFUSE_OK; for
// asynchronous solves, whose return value cannot report it
int solve_async_status(cudaStream_t st, int precision);
// bytes of the pyramids and FP64 iterates held by the cached plan of (current device, stream,
// precision): a later solve on that stream reuses them
size_t cached_plan_bytes(cudaStream_t st, int precision);

// ---- direct solve by fast transforms (dct_solve.cu): uniform batch of n slices of ny x nx,
// precision EMFUSE_PREC_FP32 or EMFUSE_PREC_FP64; FFT plans cached until release_fft_plans()
int solve_dct_batch(const float* s, const float* o, float* f, int64_t n, int64_t nx, int64_t ny, double alpha,
                    int precision, cudaStream_t st);
// 3-D gradient-domain smoothing (dct_solve.cu): out = argmin alpha |f - in|^2 +
// |grad_xy f - grad_xy in|^2 + |d_z f|^2 over an nz x ny x nx stack, exact: a DCT along z
// (GEMM) splits it into nz slice problems solved by the mirror-extension FFT; in uint8
// (dt EMFUSE_U8) or float, transforms in `precision`
int smooth_gradient_domain(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha,
                           int precision, cudaStream_t st);
// mg3d.cu
int gd_multigrid(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha,
                 const emfuse_solve_opts& opts, emfuse_slice_stats* stats, cudaStream_t st);
void release_fft_plans();  // and the cuBLAS handles

// elementwise helpers used by the adjoint (multigrid.cu)
int apply_laplacian_stack(const float* in, float* out, int64_t nx, int64_t ny, int64_t nz,
                          float scale, cudaStream_t st);
// sum_j <a_j, b_j - c_j> in FP64 over a dense float stack; result copied to host
int dot_diff(const float* a, const float* b, const float* c, int64_t n, double* host_out,
             cudaStream_t st);
int scale_copy(const float* in, float* out, int64_t n, float a, cudaStream_t st);
int axpy(const float* x, float* y, int64_t n, float a, cudaStream_t st);

}  // namespace emfuse
