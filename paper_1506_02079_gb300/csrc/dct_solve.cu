// Direct solve of Eq. (1) by fast Fourier transforms: the frequency-space interpretation of
// Sec. 3 ("Frequency-Space Interpretation": every frequency of the result is a weighted average
// of the two inputs' frequencies) turned into a solver.  Sec. 3 "Alternate Solutions" weighs an
// FFT solver against multigrid and rejects it for out-of-core CPUs (log-linear work and an
// out-of-core transpose); with a slice in HBM neither objection holds, so it serves here as an
// exact second GPU solver to compare the multigrid against.
//
// The Neumann graph Laplacian of an ny x nx slice is the periodic Laplacian of its mirror
// extension to 2ny x 2nx (reflection across the cell edges: the ghost of a boundary cell is the
// cell itself), whose Fourier modes have eigenvalues 4 sin^2(pi k / 2ny) + 4 sin^2(pi l / 2nx),
// the eigenvalues of the discrete cosine modes of the slice.  In correction form f = o + d,
// (alpha I + L) d = alpha (s - o), so
//     d = first quadrant of IFFT( FFT(mirror(s - o)) * alpha / (alpha + lambda) ).
// The transforms are cuFFT (R2C / C2R, batched over the slices); the mirror extension, the
// spectral scaling and the extraction are the kernels below.
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cufft.h>

#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"

namespace emfuse {
namespace {

template <class T>
struct Fft;
template <>
struct Fft<float> {
    using C = cufftComplex;
    static constexpr cufftType kR2C = CUFFT_R2C, kC2R = CUFFT_C2R;
    static cufftResult fwd(cufftHandle p, float* in, C* out) { return cufftExecR2C(p, in, out); }
    static cufftResult inv(cufftHandle p, C* in, float* out) { return cufftExecC2R(p, in, out); }
};
template <>
struct Fft<double> {
    using C = cufftDoubleComplex;
    static constexpr cufftType kR2C = CUFFT_D2Z, kC2R = CUFFT_Z2D;
    static cufftResult fwd(cufftHandle p, double* in, C* out) { return cufftExecD2Z(p, in, out); }
    static cufftResult inv(cufftHandle p, C* in, double* out) { return cufftExecZ2D(p, in, out); }
};

inline unsigned grid_of(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)kNumSMs * 32));
}

// ext = mirror extension of s - o: plane j of 2ny x 2nx, row Y, column X reads (y, x) with
// y = Y or 2ny - 1 - Y, x = X or 2nx - 1 - X.
template <class T>
__global__ void k_mirror(const float* __restrict__ s, const float* __restrict__ o, T* __restrict__ ext, int nx,
                         int ny, int64_t nslices) {
    const int64_t NX = 2 * (int64_t)nx, NY = 2 * (int64_t)ny, plane = NX * NY, total = nslices * plane;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / plane, q = i - j * plane;
        const int64_t Y = q / NX, X = q - Y * NX;
        const int64_t y = Y < ny ? Y : NY - 1 - Y, x = X < nx ? X : NX - 1 - X;
        const int64_t p = (j * ny + y) * nx + x;
        ext[i] = T(s[p]) - T(o[p]);
    }
}

// spec(k, l) *= alpha / (alpha + lam_y[k] + lam_x[l]) / (4 nx ny)   (half spectrum: nx + 1 columns)
template <class T, class C>
__global__ void k_scale(C* __restrict__ spec, const T* __restrict__ lam_y, const T* __restrict__ lam_x, T alpha,
                        T norm, int64_t rows, int64_t cols, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i % cols, k = (i / cols) % rows;
        const T g = alpha / (alpha + lam_y[k] + lam_x[l]) * norm;
        spec[i].x *= g;
        spec[i].y *= g;
    }
}

// f = o + first quadrant of ext
template <class T>
__global__ void k_extract(const T* __restrict__ ext, const float* __restrict__ o, float* __restrict__ f, int nx,
                          int ny, int64_t nslices) {
    const int64_t total = nslices * nx * (int64_t)ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / ((int64_t)nx * ny), q = i - j * nx * (int64_t)ny;
        const int64_t y = q / nx, x = q - y * nx;
        f[i] = float(T(o[i]) + ext[(j * 2 * ny + y) * 2 * nx + x]);
    }
}

// cuFFT plans (forward R2C and inverse C2R over a batch), kept per device, size, batch and
// precision until emfuse_release_cache.
struct FftPlans {
    cufftHandle fwd = 0, inv = 0;
    bool ok = false;
    std::mutex mu;  // held around cufftSetStream + exec: one plan, calls on several streams
    ~FftPlans() {
        if (fwd) cufftDestroy(fwd);
        if (inv) cufftDestroy(inv);
    }
};
// key: device, batch, ny, nx, element size
using FftKey = std::tuple<int, int64_t, int64_t, int64_t, int>;
std::mutex g_fft_mu;
std::map<FftKey, std::shared_ptr<FftPlans>>& g_fft = *new std::map<FftKey, std::shared_ptr<FftPlans>>();

int fft_error(const char* what, cufftResult r) {
    set_error(std::string("cuFFT ") + what + " failed (cufftResult " + std::to_string((int)r) + ")");
    return r == CUFFT_ALLOC_FAILED ? EMFUSE_ENOMEM : EMFUSE_ECUDA;
}

// n transforms of 2ny x 2nx (the mirror extensions of n slices)
template <class T>
int get_plans(int64_t nx, int64_t ny, int64_t n, std::shared_ptr<FftPlans>& out) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    const FftKey key = std::make_tuple(dev, n, ny, nx, (int)sizeof(T));
    std::lock_guard<std::mutex> lk(g_fft_mu);
    auto it = g_fft.find(key);
    if (it != g_fft.end()) {
        out = it->second;
        return EMFUSE_OK;
    }
    auto p = std::make_shared<FftPlans>();
    long long dims[2] = {2 * (long long)ny, 2 * (long long)nx};
    const long long rdist = 4LL * nx * ny, cdist = 2LL * ny * (nx + 1);
    size_t work = 0;
    cufftResult r = cufftCreate(&p->fwd);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(p->fwd, 2, dims, nullptr, 1, rdist, nullptr, 1, cdist, Fft<T>::kR2C, n, &work);
    if (r != CUFFT_SUCCESS) return fft_error("forward plan", r);
    r = cufftCreate(&p->inv);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(p->inv, 2, dims, nullptr, 1, cdist, nullptr, 1, rdist, Fft<T>::kC2R, n, &work);
    if (r != CUFFT_SUCCESS) return fft_error("inverse plan", r);
    p->ok = true;
    g_fft[key] = p;
    out = p;
    return EMFUSE_OK;
}

// forward / inverse transform of the batch on stream st (the plan's lock orders callers on
// different streams; the transforms themselves run asynchronously)
template <class T>
cufftResult fft_forward(FftPlans& p, T* in, typename Fft<T>::C* out, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(p.mu);
    cufftResult r = cufftSetStream(p.fwd, st);
    return r == CUFFT_SUCCESS ? Fft<T>::fwd(p.fwd, in, out) : r;
}
template <class T>
cufftResult fft_inverse(FftPlans& p, typename Fft<T>::C* in, T* out, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(p.mu);
    cufftResult r = cufftSetStream(p.inv, st);
    return r == CUFFT_SUCCESS ? Fft<T>::inv(p.inv, in, out) : r;
}

template <class T>
int dct_solve(const float* s, const float* o, float* f, int64_t n, int64_t nx, int64_t ny, double alpha,
              cudaStream_t st) {
    using C = typename Fft<T>::C;
    std::shared_ptr<FftPlans> plans;
    EMF_TRY(get_plans<T>(nx, ny, n, plans));
    const int64_t rows = 2 * ny, cols = nx + 1;
    DeviceBuffer ext, spec, lam;
    EMF_TRY(ext.alloc((size_t)(n * 4 * nx * ny) * sizeof(T), st));
    EMF_TRY(spec.alloc((size_t)(n * rows * cols) * sizeof(C), st));
    // eigenvalues of the periodic 1-D Laplacian on 2ny and 2nx points (FP64 on the host)
    std::vector<T> host((size_t)(rows + cols));
    for (int64_t k = 0; k < rows; ++k) {
        const double sn = std::sin(M_PI * (double)k / (2.0 * (double)ny));
        host[(size_t)k] = T(4.0 * sn * sn);
    }
    for (int64_t l = 0; l < cols; ++l) {
        const double sn = std::sin(M_PI * (double)l / (2.0 * (double)nx));
        host[(size_t)(rows + l)] = T(4.0 * sn * sn);
    }
    EMF_TRY(lam.alloc(host.size() * sizeof(T), st));
    EMF_CUDA(cudaMemcpyAsync(lam.as<T>(), host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    {
        KernelScope ks("dct_mirror", st, (double)n * nx * ny * 8.0 + (double)n * 4 * nx * ny * sizeof(T));
        k_mirror<T><<<grid_of(n * 4 * nx * ny), 256, 0, st>>>(s, o, ext.as<T>(), (int)nx, (int)ny, n);
        EMF_CHECK_LAUNCH();
    }
    cufftResult r = fft_forward<T>(*plans, ext.as<T>(), spec.as<C>(), st);
    if (r != CUFFT_SUCCESS) return fft_error("forward transform", r);
    {
        KernelScope ks("dct_scale", st, (double)n * rows * cols * 2.0 * sizeof(C));
        k_scale<T, C><<<grid_of(n * rows * cols), 256, 0, st>>>(spec.as<C>(), lam.as<T>(), lam.as<T>() + rows,
                                                                 T(alpha), T(1.0 / (4.0 * (double)nx * (double)ny)),
                                                                 rows, cols, n * rows * cols);
        EMF_CHECK_LAUNCH();
    }
    r = fft_inverse<T>(*plans, spec.as<C>(), ext.as<T>(), st);
    if (r != CUFFT_SUCCESS) return fft_error("inverse transform", r);
    {
        KernelScope ks("dct_extract", st, (double)n * nx * ny * (4.0 + 4.0 + sizeof(T)));
        k_extract<T><<<grid_of(n * nx * ny), 256, 0, st>>>(ext.as<T>(), o, f, (int)nx, (int)ny, n);
        EMF_CHECK_LAUNCH();
    }
    // the temporaries go back to the pool stream-ordered; the caller's stream orders f
    return EMFUSE_OK;
}

// ---------------------------------------------------------------- 3-D gradient-domain smoothing
// The smoothing of the earlier method (Sec. 3 "Alternate Solutions"): the stack f minimising
// alpha |f - I0|^2 + |grad_xy f - grad_xy I0|^2 + |d_z f|^2 on the 6-neighbour graph with
// Neumann boundaries, (alpha I + L_xy + L_z) f = alpha I0 + L_xy I0.  In correction form
// f = I0 + d, (alpha I + L_xy + L_z) d = -L_z I0.  The orthonormal DCT-II along z,
// C[k][z] = c_k cos(pi k (2z + 1) / 2nz), diagonalises L_z (eigenvalues lam_z[k] =
// 4 sin^2(pi k / 2nz)), so with I~ = C I0 and d~ = C d (per pixel column) the problem falls
// apart into nz independent slice problems
//     (alpha + lam_z[k]) d~_k + L_xy d~_k = -lam_z[k] I~_k,
// each a screened Poisson equation of the kind of Eq. (1) with its own screening, solved
// exactly by the mirror-extension transform of the 2-D direct solver above.  The two z
// transforms are dense nz x nz contractions over all pixels: cuBLAS GEMMs.

template <class T, class Tin>
__global__ void k_to_type(const Tin* __restrict__ in, T* __restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = T(in[i]);
}

// ext = mirror extension of every slice of x to 2ny x 2nx
template <class T>
__global__ void k_mirror_plain(const T* __restrict__ x, T* __restrict__ ext, int nx, int ny, int64_t nslices) {
    const int64_t NX = 2 * (int64_t)nx, NY = 2 * (int64_t)ny, plane = NX * NY, total = nslices * plane;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / plane, q = i - j * plane;
        const int64_t Y = q / NX, X = q - Y * NX;
        const int64_t y = Y < ny ? Y : NY - 1 - Y, xx = X < nx ? X : NX - 1 - X;
        ext[i] = x[(j * ny + y) * nx + xx];
    }
}

// spectrum of slice k: *= -lam_z[k] / (alpha + lam_z[k] + lam_y[l] + lam_x[m]) / (4 nx ny)
template <class T, class C>
__global__ void k_scale_z(C* __restrict__ spec, const T* __restrict__ lam_z, const T* __restrict__ lam_y,
                          const T* __restrict__ lam_x, T alpha, T norm, int64_t rows, int64_t cols, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i % cols, l = (i / cols) % rows, k = i / (cols * rows);
        const T lz = lam_z[k];
        const T g = -lz / (alpha + lz + lam_y[l] + lam_x[m]) * norm;
        spec[i].x *= g;
        spec[i].y *= g;
    }
}

// x = first quadrant of every extended slice
template <class T>
__global__ void k_quadrant(const T* __restrict__ ext, T* __restrict__ x, int nx, int ny, int64_t nslices) {
    const int64_t total = nslices * nx * (int64_t)ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / ((int64_t)nx * ny), q = i - j * nx * (int64_t)ny;
        const int64_t y = q / nx, xx = q - y * nx;
        x[i] = ext[(j * 2 * ny + y) * 2 * nx + xx];
    }
}

// out = I0 + d
template <class T, class Tin>
__global__ void k_add_out(const Tin* __restrict__ in, const T* __restrict__ d, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = float(T(in[i]) + d[i]);
}

// cuBLAS handles, one per device, kept until emfuse_release_cache (the lock orders callers on
// different streams around cublasSetStream + GEMM)
struct BlasHandle {
    cublasHandle_t h = nullptr;
    std::mutex mu;
    ~BlasHandle() {
        if (h) cublasDestroy(h);
    }
};
std::mutex g_blas_mu;
std::map<int, std::shared_ptr<BlasHandle>>& g_blas = *new std::map<int, std::shared_ptr<BlasHandle>>();

int get_blas(std::shared_ptr<BlasHandle>& out) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_blas_mu);
    auto it = g_blas.find(dev);
    if (it != g_blas.end()) {
        out = it->second;
        return EMFUSE_OK;
    }
    auto b = std::make_shared<BlasHandle>();
    const cublasStatus_t s = cublasCreate(&b->h);
    if (s != CUBLAS_STATUS_SUCCESS) {
        b->h = nullptr;
        set_error("cuBLAS handle creation failed (cublasStatus " + std::to_string((int)s) + ")");
        return s == CUBLAS_STATUS_ALLOC_FAILED ? EMFUSE_ENOMEM : EMFUSE_ECUDA;
    }
    g_blas[dev] = b;
    out = b;
    return EMFUSE_OK;
}

template <class T>
struct Gemm;
template <>
struct Gemm<float> {
    static cublasStatus_t run(cublasHandle_t h, cublasOperation_t tb, int64_t m, int64_t n, const float* A,
                              const float* B, float* Cm) {
        const float one = 1.f, zero = 0.f;
        return cublasSgemm_64(h, CUBLAS_OP_N, tb, m, n, n, &one, A, m, B, n, &zero, Cm, m);
    }
};
template <>
struct Gemm<double> {
    static cublasStatus_t run(cublasHandle_t h, cublasOperation_t tb, int64_t m, int64_t n, const double* A,
                              const double* B, double* Cm) {
        const double one = 1.0, zero = 0.0;
        return cublasDgemm_64(h, CUBLAS_OP_N, tb, m, n, n, &one, A, m, B, n, &zero, Cm, m);
    }
};

// The stack x as [nz][P] row-major is the P x nz column-major matrix X; the row-major DCT
// matrix C[k][z] read column-major is C^T.  Forward: Y = X C^T (Y[k][p] = sum_z C[k][z] x[z][p]);
// inverse: Y = X C (Y[z][p] = sum_k C[k][z] x[k][p]).
template <class T>
int z_transform(BlasHandle& b, const T* x, const T* cmat, T* y, int64_t P, int64_t nz, bool inverse,
                cudaStream_t st) {
    std::lock_guard<std::mutex> lk(b.mu);
    cublasStatus_t s = cublasSetStream(b.h, st);
    if (s == CUBLAS_STATUS_SUCCESS) s = Gemm<T>::run(b.h, inverse ? CUBLAS_OP_T : CUBLAS_OP_N, P, nz, x, cmat, y);
    if (s != CUBLAS_STATUS_SUCCESS) {
        set_error("cuBLAS GEMM of the z transform failed (cublasStatus " + std::to_string((int)s) + ")");
        return EMFUSE_ECUDA;
    }
    return EMFUSE_OK;
}

template <class T, class Tin>
int gd_smooth(const Tin* in, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha, cudaStream_t st) {
    using C = typename Fft<T>::C;
    const int64_t P = nx * ny, N = P * nz;
    const int64_t rows = 2 * ny, cols = nx + 1, ncplx = nz * rows * cols;
    std::shared_ptr<FftPlans> plans;
    std::shared_ptr<BlasHandle> blas;
    EMF_TRY(get_plans<T>(nx, ny, nz, plans));
    EMF_TRY(get_blas(blas));
    DeviceBuffer x, y, ext, spec, tabs;
    EMF_TRY(x.alloc((size_t)N * sizeof(T), st));
    EMF_TRY(y.alloc((size_t)N * sizeof(T), st));
    EMF_TRY(ext.alloc((size_t)(4 * N) * sizeof(T), st));
    EMF_TRY(spec.alloc((size_t)ncplx * sizeof(C), st));
    // the z DCT matrix and the eigenvalues along z (nz points, Neumann) and of the periodic
    // extensions along y and x (2ny and 2nx points), formed in FP64 on the host
    std::vector<T> host((size_t)(nz * nz + nz + rows + cols));
    for (int64_t k = 0; k < nz; ++k) {
        const double ck = std::sqrt((k == 0 ? 1.0 : 2.0) / (double)nz);
        for (int64_t z = 0; z < nz; ++z)
            host[(size_t)(k * nz + z)] = T(ck * std::cos(M_PI * (double)k * (double)(2 * z + 1) / (2.0 * (double)nz)));
    }
    auto eig = [&](size_t at, int64_t count, int64_t n) {
        for (int64_t q = 0; q < count; ++q) {
            const double sn = std::sin(M_PI * (double)q / (2.0 * (double)n));
            host[at + (size_t)q] = T(4.0 * sn * sn);
        }
    };
    eig((size_t)(nz * nz), nz, nz);
    eig((size_t)(nz * nz + nz), rows, ny);
    eig((size_t)(nz * nz + nz + rows), cols, nx);
    EMF_TRY(tabs.alloc(host.size() * sizeof(T), st));
    EMF_CUDA(cudaMemcpyAsync(tabs.as<T>(), host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    const T* cmat = tabs.as<T>();
    const T* lz = cmat + nz * nz;
    const T* ly = lz + nz;
    const T* lx = ly + rows;
    {
        KernelScope ks("gd_convert", st, (double)N * (sizeof(Tin) + sizeof(T)));
        k_to_type<T, Tin><<<grid_of(N), 256, 0, st>>>(in, x.as<T>(), N);
        EMF_CHECK_LAUNCH();
    }
    EMF_TRY(z_transform<T>(*blas, x.as<T>(), cmat, y.as<T>(), P, nz, false, st));
    {
        KernelScope ks("gd_mirror", st, (double)N * 5.0 * sizeof(T));
        k_mirror_plain<T><<<grid_of(4 * N), 256, 0, st>>>(y.as<T>(), ext.as<T>(), (int)nx, (int)ny, nz);
        EMF_CHECK_LAUNCH();
    }
    cufftResult r = fft_forward<T>(*plans, ext.as<T>(), spec.as<C>(), st);
    if (r != CUFFT_SUCCESS) return fft_error("forward transform", r);
    {
        KernelScope ks("gd_scale", st, (double)ncplx * 2.0 * sizeof(C));
        k_scale_z<T, C><<<grid_of(ncplx), 256, 0, st>>>(spec.as<C>(), lz, ly, lx, T(alpha),
                                                         T(1.0 / (4.0 * (double)nx * (double)ny)), rows, cols, ncplx);
        EMF_CHECK_LAUNCH();
    }
    r = fft_inverse<T>(*plans, spec.as<C>(), ext.as<T>(), st);
    if (r != CUFFT_SUCCESS) return fft_error("inverse transform", r);
    {
        KernelScope ks("gd_quadrant", st, (double)N * 2.0 * sizeof(T));
        k_quadrant<T><<<grid_of(N), 256, 0, st>>>(ext.as<T>(), x.as<T>(), (int)nx, (int)ny, nz);
        EMF_CHECK_LAUNCH();
    }
    EMF_TRY(z_transform<T>(*blas, x.as<T>(), cmat, y.as<T>(), P, nz, true, st));
    {
        KernelScope ks("gd_out", st, (double)N * (sizeof(Tin) + sizeof(T) + 4.0));
        k_add_out<T, Tin><<<grid_of(N), 256, 0, st>>>(in, y.as<T>(), out, N);
        EMF_CHECK_LAUNCH();
    }
    return EMFUSE_OK;
}

}  // namespace

int smooth_gradient_domain(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha,
                           int precision, cudaStream_t st) {
    if (dt == EMFUSE_U8) {
        const uint8_t* p = static_cast<const uint8_t*>(in);
        return precision == EMFUSE_PREC_FP32 ? gd_smooth<float>(p, out, nx, ny, nz, alpha, st)
                                             : gd_smooth<double>(p, out, nx, ny, nz, alpha, st);
    }
    const float* p = static_cast<const float*>(in);
    return precision == EMFUSE_PREC_FP32 ? gd_smooth<float>(p, out, nx, ny, nz, alpha, st)
                                         : gd_smooth<double>(p, out, nx, ny, nz, alpha, st);
}

int solve_dct_batch(const float* s, const float* o, float* f, int64_t n, int64_t nx, int64_t ny, double alpha,
                    int precision, cudaStream_t st) {
    return precision == EMFUSE_PREC_FP32 ? dct_solve<float>(s, o, f, n, nx, ny, alpha, st)
                                         : dct_solve<double>(s, o, f, n, nx, ny, alpha, st);
}

void release_fft_plans() {
    {
        std::lock_guard<std::mutex> lk(g_fft_mu);
        g_fft.clear();
    }
    std::lock_guard<std::mutex> lk(g_blas_mu);
    g_blas.clear();
}

}  // namespace emfuse
