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
    ~FftPlans() {
        if (fwd) cufftDestroy(fwd);
        if (inv) cufftDestroy(inv);
    }
};
// key: device, rank (2: a batch of slices, 3: one volume), three extents (batch or nz, ny,
// nx), element size
using FftKey = std::tuple<int, int, int64_t, int64_t, int64_t, int>;
std::mutex g_fft_mu;
std::map<FftKey, std::shared_ptr<FftPlans>>& g_fft = *new std::map<FftKey, std::shared_ptr<FftPlans>>();

int fft_error(const char* what, cufftResult r) {
    set_error(std::string("cuFFT ") + what + " failed (cufftResult " + std::to_string((int)r) + ")");
    return r == CUFFT_ALLOC_FAILED ? EMFUSE_ENOMEM : EMFUSE_ECUDA;
}

// rank 2: n transforms of 2ny x 2nx; rank 3: one transform of 2nz x 2ny x 2nx (n = nz)
template <class T>
int get_plans(int rank, int64_t nx, int64_t ny, int64_t n, std::shared_ptr<FftPlans>& out) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    const FftKey key = std::make_tuple(dev, rank, n, ny, nx, (int)sizeof(T));
    std::lock_guard<std::mutex> lk(g_fft_mu);
    auto it = g_fft.find(key);
    if (it != g_fft.end()) {
        out = it->second;
        return EMFUSE_OK;
    }
    auto p = std::make_shared<FftPlans>();
    long long dims[3] = {2 * (long long)n, 2 * (long long)ny, 2 * (long long)nx};
    long long* d = rank == 3 ? dims : dims + 1;
    const long long batch = rank == 3 ? 1 : n;
    const long long rdist = (rank == 3 ? 2LL * n : 1LL) * 4LL * nx * ny;
    const long long cdist = (rank == 3 ? 2LL * n : 1LL) * 2LL * ny * (nx + 1);
    size_t work = 0;
    cufftResult r = cufftCreate(&p->fwd);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(p->fwd, rank, d, nullptr, 1, rdist, nullptr, 1, cdist, Fft<T>::kR2C, batch, &work);
    if (r != CUFFT_SUCCESS) return fft_error("forward plan", r);
    r = cufftCreate(&p->inv);
    if (r == CUFFT_SUCCESS)
        r = cufftMakePlanMany64(p->inv, rank, d, nullptr, 1, cdist, nullptr, 1, rdist, Fft<T>::kC2R, batch, &work);
    if (r != CUFFT_SUCCESS) return fft_error("inverse plan", r);
    p->ok = true;
    g_fft[key] = p;
    out = p;
    return EMFUSE_OK;
}

template <class T>
int dct_solve(const float* s, const float* o, float* f, int64_t n, int64_t nx, int64_t ny, double alpha,
              cudaStream_t st) {
    using C = typename Fft<T>::C;
    std::shared_ptr<FftPlans> plans;
    EMF_TRY(get_plans<T>(2, nx, ny, n, plans));
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
    cufftResult r = cufftSetStream(plans->fwd, st);
    if (r == CUFFT_SUCCESS) r = Fft<T>::fwd(plans->fwd, ext.as<T>(), spec.as<C>());
    if (r != CUFFT_SUCCESS) return fft_error("forward transform", r);
    {
        KernelScope ks("dct_scale", st, (double)n * rows * cols * 2.0 * sizeof(C));
        k_scale<T, C><<<grid_of(n * rows * cols), 256, 0, st>>>(spec.as<C>(), lam.as<T>(), lam.as<T>() + rows,
                                                                 T(alpha), T(1.0 / (4.0 * (double)nx * (double)ny)),
                                                                 rows, cols, n * rows * cols);
        EMF_CHECK_LAUNCH();
    }
    r = cufftSetStream(plans->inv, st);
    if (r == CUFFT_SUCCESS) r = Fft<T>::inv(plans->inv, spec.as<C>(), ext.as<T>());
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
// f = I0 + d, (alpha I + L) d = -L_z I0, and on the mirror extension of the stack to
// 2nz x 2ny x 2nx (periodic, so one 3-D FFT diagonalises L):
//     d = first octant of IFFT( FFT(mirror(I0)) * (-lam_z) / (alpha + lam_z + lam_y + lam_x) ).

// ext = mirror extension of I0 (uint8 or float) to 2nz x 2ny x 2nx
template <class T, class Tin>
__global__ void k_mirror3(const Tin* __restrict__ in, T* __restrict__ ext, int64_t nx, int64_t ny, int64_t nz) {
    const int64_t NX = 2 * nx, NY = 2 * ny, NZ = 2 * nz, total = NX * NY * NZ;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t Z = i / (NX * NY), q = i - Z * NX * NY;
        const int64_t Y = q / NX, X = q - Y * NX;
        const int64_t z = Z < nz ? Z : NZ - 1 - Z, y = Y < ny ? Y : NY - 1 - Y, x = X < nx ? X : NX - 1 - X;
        ext[i] = T(in[(z * ny + y) * nx + x]);
    }
}

// spec(k, l, m) *= -lam_z[k] / (alpha + lam_z[k] + lam_y[l] + lam_x[m]) / (8 nx ny nz)
template <class T, class C>
__global__ void k_scale3(C* __restrict__ spec, const T* __restrict__ lam_z, const T* __restrict__ lam_y,
                         const T* __restrict__ lam_x, T alpha, T norm, int64_t NY, int64_t cols, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i % cols, l = (i / cols) % NY, k = i / (cols * NY);
        const T lz = lam_z[k];
        const T g = -lz / (alpha + lz + lam_y[l] + lam_x[m]) * norm;
        spec[i].x *= g;
        spec[i].y *= g;
    }
}

// out = I0 + first octant of ext
template <class T, class Tin>
__global__ void k_extract3(const T* __restrict__ ext, const Tin* __restrict__ in, float* __restrict__ out,
                           int64_t nx, int64_t ny, int64_t nz) {
    const int64_t total = nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = i / (nx * ny), q = i - z * nx * ny;
        const int64_t y = q / nx, x = q - y * nx;
        out[i] = float(T(in[i]) + ext[(z * 2 * ny + y) * 2 * nx + x]);
    }
}

template <class T, class Tin>
int gd_smooth(const Tin* in, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha, cudaStream_t st) {
    using C = typename Fft<T>::C;
    std::shared_ptr<FftPlans> plans;
    EMF_TRY(get_plans<T>(3, nx, ny, nz, plans));
    const int64_t NZ = 2 * nz, NY = 2 * ny, cols = nx + 1;
    const int64_t nreal = NZ * NY * 2 * nx, ncplx = NZ * NY * cols;
    DeviceBuffer ext, spec, lam;
    EMF_TRY(ext.alloc((size_t)nreal * sizeof(T), st));
    EMF_TRY(spec.alloc((size_t)ncplx * sizeof(C), st));
    // eigenvalues of the periodic 1-D Laplacian on 2nz, 2ny and 2nx points (FP64 on the host)
    std::vector<T> host((size_t)(NZ + NY + cols));
    auto fill = [&](size_t at, int64_t count, int64_t n) {
        for (int64_t k = 0; k < count; ++k) {
            const double sn = std::sin(M_PI * (double)k / (2.0 * (double)n));
            host[at + (size_t)k] = T(4.0 * sn * sn);
        }
    };
    fill(0, NZ, nz);
    fill((size_t)NZ, NY, ny);
    fill((size_t)(NZ + NY), cols, nx);
    EMF_TRY(lam.alloc(host.size() * sizeof(T), st));
    EMF_CUDA(cudaMemcpyAsync(lam.as<T>(), host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    const T* lz = lam.as<T>();
    {
        KernelScope ks("gd_mirror", st, (double)nx * ny * nz * sizeof(Tin) + (double)nreal * sizeof(T));
        k_mirror3<T, Tin><<<grid_of(nreal), 256, 0, st>>>(in, ext.as<T>(), nx, ny, nz);
        EMF_CHECK_LAUNCH();
    }
    cufftResult r = cufftSetStream(plans->fwd, st);
    if (r == CUFFT_SUCCESS) r = Fft<T>::fwd(plans->fwd, ext.as<T>(), spec.as<C>());
    if (r != CUFFT_SUCCESS) return fft_error("forward transform", r);
    {
        KernelScope ks("gd_scale", st, (double)ncplx * 2.0 * sizeof(C));
        k_scale3<T, C><<<grid_of(ncplx), 256, 0, st>>>(spec.as<C>(), lz, lz + NZ, lz + NZ + NY, T(alpha),
                                                        T(1.0 / (8.0 * (double)nx * (double)ny * (double)nz)), NY,
                                                        cols, ncplx);
        EMF_CHECK_LAUNCH();
    }
    r = cufftSetStream(plans->inv, st);
    if (r == CUFFT_SUCCESS) r = Fft<T>::inv(plans->inv, spec.as<C>(), ext.as<T>());
    if (r != CUFFT_SUCCESS) return fft_error("inverse transform", r);
    {
        KernelScope ks("gd_extract", st, (double)nx * ny * nz * (sizeof(Tin) + 4.0 + sizeof(T)));
        k_extract3<T, Tin><<<grid_of(nx * ny * nz), 256, 0, st>>>(ext.as<T>(), in, out, nx, ny, nz);
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
    std::lock_guard<std::mutex> lk(g_fft_mu);
    g_fft.clear();
}

}  // namespace emfuse
