// Phase 2 of the method: per-slice screened-Poisson solve of Eq. (1),
//     (alpha I + L) f = alpha s + L o,    L = -Lap (5-point, Neumann),
// by multigrid V-cycles inside a defect-correction loop (Sec. 3 "Implementation" uses a
// multigrid solver; its internals are not given, the choices below are this library's).
//
// Outer loop (per batch of slices, all slices advance together, converged ones are masked):
//     f = o
//     repeat:  r = b - A f            (residual kernel, arithmetic in TF: FP64 when mixed)
//              stop if ||r|| / ||b|| <= tol for every slice
//              e = Vcycle(A e = r)     (arithmetic in TV: FP32 when mixed, from e = 0)
//              f += e
//
// Multigrid hierarchy: level k has ceil(n/2^k) cells per axis, down to 1 x 1.  Cell I of
// level k covers fine pixels [I 2^k, min((I+1) 2^k, n)); only the last cell of an axis can be
// partial.  The level-k operator is the finite-volume rediscretisation on those true cells,
// scaled by 4^-k:
//     (A_k u)_p = alpha wx wy u_p + 4^-k sum_faces c_pq (u_p - u_q),
//     c_x = wy * 2 / (wx_I + wx_I+1),  c_y = wx * 2 / (wy_J + wy_J+1),
// with w the cell widths in level units (1 for full cells).  Interior cells give the usual
// alpha + L/4^k.  Restriction sums the (at most 4) child residuals and divides by 4;
// prolongation interpolates linearly between true cell centres.  Smoother: red-black
// Gauss-Seidel, colour (x + y) mod 2, nu_pre / nu_post sweeps.  The 1 x 1 coarsest level is
// solved exactly by one sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"
#include "mg_fused.cuh"

namespace emfuse {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;

__device__ __forceinline__ int find_slice(const int64_t* __restrict__ ts, int n, int64_t t) {
    int lo = 0, hi = n;  // ts[0] = 0 <= t < ts[n]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ts[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

template <class T>
struct LevelArgs {
    const LSlice<T>* sl;
    const int64_t* tile_start;
    int nsl;
    int k;
    T alpha;
    T sk;          // 4^-k
    const int* active;
};

// ---------------------------------------------------------------- reference kernels
template <class T>
__global__ void __launch_bounds__(kBX* kBY) k_relax(LevelArgs<T> a, int color) {
    const int64_t t = blockIdx.x;
    const int j = find_slice(a.tile_start, a.nsl, t);
    const LSlice<T> S = a.sl[j];
    if (a.active && !a.active[S.slice]) return;
    const int lt = int(t - a.tile_start[j]);
    const int x = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int y = (lt / S.tiles_x) * kBY + threadIdx.y;
    if (x >= S.nx || y >= S.ny || ((x + y) & 1) != color) return;
    const Coef<T> c = coef_at<T>(x, y, S.nx, S.ny, S.n0x, S.n0y, a.k, a.alpha, a.sk);
    T* u = S.u;
    const int64_t p = (int64_t)y * S.pitch + x;
    const T uw = x > 0 ? u[p - 1] : T(0);
    const T ue = x + 1 < S.nx ? u[p + 1] : T(0);
    const T un = y > 0 ? u[p - S.pitch] : T(0);
    const T us = y + 1 < S.ny ? u[p + S.pitch] : T(0);
    u[p] = gs_update(c, S.b[p], uw, ue, un, us);
}

// Launched over the tiles of level k (coarse); reads level k-1 (fine).
template <class T>
__global__ void __launch_bounds__(kBX* kBY) k_residual_restrict(LevelArgs<T> a, T sk_fine) {
    const int64_t t = blockIdx.x;
    const int j = find_slice(a.tile_start, a.nsl, t);
    const LSlice<T> S = a.sl[j];
    if (a.active && !a.active[S.slice]) return;
    const int lt = int(t - a.tile_start[j]);
    const int I = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int J = (lt / S.tiles_x) * kBY + threadIdx.y;
    if (I >= S.nx || J >= S.ny) return;
    T sum = T(0);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int x = 2 * I + dx, y = 2 * J + dy;
            if (x < S.nfx && y < S.nfy) {
                const Coef<T> c = coef_at<T>(x, y, S.nfx, S.nfy, S.n0x, S.n0y, a.k - 1, a.alpha, sk_fine);
                const T* u = S.uf;
                const int64_t p = (int64_t)y * S.pitchf + x;
                const T uw = x > 0 ? u[p - 1] : T(0);
                const T ue = x + 1 < S.nfx ? u[p + 1] : T(0);
                const T un = y > 0 ? u[p - S.pitchf] : T(0);
                const T us = y + 1 < S.nfy ? u[p + S.pitchf] : T(0);
                sum += residual_at(c, S.bf[p], u[p], uw, ue, un, us);
            }
        }
    const int64_t q = (int64_t)J * S.pitch + I;
    S.b[q] = sum * T(0.25);
    S.u[q] = T(0);
}

// Launched over the tiles of level k (fine); adds the interpolated level-(k+1) correction.
template <class T>
__global__ void __launch_bounds__(kBX* kBY) k_prolong_add(LevelArgs<T> a) {
    const int64_t t = blockIdx.x;
    const int j = find_slice(a.tile_start, a.nsl, t);
    const LSlice<T> S = a.sl[j];
    if (!S.uc) return;
    if (a.active && !a.active[S.slice]) return;
    const int lt = int(t - a.tile_start[j]);
    const int x = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int y = (lt / S.tiles_x) * kBY + threadIdx.y;
    if (x >= S.nx || y >= S.ny) return;
    S.u[(int64_t)y * S.pitch + x] += prolong_at<T>(S.uc, S.pitchc, x, y, S.ncx, S.ncy, S.n0x, S.n0y, a.k);
}

// ---------------------------------------------------------------- finest-level kernels
struct TopSlice {
    int64_t off;   // element offset of the slice in the packed s / o / f / out buffers
    int nx, ny;
};

template <class TF, class TV, class To>
__global__ void __launch_bounds__(kBX* kBY)
k_residual_top(LevelArgs<TV> a, const TopSlice* __restrict__ top, const float* __restrict__ s,
               const To* __restrict__ o, const float* __restrict__ rhs, const TF* __restrict__ f,
               double alpha, double* __restrict__ norms) {
    const int64_t t = blockIdx.x;
    const int j = find_slice(a.tile_start, a.nsl, t);
    const LSlice<TV> S = a.sl[j];
    if (a.active && !a.active[S.slice]) return;
    const TopSlice G = top[S.slice];
    const int lt = int(t - a.tile_start[j]);
    const int x = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int y = (lt / S.tiles_x) * kBY + threadIdx.y;
    double rr = 0.0, bb = 0.0;
    if (x < S.nx && y < S.ny) {
        const int64_t p = G.off + (int64_t)y * G.nx + x;
        const bool hw = x > 0, he = x + 1 < G.nx, hn = y > 0, hs = y + 1 < G.ny;
        const TF deg = TF(int(hw) + int(he) + int(hn) + int(hs));
        TF b;
        if (rhs) {
            b = TF(rhs[p]);
        } else {
            const TF oc = TF(o[p]);
            TF Lo = deg * oc;
            if (hw) Lo -= TF(o[p - 1]);
            if (he) Lo -= TF(o[p + 1]);
            if (hn) Lo -= TF(o[p - G.nx]);
            if (hs) Lo -= TF(o[p + G.nx]);
            b = TF(alpha) * TF(s[p]) + Lo;
        }
        const TF fc = f[p];
        TF Lf = deg * fc;
        if (hw) Lf -= f[p - 1];
        if (he) Lf -= f[p + 1];
        if (hn) Lf -= f[p - G.nx];
        if (hs) Lf -= f[p + G.nx];
        const TF r = b - (TF(alpha) * fc + Lf);
        const int64_t q = (int64_t)y * S.pitch + x;
        S.b[q] = TV(r);
        S.u[q] = TV(0);
        rr = double(r) * double(r);
        bb = double(b) * double(b);
    }
    // block reduction in FP64: warp shuffles, then one atomic pair per block
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, m);
        bb += __shfl_xor_sync(0xffffffffu, bb, m);
    }
    __shared__ double red[2][kBY];
    if (threadIdx.x == 0) { red[0][threadIdx.y] = rr; red[1][threadIdx.y] = bb; }
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.x == 0) {
        double r2 = 0.0, b2 = 0.0;
        for (int w = 0; w < kBY; ++w) { r2 += red[0][w]; b2 += red[1][w]; }
        atomicAdd(&norms[2 * S.slice], r2);
        atomicAdd(&norms[2 * S.slice + 1], b2);
    }
}

template <class TF, class TV>
__global__ void __launch_bounds__(kBX* kBY)
k_update_top(LevelArgs<TV> a, const TopSlice* __restrict__ top, TF* __restrict__ f) {
    const int64_t t = blockIdx.x;
    const int j = find_slice(a.tile_start, a.nsl, t);
    const LSlice<TV> S = a.sl[j];
    if (a.active && !a.active[S.slice]) return;
    const TopSlice G = top[S.slice];
    const int lt = int(t - a.tile_start[j]);
    const int x = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int y = (lt / S.tiles_x) * kBY + threadIdx.y;
    if (x >= S.nx || y >= S.ny) return;
    f[G.off + (int64_t)y * G.nx + x] += TF(S.u[(int64_t)y * S.pitch + x]);
}

template <class TF, class To>
__global__ void k_init_f(TF* __restrict__ f, const To* __restrict__ o, int64_t n, int zero) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f[i] = zero ? TF(0) : TF(o[i]);
}

__global__ void k_store(const double* __restrict__ f, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = float(f[i]);
}

inline unsigned grid_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)kNumSMs * 16));
}

// ---------------------------------------------------------------- host-side plan
template <class T>
struct LevelPlan {
    std::vector<LSlice<T>> sl;
    std::vector<int64_t> tile_start;   // size nsl + 1
    LSlice<T>* d_sl = nullptr;
    int64_t* d_ts = nullptr;
    int k = 0;
    double cells = 0;   // cells of this level summed over its slices
    int64_t ntiles() const { return tile_start.empty() ? 0 : tile_start.back(); }
};

inline int num_levels(int64_t nx, int64_t ny) {
    int K = 0;
    while (level_size((int)nx, K) > 1 || level_size((int)ny, K) > 1) ++K;
    return K + 1;
}

template <class TF, class TV>
struct Solver {
    const SolveRequest& req;
    cudaStream_t st;
    std::vector<LevelPlan<TV>> levels;
    DeviceBuffer ws_levels, ws_desc, ws_f, ws_norms, ws_active, ws_top;
    std::vector<int> nlev;
    int Kmax = 0;
    TF* f = nullptr;
    double* d_norms = nullptr;
    int* d_active = nullptr;
    TopSlice* d_top = nullptr;

    Solver(const SolveRequest& r, cudaStream_t s) : req(r), st(s) {}

    int build() {
        const int64_t n = req.nslices;
        nlev.resize(n);
        for (int64_t j = 0; j < n; ++j) {
            nlev[j] = num_levels(req.nx[j], req.ny[j]);
            Kmax = std::max(Kmax, nlev[j]);
        }
        // level arrays: u and b of every slice and level, rows padded to 128 bytes
        const int64_t align = 128 / (int64_t)sizeof(TV);
        std::vector<std::vector<int64_t>> off(n);
        int64_t total = 0;
        for (int64_t j = 0; j < n; ++j) {
            off[j].resize(nlev[j]);
            for (int k = 0; k < nlev[j]; ++k) {
                const int64_t lx = level_size((int)req.nx[j], k), ly = level_size((int)req.ny[j], k);
                off[j][k] = total;
                total += 2 * round_up(lx, align) * ly;
            }
        }
        EMF_TRY(ws_levels.alloc((size_t)total * sizeof(TV), st));
        TV* base = ws_levels.as<TV>();
        levels.resize(Kmax);
        for (int k = 0; k < Kmax; ++k) {
            LevelPlan<TV>& L = levels[k];
            L.k = k;
            L.tile_start.push_back(0);
            for (int64_t j = 0; j < n; ++j) {
                if (nlev[j] <= k) continue;
                LSlice<TV> S{};
                const int n0x = (int)req.nx[j], n0y = (int)req.ny[j];
                S.nx = level_size(n0x, k);
                S.ny = level_size(n0y, k);
                S.pitch = (int)round_up(S.nx, align);
                S.u = base + off[j][k];
                S.b = S.u + (int64_t)S.pitch * S.ny;
                if (k + 1 < nlev[j]) {
                    S.ncx = level_size(n0x, k + 1);
                    S.ncy = level_size(n0y, k + 1);
                    S.pitchc = (int)round_up(S.ncx, align);
                    S.uc = base + off[j][k + 1];
                }
                if (k > 0) {
                    S.nfx = level_size(n0x, k - 1);
                    S.nfy = level_size(n0y, k - 1);
                    S.pitchf = (int)round_up(S.nfx, align);
                    S.uf = base + off[j][k - 1];
                    S.bf = S.uf + (int64_t)S.pitchf * S.nfy;
                }
                S.n0x = n0x;
                S.n0y = n0y;
                S.slice = (int)j;
                S.tiles_x = (int)ceil_div(S.nx, kBX);
                const int64_t tiles = (int64_t)S.tiles_x * ceil_div(S.ny, kBY);
                L.sl.push_back(S);
                L.tile_start.push_back(L.tile_start.back() + tiles);
                L.cells += (double)S.nx * S.ny;
            }
        }
        // descriptors: one upload of all levels
        size_t bytes = 0;
        for (auto& L : levels) bytes += round_up(L.sl.size() * sizeof(LSlice<TV>), 256) + round_up(L.tile_start.size() * 8, 256);
        std::vector<char> blob(bytes);
        EMF_TRY(ws_desc.alloc(bytes, st));
        size_t pos = 0;
        for (auto& L : levels) {
            std::memcpy(blob.data() + pos, L.sl.data(), L.sl.size() * sizeof(LSlice<TV>));
            L.d_sl = reinterpret_cast<LSlice<TV>*>(ws_desc.as<char>() + pos);
            pos += round_up(L.sl.size() * sizeof(LSlice<TV>), 256);
            std::memcpy(blob.data() + pos, L.tile_start.data(), L.tile_start.size() * 8);
            L.d_ts = reinterpret_cast<int64_t*>(ws_desc.as<char>() + pos);
            pos += round_up(L.tile_start.size() * 8, 256);
        }
        EMF_CUDA(cudaMemcpyAsync(ws_desc.as<char>(), blob.data(), bytes, cudaMemcpyHostToDevice, st));
        std::vector<TopSlice> top(n);
        for (int64_t j = 0; j < n; ++j) top[j] = TopSlice{req.offsets[j], (int)req.nx[j], (int)req.ny[j]};
        EMF_TRY(ws_top.alloc(n * sizeof(TopSlice), st));
        EMF_CUDA(cudaMemcpyAsync(ws_top.as<TopSlice>(), top.data(), n * sizeof(TopSlice), cudaMemcpyHostToDevice, st));
        d_top = ws_top.as<TopSlice>();
        EMF_TRY(ws_norms.alloc(2 * n * sizeof(double), st));
        d_norms = ws_norms.as<double>();
        EMF_TRY(ws_active.alloc(n * sizeof(int), st));
        d_active = ws_active.as<int>();
        EMF_CUDA(cudaStreamSynchronize(st));  // host staging vectors go out of scope
        return EMFUSE_OK;
    }

    LevelArgs<TV> args(int k) const {
        LevelArgs<TV> a;
        a.sl = levels[k].d_sl;
        a.tile_start = levels[k].d_ts;
        a.nsl = (int)levels[k].sl.size();
        a.k = k;
        a.alpha = TV(req.alpha);
        a.sk = TV(std::ldexp(1.0, -2 * k));
        a.active = d_active;
        return a;
    }

    int relax(int k, int sweeps) {
        const auto a = args(k);
        const unsigned g = (unsigned)levels[k].ntiles();
        // a half-sweep reads the other colour and b of its colour, writes its colour
        const double bytes = 1.5 * sizeof(TV) * levels[k].cells;
        for (int s = 0; s < sweeps; ++s)
            for (int color = 0; color < 2; ++color) {
                KernelScope ks(k == 0 ? "relax_l0" : "relax_coarse", st, bytes);
                k_relax<TV><<<g, dim3(kBX, kBY), 0, st>>>(a, color);
                EMF_CHECK_LAUNCH();
            }
        return EMFUSE_OK;
    }

    int vcycle() {
        const int nu1 = req.opts.nu_pre, nu2 = req.opts.nu_post;
        for (int k = 0; k < Kmax; ++k) {
            EMF_TRY(relax(k, nu1));
            if (k + 1 < Kmax) {
                const auto a = args(k + 1);
                const double bytes = sizeof(TV) * (2.0 * levels[k].cells + 2.0 * levels[k + 1].cells);
                KernelScope ks(k == 0 ? "restrict_l0" : "restrict_coarse", st, bytes);
                k_residual_restrict<TV><<<(unsigned)levels[k + 1].ntiles(), dim3(kBX, kBY), 0, st>>>(
                    a, TV(std::ldexp(1.0, -2 * k)));
                EMF_CHECK_LAUNCH();
            }
        }
        for (int k = Kmax - 2; k >= 0; --k) {
            {
                const double bytes = sizeof(TV) * (2.0 * levels[k].cells + levels[k + 1].cells);
                KernelScope ks(k == 0 ? "prolong_l0" : "prolong_coarse", st, bytes);
                k_prolong_add<TV><<<(unsigned)levels[k].ntiles(), dim3(kBX, kBY), 0, st>>>(args(k));
                EMF_CHECK_LAUNCH();
            }
            EMF_TRY(relax(k, nu2));
        }
        return EMFUSE_OK;
    }

    template <class To>
    int run(const To* o) {
        EMF_TRY(build());
        const int64_t n = req.nslices;
        int64_t total = 0;
        for (int64_t j = 0; j < n; ++j) total = std::max(total, req.offsets[j] + req.nx[j] * req.ny[j]);
        if (std::is_same<TF, float>::value) {
            f = reinterpret_cast<TF*>(req.out);
        } else {
            EMF_TRY(ws_f.alloc((size_t)total * sizeof(TF), st));
            f = ws_f.as<TF>();
        }
        {
            KernelScope ks("init_iterate", st, (double)total * (sizeof(TF) + (req.rhs ? 0 : sizeof(To))));
            k_init_f<TF, To><<<grid_for(total, 256), 256, 0, st>>>(f, o, total, req.rhs ? 1 : 0);
            EMF_CHECK_LAUNCH();
        }

        std::vector<int> active(n, 1), vcycles(n, 0);
        std::vector<double> norms(2 * n), rel(n, 0.0), bnorm(n, 0.0);
        std::vector<char> done(n, 0);
        EMF_CUDA(cudaMemcpyAsync(d_active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        const int maxit = std::max(0, req.opts.max_vcycles);
        bool all_done = false;
        for (int it = 0;; ++it) {
            EMF_CUDA(cudaMemsetAsync(d_norms, 0, 2 * n * sizeof(double), st));
            {
                const double in_b = req.rhs ? 4.0 : 4.0 + sizeof(To);
                KernelScope ks("residual_top", st, levels[0].cells * (in_b + sizeof(TF) + 2.0 * sizeof(TV)));
                k_residual_top<TF, TV, To><<<(unsigned)levels[0].ntiles(), dim3(kBX, kBY), 0, st>>>(
                    args(0), d_top, req.s, o, req.rhs, f, req.alpha, d_norms);
                EMF_CHECK_LAUNCH();
            }
            EMF_CUDA(cudaMemcpyAsync(norms.data(), d_norms, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
            EMF_CUDA(cudaStreamSynchronize(st));
            all_done = true;
            for (int64_t j = 0; j < n; ++j) {
                if (done[j]) continue;
                const double rr = norms[2 * j], bb = norms[2 * j + 1];
                bnorm[j] = std::sqrt(bb);
                rel[j] = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
                if (rel[j] <= req.opts.tol || !std::isfinite(rel[j])) {
                    done[j] = 1;
                    active[j] = 0;
                } else {
                    all_done = false;
                }
            }
            if (all_done || it >= maxit) break;
            EMF_CUDA(cudaMemcpyAsync(d_active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
            EMF_TRY(vcycle());
            {
                KernelScope ks("update_top", st, levels[0].cells * (2.0 * sizeof(TF) + sizeof(TV)));
                k_update_top<TF, TV><<<(unsigned)levels[0].ntiles(), dim3(kBX, kBY), 0, st>>>(args(0), d_top, f);
                EMF_CHECK_LAUNCH();
            }
            for (int64_t j = 0; j < n; ++j)
                if (active[j]) ++vcycles[j];
        }
        if (!std::is_same<TF, float>::value) {
            KernelScope ks("store_output", st, (double)total * 12.0);
            k_store<<<grid_for(total, 256), 256, 0, st>>>(reinterpret_cast<const double*>(f), req.out, total);
            EMF_CHECK_LAUNCH();
        }
        bool nonfinite = false;
        if (req.stats) {
            for (int64_t j = 0; j < n; ++j) {
                req.stats[j].vcycles = vcycles[j];
                req.stats[j].rel_residual = rel[j];
                req.stats[j].b_norm = bnorm[j];
                req.stats[j].converged = rel[j] <= req.opts.tol ? 1 : 0;
            }
        }
        for (int64_t j = 0; j < n; ++j) nonfinite |= !std::isfinite(rel[j]);
        EMF_CUDA(cudaStreamSynchronize(st));
        if (nonfinite) {
            set_error("non-finite residual (NaN or Inf in the inputs?)");
            return EMFUSE_EINVAL;
        }
        if (!all_done) {
            set_error("tolerance not reached within max_vcycles");
            return EMFUSE_ENOCONV;
        }
        return EMFUSE_OK;
    }
};

template <class TF, class TV>
int run_precision(const SolveRequest& req, cudaStream_t st) {
    Solver<TF, TV> solver(req, st);
    if (req.rhs || req.o_dtype == EMFUSE_F32) return solver.run(static_cast<const float*>(req.o));
    return solver.run(static_cast<const uint8_t*>(req.o));
}

// ---------------------------------------------------------------- adjoint helpers
__global__ void k_laplacian(const float* __restrict__ in, float* __restrict__ out, int64_t nx,
                            int64_t ny, int64_t nz, float scale) {
    const int64_t n = nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = i % nx, y = (i / nx) % ny;
        const float c = in[i];
        float acc = 0.f;
        if (x > 0) acc += c - in[i - 1];
        if (x + 1 < nx) acc += c - in[i + 1];
        if (y > 0) acc += c - in[i - nx];
        if (y + 1 < ny) acc += c - in[i + nx];
        out[i] = scale * acc;
    }
}

__global__ void k_dot_diff(const float* __restrict__ a, const float* __restrict__ b,
                           const float* __restrict__ c, int64_t n, double* __restrict__ acc) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += double(a[i]) * (double(b[i]) - (c ? double(c[i]) : 0.0));
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(acc, t);
    }
}

__global__ void k_axpy(const float* __restrict__ x, float* __restrict__ y, int64_t n, float a, int overwrite) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = overwrite ? a * x[i] : fmaf(a, x[i], y[i]);
}

}  // namespace

int solve_batch(const SolveRequest& req, cudaStream_t st) {
    switch (req.opts.precision) {
        case EMFUSE_PREC_FP32: return run_precision<float, float>(req, st);
        case EMFUSE_PREC_MIXED: return run_precision<double, float>(req, st);
        case EMFUSE_PREC_FP64: return run_precision<double, double>(req, st);
        default: set_error("unknown precision mode"); return EMFUSE_EINVAL;
    }
}

int apply_laplacian_stack(const float* in, float* out, int64_t nx, int64_t ny, int64_t nz,
                          float scale, cudaStream_t st) {
    KernelScope ks("laplacian", st, 8.0 * nx * ny * nz);
    k_laplacian<<<grid_for(nx * ny * nz, 256), 256, 0, st>>>(in, out, nx, ny, nz, scale);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

int dot_diff(const float* a, const float* b, const float* c, int64_t n, double* host_out, cudaStream_t st) {
    DeviceBuffer acc;
    EMF_TRY(acc.alloc(sizeof(double), st));
    EMF_CUDA(cudaMemsetAsync(acc.as<double>(), 0, sizeof(double), st));
    {
        KernelScope ks("dot_diff", st, (c ? 12.0 : 8.0) * n);
        k_dot_diff<<<grid_for(n, 256), 256, 0, st>>>(a, b, c, n, acc.as<double>());
        EMF_CHECK_LAUNCH();
    }
    EMF_CUDA(cudaMemcpyAsync(host_out, acc.as<double>(), sizeof(double), cudaMemcpyDeviceToHost, st));
    EMF_CUDA(cudaStreamSynchronize(st));
    return EMFUSE_OK;
}

int scale_copy(const float* in, float* out, int64_t n, float a, cudaStream_t st) {
    KernelScope ks("scale_copy", st, 8.0 * n);
    k_axpy<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, a, 1);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

int axpy(const float* x, float* y, int64_t n, float a, cudaStream_t st) {
    KernelScope ks("axpy", st, 12.0 * n);
    k_axpy<<<grid_for(n, 256), 256, 0, st>>>(x, y, n, a, 0);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

}  // namespace emfuse
