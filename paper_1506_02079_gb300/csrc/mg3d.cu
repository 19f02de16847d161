// 3-D multigrid for the gradient-domain smoothing of the earlier method (Sec. 3 "Alternate
// Solutions": the target gradient field is the stack's gradient with its z-components set to
// zero), screened as in Eq. (1):
//     (alpha I + L_xy + L_z) f = alpha I0 + L_xy I0
// on the 6-neighbour graph of the stack (Neumann boundaries, unit spacing on every axis).  The
// paper solved this problem with a streaming multigrid; this is a multigrid on the stack held in
// HBM, the 3-D counterpart of the slice solver:
//   * correction form f = I0 + d, so the right-hand side of the correction equation is
//     alpha I0 + L_xy I0 - A I0 = -L_z I0 (z differences only), and A d = -L_z I0;
//   * cell-centred coarsening to 1 x 1 x 1 (an axis that reaches one cell stays at one), the
//     finite-volume operator of each level on its true (possibly partial) cells, face
//     coefficients 2 / (w_I + w_{I+1}) times the face area, scaled by 4^-k;
//   * restriction: the sum of the (up to 8) child residuals / 8; prolongation: trilinear
//     interpolation between true cell centres; red-black Gauss-Seidel (colour = parity of
//     x + y + z) with nu_pre / nu_post sweeps;
//   * V-cycles in FP32 on the correction equation, outer defect-correction passes in FP64:
//     d += e, r = -L_z I0 - A d (every operation and the norms in FP64), out = I0 + d, until
//     ||r|| / ||alpha I0 + L_xy I0|| <= tol.
// One thread per cell (one per cell of the updated colour in the relaxation); the level-0
// passes are HBM bound.  The host checks the residual norm after every defect pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"
#include "fpconv.cuh"
#include "mg_fused.cuh"

namespace emfuse {
namespace {

constexpr int kThreads3 = 256;

struct Lev3 {
    float* u;
    float* b;
    int nx, ny, nz;
};

struct AdegTab {
    double v[7];  // alpha + q, q = 0..6 (the diagonal of A for a cell with q neighbours)
};

struct Geo3 {
    int n0x, n0y, n0z;  // finest sizes (fix the cell geometry of every level)
};

__device__ __forceinline__ int64_t idx3(int x, int y, int z, int nx, int ny) {
    return ((int64_t)z * ny + y) * nx + x;
}

// The 7-point finite-volume stencil of level k at cell (x, y, z).
struct Coef3 {
    float cw, ce, cn, cs, cd, cu, D;
};

__device__ __forceinline__ Coef3 coef3(int x, int y, int z, const Lev3& L, const Geo3& g, int k, float alpha,
                                       float sk) {
    const AxisCoef<float> ax = axis_coef<float>(x, L.nx, g.n0x, k);
    const AxisCoef<float> ay = axis_coef<float>(y, L.ny, g.n0y, k);
    const AxisCoef<float> az = axis_coef<float>(z, L.nz, g.n0z, k);
    Coef3 c;
    const float ayz = ay.w * az.w, axz = ax.w * az.w, axy = ax.w * ay.w;
    c.cw = sk * (ayz * ax.gm);
    c.ce = sk * (ayz * ax.gp);
    c.cn = sk * (axz * ay.gm);
    c.cs = sk * (axz * ay.gp);
    c.cd = sk * (axy * az.gm);
    c.cu = sk * (axy * az.gp);
    c.D = fmaf(alpha, axy * az.w, ((c.cw + c.ce) + (c.cn + c.cs)) + (c.cd + c.cu));
    return c;
}

// sum_q c_pq u_q over the neighbours that exist (a zero coefficient marks a missing one)
__device__ __forceinline__ float nbr_sum(const float* __restrict__ u, const Coef3& c, int x, int y, int z,
                                         const Lev3& L) {
    const int64_t p = idx3(x, y, z, L.nx, L.ny);
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    float acc = 0.f;
    if (c.cw != 0.f) acc = fmaf(c.cw, u[p - 1], acc);
    if (c.ce != 0.f) acc = fmaf(c.ce, u[p + 1], acc);
    if (c.cn != 0.f) acc = fmaf(c.cn, u[p - sy], acc);
    if (c.cs != 0.f) acc = fmaf(c.cs, u[p + sy], acc);
    if (c.cd != 0.f) acc = fmaf(c.cd, u[p - sz], acc);
    if (c.cu != 0.f) acc = fmaf(c.cu, u[p + sz], acc);
    return acc;
}

// Cells whose three axes are interior at level k (axis_coef gives w = 1 and both faces 1
// there): the stencil is sk on every face and D = alpha + 6 sk.
__device__ __forceinline__ bool interior3(int x, int y, int z, const Lev3& L, int k) {
    return interior_row(x, L.nx, k) && interior_row(y, L.ny, k) && interior_row(z, L.nz, k);
}

// The interior diagonal of level k and its reciprocal (the general formula of coef3 with unit
// widths and faces), passed to the kernels from the host.
struct Diag3 {
    float D, iD;
};

// One red-black half-sweep: the cells of colour `colour` ((x + y + z) & 1) get
// u = (b + sum_q c_pq u_q) / D.  One thread per pair of cells along x.
__global__ void __launch_bounds__(kThreads3) k3_relax(Lev3 L, Geo3 g, int k, float alpha, float sk, Diag3 di,
                                                      int colour) {
    const int nxp = (L.nx + 1) >> 1;
    const int64_t rows = (int64_t)L.ny * L.nz;
    const int64_t sy = L.nx, sz = (int64_t)L.nx * L.ny;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x)  // one (y, z) row at a time
    for (int xp = threadIdx.x; xp < nxp; xp += blockDim.x) {
        const int y = int(row % L.ny), z = int(row / L.ny);
        const int x = 2 * xp + ((y + z + colour) & 1);
        if (x >= L.nx) continue;
        const int64_t p = row * L.nx + x;
        if (interior3(x, y, z, L, k)) {
            const float* u = L.u;
            const float acc = ((u[p - 1] + u[p + 1]) + (u[p - sy] + u[p + sy])) + (u[p - sz] + u[p + sz]);
            L.u[p] = fmaf(sk, acc, L.b[p]) * di.iD;
        } else {
            const Coef3 c = coef3(x, y, z, L, g, k, alpha, sk);
            L.u[p] = (L.b[p] + nbr_sum(L.u, c, x, y, z, L)) / c.D;
        }
    }
}

// Residual of level k restricted to level k + 1: C.b = (sum of the child residuals) / 8,
// C.u = 0.  One thread per coarse cell.
__global__ void __launch_bounds__(kThreads3) k3_residual_restrict(Lev3 F, Lev3 C, Geo3 g, int k, float alpha,
                                                                  float skf, Diag3 di) {
    const int64_t rows = (int64_t)C.ny * C.nz;
    const int64_t sy = F.nx, sz = (int64_t)F.nx * F.ny;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x)
    for (int X = threadIdx.x; X < C.nx; X += blockDim.x) {
        const int Y = int(row % C.ny), Z = int(row / C.ny);
        const int64_t t = row * C.nx + X;
        float sum = 0.f;
        for (int dz = 0; dz < 2; ++dz) {
            const int z = 2 * Z + dz;
            if (z >= F.nz) break;
            for (int dy = 0; dy < 2; ++dy) {
                const int y = 2 * Y + dy;
                if (y >= F.ny) break;
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx;
                    if (x >= F.nx) break;
                    const int64_t p = idx3(x, y, z, F.nx, F.ny);
                    if (interior3(x, y, z, F, k)) {
                        const float* u = F.u;
                        const float acc =
                            ((u[p - 1] + u[p + 1]) + (u[p - sy] + u[p + sy])) + (u[p - sz] + u[p + sz]);
                        sum += F.b[p] - fmaf(di.D, u[p], -skf * acc);
                    } else {
                        const Coef3 c = coef3(x, y, z, F, g, k, alpha, skf);
                        sum += F.b[p] - fmaf(c.D, F.u[p], -nbr_sum(F.u, c, x, y, z, F));
                    }
                }
            }
        }
        C.b[t] = sum * 0.125f;
        C.u[t] = 0.f;
    }
}

// F.u += trilinear interpolation of C.u (level k + 1) at the fine cell centres.
__global__ void __launch_bounds__(kThreads3) k3_prolong_add(Lev3 F, Lev3 C, Geo3 g, int k) {
    const int64_t rows = (int64_t)F.ny * F.nz;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x)
    for (int x = threadIdx.x; x < F.nx; x += blockDim.x) {
        const int y = int(row % F.ny), z = int(row / F.ny);
        const int64_t t = row * F.nx + x;
        int Ix, Jx, Iy, Jy, Iz, Jz;
        float wx, wy, wz;
        if (x >= 2 && (x >> 1) + 2 < C.nx && y >= 2 && (y >> 1) + 2 < C.ny && z >= 2 && (z >> 1) + 2 < C.nz) {
            // all three axes in the regular pattern of interp_axis: weight 1/4 toward the
            // neighbouring coarse centre on the side of the fine cell
            Ix = x >> 1; Jx = (x & 1) ? Ix + 1 : Ix - 1;
            Iy = y >> 1; Jy = (y & 1) ? Iy + 1 : Iy - 1;
            Iz = z >> 1; Jz = (z & 1) ? Iz + 1 : Iz - 1;
            wx = wy = wz = 0.25f;
        } else {
            interp_axis<float>(x, g.n0x, k, C.nx, Ix, Jx, wx);
            interp_axis<float>(y, g.n0y, k, C.ny, Iy, Jy, wy);
            interp_axis<float>(z, g.n0z, k, C.nz, Iz, Jz, wz);
        }
        const float* u0 = C.u + (int64_t)Iz * C.ny * C.nx;
        const float* u1 = C.u + (int64_t)Jz * C.ny * C.nx;
        const float a = bilinear<float>(u0[(int64_t)Iy * C.nx + Ix], u0[(int64_t)Iy * C.nx + Jx],
                                        u0[(int64_t)Jy * C.nx + Ix], u0[(int64_t)Jy * C.nx + Jx], wx, wy);
        const float b = bilinear<float>(u1[(int64_t)Iy * C.nx + Ix], u1[(int64_t)Iy * C.nx + Jx],
                                        u1[(int64_t)Jy * C.nx + Ix], u1[(int64_t)Jy * C.nx + Jx], wx, wy);
        F.u[t] += fmaf(wz, b - a, a);
    }
}


// Block sum of two doubles into sums[0], sums[1] (shuffle tree, one atomic per block).
__device__ __forceinline__ void block_sum2(double a, double b, double* sums) {
    __shared__ double red[2][kThreads3 / 32];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, m);
        b += __shfl_xor_sync(0xffffffffu, b, m);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = a; red[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < kThreads3 / 32 ? red[0][l] : 0.0;
        b = l < kThreads3 / 32 ? red[1][l] : 0.0;
#pragma unroll
        for (int m = 4; m > 0; m >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, m);
            b += __shfl_xor_sync(0xffffffffu, b, m);
        }
        if (l == 0) {
            atomicAdd(&sums[0], a);
            atomicAdd(&sums[1], b);
        }
    }
}

// d += e (FP64), e = the level-0 result of the last V-cycle.
__global__ void __launch_bounds__(kThreads3) k3_update(double* __restrict__ d, const float* __restrict__ e, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        d[t] += f2d_ieee(e[t]);
}

// FP64 defect pass on the finest level: r = -L_z I0 - A d (A = alpha I + L, 7-point, Neumann),
// out = I0 + d; r goes to the level-0 right-hand side (FP32) and the level-0 iterate is zeroed
// for the next V-cycle.  A d is formed in FP64 on the FP64 iterate (sum of the neighbours and
// one fma with alpha + degree, where the cancellation happens), rounded once to FP32 and taken
// from the FP32-formed -L_z I0 (exact for 8-bit input; its own rounding bounds what FP64 could
// add there), as the slice solver's correction passes do.  sums[0] += ||r||^2 (FP64); with
// `first` (d = 0, not read) also sums[1] += ||alpha I0 + L_xy I0||^2.  Conversions run on the
// integer pipe.  adeg[q] = alpha + q for q = 0..6.  EXACT (tolerances below 1e-7, where the
// FP32 rounding of the subtraction would cap the reachable residual): -L_z I0 and the
// subtraction in FP64 too.
template <class Tin, bool EXACT>
__global__ void __launch_bounds__(kThreads3) k3_defect(const Tin* __restrict__ I0, const double* __restrict__ d,
                                                       float* __restrict__ r0, float* __restrict__ u0,
                                                       float* __restrict__ out, int nx, int ny, int nz,
                                                       float alpha, AdegTab adeg, int first,
                                                       double* __restrict__ sums) {
    const int64_t rows = (int64_t)ny * nz, sy = nx, sz = (int64_t)nx * ny;
    double rr = 0.0, bb = 0.0;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x)
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const int y = int(row % ny), z = int(row / ny);
        const int64_t t = row * nx + x;
        const bool hw = x > 0, he = x + 1 < nx, hn = y > 0, hs = y + 1 < ny, hd = z > 0, hu = z + 1 < nz;
        const float ip = (float)I0[t];
        // -L_z I0: the z neighbours minus the cell
        float rhs = 0.f;
        if (hd) rhs += (float)I0[t - sz] - ip;
        if (hu) rhs += (float)I0[t + sz] - ip;
        float r = rhs, o = ip;
        double rd = 0.0;  // r in FP64 (EXACT)
        if (EXACT) {
            const double ipd = f2d_ieee(ip);
            if (hd) rd += f2d_ieee((float)I0[t - sz]) - ipd;
            if (hu) rd += f2d_ieee((float)I0[t + sz]) - ipd;
        }
        if (!first) {
            const double dp = d[t];
            double nb = 0.0;
            if (hw) nb += d[t - 1];
            if (he) nb += d[t + 1];
            if (hn) nb += d[t - sy];
            if (hs) nb += d[t + sy];
            if (hd) nb += d[t - sz];
            if (hu) nb += d[t + sz];
            const int deg = int(hw) + int(he) + int(hn) + int(hs) + int(hd) + int(hu);
            const double ad = deg == 6 ? adeg.v[6] : deg == 5 ? adeg.v[5] : deg == 4 ? adeg.v[4] :
                              deg == 3 ? adeg.v[3] : deg == 2 ? adeg.v[2] : deg == 1 ? adeg.v[1] : adeg.v[0];
            const double Ad = fma(ad, dp, -nb);
            if (EXACT) {
                rd -= Ad;
                r = d2f_ieee(rd);
            } else {
                r = rhs - d2f_ieee(Ad);
            }
            o = ip + d2f_ieee(dp);
        } else {
            float lxy = 0.f;  // L_xy I0
            if (hw) lxy += ip - (float)I0[t - 1];
            if (he) lxy += ip - (float)I0[t + 1];
            if (hn) lxy += ip - (float)I0[t - sy];
            if (hs) lxy += ip - (float)I0[t + sy];
            const double b = f2d_ieee(fmaf(alpha, ip, lxy));
            bb = fma(b, b, bb);
        }
        if (!EXACT) rd = f2d_ieee(r);
        rr = fma(rd, rd, rr);
        r0[t] = r;
        u0[t] = 0.f;
        out[t] = o;
    }
    block_sum2(rr, bb, sums);
}

// Blocks for a pass over `rows` rows of `nx` cells: one block per row (threads across the
// row), at most 16 per SM; blocks loop over rows.
unsigned grid_rows(int64_t rows) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)kNumSMs * 16));
}
unsigned grid_for(int64_t n) {
    const int64_t blocks = (n + kThreads3 - 1) / kThreads3;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)kNumSMs * 16));
}

}  // namespace

int gd_multigrid(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz, double alpha,
                 const emfuse_solve_opts& opts, emfuse_slice_stats* stats, cudaStream_t st) {
    // levels: ceil halving per axis down to 1 x 1 x 1
    std::vector<Lev3> lev;
    {
        int k = 0;
        for (;; ++k) {
            Lev3 L{};
            L.nx = (int)(((nx - 1) >> k) + 1);
            L.ny = (int)(((ny - 1) >> k) + 1);
            L.nz = (int)(((nz - 1) >> k) + 1);
            lev.push_back(L);
            if (L.nx == 1 && L.ny == 1 && L.nz == 1) break;
        }
    }
    const int nlev = (int)lev.size();
    size_t cells = 0;
    for (const auto& L : lev) cells += (size_t)L.nx * L.ny * L.nz;
    const int64_t n0 = nx * ny * nz;
    DeviceBuffer ub, bbuf, dbuf, sums;
    EMF_TRY(ub.alloc(cells * sizeof(float), st));
    EMF_TRY(bbuf.alloc(cells * sizeof(float), st));
    EMF_TRY(dbuf.alloc((size_t)n0 * sizeof(double), st));
    EMF_TRY(sums.alloc(2 * sizeof(double), st));
    {
        size_t off = 0;
        for (auto& L : lev) {
            L.u = ub.as<float>() + off;
            L.b = bbuf.as<float>() + off;
            off += (size_t)L.nx * L.ny * L.nz;
        }
    }
    EMF_CUDA(cudaMemsetAsync(dbuf.as<double>(), 0, (size_t)n0 * sizeof(double), st));  // d = 0
    const Geo3 g{(int)nx, (int)ny, (int)nz};
    const float af = (float)alpha;
    double* d = dbuf.as<double>();
    double* hs = nullptr;  // pinned copy of the norms
    EMF_CUDA(cudaMallocHost(&hs, 2 * sizeof(double)));
    struct HostFree {
        double* p;
        ~HostFree() { cudaFreeHost(p); }
    } hs_guard{hs};

    auto defect = [&](int first) -> int {
        EMF_CUDA(cudaMemsetAsync(sums.as<double>(), 0, 2 * sizeof(double), st));
        KernelScope ks("gd3_defect", st, (double)n0 * ((dt == EMFUSE_U8 ? 1.0 : 4.0) + (first ? 0.0 : 8.0) + 12.0),
                       first ? 0.0 : (double)n0 * 8.0);
        AdegTab adeg;
        for (int q = 0; q <= 6; ++q) adeg.v[q] = alpha + (double)q;
        const bool exact = opts.tol < 1e-7;
        const unsigned gr = grid_rows(ny * nz);
#define EMF_GD3_DEFECT(TT, EX)                                                                            \
    k3_defect<TT, EX><<<gr, kThreads3, 0, st>>>((const TT*)in, d, lev[0].b, lev[0].u, out, (int)nx, (int)ny, \
                                                (int)nz, af, adeg, first, sums.as<double>())
        if (dt == EMFUSE_U8) {
            if (exact) EMF_GD3_DEFECT(uint8_t, true);
            else EMF_GD3_DEFECT(uint8_t, false);
        } else {
            if (exact) EMF_GD3_DEFECT(float, true);
            else EMF_GD3_DEFECT(float, false);
        }
#undef EMF_GD3_DEFECT
        EMF_CHECK_LAUNCH();
        EMF_CUDA(cudaMemcpyAsync(hs, sums.as<double>(), 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        EMF_CUDA(cudaStreamSynchronize(st));
        return EMFUSE_OK;
    };
    // interior diagonal of level k: coef3's formula with unit widths and faces
    auto diag = [&](int k) {
        const float sk = std::ldexp(1.f, -2 * k);
        Diag3 di;
        di.D = std::fmaf(af, 1.f, ((sk + sk) + (sk + sk)) + (sk + sk));
        di.iD = (float)(1.0 / (double)di.D);
        return di;
    };
    auto relax = [&](int k, int sweeps) -> int {
        const Lev3& L = lev[k];
        const float sk = std::ldexp(1.f, -2 * k);
        const int64_t n = (int64_t)L.ny * L.nz;  // rows
        for (int s = 0; s < sweeps; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                KernelScope ks(k == 0 ? "gd3_relax_l0" : "gd3_relax", st, (double)L.nx * L.ny * L.nz * 6.0);
                k3_relax<<<grid_rows(n), kThreads3, 0, st>>>(L, g, k, af, sk, diag(k), colour);
                EMF_CHECK_LAUNCH();
            }
        return EMFUSE_OK;
    };
    auto vcycle = [&]() -> int {
        for (int k = 0; k + 1 < nlev; ++k) {
            EMF_TRY(relax(k, opts.nu_pre));
            const Lev3 &F = lev[k], &C = lev[k + 1];
            KernelScope ks(k == 0 ? "gd3_restrict_l0" : "gd3_restrict", st, (double)F.nx * F.ny * F.nz * 8.0);
            k3_residual_restrict<<<grid_rows((int64_t)C.ny * C.nz), kThreads3, 0, st>>>(
                F, C, g, k, af, std::ldexp(1.f, -2 * k), diag(k));
            EMF_CHECK_LAUNCH();
        }
        EMF_TRY(relax(nlev - 1, 1));  // 1 x 1 x 1: one half-sweep solves it
        for (int k = nlev - 2; k >= 0; --k) {
            const Lev3 &F = lev[k], &C = lev[k + 1];
            {
                KernelScope ks(k == 0 ? "gd3_prolong_l0" : "gd3_prolong", st, (double)F.nx * F.ny * F.nz * 8.0);
                k3_prolong_add<<<grid_rows((int64_t)F.ny * F.nz), kThreads3, 0, st>>>(F, C, g, k);
                EMF_CHECK_LAUNCH();
            }
            EMF_TRY(relax(k, opts.nu_post));
        }
        return EMFUSE_OK;
    };

    // relative residual; a NaN or Inf anywhere in the input makes a norm non-finite
    auto relres = [&](double bnorm) {
        if (!std::isfinite(hs[0]) || !std::isfinite(bnorm)) return std::nan("");
        return bnorm > 0.0 ? std::sqrt(hs[0]) / bnorm : (hs[0] > 0.0 ? HUGE_VAL : 0.0);
    };
    EMF_TRY(defect(1));
    const double bnorm = std::sqrt(hs[1]);
    double rel = relres(bnorm);
    int v = 0;
    bool finite = std::isfinite(rel);
    while (finite && rel > opts.tol && v < opts.max_vcycles) {
        EMF_TRY(vcycle());
        // before the first FP64 pass, further FP32 V-cycles continue from the last iterate
        // (their fine residual is formed in FP32 inside the cycle), as in the slice solver
        if (v == 0)
            for (int extra = 1; extra < opts.first_vcycles && extra < opts.max_vcycles; ++extra, ++v)
                EMF_TRY(vcycle());
        {
            KernelScope ks("gd3_update", st, (double)n0 * 20.0);
            k3_update<<<grid_for(n0), kThreads3, 0, st>>>(d, lev[0].u, n0);
            EMF_CHECK_LAUNCH();
        }
        EMF_TRY(defect(0));
        rel = relres(bnorm);
        finite = std::isfinite(rel);
        ++v;
    }
    if (stats) {
        stats->vcycles = v;
        stats->converged = finite && rel <= opts.tol ? 1 : 0;
        stats->rel_residual = rel;
        stats->b_norm = bnorm;
        stats->rel_residual_check = -1.0;
    }
    if (!finite) {
        set_error("emfuse_smooth_gradient_domain_mg: non-finite residual (NaN or Inf in the input?)");
        return EMFUSE_EINVAL;
    }
    if (rel > opts.tol) {
        set_error("emfuse_smooth_gradient_domain_mg: tolerance not reached within max_vcycles");
        return EMFUSE_ENOCONV;
    }
    return EMFUSE_OK;
}

}  // namespace emfuse
