// Device-side pieces of the multigrid shared by the reference (one kernel per half-sweep)
// and the fused kernels: the level descriptor, the finite-volume stencil of a level, the
// Gauss-Seidel update, the residual and the prolongation weights.  Both schedules call the
// same inline functions with explicit fma ordering, so they produce bit-identical iterates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "emfuse_common.cuh"

namespace emfuse {

// One slice at one multigrid level (device-visible).
template <class T>
struct LSlice {
    T* u;              // iterate, `pitch` elements per row
    T* b;              // right-hand side
    int nx, ny, pitch;
    const T* uc;       // level k+1 iterate (null at the coarsest level of this slice)
    int ncx, ncy, pitchc;
    const T* uf;       // level k-1 iterate and rhs (null at k = 0)
    const T* bf;
    int nfx, nfy, pitchf;
    int n0x, n0y;      // finest-level size (fixes the cell geometry of every level)
    int slice;         // index of the slice in the caller's batch
    int tiles_x;       // reference-kernel tiles along x
};

template <class T>
struct Coef {
    T cw, ce, cn, cs, D;
};

// Finite-volume stencil of level k at cell (x, y) (interior: alpha + L/4^k).
template <class T>
__device__ __forceinline__ Coef<T> coef_at(int x, int y, int nx, int ny, int n0x, int n0y, int k,
                                           T alpha, T sk) {
    Coef<T> c;
    if (k == 0) {
        c.cw = x > 0 ? T(1) : T(0);
        c.ce = x + 1 < nx ? T(1) : T(0);
        c.cn = y > 0 ? T(1) : T(0);
        c.cs = y + 1 < ny ? T(1) : T(0);
        c.D = alpha + (((c.cw + c.ce) + c.cn) + c.cs);
        return c;
    }
    const T wx = cell_width<T>(x, n0x, k), wy = cell_width<T>(y, n0y, k);
    c.cw = sk * (wy * face_coeff<T>(x - 1, nx, n0x, k));
    c.ce = sk * (wy * face_coeff<T>(x, nx, n0x, k));
    c.cn = sk * (wx * face_coeff<T>(y - 1, ny, n0y, k));
    c.cs = sk * (wx * face_coeff<T>(y, ny, n0y, k));
    c.D = alpha * (wx * wy) + (((c.cw + c.ce) + c.cn) + c.cs);
    return c;
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float div_t(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_t(double a, double b) { return __ddiv_rn(a, b); }

// Gauss-Seidel update u_p = (b_p + sum_q c_pq u_q) / D_p.
template <class T>
__device__ __forceinline__ T gs_update(const Coef<T>& c, T b, T uw, T ue, T un, T us) {
    T acc = fma_t(c.cw, uw, b);
    acc = fma_t(c.ce, ue, acc);
    acc = fma_t(c.cn, un, acc);
    acc = fma_t(c.cs, us, acc);
    return div_t(acc, c.D);
}

// Residual b_p - (D_p u_p - sum_q c_pq u_q).
template <class T>
__device__ __forceinline__ T residual_at(const Coef<T>& c, T b, T u, T uw, T ue, T un, T us) {
    T acc = fma_t(c.cw, uw, b);
    acc = fma_t(c.ce, ue, acc);
    acc = fma_t(c.cn, un, acc);
    acc = fma_t(c.cs, us, acc);
    return fma_t(-c.D, u, acc);
}

// Linear interpolation weight along one axis from level k+1 (coarse) to level k (fine):
// fine cell x lies between coarse centres I = x/2 and J; returns J and its weight.
template <class T>
__device__ __forceinline__ void interp_axis(int x, int n0, int k, int nc, int& I, int& J, T& wJ) {
    I = x >> 1;
    const long long fs = (long long)x << k, cs = (long long)I << (k + 1);
    const long long hf = min((long long)1 << k, (long long)n0 - fs);
    const long long hc = min((long long)1 << (k + 1), (long long)n0 - cs);
    const long long cf2 = 2 * fs + hf, cc2 = 2 * cs + hc;  // twice the centres
    J = I;
    wJ = T(0);
    if (cf2 == cc2) return;
    const int Jn = cf2 < cc2 ? I - 1 : I + 1;
    if (Jn < 0 || Jn >= nc) return;
    const long long js = (long long)Jn << (k + 1);
    const long long hj = min((long long)1 << (k + 1), (long long)n0 - js);
    const long long cj2 = 2 * js + hj;
    J = Jn;
    wJ = T(cf2 > cc2 ? cf2 - cc2 : cc2 - cf2) / T(cj2 > cc2 ? cj2 - cc2 : cc2 - cj2);
}

// Bilinear correction at fine cell (x, y) of level k from the level k+1 iterate.
template <class T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ uc, int pitchc, int x, int y, int ncx,
                                        int ncy, int n0x, int n0y, int k) {
    int Ix, Jx, Iy, Jy;
    T wx, wy;
    interp_axis<T>(x, n0x, k, ncx, Ix, Jx, wx);
    interp_axis<T>(y, n0y, k, ncy, Iy, Jy, wy);
    const T* r0 = uc + (int64_t)Iy * pitchc;
    const T* r1 = uc + (int64_t)Jy * pitchc;
    const T a = fma_t(wx, r0[Jx] - r0[Ix], r0[Ix]);
    const T b = fma_t(wx, r1[Jx] - r1[Ix], r1[Ix]);
    return fma_t(wy, b - a, a);
}

}  // namespace emfuse
