// Device-side pieces of the multigrid shared by the reference schedule (one kernel per
// half-sweep) and the fused schedule (wavefront kernels + coarse tail): the level
// descriptor, the finite-volume stencil of a level, the Gauss-Seidel update, the residual and
// the prolongation weights.  Both schedules call the same inline functions with explicit
// fma ordering, so they produce bit-identical iterates.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda.h>

#include "emfuse_common.cuh"

namespace emfuse {

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rcp_t(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcp_t(double a) { return __drcp_rn(a); }
__device__ __forceinline__ float mul_t(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_t(double a, double b) { return __dmul_rn(a, b); }

// One slice at one multigrid level (device-visible).
template <class T>
struct LSlice {
    T* u;              // iterate, `pitch` elements per row
    T* b;              // right-hand side
    int nx, ny, pitch;
    T* uo;             // where the final (post-smoothed) iterate of this level goes: a second
                       // buffer on wavefront levels, whose UP kernel reads u on halos that
                       // other warps would otherwise overwrite; u itself elsewhere
    T* uc;             // level k+1 iterate and rhs (null at the coarsest level of this slice)
    T* bc;
    T* uco;            // level k+1 final iterate (its uo)
    int ncx, ncy, pitchc;
    T* uf;             // level k-1 iterate and rhs (null at k = 0)
    T* bf;
    int nfx, nfy, pitchf;
    int n0x, n0y;      // finest-level size (fixes the cell geometry of every level)
    int slice;         // index of the slice in the caller's batch
    int tiles_x;       // reference-kernel tiles along x
    int fstrips;       // wavefront-kernel strips along x
};

// Per-axis geometry of a cell: its width (level units) and the face coefficients
// 2 / (w_i + w_{i+-1}) to its lower / upper neighbour (0 at the slice boundary).
template <class T>
struct AxisCoef {
    T w, gm, gp;
};

template <class T>
__device__ __forceinline__ AxisCoef<T> axis_coef(int i, int n, int n0, int k) {
    AxisCoef<T> a;
    if (i < 0 || i >= n) {  // outside the level: a finite, decoupled cell (never written back)
        a.w = T(1);
        a.gm = T(0);
        a.gp = T(0);
        return a;
    }
    if (k == 0) {
        a.w = T(1);
        a.gm = i > 0 ? T(1) : T(0);
        a.gp = i + 1 < n ? T(1) : T(0);
        return a;
    }
    if (i >= 1 && i + 2 < n) {  // cells i-1, i, i+1 are all full: every coefficient is 1
        a.w = T(1);
        a.gm = T(1);
        a.gp = T(1);
        return a;
    }
    a.w = cell_width<T>(i, n0, k);
    a.gm = face_coeff<T>(i - 1, n, n0, k);
    a.gp = face_coeff<T>(i, n, n0, k);
    return a;
}

template <class T>
struct Coef {
    T cw, ce, cn, cs, D, iD;  // iD = correctly rounded 1 / D
};

// Finite-volume stencil of level k at a cell (interior cells: alpha + L/4^k).
template <class T>
__device__ __forceinline__ Coef<T> make_coef(const AxisCoef<T>& ax, const AxisCoef<T>& ay, int k,
                                             T alpha, T sk) {
    Coef<T> c;
    if (k == 0) {
        c.cw = ax.gm;
        c.ce = ax.gp;
        c.cn = ay.gm;
        c.cs = ay.gp;
        c.D = alpha + (((c.cw + c.ce) + c.cn) + c.cs);
        c.iD = rcp_t(c.D);
        return c;
    }
    c.cw = sk * (ay.w * ax.gm);
    c.ce = sk * (ay.w * ax.gp);
    c.cn = sk * (ax.w * ay.gm);
    c.cs = sk * (ax.w * ay.gp);
    c.D = fma_t(alpha, ax.w * ay.w, ((c.cw + c.ce) + c.cn) + c.cs);
    c.iD = rcp_t(c.D);
    return c;
}

// The stencil of a cell on an interior row (ay = {1, 1, 1}) with D and 1/D taken from a
// per-column cache (d, id) computed by make_coef on such a row: the same values make_coef
// returns, without recomputing the diagonal and its reciprocal.
template <class T>
__device__ __forceinline__ Coef<T> interior_row_coef(const AxisCoef<T>& ax, int k, T sk, T d, T id) {
    Coef<T> c;
    if (k == 0) {
        c.cw = ax.gm;
        c.ce = ax.gp;
        c.cn = T(1);
        c.cs = T(1);
    } else {
        c.cw = sk * (T(1) * ax.gm);
        c.ce = sk * (T(1) * ax.gp);
        c.cn = sk * (ax.w * T(1));
        c.cs = sk * (ax.w * T(1));
    }
    c.D = d;
    c.iD = id;
    return c;
}

// Rows whose axis_coef is {1, 1, 1} (see axis_coef).
__device__ __forceinline__ bool interior_row(int r, int n, int k) {
    return k == 0 ? (r >= 1 && r + 1 < n) : (r >= 1 && r + 2 < n);
}

template <class T>
__device__ __forceinline__ Coef<T> coef_at(int x, int y, int nx, int ny, int n0x, int n0y, int k,
                                           T alpha, T sk) {
    return make_coef<T>(axis_coef<T>(x, nx, n0x, k), axis_coef<T>(y, ny, n0y, k), k, alpha, sk);
}


// Gauss-Seidel update u_p = (b_p + sum_q c_pq u_q) * (1 / D_p).
template <class T>
__device__ __forceinline__ T gs_update(const Coef<T>& c, T b, T uw, T ue, T un, T us) {
    T acc = fma_t(c.cw, uw, b);
    acc = fma_t(c.ce, ue, acc);
    acc = fma_t(c.cn, un, acc);
    acc = fma_t(c.cs, us, acc);
    return mul_t(acc, c.iD);
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

// Linear interpolation along one axis from level k+1 (coarse) to level k (fine): fine cell x
// lies between coarse centres I = x/2 and J; returns J and its weight (0 if J = I).
template <class T>
__device__ __forceinline__ void interp_axis(int x, int n0, int k, int nc, int& I, int& J, T& wJ) {
    I = x >> 1;
    if (x >= 2 && I + 2 < nc) {  // fine cell and both coarse cells full: weight exactly 1/4
        J = (x & 1) ? I + 1 : I - 1;
        wJ = T(0.25);
        return;
    }
    const int fs = x << k, cs = I << (k + 1);  // sides are < 2^29, so twice them fit an int
    const int hf = min(1 << k, n0 - fs);
    const int hc = min(1 << (k + 1), n0 - cs);
    const int cf2 = 2 * fs + hf, cc2 = 2 * cs + hc;  // twice the centres
    J = I;
    wJ = T(0);
    if (cf2 == cc2) return;
    const int Jn = cf2 < cc2 ? I - 1 : I + 1;
    if (Jn < 0 || Jn >= nc) return;
    const int js = Jn << (k + 1);
    const int hj = min(1 << (k + 1), n0 - js);
    const int cj2 = 2 * js + hj;
    J = Jn;
    wJ = T(cf2 > cc2 ? cf2 - cc2 : cc2 - cf2) / T(cj2 > cc2 ? cj2 - cc2 : cc2 - cj2);
}

// Bilinear combination of the four coarse values around a fine cell.
template <class T>
__device__ __forceinline__ T bilinear(T r0I, T r0J, T r1I, T r1J, T wx, T wy) {
    const T a = fma_t(wx, r0J - r0I, r0I);
    const T b = fma_t(wx, r1J - r1I, r1I);
    return fma_t(wy, b - a, a);
}

// Correction at fine cell (x, y) of level k interpolated from the level k+1 iterate.
template <class T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ uc, int pitchc, int x, int y, int ncx,
                                        int ncy, int n0x, int n0y, int k) {
    int Ix, Jx, Iy, Jy;
    T wx, wy;
    interp_axis<T>(x, n0x, k, ncx, Ix, Jx, wx);
    interp_axis<T>(y, n0y, k, ncy, Iy, Jy, wy);
    const T* r0 = uc + (int64_t)Iy * pitchc;
    const T* r1 = uc + (int64_t)Jy * pitchc;
    return bilinear<T>(r0[Ix], r0[Jx], r1[Ix], r1[Jx], wx, wy);
}

__device__ __forceinline__ int find_item(const int64_t* __restrict__ ts, int n, int64_t t) {
    int lo = 0, hi = n;  // ts[0] = 0 <= t < ts[n]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ts[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Shared-memory bytes of the coarse tail of a slice whose first tail level has nx x ny cells
// (u and b of every level down to 1 x 1, dense rows).
template <class T>
__host__ __device__ inline size_t tail_smem_bytes(int nx, int ny) {
    size_t cells = 0;
    for (int k = 0;; ++k) {
        const int lx = ((nx - 1) >> k) + 1, ly = ((ny - 1) >> k) + 1;
        cells += (size_t)lx * ly;
        if (lx == 1 && ly == 1) break;
    }
    return 2 * cells * sizeof(T);
}

// ---------------------------------------------------------------- fused schedule (fused.cu)
constexpr int kWaveHalo = 8;                      // x halo of a strip (cells, multiple of 4)
constexpr int kWaveWidth = 128;                   // strip width: 32 lanes x 4 cells
constexpr int kWaveIW = kWaveWidth - 2 * kWaveHalo;  // interior cells per strip
constexpr int kTailMax = 64;                      // levels with max side <= this go to the tail
constexpr int kWaveCoarseW = 72;                  // coarse columns staged per strip (UP)

template <class T>
struct WaveArgs {
    const LSlice<T>* sl;         // slices that use the wavefront kernel at this level
    const int64_t* item_start;   // warp work items per slice, prefix sums (nsl + 1)
    int nsl;
    int64_t nitems;
    int k;
    int ch;                      // rows per work item (even)
    T alpha;
    T sk;
    const int* active;
    const CUtensorMap* maps;     // per wavefront slice: u, b, coarse output iterate, uo
    int u_map;                   // map the initial u is read from: 0 (u) or 3 (uo, to continue
                                 // from the previous V-cycle's result)
    int* err;                    // set to 1 when a bounded wait gives up
    unsigned int* work;          // [0]: next work item, [1]: warps finished (both 0 at launch)
};

template <class T>
struct TailArgs {
    const LSlice<T>* table;      // all levels of all slices
    const int* level_off;        // first table entry of each slice
    const int* nlev;             // levels of each slice
    const int* kc;               // first level handled by the tail, per slice
    int nslices;
    T alpha;
    int nu_pre, nu_post;
    const int* active;
    int cont;                    // 1: a slice whose tail starts at level 0 continues from u
    int smem_bytes;              // dynamic shared memory of the launch (the largest slice's tail)
};

template <class T>
int launch_wave(const WaveArgs<T>& a, int S, bool zero_init, bool up, cudaStream_t st, double bytes);
template <class T>
int launch_tail(const TailArgs<T>& a, cudaStream_t st, double bytes);

}  // namespace emfuse
