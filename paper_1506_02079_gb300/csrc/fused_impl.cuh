// Fused multigrid schedule.
//
// Wavefront kernel (k_wave).  One warp owns a strip of 128 cells (32 lanes x 4 consecutive
// cells) and marches down a chunk of rows.  All nu red-black sweeps are pipelined in one
// pass: at step t the warp loads row t and applies half-sweep s (s = 1..S, S = 2 nu) to row
// t - s.  Half-sweep s only reads the other colour, whose latest update (half-sweep s - 1)
// reached rows t-s-1 .. t-s+1 before half-sweep s + 1 touches them, so the result is exactly
// that of S global half-sweeps (Gauss-Seidel red-black, colour (x + y) mod 2).  The rows in
// flight live in registers (a window of S + 3 rows plus the prefetch distance); the window is
// indexed with compile-time slots by unrolling the march by the window length.  Neighbours
// along x come from warp shuffles, so the strip edges are recomputed by the adjacent strips
// (8-cell overlap on each side).
//
//   DOWN (restriction leg): optional zero initial guess (the first half-sweep then needs no
//        load of u), S half-sweeps, the residual of the row S + 1 behind, and the 2x2 sum /4
//        of residual pairs written as the next level's right-hand side.  One read of b
//        (and u), one write of u and of the coarse rhs per cell.
//   UP   (prolongation leg): the interpolated coarse correction is added as each row
//        arrives, then S half-sweeps; one read of u, b and the coarse iterate, one write of
//        the result into a second buffer (uo): the warps read u on their halos, so no warp may
//        overwrite it in place.
//
// Coarse tail (k_tail).  Levels whose larger side is <= 64 are run by one CTA per slice: the
// remaining down and up legs of the V-cycle with __syncthreads() between half-sweeps, on
// L1-resident data.  Same per-cell arithmetic as every other schedule.
#pragma once
#include <cuda_runtime.h>

#include "emfuse_common.cuh"
#include "mg_fused.cuh"

namespace emfuse {
namespace fused_detail {

template <class T>
struct Vec4;
template <>
struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double (&v)[4]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
};

template <class T>
struct Vec2;
template <>
struct Vec2<float> {
    static __device__ __forceinline__ void load(const float* p, float& a, float& b) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        a = q.x; b = q.y;
    }
    static __device__ __forceinline__ void store(float* p, float a, float b) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
};
template <>
struct Vec2<double> {
    static __device__ __forceinline__ void load(const double* p, double& a, double& b) {
        const double2 q = *reinterpret_cast<const double2*>(p);
        a = q.x; b = q.y;
    }
    static __device__ __forceinline__ void store(double* p, double a, double b) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    }
};

constexpr int kWaveWarps = 8;


__host__ __device__ constexpr int wmod(int a, int w) { return ((a % w) + w) % w; }

// v[i] for a runtime i in 0..3 without dynamic register indexing.
template <class T>
__device__ __forceinline__ T pick4(const T (&v)[4], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// Loads row t of u (unless ZERO) and b for the lane's 4 cells; zero outside the level.
template <class T, bool ZERO>
__device__ __forceinline__ void load_row(const LSlice<T>& L, int t, int xlane, bool lane_in,
                                         T (&u)[4], T (&b)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) { u[i] = T(0); b[i] = T(0); }
    if (t < 0 || t >= L.ny || !lane_in) return;
    const int64_t off = (int64_t)t * L.pitch + xlane;
    Vec4<T>::load(L.b + off, b);
    if (!ZERO) Vec4<T>::load(L.u + off, u);
    // cells past nx sit in the row padding: mask them
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (xlane + i >= L.nx) { u[i] = T(0); b[i] = T(0); }
}

// FP32 kernels keep two CTAs per SM; FP64 windows need twice the registers.
template <class T>
struct WaveOcc { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

template <class T, int S, bool ZERO, bool UP>
__global__ void __launch_bounds__(kWaveWarps * 32, WaveOcc<T>::value) k_wave(WaveArgs<T> a) {
    constexpr int kPF = 2;                  // rows fetched ahead of the row being consumed
    constexpr int NR = UP ? S + 2 : S + 3;  // rows t .. t-NR+1 are live
    constexpr int W = NR + kPF;
    const int lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWaveWarps + (threadIdx.x >> 5);
    if (item >= a.nitems) return;
    const int j = find_item(a.item_start, a.nsl, item);
    const LSlice<T> L = a.sl[j];
    if (a.active && !a.active[L.slice]) return;
    const int li = int(item - a.item_start[j]);
    const int strip = li % L.fstrips;
    const int chunk = li / L.fstrips;
    const int X0 = strip * kWaveIW - kWaveHalo;
    const int Y0 = chunk * a.ch;
    const int Y1 = min(Y0 + a.ch, L.ny);
    const int Y1e = Y1 + (Y1 & 1);                 // residual rows run to an even end
    const int tb = Y0 - (UP ? S : S + 1);          // first row of the march
    const int te = UP ? Y1 - 1 + S : Y1e + S;      // last step (and last row loaded)
    const int k = a.k;
    const T alpha = a.alpha, sk = a.sk;

    const int xlane = X0 + 4 * lane;
    const bool lane_in = xlane >= 0 && xlane < L.nx;  // X0 is a multiple of 4: all-or-none
    const bool interior_lane = lane >= kWaveHalo / 4 && lane < 32 - kWaveHalo / 4;
    AxisCoef<T> ax[4];
    T dint[4], idint[4];  // diagonal and its reciprocal on interior rows
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        ax[i] = axis_coef<T>(xlane + i, L.nx, L.n0x, k);
        AxisCoef<T> one;
        one.w = T(1); one.gm = T(1); one.gp = T(1);
        const Coef<T> c = make_coef<T>(ax[i], one, k, alpha, sk);
        dint[i] = c.D;
        idint[i] = c.iD;
    }

    // prolongation geometry along x (UP): coarse columns cx0-1 .. cx0+2 around the lane
    const int cx0 = X0 / 2 + 2 * lane;
    int oI[4], oJ[4];
    T cwx[4];
    bool std_lane = true;  // interior pattern: J = I-1, I+1, I-1, I+1 with weight 1/4
    if (UP) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int I = 0, J = 0;
            T w = T(0);
            if (L.uco && lane_in) interp_axis<T>(xlane + i, L.n0x, k, L.ncx, I, J, w);
            oI[i] = I - cx0 + 1;
            oJ[i] = J - cx0 + 1;
            cwx[i] = w;
        }
        std_lane = oI[0] == 1 && oJ[0] == 0 && oI[1] == 1 && oJ[1] == 2 && oI[2] == 2 && oJ[2] == 1 &&
                   oI[3] == 2 && oJ[3] == 3 && cwx[0] == T(0.25) && cwx[1] == T(0.25) &&
                   cwx[2] == T(0.25) && cwx[3] == T(0.25);
    }

    T u[W][4], b[W][4];
#pragma unroll
    for (int r = 0; r < W; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) { u[r][i] = T(0); b[r][i] = T(0); }
    // UP: coarse values (rows Iy, Jy; columns cx0, cx0+1) and row weight of the row fetched
    // last, consumed one step later when the correction is added to that row
    T pc[4] = {T(0), T(0), T(0), T(0)};
    T pwy = T(0);
    bool pok = false;
    T rsum[2] = {T(0), T(0)};  // restriction partial sums (DOWN)

    auto fetch = [&](int t, T (&uu)[4], T (&bb)[4]) {
        load_row<T, (UP ? false : ZERO)>(L, t, xlane, lane_in, uu, bb);
        if (UP) {
            pok = L.uco && t >= 0 && t < L.ny;
            if (pok) {
                int Iy, Jy;
                interp_axis<T>(t, L.n0y, k, L.ncy, Iy, Jy, pwy);
                pc[0] = pc[1] = pc[2] = pc[3] = T(0);
                if (cx0 >= 0 && cx0 < L.ncx) {
                    Vec2<T>::load(L.uco + (int64_t)Iy * L.pitchc + cx0, pc[0], pc[1]);
                    Vec2<T>::load(L.uco + (int64_t)Jy * L.pitchc + cx0, pc[2], pc[3]);
                }
            }
        }
    };
    // UP: add the interpolated coarse correction (staged in pc / pwy) to row slot rs
    auto prolong = [&](T (&uu)[4]) {
        if (!pok) return;  // uniform across the warp
        const T r0m = __shfl_up_sync(0xffffffffu, pc[1], 1);    // column cx0-1 (lane-1)
        const T r0p = __shfl_down_sync(0xffffffffu, pc[0], 1);  // column cx0+2 (lane+1)
        const T r1m = __shfl_up_sync(0xffffffffu, pc[3], 1);
        const T r1p = __shfl_down_sync(0xffffffffu, pc[2], 1);
        if (!lane_in) return;
        const T v0[4] = {r0m, pc[0], pc[1], r0p};
        const T v1[4] = {r1m, pc[2], pc[3], r1p};
        if (std_lane && xlane + 3 < L.nx) {
            const T q = T(0.25);
            uu[0] = uu[0] + bilinear<T>(v0[1], v0[0], v1[1], v1[0], q, pwy);
            uu[1] = uu[1] + bilinear<T>(v0[1], v0[2], v1[1], v1[2], q, pwy);
            uu[2] = uu[2] + bilinear<T>(v0[2], v0[1], v1[2], v1[1], q, pwy);
            uu[3] = uu[3] + bilinear<T>(v0[2], v0[3], v1[2], v1[3], q, pwy);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (xlane + i >= L.nx) continue;
                uu[i] = uu[i] + bilinear<T>(pick4<T>(v0, oI[i]), pick4<T>(v0, oJ[i]), pick4<T>(v1, oI[i]),
                                            pick4<T>(v1, oJ[i]), cwx[i], pwy);
            }
        }
    };

    // rows tb and tb+1 are in flight before the march; in UP the correction of a row is added
    // one step after its fetch (when the coarse loads have landed)
    fetch(tb, u[0], b[0]);
    if (UP) prolong(u[0]);
    fetch(tb + 1, u[1], b[1]);

    for (int t0 = tb; t0 <= te; t0 += W) {
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const int t = t0 + q;
            if (t > te) break;
            // UP: finish row t + 1 (fetched one step ago), then fetch row t + 2 into the slot
            // of row t + 2 - W, which is no longer live
            if (UP) prolong(u[wmod(q + 1, W)]);
            if (t + kPF <= te) fetch(t + kPF, u[wmod(q + kPF, W)], b[wmod(q + kPF, W)]);
            // half-sweeps: stage s updates row t - s with colour (s - 1) & 1
#pragma unroll
            for (int s = 1; s <= S; ++s) {
                const int r = t - s;
                if (r < tb || r < 0 || r >= L.ny) continue;
                const int sc = wmod(q - s, W), sn = wmod(q - s - 1, W), ss = wmod(q - s + 1, W);
                const int color = (s - 1) & 1;
                const int first = (xlane + r + color) & 1;  // first cell index with this colour
                // neighbour from the adjacent lane: cell 3 of lane-1 or cell 0 of lane+1
                const T west = __shfl_up_sync(0xffffffffu, u[sc][3], 1);
                const T east = __shfl_down_sync(0xffffffffu, u[sc][0], 1);
                if (!lane_in) continue;
                const bool irow = interior_row(r, L.ny, k);
                const AxisCoef<T> ay = axis_coef<T>(r, L.ny, L.n0y, k);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    T* row = u[sc];
                    if (first == 0) {  // cells 0 and 2
                        const int i = 2 * h;
                        if (xlane + i < L.nx) {
                            const T uw = (i == 0) ? west : row[i - 1];
                            const T ue = row[i + 1];
                            const Coef<T> c = irow ? interior_row_coef<T>(ax[i], k, sk, dint[i], idint[i])
                                                   : make_coef<T>(ax[i], ay, k, alpha, sk);
                            row[i] = gs_update<T>(c, b[sc][i], uw, ue, u[sn][i], u[ss][i]);
                        }
                    } else {           // cells 1 and 3
                        const int i = 2 * h + 1;
                        if (xlane + i < L.nx) {
                            const T uw = row[i - 1];
                            const T ue = (i == 3) ? east : row[i + 1];
                            const Coef<T> c = irow ? interior_row_coef<T>(ax[i], k, sk, dint[i], idint[i])
                                                   : make_coef<T>(ax[i], ay, k, alpha, sk);
                            row[i] = gs_update<T>(c, b[sc][i], uw, ue, u[sn][i], u[ss][i]);
                        }
                    }
                }
            }
            // output of the row that completed all half-sweeps
            {
                const int r = t - S;
                const int so = wmod(q - S, W);
                if (r >= Y0 && r < Y1 && interior_lane && lane_in) {
                    T* dst = (UP ? L.uo : L.u) + (int64_t)r * L.pitch + xlane;
                    if (xlane + 3 < L.nx) {
                        Vec4<T>::store(dst, u[so]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (xlane + i < L.nx) dst[i] = u[so][i];
                    }
                }
            }
            if (!UP) {
                // residual of row t - S - 1 and its 2x2 restriction
                const int r = t - S - 1;
                const int sr = wmod(q - S - 1, W), srn = wmod(q - S - 2, W), srs = wmod(q - S, W);
                const T west = __shfl_up_sync(0xffffffffu, u[sr][3], 1);
                const T east = __shfl_down_sync(0xffffffffu, u[sr][0], 1);
                if (r >= Y0 && r < Y1e && L.bc) {
                    const bool row_in = r < L.ny && lane_in;
                    T res[4] = {T(0), T(0), T(0), T(0)};
                    if (row_in) {
                        const bool irow = interior_row(r, L.ny, k);
                        const AxisCoef<T> ay = axis_coef<T>(r, L.ny, L.n0y, k);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const T uw = i == 0 ? west : u[sr][i - 1];
                            const T ue = i == 3 ? east : u[sr][i + 1];
                            const Coef<T> c = irow ? interior_row_coef<T>(ax[i], k, sk, dint[i], idint[i])
                                                   : make_coef<T>(ax[i], ay, k, alpha, sk);
                            res[i] = residual_at<T>(c, b[sr][i], u[sr][i], uw, ue, u[srn][i], u[srs][i]);
                        }
                    }
                    // same summation order as the reference restriction:
                    // (((0 + r00) + r01) + r10) + r11
                    if ((r & 1) == 0) {
                        rsum[0] = T(0);
                        rsum[1] = T(0);
                    }
                    if (row_in) {
                        if (xlane + 0 < L.nx) rsum[0] = rsum[0] + res[0];
                        if (xlane + 1 < L.nx) rsum[0] = rsum[0] + res[1];
                        if (xlane + 2 < L.nx) rsum[1] = rsum[1] + res[2];
                        if (xlane + 3 < L.nx) rsum[1] = rsum[1] + res[3];
                    }
                    if (r & 1) {
                        const int J = r >> 1;
                        if (interior_lane && lane_in && J < L.ncy) {
                            T* dst = L.bc + (int64_t)J * L.pitchc + cx0;
                            const T v0 = rsum[0] * T(0.25), v1 = rsum[1] * T(0.25);
                            if (cx0 + 1 < L.ncx) Vec2<T>::store(dst, v0, v1);
                            else if (cx0 < L.ncx) dst[0] = v0;
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- coarse tail
template <class T>
__device__ void tail_relax(const LSlice<T>& L, int k, T alpha, T sk, int sweeps) {
    const int n = L.nx * L.ny;
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                const int y = p / L.nx, x = p - y * L.nx;
                if (((x + y) & 1) != color) continue;
                const Coef<T> c = coef_at<T>(x, y, L.nx, L.ny, L.n0x, L.n0y, k, alpha, sk);
                const int64_t q = (int64_t)y * L.pitch + x;
                const T uw = x > 0 ? L.u[q - 1] : T(0);
                const T ue = x + 1 < L.nx ? L.u[q + 1] : T(0);
                const T un = y > 0 ? L.u[q - L.pitch] : T(0);
                const T us = y + 1 < L.ny ? L.u[q + L.pitch] : T(0);
                L.u[q] = gs_update<T>(c, L.b[q], uw, ue, un, us);
            }
            __syncthreads();
        }
}

template <class T>
__global__ void __launch_bounds__(512) k_tail(TailArgs<T> a) {
    const int j = blockIdx.x;
    if (a.active && !a.active[j]) return;
    const LSlice<T>* lv = a.table + a.level_off[j];
    const int kc = a.kc[j];
    const int K = a.nlev[j] - 1;
    for (int k = kc; k <= K; ++k) {
        const LSlice<T> L = lv[k];
        const T sk = T(ldexp(1.0, -2 * k));
        for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
            const int y = p / L.nx, x = p - y * L.nx;
            L.u[(int64_t)y * L.pitch + x] = T(0);
        }
        __syncthreads();
        tail_relax<T>(L, k, a.alpha, sk, a.nu_pre);
        if (k < K) {
            const LSlice<T> C = lv[k + 1];
            for (int p = threadIdx.x; p < C.nx * C.ny; p += blockDim.x) {
                const int J = p / C.nx, I = p - J * C.nx;
                T sum = T(0);
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int x = 2 * I + dx, y = 2 * J + dy;
                        if (x < L.nx && y < L.ny) {
                            const Coef<T> c = coef_at<T>(x, y, L.nx, L.ny, L.n0x, L.n0y, k, a.alpha, sk);
                            const int64_t q = (int64_t)y * L.pitch + x;
                            const T uw = x > 0 ? L.u[q - 1] : T(0);
                            const T ue = x + 1 < L.nx ? L.u[q + 1] : T(0);
                            const T un = y > 0 ? L.u[q - L.pitch] : T(0);
                            const T us = y + 1 < L.ny ? L.u[q + L.pitch] : T(0);
                            sum += residual_at<T>(c, L.b[q], L.u[q], uw, ue, un, us);
                        }
                    }
                C.b[(int64_t)J * C.pitch + I] = sum * T(0.25);
            }
            __syncthreads();
        }
    }
    for (int k = K - 1; k >= kc; --k) {
        const LSlice<T> L = lv[k];
        const T sk = T(ldexp(1.0, -2 * k));
        for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
            const int y = p / L.nx, x = p - y * L.nx;
            L.u[(int64_t)y * L.pitch + x] += prolong_at<T>(L.uc, L.pitchc, x, y, L.ncx, L.ncy, L.n0x, L.n0y, k);
        }
        __syncthreads();
        tail_relax<T>(L, k, a.alpha, sk, a.nu_post);
    }
}

}  // namespace fused_detail
}  // namespace emfuse
