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
#include "tma.cuh"

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

constexpr int kWaveWarps = 4;  // warps (strips) per CTA


__host__ __device__ constexpr int wmod(int a, int w) { return ((a % w) + w) % w; }

// v[i] for a runtime i in 0..3 without dynamic register indexing.
template <class T>
__device__ __forceinline__ T pick4(const T (&v)[4], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// CTAs per SM the register budget is sized for (FP64 windows take twice the registers).
template <class T>
struct WaveOcc { static constexpr int value = sizeof(T) == 4 ? 4 : 2; };

// Half-sweep of one colour for a lane on a boundary row or with a boundary cell: per-cell
// stencils (rare, so kept out of line to keep the march small).
template <class T>
__device__ __noinline__ void edge_update(T (&row)[4], const T (&brow)[4], const T (&nrow)[4], const T (&srow)[4],
                                         int first, T west, T east, int xlane, int r, int nx, int ny, int n0x,
                                         int n0y, int k, T alpha, T sk) {
    const AxisCoef<T> ay = axis_coef<T>(r, ny, n0y, k);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = 2 * h + first;
        const T uw = i == 0 ? west : row[i - 1];
        const T ue = i == 3 ? east : row[i + 1];
        const Coef<T> c = make_coef<T>(axis_coef<T>(xlane + i, nx, n0x, k), ay, k, alpha, sk);
        row[i] = gs_update<T>(c, brow[i], uw, ue, nrow[i], srow[i]);
    }
}

// Residuals of a lane's 4 cells with per-cell stencils (boundary lanes and rows).
template <class T>
__device__ __noinline__ void edge_residual(T (&res)[4], const T (&rrow)[4], const T (&brow)[4], const T (&nrow)[4],
                                           const T (&srow)[4], T west, T east, int xlane, int r, int nx, int ny,
                                           int n0x, int n0y, int k, T alpha, T sk) {
    const AxisCoef<T> ay = axis_coef<T>(r, ny, n0y, k);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T uw = i == 0 ? west : rrow[i - 1];
        const T ue = i == 3 ? east : rrow[i + 1];
        const Coef<T> c = make_coef<T>(axis_coef<T>(xlane + i, nx, n0x, k), ay, k, alpha, sk);
        res[i] = residual_at<T>(c, brow[i], rrow[i], uw, ue, nrow[i], srow[i]);
    }
}

// Prolongation for lanes whose cells do not follow the interior 1/4-3/4 pattern.
template <class T>
__device__ __noinline__ void prolong_generic(T (&uu)[4], const T (&v0)[4], const T (&v1)[4], const int (&oI)[4],
                                             const int (&oJ)[4], const T (&cwx)[4], T wy, int xlane, int nx) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (xlane + i >= nx) continue;
        uu[i] = uu[i] + bilinear<T>(pick4<T>(v0, oI[i]), pick4<T>(v0, oJ[i]), pick4<T>(v1, oI[i]),
                                    pick4<T>(v1, oJ[i]), cwx[i], wy);
    }
}

// Shared-memory ring of one warp: one slot per row from the oldest row still needed (the
// residual row, S + 1 behind the newest) to the newest row in flight (kAhead - 1 ahead).  A
// slot holds the strip's row of u and b (128 cells) and, for the prolongation leg, the two
// coarse rows around it.  b is read from the ring when a half-sweep needs it; u moves into a
// register window when its row arrives.
template <class T, int S, bool ZERO, bool UP>
struct WaveRing {
    static constexpr int kAhead = sizeof(T) == 4 ? 8 : 4;            // rows in flight
    static constexpr int kNB = 16;                                   // b slots (and barriers)
    static_assert(kAhead + S + 2 <= kNB, "b ring too short for the half-sweep window");
    static constexpr int kRowBytes = kWaveWidth * (int)sizeof(T);
    static constexpr int kCoarseBytes = UP ? (kWaveCoarseW * 2 * (int)sizeof(T) + 127) / 128 * 128 : 0;
    // u and the coarse rows are consumed when their row arrives: kAhead slots suffice
    static constexpr int kUSlotBytes = (ZERO ? 0 : kRowBytes) + kCoarseBytes;
    static constexpr int kBRingBytes = kNB * kRowBytes;
    static constexpr int kURingBytes = kAhead * kUSlotBytes;
    static constexpr int kWarpBytes = kBRingBytes + kURingBytes + (kNB * 8 + 127) / 128 * 128;
};

template <class T, int S, bool ZERO, bool UP>
constexpr int wave_smem_bytes() { return kWaveWarps * WaveRing<T, S, ZERO, UP>::kWarpBytes; }

template <class T, int S, bool ZERO, bool UP>
__global__ void __launch_bounds__(kWaveWarps * 32, WaveOcc<T>::value) k_wave(WaveArgs<T> a) {
    using R = WaveRing<T, S, ZERO, UP>;
    constexpr int NB = R::kNB;
    constexpr int AHEAD = R::kAhead;
    constexpr int NR = UP ? S + 2 : S + 3;  // window: rows t-NR+1 .. t, slot NR-1 = row t
    extern __shared__ __align__(128) unsigned char wave_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t item = (int64_t)blockIdx.x * kWaveWarps + warp;
    if (item >= a.nitems) return;
    const int j = find_item(a.item_start, a.nsl, item);
    const LSlice<T> L = a.sl[j];
    if (a.active && !a.active[L.slice]) return;
    const CUtensorMap* map_b = a.maps + 4 * j + 1;
    const CUtensorMap* map_c = a.maps + 4 * j + 2;
    const CUtensorMap* map_u = a.maps + 4 * j + a.u_map;
    const int li = int(item - a.item_start[j]);
    const int strip = li % L.fstrips;
    const int chunk = li / L.fstrips;
    const int X0 = strip * kWaveIW - kWaveHalo;
    const int Y0 = chunk * a.ch;
    const int Y1 = min(Y0 + a.ch, L.ny);
    const int Y1e = Y1 + (Y1 & 1);                 // residual rows run to an even end
    const int tb = Y0 - (UP ? S : S + 1);          // first row of the march
    const int te = UP ? Y1 - 1 + S : Y1e + S;      // last row (each row is loaded once)
    const int k = a.k;
    const T alpha = a.alpha, sk = a.sk;

    const int xlane = X0 + 4 * lane;
    const bool lane_in = xlane >= 0 && xlane < L.nx;  // X0 is a multiple of 4: all-or-none
    const bool interior_lane = lane >= kWaveHalo / 4 && lane < 32 - kWaveHalo / 4;
    // Interior cells (full cells with full neighbours) all share one stencil: the values
    // make_coef returns for them, computed once.  xint: all 4 cells of the lane are interior
    // along x; rows are checked with interior_row.
    AxisCoef<T> one;
    one.w = T(1); one.gm = T(1); one.gp = T(1);
    const Coef<T> ci = make_coef<T>(one, one, k, alpha, sk);
    bool xint = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const AxisCoef<T> q = axis_coef<T>(xlane + i, L.nx, L.n0x, k);
        xint = xint && q.w == T(1) && q.gm == T(1) && q.gp == T(1);
    }

    // prolongation geometry along x (UP): coarse columns cx0-1 .. cx0+2 around the lane
    const int cx0 = X0 / 2 + 2 * lane;
    const int cbox_x = X0 / 2 - 4;  // first coarse column staged (a multiple of 2 elements x 16 B)
    int oI[4], oJ[4];
    T cwx[4];
    bool std_lane = true;  // interior pattern: J = I-1, I+1, I-1, I+1 with weight 1/4
    const bool has_coarse = UP && L.uco != nullptr;
    if (UP) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int I = 0, J = 0;
            T w = T(0);
            if (has_coarse && lane_in) interp_axis<T>(xlane + i, L.n0x, k, L.ncx, I, J, w);
            oI[i] = I - cx0 + 1;
            oJ[i] = J - cx0 + 1;
            cwx[i] = w;
        }
        std_lane = oI[0] == 1 && oJ[0] == 0 && oI[1] == 1 && oJ[1] == 2 && oI[2] == 2 && oJ[2] == 1 &&
                   oI[3] == 2 && oJ[3] == 3 && cwx[0] == T(0.25) && cwx[1] == T(0.25) &&
                   cwx[2] == T(0.25) && cwx[3] == T(0.25);
    }

    // ---- shared-memory ring and its barriers
    unsigned char* ring = wave_smem + (size_t)warp * R::kWarpBytes;   // b rows, then u row + coarse rows
    const uint32_t ring_s = smem_addr(ring);
    const uint32_t uring_s = ring_s + R::kBRingBytes;
    const uint32_t bar_s = uring_s + R::kURingBytes;
    if (lane == 0) {
        for (int s = 0; s < NB; ++s) mbar_init(bar_s + 8 * s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    constexpr uint32_t kRowB = R::kRowBytes;
    // issue the TMA loads of row t into its slot (lane 0 only)
    auto issue = [&](int t) {
        const int slot = (t - tb) & (NB - 1);
        const uint32_t bdst = ring_s + slot * kRowB, bar = bar_s + 8 * slot;
        const uint32_t udst = uring_s + ((t - tb) & (AHEAD - 1)) * R::kUSlotBytes;
        const bool coarse = has_coarse && t >= 0 && t < L.ny;
        uint32_t bytes = kRowB + (ZERO ? 0u : kRowB);
        int y0c = 0;
        if (coarse) {
            int Iy, Jy;
            T wy;
            interp_axis<T>(t, L.n0y, k, L.ncy, Iy, Jy, wy);
            y0c = min(Iy, Jy);
            bytes += kWaveCoarseW * 2 * (uint32_t)sizeof(T);
        }
        // No proxy fence here: the u/coarse slot being refilled was read (LDS) and its values
        // consumed before the __syncwarp that precedes this issue, and the b slot was last
        // read NB - AHEAD - S - 1 >= 5 rows ago.
        mbar_expect_tx(bar, bytes);
        tma_load_2d(bdst, map_b, X0, t, bar);
        if (!ZERO) tma_load_2d(udst, map_u, X0, t, bar);
        if (coarse) tma_load_2d(udst + (ZERO ? 0 : kRowB), map_c, cbox_x, y0c, bar);
    };
    if (lane == 0)
        for (int p = 0; p < AHEAD && tb + p <= te; ++p) issue(tb + p);

    T u[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) u[r][i] = T(0);
    // b of row t - d lives in ring slot (t - d - tb) mod NB; rows before tb read as zero
    auto brow_of = [&](int rr, T (&v)[4]) {
        if (rr < tb) {
            v[0] = v[1] = v[2] = v[3] = T(0);
        } else {
            lds4(ring_s + ((rr - tb) & (NB - 1)) * kRowB + 4 * lane * (uint32_t)sizeof(T), v);
        }
    };
    T rsum[2] = {T(0), T(0)};  // restriction partial sums (DOWN)

#pragma unroll 1
    for (int t = tb; t <= te; ++t) {
        const int n = t - tb;
        const int slot = n & (NB - 1);
        const uint32_t bar = bar_s + 8 * slot;
        if (!mbar_wait_warp(bar, (n / NB) & 1)) {
            // give up: flag the host, let the copies already issued land, leave
            if (lane == 0) atomicExch(a.err, 1);
            for (int tt = t + 1; tt <= te && tt < t + AHEAD; ++tt)
                mbar_wait_warp(bar_s + 8 * ((tt - tb) & (NB - 1)), ((tt - tb) / NB) & 1);
            return;
        }
        // shift the window and bring in row t
#pragma unroll
        for (int r = 0; r < NR - 1; ++r)
#pragma unroll
            for (int i = 0; i < 4; ++i) u[r][i] = u[r + 1][i];
        const uint32_t us_addr = uring_s + (n & (AHEAD - 1)) * R::kUSlotBytes;
        if (ZERO) {
#pragma unroll
            for (int i = 0; i < 4; ++i) u[NR - 1][i] = T(0);
        } else {
            lds4(us_addr + 4 * lane * (uint32_t)sizeof(T), u[NR - 1]);
        }
        // UP: add the interpolated coarse correction to row t
        if (has_coarse && t >= 0 && t < L.ny) {
            int Iy, Jy;
            T wy;
            interp_axis<T>(t, L.n0y, k, L.ncy, Iy, Jy, wy);
            const int y0c = min(Iy, Jy);
            const uint32_t cb = us_addr + (ZERO ? 0 : kRowB);
            const uint32_t c0 = cb + ((Iy - y0c) * kWaveCoarseW + 2 * lane + 3) * (uint32_t)sizeof(T);  // col cx0-1
            const uint32_t c1 = cb + ((Jy - y0c) * kWaveCoarseW + 2 * lane + 3) * (uint32_t)sizeof(T);
            const T v0[4] = {lds1(c0, T(0)), lds1(c0 + sizeof(T), T(0)), lds1(c0 + 2 * sizeof(T), T(0)),
                             lds1(c0 + 3 * sizeof(T), T(0))};
            const T v1[4] = {lds1(c1, T(0)), lds1(c1 + sizeof(T), T(0)), lds1(c1 + 2 * sizeof(T), T(0)),
                             lds1(c1 + 3 * sizeof(T), T(0))};
            if (lane_in) {
                T(&row)[4] = u[NR - 1];
                if (std_lane && xlane + 3 < L.nx) {
                    const T q = T(0.25);
                    row[0] = row[0] + bilinear<T>(v0[1], v0[0], v1[1], v1[0], q, wy);
                    row[1] = row[1] + bilinear<T>(v0[1], v0[2], v1[1], v1[2], q, wy);
                    row[2] = row[2] + bilinear<T>(v0[2], v0[1], v1[2], v1[1], q, wy);
                    row[3] = row[3] + bilinear<T>(v0[2], v0[3], v1[2], v1[3], q, wy);
                } else {
                    prolong_generic<T>(row, v0, v1, oI, oJ, cwx, wy, xlane, L.nx);
                }
            }
        }
        // refill the slot of row t + AHEAD - NB (whose b is no longer needed) with row t + AHEAD
        __syncwarp();
        if (lane == 0 && t + AHEAD <= te) issue(t + AHEAD);

        // half-sweeps: stage s updates row t - s (window slot NR-1-s) with colour (s - 1) & 1
#pragma unroll
        for (int s = 1; s <= S; ++s) {
            const int r = t - s;
            if (r < tb || r < 0 || r >= L.ny) continue;
            T(&row)[4] = u[NR - 1 - s];
            const T(&nrow)[4] = u[NR - 2 - s];
            const T(&srow)[4] = u[NR - s];
            T brow[4];
            brow_of(r, brow);
            const int color = (s - 1) & 1;
            const int first = (xlane + r + color) & 1;  // first cell index with this colour
            const T west = __shfl_up_sync(0xffffffffu, row[3], 1);   // cell 3 of lane-1
            const T east = __shfl_down_sync(0xffffffffu, row[0], 1);  // cell 0 of lane+1
            // Cells outside the level (x < 0 or x >= nx) are updated too: their coefficients
            // decouple them (zero faces), in-level cells give them zero weight, and they are
            // never written back, so no per-cell bounds test is needed.
            if (xint && interior_row(r, L.ny, k)) {
                if (first == 0) {  // cells 0 and 2
                    row[0] = gs_update<T>(ci, brow[0], west, row[1], nrow[0], srow[0]);
                    row[2] = gs_update<T>(ci, brow[2], row[1], row[3], nrow[2], srow[2]);
                } else {           // cells 1 and 3
                    row[1] = gs_update<T>(ci, brow[1], row[0], row[2], nrow[1], srow[1]);
                    row[3] = gs_update<T>(ci, brow[3], row[2], east, nrow[3], srow[3]);
                }
            } else {
                edge_update<T>(row, brow, nrow, srow, first, west, east, xlane, r, L.nx, L.ny, L.n0x, L.n0y, k,
                               alpha, sk);
            }
        }
        // output of the row that completed all half-sweeps
        {
            const int r = t - S;
            if (r >= Y0 && r < Y1 && interior_lane && lane_in) {
                const T(&orow)[4] = u[NR - 1 - S];
                T* dst = (UP ? L.uo : L.u) + (int64_t)r * L.pitch + xlane;
                if (xlane + 3 < L.nx) {
                    Vec4<T>::store(dst, orow);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (xlane + i < L.nx) dst[i] = orow[i];
                }
            }
        }
        if (!UP) {
            // residual of row t - S - 1 (slot 1; neighbours in slots 0 and 2) and its restriction
            const int r = t - S - 1;
            const T(&rrow)[4] = u[1];
            const T west = __shfl_up_sync(0xffffffffu, rrow[3], 1);
            const T east = __shfl_down_sync(0xffffffffu, rrow[0], 1);
            if (r >= Y0 && r < Y1e && L.bc) {
                const bool row_in = r < L.ny && lane_in;
                T res[4] = {T(0), T(0), T(0), T(0)};
                if (row_in) {
                    T brow[4];
                    brow_of(r, brow);
                    if (xint && interior_row(r, L.ny, k)) {
                        res[0] = residual_at<T>(ci, brow[0], rrow[0], west, rrow[1], u[0][0], u[2][0]);
                        res[1] = residual_at<T>(ci, brow[1], rrow[1], rrow[0], rrow[2], u[0][1], u[2][1]);
                        res[2] = residual_at<T>(ci, brow[2], rrow[2], rrow[1], rrow[3], u[0][2], u[2][2]);
                        res[3] = residual_at<T>(ci, brow[3], rrow[3], rrow[2], east, u[0][3], u[2][3]);
                    } else {
                        edge_residual<T>(res, rrow, brow, u[0], u[2], west, east, xlane, r, L.nx, L.ny, L.n0x,
                                         L.n0y, k, alpha, sk);
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
        if (!(a.cont && k == 0)) {  // coarse levels solve for a correction from zero
            for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
                const int y = p / L.nx, x = p - y * L.nx;
                L.u[(int64_t)y * L.pitch + x] = T(0);
            }
            __syncthreads();
        }
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
