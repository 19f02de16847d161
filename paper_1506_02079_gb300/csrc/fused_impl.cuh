// Fused multigrid schedule.
//
// Wavefront kernel (k_wave).  One warp owns a strip of 128 cells (32 lanes x 4 consecutive
// cells) and marches down a chunk of rows two at a time.  All nu red-black sweeps are
// pipelined in one pass: at step T the warp receives row pair T (rows 2T, 2T+1) and applies
// half-sweep s (s = 1..S, S = 2 nu) to pair T - s.  Half-sweep s only reads the other colour,
// whose latest update (half-sweep s - 1) reached pairs T-s-1 .. T-s+1 before half-sweep s + 1
// touches them, so the result is exactly that of S global half-sweeps (Gauss-Seidel
// red-black, colour (x + y) mod 2).  Row pairs arrive by TMA (one 128 x 2 box per array) into
// a per-warp shared-memory ring guarded by mbarriers with bounded waits; u moves into a
// register window of S + 3 pairs, b is read from the ring when a half-sweep needs it.
// Neighbours along x come from warp shuffles, so strip edges are recomputed by the adjacent
// strips (8-cell overlap on each side).
//
//   DOWN (restriction leg): optional zero initial guess (the first half-sweep then needs no
//        load of u), S half-sweeps, the residual of the pair S + 1 behind, and its 2x2 sums / 4
//        written as one row of the next level's right-hand side.  One read of b
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

#include <type_traits>

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

// CTAs per SM the register budget is sized for: the register window grows with the sweeps (S + 3
// row pairs) and FP64 windows take twice the registers.
template <class T, int S>
struct WaveOcc { static constexpr int value = (sizeof(T) == 4 && S <= 4) ? 4 : 2; };

// ---------------------------------------------------------------- per-cell stencils
// Interior cells (full cells with full neighbours) all share one stencil.  Cells on a slice
// edge, a partial coarse cell or outside the level take per-cell stencils: selects at level 0
// (alpha + degree and its reciprocal formed when needed, so that nothing of these rare paths
// stays live in registers across the march), the general finite-volume formula out of line on
// coarse levels.
template <class T>
struct StencilTab {
    Coef<T> ci;   // interior stencil
};

// Per-lane diagonal of the interior body (see "ghost strips" in k_wave): 1 / D of cell 0, of
// cells 1 and 2 and of cell 3 of the lane, and D of cells 0 and 3 (cells 1 and 2 always have the
// interior D).  Interior lanes hold the interior values; lanes outside the level 1 / D = 0.
template <class T>
struct LaneDiag {
    T iD0, iD12, iD3;
    T D0, D3;
};

// gs_update with the reciprocal diagonal given separately (same operations, same order).
template <class T>
__device__ __forceinline__ T gs_update_iD(const Coef<T>& c, T iD, T b, T uw, T ue, T un, T us) {
    T acc = fma_t(c.cw, uw, b);
    acc = fma_t(c.ce, ue, acc);
    acc = fma_t(c.cn, un, acc);
    acc = fma_t(c.cs, us, acc);
    return mul_t(acc, iD);
}

// residual_at with the diagonal given separately (same operations, same order).
template <class T>
__device__ __forceinline__ T residual_at_D(const Coef<T>& c, T D, T b, T u, T uw, T ue, T un, T us) {
    T acc = fma_t(c.cw, uw, b);
    acc = fma_t(c.ce, ue, acc);
    acc = fma_t(c.cn, un, acc);
    acc = fma_t(c.cs, us, acc);
    return fma_t(-D, u, acc);
}

template <class T>
__device__ __forceinline__ void make_stencil_tab(StencilTab<T>& tab, int k, T alpha, T sk) {
    AxisCoef<T> one;
    one.w = T(1); one.gm = T(1); one.gp = T(1);
    tab.ci = make_coef<T>(one, one, k, alpha, sk);
}

// Level-0 stencil of cell (x, r) from selects; equal to make_coef at level 0.
template <class T>
__device__ __forceinline__ Coef<T> level0_coef(int x, int r, int nx, int ny, T alpha) {
    Coef<T> c;
    const bool in = x >= 0 && x < nx && r >= 0 && r < ny;
    const int w = in && x > 0, e = in && x + 1 < nx, n = in && r > 0, s = in && r + 1 < ny;
    c.cw = T(w); c.ce = T(e); c.cn = T(n); c.cs = T(s);
    // alpha + (((cw + ce) + cn) + cs) for 0/1 coefficients; outside the level the cell is
    // decoupled (the w = 1 cell of axis_coef): D = alpha
    c.D = alpha + T(w + e + n + s);
    c.iD = rcp_t(c.D);
    return c;
}

template <class T>
__device__ __noinline__ Coef<T> coarse_cell_coef(int x, int r, int nx, int ny, int n0x, int n0y, int k, T alpha,
                                                 T sk) {
    return make_coef<T>(axis_coef<T>(x, nx, n0x, k), axis_coef<T>(r, ny, n0y, k), k, alpha, sk);
}

template <class T>
__device__ __forceinline__ Coef<T> edge_coef(const StencilTab<T>& tab, int x, int r, int nx, int ny, int n0x,
                                             int n0y, int k, T alpha, T sk) {
    return k == 0 ? level0_coef<T>(x, r, nx, ny, alpha) : coarse_cell_coef<T>(x, r, nx, ny, n0x, n0y, k, alpha, sk);
}

// Stencil of cell i of the lane on an interior row, from the lane's shared-memory cache
// (cw, ce, cn = cs, D, 1/D per cell, as make_coef returns them on such a row).
template <class T>
__device__ __forceinline__ Coef<T> cached_coef(uint32_t cache, int i) {
    Coef<T> c;
    const uint32_t a = cache + i * 5 * (uint32_t)sizeof(T);
    c.cw = lds1(a, T(0));
    c.ce = lds1(a + sizeof(T), T(0));
    c.cn = lds1(a + 2 * sizeof(T), T(0));
    c.cs = c.cn;
    c.D = lds1(a + 3 * sizeof(T), T(0));
    c.iD = lds1(a + 4 * sizeof(T), T(0));
    return c;
}

// Half-sweep of one colour on one row of the lane's 4 cells (cells f and f + 2).
template <class T, bool FAST>
__device__ __forceinline__ void sweep_row(T (&row)[4], const T (&brow)[4], const T (&nrow)[4], const T (&srow)[4],
                                          int f, T west, T east, bool fast, bool irow, uint32_t cache,
                                          const StencilTab<T>& tab, const LaneDiag<T>& g, int xlane, int r, int nx,
                                          int ny, int n0x, int n0y, int k, T alpha, T sk) {
    if (FAST || fast) {
        if (f == 0) {
            row[0] = gs_update_iD<T>(tab.ci, g.iD0, brow[0], west, row[1], nrow[0], srow[0]);
            row[2] = gs_update_iD<T>(tab.ci, g.iD12, brow[2], row[1], row[3], nrow[2], srow[2]);
        } else {
            row[1] = gs_update_iD<T>(tab.ci, g.iD12, brow[1], row[0], row[2], nrow[1], srow[1]);
            row[3] = gs_update_iD<T>(tab.ci, g.iD3, brow[3], row[2], east, nrow[3], srow[3]);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = 2 * h + f;
            const T uw = i == 0 ? west : row[i - 1];
            const T ue = i == 3 ? east : row[i + 1];
            const Coef<T> c = irow ? cached_coef<T>(cache, i)
                                   : edge_coef<T>(tab, xlane + i, r, nx, ny, n0x, n0y, k, alpha, sk);
            row[i] = gs_update<T>(c, brow[i], uw, ue, nrow[i], srow[i]);
        }
    }
}

// Residuals of one row of the lane's 4 cells.
template <class T, bool FAST>
__device__ __forceinline__ void residual_row(T (&res)[4], const T (&row)[4], const T (&brow)[4], const T (&nrow)[4],
                                             const T (&srow)[4], T west, T east, bool fast, bool irow,
                                             uint32_t cache, const StencilTab<T>& tab, const LaneDiag<T>& g,
                                             int xlane, int r, int nx, int ny, int n0x, int n0y, int k, T alpha,
                                             T sk) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T uw = i == 0 ? west : row[i - 1];
        const T ue = i == 3 ? east : row[i + 1];
        if (FAST || fast) {
            const T D = i == 0 ? g.D0 : (i == 3 ? g.D3 : tab.ci.D);
            res[i] = residual_at_D<T>(tab.ci, D, brow[i], row[i], uw, ue, nrow[i], srow[i]);
        } else {
            const Coef<T> c = irow ? cached_coef<T>(cache, i)
                                   : edge_coef<T>(tab, xlane + i, r, nx, ny, n0x, n0y, k, alpha, sk);
            res[i] = residual_at<T>(c, brow[i], row[i], uw, ue, nrow[i], srow[i]);
        }
    }
}

// Prolongation for lanes whose cells do not follow the interior 1/4-3/4 pattern; v0 / v1 hold
// coarse columns cx0 - 1 .. cx0 + 2.  The interpolation along x is formed here, when needed,
// so that nothing of this rare path stays live in registers across the march.
template <class T>
__device__ __forceinline__ void prolong_generic(T (&uu)[4], const T (&v0)[4], const T (&v1)[4], int cx0, T wy,
                                                int xlane, int nx, int n0x, int k, int ncx) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (xlane + i >= nx) continue;
        int I, J;
        T wx;
        interp_axis<T>(xlane + i, n0x, k, ncx, I, J, wx);
        const int oI = I - cx0 + 1, oJ = J - cx0 + 1;
        uu[i] = uu[i] + bilinear<T>(pick4<T>(v0, oI), pick4<T>(v0, oJ), pick4<T>(v1, oI), pick4<T>(v1, oJ), wx, wy);
    }
}

// Shared-memory rings of one warp, in units of row pairs.  b: one slot per pair from the
// oldest pair still needed (the residual pair, S + 1 behind the newest) to the newest pair in
// flight; u and the coarse rows (UP) are consumed when their pair arrives, so kAhead slots.
template <class T, int S, bool ZERO, bool UP>
struct WaveRing {
    static constexpr int kAhead = 2;                                         // pairs in flight
    static constexpr int kNB = kAhead + S + (UP ? 1 : 2);                    // b slots = barriers
    static constexpr int kPairBytes = 2 * kWaveWidth * (int)sizeof(T);
    static constexpr int kCoarseBytes = UP ? (kWaveCoarseW * 3 * (int)sizeof(T) + 127) / 128 * 128 : 0;
    static constexpr int kUSlotBytes = (ZERO ? 0 : kPairBytes) + kCoarseBytes;
    static constexpr int kBRingBytes = kNB * kPairBytes;
    static constexpr int kURingBytes = kAhead * kUSlotBytes;
    static constexpr int kCoefBytes = 32 * 4 * 5 * (int)sizeof(T);       // per-lane stencil cache
    static constexpr int kWarpBytes = kBRingBytes + kURingBytes + kCoefBytes + (kNB * 8 + 127) / 128 * 128;
};

template <class T, int S, bool ZERO, bool UP>
constexpr int wave_smem_bytes() { return kWaveWarps * WaveRing<T, S, ZERO, UP>::kWarpBytes; }

template <class T, int S, bool ZERO, bool UP>
__global__ void __launch_bounds__(kWaveWarps * 32, WaveOcc<T, S>::value) k_wave(WaveArgs<T> a) {
    using R = WaveRing<T, S, ZERO, UP>;
    constexpr int NB = R::kNB;
    constexpr int AHEAD = R::kAhead;
    constexpr int NR = UP ? S + 2 : S + 3;      // window: pairs T-NR+1 .. T (slot NR-1 = pair T)
    constexpr int HP = UP ? (S + 1) / 2 : (S + 2) / 2;  // halo pairs above the chunk
    constexpr uint32_t kRowB = kWaveWidth * sizeof(T);
    extern __shared__ __align__(128) unsigned char wave_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // ---- rings and barriers of this warp, set up once: the warp runs work items back to back
    // through them, taking the next item from the launch's work counter (items are independent,
    // so the order does not change any result)
    unsigned char* ring = wave_smem + (size_t)warp * R::kWarpBytes;
    const uint32_t ring_s = smem_addr(ring);
    const uint32_t uring_s = ring_s + R::kBRingBytes;
    const uint32_t coef_s = uring_s + R::kURingBytes + lane * 20 * (uint32_t)sizeof(T);
    const uint32_t bar_s = uring_s + R::kURingBytes + R::kCoefBytes;
    if (lane == 0) {
        for (int q = 0; q < NB; ++q) mbar_init(bar_s + 8 * q, 1);
        mbar_init_fence();
    }
    __syncwarp();
    int bs = 0, us = 0;  // ring slots of the next pair
    uint32_t phase = 0;  // parity of the b-slot barriers in the current lap

    // One work item: a strip of 128 columns and a chunk of rows of one slice.  Returns false
    // when a bounded wait gave up.
    auto run_item = [&](const int64_t item) -> bool {
    const int j = find_item(a.item_start, a.nsl, item);
    const LSlice<T> L = a.sl[j];
    if (a.active && !a.active[L.slice]) return true;
    const CUtensorMap* map_b = a.maps + 4 * j + 1;
    const CUtensorMap* map_c = a.maps + 4 * j + 2;
    const CUtensorMap* map_u = a.maps + 4 * j + a.u_map;
    const int li = int(item - a.item_start[j]);
    // consecutive items walk down one strip; the two edge strips (slower: per-cell stencils on
    // all their lanes) are handed out first, so that they do not finish last
    const int nchunks = (L.ny + a.ch - 1) / a.ch;
    const int sidx = li / nchunks;
    const int strip = L.fstrips < 2 || sidx == 0 ? sidx : (sidx == 1 ? L.fstrips - 1 : sidx - 1);
    const int chunk = li - sidx * nchunks;
    const int X0 = strip * kWaveIW - kWaveHalo;
    const int Y0 = chunk * a.ch;                  // even
    const int Y1 = min(Y0 + a.ch, L.ny);
    const int P0 = Y0 >> 1, P1 = (Y1 + 1) >> 1;   // output pairs [P0, P1)
    const int pb = P0 - HP;                       // first pair of the march
    const int te = UP ? P1 - 1 + S : P1 + S;      // last pair (each pair is loaded once)
    const int k = a.k;
    const T alpha = a.alpha, sk = a.sk;
    const int nx = L.nx, ny = L.ny;

    const int xlane = X0 + 4 * lane;
    const bool lane_in = xlane >= 0 && xlane < nx;  // X0 is a multiple of 4: all-or-none
    const bool interior_lane = lane >= kWaveHalo / 4 && lane < 32 - kWaveHalo / 4;
    StencilTab<T> tab;
    make_stencil_tab<T>(tab, k, alpha, sk);

    // Ghost strips.  A strip whose lanes are each wholly inside or wholly outside the level, and
    // whose in-level cells are all interior along x except the level's first cell (cell 0 of a
    // lane) and last cell (cell 3 of a lane) with their one-sided stencils (and for UP, there,
    // the injection from the coarse cell), runs its interior rows with the interior body too.
    // Cells outside the level are kept at exactly 0 there: their 1 / D is 0 and no coarse
    // correction is added to them (weight pm = 0; TMA fills them with 0 on every load).  A
    // boundary cell's missing neighbour then enters the interior stencil as 0, which adds
    // nothing (fma(c, 0, acc) = acc), and only its diagonal differs from the interior one: the
    // lane's iD0 / D0 or iD3 / D3 (LaneDiag), and its interpolation weight along x is 0 (wx0 /
    // wx3).  The operations and their order are those of the per-cell stencils, so the results
    // are the same bit for bit.  Every strip of a level whose width is a multiple of 4 and whose
    // coarse cells are full qualifies; others take the general body.
    const bool all_in = xlane >= 0 && xlane + 3 < nx;
    const bool all_out = xlane + 3 < 0 || xlane >= nx;
    bool ghost_ok = all_in || all_out;
    LaneDiag<T> g;
    g.iD0 = g.iD12 = g.iD3 = all_out ? T(0) : tab.ci.iD;
    g.D0 = g.D3 = tab.ci.D;
    T wx0 = T(0.25), wx3 = T(0.25);
    const T pm = all_out ? T(0) : T(1);
    if (all_in) {
        AxisCoef<T> one;
        one.w = T(1); one.gm = T(1); one.gp = T(1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const AxisCoef<T> q = axis_coef<T>(xlane + i, nx, L.n0x, k);
            if (q.w == T(1) && q.gm == T(1) && q.gp == T(1)) continue;
            const bool first = i == 0 && xlane == 0 && q.w == T(1) && q.gm == T(0) && q.gp == T(1);
            const bool last = i == 3 && xlane + 3 == nx - 1 && q.w == T(1) && q.gm == T(1) && q.gp == T(0);
            if (!(first || last)) {
                ghost_ok = false;
                continue;
            }
            const Coef<T> c = make_coef<T>(q, one, k, alpha, sk);
            if (i == 0) { g.iD0 = c.iD; g.D0 = c.D; }
            if (i == 3) { g.iD3 = c.iD; g.D3 = c.D; }
        }
    }

    // prolongation geometry along x (UP): coarse columns cx0-1 .. cx0+2 around the lane
    const int cx0 = X0 / 2 + 2 * lane;
    const int cbox_x = X0 / 2 - 4;  // first staged coarse column (x * size stays 16-B aligned)
    bool std_lane = true;  // interior pattern: J = I-1, I+1, I-1, I+1 with weight 1/4
    const bool has_coarse = UP && L.uco != nullptr;
    if (UP) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int I = 0, J = 0;
            T w = T(0);
            if (has_coarse && lane_in) interp_axis<T>(xlane + i, L.n0x, k, L.ncx, I, J, w);
            const int oI = I - cx0 + 1, oJ = J - cx0 + 1;
            const int sI = i < 2 ? 1 : 2, sJ = (i == 0 || i == 2) ? sI - 1 : sI + 1;  // interior pattern
            if (oI == sI && oJ == sJ && w == T(0.25)) continue;
            std_lane = false;
            // injection (J = I, weight 0) at the level's first / last cell keeps a ghost strip
            const bool edge_cell = (i == 0 && xlane == 0) || (i == 3 && xlane + 3 == nx - 1);
            if (has_coarse && all_in && edge_cell && oI == sI && J == I && w == T(0)) {
                if (i == 0) wx0 = T(0);
                if (i == 3) wx3 = T(0);
            } else if (has_coarse && all_in) {
                ghost_ok = false;
            }
        }
    }

    {  // cache this lane's stencils for interior rows (read when the row pair is not all-interior)
        AxisCoef<T> one;
        one.w = T(1); one.gm = T(1); one.gp = T(1);
        T* cc = reinterpret_cast<T*>(ring + (coef_s - ring_s));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const Coef<T> c = make_coef<T>(axis_coef<T>(xlane + i, nx, L.n0x, k), one, k, alpha, sk);
            cc[5 * i + 0] = c.cw;
            cc[5 * i + 1] = c.ce;
            cc[5 * i + 2] = c.cn;
            cc[5 * i + 3] = c.D;
            cc[5 * i + 4] = c.iD;
        }
    }
    __syncwarp();
    // TMA loads of pair P (lane 0): b (and u) rows 2P, 2P+1; coarse rows P-1 .. P+1 (UP)
    auto issue = [&](int P, int bslot, int uslot) {
        const uint32_t bar = bar_s + 8 * bslot;
        const uint32_t udst = uring_s + uslot * R::kUSlotBytes;
        const bool coarse = has_coarse && 2 * P < ny && 2 * P + 1 >= 0;
        const uint32_t bytes = R::kPairBytes + (ZERO ? 0u : (uint32_t)R::kPairBytes) +
                               (coarse ? (uint32_t)(kWaveCoarseW * 3 * sizeof(T)) : 0u);
        mbar_expect_tx(bar, bytes);
        tma_load_2d(ring_s + bslot * R::kPairBytes, map_b, X0, 2 * P, bar);
        if (!ZERO) tma_load_2d(udst, map_u, X0, 2 * P, bar);
        if (coarse) tma_load_2d(udst + (ZERO ? 0 : R::kPairBytes), map_c, cbox_x, P - 1, bar);
    };
    // the ring's slots were last read by the previous item: order those reads before the
    // copies that overwrite them
    fence_proxy_async();
    if (lane == 0)
        for (int p = 0; p < AHEAD && pb + p <= te; ++p) {
            const int b2 = bs + p, u2 = us + p;
            issue(pb + p, b2 >= NB ? b2 - NB : b2, u2 >= AHEAD ? u2 - AHEAD : u2);
        }

    T w[NR][2][4];  // window of u pairs in registers
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 4; ++i) w[q][h][i] = T(0);
    auto bslot_of = [&](int bs, int back) { const int q = bs - back; return q < 0 ? q + NB : q; };
    auto load_b = [&](int bslot, int h, T (&v)[4]) {
        lds4(ring_s + bslot * R::kPairBytes + h * kRowB + 4 * lane * (uint32_t)sizeof(T), v);
    };

    // Steps whose every updated row is an interior row, in a strip whose lanes all take the
    // interior stencil along x (and for UP the regular 1/4-3/4 prolongation pattern), run a
    // step body specialised to the interior stencil; the others the general one.  The choice
    // is warp-uniform, so each step executes exactly one of the two bodies.
    const bool x_ghost = __all_sync(0xffffffffu, ghost_ok);

    auto step = [&](auto fast_tag, const int T_) {
        constexpr bool FAST = decltype(fast_tag)::value;
        {
            // shift the window and bring in pair T
#pragma unroll
            for (int q = 0; q < NR - 1; ++q)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int i = 0; i < 4; ++i) w[q][h][i] = w[q + 1][h][i];
            const uint32_t us_addr = uring_s + us * R::kUSlotBytes;
            if (ZERO) {
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int i = 0; i < 4; ++i) w[NR - 1][h][i] = T(0);
            } else {
                lds4(us_addr + 4 * lane * (uint32_t)sizeof(T), w[NR - 1][0]);
                lds4(us_addr + kRowB + 4 * lane * (uint32_t)sizeof(T), w[NR - 1][1]);
            }
            // UP: add the interpolated coarse correction to rows 2T and 2T+1
            if (has_coarse && (FAST || (2 * T_ < ny && 2 * T_ + 1 >= 0))) {
                const uint32_t cb = us_addr + (ZERO ? 0 : R::kPairBytes);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = 2 * T_ + h;
                    if (!FAST && (r < 0 || r >= ny)) continue;
                    int Iy, Jy;
                    T wy;
                    if (FAST) {  // interior pattern along y (the step's rows are >= 2 and below the last two coarse rows)
                        Iy = T_;
                        Jy = h ? T_ + 1 : T_ - 1;
                        wy = T(0.25);
                    } else {
                        interp_axis<T>(r, L.n0y, k, L.ncy, Iy, Jy, wy);
                    }
                    // coarse row q sits at box row q - (T - 1); columns cx0-1 .. cx0+2 at 2l+3 .. 2l+6
                    const uint32_t c0 = cb + ((Iy - T_ + 1) * kWaveCoarseW + 2 * lane + 2) * (uint32_t)sizeof(T);
                    const uint32_t c1 = cb + ((Jy - T_ + 1) * kWaveCoarseW + 2 * lane + 2) * (uint32_t)sizeof(T);
                    T a0[6], a1[6];  // columns 2l+2 .. 2l+7 of the box (8-byte aligned pairs)
#pragma unroll
                    for (int m = 0; m < 6; m += 2) {
                        lds2(c0 + m * sizeof(T), a0[m], a0[m + 1]);
                        lds2(c1 + m * sizeof(T), a1[m], a1[m + 1]);
                    }
                    const T v0[4] = {a0[1], a0[2], a0[3], a0[4]};
                    const T v1[4] = {a1[1], a1[2], a1[3], a1[4]};
                    if (!FAST && !lane_in) continue;
                    T(&row)[4] = w[NR - 1][h];
                    const T q4 = T(0.25);
                    if (FAST) {
                        // interior pattern, with the ghost-strip weights (fma(1, p, u) = u + p)
                        row[0] = fma_t(pm, bilinear<T>(v0[1], v0[0], v1[1], v1[0], wx0, wy), row[0]);
                        row[1] = fma_t(pm, bilinear<T>(v0[1], v0[2], v1[1], v1[2], q4, wy), row[1]);
                        row[2] = fma_t(pm, bilinear<T>(v0[2], v0[1], v1[2], v1[1], q4, wy), row[2]);
                        row[3] = fma_t(pm, bilinear<T>(v0[2], v0[3], v1[2], v1[3], wx3, wy), row[3]);
                    } else if (std_lane && xlane + 3 < nx) {
                        row[0] = row[0] + bilinear<T>(v0[1], v0[0], v1[1], v1[0], q4, wy);
                        row[1] = row[1] + bilinear<T>(v0[1], v0[2], v1[1], v1[2], q4, wy);
                        row[2] = row[2] + bilinear<T>(v0[2], v0[1], v1[2], v1[1], q4, wy);
                        row[3] = row[3] + bilinear<T>(v0[2], v0[3], v1[2], v1[3], q4, wy);
                    } else {
                        prolong_generic<T>(row, v0, v1, cx0, wy, xlane, nx, L.n0x, k, L.ncx);
                    }
                }
            }
            // refill: pair T + AHEAD into the b slot of pair T + AHEAD - NB (no longer needed)
            // and the u/coarse slot of pair T (just consumed)
            __syncwarp();
            {
                int nbs = bs + AHEAD;
                if (nbs >= NB) nbs -= NB;
                if (lane == 0 && T_ + AHEAD <= te) issue(T_ + AHEAD, nbs, us);
            }

            // half-sweeps: stage s updates pair T - s (window slot NR-1-s) with colour (s - 1) & 1
#pragma unroll
            for (int s = 1; s <= S; ++s) {
                const int m = T_ - s;
                const int r0 = 2 * m, r1 = 2 * m + 1;
                if (!FAST && (m < pb || r0 >= ny || r1 < 0)) continue;
                T(&p0)[4] = w[NR - 1 - s][0];
                T(&p1)[4] = w[NR - 1 - s][1];
                const T(&north)[4] = w[NR - 2 - s][1];  // row 2m - 1
                const T(&south)[4] = w[NR - s][0];      // row 2m + 2
                const int bq = bslot_of(bs, s);
                T b0[4], b1[4];
                load_b(bq, 0, b0);
                load_b(bq, 1, b1);
                const int f0 = (r0 + ((s - 1) & 1)) & 1;  // first cell of the colour on row r0
                // Row r0 updates cells {0, 2} (needs cell 3 of lane-1) when f0 == 0, else {1, 3}
                // (needs cell 0 of lane+1); row r1 the other way round.  One shuffle per row.
                const int d0 = f0 == 0 ? -1 : 1;
                const T x0 = __shfl_sync(0xffffffffu, f0 == 0 ? p0[3] : p0[0], lane + d0);
                const T x1 = __shfl_sync(0xffffffffu, f0 == 0 ? p1[0] : p1[3], lane - d0);
                const bool ir0 = FAST || interior_row(r0, ny, k), ir1 = FAST || interior_row(r1, ny, k);
                // warp-uniform: in a strip with edge lanes every lane reads its cached stencil
                // (an interior lane's cached stencil is the interior one), so no lane diverges
                const bool fast = FAST || (x_ghost && ir0 && ir1);
                sweep_row<T, FAST>(p0, b0, north, p1, f0, x0, x0, fast, ir0, coef_s, tab, g, xlane, r0, nx, ny,
                                   L.n0x, L.n0y, k, alpha, sk);
                if (FAST || r1 < ny)
                    sweep_row<T, FAST>(p1, b1, p0, south, f0 ^ 1, x1, x1, fast, ir1, coef_s, tab, g, xlane, r1, nx,
                                       ny, L.n0x, L.n0y, k, alpha, sk);
            }
            // output of the pair that completed all half-sweeps
            {
                const int m = T_ - S;
                if (interior_lane && lane_in && (FAST || (m >= P0 && m < P1))) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int r = 2 * m + h;
                        if (!FAST && r >= Y1) continue;
                        const T(&orow)[4] = w[NR - 1 - S][h];
                        T* dst = (UP ? L.uo : L.u) + (int64_t)r * L.pitch + xlane;
                        if (FAST || xlane + 3 < nx) {
                            Vec4<T>::store(dst, orow);
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (xlane + i < nx) dst[i] = orow[i];
                        }
                    }
                }
            }
            if (!UP) {
                // residual of pair m = T - S - 1 (slot 1; neighbours in slots 0 and 2) and its
                // 2x2 restriction: rows 2m and 2m+1 form coarse row m
                const int m = T_ - S - 1;
                const T(&q0)[4] = w[1][0];
                const T(&q1)[4] = w[1][1];
                const T w0 = __shfl_up_sync(0xffffffffu, q0[3], 1);
                const T e0 = __shfl_down_sync(0xffffffffu, q0[0], 1);
                const T w1 = __shfl_up_sync(0xffffffffu, q1[3], 1);
                const T e1 = __shfl_down_sync(0xffffffffu, q1[0], 1);
                if (L.bc && (FAST || (m >= P0 && m < P1 && lane_in))) {
                    const int r0 = 2 * m, r1 = 2 * m + 1;
                    const int bq = bslot_of(bs, S + 1);
                    T b0[4], b1[4];
                    load_b(bq, 0, b0);
                    load_b(bq, 1, b1);
                    const bool ir0 = FAST || interior_row(r0, ny, k), ir1 = FAST || interior_row(r1, ny, k);
                    const bool fast = FAST || (x_ghost && ir0 && ir1);
                    T res0[4], res1[4] = {T(0), T(0), T(0), T(0)};
                    residual_row<T, FAST>(res0, q0, b0, w[0][1], q1, w0, e0, fast, ir0, coef_s, tab, g, xlane, r0,
                                          nx, ny, L.n0x, L.n0y, k, alpha, sk);
                    const bool has_r1 = FAST || r1 < ny;
                    if (has_r1)
                        residual_row<T, FAST>(res1, q1, b1, q0, w[2][0], w1, e1, fast, ir1, coef_s, tab, g, xlane,
                                              r1, nx, ny, L.n0x, L.n0y, k, alpha, sk);
                    // same summation order as the reference restriction: (((0 + r00) + r01) + r10) + r11
                    T c0 = T(0), c1 = T(0);
                    if (FAST || xlane + 0 < nx) c0 = c0 + res0[0];
                    if (FAST || xlane + 1 < nx) c0 = c0 + res0[1];
                    if (FAST || xlane + 2 < nx) c1 = c1 + res0[2];
                    if (FAST || xlane + 3 < nx) c1 = c1 + res0[3];
                    if (has_r1) {
                        if (FAST || xlane + 0 < nx) c0 = c0 + res1[0];
                        if (FAST || xlane + 1 < nx) c0 = c0 + res1[1];
                        if (FAST || xlane + 2 < nx) c1 = c1 + res1[2];
                        if (FAST || xlane + 3 < nx) c1 = c1 + res1[3];
                    }
                    if (interior_lane && m < L.ncy) {
                        T* dst = L.bc + (int64_t)m * L.pitchc + cx0;
                        const T v0 = c0 * T(0.25), v1 = c1 * T(0.25);
                        if (cx0 + 1 < L.ncx) Vec2<T>::store(dst, v0, v1);
                        else if (cx0 < L.ncx) dst[0] = v0;
                    }
                }
            }
        }
    };
#pragma unroll 1
    for (int T_ = pb; T_ <= te; ++T_) {
        if (!mbar_wait_warp(bar_s + 8 * bs, phase)) {
            // give up: flag the host, let the copies already issued land, leave
            if (lane == 0) atomicExch(a.err, 1);
            int b2 = bs, ph2 = phase;
            for (int tt = T_ + 1; tt <= te && tt < T_ + AHEAD; ++tt) {
                if (++b2 == NB) { b2 = 0; ph2 ^= 1; }
                mbar_wait_warp(bar_s + 8 * b2, ph2);
            }
            return false;
        }
        // The interior body also drops the range checks of a march step, so it is taken where
        // every stage has its pair (T - S >= first pair of the march), the output pair T - S
        // and the residual pair T - S - 1 (DOWN) lie in this chunk, the prolongation rows 2T,
        // 2T + 1 (UP) in the level with the interior interpolation pattern along y (coarse rows
        // T - 1 .. T + 1 all full: T + 2 < the coarse level's rows), and every row the step
        // updates is an interior row
        // (pairs T - S - 1 .. T - 1; interior rows form one contiguous range).
        const int rlo = 2 * (T_ - S - (UP ? 0 : 1)), rhi = 2 * T_ - 1;
        const bool steady = T_ >= P0 + S + (UP ? 0 : 1) && 2 * (T_ - S) + 1 < Y1 && T_ - S < P1 &&
                            (!UP || (2 * T_ + 1 < ny && (!has_coarse || T_ + 2 < L.ncy)));
        if (x_ghost && steady && interior_row(rlo, ny, k) && interior_row(rhi, ny, k))
            step(std::true_type{}, T_);
        else
            step(std::false_type{}, T_);
        if (++bs == NB) { bs = 0; phase ^= 1; }
        if (++us == AHEAD) us = 0;
    }
    return true;
    };

    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(a.work, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= a.nitems) break;
        if (!run_item((int64_t)item)) return;  // the host sees the error word and resets the counters
    }
    // the last warp of the launch to finish resets the counters for the next launch on this stream
    if (lane == 0) {
        const unsigned int total = gridDim.x * (unsigned int)kWaveWarps;
        if (atomicAdd(a.work + 1, 1u) == total - 1) {
            atomicExch(a.work, 0u);
            atomicExch(a.work + 1, 0u);
        }
    }
}

// ---------------------------------------------------------------- coarse tail
// The levels of one slice from kc (the first with both sides <= kTailMax) down to 1 x 1 are run
// by one CTA on copies in shared memory (dense rows): at most 64 x 64 + 32 x 32 + ... cells, u and
// b each.  Only level kc touches global memory: its right-hand side (and, continuing at level 0,
// its iterate) is read at the start and its final iterate written at the end, where the wavefront
// UP kernel of level kc - 1 (or the residual kernel, at kc = 0) reads it.  The per-cell arithmetic
// and its order are those of every other schedule.
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

constexpr int kTailMaxLevels = 16;

template <class T>
__global__ void __launch_bounds__(512) k_tail(TailArgs<T> a) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    const int j = blockIdx.x;
    if (a.active && !a.active[j]) return;
    const LSlice<T>* lv = a.table + a.level_off[j];
    const int kc = a.kc[j];
    const int K = a.nlev[j] - 1;
    if (K - kc + 1 > kTailMaxLevels) return;  // never: a 64 x 64 level has 7 levels below it
    // shared-memory copies of levels kc .. K: u then b, dense rows; their descriptors once per CTA
    __shared__ LSlice<T> sl[kTailMaxLevels];
    if (threadIdx.x == 0) {
        T* q = reinterpret_cast<T*>(tail_smem);
        for (int k = kc; k <= K; ++k) {
            LSlice<T> L = lv[k];
            L.pitch = L.nx;
            L.u = q;
            q += (size_t)L.nx * L.ny;
            L.b = q;
            q += (size_t)L.nx * L.ny;
            sl[k - kc] = L;
        }
        for (int k = kc; k < K; ++k) {
            sl[k - kc].uc = sl[k + 1 - kc].u;
            sl[k - kc].bc = sl[k + 1 - kc].b;
            sl[k - kc].pitchc = sl[k + 1 - kc].pitch;
        }
    }
    __syncthreads();
    {   // level kc from global memory: its rhs, and its iterate when continuing at level 0
        const LSlice<T>& G = lv[kc];
        const LSlice<T>& L = sl[0];
        const bool cont = a.cont && kc == 0;
        for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
            const int y = p / L.nx, x = p - y * L.nx;
            const int64_t g = (int64_t)y * G.pitch + x;
            L.b[p] = G.b[g];
            L.u[p] = cont ? G.u[g] : T(0);  // coarse levels solve for a correction from zero
        }
        __syncthreads();
    }
    for (int k = kc; k <= K; ++k) {
        const LSlice<T>& L = sl[k - kc];
        const T sk = T(ldexp(1.0, -2 * k));
        if (k > kc) {
            for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) L.u[p] = T(0);
            __syncthreads();
        }
        tail_relax<T>(L, k, a.alpha, sk, a.nu_pre);
        if (k < K) {
            const LSlice<T>& C = sl[k + 1 - kc];
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
        const LSlice<T>& L = sl[k - kc];
        const T sk = T(ldexp(1.0, -2 * k));
        for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
            const int y = p / L.nx, x = p - y * L.nx;
            L.u[(int64_t)y * L.pitch + x] += prolong_at<T>(L.uc, L.pitchc, x, y, L.ncx, L.ncy, L.n0x, L.n0y, k);
        }
        __syncthreads();
        tail_relax<T>(L, k, a.alpha, sk, a.nu_post);
    }
    {   // the final iterate of level kc back to global memory
        const LSlice<T>& G = lv[kc];
        const LSlice<T>& L = sl[0];
        for (int p = threadIdx.x; p < L.nx * L.ny; p += blockDim.x) {
            const int y = p / L.nx, x = p - y * L.nx;
            G.u[(int64_t)y * G.pitch + x] = L.u[p];
        }
    }
}

}  // namespace fused_detail
}  // namespace emfuse
