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
#include <map>
#include <memory>
#include <tuple>
#include <mutex>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"
#include "fpconv.cuh"
#include "mg_fused.cuh"
#include "tma.cuh"

namespace emfuse {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;


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
    const int j = find_item(a.tile_start, a.nsl, t);
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
    const int j = find_item(a.tile_start, a.nsl, t);
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
    const int j = find_item(a.tile_start, a.nsl, t);
    const LSlice<T> S = a.sl[j];
    if (!S.uc) return;  // coarsest level of this slice
    if (a.active && !a.active[S.slice]) return;
    const int lt = int(t - a.tile_start[j]);
    const int x = (lt % S.tiles_x) * kBX + threadIdx.x;
    const int y = (lt / S.tiles_x) * kBY + threadIdx.y;
    if (x >= S.nx || y >= S.ny) return;
    S.u[(int64_t)y * S.pitch + x] += prolong_at<T>(S.uc, S.pitchc, x, y, S.ncx, S.ncy, S.n0x, S.n0y, a.k);
}

// ---------------------------------------------------------------- finest-level kernels
// The iterate is kept in correction form f = o + d (d = 0 initially), so the residual
//     r = b - A f = alpha (s - o) - A d
// never subtracts the large L o and L f from each other.  In the adjoint (rhs) mode the
// system is A x = rhs with x = d and o = 0.
struct TopSlice {
    int64_t off;   // element offset of the slice in the packed s / o / d / out buffers
    int nx, ny;
    int tiles_x;   // 64 x 32 tiles of the residual kernel
    int pitch0;    // level-0 row pitch
    void* u0;      // level-0 iterate of the V-cycle (the correction e)
    void* b0;      // level-0 right-hand side (the residual r)
};

// alpha + deg in the iterate type for deg = 0..4 (the diagonal of A), formed once on the host
// (IEEE addition gives the same values there as on the device)
template <class TF>
struct AlphaDeg {
    TF v[5];
    float alpha_f;  // alpha rounded to float once on the host (a conversion per thread would
                    // take the FP64 pipe)
};

// Device-side state of the outer loop of one solve (one per plan).  The loop (residual pass,
// convergence check, V-cycle, residual pass, ...) is decided on the device by k_check after
// every residual pass, so that a solve is one CUDA graph whose loop is a conditional WHILE node
// (without graphs the same kernels are launched by a host loop that reads `cont`).
struct SolveState {
    int it;         // index of the next residual pass (0 = the first residual)
    int vdone;      // V-cycles applied so far to the slices still iterating
    int cont;       // 1 while another V-cycle and residual pass follow
    int nonfinite;  // some slice's residual was not finite
    int timeout;    // a bounded wait of a V-cycle kernel expired
    int pad[3];
};

// The caller's buffers of the current call, which the residual kernels read through this
// struct (written by k_set_call before every solve), so a captured solve graph stays valid
// when they change.
struct CallPtrs {
    const float* s;
    const void* o;
    const float* rhs;
    float* out;
};

constexpr int kTopTX = 64;
constexpr int kTopTY = 32;  // two rows of 4 cells per thread; the one-cell halo of d is 9 % extra

// MODE 0: d = 0, r = alpha (s - o)          (first residual; also accumulates ||b||^2)
// MODE 1: d_new = e                          (first correction)
// MODE 2: d_new = d_old + e                  (later corrections)
// and in MODE 1 and 2: r = b - A d_new, out = o + d_new (the solution for the iterate whose
// residual this pass measures, so the output is always the latest iterate).
// d_old and d_new are different buffers (they alternate between passes): a tile reads d_old
// and e on a one-cell halo while its neighbours write d_new.  Arithmetic on d and r in TF
// (FP64 when mixed); the FP64 work per cell is the 5-point operator on d (and in MODE 2 the
// update d_old + e).  Conversions between TV and TF run on the integer pipe (fpconv.cuh).
template <class TF, class TV, class To, int MODE, bool EXACT>
__global__ void __launch_bounds__(256)
k_top(const TopSlice* __restrict__ top, const int64_t* __restrict__ tile_start, int nslices,
      const int* __restrict__ active, const CallPtrs* __restrict__ call, const SolveState* __restrict__ state,
      TF* __restrict__ dbuf0, TF* __restrict__ dbuf1, double alpha, AlphaDeg<TF> ad,
      double* __restrict__ norms) {
    const int64_t t = blockIdx.x;
    const int j = find_item(tile_start, nslices, t);
    if (active && !active[j]) return;
    // the caller's buffers, and the iterate buffers of this pass: pass `it` writes buffer it & 1
    // and reads the other (they alternate, so that a tile can read d_old on its halo while its
    // neighbours write d_new)
    const float* __restrict__ s = call->s;
    const To* __restrict__ o = static_cast<const To*>(call->o);
    const float* __restrict__ rhs = call->rhs;
    float* __restrict__ out = call->out;
    const int it = state->it;
    const TF* __restrict__ d_old = (it & 1) ? dbuf0 : dbuf1;
    TF* __restrict__ d_new = (it & 1) ? dbuf1 : dbuf0;
    const TopSlice G = top[j];
    const int lt = int(t - tile_start[j]);
    const int tx0 = (lt % G.tiles_x) * kTopTX;
    const int ty0 = (lt / G.tiles_x) * kTopTY;
    const int tid = threadIdx.x;
    const TV* e = static_cast<const TV*>(G.u0);
    TV* r0 = static_cast<TV*>(G.b0);
    __shared__ TF dsm[kTopTY + 2][kTopTX + 2];
    if (MODE >= 1) {
        for (int q = tid; q < (kTopTY + 2) * (kTopTX + 2); q += 256) {
            const int rr = q / (kTopTX + 2), cc = q - rr * (kTopTX + 2);
            const int gx = tx0 - 1 + cc, gy = ty0 - 1 + rr;
            TF v = TF(0);
            if (gx >= 0 && gx < G.nx && gy >= 0 && gy < G.ny) {
                const TF ev = cvt<TF>(e[(int64_t)gy * G.pitch0 + gx]);
                v = MODE == 1 ? ev : d_old[G.off + (int64_t)gy * G.nx + gx] + ev;
            }
            dsm[rr][cc] = v;
        }
        __syncthreads();
    }
    const float af = ad.alpha_f;
    // squared norms: FP32 partial sums over a warp's 256 cells, FP64 from there on (per-block
    // sums, per-slice atomics); this keeps the FP64 pipe for the residual itself
    float rrf = 0.f, bbf = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int ly = tid / 16 + 16 * (i >> 2);  // rows tid / 16 and tid / 16 + 16
        const int y = ty0 + ly;
        const int lx = (tid % 16) + 16 * (i & 3);  // consecutive threads, consecutive cells
        const int x = tx0 + lx;
        if (x >= G.nx || y >= G.ny) continue;
        const int64_t p = G.off + (int64_t)y * G.nx + x;
        const bool hw = x > 0, he = x + 1 < G.nx, hn = y > 0, hs = y + 1 < G.ny;
        float bc, ov = 0.f;
        if (rhs) {
            bc = rhs[p];
            if (MODE == 0) bbf = fmaf(bc, bc, bbf);
        } else {
            const float sv = s[p];
            ov = float(o[p]);
            bc = af * (sv - ov);
            if (MODE == 0) {
                // ||b||^2 with b = alpha s + L o, for the relative-residual denominator
                float lo = 0.f;
                if (hw) lo += ov - float(o[p - 1]);
                if (he) lo += ov - float(o[p + 1]);
                if (hn) lo += ov - float(o[p - G.nx]);
                if (hs) lo += ov - float(o[p + G.nx]);
                const float b = fmaf(af, sv, lo);
                bbf = fmaf(b, b, bbf);
            }
        }
        TV rv;
        if (MODE == 0) {
            rv = cvt<TV>(bc);
        } else {
            const TF c = dsm[ly + 1][lx + 1];
            const TF nsum = (dsm[ly + 1][lx] + dsm[ly + 1][lx + 2]) + (dsm[ly][lx + 1] + dsm[ly + 2][lx + 1]);
            const int deg = int(hw) + int(he) + int(hn) + int(hs);
            const TF adeg = deg == 4 ? ad.v[4] : (deg == 3 ? ad.v[3] : (deg == 2 ? ad.v[2] : (deg == 1 ? ad.v[1] : ad.v[0])));
            // A d in TF (FP64 when mixed): the operator on the high-precision iterate, where
            // the cancellation between alpha d + L d and the right-hand side happens
            const TF Ad = fma_t(adeg, c, -nsum);
            // r = bc - A d.  bc = alpha (s - o) is formed in FP32, so its own rounding (~6e-8
            // |bc|) bounds what FP64 could add here: unless EXACT, A d is rounded to the
            // V-cycle type before the subtraction (same order of error, one FP64 operation per
            // cell less).  That caps the reachable relative residual near 6e-8 ||bc|| / ||b||;
            // tolerances below 1e-7 select EXACT.
            if constexpr (!EXACT && sizeof(TV) < sizeof(TF)) rv = bc - cvt<TV>(Ad);
            else rv = cvt<TV>(cvt<TF>(bc) - Ad);
            d_new[p] = c;
            // output: d alone in the adjoint mode, else o + d (in FP64 when TV is FP64)
            float f;
            if (rhs) f = cvt<float>(c);
            else if constexpr (sizeof(TV) == 8) f = cvt<float>(cvt<double>(ov) + c);
            else f = ov + cvt<float>(c);
            out[p] = f;
        }
        r0[(int64_t)y * G.pitch0 + x] = rv;
        const float rf = cvt<float>(rv);
        rrf = fmaf(rf, rf, rrf);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        rrf += __shfl_xor_sync(0xffffffffu, rrf, m);
        if (MODE == 0) bbf += __shfl_xor_sync(0xffffffffu, bbf, m);
    }
    // the 8 warp partials: converted on the integer pipe and added in FP64 by a shuffle tree in
    // the first warp (lanes l and l + 8, l + 16, l + 24 hold the same partial), 3 FP64 adds per
    // norm: on this part one warp-wide FP64 instruction holds the pipe for 16 cycles, so a serial
    // per-block loop would cost a sizeable share of the whole pass
    __shared__ float red[2][8];
    if ((tid & 31) == 0) { red[0][tid >> 5] = rrf; red[1][tid >> 5] = bbf; }
    __syncthreads();
    if (tid < 32) {
        const int l = tid & 7;
        double r2 = cvt<double>(red[0][l]);
        double b2 = MODE == 0 ? cvt<double>(red[1][l]) : 0.0;
#pragma unroll
        for (int m = 4; m > 0; m >>= 1) {
            r2 += __shfl_xor_sync(0xffffffffu, r2, m);
            if (MODE == 0) b2 += __shfl_xor_sync(0xffffffffu, b2, m);
        }
        if (tid == 0) {
            atomicAdd(&norms[2 * j], r2);
            if (MODE == 0) atomicAdd(&norms[2 * j + 1], b2);
        }
    }
}

// Independent check of the reported residual (opts.verify_residual): ||b - A f||^2 and ||b||^2
// per slice for the final iterate f = o + d, with every operation in FP64 (hardware
// conversions), b = alpha s + L o formed directly (not the correction form of k_top) and the
// squares summed in FP64 (per-block shuffle tree, one FP64 atomic per block and slice).
// last_pass[j] is the residual pass that last wrote slice j's iterate (0: never iterated, d = 0).
// Neighbours are read from global memory (a one-off pass).
template <class TF, class To>
__global__ void __launch_bounds__(256)
k_verify(const TopSlice* __restrict__ top, const int64_t* __restrict__ tile_start, int nslices,
         const int* __restrict__ last_pass, const float* __restrict__ s, const To* __restrict__ o,
         const float* __restrict__ rhs, const TF* __restrict__ d0, const TF* __restrict__ d1, double alpha,
         double* __restrict__ sums) {
    const int64_t t = blockIdx.x;
    const int j = find_item(tile_start, nslices, t);
    const TopSlice G = top[j];
    const int lt = int(t - tile_start[j]);
    const int tx0 = (lt % G.tiles_x) * kTopTX;
    const int ty0 = (lt / G.tiles_x) * kTopTY;
    const int tid = threadIdx.x;
    // the iterate of slice j: written by its last residual pass p (buffer p & 1), none if p = 0
    const int lp = last_pass[j];
    const TF* d = lp == 0 ? nullptr : ((lp & 1) ? d1 : d0);
    auto fval = [&](int64_t q) -> double {  // f = o + d (rhs mode: f = d)
        const double dv = d ? (double)d[q] : 0.0;
        return rhs ? dv : (double)o[q] + dv;
    };
    double rr = 0.0, bb = 0.0;
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const int y = ty0 + tid / 16 + 16 * (i >> 2);
        const int x = tx0 + (tid % 16) + 16 * (i & 3);
        if (x >= G.nx || y >= G.ny) continue;
        const int64_t p = G.off + (int64_t)y * G.nx + x;
        const bool hw = x > 0, he = x + 1 < G.nx, hn = y > 0, hs = y + 1 < G.ny;
        double b, Lf = 0.0;
        const double fc = fval(p);
        if (hw) Lf += fc - fval(p - 1);
        if (he) Lf += fc - fval(p + 1);
        if (hn) Lf += fc - fval(p - G.nx);
        if (hs) Lf += fc - fval(p + G.nx);
        if (rhs) {
            b = (double)rhs[p];
        } else {
            const double oc = (double)o[p];
            double Lo = 0.0;
            if (hw) Lo += oc - (double)o[p - 1];
            if (he) Lo += oc - (double)o[p + 1];
            if (hn) Lo += oc - (double)o[p - G.nx];
            if (hs) Lo += oc - (double)o[p + G.nx];
            b = alpha * (double)s[p] + Lo;
        }
        const double r = b - (alpha * fc + Lf);
        rr += r * r;
        bb += b * b;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, m);
        bb += __shfl_xor_sync(0xffffffffu, bb, m);
    }
    __shared__ double red[2][8];
    if ((tid & 31) == 0) { red[0][tid >> 5] = rr; red[1][tid >> 5] = bb; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < 8; ++w) { a += red[0][w]; c += red[1][w]; }
        atomicAdd(&sums[2 * j], a);
        atomicAdd(&sums[2 * j + 1], c);
    }
}

// ---------------------------------------------------------------- device-side outer loop
__global__ void k_set_call(CallPtrs* __restrict__ dst, CallPtrs v) { *dst = v; }

// Start of a solve: every slice active, no V-cycle yet, norms and wavefront work counters zero.
__global__ void k_init(SolveState* __restrict__ st, int n, int* __restrict__ done, int* __restrict__ active,
                       int* __restrict__ vcycles, int* __restrict__ last_pass, double* __restrict__ norms,
                       unsigned int* __restrict__ work) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        done[j] = 0;
        active[j] = 1;
        vcycles[j] = 0;
        last_pass[j] = 0;
        norms[2 * j] = 0.0;
        norms[2 * j + 1] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->it = 0;
        st->vdone = 0;
        st->cont = 0;
        st->nonfinite = 0;
        st->timeout = 0;
        work[0] = 0u;
        work[1] = 0u;
    }
}

// Convergence check after residual pass st->it, one CTA: per slice, ||r|| / ||b|| from the
// squared norms the pass accumulated (||b|| from pass 0); a slice at or below tol (or with a
// non-finite residual) is done and leaves the active set.  Another V-cycle follows (cont) while
// some slice is left, fewer than maxit V-cycles were applied and no bounded wait expired; it is
// then counted (nv V-cycles) for the slices left.  The norms are cleared for the next pass.
// With use_handle, the decision is also the condition of the solve graph's WHILE node: it is
// set on every call, and cont is 0 once maxit V-cycles are done, so the loop ends.
__global__ void __launch_bounds__(256)
k_check(SolveState* __restrict__ st, int n, double* __restrict__ norms, double* __restrict__ bnorm,
        double* __restrict__ rel, int* __restrict__ done, int* __restrict__ active, int* __restrict__ vcycles,
        int* __restrict__ last_pass, double tol, int maxit, int nv, const int* __restrict__ err, int use_handle,
        cudaGraphConditionalHandle h) {
    __shared__ int s_left, s_nonfinite;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_left = 0;
        s_nonfinite = 0;
    }
    __syncthreads();
    const int it = st->it;
    int left = 0, nonfinite = 0;
    for (int j = tid; j < n; j += blockDim.x) {
        if (done[j]) continue;
        last_pass[j] = it;
        if (it == 0) bnorm[j] = sqrt(norms[2 * j + 1]);
        const double rn = sqrt(norms[2 * j]);
        const double b = bnorm[j];
        const double r = b > 0.0 ? rn / b : rn;
        rel[j] = r;
        if (r <= tol || !isfinite(r)) {
            done[j] = 1;
            active[j] = 0;
            nonfinite += !isfinite(r);
        } else {
            ++left;
        }
    }
    if (left) atomicAdd(&s_left, left);
    if (nonfinite) atomicAdd(&s_nonfinite, nonfinite);
    __syncthreads();
    const int timeout = *err != 0;
    const int cont = (s_left > 0 && st->vdone < maxit && !timeout && it <= maxit + 1) ? 1 : 0;
    __syncthreads();  // every thread has read st before thread 0 updates it
    for (int j = tid; j < n; j += blockDim.x) {
        norms[2 * j] = 0.0;
        norms[2 * j + 1] = 0.0;
        if (cont && !done[j]) vcycles[j] += nv;
    }
    if (tid == 0) {
        st->it = it + 1;
        if (cont) st->vdone += nv;
        st->cont = cont;
        if (s_nonfinite) st->nonfinite = 1;
        if (timeout) st->timeout = 1;
        if (use_handle) cudaGraphSetConditional(h, cont ? 1u : 0u);
    }
}

// out = o (or 0 in the adjoint mode) on the slices that were never iterated (they met the
// tolerance at the initial iterate f = o): kFinishBlocks CTAs per slice, which return at once
// for the slices that were iterated.
constexpr int kFinishBlocks = 8;
template <class To>
__global__ void __launch_bounds__(256)
k_finish(const TopSlice* __restrict__ top, const int* __restrict__ vcycles, const CallPtrs* __restrict__ call) {
    const int j = blockIdx.x / kFinishBlocks;
    if (vcycles[j] != 0) return;
    const TopSlice G = top[j];
    const To* o = static_cast<const To*>(call->o);
    const bool zero = call->rhs != nullptr;
    const int64_t cells = (int64_t)G.nx * G.ny;
    for (int64_t q = (int64_t)(blockIdx.x % kFinishBlocks) * blockDim.x + threadIdx.x; q < cells;
         q += (int64_t)kFinishBlocks * blockDim.x)
        call->out[G.off + q] = zero ? 0.f : float(o[G.off + q]);
}

// Per-slice results of a solve in the layout of emfuse_slice_stats (vsums: the squared norms of
// the verification pass, or null).
__global__ void k_stats(int n, const int* __restrict__ vcycles, const double* __restrict__ rel,
                        const double* __restrict__ bnorm, const double* __restrict__ vsums, double tol,
                        emfuse_slice_stats* __restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        emfuse_slice_stats r;
        r.vcycles = vcycles[j];
        r.rel_residual = rel[j];
        r.b_norm = bnorm[j];
        r.converged = rel[j] <= tol ? 1 : 0;
        if (vsums) {
            const double rn = sqrt(vsums[2 * j]), bn = sqrt(vsums[2 * j + 1]);
            r.rel_residual_check = bn > 0.0 ? rn / bn : rn;
        } else {
            r.rel_residual_check = -1.0;
        }
        out[j] = r;
    }
}

// A workspace larger than the device's whole memory can never be allocated: such a request
// fails here with EMFUSE_ENOMEM, before any allocation and before any kernel reads the caller's
// buffers.  (Smaller requests that exceed the free memory fail in the allocator, also ENOMEM.)
inline int check_device_capacity(double bytes, const char* what) {
    size_t free_b = 0, total_b = 0;
    EMF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (bytes > (double)total_b) {
        set_error(std::string(what) + ": the solver workspace needs " + std::to_string(bytes / 1e9) +
                  " GB, more than the device's " + std::to_string((double)total_b / 1e9) + " GB");
        return EMFUSE_ENOMEM;
    }
    return EMFUSE_OK;
}

inline unsigned grid_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)kNumSMs * 16));
}

// ---------------------------------------------------------------- host-side plan
template <class T>
struct LevelPlan {
    std::vector<LSlice<T>> sl;          // every slice that has this level
    std::vector<int64_t> tile_start;    // reference-kernel tiles, prefix sums (nsl + 1)
    std::vector<LSlice<T>> wsl;         // slices that run the wavefront kernels here
    std::vector<int64_t> item_start;    // wavefront work items, prefix sums
    LSlice<T>* d_sl = nullptr;
    int64_t* d_ts = nullptr;
    LSlice<T>* d_wsl = nullptr;
    int64_t* d_is = nullptr;
    std::vector<CUtensorMap> maps;      // per wavefront slice: u, b, coarse output iterate
    CUtensorMap* d_maps = nullptr;
    int k = 0;
    int ch = 64;                        // wavefront rows per work item
    double cells = 0;                   // cells of this level summed over its slices
    double wcells = 0;                  // ... over the wavefront slices
    int64_t ntiles() const { return tile_start.empty() ? 0 : tile_start.back(); }
    int64_t nitems() const { return item_start.empty() ? 0 : item_start.back(); }
};

inline int num_levels(int64_t nx, int64_t ny) {
    int K = 0;
    while (level_size((int)nx, K) > 1 || level_size((int)ny, K) > 1) ++K;
    return K + 1;
}

// Small descriptor uploads: packs host vectors into one device blob.
struct Blob {
    std::vector<char> host;
    template <class V>
    size_t add(const std::vector<V>& v) {
        const size_t pos = host.size();
        host.resize(pos + round_up(std::max<size_t>(1, v.size() * sizeof(V)), 256));
        if (!v.empty()) std::memcpy(host.data() + pos, v.data(), v.size() * sizeof(V));
        return pos;
    }
};

template <class TF, class TV>
struct Solver {
    const SolveRequest* rq = nullptr;  // the call being served
    cudaStream_t st;
    std::vector<LevelPlan<TV>> levels;
    DeviceBuffer ws_levels, ws_desc, ws_f, ws_norms, ws_active, ws_loop;
    std::vector<int> nlev, kc;
    int Kmax = 0, Kw = 0;       // levels, and levels with wavefront work
    TF* dbuf[2] = {nullptr, nullptr};  // FP64 iterates d, alternating between passes
    double* d_norms = nullptr;
    int* d_active = nullptr;
    int* d_err = nullptr;            // this plan's error word (bounded waits of its V-cycle kernels)
    unsigned int* d_work = nullptr;  // wavefront work counters (reset by each launch's last warp)
    TopSlice* d_top = nullptr;
    int64_t* d_top_ts = nullptr;
    int64_t top_tiles = 0;
    double top_cells = 0;
    TailArgs<TV> tail{};
    double tail_cells = 0;
    bool fused = true;

    // device-side outer loop (ws_loop): state, the caller's buffers, per-slice arrays, results
    SolveState* d_state = nullptr;
    CallPtrs* d_call = nullptr;
    int *d_done = nullptr, *d_vcyc = nullptr, *d_lastp = nullptr;
    double *d_bnorm = nullptr, *d_rel = nullptr, *d_vsums = nullptr;
    emfuse_slice_stats* d_stats = nullptr;
    // page-locked host copies of the results (read after a synchronisation, or by the stream
    // callback of an asynchronous solve)
    emfuse_slice_stats* h_stats = nullptr;
    SolveState* h_state = nullptr;
    cudaEvent_t async_done = nullptr;  // recorded after the last asynchronous solve's callback

    // The whole solve as one CUDA graph with a WHILE node (see solve_graph), captured on private
    // streams and replayed on the caller's; rebuilt when one of the values it bakes in changes.
    cudaGraphExec_t sexec = nullptr;
    std::vector<double> skey;
    int64_t s_pro_nodes = 0, s_body_nodes = 0;  // kernel nodes outside / inside the loop
    int s_pro_passes = 0;                       // residual passes outside the loop
    cudaStream_t cap_st = nullptr, cap_body = nullptr;

    explicit Solver(cudaStream_t s) : st(s) {}
    ~Solver() {
        if (async_done) {  // the stream callback of an asynchronous solve reads h_stats / h_state
            cudaEventSynchronize(async_done);
            cudaEventDestroy(async_done);
        }
        drop_graphs();
        if (cap_st) cudaStreamDestroy(cap_st);
        if (cap_body) cudaStreamDestroy(cap_body);
        free_host();
    }
    void drop_graphs() {
        if (sexec) cudaGraphExecDestroy(sexec);
        sexec = nullptr;
        skey.clear();
    }
    void free_host() {
        if (h_stats) cudaFreeHost(h_stats);
        if (h_state) cudaFreeHost(h_state);
        h_stats = nullptr;
        h_state = nullptr;
    }

    // What the plan depends on: the slice geometry and the schedule options.
    std::vector<int64_t> sig;
    bool built = false;
    static std::vector<int64_t> signature(const SolveRequest& r) {
        std::vector<int64_t> v = {r.nslices, r.opts.fused, r.opts.nu_pre, r.opts.nu_post, r.opts.tile_rows};
        for (int64_t j = 0; j < r.nslices; ++j) {
            v.push_back(r.nx[j]);
            v.push_back(r.ny[j]);
            v.push_back(r.offsets[j]);
        }
        return v;
    }

    // The wavefront kernels' strips overlap by kWaveHalo = 8 cells, and every half-sweep carries
    // the wrong values at a strip's outer edge one cell further in: the UP leg (S = 2 nu
    // half-sweeps) needs S <= 8, the DOWN leg, whose residual reaches one cell further, S + 1 <= 8.
    static bool wave_ok_pre(int nu) { return nu >= 1 && 2 * nu + 1 <= kWaveHalo; }
    static bool wave_ok_post(int nu) { return nu >= 1 && 2 * nu <= kWaveHalo; }

    // Drops the plan but keeps the two large buffers (pyramids, FP64 iterates): their layout
    // is recomputed by build() and they are only reallocated when a batch needs more.
    void reset() {
        drop_graphs();
        levels.clear();
        ws_desc.release();
        ws_norms.release();
        ws_active.release();
        ws_loop.release();
        if (async_done) cudaEventSynchronize(async_done);
        free_host();
        nlev.clear();
        kc.clear();
        Kmax = Kw = 0;
        top_tiles = 0;
        top_cells = tail_cells = 0;
        tail = TailArgs<TV>{};
        built = false;
    }

    int build() {
        std::vector<int64_t> want = signature(*rq);
        if (built && want == sig) {
            tail.alpha = TV(rq->alpha);  // the only planned value that depends on alpha
            return EMFUSE_OK;
        }
        reset();
        sig = std::move(want);
        const int64_t n = rq->nslices;
        fused = rq->opts.fused != 0 && wave_ok_pre(rq->opts.nu_pre) && wave_ok_post(rq->opts.nu_post);
        nlev.resize(n);
        kc.resize(n);
        for (int64_t j = 0; j < n; ++j) {
            nlev[j] = num_levels(rq->nx[j], rq->ny[j]);
            Kmax = std::max(Kmax, nlev[j]);
            int k = 0;  // first level small enough for the coarse tail
            while (std::max(level_size((int)rq->nx[j], k), level_size((int)rq->ny[j], k)) > kTailMax) ++k;
            kc[j] = fused ? k : nlev[j];
            Kw = std::max(Kw, kc[j]);
        }
        // levels run by the wavefront kernels (the others by the coarse tail / reference)
        auto wave = [&](int64_t j, int k) { return fused && k < kc[j]; };
        // level arrays: u and b of every slice and level, rows padded to 128 bytes
        const int64_t align = 128 / (int64_t)sizeof(TV);
        std::vector<std::vector<int64_t>> off(n);
        int64_t total = 0;
        for (int64_t j = 0; j < n; ++j) {
            off[j].resize(nlev[j]);
            for (int k = 0; k < nlev[j]; ++k) {
                const int64_t lx = level_size((int)rq->nx[j], k), ly = level_size((int)rq->ny[j], k);
                off[j][k] = total;
                // u, b, and on wavefront levels the output iterate uo
                total += (wave(j, k) ? 3 : 2) * round_up(lx, align) * ly;
            }
        }
        {
            double fine = 0.0;  // the two FP64 iterates of run(): 2 x the finest levels
            for (int64_t j = 0; j < n; ++j) fine += (double)rq->nx[j] * (double)rq->ny[j];
            EMF_TRY(check_device_capacity((double)total * sizeof(TV) + 2.0 * fine * sizeof(TF), "solve"));
        }
        if (ws_levels.bytes() < (size_t)total * sizeof(TV))
            EMF_TRY(ws_levels.alloc_persistent((size_t)total * sizeof(TV)));
        TV* base = ws_levels.as<TV>();
        auto make = [&](int64_t j, int k) {
            LSlice<TV> S{};
            const int n0x = (int)rq->nx[j], n0y = (int)rq->ny[j];
            S.nx = level_size(n0x, k);
            S.ny = level_size(n0y, k);
            S.pitch = (int)round_up(S.nx, align);
            S.u = base + off[j][k];
            S.b = S.u + (int64_t)S.pitch * S.ny;
            S.uo = wave(j, k) ? S.b + (int64_t)S.pitch * S.ny : S.u;
            if (k + 1 < nlev[j]) {
                S.ncx = level_size(n0x, k + 1);
                S.ncy = level_size(n0y, k + 1);
                S.pitchc = (int)round_up(S.ncx, align);
                S.uc = base + off[j][k + 1];
                S.bc = S.uc + (int64_t)S.pitchc * S.ncy;
                S.uco = wave(j, k + 1) ? S.bc + (int64_t)S.pitchc * S.ncy : S.uc;
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
            S.fstrips = (int)ceil_div(S.nx, kWaveIW);
            return S;
        };
        levels.resize(Kmax);
        std::vector<LSlice<TV>> table;
        std::vector<int> level_off(n);
        for (int64_t j = 0; j < n; ++j) {
            level_off[j] = (int)table.size();
            for (int k = 0; k < nlev[j]; ++k) table.push_back(make(j, k));
        }
        for (int k = 0; k < Kmax; ++k) {
            LevelPlan<TV>& L = levels[k];
            L.k = k;
            L.tile_start.push_back(0);
            L.item_start.push_back(0);
            int64_t want = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (nlev[j] <= k) continue;
                const LSlice<TV> S = make(j, k);
                L.sl.push_back(S);
                L.tile_start.push_back(L.tile_start.back() + (int64_t)S.tiles_x * ceil_div(S.ny, kBY));
                L.cells += (double)S.nx * S.ny;
                if (wave(j, k)) {
                    L.wsl.push_back(S);
                    L.wcells += (double)S.nx * S.ny;
                    want += (int64_t)S.fstrips * S.ny;
                }
            }
            // rows per work item: tall chunks amortise the halo rows (about 2 nu + 3 pairs per
            // chunk) and the per-item set-up; 256 rows only where every resident warp still gets
            // several items (the last ones would otherwise leave SMs idle), shorter ones while the
            // level would leave SMs idle (down to 8 rows on small levels, where a march's latency,
            // not its work, is the cost)
            const int64_t resident = (int64_t)kNumSMs * 16;  // resident wavefront warps, about
            L.ch = want / 256 >= 4 * resident ? 256 : 128;
            while (L.ch > 8 && want / L.ch < resident) L.ch /= 2;  // about one item per resident warp
            if (k == 0 && rq->opts.tile_rows > 0) L.ch = rq->opts.tile_rows;
            for (const auto& S : L.wsl) {
                L.item_start.push_back(L.item_start.back() + (int64_t)S.fstrips * ceil_div(S.ny, L.ch));
                // TMA maps: row pairs of u, b and uo (one 128 x 2 box per strip step) and the
                // three coarse rows around a fine row pair for the prolongation
                CUtensorMap mu, mb, mc;
                EMF_TRY(encode_tensor_map_2d(&mu, S.u, sizeof(TV), S.nx, S.ny, S.pitch, kWaveWidth, 2));
                EMF_TRY(encode_tensor_map_2d(&mb, S.b, sizeof(TV), S.nx, S.ny, S.pitch, kWaveWidth, 2));
                if (S.uco)
                    EMF_TRY(encode_tensor_map_2d(&mc, S.uco, sizeof(TV), S.ncx, S.ncy, S.pitchc, kWaveCoarseW, 3));
                else
                    mc = mu;
                CUtensorMap mo;
                EMF_TRY(encode_tensor_map_2d(&mo, S.uo, sizeof(TV), S.nx, S.ny, S.pitch, kWaveWidth, 2));
                L.maps.push_back(mu);
                L.maps.push_back(mb);
                L.maps.push_back(mc);
                L.maps.push_back(mo);
            }
        }
        // finest-level (residual kernel) tiling
        std::vector<TopSlice> top(n);
        std::vector<int64_t> top_ts(n + 1, 0);
        for (int64_t j = 0; j < n; ++j) {
            const LSlice<TV> S0 = table[level_off[j]];
            top[j] = TopSlice{rq->offsets[j], (int)rq->nx[j], (int)rq->ny[j],
                              (int)ceil_div(rq->nx[j], kTopTX), S0.pitch, S0.uo, S0.b};
            top_ts[j + 1] = top_ts[j] + (int64_t)top[j].tiles_x * ceil_div(rq->ny[j], kTopTY);
            top_cells += (double)rq->nx[j] * rq->ny[j];
        }
        top_tiles = top_ts[n];
        std::vector<int> vkc(kc), vnlev(nlev);
        for (int64_t j = 0; j < n; ++j)
            for (int k = kc[j]; k < nlev[j]; ++k) {
                const auto& S = table[level_off[j] + k];
                tail_cells += (double)S.nx * S.ny;
            }
        Blob blob;
        std::vector<size_t> pos_sl(Kmax), pos_ts(Kmax), pos_wsl(Kmax), pos_is(Kmax), pos_maps(Kmax);
        for (int k = 0; k < Kmax; ++k) {
            pos_maps[k] = blob.add(levels[k].maps);
            pos_sl[k] = blob.add(levels[k].sl);
            pos_ts[k] = blob.add(levels[k].tile_start);
            pos_wsl[k] = blob.add(levels[k].wsl);
            pos_is[k] = blob.add(levels[k].item_start);
        }
        const size_t pos_top = blob.add(top), pos_top_ts = blob.add(top_ts);
        const size_t pos_table = blob.add(table), pos_loff = blob.add(level_off);
        const size_t pos_nlev = blob.add(vnlev), pos_kc = blob.add(vkc);
        EMF_TRY(ws_desc.alloc_persistent(blob.host.size()));
        char* dbase = ws_desc.as<char>();
        EMF_CUDA(cudaMemcpyAsync(dbase, blob.host.data(), blob.host.size(), cudaMemcpyHostToDevice, st));
        for (int k = 0; k < Kmax; ++k) {
            levels[k].d_sl = reinterpret_cast<LSlice<TV>*>(dbase + pos_sl[k]);
            levels[k].d_ts = reinterpret_cast<int64_t*>(dbase + pos_ts[k]);
            levels[k].d_wsl = reinterpret_cast<LSlice<TV>*>(dbase + pos_wsl[k]);
            levels[k].d_is = reinterpret_cast<int64_t*>(dbase + pos_is[k]);
            levels[k].d_maps = reinterpret_cast<CUtensorMap*>(dbase + pos_maps[k]);
        }
        d_top = reinterpret_cast<TopSlice*>(dbase + pos_top);
        d_top_ts = reinterpret_cast<int64_t*>(dbase + pos_top_ts);
        EMF_TRY(ws_norms.alloc_persistent(2 * n * sizeof(double)));
        d_norms = ws_norms.as<double>();
        // active flags of the slices, then the two work counters of the wavefront kernels
        EMF_TRY(ws_active.alloc_persistent((n + 2) * sizeof(int)));
        d_active = ws_active.as<int>();
        d_work = reinterpret_cast<unsigned int*>(d_active + n);
        EMF_CUDA(cudaMemsetAsync(d_work, 0, 2 * sizeof(unsigned int), st));
        {
            // loop state, call buffers and this plan's error word, then the per-slice arrays
            const size_t head = 256, ints = round_up(n * sizeof(int), 256), dbls = round_up(n * sizeof(double), 256);
            const size_t stats = round_up(n * sizeof(emfuse_slice_stats), 256);
            EMF_TRY(ws_loop.alloc_persistent(head + 3 * ints + 4 * dbls + stats));
            char* q = ws_loop.as<char>();
            d_state = reinterpret_cast<SolveState*>(q);
            d_call = reinterpret_cast<CallPtrs*>(q + 64);
            d_err = reinterpret_cast<int*>(q + 128);
            q += head;
            d_done = reinterpret_cast<int*>(q); q += ints;
            d_vcyc = reinterpret_cast<int*>(q); q += ints;
            d_lastp = reinterpret_cast<int*>(q); q += ints;
            d_bnorm = reinterpret_cast<double*>(q); q += dbls;
            d_rel = reinterpret_cast<double*>(q); q += dbls;
            d_vsums = reinterpret_cast<double*>(q); q += 2 * dbls;
            d_stats = reinterpret_cast<emfuse_slice_stats*>(q);
            EMF_CUDA(cudaMemsetAsync(ws_loop.as<char>(), 0, head, st));
            EMF_CUDA(cudaMallocHost(&h_stats, std::max<size_t>(1, n) * sizeof(emfuse_slice_stats)));
            EMF_CUDA(cudaMallocHost(&h_state, sizeof(SolveState)));
        }
        tail.table = reinterpret_cast<const LSlice<TV>*>(dbase + pos_table);
        tail.level_off = reinterpret_cast<const int*>(dbase + pos_loff);
        tail.nlev = reinterpret_cast<const int*>(dbase + pos_nlev);
        tail.kc = reinterpret_cast<const int*>(dbase + pos_kc);
        tail.nslices = (int)n;
        tail.alpha = TV(rq->alpha);
        tail.nu_pre = rq->opts.nu_pre;
        tail.nu_post = rq->opts.nu_post;
        tail.active = d_active;
        tail.cont = 0;
        tail.smem_bytes = 0;
        for (int64_t j = 0; j < n; ++j)
            if (kc[j] < nlev[j])
                tail.smem_bytes = std::max<int>(tail.smem_bytes, (int)tail_smem_bytes<TV>(
                    level_size((int)rq->nx[j], kc[j]), level_size((int)rq->ny[j], kc[j])));
        EMF_CUDA(cudaStreamSynchronize(st));  // the host staging blob goes out of scope
        built = true;
        return EMFUSE_OK;
    }

    LevelArgs<TV> args(int k) const {
        LevelArgs<TV> a;
        a.sl = levels[k].d_sl;
        a.tile_start = levels[k].d_ts;
        a.nsl = (int)levels[k].sl.size();
        a.k = k;
        a.alpha = TV(rq->alpha);
        a.sk = TV(std::ldexp(1.0, -2 * k));
        a.active = d_active;
        return a;
    }

    WaveArgs<TV> wargs(int k) const {
        WaveArgs<TV> a;
        a.sl = levels[k].d_wsl;
        a.item_start = levels[k].d_is;
        a.nsl = (int)levels[k].wsl.size();
        a.nitems = levels[k].nitems();
        a.k = k;
        a.ch = levels[k].ch;
        a.alpha = TV(rq->alpha);
        a.sk = TV(std::ldexp(1.0, -2 * k));
        a.active = d_active;
        a.maps = levels[k].d_maps;
        a.u_map = 0;
        a.err = d_err;
        a.work = d_work;
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

    // Reference schedule: one kernel per half-sweep, restriction and prolongation.
    // cont = continue from the level-0 iterate of the previous V-cycle instead of zero.
    int vcycle_reference(bool cont) {
        const int nu1 = rq->opts.nu_pre, nu2 = rq->opts.nu_post;
        if (!cont)
            for (const auto& S : levels[0].sl)
                EMF_CUDA(cudaMemsetAsync(S.u, 0, (size_t)S.pitch * S.ny * sizeof(TV), st));
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

    // Fused schedule: wavefront DOWN on large levels, one coarse-tail kernel, wavefront UP.
    // cont = continue from the previous V-cycle's level-0 result (read from uo).
    int vcycle_fused(bool cont) {
        const int S1 = 2 * rq->opts.nu_pre, S2 = 2 * rq->opts.nu_post;
        for (int k = 0; k < Kw; ++k) {
            const auto& L = levels[k];
            const bool from_prev = cont && k == 0;
            // reads b (and u when continuing), writes u and the coarse rhs
            const double bytes = sizeof(TV) * ((from_prev ? 3.0 : 2.0) * L.wcells + 0.25 * L.wcells);
            WaveArgs<TV> a = wargs(k);
            a.u_map = from_prev ? 3 : 0;
            EMF_TRY(launch_wave<TV>(a, S1, !from_prev, false, st, bytes));
        }
        TailArgs<TV> ta = tail;
        ta.cont = cont ? 1 : 0;  // slices that start in the tail continue from their level-0 u
        EMF_TRY(launch_tail<TV>(ta, st, sizeof(TV) * 2.0 * tail_cells));
        for (int k = Kw - 1; k >= 0; --k) {
            const auto& L = levels[k];
            // reads u, b and the coarse iterate, writes u
            const double bytes = sizeof(TV) * (3.0 * L.wcells + 0.25 * L.wcells);
            EMF_TRY(launch_wave<TV>(wargs(k), S2, false, true, st, bytes));
        }
        return EMFUSE_OK;
    }

    // One V-cycle (launched directly, or recorded while a solve graph is captured).
    int vcycle(bool cont) { return fused ? vcycle_fused(cont) : vcycle_reference(cont); }

    // Residual pass MODE (0: first residual, 1: first correction, 2: later corrections) on the
    // iterate buffers the device-side pass index selects.
    template <class To, int MODE>
    int top_pass() {
        // algorithmic bytes: s and o (or rhs) read, r written; MODE >= 1 also reads e (and
        // d_old in MODE 2) and writes d_new and the output
        const double in_b = rq->rhs ? 4.0 : 4.0 + sizeof(To);
        const double it_b = MODE == 0 ? 0.0 : sizeof(TV) + sizeof(TF) + 4.0 + (MODE == 2 ? sizeof(TF) : 0.0);
        const double bytes = top_cells * (in_b + it_b + sizeof(TV));
        // FP64 work of the pass (when the iterate is FP64): the 5-point operator on d, three
        // adds and one fma per cell, plus the update d_old + e in MODE 2
        const double flops = sizeof(TF) == 8 && MODE > 0 ? top_cells * (MODE == 2 ? 6.0 : 5.0) : 0.0;
        KernelScope ks(MODE == 0 ? "residual_first" : "residual_update", st, bytes, flops);
        AlphaDeg<TF> ad;
        for (int q = 0; q < 5; ++q) ad.v[q] = TF(rq->alpha) + TF(q);
        ad.alpha_f = float(rq->alpha);
        if (rq->opts.tol < 1e-7)
            k_top<TF, TV, To, MODE, true><<<(unsigned)top_tiles, 256, 0, st>>>(
                d_top, d_top_ts, (int)rq->nslices, d_active, d_call, d_state, dbuf[0], dbuf[1], rq->alpha, ad,
                d_norms);
        else
            k_top<TF, TV, To, MODE, false><<<(unsigned)top_tiles, 256, 0, st>>>(
                d_top, d_top_ts, (int)rq->nslices, d_active, d_call, d_state, dbuf[0], dbuf[1], rq->alpha, ad,
                d_norms);
        EMF_CHECK_LAUNCH();
        return EMFUSE_OK;
    }

    int launch_init() {
        const int n = (int)rq->nslices;
        KernelScope ks("solve_control", st, 0.0);
        k_init<<<(unsigned)std::max<int64_t>(1, ceil_div(n, 256)), 256, 0, st>>>(d_state, n, d_done, d_active, d_vcyc,
                                                                                 d_lastp, d_norms, d_work);
        EMF_CHECK_LAUNCH();
        return EMFUSE_OK;
    }

    int launch_check(int nv, bool handle, cudaGraphConditionalHandle h) {
        KernelScope ks("solve_control", st, 0.0);
        k_check<<<1, 256, 0, st>>>(d_state, (int)rq->nslices, d_norms, d_bnorm, d_rel, d_done, d_active, d_vcyc,
                                   d_lastp, rq->opts.tol, std::max(0, rq->opts.max_vcycles), nv, d_err,
                                   handle ? 1 : 0, h);
        EMF_CHECK_LAUNCH();
        return EMFUSE_OK;
    }

    template <class To>
    int launch_finish() {
        KernelScope ks("store_initial", st, 0.0);
        k_finish<To><<<(unsigned)(rq->nslices * kFinishBlocks), 256, 0, st>>>(d_top, d_vcyc, d_call);
        EMF_CHECK_LAUNCH();
        return EMFUSE_OK;
    }

    // V-cycles of the first outer iteration (the second continues from the first's correction)
    int first_vcycles() const { return std::min(rq->opts.first_vcycles, std::max(0, rq->opts.max_vcycles)); }

    // The outer loop, recorded on `st`:  first residual, check; then (when the first iteration
    // has V-cycles) those V-cycles, the first correction pass and a check that sets the loop
    // condition; the loop body is one V-cycle, a correction pass and a check.  Slices that are
    // done are inactive, so the first iteration's kernels do nothing for them even when the
    // first check finds every slice done.
    template <class To>
    int record_prologue(cudaGraphConditionalHandle h, bool handle) {
        EMF_TRY(launch_init());
        EMF_TRY((top_pass<To, 0>()));
        const int nv = first_vcycles();
        EMF_TRY(launch_check(nv, false, h));
        if (nv == 0) return EMFUSE_OK;
        for (int v = 0; v < nv; ++v) EMF_TRY(vcycle(v > 0));
        EMF_TRY((top_pass<To, 1>()));
        return launch_check(1, handle, h);
    }
    template <class To>
    int record_body(cudaGraphConditionalHandle h, bool handle) {
        EMF_TRY(vcycle(false));
        EMF_TRY((top_pass<To, 2>()));
        return launch_check(1, handle, h);
    }

    // The solve as one graph: the prologue, a conditional WHILE node whose condition k_check
    // sets after every residual pass (the body captured into the node's child graph on a second
    // private stream), and the store of the never-iterated slices.  Captured once per plan and
    // per value baked into its kernels (alpha, tol, max_vcycles, first V-cycles, iterate and
    // constraint types); the caller's buffers go through d_call.
    template <class To>
    int solve_graph() {
        const std::vector<double> key = {rq->alpha, rq->opts.tol, (double)rq->opts.max_vcycles,
                                         (double)first_vcycles(), rq->rhs ? 1.0 : 0.0, (double)sizeof(To)};
        if (sexec && key == skey) return EMFUSE_OK;
        drop_graphs();
        if (!cap_st) EMF_CUDA(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
        if (!cap_body) EMF_CUDA(cudaStreamCreateWithFlags(&cap_body, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        EMF_CUDA(cudaGraphCreate(&g, 0));
        // the loop's condition handle (a graph without the loop node may hold no handle)
        cudaGraphConditionalHandle h{};
        cudaError_t e = first_vcycles() > 0 ? cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)
                                            : cudaSuccess;
        int rc = EMFUSE_OK;
        int64_t n_pro = 0, n_body = 0;
        const cudaStream_t user = st;
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap_st, g, nullptr, nullptr, 0,
                                                                cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const uint64_t c0 = launch_count();
            st = cap_st;
            rc = record_prologue<To>(h, first_vcycles() > 0);
            if (rc == EMFUSE_OK && first_vcycles() > 0) {
                cudaStreamCaptureStatus cs;
                cudaGraph_t cg = nullptr;
                const cudaGraphNode_t* deps = nullptr;
                size_t ndeps = 0;
                e = cudaStreamGetCaptureInfo(cap_st, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
                cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t loop = nullptr;
                if (e == cudaSuccess) e = cudaGraphAddNode(&loop, cg, deps, nullptr, ndeps, &cp);
                if (e == cudaSuccess)
                    e = cudaStreamUpdateCaptureDependencies(cap_st, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
                if (e == cudaSuccess)
                    e = cudaStreamBeginCaptureToGraph(cap_body, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const uint64_t b0 = launch_count();
                    st = cap_body;
                    rc = record_body<To>(h, true);
                    n_body = (int64_t)(launch_count() - b0);
                    cudaGraph_t body = nullptr;
                    const cudaError_t eb = cudaStreamEndCapture(cap_body, &body);
                    if (e == cudaSuccess) e = eb;
                    st = cap_st;
                }
            }
            if (rc == EMFUSE_OK && e == cudaSuccess) rc = launch_finish<To>();
            n_pro = (int64_t)(launch_count() - c0) - n_body;
            const cudaError_t ee = cudaStreamEndCapture(cap_st, &g);
            if (e == cudaSuccess) e = ee;
            add_launches(-(n_pro + n_body));  // recorded, not run
        }
        st = user;
        if (rc == EMFUSE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&sexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (rc != EMFUSE_OK) {
            sexec = nullptr;
            return rc;
        }
        if (e != cudaSuccess) {
            sexec = nullptr;
            set_error(std::string("solve graph: ") + cudaGetErrorString(e));
            return EMFUSE_ECUDA;
        }
        skey = key;
        s_pro_nodes = n_pro;
        s_body_nodes = n_body;
        s_pro_passes = first_vcycles() > 0 ? 2 : 1;
        return EMFUSE_OK;
    }

    // The same kernels launched directly, the host reading the loop decision after every check
    // (per-launch profiling, opts.no_graphs, the reference schedule).
    template <class To>
    int solve_direct() {
        auto cont = [&](int& c) -> int {
            EMF_CUDA(cudaMemcpyAsync(h_state, d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
            EMF_CUDA(cudaStreamSynchronize(st));
            c = h_state->cont;
            return EMFUSE_OK;
        };
        cudaGraphConditionalHandle none{};
        EMF_TRY(launch_init());
        EMF_TRY((top_pass<To, 0>()));
        const int nv = first_vcycles();
        EMF_TRY(launch_check(nv, false, none));
        int c = 0;
        EMF_TRY(cont(c));
        if (c && nv > 0) {
            for (int v = 0; v < nv; ++v) EMF_TRY(vcycle(v > 0));
            EMF_TRY((top_pass<To, 1>()));
            EMF_TRY(launch_check(1, false, none));
            EMF_TRY(cont(c));
            while (c) {
                EMF_TRY((record_body<To>(none, false)));
                EMF_TRY(cont(c));
            }
        }
        return launch_finish<To>();
    }

    // Stream callback of an asynchronous solve: copies the results to the caller's array and
    // counts the kernels the graph ran (its loop ran a data-dependent number of times).
    struct AsyncJob {
        const emfuse_slice_stats* src;
        emfuse_slice_stats* dst;
        int64_t n;
        const SolveState* state;
        int64_t pro_nodes, body_nodes;
        int pro_passes;
    };
    static void CUDART_CB async_done_cb(void* p) {
        AsyncJob* j = static_cast<AsyncJob*>(p);
        if (j->dst) std::memcpy(j->dst, j->src, (size_t)j->n * sizeof(emfuse_slice_stats));
        add_launches(j->pro_nodes + j->body_nodes * std::max(0, j->state->it - j->pro_passes));
        delete j;
    }

    template <class To>
    int run(const To* o) {
        EMF_TRY(build());
        const int64_t n = rq->nslices;
        int64_t total = 0;
        for (int64_t j = 0; j < n; ++j) total = std::max(total, rq->offsets[j] + rq->nx[j] * rq->ny[j]);
        const int64_t half = round_up(total, 64);
        if (ws_f.bytes() < (size_t)(2 * half) * sizeof(TF))
            EMF_TRY(ws_f.alloc_persistent((size_t)(2 * half) * sizeof(TF)));
        dbuf[0] = ws_f.as<TF>();
        dbuf[1] = ws_f.as<TF>() + half;
        // the graph path needs the fused schedule; instrumented runs time every launch directly
        const bool graph = fused && !rq->opts.no_graphs && !profiling_active();
        const bool async = graph && rq->opts.async_solve;
        {
            KernelScope ks("solve_control", st, 0.0);
            k_set_call<<<1, 1, 0, st>>>(d_call, CallPtrs{rq->s, o, rq->rhs, rq->out});
            EMF_CHECK_LAUNCH();
        }
        if (graph) {
            EMF_TRY(solve_graph<To>());
            EMF_CUDA(cudaGraphLaunch(sexec, st));
        } else {
            EMF_TRY(solve_direct<To>());
        }
        if (rq->opts.verify_residual) {
            EMF_CUDA(cudaMemsetAsync(d_vsums, 0, 2 * n * sizeof(double), st));
            KernelScope ks("residual_verify", st, top_cells * (12.0 + sizeof(TF) + sizeof(To)));
            k_verify<TF, To><<<(unsigned)top_tiles, 256, 0, st>>>(d_top, d_top_ts, (int)n, d_lastp, rq->s, o, rq->rhs,
                                                                    dbuf[0], dbuf[1], rq->alpha, d_vsums);
            EMF_CHECK_LAUNCH();
        }
        {
            KernelScope ks("solve_control", st, 0.0);
            k_stats<<<(unsigned)std::max<int64_t>(1, ceil_div(n, 256)), 256, 0, st>>>(
                (int)n, d_vcyc, d_rel, d_bnorm, rq->opts.verify_residual ? d_vsums : nullptr, rq->opts.tol, d_stats);
            EMF_CHECK_LAUNCH();
        }
        EMF_CUDA(cudaMemcpyAsync(h_stats, d_stats, n * sizeof(emfuse_slice_stats), cudaMemcpyDeviceToHost, st));
        EMF_CUDA(cudaMemcpyAsync(h_state, d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
        if (async) {
            // results reach the caller's array from a stream callback: valid after the stream
            // (or an event recorded after this call) has completed
            AsyncJob* job = new AsyncJob{h_stats, rq->stats, n, h_state, s_pro_nodes, s_body_nodes, s_pro_passes};
            const cudaError_t e = cudaLaunchHostFunc(st, async_done_cb, job);
            if (e != cudaSuccess) {
                delete job;
                set_error(std::string("cudaLaunchHostFunc: ") + cudaGetErrorString(e));
                return EMFUSE_ECUDA;
            }
            if (!async_done) EMF_CUDA(cudaEventCreateWithFlags(&async_done, cudaEventDisableTiming));
            EMF_CUDA(cudaEventRecord(async_done, st));
            return EMFUSE_OK;
        }
        int* dev_err = device_error_flag();  // bounded waits of other kernels (smoothing)
        int dev_flag = 0;
        if (dev_err) EMF_CUDA(cudaMemcpyAsync(&dev_flag, dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        EMF_CUDA(cudaStreamSynchronize(st));
        if (graph) add_launches(s_pro_nodes + s_body_nodes * std::max(0, h_state->it - s_pro_passes));
        if (rq->stats) std::memcpy(rq->stats, h_stats, (size_t)n * sizeof(emfuse_slice_stats));
        if (h_state->timeout || dev_flag) {
            cudaMemsetAsync(d_err, 0, sizeof(int), st);
            if (dev_err) cudaMemsetAsync(dev_err, 0, sizeof(int), st);
            cudaStreamSynchronize(st);
            set_error("a bounded device-side wait (TMA staging) expired");
            return EMFUSE_ETIMEOUT;
        }
        bool nonfinite = false, converged = true;
        for (int64_t j = 0; j < n; ++j) {
            nonfinite |= !std::isfinite(h_stats[j].rel_residual);
            converged &= h_stats[j].rel_residual <= rq->opts.tol;
        }
        if (nonfinite) {
            set_error("non-finite residual (NaN or Inf in the inputs?)");
            return EMFUSE_EINVAL;
        }
        if (!converged) {
            set_error("tolerance not reached within max_vcycles");
            return EMFUSE_ENOCONV;
        }
        return EMFUSE_OK;
    }
};

// Solver plans (descriptor tables, TMA tensor maps, multigrid pyramids, FP64 iterate) are
// kept between calls, one per (device, stream, precision), and rebuilt when the slice
// geometry or the schedule options change.  A plan is used by one call at a time.
struct PlanEntry {
    int dev;
    cudaStream_t st;
    int prec;
    std::shared_ptr<void> solver;
    std::shared_ptr<std::mutex> mu;
    size_t (*bytes)(const void*);  // large buffers held by the solver
};
std::mutex g_plans_mu;
// heap-allocated and never destroyed: no CUDA call from a static destructor at process exit
std::vector<PlanEntry>& g_plans = *new std::vector<PlanEntry>();
constexpr size_t kMaxPlans = 4;

template <class TF, class TV>
int run_precision(const SolveRequest& req, cudaStream_t st) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    const int prec = req.opts.precision;
    std::shared_ptr<Solver<TF, TV>> solver;
    std::shared_ptr<std::mutex> mu;
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        for (auto& e : g_plans)
            if (e.dev == dev && e.st == st && e.prec == prec) {
                solver = std::static_pointer_cast<Solver<TF, TV>>(e.solver);
                mu = e.mu;
            }
        if (!solver) {
            if (g_plans.size() >= kMaxPlans) g_plans.erase(g_plans.begin());
            solver = std::make_shared<Solver<TF, TV>>(st);
            mu = std::make_shared<std::mutex>();
            g_plans.push_back(PlanEntry{dev, st, prec, solver, mu, [](const void* p) -> size_t {
                const auto* s = static_cast<const Solver<TF, TV>*>(p);
                return s->ws_levels.bytes() + s->ws_f.bytes();
            }});
        }
    }
    std::lock_guard<std::mutex> lk(*mu);
    solver->rq = &req;
    int rc;
    if (req.rhs || req.o_dtype == EMFUSE_F32) rc = solver->run(static_cast<const float*>(req.o));
    else rc = solver->run(static_cast<const uint8_t*>(req.o));
    if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) solver->built = false;  // rebuild after an error
    return rc;
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

static int solve_batch_once(const SolveRequest& req, cudaStream_t st) {
    switch (req.opts.precision) {
        case EMFUSE_PREC_FP32: return run_precision<float, float>(req, st);
        case EMFUSE_PREC_MIXED: return run_precision<double, float>(req, st);
        case EMFUSE_PREC_FP64: return run_precision<double, double>(req, st);
        default: set_error("unknown precision mode"); return EMFUSE_EINVAL;
    }
}

// ---------------------------------------------------------------- autotuner
// Schedules are compared by the time of a complete solve to the requested tolerance (a
// schedule with fewer sweeps is cheaper per V-cycle but may need more V-cycles).  The search
// is staged: rows per work item on the finest level in {32, 64, 128, 256} with nu = (2, 2),
// then (nu_pre, nu_post) in {(1, 1), (1, 2), (2, 1), (2, 3), (3, 2), (3, 3), (3, 4)} with the best
// rows (one to four red-black sweeps per leg, all in the fused wavefront kernels).  Each candidate runs twice (the
// first run builds its plan and captures its graphs) and the second run is timed.  The winner
// is cached per batch geometry, alpha, precision and tol.
namespace {
struct TuneKey {
    std::vector<int64_t> geom;
    int precision;
    double tol, alpha;
    int first_vcycles, max_vcycles;
    bool operator<(const TuneKey& o) const {
        return std::tie(geom, precision, tol, alpha, first_vcycles, max_vcycles) <
               std::tie(o.geom, o.precision, o.tol, o.alpha, o.first_vcycles, o.max_vcycles);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, emfuse_tune_entry>& g_tune_cache = *new std::map<TuneKey, emfuse_tune_entry>();
thread_local std::vector<emfuse_tune_entry> t_last_tune;

int time_solve(const SolveRequest& req, cudaStream_t st, emfuse_tune_entry& e) {
    std::vector<emfuse_slice_stats> stats((size_t)req.nslices);
    SolveRequest r = req;
    r.stats = stats.data();
    cudaEvent_t a = nullptr, b = nullptr;
    EMF_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        set_error("autotune: cudaEventCreate failed");
        return EMFUSE_ECUDA;
    }
    cudaEventRecord(a, st);
    const int rc = solve_batch_once(r, st);
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) ms = -1.f;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e.ms = ms;
    e.vcycles = 0;
    for (const auto& s : stats) e.vcycles = std::max(e.vcycles, s.vcycles);
    return rc;
}
}  // namespace

int solve_batch(const SolveRequest& req, cudaStream_t st) {
    if (!req.opts.autotune || !req.opts.fused) return solve_batch_once(req, st);
    TuneKey key;
    key.geom.reserve(3 * (size_t)req.nslices);
    for (int64_t j = 0; j < req.nslices; ++j) {
        key.geom.push_back(req.nx[j]);
        key.geom.push_back(req.ny[j]);
        key.geom.push_back(req.offsets[j]);
    }
    key.precision = req.opts.precision;
    key.tol = req.opts.tol;
    key.alpha = req.alpha;
    key.first_vcycles = req.opts.first_vcycles;
    key.max_vcycles = req.opts.max_vcycles;
    SolveRequest r = req;
    r.opts.autotune = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            r.opts.nu_pre = it->second.nu_pre;
            r.opts.nu_post = it->second.nu_post;
            r.opts.tile_rows = it->second.tile_rows;
            return solve_batch_once(r, st);
        }
    }
    std::vector<emfuse_tune_entry> table;
    auto trial = [&](int np, int nq, int rows) -> int {
        SolveRequest c = r;
        c.stats = nullptr;
        c.opts.verify_residual = 0;
        c.opts.async_solve = 0;
        c.opts.nu_pre = np;
        c.opts.nu_post = nq;
        c.opts.tile_rows = rows;
        emfuse_tune_entry e{np, nq, rows, 0, 0.0};
        int rc = solve_batch_once(c, st);  // builds the plan and its graphs
        if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) return rc;
        rc = time_solve(c, st, e);
        if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) return rc;
        if (rc == EMFUSE_ENOCONV) e.ms = -1.0;  // did not reach tol: never chosen
        table.push_back(e);
        return EMFUSE_OK;
    };
    auto best_of = [&]() {
        int b = -1;
        for (int i = 0; i < (int)table.size(); ++i)
            if (table[i].ms >= 0 && (b < 0 || table[i].ms < table[b].ms)) b = i;
        return b;
    };
    // rows per work item (the tile height of a 128-column strip) at nu = (2, 2), then every
    // other sweep count with the two fastest tile heights
    for (int rows : {32, 64, 128, 256}) EMF_TRY(trial(2, 2, rows));
    std::vector<emfuse_tune_entry> by_rows(table);
    std::stable_sort(by_rows.begin(), by_rows.end(), [](const emfuse_tune_entry& x, const emfuse_tune_entry& y) {
        const double a = x.ms < 0 ? 1e300 : x.ms, c = y.ms < 0 ? 1e300 : y.ms;
        return a < c;
    });
    for (auto nu : {std::pair<int, int>{1, 1}, {1, 2}, {2, 1}, {2, 3}, {3, 2}, {3, 3}, {3, 4}, {4, 4}})
        for (int q = 0; q < 2; ++q) EMF_TRY(trial(nu.first, nu.second, by_rows[q].tile_rows));
    int b = best_of();
    if (b < 0) {
        t_last_tune = table;
        set_error("autotune: no candidate schedule reached the tolerance");
        return EMFUSE_ENOCONV;
    }
    std::swap(table[0], table[b]);
    t_last_tune = table;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = table[0];
    }
    r.opts.nu_pre = table[0].nu_pre;
    r.opts.nu_post = table[0].nu_post;
    r.opts.tile_rows = table[0].tile_rows;
    return solve_batch_once(r, st);
}

const std::vector<emfuse_tune_entry>& last_autotune() { return t_last_tune; }

int solve_async_status(cudaStream_t st, int precision) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    std::shared_ptr<void> solver;
    std::shared_ptr<std::mutex> mu;
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        for (auto& e : g_plans)
            if (e.dev == dev && e.st == st && e.prec == precision) {
                solver = e.solver;
                mu = e.mu;
            }
    }
    if (!solver) return EMFUSE_OK;
    std::lock_guard<std::mutex> lk(*mu);
    auto status = [&](auto* sv) -> int {
        if (!sv->h_state || !sv->d_err) return EMFUSE_OK;
        int flag = 0;
        EMF_CUDA(cudaMemcpyAsync(&flag, sv->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        EMF_CUDA(cudaStreamSynchronize(st));
        if (!flag && !sv->h_state->timeout) return EMFUSE_OK;
        cudaMemsetAsync(sv->d_err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        set_error("a bounded device-side wait (TMA staging) expired");
        return EMFUSE_ETIMEOUT;
    };
    switch (precision) {
        case EMFUSE_PREC_FP32: return status(static_cast<Solver<float, float>*>(solver.get()));
        case EMFUSE_PREC_MIXED: return status(static_cast<Solver<double, float>*>(solver.get()));
        default: return status(static_cast<Solver<double, double>*>(solver.get()));
    }
}

size_t cached_plan_bytes(cudaStream_t st, int precision) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_plans_mu);
    size_t b = 0;
    for (auto& e : g_plans)
        if (e.dev == dev && e.st == st && e.prec == precision && e.bytes) b += e.bytes(e.solver.get());
    return b;
}

void release_plans() {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    g_plans.clear();
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
