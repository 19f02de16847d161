// Phase 1 of the method: anisotropic Gaussian smoothing I1 = I0 * G_{sigma_xy, sigma_z}
// (Sec. 3 "Anisotropic Smoothing"), with the Gaussian cut off beyond three standard deviations
// (Sec. 3 "Implementation") and the weights renormalised over the taps inside the stack.
//
// Three implementations:
//   * smooth_tma_kernel (default): one HBM pass.  A CTA owns a 64x16 xy-tile and marches
//     along z.  Input planes (tile plus xy halo) arrive by TMA bulk tensor copies into a ring of
//     shared-memory buffers, all but one in flight while a plane is blurred; the hardware
//     zero-fills the halo outside the stack.  x blur in items of 8 outputs, one barrier per
//     plane, y blur of 2 x 2 outputs per thread, then a 19-plane register ring along z (moved
//     once per block of planes, so the march stays a small rolled loop).  Needs rows whose
//     byte pitch is a multiple of 16.
//   * smooth_fused_kernel: the same data flow with plain loads, for any pitch.
//     Each input plane is staged in shared memory with its xy halo, blurred in x then y,
//     and pushed into a per-thread ring of the last P planes held in registers; the z-blur of
//     the plane R behind is emitted from the ring.  The ring index is a compile-time constant
//     (the z loop is unrolled by the ring period P), so the ring never leaves registers.
//     Reads I0 once (plus L2-resident halo) and writes I1 once.
//   * axis_conv_kernel: one renormalised 1-D pass along x, y or z with optional pre/post
//     scaling.  Used for large supports, for the transpose K^T and for dK/dsigma_z in the
//     adjoint, and as an independent cross-check of the fused kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"
#include "tma.cuh"

namespace emfuse {

namespace {

constexpr int kTX = 64;   // tile width (outputs)
constexpr int kTY = 16;   // tile height (outputs)
constexpr int kThreads = 256;
constexpr int kMaxRxy = 8;

struct SmoothParams {
    float wxy[2 * kMaxRxy + 1];  // taps w(d), d = -Rxy..Rxy
    float wz[19];                // wz[j] = w(Rz - j), j = 0..2Rz (zero beyond)
    int Rxy, Rz;
    float kappa2;                // robust averaging: squared threshold in standard deviations
};

// Robust z-average of one voxel (Sec. 3, the outlier example: only values within kappa
// weighted standard deviations of the window's weighted mean are averaged).  v[j] are the
// xy-smoothed window values, w[j] their tap weights (0 for taps outside the stack).
template <int P>
__device__ __forceinline__ float robust_window(const float (&v)[P], const float (&w)[P], float kappa2) {
    float W = 0.f, m = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        W += w[j];
        m = fmaf(w[j], v[j], m);
    }
    const float mu = m / W;
    float s2 = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const float dv = v[j] - mu;
        s2 = fmaf(w[j] * dv, dv, s2);
    }
    const float thr = kappa2 * (s2 / W);
    float sk = 0.f, wk = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const float dv = v[j] - mu;
        const float wj = dv * dv <= thr ? w[j] : 0.f;
        wk += wj;
        sk = fmaf(wj, v[j], sk);
    }
    return sk / wk;
}

template <class Tin>
__device__ __forceinline__ float load_in(const Tin* p) { return float(*p); }

template <class Tin, int P, bool ROB>
__global__ void __launch_bounds__(kThreads, 2)
smooth_fused_kernel(const Tin* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz,
                    int64_t pitch, int z0, int z1, const float* __restrict__ inv_nx,
                    const float* __restrict__ inv_ny, const float* __restrict__ inv_nz,
                    SmoothParams prm) {
    constexpr int MAXH = kTY + 2 * kMaxRxy;
    __shared__ float s_in[MAXH][kTX + 2 * kMaxRxy + 1];
    __shared__ float s_x[MAXH][kTX];

    const int R = prm.Rxy;
    const int Rz = prm.Rz;
    const int x0 = blockIdx.x * kTX;
    const int y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    const int tx = tid % 16;  // 4 consecutive x per thread
    const int ty = tid / 16;  // one row per thread
    const int W = kTX + 2 * R;
    const int H = kTY + 2 * R;
    const int64_t plane = pitch * (int64_t)ny;

    float ring[P][4];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) ring[q][i] = 0.f;

    // input planes that influence outputs [z0, z1)
    const int zin_lo = max(0, z0 - Rz);
    const int zin_hi = min(nz, z1 + Rz);  // exclusive
    // zi runs from zin_lo to z1 - 1 + Rz; output zo = zi - Rz
    const int zi_end = z1 + Rz;

    for (int zb = zin_lo; zb < zi_end; zb += P) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int zi = zb + q;
            if (zi >= zi_end) break;  // uniform across the CTA
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (zi < zin_hi) {
                const Tin* src = in + (int64_t)zi * plane;
                __syncthreads();
                for (int e = tid; e < W * H; e += kThreads) {
                    const int r = e / W, c = e - r * W;
                    const int gy = y0 - R + r, gx = x0 - R + c;
                    float val = 0.f;
                    if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) val = load_in(src + (int64_t)gy * pitch + gx);
                    s_in[r][c] = val;
                }
                __syncthreads();
                for (int e = tid; e < kTX * H; e += kThreads) {
                    const int r = e / kTX, c = e - r * kTX;
                    float acc = 0.f;
                    for (int d = -R; d <= R; ++d) acc = fmaf(prm.wxy[d + R], s_in[r][c + R + d], acc);
                    const int gx = min(x0 + c, nx - 1);
                    s_x[r][c] = acc * inv_nx[gx];
                }
                __syncthreads();
                const int gy = min(y0 + ty, ny - 1);
                const float iny = inv_ny[gy];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float acc = 0.f;
                    for (int d = -R; d <= R; ++d) acc = fmaf(prm.wxy[d + R], s_x[ty + R + d][4 * tx + i], acc);
                    v[i] = acc * iny;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) ring[q][i] = v[i];
            const int zo = zi - Rz;
            if (zo >= z0 && zo < z1) {
                float o4[4] = {0.f, 0.f, 0.f, 0.f};
                float inz = 1.f;
                if constexpr (ROB) {
                    float wv[P];
#pragma unroll
                    for (int j = 0; j < P; ++j) wv[j] = (zi - j >= 0 && zi - j < nz) ? prm.wz[j] : 0.f;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float vv[P];
#pragma unroll
                        for (int j = 0; j < P; ++j) vv[j] = ring[(q - j + P * 4) % P][i];
                        o4[i] = robust_window<P>(vv, wv, prm.kappa2);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < P; ++j) {
                        const float w = prm.wz[j];
                        const int slot = (q - j + P * 4) % P;
#pragma unroll
                        for (int i = 0; i < 4; ++i) o4[i] = fmaf(w, ring[slot][i], o4[i]);
                    }
                    inz = inv_nz[zo];
                }
                const int gy = y0 + ty;
                if (gy < ny) {
                    float* dst = out + (int64_t)(zo - z0) * plane + (int64_t)gy * pitch;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int gx = x0 + 4 * tx + i;
                        if (gx < nx) dst[gx] = o4[i] * inz;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- TMA-staged kernel
// Shared-memory layout of the TMA kernel for input type Tin and xy radius R.
template <class Tin, int R>
struct SmTile {
    static constexpr int HX = sizeof(Tin) == 1 ? 16 : 4;   // staged columns left of the tile: the
                                                          // copy's x-start stays 16-byte aligned
    static constexpr int HXR = sizeof(Tin) == 1 ? 16 : 8;  // right: a float row of 76 words is
                                                          // 304 B, so 8 consecutive rows start in
                                                          // 8 different 16-B bank groups
    static constexpr int BX = kTX + HX + HXR;
    static constexpr int BY = kTY + 2 * R;
    static constexpr int kPlaneBytes = BX * BY * (int)sizeof(Tin);
    static constexpr int kPlaneStride = (kPlaneBytes + 127) / 128 * 128;  // TMA destinations 128-B aligned
    // plane buffers, all in flight except the one being blurred (about 64 KiB of copies in
    // flight per SM with two CTAs per SM for float input)
    static constexpr int NBUF = sizeof(Tin) == 1 ? 8 : 5;
    static constexpr int SXW = kTX + 4;                    // x-blurred row stride (words): 272 B,
                                                          // 8 rows -> 8 different bank groups
    static constexpr int kRowBlocks = (BY + 7) / 8;        // x-blur items: 8 rows x 8 groups each
    static constexpr int kXItems = 64 * kRowBlocks;        // <= 256 for R <= 4
    static constexpr int kSmemBytes = NBUF * kPlaneStride + 2 * BY * SXW * 4 + NBUF * 8;
};

// 16 consecutive staged values (as float) starting at p.
template <class Tin>
__device__ __forceinline__ void load16(const Tin* p, float (&s)[16]);
template <>
__device__ __forceinline__ void load16<float>(const float* p, float (&s)[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = reinterpret_cast<const float4*>(p)[k];
        s[4 * k] = q.x; s[4 * k + 1] = q.y; s[4 * k + 2] = q.z; s[4 * k + 3] = q.w;
    }
}
template <>
__device__ __forceinline__ void load16<uint8_t>(const uint8_t* p, float (&s)[16]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uchar4 q = reinterpret_cast<const uchar4*>(p)[k];
        s[4 * k] = q.x; s[4 * k + 1] = q.y; s[4 * k + 2] = q.z; s[4 * k + 3] = q.w;
    }
}

// One HBM pass of the separable smoothing.  A CTA owns a 64 x 16 xy-tile and marches along z.
// Per input plane (arriving by TMA into a ring of NBUF shared-memory buffers, zero-filled
// outside the stack):
//   x blur   items of 8 outputs on one staged row (rows tile + y halo), written to one of two
//            x-blurred planes; 8 consecutive lanes take 8 rows, so the vector loads and
//            stores of a quarter-warp fall in distinct banks;
//   barrier  the only one per plane: the x-blurred plane is complete, the staged buffer is
//            free and is refilled with the plane NBUF ahead;
//   y blur   each thread 2 columns x 2 rows into a register ring of the last 19 planes;
//   z blur   the plane Rz behind is emitted from the ring, scaled by the product of the three
//            inverse normalisers.
// The taps are kernel parameters with compile-time indices, i.e. constant-bank operands of the
// FMAs.  The blurs sum in their own order and scale once at the end, so results agree with the
// other implementations to rounding.
template <class Tin, int R, bool ROB>
__global__ void __launch_bounds__(kThreads, 2)
smooth_tma_kernel(const __grid_constant__ CUtensorMap map, float* __restrict__ out, int nx, int ny, int nz,
                  int64_t pitch, int z0, int z1, const float* __restrict__ inv_nx,
                  const float* __restrict__ inv_ny, const float* __restrict__ inv_nz, SmoothParams prm,
                  int* __restrict__ err) {
    using G = SmTile<Tin, R>;
    constexpr int P = 19;  // z taps: supports floor(3 sigma_z) <= 9
    constexpr int NB = G::NBUF;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_raw = smem;
    float* s_x = reinterpret_cast<float*>(smem + NB * G::kPlaneStride);  // [2][BY][SXW]
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + NB * G::kPlaneStride + 2 * G::BY * G::SXW * 4);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int Rz = prm.Rz;
    const int zin_lo = max(0, z0 - Rz), zin_hi = min(nz, z1 + Rz), zi_end = z1 + Rz;
    const uint32_t bar0 = smem_addr(&s_bar[0]);
    if (tid == 0) {
        for (int q = 0; q < NB; ++q) mbar_init(bar0 + 8 * q, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0: plane zi into buffer slot (zi - zin_lo) mod NB; a slot is refilled only after
    // the barrier that ended the x blur of the plane it held
    auto issue = [&](int zi, int slot) {
        fence_proxy_async();
        mbar_expect_tx(bar0 + 8 * slot, G::kPlaneBytes);
        tma_load_3d(smem_addr(s_raw + slot * G::kPlaneStride), &map, x0 - G::HX, y0 - R, zi, bar0 + 8 * slot);
    };
    if (tid == 0)
        for (int q = 0; q < NB && zin_lo + q < zin_hi; ++q) issue(zin_lo + q, q);

    // x-blur item of this thread (warp-uniform participation: kXItems is a multiple of 64)
    const bool xw = tid < G::kXItems;
    const int xr = (tid >> 6) * 8 + (tid & 7);  // staged row
    const int xg = (tid >> 3) & 7;              // group of 8 output columns
    const bool xitem = xw && xr < G::BY;
    const Tin* const s_in0 = reinterpret_cast<const Tin*>(s_raw) + xr * G::BX + 8 * xg + G::HX - 4;
    float* const sx_item = s_x + xr * G::SXW + 8 * xg;
    // y/z outputs of this thread: columns 2 lane, 2 lane + 1 of rows 2 warp, 2 warp + 1
    const int lane = tid & 31, wrp = tid >> 5;
    const int gx = x0 + 2 * lane;
    const int gy0 = y0 + 2 * wrp, gy1 = gy0 + 1;
    const float* const sy_col = s_x + (2 * wrp) * G::SXW + 2 * lane;
    float sxy[4];  // inv_x * inv_y of the 4 outputs (row 0 x, row 0 x+1, row 1 x, row 1 x+1)
    {
        const float ix0 = inv_nx[min(gx, nx - 1)], ix1 = inv_nx[min(gx + 1, nx - 1)];
        const float iy0 = inv_ny[min(gy0, ny - 1)], iy1 = inv_ny[min(gy1, ny - 1)];
        sxy[0] = ix0 * iy0; sxy[1] = ix1 * iy0; sxy[2] = ix0 * iy1; sxy[3] = ix1 * iy1;
    }
    const bool st0 = gy0 < ny, st1 = gy1 < ny;
    const bool vec2 = (pitch & 1) == 0 && (reinterpret_cast<uintptr_t>(out) & 7) == 0 && gx + 1 < nx;
    float* const dst0 = out + (int64_t)min(gy0, ny - 1) * pitch + gx;
    float* const dst1 = out + (int64_t)min(gy1, ny - 1) * pitch + gx;

    // z ring: slots 0 .. P-2 hold the P-1 planes before the current block of U planes, slots
    // P-1 .. P-2+U the block; the ring moves by U slots once per block (the loop over a block is
    // unrolled, so every slot index is a constant)
    constexpr int U = ROB ? 2 : 4;  // the robust window needs more registers of its own
    float ring[P - 1 + U][4];
#pragma unroll
    for (int q = 0; q < P - 1 + U; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) ring[q][c] = 0.f;
    const int64_t plane = pitch * (int64_t)ny;

    int slot = 0;        // buffer slot of plane zi
    uint32_t phase = 0;  // barrier parity of the current lap over the slots
    int buf = 0;         // x-blurred plane buffer (0 or 1)
#pragma unroll 1
    for (int zb = zin_lo; zb < zi_end; zb += U) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int zi = zb + u;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (zi < zin_hi) {  // uniform across the CTA
                bool ok = true;
                const int boff = buf * (G::BY * G::SXW);
                if (xw) {
                    ok = mbar_wait_warp(bar0 + 8 * slot, phase);
                    if (ok && xitem) {
                        float s[16];
                        load16<Tin>(s_in0 + slot * (G::kPlaneStride / (int)sizeof(Tin)), s);
                        // output i sits at s[4 + i]
                        float o[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float acc = prm.wxy[0] * s[4 + i - R];
#pragma unroll
                            for (int d = -R + 1; d <= R; ++d) acc = fmaf(prm.wxy[d + R], s[4 + i + d], acc);
                            o[i] = acc;
                        }
                        float4* dst = reinterpret_cast<float4*>(sx_item + boff);
                        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
                        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
                    }
                }
                if (!__syncthreads_and(ok)) {
                    // give up: flag the host, let the copies in flight land, leave
                    if (tid == 0) {
                        atomicExch(err, 1);
                        for (int zz = zi; zz < zin_hi && zz < zi + NB; ++zz) {
                            const int k = zz - zin_lo;
                            const uint32_t b = bar0 + 8 * (k % NB), ph = (uint32_t)((k / NB) & 1);
                            for (int it = 0; it < kWaitLimit; ++it)
                                if (mbar_try_wait(b, ph)) break;
                        }
                    }
                    __syncthreads();
                    return;
                }
                if (tid == 0 && zi + NB < zin_hi) issue(zi + NB, slot);
                // y blur of rows 2 warp, 2 warp + 1 (x-blurred rows 2 warp .. 2 warp + 2R + 1)
#pragma unroll
                for (int t = 0; t <= 2 * R + 1; ++t) {
                    const float2 q = *reinterpret_cast<const float2*>(sy_col + boff + t * G::SXW);
                    if (t == 0) {
                        v[0] = prm.wxy[0] * q.x;
                        v[1] = prm.wxy[0] * q.y;
                    } else if (t <= 2 * R) {
                        v[0] = fmaf(prm.wxy[t], q.x, v[0]);
                        v[1] = fmaf(prm.wxy[t], q.y, v[1]);
                    }
                    if (t == 1) {
                        v[2] = prm.wxy[0] * q.x;
                        v[3] = prm.wxy[0] * q.y;
                    } else if (t >= 2) {
                        v[2] = fmaf(prm.wxy[t - 1], q.x, v[2]);
                        v[3] = fmaf(prm.wxy[t - 1], q.y, v[3]);
                    }
                }
                if (R == 0) {  // 2R + 1 = 1 row per output
                    const float2 q = *reinterpret_cast<const float2*>(sy_col + boff + G::SXW);
                    v[2] = prm.wxy[0] * q.x;
                    v[3] = prm.wxy[0] * q.y;
                }
                if (++slot == NB) { slot = 0; phase ^= 1u; }
                buf ^= 1;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[P - 1 + u][c] = v[c];
            // emit plane zi - Rz from ring slots u .. u + P - 1 (slot u + P - 1 = plane zi)
            const int zo = zi - Rz;
            if (zo >= z0 && zo < z1) {  // uniform across the CTA
                float o[4];
                if constexpr (ROB) {
                    float wv[P];
#pragma unroll
                    for (int jj = 0; jj < P; ++jj) wv[jj] = (zi - jj >= 0 && zi - jj < nz) ? prm.wz[jj] : 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float vv[P];
#pragma unroll
                        for (int jj = 0; jj < P; ++jj) vv[jj] = ring[u + P - 1 - jj][c];
                        o[c] = robust_window<P>(vv, wv, prm.kappa2) * sxy[c];
                    }
                } else {
                    const float inz = inv_nz[zo];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float acc = prm.wz[0] * ring[u + P - 1][c];
#pragma unroll
                        for (int jj = 1; jj < P; ++jj) acc = fmaf(prm.wz[jj], ring[u + P - 1 - jj][c], acc);
                        o[c] = acc * (sxy[c] * inz);
                    }
                }
                const int64_t zoff = (int64_t)(zo - z0) * plane;
                if (vec2) {
                    if (st0) *reinterpret_cast<float2*>(dst0 + zoff) = make_float2(o[0], o[1]);
                    if (st1) *reinterpret_cast<float2*>(dst1 + zoff) = make_float2(o[2], o[3]);
                } else {
                    if (st0 && gx < nx) dst0[zoff] = o[0];
                    if (st0 && gx + 1 < nx) dst0[zoff + 1] = o[1];
                    if (st1 && gx < nx) dst1[zoff] = o[2];
                    if (st1 && gx + 1 < nx) dst1[zoff + 1] = o[3];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P - 1; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) ring[q][c] = ring[q + U][c];
    }
}

// Opt in to the TMA kernel's dynamic shared memory once per instantiation and device.
template <class Tin, int R, bool ROB>
int smooth_tma_prepare() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return EMFUSE_OK;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        EMF_CUDA(cudaFuncSetAttribute(smooth_tma_kernel<Tin, R, ROB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SmTile<Tin, R>::kSmemBytes));
        done[dev] = true;
    }
    return EMFUSE_OK;
}

struct AxisParams {
    float w[65];
    int R;
};

// out[p] = beta * out[p] + post[idx_a(p)] * sum_{|d|<=R, inside} w(d) pre[idx_a(p+d)] in[p+d]
// along axis a (0 = x, 1 = y, 2 = z).  pre / post may be null (= 1).
template <class Tin>
__global__ void axis_conv_kernel(const Tin* __restrict__ in, float* __restrict__ out, int nx,
                                 int ny, int nz, int64_t pitch_in, int64_t pitch_out, int axis,
                                 const float* __restrict__ pre, const float* __restrict__ post,
                                 float beta, AxisParams prm) {
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = int(i % nx);
        const int y = int((i / nx) % ny);
        const int z = int(i / ((int64_t)nx * ny));
        const int c = axis == 0 ? x : (axis == 1 ? y : z);
        const int len = axis == 0 ? nx : (axis == 1 ? ny : nz);
        const int64_t stride = axis == 0 ? 1 : (axis == 1 ? pitch_in : pitch_in * ny);
        const int64_t base = (int64_t)z * pitch_in * ny + (int64_t)y * pitch_in + x;
        float acc = 0.f;
        for (int d = -prm.R; d <= prm.R; ++d) {
            const int cc = c + d;
            if (cc < 0 || cc >= len) continue;
            float v = float(in[base + (int64_t)d * stride]);
            if (pre) v *= pre[cc];
            acc = fmaf(prm.w[d + prm.R], v, acc);
        }
        if (post) acc *= post[c];
        const int64_t o = (int64_t)z * pitch_out * ny + (int64_t)y * pitch_out + x;
        out[o] = beta == 0.f ? acc : fmaf(beta, out[o], acc);
    }
}

}  // namespace

int support_radius(float sigma) {
    if (!(sigma > 0.f)) return 0;
    return (int)std::floor(3.0 * (double)sigma + 1e-9);
}

std::vector<float> gaussian_taps(float sigma, int R) {
    std::vector<float> w(2 * R + 1, 1.f);
    if (sigma > 0.f)
        for (int d = -R; d <= R; ++d) w[d + R] = (float)std::exp(-(double)d * d / (2.0 * (double)sigma * sigma));
    return w;
}

// 1 / (sum of in-range taps) for every index 0..n-1 of an axis of length n.
std::vector<float> inverse_norms(const std::vector<float>& w, int n) {
    const int R = ((int)w.size() - 1) / 2;
    std::vector<float> inv(n);
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int d = -R; d <= R; ++d)
            if (i + d >= 0 && i + d < n) s += w[d + R];
        inv[i] = (float)(1.0 / s);
    }
    return inv;
}

static int launch_axis(const void* in, int dt, float* out, int nx, int ny, int nz, int64_t pin,
                       int64_t pout, int axis, const std::vector<float>& w, const float* pre,
                       const float* post, float beta, cudaStream_t st) {
    AxisParams prm{};
    prm.R = ((int)w.size() - 1) / 2;
    if (prm.R > 32) {
        set_error("smoothing support radius above 32 taps is not supported");
        return EMFUSE_EINVAL;
    }
    for (size_t i = 0; i < w.size(); ++i) prm.w[i] = w[i];
    const int64_t n = (int64_t)nx * ny * nz;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, threads), (int64_t)kNumSMs * 32);
    KernelScope ks("smooth_axis", st, (double)n * ((dt == EMFUSE_U8 ? 1.0 : 4.0) + 4.0 + (beta != 0.f ? 4.0 : 0.0)));
    if (dt == EMFUSE_U8)
        axis_conv_kernel<uint8_t><<<(unsigned)blocks, threads, 0, st>>>(
            (const uint8_t*)in, out, nx, ny, nz, pin, pout, axis, pre, post, beta, prm);
    else
        axis_conv_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            (const float*)in, out, nx, ny, nz, pin, pout, axis, pre, post, beta, prm);
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}

// Device table of the inverse normalisers of the three axes: [inv_x | inv_y | inv_z].
static int upload_norms(DeviceBuffer& buf, const std::vector<float>& ix, const std::vector<float>& iy,
                        const std::vector<float>& iz, cudaStream_t st, std::vector<float>& host) {
    host.clear();
    host.insert(host.end(), ix.begin(), ix.end());
    host.insert(host.end(), iy.begin(), iy.end());
    host.insert(host.end(), iz.begin(), iz.end());
    EMF_TRY(buf.alloc(host.size() * sizeof(float), st));
    EMF_CUDA(cudaMemcpyAsync(buf.as<float>(), host.data(), host.size() * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    return EMFUSE_OK;
}

int smooth_stack(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                 int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                 cudaStream_t st, int force_path, float kappa) {
    const int Rxy = support_radius(sigma_xy);
    const int Rz = support_radius(sigma_z);
    const bool rob = kappa > 0.f;
    if (rob && (Rxy > kMaxRxy || Rz > 9 || force_path == 1)) {
        set_error("robust averaging needs floor(3 sigma_xy) <= 8 and floor(3 sigma_z) <= 9");
        return EMFUSE_EINVAL;
    }
    const auto wxy = gaussian_taps(sigma_xy, Rxy);
    const auto wz = gaussian_taps(sigma_z, Rz);
    std::vector<float> host;
    DeviceBuffer norms;
    EMF_TRY(upload_norms(norms, inverse_norms(wxy, (int)nx), inverse_norms(wxy, (int)ny),
                         inverse_norms(wz, (int)nz), st, host));
    const float* inv_x = norms.as<float>();
    const float* inv_y = inv_x + nx;
    const float* inv_z = inv_y + ny;

    const size_t esz = dt == EMFUSE_U8 ? 1 : 4;
    const bool tma_ok = Rxy <= 4 && Rz <= 9 && force_path == 0 && (pitch * (int64_t)esz) % 16 == 0 &&
                        (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    if (tma_ok) {
        SmoothParams prm{};
        prm.Rxy = Rxy;
        prm.Rz = Rz;
        for (int d = 0; d < 2 * Rxy + 1; ++d) prm.wxy[d] = wxy[d];
        for (int j = 0; j < 2 * Rz + 1; ++j) prm.wz[j] = wz[2 * Rz - j];
        prm.kappa2 = kappa * kappa;
        CUtensorMap map;
        const int hx = dt == EMFUSE_U8 ? 16 : 4, hxr = dt == EMFUSE_U8 ? 16 : 8;
        EMF_TRY(encode_tensor_map_3d(&map, in, (int)esz, nx, ny, nz, pitch, kTX + hx + hxr, kTY + 2 * Rxy));
        int* err = device_error_flag();
        if (!err) {
            set_error("could not allocate the device error word");
            return EMFUSE_ECUDA;
        }
        dim3 grid((unsigned)ceil_div(nx, kTX), (unsigned)ceil_div(ny, kTY));
        const int64_t zin0 = std::max<int64_t>(0, z0 - Rz), zin1 = std::min<int64_t>(nz, z1 + Rz);
        {
            KernelScope ks(rob ? "smooth_tma_robust" : "smooth_tma", st,
                           (double)nx * ny * ((zin1 - zin0) * (double)esz + (z1 - z0) * 4.0));
#define EMF_SMOOTH_TMA2(TT, RR, RB)                                                                \
    do {                                                                                           \
        EMF_TRY((smooth_tma_prepare<TT, RR, RB>()));                                               \
        smooth_tma_kernel<TT, RR, RB><<<grid, kThreads, SmTile<TT, RR>::kSmemBytes, st>>>(          \
            map, out, (int)nx, (int)ny, (int)nz, pitch, (int)z0, (int)z1, inv_x, inv_y, inv_z, prm, err);       \
    } while (0)
#define EMF_SMOOTH_TMA1(RR, RB)                                                                    \
    do {                                                                                           \
        if (dt == EMFUSE_U8) EMF_SMOOTH_TMA2(uint8_t, RR, RB);                                     \
        else EMF_SMOOTH_TMA2(float, RR, RB);                                                       \
    } while (0)
#define EMF_SMOOTH_TMA(RR)                                                                         \
    do {                                                                                           \
        if (rob) EMF_SMOOTH_TMA1(RR, true);                                                        \
        else EMF_SMOOTH_TMA1(RR, false);                                                           \
    } while (0)
            switch (Rxy) {
                case 0: EMF_SMOOTH_TMA(0); break;
                case 1: EMF_SMOOTH_TMA(1); break;
                case 2: EMF_SMOOTH_TMA(2); break;
                case 3: EMF_SMOOTH_TMA(3); break;
                default: EMF_SMOOTH_TMA(4); break;
            }
#undef EMF_SMOOTH_TMA
#undef EMF_SMOOTH_TMA1
#undef EMF_SMOOTH_TMA2
            EMF_CHECK_LAUNCH();
        }
        // a timed-out wait is reported by the next call that synchronises (the solves)
        return EMFUSE_OK;
    }
    const bool fused_ok = Rxy <= kMaxRxy && Rz <= 9 && force_path != 1;
    if (fused_ok) {
        SmoothParams prm{};
        prm.Rxy = Rxy;
        prm.Rz = Rz;
        for (int d = 0; d < 2 * Rxy + 1; ++d) prm.wxy[d] = wxy[d];
        for (int j = 0; j < 2 * Rz + 1; ++j) prm.wz[j] = wz[2 * Rz - j];
        prm.kappa2 = kappa * kappa;
        dim3 grid((unsigned)ceil_div(nx, kTX), (unsigned)ceil_div(ny, kTY));
        const int P = 2 * Rz + 1;
        const int64_t zin0 = std::max<int64_t>(0, z0 - Rz), zin1 = std::min<int64_t>(nz, z1 + Rz);
        KernelScope ks(rob ? "smooth_fused_robust" : "smooth_fused", st,
                       (double)nx * ny * ((zin1 - zin0) * (dt == EMFUSE_U8 ? 1.0 : 4.0) + (z1 - z0) * 4.0));
#define EMF_SMOOTH_LAUNCH1(PP, RB)                                                             \
    do {                                                                                       \
        if (dt == EMFUSE_U8)                                                                   \
            smooth_fused_kernel<uint8_t, PP, RB><<<grid, kThreads, 0, st>>>(                   \
                (const uint8_t*)in, out, (int)nx, (int)ny, (int)nz, pitch, (int)z0, (int)z1,   \
                inv_x, inv_y, inv_z, prm);                                                     \
        else                                                                                   \
            smooth_fused_kernel<float, PP, RB><<<grid, kThreads, 0, st>>>(                     \
                (const float*)in, out, (int)nx, (int)ny, (int)nz, pitch, (int)z0, (int)z1,     \
                inv_x, inv_y, inv_z, prm);                                                     \
    } while (0)
#define EMF_SMOOTH_LAUNCH(PP)                                                                  \
    do {                                                                                       \
        if (rob) EMF_SMOOTH_LAUNCH1(PP, true);                                                 \
        else EMF_SMOOTH_LAUNCH1(PP, false);                                                    \
    } while (0)
        if (P <= 1) EMF_SMOOTH_LAUNCH(1);
        else if (P <= 7) EMF_SMOOTH_LAUNCH(7);
        else EMF_SMOOTH_LAUNCH(19);
#undef EMF_SMOOTH_LAUNCH
#undef EMF_SMOOTH_LAUNCH1
        EMF_CHECK_LAUNCH();
        return EMFUSE_OK;
    }
    // Three renormalised 1-D passes (x, y over the needed input planes; then z).
    const int64_t zin0 = std::max<int64_t>(0, z0 - Rz), zin1 = std::min<int64_t>(nz, z1 + Rz);
    const int64_t nzin = zin1 - zin0;
    DeviceBuffer t1, t2;
    EMF_TRY(t1.alloc((size_t)(nzin * ny * nx) * sizeof(float), st));
    EMF_TRY(t2.alloc((size_t)(nzin * ny * nx) * sizeof(float), st));
    const void* in0 = (const char*)in + (size_t)(zin0 * ny * pitch) * esz;
    EMF_TRY(launch_axis(in0, dt, t1.as<float>(), (int)nx, (int)ny, (int)nzin, pitch, nx, 0, wxy,
                        nullptr, inv_x, 0.f, st));
    EMF_TRY(launch_axis(t1.as<float>(), EMFUSE_F32, t2.as<float>(), (int)nx, (int)ny, (int)nzin,
                        nx, nx, 1, wxy, nullptr, inv_y, 0.f, st));
    // z pass: only the requested output planes, normaliser indexed by absolute z
    DeviceBuffer tz;
    EMF_TRY(tz.alloc((size_t)(nzin * ny * nx) * sizeof(float), st));
    std::vector<float> iz_local(host.begin() + nx + ny + zin0, host.begin() + nx + ny + zin1);
    // renormalisation by the absolute-z table: recompute in local coordinates would be wrong
    // when the slab is a sub-range, so scale with the global table slice.
    DeviceBuffer izb;
    EMF_TRY(izb.alloc(iz_local.size() * sizeof(float), st));
    EMF_CUDA(cudaMemcpyAsync(izb.as<float>(), iz_local.data(), iz_local.size() * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    EMF_TRY(launch_axis(t2.as<float>(), EMFUSE_F32, tz.as<float>(), (int)nx, (int)ny, (int)nzin,
                        nx, nx, 2, wz, nullptr, izb.as<float>(), 0.f, st));
    EMF_CUDA(cudaMemcpy2DAsync(out, pitch * sizeof(float),
                               tz.as<float>() + (z0 - zin0) * ny * nx, nx * sizeof(float),
                               nx * sizeof(float), (size_t)((z1 - z0) * ny), cudaMemcpyDeviceToDevice, st));
    EMF_CUDA(cudaStreamSynchronize(st));  // host vectors above must outlive the async copies
    return EMFUSE_OK;
}

// K^T g for K = Kz Ky Kx (dense float stack, pitch nx):  (K_a^T v)(q) = sum_p w(p-q) v(p)/N(p).
int smooth_transpose(const float* g, float* out, int64_t nx, int64_t ny, int64_t nz,
                     float sigma_xy, float sigma_z, cudaStream_t st) {
    const int Rxy = support_radius(sigma_xy), Rz = support_radius(sigma_z);
    const auto wxy = gaussian_taps(sigma_xy, Rxy);
    const auto wz = gaussian_taps(sigma_z, Rz);
    std::vector<float> host;
    DeviceBuffer norms;
    EMF_TRY(upload_norms(norms, inverse_norms(wxy, (int)nx), inverse_norms(wxy, (int)ny),
                         inverse_norms(wz, (int)nz), st, host));
    const float* inv_x = norms.as<float>();
    const float* inv_y = inv_x + nx;
    const float* inv_z = inv_y + ny;
    DeviceBuffer t1;
    EMF_TRY(t1.alloc((size_t)(nx * ny * nz) * sizeof(float), st));
    EMF_TRY(launch_axis(g, EMFUSE_F32, out, (int)nx, (int)ny, (int)nz, nx, nx, 2, wz, inv_z, nullptr, 0.f, st));
    EMF_TRY(launch_axis(out, EMFUSE_F32, t1.as<float>(), (int)nx, (int)ny, (int)nz, nx, nx, 1, wxy, inv_y, nullptr, 0.f, st));
    EMF_TRY(launch_axis(t1.as<float>(), EMFUSE_F32, out, (int)nx, (int)ny, (int)nz, nx, nx, 0, wxy, inv_x, nullptr, 0.f, st));
    EMF_CUDA(cudaStreamSynchronize(st));
    return EMFUSE_OK;
}

// (dK/dsigma_z) I0 with the support radius fixed at floor(3 sigma_z):
//   Kz' v = (sum w' v) / N - (sum w v) N' / N^2,  w'(d) = w(d) d^2 / sigma^3.
int smooth_dsigma_z(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                    float sigma_xy, float sigma_z, cudaStream_t st) {
    const int Rxy = support_radius(sigma_xy), Rz = support_radius(sigma_z);
    const auto wxy = gaussian_taps(sigma_xy, Rxy);
    const auto wz = gaussian_taps(sigma_z, Rz);
    std::vector<float> dwz(wz.size());
    for (int d = -Rz; d <= Rz; ++d)
        dwz[d + Rz] = sigma_z > 0.f ? (float)((double)wz[d + Rz] * d * d / std::pow((double)sigma_z, 3)) : 0.f;
    const auto ix = inverse_norms(wxy, (int)nx), iy = inverse_norms(wxy, (int)ny), iz = inverse_norms(wz, (int)nz);
    std::vector<float> c1(nz), c2(nz);  // 1/N and -N'/N^2 per plane
    for (int z = 0; z < nz; ++z) {
        double N = 0, dN = 0;
        for (int d = -Rz; d <= Rz; ++d)
            if (z + d >= 0 && z + d < nz) { N += wz[d + Rz]; dN += dwz[d + Rz]; }
        c1[z] = (float)(1.0 / N);
        c2[z] = (float)(-dN / (N * N));
    }
    std::vector<float> host;
    DeviceBuffer norms, cz;
    EMF_TRY(upload_norms(norms, ix, iy, iz, st, host));
    std::vector<float> hc(c1);
    hc.insert(hc.end(), c2.begin(), c2.end());
    EMF_TRY(cz.alloc(hc.size() * sizeof(float), st));
    EMF_CUDA(cudaMemcpyAsync(cz.as<float>(), hc.data(), hc.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    DeviceBuffer t1, t2;
    EMF_TRY(t1.alloc((size_t)(nx * ny * nz) * sizeof(float), st));
    EMF_TRY(t2.alloc((size_t)(nx * ny * nz) * sizeof(float), st));
    const float* inv_x = norms.as<float>();
    const float* inv_y = inv_x + nx;
    EMF_TRY(launch_axis(in, dt, t1.as<float>(), (int)nx, (int)ny, (int)nz, nx, nx, 0, wxy, nullptr, inv_x, 0.f, st));
    EMF_TRY(launch_axis(t1.as<float>(), EMFUSE_F32, t2.as<float>(), (int)nx, (int)ny, (int)nz, nx, nx, 1, wxy, nullptr, inv_y, 0.f, st));
    EMF_TRY(launch_axis(t2.as<float>(), EMFUSE_F32, out, (int)nx, (int)ny, (int)nz, nx, nx, 2, dwz, nullptr, cz.as<float>(), 0.f, st));
    EMF_TRY(launch_axis(t2.as<float>(), EMFUSE_F32, out, (int)nx, (int)ny, (int)nz, nx, nx, 2, wz, nullptr, cz.as<float>() + nz, 1.f, st));
    EMF_CUDA(cudaStreamSynchronize(st));
    return EMFUSE_OK;
}

// ---------------------------------------------------------------- allocation-free variant
// emfuse_smooth_z_noalloc runs smooth_fused_kernel with its only scratch, the three per-axis
// tables of inverse normalisers, in a file-scope device array instead of memory from the CUDA
// allocator.  It exists for callers that cannot allocate device memory while they run: a host
// that has handed all device memory to its own pool or works under a fixed memory budget, and
// code on a latency-critical path where cudaMalloc / cudaFree would synchronise the device.
// Every GPU that loads this library holds the array (kNoAllocMaxNorms floats, 384 KiB) until
// the process exits.
constexpr int64_t kNoAllocMaxNorms = 3 * 32768;  // nx + ny + nz of one call
static __device__ __align__(256) float g_noalloc_norms[kNoAllocMaxNorms];

namespace {

// Fills the table [inv_x | inv_y | inv_z] of the allocation-free variant on the device, from the
// taps passed by value: entry i of an axis of length n is 1 / (sum of the taps w(d), |d| <= R,
// with 0 <= i + d < n), summed in double over d = -R..R and rounded once to float, i.e. the
// values inverse_norms() forms on the host.  (prm.wz holds w(R_z - j); the taps are symmetric,
// so prm.wz[d + R_z] = w(d).)
__global__ void k_noalloc_norms(float* __restrict__ tab, int nx, int ny, int nz, SmoothParams prm) {
    const int total = nx + ny + nz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const bool zax = t >= nx + ny;
        const int i = t < nx ? t : (zax ? t - nx - ny : t - nx);
        const int n = t < nx ? nx : (zax ? nz : ny);
        const int R = zax ? prm.Rz : prm.Rxy;
        double sum = 0.0;
        for (int d = -R; d <= R; ++d)
            if (i + d >= 0 && i + d < n) sum += (double)(zax ? prm.wz[d + R] : prm.wxy[d + R]);
        tab[t] = (float)(1.0 / sum);
    }
}

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_norms on the current device, looked up once per device with
// that device current (in host code the array's name is only a host-side stand-in).
int noalloc_norms(float** out) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("emfuse_smooth_z_noalloc: device ordinal out of range");
        return EMFUSE_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_norms);
        if (e != cudaSuccess || !p) {
            set_error(std::string("emfuse_smooth_z_noalloc: cudaGetSymbolAddress failed: ") +
                      cudaGetErrorString(e));
            return EMFUSE_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return EMFUSE_OK;
}

}  // namespace

}  // namespace emfuse

extern "C" int emfuse_smooth_z_noalloc(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                       int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                                       void* stream) {
    using namespace emfuse;
    set_error("");
    if (!in || !out) {
        set_error("emfuse_smooth_z_noalloc: null pointer");
        return EMFUSE_EINVAL;
    }
    if (dt != EMFUSE_U8 && dt != EMFUSE_F32) {
        set_error("emfuse_smooth_z_noalloc: dtype must be EMFUSE_U8 or EMFUSE_F32");
        return EMFUSE_EINVAL;
    }
    if (nx < 1 || ny < 1 || nz < 1 || pitch < nx || z0 < 0 || z1 > nz || z0 >= z1) {
        set_error("emfuse_smooth_z_noalloc: need sizes >= 1, pitch >= nx and 0 <= z0 < z1 <= nz");
        return EMFUSE_EINVAL;
    }
    if (nx + ny + nz > kNoAllocMaxNorms) {
        set_error("emfuse_smooth_z_noalloc: nx + ny + nz = " + std::to_string(nx + ny + nz) +
                  " exceeds the static scratch of " + std::to_string(kNoAllocMaxNorms) +
                  " entries; use emfuse_smooth_z");
        return EMFUSE_EINVAL;
    }
    if (!std::isfinite(sigma_xy) || !std::isfinite(sigma_z) || sigma_xy < 0.f || sigma_z < 0.f) {
        set_error("emfuse_smooth_z_noalloc: sigma_xy and sigma_z must be finite and >= 0");
        return EMFUSE_EINVAL;
    }
    const int Rxy = support_radius(sigma_xy), Rz = support_radius(sigma_z);
    if (Rxy > kMaxRxy || Rz > 9) {
        set_error("emfuse_smooth_z_noalloc: needs floor(3 sigma_xy) <= 8 and floor(3 sigma_z) <= 9; wider "
                  "supports need temporaries, use emfuse_smooth_z");
        return EMFUSE_EINVAL;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    float* norms = nullptr;
    EMF_TRY(noalloc_norms(&norms));
    const auto wxy = gaussian_taps(sigma_xy, Rxy);
    const auto wz = gaussian_taps(sigma_z, Rz);
    SmoothParams prm{};
    prm.Rxy = Rxy;
    prm.Rz = Rz;
    for (int d = 0; d < 2 * Rxy + 1; ++d) prm.wxy[d] = wxy[d];
    for (int j = 0; j < 2 * Rz + 1; ++j) prm.wz[j] = wz[2 * Rz - j];
    // The normaliser tables are written on the device, stream-ordered before the smoothing
    // kernel, from the taps in `prm` (no host buffer is involved).  Every entry the smoothing
    // kernel reads is rewritten by each call.
    {
        const int total = (int)(nx + ny + nz);
        KernelScope ks("smooth_noalloc_norms", st, 4.0 * total);
        k_noalloc_norms<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(norms, (int)nx, (int)ny, (int)nz, prm);
        EMF_CHECK_LAUNCH();
    }
    const float* inv_x = norms;
    const float* inv_y = inv_x + nx;
    const float* inv_z = inv_y + ny;
    const dim3 grid((unsigned)ceil_div(nx, kTX), (unsigned)ceil_div(ny, kTY));
    const int P = 2 * Rz + 1;
    const int64_t zin0 = std::max<int64_t>(0, z0 - Rz), zin1 = std::min<int64_t>(nz, z1 + Rz);
    KernelScope ks("smooth_noalloc", st,
                   (double)nx * ny * ((zin1 - zin0) * (dt == EMFUSE_U8 ? 1.0 : 4.0) + (z1 - z0) * 4.0));
#define EMF_NOALLOC_LAUNCH(PP)                                                               \
    do {                                                                                     \
        if (dt == EMFUSE_U8)                                                                 \
            smooth_fused_kernel<uint8_t, PP, false><<<grid, kThreads, 0, st>>>(              \
                (const uint8_t*)in, out, (int)nx, (int)ny, (int)nz, pitch, (int)z0, (int)z1, \
                inv_x, inv_y, inv_z, prm);                                                   \
        else                                                                                 \
            smooth_fused_kernel<float, PP, false><<<grid, kThreads, 0, st>>>(                \
                (const float*)in, out, (int)nx, (int)ny, (int)nz, pitch, (int)z0, (int)z1,   \
                inv_x, inv_y, inv_z, prm);                                                   \
    } while (0)
    if (P <= 1) EMF_NOALLOC_LAUNCH(1);
    else if (P <= 7) EMF_NOALLOC_LAUNCH(7);
    else EMF_NOALLOC_LAUNCH(19);
#undef EMF_NOALLOC_LAUNCH
    EMF_CHECK_LAUNCH();
    return EMFUSE_OK;
}
