// extern "C" entry points of libemfuse (declared in include/emfuse.h): argument validation,
// error reporting, and the orchestration of the two phases of the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "emfuse_common.cuh"
#include "emfuse_internal.cuh"

namespace emfuse {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

static int einval(const std::string& msg) {
    set_error(msg);
    return EMFUSE_EINVAL;
}

static int resolve_opts(const emfuse_solve_opts* in, emfuse_solve_opts* out) {
    emfuse_default_opts(out);
    if (in) *out = *in;
    if (!(out->tol >= 0.0)) return einval("opts.tol must be >= 0");
    if (out->max_vcycles < 0) return einval("opts.max_vcycles must be >= 0");
    if (out->nu_pre < 0 || out->nu_post < 0 || out->nu_pre + out->nu_post < 1 || out->nu_pre > 8 || out->nu_post > 8)
        return einval("opts.nu_pre / nu_post must be in [0, 8] with at least one sweep");
    if (out->precision < EMFUSE_PREC_FP32 || out->precision > EMFUSE_PREC_FP64)
        return einval("opts.precision must be EMFUSE_PREC_FP32, _MIXED or _FP64");
    if (out->first_vcycles == 0) out->first_vcycles = 2;
    if (out->first_vcycles < 1 || out->first_vcycles > 8) return einval("opts.first_vcycles must be in [1, 8]");
    const int tr = out->tile_rows;
    if (tr != 0 && (tr < 8 || tr > 256 || (tr & (tr - 1)) != 0))
        return einval("opts.tile_rows must be 0 or a power of two in [8, 256]");
    if (out->autotune != 0 && out->autotune != 1) return einval("opts.autotune must be 0 or 1");
    if (out->no_graphs != 0 && out->no_graphs != 1) return einval("opts.no_graphs must be 0 or 1");
    if (out->host_pipeline < 0 || out->host_pipeline > 2) return einval("opts.host_pipeline must be 0, 1 or 2");
    if (out->verify_residual != 0 && out->verify_residual != 1) return einval("opts.verify_residual must be 0 or 1");
    if (out->async_solve != 0 && out->async_solve != 1) return einval("opts.async_solve must be 0 or 1");
    if (out->host_chunk < 0) return einval("opts.host_chunk must be >= 0");
    if (!(out->robust_kappa == 0.f || (out->robust_kappa >= 1.f && std::isfinite(out->robust_kappa))))
        return einval("opts.robust_kappa must be 0 (plain averaging) or finite and >= 1");
    return EMFUSE_OK;
}

static bool dtype_ok(int dt) { return dt == EMFUSE_U8 || dt == EMFUSE_F32; }
static size_t dtype_size(int dt) { return dt == EMFUSE_U8 ? 1 : 4; }

// Largest supported side: level geometry is computed in 32-bit integers.
constexpr int64_t kMaxSide = (int64_t)1 << 29;

static int check_sigma(float sxy, float sz) {
    if (!(sxy >= 0.f) || !(sz >= 0.f) || !std::isfinite(sxy) || !std::isfinite(sz))
        return einval("sigma_xy and sigma_z must be finite and >= 0");
    if (support_radius(sxy) > 32 || support_radius(sz) > 32)
        return einval("sigma too large: support radius floor(3 sigma) must be <= 32");
    return EMFUSE_OK;
}

static int check_alpha(double alpha) {
    if (!(alpha > 0.0) || !std::isfinite(alpha))
        return einval("alpha must be finite and > 0 (Eq. (1) is singular at alpha = 0 with Neumann boundaries)");
    return EMFUSE_OK;
}

// Solve every slice of a dense stack (nz slices of ny x nx).
static int solve_stack(const float* s, const void* o, int dt, float* out, int64_t nx, int64_t ny,
                       int64_t nz, double alpha, const emfuse_solve_opts& opts,
                       emfuse_slice_stats* stats, const float* rhs, cudaStream_t st) {
    std::vector<int64_t> vx(nz, nx), vy(nz, ny), off(nz);
    for (int64_t j = 0; j < nz; ++j) off[j] = j * nx * ny;
    SolveRequest req;
    req.s = s;
    req.o = o;
    req.o_dtype = dt;
    req.rhs = rhs;
    req.out = out;
    req.nslices = nz;
    req.nx = vx.data();
    req.ny = vy.data();
    req.offsets = off.data();
    req.alpha = alpha;
    req.opts = opts;
    req.stats = stats;
    return solve_batch(req, st);
}


// Host-resident stack whose input and smoothed copy fit on the device together with the
// solvers' chunk workspaces.  Everything is queued without waiting on the host, and the call
// synchronises once at the end:
//   copy-in  (side stream): the input in pieces, piece k ending at the last plane smoothing
//            chunk k reads, each with an event;
//   compute  (the caller's stream): smoothing of a chunk of C slices once its input has
//            arrived (the first chunk's input is small, so compute starts early; on a stack so
//            short that it is half the stack already, the whole stack in one launch), and the
//            chunk's solve,
//            queued asynchronously (the solve's outer loop runs on the device, so the host never
//            waits between chunks), into an output buffer of a ring of four;
//   copy-out (side stream): each chunk's output to the host as soon as its solve is done.
// A slice's result does not depend on the batch it is solved in, so the output equals the
// device path's bit for bit.  The per-slice stats of the chunks give the outcome.
// Copy streams and events of the host-buffer pipeline, kept per host thread and device for the
// life of the process (creating and destroying streams on every call costs the driver
// occasional stalls of tens of milliseconds).  Every event is complete when a call returns.
struct PipeResources {
    int dev = -1;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> events;
    size_t next = 0;
};
static thread_local PipeResources* t_pipe = nullptr;

static int pipe_resources(PipeResources** out) {
    int dev = 0;
    EMF_CUDA(cudaGetDevice(&dev));
    if (!t_pipe) t_pipe = new PipeResources();
    if (t_pipe->dev != dev) {  // first use on this thread, or another device: fresh resources
        t_pipe = new PipeResources();  // the old device's streams stay valid for that device
        EMF_CUDA(cudaStreamCreateWithFlags(&t_pipe->s_in, cudaStreamNonBlocking));
        EMF_CUDA(cudaStreamCreateWithFlags(&t_pipe->s_out, cudaStreamNonBlocking));
        t_pipe->dev = dev;
    }
    t_pipe->next = 0;
    *out = t_pipe;
    return EMFUSE_OK;
}

static int pipe_event(PipeResources* r, cudaEvent_t* e) {
    if (r->next == r->events.size()) {
        cudaEvent_t x = nullptr;
        EMF_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        r->events.push_back(x);
    }
    *e = r->events[r->next++];
    return EMFUSE_OK;
}

static int correct_stack_resident(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                  float sigma_xy, float sigma_z, double alpha, const emfuse_solve_opts& o2,
                                  emfuse_slice_stats* stats, cudaStream_t st, int64_t C) {
    const int64_t R = support_radius(sigma_z);
    const int64_t plane = nx * ny;
    const size_t esz = dtype_size(dt);
    const int64_t nchunks = (nz + C - 1) / C;            // solve chunks
    // smoothing chunks: one per solve chunk, unless the first chunk's input (its planes and R
    // more) is already half the stack; then one launch smooths the whole stack, instead of
    // each chunk marching through R halo planes on either side again
    const int64_t Cs = C + R >= (nz + 1) / 2 ? nchunks * C : C;
    const int64_t ns = (nz + Cs - 1) / Cs;
    constexpr int kRing = 4;                             // chunk output buffers
    const int nbuf = (int)std::min<int64_t>(kRing, nchunks);
    emfuse_solve_opts o3 = o2;
    o3.async_solve = 1;  // queued; the outcome is read from the stats after the final synchronisation
    std::vector<emfuse_slice_stats> hst((size_t)nz);
    DeviceBuffer din, ds, dout[kRing];
    EMF_TRY(din.alloc((size_t)(nz * plane) * esz, st));
    EMF_TRY(ds.alloc((size_t)(nz * plane) * sizeof(float), st));
    for (int q = 0; q < nbuf; ++q) EMF_TRY(dout[q].alloc((size_t)(C * plane) * sizeof(float), st));
    PipeResources* pr = nullptr;
    EMF_TRY(pipe_resources(&pr));
    cudaStream_t s_in = pr->s_in, s_out = pr->s_out;
    cudaEvent_t ev_alloc = nullptr, ev_outq = nullptr;
    std::vector<cudaEvent_t> ev_piece(ns, nullptr), ev_smooth(ns, nullptr), ev_comp(nchunks, nullptr),
        ev_free(kRing, nullptr);
    auto cleanup = [&]() {};  // streams and events are kept for the next call
    auto ev = [&](cudaEvent_t& e) -> int { return pipe_event(pr, &e); };
    auto body = [&]() -> int {
        EMF_TRY(ev(ev_alloc));
        EMF_TRY(ev(ev_outq));
        for (auto* v : {&ev_piece, &ev_smooth, &ev_comp, &ev_free})
            for (auto& e : *v) EMF_TRY(ev(e));
        // the buffers come from the caller's stream's pool: valid for the other streams after this
        EMF_CUDA(cudaEventRecord(ev_alloc, st));
        for (cudaStream_t x : {s_in, s_out}) EMF_CUDA(cudaStreamWaitEvent(x, ev_alloc, 0));
        for (int64_t k = 0, have = 0; k < ns; ++k) {
            const int64_t need = std::min(nz, std::min(nz, (k + 1) * Cs) + R);  // planes [0, need) read
            if (need > have)
                EMF_CUDA(cudaMemcpyAsync(din.as<char>() + (size_t)(have * plane) * esz,
                                         (const char*)in + (size_t)(have * plane) * esz,
                                         (size_t)((need - have) * plane) * esz, cudaMemcpyHostToDevice, s_in));
            have = std::max(have, need);
            EMF_CUDA(cudaEventRecord(ev_piece[k], s_in));
        }
        std::vector<char> smoothed(ns, 0);
        for (int64_t i = 0; i < nchunks; ++i) {
            const cudaStream_t c = st;
            const int q = int(i % nbuf);
            const int64_t z0 = i * C, z1 = std::min(nz, z0 + C);
            const int64_t k = z0 / Cs;  // chunk boundaries are multiples of C, and Cs of C
            if (!smoothed[k]) {
                const int64_t a = k * Cs, b = std::min(nz, a + Cs);
                EMF_CUDA(cudaStreamWaitEvent(c, ev_piece[k], 0));  // input planes [0, b + R) arrived
                EMF_TRY(smooth_stack(din.as<char>(), dt, ds.as<float>() + a * plane, nx, ny, nz, nx, a, b, sigma_xy,
                                     sigma_z, c, 0, o2.robust_kappa));
                EMF_CUDA(cudaEventRecord(ev_smooth[k], c));
                smoothed[k] = 1;
            } else {
                EMF_CUDA(cudaStreamWaitEvent(c, ev_smooth[k], 0));
            }
            if (i >= nbuf) EMF_CUDA(cudaStreamWaitEvent(c, ev_free[q], 0));  // dout[q] drained
            const int rc = solve_stack(ds.as<float>() + z0 * plane, din.as<char>() + (size_t)(z0 * plane) * esz, dt,
                                       dout[q].as<float>(), nx, ny, z1 - z0, alpha, o3, hst.data() + z0, nullptr, c);
            if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) return rc;
            EMF_CUDA(cudaEventRecord(ev_comp[i], c));
            EMF_CUDA(cudaStreamWaitEvent(s_out, ev_comp[i], 0));
            EMF_CUDA(cudaMemcpyAsync(out + z0 * plane, dout[q].as<float>(), (size_t)((z1 - z0) * plane) * sizeof(float),
                                     cudaMemcpyDeviceToHost, s_out));
            EMF_CUDA(cudaEventRecord(ev_free[q], s_out));
        }
        // the caller's stream waits for the copy streams (the buffers go back to its pool)
        EMF_CUDA(cudaEventRecord(ev_outq, s_out));
        EMF_CUDA(cudaStreamWaitEvent(st, ev_outq, 0));
        EMF_CUDA(cudaStreamWaitEvent(st, ev_piece[ns - 1], 0));
        return EMFUSE_OK;
    };
    int rc = body();
    // wait for everything queued (also after a failure part-way, before the buffers are released);
    // on success the caller's stream already waits for both copy streams, and the host thread
    // sleeps on a blocking-sync event instead of spinning for the whole pipeline
    cudaError_t e = cudaSuccess;
    if (rc == EMFUSE_OK) {
        cudaEvent_t done = nullptr;
        e = cudaEventCreateWithFlags(&done, cudaEventBlockingSync | cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(done, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(done);
        if (done) cudaEventDestroy(done);
    }
    if (s_in) cudaStreamSynchronize(s_in);
    if (s_out) cudaStreamSynchronize(s_out);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    cleanup();
    if (rc != EMFUSE_OK) return rc;
    if (e != cudaSuccess) {
        set_error(std::string("emfuse_correct_stack: ") + cudaGetErrorString(e));
        return EMFUSE_ECUDA;
    }
    EMF_TRY(solve_async_status(st, o2.precision));
    if (stats) std::memcpy(stats, hst.data(), hst.size() * sizeof(emfuse_slice_stats));
    bool nonfinite = false, converged = true;
    for (const auto& x : hst) {
        nonfinite |= !std::isfinite(x.rel_residual);
        converged &= x.converged != 0;
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

// Host-resident stack, streamed through the device in z-chunks of C output slices.  Chunk i
// needs input planes [a_i, b_i) = [z0 - R, z1 + R) clipped to the stack (R = floor(3 sigma_z)),
// so that smoothing the slab alone gives exactly the stack's slices.  Three streams overlap:
//   copy-in  (side stream): the planes chunk i shares with chunk i - 1 device to device from
//            the previous slab, the new planes from the host, into slab buffer i mod 2;
//   compute  (the caller's stream): smoothing and the batched solve of chunk i into output
//            buffer i mod 2 (the solve's host-side convergence checks block this thread, so
//            the copy of slab i + 1 is queued before it starts);
//   copy-out (side stream): output buffer i mod 2 to the host.
// Events order the reuse of the two slab and two output buffers.
static int correct_stack_host(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                              float sigma_xy, float sigma_z, double alpha, const emfuse_solve_opts& o2,
                              emfuse_slice_stats* stats, cudaStream_t st) {
    const int64_t R = support_radius(sigma_z);
    const int64_t plane = nx * ny;
    const size_t esz = dtype_size(dt);
    size_t free_b = 0, total_b = 0;
    EMF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    // memory this library already holds counts as available: idle pages of its pool, and the
    // buffers of this stream's cached solver plan, which the chunk solves reuse
    free_b += library_pool_idle_bytes() + cached_plan_bytes(st, o2.precision);
    // device bytes per output slice of a chunk: two slabs of input, s, two output buffers, and
    // the solver's pyramids (about 16 B/px) and FP64 iterates (16 B/px)
    const double per_slice = (double)plane * (2.0 * esz + 4.0 + 8.0 + 32.0);
    const double halo = (double)plane * 2.0 * esz * 2.0 * (double)R;
    int64_t cmax = (int64_t)std::floor((0.7 * (double)free_b - halo) / per_slice);
    if (cmax < 1) {
        set_error("emfuse_correct_stack: not enough free device memory for one slice of " +
                  std::to_string(ny) + " x " + std::to_string(nx) + " plus halo planes");
        return EMFUSE_ENOMEM;
    }
    // at least two chunks when the stack allows it, so that copies overlap compute (every extra
    // chunk costs a solve's fixed, latency-bound coarse-level time, so no more than needed);
    // equal chunk sizes (but the last) keep the solver's cached plan valid from chunk to chunk
    cmax = std::min<int64_t>({cmax, 64, std::max<int64_t>(1, (nz + 1) / 2)});
    if (o2.host_chunk > 0) cmax = std::min<int64_t>(cmax, o2.host_chunk);
    const int64_t nchunks = (nz + cmax - 1) / cmax;
    const int64_t C = (nz + nchunks - 1) / nchunks;
    // the resident schedule: the whole input and its smoothed copy on the device, chunks of Cr
    // slices (four chunks unless opts.host_chunk says otherwise), the solver plan (about 48 B per
    // pixel: pyramids and FP64 iterates) and a ring of four chunk output buffers
    const int64_t Cr = std::min<int64_t>(nz, o2.host_chunk > 0 ? o2.host_chunk : std::max<int64_t>(1, (nz + 3) / 4));
    const double resident = (double)(nz * plane) * (esz + 4.0) + (double)(Cr * plane) * (4.0 * 4.0 + 48.0);
    const bool fits = resident <= 0.7 * (double)free_b;
    if (o2.host_pipeline == 2 && !fits) {
        set_error("emfuse_correct_stack: the whole input and its smoothed copy do not fit on the device");
        return EMFUSE_ENOMEM;
    }
    if (o2.host_pipeline == 2 || (o2.host_pipeline == 0 && fits))
        return correct_stack_resident(in, dt, out, nx, ny, nz, sigma_xy, sigma_z, alpha, o2, stats, st, Cr);
    const int64_t slab_cap = std::min<int64_t>(nz, C + 2 * R);

    DeviceBuffer din[2], dout[2], ds;
    for (int q = 0; q < 2; ++q) {
        EMF_TRY(din[q].alloc((size_t)(slab_cap * plane) * esz, st));
        EMF_TRY(dout[q].alloc((size_t)(C * plane) * sizeof(float), st));
    }
    EMF_TRY(ds.alloc((size_t)(C * plane) * sizeof(float), st));
    // the buffers come from the caller's stream's pool: make them valid for the side streams
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_alloc = nullptr, ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr};
    int rc_all = EMFUSE_OK;
    auto cleanup = [&]() {
        for (int q = 0; q < 2; ++q) {
            if (ev_in[q]) cudaEventDestroy(ev_in[q]);
            if (ev_comp[q]) cudaEventDestroy(ev_comp[q]);
            if (ev_out[q]) cudaEventDestroy(ev_out[q]);
        }
        if (ev_alloc) cudaEventDestroy(ev_alloc);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_out) cudaStreamDestroy(s_out);
    };
    auto body = [&]() -> int {
        EMF_CUDA(cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking));
        EMF_CUDA(cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking));
        EMF_CUDA(cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming));
        for (int q = 0; q < 2; ++q) {
            EMF_CUDA(cudaEventCreateWithFlags(&ev_in[q], cudaEventDisableTiming));
            EMF_CUDA(cudaEventCreateWithFlags(&ev_comp[q], cudaEventDisableTiming));
            EMF_CUDA(cudaEventCreateWithFlags(&ev_out[q], cudaEventDisableTiming));
        }
        EMF_CUDA(cudaEventRecord(ev_alloc, st));
        EMF_CUDA(cudaStreamWaitEvent(s_in, ev_alloc, 0));
        EMF_CUDA(cudaStreamWaitEvent(s_out, ev_alloc, 0));
        auto slab = [&](int64_t i, int64_t& a, int64_t& b, int64_t& z0, int64_t& z1) {
            z0 = i * C;
            z1 = std::min(nz, z0 + C);
            a = std::max<int64_t>(0, z0 - R);
            b = std::min<int64_t>(nz, z1 + R);
        };
        // queue the copy of slab i into din[i & 1]
        auto copy_in = [&](int64_t i) -> int {
            const int q = int(i & 1);
            int64_t a, b, z0, z1;
            slab(i, a, b, z0, z1);
            if (i >= 2) EMF_CUDA(cudaStreamWaitEvent(s_in, ev_comp[q], 0));  // chunk i-2 done with it
            int64_t have = a;  // planes [a, have) come from the previous slab
            if (i >= 1) {
                int64_t pa, pb, pz0, pz1;
                slab(i - 1, pa, pb, pz0, pz1);
                if (pb > a) {
                    EMF_CUDA(cudaMemcpyAsync(din[q].as<char>(), din[q ^ 1].as<char>() + (size_t)((a - pa) * plane) * esz,
                                             (size_t)((pb - a) * plane) * esz, cudaMemcpyDeviceToDevice, s_in));
                    have = pb;
                }
            }
            if (b > have)
                EMF_CUDA(cudaMemcpyAsync(din[q].as<char>() + (size_t)((have - a) * plane) * esz,
                                         (const char*)in + (size_t)(have * plane) * esz,
                                         (size_t)((b - have) * plane) * esz, cudaMemcpyHostToDevice, s_in));
            EMF_CUDA(cudaEventRecord(ev_in[q], s_in));
            return EMFUSE_OK;
        };
        EMF_TRY(copy_in(0));
        for (int64_t i = 0; i < nchunks; ++i) {
            const int q = int(i & 1);
            int64_t a, b, z0, z1;
            slab(i, a, b, z0, z1);
            if (i + 1 < nchunks) EMF_TRY(copy_in(i + 1));
            EMF_CUDA(cudaStreamWaitEvent(st, ev_in[q], 0));
            if (i >= 2) EMF_CUDA(cudaStreamWaitEvent(st, ev_out[q], 0));  // dout[q] drained
            EMF_TRY(smooth_stack(din[q].as<char>(), dt, ds.as<float>(), nx, ny, b - a, nx, z0 - a, z1 - a,
                                 sigma_xy, sigma_z, st, 0, o2.robust_kappa));
            const char* o_chunk = din[q].as<char>() + (size_t)((z0 - a) * plane) * esz;
            const int rc = solve_stack(ds.as<float>(), o_chunk, dt, dout[q].as<float>(), nx, ny, z1 - z0, alpha,
                                       o2, stats ? stats + z0 : nullptr, nullptr, st);
            if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) return rc;
            if (rc == EMFUSE_ENOCONV) rc_all = rc;
            EMF_CUDA(cudaEventRecord(ev_comp[q], st));
            EMF_CUDA(cudaStreamWaitEvent(s_out, ev_comp[q], 0));
            EMF_CUDA(cudaMemcpyAsync(out + z0 * plane, dout[q].as<float>(), (size_t)((z1 - z0) * plane) * sizeof(float),
                                     cudaMemcpyDeviceToHost, s_out));
            EMF_CUDA(cudaEventRecord(ev_out[q], s_out));
        }
        // the buffers go back to the caller's stream's pool after the side streams are done
        for (int q = 0; q < 2; ++q) {
            EMF_CUDA(cudaStreamWaitEvent(st, ev_out[q], 0));
            EMF_CUDA(cudaStreamWaitEvent(st, ev_in[q], 0));
        }
        return EMFUSE_OK;
    };
    int rc = body();
    if (rc != EMFUSE_OK) {
        // a failure part-way: let queued copies finish before the buffers are released
        if (s_in) cudaStreamSynchronize(s_in);
        if (s_out) cudaStreamSynchronize(s_out);
        cudaStreamSynchronize(st);
        cleanup();
        return rc;
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) {
        set_error(std::string("emfuse_correct_stack: ") + cudaGetErrorString(e));
        return EMFUSE_ECUDA;
    }
    return rc_all;
}

}  // namespace emfuse

using namespace emfuse;

extern "C" {

void emfuse_default_opts(emfuse_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_vcycles = 40;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->precision = EMFUSE_PREC_MIXED;
    o->fused = 1;
    o->first_vcycles = 2;
}

const char* emfuse_last_error(void) { return last_error(); }

int emfuse_autotune_result(emfuse_tune_entry* out, int max_entries) {
    const auto& v = last_autotune();
    for (int i = 0; out && i < max_entries && i < (int)v.size(); ++i) out[i] = v[i];
    return (int)v.size();
}

void emfuse_release_cache(void) {
    cudaDeviceSynchronize();
    release_plans();
    release_fft_plans();
    trim_library_pools();
}

const char* emfuse_version(void) { return "emfuse 0.1 (sm_103a)"; }

int emfuse_smooth_z(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                    int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                    void* stream) {
    set_error("");
    if (!in || !out) return einval("emfuse_smooth_z: null pointer");
    if (!dtype_ok(dt)) return einval("emfuse_smooth_z: dtype must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_smooth_z: sizes must be in [1, 2^29]");
    if (pitch < nx) return einval("emfuse_smooth_z: pitch must be >= nx");
    if (z0 < 0 || z1 > nz || z0 >= z1) return einval("emfuse_smooth_z: need 0 <= z0 < z1 <= nz");
    EMF_TRY(check_sigma(sigma_xy, sigma_z));
    return smooth_stack(in, dt, out, nx, ny, nz, pitch, z0, z1, sigma_xy, sigma_z,
                        (cudaStream_t)stream, 0);
}

int emfuse_smooth_z_robust(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                           int64_t pitch, int64_t z0, int64_t z1, float sigma_xy, float sigma_z,
                           float kappa, void* stream) {
    set_error("");
    if (!in || !out) return einval("emfuse_smooth_z_robust: null pointer");
    if (!dtype_ok(dt)) return einval("emfuse_smooth_z_robust: dtype must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_smooth_z_robust: sizes must be in [1, 2^29]");
    if (pitch < nx) return einval("emfuse_smooth_z_robust: pitch must be >= nx");
    if (z0 < 0 || z1 > nz || z0 >= z1) return einval("emfuse_smooth_z_robust: need 0 <= z0 < z1 <= nz");
    if (!(kappa >= 1.f) || !std::isfinite(kappa)) return einval("emfuse_smooth_z_robust: kappa must be finite and >= 1");
    EMF_TRY(check_sigma(sigma_xy, sigma_z));
    return smooth_stack(in, dt, out, nx, ny, nz, pitch, z0, z1, sigma_xy, sigma_z, (cudaStream_t)stream, 0,
                        kappa);
}

int emfuse_screened_poisson(const float* s, const float* o, float* f, int64_t nslices,
                            const int64_t* nx, const int64_t* ny, const int64_t* offsets,
                            double alpha, const emfuse_solve_opts* opts,
                            emfuse_slice_stats* stats, void* stream) {
    set_error("");
    if (!s || !o || !f || !nx || !ny || !offsets) return einval("emfuse_screened_poisson: null pointer");
    if (nslices < 1) return einval("emfuse_screened_poisson: nslices must be >= 1");
    if (f == s || f == o) return einval("emfuse_screened_poisson: f must not alias s or o");
    for (int64_t j = 0; j < nslices; ++j) {
        if (nx[j] < 1 || ny[j] < 1 || nx[j] > kMaxSide || ny[j] > kMaxSide)
            return einval("emfuse_screened_poisson: slice sizes must be in [1, 2^29]");
        if (offsets[j] < 0) return einval("emfuse_screened_poisson: negative offset");
    }
    EMF_TRY(check_alpha(alpha));
    emfuse_solve_opts o2;
    EMF_TRY(resolve_opts(opts, &o2));
    SolveRequest req;
    req.s = s;
    req.o = o;
    req.o_dtype = EMFUSE_F32;
    req.out = f;
    req.nslices = nslices;
    req.nx = nx;
    req.ny = ny;
    req.offsets = offsets;
    req.alpha = alpha;
    req.opts = o2;
    req.stats = stats;
    return solve_batch(req, (cudaStream_t)stream);
}

int emfuse_screened_poisson_dct(const float* s, const float* o, float* f, int64_t nslices, int64_t nx,
                                int64_t ny, double alpha, int precision, void* stream) {
    set_error("");
    if (!s || !o || !f) return einval("emfuse_screened_poisson_dct: null pointer");
    if (nslices < 1 || nx < 1 || ny < 1 || nx > kMaxSide || ny > kMaxSide)
        return einval("emfuse_screened_poisson_dct: need nslices >= 1 and sizes in [1, 2^29]");
    if (f == s || f == o) return einval("emfuse_screened_poisson_dct: f must not alias s or o");
    if (precision != EMFUSE_PREC_FP32 && precision != EMFUSE_PREC_FP64)
        return einval("emfuse_screened_poisson_dct: precision must be EMFUSE_PREC_FP32 or EMFUSE_PREC_FP64");
    EMF_TRY(check_alpha(alpha));
    return solve_dct_batch(s, o, f, nslices, nx, ny, alpha, precision, (cudaStream_t)stream);
}

int emfuse_smooth_gradient_domain(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                  double alpha, int precision, void* stream) {
    set_error("");
    if (!in || !out) return einval("emfuse_smooth_gradient_domain: null pointer");
    if (dt != EMFUSE_U8 && dt != EMFUSE_F32) return einval("emfuse_smooth_gradient_domain: dt must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_smooth_gradient_domain: need sizes in [1, 2^29]");
    if ((double)nx * (double)ny * (double)nz > 1099511627776.0)
        return einval("emfuse_smooth_gradient_domain: more than 2^40 cells");
    if ((const void*)out == in) return einval("emfuse_smooth_gradient_domain: out must not alias in");
    if (precision != EMFUSE_PREC_FP32 && precision != EMFUSE_PREC_FP64)
        return einval("emfuse_smooth_gradient_domain: precision must be EMFUSE_PREC_FP32 or EMFUSE_PREC_FP64");
    EMF_TRY(check_alpha(alpha));
    return smooth_gradient_domain(in, dt, out, nx, ny, nz, alpha, precision, (cudaStream_t)stream);
}

int emfuse_smooth_gradient_domain_mg(const void* in, int dt, float* out, int64_t nx, int64_t ny, int64_t nz,
                                     double alpha, const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                                     void* stream) {
    set_error("");
    if (!in || !out) return einval("emfuse_smooth_gradient_domain_mg: null pointer");
    if (dt != EMFUSE_U8 && dt != EMFUSE_F32)
        return einval("emfuse_smooth_gradient_domain_mg: dt must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_smooth_gradient_domain_mg: need sizes in [1, 2^29]");
    if ((double)nx * (double)ny * (double)nz > 1099511627776.0)
        return einval("emfuse_smooth_gradient_domain_mg: more than 2^40 cells");
    if ((const void*)out == in) return einval("emfuse_smooth_gradient_domain_mg: out must not alias in");
    EMF_TRY(check_alpha(alpha));
    emfuse_solve_opts o2;
    EMF_TRY(resolve_opts(opts, &o2));
    return gd_multigrid(in, dt, out, nx, ny, nz, alpha, o2, stats, (cudaStream_t)stream);
}

int emfuse_fuse_color(const float* s_rgb, const float* o_grey, float* f_rgb, int64_t nimages, int64_t nx,
                      int64_t ny, double alpha, const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                      void* stream) {
    set_error("");
    if (!s_rgb || !o_grey || !f_rgb) return einval("emfuse_fuse_color: null pointer");
    if (nimages < 1 || nx < 1 || ny < 1 || nx > kMaxSide || ny > kMaxSide)
        return einval("emfuse_fuse_color: need nimages >= 1 and sizes in [1, 2^29]");
    if (f_rgb == s_rgb) return einval("emfuse_fuse_color: f_rgb must not alias s_rgb");
    EMF_TRY(check_alpha(alpha));
    emfuse_solve_opts o2;
    EMF_TRY(resolve_opts(opts, &o2));
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t plane = nx * ny, n = 3 * nimages;
    // the grey image is the gradient constraint of every channel: one copy per channel
    DeviceBuffer o3;
    EMF_TRY(o3.alloc((size_t)(n * plane) * sizeof(float), st));
    for (int64_t i = 0; i < nimages; ++i)
        for (int c = 0; c < 3; ++c)
            EMF_CUDA(cudaMemcpyAsync(o3.as<float>() + (3 * i + c) * plane, o_grey + i * plane,
                                     (size_t)plane * sizeof(float), cudaMemcpyDeviceToDevice, st));
    std::vector<int64_t> vx(n, nx), vy(n, ny), off(n);
    for (int64_t j = 0; j < n; ++j) off[j] = j * plane;
    SolveRequest req;
    req.s = s_rgb;
    req.o = o3.as<float>();
    req.o_dtype = EMFUSE_F32;
    req.out = f_rgb;
    req.nslices = n;
    req.nx = vx.data();
    req.ny = vy.data();
    req.offsets = off.data();
    req.alpha = alpha;
    req.opts = o2;
    req.stats = stats;
    return solve_batch(req, st);
}

int emfuse_correct_stack(const void* in, int dt, int in_is_host, float* out, int64_t nx,
                         int64_t ny, int64_t nz, float sigma_xy, float sigma_z, double alpha,
                         const emfuse_solve_opts* opts, emfuse_slice_stats* stats,
                         void* stream) {
    set_error("");
    if (!in || !out) return einval("emfuse_correct_stack: null pointer");
    if (!dtype_ok(dt)) return einval("emfuse_correct_stack: dtype must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_correct_stack: sizes must be in [1, 2^29]");
    EMF_TRY(check_sigma(sigma_xy, sigma_z));
    EMF_TRY(check_alpha(alpha));
    emfuse_solve_opts o2;
    EMF_TRY(resolve_opts(opts, &o2));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t plane = nx * ny;
    if (!in_is_host) {
        DeviceBuffer sbuf;
        EMF_TRY(sbuf.alloc((size_t)(plane * nz) * sizeof(float), st));
        EMF_TRY(smooth_stack(in, dt, sbuf.as<float>(), nx, ny, nz, nx, 0, nz, sigma_xy, sigma_z, st, 0,
                             o2.robust_kappa));
        return solve_stack(sbuf.as<float>(), in, dt, out, nx, ny, nz, alpha, o2, stats, nullptr, st);
    }
    o2.async_solve = 0;  // host buffers: the call returns when out is written
    return correct_stack_host(in, dt, out, nx, ny, nz, sigma_xy, sigma_z, alpha, o2, stats, st);
}

int emfuse_backward(const float* grad_f, const float* f, const float* s, const void* o, int dt,
                    int64_t nx, int64_t ny, int64_t nz, float sigma_xy, float sigma_z,
                    double alpha, float* grad_s, float* grad_o, float* grad_in0,
                    double* grad_alpha, double* grad_sigma_z, const emfuse_solve_opts* opts,
                    void* stream) {
    set_error("");
    if (!grad_f) return einval("emfuse_backward: grad_f is null");
    if (!dtype_ok(dt)) return einval("emfuse_backward: dtype must be EMFUSE_U8 or EMFUSE_F32");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxSide || ny > kMaxSide || nz > kMaxSide)
        return einval("emfuse_backward: sizes must be in [1, 2^29]");
    if (grad_alpha && (!f || !s)) return einval("emfuse_backward: grad_alpha needs f and s");
    if (grad_sigma_z && !o) return einval("emfuse_backward: grad_sigma_z needs o (I0)");
    EMF_TRY(check_alpha(alpha));
    EMF_TRY(check_sigma(sigma_xy, sigma_z));
    emfuse_solve_opts o2;
    EMF_TRY(resolve_opts(opts, &o2));
    o2.async_solve = 0;  // the gradients below need the solve's outcome
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = nx * ny * nz;
    DeviceBuffer lam;
    EMF_TRY(lam.alloc((size_t)n * sizeof(float), st));
    // lam = A^{-1} grad_f (A symmetric)
    int rc = solve_stack(nullptr, nullptr, EMFUSE_F32, lam.as<float>(), nx, ny, nz, alpha, o2,
                         nullptr, grad_f, st);
    if (rc != EMFUSE_OK && rc != EMFUSE_ENOCONV) return rc;
    DeviceBuffer tmp_s;
    float* gs = grad_s;
    if (!gs && (grad_in0 || grad_sigma_z)) {
        EMF_TRY(tmp_s.alloc((size_t)n * sizeof(float), st));
        gs = tmp_s.as<float>();
    }
    if (gs) EMF_TRY(scale_copy(lam.as<float>(), gs, n, (float)alpha, st));
    if (grad_o) EMF_TRY(apply_laplacian_stack(lam.as<float>(), grad_o, nx, ny, nz, 1.f, st));
    if (grad_alpha) EMF_TRY(dot_diff(lam.as<float>(), s, f, n, grad_alpha, st));
    if (grad_in0) {
        // dl/dI0 = L lam + K^T (alpha lam)
        EMF_TRY(smooth_transpose(gs, grad_in0, nx, ny, nz, sigma_xy, sigma_z, st));
        DeviceBuffer lap;
        EMF_TRY(lap.alloc((size_t)n * sizeof(float), st));
        EMF_TRY(apply_laplacian_stack(lam.as<float>(), lap.as<float>(), nx, ny, nz, 1.f, st));
        EMF_TRY(axpy(lap.as<float>(), grad_in0, n, 1.f, st));
    }
    if (grad_sigma_z) {
        DeviceBuffer dk;
        EMF_TRY(dk.alloc((size_t)n * sizeof(float), st));
        EMF_TRY(smooth_dsigma_z(o, dt, dk.as<float>(), nx, ny, nz, sigma_xy, sigma_z, st));
        EMF_TRY(dot_diff(gs, dk.as<float>(), nullptr, n, grad_sigma_z, st));
    }
    EMF_CUDA(cudaStreamSynchronize(st));
    return rc;
}

}  // extern "C"
