// Context API of libjac: one grid resident in device memory.  jac_upload is
// the hoisted copy-in, jac_sweep runs every sweep on the resident arrays,
// jac_download is the hoisted copy-out -- the transfer structure the paper
// builds its offloading on (Sections 3.2-3.3: transfer nested-loop variables
// once, outside the outermost loop, batch the copies and mark data already
// present on the device).
//
// Two ownership models.  jac_create allocates the field storage and every
// scratch array itself (cudaMalloc).  jac_create_borrowed takes the fourteen
// storage arrays and one workspace from the caller (for example torch
// tensors) and allocates no device memory at all: staging, sweep scratch and
// the checkpoint tape are carved out of the workspace, whose size
// jac_workspace_size reports.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "jac_common.cuh"
#include "jac_internal.h"

struct jac_ctx {
    int I = 0, J = 0, K = 0, pitch = 0;
    jac_prec prec = JAC_F32;
    double omega = 0.0;
    cudaStream_t stream = nullptr;
    void *arena = nullptr;            // field storage: both states and 12 arrays
    void *arr[JAC_NFIELDS] = {};      // arr[JAC_A0..JAC_BND]; arr[JAC_P] unused
    void *pbuf[2] = {nullptr, nullptr};
    int cur = 0;                      // which pbuf holds the current state
    double *staging = nullptr;        // I*J*K doubles
    double *stage_all = nullptr;      // JAC_NFIELDS*I*J*K doubles, jac_upload_async only (first use)
    void *ws = nullptr;               // sweep workspace
    size_t ws_bytes = 0;
    jac_plan plan{0, 0, 0, 0};
    long long count = 0;
    bool uploaded = false;
    bool has_res = false;
    unsigned long long stall_ns = 0;  // jac_inject_stall: the next sweep launch's wait limit
    // borrowed contexts: caller memory, carved by ws_carve()
    bool borrowed = false;
    char *tape_region = nullptr;      // room for tape_cap state arrays plus 256 bytes
    int tape_cap = 0;
    std::string err;
    // checkpoint tape of the sweeps since jac_tape_begin
    struct Tape {
        int C = 0, max_sweeps = 0, taped = 0;
        void *mem = nullptr;      // checkpoints, segment states 1..C-1, two lambda buffers, one double
        size_t state_bytes = 0;
        int n_ckpt = 0;
        char *ckpt(int s) const { return static_cast<char *>(mem) + (size_t)s * state_bytes; }
        // state m (1 <= m < C) of a segment; state 0 is the segment's checkpoint
        char *seg(int m) const { return ckpt(n_ckpt) + (size_t)(m - 1) * state_bytes; }
        char *lam(int b) const { return seg(C) + (size_t)b * state_bytes; }
        double *scratch() const { return reinterpret_cast<double *>(lam(2)); }
    } tape;
};

namespace {

jac_status ctx_fail(jac_ctx *c, jac_status s, const std::string &m)
{
    if (c) c->err = m;
    jac::set_thread_error(m);
    return s;
}

jac_status ctx_from_thread(jac_ctx *c, jac_status s)
{
    if (s != JAC_OK && c) c->err = jac::thread_last_error();
    return s;
}

jac_status ctx_cuda(jac_ctx *c, cudaError_t e, const char *what)
{
    return ctx_fail(c, JAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Bytes of data in storage array `which` (what a borrowed buffer holds).
size_t data_bytes(const jac_ctx *c, int which)
{
    return (size_t)c->pitch * c->J * c->K * jac::elem_bytes(c->prec, which);
}

// The same rounded up to 256 bytes: the spacing of arrays inside the
// context's own memory (arena, tape).
size_t array_bytes(const jac_ctx *c, int which)
{
    return jac::round_up((size_t)c->pitch * c->J * c->K * jac::elem_bytes(c->prec, which), 256);
}

jac_grid make_grid(const jac_ctx *c)
{
    jac_grid g;
    std::memset(&g, 0, sizeof(g));
    g.I = c->I; g.J = c->J; g.K = c->K;
    g.prec = c->prec;
    g.omega = c->omega;
    g.p[0] = c->pbuf[c->cur];
    g.p[1] = c->pbuf[c->cur ^ 1];
    for (int q = JAC_A0; q <= JAC_BND; ++q) g.coef[q] = c->arr[q];
    return g;
}

// Sweep scratch of a borrowed context: the 256-byte header and one FP64
// partial for each of up to JAC_NOALLOC_MAX_CTAS CTAs.  A sweep launches at
// most one CTA per SM, so this covers every plan on any current GPU.
constexpr size_t kBorrowedSweepScratch = jac::kWsHeaderBytes + (size_t)JAC_NOALLOC_MAX_CTAS * sizeof(double);

// State arrays a tape of max_sweeps sweeps with a checkpoint every C holds:
// its checkpoints, C - 1 segment states and two adjoint buffers.
int tape_states(int C, int max_sweeps)
{
    if (C < 1 || max_sweeps < 1) return 0;
    const int c = std::min(C, max_sweeps);
    return (max_sweeps + c - 1) / c + c + 1;
}

// Layout of a borrowed context's workspace (every region 256-byte aligned).
struct WsLayout {
    size_t sweep = 0, staging = 0, stage_all = 0, tape = 0, total = 0;
    int tape_states = 0;
};

WsLayout ws_layout(int I, int J, int K, jac_prec prec, const jac_ws_spec *spec)
{
    WsLayout L;
    const size_t n = (size_t)I * J * K;
    const size_t state = jac::round_up((size_t)jac_pitch(I) * J * K * jac::elem_bytes(prec, JAC_P), 256);
    L.sweep = kBorrowedSweepScratch;
    L.staging = jac::round_up(n * sizeof(double), 256);
    L.stage_all = (spec && spec->async_upload) ? jac::round_up(JAC_NFIELDS * n * sizeof(double), 256) : 0;
    L.tape_states = spec ? tape_states(spec->tape_C, spec->tape_max) : 0;
    L.tape = L.tape_states ? (size_t)L.tape_states * state + 256 : 0;
    L.total = L.sweep + L.staging + L.stage_all + L.tape;
    return L;
}

jac_status check_spec(jac_ctx *c, const jac_ws_spec *spec)
{
    if (spec && (spec->tape_C < 0 || spec->tape_max < 0))
        return ctx_fail(c, JAC_EINVAL, "negative tape size in the workspace spec");
    return JAC_OK;
}

// Points the context at the regions of a borrowed workspace and clears its
// sweep scratch (the kernels need a zero header).
jac_status ws_carve(jac_ctx *c, void *ws, size_t ws_bytes, const jac_ws_spec *spec)
{
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
        return ctx_fail(c, JAC_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    const WsLayout L = ws_layout(c->I, c->J, c->K, c->prec, spec);
    if (ws_bytes < L.total)
        return ctx_fail(c, JAC_EINVAL, "workspace too small: " + std::to_string(ws_bytes) + " bytes, need " +
                                           std::to_string(L.total) + " (jac_workspace_size)");
    char *p = static_cast<char *>(ws);
    c->ws = p;
    c->ws_bytes = L.sweep;
    p += L.sweep;
    c->staging = reinterpret_cast<double *>(p);
    p += L.staging;
    c->stage_all = L.stage_all ? reinterpret_cast<double *>(p) : nullptr;
    p += L.stage_all;
    c->tape_region = L.tape ? p : nullptr;
    c->tape_cap = L.tape_states;
    cudaError_t e = cudaMemsetAsync(c->ws, 0, L.sweep, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "cudaMemsetAsync");
    return JAC_OK;
}

jac_status ensure_workspace(jac_ctx *c)
{
    jac_grid g = make_grid(c);
    size_t need = 0;
    jac_status s = jac_sweep_workspace_size(&g, &c->plan, &need);
    if (s != JAC_OK) return ctx_from_thread(c, s);
    if (need <= c->ws_bytes) return JAC_OK;
    if (c->borrowed)
        return ctx_fail(c, JAC_EINVAL, "the sweep needs " + std::to_string(need) +
                                           " bytes of scratch, more than a borrowed workspace holds");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "cudaStreamSynchronize");
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    e = cudaMalloc(&c->ws, need);
    if (e != cudaSuccess) return ctx_fail(c, JAC_ENOMEM, "workspace allocation failed");
    e = cudaMemsetAsync(c->ws, 0, need, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "cudaMemsetAsync");
    c->ws_bytes = need;
    return JAC_OK;
}

void tape_free(jac_ctx *c)
{
    if (c->tape.mem) {
        cudaStreamSynchronize(c->stream);
        if (!c->borrowed) cudaFree(c->tape.mem);
    }
    c->tape = jac_ctx::Tape();
}

// Sweeps on the resident state; while a tape is active, the state at the
// start of every C-sweep segment is saved first.
jac_status sweep_impl(jac_ctx *c, int n_iter)
{
    jac_status s = ensure_workspace(c);
    if (s != JAC_OK) return s;
    jac::WsHeader *hdr = static_cast<jac::WsHeader *>(c->ws);
    jac_ctx::Tape &tp = c->tape;
    if (tp.mem && tp.taped + n_iter > tp.max_sweeps)
        return ctx_fail(c, JAC_ESTATE, "more sweeps than the tape was sized for");
    while (n_iter > 0) {
        int chunk = n_iter;
        if (tp.mem) {
            if (tp.taped % tp.C == 0) {
                cudaError_t e = cudaMemcpyAsync(tp.ckpt(tp.taped / tp.C), c->pbuf[c->cur], data_bytes(c, JAC_P),
                                                cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) return ctx_cuda(c, e, "checkpoint copy");
            }
            chunk = std::min(n_iter, tp.C - tp.taped % tp.C);
        }
        jac_grid g = make_grid(c);
        jac::LaunchOpts opts;
        if (c->stall_ns) {            // the grid barrier of this launch is never reached
            opts.wait_ns = c->stall_ns;
            opts.gbar_extra = 1;
            c->stall_ns = 0;
        }
        s = jac::sweep_dev(&g, &c->plan, chunk, &hdr->residual, c->ws, c->ws_bytes, c->stream, &opts);
        if (s != JAC_OK) return ctx_from_thread(c, s);
        c->cur = (c->cur + chunk) & 1;
        c->count += chunk;
        if (tp.mem) tp.taped += chunk;
        n_iter -= chunk;
    }
    c->has_res = true;
    return JAC_OK;
}

enum class Src { host, device, host_async, host_async_f32 };

// The copy-in.  Host sources go through device staging: one array reused
// per field (synchronous), or, for the asynchronous form, one staging array
// per field, so that all thirteen host-to-device copies run on the copy
// engine without waiting for the packing kernels (which need free SMs).
jac_status upload_impl(jac_ctx *c, const jac_fields *f, Src from)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    if (!f) return ctx_fail(c, JAC_EINVAL, "fields is NULL");
    for (int q = 0; q < JAC_NFIELDS; ++q)
        if (!f->f[q]) return ctx_fail(c, JAC_EINVAL, "field " + std::to_string(q) + " is NULL");
    const size_t n = (size_t)c->I * c->J * c->K;
    const bool async = from == Src::host_async || from == Src::host_async_f32;
    if (async && !c->stage_all && c->borrowed)
        return ctx_fail(c, JAC_ENOMEM, "the borrowed workspace has no room for the asynchronous staging arrays "
                                       "(jac_set_workspace with async_upload set)");
    if (from == Src::host_async_f32) {
        // thirteen FP32 copies into the asynchronous staging (as floats), then the packing kernels
        const float *const *src32 = reinterpret_cast<const float *const *>(f->f);
        if (!c->stage_all) {
            cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&c->stage_all), JAC_NFIELDS * n * sizeof(double));
            if (e != cudaSuccess) {
                c->stage_all = nullptr;
                return ctx_fail(c, JAC_ENOMEM, "device allocation of the asynchronous staging arrays failed");
            }
        }
        float *st32 = reinterpret_cast<float *>(c->stage_all);
        for (int q = 0; q < JAC_NFIELDS; ++q) {
            cudaError_t e = cudaMemcpyAsync(st32 + (size_t)q * n, src32[q], n * sizeof(float), cudaMemcpyHostToDevice,
                                            c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "host-to-device copy");
        }
        for (int q = 0; q < JAC_NFIELDS; ++q) {
            jac_status s = jac::pack_dev_f32(c->I, c->J, c->K, c->prec, q, st32 + (size_t)q * n,
                                             q == JAC_P ? c->pbuf[0] : c->arr[q], c->stream);
            if (s != JAC_OK) return ctx_from_thread(c, s);
        }
        cudaError_t e = cudaMemcpyAsync(c->pbuf[1], c->pbuf[0], data_bytes(c, JAC_P), cudaMemcpyDeviceToDevice,
                                        c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "device copy of p0");
        c->cur = 0;
        c->count = 0;
        c->uploaded = true;
        c->has_res = false;
        tape_free(c);
        return JAC_OK;
    }
    if (from == Src::host_async && !c->stage_all) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&c->stage_all), JAC_NFIELDS * n * sizeof(double));
        if (e != cudaSuccess) {
            c->stage_all = nullptr;
            return ctx_fail(c, JAC_ENOMEM, "device allocation of the asynchronous staging arrays failed");
        }
    }
    const double *src[JAC_NFIELDS];
    for (int q = 0; q < JAC_NFIELDS; ++q) {
        src[q] = f->f[q];
        if (from != Src::device) {
            double *stage = (from == Src::host) ? c->staging : c->stage_all + (size_t)q * n;
            cudaError_t e = cudaMemcpyAsync(stage, src[q], n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return ctx_cuda(c, e, "host-to-device copy");
            src[q] = stage;
        }
        // one reused staging array: pack each field before the next copy
        if (from == Src::host) {
            jac_status s = jac::pack_dev(c->I, c->J, c->K, c->prec, q, src[q],
                                         q == JAC_P ? c->pbuf[0] : c->arr[q], c->stream);
            if (s != JAC_OK) return ctx_from_thread(c, s);
        }
    }
    for (int q = 0; q < JAC_NFIELDS && from != Src::host; ++q) {
        jac_status s = jac::pack_dev(c->I, c->J, c->K, c->prec, q, src[q], q == JAC_P ? c->pbuf[0] : c->arr[q],
                                     c->stream);
        if (s != JAC_OK) return ctx_from_thread(c, s);
    }
    cudaError_t e = cudaMemcpyAsync(c->pbuf[1], c->pbuf[0], data_bytes(c, JAC_P), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "device copy of p0");
    if (from == Src::host) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "cudaStreamSynchronize");
    }
    c->cur = 0;
    c->count = 0;
    c->uploaded = true;
    c->has_res = false;
    tape_free(c);
    return JAC_OK;
}

}  // namespace

extern "C" {

jac_status jac_create(jac_ctx **out, int I, int J, int K, jac_prec prec, double omega, void *stream)
{
    if (!out) return ctx_fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    if (I < 3 || J < 3 || K < 3) return ctx_fail(nullptr, JAC_EINVAL, "every grid dimension must be >= 3");
    if (prec != JAC_F64 && prec != JAC_F32 && prec != JAC_F32_BF16COEF)
        return ctx_fail(nullptr, JAC_EINVAL, "unknown precision");
    if (!std::isfinite(omega)) return ctx_fail(nullptr, JAC_EINVAL, "omega must be finite");
    jac_ctx *c = new (std::nothrow) jac_ctx;
    if (!c) return ctx_fail(nullptr, JAC_ENOMEM, "host allocation failed");
    c->I = I; c->J = J; c->K = K;
    c->pitch = jac_pitch(I);
    c->prec = prec;
    c->omega = omega;
    c->stream = static_cast<cudaStream_t>(stream);
    size_t total = 2 * array_bytes(c, JAC_P);
    for (int q = JAC_A0; q <= JAC_BND; ++q) total += array_bytes(c, q);
    cudaError_t e = cudaMalloc(&c->arena, total);
    if (e != cudaSuccess) {
        delete c;
        return ctx_fail(nullptr, JAC_ENOMEM, "device allocation of the fields failed");
    }
    char *p = static_cast<char *>(c->arena);
    c->pbuf[0] = p; p += array_bytes(c, JAC_P);
    c->pbuf[1] = p; p += array_bytes(c, JAC_P);
    for (int q = JAC_A0; q <= JAC_BND; ++q) {
        c->arr[q] = p;
        p += array_bytes(c, q);
    }
    e = cudaMalloc(reinterpret_cast<void **>(&c->staging), (size_t)I * J * K * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        return ctx_fail(nullptr, JAC_ENOMEM, "device allocation of the staging array failed");
    }
    e = cudaMemsetAsync(c->arena, 0, total, c->stream);
    if (e != cudaSuccess) {
        jac_status s = ctx_cuda(nullptr, e, "cudaMemsetAsync");
        cudaFree(c->staging);
        cudaFree(c->arena);
        delete c;
        return s;
    }
    jac_status s = ensure_workspace(c);
    if (s != JAC_OK) {
        cudaFree(c->staging);
        cudaFree(c->arena);
        delete c;
        return s;
    }
    *out = c;
    return JAC_OK;
}

jac_status jac_destroy(jac_ctx *c)
{
    if (!c) return JAC_OK;
    tape_free(c);
    cudaStreamSynchronize(c->stream);
    if (c->borrowed) {                // nothing of the device memory is the context's
        delete c;
        return JAC_OK;
    }
    if (c->ws) cudaFree(c->ws);
    if (c->staging) cudaFree(c->staging);
    if (c->stage_all) cudaFree(c->stage_all);
    if (c->arena) cudaFree(c->arena);
    delete c;
    return JAC_OK;
}

jac_status jac_field_bytes(int I, int J, int K, jac_prec prec, int which, size_t *bytes)
{
    if (!bytes) return ctx_fail(nullptr, JAC_EINVAL, "bytes is NULL");
    if (I < 3 || J < 3 || K < 3) return ctx_fail(nullptr, JAC_EINVAL, "every grid dimension must be >= 3");
    if (prec != JAC_F64 && prec != JAC_F32 && prec != JAC_F32_BF16COEF)
        return ctx_fail(nullptr, JAC_EINVAL, "unknown precision");
    if (which < 0 || which >= JAC_NFIELDS) return ctx_fail(nullptr, JAC_EINVAL, "bad array index");
    *bytes = (size_t)jac_pitch(I) * J * K * jac::elem_bytes(prec, which);
    return JAC_OK;
}

jac_status jac_workspace_size(int I, int J, int K, jac_prec prec, const jac_ws_spec *spec, size_t *bytes)
{
    if (!bytes) return ctx_fail(nullptr, JAC_EINVAL, "bytes is NULL");
    if (I < 3 || J < 3 || K < 3) return ctx_fail(nullptr, JAC_EINVAL, "every grid dimension must be >= 3");
    if (prec != JAC_F64 && prec != JAC_F32 && prec != JAC_F32_BF16COEF)
        return ctx_fail(nullptr, JAC_EINVAL, "unknown precision");
    jac_status s = check_spec(nullptr, spec);
    if (s != JAC_OK) return s;
    *bytes = ws_layout(I, J, K, prec, spec).total;
    return JAC_OK;
}

jac_status jac_create_borrowed(jac_ctx **out, const jac_grid *fields, void *stream, void *workspace,
                               size_t ws_bytes, const jac_ws_spec *spec)
{
    if (!out) return ctx_fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    jac_status s = jac::validate_grid(fields);
    if (s != JAC_OK) return s;
    if ((s = check_spec(nullptr, spec)) != JAC_OK) return s;
    jac_ctx *c = new (std::nothrow) jac_ctx;
    if (!c) return ctx_fail(nullptr, JAC_ENOMEM, "host allocation failed");
    c->borrowed = true;
    c->I = fields->I; c->J = fields->J; c->K = fields->K;
    c->pitch = jac_pitch(c->I);
    c->prec = fields->prec;
    c->omega = fields->omega;
    c->stream = static_cast<cudaStream_t>(stream);
    c->pbuf[0] = fields->p[0];
    c->pbuf[1] = fields->p[1];
    for (int q = JAC_A0; q <= JAC_BND; ++q) c->arr[q] = const_cast<void *>(fields->coef[q]);
    if ((s = ws_carve(c, workspace, ws_bytes, spec)) != JAC_OK || (s = ensure_workspace(c)) != JAC_OK) {
        delete c;
        return s;
    }
    *out = c;
    return JAC_OK;
}

jac_status jac_set_workspace(jac_ctx *c, void *workspace, size_t ws_bytes, const jac_ws_spec *spec)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    if (!c->borrowed) return ctx_fail(c, JAC_ESTATE, "jac_set_workspace needs a context from jac_create_borrowed");
    jac_status s = check_spec(c, spec);
    if (s != JAC_OK) return s;
    tape_free(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "cudaStreamSynchronize");
    c->has_res = false;                // the residual lived in the old workspace
    if ((s = ws_carve(c, workspace, ws_bytes, spec)) != JAC_OK) {
        c->ws = nullptr;               // no sweep until a workspace is set
        c->ws_bytes = 0;
        c->staging = c->stage_all = nullptr;
        c->tape_region = nullptr;
        c->tape_cap = 0;
        return s;
    }
    return ensure_workspace(c);
}

const char *jac_last_error(const jac_ctx *c) { return c ? c->err.c_str() : jac::thread_last_error(); }

jac_status jac_set_plan(jac_ctx *c, const jac_plan *plan)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    jac_plan p{0, 0, 0, 0};
    if (plan) p = *plan;
    if (p.tile_j < 0 || p.tile_i < 0 || (p.kdepth < 0 && p.kdepth != JAC_KDEPTH_BALANCED))
        return ctx_fail(c, JAC_EINVAL, "negative plan entry");
    if (p.kdepth == JAC_KDEPTH_BALANCED && c->prec != JAC_F64)
        return ctx_fail(c, JAC_EINVAL, "balanced ranges (JAC_KDEPTH_BALANCED) are for FP64 storage");
    if (p.fuse < 0 || p.fuse > 2) return ctx_fail(c, JAC_EINVAL, "fuse must be 0, 1 or 2");
    if (p.tile_i || p.tile_j) {
        jac_grid g = make_grid(c);
        int rw = 0, tj = 0;
        jac_status s = jac::check_plan(c->prec, jac::resolve_plan(&g, &p), &rw, &tj);
        if (s != JAC_OK) return ctx_from_thread(c, s);
    }
    c->plan = p;
    return ensure_workspace(c);
}

jac_status jac_upload(jac_ctx *c, const jac_fields *host) { return upload_impl(c, host, Src::host); }

jac_status jac_upload_async(jac_ctx *c, const jac_fields *host) { return upload_impl(c, host, Src::host_async); }

jac_status jac_upload_dev(jac_ctx *c, const jac_fields *dev) { return upload_impl(c, dev, Src::device); }

jac_status jac_upload_f32_async(jac_ctx *c, const jac_fields_f32 *host)
{
    if (!host) return ctx_fail(c, JAC_EINVAL, "fields is NULL");
    jac_fields f;
    for (int q = 0; q < JAC_NFIELDS; ++q) f.f[q] = reinterpret_cast<const double *>(host->f[q]);
    return upload_impl(c, &f, Src::host_async_f32);
}

jac_status jac_sweep(jac_ctx *c, int n_iter)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    if (!c->uploaded) return ctx_fail(c, JAC_ESTATE, "jac_sweep before jac_upload");
    if (n_iter < 0) return ctx_fail(c, JAC_EINVAL, "n_iter must be >= 0");
    if (n_iter == 0) return JAC_OK;
    return sweep_impl(c, n_iter);
}

jac_status jac_residual(jac_ctx *c, double *out)
{
    if (!c || !out) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    if (!c->has_res) return ctx_fail(c, JAC_ESTATE, "no sweep since the last upload");
    jac_status s = jac::workspace_check(c->ws, c->stream);
    if (s != JAC_OK) return ctx_from_thread(c, s);
    jac::WsHeader *hdr = static_cast<jac::WsHeader *>(c->ws);
    cudaError_t e = cudaMemcpyAsync(out, &hdr->residual, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "residual copy");
    return JAC_OK;
}

jac_status jac_download_dev(jac_ctx *c, double *p_dev)
{
    if (!c || !p_dev) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    if (!c->uploaded) return ctx_fail(c, JAC_ESTATE, "download before upload");
    return ctx_from_thread(c, jac::unpack_dev(c->I, c->J, c->K, c->prec, JAC_P, c->pbuf[c->cur], p_dev, c->stream));
}

jac_status jac_download(jac_ctx *c, double *p_host)
{
    if (!c || !p_host) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    jac_status s = jac_download_dev(c, c ? c->staging : nullptr);
    if (s != JAC_OK) return s;
    const size_t n = (size_t)c->I * c->J * c->K;
    cudaError_t e = cudaMemcpyAsync(p_host, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "device-to-host copy");
    s = jac::workspace_check(c->ws, c->stream);  // synchronises
    return ctx_from_thread(c, s);
}

jac_status jac_download_async(jac_ctx *c, double *p_host, double *res_host)
{
    if (!c || !p_host) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    if (res_host && !c->has_res) return ctx_fail(c, JAC_ESTATE, "no sweep since the last upload");
    jac_status s = jac_download_dev(c, c->staging);
    if (s != JAC_OK) return s;
    const size_t n = (size_t)c->I * c->J * c->K;
    cudaError_t e = cudaMemcpyAsync(p_host, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "device-to-host copy");
    if (res_host) {
        jac::WsHeader *hdr = static_cast<jac::WsHeader *>(c->ws);
        e = cudaMemcpyAsync(res_host, &hdr->residual, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "residual copy");
    }
    return JAC_OK;
}

jac_status jac_download_f32_async(jac_ctx *c, float *p_host, double *res_host)
{
    if (!c || !p_host) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    if (!c->uploaded) return ctx_fail(c, JAC_ESTATE, "download before upload");
    if (res_host && !c->has_res) return ctx_fail(c, JAC_ESTATE, "no sweep since the last upload");
    float *st32 = reinterpret_cast<float *>(c->staging);
    if (!st32) return ctx_fail(c, JAC_ESTATE, "no staging array (workspace not set)");
    jac_status s = jac::unpack_dev_f32(c->I, c->J, c->K, c->prec, JAC_P, c->pbuf[c->cur], st32, c->stream);
    if (s != JAC_OK) return ctx_from_thread(c, s);
    const size_t n = (size_t)c->I * c->J * c->K;
    cudaError_t e = cudaMemcpyAsync(p_host, st32, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return ctx_cuda(c, e, "device-to-host copy");
    if (res_host) {
        jac::WsHeader *hdr = static_cast<jac::WsHeader *>(c->ws);
        e = cudaMemcpyAsync(res_host, &hdr->residual, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "residual copy");
    }
    return JAC_OK;
}

jac_status jac_sync(jac_ctx *c)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    return ctx_from_thread(c, jac::workspace_check(c->ws, c->stream));
}

jac_status jac_sweep_count(const jac_ctx *c, long long *out)
{
    if (!c || !out) return JAC_EINVAL;
    *out = c->count;
    return JAC_OK;
}

jac_status jac_get_grid(const jac_ctx *c, jac_grid *g)
{
    if (!c || !g) return JAC_EINVAL;
    *g = make_grid(c);
    return JAC_OK;
}

jac_status jac_tape_begin(jac_ctx *c, int C, int max_sweeps)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    if (!c->uploaded) return ctx_fail(c, JAC_ESTATE, "jac_tape_begin before jac_upload");
    if (C < 1 || max_sweeps < 1) return ctx_fail(c, JAC_EINVAL, "C and max_sweeps must be >= 1");
    tape_free(c);
    jac_ctx::Tape tp;
    tp.C = std::min(C, max_sweeps);
    tp.max_sweeps = max_sweeps;
    tp.state_bytes = array_bytes(c, JAC_P);
    tp.n_ckpt = (max_sweeps + tp.C - 1) / tp.C;
    const size_t bytes = (size_t)(tp.n_ckpt + tp.C + 1) * tp.state_bytes + 256;
    if (c->borrowed) {
        const int need = tape_states(C, max_sweeps);
        if (need > c->tape_cap)
            return ctx_fail(c, JAC_ENOMEM, "this tape needs " + std::to_string(need) +
                                               " state arrays; the borrowed workspace holds " +
                                               std::to_string(c->tape_cap) + " (jac_set_workspace with a larger tape)");
        tp.mem = c->tape_region;
        c->tape = tp;
        return JAC_OK;
    }
    cudaError_t e = cudaMalloc(&tp.mem, bytes);
    if (e != cudaSuccess) return ctx_fail(c, JAC_ENOMEM, "tape allocation failed (" + std::to_string(bytes) + " bytes)");
    c->tape = tp;
    return JAC_OK;
}

jac_status jac_tape_end(jac_ctx *c)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    tape_free(c);
    return JAC_OK;
}

jac_status jac_sweep_adjoint(jac_ctx *c, const double *lam_T, double *g_wrk1, double *g_a3, double *const *g_coef,
                             double *g_p0)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    jac_ctx::Tape &tp = c->tape;
    if (!tp.mem || tp.taped == 0) return ctx_fail(c, JAC_ESTATE, "no taped sweeps: call jac_tape_begin, then jac_sweep");
    if (!lam_T || !g_wrk1 || !g_a3) return ctx_fail(c, JAC_EINVAL, "lambda_T, g_wrk1 and g_a3 are required");
    jac_status s = ensure_workspace(c);
    if (s != JAC_OK) return s;
    const size_t n = (size_t)c->I * c->J * c->K;
    cudaError_t e = cudaMemsetAsync(g_wrk1, 0, n * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_a3, 0, n * sizeof(double), c->stream);
    for (int q = 0; g_coef && q < 9 && e == cudaSuccess; ++q) {
        if (!g_coef[q]) return ctx_fail(c, JAC_EINVAL, "g_coef needs all nine arrays");
        e = cudaMemsetAsync(g_coef[q], 0, n * sizeof(double), c->stream);
    }
    if (e != cudaSuccess) return ctx_cuda(c, e, "gradient clear");
    // lambda_T into storage layout
    s = jac::pack_dev(c->I, c->J, c->K, c->prec, JAC_P, lam_T, tp.lam(0), c->stream);
    if (s != JAC_OK) return ctx_from_thread(c, s);
    // faces never change: give every segment slot the faces of the first checkpoint
    for (int m = 1; m < tp.C; ++m) {
        e = cudaMemcpyAsync(tp.seg(m), tp.ckpt(0), tp.state_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return ctx_cuda(c, e, "segment init");
    }
    jac_grid g = make_grid(c);
    const bool pairs = c->prec == JAC_F32 && jac::resolve_plan(&g, &c->plan).fuse == 2;
    int lc = 0;
    const int nseg = (tp.taped + tp.C - 1) / tp.C;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int t0 = sgi * tp.C;
        const int len = std::min(tp.C, tp.taped - t0);
        // state m of this segment: the checkpoint itself for m = 0
        auto state = [&](int m) -> void * { return m == 0 ? tp.ckpt(sgi) : tp.seg(m); };
        // recompute the segment's states: where the plan takes two-sweep
        // passes, one pass gives two states (the intermediate one stored on
        // the way), bitwise those of single sweeps
        for (int m = 1; m < len;) {
            g.p[0] = state(m - 1);
            if (pairs && m + 1 < len) {
                g.p[1] = tp.seg(m + 1);
                s = jac::sweep2_run(&g, 0, 1, nullptr, c->ws, c->ws_bytes, c->stream, tp.seg(m));
                m += 2;
            } else {
                g.p[1] = tp.seg(m);
                s = jac::sweep_dev(&g, &c->plan, 1, tp.scratch(), c->ws, c->ws_bytes, c->stream);
                m += 1;
            }
            if (s != JAC_OK) return ctx_from_thread(c, s);
        }
        for (int m = len - 1; m >= 0; --m) {     // reverse sweeps of the segment
            s = jac::adjoint_step_dev(&g, state(m), tp.lam(lc), tp.lam(lc ^ 1), g_wrk1, g_a3, g_coef, 0, c->ws,
                                      c->ws_bytes, c->stream);
            if (s != JAC_OK) return ctx_from_thread(c, s);
            lc ^= 1;
        }
    }
    if (g_p0) {
        s = jac::unpack_dev(c->I, c->J, c->K, c->prec, JAC_P, tp.lam(lc), g_p0, c->stream);
        if (s != JAC_OK) return ctx_from_thread(c, s);
    }
    return JAC_OK;
}

jac_status jac_inject_stall(jac_ctx *c, unsigned long long wait_ns)
{
    if (!c) return ctx_fail(c, JAC_EINVAL, "ctx is NULL");
    if (wait_ns > jac::kWaitLimitNs) return ctx_fail(c, JAC_EINVAL, "wait_ns above the library's wait limit");
    c->stall_ns = wait_ns;
    return JAC_OK;
}

jac_status jac_tape_count(const jac_ctx *c, int *out)
{
    if (!c || !out) return JAC_EINVAL;
    *out = c->tape.mem ? c->tape.taped : 0;
    return JAC_OK;
}

jac_status jac_sweep_unhoisted(jac_ctx *c, int n_iter, const jac_fields *host, double *p_host)
{
    if (!c || !host || !p_host) return ctx_fail(c, JAC_EINVAL, "NULL argument");
    if (n_iter < 0) return ctx_fail(c, JAC_EINVAL, "n_iter must be >= 0");
    jac_fields f = *host;
    f.f[JAC_P] = p_host;
    for (int t = 0; t < n_iter; ++t) {
        jac_status s = upload_impl(c, &f, Src::host);
        if (s == JAC_OK) s = jac_sweep(c, 1);
        if (s == JAC_OK) s = jac_download(c, p_host);
        if (s != JAC_OK) return s;
    }
    c->count = n_iter;
    return JAC_OK;
}

}  // extern "C"
