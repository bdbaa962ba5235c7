// Batched sweeps of libjac: many independent grids of uneven sizes in one
// persistent, cooperative launch, captured once in a CUDA graph and replayed.
//
// Every grid keeps its own compact storage (the single-grid layout) and gets
// a descriptor -- its tensor maps, tiling (tile width, row fold, k-block
// depth) and first work item -- in a device table.  The forward kernel of
// jac_sweep_kernel.cuh walks the concatenated work items of all grids; a
// bounded grid barrier separates sweeps across the whole batch and the
// residual of each grid is reduced deterministically.  Tile widths and
// k-block depths come per grid from a plan (an autotuner chooses them per
// size class by measurement).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "jac_internal.h"
#include "jac_sweep_kernel.cuh"

struct jac_batch {
    int n = 0;
    jac_prec prec = JAC_F32;
    double omega = 0.8;
    cudaStream_t stream = nullptr;
    std::vector<int> I, J, K;
    std::vector<jac::GridDesc> host_descs;
    std::vector<jac_grid> grids;           // storage pointers, p[0]/p[1] = buffers 0/1
    void *arena = nullptr;
    double *staging = nullptr;             // largest I*J*K doubles
    double *d_res = nullptr;               // n residuals
    jac::GridDesc *d_descs = nullptr;
    int *d_item_base = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int warps = 8;
    std::vector<int> tile_i, kdepth;       // per grid, 0 = default
    bool tables_ok = false;
    int nitems = 0;
    unsigned nblocks = 0;
    int par = 0;                           // buffer holding the current state
    long long count = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (n_iter, par) -> graph
    std::string err;
};

namespace {

jac_status bfail(jac_batch *b, jac_status s, const std::string &m)
{
    if (b) b->err = m;
    jac::set_thread_error(m);
    return s;
}

jac_status bcuda(jac_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, JAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

jac_status bthread(jac_batch *b, jac_status s)
{
    if (s != JAC_OK && b) b->err = jac::thread_last_error();
    return s;
}

size_t arr_bytes(const jac_batch *b, int g, int which)
{
    return jac::round_up((size_t)jac_pitch(b->I[g]) * b->J[g] * b->K[g] * jac::elem_bytes(b->prec, which), 256);
}

void drop_graphs(jac_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

void drop_tables(jac_batch *b)
{
    drop_graphs(b);
    if (b->d_descs) cudaFree(b->d_descs);
    if (b->d_item_base) cudaFree(b->d_item_base);
    if (b->ws) cudaFree(b->ws);
    b->d_descs = nullptr;
    b->d_item_base = nullptr;
    b->ws = nullptr;
    b->ws_bytes = 0;
    b->tables_ok = false;
}

jac_plan grid_plan(const jac_batch *b, int g)
{
    const int full = 32 * jac::vector_points(b->prec);
    jac_plan p;
    p.fuse = 1;   // batched grids sweep one sweep per pass
    p.tile_i = b->tile_i[g] > 0 ? b->tile_i[g] : jac::best_tile_i(b->I[g], b->J[g], b->prec, b->warps);
    p.tile_j = b->warps * (full / p.tile_i);
    p.kdepth = b->kdepth[g];
    if (p.kdepth <= 0) {
        // one k-block per about 16 output planes of the grid
        p.kdepth = std::max(2, std::min(b->K[g] - 2, 16));
    }
    return p;
}

// Descriptors, item bases and workspace for the current plan.
jac_status build_tables(jac_batch *b)
{
    if (b->tables_ok) return JAC_OK;
    drop_tables(b);
    b->host_descs.assign(b->n, jac::GridDesc());
    std::vector<int> base(b->n);
    long long items = 0;
    for (int g = 0; g < b->n; ++g) {
        const jac_plan p = grid_plan(b, g);
        int rw = 0, tj = 0;
        jac_status s = jac::check_plan(b->prec, p, &rw, &tj);
        if (s != JAC_OK) return bthread(b, s);
        if (tj != b->warps) return bfail(b, JAC_EINVAL, "plan of grid " + std::to_string(g) + " needs another warp count");
        base[g] = (int)items;
        if ((s = jac::build_desc(&b->host_descs[g], &b->grids[g], p, (int)items)) != JAC_OK) return bthread(b, s);
        items += b->host_descs[g].nitems;
        if (items > 0x3fffffffLL) return bfail(b, JAC_EINVAL, "too many work items");
    }
    b->nitems = (int)items;
    b->nblocks = (unsigned)std::min<long long>(items, jac::device_sm_count());
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_descs), sizeof(jac::GridDesc) * b->n);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_item_base), sizeof(int) * b->n);
    b->ws_bytes = jac::kWsHeaderBytes + jac::round_up((size_t)b->n * b->nblocks * sizeof(double), 256);
    if (e == cudaSuccess) e = cudaMalloc(&b->ws, b->ws_bytes);
    if (e != cudaSuccess) {
        drop_tables(b);
        return bfail(b, JAC_ENOMEM, "batch table allocation failed");
    }
    e = cudaMemcpy(b->d_descs, b->host_descs.data(), sizeof(jac::GridDesc) * b->n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_item_base, base.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->ws, 0, b->ws_bytes);
    if (e != cudaSuccess) {
        drop_tables(b);
        return bcuda(b, e, "batch table upload");
    }
    b->tables_ok = true;
    return JAC_OK;
}

jac::SweepArgs batch_args(const jac_batch *b, int n_iter)
{
    jac::SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.descs = b->d_descs;
    a.item_base = b->d_item_base;
    a.ngrids = b->n;
    a.nitems = b->nitems;
    a.n_iter = n_iter;
    a.par = b->par;
    a.omega = b->omega;
    a.hdr = static_cast<jac::WsHeader *>(b->ws);
    a.partials = reinterpret_cast<double *>(static_cast<char *>(b->ws) + jac::kWsHeaderBytes);
    a.res = b->d_res;
    size_t points = 0;
    for (int g = 0; g < b->n; ++g) points += (size_t)jac_pitch(b->I[g]) * b->J[g] * b->K[g];
    jac::set_l2_policy(a, b->prec, points);
    return a;
}

jac_status read_residuals(jac_batch *b, double *res_host)
{
    if (res_host) {
        cudaError_t e = cudaMemcpyAsync(res_host, b->d_res, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "residual copy");
    }
    jac_status s = jac::workspace_check(b->ws, b->stream);   // synchronises
    return bthread(b, s);
}

jac_grid current_grid(const jac_batch *b, int g)
{
    jac_grid gr = b->grids[g];
    gr.p[0] = b->grids[g].p[b->par];
    gr.p[1] = b->grids[g].p[b->par ^ 1];
    return gr;
}

}  // namespace

extern "C" {

jac_status jac_batch_create(jac_batch **out, int n, const int *dims, jac_prec prec, double omega, void *stream)
{
    if (!out) return bfail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !dims) return bfail(nullptr, JAC_EINVAL, "need at least one grid");
    if (prec != JAC_F64 && prec != JAC_F32 && prec != JAC_F32_BF16COEF)
        return bfail(nullptr, JAC_EINVAL, "unknown precision");
    if (!std::isfinite(omega)) return bfail(nullptr, JAC_EINVAL, "omega must be finite");
    for (int g = 0; g < n; ++g)
        if (dims[3 * g] < 3 || dims[3 * g + 1] < 3 || dims[3 * g + 2] < 3)
            return bfail(nullptr, JAC_EINVAL, "every grid dimension must be >= 3");
    jac_batch *b = new (std::nothrow) jac_batch;
    if (!b) return bfail(nullptr, JAC_ENOMEM, "host allocation failed");
    b->n = n;
    b->prec = prec;
    b->omega = omega;
    b->stream = static_cast<cudaStream_t>(stream);
    b->I.resize(n); b->J.resize(n); b->K.resize(n);
    b->tile_i.assign(n, 0);
    b->kdepth.assign(n, 0);
    size_t total = 0, max_n = 0;
    for (int g = 0; g < n; ++g) {
        b->I[g] = dims[3 * g]; b->J[g] = dims[3 * g + 1]; b->K[g] = dims[3 * g + 2];
        total += 2 * arr_bytes(b, g, JAC_P);
        for (int q = JAC_A0; q <= JAC_BND; ++q) total += arr_bytes(b, g, q);
        max_n = std::max(max_n, (size_t)b->I[g] * b->J[g] * b->K[g]);
    }
    b->warps = 8;
    cudaError_t e = cudaMalloc(&b->arena, total);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->staging), max_n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_res), n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena, 0, total, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_res, 0, n * sizeof(double), b->stream);
    if (e != cudaSuccess) {
        if (b->arena) cudaFree(b->arena);
        if (b->staging) cudaFree(b->staging);
        if (b->d_res) cudaFree(b->d_res);
        delete b;
        return bfail(nullptr, JAC_ENOMEM, "batch device allocation failed");
    }
    char *p = static_cast<char *>(b->arena);
    b->grids.resize(n);
    for (int g = 0; g < n; ++g) {
        jac_grid &gr = b->grids[g];
        std::memset(&gr, 0, sizeof(gr));
        gr.I = b->I[g]; gr.J = b->J[g]; gr.K = b->K[g];
        gr.prec = prec;
        gr.omega = omega;
        gr.p[0] = p; p += arr_bytes(b, g, JAC_P);
        gr.p[1] = p; p += arr_bytes(b, g, JAC_P);
        for (int q = JAC_A0; q <= JAC_BND; ++q) {
            gr.coef[q] = p;
            p += arr_bytes(b, g, q);
        }
    }
    *out = b;
    return JAC_OK;
}

jac_status jac_batch_destroy(jac_batch *b)
{
    if (!b) return JAC_OK;
    cudaStreamSynchronize(b->stream);
    drop_tables(b);
    if (b->arena) cudaFree(b->arena);
    if (b->staging) cudaFree(b->staging);
    if (b->d_res) cudaFree(b->d_res);
    delete b;
    return JAC_OK;
}

const char *jac_batch_last_error(const jac_batch *b) { return b ? b->err.c_str() : jac::thread_last_error(); }

static jac_status batch_upload_impl(jac_batch *b, int g, const jac_fields *f, bool on_device)
{
    if (!b || !f) return bfail(b, JAC_EINVAL, "NULL argument");
    if (g < 0 || g >= b->n) return bfail(b, JAC_EINVAL, "grid index out of range");
    for (int q = 0; q < JAC_NFIELDS; ++q)
        if (!f->f[q]) return bfail(b, JAC_EINVAL, "field " + std::to_string(q) + " is NULL");
    const size_t n = (size_t)b->I[g] * b->J[g] * b->K[g];
    const jac_grid &gr = b->grids[g];
    for (int q = 0; q < JAC_NFIELDS; ++q) {
        const double *src = f->f[q];
        if (!on_device) {
            cudaError_t e = cudaMemcpyAsync(b->staging, src, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "host-to-device copy");
            src = b->staging;
        }
        void *dst = (q == JAC_P) ? gr.p[0] : const_cast<void *>(gr.coef[q]);
        jac_status s = jac::pack_dev(b->I[g], b->J[g], b->K[g], b->prec, q, src, dst, b->stream);
        if (s != JAC_OK) return bthread(b, s);
    }
    cudaError_t e = cudaMemcpyAsync(gr.p[1], gr.p[0], arr_bytes(b, g, JAC_P), cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "device copy of p0");
    if (!on_device) {
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
    }
    return JAC_OK;
}

jac_status jac_batch_upload(jac_batch *b, int g, const jac_fields *host) { return batch_upload_impl(b, g, host, false); }

jac_status jac_batch_upload_dev(jac_batch *b, int g, const jac_fields *dev) { return batch_upload_impl(b, g, dev, true); }

jac_status jac_batch_set_plan(jac_batch *b, int warps, const int *tile_i, const int *kdepth)
{
    if (!b) return bfail(b, JAC_EINVAL, "batch is NULL");
    if (warps != 0 && !jac::warps_supported(b->prec, warps)) return bfail(b, JAC_EINVAL, "unsupported warp count");
    b->warps = warps ? warps : 8;
    for (int g = 0; g < b->n; ++g) {
        b->tile_i[g] = tile_i ? tile_i[g] : 0;
        b->kdepth[g] = kdepth ? kdepth[g] : 0;
        if (b->tile_i[g] < 0 || b->kdepth[g] < 0) return bfail(b, JAC_EINVAL, "negative plan entry");
    }
    drop_tables(b);
    return JAC_OK;
}

jac_status jac_batch_sweep(jac_batch *b, int n_iter, double *res_host)
{
    if (!b) return bfail(b, JAC_EINVAL, "batch is NULL");
    if (n_iter < 0) return bfail(b, JAC_EINVAL, "n_iter must be >= 0");
    if (n_iter == 0) return JAC_OK;
    jac_status s = build_tables(b);
    if (s != JAC_OK) return s;
    const std::pair<int, int> key(n_iter, b->par);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        // capture the single persistent launch once; later calls replay it
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(b, e, "capture stream");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return bcuda(b, e, "cudaStreamBeginCapture");
        }
        const jac::SweepArgs a = batch_args(b, n_iter);
        s = jac::launch_sweep<true>(b->prec, b->warps, b->host_descs[0], a, b->nblocks, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (s != JAC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return bthread(b, s);
        }
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
        it = b->graphs.emplace(key, exec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
    b->par = (b->par + n_iter) & 1;
    b->count += n_iter;
    return read_residuals(b, res_host);
}

jac_status jac_batch_sweep_loop(jac_batch *b, int n_iter, int per_sweep, double *res_host)
{
    if (!b) return bfail(b, JAC_EINVAL, "batch is NULL");
    if (n_iter < 0) return bfail(b, JAC_EINVAL, "n_iter must be >= 0");
    if (n_iter == 0) return JAC_OK;
    jac_status s = build_tables(b);
    if (s != JAC_OK) return s;
    for (int g = 0; g < b->n; ++g) {
        jac_grid gr = current_grid(b, g);
        const jac_plan p = grid_plan(b, g);
        if (per_sweep) {
            for (int t = 0; t < n_iter; ++t) {
                jac_grid gt = gr;
                gt.p[0] = gr.p[t & 1];
                gt.p[1] = gr.p[(t + 1) & 1];
                s = jac::sweep_dev(&gt, &p, 1, b->d_res + g, b->ws, b->ws_bytes, b->stream);
                if (s != JAC_OK) return bthread(b, s);
            }
        } else {
            s = jac::sweep_dev(&gr, &p, n_iter, b->d_res + g, b->ws, b->ws_bytes, b->stream);
            if (s != JAC_OK) return bthread(b, s);
        }
    }
    b->par = (b->par + n_iter) & 1;
    b->count += n_iter;
    return read_residuals(b, res_host);
}

jac_status jac_batch_download_dev(jac_batch *b, int g, double *p_dev)
{
    if (!b || !p_dev) return bfail(b, JAC_EINVAL, "NULL argument");
    if (g < 0 || g >= b->n) return bfail(b, JAC_EINVAL, "grid index out of range");
    return bthread(b, jac::unpack_dev(b->I[g], b->J[g], b->K[g], b->prec, JAC_P, b->grids[g].p[b->par], p_dev,
                                      b->stream));
}

jac_status jac_batch_download(jac_batch *b, int g, double *p_host)
{
    if (!b || !p_host) return bfail(b, JAC_EINVAL, "NULL argument");
    jac_status s = jac_batch_download_dev(b, g, b ? b->staging : nullptr);
    if (s != JAC_OK) return s;
    const size_t n = (size_t)b->I[g] * b->J[g] * b->K[g];
    cudaError_t e = cudaMemcpyAsync(p_host, b->staging, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "device-to-host copy");
    return JAC_OK;
}

jac_status jac_batch_info(const jac_batch *b, int *n_items, int *n_ctas, int *warps, long long *sweeps)
{
    if (!b) return JAC_EINVAL;
    if (n_items) *n_items = b->tables_ok ? b->nitems : 0;
    if (n_ctas) *n_ctas = b->tables_ok ? (int)b->nblocks : 0;
    if (warps) *warps = b->warps;
    if (sweeps) *sweeps = b->count;
    return JAC_OK;
}

jac_status jac_batch_grid_plan(const jac_batch *b, int g, jac_plan *out)
{
    if (!b || !out || g < 0 || g >= b->n) return JAC_EINVAL;
    *out = grid_plan(b, g);
    return JAC_OK;
}

}  // extern "C"
