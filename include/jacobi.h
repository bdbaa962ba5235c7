/*
 * jacobi.h -- C ABI of libjac, a GB300 (sm_103a) library for the 3-D
 * 19-point variable-coefficient Jacobi relaxation with a fused residual.
 *
 * The operation.  The paper (Yamato, "Improvement of Automatic GPU Offloading
 * Technology for Application Loop Statements") offloads the loop nests of
 * C/C++ applications, evaluated on the Himeno benchmark, a Poisson solve by
 * Jacobi iteration (Section 5.1.1).  One sweep, for every interior point
 * x = (i, j, k) (1 <= i <= I-2, same for j and k), reading state p and writing
 * state p':
 *
 *   s0 = a0 p[i+1] + a1 p[j+1] + a2 p[k+1]
 *      + b0 (p[i+1,j+1] - p[i+1,j-1] - p[i-1,j+1] + p[i-1,j-1])
 *      + b1 (p[j+1,k+1] - p[j+1,k-1] - p[j-1,k+1] + p[j-1,k-1])
 *      + b2 (p[i+1,k+1] - p[i+1,k-1] - p[i-1,k+1] + p[i-1,k-1])
 *      + c0 p[i-1] + c1 p[j-1] + c2 p[k-1] + wrk1
 *   ss = (s0 a3 - p[x]) bnd
 *   p'[x] = p[x] + omega ss
 *
 * with every coefficient read at x.  Faces are never written.  The residual
 * of a sweep is gosa = sum over the interior of ss^2, taken from that sweep's
 * input state.  The paper's transfer hoisting (Section 3.2-3.3: copy data
 * once, outside the outermost loop, and mark it present on the device
 * afterwards) is the structure of this API: jac_upload once, jac_sweep n
 * times with every array resident in device memory, jac_download once.
 *
 * Conventions.
 *   - Every call returns a jac_status.  No call aborts or prints;
 *     jac_last_error() gives the message of the last failure of a context.
 *   - Host arrays ("host fields") are dense FP64, i fastest, then j, then k:
 *     element (i, j, k) at index (k*J + j)*I + i.
 *   - Device storage ("storage layout") is pitched: element (i, j, k) of an
 *     array at offset (k*J + j)*pitch + i elements, pitch = jac_pitch(I).
 *     Element types by precision:
 *       JAC_F64:          every array double;
 *       JAC_F32:          every array float;
 *       JAC_F32_BF16COEF: p and wrk1 float, the eleven coefficient arrays
 *                         a0..a3, b0..b2, c0..c2 and bnd __nv_bfloat16.
 *     Storage values are RNE roundings of the FP64 inputs (BF16 values are
 *     RNE of the FP32-rounded value).  Arithmetic is in the element type of
 *     p; residuals are accumulated in FP64.
 *   - Calls that take a stream enqueue asynchronously on it unless they
 *     return host data, in which case they synchronise that stream.
 *   - The library never calls exit or abort, and device-side waits are
 *     bounded: a wait that runs out sets an error word that the next
 *     synchronising call reports as JAC_ETIMEOUT.
 */
#ifndef JACOBI_H
#define JACOBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum jac_status {
    JAC_OK = 0,
    JAC_EINVAL = 1,    /* bad argument: size, pointer, alignment, precision */
    JAC_ENOMEM = 2,    /* a device or host allocation failed */
    JAC_ECUDA = 3,     /* a CUDA runtime or driver call failed */
    JAC_ESTATE = 4,    /* call not valid in the current state */
    JAC_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    JAC_EINTERNAL = 6  /* an internal consistency check failed */
} jac_status;

typedef enum jac_prec {
    JAC_F64 = 0,          /* FP64 storage and arithmetic */
    JAC_F32 = 1,          /* FP32 storage and arithmetic */
    JAC_F32_BF16COEF = 2  /* FP32 p/wrk1 and arithmetic, BF16 coefficients */
} jac_prec;

/* Array indices of a field set. */
enum {
    JAC_P = 0, JAC_A0, JAC_A1, JAC_A2, JAC_A3, JAC_B0, JAC_B1, JAC_B2,
    JAC_C0, JAC_C1, JAC_C2, JAC_WRK1, JAC_BND, JAC_NFIELDS
};

/* Thirteen dense FP64 arrays (host or device memory, as the call says),
 * indexed by the enum above.  Borrowed for the duration of the call. */
typedef struct jac_fields {
    const double *f[JAC_NFIELDS];
} jac_fields;

/* The same thirteen arrays as dense FP32 values (host memory), for problems
 * whose inputs are FP32 numbers. */
typedef struct jac_fields_f32 {
    const float *f[JAC_NFIELDS];
} jac_fields_f32;

/* Storage pitch (elements) of every array of an I-wide grid: I rounded up to
 * a multiple of 8, so that each row starts on a 16-byte boundary in every
 * element type (the TMA stride rule) and vector loads stay aligned.  No
 * paper counterpart (device layout). */
int jac_pitch(int I);

/* Library version string (static storage).  No paper counterpart. */
const char *jac_version(void);

/* =====================================================================
 * Stateless device API.  The caller owns every buffer.
 * ===================================================================== */

/* One grid in storage layout.  p[0] and p[1] are the two state buffers:
 * sweep t (t = 0, 1, ...) of a call reads p[t % 2] and writes p[(t+1) % 2],
 * so after n sweeps the state is in p[n % 2].  Faces (and the padding
 * columns I..pitch-1) of both buffers must hold the same values; sweeps never
 * write faces.  coef[q] for q = JAC_A0..JAC_BND (q = 1..12, JAC_WRK1
 * included) points at that array; coef[0] is unused.  Every pointer must be
 * 16-byte aligned. */
typedef struct jac_grid {
    int I, J, K;          /* >= 3 each */
    jac_prec prec;
    double omega;
    void *p[2];
    const void *coef[JAC_NFIELDS];
} jac_grid;

/* Launch shape of the sweep kernel.  A work item is tile_i x tile_j points
 * in (i, j) over kdepth consecutive k-planes.  The kernel runs W consumer
 * warps; each covers tile_j / W rows of tile_i points (so W = tile_j * tile_i
 * / 128 for FP32/BF16, tile_j * tile_i / 64 for FP64).  tile_i: a power of
 * two in [16, 128] (FP64: [16, 64]); W must be 4 or 8, or 16 with BF16
 * coefficients and tile_i >= 32.  Zero fields pick defaults: W = 8 (16 for
 * BF16 on grids a 128-wide tile covers fully), the tile width with the best
 * lane use, and a kdepth by precision: FP32/BF16 take the smallest depth
 * (at most 256) at which every work item of a sweep fits one round of CTAs,
 * else 8; FP64 minimises (work-item rounds per CTA) x (kdepth + 3), or
 * takes balanced ranges where their cost (planes per CTA + 3 per tile a
 * range touches) is lower.  kdepth = JAC_KDEPTH_BALANCED: no fixed depth; with T tiles per plane and
 * G CTAs, CTA b takes the tile-planes b*U/G .. (b+1)*U/G - 1 of the
 * tile-major order of all U = T * (K - 2) tile-planes, one work item per
 * tile that range touches, so every CTA gets the same number of planes
 * (FP64 storage only; with FP32 storage they measured slower than the
 * rule above, and the call returns JAC_EINVAL).
 * Unsupported shapes: JAC_EINVAL at launch. */
enum { JAC_KDEPTH_BALANCED = -1 };
typedef struct jac_plan {
    int tile_j;   /* rows per work item */
    int kdepth;   /* k-planes per work item, >= 1, or JAC_KDEPTH_BALANCED */
    int tile_i;   /* points per row */
    int fuse;     /* two sweeps per pass (FP32 storage only; temporal
                     blocking by two): 0 the library's choice, 1 never, 2
                     whenever n_iter >= 4.  The library's choice (what
                     jac_resolve_plan returns for 0) is 2 for FP32 grids
                     whose two state buffers take more than half the L2
                     (the device's, 128 MiB without one), where single sweeps
                     are bound by DRAM bandwidth and a pass, which moves half
                     the bytes per sweep, measured up to 1.26x faster on
                     GB300; else 1 (a state that stays in L2 makes the single
                     sweep faster).  A pass reads the state once and writes it
                     two sweeps later; the state is bitwise that of single
                     sweeps.  Its tile shape is fixed; tile_i, tile_j and
                     kdepth then apply to the 0..3 single sweeps that follow
                     an even number of passes. */
} jac_plan;

/* Paper: launch parameters chosen by rule where the rule is known and by
 * measurement otherwise (Section 4).
 * The plan a sweep of this grid would run with on a device of sm_count SMs
 * (one CTA per SM; sm_count <= 0: the current device's count): the zero
 * fields of *plan (NULL: all zero) filled in by the rules above.  Only the
 * dimensions and the precision of *g are read; no device memory is touched,
 * and with sm_count > 0 no GPU is needed.  Errors: JAC_EINVAL for bad
 * dimensions, precision or plan entries, or a shape the kernels lack. */
jac_status jac_resolve_plan(const jac_grid *g, const jac_plan *plan, int sm_count, jac_plan *out);

/* Bytes of device workspace jac_sweep_dev needs for this grid and plan
 * (host only).  No paper counterpart (the caller-owned scratch of the
 * stateless form). */
jac_status jac_sweep_workspace_size(const jac_grid *g, const jac_plan *plan, size_t *bytes);

/* n_iter sweeps of grid g on the given stream (a cudaStream_t, NULL for the
 * legacy default stream): the Himeno relaxation loop of Section 5.1.1 on
 * arrays already present on the device (Section 3.3).  If d_residual is not
 * NULL, the residual of the last sweep is written there (one double, device
 * memory); if a bounded device wait gave up, that residual is NaN and the
 * workspace's error word is set (jac_workspace_check).  workspace: device
 * memory of at least jac_sweep_workspace_size bytes, 16-byte aligned; its
 * first 256 bytes must be zero before the first call that uses it (the
 * kernels leave them zero again).  Calls that share a workspace must not
 * overlap in time.  n_iter == 0 is a no-op.  Errors: JAC_EINVAL for a bad
 * grid, plan or size; JAC_ECUDA if a launch fails. */
jac_status jac_sweep_dev(const jac_grid *g, const jac_plan *plan, int n_iter,
                         double *d_residual, void *workspace, size_t ws_bytes,
                         void *stream);

/* Reads the device error word kept in a workspace (synchronises the
 * stream): JAC_OK, or JAC_ETIMEOUT if a bounded wait gave up; clears it.
 * Paper: the offload search gives up a measurement after a time limit
 * (Section 5.1.2); the kernels give up their device waits likewise. */
jac_status jac_workspace_check(void *workspace, void *stream);

/* Convert one dense FP64 device array (I*J*K doubles) into storage layout of
 * element type `prec` uses for array `which` (JAC_P .. JAC_BND), on stream.
 * Padding columns are set to zero.  Paper: the device side of the hoisted
 * copy-in (Sections 3.2-3.3). */
jac_status jac_pack_dev(int I, int J, int K, jac_prec prec, int which,
                        const double *d_src, void *d_dst, void *stream);

/* Convert one storage-layout array back to dense FP64 (device memory).
 * Paper: the device side of the hoisted copy-out (Section 3.3). */
jac_status jac_unpack_dev(int I, int J, int K, jac_prec prec, int which,
                          const void *d_src, double *d_dst, void *stream);

/* Largest launch (CTAs) that jac_sweep_dev_noalloc serves: its scratch is
 * 256 + 8 * JAC_NOALLOC_MAX_CTAS bytes (16.6 KiB).  The sweep launches at
 * most one CTA per SM, so every current GPU fits. */
#define JAC_NOALLOC_MAX_CTAS 2048

/* jac_sweep_dev without a workspace argument, for callers that cannot
 * allocate device memory: a plugin whose host application owns the GPU's
 * memory through its own pool and passes in only input and output buffers,
 * or a loop that cannot take the device-wide synchronisation cudaMalloc and
 * cudaFree may cause.  The paper has no counterpart; this is an interface
 * addition of this library.
 *
 * Same grid, plan, n_iter, d_residual and stream meaning as jac_sweep_dev.
 * The scratch lives in one fixed array of this library's device memory, held
 * on every GPU that loads the library until the process exits.  The call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, with the device current); make that first call
 *     before any stream capture on the device.  The address is kept for the
 *     life of the process: after cudaDeviceReset (which unloads the
 *     library's device memory) do not call this entry point again on that
 *     device in the same process.
 *   - Every call shares the array and overwrites what the previous call left
 *     there; its header is cleared (cudaMemsetAsync) at the start of each
 *     call.  Calls that overlap on the GPU (other streams, other host threads)
 *     race on it: serialise them.
 *   - Pass d_residual (device memory) to receive the residual; with NULL it
 *     lands in the shared array and is lost to the next call.
 *   - A bounded device wait that gives up is reported through the residual:
 *     the kernel writes NaN to d_residual instead of a sum (the error word
 *     itself stays in the shared array and is cleared by the next call).
 *     Callers who need the status code use jac_sweep_dev with their own
 *     workspace and jac_workspace_check.
 * Errors: as jac_sweep_dev, plus JAC_EINVAL when the launch would need more
 * than JAC_NOALLOC_MAX_CTAS CTAs (a device with more SMs than that), and
 * JAC_ECUDA if the array's address cannot be obtained. */
jac_status jac_sweep_dev_noalloc(const jac_grid *g, const jac_plan *plan, int n_iter,
                                 double *d_residual, void *stream);

/* =====================================================================
 * Context API: one grid resident in device memory between the hoisted
 * copy-in and copy-out (Sections 3.2-3.3: data transferred once, outside
 * the outermost loop, and kept present on the device).  A context either
 * owns its device memory (jac_create) or borrows all of it from the caller
 * (jac_create_borrowed).
 * ===================================================================== */
typedef struct jac_ctx jac_ctx;

/* Create a context for an I x J x K grid that owns its device memory: it
 * allocates (cudaMalloc on the current device) the storage of all fields,
 * both state buffers, a FP64 staging array of I*J*K doubles and the sweep
 * workspace, and later the checkpoint tape (jac_tape_begin) and the
 * asynchronous staging arrays (jac_upload_async).  stream: the cudaStream_t
 * every call of this context uses (NULL: legacy default).
 * Errors: JAC_EINVAL (dims < 3, bad precision, omega not finite),
 * JAC_ENOMEM, JAC_ECUDA. */
jac_status jac_create(jac_ctx **out, int I, int J, int K, jac_prec prec,
                      double omega, void *stream);

/* What a borrowed context's workspace must hold besides the sweep scratch
 * and one FP64 staging array: room for jac_upload_async's thirteen staging
 * arrays (async_upload != 0), and a checkpoint tape of up to tape_max
 * sweeps with a checkpoint every tape_C (tape_C = 0 or tape_max = 0: none);
 * a later jac_tape_begin(C, max) fits if it needs no more state arrays
 * (ceil(max / C) + C + 1) than that. */
typedef struct jac_ws_spec {
    int async_upload;
    int tape_C;
    int tape_max;
} jac_ws_spec;

/* Bytes of storage array `which` (JAC_P .. JAC_BND) of an I x J x K grid in
 * precision prec: jac_pitch(I) * J * K elements of its element type.  Host
 * only (no GPU needed).  Errors: JAC_EINVAL. */
jac_status jac_field_bytes(int I, int J, int K, jac_prec prec, int which, size_t *bytes);

/* Bytes of the workspace jac_create_borrowed needs for this grid and spec
 * (NULL spec: no asynchronous staging, no tape): 256 + 8 *
 * JAC_NOALLOC_MAX_CTAS bytes of sweep scratch, I*J*K doubles of staging,
 * 13*I*J*K doubles with async_upload, and (ceil(max/C) + C + 1) state
 * arrays plus 256 bytes for a tape; each part rounded up to 256 bytes.
 * Host only (no GPU needed).  Errors: JAC_EINVAL. */
jac_status jac_workspace_size(int I, int J, int K, jac_prec prec, const jac_ws_spec *spec,
                              size_t *bytes);

/* Create a context that allocates no device memory: the caller passes the
 * grid's fourteen storage arrays in *fields (the jac_grid of the stateless
 * API: dims, precision, omega, the two state buffers p[0], p[1] and
 * coef[JAC_A0..JAC_BND], each of jac_field_bytes bytes, 16-byte aligned)
 * and one workspace of at least jac_workspace_size(spec) bytes, 256-byte
 * aligned.  All of it stays the caller's: it must outlive the context and
 * is not freed by jac_destroy; the context only reads and writes it, on
 * `stream`.  Upload, sweeps, residual, download, tape and adjoint work as
 * for jac_create; the array contents are undefined until the first upload.
 * jac_upload_async needs spec->async_upload, and jac_tape_begin a tape that
 * fits spec; otherwise they return JAC_ENOMEM (jac_set_workspace gives the
 * context a larger workspace).  Errors: JAC_EINVAL (bad grid, pointers,
 * alignment or workspace size), JAC_ECUDA. */
jac_status jac_create_borrowed(jac_ctx **out, const jac_grid *fields, void *stream,
                               void *workspace, size_t ws_bytes, const jac_ws_spec *spec);

/* Give a borrowed context another workspace (for example a larger one
 * before a longer tape).  Synchronises the stream; the tape and the last
 * residual are dropped (the field storage, and with it the state, is kept).
 * The old workspace is no longer used once the call returns.  Errors:
 * JAC_ESTATE for a context from jac_create, JAC_EINVAL as for
 * jac_create_borrowed, JAC_ECUDA. */
jac_status jac_set_workspace(jac_ctx *ctx, void *workspace, size_t ws_bytes, const jac_ws_spec *spec);

/* Free everything the context owns (synchronises its stream); a borrowed
 * context's memory stays the caller's.  NULL is ok.  No paper counterpart. */
jac_status jac_destroy(jac_ctx *ctx);

/* Message of the last failed call on this context ("" if none; NULL: the
 * calling thread's last message).  No paper counterpart. */
const char *jac_last_error(const jac_ctx *ctx);

/* Set the launch plan of later sweeps ({0,0} = defaults).  Paper: launch
 * parameters chosen by rule or by measurement (Section 4, the search by
 * measurement that the autotuner applies to launch plans). */
jac_status jac_set_plan(jac_ctx *ctx, const jac_plan *plan);

/* The hoisted copy-in (Sections 3.2-3.3: all variables copied once, before
 * all GPU work): all thirteen host FP64 arrays, rounded to the storage
 * precision on the device; p0 goes to both state buffers.  Resets the sweep
 * count and the residual.  Returns after the copies are enqueued (host
 * arrays may be reused once the call returns: pageable sources are copied
 * synchronously, and the call synchronises before returning). */
jac_status jac_upload(jac_ctx *ctx, const jac_fields *host);

/* Same as jac_upload without waiting (Sections 3.2-3.3, with the copies
 * overlapping other work): the thirteen host-to-device copies go
 * into thirteen device staging arrays (13*I*J*K doubles, allocated by the
 * first call and owned by the context), and the rounding kernels follow them
 * on the stream, so the copies can run on the copy engine while another
 * stream's sweeps hold the SMs.  The host arrays must stay unchanged until
 * the stream has passed the copies (jac_sync); pinned arrays give
 * asynchronous copies, pageable ones are copied by the driver before the
 * call returns.  Synchronises when a tape is active (the tape is freed).
 * Errors: as jac_upload, JAC_ENOMEM if the staging arrays cannot be
 * allocated. */
jac_status jac_upload_async(jac_ctx *ctx, const jac_fields *host);

/* jac_upload_async for inputs that are FP32 numbers, as dense FP32 host
 * arrays: half the host-to-device bytes of the FP64 form (52 instead of 104
 * bytes per point), the same transfer hoisting (Section 3.2-3.3).  FP64 and
 * FP32 storage keep each value; BF16-stored coefficients are its RNE
 * rounding -- for FP64 inputs that are FP32 numbers, exactly the storage
 * values jac_upload_async gives.  Uses the same staging arrays (a borrowed
 * context needs async_upload in its workspace spec).  Errors: as
 * jac_upload_async. */
jac_status jac_upload_f32_async(jac_ctx *ctx, const jac_fields_f32 *host);

/* Same as jac_upload with the thirteen arrays in device memory (dense FP64);
 * asynchronous.  Paper: data already present on the device (Section 3.3). */
jac_status jac_upload_dev(jac_ctx *ctx, const jac_fields *dev);

/* n_iter sweeps, asynchronous; the residual of the last one is kept on the
 * device.  JAC_ESTATE before the first upload.  Paper: the Himeno Jacobi
 * loop (Section 5.1.1) on arrays present on the device (Section 3.3). */
jac_status jac_sweep(jac_ctx *ctx, int n_iter);

/* Residual of the last sweep (synchronises).  JAC_ESTATE if no sweep ran
 * since the last upload; JAC_ETIMEOUT if a device wait gave up.  Paper: the
 * Himeno residual (Section 5.1.1), the value the result check compares
 * between CPU and GPU runs (Section 4). */
jac_status jac_residual(jac_ctx *ctx, double *out);

/* The hoisted copy-out (Section 3.3: copied back once, after all GPU
 * work): current state as dense FP64 into host memory (I*J*K doubles;
 * synchronises). */
jac_status jac_download(jac_ctx *ctx, double *p_host);

/* Current state as dense FP64 into device memory (asynchronous).  Paper:
 * Section 3.3 (the result stays on the device for later GPU work). */
jac_status jac_download_dev(jac_ctx *ctx, double *p_dev);

/* jac_download and jac_residual without waiting (Section 3.3, overlapped
 * with other work): enqueues the copy of the
 * current state (I*J*K doubles) to p_host and, if res_host is not NULL, of
 * the residual of the last sweep to *res_host.  Both are valid once the
 * stream has passed them (jac_sync); pinned destinations give asynchronous
 * copies.  A device wait that gave up is reported by jac_sync.  Errors:
 * JAC_EINVAL (NULL ctx or p_host), JAC_ESTATE (res_host given and no sweep
 * since the last upload), JAC_ECUDA. */
jac_status jac_download_async(jac_ctx *ctx, double *p_host, double *res_host);

/* jac_download_async with the state as dense FP32 (I*J*K floats): exact for
 * FP32 state storage, RNE of the value for FP64 storage; the residual stays
 * FP64.  Valid after jac_sync.  Errors: as jac_download_async. */
jac_status jac_download_f32_async(jac_ctx *ctx, float *p_host, double *res_host);

/* Paper: Section 5.1.2 (time-limited waits, as for jac_workspace_check).
 * Wait for the context's stream and check the sweep workspace's error word:
 * JAC_ETIMEOUT if a bounded device wait of an earlier sweep gave up (the
 * word is cleared), JAC_ECUDA on a CUDA error. */
jac_status jac_sync(jac_ctx *ctx);

/* Failure-path test aid (host-side injection; the paper has no counterpart:
 * its offload search gives up on a measurement after a time limit, Section
 * 5.1.2, and this library's kernels likewise give up their device waits).
 * The next sweep launch of this context is made with a grid-barrier target
 * between sweeps that no CTA ever reaches, and with wait_ns nanoseconds as
 * the limit of every wait on other warps and CTAs (wait_ns = 0 cancels;
 * at most 2 s).  A launch of at least two sweeps then gives up its waits,
 * every CTA drains its own copies and exits, the workspace error word is
 * set and the residual of the launch is NaN: jac_residual, jac_sync and
 * jac_download report JAC_ETIMEOUT and clear the word.  The state of that
 * launch is partly swept; upload again before sweeping on.  Nothing faults
 * or hangs: every wait is bounded.  Errors: JAC_EINVAL. */
jac_status jac_inject_stall(jac_ctx *ctx, unsigned long long wait_ns);

/* Sweeps completed since the last upload.  No paper counterpart. */
jac_status jac_sweep_count(const jac_ctx *ctx, long long *out);

/* The context's grid descriptor (current state in p[count % 2] order is
 * handled by the context; g->p[0] is the current state after this call).
 * No paper counterpart. */
jac_status jac_get_grid(const jac_ctx *ctx, jac_grid *g);

/* ---------------------------------------------------------------------
 * Adjoint (reverse mode).  For a terminal loss L(p_T), the adjoint of one
 * sweep maps lambda_{t+1} = dL/dp_{t+1} to lambda_t in gather form:
 *   lambda_t[y] = lambda_{t+1}[y] - mu[y] + sum over the 18 neighbours x of y
 *                 of w[x] * (coefficient of p[y] in the update of x),
 * mu[x] = omega bnd[x] lambda_{t+1}[x] on interior x (0 on faces),
 * w[x] = a3[x] mu[x]; its parameter gradients at interior x are
 * dL/dwrk1 += w, dL/da3 += mu s0_t, dL/da0 += w p_t[i+1], dL/dc0 += w p_t[i-1]
 * (and likewise a1, a2, c1, c2), dL/db0 += w * (b0 bracket of p_t), etc.
 * Gradients accumulate in FP64; lambda is kept in the element type of p.
 * There is no paper counterpart: this is the differentiation addition of
 * this library (the sweep itself is the Himeno relaxation of Section 5.1.1).
 * --------------------------------------------------------------------- */

/* One adjoint sweep, stateless.  g describes the grid (coefficients; p[0]
 * and p[1] unused).  p_t: the state before the sweep, lam_in: lambda_{t+1},
 * lam_out: lambda_t (storage layout, element type of p, 16-byte aligned;
 * lam_out != lam_in; every point including faces is written, the row
 * padding may be written too).  g_wrk1, g_a3: dense FP64 (I*J*K) arrays,
 * accumulated (+=).  g_coef: NULL, or nine dense FP64 arrays for a0, a1, a2,
 * b0, b1, b2, c0, c1, c2, accumulated.  kdepth: output planes per work item
 * (0: chosen from the grid).  workspace: at least 256 bytes, 256-byte
 * aligned (a sweep workspace serves); a device wait that gives up sets its
 * error word, which jac_workspace_check reports as JAC_ETIMEOUT.
 * Asynchronous on stream; coefficient arrays must be finite on the faces
 * too (a face's w is 0, and 0 * coefficient must be 0). */
jac_status jac_adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out,
                                double *g_wrk1, double *g_a3, double *const *g_coef, int kdepth,
                                void *workspace, size_t ws_bytes, void *stream);

/* No paper counterpart (differentiation addition).
 * Start a checkpoint tape: the next sweeps (at most max_sweeps, across any
 * number of jac_sweep calls) are recorded by saving the state at the start
 * of every C-sweep segment.  Allocates ceil(max_sweeps/C) + C + 1 state
 * arrays.  A new upload or jac_tape_end discards the tape. */
jac_status jac_tape_begin(jac_ctx *ctx, int C, int max_sweeps);
jac_status jac_tape_end(jac_ctx *ctx);

/* Sweeps recorded on the tape so far.  No paper counterpart. */
jac_status jac_tape_count(const jac_ctx *ctx, int *out);

/* No paper counterpart (differentiation addition).
 * Reverse pass over the taped sweeps for a terminal adjoint lambda_T
 * (dense FP64, device; e.g. p_T - target for L = 1/2 |p_T - target|^2).
 * Each segment is recomputed from its checkpoint into C state buffers, then
 * swept backwards.  Outputs (dense FP64, device, overwritten): g_wrk1,
 * g_a3, and if not NULL the nine arrays of g_coef (a0 a1 a2 b0 b1 b2 c0 c1
 * c2) and g_p0 = dL/d(state at tape start).  The forward state, count and
 * residual are unchanged.  Asynchronous.  JAC_ESTATE without taped sweeps. */
jac_status jac_sweep_adjoint(jac_ctx *ctx, const double *lambda_T, double *g_wrk1, double *g_a3,
                             double *const *g_coef, double *g_p0);

/* ---------------------------------------------------------------------
 * Batched grids: many independent grids of uneven sizes swept together in
 * one persistent launch (a CUDA graph replayed on every call), each grid in
 * its own device storage.  No paper counterpart: the paper offloads one
 * application at a time; this serves many small Himeno-style problems.
 * --------------------------------------------------------------------- */
typedef struct jac_batch jac_batch;

/* No paper counterpart (see above).
 * n grids, dims[3g..3g+2] = I, J, K of grid g (each >= 3).  Allocates every
 * grid's storage (cudaMalloc), a staging array of the largest grid and n
 * residuals.  stream: the cudaStream_t of every call. */
jac_status jac_batch_create(jac_batch **out, int n, const int *dims, jac_prec prec, double omega,
                            void *stream);
jac_status jac_batch_destroy(jac_batch *b);
const char *jac_batch_last_error(const jac_batch *b);

/* Hoisted copy-in of grid g (host or device dense FP64 arrays, as for
 * jac_upload / jac_upload_dev; Sections 3.2-3.3). */
jac_status jac_batch_upload(jac_batch *b, int g, const jac_fields *host);
jac_status jac_batch_upload_dev(jac_batch *b, int g, const jac_fields *dev);

/* Paper: the plan the autotuner finds by measurement (Section 4, the GA's
 * search by measured run time, Section 5.1.2 for its settings).
 * Launch plan: `warps` consumer warps per CTA for the whole launch (4 or 8;
 * 16 with BF16 coefficients; 0 = 8) and per grid a tile width tile_i[g] (a
 * power of two in [16, 128] for FP32/BF16, [16, 64] for FP64; 0 = the width
 * with the best lane use) and k-block depth kdepth[g] (0 = default).  NULL
 * arrays mean all defaults.  The next sweep rebuilds the device tables. */
jac_status jac_batch_set_plan(jac_batch *b, int warps, const int *tile_i, const int *kdepth);

/* The plan grid g will run with (after defaults).  No paper counterpart. */
jac_status jac_batch_grid_plan(const jac_batch *b, int g, jac_plan *out);

/* Paper: the Himeno loop (Section 5.1.1) for many grids at once.
 * n_iter sweeps of every grid in one persistent launch (captured in a CUDA
 * graph on first use for this n_iter and buffer parity, then replayed).
 * If res_host is not NULL it receives the n residuals of the last sweep.
 * Synchronises.  JAC_ETIMEOUT if a bounded device wait gave up. */
jac_status jac_batch_sweep(jac_batch *b, int n_iter, double *res_host);

/* No paper counterpart (measurement contrast).
 * The same sweeps as a loop of per-grid launches, for comparison: one
 * cooperative launch of n_iter sweeps per grid (per_sweep = 0), or one
 * launch per sweep per grid (per_sweep != 0). */
jac_status jac_batch_sweep_loop(jac_batch *b, int n_iter, int per_sweep, double *res_host);

/* Current state of grid g as dense FP64 (host: synchronises; device:
 * async).  Paper: the hoisted copy-out (Section 3.3). */
jac_status jac_batch_download(jac_batch *b, int g, double *p_host);
jac_status jac_batch_download_dev(jac_batch *b, int g, double *p_dev);

/* Work items and CTAs of the current plan (0 before the first sweep), the
 * warp count and the sweeps run so far.  No paper counterpart. */
jac_status jac_batch_info(const jac_batch *b, int *n_items, int *n_ctas, int *warps, long long *sweeps);

/* Paper: what transfer hoisting avoids (Section 3.2: copies inside the
 * loop nest instead of outside it).
 * The contrast to hoisting, for measurement only: for each of n_iter
 * sweeps, copy all thirteen host arrays in (the current host state as p),
 * run one sweep, copy p back out to p_host.  On entry p_host holds p0; on
 * return it holds p_n, and the context's residual is that of sweep n. */
jac_status jac_sweep_unhoisted(jac_ctx *ctx, int n_iter, const jac_fields *host,
                               double *p_host);

#ifdef __cplusplus
}
#endif
#endif /* JACOBI_H */
