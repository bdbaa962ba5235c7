// Single-grid host side of the forward sweep (the kernel is in
// jac_sweep_kernel.cuh), the storage-layout conversions and the stateless
// device entry points of libjac.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_internal.h"
#include "jac_sweep_kernel.cuh"

namespace jac {

// ------------------------------------------------------- pack / unpack
template <typename C>
__device__ __forceinline__ C cvt_from_f64(double x);
template <>
__device__ __forceinline__ double cvt_from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ float cvt_from_f64<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_f64<__nv_bfloat16>(double x)
{
    return __float2bfloat16_rn(__double2float_rn(x));  // FP64 -> FP32 -> BF16, each RNE
}

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return (double)x; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename C>
__global__ void k_pack(const double *__restrict__ src, C *__restrict__ dst, int I, int J, int K, int pitch)
{
    const size_t total = (size_t)pitch * J * K;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(x % (size_t)pitch);
        const size_t row = x / (size_t)pitch;
        dst[x] = (i < I) ? cvt_from_f64<C>(src[row * I + i]) : cvt_from_f64<C>(0.0);
    }
}

// The same from dense FP32 values (inputs that are FP32 numbers): FP64 and
// FP32 storage keep the value, BF16 storage rounds it RNE -- the storage
// values k_pack gives for the same numbers in FP64.
template <typename C>
__device__ __forceinline__ C cvt_from_f32(float x);
template <>
__device__ __forceinline__ double cvt_from_f32<double>(float x) { return (double)x; }
template <>
__device__ __forceinline__ float cvt_from_f32<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_f32<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename C>
__global__ void k_pack_f32(const float *__restrict__ src, C *__restrict__ dst, int I, int J, int K, int pitch)
{
    const size_t total = (size_t)pitch * J * K;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(x % (size_t)pitch);
        const size_t row = x / (size_t)pitch;
        dst[x] = (i < I) ? cvt_from_f32<C>(src[row * I + i]) : cvt_from_f32<C>(0.0f);
    }
}

// Storage layout to dense FP32 (RNE from FP64 storage; exact otherwise).
template <typename C>
__global__ void k_unpack_f32(const C *__restrict__ src, float *__restrict__ dst, int I, int J, int K, int pitch)
{
    const size_t total = (size_t)I * J * K;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(x % (size_t)I);
        const size_t row = x / (size_t)I;
        dst[x] = (float)to_f64(src[row * pitch + i]);
    }
}

template <typename C>
__global__ void k_unpack(const C *__restrict__ src, double *__restrict__ dst, int I, int J, int K, int pitch)
{
    const size_t total = (size_t)I * J * K;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(x % (size_t)I);
        const size_t row = x / (size_t)I;
        dst[x] = to_f64(src[row * pitch + i]);
    }
}

// ------------------------------------------------------------ host side
namespace {

thread_local std::string g_err;

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

// Per-device attributes, cached by device ordinal (a process may drive
// several GPUs of different kinds).
constexpr int kMaxDevices = 64;
std::mutex g_attr_mu;
int g_num_sms[kMaxDevices] = {};
size_t g_l2_bytes[kMaxDevices] = {};

// Attribute `attr` of the current device, cached in table[dev]; `fallback`
// when the device cannot be queried.
template <typename V>
V device_attr(V *table, cudaDeviceAttr attr, V fallback)
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return fallback;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (dev < kMaxDevices && table[dev] != 0) return table[dev];
    if (cudaDeviceGetAttribute(&v, attr, dev) != cudaSuccess || v <= 0) return fallback;
    if (dev < kMaxDevices) table[dev] = (V)v;
    return (V)v;
}

jac_status fail(jac_status st, const std::string &msg)
{
    g_err = msg;
    return st;
}

jac_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(JAC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

jac_status ensure_encode()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? JAC_OK : fail(JAC_ECUDA, "cuTensorMapEncodeTiled entry point not available");
}

CUtensorMapDataType map_type(size_t elem)
{
    return elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                     : (elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
}

// 3-D tensor map of one storage-layout array with a (bx, by, 1) box.
jac_status encode_map(CUtensorMap *m, const void *base, size_t elem, int pitch, int J, int K, int bx, int by)
{
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)J, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * elem, (cuuint64_t)pitch * J * elem};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = g_encode(m, map_type(elem), 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(JAC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return JAC_OK;
}

// SM count of the current device (148 if it cannot be queried).
int num_sms() { return device_attr<int>(g_num_sms, cudaDevAttrMultiProcessorCount, 148); }

}  // namespace

jac_status encode_box_map(CUtensorMap *m, const void *base, size_t elem, int extent_i, int pitch, int J, int K,
                          int bx, int by)
{
    jac_status s = ensure_encode();
    if (s != JAC_OK) return s;
    const cuuint64_t dims[3] = {(cuuint64_t)extent_i, (cuuint64_t)J, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * elem, (cuuint64_t)pitch * J * elem};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = g_encode(m, map_type(elem), 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(JAC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return JAC_OK;
}

const char *thread_last_error() { return g_err.c_str(); }
void set_thread_error(const std::string &m) { g_err = m; }
int device_sm_count() { return num_sms(); }

// Share of the L2 that the state and the coefficient arrays kept with it
// may claim together.  Measured on GB300 (129 x 129 x 257): 0.6 keeps the
// state and two FP32 arrays (72 MB) and gains 2-3% over the state alone;
// 90 MB and more of evict_last lines thrash and lose up to 15%.
constexpr double kL2KeepFraction = 0.6;

// L2 residency for one launch: keep the state when both buffers fit in half
// the L2; then keep whole coefficient arrays, in a fixed order, while state
// and kept arrays together stay within kL2KeepFraction of the L2.  `points` =
// stored points of all grids.
void set_l2_policy(SweepArgs &a, jac_prec prec, size_t points)
{
    const size_t l2 = device_l2_bytes();
    const size_t state = 2 * points * (prec == JAC_F64 ? 8 : 4);
    a.l2_keep_state = state <= l2 / 2;
    a.l2_keep_coef = 0;
    if (!a.l2_keep_state) return;
    const double budget = kL2KeepFraction * (double)l2;
    static const int order[12] = {JAC_WRK1, JAC_A3, JAC_BND, JAC_A0, JAC_A1, JAC_A2,
                                  JAC_C0,   JAC_C1, JAC_C2,  JAC_B0, JAC_B1, JAC_B2};
    double used = (double)state;
    for (int q : order) {
        const double bytes = (double)points * (double)elem_bytes(prec, q);
        if (used + bytes > budget) break;
        used += bytes;
        a.l2_keep_coef |= 1u << q;
    }
}

size_t device_l2_bytes() { return device_attr<size_t>(g_l2_bytes, cudaDevAttrL2CacheSize, 1); }

int vector_points(jac_prec prec) { return prec == JAC_F64 ? 2 : 4; }

int max_row_fold(jac_prec prec, int tj)
{
    if (prec == JAC_F64) return 4;
    return tj >= 16 ? 4 : 8;
}

bool warps_supported(jac_prec prec, int tj) { return tj == 4 || tj == 8 || (tj == 16 && prec == JAC_F32_BF16COEF); }

// Tile width with the best lane use for an I x J grid when each consumer warp
// takes 32*VI/ti rows (ties go to the wider tile).
int best_tile_i(int I, int J, jac_prec prec, int tj)
{
    const int vi = vector_points(prec), full = 32 * vi;
    int best = full;
    double best_u = -1.0;
    for (int ti = full; ti >= 16; ti >>= 1) {
        const int rw = full / ti;
        if (rw > max_row_fold(prec, tj)) break;
        const int rows = tj * rw;
        const double cover_i = (double)((I - 2) / ti + 1) * ti;
        const double cover_j = (double)((J - 2 + rows - 1) / rows) * rows;
        const double u = (double)(I - 2) * (J - 2) / (cover_i * cover_j);
        if (u > best_u + 1e-12) { best_u = u; best = ti; }
    }
    return best;
}

// k-planes per work item when the plan leaves it open, by what bounds the
// sweep (both rules measured on GB300 over 129x129x257 .. 513x513x1025):
//  * FP32 and BF16 coefficients (memory-bound).  If every item of a sweep
//    fits in one round of CTAs at a depth of at most 256 planes, the smallest
//    such depth: each CTA does one item per sweep, so none waits at the
//    sweep's grid barrier for another's extra item and no ring refills
//    mid-sweep.  Otherwise shallow items of 8 planes: consecutive items are
//    row-adjacent tiles of one thin slab of the grid, so the CTAs at work at
//    any moment read neighbouring rows and share halo planes in L2.
//  * FP64 (bound by the FP64 pipe).  A sweep takes about rounds x (kdepth +
//    h) plane-times, rounds = ceil(items / CTAs), h = 3 for an item's two
//    extra state planes and its ring refill, during which the FP64 pipe
//    idles; the smallest such cost wins (ties: the deeper item); depth 1
//    counts too (33x33x65: 126 one-plane items on 126 SMs, 6.3 us per
//    sweep, against 9.6 us for the 64 two-plane items of depth 2).  Balanced
//    ranges (JAC_KDEPTH_BALANCED) cost ceil(cols nk / CTAs) planes plus h
//    for each tile a CTA's range can touch; they win where whole items
//    leave the last round part-empty (129x129x257: 21.1 -> 22.9, and
//    513x513x1025: 23.9 -> 24.3 Gpoint-updates/s, measured).  For FP32 and
//    BF16 balanced ranges measured 1-5% slower than the rule above.
int default_kdepth(long cols, int nk, int ctas, jac_prec prec)
{
    if (nk <= 1) return 1;
    if (prec != JAC_F64) {
        constexpr int kOneRoundMax = 256, kShallow = 8;
        if (cols <= ctas) {
            const long kblocks = ctas / cols;   // k-blocks that one round holds
            const long kd = std::max<long>(2, (nk + kblocks - 1) / kblocks);
            if (kd <= kOneRoundMax) return (int)std::min<long>(kd, nk);
        }
        return std::min(nk, kShallow);
    }
    const long h = 3;
    int best = 1;
    long best_cost = -1;
    for (int kd = 1; kd <= std::min(nk, 256); ++kd) {
        const long items = cols * ((nk + kd - 1) / kd);
        const long rounds = (items + ctas - 1) / ctas;
        const long cost = rounds * (kd + h);
        if (best_cost < 0 || cost <= best_cost) { best_cost = cost; best = kd; }
    }
    const long per = (cols * nk + ctas - 1) / ctas;               // planes per CTA
    const long bal_cost = per + h * ((per + nk - 1) / nk + 1);   // + h per tile touched
    return bal_cost < best_cost ? JAC_KDEPTH_BALANCED : best;
}

jac_plan resolve_plan(const jac_grid *g, const jac_plan *plan) { return resolve_plan_sms(g, plan, num_sms()); }

// Whether the library's choice for a grid is two-sweep passes: FP32 storage
// whose two state buffers do not stay in L2 (more than half of it; the L2
// of the current device, or 128 MiB without one).  There the single sweep is
// bound by DRAM bandwidth and a pass, which moves half the bytes per sweep,
// is faster; where the state stays in L2 the single sweep is.
bool two_sweep_default(const jac_grid *g)
{
    if (g->prec != JAC_F32) return false;
    size_t l2 = device_l2_bytes();
    if (l2 <= 1) l2 = (size_t)128 << 20;
    const size_t state = 2 * (size_t)jac_pitch(g->I) * (size_t)g->J * (size_t)g->K * 4;
    return state > l2 / 2;
}

// The plan of a grid for a device of `sms` SMs (one CTA per SM).
jac_plan resolve_plan_sms(const jac_grid *g, const jac_plan *plan, int sms)
{
    // defaults: 8 consumer warps (16 for BF16 coefficients on wide grids),
    // the tile width with the best lane use, kdepth from default_kdepth
    const int vi = vector_points(g->prec), full = 32 * vi;
    int tj = 8;
    jac_plan p;
    p.fuse = plan ? plan->fuse : 0;
    if (p.fuse == 0) p.fuse = two_sweep_default(g) ? 2 : 1;
    p.tile_i = (plan && plan->tile_i > 0) ? plan->tile_i : 0;
    p.tile_j = (plan && plan->tile_j > 0) ? plan->tile_j : 0;
    p.kdepth = (plan && (plan->kdepth > 0 || plan->kdepth == JAC_KDEPTH_BALANCED)) ? plan->kdepth : 0;
    if (p.tile_i == 0) {
        if (g->prec == JAC_F32_BF16COEF && p.tile_j == 0 && best_tile_i(g->I, g->J, g->prec, 16) == full) tj = 16;
        if (p.tile_j > 0) {
            // pick the width that turns tile_j into a supported warp count
            p.tile_i = full;
            for (int ti = full; ti >= 16; ti >>= 1) {
                const int rw = full / ti;
                if (p.tile_j % rw == 0 && warps_supported(g->prec, p.tile_j / rw) &&
                    rw <= max_row_fold(g->prec, p.tile_j / rw)) { p.tile_i = ti; break; }
            }
        } else {
            p.tile_i = best_tile_i(g->I, g->J, g->prec, tj);
        }
    }
    if (p.tile_j == 0) p.tile_j = tj * (full / std::max(p.tile_i, 1));
    if (p.kdepth == 0) {
        const int ti = std::max(p.tile_i, 1), rows = std::max(p.tile_j, 1);
        const long cols = (long)((g->I - 2) / ti + 1) * ((g->J - 2 + rows - 1) / rows);
        p.kdepth = default_kdepth(cols, g->K - 2, sms, g->prec);
    }
    return p;
}

// Checks a plan against the kernel shapes; fills rw and the warp count.
jac_status check_plan(jac_prec prec, const jac_plan &p, int *rw_out, int *tj_out)
{
    const int full = 32 * vector_points(prec);
    if (p.tile_i < 16 || p.tile_i > full || (full % p.tile_i) != 0 || (p.tile_i & (p.tile_i - 1)) != 0)
        return fail(JAC_EINVAL, "tile_i must be a power of two in [16, " + std::to_string(full) + "]");
    const int rw = full / p.tile_i;
    if (p.tile_j <= 0 || p.tile_j % rw != 0)
        return fail(JAC_EINVAL, "tile_j must be a multiple of " + std::to_string(rw) + " for tile_i " +
                                    std::to_string(p.tile_i));
    const int tj = p.tile_j / rw;
    if (!warps_supported(prec, tj) || rw > max_row_fold(prec, tj))
        return fail(JAC_EINVAL, "unsupported tile " + std::to_string(p.tile_i) + "x" + std::to_string(p.tile_j) +
                                    ": tile_j / (" + std::to_string(full) + " / tile_i) must be 4 or 8 (16 with "
                                    "BF16 coefficients and tile_i >= 32)");
    if (p.kdepth < 1 && p.kdepth != JAC_KDEPTH_BALANCED)
        return fail(JAC_EINVAL, "kdepth must be >= 1 or JAC_KDEPTH_BALANCED");
    if (p.kdepth == JAC_KDEPTH_BALANCED && prec != JAC_F64)
        return fail(JAC_EINVAL, "balanced ranges (JAC_KDEPTH_BALANCED) are for FP64 storage");
    *rw_out = rw;
    *tj_out = tj;
    return JAC_OK;
}

// Descriptor of one grid for a plan: tensor maps, tiling and item counts.
jac_status build_desc(GridDesc *d, const jac_grid *g, const jac_plan &p, int item_base)
{
    jac_status s = ensure_encode();
    if (s != JAC_OK) return s;
    std::memset(d, 0, sizeof(*d));
    const int vi = vector_points(g->prec), full = 32 * vi;
    const size_t et = (g->prec == JAC_F64) ? 8 : 4;
    const size_t ec = (g->prec == JAC_F64) ? 8 : (g->prec == JAC_F32 ? 4 : 2);
    const int H = (int)(16 / et);
    d->I = g->I; d->J = g->J; d->K = g->K;
    d->pitch = jac_pitch(g->I);
    d->ti = p.tile_i;
    d->rw = full / p.tile_i;
    d->rows = p.tile_j;
    d->kdepth = (p.kdepth == JAC_KDEPTH_BALANCED) ? g->K - 2 : p.kdepth;   // balanced: one item per tile
    d->nti = (g->I - 2) / d->ti + 1;
    d->ntj = (g->J - 2 + d->rows - 1) / d->rows;
    d->nkb = (g->K - 2 + d->kdepth - 1) / d->kdepth;
    const long long items = (long long)d->nti * d->ntj * d->nkb;
    if (items > 0x3fffffffLL) return fail(JAC_EINVAL, "grid too large for the launch shape");
    d->nitems = (int)items;
    d->item_base = item_base;
    d->p_tx = (uint32_t)((d->ti + 2 * H) * (d->rows + 2) * et);
    d->p_buf[0] = g->p[0];
    d->p_buf[1] = g->p[1];
    for (int b = 0; b < 2; ++b)
        if ((s = encode_map(&d->p[b], g->p[b], et, d->pitch, g->J, g->K, d->ti + 2 * H, d->rows + 2)) != JAC_OK)
            return s;
    for (int q = JAC_A0; q <= JAC_BND; ++q)
        if ((s = encode_map(&d->coef[q - 1], g->coef[q], q == JAC_WRK1 ? et : ec, d->pitch, g->J, g->K, d->ti,
                            d->rows)) != JAC_OK)
            return s;
    return JAC_OK;
}

jac_status validate_grid(const jac_grid *g)
{
    if (!g) return fail(JAC_EINVAL, "grid is NULL");
    if (g->I < 3 || g->J < 3 || g->K < 3) return fail(JAC_EINVAL, "every grid dimension must be >= 3");
    if (g->prec != JAC_F64 && g->prec != JAC_F32 && g->prec != JAC_F32_BF16COEF)
        return fail(JAC_EINVAL, "unknown precision");
    if (!std::isfinite(g->omega)) return fail(JAC_EINVAL, "omega must be finite");
    if ((size_t)g->J * g->K > 0x7fffffffull) return fail(JAC_EINVAL, "J*K too large");
    for (int b = 0; b < 2; ++b)
        if (!g->p[b] || (reinterpret_cast<uintptr_t>(g->p[b]) & 15))
            return fail(JAC_EINVAL, "state buffers must be non-NULL and 16-byte aligned");
    if (g->p[0] == g->p[1]) return fail(JAC_EINVAL, "the two state buffers must differ");
    for (int q = JAC_A0; q <= JAC_BND; ++q)
        if (!g->coef[q] || (reinterpret_cast<uintptr_t>(g->coef[q]) & 15))
            return fail(JAC_EINVAL, "coefficient arrays must be non-NULL and 16-byte aligned");
    return JAC_OK;
}

template <typename T, typename C, int TJ, bool BATCH, bool DEEP = false, bool BAL = false>
jac_status launch_sweep_kernel(const GridDesc &d0, const SweepArgs &a, unsigned nblocks, cudaStream_t st)
{
    using S = SweepShape<T, C, TJ, DEEP>;
    static_assert(S::RC >= 2, "coefficient ring too shallow for the shared-memory budget");
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_sweep<T, C, TJ, BATCH, DEEP, BAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute");
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident: the grid barrier needs it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_sweep<T, C, TJ, BATCH, DEEP, BAL>, d0, a);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    return JAC_OK;
}

template <bool BATCH>
jac_status launch_sweep(jac_prec prec, int tj, const GridDesc &d0, const SweepArgs &a, unsigned nblocks,
                        cudaStream_t st)
{
    switch (prec) {
    case JAC_F64:
        if (!BATCH && a.bal_units > 0) {
            if (tj == 4) return launch_sweep_kernel<double, double, 4, false, false, true>(d0, a, nblocks, st);
            if (tj == 8) return launch_sweep_kernel<double, double, 8, false, false, true>(d0, a, nblocks, st);
            break;
        }
        if (tj == 4) return launch_sweep_kernel<double, double, 4, BATCH>(d0, a, nblocks, st);
        if (tj == 8) return launch_sweep_kernel<double, double, 8, BATCH>(d0, a, nblocks, st);
        break;
    case JAC_F32:
        if (tj == 4) return launch_sweep_kernel<float, float, 4, BATCH>(d0, a, nblocks, st);
        if (tj == 8) {
            // a fourth coefficient stage when the state stays in L2
            if (!BATCH && a.l2_keep_state) return launch_sweep_kernel<float, float, 8, false, true>(d0, a, nblocks, st);
            return launch_sweep_kernel<float, float, 8, BATCH>(d0, a, nblocks, st);
        }
        break;
    case JAC_F32_BF16COEF:
        if (tj == 4) return launch_sweep_kernel<float, __nv_bfloat16, 4, BATCH>(d0, a, nblocks, st);
        if (tj == 8) return launch_sweep_kernel<float, __nv_bfloat16, 8, BATCH>(d0, a, nblocks, st);
        if (tj == 16) return launch_sweep_kernel<float, __nv_bfloat16, 16, BATCH>(d0, a, nblocks, st);
        break;
    }
    return fail(JAC_EINVAL, "unsupported warp count " + std::to_string(tj));
}

template jac_status launch_sweep<true>(jac_prec, int, const GridDesc &, const SweepArgs &, unsigned, cudaStream_t);

// Work units of a single-grid sweep: its work items, or for balanced ranges
// its tile-planes; the launch has min(units, SMs) CTAs.
static long long sweep_units(const jac_grid *g, const jac_plan &p)
{
    const int ti = std::max(p.tile_i, 1), rows = std::max(p.tile_j, 1);
    const long long tiles = (long long)((g->I - 2) / ti + 1) * ((g->J - 2 + rows - 1) / rows);
    if (p.kdepth == JAC_KDEPTH_BALANCED) return tiles * (g->K - 2);
    const int kd = std::max(p.kdepth, 1);
    return tiles * ((g->K - 2 + kd - 1) / kd);
}

size_t sweep_workspace_bytes(const jac_grid *g, const jac_plan &p)
{
    const long long blocks = std::min<long long>(sweep_units(g, p), num_sms());
    const size_t single = kWsHeaderBytes + round_up((size_t)blocks * sizeof(double), 256);
    if (g->prec != JAC_F32 || p.fuse == 1) return single;
    return std::max(single, sweep2_workspace_bytes(g));   // two-sweep passes may run
}

// Whether a call of n_iter sweeps runs as two-sweep passes.
bool use_two_sweep_passes(const jac_grid *g, const jac_plan &p, int n_iter)
{
    if (g->prec != JAC_F32 || p.fuse == 1 || n_iter < 4) return false;
    return p.fuse == 2;
}

jac_status sweep_dev(const jac_grid *g, const jac_plan *plan, int n_iter, double *d_residual, void *workspace,
                     size_t ws_bytes, void *stream, const LaunchOpts *opts)
{
    const bool injected = opts && (opts->wait_ns != 0 || opts->gbar_extra != 0);
    jac_status s = validate_grid(g);
    if (s != JAC_OK) return s;
    if (n_iter < 0) return fail(JAC_EINVAL, "n_iter must be >= 0");
    if (n_iter == 0) return JAC_OK;
    const jac_plan p = resolve_plan(g, plan);
    int rw = 0, tj = 0;
    if ((s = check_plan(g->prec, p, &rw, &tj)) != JAC_OK) return s;
    if (p.fuse < 0 || p.fuse > 2) return fail(JAC_EINVAL, "fuse must be 0, 1 or 2");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15)) return fail(JAC_EINVAL, "bad workspace");
    const size_t need = sweep_workspace_bytes(g, p);
    if (ws_bytes < need) return fail(JAC_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
    if (!injected && use_two_sweep_passes(g, p, n_iter)) {
        // an even number of passes keeps the state of n sweeps in p[n % 2];
        // the remaining 0..3 sweeps run singly and give the residual if any
        const int n_pass = (n_iter / 2) & ~1;
        const int rest = n_iter - 2 * n_pass;
        double *res2 = nullptr;
        if (rest == 0) res2 = d_residual ? d_residual : &static_cast<WsHeader *>(workspace)->residual;
        if ((s = sweep2_run(g, 0, n_pass, res2, workspace, ws_bytes, static_cast<cudaStream_t>(stream))) != JAC_OK)
            return s;
        if (rest == 0) return JAC_OK;
        n_iter = rest;
    }
    GridDesc d0;
    if ((s = build_desc(&d0, g, p, 0)) != JAC_OK) return s;
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    SweepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.ngrids = 1;
    a.nitems = d0.nitems;
    a.n_iter = n_iter;
    a.par = 0;
    a.omega = g->omega;
    a.partials = reinterpret_cast<double *>(static_cast<char *>(workspace) + kWsHeaderBytes);
    a.res = d_residual ? d_residual : &hdr->residual;
    a.hdr = hdr;
    if (injected) {
        a.wait_ns = opts->wait_ns;
        a.gbar_extra = opts->gbar_extra;
    }
    const unsigned nblocks = (unsigned)std::min<long long>(sweep_units(g, p), num_sms());
    if (p.kdepth == JAC_KDEPTH_BALANCED) {
        // item numbers b + n G for n below the most tiles one CTA's range touches
        const long long U = sweep_units(g, p), G = nblocks, nk = g->K - 2;
        long long most = 1;
        for (long long b = 0; b < G; ++b) {
            const long long u0 = b * U / G, u1 = (b + 1) * U / G;
            if (u1 > u0) most = std::max(most, (u1 - 1) / nk - u0 / nk + 1);
        }
        a.bal_units = U;
        a.nitems = (int)(G * most);
    }
    set_l2_policy(a, g->prec, (size_t)d0.pitch * g->J * g->K);
    return launch_sweep<false>(g->prec, tj, d0, a, nblocks, static_cast<cudaStream_t>(stream));
}

jac_status pack_dev(int I, int J, int K, jac_prec prec, int which, const double *src, void *dst, cudaStream_t st)
{
    if (I < 3 || J < 3 || K < 3 || which < 0 || which >= JAC_NFIELDS || !src || !dst)
        return fail(JAC_EINVAL, "bad pack arguments");
    const int pitch = jac_pitch(I);
    const size_t total = (size_t)pitch * J * K;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, (size_t)num_sms() * 32);
    switch (elem_bytes(prec, which)) {
    case 8: k_pack<double><<<blocks, threads, 0, st>>>(src, static_cast<double *>(dst), I, J, K, pitch); break;
    case 4: k_pack<float><<<blocks, threads, 0, st>>>(src, static_cast<float *>(dst), I, J, K, pitch); break;
    default:
        k_pack<__nv_bfloat16><<<blocks, threads, 0, st>>>(src, static_cast<__nv_bfloat16 *>(dst), I, J, K, pitch);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JAC_OK : cuda_fail(e, "pack launch");
}

jac_status pack_dev_f32(int I, int J, int K, jac_prec prec, int which, const float *src, void *dst, cudaStream_t st)
{
    if (I < 3 || J < 3 || K < 3 || which < 0 || which >= JAC_NFIELDS || !src || !dst)
        return fail(JAC_EINVAL, "bad pack arguments");
    const int pitch = jac_pitch(I);
    const size_t total = (size_t)pitch * J * K;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, (size_t)num_sms() * 32);
    switch (elem_bytes(prec, which)) {
    case 8: k_pack_f32<double><<<blocks, threads, 0, st>>>(src, static_cast<double *>(dst), I, J, K, pitch); break;
    case 4: k_pack_f32<float><<<blocks, threads, 0, st>>>(src, static_cast<float *>(dst), I, J, K, pitch); break;
    default:
        k_pack_f32<__nv_bfloat16><<<blocks, threads, 0, st>>>(src, static_cast<__nv_bfloat16 *>(dst), I, J, K, pitch);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JAC_OK : cuda_fail(e, "pack launch");
}

jac_status unpack_dev_f32(int I, int J, int K, jac_prec prec, int which, const void *src, float *dst, cudaStream_t st)
{
    if (I < 3 || J < 3 || K < 3 || which < 0 || which >= JAC_NFIELDS || !src || !dst)
        return fail(JAC_EINVAL, "bad unpack arguments");
    const int pitch = jac_pitch(I);
    const size_t total = (size_t)I * J * K;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, (size_t)num_sms() * 32);
    switch (elem_bytes(prec, which)) {
    case 8: k_unpack_f32<double><<<blocks, threads, 0, st>>>(static_cast<const double *>(src), dst, I, J, K, pitch); break;
    case 4: k_unpack_f32<float><<<blocks, threads, 0, st>>>(static_cast<const float *>(src), dst, I, J, K, pitch); break;
    default:
        k_unpack_f32<__nv_bfloat16>
            <<<blocks, threads, 0, st>>>(static_cast<const __nv_bfloat16 *>(src), dst, I, J, K, pitch);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JAC_OK : cuda_fail(e, "unpack launch");
}

jac_status unpack_dev(int I, int J, int K, jac_prec prec, int which, const void *src, double *dst, cudaStream_t st)
{
    if (I < 3 || J < 3 || K < 3 || which < 0 || which >= JAC_NFIELDS || !src || !dst)
        return fail(JAC_EINVAL, "bad unpack arguments");
    const int pitch = jac_pitch(I);
    const size_t total = (size_t)I * J * K;
    const int threads = 256;
    const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, (size_t)num_sms() * 32);
    switch (elem_bytes(prec, which)) {
    case 8: k_unpack<double><<<blocks, threads, 0, st>>>(static_cast<const double *>(src), dst, I, J, K, pitch); break;
    case 4: k_unpack<float><<<blocks, threads, 0, st>>>(static_cast<const float *>(src), dst, I, J, K, pitch); break;
    default:
        k_unpack<__nv_bfloat16>
            <<<blocks, threads, 0, st>>>(static_cast<const __nv_bfloat16 *>(src), dst, I, J, K, pitch);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? JAC_OK : cuda_fail(e, "unpack launch");
}

jac_status workspace_check(void *workspace, cudaStream_t st)
{
    if (!workspace) return fail(JAC_EINVAL, "workspace is NULL");
    WsHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "workspace check");
    if (h.errword != JAC_OK) {
        WsHeader z{};
        e = cudaMemcpyAsync(workspace, &z, sizeof(int) * 2, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return fail((jac_status)h.errword, "a bounded device wait gave up");
    }
    return JAC_OK;
}

}  // namespace jac

// ------------------------------------------------------------- C ABI
extern "C" {

int jac_pitch(int I) { return (int)jac::round_up((size_t)(I < 1 ? 1 : I), 8); }

const char *jac_version(void) { return "libjac 0.1 (sm_103a)"; }

jac_status jac_sweep_workspace_size(const jac_grid *g, const jac_plan *plan, size_t *bytes)
{
    if (!bytes) return jac::fail(JAC_EINVAL, "bytes is NULL");
    jac_status s = jac::validate_grid(g);
    if (s != JAC_OK) return s;
    *bytes = jac::sweep_workspace_bytes(g, jac::resolve_plan(g, plan));
    return JAC_OK;
}

jac_status jac_sweep_dev(const jac_grid *g, const jac_plan *plan, int n_iter, double *d_residual, void *workspace,
                         size_t ws_bytes, void *stream)
{
    return jac::sweep_dev(g, plan, n_iter, d_residual, workspace, ws_bytes, stream);
}

jac_status jac_resolve_plan(const jac_grid *g, const jac_plan *plan, int sm_count, jac_plan *out)
{
    if (!g || !out) return jac::fail(JAC_EINVAL, "NULL argument");
    if (g->I < 3 || g->J < 3 || g->K < 3) return jac::fail(JAC_EINVAL, "every grid dimension must be >= 3");
    if (g->prec != JAC_F64 && g->prec != JAC_F32 && g->prec != JAC_F32_BF16COEF)
        return jac::fail(JAC_EINVAL, "unknown precision");
    if (plan && (plan->tile_j < 0 || plan->tile_i < 0 || plan->fuse < 0 || plan->fuse > 2 ||
                 (plan->kdepth < 0 && plan->kdepth != JAC_KDEPTH_BALANCED)))
        return jac::fail(JAC_EINVAL, "bad plan entry");
    const jac_plan p = jac::resolve_plan_sms(g, plan, sm_count > 0 ? sm_count : jac::device_sm_count());
    int rw = 0, tj = 0;
    jac_status s = jac::check_plan(g->prec, p, &rw, &tj);
    if (s != JAC_OK) return s;
    *out = p;
    return JAC_OK;
}

jac_status jac_workspace_check(void *workspace, void *stream)
{
    return jac::workspace_check(workspace, static_cast<cudaStream_t>(stream));
}

jac_status jac_pack_dev(int I, int J, int K, jac_prec prec, int which, const double *d_src, void *d_dst, void *stream)
{
    return jac::pack_dev(I, J, K, prec, which, d_src, d_dst, static_cast<cudaStream_t>(stream));
}

jac_status jac_unpack_dev(int I, int J, int K, jac_prec prec, int which, const void *d_src, double *d_dst,
                          void *stream)
{
    return jac::unpack_dev(I, J, K, prec, which, d_src, d_dst, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
