// Forward Jacobi sweep kernels and the stateless device API of libjac.
//
// One sweep of the 19-point variable-coefficient relaxation (the Himeno-style
// loop nest of the paper's evaluation, Section 5.1.1; the stencil is written
// out in include/jacobi.h) over a grid resident in device memory.
//
// Kernel design (2.5-D blocking, k-streaming):
//   * a CTA owns a tile of TI x TJ interior points in (i, j) -- one warp per
//     j-row, each lane VI consecutive i points (16 bytes of state) -- and
//     marches along k over `kdepth` planes;
//   * state planes k-1 .. ke arrive in shared memory by TMA (one 3-D tile per
//     plane, (TI + 2H) x (TJ + 2) elements with the i/j halo; H = 16 bytes
//     of columns so every copy starts on a 16-byte boundary), through a ring
//     of kRing slots filled kRing-2 planes ahead of use, each slot with its
//     own mbarrier;
//   * coefficient arrays are streamed straight from HBM with 16-byte (8-byte
//     for BF16) non-allocating loads, issued before the wait on the plane;
//   * i-neighbours come from warp shuffles, j/k-neighbours from the ring;
//   * the update is evaluated in difference form,
//       ss = a3 * (sum_d coef_d (p_nb - p) + b-terms + wrk1) + p (a3 S - 1),
//     S = a0 + a1 + a2 + c0 + c1 + c2, which is algebraically the definition
//     but avoids cancelling s0*a3 against p; for FP32, S is accumulated with
//     Knuth's TwoSum so that a3 S - 1 (a few ulp) keeps its digits;
//   * the last sweep of a call also accumulates ss^2 in FP64 per thread,
//     reduces it over the warp and the CTA (Neumaier), writes one partial per
//     CTA and lets the last CTA to arrive sum the partials in a fixed order,
//     so the residual is bitwise reproducible.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_common.cuh"
#include "jac_internal.h"

namespace jac {

constexpr int kRing = 6;

struct SweepArgs {
    const void *coef[JAC_NFIELDS];
    void *p_out;
    int I, J, K, pitch, kdepth;
    double omega;
    double *partials;
    WsHeader *hdr;
    double *d_res;
    unsigned nblocks;
};

__host__ __device__ constexpr int sweep_vi(int elem) { return 16 / elem; }

template <typename T>
__device__ __forceinline__ void two_sum_acc(T &hi, T &lo, T b)
{
    const T s = hi + b;
    const T bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

__device__ __forceinline__ void neumaier_add(double &s, double &c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// a3 * S - 1 for the six a/c coefficients of one point.
template <typename T>
__device__ __forceinline__ T a3s_minus_one(T a3, T a0, T a1, T a2, T c0, T c1, T c2)
{
    if constexpr (sizeof(T) == 4) {
        T hi = a0, lo = T(0);
        two_sum_acc(hi, lo, c0);
        two_sum_acc(hi, lo, a1);
        two_sum_acc(hi, lo, c1);
        two_sum_acc(hi, lo, a2);
        two_sum_acc(hi, lo, c2);
        T e = fmaf(a3, hi, -1.0f);
        return fmaf(a3, lo, e);
    } else {
        const T S = ((a0 + c0) + (a1 + c1)) + (a2 + c2);
        return fma(a3, S, -1.0);
    }
}

// One row segment of a ring plane: VI values for this lane plus the left and
// right neighbours (shuffles; lanes 0 and 31 read the halo column).
template <typename T, int VI, int H>
__device__ __forceinline__ void load_ext(const T *row, int lane, T (&e)[VI + 2])
{
    const int col = H + VI * lane;
    if constexpr (VI == 4) {
        float4 v = *reinterpret_cast<const float4 *>(row + col);
        e[1] = v.x; e[2] = v.y; e[3] = v.z; e[4] = v.w;
    } else {
        double2 v = *reinterpret_cast<const double2 *>(row + col);
        e[1] = v.x; e[2] = v.y;
    }
    T l = __shfl_up_sync(0xffffffffu, e[VI], 1);
    T r = __shfl_down_sync(0xffffffffu, e[1], 1);
    if (lane == 0) l = row[col - 1];
    if (lane == 31) r = row[col + VI];
    e[0] = l;
    e[VI + 1] = r;
}

template <typename T, int VI, int H>
__device__ __forceinline__ void load_vec(const T *row, int lane, T (&v)[VI])
{
    const int col = H + VI * lane;
    if constexpr (VI == 4) {
        float4 x = *reinterpret_cast<const float4 *>(row + col);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
        double2 x = *reinterpret_cast<const double2 *>(row + col);
        v[0] = x.x; v[1] = x.y;
    }
}

template <typename T, int VI>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VI])
{
    if constexpr (VI == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
}

template <typename T, int TJ>
struct SweepShape {
    static constexpr int VI = 16 / (int)sizeof(T);
    static constexpr int TI = 32 * VI;
    static constexpr int H = VI;
    static constexpr int W = TI + 2 * H;
    static constexpr int ROWS = TJ + 2;
    static constexpr uint32_t SLOT_TX = (uint32_t)(W * ROWS * sizeof(T));
    static constexpr int SLOT_STRIDE = (int)(((SLOT_TX + 127) / 128 * 128) / sizeof(T));
    static constexpr size_t SMEM = (size_t)kRing * SLOT_STRIDE * sizeof(T) + 128;
};

template <typename T, typename C, int TJ, bool RES>
__global__ void __launch_bounds__(32 * TJ)
k_sweep(const __grid_constant__ CUtensorMap tm_in, const SweepArgs a)
{
    using S = SweepShape<T, TJ>;
    constexpr int VI = S::VI, TI = S::TI, H = S::H, W = S::W;
    extern __shared__ unsigned char dsm_raw[];
    T *ring = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~uintptr_t(127));
    __shared__ __align__(8) uint64_t full[kRing];
    __shared__ int s_abort;
    __shared__ int s_last;
    __shared__ double s_part[TJ];

    const int lane = threadIdx.x & 31;
    const int wy = threadIdx.x >> 5;
    const int i0 = blockIdx.x * TI;
    const int j0 = 1 + blockIdx.y * TJ;
    const int kb = 1 + blockIdx.z * a.kdepth;
    const int ke = min(a.K - 1, kb + a.kdepth);
    const int nout = ke - kb;
    const int L = nout + 2;
    const int j = j0 + wy;
    const int ib = i0 + VI * lane;
    const bool row_ok = (j <= a.J - 2);
    const bool vec_ok = row_ok && (ib < a.pitch);

    int issued = 0;  // meaningful in thread 0 only
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) mbar_init(&full[s], 1);
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int pre = min(kRing, L);
        for (int q = 0; q < pre; ++q) {
            mbar_arrive_expect_tx(&full[q], S::SLOT_TX);
            tma_load_3d(ring + q * S::SLOT_STRIDE, &tm_in, &full[q], i0 - H, j0 - 1, kb - 1 + q);
        }
        issued = pre;
    }

    const T omega = (T)a.omega;
    const size_t plane = (size_t)a.J * (size_t)a.pitch;
    size_t off = ((size_t)kb * a.J + (size_t)j) * (size_t)a.pitch + (size_t)ib;
    double acc = 0.0;
    bool interior[VI];
#pragma unroll
    for (int e = 0; e < VI; ++e) interior[e] = row_ok && (ib + e >= 1) && (ib + e <= a.I - 2);

    int m = 0;
    for (; m < nout; ++m, off += plane) {
        T cf[12][VI];
        if (vec_ok) {
#pragma unroll
            for (int q = 1; q <= 12; ++q) {
                const char *base = static_cast<const char *>(a.coef[q]);
                if (q == JAC_WRK1) {
                    CoefLoad<T, T, VI>::run(base + off * sizeof(T), cf[q - 1]);
                } else {
                    CoefLoad<T, C, VI>::run(base + off * sizeof(C), cf[q - 1]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q)
#pragma unroll
                for (int e = 0; e < VI; ++e) cf[q][e] = T(0);
        }

        bool ok = true;
        if (m == 0) {
            ok = mbar_wait_bounded(&full[0], 0u) && mbar_wait_bounded(&full[1], 0u);
        }
        {
            const int q = m + 2;
            ok = ok && mbar_wait_bounded(&full[q % kRing], (uint32_t)((q / kRing) & 1));
        }
        if (!ok) {
            s_abort = 1;
            atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
        }

        const T *Pm = ring + (m % kRing) * S::SLOT_STRIDE;        // plane k-1
        const T *Pk = ring + ((m + 1) % kRing) * S::SLOT_STRIDE;  // plane k
        const T *Pp = ring + ((m + 2) % kRing) * S::SLOT_STRIDE;  // plane k+1
        const int r0 = wy * W, r1 = (wy + 1) * W, r2 = (wy + 2) * W;  // rows j-1, j, j+1

        T ek0[VI + 2], ek1[VI + 2], ek2[VI + 2], em1[VI + 2], ep1[VI + 2];
        T vm0[VI], vm2[VI], vp0[VI], vp2[VI];
        load_ext<T, VI, H>(Pk + r0, lane, ek0);
        load_ext<T, VI, H>(Pk + r1, lane, ek1);
        load_ext<T, VI, H>(Pk + r2, lane, ek2);
        load_ext<T, VI, H>(Pm + r1, lane, em1);
        load_ext<T, VI, H>(Pp + r1, lane, ep1);
        load_vec<T, VI, H>(Pm + r0, lane, vm0);
        load_vec<T, VI, H>(Pm + r2, lane, vm2);
        load_vec<T, VI, H>(Pp + r0, lane, vp0);
        load_vec<T, VI, H>(Pp + r2, lane, vp2);

        T out[VI];
#pragma unroll
        for (int e = 0; e < VI; ++e) {
            const T a0 = cf[JAC_A0 - 1][e], a1 = cf[JAC_A1 - 1][e], a2 = cf[JAC_A2 - 1][e];
            const T a3 = cf[JAC_A3 - 1][e];
            const T b0 = cf[JAC_B0 - 1][e], b1 = cf[JAC_B1 - 1][e], b2 = cf[JAC_B2 - 1][e];
            const T c0 = cf[JAC_C0 - 1][e], c1 = cf[JAC_C1 - 1][e], c2 = cf[JAC_C2 - 1][e];
            const T wk = cf[JAC_WRK1 - 1][e], bnd = cf[JAC_BND - 1][e];
            const T c = ek1[e + 1];
            const T bij = ((ek2[e + 2] - ek0[e + 2]) - ek2[e]) + ek0[e];
            const T bjk = ((vp2[e] - vm2[e]) - vp0[e]) + vm0[e];
            const T bik = ((ep1[e + 2] - em1[e + 2]) - ep1[e]) + em1[e];
            T d = wk;
            d = fma(a0, ek1[e + 2] - c, d);
            d = fma(a1, ek2[e + 1] - c, d);
            d = fma(a2, ep1[e + 1] - c, d);
            d = fma(c0, ek1[e] - c, d);
            d = fma(c1, ek0[e + 1] - c, d);
            d = fma(c2, em1[e + 1] - c, d);
            d = fma(b0, bij, d);
            d = fma(b1, bjk, d);
            d = fma(b2, bik, d);
            const T ec = a3s_minus_one<T>(a3, a0, a1, a2, c0, c1, c2);
            const T ss = fma(a3, d, c * ec) * bnd;
            out[e] = interior[e] ? fma(omega, ss, c) : c;
            if constexpr (RES) {
                if (interior[e]) acc = fma((double)ss, (double)ss, acc);
            }
        }
        if (vec_ok && ok) store_vec<T, VI>(static_cast<T *>(a.p_out) + off, out);

        __syncthreads();
        if (s_abort) break;
        if (threadIdx.x == 0 && issued < L) {
            const int q = issued;
            const int s = q % kRing;
            mbar_arrive_expect_tx(&full[s], S::SLOT_TX);
            tma_load_3d(ring + s * S::SLOT_STRIDE, &tm_in, &full[s], i0 - H, j0 - 1, kb - 1 + q);
            ++issued;
        }
    }

    if (s_abort) {
        // let the copies still in flight land before the CTA's shared memory
        // is released (each wait bounded again)
        if (threadIdx.x == 0) {
            for (int q = m; q < issued; ++q) (void)mbar_wait_bounded(&full[q % kRing], (uint32_t)((q / kRing) & 1));
        }
        __syncthreads();
    }

    if constexpr (RES) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) s_part[wy] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0, c = 0.0;
            for (int w = 0; w < TJ; ++w) neumaier_add(s, c, s_part[w]);
            const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            a.partials[bid] = s + c;
            __threadfence();
            const unsigned prev = atomicAdd(&a.hdr->counter, 1u);
            s_last = (prev == a.nblocks - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double s = 0.0, c = 0.0;
            for (unsigned b = threadIdx.x; b < a.nblocks; b += blockDim.x) neumaier_add(s, c, __ldcg(&a.partials[b]));
            double *tot = reinterpret_cast<double *>(ring);
            tot[threadIdx.x] = s + c;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s2 = 0.0, c2 = 0.0;
                for (unsigned t = 0; t < blockDim.x; ++t) neumaier_add(s2, c2, tot[t]);
                *a.d_res = s2 + c2;
                a.hdr->counter = 0u;
                __threadfence();
            }
        }
    }
}

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
int g_num_sms = 0;

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

template <typename T, int TJ>
jac_status encode_state_map(CUtensorMap *m, void *base, int pitch, int J, int K)
{
    using S = SweepShape<T, TJ>;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)J, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(T), (cuuint64_t)pitch * J * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)S::W, (cuuint32_t)S::ROWS, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = g_encode(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(JAC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return JAC_OK;
}

struct Geometry {
    int vi, ti, nti, ntj, nkb;
    unsigned nblocks;
};

Geometry geometry(const jac_grid *g, int tj, int kdepth)
{
    Geometry G;
    G.vi = g->prec == JAC_F64 ? 2 : 4;
    G.ti = 32 * G.vi;
    G.nti = (g->I - 2) / G.ti + 1;
    G.ntj = (g->J - 2 + tj - 1) / tj;
    G.nkb = (g->K - 2 + kdepth - 1) / kdepth;
    G.nblocks = (unsigned)G.nti * (unsigned)G.ntj * (unsigned)G.nkb;
    return G;
}

int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            g_num_sms = n;
        else
            g_num_sms = 148;
    }
    return g_num_sms;
}

}  // namespace

const char *thread_last_error() { return g_err.c_str(); }
void set_thread_error(const std::string &m) { g_err = m; }

jac_plan resolve_plan(const jac_grid *g, const jac_plan *plan)
{
    jac_plan p{8, 0};
    if (plan && plan->tile_j > 0) p.tile_j = plan->tile_j;
    if (plan && plan->kdepth > 0) {
        p.kdepth = plan->kdepth;
    } else {
        // aim at about 16 CTAs per SM over the whole launch
        const int vi = g->prec == JAC_F64 ? 2 : 4;
        const long cols = (long)((g->I - 2) / (32 * vi) + 1) * ((g->J - 2 + p.tile_j - 1) / p.tile_j);
        const long target = 16L * num_sms();
        long kd = (cols * (g->K - 2) + target - 1) / target;
        if (kd < 2) kd = 2;
        if (kd > g->K - 2) kd = g->K - 2;
        p.kdepth = (int)kd;
    }
    return p;
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

namespace {

using KernelFn = void (*)(const CUtensorMap, const SweepArgs);

template <typename T, typename C, int TJ>
jac_status launch_one(const jac_grid *g, const Geometry &G, int kdepth, int n_iter, double *d_res, WsHeader *hdr,
                      double *partials, cudaStream_t st)
{
    using S = SweepShape<T, TJ>;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_sweep<T, C, TJ, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)S::SMEM);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(k_sweep<T, C, TJ, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)S::SMEM);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute");

    const int pitch = jac_pitch(g->I);
    CUtensorMap maps[2];
    for (int b = 0; b < 2; ++b) {
        jac_status s = encode_state_map<T, TJ>(&maps[b], g->p[b], pitch, g->J, g->K);
        if (s != JAC_OK) return s;
    }
    SweepArgs a;
    for (int q = 0; q < JAC_NFIELDS; ++q) a.coef[q] = g->coef[q];
    a.I = g->I; a.J = g->J; a.K = g->K; a.pitch = pitch; a.kdepth = kdepth;
    a.omega = g->omega;
    a.partials = partials;
    a.hdr = hdr;
    a.d_res = d_res ? d_res : &hdr->residual;
    a.nblocks = G.nblocks;
    const dim3 grid(G.nti, G.ntj, G.nkb), block(32 * TJ);
    for (int t = 0; t < n_iter; ++t) {
        a.p_out = g->p[(t + 1) & 1];
        const bool res = (t == n_iter - 1);
        if (res) k_sweep<T, C, TJ, true><<<grid, block, S::SMEM, st>>>(maps[t & 1], a);
        else k_sweep<T, C, TJ, false><<<grid, block, S::SMEM, st>>>(maps[t & 1], a);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    return JAC_OK;
}

template <typename T, typename C>
jac_status dispatch_tj(const jac_grid *g, const jac_plan &p, const Geometry &G, int n_iter, double *d_res,
                       WsHeader *hdr, double *partials, cudaStream_t st)
{
    switch (p.tile_j) {
    case 4: return launch_one<T, C, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    case 8: return launch_one<T, C, 8>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    case 16: return launch_one<T, C, 16>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    default: return fail(JAC_EINVAL, "tile_j must be 4, 8 or 16");
    }
}

}  // namespace

size_t sweep_workspace_bytes(const jac_grid *g, const jac_plan &p)
{
    Geometry G = geometry(g, p.tile_j, p.kdepth);
    return kWsHeaderBytes + round_up((size_t)G.nblocks * sizeof(double), 256);
}

jac_status sweep_dev(const jac_grid *g, const jac_plan *plan, int n_iter, double *d_residual, void *workspace,
                     size_t ws_bytes, void *stream)
{
    jac_status s = validate_grid(g);
    if (s != JAC_OK) return s;
    if (n_iter < 0) return fail(JAC_EINVAL, "n_iter must be >= 0");
    if (n_iter == 0) return JAC_OK;
    const jac_plan p = resolve_plan(g, plan);
    if (p.tile_j != 4 && p.tile_j != 8 && p.tile_j != 16) return fail(JAC_EINVAL, "tile_j must be 4, 8 or 16");
    if (p.kdepth < 1) return fail(JAC_EINVAL, "kdepth must be >= 1");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15)) return fail(JAC_EINVAL, "bad workspace");
    const size_t need = sweep_workspace_bytes(g, p);
    if (ws_bytes < need) return fail(JAC_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
    const Geometry G = geometry(g, p.tile_j, p.kdepth);
    if (G.nkb > 65535 || G.ntj > 65535) return fail(JAC_EINVAL, "grid too large for the launch shape");
    if ((s = ensure_encode()) != JAC_OK) return s;
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(workspace) + kWsHeaderBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (g->prec) {
    case JAC_F64: return dispatch_tj<double, double>(g, p, G, n_iter, d_residual, hdr, partials, st);
    case JAC_F32: return dispatch_tj<float, float>(g, p, G, n_iter, d_residual, hdr, partials, st);
    case JAC_F32_BF16COEF: return dispatch_tj<float, __nv_bfloat16>(g, p, G, n_iter, d_residual, hdr, partials, st);
    }
    return fail(JAC_EINVAL, "unknown precision");
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
