// Adjoint (transposed-stencil) sweep of libjac.
//
// Reverse mode of one Jacobi sweep p_{t+1} = F(p_t): given
// lambda_{t+1} = dL/dp_{t+1}, every point y (faces included) gets
//   lambda_t[y] = lambda_{t+1}[y] - mu[y] + sum over the 18 neighbours x of y
//                 of w[x] * (the coefficient of p[y] in the row of x),
// with mu[x] = omega * bnd[x] * lambda_{t+1}[x] on interior points (0 on
// faces, which the sweep does not update) and w[x] = a3[x] * mu[x].  The
// parameter gradients of the same sweep, at interior x, are
//   dL/dwrk1 += w,  dL/da3 += mu * s0_t,  dL/da0 += w * p_t[x+e_i], ...,
//   dL/db0 += w * (the b0 bracket of p_t), ...
// accumulated in FP64 across sweeps.
//
// Kernel design (gather form, 2.5-D k-streaming, one point per thread): a
// CTA of 32 x TJ threads owns a 32 x TJ tile of (i, j) over kdepth planes.
// For each plane it loads, per point of the tile and its one-point halo,
// lambda_{t+1}, a3, bnd, the nine stencil coefficients and p_t, and stores in
// shared memory the nine products coef * w (with halo), p_t (with halo) and
// the centre values needed for the gradients.  A plane is loaded into
// registers one step ahead while the previous step computes, so global
// latency overlaps the gather; a ring of three plane slots holds k-1, k, k+1
// (a fourth slot with one barrier per plane was measured slower: the stores of
// the next plane then contend with the gather for shared memory).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_common.cuh"
#include "jac_internal.h"

namespace jac {

struct AdjArgs {
    const void *coef[JAC_NFIELDS];   // storage layout, JAC_A0..JAC_BND
    const void *p_t;                 // state before the sweep (storage layout, T)
    const void *lam_in;              // lambda_{t+1} (storage layout, T)
    void *lam_out;                   // lambda_t (storage layout, T)
    double *g_wrk1, *g_a3;           // dense FP64, accumulated
    double *g_coef[9];               // dense FP64 a0 a1 a2 b0 b1 b2 c0 c1 c2, or all NULL
    int I, J, K, pitch, kdepth;
    double omega;
};

template <typename T, int TJ>
struct AdjShape {
    static constexpr int TW = 32;           // points per row
    static constexpr int HW = TW + 2;       // row length with halo
    static constexpr int HR = TJ + 2;       // rows with halo
    static constexpr int HALO_TILE = HW * HR;
    static constexpr int CEN_TILE = TW * TJ;
    // halo tiles: products a0 w, c0 w, a1 w, c1 w, a2 w, c2 w, b0 w, b1 w, b2 w and p_t
    enum { QA0, QC0, QA1, QC1, QA2, QC2, QB0, QB1, QB2, PT, NHALO };
    // centre tiles: lambda, mu, w, wrk1 and the nine raw coefficients
    enum { CLAM, CMU, CW, CWK, CA0, CA1, CA2, CB0, CB1, CB2, CC0, CC1, CC2, NCEN };
    static constexpr int SLOT = NHALO * HALO_TILE + NCEN * CEN_TILE;   // elements of T
    static constexpr int NSLOT = 3;          // planes k-1, k, k+1
    static constexpr size_t SMEM = NSLOT * (size_t)SLOT * sizeof(T);
    static constexpr int NHALO_PTS = 2 * HW + 2 * TJ;                  // halo points per plane
};

template <typename T>
struct PointVals {
    T lam, a3, bnd, a0, a1, a2, b0, b1, b2, c0, c1, c2, p, wrk1;
};

template <typename C>
__device__ __forceinline__ float ld_coef(const void *base, size_t off);
template <>
__device__ __forceinline__ float ld_coef<float>(const void *base, size_t off)
{
    return __ldg(static_cast<const float *>(base) + off);
}
template <>
__device__ __forceinline__ float ld_coef<__nv_bfloat16>(const void *base, size_t off)
{
    return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(base) + off));
}

template <typename T, typename C>
__device__ __forceinline__ T ld_c(const void *base, size_t off)
{
    if constexpr (sizeof(T) == 8) return __ldg(static_cast<const double *>(base) + off);
    else return ld_coef<C>(base, off);
}

// Values of point (i, j, k); zeros outside the grid.
template <typename T, typename C>
__device__ __forceinline__ void load_point(const AdjArgs &a, int i, int j, int k, bool centre, PointVals<T> &v)
{
    if (i < 0 || i >= a.I || j < 0 || j >= a.J || k < 0 || k >= a.K) {
        v.lam = v.a3 = v.bnd = v.a0 = v.a1 = v.a2 = v.b0 = v.b1 = v.b2 = v.c0 = v.c1 = v.c2 = v.p = v.wrk1 = T(0);
        return;
    }
    const size_t off = ((size_t)k * a.J + (size_t)j) * (size_t)a.pitch + (size_t)i;
    v.lam = __ldg(static_cast<const T *>(a.lam_in) + off);
    v.p = __ldg(static_cast<const T *>(a.p_t) + off);
    v.a3 = ld_c<T, C>(a.coef[JAC_A3], off);
    v.bnd = ld_c<T, C>(a.coef[JAC_BND], off);
    v.a0 = ld_c<T, C>(a.coef[JAC_A0], off);
    v.a1 = ld_c<T, C>(a.coef[JAC_A1], off);
    v.a2 = ld_c<T, C>(a.coef[JAC_A2], off);
    v.b0 = ld_c<T, C>(a.coef[JAC_B0], off);
    v.b1 = ld_c<T, C>(a.coef[JAC_B1], off);
    v.b2 = ld_c<T, C>(a.coef[JAC_B2], off);
    v.c0 = ld_c<T, C>(a.coef[JAC_C0], off);
    v.c1 = ld_c<T, C>(a.coef[JAC_C1], off);
    v.c2 = ld_c<T, C>(a.coef[JAC_C2], off);
    v.wrk1 = centre ? __ldg(static_cast<const T *>(a.coef[JAC_WRK1]) + off) : T(0);
}

template <typename T, int TJ>
__device__ __forceinline__ void store_point(T *slot, int hpos, int cpos, const PointVals<T> &v, bool interior, T omega)
{
    using S = AdjShape<T, TJ>;
    const T mu = interior ? omega * v.bnd * v.lam : T(0);
    const T w = v.a3 * mu;
    T *h = slot + hpos;
    h[S::QA0 * S::HALO_TILE] = v.a0 * w;
    h[S::QC0 * S::HALO_TILE] = v.c0 * w;
    h[S::QA1 * S::HALO_TILE] = v.a1 * w;
    h[S::QC1 * S::HALO_TILE] = v.c1 * w;
    h[S::QA2 * S::HALO_TILE] = v.a2 * w;
    h[S::QC2 * S::HALO_TILE] = v.c2 * w;
    h[S::QB0 * S::HALO_TILE] = v.b0 * w;
    h[S::QB1 * S::HALO_TILE] = v.b1 * w;
    h[S::QB2 * S::HALO_TILE] = v.b2 * w;
    h[S::PT * S::HALO_TILE] = v.p;
    if (cpos >= 0) {
        T *c = slot + S::NHALO * S::HALO_TILE + cpos;
        c[S::CLAM * S::CEN_TILE] = v.lam;
        c[S::CMU * S::CEN_TILE] = mu;
        c[S::CW * S::CEN_TILE] = w;
        c[S::CWK * S::CEN_TILE] = v.wrk1;
        c[S::CA0 * S::CEN_TILE] = v.a0;
        c[S::CA1 * S::CEN_TILE] = v.a1;
        c[S::CA2 * S::CEN_TILE] = v.a2;
        c[S::CB0 * S::CEN_TILE] = v.b0;
        c[S::CB1 * S::CEN_TILE] = v.b1;
        c[S::CB2 * S::CEN_TILE] = v.b2;
        c[S::CC0 * S::CEN_TILE] = v.c0;
        c[S::CC1 * S::CEN_TILE] = v.c1;
        c[S::CC2 * S::CEN_TILE] = v.c2;
    }
}

__device__ __forceinline__ bool is_interior(const AdjArgs &a, int i, int j, int k)
{
    return i >= 1 && i <= a.I - 2 && j >= 1 && j <= a.J - 2 && k >= 1 && k <= a.K - 2;
}

// Halo point number h (0 <= h < NHALO_PTS) of a tile -> (row, col) in halo
// coordinates: the top and bottom rows, then the left and right columns.
template <int TJ>
__device__ __forceinline__ void halo_rc(int h, int &r, int &c)
{
    constexpr int HW = 34;
    if (h < HW) { r = 0; c = h; }
    else if (h < 2 * HW) { r = TJ + 1; c = h - HW; }
    else if (h < 2 * HW + TJ) { r = 1 + (h - 2 * HW); c = 0; }
    else { r = 1 + (h - 2 * HW - TJ); c = HW - 1; }
}

template <typename T, typename C, int TJ, bool CGRAD>
__global__ void __launch_bounds__(32 * TJ)
k_adjoint(const AdjArgs a)
{
    using S = AdjShape<T, TJ>;
    extern __shared__ __align__(16) unsigned char adj_smem[];
    T *ring = reinterpret_cast<T *>(adj_smem);

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TJ;
    const int kb = blockIdx.z * a.kdepth;
    const int ke = min(a.K, kb + a.kdepth);
    const int i = i0 + tx, j = j0 + ty;
    const T omega = (T)a.omega;
    const int hc = (ty + 1) * S::HW + (tx + 1);   // this thread's point in halo coordinates
    const int cpos = ty * S::TW + tx;
    // the halo point this thread loads, if any
    int hr = 0, hcol = 0;
    const bool has_halo = threadIdx.x < S::NHALO_PTS;
    if (has_halo) halo_rc<TJ>(threadIdx.x, hr, hcol);
    const int hi = i0 + hcol - 1, hj = j0 + hr - 1;

    PointVals<T> vc, vh;
    auto load_plane = [&](int kk) {
        load_point<T, C>(a, i, j, kk, true, vc);
        if (has_halo) load_point<T, C>(a, hi, hj, kk, false, vh);
    };
    auto slot_of = [&](int kk) { return ring + (size_t)(((kk % S::NSLOT) + S::NSLOT) % S::NSLOT) * S::SLOT; };
    auto store_plane = [&](int kk) {
        T *slot = slot_of(kk);
        store_point<T, TJ>(slot, hc, cpos, vc, is_interior(a, i, j, kk), omega);
        if (has_halo) store_point<T, TJ>(slot, hr * S::HW + hcol, -1, vh, is_interior(a, hi, hj, kk), omega);
    };

    // planes kb-1, kb, kb+1 into the ring
    for (int kk = kb - 1; kk <= kb + 1; ++kk) {
        load_plane(kk);
        store_plane(kk);
    }
    __syncthreads();

    const bool mine = (i < a.I) && (j < a.J);
    for (int k = kb; k < ke; ++k) {
        const bool more = (k + 2 <= ke);        // plane k+2 is needed by output k+1
        if (more) load_plane(k + 2);

        const T *Sm = slot_of(k - 1);
        const T *Sk = slot_of(k);
        const T *Sp = slot_of(k + 1);
        if (mine) {
            auto H = [&](const T *sl, int tile, int pos) { return sl[tile * S::HALO_TILE + pos]; };
            auto Cn = [&](const T *sl, int tile) { return sl[S::NHALO * S::HALO_TILE + tile * S::CEN_TILE + cpos]; };
            const constexpr int HWc = S::HW;
            T lam = Cn(Sk, S::CLAM) - Cn(Sk, S::CMU);
            lam += H(Sk, S::QA0, hc - 1);
            lam += H(Sk, S::QC0, hc + 1);
            lam += H(Sk, S::QA1, hc - HWc);
            lam += H(Sk, S::QC1, hc + HWc);
            lam += H(Sm, S::QA2, hc);
            lam += H(Sp, S::QC2, hc);
            lam += ((H(Sk, S::QB0, hc - 1 - HWc) - H(Sk, S::QB0, hc - 1 + HWc)) - H(Sk, S::QB0, hc + 1 - HWc)) +
                   H(Sk, S::QB0, hc + 1 + HWc);
            lam += ((H(Sm, S::QB1, hc - HWc) - H(Sm, S::QB1, hc + HWc)) - H(Sp, S::QB1, hc - HWc)) +
                   H(Sp, S::QB1, hc + HWc);
            lam += ((H(Sm, S::QB2, hc - 1) - H(Sm, S::QB2, hc + 1)) - H(Sp, S::QB2, hc - 1)) + H(Sp, S::QB2, hc + 1);
            const size_t off = ((size_t)k * a.J + (size_t)j) * (size_t)a.pitch + (size_t)i;
            static_cast<T *>(a.lam_out)[off] = lam;

            if (is_interior(a, i, j, k)) {
                const T w = Cn(Sk, S::CW), mu = Cn(Sk, S::CMU);
                const T pc = H(Sk, S::PT, hc);
                const T xp = H(Sk, S::PT, hc + 1), xm = H(Sk, S::PT, hc - 1);
                const T yp = H(Sk, S::PT, hc + HWc), ym = H(Sk, S::PT, hc - HWc);
                const T zp = H(Sp, S::PT, hc), zm = H(Sm, S::PT, hc);
                const T bij = ((H(Sk, S::PT, hc + 1 + HWc) - H(Sk, S::PT, hc + 1 - HWc)) - H(Sk, S::PT, hc - 1 + HWc)) +
                              H(Sk, S::PT, hc - 1 - HWc);
                const T bjk = ((H(Sp, S::PT, hc + HWc) - H(Sm, S::PT, hc + HWc)) - H(Sp, S::PT, hc - HWc)) +
                              H(Sm, S::PT, hc - HWc);
                const T bik = ((H(Sp, S::PT, hc + 1) - H(Sm, S::PT, hc + 1)) - H(Sp, S::PT, hc - 1)) +
                              H(Sm, S::PT, hc - 1);
                (void)pc;
                T s0 = Cn(Sk, S::CWK);
                s0 = fma(Cn(Sk, S::CA0), xp, s0);
                s0 = fma(Cn(Sk, S::CA1), yp, s0);
                s0 = fma(Cn(Sk, S::CA2), zp, s0);
                s0 = fma(Cn(Sk, S::CB0), bij, s0);
                s0 = fma(Cn(Sk, S::CB1), bjk, s0);
                s0 = fma(Cn(Sk, S::CB2), bik, s0);
                s0 = fma(Cn(Sk, S::CC0), xm, s0);
                s0 = fma(Cn(Sk, S::CC1), ym, s0);
                s0 = fma(Cn(Sk, S::CC2), zm, s0);
                const size_t d = ((size_t)k * a.J + (size_t)j) * (size_t)a.I + (size_t)i;
                // each sweep's term is formed in T and accumulated in FP64
                a.g_wrk1[d] += (double)w;
                a.g_a3[d] += (double)(mu * s0);
                if constexpr (CGRAD) {
                    a.g_coef[0][d] += (double)(w * xp);
                    a.g_coef[1][d] += (double)(w * yp);
                    a.g_coef[2][d] += (double)(w * zp);
                    a.g_coef[3][d] += (double)(w * bij);
                    a.g_coef[4][d] += (double)(w * bjk);
                    a.g_coef[5][d] += (double)(w * bik);
                    a.g_coef[6][d] += (double)(w * xm);
                    a.g_coef[7][d] += (double)(w * ym);
                    a.g_coef[8][d] += (double)(w * zm);
                }
            }
        }
        // plane k+2 replaces plane k-1 once every thread is done with it
        __syncthreads();
        if (more) store_plane(k + 2);
        __syncthreads();
    }
}

// ------------------------------------------------------------ host side
namespace {

jac_status adj_fail(jac_status s, const std::string &m)
{
    set_thread_error(m);
    return s;
}

template <typename T, typename C, int TJ, bool CGRAD>
jac_status launch_adj(const AdjArgs &a, cudaStream_t st)
{
    using S = AdjShape<T, TJ>;
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(k_adjoint<T, C, TJ, CGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)S::SMEM);
    });
    if (err != cudaSuccess) return adj_fail(JAC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
    const dim3 grid((a.I + 31) / 32, (a.J + TJ - 1) / TJ, (a.K + a.kdepth - 1) / a.kdepth);
    k_adjoint<T, C, TJ, CGRAD><<<grid, 32 * TJ, S::SMEM, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(JAC_ECUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
    return JAC_OK;
}

template <typename T, typename C, int TJ>
jac_status launch_adj_cg(const AdjArgs &a, bool cgrad, cudaStream_t st)
{
    return cgrad ? launch_adj<T, C, TJ, true>(a, st) : launch_adj<T, C, TJ, false>(a, st);
}

}  // namespace

jac_status adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out, double *g_wrk1,
                            double *g_a3, double *const *g_coef, int kdepth, cudaStream_t st)
{
    jac_status s = validate_grid(g);
    if (s != JAC_OK) return s;
    if (!p_t || !lam_in || !lam_out || !g_wrk1 || !g_a3 || lam_in == lam_out)
        return adj_fail(JAC_EINVAL, "adjoint: state, lambda (two distinct buffers) and gradient arrays are required");
    AdjArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int q = 0; q < JAC_NFIELDS; ++q) a.coef[q] = g->coef[q];
    a.p_t = p_t;
    a.lam_in = lam_in;
    a.lam_out = lam_out;
    a.g_wrk1 = g_wrk1;
    a.g_a3 = g_a3;
    bool cgrad = false;
    if (g_coef) {
        cgrad = true;
        for (int q = 0; q < 9; ++q) {
            a.g_coef[q] = g_coef[q];
            if (!g_coef[q]) return adj_fail(JAC_EINVAL, "adjoint: g_coef needs all nine arrays");
        }
    }
    a.I = g->I; a.J = g->J; a.K = g->K;
    a.pitch = jac_pitch(g->I);
    a.kdepth = kdepth > 0 ? kdepth : 16;
    a.omega = g->omega;
    if ((a.K + a.kdepth - 1) / a.kdepth > 65535 || (a.J + 7) / 8 > 65535)
        return adj_fail(JAC_EINVAL, "adjoint: grid too large for the launch shape");
    switch (g->prec) {
    case JAC_F64: return launch_adj_cg<double, double, 4>(a, cgrad, st);
    case JAC_F32: return launch_adj_cg<float, float, 8>(a, cgrad, st);
    case JAC_F32_BF16COEF: return launch_adj_cg<float, __nv_bfloat16, 8>(a, cgrad, st);
    }
    return adj_fail(JAC_EINVAL, "unknown precision");
}

}  // namespace jac

extern "C" jac_status jac_adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out,
                                           double *g_wrk1, double *g_a3, double *const *g_coef, int kdepth,
                                           void *stream)
{
    return jac::adjoint_step_dev(g, p_t, lam_in, lam_out, g_wrk1, g_a3, g_coef, kdepth,
                                 static_cast<cudaStream_t>(stream));
}
