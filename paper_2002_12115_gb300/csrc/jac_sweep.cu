// Forward Jacobi sweep kernels and the stateless device API of libjac.
//
// One sweep of the 19-point variable-coefficient relaxation (the Himeno-style
// loop nest of the paper's evaluation, Section 5.1.1; the stencil is written
// out in include/jacobi.h) over a grid resident in device memory.
//
// Kernel design (2.5-D blocking, k-streaming, persistent and warp-specialised):
//   * a work item is a tile of TI x TJ points in (i, j) -- one consumer warp
//     per j-row, each lane VI consecutive i points (16 bytes of state) -- over
//     `kdepth` consecutive k-planes; a persistent CTA per SM takes items
//     blockIdx.x, blockIdx.x + gridDim.x, ...;
//   * one producer warp (one lane) issues every TMA copy: the state plane with
//     its i/j halo ((TI + 2H) x (TJ + 2), H = 16 bytes of columns so every copy
//     starts 16-byte aligned) into a ring of RP slots, and the twelve
//     coefficient tiles of each output plane into a ring of RC stages; full
//     and empty mbarriers per slot let it run ahead across item boundaries;
//   * with programmatic dependent launch the next sweep's CTAs start while the
//     previous sweep drains and prefetch coefficient stages (which do not
//     depend on it) before griddepcontrol.wait;
//   * consumers take i-neighbours from warp shuffles and j/k-neighbours from
//     the ring; the update is evaluated in FP32 in difference form,
//       ss = a3 * (sum_d coef_d (p_nb - p) + b-terms + wrk1) + p (a3 S - 1),
//     S = a0 + a1 + a2 + c0 + c1 + c2, algebraically the definition but
//     without cancelling s0*a3 against p; S is accumulated with Knuth's TwoSum
//     so that a3 S - 1 (a few ulp) keeps its digits.  FP64 uses the written
//     form with fused multiply-adds (its rounding is far below the bar, and the
//     FP64 pipe is the bottleneck on this part);
//   * the last sweep of a call sums each lane's squares of one step in FP32,
//     accumulates those in FP64, reduces over the warp and the CTA (Neumaier),
//     writes one partial per CTA and lets the last CTA to arrive sum the
//     partials in a fixed order: the residual is bitwise reproducible.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_common.cuh"
#include "jac_internal.h"

namespace jac {

struct SweepArgs {
    int I, J, K, pitch, kdepth;
    int nti, ntj, nkb, nitems;
    int n_iter;              // sweeps of this launch; sweep t writes p_buf[(t+1) & 1]
    void *p_buf[2];
    double omega;
    double *partials;        // one per CTA
    WsHeader *hdr;
    double *d_res;           // residual of the last sweep (NULL: none)
};

// Tensor maps of one launch: both state buffers and the twelve
// coefficient-like arrays (index q-1 for q = JAC_A0 .. JAC_BND).
struct SweepMaps {
    CUtensorMap p[2];
    CUtensorMap coef[12];
};

// Fast2Sum step (Dekker): hi + b = s + err exactly when |hi| >= |b|.
__device__ __forceinline__ void fast_two_sum_acc(float &hi, float &lo, float b)
{
    const float s = hi + b;
    lo += b - (s - hi);
    hi = s;
}

// a3 * S - 1 with S = a0 + a1 + a2 + c0 + c1 + c2, for FP32 arithmetic.
// Every coefficient lies near 1, so after ordering the first pair the running
// sum always dominates the next term and Fast2Sum is exact: S = hi + lo
// exactly.  When the coefficients are BF16 values (8 significant bits, all
// multiples of 2^-8 below 8) their plain FP32 sum is already exact.
template <bool EXACT_SUM>
__device__ __forceinline__ float a3s_minus_one(float a3, float a0, float a1, float a2, float c0, float c1,
                                               float c2)
{
    if constexpr (EXACT_SUM) {
        const float S = ((a0 + c0) + (a1 + c1)) + (a2 + c2);
        return fmaf(a3, S, -1.0f);
    } else {
        float hi = fmaxf(a0, c0), lo = 0.0f;
        fast_two_sum_acc(hi, lo, fminf(a0, c0));
        fast_two_sum_acc(hi, lo, a1);
        fast_two_sum_acc(hi, lo, c1);
        fast_two_sum_acc(hi, lo, a2);
        fast_two_sum_acc(hi, lo, c2);
        return fmaf(a3, lo, fmaf(a3, hi, -1.0f));
    }
}

__device__ __forceinline__ void neumaier_add(double &s, double &c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// Launch geometry of the sweep kernel for element type T, TJ rows per CTA and
// VI points per lane.
template <typename T, typename C, int TJ, int VI_>
struct SweepShape {
    static constexpr int VI = VI_;                        // points per lane
    static constexpr int TI = 32 * VI;                    // points per row
    static constexpr int H = 16 / (int)sizeof(T);         // halo columns (16 bytes)
    static constexpr int W = TI + 2 * H;                  // state tile row length
    static constexpr int ROWS = TJ + 2;
    static constexpr uint32_t P_TX = (uint32_t)(W * ROWS * sizeof(T));
    static constexpr int P_STRIDE = (int)((P_TX + 127) / 128 * 128);
    static constexpr int RP = 5;                          // state ring: 3 in use + 2 ahead
    static constexpr int TILE_C = TI * TJ * (int)sizeof(C);
    static constexpr int TILE_T = TI * TJ * (int)sizeof(T);
    static constexpr uint32_t C_TX = (uint32_t)(11 * TILE_C + TILE_T);
    static constexpr int C_STRIDE = (int)((C_TX + 127) / 128 * 128);
    static constexpr int BUDGET = 220 * 1024;
    static constexpr int RC_FIT = (BUDGET - RP * P_STRIDE - 1024) / C_STRIDE;
    static constexpr int RC = RC_FIT > 8 ? 8 : RC_FIT;    // coefficient stages
    static constexpr size_t SMEM = (size_t)RP * P_STRIDE + (size_t)RC * C_STRIDE + 128;
    static constexpr int THREADS = 32 * (TJ + 2);         // TJ consumers, state and coefficient producers
    // byte offset of array q (JAC_A0..JAC_BND) inside a coefficient stage
    static __host__ __device__ constexpr int tile_off(int q)
    {
        return (q - 1) * TILE_C + (q > JAC_WRK1 ? TILE_T - TILE_C : 0);
    }
};

// VI consecutive T values from shared memory (8- or 16-byte aligned).
template <typename T, int VI>
__device__ __forceinline__ void lds_vec(const T *p, T (&v)[VI])
{
    if constexpr (sizeof(T) == 4 && VI == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if constexpr (sizeof(T) == 4 && VI == 2) {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x; v[1] = x.y;
    } else {
        static_assert(sizeof(T) == 8 && VI == 2, "unsupported vector shape");
        const double2 x = *reinterpret_cast<const double2 *>(p);
        v[0] = x.x; v[1] = x.y;
    }
}

// VI coefficient values of one lane from a shared-memory tile, as T.
template <typename T, typename C, int VI>
__device__ __forceinline__ void smem_coef(const unsigned char *tile, int idx, T (&o)[VI])
{
    if constexpr (sizeof(C) == 2) {
        // BF16 -> FP32 is exact: the BF16 bits are the high half of the FP32 word.
        if constexpr (VI == 4) {
            const uint2 v = *reinterpret_cast<const uint2 *>(tile + (size_t)idx * 2);
            o[0] = __uint_as_float(v.x << 16);
            o[1] = __uint_as_float(v.x & 0xffff0000u);
            o[2] = __uint_as_float(v.y << 16);
            o[3] = __uint_as_float(v.y & 0xffff0000u);
        } else {
            const unsigned v = *reinterpret_cast<const unsigned *>(tile + (size_t)idx * 2);
            o[0] = __uint_as_float(v << 16);
            o[1] = __uint_as_float(v & 0xffff0000u);
        }
    } else {
        lds_vec<T, VI>(reinterpret_cast<const T *>(tile) + idx, o);
    }
}

// One row segment of a ring plane: VI values for this lane plus the left and
// right neighbours (shuffles; lanes 0 and 31 read the halo column).
template <typename T, int VI, int H>
__device__ __forceinline__ void load_ext(const T *row, int lane, T (&e)[VI + 2])
{
    const int col = H + VI * lane;
    T v[VI];
    lds_vec<T, VI>(row + col, v);
#pragma unroll
    for (int q = 0; q < VI; ++q) e[q + 1] = v[q];
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
    lds_vec<T, VI>(row + H + VI * lane, v);
}

template <typename T, int VI>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VI])
{
    if constexpr (sizeof(T) == 4 && VI == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (sizeof(T) == 4 && VI == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
}

struct Item {
    int i0, j0, kb, nout;
};

__device__ __forceinline__ Item decode_item(const SweepArgs &a, int item, int TI, int TJ)
{
    const int tj = item % a.ntj;
    const int r = item / a.ntj;
    const int ti = r % a.nti;
    const int kk = r / a.nti;
    Item it;
    it.i0 = ti * TI;
    it.j0 = 1 + tj * TJ;
    it.kb = 1 + kk * a.kdepth;
    it.nout = min(a.K - 1, it.kb + a.kdepth) - it.kb;
    return it;
}

// Persistent, warp-specialised sweeps.  One launch runs all n_iter sweeps:
//   * warp TJ (one lane) issues the state-plane TMA copies into a ring of RP
//     slots; before sweep t >= 1 it waits on a grid barrier that every CTA
//     passes once its consumers have stored sweep t-1;
//   * warp TJ+1 (one lane) issues the twelve coefficient tiles of every
//     output plane into a ring of RC stages; the coefficients never change,
//     so it streams on across sweep boundaries and barriers;
//   * warps 0..TJ-1 consume, one j-row each, and release slots through
//     per-slot "empty" mbarriers.
// Each CTA takes the work items blockIdx.x, blockIdx.x + gridDim.x, ... of
// every sweep.  The launch is cooperative, so all CTAs are resident and the
// grid barrier cannot wait on an unscheduled CTA; every wait is bounded.
template <typename T, typename C, int TJ, int VI_>
__global__ void __launch_bounds__(SweepShape<T, C, TJ, VI_>::THREADS, 1)
k_sweep(const __grid_constant__ SweepMaps maps, const SweepArgs a)
{
    using S = SweepShape<T, C, TJ, VI_>;
    constexpr int VI = S::VI, TI = S::TI, H = S::H, W = S::W, RP = S::RP, RC = S::RC;
    constexpr bool EXACT_SUM = sizeof(C) == 2;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) &
                                                            ~uintptr_t(127));
    T *ring_p = reinterpret_cast<T *>(base);
    unsigned char *ring_c = base + (size_t)RP * S::P_STRIDE;
    __shared__ __align__(8) uint64_t p_full[RP], p_empty[RP], c_full[RC], c_empty[RC];
    __shared__ volatile int s_abort;
    __shared__ double s_part[TJ];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int n_iter = a.n_iter;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RP; ++s) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], TJ); }
        for (int s = 0; s < RC; ++s) { mbar_init(&c_full[s], 1); mbar_init(&c_empty[s], TJ); }
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    double acc = 0.0;

    if (warp == TJ + 1) {
        // -------------------------------------------- coefficient producer
        if (lane == 0) {
            uint32_t cc = 0;
            bool ok = true;
            for (int t = 0; t < n_iter && ok; ++t)
                for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
                    const Item it = decode_item(a, item, TI, TJ);
                    for (int m = 0; m < it.nout; ++m, ++cc) {
                        const uint32_t slot = cc % RC, use = cc / RC;
                        if (use > 0 && !mbar_wait_bounded(&c_empty[slot], (use - 1) & 1)) { ok = false; break; }
                        if (s_abort) { ok = false; break; }
                        unsigned char *st = ring_c + (size_t)slot * S::C_STRIDE;
                        mbar_arrive_expect_tx(&c_full[slot], S::C_TX);
                        for (int q = JAC_A0; q <= JAC_BND; ++q)
                            tma_load_3d(st + S::tile_off(q), &maps.coef[q - 1], &c_full[slot], it.i0, it.j0,
                                        it.kb + m);
                    }
                }
            if (!ok) {
                s_abort = 1;
                atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
            }
            // every copy this thread issued must land before the CTA exits
            for (uint32_t s = 0; s < (uint32_t)RC && s < cc; ++s) {
                const uint32_t last = cc - 1 - ((cc - 1 - s) % RC);
                (void)mbar_wait_bounded(&c_full[s], (last / RC) & 1);
            }
        }
    } else if (warp == TJ) {
        // -------------------------------------------------- state producer
        if (lane == 0) {
            uint32_t pc = 0;
            bool ok = true;
            for (int t = 0; t < n_iter && ok; ++t) {
                if (t > 0) {
                    // all CTAs have stored sweep t-1
                    if (!wait_counter_bounded(&a.hdr->gbar, (unsigned)t * gridDim.x)) { ok = false; break; }
                    fence_proxy_async_global();
                }
                const CUtensorMap *pm = (t & 1) ? &maps.p[1] : &maps.p[0];
                for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
                    const Item it = decode_item(a, item, TI, TJ);
                    for (int q = 0; q < it.nout + 2; ++q, ++pc) {
                        const uint32_t slot = pc % RP, use = pc / RP;
                        if (use > 0 && !mbar_wait_bounded(&p_empty[slot], (use - 1) & 1)) { ok = false; break; }
                        if (s_abort) { ok = false; break; }
                        mbar_arrive_expect_tx(&p_full[slot], S::P_TX);
                        tma_load_3d(ring_p + (size_t)slot * (S::P_STRIDE / sizeof(T)), pm, &p_full[slot],
                                    it.i0 - H, it.j0 - 1, it.kb - 1 + q);
                    }
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
            }
            for (uint32_t s = 0; s < (uint32_t)RP && s < pc; ++s) {
                const uint32_t last = pc - 1 - ((pc - 1 - s) % RP);
                (void)mbar_wait_bounded(&p_full[s], (last / RP) & 1);
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int wy = warp;
        const T omega = (T)a.omega;
        const size_t plane = (size_t)a.J * (size_t)a.pitch;
        const int cidx = wy * TI + VI * lane;   // element index inside a coefficient tile
        uint32_t pc = 0, cc = 0;
        bool ok = true;
        for (int t = 0; t < n_iter && ok; ++t) {
            const bool res = (t == n_iter - 1) && (a.d_res != nullptr);
            T *p_out = static_cast<T *>((t & 1) ? a.p_buf[0] : a.p_buf[1]);
            for (int item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
                const Item it = decode_item(a, item, TI, TJ);
                const int j = it.j0 + wy;
                const int ib = it.i0 + VI * lane;
                const bool row_ok = (j <= a.J - 2);
                const bool vec_ok = row_ok && (ib < a.pitch);
                bool interior[VI];
#pragma unroll
                for (int e = 0; e < VI; ++e) interior[e] = row_ok && (ib + e >= 1) && (ib + e <= a.I - 2);
                size_t off = ((size_t)it.kb * a.J + (size_t)j) * (size_t)a.pitch + (size_t)ib;

                for (int m = 0; m < it.nout; ++m, off += plane) {
                    if (m == 0) {
                        ok = mbar_wait_bounded(&p_full[pc % RP], (pc / RP) & 1) &&
                             mbar_wait_bounded(&p_full[(pc + 1) % RP], ((pc + 1) / RP) & 1);
                    }
                    const uint32_t q2 = pc + m + 2;
                    ok = ok && mbar_wait_bounded(&p_full[q2 % RP], (q2 / RP) & 1);
                    ok = ok && mbar_wait_bounded(&c_full[cc % RC], (cc / RC) & 1);
                    ok = __all_sync(0xffffffffu, ok && !s_abort);
                    if (!ok) break;

                    const T *Pm = ring_p + (size_t)((pc + m) % RP) * (S::P_STRIDE / sizeof(T));      // k-1
                    const T *Pk = ring_p + (size_t)((pc + m + 1) % RP) * (S::P_STRIDE / sizeof(T));  // k
                    const T *Pp = ring_p + (size_t)(q2 % RP) * (S::P_STRIDE / sizeof(T));            // k+1
                    const unsigned char *cs = ring_c + (size_t)(cc % RC) * S::C_STRIDE;
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

                    T ca0[VI], ca1[VI], ca2[VI], ca3[VI], cb0[VI], cb1[VI], cb2[VI], cc0[VI], cc1[VI], cc2[VI],
                        cwk[VI], cbn[VI];
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_A0), cidx, ca0);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_A1), cidx, ca1);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_A2), cidx, ca2);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_A3), cidx, ca3);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_B0), cidx, cb0);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_B1), cidx, cb1);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_B2), cidx, cb2);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_C0), cidx, cc0);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_C1), cidx, cc1);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_C2), cidx, cc2);
                    smem_coef<T, T, VI>(cs + S::tile_off(JAC_WRK1), cidx, cwk);
                    smem_coef<T, C, VI>(cs + S::tile_off(JAC_BND), cidx, cbn);

                    T out[VI];
                    float ss2 = 0.0f;   // FP32 sum of this step's (at most 4) squares
#pragma unroll
                    for (int e = 0; e < VI; ++e) {
                        const T c = ek1[e + 1];
                        const T bij = ((ek2[e + 2] - ek0[e + 2]) - ek2[e]) + ek0[e];
                        const T bjk = ((vp2[e] - vm2[e]) - vp0[e]) + vm0[e];
                        const T bik = ((ep1[e + 2] - em1[e + 2]) - ep1[e]) + em1[e];
                        T ss;
                        if constexpr (sizeof(T) == 4) {
                            // difference form with an exact a3*S - 1
                            T d = cwk[e];
                            d = fmaf(ca0[e], ek1[e + 2] - c, d);
                            d = fmaf(ca1[e], ek2[e + 1] - c, d);
                            d = fmaf(ca2[e], ep1[e + 1] - c, d);
                            d = fmaf(cc0[e], ek1[e] - c, d);
                            d = fmaf(cc1[e], ek0[e + 1] - c, d);
                            d = fmaf(cc2[e], em1[e + 1] - c, d);
                            d = fmaf(cb0[e], bij, d);
                            d = fmaf(cb1[e], bjk, d);
                            d = fmaf(cb2[e], bik, d);
                            const T ec = a3s_minus_one<EXACT_SUM>(ca3[e], ca0[e], ca1[e], ca2[e], cc0[e], cc1[e],
                                                                  cc2[e]);
                            ss = fmaf(ca3[e], d, c * ec) * cbn[e];
                        } else {
                            // FP64: the written form, fused
                            T s0 = cwk[e];
                            s0 = fma(ca0[e], ek1[e + 2], s0);
                            s0 = fma(ca1[e], ek2[e + 1], s0);
                            s0 = fma(ca2[e], ep1[e + 1], s0);
                            s0 = fma(cb0[e], bij, s0);
                            s0 = fma(cb1[e], bjk, s0);
                            s0 = fma(cb2[e], bik, s0);
                            s0 = fma(cc0[e], ek1[e], s0);
                            s0 = fma(cc1[e], ek0[e + 1], s0);
                            s0 = fma(cc2[e], em1[e + 1], s0);
                            ss = fma(s0, ca3[e], -c) * cbn[e];
                        }
                        out[e] = interior[e] ? fma(omega, ss, c) : c;
                        if (res && interior[e]) {
                            if constexpr (sizeof(T) == 4) ss2 = fmaf(ss, ss, ss2);
                            else acc = fma(ss, ss, acc);
                        }
                    }
                    if constexpr (sizeof(T) == 4) {
                        if (res) acc += (double)ss2;
                    }
                    if (vec_ok) store_vec<T, VI>(p_out + off, out);
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&c_empty[cc % RC]);
                        mbar_arrive(&p_empty[(pc + m) % RP]);  // plane k-1 is done
                    }
                    ++cc;
                }
                if (!ok) break;
                // the last two planes of the item are done too
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&p_empty[(pc + it.nout) % RP]);
                    mbar_arrive(&p_empty[(pc + it.nout + 1) % RP]);
                }
                pc += it.nout + 2;
            }
            if (!ok) break;
            if (t + 1 < n_iter) {
                // publish this CTA's part of sweep t to every CTA's TMA reads
                fence_proxy_async_global();
                named_barrier_sync(1, 32 * TJ);
                if (threadIdx.x == 0) {
                    __threadfence();
                    atomicAdd(&a.hdr->gbar, 1u);
                }
            }
        }
        if (!ok) {
            s_abort = 1;
            atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
        }
        if (a.d_res != nullptr) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) s_part[wy] = acc;
        }
    }

    // CTA epilogue: the last CTA to finish sums the residual partials in a
    // fixed order and resets the workspace counters for the next launch.
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.d_res != nullptr) {
            double s = 0.0, c = 0.0;
            for (int w = 0; w < TJ; ++w) neumaier_add(s, c, s_part[w]);
            a.partials[blockIdx.x] = s + c;
        }
        __threadfence();
        const unsigned prev = atomicAdd(&a.hdr->counter, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            if (a.d_res != nullptr) {
                double s = 0.0, c = 0.0;
                for (unsigned b = 0; b < gridDim.x; ++b) neumaier_add(s, c, __ldcg(&a.partials[b]));
                *a.d_res = s + c;
            }
            a.hdr->gbar = 0u;
            a.hdr->counter = 0u;
            __threadfence();
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

struct Geometry {
    int vi, ti, nti, ntj, nkb, nitems;
    unsigned nblocks;  // CTAs of the persistent launch
};

int num_sms();

Geometry geometry(const jac_grid *g, int ti, int tj, int kdepth)
{
    Geometry G;
    G.ti = ti;
    G.vi = ti / 32;
    G.nti = (g->I - 2) / G.ti + 1;
    G.ntj = (g->J - 2 + tj - 1) / tj;
    G.nkb = (g->K - 2 + kdepth - 1) / kdepth;
    const long long items = (long long)G.nti * G.ntj * G.nkb;
    G.nitems = items > 0x7fffffffLL ? 0x7fffffff : (int)items;
    G.nblocks = (unsigned)std::min<long long>(items, (long long)num_sms());
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
    // defaults: FP64 64 x 8; FP32 128 x 8; BF16 coefficients 128 x 16
    jac_plan p;
    p.tile_i = (g->prec == JAC_F64) ? 64 : 128;
    p.tile_j = (g->prec == JAC_F32_BF16COEF) ? 16 : 8;
    p.kdepth = 0;
    if (plan && plan->tile_i > 0) p.tile_i = plan->tile_i;
    if (plan && plan->tile_j > 0) p.tile_j = plan->tile_j;
    if (plan && plan->kdepth > 0) {
        p.kdepth = plan->kdepth;
    } else {
        // persistent CTAs, one per SM: about 12 work items per CTA keeps the
        // static round-robin balanced within ~8%, deeper k-blocks re-read
        // fewer halo planes
        const int ti = p.tile_i > 0 ? p.tile_i : 64;
        const int tj = p.tile_j > 0 ? p.tile_j : 8;
        const long cols = (long)((g->I - 2) / ti + 1) * ((g->J - 2 + tj - 1) / tj);
        const long target = 12L * num_sms();
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

template <typename T, typename C, int TJ, int VI>
jac_status launch_one(const jac_grid *g, const Geometry &G, int kdepth, int n_iter, double *d_res, WsHeader *hdr,
                      double *partials, cudaStream_t st)
{
    using S = SweepShape<T, C, TJ, VI>;
    static_assert(S::RC >= 2, "coefficient ring too shallow for the shared-memory budget");
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_sweep<T, C, TJ, VI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    });
    if (attr_err != cudaSuccess) return cuda_fail(attr_err, "cudaFuncSetAttribute");

    const int pitch = jac_pitch(g->I);
    SweepMaps maps;
    for (int b = 0; b < 2; ++b) {
        jac_status s = encode_map(&maps.p[b], g->p[b], sizeof(T), pitch, g->J, g->K, S::W, S::ROWS);
        if (s != JAC_OK) return s;
    }
    for (int q = JAC_A0; q <= JAC_BND; ++q) {
        const size_t elem = (q == JAC_WRK1) ? sizeof(T) : sizeof(C);
        jac_status s = encode_map(&maps.coef[q - 1], g->coef[q], elem, pitch, g->J, g->K, S::TI, TJ);
        if (s != JAC_OK) return s;
    }
    SweepArgs a;
    a.I = g->I; a.J = g->J; a.K = g->K; a.pitch = pitch; a.kdepth = kdepth;
    a.nti = G.nti; a.ntj = G.ntj; a.nkb = G.nkb; a.nitems = G.nitems;
    a.n_iter = n_iter;
    a.p_buf[0] = g->p[0];
    a.p_buf[1] = g->p[1];
    a.omega = g->omega;
    a.partials = partials;
    a.hdr = hdr;
    a.d_res = d_res ? d_res : &hdr->residual;

    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(G.nblocks);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs resident: the grid barrier needs it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_sweep<T, C, TJ, VI>, maps, a);
    if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
    return JAC_OK;
}

// Supported (tile_i, tile_j) shapes per precision; the shared-memory budget
// bounds the coefficient stage (12 tiles of tile_i x tile_j elements).
template <typename T, typename C>
jac_status dispatch_shape(const jac_grid *g, const jac_plan &p, const Geometry &G, int n_iter, double *d_res,
                          WsHeader *hdr, double *partials, cudaStream_t st)
{
    const int ti = p.tile_i, tj = p.tile_j;
    if constexpr (sizeof(T) == 8) {
        if (ti == 64 && tj == 4) return launch_one<T, C, 4, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 64 && tj == 8) return launch_one<T, C, 8, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    } else if constexpr (sizeof(C) == 4) {
        if (ti == 128 && tj == 4) return launch_one<T, C, 4, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 128 && tj == 8) return launch_one<T, C, 8, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 64 && tj == 8) return launch_one<T, C, 8, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 64 && tj == 16) return launch_one<T, C, 16, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    } else {
        if (ti == 128 && tj == 4) return launch_one<T, C, 4, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 128 && tj == 8) return launch_one<T, C, 8, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 128 && tj == 16) return launch_one<T, C, 16, 4>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 64 && tj == 8) return launch_one<T, C, 8, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
        if (ti == 64 && tj == 16) return launch_one<T, C, 16, 2>(g, G, p.kdepth, n_iter, d_res, hdr, partials, st);
    }
    return fail(JAC_EINVAL, "unsupported tile shape " + std::to_string(ti) + "x" + std::to_string(tj) +
                                " for this precision (FP64: 64x4, 64x8; FP32: 128x4, 128x8, 64x8, 64x16; "
                                "BF16 coefficients: 128x4, 128x8, 128x16, 64x8, 64x16)");
}

}  // namespace

size_t sweep_workspace_bytes(const jac_grid *g, const jac_plan &p)
{
    Geometry G = geometry(g, p.tile_i, p.tile_j, p.kdepth);
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
    if ((p.tile_i != 64 && p.tile_i != 128) || (p.tile_j != 4 && p.tile_j != 8 && p.tile_j != 16))
        return fail(JAC_EINVAL, "tile_i must be 64 or 128 and tile_j 4, 8 or 16");
    if (p.kdepth < 1) return fail(JAC_EINVAL, "kdepth must be >= 1");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15)) return fail(JAC_EINVAL, "bad workspace");
    const size_t need = sweep_workspace_bytes(g, p);
    if (ws_bytes < need) return fail(JAC_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes");
    const Geometry G = geometry(g, p.tile_i, p.tile_j, p.kdepth);
    if (G.nitems == 0x7fffffff) return fail(JAC_EINVAL, "grid too large for the launch shape");
    if ((s = ensure_encode()) != JAC_OK) return s;
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(workspace) + kWsHeaderBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (g->prec) {
    case JAC_F64: return dispatch_shape<double, double>(g, p, G, n_iter, d_residual, hdr, partials, st);
    case JAC_F32: return dispatch_shape<float, float>(g, p, G, n_iter, d_residual, hdr, partials, st);
    case JAC_F32_BF16COEF:
        return dispatch_shape<float, __nv_bfloat16>(g, p, G, n_iter, d_residual, hdr, partials, st);
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
