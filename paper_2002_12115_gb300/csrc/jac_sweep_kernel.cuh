// The forward sweep kernel of libjac, shared by the single-grid entry points
// (jac_sweep.cu) and the batched ones (jac_batch.cu).
//
// One sweep of the 19-point variable-coefficient relaxation (the Himeno-style
// loop nest of the paper's evaluation, Section 5.1.1; the stencil is written
// out in include/jacobi.h) over grids resident in device memory.
//
// Kernel design (2.5-D blocking, k-streaming, persistent, warp-specialised):
//   * one cooperative launch runs all n sweeps of a call, one CTA per SM;
//   * a work item is a tile of ti x rows points in (i, j) of one grid over
//     `kdepth` consecutive k-planes.  Consumer warp w owns rows w*rw .. w*rw +
//     rw-1 of the tile; each of its rw row segments has 32/rw lanes of VI
//     points (i-folding: narrow grids use narrow, tall tiles, so no lane
//     idles on a 17-point row);  CTA b takes items b, b + G, b + 2G, ...;
//   * warp TJ (one lane) issues the state-plane TMA copies -- the plane with
//     its i/j halo, (ti + 2H) x (rows + 2), H = 16 bytes of columns so every
//     copy starts 16-byte aligned -- into a ring of RP slots; before sweep
//     t >= 1 it waits on a grid barrier that every CTA passes once its
//     consumers have stored sweep t-1;
//   * warp TJ+1 (one lane) issues the twelve coefficient tiles of every
//     output plane into a ring of RC stages; coefficients never change, so it
//     streams on across sweep boundaries;
//   * consumers take i-neighbours from segment shuffles and j/k-neighbours
//     from the ring, and release slots through per-slot empty mbarriers;
//   * FP32 update in difference form,
//       ss = a3 * (sum_d coef_d (p_nb - p) + b-terms + wrk1) + p (a3 S - 1),
//     with S = a0 + a1 + a2 + c0 + c1 + c2 summed exactly (Fast2Sum, or a
//     plain sum for BF16 coefficients): algebraically the definition, without
//     cancelling s0*a3 against p.  FP64 uses the written form with FMAs;
//   * the last sweep sums each lane's squares of one step in FP32 and
//     accumulates them in FP64; at every change of grid in a CTA's item list
//     the consumer warps reduce (shuffle, then Neumaier) into one partial per
//     (grid, CTA); the last CTA to finish sums each grid's partials in CTA
//     order, so every residual is bitwise reproducible;
//   * when both state buffers fit in half the L2 (129 MB on GB300), the state
//     copies and stores carry an evict_last policy and the coefficient copies
//     evict_first: the state then stays L2-resident from one sweep to the
//     next and only the coefficients stream from HBM.  Whole coefficient
//     arrays that still fit a resident budget beside the state are marked
//     evict_last as well (l2_keep_coef), so that they too are read from L2
//     on every sweep after the first;
//   * every wait is bounded; on expiry the kernel sets the workspace error
//     word, drains its own copies and returns.
#pragma once

#include "jac_common.cuh"

namespace jac {

// Per-grid descriptor (device memory for batches, kernel parameter for one
// grid).  Tensor maps first: they must be 64-byte aligned.
struct GridDesc {
    CUtensorMap p[2];          // state buffers, box (ti + 2H, rows + 2, 1)
    CUtensorMap coef[12];      // JAC_A0..JAC_BND (index q-1), box (ti, rows, 1)
    void *p_buf[2];
    int I, J, K, pitch;
    int ti, rw, rows;          // tile width, rows per consumer warp, rows per item
    int kdepth, nti, ntj, nkb, nitems, item_base;
    uint32_t p_tx;             // bytes of one state-plane copy
};

struct SweepArgs {
    const GridDesc *descs;     // batched: one per grid
    const int *item_base;      // batched: first item of each grid (ascending)
    int ngrids, nitems, n_iter;
    int par;                   // sweep t reads p[(t + par) & 1], writes the other
    double omega;
    double *partials;          // ngrids * gridDim.x
    double *res;               // residual of the last sweep per grid (NULL: none)
    WsHeader *hdr;
    int l2_keep_state;         // 1: state copies/stores evict_last, coefficients evict_first
    unsigned l2_keep_coef;     // bit q (JAC_A0..JAC_BND): array q's copies evict_last too
    long long bal_units;       // balanced ranges (BAL kernels): tile-planes of the grid
    unsigned long long wait_ns;  // limit of the waits on other warps and CTAs (0: kWaitLimitNs)
    unsigned gbar_extra;       // added to every grid-barrier target: 0, except when a test
                               // makes the barrier unreachable so that its bounded wait runs out
};

// The limit of a launch's progress waits.
__device__ __forceinline__ unsigned long long progress_limit(const SweepArgs &a)
{
    return a.wait_ns ? a.wait_ns : kWaitLimitNs;
}

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

// ss of one point for FP32 arithmetic, in difference form: the coefficients
// times (neighbour - centre), the three b brackets and wrk1, then
// a3 * that + p (a3 S - 1) with a3 S - 1 exact; times bnd.  Shared by the
// single-sweep and the two-sweep kernels, so that both round alike.
// ss_f32_ec takes ec = a3 S - 1 already formed (it depends only on the
// coefficients, so a kernel that updates the same point twice forms it once).
__device__ __forceinline__ float ss_f32_ec(float c, float xp, float xm, float yp, float ym, float zp, float zm,
                                           float bij, float bjk, float bik, float a0, float a1, float a2, float a3,
                                           float b0, float b1, float b2, float c0, float c1, float c2, float wk,
                                           float bnd, float ec)
{
    float d = wk;
    d = fmaf(a0, xp - c, d);
    d = fmaf(a1, yp - c, d);
    d = fmaf(a2, zp - c, d);
    d = fmaf(c0, xm - c, d);
    d = fmaf(c1, ym - c, d);
    d = fmaf(c2, zm - c, d);
    d = fmaf(b0, bij, d);
    d = fmaf(b1, bjk, d);
    d = fmaf(b2, bik, d);
    return fmaf(a3, d, c * ec) * bnd;
}

template <bool EXACT_SUM>
__device__ __forceinline__ float ss_f32(float c, float xp, float xm, float yp, float ym, float zp, float zm,
                                        float bij, float bjk, float bik, float a0, float a1, float a2, float a3,
                                        float b0, float b1, float b2, float c0, float c1, float c2, float wk,
                                        float bnd)
{
    return ss_f32_ec(c, xp, xm, yp, ym, zp, zm, bij, bjk, bik, a0, a1, a2, a3, b0, b1, b2, c0, c1, c2, wk, bnd,
                     a3s_minus_one<EXACT_SUM>(a3, a0, a1, a2, c0, c1, c2));
}

__device__ __forceinline__ void neumaier_add(double &s, double &c, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

// Compile-time shape of a kernel instantiation: TJ consumer warps, VI points
// per lane, row folds rw in {1, .., RW_MAX}.
// DEEP: the larger shared-memory budget, which gives FP32 with 8 consumer
// warps a fourth coefficient stage; it pays where the state stays in L2
// (more coefficient bytes in flight) and costs where the state streams from
// DRAM (the deeper coefficient queue delays the state copies).
template <typename T, typename C, int TJ, bool DEEP = false>
struct SweepShape {
    static constexpr int VI = 16 / (int)sizeof(T);        // points per lane (16 bytes)
    static constexpr int TI = 32 * VI;                     // tile width at rw = 1
    static constexpr int H = 16 / (int)sizeof(T);          // halo columns (16 bytes)
    static constexpr int RW_MAX = (sizeof(T) == 8) ? 4 : (TJ >= 16 ? 4 : 8);
    static constexpr int p_elems(int rw) { return (TI / rw + 2 * H) * (TJ * rw + 2); }
    static constexpr int max2(int a, int b) { return a > b ? a : b; }
    static constexpr int P_MAX =
        max2(max2(p_elems(1), p_elems(2)), max2(p_elems(4), RW_MAX >= 8 ? p_elems(8) : 0));
    static constexpr int P_STRIDE = (int)((P_MAX * sizeof(T) + 127) / 128 * 128);   // bytes
    static constexpr int RP = 5;                           // state ring: 3 in use + 2 ahead
    static constexpr int TILE_C = TI * TJ * (int)sizeof(C);   // a coefficient tile (any rw)
    static constexpr int TILE_T = TI * TJ * (int)sizeof(T);
    static constexpr uint32_t C_TX = (uint32_t)(11 * TILE_C + TILE_T);
    static constexpr int C_STRIDE = (int)((C_TX + 127) / 128 * 128);
    static constexpr int BUDGET = (DEEP ? 226 : 220) * 1024;
    static constexpr int RC_FIT = (BUDGET - RP * P_STRIDE - 1024) / C_STRIDE;
    static constexpr int RC = RC_FIT > 8 ? 8 : RC_FIT;     // coefficient stages
    static constexpr size_t SMEM = (size_t)RP * P_STRIDE + (size_t)RC * C_STRIDE + 128;
    static constexpr int THREADS = 32 * (TJ + 2);          // TJ consumers, state and coefficient producers
    static __host__ __device__ constexpr int tile_off(int q)
    {
        return (q - 1) * TILE_C + (q > JAC_WRK1 ? TILE_T - TILE_C : 0);
    }
};

template <typename T, int VI>
__device__ __forceinline__ void lds_vec(const T *p, T (&v)[VI])
{
    if constexpr (sizeof(T) == 4 && VI == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
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
        const uint2 v = *reinterpret_cast<const uint2 *>(tile + (size_t)idx * 2);
        o[0] = __uint_as_float(v.x << 16);
        o[1] = __uint_as_float(v.x & 0xffff0000u);
        o[2] = __uint_as_float(v.y << 16);
        o[3] = __uint_as_float(v.y & 0xffff0000u);
    } else {
        lds_vec<T, VI>(reinterpret_cast<const T *>(tile) + idx, o);
    }
}

// VI values of this lane's row segment plus the left and right neighbours:
// shuffles within segments of `seg` lanes; the segment's end lanes read the
// halo column.
template <typename T, int VI, int H>
__device__ __forceinline__ void load_ext(const T *row, int lin, int seg, T (&e)[VI + 2])
{
    const int col = H + VI * lin;
    T v[VI];
    lds_vec<T, VI>(row + col, v);
#pragma unroll
    for (int q = 0; q < VI; ++q) e[q + 1] = v[q];
    T l = __shfl_up_sync(0xffffffffu, e[VI], 1, seg);
    T r = __shfl_down_sync(0xffffffffu, e[1], 1, seg);
    if (lin == 0) l = row[col - 1];
    if (lin == seg - 1) r = row[col + VI];
    e[0] = l;
    e[VI + 1] = r;
}

template <typename T, int VI>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VI], uint64_t policy)
{
    if constexpr (sizeof(T) == 4 && VI == 4) {
        st_v4_hint(p, v[0], v[1], v[2], v[3], policy);
    } else {
        st_v2d_hint(p, v[0], v[1], policy);
    }
}

struct Item {
    const GridDesc *D;
    int g, i0, j0, kb, nout;
};

template <bool BATCH>
__device__ __forceinline__ Item decode_item(const SweepArgs &a, const GridDesc *d0, int item)
{
    Item it;
    int local = item;
    if constexpr (BATCH) {
        int lo = 0, hi = a.ngrids - 1;   // last grid whose first item <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&a.item_base[mid]) <= item) lo = mid;
            else hi = mid - 1;
        }
        it.g = lo;
        it.D = a.descs + lo;
        local = item - __ldg(&a.item_base[lo]);
    } else {
        it.g = 0;
        it.D = d0;
    }
    const GridDesc *D = it.D;
    const int ntj = D->ntj, nti = D->nti;
    const int tj = local % ntj;
    const int r = local / ntj;
    const int ti = r % nti;
    const int kk = r / nti;
    it.i0 = ti * D->ti;
    it.j0 = 1 + tj * D->rows;
    it.kb = 1 + kk * D->kdepth;
    it.nout = min(D->K - 1, it.kb + D->kdepth) - it.kb;
    return it;
}

// Balanced ranges (single grid, a.bal_units = U tile-planes; tile
// t = tj + ntj * ti covers tile-planes t (K-2) .. (t+1) (K-2) - 1): CTA b
// takes the tile-planes b U / G .. (b+1) U / G - 1, as one item per tile
// they touch.  Its n-th such item has the number b + n G; numbers past its
// last item are empty (nout = 0).
__device__ __forceinline__ Item balanced_item(const SweepArgs &a, const GridDesc *d0, int item)
{
    const long long G = gridDim.x, b = blockIdx.x, U = a.bal_units;
    const long long u0 = b * U / G, u1 = (b + 1) * U / G;
    const long long nk = d0->K - 2;
    const int n = (item - (int)blockIdx.x) / (int)gridDim.x;
    const long long start = (n == 0) ? u0 : (u0 / nk + n) * nk;
    const long long tile = start / nk;
    Item it;
    it.D = d0;
    it.g = 0;
    it.i0 = (int)(tile / d0->ntj) * d0->ti;
    it.j0 = 1 + (int)(tile % d0->ntj) * d0->rows;
    it.kb = 1 + (int)(start - tile * nk);
    it.nout = (start < u1) ? (int)(min(u1, (tile + 1) * nk) - start) : 0;
    return it;
}

template <bool BATCH, bool BAL>
__device__ __forceinline__ Item get_item(const SweepArgs &a, const GridDesc *d0, int item)
{
    if constexpr (BAL) return balanced_item(a, d0, item);
    else return decode_item<BATCH>(a, d0, item);
}

// BAL: work items from balanced ranges (single grid) instead of fixed-depth
// items; a separate instantiation, so that the fixed-depth kernels are
// compiled exactly as without it.
template <typename T, typename C, int TJ, bool BATCH, bool DEEP = false, bool BAL = false>
__global__ void __launch_bounds__(SweepShape<T, C, TJ, DEEP>::THREADS, 1)
k_sweep(const __grid_constant__ GridDesc d0, const SweepArgs a)
{
    static_assert(!(BATCH && BAL), "balanced ranges are for single grids");
    using S = SweepShape<T, C, TJ, DEEP>;
    constexpr int VI = S::VI, H = S::H, RP = S::RP, RC = S::RC;
    constexpr bool EXACT_SUM = sizeof(C) == 2;
    extern __shared__ unsigned char dsm_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm_raw) + 127) &
                                                            ~uintptr_t(127));
    unsigned char *ring_c = base + (size_t)RP * S::P_STRIDE;
    __shared__ __align__(8) uint64_t p_full[RP], p_empty[RP], c_full[RC], c_empty[RC], cons_bar;
    __shared__ volatile int s_abort;
    __shared__ double s_part[TJ];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int n_iter = a.n_iter;
    const int G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RP; ++s) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], TJ); }
        for (int s = 0; s < RC; ++s) { mbar_init(&c_full[s], 1); mbar_init(&c_empty[s], TJ); }
        mbar_init(&cons_bar, TJ);
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == TJ + 1) {
        // -------------------------------------------- coefficient producer
        if (lane == 0) {
            const uint64_t pol = l2_policy(a.l2_keep_state ? -1 : 0);
            const uint64_t pol_keep = l2_policy(1);
            const unsigned long long wlim = progress_limit(a);
            uint32_t cc = 0;
            bool ok = true;
            for (int t = 0; t < n_iter && ok; ++t)
                for (int item = blockIdx.x; item < a.nitems && ok; item += G) {
                    const Item it = get_item<BATCH, BAL>(a, &d0, item);
                    if (BAL && it.nout == 0) continue;
                    for (int m = 0; m < it.nout; ++m, ++cc) {
                        const uint32_t slot = cc % RC, use = cc / RC;
                        if (use > 0 && !mbar_wait_bounded(&c_empty[slot], (use - 1) & 1, wlim)) { ok = false; break; }
                        if (s_abort) { ok = false; break; }
                        unsigned char *st = ring_c + (size_t)slot * S::C_STRIDE;
                        mbar_arrive_expect_tx(&c_full[slot], S::C_TX);
                        for (int q = JAC_A0; q <= JAC_BND; ++q)
                            tma_load_3d_hint(st + S::tile_off(q), &it.D->coef[q - 1], &c_full[slot], it.i0,
                                             it.j0, it.kb + m, ((a.l2_keep_coef >> q) & 1u) ? pol_keep : pol);
                    }
                }
            if (!ok) {
                s_abort = 1;
                atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
            }
            for (uint32_t s = 0; s < (uint32_t)RC && s < cc; ++s) {   // land every issued copy
                const uint32_t last = cc - 1 - ((cc - 1 - s) % RC);
                (void)mbar_wait_bounded(&c_full[s], (last / RC) & 1);
            }
        }
    } else if (warp == TJ) {
        // -------------------------------------------------- state producer
        if (lane == 0) {
            const uint64_t pol = l2_policy(a.l2_keep_state ? 1 : 0);
            const unsigned long long wlim = progress_limit(a);
            uint32_t pc = 0;
            bool ok = true;
            for (int t = 0; t < n_iter && ok; ++t) {
                if (t > 0) {
                    if (!wait_counter_bounded(&a.hdr->gbar, (unsigned)t * G + a.gbar_extra, wlim)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_global();
                }
                const int rb = (t + a.par) & 1;
                for (int item = blockIdx.x; item < a.nitems && ok; item += G) {
                    const Item it = get_item<BATCH, BAL>(a, &d0, item);
                    if (BAL && it.nout == 0) continue;
                    const CUtensorMap *pm = rb ? &it.D->p[1] : &it.D->p[0];
                    const uint32_t tx = it.D->p_tx;
                    for (int q = 0; q < it.nout + 2; ++q, ++pc) {
                        const uint32_t slot = pc % RP, use = pc / RP;
                        if (use > 0 && !mbar_wait_bounded(&p_empty[slot], (use - 1) & 1, wlim)) { ok = false; break; }
                        if (s_abort) { ok = false; break; }
                        mbar_arrive_expect_tx(&p_full[slot], tx);
                        tma_load_3d_hint(base + (size_t)slot * S::P_STRIDE, pm, &p_full[slot], it.i0 - H,
                                         it.j0 - 1, it.kb - 1 + q, pol);
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
        const uint64_t st_pol = l2_policy(a.l2_keep_state ? 1 : 0);
        const unsigned long long wlim = progress_limit(a);
        uint32_t pc = 0, cc = 0;
        bool ok = true;
        double acc = 0.0;
        int g_open = -1;            // grid whose residual partial is being accumulated
        uint32_t sync_phase = 0;
        // barrier of the consumer warps (an mbarrier, so that the wait is bounded)
        auto cons_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(&cons_bar);
            const bool r = mbar_wait_bounded(&cons_bar, sync_phase & 1, wlim);
            ++sync_phase;
            return __all_sync(0xffffffffu, r);
        };
        // one partial per (grid, CTA): reduce the warps' sums and store it
        auto flush = [&](int g) -> bool {
            double v = acc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_part[wy] = v;
            if (!cons_sync()) return false;
            if (threadIdx.x == 0) {
                double s = 0.0, c = 0.0;
                for (int w = 0; w < TJ; ++w) neumaier_add(s, c, s_part[w]);
                a.partials[(size_t)g * G + blockIdx.x] = s + c;
            }
            acc = 0.0;
            return cons_sync();
        };
        // grids this CTA has no item of get an explicit zero partial
        auto zero_range = [&](int g0, int g1) {
            if (threadIdx.x == 0)
                for (int g = g0; g < g1; ++g) a.partials[(size_t)g * G + blockIdx.x] = 0.0;
        };

        for (int t = 0; t < n_iter && ok; ++t) {
            const bool res = (t == n_iter - 1) && (a.res != nullptr);
            const int wb = (t + 1 + a.par) & 1;
            for (int item = blockIdx.x; item < a.nitems && ok; item += G) {
                const Item it = get_item<BATCH, BAL>(a, &d0, item);
                if (BAL && it.nout == 0) continue;
                const GridDesc *D = it.D;
                if (res && it.g != g_open) {
                    if (g_open >= 0 && !flush(g_open)) { ok = false; break; }
                    zero_range(g_open + 1, it.g);
                    g_open = it.g;
                }
                const int rw = D->rw, seg = 32 / rw;
                const int rin = lane / seg, lin = lane - rin * seg;
                const int row = wy * rw + rin;                  // row of the item, 0 .. rows-1
                const int j = it.j0 + row;
                const int ib = it.i0 + VI * lin;
                const int I = D->I, J = D->J, pitch = D->pitch;
                const int W = D->ti + 2 * H;                    // ring row length
                const bool row_ok = (j <= J - 2);
                const bool vec_ok = row_ok && (ib < pitch);
                bool interior[VI];
#pragma unroll
                for (int e = 0; e < VI; ++e) interior[e] = row_ok && (ib + e >= 1) && (ib + e <= I - 2);
                T *p_out = static_cast<T *>(wb ? D->p_buf[1] : D->p_buf[0]);
                const size_t plane = (size_t)J * (size_t)pitch;
                size_t off = ((size_t)it.kb * J + (size_t)j) * (size_t)pitch + (size_t)ib;
                const int cidx = row * D->ti + VI * lin;        // element index in a coefficient tile
                const int r0 = row * W, r1 = (row + 1) * W, r2 = (row + 2) * W;   // rows j-1, j, j+1

                for (int m = 0; m < it.nout; ++m, off += plane) {
                    if (m == 0) {
                        ok = mbar_wait_bounded(&p_full[pc % RP], (pc / RP) & 1, wlim) &&
                             mbar_wait_bounded(&p_full[(pc + 1) % RP], ((pc + 1) / RP) & 1, wlim);
                    }
                    const uint32_t q2 = pc + m + 2;
                    ok = ok && mbar_wait_bounded(&p_full[q2 % RP], (q2 / RP) & 1, wlim);
                    ok = ok && mbar_wait_bounded(&c_full[cc % RC], (cc / RC) & 1, wlim);
                    ok = __all_sync(0xffffffffu, ok && !s_abort);
                    if (!ok) break;

                    const T *Pm = reinterpret_cast<const T *>(base + (size_t)((pc + m) % RP) * S::P_STRIDE);
                    const T *Pk = reinterpret_cast<const T *>(base + (size_t)((pc + m + 1) % RP) * S::P_STRIDE);
                    const T *Pp = reinterpret_cast<const T *>(base + (size_t)(q2 % RP) * S::P_STRIDE);
                    const unsigned char *cs = ring_c + (size_t)(cc % RC) * S::C_STRIDE;

                    T ek0[VI + 2], ek1[VI + 2], ek2[VI + 2], em1[VI + 2], ep1[VI + 2];
                    T vm0[VI], vm2[VI], vp0[VI], vp2[VI];
                    load_ext<T, VI, H>(Pk + r0, lin, seg, ek0);
                    load_ext<T, VI, H>(Pk + r1, lin, seg, ek1);
                    load_ext<T, VI, H>(Pk + r2, lin, seg, ek2);
                    load_ext<T, VI, H>(Pm + r1, lin, seg, em1);
                    load_ext<T, VI, H>(Pp + r1, lin, seg, ep1);
                    lds_vec<T, VI>(Pm + r0 + H + VI * lin, vm0);
                    lds_vec<T, VI>(Pm + r2 + H + VI * lin, vm2);
                    lds_vec<T, VI>(Pp + r0 + H + VI * lin, vp0);
                    lds_vec<T, VI>(Pp + r2 + H + VI * lin, vp2);

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
                            ss = ss_f32<EXACT_SUM>(c, ek1[e + 2], ek1[e], ek2[e + 1], ek0[e + 1], ep1[e + 1],
                                                   em1[e + 1], bij, bjk, bik, ca0[e], ca1[e], ca2[e], ca3[e],
                                                   cb0[e], cb1[e], cb2[e], cc0[e], cc1[e], cc2[e], cwk[e], cbn[e]);
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
                    if (vec_ok) store_vec<T, VI>(p_out + off, out, st_pol);
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
            if (res) {
                if (g_open >= 0 && !flush(g_open)) { ok = false; break; }
                zero_range(g_open + 1, a.ngrids);
            }
            if (t + 1 < n_iter) {
                // publish this CTA's part of sweep t to every CTA's TMA reads
                fence_proxy_async_global();
                if (!cons_sync()) { ok = false; break; }
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
    }

    // CTA epilogue: the last CTA to finish sums each grid's partials in CTA
    // order and resets the workspace counters for the next launch.  If any
    // CTA gave up a wait (the error word is set), the partials may be stale
    // and every residual is written as NaN instead, so that a caller who
    // reads only the residual still sees the failure.
    __syncthreads();
    __shared__ int s_last, s_failed;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.hdr->counter, 1u);
        s_last = (prev == (unsigned)G - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) s_failed = s_abort || workspace_failed(a.hdr);
        __syncthreads();
        if (a.res != nullptr) {
            for (int g = threadIdx.x; g < a.ngrids; g += blockDim.x) {
                double s = 0.0, c = 0.0;
                if (!s_failed)
                    for (int b = 0; b < G; ++b) neumaier_add(s, c, __ldcg(&a.partials[(size_t)g * G + b]));
                a.res[g] = s_failed ? __longlong_as_double(0x7ff8000000000000ll) : s + c;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            a.hdr->gbar = 0u;
            a.hdr->counter = 0u;
            __threadfence();
        }
    }
}

}  // namespace jac
