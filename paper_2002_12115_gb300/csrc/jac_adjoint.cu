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
// Grouped by the plane of the neighbour, the gather at x = (i, j, k) takes
//   from plane k:   a0 w (i-1), c0 w (i+1), a1 w (j-1), c1 w (j+1),
//                   b0 w (i-1,j-1) - b0 w (i-1,j+1) - b0 w (i+1,j-1) + b0 w (i+1,j+1);
//   from plane k-1: a2 w (i,j) - D1 - D2;   from plane k+1: c2 w (i,j) + D1 + D2,
// with D1 = b1 w (j+1) - b1 w (j-1) and D2 = b2 w (i+1) - b2 w (i-1) taken in
// that neighbour plane.
//
// Kernel design (gather form, streamed over k, persistent, warp-specialised):
//   * a work item is a tile of TI x TJ points in (i, j) over `kdepth` output
//     planes kb .. ke-1; CTA b takes items b, b + G, b + 2G, ...;
//   * the kernel walks the planes m = kb-1 .. ke of an item once and adds
//     each plane's products to three register accumulators: output planes
//     m+1 (its "from k-1" part), m (the in-plane part) and m-1 (its last
//     part, after which it is stored).  So a stage holds one plane of the
//     thirteen inputs (lambda, a3, bnd, the nine coefficients, wrk1), each
//     with only the halo its products need; the planes kb-1 and ke carry
//     only the six arrays of the cross-plane products;
//   * warp TJ (one lane) issues the TMA copies: the planes of p_t (halo both
//     ways, for s0 of the gradients) into a ring of RP slots, the stages into
//     a ring of RC; slots are released through per-slot empty mbarriers;
//   * consumer warp r owns row r of the tile, VI points per lane: it forms w
//     on rows r-1, r, r+1, takes i-neighbours by lane shuffles and the
//     tile's halo columns from the stage (lanes 0 and 31);
//   * the FP64 gradient arrays are read-modify-written by the consumers,
//     loaded one plane ahead;
//   * column i = I-1 is a face that gathers only from column I-2.  When it
//     lies just past the last tile (I-1 a multiple of TI), lane 31 of that
//     tile emits it, so no tile is spent on a single column;
//   * every wait is bounded; on expiry the kernel sets the workspace error
//     word, drains its own copies and returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_internal.h"
#include "jac_sweep_kernel.cuh"

namespace jac {

// Stage geometry of one kernel instantiation: element type T of p, lambda
// and wrk1, coefficient storage C, TJ consumer warps (rows per tile), VI
// points per lane.
template <typename T, typename C, int TJ, int VI_>
struct AdjGeom {
    static constexpr int VI = VI_;                       // points per lane
    static constexpr int TI = 32 * VI;                   // tile width
    static constexpr int HT = 16 / (int)sizeof(T);       // halo columns of a T array (16 bytes)
    static constexpr int HC = 16 / (int)sizeof(C);       // halo columns of a C array
    enum { LAM, A3, BND, A0, C0, A1, C1, B0, B1, B2, A2, C2, WRK1, NQ };
    static constexpr int esz(int q) { return (q == LAM || q == WRK1) ? (int)sizeof(T) : (int)sizeof(C); }
    static constexpr int hw(int q) { return q == LAM ? HT : HC; }
    static constexpr bool w_in(int q) { return q == LAM || q == A3 || q == BND; }   // w needs every halo
    static constexpr int hl(int q) { return (w_in(q) || q == A0 || q == B0 || q == B2) ? hw(q) : 0; }
    static constexpr int hr(int q) { return (w_in(q) || q == C0 || q == B0 || q == B2) ? hw(q) : 0; }
    static constexpr int up(int q) { return (w_in(q) || q == A1 || q == B0 || q == B1) ? 1 : 0; }
    static constexpr int dn(int q) { return (w_in(q) || q == C1 || q == B0 || q == B1) ? 1 : 0; }
    static constexpr int width(int q) { return TI + hl(q) + hr(q); }
    static constexpr int height(int q) { return TJ + up(q) + dn(q); }
    static constexpr int box_bytes(int q) { return width(q) * height(q) * esz(q); }
    static constexpr int slot_bytes(int q) { return (box_bytes(q) + 127) / 128 * 128; }
    static constexpr int off(int q)
    {
        int o = 0;
        for (int s = 0; s < q; ++s) o += slot_bytes(s);
        return o;
    }
    static constexpr int STAGE = off(NQ);
    // kind 0: an output plane (every array); 1: plane kb-1; 2: plane ke
    static constexpr bool loads(int q, int kind)
    {
        return kind == 0 || w_in(q) || q == B1 || q == B2 || q == (kind == 1 ? A2 : C2);
    }
    static constexpr uint32_t tx(int kind)
    {
        uint32_t b = 0;
        for (int q = 0; q < NQ; ++q)
            if (loads(q, kind)) b += (uint32_t)box_bytes(q);
        return b;
    }
    static constexpr int PW = TI + 2 * HT, PH = TJ + 2;  // state plane with its halo
    static constexpr uint32_t P_TX = (uint32_t)(PW * PH * (int)sizeof(T));
    static constexpr int P_BYTES = (int)((P_TX + 127) / 128 * 128);
    static constexpr int RP = 5;                          // state ring: planes m-1..m+1 and two ahead
    static constexpr int BUDGET = 220 * 1024;
    static constexpr int RC_FIT = (BUDGET - RP * P_BYTES - 1024) / STAGE;
    static constexpr int RC = RC_FIT > 8 ? 8 : RC_FIT;    // stages
    static constexpr size_t SMEM = (size_t)RP * P_BYTES + (size_t)RC * STAGE + 128;
    static constexpr int THREADS = 32 * (TJ + 1);
};

struct AdjDesc {
    CUtensorMap map[13];       // stage arrays, AdjGeom order (LAM .. WRK1)
    CUtensorMap pmap;          // p_t, box (TI + 2 HT, TJ + 2)
    void *lam_out;             // lambda_t (storage layout, T)
    double *g_wrk1, *g_a3;     // dense FP64, accumulated
    double *g_coef[9];         // a0 a1 a2 b0 b1 b2 c0 c1 c2, or all NULL
    WsHeader *hdr;
    int I, J, K, pitch, kdepth, nti, ntj, nitems;
    double omega;
};

struct AdjItem {
    int i0, j0, kb, ke, m_lo, m_hi;
};

template <int TI, int TJ>
__device__ __forceinline__ AdjItem adj_item(const AdjDesc &d, int item)
{
    AdjItem it;
    const int tj = item % d.ntj;
    const int r = item / d.ntj;
    const int ti = r % d.nti;
    const int kk = r / d.nti;
    it.i0 = ti * TI;
    it.j0 = tj * TJ;
    it.kb = kk * d.kdepth;
    it.ke = min(d.K, it.kb + d.kdepth);
    it.m_lo = max(it.kb - 1, 0);
    it.m_hi = min(it.ke, d.K - 1);
    return it;
}

// VI consecutive values of T from shared memory (16- or 8-byte aligned).
template <typename T, int VI>
__device__ __forceinline__ void adj_lds(const T *p, T (&v)[VI])
{
    if constexpr (sizeof(T) * VI == 16) {
        lds_vec<T, VI>(p, v);
    } else if constexpr (sizeof(T) == 4 && VI == 2) {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x; v[1] = x.y;
    } else {
        static_assert(sizeof(T) == 8 && VI == 1, "unsupported vector shape");
        v[0] = *p;
    }
}

// VI BF16 values from shared memory as FP32 (exact: the BF16 bits are the
// high half of the FP32 word), or VI values of T.
template <typename T, typename C, int VI>
__device__ __forceinline__ void adj_coef(const unsigned char *tile, int idx, T (&o)[VI])
{
    if constexpr (sizeof(C) == 2 && VI == 2) {
        const uint32_t v = *reinterpret_cast<const uint32_t *>(tile + (size_t)idx * 2);
        o[0] = __uint_as_float(v << 16);
        o[1] = __uint_as_float(v & 0xffff0000u);
    } else if constexpr (sizeof(C) == 2) {
        smem_coef<T, C, VI>(tile, idx, o);
    } else {
        adj_lds<T, VI>(reinterpret_cast<const T *>(tile) + idx, o);
    }
}

// VI values of a state row plus the left and right neighbours: lane
// shuffles inside the warp, the halo columns for lanes 0 and 31.
template <typename T, int VI, int H>
__device__ __forceinline__ void adj_load_ext(const T *row, int lane, T (&e)[VI + 2])
{
    const int col = H + VI * lane;
    T v[VI];
    adj_lds<T, VI>(row + col, v);
#pragma unroll
    for (int q = 0; q < VI; ++q) e[q + 1] = v[q];
    T l = __shfl_up_sync(0xffffffffu, e[VI], 1);
    T r = __shfl_down_sync(0xffffffffu, e[1], 1);
    if (lane == 0) l = row[col - 1];
    if (lane == 31) r = row[col + VI];
    e[0] = l;
    e[VI + 1] = r;
}

// VI values of stage array Q at tile row `row` (-up .. TJ-1+dn) and tile
// column `col` (a multiple of VI), as T.
template <typename G, int Q, typename T, int VI>
__device__ __forceinline__ void st_vec(const unsigned char *st, int row, int col, T (&o)[VI])
{
    const int idx = (row + G::up(Q)) * G::width(Q) + col + G::hl(Q);
    if constexpr (G::esz(Q) == (int)sizeof(T)) adj_lds<T, VI>(reinterpret_cast<const T *>(st + G::off(Q)) + idx, o);
    else adj_coef<T, __nv_bfloat16, VI>(st + G::off(Q), idx, o);
}

// One value of stage array Q (col may be -1 or TI, the halo columns), as T.
template <typename G, int Q, typename T>
__device__ __forceinline__ T st_one(const unsigned char *st, int row, int col)
{
    const int idx = (row + G::up(Q)) * G::width(Q) + col + G::hl(Q);
    if constexpr (G::esz(Q) == (int)sizeof(T)) {
        return reinterpret_cast<const T *>(st + G::off(Q))[idx];
    } else {
        const unsigned short b = reinterpret_cast<const unsigned short *>(st + G::off(Q))[idx];
        return __uint_as_float((uint32_t)b << 16);
    }
}

template <typename T, int VI>
__device__ __forceinline__ void stg_vec(T *p, const T (&v)[VI])
{
    if constexpr (sizeof(T) == 4 && VI == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (sizeof(T) == 4 && VI == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else if constexpr (VI == 2) *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    else *p = v[0];
}

template <typename T, typename C, int TJ, int VI_, bool CGRAD>
__global__ void __launch_bounds__(AdjGeom<T, C, TJ, VI_>::THREADS, 1)
k_adjoint(const __grid_constant__ AdjDesc d)
{
    using G = AdjGeom<T, C, TJ, VI_>;
    constexpr int VI = G::VI, TI = G::TI, HT = G::HT, RP = G::RP, RC = G::RC;
    extern __shared__ unsigned char adj_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(adj_raw) + 127) & ~uintptr_t(127));
    unsigned char *ring_s = base + (size_t)RP * G::P_BYTES;
    __shared__ __align__(8) uint64_t p_full[RP], p_empty[RP], c_full[RC], c_empty[RC];
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int NB = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RP; ++s) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], TJ); }
        for (int s = 0; s < RC; ++s) { mbar_init(&c_full[s], 1); mbar_init(&c_empty[s], TJ); }
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == TJ) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t pc = 0, cc = 0;
            bool ok = true;
            auto issue_p = [&](const AdjItem &it, int m) -> bool {
                const uint32_t slot = pc % RP, use = pc / RP;
                if (use > 0 && !mbar_wait_bounded(&p_empty[slot], (use - 1) & 1)) return false;
                if (s_abort) return false;
                mbar_arrive_expect_tx(&p_full[slot], G::P_TX);
                tma_load_3d(base + (size_t)slot * G::P_BYTES, &d.pmap, &p_full[slot], it.i0 - HT, it.j0 - 1, m);
                ++pc;
                return true;
            };
            auto issue_s = [&](const AdjItem &it, int m) -> bool {
                const uint32_t slot = cc % RC, use = cc / RC;
                if (use > 0 && !mbar_wait_bounded(&c_empty[slot], (use - 1) & 1)) return false;
                if (s_abort) return false;
                const int kind = (m < it.kb) ? 1 : (m >= it.ke ? 2 : 0);
                unsigned char *st = ring_s + (size_t)slot * G::STAGE;
                mbar_arrive_expect_tx(&c_full[slot], kind == 0 ? G::tx(0) : (kind == 1 ? G::tx(1) : G::tx(2)));
#pragma unroll
                for (int q = 0; q < G::NQ; ++q)
                    if (G::loads(q, kind))
                        tma_load_3d(st + G::off(q), &d.map[q], &c_full[slot], it.i0 - G::hl(q), it.j0 - G::up(q),
                                    m);
                ++cc;
                return true;
            };
            for (int item = blockIdx.x; item < d.nitems && ok; item += NB) {
                const AdjItem it = adj_item<TI, TJ>(d, item);
                ok = issue_p(it, it.m_lo) && (it.m_lo + 1 > it.m_hi || issue_p(it, it.m_lo + 1));
                for (int m = it.m_lo; m <= it.m_hi && ok; ++m) {
                    if (m + 2 <= it.m_hi) ok = issue_p(it, m + 2);
                    ok = ok && issue_s(it, m);
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(&d.hdr->errword, (int)JAC_ETIMEOUT);
            }
            for (uint32_t s = 0; s < (uint32_t)RP && s < pc; ++s) {   // land every issued copy
                const uint32_t last = pc - 1 - ((pc - 1 - s) % RP);
                (void)mbar_wait_bounded(&p_full[s], (last / RP) & 1);
            }
            for (uint32_t s = 0; s < (uint32_t)RC && s < cc; ++s) {
                const uint32_t last = cc - 1 - ((cc - 1 - s) % RC);
                (void)mbar_wait_bounded(&c_full[s], (last / RC) & 1);
            }
        }
        return;
    }

    // -------------------------------------------------------------- consumers
    const int r = warp;                       // tile row of this warp
    const T omega = (T)d.omega;
    const int I = d.I, J = d.J, K = d.K, pitch = d.pitch;
    T *lam_out = static_cast<T *>(d.lam_out);
    uint32_t pc = 0, cc = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < d.nitems && ok; item += NB) {
        const AdjItem it = adj_item<TI, TJ>(d, item);
        const int j = it.j0 + r;
        const int ib = it.i0 + VI * lane;
        const bool row_ok = j < J;
        const bool vec_ok = row_ok && ib < pitch;
        // column I-1 just past the tile: lane 31 emits it
        const bool extra = row_ok && lane == 31 && (it.i0 + TI == I - 1);
        bool inI[VI];
#pragma unroll
        for (int e = 0; e < VI; ++e) inI[e] = (ib + e >= 1) && (ib + e <= I - 2);
        const bool inI_l = (it.i0 - 1 >= 1) && (it.i0 - 1 <= I - 2);
        const bool inI_r = (it.i0 + TI >= 1) && (it.i0 + TI <= I - 2);
        // the tile halo column on this lane's side: lane 0 the left one, the
        // others the right one (only lane 31 uses it)
        const int hcol = (lane == 0) ? -1 : TI;
        const bool hin = (lane == 0) ? inI_l : inI_r;
        bool inJ[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) inJ[s] = (j - 1 + s >= 1) && (j - 1 + s <= J - 2);

        T Qm[VI], Qm1[VI];                    // partial lambda of output planes m and m-1
        T Xm = T(0), Xm1 = T(0);              // the same at column I-1 (extra)
#pragma unroll
        for (int e = 0; e < VI; ++e) Qm[e] = Qm1[e] = T(0);
        double gw[VI], ga[VI];                // gradients of the next plane, loaded one plane ahead
#pragma unroll
        for (int e = 0; e < VI; ++e) gw[e] = ga[e] = 0.0;
        auto load_grads = [&](int m) {
            if (!(m >= it.kb && m < it.ke && m >= 1 && m <= K - 2 && row_ok && inJ[1])) return;
            const size_t dd = ((size_t)m * J + (size_t)j) * (size_t)I + (size_t)ib;
#pragma unroll
            for (int e = 0; e < VI; ++e)
                if (inI[e]) {
                    gw[e] = __ldcg(d.g_wrk1 + dd + e);
                    ga[e] = __ldcg(d.g_a3 + dd + e);
                }
        };
        int pw = 0;                           // state planes of this item waited for
        const int np = it.m_hi - it.m_lo + 1;

        for (int m = it.m_lo; m <= it.m_hi; ++m) {
            const int kind = (m < it.kb) ? 1 : (m >= it.ke ? 2 : 0);
            const uint32_t cs = cc;
            const int need = min(m + 1, it.m_hi) - it.m_lo + 1;
            double gwc[VI], gac[VI];          // this plane's gradients, loaded one plane ago
#pragma unroll
            for (int e = 0; e < VI; ++e) { gwc[e] = gw[e]; gac[e] = ga[e]; }
            load_grads(m + 1);
            ok = mbar_wait_bounded(&c_full[cs % RC], (cs / RC) & 1);
            while (ok && pw < need) {
                const uint32_t q = pc + (uint32_t)pw;
                ok = mbar_wait_bounded(&p_full[q % RP], (q / RP) & 1);
                ++pw;
            }
            ok = __all_sync(0xffffffffu, ok && !s_abort);
            if (!ok) break;
            const unsigned char *st = ring_s + (size_t)(cs % RC) * G::STAGE;
            const bool inK = (m >= 1) && (m <= K - 2);

            // w on rows r-1, r, r+1, extended by one point on each side
            T w[3][VI + 2];
            T lam_c[VI], mu_c[VI];
            T lam_x = T(0);                   // lambda_{t+1} at column I-1 (extra)
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int row = r - 1 + s;
                T lv[VI], av[VI], bv[VI];
                st_vec<G, G::LAM, T, VI>(st, row, VI * lane, lv);
                st_vec<G, G::A3, T, VI>(st, row, VI * lane, av);
                st_vec<G, G::BND, T, VI>(st, row, VI * lane, bv);
                const bool rin = inK && inJ[s];
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    const T mu = (rin && inI[e]) ? omega * bv[e] * lv[e] : T(0);
                    w[s][e + 1] = av[e] * mu;
                    if (s == 1) { lam_c[e] = lv[e]; mu_c[e] = mu; }
                }
                T wl = __shfl_up_sync(0xffffffffu, w[s][VI], 1);
                T wr = __shfl_down_sync(0xffffffffu, w[s][1], 1);
                {
                    // w at the tile's halo column on this lane's side (lane 0: left,
                    // the others: right), without a divergent branch; lanes 1..30
                    // discard it
                    const T lam_h = st_one<G, G::LAM, T>(st, row, hcol);
                    const T mu = (rin && hin) ? omega * st_one<G, G::BND, T>(st, row, hcol) * lam_h : T(0);
                    const T wh = st_one<G, G::A3, T>(st, row, hcol) * mu;
                    wl = (lane == 0) ? wh : wl;
                    wr = (lane == 31) ? wh : wr;
                    if (s == 1) lam_x = lam_h;        // used by lane 31 only
                }
                w[s][0] = wl;
                w[s][VI + 1] = wr;
            }

            // cross-plane products: D = D1 (b1, rows r-1 and r+1) + D2 (b2, row r)
            T D[VI], b2x;
            {
                T bm[VI], bp[VI], b2[VI], P2[VI];
                st_vec<G, G::B1, T, VI>(st, r - 1, VI * lane, bm);
                st_vec<G, G::B1, T, VI>(st, r + 1, VI * lane, bp);
                st_vec<G, G::B2, T, VI>(st, r, VI * lane, b2);
#pragma unroll
                for (int e = 0; e < VI; ++e) P2[e] = b2[e] * w[1][e + 1];
                T l2 = __shfl_up_sync(0xffffffffu, P2[VI - 1], 1);
                T r2 = __shfl_down_sync(0xffffffffu, P2[0], 1);
                {
                    const T p2h = st_one<G, G::B2, T>(st, r, hcol) * (lane == 0 ? w[1][0] : w[1][VI + 1]);
                    l2 = (lane == 0) ? p2h : l2;
                    r2 = (lane == 31) ? p2h : r2;
                }
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    const T lft = (e == 0) ? l2 : P2[e - 1];
                    const T rgt = (e == VI - 1) ? r2 : P2[e + 1];
                    D[e] = (bp[e] * w[2][e + 1] - bm[e] * w[0][e + 1]) + (rgt - lft);
                }
                b2x = P2[VI - 1];             // b2 w at column I-2 (extra)
            }

            // plane m-1 is complete: its last part comes from plane m
            if (kind != 1 && m - 1 >= it.kb) {
                T cv[VI], o[VI];
                st_vec<G, G::C2, T, VI>(st, r, VI * lane, cv);
#pragma unroll
                for (int e = 0; e < VI; ++e) o[e] = Qm1[e] + (cv[e] * w[1][e + 1] + D[e]);
                const size_t off = ((size_t)(m - 1) * J + (size_t)j) * (size_t)pitch + (size_t)ib;
                if (vec_ok) stg_vec<T, VI>(lam_out + off, o);
                if (extra) lam_out[off - (size_t)ib + (size_t)(I - 1)] = Xm1 - b2x;
            }
            // the "from k-1" part of plane m+1
            T Qn[VI];
            T Xn = T(0);
            if (kind != 2 && m + 1 < it.ke) {
                T av[VI];
                st_vec<G, G::A2, T, VI>(st, r, VI * lane, av);
#pragma unroll
                for (int e = 0; e < VI; ++e) Qn[e] = av[e] * w[1][e + 1] - D[e];
                Xn = b2x;
            } else {
#pragma unroll
                for (int e = 0; e < VI; ++e) Qn[e] = T(0);
            }

            if (kind == 0) {
                // in-plane part of plane m
                T a0[VI], c0[VI], a1[VI], c1[VI], b0m[VI], b0p[VI];
                st_vec<G, G::A0, T, VI>(st, r, VI * lane, a0);
                st_vec<G, G::C0, T, VI>(st, r, VI * lane, c0);
                st_vec<G, G::A1, T, VI>(st, r - 1, VI * lane, a1);
                st_vec<G, G::C1, T, VI>(st, r + 1, VI * lane, c1);
                st_vec<G, G::B0, T, VI>(st, r - 1, VI * lane, b0m);
                st_vec<G, G::B0, T, VI>(st, r + 1, VI * lane, b0p);
                T Pa0[VI], Pc0[VI], Pbm[VI], Pbp[VI];
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    Pa0[e] = a0[e] * w[1][e + 1];
                    Pc0[e] = c0[e] * w[1][e + 1];
                    Pbm[e] = b0m[e] * w[0][e + 1];
                    Pbp[e] = b0p[e] * w[2][e + 1];
                }
                T la0 = __shfl_up_sync(0xffffffffu, Pa0[VI - 1], 1);
                T rc0 = __shfl_down_sync(0xffffffffu, Pc0[0], 1);
                T lbm = __shfl_up_sync(0xffffffffu, Pbm[VI - 1], 1);
                T rbm = __shfl_down_sync(0xffffffffu, Pbm[0], 1);
                T lbp = __shfl_up_sync(0xffffffffu, Pbp[VI - 1], 1);
                T rbp = __shfl_down_sync(0xffffffffu, Pbp[0], 1);
                {
                    const T bmh = st_one<G, G::B0, T>(st, r - 1, hcol) * (lane == 0 ? w[0][0] : w[0][VI + 1]);
                    const T bph = st_one<G, G::B0, T>(st, r + 1, hcol) * (lane == 0 ? w[2][0] : w[2][VI + 1]);
                    lbm = (lane == 0) ? bmh : lbm;
                    rbm = (lane == 31) ? bmh : rbm;
                    lbp = (lane == 0) ? bph : lbp;
                    rbp = (lane == 31) ? bph : rbp;
                }
                if (lane == 0) la0 = st_one<G, G::A0, T>(st, r, -1) * w[1][0];
                if (lane == 31) rc0 = st_one<G, G::C0, T>(st, r, TI) * w[1][VI + 1];
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    const T a0w = (e == 0) ? la0 : Pa0[e - 1];
                    const T c0w = (e == VI - 1) ? rc0 : Pc0[e + 1];
                    const T bmm = (e == 0) ? lbm : Pbm[e - 1];        // (i-1, j-1)
                    const T bpm = (e == 0) ? lbp : Pbp[e - 1];        // (i-1, j+1)
                    const T bmp = (e == VI - 1) ? rbm : Pbm[e + 1];   // (i+1, j-1)
                    const T bpp = (e == VI - 1) ? rbp : Pbp[e + 1];   // (i+1, j+1)
                    const T in = ((a0w + c0w) + (a1[e] * w[0][e + 1] + c1[e] * w[2][e + 1])) +
                                 (((bmm - bpm) - bmp) + bpp);
                    Qm[e] += (lam_c[e] - mu_c[e]) + in;
                }
                // column I-2's products into the face column I-1
                Xm += lam_x + (Pa0[VI - 1] + (Pbm[VI - 1] - Pbp[VI - 1]));

                // parameter gradients at the interior points of the row
                if (inK && row_ok && inJ[1]) {
                    constexpr int W = G::PW;
                    const int pm = (int)((pc + (uint32_t)(m - 1 - it.m_lo)) % RP);
                    const T *Pm = reinterpret_cast<const T *>(base + (size_t)pm * G::P_BYTES);
                    const T *Pk = reinterpret_cast<const T *>(base + (size_t)((pm + 1) % RP) * G::P_BYTES);
                    const T *Pp = reinterpret_cast<const T *>(base + (size_t)((pm + 2) % RP) * G::P_BYTES);
                    const int r0 = r * W, r1 = (r + 1) * W, r2 = (r + 2) * W;   // rows j-1, j, j+1
                    T ek0[VI + 2], ek1[VI + 2], ek2[VI + 2], em1[VI + 2], ep1[VI + 2];
                    T vm0[VI], vm2[VI], vp0[VI], vp2[VI];
                    adj_load_ext<T, VI, HT>(Pk + r0, lane, ek0);
                    adj_load_ext<T, VI, HT>(Pk + r1, lane, ek1);
                    adj_load_ext<T, VI, HT>(Pk + r2, lane, ek2);
                    adj_load_ext<T, VI, HT>(Pm + r1, lane, em1);
                    adj_load_ext<T, VI, HT>(Pp + r1, lane, ep1);
                    adj_lds<T, VI>(Pm + r0 + HT + VI * lane, vm0);
                    adj_lds<T, VI>(Pm + r2 + HT + VI * lane, vm2);
                    adj_lds<T, VI>(Pp + r0 + HT + VI * lane, vp0);
                    adj_lds<T, VI>(Pp + r2 + HT + VI * lane, vp2);
                    T a1c[VI], a2c[VI], b0c[VI], b1c[VI], b2c[VI], c1c[VI], c2c[VI], wk[VI];
                    st_vec<G, G::A1, T, VI>(st, r, VI * lane, a1c);
                    st_vec<G, G::A2, T, VI>(st, r, VI * lane, a2c);
                    st_vec<G, G::B0, T, VI>(st, r, VI * lane, b0c);
                    st_vec<G, G::B1, T, VI>(st, r, VI * lane, b1c);
                    st_vec<G, G::B2, T, VI>(st, r, VI * lane, b2c);
                    st_vec<G, G::C1, T, VI>(st, r, VI * lane, c1c);
                    st_vec<G, G::C2, T, VI>(st, r, VI * lane, c2c);
                    st_vec<G, G::WRK1, T, VI>(st, r, VI * lane, wk);
                    const size_t dd = ((size_t)m * J + (size_t)j) * (size_t)I + (size_t)ib;
#pragma unroll
                    for (int e = 0; e < VI; ++e) {
                        if (!inI[e]) continue;
                        const T xp = ek1[e + 2], xm = ek1[e], yp = ek2[e + 1], ym = ek0[e + 1];
                        const T zp = ep1[e + 1], zm = em1[e + 1];
                        const T bij = ((ek2[e + 2] - ek0[e + 2]) - ek2[e]) + ek0[e];
                        const T bjk = ((vp2[e] - vm2[e]) - vp0[e]) + vm0[e];
                        const T bik = ((ep1[e + 2] - em1[e + 2]) - ep1[e]) + em1[e];
                        T s0 = wk[e];
                        s0 = fma(a0[e], xp, s0);
                        s0 = fma(a1c[e], yp, s0);
                        s0 = fma(a2c[e], zp, s0);
                        s0 = fma(b0c[e], bij, s0);
                        s0 = fma(b1c[e], bjk, s0);
                        s0 = fma(b2c[e], bik, s0);
                        s0 = fma(c0[e], xm, s0);
                        s0 = fma(c1c[e], ym, s0);
                        s0 = fma(c2c[e], zm, s0);
                        const T we = w[1][e + 1];
                        // each sweep's term is formed in T and accumulated in FP64
                        d.g_wrk1[dd + e] = gwc[e] + (double)we;
                        d.g_a3[dd + e] = gac[e] + (double)(mu_c[e] * s0);
                        if constexpr (CGRAD) {
                            const T tv[9] = {xp, yp, zp, bij, bjk, bik, xm, ym, zm};
#pragma unroll
                            for (int q = 0; q < 9; ++q) d.g_coef[q][dd + e] += (double)(we * tv[q]);
                        }
                    }
                }
            }

#pragma unroll
            for (int e = 0; e < VI; ++e) { Qm1[e] = Qm[e]; Qm[e] = Qn[e]; }
            Xm1 = Xm;
            Xm = Xn;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&c_empty[cs % RC]);
                if (m > it.m_lo) mbar_arrive(&p_empty[(pc + (uint32_t)(m - 1 - it.m_lo)) % RP]);
            }
            ++cc;
        }
        if (!ok) break;
        // an output plane K-1 has no plane above it
        if (it.m_hi == it.ke - 1) {
            const size_t off = ((size_t)it.m_hi * J + (size_t)j) * (size_t)pitch + (size_t)ib;
            if (vec_ok) stg_vec<T, VI>(lam_out + off, Qm1);
            if (extra) lam_out[off - (size_t)ib + (size_t)(I - 1)] = Xm1;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&p_empty[(pc + (uint32_t)(np - 1)) % RP]);
        pc += (uint32_t)np;
    }
    if (!ok) {
        s_abort = 1;
        atomicExch(&d.hdr->errword, (int)JAC_ETIMEOUT);
    }
}

// ------------------------------------------------------------ host side
namespace {

jac_status adj_fail(jac_status s, const std::string &m)
{
    set_thread_error(m);
    return s;
}

template <typename T, typename C, int TJ, int VI, bool CGRAD>
jac_status launch_adj(const AdjDesc &d, unsigned nblocks, cudaStream_t st)
{
    using G = AdjGeom<T, C, TJ, VI>;
    static_assert(G::RC >= 2, "stage ring too shallow for the shared-memory budget");
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(k_adjoint<T, C, TJ, VI, CGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)G::SMEM);
    });
    if (err != cudaSuccess) return adj_fail(JAC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
    k_adjoint<T, C, TJ, VI, CGRAD><<<nblocks, G::THREADS, G::SMEM, st>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return adj_fail(JAC_ECUDA, std::string("adjoint launch: ") + cudaGetErrorString(e));
    return JAC_OK;
}


// Launch shapes: consumer warps (tile rows) and points per lane.  FP32
// state: 15 rows of 64 points (two per lane), so that with the producer the
// CTA has 16 warps, four per SM sub-partition, and each thread may hold 128
// registers of the sub-partition's 16 K (a 17th warp would put five warps on
// one sub-partition and cap every thread at 96).  FP64: 8 rows of 64 points.
constexpr int kAdjRowsF32 = 15, kAdjVIF32 = 2, kAdjRowsF64 = 8;

// Output planes per item: 32, fewer while the grid has too few items to give
// every SM two.
int adj_kdepth(int K, long long tiles_ij, int sms)
{
    int kd = 32;
    while (kd > 4 && tiles_ij * ((K + kd - 1) / kd) < 2LL * sms) kd /= 2;
    return kd;
}

// TJ consumer warps (tile rows) of VI points per lane.
template <typename T, typename C, int TJ, int VI>
jac_status run_adj(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out, double *g_wrk1,
                   double *g_a3, double *const *g_coef, int kdepth, WsHeader *hdr, cudaStream_t st)
{
    using G = AdjGeom<T, C, TJ, VI>;
    AdjDesc d;
    std::memset(&d, 0, sizeof(d));
    d.I = g->I; d.J = g->J; d.K = g->K;
    d.pitch = jac_pitch(g->I);
    d.nti = std::max(1, (g->I - 1 + G::TI - 1) / G::TI);   // column I-1 may be a tile's extra column
    d.ntj = (g->J + TJ - 1) / TJ;
    const int sms = device_sm_count();
    d.kdepth = kdepth > 0 ? kdepth : adj_kdepth(g->K, (long long)d.nti * d.ntj, sms);
    const long long items = (long long)d.nti * d.ntj * ((g->K + d.kdepth - 1) / d.kdepth);
    if (items > 0x3fffffffLL) return adj_fail(JAC_EINVAL, "adjoint: grid too large for the launch shape");
    d.nitems = (int)items;
    d.omega = g->omega;
    d.lam_out = lam_out;
    d.g_wrk1 = g_wrk1;
    d.g_a3 = g_a3;
    bool cgrad = false;
    if (g_coef) {
        cgrad = true;
        for (int q = 0; q < 9; ++q) {
            if (!g_coef[q]) return adj_fail(JAC_EINVAL, "adjoint: g_coef needs all nine arrays");
            d.g_coef[q] = g_coef[q];
        }
    }
    d.hdr = hdr;
    // stage arrays in AdjGeom order; each box carries the array's halo, and
    // the extent in i is I, so that columns past the grid read as zero
    static const int field[G::NQ] = {-1,     JAC_A3, JAC_BND, JAC_A0, JAC_C0, JAC_A1, JAC_C1,
                                     JAC_B0, JAC_B1, JAC_B2,  JAC_A2, JAC_C2, JAC_WRK1};
    jac_status s;
    for (int q = 0; q < G::NQ; ++q) {
        const void *ptr = q == G::LAM ? lam_in : g->coef[field[q]];
        if ((s = encode_box_map(&d.map[q], ptr, (size_t)G::esz(q), g->I, d.pitch, g->J, g->K, G::width(q),
                                G::height(q))) != JAC_OK)
            return s;
    }
    if ((s = encode_box_map(&d.pmap, p_t, sizeof(T), g->I, d.pitch, g->J, g->K, G::PW, G::PH)) != JAC_OK) return s;
    const unsigned nblocks = (unsigned)std::min<long long>(items, sms);
    return cgrad ? launch_adj<T, C, TJ, VI, true>(d, nblocks, st) : launch_adj<T, C, TJ, VI, false>(d, nblocks, st);
}

}  // namespace

jac_status adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out, double *g_wrk1,
                            double *g_a3, double *const *g_coef, int kdepth, void *workspace, size_t ws_bytes,
                            cudaStream_t st)
{
    jac_status s = validate_grid(g);
    if (s != JAC_OK) return s;
    if (!p_t || !lam_in || !lam_out || !g_wrk1 || !g_a3 || lam_in == lam_out)
        return adj_fail(JAC_EINVAL, "adjoint: state, lambda (two distinct buffers) and gradient arrays are required");
    const uintptr_t al = reinterpret_cast<uintptr_t>(p_t) | reinterpret_cast<uintptr_t>(lam_in) |
                         reinterpret_cast<uintptr_t>(lam_out);
    if (al & 15) return adj_fail(JAC_EINVAL, "adjoint: state and lambda buffers must be 16-byte aligned");
    if (!workspace || ws_bytes < kWsHeaderBytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return adj_fail(JAC_EINVAL, "adjoint: a workspace of at least 256 bytes, 256-byte aligned, is required");
    if (kdepth < 0) return adj_fail(JAC_EINVAL, "adjoint: kdepth must be >= 0");
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    switch (g->prec) {
    case JAC_F64:
        return run_adj<double, double, kAdjRowsF64, 2>(g, p_t, lam_in, lam_out, g_wrk1, g_a3, g_coef, kdepth, hdr,
                                                        st);
    case JAC_F32:
        return run_adj<float, float, kAdjRowsF32, kAdjVIF32>(g, p_t, lam_in, lam_out, g_wrk1, g_a3, g_coef, kdepth,
                                                             hdr, st);
    case JAC_F32_BF16COEF:
        return run_adj<float, __nv_bfloat16, kAdjRowsF32, kAdjVIF32>(g, p_t, lam_in, lam_out, g_wrk1, g_a3, g_coef,
                                                                     kdepth, hdr, st);
    }
    return adj_fail(JAC_EINVAL, "unknown precision");
}

}  // namespace jac

extern "C" jac_status jac_adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out,
                                           double *g_wrk1, double *g_a3, double *const *g_coef, int kdepth,
                                           void *workspace, size_t ws_bytes, void *stream)
{
    return jac::adjoint_step_dev(g, p_t, lam_in, lam_out, g_wrk1, g_a3, g_coef, kdepth, workspace, ws_bytes,
                                 static_cast<cudaStream_t>(stream));
}
