// Two fused sweeps per pass (temporal blocking by two) for FP32 storage.
//
// A pass reads the state p_t and writes p_{t+2}; the intermediate state
// p_{t+1} of a tile lives only in shared memory.  Every coefficient plane is
// then read from memory once for two point-updates.  Each update is the
// same arithmetic as the single-sweep kernel (ss_f32_ec; a3 S - 1, which
// depends only on the coefficients, is formed by sweep 1 and carried in
// registers to sweep 2 at the same point), so a pass gives bitwise the state
// of two single sweeps.
//
// Kernel design (persistent, warp-specialised, one CTA per SM, all passes of
// a call in one cooperative launch):
//   * an item is a tile of the 128 columns i0 .. i0+127 (i0 a multiple of
//     128) x R2 = 8 rows in (i, j) of output points over `kdepth` output
//     planes kb .. ke-1.  Sweep 1 runs over the tile's columns, the
//     R1 = R2 + 2 rows j0-1 .. j0+R2 and the planes kb-1 .. ke; sweep 2 over
//     the R2 inner rows and planes kb .. ke-1.  Tiles do not overlap: sweep 2
//     at columns i0 and i0+127 needs sweep 1 at columns i0-1 and i0+128 too;
//   * warp 10 (one lane) copies, in the order they are used, the planes of
//     p_t with a halo of 4 columns and 2 rows into a ring of 4 slots, and the
//     twelve coefficient tiles (128 x R1) of every sweep-1 plane into a ring
//     of 2 stages, which sweep 1 alone uses.  Before the state of pass
//     t >= 1 it waits on the grid barrier of the pass before;
//   * consumer warp w (0 .. R1-1) owns row j0-1+w.  At step s (plane
//     m = kb-1+s) it computes sweep 1 there into a ring of 4 intermediate
//     planes, then (warps 1 .. R1-2, s >= 3) sweep 2 at plane m-2 from the
//     intermediate planes m-3 .. m-1.  Sweep 2 trails by two planes so that
//     its wait (every row of plane m-1 written: an mbarrier per
//     intermediate plane) is for work the other warps finished a step ago,
//     not for the step in flight.  Its coefficients come from global memory
//     (the tiles were copied for sweep 1 two steps earlier, so they are read
//     from L2) into a 6 KB buffer per warp: each lane copies its own 12 x 16
//     bytes with cp.async at the end of a step, for the next step's sweep 2,
//     so the L2 latency is hidden behind sweep 1.  (Keeping the stages for
//     three steps would need four 61 KB stages in flight.)
//   * warp 11 (the edge warp, 20 lanes) computes sweep 1 at columns i0-1 and
//     i0+128 of the R1 rows at every step, from the state ring and
//     coefficients it loads from global memory one plane ahead (those
//     columns belong to the neighbouring tiles, whose CTAs copy them at
//     about the same time);
//   * the residual of the last pass's second sweep is reduced as in the
//     single-sweep kernel; every wait is bounded;
//   * a one-pass call may also store sweep 1's state at the points the
//     items own (Sweep2Args::mid): the reverse pass recomputes two
//     checkpoint-segment states per launch that way.
//
// Twelve warps leave 168 registers a thread (a thirteenth would put four
// warps on one SM sub-partition and cap them at 128).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "jac_internal.h"
#include "jac_sweep_kernel.cuh"

namespace jac {

struct Sweep2Shape {
    static constexpr int VI = 4, TI = 128, H = 4;
    static constexpr int R2 = 8, R1 = R2 + 2;                // output rows, sweep-1 rows (= consumer warps)
    static constexpr int PW = TI + 2 * H, PH = R1 + 2;       // state plane box
    static constexpr int P_BYTES = PW * PH * 4;              // 6528
    static constexpr int TILE = TI * R1 * 4;                 // one coefficient tile, 5120
    static constexpr int C_BYTES = 12 * TILE;                // one stage
    static constexpr int Q_BYTES = TI * R1 * 4;              // one intermediate plane
    static constexpr int B_BYTES = 12 * TI * 4;              // one warp's sweep-2 coefficients of one row
    static constexpr int RP = 4, RC = 2, RQ = 4;
    static constexpr size_t SMEM =
        (size_t)RP * P_BYTES + (size_t)RQ * Q_BYTES + (size_t)RC * C_BYTES + (size_t)R2 * B_BYTES + 128;
    static constexpr int EDGE_WARP = R1 + 1;                 // sweep 1 at the two columns past the tile
    static constexpr int THREADS = 32 * (R1 + 2);
    static_assert(P_BYTES % 128 == 0 && Q_BYTES % 128 == 0 && C_BYTES % 128 == 0 && B_BYTES % 128 == 0,
                  "slot alignment");
};

struct Sweep2Desc {
    CUtensorMap p[2];          // state buffers, box (PW, PH, 1)
    CUtensorMap coef[12];      // JAC_A0 .. JAC_BND (index q-1), box (TI, R1, 1)
    const float *coef_ptr[12]; // the same arrays, for the edge warp's loads
    void *p_buf[2];
    int I, J, K, pitch;
    int kdepth, nti, ntj, nkb, nitems;
};

struct Sweep2Args {
    int n_pass, par;           // pass t reads p[(t + par) & 1], writes the other
    double omega;
    double *partials;          // gridDim.x
    double *res;               // residual of the last pass's second sweep (NULL: none)
    float *mid;                // one-pass calls: also store sweep 1's state here (NULL: no)
    WsHeader *hdr;
    int l2_keep_state;
    unsigned l2_keep_coef;
};

struct Item2 {
    int ti, i0, j0, kb, nout;
};

__device__ __forceinline__ Item2 decode_item2(const Sweep2Desc &d, int item)
{
    using S = Sweep2Shape;
    Item2 it;
    const int tj = item % d.ntj;
    const int r = item / d.ntj;
    it.ti = r % d.nti;
    const int kk = r / d.nti;
    it.i0 = it.ti * S::TI;
    it.j0 = 1 + tj * S::R2;
    it.kb = 1 + kk * d.kdepth;
    it.nout = min(d.K - 1, it.kb + d.kdepth) - it.kb;
    return it;
}

// VI values of an intermediate-plane row (no halo) with the left and right
// neighbours by lane shuffles; the edge lanes get `left` / `right`.
__device__ __forceinline__ void q_ext(const float *row, int lane, float left, float right, float (&e)[6])
{
    const float4 v = *reinterpret_cast<const float4 *>(row + 4 * lane);
    e[1] = v.x; e[2] = v.y; e[3] = v.z; e[4] = v.w;
    const float l = __shfl_up_sync(0xffffffffu, e[4], 1);
    const float r = __shfl_down_sync(0xffffffffu, e[1], 1);
    e[0] = (lane == 0) ? left : l;
    e[5] = (lane == 31) ? right : r;
}

// 16 bytes global -> shared without a register round trip (cached in L2
// only); the copies of a thread complete at cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(Sweep2Shape::THREADS, 1)
k_sweep2(const __grid_constant__ Sweep2Desc d, const Sweep2Args a)
{
    using S = Sweep2Shape;
    constexpr int VI = S::VI, TI = S::TI, H = S::H, R1 = S::R1, RP = S::RP, RC = S::RC, RQ = S::RQ;
    extern __shared__ unsigned char dsm2_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(dsm2_raw) + 127) & ~uintptr_t(127));
    unsigned char *ring_q = base + (size_t)RP * S::P_BYTES;
    unsigned char *ring_c = ring_q + (size_t)RQ * S::Q_BYTES;
    unsigned char *bufs2 = ring_c + (size_t)RC * S::C_BYTES;   // per sweep-2 warp
    __shared__ __align__(8) uint64_t p_full[RP], p_empty[RP], c_full[RC], c_empty[RC], q_full[RQ], q_empty[RQ],
        cons_bar;
    __shared__ volatile int s_abort;
    __shared__ double s_part[R1];
    __shared__ float q_edge[RQ][R1][2];   // sweep-1 values at columns i0-1 and i0+128, per row

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RP; ++s) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], R1 + 1); }
        for (int s = 0; s < RC; ++s) { mbar_init(&c_full[s], 1); mbar_init(&c_empty[s], R1); }
        for (int s = 0; s < RQ; ++s) { mbar_init(&q_full[s], R1 + 1); mbar_init(&q_empty[s], R1); }
        mbar_init(&cons_bar, R1);
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == R1) {
        // ------------------------------------------------------------ producer
        // One lane copies, per item, the coefficient stage of each sweep-1
        // plane (twelve 128 x R1 tiles) and the state planes of p_t with a
        // halo of 4 columns and 2 rows, in the order the consumers use them:
        // state planes 0 and 1, then per step s state plane s+2 and stage
        // s+1.  Before the state of pass t >= 1 it waits on the grid barrier
        // of the pass before (the first stage of the pass does not need it).
        if (lane == 0) {
            const uint64_t pol_c = l2_policy(0);   // sweep 2 reads the tiles again from L2
            const uint64_t pol_keep = l2_policy(1);
            const uint64_t pol_p = l2_policy(a.l2_keep_state ? 1 : 0);
            uint32_t pc = 0, cc = 0;
            bool ok = true;
            const CUtensorMap *pm = nullptr;
            auto put_state = [&](const Item2 &it, int q) -> bool {
                const uint32_t slot = pc % RP, use = pc / RP;
                if (use > 0 && !mbar_wait_bounded(&p_empty[slot], (use - 1) & 1)) return false;
                if (s_abort) return false;
                mbar_arrive_expect_tx(&p_full[slot], (uint32_t)S::P_BYTES);
                tma_load_3d_hint(base + (size_t)slot * S::P_BYTES, pm, &p_full[slot], it.i0 - H, it.j0 - 2,
                                 it.kb - 2 + q, pol_p);
                ++pc;
                return true;
            };
            auto put_coef = [&](const Item2 &it, int q) -> bool {
                const uint32_t slot = cc % RC, use = cc / RC;
                if (use > 0 && !mbar_wait_bounded(&c_empty[slot], (use - 1) & 1)) return false;
                if (s_abort) return false;
                unsigned char *st = ring_c + (size_t)slot * S::C_BYTES;
                mbar_arrive_expect_tx(&c_full[slot], (uint32_t)S::C_BYTES);
                for (int k = JAC_A0; k <= JAC_BND; ++k)
                    tma_load_3d_hint(st + (size_t)(k - 1) * S::TILE, &d.coef[k - 1], &c_full[slot], it.i0,
                                     it.j0 - 1, it.kb - 1 + q, ((a.l2_keep_coef >> k) & 1u) ? pol_keep : pol_c);
                ++cc;
                return true;
            };
            for (int t = 0; t < a.n_pass && ok; ++t) {
                pm = ((t + a.par) & 1) ? &d.p[1] : &d.p[0];
                bool first = true;
                for (int item = blockIdx.x; item < d.nitems && ok; item += G) {
                    const Item2 it = decode_item2(d, item);
                    if (!(ok = put_coef(it, 0))) break;
                    if (t > 0 && first) {
                        if (!(ok = wait_counter_bounded(&a.hdr->gbar, (unsigned)t * G))) break;
                        fence_proxy_async_global();
                    }
                    first = false;
                    if (!(ok = put_state(it, 0) && put_state(it, 1))) break;
                    for (int q = 0; q < it.nout + 2 && ok; ++q) {
                        ok = put_state(it, q + 2);
                        if (ok && q + 1 < it.nout + 2) ok = put_coef(it, q + 1);
                    }
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
            for (uint32_t s = 0; s < (uint32_t)RP && s < pc; ++s) {
                const uint32_t last = pc - 1 - ((pc - 1 - s) % RP);
                (void)mbar_wait_bounded(&p_full[s], (last / RP) & 1);
            }
        }
    } else if (warp == S::EDGE_WARP) {
        // ----------------------------------------------------------- edge warp
        // Lane 2r + e (r < R1) computes sweep 1 at row j0-1+r and column
        // i0-1 (e = 0) or i0+128 (e = 1), the neighbours that sweep 2 needs
        // past the tile's 128 columns, with the consumers' arithmetic.  Its
        // twelve coefficients come from global memory one plane ahead.
        const int r = lane >> 1, side = lane & 1;
        const bool act = lane < 2 * R1;
        const float omega = (float)a.omega;
        const int I = d.I, J = d.J, K = d.K, pitch = d.pitch;
        const int x = side ? H + TI : H - 1;             // the column in the state box
        const int r0 = r * S::PW, r1 = (r + 1) * S::PW, r2 = (r + 2) * S::PW;
        uint32_t pc = 0, qc = 0;
        bool ok = true;
        for (int t = 0; t < a.n_pass && ok; ++t) {
            for (int item = blockIdx.x; item < d.nitems && ok; item += G) {
                const Item2 it = decode_item2(d, item);
                const int j = it.j0 - 1 + r;
                const int ie = side ? it.i0 + TI : it.i0 - 1;
                const bool col_in = act && (j >= 1) && (j <= J - 2) && (ie >= 1) && (ie <= I - 2);
                float cf[12], cn[12];
                auto load_coef = [&](int m, float (&v)[12]) {
                    if (col_in && m >= 1 && m <= K - 2) {
                        const size_t off = ((size_t)m * J + (size_t)j) * (size_t)pitch + (size_t)ie;
#pragma unroll
                        for (int q = 0; q < 12; ++q) v[q] = __ldg(d.coef_ptr[q] + off);
                    } else {
#pragma unroll
                        for (int q = 0; q < 12; ++q) v[q] = 0.0f;
                    }
                };
                load_coef(it.kb - 1, cf);
                for (int s = 0; s < it.nout + 2; ++s) {
                    const int m = it.kb - 1 + s;
                    if (s == 0) {
                        ok = mbar_wait_bounded(&p_full[pc % RP], (pc / RP) & 1) &&
                             mbar_wait_bounded(&p_full[(pc + 1) % RP], ((pc + 1) / RP) & 1);
                    }
                    const uint32_t q2 = pc + s + 2;
                    ok = ok && mbar_wait_bounded(&p_full[q2 % RP], (q2 / RP) & 1);
                    const uint32_t qs = qc + s;
                    if (qs >= RQ) ok = ok && mbar_wait_bounded(&q_empty[qs % RQ], ((qs / RQ) - 1) & 1);
                    ok = __all_sync(0xffffffffu, ok && !s_abort);
                    if (!ok) break;
                    if (s + 1 < it.nout + 2) load_coef(m + 1, cn);
                    if (act) {
                        const float *Pm = reinterpret_cast<const float *>(base + (size_t)((pc + s) % RP) * S::P_BYTES);
                        const float *Pk =
                            reinterpret_cast<const float *>(base + (size_t)((pc + s + 1) % RP) * S::P_BYTES);
                        const float *Pp = reinterpret_cast<const float *>(base + (size_t)(q2 % RP) * S::P_BYTES);
                        const float c = Pk[r1 + x];
                        float out = c;
                        if (col_in && m >= 1 && m <= K - 2) {
                            const float bij = ((Pk[r2 + x + 1] - Pk[r0 + x + 1]) - Pk[r2 + x - 1]) + Pk[r0 + x - 1];
                            const float bjk = ((Pp[r2 + x] - Pm[r2 + x]) - Pp[r0 + x]) + Pm[r0 + x];
                            const float bik = ((Pp[r1 + x + 1] - Pm[r1 + x + 1]) - Pp[r1 + x - 1]) + Pm[r1 + x - 1];
                            const float ss = ss_f32<false>(c, Pk[r1 + x + 1], Pk[r1 + x - 1], Pk[r2 + x], Pk[r0 + x],
                                                           Pp[r1 + x], Pm[r1 + x], bij, bjk, bik, cf[0], cf[1], cf[2],
                                                           cf[3], cf[4], cf[5], cf[6], cf[7], cf[8], cf[9], cf[10],
                                                           cf[11]);
                            out = fmaf(omega, ss, c);
                        }
                        q_edge[qs % RQ][r][side] = out;
                    }
#pragma unroll
                    for (int q = 0; q < 12; ++q) cf[q] = cn[q];
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&q_full[qs % RQ]);            // the edge values of intermediate plane s
                        mbar_arrive(&p_empty[(pc + s) % RP]);     // state plane m-1 is done
                    }
                }
                if (!ok) break;
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&p_empty[(pc + it.nout + 2) % RP]);
                    mbar_arrive(&p_empty[(pc + it.nout + 3) % RP]);
                }
                pc += it.nout + 4;
                qc += it.nout + 2;
            }
        }
        if (!ok) {
            s_abort = 1;
            atomicExch(&a.hdr->errword, (int)JAC_ETIMEOUT);
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int w = warp;                         // row j0-1+w of every item
        const float omega = (float)a.omega;
        const uint64_t st_pol = l2_policy(a.l2_keep_state ? 1 : 0);
        const int I = d.I, J = d.J, K = d.K, pitch = d.pitch;
        uint32_t pc = 0, cc = 0, qc = 0;
        bool ok = true;
        double acc = 0.0;
        uint32_t sync_phase = 0;
        auto cons_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(&cons_bar);
            const bool r = mbar_wait_bounded(&cons_bar, sync_phase & 1);
            ++sync_phase;
            return __all_sync(0xffffffffu, r);
        };
        const bool do2 = (w >= 1) && (w <= R1 - 2);  // this warp's row is an output row too

        for (int t = 0; t < a.n_pass && ok; ++t) {
            const bool res = (t == a.n_pass - 1) && (a.res != nullptr);
            float *p_out = static_cast<float *>(((t + 1 + a.par) & 1) ? d.p_buf[1] : d.p_buf[0]);
            for (int item = blockIdx.x; item < d.nitems && ok; item += G) {
                const Item2 it = decode_item2(d, item);
                const int j = it.j0 - 1 + w;
                const int ib = it.i0 + VI * lane;
                const bool row1_in = (j >= 1) && (j <= J - 2);
                bool in_i[VI], owned[VI];
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    in_i[e] = (ib + e >= 1) && (ib + e <= I - 2);
                    owned[e] = do2 && row1_in && in_i[e];
                }
                bool all_owned = true, any_owned = false;
#pragma unroll
                for (int e = 0; e < VI; ++e) {
                    all_owned = all_owned && owned[e];
                    any_owned = any_owned || owned[e];
                }
                const int r0 = w * S::PW, r1 = (w + 1) * S::PW, r2 = (w + 2) * S::PW;   // rows j-1, j, j+1
                const int cidx = w * TI + VI * lane;
                float *buf2 = reinterpret_cast<float *>(bufs2 + (size_t)(do2 ? w - 1 : 0) * S::B_BYTES);
                // a3 S - 1 of this row's points at the sweep-1 planes of the
                // last two steps, carried to sweep 2 at those planes
                float ec1[VI], ec2[VI];
#pragma unroll
                for (int e = 0; e < VI; ++e) ec1[e] = ec2[e] = 0.0f;

                for (int s = 0; s < it.nout + 3; ++s) {
                    const int m = it.kb - 1 + s;                 // sweep-1 plane
                    const uint32_t qs = qc + s;
                    float ec0[VI];
#pragma unroll
                    for (int e = 0; e < VI; ++e) ec0[e] = 0.0f;
                    if (s < it.nout + 2) {
                        // ---- sweep 1 at plane m, row j, into intermediate plane s
                        if (s == 0) {
                            ok = mbar_wait_bounded(&p_full[pc % RP], (pc / RP) & 1) &&
                                 mbar_wait_bounded(&p_full[(pc + 1) % RP], ((pc + 1) / RP) & 1);
                        }
                        const uint32_t q2 = pc + s + 2;
                        ok = ok && mbar_wait_bounded(&p_full[q2 % RP], (q2 / RP) & 1);
                        ok = ok && mbar_wait_bounded(&c_full[(cc + s) % RC], ((cc + s) / RC) & 1);
                        if (qs >= RQ) ok = ok && mbar_wait_bounded(&q_empty[qs % RQ], ((qs / RQ) - 1) & 1);
                        ok = __all_sync(0xffffffffu, ok && !s_abort);
                        if (!ok) break;
                        const float *Pm = reinterpret_cast<const float *>(base + (size_t)((pc + s) % RP) * S::P_BYTES);
                        const float *Pk =
                            reinterpret_cast<const float *>(base + (size_t)((pc + s + 1) % RP) * S::P_BYTES);
                        const float *Pp = reinterpret_cast<const float *>(base + (size_t)(q2 % RP) * S::P_BYTES);
                        const unsigned char *cs = ring_c + (size_t)((cc + s) % RC) * S::C_BYTES;
                        float ek0[VI + 2], ek1[VI + 2], ek2[VI + 2], em1[VI + 2], ep1[VI + 2];
                        float vm0[VI], vm2[VI], vp0[VI], vp2[VI];
                        load_ext<float, VI, H>(Pk + r0, lane, 32, ek0);
                        load_ext<float, VI, H>(Pk + r1, lane, 32, ek1);
                        load_ext<float, VI, H>(Pk + r2, lane, 32, ek2);
                        load_ext<float, VI, H>(Pm + r1, lane, 32, em1);
                        load_ext<float, VI, H>(Pp + r1, lane, 32, ep1);
                        lds_vec<float, VI>(Pm + r0 + H + VI * lane, vm0);
                        lds_vec<float, VI>(Pm + r2 + H + VI * lane, vm2);
                        lds_vec<float, VI>(Pp + r0 + H + VI * lane, vp0);
                        lds_vec<float, VI>(Pp + r2 + H + VI * lane, vp2);
                        float ca0[VI], ca1[VI], ca2[VI], ca3[VI], cb0[VI], cb1[VI], cb2[VI], cc0[VI], cc1[VI],
                            cc2[VI], cwk[VI], cbn[VI];
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 0 * S::TILE) + cidx, ca0);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 1 * S::TILE) + cidx, ca1);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 2 * S::TILE) + cidx, ca2);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 3 * S::TILE) + cidx, ca3);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 4 * S::TILE) + cidx, cb0);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 5 * S::TILE) + cidx, cb1);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 6 * S::TILE) + cidx, cb2);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 7 * S::TILE) + cidx, cc0);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 8 * S::TILE) + cidx, cc1);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 9 * S::TILE) + cidx, cc2);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 10 * S::TILE) + cidx, cwk);
                        lds_vec<float, VI>(reinterpret_cast<const float *>(cs + 11 * S::TILE) + cidx, cbn);
                        const bool in1 = row1_in && (m >= 1) && (m <= K - 2);
                        float out[VI];
#pragma unroll
                        for (int e = 0; e < VI; ++e) {
                            const float c = ek1[e + 1];
                            const float bij = ((ek2[e + 2] - ek0[e + 2]) - ek2[e]) + ek0[e];
                            const float bjk = ((vp2[e] - vm2[e]) - vp0[e]) + vm0[e];
                            const float bik = ((ep1[e + 2] - em1[e + 2]) - ep1[e]) + em1[e];
                            ec0[e] = a3s_minus_one<false>(ca3[e], ca0[e], ca1[e], ca2[e], cc0[e], cc1[e], cc2[e]);
                            const float ss = ss_f32_ec(c, ek1[e + 2], ek1[e], ek2[e + 1], ek0[e + 1], ep1[e + 1],
                                                       em1[e + 1], bij, bjk, bik, ca0[e], ca1[e], ca2[e], ca3[e],
                                                       cb0[e], cb1[e], cb2[e], cc0[e], cc1[e], cc2[e], cwk[e], cbn[e],
                                                       ec0[e]);
                            out[e] = (in1 && in_i[e]) ? fmaf(omega, ss, c) : c;
                        }
                        float *qrow = reinterpret_cast<float *>(ring_q + (size_t)(qs % RQ) * S::Q_BYTES) + w * TI;
                        *reinterpret_cast<float4 *>(qrow + VI * lane) = make_float4(out[0], out[1], out[2], out[3]);
                        if (a.mid != nullptr && m >= it.kb && m < it.kb + it.nout) {
                            // the intermediate state at this item's own points
                            const size_t offm = ((size_t)m * J + (size_t)j) * (size_t)pitch + (size_t)ib;
                            if (all_owned) {
                                store_vec<float, VI>(a.mid + offm, out, st_pol);
                            } else {
#pragma unroll
                                for (int e = 0; e < VI; ++e)
                                    if (owned[e]) a.mid[offm + e] = out[e];
                            }
                        }
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&q_full[qs % RQ]);            // intermediate plane s: this row written
                            mbar_arrive(&p_empty[(pc + s) % RP]);     // state plane m-1 is done
                            mbar_arrive(&c_empty[(cc + s) % RC]);     // stage s is done
                        }
                    }

                    if (s >= 3) {
                        // ---- sweep 2 at plane m-2 from intermediate planes s-3 .. s-1;
                        // its coefficients come from global memory (the stage
                        // that held them served sweep 1 two steps ago)
                        const int m2 = m - 2;
                        const size_t off = ((size_t)m2 * J + (size_t)j) * (size_t)pitch + (size_t)ib;
                        for (int qq = 0; qq < 3 && ok; ++qq) {
                            const uint32_t qw = qc + s - 3 + qq;
                            ok = mbar_wait_bounded(&q_full[qw % RQ], (qw / RQ) & 1);
                        }
                        ok = __all_sync(0xffffffffu, ok && !s_abort);
                        if (!ok) break;
                        if (do2) {
                            const float *Qm =
                                reinterpret_cast<const float *>(ring_q + (size_t)((qs - 3) % RQ) * S::Q_BYTES);
                            const float *Qk =
                                reinterpret_cast<const float *>(ring_q + (size_t)((qs - 2) % RQ) * S::Q_BYTES);
                            const float *Qp =
                                reinterpret_cast<const float *>(ring_q + (size_t)((qs - 1) % RQ) * S::Q_BYTES);
                            const int q0 = (w - 1) * TI, q1 = w * TI, q2r = (w + 1) * TI;
                            // columns i0-1 and i0+128 come from the edge warp
                            const float(*Em)[2] = q_edge[(qs - 3) % RQ];
                            const float(*Ek)[2] = q_edge[(qs - 2) % RQ];
                            const float(*Ep)[2] = q_edge[(qs - 1) % RQ];
                            float ek0[VI + 2], ek1[VI + 2], ek2[VI + 2], em1[VI + 2], ep1[VI + 2];
                            float vm0[VI], vm2[VI], vp0[VI], vp2[VI];
                            q_ext(Qk + q0, lane, Ek[w - 1][0], Ek[w - 1][1], ek0);
                            q_ext(Qk + q1, lane, Ek[w][0], Ek[w][1], ek1);
                            q_ext(Qk + q2r, lane, Ek[w + 1][0], Ek[w + 1][1], ek2);
                            q_ext(Qm + q1, lane, Em[w][0], Em[w][1], em1);
                            q_ext(Qp + q1, lane, Ep[w][0], Ep[w][1], ep1);
                            lds_vec<float, VI>(Qm + q0 + VI * lane, vm0);
                            lds_vec<float, VI>(Qm + q2r + VI * lane, vm2);
                            lds_vec<float, VI>(Qp + q0 + VI * lane, vp0);
                            lds_vec<float, VI>(Qp + q2r + VI * lane, vp2);
                            // this lane's own copies (issued a step ago) have landed
                            cp_async_wait_all();
                            float ca0[VI], ca1[VI], ca2[VI], ca3[VI], cb0[VI], cb1[VI], cb2[VI], cc0[VI], cc1[VI],
                                cc2[VI], cwk[VI], cbn[VI];
                            lds_vec<float, VI>(buf2 + 0 * TI + VI * lane, ca0);
                            lds_vec<float, VI>(buf2 + 1 * TI + VI * lane, ca1);
                            lds_vec<float, VI>(buf2 + 2 * TI + VI * lane, ca2);
                            lds_vec<float, VI>(buf2 + 3 * TI + VI * lane, ca3);
                            lds_vec<float, VI>(buf2 + 4 * TI + VI * lane, cb0);
                            lds_vec<float, VI>(buf2 + 5 * TI + VI * lane, cb1);
                            lds_vec<float, VI>(buf2 + 6 * TI + VI * lane, cb2);
                            lds_vec<float, VI>(buf2 + 7 * TI + VI * lane, cc0);
                            lds_vec<float, VI>(buf2 + 8 * TI + VI * lane, cc1);
                            lds_vec<float, VI>(buf2 + 9 * TI + VI * lane, cc2);
                            lds_vec<float, VI>(buf2 + 10 * TI + VI * lane, cwk);
                            lds_vec<float, VI>(buf2 + 11 * TI + VI * lane, cbn);
                            float out[VI];
                            float ss2 = 0.0f;
#pragma unroll
                            for (int e = 0; e < VI; ++e) {
                                const float c = ek1[e + 1];
                                const float bij = ((ek2[e + 2] - ek0[e + 2]) - ek2[e]) + ek0[e];
                                const float bjk = ((vp2[e] - vm2[e]) - vp0[e]) + vm0[e];
                                const float bik = ((ep1[e + 2] - em1[e + 2]) - ep1[e]) + em1[e];
                                const float ss = ss_f32_ec(c, ek1[e + 2], ek1[e], ek2[e + 1], ek0[e + 1], ep1[e + 1],
                                                           em1[e + 1], bij, bjk, bik, ca0[e], ca1[e], ca2[e], ca3[e],
                                                           cb0[e], cb1[e], cb2[e], cc0[e], cc1[e], cc2[e], cwk[e],
                                                           cbn[e], ec2[e]);
                                out[e] = owned[e] ? fmaf(omega, ss, c) : c;
                                if (res && owned[e]) ss2 = fmaf(ss, ss, ss2);
                            }
                            if (res) acc += (double)ss2;
                            if (all_owned) {
                                store_vec<float, VI>(p_out + off, out, st_pol);
                            } else {
#pragma unroll
                                for (int e = 0; e < VI; ++e)
                                    if (owned[e]) p_out[off + e] = out[e];
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&q_empty[(qs - 3) % RQ]);   // intermediate plane s-3 done
                    }
                    // the coefficients of the next step's sweep 2 (plane m-1),
                    // into this warp's buffer, which sweep 2 above has read
                    if (do2 && s + 1 >= 3 && s + 1 <= it.nout + 2) {   // the same for every lane
                        __syncwarp();
                        if (any_owned) {
                            const size_t offn = ((size_t)(m - 1) * J + (size_t)j) * (size_t)pitch + (size_t)ib;
#pragma unroll
                            for (int q = 0; q < 12; ++q)
                                cp_async16(buf2 + q * TI + VI * lane, d.coef_ptr[q] + offn);
                        }
                        cp_async_commit();
                    }
#pragma unroll
                    for (int e = 0; e < VI; ++e) {
                        ec2[e] = ec1[e];
                        ec1[e] = ec0[e];
                    }
                }
                if (!ok) break;
                // the item's last state planes and intermediate planes
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&p_empty[(pc + it.nout + 2) % RP]);
                    mbar_arrive(&p_empty[(pc + it.nout + 3) % RP]);
                    mbar_arrive(&q_empty[(qc + it.nout) % RQ]);
                    mbar_arrive(&q_empty[(qc + it.nout + 1) % RQ]);
                }
                pc += it.nout + 4;
                cc += it.nout + 2;
                qc += it.nout + 2;
            }
            if (!ok) break;
            if (res) {
                double v = acc;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) s_part[w] = v;
                if (!cons_sync()) { ok = false; break; }
                if (threadIdx.x == 0) {
                    double sum = 0.0, comp = 0.0;
                    for (int q = 0; q < R1; ++q) neumaier_add(sum, comp, s_part[q]);
                    a.partials[blockIdx.x] = sum + comp;
                }
                acc = 0.0;
                if (!cons_sync()) { ok = false; break; }
            }
            if (t + 1 < a.n_pass) {
                // publish this CTA's part of the pass to every CTA's TMA reads
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
        cp_async_wait_all();   // no copy into this CTA's shared memory outlives it
    }

    // CTA epilogue: the last CTA to finish sums the partials in CTA order
    // and resets the workspace counters for the next launch.
    // If any CTA gave up a wait, the residual is written as NaN.
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.hdr->counter, 1u);
        s_last = (prev == (unsigned)G - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x == 0) {
            if (a.res != nullptr) {
                if (s_abort || workspace_failed(a.hdr)) {
                    *a.res = __longlong_as_double(0x7ff8000000000000ll);
                } else {
                    double sum = 0.0, comp = 0.0;
                    for (int b = 0; b < G; ++b) neumaier_add(sum, comp, __ldcg(&a.partials[b]));
                    *a.res = sum + comp;
                }
            }
            a.hdr->gbar = 0u;
            a.hdr->counter = 0u;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------ host side
namespace {

jac_status fail2(jac_status st, const std::string &msg)
{
    set_thread_error(msg);
    return st;
}

}  // namespace

// Tiles in i: columns 128 n .. 128 n + 127, until one holds column I-2.
int sweep2_tiles_i(int I)
{
    using S = Sweep2Shape;
    return (I - 2) / S::TI + 1;
}

// Output planes per item: the depth that minimises the rounds of items over
// `ctas` CTAs times the steps of an item (its planes, the two extra planes
// of sweep 1 and about two steps of start-up); ties go to the shallower.
int sweep2_kdepth(long cols, int nk, int ctas)
{
    if (nk <= 2) return std::max(nk, 1);
    long best_cost = -1;
    int best = 2;
    int prev = -1;
    for (int n = 1; n <= nk; ++n) {
        const int kd = std::max(2, (nk + n - 1) / n);
        if (kd == prev) continue;
        prev = kd;
        const long items = cols * (long)((nk + kd - 1) / kd);
        const long rounds = (items + ctas - 1) / ctas;
        const long cost = rounds * (long)(kd + 4);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && kd < best)) {
            best_cost = cost;
            best = kd;
        }
    }
    return best;
}

size_t sweep2_workspace_bytes(const jac_grid *g)
{
    using S = Sweep2Shape;
    const long long cols = (long long)sweep2_tiles_i(g->I) * ((g->J - 2 + S::R2 - 1) / S::R2);
    const int sms = device_sm_count();
    const int kd = sweep2_kdepth(cols, g->K - 2, sms);
    const long long items = cols * ((g->K - 2 + kd - 1) / kd);
    return kWsHeaderBytes + round_up((size_t)std::min<long long>(items, sms) * sizeof(double), 256);
}

jac_status sweep2_run(const jac_grid *g, int kdepth, int n_pass, double *d_residual, void *workspace,
                      size_t ws_bytes, cudaStream_t st, void *mid)
{
    using S = Sweep2Shape;
    if (mid != nullptr && n_pass != 1) return fail2(JAC_EINVAL, "the intermediate state needs a one-pass call");
    Sweep2Desc d;
    std::memset(&d, 0, sizeof(d));
    d.I = g->I; d.J = g->J; d.K = g->K;
    d.pitch = jac_pitch(g->I);
    d.nti = sweep2_tiles_i(g->I);
    d.ntj = (g->J - 2 + S::R2 - 1) / S::R2;
    const int sms = device_sm_count();
    d.kdepth = kdepth > 0 ? kdepth : sweep2_kdepth((long)d.nti * d.ntj, g->K - 2, sms);
    d.nkb = (g->K - 2 + d.kdepth - 1) / d.kdepth;
    const long long items = (long long)d.nti * d.ntj * d.nkb;
    if (items > 0x3fffffffLL) return fail2(JAC_EINVAL, "grid too large for the two-sweep launch shape");
    d.nitems = (int)items;
    d.p_buf[0] = g->p[0];
    d.p_buf[1] = g->p[1];
    jac_status s;
    for (int b = 0; b < 2; ++b)
        if ((s = encode_box_map(&d.p[b], g->p[b], 4, d.pitch, d.pitch, g->J, g->K, S::PW, S::PH)) != JAC_OK)
            return s;
    for (int q = JAC_A0; q <= JAC_BND; ++q) {
        if ((s = encode_box_map(&d.coef[q - 1], g->coef[q], 4, d.pitch, d.pitch, g->J, g->K, S::TI, S::R1)) !=
            JAC_OK)
            return s;
        d.coef_ptr[q - 1] = static_cast<const float *>(g->coef[q]);
    }
    const unsigned nblocks = (unsigned)std::min<long long>(items, sms);
    if (ws_bytes < kWsHeaderBytes + (size_t)nblocks * sizeof(double))
        return fail2(JAC_EINVAL, "workspace too small for the two-sweep launch");
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    Sweep2Args a;
    std::memset(&a, 0, sizeof(a));
    a.n_pass = n_pass;
    a.par = 0;
    a.omega = g->omega;
    a.partials = reinterpret_cast<double *>(static_cast<char *>(workspace) + kWsHeaderBytes);
    a.res = d_residual;
    a.mid = static_cast<float *>(mid);
    a.hdr = hdr;
    SweepArgs la;
    std::memset(&la, 0, sizeof(la));
    set_l2_policy(la, g->prec, (size_t)d.pitch * g->J * g->K);
    a.l2_keep_state = la.l2_keep_state;
    a.l2_keep_coef = la.l2_keep_coef;

    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(k_sweep2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    });
    if (attr_err != cudaSuccess)
        return fail2(JAC_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(attr_err));
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(S::THREADS);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_sweep2, d, a);
    if (e != cudaSuccess) return fail2(JAC_ECUDA, std::string("two-sweep launch: ") + cudaGetErrorString(e));
    return JAC_OK;
}

}  // namespace jac
