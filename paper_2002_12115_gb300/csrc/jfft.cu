// 3-D complex FFT block of libjac (include/jfft.h): the FFT workload of the
// paper's evaluation (NAS.FT, Section 5.1.1) and the function-block offload
// it names as next step (Section 6), device-resident on GB300.
//
// One kernel launch per axis.  A CTA owns W whole lines along the axis of
// the pass and transforms them in registers and shared memory:
//   * mixed-radix Stockham FFT of length N = R1 R2 R3 (radices 2..16):
//     stage s reads R values at stride N / R, multiplies by the twiddles
//     W_{Ns R}^{(j mod Ns) r} (from a table of W_N^m computed on the host in
//     FP64), does an R-point DFT in registers (radix-2 decimation in
//     frequency with constant twiddles, its bit-reversed output order folded
//     into the register indices) and writes R values at stride Ns, Ns = R1
//     ... R(s-1);
//   * the first stage reads global memory and the last writes it; the
//     stages between exchange through a padded shared-memory tile;
//   * passes along y and z give a CTA W lines of consecutive x (W * element
//     size = 128 bytes), lanes running over those lines, so every global
//     access is a run of 128 bytes; the pass along x gives a CTA W rows with
//     lanes running along the row;
//   * the spectral step multiplies the data by exp(-4 pi^2 alpha t |kbar|^2)
//     as the first pass loads it (a per-CTA table of the factor along the
//     axis times one factor per line), and the last pass scales by 1/N as it
//     stores and sums |u|^2 per CTA in FP64; a one-CTA kernel then adds the
//     per-CTA sums in a fixed order, so the energy is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/jfft.h"
#include "jac_internal.h"

namespace jfft {

template <typename T>
struct alignas(2 * sizeof(T)) C2 {
    T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }

// z * w (INV = false) or z * conj(w) (INV = true)
template <typename T, bool INV>
__device__ __forceinline__ C2<T> cmul(C2<T> z, C2<T> w)
{
    if (INV) return {z.x * w.x + z.y * w.y, z.y * w.x - z.x * w.y};
    return {z.x * w.x - z.y * w.y, z.x * w.y + z.y * w.x};
}

// cos(2 pi m / 16)
__host__ __device__ constexpr double cos16(int m)
{
    m &= 15;
    if (m > 8) m = 16 - m;
    return m == 0   ? 1.0
           : m == 1 ? 0.92387953251128675613
           : m == 2 ? 0.70710678118654752440
           : m == 3 ? 0.38268343236508977173
           : m == 4 ? 0.0
           : m == 5 ? -0.38268343236508977173
           : m == 6 ? -0.70710678118654752440
           : m == 7 ? -0.92387953251128675613
                    : -1.0;
}

// z * exp(-+ 2 pi i m / 16) (forward: minus), m a compile-time constant
// after unrolling; the trivial factors 1 and -+i cost no multiply.
template <typename T, bool INV, int M>
__device__ __forceinline__ C2<T> rot16(C2<T> z)
{
    constexpr int m = M & 15;
    if constexpr (m == 0) {
        return z;
    } else if constexpr (m == 4) {
        return INV ? C2<T>{-z.y, z.x} : C2<T>{z.y, -z.x};
    } else {
        constexpr T c = (T)cos16(m), s = (T)cos16(m + 12);   // sin(2 pi m / 16)
        return INV ? C2<T>{z.x * c - z.y * s, z.x * s + z.y * c} : C2<T>{z.x * c + z.y * s, z.y * c - z.x * s};
    }
}

// One level of the in-register radix-2 decimation-in-frequency DFT of R
// points: butterflies of span HALF, then the next level.  After all levels
// X[k] sits at v[brev(k)].
template <typename T, int R, int HALF, bool INV>
struct Dif {
    template <int BLK, int K>
    static __device__ __forceinline__ void bfly(C2<T> *v)
    {
        if constexpr (BLK < R) {
            if constexpr (K < HALF) {
                const C2<T> a = v[BLK + K], b = v[BLK + K + HALF];
                v[BLK + K] = a + b;
                v[BLK + K + HALF] = rot16<T, INV, K * (8 / HALF)>(a - b);
                bfly<BLK, K + 1>(v);
            } else {
                bfly<BLK + 2 * HALF, 0>(v);
            }
        }
    }
    static __device__ __forceinline__ void run(C2<T> *v)
    {
        bfly<0, 0>(v);
        Dif<T, R, HALF / 2, INV>::run(v);
    }
};
template <typename T, int R, bool INV>
struct Dif<T, R, 0, INV> {
    static __device__ __forceinline__ void run(C2<T> *) {}
};

__host__ __device__ constexpr int brev(int k, int R)
{
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

// Radices of a length-N transform: up to three stages of at most 16.
template <int N>
struct Radix {
    static constexpr int R1 = N <= 16 ? N : (N == 32 ? 4 : (N == 64 ? 8 : (N == 128 ? 8 : (N == 256 ? 16 :
                                                            (N == 512 ? 8 : 4)))));
    static constexpr int R2 = N <= 16 ? 1 : (N == 32 ? 8 : (N == 64 ? 8 : (N == 128 ? 16 : (N == 256 ? 16 :
                                                            (N == 512 ? 8 : 16)))));
    static constexpr int R3 = N <= 256 ? 1 : (N == 512 ? 8 : 16);
    static constexpr int RMAX = R1 > R2 ? (R1 > R3 ? R1 : R3) : (R2 > R3 ? R2 : R3);
    static_assert(R1 * R2 * R3 == N, "radix plan");
};

// Elements of a line each thread holds.  The pass along x keeps the
// largest radix (more lanes along each row); the passes along y and z take
// up to 16, so that fewer threads serve a line and a CTA of at most 512
// threads covers up to 256 bytes of consecutive x.
template <typename T, int N, bool YZ>
__host__ __device__ constexpr int elems_per_thread()
{
    constexpr int rmax = Radix<N>::RMAX;
    constexpr int want = N / 16 > rmax ? N / 16 : rmax;
    return YZ ? (want < 16 ? want : 16) : rmax;
}

// CTAs per SM the kernel is built for: for FP32, two 512-thread CTAs of the
// passes along y and z and four 256-thread CTAs of the pass along x (at
// most 64 registers a thread), so that one CTA's loads overlap another's
// butterflies; FP64 (bound by its ALU) keeps the registers it wants.
template <typename T, bool YZ>
__host__ __device__ constexpr int min_ctas_per_sm()
{
    return sizeof(T) == 4 ? (YZ ? 2 : 4) : 1;
}

// Shared-memory index of element e of a line: one pad element after every
// 16 (FP32) or 8 (FP64) elements, so that butterfly writes at stride R do
// not fall on one bank.
template <typename T>
__host__ __device__ constexpr int pad_idx(int e)
{
    return sizeof(T) == 4 ? e + (e >> 4) : e + (e >> 3);
}

// Row stride of the tile (elements): the padded line plus one, with the
// stride odd in units of 32 bytes, so that lanes on different lines at the
// same element do not share a bank.
template <typename T, int N>
__host__ __device__ constexpr int row_stride()
{
    constexpr int a = sizeof(T) == 4 ? 16 : 8;
    return (pad_idx<T>(N - 1) + 1 + a - 1) / a * a + 1;
}

struct PassArgs {
    const void *in;
    void *out;
    const void *tw;          // W_N^m, m = 0 .. N-1, of this axis (forward sign)
    int n1, n2, n3;
    int axis;                // 0: x, 1: y, 2: z
    int W;                   // lines per CTA
    double scale;            // applied by the last stage (1 or 1/N)
    int factor;              // multiply by the spectral factor on load (first pass of a step)
    const void *fa;          // factor tables exp(c kbar^2) (element type T): this pass's axis,
    const void *fb;          // and the line's other two axes (for the pass along x: y, then z)
    const void *fc;
    double *partials;        // per-CTA sums of |u|^2 (written when energy != NULL)
    double *energy;
};

__device__ __forceinline__ double kbar2(int k, int n)
{
    const int s = k < (n + 1) / 2 ? k : k - n;
    return (double)s * (double)s;
}

// The spectral factor along each axis, exp(c kbar^2) for every index of
// n1, then n2, then n3 (FP64 exp, stored as T): one small launch per step,
// so that a pass multiplies by a table entry per element and one per line.
template <typename T>
__global__ void k_fft_factors(double c, int n1, int n2, int n3, T *f1, T *f2, T *f3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) f1[i] = (T)exp(c * kbar2(i, n1));
    else if (i < n1 + n2) f2[i - n1] = (T)exp(c * kbar2(i - n1, n2));
    else if (i < n1 + n2 + n3) f3[i - n1 - n2] = (T)exp(c * kbar2(i - n1 - n2, n3));
}

// One Stockham stage for the BPT = RMAX / R butterflies of this thread.
template <typename T, int N, int R, int RMAX, int NS, bool INV, bool FIRST, bool LAST>
__device__ __forceinline__ void stage(C2<T> (&v)[RMAX], C2<T> *tile, const C2<T> *tw, const C2<T> *gin, C2<T> *gout,
                                      long long lb, long long es, int w, int t, const T *fe, T fl, T scale,
                                      bool factor, T &esum, bool want_energy)
{
    constexpr int TT = N / RMAX;       // threads per line
    constexpr int BPT = RMAX / R;      // butterflies per thread
    constexpr int RS = row_stride<T, N>();
    C2<T> *row = tile + w * RS;
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int j = t + q * TT;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * (N / R);
            if constexpr (FIRST) {
                C2<T> x = gin[lb + (long long)e * es];
                if (factor) {
                    const T f = fe[e] * fl;
                    x.x *= f;
                    x.y *= f;
                }
                v[q * R + r] = x;
            } else {
                v[q * R + r] = row[pad_idx<T>(e)];
            }
        }
    }
    if constexpr (!FIRST && !LAST) __syncthreads();   // every read of the tile before any write
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int j = t + q * TT;
        if constexpr (NS > 1) {
            const int jm = j & (NS - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[q * R + r] = cmul<T, INV>(v[q * R + r], tw[jm * r * (N / (NS * R))]);
        }
        Dif<T, R, R / 2, INV>::run(&v[q * R]);
    }
    T e_loc = (T)0;     // this thread's |u|^2, summed in T over its outputs
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int j = t + q * TT;
        const int idx = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = idx + r * NS;
            C2<T> x = v[q * R + brev(r, R)];
            if constexpr (LAST) {
                x.x *= scale;
                x.y *= scale;
                gout[lb + (long long)e * es] = x;
                if (want_energy) e_loc = fma(x.x, x.x, fma(x.y, x.y, e_loc));
            } else {
                row[pad_idx<T>(e)] = x;
            }
        }
    }
    if constexpr (LAST) esum += e_loc;
    if constexpr (!LAST) __syncthreads();
}

template <typename T, int N, bool INV, bool YZ>
__global__ void __launch_bounds__(YZ ? 512 : 256, min_ctas_per_sm<T, YZ>()) k_fft_pass(const PassArgs a)
{
    using RX = Radix<N>;
    constexpr int RMAX = elems_per_thread<T, N, YZ>();   // elements per thread
    constexpr int TT = N / RMAX;
    constexpr int RS = row_stride<T, N>();
    extern __shared__ __align__(16) unsigned char jfft_smem[];
    const int W = a.W;
    C2<T> *tile = reinterpret_cast<C2<T> *>(jfft_smem);
    C2<T> *tw = tile + (RX::R2 > 1 ? W * RS : 0);
    T *fe = reinterpret_cast<T *>(tw + N);
    T *fl = fe + N;
    __shared__ double red[512];

    // this thread's line and position in it
    int w, t;
    if (a.axis == 0) { t = threadIdx.x % TT; w = threadIdx.x / TT; }
    else { w = threadIdx.x % W; t = threadIdx.x / W; }
    const long long n1 = a.n1, n2 = a.n2;
    long long lb, es;              // first element of the line, element stride
    int ia, ib, na, nb;            // the line's indices on the other two axes, and their extents
    if (a.axis == 0) {
        const long long row = (long long)blockIdx.x * W + w;     // row = z * n2 + y
        lb = row * n1;
        es = 1;
        ia = (int)(row % n2); na = a.n2;
        ib = (int)(row / n2); nb = a.n3;
    } else {
        const int xt = blockIdx.x % (a.n1 / W);
        const int o = blockIdx.x / (a.n1 / W);                   // z (y pass) or y (z pass)
        const int x = xt * W + w;
        ia = x; na = a.n1;
        ib = o; nb = a.axis == 1 ? a.n3 : a.n2;
        lb = a.axis == 1 ? (long long)o * n1 * n2 + x : (long long)o * n1 + x;
        es = a.axis == 1 ? n1 : n1 * n2;
    }

    // twiddles (and the spectral factor along this axis) into shared memory
    const C2<T> *gtw = static_cast<const C2<T> *>(a.tw);
    const T *gfa = static_cast<const T *>(a.fa);
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        if constexpr (RX::R2 > 1) tw[m] = gtw[m];
        if (a.factor) fe[m] = gfa[m];
    }
    if (a.factor && t == 0) fl[w] = static_cast<const T *>(a.fb)[ia] * static_cast<const T *>(a.fc)[ib];
    (void)na;
    (void)nb;
    __syncthreads();

    const C2<T> *gin = static_cast<const C2<T> *>(a.in);
    C2<T> *gout = static_cast<C2<T> *>(a.out);
    const bool want_energy = a.energy != nullptr;
    const T scale = (T)a.scale;
    const T flw = a.factor ? fl[w] : (T)1;
    T esum = (T)0;
    C2<T> v[RMAX];
    constexpr int R1 = RX::R1, R2 = RX::R2, R3 = RX::R3;
    if constexpr (R2 == 1) {
        stage<T, N, R1, RMAX, 1, INV, true, true>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                  a.factor, esum, want_energy);
    } else if constexpr (R3 == 1) {
        stage<T, N, R1, RMAX, 1, INV, true, false>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                   a.factor, esum, want_energy);
        stage<T, N, R2, RMAX, R1, INV, false, true>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                    a.factor, esum, want_energy);
    } else {
        stage<T, N, R1, RMAX, 1, INV, true, false>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                   a.factor, esum, want_energy);
        stage<T, N, R2, RMAX, R1, INV, false, false>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                     a.factor, esum, want_energy);
        stage<T, N, R3, RMAX, R1 * R2, INV, false, true>(v, tile, tw, gin, gout, lb, es, w, t, fe, flw, scale,
                                                         a.factor, esum, want_energy);
    }
    if (!want_energy) return;

    // energy: a pairwise tree over the block in T (warp shuffles, then the
    // warps' sums in shared memory; log2 of the block's size roundings, and
    // FP64 only for the CTA's one partial -- GB300's FP64 pipe is narrow);
    // k_fft_energy adds the partials after the pass
    __shared__ T tred[32];
    T v_e = esum;
    if ((blockDim.x & 31) == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v_e += __shfl_down_sync(0xffffffffu, v_e, o);
        if ((threadIdx.x & 31) == 0) tred[threadIdx.x >> 5] = v_e;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            T x = threadIdx.x < nw ? tred[threadIdx.x] : (T)0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (threadIdx.x == 0) a.partials[blockIdx.x] = (double)x;
        }
    } else {                                   // blocks of fewer than 32 threads (short lines)
        red[threadIdx.x] = (double)v_e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (unsigned i = 0; i < blockDim.x; ++i) sum += red[i];
            a.partials[blockIdx.x] = sum;
        }
    }
}

// Sum of the n per-CTA energy partials of the last pass, in a fixed order:
// thread t adds the partials t, t + 512, ... (four independent loads in
// flight), then a pairwise tree over the 512 threads.  One CTA of 512
// threads.
__global__ void __launch_bounds__(512) k_fft_energy(const double *__restrict__ partials, int n, double *energy)
{
    __shared__ double red[512];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int b = t; b < n; b += 4 * 512) {
        s0 += partials[b];
        if (b + 512 < n) s1 += partials[b + 512];
        if (b + 1024 < n) s2 += partials[b + 1024];
        if (b + 1536 < n) s3 += partials[b + 1536];
    }
    red[t] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    for (int h = 256; h > 0; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) *energy = red[0];
}

// ---------------------------------------------------------------- host
namespace {

bool pow2_in_range(int n) { return n >= JFFT_MIN_N && n <= JFFT_MAX_N && (n & (n - 1)) == 0; }

size_t elem_bytes(jfft_prec p) { return p == JFFT_C64 ? 16 : 8; }

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Largest radix of a length-N transform (Radix<N>::RMAX), on the host.
int rmax_of(int N)
{
    if (N <= 16) return N;
    return (N == 32 || N == 64 || N == 512) ? 8 : 16;
}

// Elements per thread (elems_per_thread<T, N, YZ> on the host).
int elems_of(int N, jfft_prec prec, bool yz)
{
    (void)prec;
    const int rmax = rmax_of(N);
    if (!yz) return rmax;
    return std::min(std::max(N / 16, rmax), 16);
}

// Lines per CTA of a pass (see the kernel's mapping): rows of about 256
// threads for the pass along x; for y and z, 256 bytes of consecutive x
// (32 FP32 or 16 FP64 complex values), at most 512 threads.
int lines_per_cta(int axis, int N, const int n[3], jfft_prec prec)
{
    const int tt = N / elems_of(N, prec, axis != 0);
    if (axis == 0) return std::max(1, std::min(256 / tt, n[1] * n[2]));
    return std::max(1, std::min(std::min(prec == JFFT_C64 ? 16 : 32, n[0]), 512 / tt));
}

long long ctas_of_pass(int axis, const int n[3], int W)
{
    if (axis == 0) return (long long)n[1] * n[2] / W;
    return (long long)(n[0] / W) * (axis == 1 ? n[2] : n[1]);
}

int threads_of_pass(int N, int W, jfft_prec prec, bool yz) { return (N / elems_of(N, prec, yz)) * W; }

struct Layout {
    size_t tw[3];       // offsets of the twiddle tables
    size_t fac[3];      // offsets of the spectral factor tables
    size_t partials;
    size_t total;
    long long max_ctas;
};

Layout layout(const int n[3], jfft_prec prec)
{
    Layout L;
    size_t off = 256;                     // header (reserved)
    for (int a = 0; a < 3; ++a) {
        L.tw[a] = off;
        off += round256((size_t)n[a] * elem_bytes(prec));
    }
    for (int a = 0; a < 3; ++a) {
        L.fac[a] = off;
        off += round256((size_t)n[a] * elem_bytes(prec) / 2);
    }
    L.max_ctas = 0;
    for (int a = 0; a < 3; ++a)
        L.max_ctas = std::max(L.max_ctas, ctas_of_pass(a, n, lines_per_cta(a, n[a], n, prec)));
    L.partials = off;
    off += round256((size_t)L.max_ctas * sizeof(double));
    L.total = off;
    return L;
}

jac_status check_shape(int n1, int n2, int n3, jfft_prec prec)
{
    if (!pow2_in_range(n1) || !pow2_in_range(n2) || !pow2_in_range(n3)) {
        jac::set_thread_error("every extent must be a power of two in [" + std::to_string(JFFT_MIN_N) + ", " +
                              std::to_string(JFFT_MAX_N) + "]");
        return JAC_EINVAL;
    }
    if (prec != JFFT_C64 && prec != JFFT_C32) {
        jac::set_thread_error("unknown FFT precision");
        return JAC_EINVAL;
    }
    return JAC_OK;
}

}  // namespace

// Launch of one pass: the kernel instantiation for (T, N, INV).
template <typename T, bool INV, bool YZ>
jac_status launch_pass_t(int N, const PassArgs &a, unsigned grid, unsigned block, cudaStream_t st)
{
    size_t smem = 0;
    void (*kern)(PassArgs) = nullptr;
    switch (N) {
#define JFFT_CASE(NN)                                                                                       \
    case NN:                                                                                                \
        kern = k_fft_pass<T, NN, INV, YZ>;                                                                  \
        smem = (Radix<NN>::R2 > 1 ? (size_t)a.W * row_stride<T, NN>() * sizeof(C2<T>) : 0) +               \
               (size_t)NN * sizeof(C2<T>) + (size_t)NN * sizeof(T) + (size_t)a.W * sizeof(T);               \
        break;
        JFFT_CASE(2) JFFT_CASE(4) JFFT_CASE(8) JFFT_CASE(16) JFFT_CASE(32) JFFT_CASE(64) JFFT_CASE(128)
        JFFT_CASE(256) JFFT_CASE(512) JFFT_CASE(1024)
#undef JFFT_CASE
    default:
        jac::set_thread_error("unsupported FFT length");
        return JAC_EINVAL;
    }
    smem = (smem + 15) / 16 * 16;
    // opt in to more than the default dynamic shared memory (the kernel's
    // static reduction buffer counts against the same 48 KB); once per
    // kernel and size
    if (smem > 32 * 1024) {
        static std::mutex mu;
        static std::vector<std::pair<const void *, size_t>> done;
        std::lock_guard<std::mutex> lk(mu);
        auto it = std::find_if(done.begin(), done.end(), [&](const std::pair<const void *, size_t> &d) {
            return d.first == (const void *)kern;
        });
        if (it == done.end() || it->second < smem) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) {
                jac::set_thread_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
                return JAC_ECUDA;
            }
            if (it == done.end()) done.emplace_back((const void *)kern, smem);
            else it->second = smem;
        }
    }
    kern<<<grid, block, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        jac::set_thread_error(std::string("FFT pass launch: ") + cudaGetErrorString(e));
        return JAC_ECUDA;
    }
    return JAC_OK;
}

}  // namespace jfft

struct jfft_plan {
    int n[3] = {0, 0, 0};
    jfft_prec prec = JFFT_C32;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    jfft::Layout L{};
    std::string err;
};

namespace {

jac_status plan_fail(jfft_plan *p, jac_status s, const std::string &m)
{
    if (p) p->err = m;
    jac::set_thread_error(m);
    return s;
}

jac_status plan_from_thread(jfft_plan *p, jac_status s)
{
    if (s != JAC_OK && p) p->err = jac::thread_last_error();
    return s;
}

// The three passes of one transform.  first_in: the input of the first
// pass; every later pass works in place on `out`.
jac_status run3(jfft_plan *p, const void *in, void *out, bool inv, double scale, bool factor, double c,
                double *energy)
{
    if (!p) return plan_fail(p, JAC_EINVAL, "plan is NULL");
    if (!in || !out || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return plan_fail(p, JAC_EINVAL, "data arrays must be non-NULL and 16-byte aligned");
    if (in != out) {
        const size_t bytes = (size_t)p->n[0] * p->n[1] * p->n[2] * jfft::elem_bytes(p->prec);
        const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
        if (a < b + bytes && b < a + bytes) return plan_fail(p, JAC_EINVAL, "in and out overlap without being equal");
    }
    if (factor) {
        const int nt = p->n[0] + p->n[1] + p->n[2];
        if (p->prec == JFFT_C32)
            jfft::k_fft_factors<float><<<(nt + 255) / 256, 256, 0, p->stream>>>(
                c, p->n[0], p->n[1], p->n[2], reinterpret_cast<float *>(p->ws + p->L.fac[0]),
                reinterpret_cast<float *>(p->ws + p->L.fac[1]), reinterpret_cast<float *>(p->ws + p->L.fac[2]));
        else
            jfft::k_fft_factors<double><<<(nt + 255) / 256, 256, 0, p->stream>>>(
                c, p->n[0], p->n[1], p->n[2], reinterpret_cast<double *>(p->ws + p->L.fac[0]),
                reinterpret_cast<double *>(p->ws + p->L.fac[1]), reinterpret_cast<double *>(p->ws + p->L.fac[2]));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return plan_fail(p, JAC_ECUDA, std::string("factor launch: ") + cudaGetErrorString(e));
    }
    for (int axis = 0; axis < 3; ++axis) {
        const int N = p->n[axis];
        jfft::PassArgs a;
        std::memset(&a, 0, sizeof(a));
        a.in = axis == 0 ? in : out;
        a.out = out;
        a.tw = p->ws + p->L.tw[axis];
        a.n1 = p->n[0]; a.n2 = p->n[1]; a.n3 = p->n[2];
        a.axis = axis;
        a.W = jfft::lines_per_cta(axis, N, p->n, p->prec);
        a.scale = axis == 2 ? scale : 1.0;
        a.factor = (factor && axis == 0) ? 1 : 0;
        a.fa = p->ws + p->L.fac[0];
        a.fb = p->ws + p->L.fac[1];
        a.fc = p->ws + p->L.fac[2];
        if (axis == 2 && energy) {
            a.energy = energy;
            a.partials = reinterpret_cast<double *>(p->ws + p->L.partials);
        }
        const unsigned grid = (unsigned)jfft::ctas_of_pass(axis, p->n, a.W);
        const unsigned block = (unsigned)jfft::threads_of_pass(N, a.W, p->prec, axis != 0);
        jac_status s;
        const bool yz = axis != 0;
        if (p->prec == JFFT_C32)
            s = inv ? (yz ? jfft::launch_pass_t<float, true, true>(N, a, grid, block, p->stream)
                          : jfft::launch_pass_t<float, true, false>(N, a, grid, block, p->stream))
                    : (yz ? jfft::launch_pass_t<float, false, true>(N, a, grid, block, p->stream)
                          : jfft::launch_pass_t<float, false, false>(N, a, grid, block, p->stream));
        else
            s = inv ? (yz ? jfft::launch_pass_t<double, true, true>(N, a, grid, block, p->stream)
                          : jfft::launch_pass_t<double, true, false>(N, a, grid, block, p->stream))
                    : (yz ? jfft::launch_pass_t<double, false, true>(N, a, grid, block, p->stream)
                          : jfft::launch_pass_t<double, false, false>(N, a, grid, block, p->stream));
        if (s != JAC_OK) return plan_from_thread(p, s);
        if (axis == 2 && energy) {
            jfft::k_fft_energy<<<1, 512, 0, p->stream>>>(reinterpret_cast<double *>(p->ws + p->L.partials), (int)grid,
                                                         energy);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return plan_fail(p, JAC_ECUDA, std::string("energy launch: ") + cudaGetErrorString(e));
        }
    }
    return JAC_OK;
}

}  // namespace

extern "C" {

jac_status jfft_workspace_size(int n1, int n2, int n3, jfft_prec prec, size_t *bytes)
{
    if (!bytes) return plan_fail(nullptr, JAC_EINVAL, "bytes is NULL");
    jac_status s = jfft::check_shape(n1, n2, n3, prec);
    if (s != JAC_OK) return s;
    const int n[3] = {n1, n2, n3};
    *bytes = jfft::layout(n, prec).total;
    return JAC_OK;
}

jac_status jfft_plan_create(jfft_plan **out, int n1, int n2, int n3, jfft_prec prec, void *stream, void *workspace,
                            size_t ws_bytes)
{
    if (!out) return plan_fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    jac_status s = jfft::check_shape(n1, n2, n3, prec);
    if (s != JAC_OK) return s;
    const int n[3] = {n1, n2, n3};
    const jfft::Layout L = jfft::layout(n, prec);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return plan_fail(nullptr, JAC_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (ws_bytes < L.total)
        return plan_fail(nullptr, JAC_EINVAL, "workspace too small: need " + std::to_string(L.total) + " bytes");
    jfft_plan *p = new (std::nothrow) jfft_plan;
    if (!p) return plan_fail(nullptr, JAC_ENOMEM, "host allocation failed");
    p->n[0] = n1; p->n[1] = n2; p->n[2] = n3;
    p->prec = prec;
    p->stream = static_cast<cudaStream_t>(stream);
    p->ws = static_cast<char *>(workspace);
    p->L = L;
    // twiddle tables W_N^m = exp(-2 pi i m / N), in FP64 on the host, stored in the plan's precision
    std::vector<unsigned char> host(L.fac[0] - 256, 0);
    const double pi = 3.14159265358979323846264338327950288;
    for (int a = 0; a < 3; ++a) {
        unsigned char *dst = host.data() + (L.tw[a] - 256);
        for (int m = 0; m < n[a]; ++m) {
            const double re = std::cos(2.0 * pi * m / n[a]), im = -std::sin(2.0 * pi * m / n[a]);
            if (prec == JFFT_C64) {
                const double v[2] = {re, im};
                std::memcpy(dst + (size_t)m * 16, v, 16);
            } else {
                const float v[2] = {(float)re, (float)im};
                std::memcpy(dst + (size_t)m * 8, v, 8);
            }
        }
    }
    cudaError_t e = cudaMemsetAsync(p->ws, 0, 256, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->ws + 256, host.data(), host.size(), cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        delete p;
        return plan_fail(nullptr, JAC_ECUDA, std::string("plan set-up: ") + cudaGetErrorString(e));
    }
    *out = p;
    return JAC_OK;
}

jac_status jfft_destroy(jfft_plan *p)
{
    if (!p) return JAC_OK;
    cudaStreamSynchronize(p->stream);
    delete p;
    return JAC_OK;
}

const char *jfft_last_error(const jfft_plan *p) { return p ? p->err.c_str() : jac::thread_last_error(); }

jac_status jfft_forward(jfft_plan *p, const void *in, void *out)
{
    return run3(p, in, out, false, 1.0, false, 0.0, nullptr);
}

jac_status jfft_inverse(jfft_plan *p, const void *in, void *out)
{
    if (!p) return plan_fail(p, JAC_EINVAL, "plan is NULL");
    return run3(p, in, out, true, 1.0 / ((double)p->n[0] * p->n[1] * p->n[2]), false, 0.0, nullptr);
}

jac_status jfft_evolve(jfft_plan *p, const void *U, double alpha, double t, void *out, double *d_energy)
{
    if (!p) return plan_fail(p, JAC_EINVAL, "plan is NULL");
    if (!std::isfinite(alpha) || !std::isfinite(t) || alpha * t < 0.0)
        return plan_fail(p, JAC_EINVAL, "alpha and t must be finite with alpha * t >= 0");
    const double pi = 3.14159265358979323846264338327950288;
    const double c = -4.0 * pi * pi * alpha * t;
    return run3(p, U, out, true, 1.0 / ((double)p->n[0] * p->n[1] * p->n[2]), true, c, d_energy);
}

}  // extern "C"
