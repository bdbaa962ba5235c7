/*
 * FP64 CPU oracle of the 3-D complex discrete Fourier transform and of one
 * spectral time step built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The GPU
 * product path never calls it, and it shares no code with the CUDA sources.
 *
 * What it computes.  The paper evaluates its offloading on NAS.FT, an FFT
 * application, beside the Himeno benchmark (Section 5.1.1), and names the
 * offload of whole function blocks such as the FFT as its next step (Section
 * 6).  The transform is the plain definition, one axis at a time:
 *
 *   X[k] = sum_{j=0}^{n-1} x[j] exp(sign * 2 pi i j k / n),  sign = -1 forward,
 *
 * applied along x, then y, then z of an n1 x n2 x n3 array (the 3-D DFT is
 * separable, so this is its definition summed in a fixed order).  The
 * inverse uses sign = +1 and scales by 1 / (n1 n2 n3).  Each output is an
 * O(n) sum; exp(2 pi i m / n) is taken from a table of libm cos/sin at the
 * exact integer phase m = j k mod n.
 *
 * The spectral step (heat equation u_t = alpha laplace(u) on the periodic
 * unit cube, solved exactly in Fourier space): given the forward transform
 * U of an initial field, the field at time t is
 *
 *   u(t) = inverse( U[k] * exp(-4 pi^2 alpha t |kbar|^2) ),
 *
 * with kbar the signed frequency (k for k < n/2, k - n otherwise, per
 * axis); its energy sum |u(t)|^2 is accumulated with Neumaier compensation.
 *
 * Layout: interleaved complex doubles (re, im), x fastest, then y, then z:
 * the element (x, y, z) at complex index (z*n2 + y)*n1 + x.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define FFT_OK 0
#define FFT_EINVAL 1
#define FFT_ENOMEM 2

static const double kPi = 3.14159265358979323846264338327950288;

typedef struct { double s, c; } fneumaier;

static void fnm_add(fneumaier *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}

/* DFT of every line along `axis` (0: x, 1: y, 2: z) of the n1 x n2 x n3
 * array `in` into `out` (may not alias).  sign: -1 or +1.  Unscaled. */
int fft_oracle_dft_axis(int n1, int n2, int n3, int axis, int sign, const double *in, double *out)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || axis < 0 || axis > 2 || (sign != 1 && sign != -1) || !in || !out ||
        in == out)
        return FFT_EINVAL;
    const int dims[3] = {n1, n2, n3};
    const int n = dims[axis];
    const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)n1 : (size_t)n1 * n2);
    /* lines: the index of the first element of every line along `axis` */
    const size_t nlines = (size_t)n1 * n2 * n3 / (size_t)n;
    double *tw = (double *)malloc(2 * (size_t)n * sizeof(double));
    if (!tw) return FFT_ENOMEM;
    for (int m = 0; m < n; ++m) {
        tw[2 * m] = cos(2.0 * kPi * m / n);
        tw[2 * m + 1] = sign * sin(2.0 * kPi * m / n);
    }
#pragma omp parallel for schedule(static)
    for (long long l = 0; l < (long long)nlines; ++l) {
        size_t base;
        if (axis == 0) {
            base = (size_t)l * n1;
        } else if (axis == 1) {                  /* l = z*n1 + x */
            const size_t z = (size_t)l / n1, x = (size_t)l % n1;
            base = z * n1 * n2 + x;
        } else {                                 /* l = y*n1 + x */
            base = (size_t)l;
        }
        for (int k = 0; k < n; ++k) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; ++j) {
                const size_t m = ((size_t)j * (size_t)k) % (size_t)n;
                const double *a = in + 2 * (base + (size_t)j * stride);
                const double wr = tw[2 * m], wi = tw[2 * m + 1];
                re += a[0] * wr - a[1] * wi;
                im += a[0] * wi + a[1] * wr;
            }
            double *b = out + 2 * (base + (size_t)k * stride);
            b[0] = re;
            b[1] = im;
        }
    }
    free(tw);
    return FFT_OK;
}

/* 3-D transform: the axis DFTs along x, y, z in that order.  sign = -1:
 * forward, unscaled; sign = +1: inverse, scaled by 1 / (n1 n2 n3).
 * `out` may equal `in`. */
int fft_oracle_fft3(int n1, int n2, int n3, int sign, const double *in, double *out)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || !in || !out) return FFT_EINVAL;
    const size_t N = (size_t)n1 * n2 * n3;
    double *a = (double *)malloc(2 * N * sizeof(double));
    double *b = (double *)malloc(2 * N * sizeof(double));
    if (!a || !b) { free(a); free(b); return FFT_ENOMEM; }
    int rc = fft_oracle_dft_axis(n1, n2, n3, 0, sign, in, a);
    if (!rc) rc = fft_oracle_dft_axis(n1, n2, n3, 1, sign, a, b);
    if (!rc) rc = fft_oracle_dft_axis(n1, n2, n3, 2, sign, b, a);
    if (!rc) {
        if (sign == 1) {
            const double s = 1.0 / (double)N;
            for (size_t q = 0; q < 2 * N; ++q) a[q] *= s;
        }
        memcpy(out, a, 2 * N * sizeof(double));
    }
    free(a);
    free(b);
    return rc;
}

/* Signed frequency of index k on an axis of n points. */
static double kbar(int k, int n) { return (double)(k < (n + 1) / 2 ? k : k - n); }

/* The spectral step: out = inverse(U * exp(-4 pi^2 alpha t |kbar|^2)) and
 * *energy = sum |out|^2.  `out` may equal `U`. */
int fft_oracle_evolve(int n1, int n2, int n3, double alpha, double t, const double *U, double *out,
                      double *energy)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || !U || !out) return FFT_EINVAL;
    const size_t N = (size_t)n1 * n2 * n3;
    double *w = (double *)malloc(2 * N * sizeof(double));
    if (!w) return FFT_ENOMEM;
    const double c = -4.0 * kPi * kPi * alpha * t;
    for (int z = 0; z < n3; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n1; ++x) {
                const double kx = kbar(x, n1), ky = kbar(y, n2), kz = kbar(z, n3);
                const double f = exp(c * (kx * kx + ky * ky + kz * kz));
                const size_t q = ((size_t)z * n2 + y) * n1 + x;
                w[2 * q] = U[2 * q] * f;
                w[2 * q + 1] = U[2 * q + 1] * f;
            }
    int rc = fft_oracle_fft3(n1, n2, n3, 1, w, out);
    free(w);
    if (rc) return rc;
    if (energy) {
        fneumaier e = {0.0, 0.0};
        for (size_t q = 0; q < 2 * N; ++q) fnm_add(&e, out[q] * out[q]);
        *energy = e.s + e.c;
    }
    return FFT_OK;
}

/* One output of the 3-D DFT straight from its definition (a single O(N)
 * sum over all points, not separated by axis): X[kx, ky, kz] for sign = -1
 * (unscaled), or the unscaled inverse for sign = +1.  out: 2 doubles. */
int fft_oracle_point(int n1, int n2, int n3, int sign, const double *in, int kx, int ky, int kz, double *out)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || (sign != 1 && sign != -1) || !in || !out || kx < 0 || kx >= n1 ||
        ky < 0 || ky >= n2 || kz < 0 || kz >= n3)
        return FFT_EINVAL;
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int z = 0; z < n3; ++z)
        for (int y = 0; y < n2; ++y)
            for (int x = 0; x < n1; ++x) {
                /* phase = kx x / n1 + ky y / n2 + kz z / n3, in turns, from exact integer products */
                const double ph = (double)(((long long)kx * x) % n1) / n1 + (double)(((long long)ky * y) % n2) / n2 +
                                  (double)(((long long)kz * z) % n3) / n3;
                const double wr = cos(2.0 * kPi * ph), wi = sign * sin(2.0 * kPi * ph);
                const double *a = in + 2 * (((size_t)z * n2 + y) * n1 + x);
                re += a[0] * wr - a[1] * wi;
                im += a[0] * wi + a[1] * wr;
            }
    out[0] = re;
    out[1] = im;
    return FFT_OK;
}
