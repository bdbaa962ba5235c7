/*
 * FP64 CPU oracle of the 19-point variable-coefficient Jacobi sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The GPU
 * product path never calls it, and it shares no code with the CUDA sources.
 *
 * What it computes (the Himeno-style Poisson relaxation that the paper's
 * offloading method targets, Section 5.1.1, with the stencil fixed by the
 * workload definition since the paper does not write it out):
 *
 *   for every interior point x = (i, j, k), 1 <= i <= I-2 (same for j, k):
 *     s0 = a0*p[i+1] + a1*p[j+1] + a2*p[k+1]
 *        + b0*(p[i+1,j+1] - p[i+1,j-1] - p[i-1,j+1] + p[i-1,j-1])
 *        + b1*(p[j+1,k+1] - p[j+1,k-1] - p[j-1,k+1] + p[j-1,k-1])
 *        + b2*(p[i+1,k+1] - p[i+1,k-1] - p[i-1,k+1] + p[i-1,k-1])
 *        + c0*p[i-1] + c1*p[j-1] + c2*p[k-1] + wrk1
 *     ss = (s0*a3 - p[x]) * bnd
 *     p'[x] = p[x] + omega*ss
 *   Coefficients are read at x.  Faces are never written.  Every read comes
 *   from the previous sweep (Jacobi, double buffered).  The residual of a
 *   sweep is gosa = sum over the interior of ss^2, computed from that sweep's
 *   input state.
 *
 * Arithmetic: plain FP64, terms summed in the order written above.  Build with
 * -ffp-contract=off so that no multiply-add is fused.  The residual is a
 * Neumaier-compensated sum, taken per k-plane in (j, i) order and then over
 * planes in k order, so its value does not depend on the thread count.
 *
 * The reverse-mode adjoint keeps every state p_0 .. p_T and applies the
 * transposed sweep in scatter form: each interior point x pushes
 * coef(x) * w(x) into the neighbour that coefficient multiplied in x's row.
 *
 * Layout: dense arrays, i fastest, then j, then k: index (k*J + j)*I + i.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    const double *a0, *a1, *a2, *a3;
    const double *b0, *b1, *b2;
    const double *c0, *c1, *c2;
    const double *wrk1, *bnd;
} oracle_fields;

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

typedef struct { double s, c; } neumaier;

static void nm_add(neumaier *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}

/* s0 at interior point (i, j, k) of state p, terms in the written order. */
static double s0_at(const oracle_fields *f, const double *p,
                    int I, int J, int i, int j, int k)
{
    const size_t sj = (size_t)I, sk = (size_t)I * (size_t)J;
    const size_t x = (size_t)k * sk + (size_t)j * sj + (size_t)i;
    double bij = p[x + 1 + sj] - p[x + 1 - sj] - p[x - 1 + sj] + p[x - 1 - sj];
    double bjk = p[x + sj + sk] - p[x + sj - sk] - p[x - sj + sk] + p[x - sj - sk];
    double bik = p[x + 1 + sk] - p[x + 1 - sk] - p[x - 1 + sk] + p[x - 1 - sk];
    double s0 = f->a0[x] * p[x + 1] + f->a1[x] * p[x + sj] + f->a2[x] * p[x + sk]
              + f->b0[x] * bij + f->b1[x] * bjk + f->b2[x] * bik
              + f->c0[x] * p[x - 1] + f->c1[x] * p[x - sj] + f->c2[x] * p[x - sk]
              + f->wrk1[x];
    return s0;
}

/* One Jacobi sweep p_in -> p_out; *gosa receives the sweep's residual.
 * state_f32 != 0 models a state stored in FP32: each new interior value is
 * rounded to the nearest FP32 number (the arithmetic stays FP64). */
int oracle_sweep(int I, int J, int K, const oracle_fields *f, double omega,
                 const double *p_in, double *p_out, double *gosa, int state_f32)
{
    if (I < 3 || J < 3 || K < 3 || !f || !p_in || !p_out || p_in == p_out)
        return ORACLE_EINVAL;
    const size_t N = (size_t)I * J * K;
    memcpy(p_out, p_in, N * sizeof(double));        /* faces keep their values */
    double *plane = (double *)calloc((size_t)K, sizeof(double));
    if (!plane) return ORACLE_ENOMEM;
    const size_t sk = (size_t)I * J;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < K - 1; ++k) {
        neumaier acc = {0.0, 0.0};
        for (int j = 1; j < J - 1; ++j) {
            for (int i = 1; i < I - 1; ++i) {
                const size_t x = (size_t)k * sk + (size_t)j * I + (size_t)i;
                double s0 = s0_at(f, p_in, I, J, i, j, k);
                double ss = (s0 * f->a3[x] - p_in[x]) * f->bnd[x];
                nm_add(&acc, ss * ss);
                double pn = p_in[x] + omega * ss;
                p_out[x] = state_f32 ? (double)(float)pn : pn;
            }
        }
        plane[k] = acc.s + acc.c;
    }
    neumaier tot = {0.0, 0.0};
    for (int k = 1; k < K - 1; ++k) nm_add(&tot, plane[k]);
    free(plane);
    if (gosa) *gosa = tot.s + tot.c;
    return ORACLE_OK;
}

/* n sweeps starting from p (overwritten with p_n); *gosa = residual of sweep n
 * (0 when n == 0).  state_f32 as for oracle_sweep. */
int oracle_run(int I, int J, int K, const oracle_fields *f, double omega, int n,
               double *p, double *gosa, int state_f32)
{
    if (I < 3 || J < 3 || K < 3 || !f || !p || n < 0) return ORACLE_EINVAL;
    const size_t N = (size_t)I * J * K;
    if (gosa) *gosa = 0.0;
    if (n == 0) return ORACLE_OK;
    double *tmp = (double *)malloc(N * sizeof(double));
    if (!tmp) return ORACLE_ENOMEM;
    double *src = p, *dst = tmp;
    for (int t = 0; t < n; ++t) {
        int rc = oracle_sweep(I, J, K, f, omega, src, dst, gosa, state_f32);
        if (rc) { free(tmp); return rc; }
        double *sw = src; src = dst; dst = sw;
    }
    if (src != p) memcpy(p, src, N * sizeof(double));
    free(tmp);
    return ORACLE_OK;
}

/*
 * Reverse-mode gradient of L = 1/2 * sum over all points of (p_T - target)^2
 * after T sweeps from p0.  Outputs (each N doubles unless noted):
 *   loss (1 double), pT, g_p0 = dL/dp0, g_wrk1, g_a3, and, if g_coef is not
 *   NULL, 9*N doubles holding dL/d{a0,a1,a2,b0,b1,b2,c0,c1,c2} in that order.
 * The bnd array is treated as fixed data (no gradient).
 */
int oracle_adjoint(int I, int J, int K, const oracle_fields *f, double omega, int T,
                   const double *p0, const double *target, double *loss, double *pT,
                   double *g_p0, double *g_wrk1, double *g_a3, double *g_coef)
{
    if (I < 3 || J < 3 || K < 3 || !f || !p0 || !target || T < 0 ||
        !loss || !pT || !g_p0 || !g_wrk1 || !g_a3)
        return ORACLE_EINVAL;
    const size_t N = (size_t)I * J * K;
    const size_t sj = (size_t)I, sk = (size_t)I * J;
    double *states = (double *)malloc((size_t)(T + 1) * N * sizeof(double));
    double *lam_next = (double *)malloc(N * sizeof(double));
    if (!states || !lam_next) { free(states); free(lam_next); return ORACLE_ENOMEM; }

    /* forward pass, keeping every state */
    memcpy(states, p0, N * sizeof(double));
    for (int t = 0; t < T; ++t)
        oracle_sweep(I, J, K, f, omega, states + (size_t)t * N, states + (size_t)(t + 1) * N, NULL, 0);
    const double *p_last = states + (size_t)T * N;
    memcpy(pT, p_last, N * sizeof(double));

    /* terminal adjoint lambda_T = dL/dp_T */
    double *lam = g_p0;
    neumaier L = {0.0, 0.0};
    for (size_t x = 0; x < N; ++x) {
        double d = p_last[x] - target[x];
        lam[x] = d;
        nm_add(&L, 0.5 * d * d);
    }
    *loss = L.s + L.c;

    memset(g_wrk1, 0, N * sizeof(double));
    memset(g_a3, 0, N * sizeof(double));
    double *ga[9] = {0};
    if (g_coef) {
        memset(g_coef, 0, 9 * N * sizeof(double));
        for (int q = 0; q < 9; ++q) ga[q] = g_coef + (size_t)q * N;
    }

    for (int t = T - 1; t >= 0; --t) {
        const double *p = states + (size_t)t * N;
        memcpy(lam_next, lam, N * sizeof(double));   /* identity part */
        for (int k = 1; k < K - 1; ++k)
            for (int j = 1; j < J - 1; ++j)
                for (int i = 1; i < I - 1; ++i) {
                    const size_t x = (size_t)k * sk + (size_t)j * sj + (size_t)i;
                    double mu = omega * f->bnd[x] * lam_next[x];
                    double w = f->a3[x] * mu;
                    /* p'[x] = (1 - omega*bnd) p[x] + omega*bnd*a3*s0: the -p part */
                    lam[x] -= mu;
                    /* scatter: s0's coefficient of each neighbour, times w */
                    lam[x + 1]  += f->a0[x] * w;
                    lam[x + sj] += f->a1[x] * w;
                    lam[x + sk] += f->a2[x] * w;
                    lam[x + 1 + sj] += f->b0[x] * w;
                    lam[x + 1 - sj] -= f->b0[x] * w;
                    lam[x - 1 + sj] -= f->b0[x] * w;
                    lam[x - 1 - sj] += f->b0[x] * w;
                    lam[x + sj + sk] += f->b1[x] * w;
                    lam[x + sj - sk] -= f->b1[x] * w;
                    lam[x - sj + sk] -= f->b1[x] * w;
                    lam[x - sj - sk] += f->b1[x] * w;
                    lam[x + 1 + sk] += f->b2[x] * w;
                    lam[x + 1 - sk] -= f->b2[x] * w;
                    lam[x - 1 + sk] -= f->b2[x] * w;
                    lam[x - 1 - sk] += f->b2[x] * w;
                    lam[x - 1]  += f->c0[x] * w;
                    lam[x - sj] += f->c1[x] * w;
                    lam[x - sk] += f->c2[x] * w;
                    /* parameter gradients of sweep t */
                    g_wrk1[x] += w;
                    g_a3[x] += mu * s0_at(f, p, I, J, i, j, k);
                    if (g_coef) {
                        ga[0][x] += w * p[x + 1];
                        ga[1][x] += w * p[x + sj];
                        ga[2][x] += w * p[x + sk];
                        ga[3][x] += w * (p[x + 1 + sj] - p[x + 1 - sj] - p[x - 1 + sj] + p[x - 1 - sj]);
                        ga[4][x] += w * (p[x + sj + sk] - p[x + sj - sk] - p[x - sj + sk] + p[x - sj - sk]);
                        ga[5][x] += w * (p[x + 1 + sk] - p[x + 1 - sk] - p[x - 1 + sk] + p[x - 1 - sk]);
                        ga[6][x] += w * p[x - 1];
                        ga[7][x] += w * p[x - sj];
                        ga[8][x] += w * p[x - sk];
                    }
                }
    }
    free(states);
    free(lam_next);
    return ORACLE_OK;
}
