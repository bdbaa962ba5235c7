/* A plain C client of libjac (include/jacobi.h), used by the GPU tests: it
 * reads the thirteen FP64 arrays of one grid from a file, runs the hoisted
 * path (create, upload, n sweeps, residual, download) on the legacy default
 * stream and writes the state and the residual to a file.  No Python, no
 * torch: only the C ABI, the library and (for a borrowed context) the CUDA
 * runtime's cudaMalloc.
 *
 *   jac_client I J K prec n in.bin out.bin [borrowed]
 *
 * in.bin: the arrays p, a0, a1, a2, a3, b0, b1, b2, c0, c1, c2, wrk1, bnd in
 * that order, each I*J*K doubles (i fastest).  out.bin: I*J*K doubles of the
 * state, then the residual.  prec: 0 FP64, 1 FP32, 2 FP32 with BF16
 * coefficients.  With "borrowed" the client allocates the fourteen storage
 * arrays and the workspace itself and hands them to jac_create_borrowed;
 * otherwise jac_create allocates them.  Exit status 0 on success; otherwise
 * the failing call and jac_last_error are printed. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "jacobi.h"

static int check(jac_status s, const char *what, const jac_ctx *c)
{
    if (s == JAC_OK) return 0;
    fprintf(stderr, "%s failed (%d): %s\n", what, (int)s, jac_last_error(c));
    return 1;
}

/* The caller-owned storage and workspace of a borrowed context. */
static void *g_dev[JAC_NFIELDS + 2];

static int create_borrowed(jac_ctx **c, int I, int J, int K, jac_prec prec)
{
    jac_grid g;
    memset(&g, 0, sizeof(g));
    g.I = I; g.J = J; g.K = K; g.prec = prec; g.omega = 0.8;
    for (int q = 0; q <= JAC_NFIELDS; ++q) {       /* q = 0, 1: the state buffers; 2.. : coef[1..12] */
        size_t bytes = 0;
        const int which = q < 2 ? JAC_P : q - 1;
        if (check(jac_field_bytes(I, J, K, prec, which, &bytes), "jac_field_bytes", NULL)) return 1;
        if (cudaMalloc(&g_dev[q], bytes) != cudaSuccess) return 1;
        if (q < 2) g.p[q] = g_dev[q];
        else g.coef[which] = g_dev[q];
    }
    size_t ws = 0;
    if (check(jac_workspace_size(I, J, K, prec, NULL, &ws), "jac_workspace_size", NULL)) return 1;
    if (cudaMalloc(&g_dev[JAC_NFIELDS + 1], ws) != cudaSuccess) return 1;
    return check(jac_create_borrowed(c, &g, NULL, g_dev[JAC_NFIELDS + 1], ws, NULL), "jac_create_borrowed", NULL);
}

int main(int argc, char **argv)
{
    if (argc != 8 && argc != 9) {
        fprintf(stderr, "usage: %s I J K prec n in.bin out.bin [borrowed]\n", argv[0]);
        return 2;
    }
    const int I = atoi(argv[1]), J = atoi(argv[2]), K = atoi(argv[3]);
    const int prec = atoi(argv[4]), n = atoi(argv[5]);
    const int borrowed = argc == 9 && strcmp(argv[8], "borrowed") == 0;
    const size_t N = (size_t)I * J * K;
    double *in = malloc(N * JAC_NFIELDS * sizeof(double));
    double *p = malloc((N + 1) * sizeof(double));
    if (!in || !p) return 3;
    FILE *fi = fopen(argv[6], "rb");
    if (!fi || fread(in, sizeof(double), N * JAC_NFIELDS, fi) != N * JAC_NFIELDS) return 4;
    fclose(fi);

    jac_fields f;
    for (int q = 0; q < JAC_NFIELDS; ++q) f.f[q] = in + (size_t)q * N;
    jac_ctx *c = NULL;
    if (borrowed) {
        if (create_borrowed(&c, I, J, K, (jac_prec)prec)) return 5;
    } else if (check(jac_create(&c, I, J, K, (jac_prec)prec, 0.8, NULL), "jac_create", NULL)) {
        return 5;
    }
    int bad = check(jac_upload(c, &f), "jac_upload", c);
    if (!bad) bad = check(jac_sweep(c, n), "jac_sweep", c);
    if (!bad) bad = check(jac_residual(c, &p[N]), "jac_residual", c);
    if (!bad) bad = check(jac_download(c, p), "jac_download", c);
    jac_destroy(c);
    for (int q = 0; borrowed && q < JAC_NFIELDS + 2; ++q) cudaFree(g_dev[q]);
    if (bad) return 6;

    FILE *fo = fopen(argv[7], "wb");
    if (!fo || fwrite(p, sizeof(double), N + 1, fo) != N + 1) return 7;
    fclose(fo);
    free(in);
    free(p);
    return 0;
}
