/*
 * jfft.h -- C ABI of the 3-D complex FFT block of libjac (sm_103a).
 *
 * The paper evaluates its automatic offloading on two applications: the
 * Himeno benchmark and NAS.FT, an FFT code (Section 5.1.1), and names the
 * offload of whole function blocks such as the FFT, not only loop
 * statements, as the next step (Section 6).  This block is that FFT,
 * device-resident and hand-written for GB300, with the time loop of a
 * spectral PDE solver built on it.
 *
 * Transforms of an n1 x n2 x n3 complex array (interleaved re, im; x
 * fastest: element (x, y, z) at complex index (z*n2 + y)*n1 + x):
 *
 *   forward:  X[kx,ky,kz] = sum_{x,y,z} u[x,y,z] exp(-2 pi i (kx x/n1 + ky y/n2 + kz z/n3))
 *   inverse:  u = (1 / (n1 n2 n3)) sum_k X[k] exp(+2 pi i (...))
 *
 * computed as one pass per axis (x, then y, then z), each a batched 1-D FFT
 * of every line along that axis in shared memory and registers (a
 * mixed-radix Stockham FFT: radix-2 to radix-16 butterflies in registers,
 * twiddle factors from a table computed on the host in FP64).
 *
 * The spectral step (jfft_evolve) is the exact Fourier-space solution of the
 * heat equation u_t = alpha * laplace(u) on the periodic unit cube: from the
 * forward transform U of the initial field (computed once, outside the time
 * loop, as the paper hoists transfers out of loops),
 *
 *   u(t) = inverse( U[k] * exp(-4 pi^2 alpha t |kbar|^2) ),
 *
 * kbar the signed frequency per axis (k for k < n/2, k - n otherwise), and
 * its energy sum |u(t)|^2 accumulated in FP64.  The factor is applied as the
 * first pass loads its data, the 1/N scale and the energy as the last pass
 * stores it.
 *
 * Precisions: JFFT_C64 (complex double storage and arithmetic), JFFT_C32
 * (complex float storage and arithmetic, FP64 energy accumulation).
 *
 * Ownership: the plan allocates no device memory.  The caller passes a
 * workspace (jfft_workspace_size bytes) that holds the twiddle tables and
 * the energy partials; data arrays are the caller's too.  Every call
 * enqueues on the plan's stream and returns without waiting; calls on one
 * plan must not overlap in time on different streams.
 *
 * Errors are jac_status values (jacobi.h); jfft_last_error gives the message.
 */
#ifndef JFFT_H
#define JFFT_H

#include <stddef.h>

#include "jacobi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum jfft_prec {
    JFFT_C64 = 0,  /* complex double */
    JFFT_C32 = 1   /* complex float */
} jfft_prec;

typedef struct jfft_plan jfft_plan;

/* Largest and smallest supported extent of each axis (powers of two). */
#define JFFT_MIN_N 2
#define JFFT_MAX_N 1024

/* Bytes of workspace a plan for this shape needs (host only, no GPU):
 * twiddle tables of n1 + n2 + n3 complex values and the energy partials.
 * Errors: JAC_EINVAL for an extent that is not a power of two in
 * [JFFT_MIN_N, JFFT_MAX_N] or an unknown precision. */
jac_status jfft_workspace_size(int n1, int n2, int n3, jfft_prec prec, size_t *bytes);

/* Create a plan on the current device.  stream: the cudaStream_t of every
 * call (NULL: legacy default).  workspace: device memory of at least
 * jfft_workspace_size bytes, 256-byte aligned, owned by the caller and kept
 * by the plan until jfft_destroy; the twiddle tables are copied into it
 * (this call synchronises the stream once).  Errors: JAC_EINVAL, JAC_ECUDA. */
jac_status jfft_plan_create(jfft_plan **out, int n1, int n2, int n3, jfft_prec prec, void *stream,
                            void *workspace, size_t ws_bytes);

/* Free the plan (host memory only; the workspace stays the caller's).  NULL is ok. */
jac_status jfft_destroy(jfft_plan *plan);

/* Message of the last failed call on this plan (NULL: of this thread). */
const char *jfft_last_error(const jfft_plan *plan);

/* Forward 3-D transform (unscaled) of `in` into `out`, device arrays of
 * n1*n2*n3 complex values of the plan's precision, 16-byte aligned; out may
 * equal in (in place), otherwise they must not overlap.  Three launches. */
jac_status jfft_forward(jfft_plan *plan, const void *in, void *out);

/* Inverse 3-D transform scaled by 1 / (n1 n2 n3); as jfft_forward. */
jac_status jfft_inverse(jfft_plan *plan, const void *in, void *out);

/* The spectral step: out = inverse(U * exp(-4 pi^2 alpha t |kbar|^2)), and,
 * if d_energy is not NULL, the FP64 sum of |out|^2 over all points written
 * to d_energy (one double in device memory).  U is read only; out may equal
 * U only if U is not needed again.  alpha and t must be finite and
 * alpha * t >= 0.  Three launches. */
jac_status jfft_evolve(jfft_plan *plan, const void *U, double alpha, double t, void *out, double *d_energy);

#ifdef __cplusplus
}
#endif
#endif /* JFFT_H */
