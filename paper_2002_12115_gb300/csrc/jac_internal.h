// Internal interfaces shared by the translation units of libjac.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/jacobi.h"

namespace jac {

struct GridDesc;
struct SweepArgs;

const char *thread_last_error();
void set_thread_error(const std::string &m);

jac_status validate_grid(const jac_grid *g);
jac_plan resolve_plan(const jac_grid *g, const jac_plan *plan);
jac_plan resolve_plan_sms(const jac_grid *g, const jac_plan *plan, int sms);
size_t sweep_workspace_bytes(const jac_grid *g, const jac_plan &p);
// Launch options of the single-grid sweep that only a test of the failure
// path sets: a shorter limit for the waits on other warps and CTAs, and an
// offset that makes the grid barrier between sweeps unreachable.  Either one
// set runs single sweeps (no two-sweep passes).
struct LaunchOpts {
    unsigned long long wait_ns = 0;
    unsigned gbar_extra = 0;
};
jac_status sweep_dev(const jac_grid *g, const jac_plan *plan, int n_iter, double *d_residual, void *workspace,
                     size_t ws_bytes, void *stream, const LaunchOpts *opts = nullptr);
jac_status pack_dev(int I, int J, int K, jac_prec prec, int which, const double *src, void *dst, cudaStream_t st);
jac_status unpack_dev(int I, int J, int K, jac_prec prec, int which, const void *src, double *dst,
                      cudaStream_t st);
jac_status pack_dev_f32(int I, int J, int K, jac_prec prec, int which, const float *src, void *dst, cudaStream_t st);
jac_status unpack_dev_f32(int I, int J, int K, jac_prec prec, int which, const void *src, float *dst,
                          cudaStream_t st);
jac_status workspace_check(void *workspace, cudaStream_t st);
int device_sm_count();
size_t device_l2_bytes();
void set_l2_policy(SweepArgs &a, jac_prec prec, size_t points);
int vector_points(jac_prec prec);
int max_row_fold(jac_prec prec, int tj);
bool warps_supported(jac_prec prec, int tj);
int best_tile_i(int I, int J, jac_prec prec, int tj);
jac_status check_plan(jac_prec prec, const jac_plan &p, int *rw_out, int *tj_out);
jac_status build_desc(GridDesc *d, const jac_grid *g, const jac_plan &p, int item_base);
template <bool BATCH>
jac_status launch_sweep(jac_prec prec, int tj, const GridDesc &d0, const SweepArgs &a, unsigned nblocks,
                        cudaStream_t st);
// Two-sweep passes (FP32 storage): n_pass passes of two sweeps each, in one
// cooperative launch; the residual of the last sweep to d_residual (NULL:
// none).  kdepth 0: the default depth.
// Two-sweep passes (FP32 storage): pass t reads p[t & 1] and writes the other
// buffer.  mid (one-pass calls only) also receives the state after the first
// sweep at every interior point; its faces are left as they are.
jac_status sweep2_run(const jac_grid *g, int kdepth, int n_pass, double *d_residual, void *workspace,
                      size_t ws_bytes, cudaStream_t st, void *mid = nullptr);
// Whether the library's plan for this grid takes two-sweep passes (fuse 0).
bool two_sweep_default(const jac_grid *g);
size_t sweep2_workspace_bytes(const jac_grid *g);
jac_status adjoint_step_dev(const jac_grid *g, const void *p_t, const void *lam_in, void *lam_out, double *g_wrk1,
                            double *g_a3, double *const *g_coef, int kdepth, void *workspace, size_t ws_bytes,
                            cudaStream_t st);
// 3-D tensor map of one storage-layout array (row pitch `pitch` elements)
// with extent (extent_i, J, K), so that columns at i >= extent_i read as
// zero, and a (bx, by, 1) box.
jac_status encode_box_map(CUtensorMap *m, const void *base, size_t elem, int extent_i, int pitch, int J, int K,
                          int bx, int by);

}  // namespace jac
