// igm_launch.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "../../include/igm.h"
#include "igm_internal.h"

namespace igm {

// set-up (one system)
void launch_validate(int n, int nnz, const int *rowptr, const int *col, int *diagpos,
                     unsigned *err, cudaStream_t st);
void launch_scale(int n, const int *rowptr, const double *ahat, int alpha, double *a,
                  double *d, unsigned *err, cudaStream_t st);
void launch_cast(long long nnz, const double *a, i64 *abar, unsigned *err, cudaStream_t st);
void launch_levels(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                   int *level, int *flag, int epoch, unsigned *ticket, int *maxlev,
                   unsigned *err, cudaStream_t st);
void launch_level_order(int n, int L, const int *level, int *cnt, int *order,
                        cudaStream_t st);
void launch_ilu0(int n, const int *rowptr, const int *col, const int *diagpos,
                 const int *lorder, double *f, int *flag, int epoch, unsigned *ticket,
                 unsigned *err, cudaStream_t st);
void launch_ilu_int(int n, const int *rowptr, const int *col, const int *diagpos,
                    const double *f, i64 *fac, i64 *ldiag, i64 *udiag, unsigned *err,
                    cudaStream_t st);

// refinement loop and inner solve (a batch of systems)
void launch_init_scal(const BatchDev &B, int mode, cudaStream_t st);
void launch_init_ir(const BatchDev &B, cudaStream_t st);
void launch_max(const BatchDev &B, int which, int gate, cudaStream_t st);
void launch_norm(const BatchDev &B, int which, int act, int gate, cudaStream_t st);
void launch_resid(const BatchDev &B, int hat, cudaStream_t st);
void launch_resid_int(const BatchDev &B, cudaStream_t st);
void launch_rhs(const BatchDev &B, cudaStream_t st);
void launch_arm(const BatchDev &B, cudaStream_t st);
void launch_trsv_fp(const BatchDev &B, int lower, cudaStream_t st);
void launch_trsv_int(const BatchDev &B, int lower, cudaStream_t st);
void launch_cast_v1(const BatchDev &B, cudaStream_t st);
void launch_spmv(const BatchDev &B, int j, cudaStream_t st);
void launch_mgs(const BatchDev &B, int i, int j, cudaStream_t st);
void launch_mgs_last(const BatchDev &B, int j, cudaStream_t st);
void launch_normalize(const BatchDev &B, int j, cudaStream_t st);
void launch_backsub(const BatchDev &B, cudaStream_t st);
void launch_update(const BatchDev &B, cudaStream_t st);

}  // namespace igm
