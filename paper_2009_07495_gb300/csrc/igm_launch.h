// igm_launch.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <vector>
#include <cuda_runtime.h>

#include "../../include/igm.h"
#include "igm_internal.h"

namespace igm {

// a launch whose own return value reports an error (cooperative or extended
// launches) records it here; the host driver checks it with the launch error
void note_launch(cudaError_t e);
// the first recorded launch error of this thread since the last call (and
// clears it), else cudaSuccess
cudaError_t take_launch_error();

// set-up (one system)
void launch_validate(int n, int nnz, const int *rowptr, const int *col, int *diagpos,
                     unsigned *err, cudaStream_t st);
void launch_bandwidth(int n, const int *rowptr, const int *col, int *bw, cudaStream_t st);
void launch_scale(int n, const int *rowptr, const double *ahat, int alpha, double *a,
                  double *d, unsigned *err, cudaStream_t st);
void launch_cast(long long nnz, const double *a, i64 *abar, unsigned *err, cudaStream_t st);
void launch_levels(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                   int R, int *level, int *flag, int epoch, unsigned *ticket, int *chunkmax,
                   unsigned *err, cudaStream_t st);
void launch_level_order(int n, int lower, int R, int L, const int *level, const int *levb,
                        int *cnt, int *lptr, int *order, cudaStream_t st);
void launch_ilu0_lv(int n, const int *rowptr, const int *col, const int *diagpos, const Tri &T,
                    int R, int single, double *f, unsigned *ticket, int epoch, unsigned *err,
                    cudaStream_t st);
void launch_chunkdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                      int R, int *dmax, cudaStream_t st);
void launch_regroup(int n, int R, const int *ord, int *lev, const int *levb_old,
                    const int *lptr_old, const int *newbase, const int *levb_new, int cap,
                    int *posof, cudaStream_t st);
void launch_ringdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                     int R, const int *ord, const int *posof, const int *lev, const int *levb,
                     const int *lptr, int *dmax, cudaStream_t st);
void launch_pringdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                      int R, const int *ord, const int *posof, const int *lev, const int *levb,
                      const int *lptr, const int *needpm, int *dmax, cudaStream_t st);
void launch_facmax(int n, const int *rowptr, const int *diagpos, int lower, const i64 *fac,
                   unsigned long long *mx, cudaStream_t st);
void launch_pack(int n, const int *rowptr, const int *col, const int *diagpos, int lower, int K,
                 int R, int single, int ring, int pring, int fac32, const int *ord,
                 const int *posof, const int *lev, const int *levb, const int *lptr,
                 const long long *boff, const long long *boffd, const i64 *fac, const i64 *ldiag,
                 const i64 *udiag, const double *f, unsigned char *blob, unsigned char *blobd,
                 cudaStream_t st);
// the widest group a factor with K dependencies per row may have
int trsv_group_cap(int K);
void launch_need(int n, const int *rowptr, const int *col, const int *diagpos, int lower, int R,
                 const int *ord, const int *levb, const int *lev, int *need, cudaStream_t st);
// substitutions: kind 0 integer (line 5'), 1 FP64 on the integer factors
// (line 1'), 2 FP64 factors (comparison solver); which 0 line 1', 1 line 5'
void launch_trsv_lv(const BatchDev &B, int kind, int lower, int which, cudaStream_t st);
void launch_trsv_color(const BatchDev &B, int kind, int lower, int which, cudaStream_t st);
void launch_maxw(int L, const int *lptr, int *out, cudaStream_t st);
void launch_permute(int n, const int *perm, const double *src, double *dst, int back,
                    cudaStream_t st);
void launch_mt_init(long long nnz, const double *a, const i64 *abar, double *R,
                    cudaStream_t st);
void launch_mt_max(long long nnz, const double *R, unsigned long long *mx, cudaStream_t st);
void launch_mt_term(long long nnz, double *R, int al, i64 *T, cudaStream_t st);
void launch_sell_fill(int n, int nsl, const int *rowptr, const int *col, const i64 *abar,
                      const long long *sptr, i64 *sval, int *scol, cudaStream_t st);
void launch_gs_factors(int n, const int *rowptr, const int *col, const int *diagpos,
                       const double *a, double *f, unsigned *err, cudaStream_t st);
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
void launch_cast_v1(const BatchDev &B, cudaStream_t st);
void launch_spmv(const BatchDev &B, int j, cudaStream_t st);
// lines 6-19 of step j: persistent MGS + norm + line 11, then Givens
void launch_mgs_step(const BatchDev &B, int j, cudaStream_t st);
void launch_fp64_mgs_step(const BatchDev &B, int j, cudaStream_t st);
int persistent_grid(int ntiles);  // CTAs of the persistent kernels
// the row partition of the integer Arnoldi step over systems of sizes n
void mgs_plan(const std::vector<int> &n, int max_ctas, int wmax, int snap, bool ring_ok, int &G,
              std::vector<int> &ptr, std::vector<Tile> &seg, int &wrows, int &rows, int &ring,
              std::vector<int> &sys_seg);
void launch_mgs_fused(const BatchDev &B, int j0, int j1, cudaStream_t st);
#ifdef IGM_CHECKS
// checked builds: the first failed device check of each translation unit
unsigned checks_read_mgs();
unsigned checks_read_trsv();
unsigned checks_read_solve();
#endif
void launch_backsub(const BatchDev &B, cudaStream_t st);
void launch_update(const BatchDev &B, cudaStream_t st);
int norm2_grid(int n);
void launch_norm2(const double *x, int n, long long *ws, double *mx, double *out,
                  cudaStream_t st);
// the same with an explicit grid (ws: 2*g partial words + 2 counter words)
void launch_norm2_grid(const double *x, int n, int g, long long *ws, double *mx, double *out,
                       cudaStream_t st);
void launch_gather_state(const BatchDev &B, int4 *out, cudaStream_t st);

// FP64 GMRES(m) comparison solver (lines 1-23 after line 1's residual)
void launch_fp64_inner(const BatchDev &B, int m, int any_ilu, cudaStream_t st);
void launch_fp64_resid_guess(const BatchDev &B, cudaStream_t st);

}  // namespace igm
