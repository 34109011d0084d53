// igm_setup.cu -- device set-up of one system (the steps of Fig. 1 before
// the refinement loop): CSR validation, the initial row scaling of eq. (1)
// and eq. (3), the cast of Sec. IV-B, the level schedule of the triangular
// factors, the FP64 ILU(0) of eq. (ilu) and the integer factors of
// eq. (dldr)-(ilu2).
#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

// CSR checks (rowptr monotone, columns in range and strictly ascending) and
// the position of each row's diagonal (-1 if absent)
__global__ void s_validate(int n, int nnz, const int *rowptr, const int *col, int *diagpos,
                           unsigned *err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int k0 = rowptr[i], k1 = rowptr[i + 1], dp = -1;
    if (k0 < 0 || k1 < k0 || k1 > nnz) {
      atomicOr(err, ERR_BADCSR);
      diagpos[i] = -1;
      continue;
    }
    int prev = -1;
    for (int k = k0; k < k1; ++k) {
      int c = col[k];
      if (c < 0 || c >= n || c <= prev) atomicOr(err, ERR_BADCSR);
      if (c == i) dp = k;
      prev = c;
    }
    diagpos[i] = dp;
  }
}

// bandwidths of the strict triangles, max (i - j) below and (j - i) above,
// and the largest number of entries of a row below / above the diagonal
// (bw[0..3]); columns are ascending, rows well formed (checked before)
__global__ void s_bandwidth(int n, const int *rowptr, const int *col, int *bw) {
  int lo = 0, hi = 0, kl = 0, ku = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int k0 = rowptr[i], k1 = rowptr[i + 1];
    if (k1 > k0) {
      lo = max(lo, i - col[k0]);
      hi = max(hi, col[k1 - 1] - i);
    }
    int nl = 0, nu = 0;
    for (int k = k0; k < k1; ++k) {
      nl += col[k] < i;
      nu += col[k] > i;
    }
    kl = max(kl, nl);
    ku = max(ku, nu);
  }
  atomicMax(bw, lo);
  atomicMax(bw + 1, hi);
  atomicMax(bw + 2, kl);
  atomicMax(bw + 3, ku);
}

// eq. (3): d_i = max_j |ahat_ij| 2^-alpha_a; eq. (1): a_ij = ahat_ij / d_i
__global__ void s_scale(int n, const int *rowptr, const double *ahat, int alpha,
                        double *a, double *d, unsigned *err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double mx = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) mx = fmax(mx, fabs(ahat[k]));
    if (mx == 0.0) {
      atomicOr(err, ERR_ZERO_ROW);
      d[i] = 1.0;
      continue;
    }
    double di = scalbn(mx, -alpha);
    d[i] = di;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) a[k] = __ddiv_rn(ahat[k], di);
  }
}

// Sec. IV-B: Abar_0 = cast(A), truncation toward zero
__global__ void s_cast(long long nnz, const double *a, i64 *abar, unsigned *err) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x) {
    double v = a[k];
    if (fabs(v) < 9223372036854775808.0) abar[k] = __double2ll_rz(v);
    else {
      abar[k] = 0;
      atomicOr(err, ERR_CAST);
    }
  }
}

// eq. (A): remainder of term 0, R = A - Abar_0 (exact)
__global__ void s_mt_init(long long nnz, const double *a, const i64 *abar, double *R) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x)
    R[k] = __dsub_rn(a[k], (double)abar[k]);
}

// max |R| as the bit pattern of a non-negative double (ordered like the value)
__global__ void s_mt_max(long long nnz, const double *R, unsigned long long *mx) {
  unsigned long long m = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(fabs(R[k])));
  atomicMax(mx, m);
}

// eq. (alpha1): Abar_l = trunc(R 2^alpha_l), then R = (R 2^alpha_l - Abar_l)
// 2^-alpha_l (both exact)
__global__ void s_mt_term(long long nnz, double *R, int al, i64 *T) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x) {
    const double t = scalbn(R[k], al);
    const i64 q = __double2ll_rz(t);
    T[k] = q;
    R[k] = scalbn(__dsub_rn(t, (double)q), -al);
  }
}

// Ā in SELL-32 (see SysDev): one thread per slot row (padding rows of the
// last slice included)
__global__ void s_sell_fill(int n, int nsl, const int *rowptr, const int *col, const i64 *abar,
                            const long long *sptr, i64 *sval, int *scol) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < 32ll * nsl;
       r += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(r >> 5), lane = (int)(r & 31);
    const long long base = sptr[s], len = (sptr[s + 1] - base) >> 5;
    const int k0 = r < n ? rowptr[r] : 0, cnt = r < n ? rowptr[r + 1] - k0 : 0;
    for (int k = 0; k < len; ++k) {
      const long long q = base + 32ll * k + lane;
      sval[q] = k < cnt ? abar[k0 + k] : 0;
      scol[q] = k < cnt ? col[k0 + k] : (r < n ? (int)r : 0);
    }
  }
}

// Chunk-local level of every row of the strict lower (lower = 1) or strict
// upper part.  Positions p = 0..n-1 run in dependency order (row p for L,
// row n-1-p for U) and are cut into chunks of R positions; the local level of
// a row is 1 + the largest local level of the rows it reads inside its own
// chunk (0 if none): rows of earlier chunks are not counted, they are waited
// for at solve time.  CTAs take 256-position chunks of work by ticket; each
// row waits (bounded) on the flags of its same-chunk dependencies.
__global__ void s_levels(int n, const int *rowptr, const int *col, const int *diagpos,
                         int lower, int R, int *level, int *flag, int epoch, unsigned *ticket,
                         int *chunkmax, unsigned *err) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  int p = s_t * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i = lower ? p : n - 1 - p;
  int c = p / R;
  int first = c * R;  // first position of the chunk
  int k0 = lower ? rowptr[i] : diagpos[i] + 1;
  int k1 = lower ? diagpos[i] : rowptr[i + 1];
  int lv = 0;
  for (int k = k0; k < k1; ++k) {
    int j = col[k];
    int pj = lower ? j : n - 1 - j;
    if (pj < first) continue;
    wait_flag_setup(flag + j, epoch, err);
    lv = max(lv, __ldcg(level + j) + 1);
  }
  level[i] = lv;
  st_release(flag + i, epoch);
  atomicMax(chunkmax + c, lv);
}

// group key of a row: first group of its chunk + its local level
__global__ void s_hist(int n, int lower, int R, const int *level, const int *levb, int *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = lower ? i : n - 1 - i;
    atomicAdd(cnt + levb[p / R] + level[i], 1);
  }
}

// exclusive scan of cnt[0..L) into out[0..L] (out[L] = total), one CTA
__global__ void s_scan(int L, const int *cnt, int *out) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < L; base += 1024) {
    int idx = base + threadIdx.x;
    int v = idx < L ? cnt[idx] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (idx < L) out[idx] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[L] = carry;
}

// scatter rows into (chunk, level) groups; the order inside a group is
// arbitrary and does not affect results (rows of one group are independent)
__global__ void s_scatter(int n, int lower, int R, const int *level, const int *levb,
                          int *cursor, int *order) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = lower ? i : n - 1 - i;
    order[atomicAdd(cursor + levb[p / R] + level[i], 1)] = i;
  }
}

// the most rows of one level group, max over g of lptr[g+1] - lptr[g]
__global__ void s_maxw(int L, const int *lptr, int *out) {
  int w = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < L; g += gridDim.x * blockDim.x)
    w = max(w, lptr[g + 1] - lptr[g]);
  atomicMax(out, w);
}

// The Gauss-Seidel preconditioner D + L_A in the ILU factor form: unit lower
// entries a_ij / a_jj, pivots a_ii, no strict upper part (precond = 2)
__global__ void s_gs_factors(int n, const int *rowptr, const int *col, const int *diagpos,
                             const double *a, double *f, unsigned *err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (a[diagpos[i]] == 0.0) atomicOr(err, ERR_ZERO_PIVOT);
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = col[k];
      f[k] = j < i ? __ddiv_rn(a[k], a[diagpos[j]]) : (j == i ? a[k] : 0.0);
    }
  }
}

// eq. (dl), (dl2), (l1), (u1), (ilu2): D_l = |d|^1/2, D_u = sgn(d)|d|^1/2,
// Lbar = trunc(L D_l), Ubar = trunc(D_u U') with U' = D^-1 U
__global__ void s_ilu_int(int n, const int *rowptr, const int *col, const int *diagpos,
                          const double *f, i64 *fac, i64 *ldiag, i64 *udiag, unsigned *err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double di = f[diagpos[i]];
    double sl = __dsqrt_rn(fabs(di));
    double su = di < 0 ? -sl : sl;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int j = col[k];
      double v;
      if (j < i) v = __dmul_rn(f[k], __dsqrt_rn(fabs(f[diagpos[j]])));
      else if (j > i) v = __dmul_rn(su, __ddiv_rn(f[k], di));
      else {
        fac[k] = 0;
        continue;
      }
      if (fabs(v) < 9223372036854775808.0) fac[k] = __double2ll_rz(v);
      else {
        fac[k] = 0;
        atomicOr(err, ERR_CAST);
      }
    }
    if (!(sl < 9223372036854775808.0)) atomicOr(err, ERR_CAST);
    i64 l = sl < 9223372036854775808.0 ? __double2ll_rz(sl) : 0;
    i64 u = sl < 9223372036854775808.0 ? __double2ll_rz(su) : 0;
    ldiag[i] = l;
    udiag[i] = u;
    if (l == 0 || u == 0) atomicOr(err, ERR_ZERO_PIVOT);
  }
}

// ---------------------------------------------------------------------------
static int grid_for(long long n, int bs) {
  long long g = (n + bs - 1) / bs;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

void launch_validate(int n, int nnz, const int *rowptr, const int *col, int *diagpos,
                     unsigned *err, cudaStream_t st) {
  s_validate<<<grid_for(n, 256), 256, 0, st>>>(n, nnz, rowptr, col, diagpos, err);
}
void launch_bandwidth(int n, const int *rowptr, const int *col, int *bw, cudaStream_t st) {
  s_bandwidth<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, bw);
}
void launch_scale(int n, const int *rowptr, const double *ahat, int alpha, double *a,
                  double *d, unsigned *err, cudaStream_t st) {
  s_scale<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, ahat, alpha, a, d, err);
}
void launch_cast(long long nnz, const double *a, i64 *abar, unsigned *err, cudaStream_t st) {
  s_cast<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, a, abar, err);
}
void launch_levels(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                   int R, int *level, int *flag, int epoch, unsigned *ticket, int *chunkmax,
                   unsigned *err, cudaStream_t st) {
  s_levels<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, col, diagpos, lower, R, level, flag,
                                             epoch, ticket, chunkmax, err);
}
void launch_level_order(int n, int lower, int R, int L, const int *level, const int *levb,
                        int *cnt, int *lptr, int *order, cudaStream_t st) {
  s_hist<<<grid_for(n, 256), 256, 0, st>>>(n, lower, R, level, levb, cnt);
  s_scan<<<1, 1024, 0, st>>>(L, cnt, lptr);
  cudaMemcpyAsync(cnt, lptr, sizeof(int) * L, cudaMemcpyDeviceToDevice, st);
  s_scatter<<<grid_for(n, 256), 256, 0, st>>>(n, lower, R, level, levb, cnt, order);
}
void launch_mt_init(long long nnz, const double *a, const i64 *abar, double *R,
                    cudaStream_t st) {
  s_mt_init<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, a, abar, R);
}
void launch_mt_max(long long nnz, const double *R, unsigned long long *mx, cudaStream_t st) {
  s_mt_max<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, R, mx);
}
void launch_mt_term(long long nnz, double *R, int al, i64 *T, cudaStream_t st) {
  s_mt_term<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, R, al, T);
}
void launch_sell_fill(int n, int nsl, const int *rowptr, const int *col, const i64 *abar,
                      const long long *sptr, i64 *sval, int *scol, cudaStream_t st) {
  s_sell_fill<<<grid_for(32ll * nsl, 256), 256, 0, st>>>(n, nsl, rowptr, col, abar, sptr, sval,
                                                         scol);
}
void launch_maxw(int L, const int *lptr, int *out, cudaStream_t st) {
  s_maxw<<<grid_for(L, 256), 256, 0, st>>>(L, lptr, out);
}
void launch_gs_factors(int n, const int *rowptr, const int *col, const int *diagpos,
                       const double *a, double *f, unsigned *err, cudaStream_t st) {
  s_gs_factors<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, diagpos, a, f, err);
}
void launch_ilu_int(int n, const int *rowptr, const int *col, const int *diagpos,
                    const double *f, i64 *fac, i64 *ldiag, i64 *udiag, unsigned *err,
                    cudaStream_t st) {
  s_ilu_int<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, diagpos, f, fac, ldiag, udiag,
                                               err);
}

}  // namespace igm
