// igm_trsv.cu -- sparse triangular substitutions on chunked level schedules:
// line 5' of Sec. VI (integer Lbar, Ubar: y_i = (z_i - sum Lbar_ij y_j) /
// Lbar_ii with an exact int128 numerator and truncating division), line 1'
// (the same in FP64 on the integer factors) and the FP64 comparison solver's
// ILU(0) apply, plus the set-up kernels that build the schedules' packed data
// and the FP64 ILU(0) factorisation (eq. ilu) on the same schedule.
//
// A CTA takes one chunk of consecutive positions (by ticket, in dependency
// order) and walks its local levels separated by CTA barriers.  Dependencies
// inside the chunk were computed at an earlier level by the same CTA (kept in
// shared memory); when the chunk size is at least the factor's bandwidth,
// every other dependency lies in the previous chunk and one thread waits,
// once per level, for that chunk's progress word to reach the level the
// group needs (precomputed); otherwise each row waits for its own
// dependencies.  A chunk publishes its progress after every level.  Each
// thread prefetches its row of the next level while computing the current.
#include <type_traits>

#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

#define IGM_TRSV_BLOCK 256
#define IGM_TRSV_KC 4  // dependencies prefetched into registers per row

// ---------------------------------------------------------------------------
// set-up: packed rows, predecessor requirements
// ---------------------------------------------------------------------------

// max strict-part entries per row of L (lower) or U
__global__ void s_maxdeps(int n, const int *rowptr, const int *diagpos, int lower, int *kmax) {
  int k = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    k = max(k, lower ? diagpos[i] - rowptr[i] : rowptr[i + 1] - diagpos[i] - 1);
  atomicMax(kmax, k);
}

// packs the strict part of the row at each position, dependency-major
__global__ void s_pack(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                       int K, const int *ord, const i64 *fac, const i64 *ldiag, const i64 *udiag,
                       const double *f, int *pcol, i64 *pfac, i64 *pdiag, double *pdinv,
                       double *pfacd, double *pdiagd) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int i = ord[p];
    int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    int k1 = lower ? diagpos[i] : rowptr[i + 1];
    for (int q = 0; q < K; ++q) {
      int k = k0 + q;
      bool in = k < k1;
      pcol[(size_t)q * n + p] = in ? col[k] : -1;
      pfac[(size_t)q * n + p] = in ? fac[k] : 0;
      if (pfacd) pfacd[(size_t)q * n + p] = in ? f[k] : 0.0;
    }
    pdiag[p] = lower ? ldiag[i] : udiag[i];
    pdinv[p] = 1.0 / (double)pdiag[p];
    if (pdiagd) pdiagd[p] = f[diagpos[i]];
  }
}

// need[g] = 1 + the largest local level, in the previous chunk, of the
// dependencies of group g's rows (0 when there are none)
__global__ void s_need(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                       int R, const int *ord, const int *levb, const int *lev, int *need) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int i = ord[p];
    int c = p / R, first = c * R;
    int g = levb[c] + lev[i];
    int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    int k1 = lower ? diagpos[i] : rowptr[i + 1];
    int nd = 0;
    for (int k = k0; k < k1; ++k) {
      int j = col[k];
      int pj = lower ? j : n - 1 - j;
      if (pj < first) nd = max(nd, lev[j] + 1);
    }
    if (nd) atomicMax(need + g, nd);
  }
}

// ---------------------------------------------------------------------------
// the substitution kernel
// ---------------------------------------------------------------------------
enum { TK_INT = 0, TK_FPI = 1, TK_FP = 2 };

template <int KIND>
struct TrsvT {
  typedef i64 V;
};
template <>
struct TrsvT<TK_FPI> {
  typedef double V;
};
template <>
struct TrsvT<TK_FP> {
  typedef double V;
};

// row data of one position, loaded ahead of its level
template <int KIND>
struct RowPre {
  typedef typename TrsvT<KIND>::V V;
  int i;
  int col[IGM_TRSV_KC];
  V fac[IGM_TRSV_KC];
  V diag;
  V rhs;
  double dinv;
};

template <int KIND>
__device__ __forceinline__ void row_load(RowPre<KIND> &r, const Tri &T, int n, int p, int row,
                                         const typename TrsvT<KIND>::V *in) {
  r.i = row;
#pragma unroll
  for (int q = 0; q < IGM_TRSV_KC; ++q) {
    if (q < T.K) {
      r.col[q] = T.pcol[(size_t)q * n + p];
      if (KIND == TK_INT) r.fac[q] = T.pfac[(size_t)q * n + p];
      else if (KIND == TK_FPI) r.fac[q] = (double)T.pfac[(size_t)q * n + p];
      else r.fac[q] = T.pfacd[(size_t)q * n + p];
    } else {
      r.col[q] = -1;
    }
  }
  if (KIND == TK_INT) {
    r.diag = T.pdiag[p];
    r.dinv = T.pdinv[p];
  } else if (KIND == TK_FPI) r.diag = (double)T.pdiag[p];
  else r.diag = T.pdiagd ? T.pdiagd[p] : 1.0;
  r.rhs = in[r.i];
}

template <int KIND>
__global__ void __launch_bounds__(IGM_TRSV_BLOCK)
    k_trsv_lv(BatchDev B, int lower, int which, int smem_rows) {
  typedef typename TrsvT<KIND>::V V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *sv = reinterpret_cast<V *>(smem_raw);
  int *sord = reinterpret_cast<int *>(smem_raw + (size_t)smem_rows * sizeof(V));
  __shared__ int s_t;
  const int tk = which == 0 ? (lower ? 0 : 1) : (lower ? 2 : 3);
  if (threadIdx.x == 0) s_t = (int)atomicAdd(&B.ticket[tk], 1u);
  __syncthreads();
  Tile ct = B.ctiles[s_t];
  const SysDev *s = B.sys[ct.sys];
  SysScal *sc = s->sc;
  if (!(sc->cyc != 0 && sc->early == 0) || !s->p.precond) return;
  const Tri &T = s->tri[lower ? 0 : 1];
  const int c = ct.row0, n = s->n, R = s->chunk;
  const int first = c * R, last = min(n, first + R);  // positions of the chunk
  const bool use_smem = (last - first) <= smem_rows;
  // vectors: line 5' (which 1) w -> yv -> w; line 1' (which 0) r -> t -> r
  const V *in;
  V *out;
  if (KIND == TK_INT) {
    in = reinterpret_cast<const V *>(lower ? s->w : s->yv);
    out = reinterpret_cast<V *>(lower ? s->yv : s->w);
  } else if (KIND == TK_FPI || which == 0) {
    in = reinterpret_cast<const V *>(lower ? s->r : s->t);
    out = reinterpret_cast<V *>(lower ? s->t : s->r);
  } else {
    in = reinterpret_cast<const V *>(lower ? reinterpret_cast<const double *>(s->w) : s->t);
    out = reinterpret_cast<V *>(lower ? s->t : reinterpret_cast<double *>(s->w));
  }
  const u64 ep = (u64)(unsigned)sc->seq << 32;
  const int g0 = T.levb[c], g1 = T.levb[c + 1];
  const bool single = s->single_pred != 0;
  unsigned ev = 0;

  // the chunk's rows in level order, staged once so that prefetching a row
  // never waits on the order array
  if (use_smem)
    for (int q = threadIdx.x; q < last - first; q += blockDim.x) sord[q] = T.ord[first + q];
  __syncthreads();
#define ROW_OF(pp) (use_smem ? sord[(pp) - first] : T.ord[pp])

  RowPre<KIND> cur, nxt;
  int pn = T.lptr[g0] + threadIdx.x;
  bool has_nxt = pn < T.lptr[g0 + 1];
  if (has_nxt) row_load<KIND>(nxt, T, n, pn, ROW_OF(pn), in);

  for (int g = g0; g < g1; ++g) {
    const int p0 = T.lptr[g], p1 = T.lptr[g + 1];
    const bool has_cur = has_nxt;
    cur = nxt;
    // prefetch this thread's first row of the next level
    if (g + 1 < g1) {
      pn = T.lptr[g + 1] + threadIdx.x;
      has_nxt = pn < T.lptr[g + 2];
      if (has_nxt) row_load<KIND>(nxt, T, n, pn, ROW_OF(pn), in);
    } else {
      has_nxt = false;
    }
    // the previous chunk must have reached the level this group reads
    if (single && c > 0) {
      if (threadIdx.x == 0) {
        int nd = T.need[g];
        if (nd) wait_prog(T.prog + c - 1, ep | (u64)nd, &sc->err);
      }
      __syncthreads();
    }
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      RowPre<KIND> rr;
      if (p == p0 + (int)threadIdx.x && has_cur) rr = cur;
      else row_load<KIND>(rr, T, n, p, ROW_OF(p), in);
      typedef typename std::conditional<KIND == TK_INT, i128, double>::type A;
      A acc = (A)rr.rhs;
      for (int q = 0; q < T.K; ++q) {
        int j;
        V a;
        if (q < IGM_TRSV_KC) {
          j = rr.col[q];
          a = rr.fac[q];
        } else {
          j = T.pcol[(size_t)q * n + p];
          if (KIND == TK_INT) a = T.pfac[(size_t)q * n + p];
          else if (KIND == TK_FPI) a = (double)T.pfac[(size_t)q * n + p];
          else a = T.pfacd[(size_t)q * n + p];
        }
        if (j < 0) break;
        const int pj = lower ? j : n - 1 - j;
        V yj;
        if (pj >= first) {
          yj = use_smem ? sv[pj - first] : out[j];
        } else {
          if (!single) wait_prog(T.prog + pj / R, ep | (u64)(T.lev[j] + 1), &sc->err);
          yj = (V)__ldcg(out + j);
        }
        if (KIND == TK_INT) acc -= (A)mulw((i64)a, (i64)yj, ev);
        else acc = __dsub_rn((double)acc, __dmul_rn((double)a, (double)yj));
      }
      V y;
      if (KIND == TK_INT) {
        ev += out64((i128)acc);
        y = (V)divt_rcp(wrap((i128)acc), (i64)rr.diag, rr.dinv, ev);
      } else if (KIND == TK_FP && lower) {
        y = (V)acc;  // unit lower factor
      } else {
        y = (V)__ddiv_rn((double)acc, (double)rr.diag);
      }
      out[rr.i] = y;
      // shared slots are indexed by the row's natural position in the chunk
      // (the order inside a level group is arbitrary)
      if (use_smem) sv[(lower ? rr.i : n - 1 - rr.i) - first] = y;
    }
    // the release by one thread after the CTA barrier covers every thread's
    // stores of the level (release is cumulative over the barrier)
    __syncthreads();
    if (threadIdx.x == 0) st_release64(T.prog + c, ep | (u64)(g - g0 + 1));
  }
  if (KIND == TK_INT) flush_ev(ev, &sc->ev[IGM_EV_L5P]);
#undef ROW_OF
}

// ---------------------------------------------------------------------------
// eq. (ilu) on the L schedule: one CTA per chunk, local levels in order;
// row i runs the IKJ update of Saad's Alg. 10.4 (k ascending over its strict
// lower part: l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for the j > k of
// row i present in row k), reading rows k of earlier levels or chunks
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(IGM_TRSV_BLOCK)
    s_ilu0_lv(int n, const int *rowptr, const int *col, const int *diagpos, Tri T, int R,
              int single, double *f, unsigned *ticket, int epoch, unsigned *err) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int c = s_t;
  const int first = c * R;
  const u64 ep = (u64)(unsigned)epoch << 32;
  const int g0 = T.levb[c], g1 = T.levb[c + 1];
  for (int g = g0; g < g1; ++g) {
    if (single && c > 0) {
      if (threadIdx.x == 0 && T.need[g]) wait_prog(T.prog + c - 1, ep | (u64)T.need[g], err);
      __syncthreads();
    }
    for (int p = T.lptr[g] + threadIdx.x; p < T.lptr[g + 1]; p += blockDim.x) {
      int i = T.ord[p];
      int end = rowptr[i + 1];
      for (int kk = rowptr[i]; kk < diagpos[i]; ++kk) {
        int k = col[kk];
        // row k: finished at an earlier level of this CTA (ordinary loads,
        // visible after the CTA barrier) or in an earlier chunk (L2 loads
        // after the acquire of its progress word)
        const bool ext = k < first;
        if (!single && ext) wait_prog(T.prog + k / R, ep | (u64)(T.lev[k] + 1), err);
        double ukk = ext ? __ldcg(f + diagpos[k]) : f[diagpos[k]];
        if (ukk == 0.0) {
          atomicOr(err, ERR_ZERO_PIVOT);
          break;
        }
        double lik = __ddiv_rn(f[kk], ukk);
        f[kk] = lik;
        int q = diagpos[k] + 1, qe = rowptr[k + 1];
        for (int jj = kk + 1; jj < end; ++jj) {
          int jc = col[jj];
          while (q < qe && col[q] < jc) ++q;
          if (q < qe && col[q] == jc)
            f[jj] = __dsub_rn(f[jj], __dmul_rn(lik, ext ? __ldcg(f + q) : f[q]));
        }
      }
      if (f[diagpos[i]] == 0.0) atomicOr(err, ERR_ZERO_PIVOT);
    }
    __syncthreads();
    if (threadIdx.x == 0) st_release64(T.prog + c, ep | (u64)(g - g0 + 1));
  }
}

// ---------------------------------------------------------------------------
static int grid_n(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

void launch_maxdeps(int n, const int *rowptr, const int *diagpos, int lower, int *kmax,
                    cudaStream_t st) {
  s_maxdeps<<<grid_n(n), 256, 0, st>>>(n, rowptr, diagpos, lower, kmax);
}

void launch_pack(int n, const int *rowptr, const int *col, const int *diagpos, int lower, int K,
                 const int *ord, const i64 *fac, const i64 *ldiag, const i64 *udiag,
                 const double *f, int *pcol, i64 *pfac, i64 *pdiag, double *pdinv,
                 double *pfacd, double *pdiagd, cudaStream_t st) {
  s_pack<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, K, ord, fac, ldiag, udiag, f,
                                     pcol, pfac, pdiag, pdinv, pfacd, pdiagd);
}

void launch_need(int n, const int *rowptr, const int *col, const int *diagpos, int lower, int R,
                 const int *ord, const int *levb, const int *lev, int *need, cudaStream_t st) {
  s_need<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, R, ord, levb, lev, need);
}

void launch_ilu0_lv(int n, const int *rowptr, const int *col, const int *diagpos, const Tri &T,
                    int R, int single, double *f, unsigned *ticket, int epoch, unsigned *err,
                    cudaStream_t st) {
  s_ilu0_lv<<<T.nchunk, IGM_TRSV_BLOCK, 0, st>>>(n, rowptr, col, diagpos, T, R, single, f, ticket,
                                                 epoch, err);
}

// shared memory for a chunk's values and order: the chunk if it fits in
// 200 KB
static int smem_rows_for(int bytes_per) { return (200 * 1024) / bytes_per; }

template <int KIND>
static void launch_lv(const BatchDev &B, int lower, int which, int max_chunk, cudaStream_t st) {
  if (B.nctiles <= 0) return;
  const int bper = 8 + 4;  // a value and an order entry per row
  int rows = smem_rows_for(bper);
  if (rows > max_chunk) rows = max_chunk;
  size_t sm = (size_t)rows * bper;
  static bool attr_set[3] = {false, false, false};
  if (!attr_set[KIND]) {
    cudaFuncSetAttribute(k_trsv_lv<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr_set[KIND] = true;
  }
  k_trsv_lv<KIND><<<B.nctiles, IGM_TRSV_BLOCK, sm, st>>>(B, lower, which, rows);
}

void launch_trsv_lv(const BatchDev &B, int kind, int lower, int which, int max_chunk,
                    cudaStream_t st) {
  if (kind == TK_INT) launch_lv<TK_INT>(B, lower, which, max_chunk, st);
  else if (kind == TK_FPI) launch_lv<TK_FPI>(B, lower, which, max_chunk, st);
  else launch_lv<TK_FP>(B, lower, which, max_chunk, st);
}

}  // namespace igm
