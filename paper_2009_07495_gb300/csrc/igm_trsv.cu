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
#include <cooperative_groups.h>
#include <type_traits>

#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

namespace cg = cooperative_groups;

#define IGM_TRSV_BLOCK 256
// dependencies of a row held in registers (and in the prefetch ring): 4 for
// 5/7-point stencils, 16 for up to 27-point ones; longer rows read the rest
// from the packed arrays
#define IGM_TRSV_KC_SMALL 4
#define IGM_TRSV_KC_LARGE 16

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
                       const double *f, int *pcol, i64 *pfac, i64 *pdiag, u64 *pdm,
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
    const i64 dg = pdiag[p];
    pdm[p] = dg == 0 ? 0 : magic_u64(dg < 0 ? 0ull - (u64)dg : (u64)dg);
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
template <int KIND, int KC>
struct RowPre {
  typedef typename TrsvT<KIND>::V V;
  int i;
  int col[KC];
  V fac[KC];
  V diag;
  V rhs;
  u64 dm;  // magic multiplier of |diag| (integer kind)
};

// read-only loads issued where they are written (a prefetch must not be
// moved next to its use)
__device__ __forceinline__ int ldnc(const int *p) {
  int v;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ long long ldnc(const long long *p) {
  long long v;
  asm volatile("ld.global.nc.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned long long ldnc(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.global.nc.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ldnc(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

template <int KIND, int KC>
__device__ __forceinline__ void row_load(RowPre<KIND, KC> &r, const Tri &T, int n, int p, int row,
                                         const typename TrsvT<KIND>::V *in) {
  r.i = row;
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    if (q < T.K) {
      r.col[q] = ldnc(T.pcol + (size_t)q * n + p);
      if (KIND == TK_INT) r.fac[q] = ldnc(T.pfac + (size_t)q * n + p);
      else if (KIND == TK_FPI) r.fac[q] = (double)ldnc(T.pfac + (size_t)q * n + p);
      else r.fac[q] = ldnc(T.pfacd + (size_t)q * n + p);
    } else {
      r.col[q] = -1;
      r.fac[q] = 0;
    }
  }
  if (KIND == TK_INT) {
    r.diag = ldnc(T.pdiag + p);
    r.dm = ldnc(T.pdm + p);
  } else if (KIND == TK_FPI) {
    r.diag = (double)ldnc(T.pdiag + p);
    r.dm = 0;
  } else {
    r.diag = T.pdiagd ? ldnc(T.pdiagd + p) : 1.0;
    r.dm = 0;
  }
  r.rhs = ldnc(in + r.i);
}

// asynchronous global -> shared copies (no register scoreboard is held while
// they are in flight; a thread waits for its own groups)
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// wait until at most n of this thread's groups are pending (n <= 3)
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
}

// One row of a level: y_i = (rhs_i - sum_q fac_q y_(col_q)) / diag_i.  FAST
// when every dependency outside the chunk lies in the previous chunk (already
// waited for) and the chunk's values are in shared memory: the register-held
// dependencies are then fetched and multiplied without branches (padding
// entries have factor 0).  Integer numerators are exact (int128); FP64 ones
// subtract in the packed (CSR) order.
template <int KIND, int KC, bool FAST>
__device__ __forceinline__ typename TrsvT<KIND>::V trsv_row(
    const RowPre<KIND, KC> &rr, int p, const Tri &T, int n, int lower, int first, int R,
    bool use_smem, bool single, u64 ep, const typename TrsvT<KIND>::V *sv,
    const typename TrsvT<KIND>::V *psv, const typename TrsvT<KIND>::V *out, unsigned *err,
    unsigned &ev) {
  typedef typename TrsvT<KIND>::V V;
  V yv[KC];
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    const int j = rr.col[q];
    const int pj = lower ? j : n - 1 - j;
    if (FAST) {
      const bool ext = j >= 0 && pj < first;
      const int si = (j >= 0 && !ext) ? pj - first : 0;
      // the previous chunk's values: its CTA's shared memory when it is in
      // this cluster, else global memory
      yv[q] = ext ? (psv ? psv[pj - first + R] : (V)__ldcg(out + j)) : sv[si];
    } else {
      V y = 0;
      if (j >= 0) {
        if (pj >= first) {
          y = use_smem ? sv[pj - first] : (V)__ldcg(out + j);
        } else {
          if (!single) wait_prog(T.prog + (size_t)IGM_PROG_STRIDE * (pj / R), ep | (u64)(T.lev[j] + 1), err);
          y = (V)__ldcg(out + j);
        }
      }
      yv[q] = y;
    }
  }
  typedef typename std::conditional<KIND == TK_INT, i128, double>::type A;
  A acc = (A)rr.rhs;
  if (KIND == TK_INT) {
    i128 sum = 0;
#pragma unroll
    for (int q = 0; q < KC; ++q) sum += (i128)mulw((i64)rr.fac[q], (i64)yv[q], ev);
    acc -= (A)sum;
  } else {
#pragma unroll
    for (int q = 0; q < KC; ++q)
      if (rr.col[q] >= 0) acc = __dsub_rn((double)acc, __dmul_rn((double)rr.fac[q], (double)yv[q]));
  }
  // rows with more dependencies than the registers hold
  for (int q = KC; q < T.K; ++q) {
    const int j = T.pcol[(size_t)q * n + p];
    if (j < 0) break;
    V a;
    if (KIND == TK_INT) a = T.pfac[(size_t)q * n + p];
    else if (KIND == TK_FPI) a = (double)T.pfac[(size_t)q * n + p];
    else a = T.pfacd[(size_t)q * n + p];
    const int pj = lower ? j : n - 1 - j;
    V yj;
    if (pj >= first) {
      yj = use_smem ? sv[pj - first] : (V)__ldcg(out + j);
    } else {
      if (!single) wait_prog(T.prog + (size_t)IGM_PROG_STRIDE * (pj / R), ep | (u64)(T.lev[j] + 1), err);
      yj = (V)__ldcg(out + j);
    }
    if (KIND == TK_INT) acc -= (A)mulw((i64)a, (i64)yj, ev);
    else acc = __dsub_rn((double)acc, __dmul_rn((double)a, (double)yj));
  }
  if (KIND == TK_INT) {
    ev += out64((i128)acc);
    return (V)divt_magic(wrap((i128)acc), (i64)rr.diag, rr.dm, ev);
  }
  if (KIND == TK_FP && lower) return (V)acc;  // unit lower factor
  return (V)__ddiv_rn((double)acc, (double)rr.diag);
}

// CTA-scope release / acquire on shared-memory counters
__device__ __forceinline__ void red_release_cta(unsigned *p, unsigned v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(p)),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ void st_release_cta(unsigned *p, unsigned v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(p)),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}

__device__ __forceinline__ u64 gtimer() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The waits of a substitution CTA are bounded in time (the system's
// p.wait_ns, 1 s unless set), nested so that a wait never expires while the
// wait it depends on can still succeed: the waiter gives up after the bound,
// the publisher (who waits on the compute warps, who wait on the waiter)
// after four times.  An iteration cap backs up each bound.
#define IGM_WAIT_ITERS (1 << 28)

// spin until the shared counter *p reaches at least v; false if the bound
// expired or another wait of the system already timed out
__device__ __forceinline__ bool wait_cta(const unsigned *p, unsigned v, unsigned *err,
                                         u64 limit_ns) {
  if (ld_acquire_cta(p) >= v) return true;
  const u64 t0 = gtimer();
  for (int it = 0; it < IGM_WAIT_ITERS; ++it) {
    if (ld_acquire_cta(p) >= v) return true;
    if (it > 64) __nanosleep(32);
    if ((it & 255) == 255 &&
        ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtimer() - t0 > limit_ns))
      break;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

// Roles in a substitution CTA: IGM_TRSV_CW compute warps walk the levels;
// the waiter warp acquires the previous chunk's progress word and joins the
// compute warps in one named barrier per level, which both lets a level start
// once its inputs are there and makes the previous level's shared values
// visible; the publisher warp turns the compute warps' count of finished
// levels into this chunk's progress word with a GPU-scope release, off the
// compute warps' path.
#define IGM_TRSV_CW 8
#define IGM_TRSV_NC (IGM_TRSV_CW * 32)
#define IGM_TRSV_THREADS (IGM_TRSV_NC + 64)

// cluster-scope signalling between the CTAs of a cluster
__device__ __forceinline__ void st_release_cluster_remote(unsigned *local_ptr, int rank,
                                                          unsigned v) {
  unsigned a = (unsigned)__cvta_generic_to_shared(local_ptr), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cluster_local(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}

// One chunk (ctile t) of a substitution.  rank/cl: the CTA's place in its
// cluster (cl = 1: no cluster).  s_done counts finished levels x warps;
// s_pred receives the previous chunk's finished levels when that chunk runs
// in the same cluster.
template <int KIND, int KC>
__device__ __forceinline__ void trsv_chunk(const BatchDev &B, int t, int rank, int cl, int lower,
                                           int which, int smem_rows, int smem_lev, int rmax,
                                           int pf, int kr, unsigned *s_done_p,
                                           unsigned *s_pred_p) {
  typedef typename TrsvT<KIND>::V V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [values: smem_rows][ring words: (pf+1) x (kr+3) x rmax][order: smem_rows]
  // [ring columns: (pf+1) x kr x rmax][level pointers: smem_lev+1][needs: smem_lev]
  const int S = pf + 1;
  V *sv = reinterpret_cast<V *>(smem_raw);
  long long *ring64 = reinterpret_cast<long long *>(sv + smem_rows);
  int *sord = reinterpret_cast<int *>(ring64 + (pf > 0 ? (size_t)S * (kr + 3) * rmax : 0));
  int *ring32 = sord + smem_rows;
  int *slptr = ring32 + (pf > 0 ? (size_t)S * kr * rmax : 0);  // level pointers (smem_lev + 1)
  int *sneed = slptr + smem_lev + 1;  // their requirements on the previous chunk
  unsigned &s_done = *s_done_p;
  if (t >= B.nctiles) return;
  const Tile ct = B.ctiles[t];
  const SysDev *s = B.sys[ct.sys];
  SysScal *sc = s->sc;
  if (!(sc->cyc != 0 && sc->early == 0) || !s->p.precond) return;
  const Tri T = s->tri[lower ? 0 : 1];
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
  const u64 wns = s->p.wait_ns;
  // tests of the bounded waits: the system's first chunk never signals
  const bool mute = s->p.stall != 0 && c == 0;
  const int g0 = T.levb[c], nlev = T.levb[c + 1] - g0;
  const bool single = s->single_pred != 0;
  const bool lev_smem = nlev <= smem_lev;
  unsigned *err = &sc->err;
  // the previous chunk (c - 1) runs in this cluster's CTA rank - 1 and keeps
  // its values in shared memory; the next chunk (c + 1) in rank + 1
  const bool pred_cl = cl > 1 && rank > 0 && c > 0 && single && R <= smem_rows;
  const bool succ_cl = cl > 1 && rank < cl - 1 && t + 1 < B.nctiles &&
                       B.ctiles[t + 1].sys == ct.sys && single && R <= smem_rows;
  // a successor in the cluster reads this chunk's values from shared memory,
  // except for dependencies beyond the KC held in registers, which it reads
  // from global memory: the global stores may wait until the chunk is done
  // only when rows have no more than KC dependencies
  const bool late_store = succ_cl && T.K <= KC;
  const V *psv = nullptr;
  if (pred_cl) psv = cg::this_cluster().map_shared_rank(sv, rank - 1);

  // stage the chunk's order and level data once
  if (use_smem)
    for (int q = threadIdx.x; q < last - first; q += blockDim.x) sord[q] = T.ord[first + q];
  if (lev_smem) {
    for (int q = threadIdx.x; q <= nlev; q += blockDim.x) slptr[q] = T.lptr[g0 + q];
    for (int q = threadIdx.x; q < nlev; q += blockDim.x) sneed[q] = T.need[g0 + q];
  }
  __syncthreads();
#define ROW_OF(pp) (use_smem ? sord[(pp) - first] : T.ord[pp])
#define LPTR(l) (lev_smem ? slptr[l] : T.lptr[g0 + (l)])
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (wid == IGM_TRSV_CW) {  // waiter: one barrier per level with the compute warps
    u64 seen = 0;  // levels of the previous chunk known to be done
    bool dead = false;
    for (int l = 0; l < nlev; ++l) {
      const int nd = (single && c > 0) ? (lev_smem ? sneed[l] : T.need[g0 + l]) : 0;
      if (lane == 0 && !dead && (u64)nd > seen && pred_cl) {
        unsigned v = ld_acquire_cluster_local(s_pred_p);
        if (v < (unsigned)nd) {
          const u64 t0 = gtimer();
          for (int it = 0; it < IGM_WAIT_ITERS; ++it) {
            if (it > 256) __nanosleep(32);
            v = ld_acquire_cluster_local(s_pred_p);
            if (v >= (unsigned)nd) break;
            if ((it & 255) == 255 &&
                ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtimer() - t0 > wns))
              break;
          }
        }
        if (v < (unsigned)nd) {
          atomicOr(err, ERR_TIMEOUT);
          dead = true;
        } else {
          seen = v;
        }
      } else if (lane == 0 && !dead && (u64)nd > seen) {
        const u64 want = ep | (u64)nd;
        u64 v = ld_acquire64(T.prog + (size_t)IGM_PROG_STRIDE * (c - 1));
        if (v < want) {
          const u64 t0 = gtimer();
          for (int it = 0; it < IGM_WAIT_ITERS; ++it) {
            if (it > 32) __nanosleep(16);
            v = ld_acquire64(T.prog + (size_t)IGM_PROG_STRIDE * (c - 1));
            if (v >= want) break;
            if ((it & 255) == 255 &&
                ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtimer() - t0 > wns))
              break;
          }
        }
        if (v < want) {  // expired: the compute warps finish unchecked, the result is flagged
          atomicOr(err, ERR_TIMEOUT);
          dead = true;
        } else {
          seen = v - ep;
        }
      }
      __syncwarp();
      asm volatile("bar.sync 2, %0;" ::"n"(IGM_TRSV_NC + 32) : "memory");
    }
    return;
  }
  if (wid == IGM_TRSV_CW + 1) {  // publisher
    if (lane == 0) {
      for (unsigned pub = 0; pub < (unsigned)nlev;) {
        // levels every compute warp has finished
        if (!wait_cta(&s_done, (pub + 1) * IGM_TRSV_CW, err, 4 * wns)) break;
        pub = ld_acquire_cta(&s_done) / IGM_TRSV_CW;
        if (mute) continue;
        if (succ_cl) st_release_cluster_remote(s_pred_p, rank + 1, pub);
        else st_release64(T.prog + (size_t)IGM_PROG_STRIDE * c, ep | (u64)pub);
      }
    }
    return;
  }

  // compute warps.  A thread's first row of a level (threads below rmax) is
  // copied into a shared-memory ring pf levels ahead with asynchronous
  // copies; other rows are loaded when they are computed.
  const int tid = threadIdx.x;
  const bool fast = single && use_smem;
  const int kk = T.K < kr ? T.K : kr;  // dependencies this system keeps in the ring
  unsigned ev = 0;
  // the packed arrays of each register-held dependency
  const int *pcq[KC];
  const void *pfq[KC];
#pragma unroll
  for (int q = 0; q < KC; ++q) {
    pcq[q] = T.pcol + (size_t)q * n;
    if (KIND == TK_FP) pfq[q] = T.pfacd + (size_t)q * n;
    else pfq[q] = T.pfac + (size_t)q * n;
  }
  auto issue = [&](int lv) {
    if (pf == 0) return;
    if (lv < nlev && tid < rmax) {
      const int pn = LPTR(lv) + tid;
      if (pn < LPTR(lv + 1)) {
        const int sl = lv % S;
        long long *r64 = ring64 + (size_t)sl * (kr + 3) * rmax + tid;
        int *r32 = ring32 + (size_t)sl * kr * rmax + tid;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          if (q < kk) {
            cp_async4(r32 + q * rmax, pcq[q] + pn);
            cp_async8(r64 + q * rmax, static_cast<const long long *>(pfq[q]) + pn);
          }
        }
        if (KIND != TK_FP) cp_async8(r64 + kr * rmax, T.pdiag + pn);
        else if (T.pdiagd) cp_async8(r64 + kr * rmax, T.pdiagd + pn);
        if (KIND == TK_INT) cp_async8(r64 + (kr + 1) * rmax, T.pdm + pn);
        cp_async8(r64 + (kr + 2) * rmax, in + ROW_OF(pn));
      }
    }
    cp_async_commit();
  };
  auto ring_row = [&](int lv, int p, RowPre<KIND, KC> &r) {
    const int sl = lv % S;
    const long long *r64 = ring64 + (size_t)sl * (kr + 3) * rmax + tid;
    const int *r32 = ring32 + (size_t)sl * kr * rmax + tid;
    r.i = ROW_OF(p);
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      if (q < kk) {
        r.col[q] = r32[q * rmax];
        const long long w = r64[q * rmax];
        if (KIND == TK_INT) r.fac[q] = (V)w;
        else if (KIND == TK_FPI) r.fac[q] = (V)(double)w;
        else r.fac[q] = (V)__longlong_as_double(w);
      } else {
        r.col[q] = -1;
        r.fac[q] = 0;
      }
    }
    const long long dw = r64[kr * rmax], rw = r64[(kr + 2) * rmax];
    if (KIND == TK_INT) {
      r.diag = (V)dw;
      r.dm = (u64)r64[(kr + 1) * rmax];
      r.rhs = (V)rw;
    } else {
      if (KIND == TK_FPI) r.diag = (V)(double)dw;
      else r.diag = (V)(T.pdiagd ? __longlong_as_double(dw) : 1.0);
      r.dm = 0;
      r.rhs = (V)__longlong_as_double(rw);
    }
  };
  for (int l = 0; l < pf; ++l) issue(l);
  for (int l = 0; l < nlev; ++l) {
    const int p0 = LPTR(l), p1 = LPTR(l + 1);
    issue(l + pf);
    // the waiter has seen the previous chunk reach what this level reads;
    // the previous level's shared values are visible
    __syncwarp();
    asm volatile("bar.sync 2, %0;" ::"n"(IGM_TRSV_NC + 32) : "memory");
    if (pf > 0) cp_async_wait(pf);  // this thread's copies of level l have landed
    for (int p = p0 + tid; p < p1; p += IGM_TRSV_NC) {
      RowPre<KIND, KC> rr;
      if (pf > 0 && p == p0 + tid && tid < rmax) ring_row(l, p, rr);
      else row_load<KIND, KC>(rr, T, n, p, ROW_OF(p), in);
      const V y = fast ? trsv_row<KIND, KC, true>(rr, p, T, n, lower, first, R, use_smem, single, ep,
                                              sv, psv, out, err, ev)
                       : trsv_row<KIND, KC, false>(rr, p, T, n, lower, first, R, use_smem, single,
                                               ep, sv, nullptr, out, err, ev);
      // shared slots are indexed by the row's natural position in the chunk
      // (the order inside a level group is arbitrary)
      if (use_smem) sv[(lower ? rr.i : n - 1 - rr.i) - first] = y;
      if (!late_store) out[rr.i] = y;
    }
    // the warp's stores of the level, then one count per warp for the
    // publisher
    __syncwarp();
    if (lane == 0) red_release_cta(&s_done, 1u);
  }
  if (late_store) {
    // the chunk's values go to global memory once, in one coalesced sweep
    // after its last level, so the publisher's releases never wait for
    // global stores
    asm volatile("bar.sync 3, %0;" ::"n"(IGM_TRSV_NC) : "memory");
    for (int q = tid; q < last - first; q += IGM_TRSV_NC)
      out[lower ? first + q : n - 1 - (first + q)] = sv[q];
  }
  if (pf > 0) cp_async_wait(0);
  if (KIND == TK_INT) flush_ev(ev, &sc->ev[IGM_EV_L5P]);
#undef ROW_OF
#undef LPTR
}

// The substitution kernel.  Without clusters each CTA takes a chunk by
// ticket; with clusters of cl CTAs, rank 0 takes a ticket for cl consecutive
// chunks (tickets keep every chunk's predecessor started before it), and all
// CTAs of a cluster stay resident until the last one is done, since later
// chunks read earlier chunks' shared memory.
template <int KIND, int KC>
__global__ void __launch_bounds__(IGM_TRSV_THREADS, 1)
    k_trsv_lv(BatchDev B, int lower, int which, int smem_rows, int smem_lev, int rmax, int pf,
              int kr, int cl) {
  __shared__ int s_t;
  __shared__ unsigned s_done, s_pred;
  const int tk = which == 0 ? (lower ? 0 : 1) : (lower ? 2 : 3);
  if (cl > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    if (threadIdx.x == 0) {
      if (rank == 0) s_t = (int)atomicAdd(&B.ticket[tk], 1u);
      s_done = 0;
      s_pred = 0;
    }
    cluster.sync();  // rank 0's ticket and every CTA's counters are set
    const int t = *cluster.map_shared_rank(&s_t, 0) * cl + rank;
    trsv_chunk<KIND, KC>(B, t, rank, cl, lower, which, smem_rows, smem_lev, rmax, pf, kr, &s_done,
                     &s_pred);
    cluster.sync();  // no CTA leaves while a later chunk may read its values
  } else {
    if (threadIdx.x == 0) {
      s_t = (int)atomicAdd(&B.ticket[tk], 1u);
      s_done = 0;
      s_pred = 0;
    }
    __syncthreads();
    trsv_chunk<KIND, KC>(B, s_t, 0, 1, lower, which, smem_rows, smem_lev, rmax, pf, kr, &s_done,
                     &s_pred);
  }
}

// ---------------------------------------------------------------------------
// Substitutions in multicolour order: every strict dependency of a row lies
// in another colour (earlier for L, later for U), so one launch per colour
// computes all its rows at once, each row from the CSR of the factors in
// CSR order (the order of the natural substitution).
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(256) k_trsv_color(BatchDev B, int lower, int which, int c) {
  typedef typename TrsvT<KIND>::V V;
  const Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!(sc->cyc != 0 && sc->early == 0) || !s->p.precond || s->ncolors == 0) return;
  const int nc = s->ncolors;
  if (c >= nc) return;
  const int cc = lower ? c : nc - 1 - c;  // U: colours from the last
  const int r0 = max(tl.row0, s->cptr[cc]), r1 = min(tl.row0 + tl.nrows, s->cptr[cc + 1]);
  if (r0 >= r1) return;
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
  unsigned ev = 0;
  for (int i = r0 + (int)threadIdx.x; i < r1; i += blockDim.x) {
    const int dp = s->diagpos[i];
    const int k0 = lower ? s->rowptr[i] : dp + 1, k1 = lower ? dp : s->rowptr[i + 1];
    typedef typename std::conditional<KIND == TK_INT, i128, double>::type A;
    A acc = (A)in[i];
    for (int k = k0; k < k1; ++k) {
      const V yj = __ldcg(out + s->col[k]);
      if (KIND == TK_INT) acc -= (A)mulw(s->fac[k], (i64)yj, ev);
      else if (KIND == TK_FPI) acc = __dsub_rn((double)acc, __dmul_rn((double)s->fac[k], (double)yj));
      else acc = __dsub_rn((double)acc, __dmul_rn(s->f[k], (double)yj));
    }
    V y;
    if (KIND == TK_INT) {
      ev += out64((i128)acc);
      y = (V)divt(wrap((i128)acc), lower ? s->ldiag[i] : s->udiag[i], ev);
    } else if (KIND == TK_FPI) {
      y = (V)__ddiv_rn((double)acc, (double)(lower ? s->ldiag[i] : s->udiag[i]));
    } else if (lower) {
      y = (V)acc;  // unit lower factor
    } else {
      y = (V)__ddiv_rn((double)acc, s->f[dp]);
    }
    out[i] = y;
  }
  if (KIND == TK_INT) flush_ev(ev, &sc->ev[IGM_EV_L5P]);
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
      if (threadIdx.x == 0 && T.need[g])
        wait_prog_setup(T.prog + (size_t)IGM_PROG_STRIDE * (c - 1), ep | (u64)T.need[g], err);
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
        if (!single && ext)
          wait_prog_setup(T.prog + (size_t)IGM_PROG_STRIDE * (k / R), ep | (u64)(T.lev[k] + 1), err);
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
    if (threadIdx.x == 0) st_release64(T.prog + (size_t)IGM_PROG_STRIDE * c, ep | (u64)(g - g0 + 1));
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
                 const double *f, int *pcol, i64 *pfac, i64 *pdiag, u64 *pdm,
                 double *pfacd, double *pdiagd, cudaStream_t st) {
  s_pack<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, K, ord, fac, ldiag, udiag, f,
                                     pcol, pfac, pdiag, pdm, pfacd, pdiagd);
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

// shared memory: a chunk's values and order if the chunk fits in 200 KB,
// its level pointers and requirements if they fit in the rest, then as deep
// a ring of prefetched rows (up to three levels ahead) as the remainder holds
static int smem_rows_for(int bytes_per) { return (200 * 1024) / bytes_per; }
#define IGM_TRSV_SMEM_MAX (226 * 1024)

template <int KIND, int KC>
static void launch_lv(const BatchDev &B, int lower, int which, int max_chunk, cudaStream_t st) {
  if (B.nctiles <= 0) return;
  const int bper = 8 + 4;  // a value and an order entry per row
  int rows = smem_rows_for(bper);
  if (rows > max_chunk) rows = max_chunk;
  size_t sm = (size_t)rows * bper;
  int lev = B.trsv_maxlev;
  if (sm + (size_t)(2 * lev + 1) * sizeof(int) > IGM_TRSV_SMEM_MAX) lev = 0;
  sm += (size_t)(2 * lev + 1) * sizeof(int);
  const int kr = B.trsv_maxk < KC ? (B.trsv_maxk > 0 ? B.trsv_maxk : 1) : KC;
  const int rmax = B.trsv_maxw < IGM_TRSV_NC ? B.trsv_maxw : IGM_TRSV_NC;
  const size_t per_slot = (size_t)rmax * ((kr + 3) * 8 + kr * 4);
  int pf = 0;
  for (int d = 3; d >= 1; --d)
    if (sm + (size_t)(d + 1) * per_slot <= IGM_TRSV_SMEM_MAX) {
      pf = d;
      break;
    }
  if (pf > 0) sm += (size_t)(pf + 1) * per_slot;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_trsv_lv<KIND, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IGM_TRSV_SMEM_MAX);
    attr_set = true;
  }
  // clusters of consecutive chunks when the GPU can co-schedule them (4 by
  // default: larger clusters are harder to place and measured slower)
  int cl = B.trsv_cluster;
  if (cl == 0) {
    cl = 1;
    for (int want = 4; want >= 2; want /= 2) {
      cudaLaunchConfig_t q = {};
      q.gridDim = dim3(want);
      q.blockDim = dim3(IGM_TRSV_THREADS);
      q.dynamicSmemBytes = sm;
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = want;
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.attrs = qa;
      q.numAttrs = 1;
      int nclus = 0;
      if (cudaOccupancyMaxActiveClusters(&nclus, k_trsv_lv<KIND, KC>, &q) == cudaSuccess && nclus >= 1) {
        cl = want;
        break;
      }
      cudaGetLastError();
    }
  }
  const int G = (B.nctiles + cl - 1) / cl * cl;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(IGM_TRSV_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  note_launch(cudaLaunchKernelEx(&cfg, k_trsv_lv<KIND, KC>, B, lower, which, rows, lev, rmax, pf,
                                 kr, cl));
}

void launch_trsv_color(const BatchDev &B, int kind, int lower, int which, cudaStream_t st) {
  for (int c = 0; c < B.max_colors; ++c) {
    if (kind == TK_INT) k_trsv_color<TK_INT><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
    else if (kind == TK_FPI) k_trsv_color<TK_FPI><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
    else k_trsv_color<TK_FP><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
  }
}

void launch_trsv_lv(const BatchDev &B, int kind, int lower, int which, int max_chunk,
                    cudaStream_t st) {
  if (B.max_colors > 0) launch_trsv_color(B, kind, lower, which, st);
  if (B.trsv_maxk <= IGM_TRSV_KC_SMALL) {
    if (kind == TK_INT) launch_lv<TK_INT, IGM_TRSV_KC_SMALL>(B, lower, which, max_chunk, st);
    else if (kind == TK_FPI) launch_lv<TK_FPI, IGM_TRSV_KC_SMALL>(B, lower, which, max_chunk, st);
    else launch_lv<TK_FP, IGM_TRSV_KC_SMALL>(B, lower, which, max_chunk, st);
  } else {
    if (kind == TK_INT) launch_lv<TK_INT, IGM_TRSV_KC_LARGE>(B, lower, which, max_chunk, st);
    else if (kind == TK_FPI) launch_lv<TK_FPI, IGM_TRSV_KC_LARGE>(B, lower, which, max_chunk, st);
    else launch_lv<TK_FP, IGM_TRSV_KC_LARGE>(B, lower, which, max_chunk, st);
  }
}

}  // namespace igm
