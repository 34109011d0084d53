// igm_trsv.cu -- sparse triangular substitutions on chunked group schedules:
// line 5' of Sec. VI (integer Lbar, Ubar: y_i = (z_i - sum Lbar_ij y_j) /
// Lbar_ii with an exact int128 numerator and truncating division), line 1'
// (the same in FP64 on the integer factors) and the FP64 comparison solver's
// ILU(0) apply, plus the set-up kernels that build the schedules' packed data
// and the FP64 ILU(0) factorisation (eq. ilu) on the same schedule.
//
// A CTA takes one chunk of consecutive positions (by ticket, in dependency
// order) and walks its groups (local levels, split to a width cap) in order,
// one named barrier per group.  Values of the chunk's recent groups stay in a
// ring in shared memory; everything else a row reads (its packed factors,
// diagonal, right-hand side, and the values of earlier chunks or of older
// groups) is brought into shared memory ahead of time: a producer warp
// bulk-copies each group's packed data (cp.async.bulk with mbarrier
// completion) several groups ahead, and the compute threads gather the
// right-hand sides and far values with cp.async two groups ahead, once a
// waiter warp has seen the previous chunk reach the groups they need.  A
// publisher warp releases the chunk's progress after each group.
#include <mutex>
#include <type_traits>

#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

#define IGM_TRSV_BLOCK 256
// dependencies of a row held in registers: 4 for 5/7-point stencils, 16 for
// up to 27-point ones; longer rows read the rest from shared memory
#define IGM_TRSV_KC_SMALL 4
#define IGM_TRSV_KC_LARGE 16

// ---------------------------------------------------------------------------
// set-up: schedules and packed rows
// ---------------------------------------------------------------------------

// max strict-part entries per row of L (lower) or U
__global__ void s_maxdeps(int n, const int *rowptr, const int *diagpos, int lower, int *kmax) {
  int k = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    k = max(k, lower ? diagpos[i] - rowptr[i] : rowptr[i + 1] - diagpos[i] - 1);
  atomicMax(kmax, k);
}

// the chunk of a row: chunks cut the dependency order (L: i, U: n-1-i)
__device__ __forceinline__ int chunk_of(int i, int n, int lower, int R) {
  return (lower ? i : n - 1 - i) / R;
}

// the largest distance, in chunks, from a row to one of its dependencies:
// at most 1 means every chunk reads only itself and its predecessor
__global__ void s_chunkdist(int n, const int *rowptr, const int *col, const int *diagpos,
                            int lower, int R, int *dmax) {
  int d = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    const int k1 = lower ? diagpos[i] : rowptr[i + 1];
    const int ci = chunk_of(i, n, lower, R);
    for (int k = k0; k < k1; ++k) d = max(d, ci - chunk_of(col[k], n, lower, R));
  }
  atomicMax(dmax, d);
}

// Splits every level group wider than `cap` rows into consecutive groups of
// at most cap rows (rows of one level are independent, so any split keeps
// the dependencies); records each row's new group index local to its chunk
// and its position.  ord is the order of the level groups (positions kept);
// lptr_old/levb_old their bounds, newbase[g] the first new group of old
// group g, levb_new the first new group of each chunk.
__global__ void s_regroup(int n, int R, const int *ord, int *lev, const int *levb_old,
                          const int *lptr_old, const int *newbase, const int *levb_new, int cap,
                          int *posof) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = ord[p];
    const int c = p / R;
    const int g = levb_old[c] + lev[i];
    const int gn = newbase[g] + (p - lptr_old[g]) / cap;
    lev[i] = gn - levb_new[c];
    posof[i] = p;
  }
}

// the largest (end of a row's group) - (position of a same-chunk dependency):
// a ring of at least this many values holds every same-chunk dependency
// until it is read
__global__ void s_ringdist(int n, const int *rowptr, const int *col, const int *diagpos,
                           int lower, int R, const int *ord, const int *posof, const int *lev,
                           const int *levb, const int *lptr, int *dmax) {
  int d = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = ord[p];
    const int c = p / R, first = c * R;
    const int b = lptr[levb[c] + lev[i] + 1];
    const int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    const int k1 = lower ? diagpos[i] : rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const int pj = posof[col[k]];
      if (pj >= first) d = max(d, b - pj);
    }
  }
  atomicMax(dmax, d);
}

// The predecessor ring: after iteration l of chunk c (the copy that serves
// group l + IGM_TRSV_PFB) the previous chunk's values up to position
// front[c][l] (+1 for the even rounding of the copies) are in the ring,
// front = lptr of the previous chunk at the largest need of groups
// 0 .. l + PFB (needpm: that prefix maximum per group).  Copies of iteration
// l must not overwrite values that groups l and later still read, so the
// ring needs front + 2 - (each such value's position) slots.
__global__ void s_pringdist(int n, const int *rowptr, const int *col, const int *diagpos,
                            int lower, int R, const int *ord, const int *posof, const int *lev,
                            const int *levb, const int *lptr, const int *needpm, int *dmax) {
  int d = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = ord[p];
    const int c = p / R, first = c * R;
    if (c == 0) continue;
    const int l = lev[i], nl = levb[c + 1] - levb[c];
    const int g = min(l + IGM_TRSV_PFB, nl - 1);
    const int front = lptr[levb[c - 1] + needpm[levb[c] + g]];
    const int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    const int k1 = lower ? diagpos[i] : rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const int pj = posof[col[k]];
      if (pj < first) d = max(d, front + 2 - pj);
    }
  }
  atomicMax(dmax, d);
}

// the largest |entry| of the strict part of L (lower) or U: whether the
// factor packs as int32
__global__ void s_facmax(int n, const int *rowptr, const int *diagpos, int lower, const i64 *fac,
                         unsigned long long *mx) {
  u64 m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    const int k1 = lower ? diagpos[i] : rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const i64 v = fac[k];
      const u64 a = v < 0 ? 0ull - (u64)v : (u64)v;
      m = a > m ? a : m;
    }
  }
  atomicMax(mx, m);
}

// Packs the rows of every group into the group's block (the layout of
// trsv_blk_bytes): each row's strict part farthest dependency first (L:
// columns ascending, U: descending) with each dependency's code
// (IGM_DEP_*): same-chunk values recent enough for the own ring at their
// chunk-local position mod ring; values of the previous chunk (single = 1,
// every dependency in this chunk or the previous one) at ring + their
// position mod pring; padding at the zero (ring + pring); the rest as late
// reads.  Factors as int32 when fac32.  The row word (IGM_ROW_*): the bound
// (with S = sum_q |fac_q| of the row, every |y_q| <= 2^bound keeps each
// product and the sum below 2^62 in magnitude: 62 - bit length of S, none
// when no such bound exists), the division shift, the late flag.  blobd
// (FP64 comparison solver, may be NULL): the same rows with FP64 factors
// and diagonals (1 for the unit lower factor), offsets boffd.
__global__ void s_pack(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                       int K, int R, int single, int ring, int pring, int fac32, const int *ord,
                       const int *posof, const int *lev, const int *levb, const int *lptr,
                       const long long *boff, const long long *boffd, const i64 *fac,
                       const i64 *ldiag, const i64 *udiag, const double *f, unsigned char *blob,
                       unsigned char *blobd) {
  const int zero = ring + pring;
  const int fb = fac32 ? 4 : 8;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = ord[p];
    const int c = p / R, first = c * R;
    const int g = levb[c] + lev[i];
    const int r = p - lptr[g], wp = (int)trsv_wp(lptr[g + 1] - lptr[g]);
    const int b = lptr[g + 1];
    unsigned char *base = blob + boff[g];
    int *bcode = reinterpret_cast<int *>(base);
    int *bord = bcode + (size_t)K * wp;
    int *byb = bord + wp;
    unsigned char *bfac = reinterpret_cast<unsigned char *>(byb + wp);
    i64 *bdiag = reinterpret_cast<i64 *>(bfac + (size_t)fb * K * wp);
    u64 *bdm = reinterpret_cast<u64 *>(bdiag + wp);
    unsigned char *based = blobd ? blobd + boffd[g] : nullptr;
    const int k0 = lower ? rowptr[i] : diagpos[i] + 1;
    const int k1 = lower ? diagpos[i] : rowptr[i + 1];
    const int cnt = k1 - k0;
    u128 sabs = 0;
    bool late = false;
    for (int q = 0; q < K; ++q) {
      int code = zero;
      i64 fv = 0;
      double fd = 0.0;
      if (q < cnt) {
        const int k = lower ? k0 + q : k1 - 1 - q;
        const int pj = posof[col[k]];
        if (pj >= first) code = (b - pj <= ring) ? ((pj - first) & (ring - 1)) : -1 - pj;
        else if (single) code = ring + (pj & (pring - 1));
        else code = -1 - pj;
        fv = fac[k];
        if (f) fd = f[k];
        sabs += (u128)(fv < 0 ? 0ull - (u64)fv : (u64)fv);
        late |= code < 0;
      }
      bcode[(size_t)q * wp + r] = code;
      if (fac32) reinterpret_cast<int *>(bfac)[(size_t)q * wp + r] = (int)fv;
      else reinterpret_cast<i64 *>(bfac)[(size_t)q * wp + r] = fv;
      if (based) {
        reinterpret_cast<int *>(based)[(size_t)q * wp + r] = code;
        reinterpret_cast<double *>(based + (size_t)(4 * K + 8) * wp)[(size_t)q * wp + r] = fd;
      }
    }
    int bl = 0;  // bit length of sabs
    while (bl < 127 && (sabs >> bl) != 0) ++bl;
    bord[r] = i;
    const i64 dg = lower ? ldiag[i] : udiag[i];
    const u64 adg = dg < 0 ? 0ull - (u64)dg : (u64)dg;
    const int bound = 62 - bl < -1 ? -1 : 62 - bl;
    byb[r] = (bound + 1) | (ceil_log2_u64(adg) << 8) | (late ? IGM_ROW_LATE : 0);
    bdiag[r] = dg;
    bdm[r] = dg == 0 ? 0 : magic_u64(adg);
    if (based) {
      int *dord = reinterpret_cast<int *>(based) + (size_t)K * wp;
      dord[r] = i;
      dord[wp + r] = late ? IGM_ROW_LATE : 0;
      double *ddg = reinterpret_cast<double *>(based + (size_t)(4 * K + 8) * wp + (size_t)8 * K * wp);
      ddg[r] = lower ? 1.0 : f[diagpos[i]];
      reinterpret_cast<u64 *>(ddg + wp)[r] = 0;
    }
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


// asynchronous 8-byte global -> shared copy (a thread waits for its own
// groups of copies)
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(src)),
               "r"(bytes)
               : "memory");
}

// CTA-scope release / acquire on shared-memory counters
__device__ __forceinline__ void red_release_cta(unsigned *p, unsigned v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}


// The waits of a substitution CTA are bounded in time (the system's
// p.wait_ns, 1 s unless set), nested so that a wait never expires while the
// wait it depends on can still succeed: the waiter gives up after the bound,
// the producer and the publisher (who wait on the compute warps, who wait on
// the waiter and on the bulk copies) after four times.  An iteration cap
// backs up each bound.

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

// spin until the shared counter *p reaches at least v, bounded by time only
// (for a wait whose giving up early would leave slots unfilled: the compute
// warps it waits on always advance, since all their own waits are bounded)
__device__ __forceinline__ bool wait_cta_own(const unsigned *p, unsigned v, unsigned *err,
                                             u64 limit_ns) {
  if (ld_acquire_cta(p) >= v) return true;
  const u64 t0 = gtimer();
  for (int it = 0; it < IGM_WAIT_ITERS; ++it) {
    if (ld_acquire_cta(p) >= v) return true;
    if (it > 64) __nanosleep(32);
    if ((it & 255) == 255 && gtimer() - t0 > limit_ns) break;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}


// Roles in a substitution CTA: IGM_TRSV_CW compute warps walk the groups,
// one named barrier per group among them (which makes the previous group's
// ring values visible; after it thread 0 releases the count of finished
// groups); the waiter warp acquires the previous chunk's progress and
// bulk-copies its values into the predecessor ring ahead of the groups that
// read them; the publisher warp turns the count of finished groups into this
// chunk's progress word; the block warp bulk-copies each group's packed
// block into a slot as slots free up (and prefetches later blocks into L2);
// the gather warp waits for each block and gathers the group's right-hand
// sides into the slot, the group's ready barrier completing when both are
// there.
#define IGM_TRSV_CW 8
#define IGM_TRSV_NC (IGM_TRSV_CW * 32)
#define IGM_TRSV_THREADS (IGM_TRSV_NC + 128)
// groups ahead of the L2 prefetch of the blocks, past the slots
#define IGM_TRSV_PFL 8

__device__ __forceinline__ void st_release_cta(unsigned *p, unsigned v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// arrives on bar once this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive_noinc(u64 *bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <int KIND, int KC>
__global__ void __launch_bounds__(IGM_TRSV_THREADS, 1)
    k_trsv_lv(BatchDev B, int lower, int which) {
  typedef typename TrsvT<KIND>::V V;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_t;
  __shared__ int s_poison;     // a compute-side wait expired: no slot is read again
  __shared__ unsigned s_done;  // groups the compute warps have finished
  __shared__ __align__(8) u64 s_blk[IGM_TRSV_NA_MAX];  // a slot's block has landed
  __shared__ __align__(8) u64 s_rdy[IGM_TRSV_NA_MAX];  // ... and its right-hand sides
  __shared__ __align__(8) u64 s_barp[IGM_TRSV_NB];     // a group's predecessor values
  const int tk = which == 0 ? (lower ? 0 : 1) : (lower ? 2 : 3);
  if (threadIdx.x == 0) {
    s_t = (int)atomicAdd(&B.ticket[tk], 1u);
    s_done = 0;
    s_poison = 0;
    for (int k = 0; k < IGM_TRSV_NA_MAX; ++k) {
      mbar_init(&s_blk[k], 1);
      mbar_init(&s_rdy[k], 33);  // the gather warp's 32 copy arrivals and lane 0
    }
    for (int k = 0; k < IGM_TRSV_NB; ++k) mbar_init(&s_barp[k], 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();
  const int t = s_t;
  if (t >= B.nctiles) return;
  const Tile ct = B.ctiles[t];
  const SysDev *s = B.sys[ct.sys];
  SysScal *sc = s->sc;
  if (!(sc->cyc != 0 && sc->early == 0) || !s->p.precond) return;
  const Tri T = s->tri[lower ? 0 : 1];
  const int c = ct.row0, n = s->n, R = s->chunk;
  const int first = c * R;
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
  const int K = T.K;
  const unsigned rmask = (unsigned)T.ring - 1u, pmask = (unsigned)T.pring - 1u;
  unsigned *err = &sc->err;
  V *xbuf = reinterpret_cast<V *>(s->xbuf);
  // factor entries of 4 bytes when they fit (the FP64 comparison solver's
  // factors are FP64)
  const bool f32 = KIND != TK_FP && T.fac32 != 0;
  const int fb = f32 ? 4 : 8;
  const unsigned char *blob = KIND == TK_FP ? T.blobd : T.blob;
  const long long *boff = KIND == TK_FP ? T.boffd : T.boff;
  const TrsvLayout Ly = trsv_layout(T.maxw, K, T.ring, T.pring, T.maxlev, fb);
  const int na = (int)Ly.na;
  // the values a row reads: own ring, predecessor ring, a zero for padding
  V *vals = reinterpret_cast<V *>(smem);
  V *pring = vals + T.ring;
  if (threadIdx.x == 0) vals[T.ring + T.pring] = (V)0;
  int *slptr = reinterpret_cast<int *>(smem + Ly.oLev);
  int *sneed = slptr + Ly.lev + 1;
  int *splptr = sneed + Ly.lev + 1;  // the previous chunk's group pointers
  const bool lev_smem = Ly.lev != 0;
  const bool pred = single && c > 0;
  const int pg0 = pred ? T.levb[c - 1] : 0, pnlev = pred ? g0 - pg0 : 0;
  const int pfirst = (c - 1) * R;  // first position of the previous chunk
  if (lev_smem) {
    for (int q = threadIdx.x; q <= nlev; q += blockDim.x) slptr[q] = T.lptr[g0 + q];
    for (int q = threadIdx.x; q < nlev; q += blockDim.x) sneed[q] = T.need[g0 + q];
    for (int q = threadIdx.x; q <= pnlev; q += blockDim.x) splptr[q] = T.lptr[pg0 + q];
  }
  __syncthreads();
#define LPTR(l) (lev_smem ? slptr[l] : T.lptr[g0 + (l)])
#define NEED(l) (lev_smem ? sneed[l] : T.need[g0 + (l)])
#define PLPTR(l) (lev_smem ? splptr[l] : T.lptr[pg0 + (l)])
  auto slot = [&](int lv) { return smem + Ly.oSlots + (size_t)(lv % na) * Ly.szSlot; };
  auto width = [&](int lv) { return LPTR(lv + 1) - LPTR(lv); };
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (wid == IGM_TRSV_CW) {  // waiter: the previous chunk's values, ahead of their groups
    if (lane == 0) {
      u64 seen = 0;   // groups of the previous chunk known to be done
      int copied = 0; // groups of the previous chunk copied into the predecessor ring
      int hi = pfirst;  // first position not yet copied
      // the copies of the last two groups (group, first and end position),
      // which may still be in flight
      int f_lb[2] = {-1, -1}, f_a[2] = {0, 0}, f_e[2] = {0, 0};
      bool dead = false;
      const u64 *pw = T.prog + (size_t)IGM_PROG_STRIDE * (c - 1);
      for (int lb = 0; lb < nlev; ++lb) {
        // the copy for group lb may overwrite values that groups up to
        // lb - 3 read (the set-up sized the ring for that): wait until the
        // compute warps are done with them (bounded by time only: slots
        // must not stay unfilled)
        if (lb >= 3 && !wait_cta_own(&s_done, (unsigned)(lb - 2), err, 8 * wns)) dead = true;
        const int nd = pred ? NEED(lb) : 0;
        if (!dead && (u64)nd > seen) {
          const u64 want = ep | (u64)nd;
          u64 v = ld_acquire64(pw);
          if (v < want) {
            const u64 t0 = gtimer();
            for (int k = 0; k < IGM_WAIT_ITERS; ++k) {
              if (k > 32) __nanosleep(16);
              v = ld_acquire64(pw);
              if (v >= want) break;
              if ((k & 255) == 255 &&
                  ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtimer() - t0 > wns))
                break;
            }
          }
          if (v < want) {  // expired: the copies still run, the result is flagged
            atomicOr(err, ERR_TIMEOUT);
            dead = true;
          } else {
            seen = v - ep;
          }
        }
        // copy the previous chunk's positions up to its end of group nd into
        // the predecessor ring (16-byte aligned pieces, split at the ring's
        // end); one arrival per group on its barrier
        u64 *bar = &s_barp[lb % IGM_TRSV_NB];
        unsigned bytes = 0;
        int a = 0, e = 0;
        if (nd > copied) {
          const int top = PLPTR(nd);
          e = (top + 1) & ~1;
          // values more than a ring behind the copy's end are never read
          // again (the set-up sized the ring so), so one copy covers at most
          // one ring
          a = max(hi & ~1, e - (int)(pmask + 1u));
          bytes = (unsigned)(e - a) * 8u;
          hi = top;
          copied = nd;
          // copies are not ordered among themselves: a copy still in flight
          // (issued for the last two groups; older ones were waited for by
          // their groups' threads) that writes slots this one writes too --
          // the last pair of the previous copy, which held a value not yet
          // computed, or slots a ring apart -- must land first
          for (int k = 0; k < 2; ++k)
            if (f_lb[k] >= 0 && f_lb[k] >= lb - 2 &&
                (a < f_e[k] || e - f_a[k] > (int)(pmask + 1u)))
              mbar_wait(&s_barp[f_lb[k] % IGM_TRSV_NB], (unsigned)(f_lb[k] / IGM_TRSV_NB) & 1u,
                        err, 4 * wns);
          f_lb[1] = f_lb[0];
          f_a[1] = f_a[0];
          f_e[1] = f_e[0];
          f_lb[0] = lb;
          f_a[0] = a;
          f_e[0] = e;
        }
        if (bytes) fence_proxy_async_global();
        mbar_expect_tx(bar, bytes);
        while (a < e) {
          const unsigned sl = (unsigned)a & pmask;  // even: a is
          const int m = min(e - a, (int)(pmask + 1u - sl));
          bulk_g2s(pring + sl, xbuf + a, (unsigned)m * 8u, bar);
          a += m;
        }
      }
      // no copy may still be in flight when the CTA exits (the compute
      // warps waited for every group's copies unless a wait expired)
      for (int lb = nlev - IGM_TRSV_NB > 0 ? nlev - IGM_TRSV_NB : 0; lb < nlev; ++lb)
        mbar_wait(&s_barp[lb % IGM_TRSV_NB], (unsigned)(lb / IGM_TRSV_NB) & 1u, err, 4 * wns);
    }
    return;
  }
  if (wid == IGM_TRSV_CW + 1) {  // publisher
    if (lane == 0) {
      for (unsigned pub = 0; pub < (unsigned)nlev;) {
        // groups the compute warps have finished
        if (!wait_cta(&s_done, pub + 1, err, 4 * wns)) break;
        pub = ld_acquire_cta(&s_done);
        if (mute) continue;
        st_release64(T.prog + (size_t)IGM_PROG_STRIDE * c, ep | (u64)pub);
      }
    }
    return;
  }
  if (wid == IGM_TRSV_CW + 2) {  // block warp
    if (lane == 0) {
      // blocks of one chunk are contiguous: each group's offset follows from
      // the widths
      long long off = boff[g0], poff = off;
      int pl = 0;  // next group to prefetch into L2
      auto bytes_of = [&](int lv) { return trsv_blk_bytes(trsv_wp(width(lv)), K, fb); };
      auto prefetch_upto = [&](int lv) {
        for (; pl <= lv && pl < nlev; ++pl) {
          const unsigned b = bytes_of(pl);
          bulk_prefetch_l2(blob + poff, b);
          poff += b;
        }
      };
      auto issue = [&](int lv) {
        const unsigned b = bytes_of(lv);
        u64 *bar = &s_blk[lv % na];
        mbar_expect_tx(bar, b);
        bulk_g2s(slot(lv), blob + off, b, bar);
        off += b;
      };
      prefetch_upto(na + IGM_TRSV_PFL - 1);
      for (int lv = 0; lv < na && lv < nlev; ++lv) issue(lv);
      // the slot of group k - 1 takes group k - 1 + na once k groups are done
      for (int k = 1; k - 1 + na < nlev; ++k) {
        if (!wait_cta_own(&s_done, (unsigned)k, err, 8 * wns)) break;
        issue(k - 1 + na);
        prefetch_upto(k - 1 + na + IGM_TRSV_PFL);
      }
      // no copy may still be in flight when the CTA exits
      for (int k = 0; k < na && k < nlev; ++k) {
        const int lastlv = k + (nlev - 1 - k) / na * na;
        mbar_wait(&s_blk[k], (unsigned)(lastlv / na) & 1u, err, 4 * wns);
      }
    }
    return;
  }
  if (wid == IGM_TRSV_CW + 3) {  // gather warp: right-hand sides into each slot
    for (int lv = 0; lv < nlev; ++lv) {
      const int k = lv % na;
      const bool ok = mbar_wait(&s_blk[k], (unsigned)(lv / na) & 1u, err, 4 * wns);
      const int w = width(lv);
      unsigned char *sl = slot(lv);
      if (ok) {  // the block's orders are in place
        const int *bord = reinterpret_cast<const int *>(sl) + (size_t)K * trsv_wp(w);
        V *rhs = reinterpret_cast<V *>(sl + Ly.szBlk);
        for (int r = lane; r < w; r += 32)
          if (IGM_OK((unsigned)bord[r] < (unsigned)n, CHK_TRSV_RHS)) cp_async8(rhs + r, in + bord[r]);
      }
      cp_async_arrive_noinc(&s_rdy[k]);
      if (lane == 0) mbar_arrive(&s_rdy[k]);
    }
    cp_async_wait<0>();
    return;
  }

  // compute warps.  One idle-most thread (the last) waits for group l's
  // slot and predecessor copies before the group's barrier, which then
  // passes their arrival on to every compute thread.  If that wait expires
  // no compute thread reads a slot's contents again (they may be stale or
  // never written): they keep their barrier obligations and leave their
  // rows alone; the call reports IGM_ETIMEOUT.
  const int tid = threadIdx.x;
  unsigned ev = 0;
  auto late = [&](int code) -> V {
    const int pj = -1 - code;
    if (!single && pj < first)
      wait_prog(T.prog + (size_t)IGM_PROG_STRIDE * (pj / R),
                ep | (u64)(T.lev[T.ord[pj]] + 1), err);
    return (V)__ldcg(xbuf + pj);
  };
  int cs = 0, us = 0;  // slot of group l and its uses before l (l mod na, l / na)
  int cb = 0, up = 0;  // barrier of group l's predecessor copy (l mod NB, l / NB)
  for (int l = 0; l < nlev; ++l) {
    if (tid == IGM_TRSV_NC - 1 && !s_poison &&
        !(mbar_wait(&s_rdy[cs], (unsigned)us & 1u, err, 2 * wns) &&
          mbar_wait(&s_barp[cb], (unsigned)up & 1u, err, 2 * wns)))
      s_poison = 1;
    __syncwarp();
    // the previous group's ring values and group l's slot are visible
    asm volatile("bar.sync 2, %0;" ::"n"(IGM_TRSV_NC) : "memory");
    if (tid == IGM_TRSV_NC - 2 && l > 0) st_release_cta(&s_done, (unsigned)l);
    const int p0 = LPTR(l), w = LPTR(l + 1) - p0;
    const bool poisoned = s_poison != 0;
    if (tid < w && !poisoned) {
      const unsigned wp = trsv_wp(w);
      const unsigned char *blk = smem + Ly.oSlots + (size_t)cs * Ly.szSlot;
      const int *scode = reinterpret_cast<const int *>(blk);
      const int *sord = scode + (size_t)K * wp;
      const int *syb = sord + wp;
      const unsigned char *sfac = reinterpret_cast<const unsigned char *>(syb + wp);
      const unsigned char *sdg = sfac + (size_t)fb * K * wp;  // diagonals, then multipliers
      const V *srhs = reinterpret_cast<const V *>(blk + Ly.szBlk);
      for (int r = tid; r < w; r += IGM_TRSV_NC) {
        const int row = sord[r];
        const int wd = syb[r];
        // rows whose dependencies are all in shared memory (the common case)
        // fetch them without branches, so all the loads issue together
        const bool onchip = (wd & IGM_ROW_LATE) == 0;
        auto dep = [&](int q) -> V {
          const int code = scode[(size_t)q * wp + r];
          return code >= 0 ? vals[code] : late(code);
        };
        auto dep_on = [&](int q) -> V { return vals[scode[(size_t)q * wp + r]]; };
        auto fac = [&](int q) -> i64 {
          return f32 ? (i64)reinterpret_cast<const int *>(sfac)[(size_t)q * wp + r]
                     : reinterpret_cast<const i64 *>(sfac)[(size_t)q * wp + r];
        };
        V y;
        if (KIND == TK_INT) {
          i64 yv[KC], fv[KC];
          u64 mag = 0;  // the largest |y| (as y ^ (y >> 63))
          if (onchip) {
#pragma unroll
            for (int q = 0; q < KC; ++q) yv[q] = q < K ? (i64)dep_on(q) : 0;
          } else {
#pragma unroll
            for (int q = 0; q < KC; ++q) yv[q] = q < K ? (i64)dep(q) : 0;
          }
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            fv[q] = q < K ? fac(q) : 0;
            mag |= (u64)(yv[q] ^ (yv[q] >> 63));
          }
          for (int q = KC; q < K; ++q) {
            const i64 v = onchip ? (i64)dep_on(q) : (i64)dep(q);
            mag |= (u64)(v ^ (v >> 63));
          }
          const i64 rhs = (i64)srhs[r];
          const int yb = IGM_ROW_BOUND(wd);
          i64 num;
          if (yb >= 0 && (mag >> yb) == 0) {
            // every product and the sum are below 2^62 (the set-up's bound):
            // exact in 64-bit words, no event possible; only the difference
            // with the right-hand side may leave the range
            i64 sum = 0;
#pragma unroll
            for (int q = 0; q < KC; ++q) sum += fv[q] * yv[q];
            for (int q = KC; q < K; ++q)
              sum += fac(q) * (onchip ? (i64)dep_on(q) : (i64)dep(q));
            num = (i64)((u64)rhs - (u64)sum);
            ev += (((rhs ^ sum) & (rhs ^ num)) < 0);
          } else {
            i128 sum = 0;
#pragma unroll
            for (int q = 0; q < KC; ++q) sum += (i128)mulw(fv[q], yv[q], ev);
            for (int q = KC; q < K; ++q)
              sum += (i128)mulw(fac(q), onchip ? (i64)dep_on(q) : (i64)dep(q), ev);
            const i128 acc = (i128)rhs - sum;
            ev += out64(acc);
            num = wrap(acc);
          }
          const i64 dg = reinterpret_cast<const i64 *>(sdg)[r];
          const u64 dm = reinterpret_cast<const u64 *>(sdg)[(size_t)wp + r];
          y = (V)divt_magic_l(num, dg, dm, IGM_ROW_SHIFT(wd), ev);
        } else {
          // FP64: subtract in CSR order (L packed ascending, U descending);
          // padding subtracts an exact zero
          auto facd = [&](int q) -> double {
            if (KIND == TK_FPI) return (double)fac(q);
            return reinterpret_cast<const double *>(sfac)[(size_t)q * wp + r];
          };
          double acc = (double)srhs[r];
          for (int k = 0; k < K; ++k) {
            const int q = lower ? k : K - 1 - k;
            acc = __dsub_rn(acc, __dmul_rn(facd(q), (double)(onchip ? dep_on(q) : dep(q))));
          }
          if (KIND == TK_FP && lower) {
            y = (V)acc;  // unit lower factor
          } else {
            const double dg = KIND == TK_FPI ? (double)reinterpret_cast<const i64 *>(sdg)[r]
                                             : reinterpret_cast<const double *>(sdg)[r];
            y = (V)__ddiv_rn(acc, dg);
          }
        }
        vals[(unsigned)(p0 + r - first) & rmask] = y;
        out[row] = y;
        xbuf[p0 + r] = y;
      }
    }
    if (++cs == na) {
      cs = 0;
      ++us;
    }
    if (++cb == IGM_TRSV_NB) {
      cb = 0;
      ++up;
    }
  }
  __syncwarp();
  asm volatile("bar.sync 2, %0;" ::"n"(IGM_TRSV_NC) : "memory");
  if (tid == IGM_TRSV_NC - 2) st_release_cta(&s_done, (unsigned)nlev);
  if (KIND == TK_INT) flush_ev(ev, &sc->ev[IGM_EV_L5P]);
#undef LPTR
#undef NEED
#undef PLPTR
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

void launch_chunkdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                      int R, int *dmax, cudaStream_t st) {
  s_chunkdist<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, R, dmax);
}

void launch_regroup(int n, int R, const int *ord, int *lev, const int *levb_old,
                    const int *lptr_old, const int *newbase, const int *levb_new, int cap,
                    int *posof, cudaStream_t st) {
  s_regroup<<<grid_n(n), 256, 0, st>>>(n, R, ord, lev, levb_old, lptr_old, newbase, levb_new, cap,
                                        posof);
}

void launch_ringdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                     int R, const int *ord, const int *posof, const int *lev, const int *levb,
                     const int *lptr, int *dmax, cudaStream_t st) {
  s_ringdist<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, R, ord, posof, lev, levb,
                                         lptr, dmax);
}

void launch_pringdist(int n, const int *rowptr, const int *col, const int *diagpos, int lower,
                      int R, const int *ord, const int *posof, const int *lev, const int *levb,
                      const int *lptr, const int *needpm, int *dmax, cudaStream_t st) {
  s_pringdist<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, R, ord, posof, lev, levb,
                                          lptr, needpm, dmax);
}

void launch_facmax(int n, const int *rowptr, const int *diagpos, int lower, const i64 *fac,
                   unsigned long long *mx, cudaStream_t st) {
  s_facmax<<<grid_n(n), 256, 0, st>>>(n, rowptr, diagpos, lower, fac, mx);
}

void launch_pack(int n, const int *rowptr, const int *col, const int *diagpos, int lower, int K,
                 int R, int single, int ring, int pring, int fac32, const int *ord,
                 const int *posof, const int *lev, const int *levb, const int *lptr,
                 const long long *boff, const long long *boffd, const i64 *fac, const i64 *ldiag,
                 const i64 *udiag, const double *f, unsigned char *blob, unsigned char *blobd,
                 cudaStream_t st) {
  s_pack<<<grid_n(n), 256, 0, st>>>(n, rowptr, col, diagpos, lower, K, R, single, ring, pring,
                                     fac32, ord, posof, lev, levb, lptr, boff, boffd, fac, ldiag,
                                     udiag, f, blob, blobd);
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

// the widest group a factor with K dependencies per row may have: every slot
// of the substitution kernel must fit in its shared memory with rings of the
// largest size
int trsv_group_cap(int K) {
  int W = 4096;
  while (W > 8 && trsv_layout(W, K, IGM_TRSV_RING_MAX, IGM_TRSV_RING_MAX, 0, 8,
                              IGM_TRSV_NA_MIN).total + 8 * 1024 > IGM_TRSV_SMEM)
    W -= 8;
  return W;
}

template <int KIND, int KC>
static void launch_lv(const BatchDev &B, int lower, int which, cudaStream_t st) {
  if (B.nctiles <= 0) return;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_trsv_lv<KIND, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IGM_TRSV_SMEM);
  });
  k_trsv_lv<KIND, KC><<<B.nctiles, IGM_TRSV_THREADS, IGM_TRSV_SMEM, st>>>(B, lower, which);
}

void launch_trsv_color(const BatchDev &B, int kind, int lower, int which, cudaStream_t st) {
  for (int c = 0; c < B.max_colors; ++c) {
    if (kind == TK_INT) k_trsv_color<TK_INT><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
    else if (kind == TK_FPI) k_trsv_color<TK_FPI><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
    else k_trsv_color<TK_FP><<<B.ntiles, 256, 0, st>>>(B, lower, which, c);
  }
}

void launch_trsv_lv(const BatchDev &B, int kind, int lower, int which, cudaStream_t st) {
  if (B.max_colors > 0) launch_trsv_color(B, kind, lower, which, st);
  if (B.trsv_maxk <= IGM_TRSV_KC_SMALL) {
    if (kind == TK_INT) launch_lv<TK_INT, IGM_TRSV_KC_SMALL>(B, lower, which, st);
    else if (kind == TK_FPI) launch_lv<TK_FPI, IGM_TRSV_KC_SMALL>(B, lower, which, st);
    else launch_lv<TK_FP, IGM_TRSV_KC_SMALL>(B, lower, which, st);
  } else {
    if (kind == TK_INT) launch_lv<TK_INT, IGM_TRSV_KC_LARGE>(B, lower, which, st);
    else if (kind == TK_FPI) launch_lv<TK_FPI, IGM_TRSV_KC_LARGE>(B, lower, which, st);
    else launch_lv<TK_FP, IGM_TRSV_KC_LARGE>(B, lower, which, st);
  }
}

IGM_CHECKS_READER(checks_read_trsv)

}  // namespace igm
