// igm_mgs.cu -- lines 6-11 of Fig. 2 (modified Gram-Schmidt, norm, division)
// for one Arnoldi step j as ONE persistent kernel: all CTAs are co-resident
// (cooperative launch) and sweep the rows of every system once per pass;
// each CTA stores its exact int128 sum of the pass per segment, a bounded
// grid barrier publishes them, and every CTA adds up the sums of its
// systems.  Pass i <= j fuses the line-8 update with h_{i-1,j} and the
// line-7 inner product with v_i; pass j+1 fuses the last update with the
// line-10 norm; then line 11 and, by the CTA holding each system's row 0,
// lines 12-19.  The basis streams from HBM once per pass; w stays in shared
// memory.  Small batches (every row in one CTA) run a one-CTA variant
// without the grid barrier.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {


__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid barrier with a bounded wait; false if it expired.  bar[0] counts
// arrivals, bar[1] is the generation.  Thread 0 arrives with an acq_rel add
// after the block barrier (so the CTA's writes before the barrier are
// released with it); the last arrival resets the count and releases the
// next generation, which the others acquire.
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned *gen = bar + 1;
    const unsigned g = ld_relaxed_u32(gen);
    const unsigned arrived = atom_add_acq_rel_u32(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      st_relaxed_u32(bar, 0u);
      st_release_u32(gen, g + 1u);
    } else {
      int it = 0;
      while (ld_acquire_u32(gen) == g) {
        if (++it > IGM_SPIN_MAX) {
          atomicOr(err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (it > 256) __nanosleep(20);
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// asynchronous 8-byte copy global -> shared (the one-CTA mode's basis staging)
__device__ __forceinline__ void mgs_cp_async8(i64 *dst, const i64 *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}

__device__ __forceinline__ void mgs_cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void mgs_cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// every group but the N most recent complete
template <int N>
__device__ __forceinline__ void mgs_cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ bool m_step(const SysDev *s, int j) {
  return s->sc->cyc != 0 && s->sc->early == 0 && j < s->p.m;
}

#define IGM_RPT 4           // rows in flight per thread
// threads of a grid-mode CTA (one CTA per SM)
#ifndef IGM_MGS_GBS
#define IGM_MGS_GBS 1024
#endif
#define IGM_MGS_GCACHE 32   // segment descriptors a CTA of the grid mode keeps in shared memory
// CTA rows of the grid mode resident in shared memory: w (int64) and two
// int32 basis vectors, 16 bytes a row (218 KB)
#define IGM_MGS_WMAX 13952
#define IGM_MGS_ROWB 16




// a segment as the step kernel sees it: its system's arrays and shifts
struct MSegC {
  i64 *V;        // basis of the system
  int *V32;      // the same as int32 words
  i64 *w;        // the segment's first row of w
  i64 *H;
  SysScal *sc;
  int n, row0, nrows, off, sys, ld;
  int df, b7, b8, b10, b11a, b11b;
  int first;   // holds row 0 of its system: records h_{i,j} and its events
  int active;  // the system takes this step
  int narrow;  // every basis entry of this inner solve fits int32 so far
};

__device__ __forceinline__ void mseg_make(const BatchDev &B, int g, int j, MSegC &c) {
  const Tile t = B.mseg[g];
  const SysDev *s = B.sys[t.sys];
  const SysParams &P = s->p;
  c.V = s->V;
  c.V32 = s->V32;
  c.w = s->w + t.row0;
  c.H = s->H;
  c.sc = s->sc;
  c.n = s->n;
  c.row0 = t.row0;
  c.nrows = t.nrows;
  c.off = t.first;
  c.sys = t.sys;
  c.ld = s->ld;
  c.df = P.df;
  c.b7 = P.b7;
  c.b8 = P.b8;
  c.b10 = P.b10;
  c.b11a = P.b11a;
  c.b11b = P.b11b;
  c.first = t.row0 == 0;
  c.active = m_step(s, j);
  c.narrow = s->sc->vwide == 0;
}

// after the barrier of pass i: the exact total of the pass; h_{i,j} (line 7)
// or h_{j+1,j} (line 10), recorded once per system with the total's event;
// returns the coefficient pass i+1 needs (line 8) or h_{j+1,j}
__device__ __forceinline__ i64 mseg_coef(const MSegC &c, i128 tot, int i, int j) {
  unsigned e = out64(tot);
  if (i <= j) {
    const i64 h = shr(wrap(tot), c.df - c.b7);
    if (c.first) {
      c.H[i + j * c.ld] = h;
      if (e) atomicAdd(&c.sc->ev[IGM_EV_L7], (u64)e);
    }
    return shr(h, c.b8);
  }
  const i64 h = fx_sqrt(wrap(tot), 2 * c.df - 2 * c.b10, c.df, e);
  if (c.first && e) atomicAdd(&c.sc->ev[IGM_EV_L10], (u64)e);
  return h;
}

// lines 10 (store of h_{j+1,j}) and 12-19 of c's system (one thread)
__device__ __forceinline__ void givens_tail(const BatchDev &B, const MSegC &c, int j, i64 hj1) {
  const SysDev *s = B.sys[c.sys];
  s->H[j + 1 + j * c.ld] = hj1;
  c.sc->hnext = hj1;
  c.sc->normj = shr(hj1, c.b11b) == 0 ? -1 : j;
  givens_col(s, c.sc, j, hj1);
}

// ---------------------------------------------------------------------------
// one-CTA mode
// ---------------------------------------------------------------------------

// One CTA of IGM_MGS_ONE_BLOCK threads holds every row of every system
// (small batches, mgs_one_cta): each system is one segment of it, w stays in
// shared memory, the pass totals stay in shared memory and a block barrier
// ends each pass; the basis vectors are staged in shared memory, v_{i+D}
// copied asynchronously while pass i runs (D = IGM_ONE_NBUF - 2 passes
// ahead, so a pass waits on no global load).
#define IGM_ONE_NBUF 5
__global__ void __launch_bounds__(IGM_MGS_ONE_BLOCK, 1) k_mgs_one(BatchDev B, int j) {
  constexpr int BS = IGM_MGS_ONE_BLOCK, NB = IGM_ONE_NBUF, D = IGM_ONE_NBUF - 2;
  extern __shared__ i64 s_dyn[];
  i64 (*s_v)[IGM_MGS_BLOCK] = reinterpret_cast<i64 (*)[IGM_MGS_BLOCK]>(s_dyn);  // v_i: s_v[i % NB]
  i64 *sw = s_dyn + NB * IGM_MGS_BLOCK;                                        // every row of w
  __shared__ MSegC s_seg[IGM_MSEG_CACHE];
  __shared__ i64 s_h[IGM_MSEG_CACHE];
  __shared__ i128 s_tot[IGM_MSEG_CACHE];
  const int ns = B.mseg_ptr[1];
  for (int k = threadIdx.x; k < ns; k += BS) mseg_make(B, k, j, s_seg[k]);
  __syncthreads();
  // stage v_i into s_v[i % NB] (nothing for i > j); one copy group either way
  auto stage = [&](int i) {
    for (int k = 0; k < ns && i <= j; ++k) {
      const MSegC &c = s_seg[k];
      if (!c.active) continue;
      const i64 *src = c.V + (size_t)i * c.n + c.row0;
      i64 *dst = &s_v[i % NB][c.off];
      for (int q = threadIdx.x; q < c.nrows; q += BS) mgs_cp_async8(dst + q, src + q);
    }
    mgs_cp_async_commit();
  };
  for (int t = 0; t < D; ++t) stage(t);
  mgs_cp_async_wait<D - 1>();  // v_0
  __syncthreads();
  for (int i = 0; i <= j + 1; ++i) {
    // into the buffer of v_{i-2}, last read in pass i - 1
    stage(i + D);
    for (int k = 0; k < ns; ++k) {
      const MSegC &c = s_seg[k];
      if (!c.active) continue;
      const i64 hs = i == 0 ? 0 : s_h[k];
      const int nr = c.nrows;
      const i64 *vp = &s_v[(i + NB - 1) % NB][c.off], *vi = &s_v[i % NB][c.off];
      const i64 *wg = c.w;
      i64 *ws = sw + c.off;
      const int s8 = shc(c.df - c.b8), s7 = shc(c.b7), s10 = shc(c.b10);
      const bool hs32 = hs == (i64)(int)hs;
      i128 part = 0;
      unsigned evA = 0, evB = 0;
      for (int q = threadIdx.x; q < nr; q += BS) {
        i64 wl = i > 0 ? ws[q] : wg[q];
        if (i > 0) {
          const i64 pv = vp[q];
          const i64 pr = (hs32 && pv == (i64)(int)pv) ? (i64)(int)hs * (i64)(int)pv
                                                      : mulw(hs, pv, evB);
          wl = subw(wl, pr >> s8, evB);
        }
        ws[q] = wl;
        if (i <= j) {
          const i64 a = wl >> s7, b = vi[q];
          part += (i128)((a == (i64)(int)a && b == (i64)(int)b) ? (i64)(int)a * (i64)(int)b
                                                                : mulw(a, b, evA));
        } else {
          const i64 a = wl >> s10;
          part += (i128)(a == (i64)(int)a ? (i64)(int)a * (i64)(int)a : mulw(a, a, evA));
        }
      }
      flush_ev(evB, &c.sc->ev[IGM_EV_L8]);
      flush_ev(evA, &c.sc->ev[i <= j ? IGM_EV_L7 : IGM_EV_L10]);
      part = block_sum_i128(part);
      if (threadIdx.x == 0) s_tot[k] = part;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += BS)
      if (s_seg[k].active) s_h[k] = mseg_coef(s_seg[k], s_tot[k], i, j);
    mgs_cp_async_wait<D - 1>();  // v_{i+1} is in place for pass i+1
    __syncthreads();
  }
  // line 11 for every system whose divisor is non-zero
  for (int k = 0; k < ns; ++k) {
    const MSegC &c = s_seg[k];
    if (!c.active) continue;
    const i64 hn = s_h[k];
    if (shr(hn, c.b11b) == 0) continue;
    i64 *vn = c.V + (size_t)(j + 1) * c.n + c.row0;
    int *vn32 = c.V32 + (size_t)(j + 1) * c.n + c.row0;
    const i64 *ws = sw + c.off;
    unsigned ev = 0, evr = 0;
    for (int q = threadIdx.x; q < c.nrows; q += BS) {
      const i64 v = fx_div(ws[q], hn, c.b11a, c.b11b, c.df, ev);
      evr += (v < INT32_MIN || v > INT32_MAX);
      vn[q] = v;
      vn32[q] = (int)v;
    }
    flush_ev(ev, &c.sc->ev[IGM_EV_L11]);
    if (__syncthreads_or(evr != 0) && threadIdx.x == 0) atomicOr(&c.sc->vwide, 1);
    flush_ev(evr, &c.sc->ev[IGM_EV_VRANGE]);
  }
  // lines 10 (store) and 12-19, one thread per system
  __syncthreads();
  for (int k = threadIdx.x; k < ns; k += BS)
    if (s_seg[k].active && s_seg[k].first) givens_tail(B, s_seg[k], j, s_h[k]);
}

// ---------------------------------------------------------------------------
// grid mode
// ---------------------------------------------------------------------------

// The exact sum of a pass over one segment travels as three 64-bit words,
// each (32 bits of the sum << 32) | tag, tag = (launch epoch << 8) | (pass
// + 1): a word is read whole or not at all (single-copy atomicity of aligned
// 64-bit accesses), so a reader that sees the current tag in all three has
// the sum, with no fence and no barrier.  |sum| < 2^95 (at most 2^31 rows of
// int64 products), so 96 bits hold it.  Slot of segment g for pass parity
// p: 4 words (32-byte aligned) at mpart[(p * nseg + g) * 4].
__device__ __forceinline__ u64 *mslot(const BatchDev &B, int par, int g) {
  return B.mpart + ((size_t)par * B.nseg + g) * 4;
}

__device__ __forceinline__ void mslot_put(u64 *sl, i128 v, unsigned tag) {
  const u128 u = (u128)v;
  const u64 w0 = ((u64)(unsigned)u << 32) | tag;
  const u64 w1 = ((u64)(unsigned)(u >> 32) << 32) | tag;
  const u64 w2 = ((u64)(unsigned)(u >> 64) << 32) | tag;
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(sl), "l"(w0), "l"(w1)
               : "memory");
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(sl + 2), "l"(w2) : "memory");
}

__device__ __forceinline__ void mslot_load(const u64 *sl, u64 &w0, u64 &w1, u64 &w2) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(w0), "=l"(w1)
               : "l"(sl)
               : "memory");
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w2) : "l"(sl + 2) : "memory");
}

__device__ __forceinline__ i128 mslot_value(u64 w0, u64 w1, u64 w2) {
  const i128 hi = (i128)(int)(unsigned)(w2 >> 32);
  return (i128)(((u128)hi << 64) | ((u128)(w1 >> 32) << 32) | (u128)(w0 >> 32));
}

// The exact total of a pass over every segment of system `sys`, gathered
// by the whole CTA from the segments' tagged slots, one slot per thread (a
// system has at most one segment per CTA); valid in thread 0.  False (in
// every thread) when a slot did not carry the tag within the wait bound or
// a CTA has reported an expired wait.
__device__ bool mseg_total(const BatchDev &B, int sys, int par, unsigned tag,
                           const unsigned *err0, i128 &tot) {
  const int lo = B.sys_seg[sys], hi = B.sys_seg[sys + 1];
  i128 t = 0;
  bool ok = true;
  for (int g = lo + threadIdx.x; g < hi && ok; g += blockDim.x) {
    for (int it = 0;; ++it) {
      u64 w0, w1, w2;
      mslot_load(mslot(B, par, g), w0, w1, w2);
      if ((unsigned)w0 == tag && (unsigned)w1 == tag && (unsigned)w2 == tag) {
        t += mslot_value(w0, w1, w2);
        break;
      }
      if (it > IGM_SPIN_MAX || ((it & 255) == 255 && (ld_relaxed_u32(err0) & ERR_TIMEOUT))) {
        ok = false;
        break;
      }
      if (it > 32) __nanosleep(32);
    }
  }
  tot = block_sum_i128(t);
  return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ bool fits32(int) { return true; }
__device__ __forceinline__ bool fits32(i64 x) { return x == (i64)(int)x; }

// Pass work on IGM_RPT rows of a segment whose values are loaded (w in wv,
// v_{i-1} in pv, v_i in qv; rows past the end hold zeros, which change
// nothing and raise no event).  MODE 0: pass 0 (line 7 with v_0); 1:
// 0 < i <= j (line 8 with h_{i-1,j}, line 7 with v_i); 2: i = j + 1 (line 8
// with h_{j,j}, line 10).  HS32: line 8's coefficient fits int32.  The
// products of lines 7 / 10 are taken as 32x32 -> 64-bit multiplies (exact,
// never out of range: the same word, no event) and redone with the general
// wrapped product only when a factor leaves int32, so the common case has
// no branch per row.  wv returns the updated w.
template <int MODE, bool HS32, int R, typename VT>
__device__ __forceinline__ void rows_pass(i64 (&wv)[R], const VT (&pv)[R], const VT (&qv)[R],
                                          i64 hs, int s8, int sA, i128 &part, unsigned &evA,
                                          unsigned &evB) {
  i64 pr[R];
  bool fast = true;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (MODE > 0) {
      i64 p;
      if (HS32 && sizeof(VT) == 4) p = (i64)(int)hs * (i64)pv[u];
      else p = mulw(hs, (i64)pv[u], evB);
      wv[u] = subw(wv[u], p >> s8, evB);
    }
    const i64 a = wv[u] >> sA;
    const i64 b = MODE == 2 ? a : (i64)qv[u];
    fast = fast && fits32(a) && fits32(b);
    pr[u] = (i64)(int)a * (i64)(int)b;
  }
  if (!fast) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const i64 a = wv[u] >> sA;
      const i64 b = MODE == 2 ? a : (i64)qv[u];
      if (!(fits32(a) && fits32(b))) pr[u] = mulw(a, b, evA);
    }
  }
#pragma unroll
  for (int u = 0; u < R; ++u) part += (i128)pr[u];
}

// a segment's pass in the grid mode (k_mgs_step_grid, k_mgs_fused)
struct MPass {
  i64 hs;
  int s8, sA;
  int qv, qw, nr;     // resident basis rows, resident w rows, rows
  bool w0s;           // line 5 left w of the resident rows in shared memory
  i64 *wg, *ws;       // w in global memory (segment) and in shared memory
  const int *vps, *vis;  // resident v_{i-1}, v_i (shared memory)
};

// resident rows [0, qv): w, v_{i-1} and v_i in shared memory (at pass 0 w
// from global memory unless line 5 left it in shared memory; stored into
// shared memory); each thread the rows q = threadIdx.x (mod IGM_MGS_GBS)
template <int MODE, bool HS32>
__device__ __forceinline__ void pass_res(const MPass &P, i128 &part, unsigned &evA,
                                         unsigned &evB) {
  for (int q0 = threadIdx.x; q0 < P.qv; q0 += IGM_RPT * IGM_MGS_GBS) {
    i64 wv[IGM_RPT];
    int pv[IGM_RPT], qq[IGM_RPT];
#pragma unroll
    for (int u = 0; u < IGM_RPT; ++u) {
      const int q = q0 + u * IGM_MGS_GBS;
      const bool ok = q < P.qv;
      wv[u] = !ok ? 0 : (MODE == 0 && !P.w0s) ? P.wg[q] : P.ws[q];
      pv[u] = (MODE > 0 && ok) ? P.vps[q] : 0;
      qq[u] = (MODE < 2 && ok) ? P.vis[q] : 0;
    }
    rows_pass<MODE, HS32>(wv, pv, qq, P.hs, P.s8, P.sA, part, evA, evB);
#pragma unroll
    for (int u = 0; u < IGM_RPT; ++u) {
      const int q = q0 + u * IGM_MGS_GBS;
      if (q < P.qv) P.ws[q] = wv[u];
    }
  }
}

// further rows [qv, nr): the basis from global memory (VT int: the int32
// copy, IGM_RPT rows in flight a thread; int64: half as many), w in shared
// memory below qw, else in global memory
template <int MODE, bool HS32, typename VT>
__device__ __forceinline__ void pass_glob(const MPass &P, const VT *vp, const VT *vi, i128 &part,
                                          unsigned &evA, unsigned &evB) {
  constexpr int R = sizeof(VT) == 4 ? IGM_RPT : IGM_RPT / 2;
  for (int q0 = P.qv + threadIdx.x; q0 < P.nr; q0 += R * IGM_MGS_GBS) {
    i64 wv[R];
    VT pv[R], qq[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int q = q0 + u * IGM_MGS_GBS;
      const bool ok = q < P.nr;
      wv[u] = !ok ? 0 : ((MODE > 0 || P.w0s) && q < P.qw) ? P.ws[q] : P.wg[q];
      pv[u] = (MODE > 0 && ok) ? vp[q] : 0;
      qq[u] = (MODE < 2 && ok) ? vi[q] : 0;
    }
    rows_pass<MODE, HS32>(wv, pv, qq, P.hs, P.s8, P.sA, part, evA, evB);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int q = q0 + u * IGM_MGS_GBS;
      if (q >= P.nr) continue;
      if (q < P.qw) P.ws[q] = wv[u];
      else if (MODE > 0) P.wg[q] = wv[u];
    }
  }
}

template <int MODE, bool HS32>
__device__ __forceinline__ void pass_seg(const MPass &P, const MSegC &c, int i, int j,
                                         i128 &part, unsigned &evA, unsigned &evB) {
  pass_res<MODE, HS32>(P, part, evA, evB);
  if (P.qv < P.nr) {
    const size_t op = (size_t)(i > 0 ? i - 1 : 0) * c.n + c.row0;
    const size_t oi = (size_t)(i <= j ? i : 0) * c.n + c.row0;
    if (c.narrow) pass_glob<MODE, HS32, int>(P, c.V32 + op, c.V32 + oi, part, evA, evB);
    else pass_glob<MODE, HS32, i64>(P, c.V + op, c.V + oi, part, evA, evB);
  }
}

// Ring mode of the single-step grid kernel (rows beyond a CTA's resident
// ones, basis as int32 words): the copy engine streams tiles of
// IGM_MGS_T rows through IGM_MGS_NST stages in shared memory, w and the
// basis words in with one mbarrier per stage, w back out with bulk stores,
// so that memory traffic and row arithmetic overlap.  A stage holds w (8T
// bytes), v_{i-1} and v_i (4T + 16 bytes each: a copy starts at the 16-byte
// boundary below the tile, the misalignment kept as an offset).
#define IGM_MGS_TR 2  // rows a thread a tile
#define IGM_MGS_T (IGM_MGS_TR * IGM_MGS_GBS)
#define IGM_MGS_NST 5
#define IGM_MGS_STG (16 * IGM_MGS_T + 32)
#define IGM_MGS_RING (IGM_MGS_NST * IGM_MGS_STG)
// resident rows of a CTA in ring mode
#define IGM_MGS_WRING 3584

struct MRing {
  unsigned char *base;  // IGM_MGS_NST stages
  u64 *full;            // one mbarrier per stage
  unsigned tt;          // tiles streamed so far in this launch (all threads)
};

// the sums a streamed span adds to its pass
struct MStreamOut {
  i128 part;
  unsigned evA, evB;
};

// rows [qa, qb) of segment c (qb - qa even; w 16-byte aligned at qa) in
// pass i, IGM_MGS_TR rows a thread a tile; thread 0 issues the copies; tt0: the
// tiles streamed before in this launch (the caller adds this span's)
template <int MODE, bool HS32>
__device__ __noinline__ MStreamOut pass_stream(const MPass P, const MSegC &c, int i, int qa,
                                               int qb, unsigned char *base, u64 *full,
                                               unsigned tt0, int *s_fail, unsigned *err0) {
  constexpr int T = IGM_MGS_T, NS = IGM_MGS_NST;
  const int L = qb - qa, nt = (L + T - 1) / T;
  i128 part = 0;
  unsigned evA = 0, evB = 0;
  const size_t ep = (size_t)(i > 0 ? i - 1 : 0) * c.n + c.row0, ei = (size_t)i * c.n + c.row0;
  auto stg = [&](int t) { return base + (size_t)((tt0 + t) % NS) * IGM_MGS_STG; };
  auto bar = [&](int t) { return &full[(tt0 + t) % NS]; };
  auto par = [&](int t) { return ((tt0 + t) / NS) & 1u; };
  auto issue = [&](int t) {
    const int r0 = qa + t * T, len = min(T, qb - r0);
    unsigned char *b = stg(t);
    const int pp = (int)((ep + r0) & 3), pc = (int)((ei + r0) & 3);
    const unsigned bw = 8u * len, bp = MODE > 0 ? 4u * ((pp + len + 3) & ~3) : 0u,
                   bc = MODE < 2 ? 4u * ((pc + len + 3) & ~3) : 0u;
    mbar_expect_tx(bar(t), bw + bp + bc);
    bulk_g2s(b, c.w + r0, bw, bar(t));
    if (MODE > 0) bulk_g2s(b + 8 * T, c.V32 + (ep + r0 - pp), bp, bar(t));
    if (MODE < 2) bulk_g2s(b + 12 * T + 16, c.V32 + (ei + r0 - pc), bc, bar(t));
  };
  int ni = 0;  // tiles issued (thread 0)
  if (threadIdx.x == 0) {
    bulk_wait<0>();       // w stored by the last pass has landed before it is read again
    fence_proxy_async();  // the stages' last generic reads before their refill
    for (; ni < nt && ni < NS - 1; ++ni) issue(ni);
  }
  __syncthreads();
  int t = 0;
  for (; t < nt && !*s_fail; ++t) {
    const int r0 = qa + t * T, len = min(T, qb - r0);
    unsigned char *b = stg(t);
    const bool ok = mbar_wait(bar(t), par(t), err0, 1000000000ull);
    if (!ok) *s_fail = 1;
    if (ok) {
      i64 *ws = reinterpret_cast<i64 *>(b);
      const int *vp = reinterpret_cast<const int *>(b + 8 * T) + ((ep + r0) & 3);
      const int *vc = reinterpret_cast<const int *>(b + 12 * T + 16) + ((ei + r0) & 3);
      i64 wv[IGM_MGS_TR];
      int pv[IGM_MGS_TR], qq[IGM_MGS_TR];
#pragma unroll
      for (int u = 0; u < IGM_MGS_TR; ++u) {
        const int q = threadIdx.x + u * IGM_MGS_GBS;
        const bool in = q < len;
        wv[u] = in ? ws[q] : 0;
        pv[u] = (MODE > 0 && in) ? vp[q] : 0;
        qq[u] = (MODE < 2 && in) ? vc[q] : 0;
      }
      rows_pass<MODE, HS32>(wv, pv, qq, P.hs, P.s8, P.sA, part, evA, evB);
      if (MODE > 0) {
#pragma unroll
        for (int u = 0; u < IGM_MGS_TR; ++u) {
          const int q = threadIdx.x + u * IGM_MGS_GBS;
          if (q < len) ws[q] = wv[u];
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !*s_fail) {
      fence_proxy_async();  // the tile's generic accesses before the async ones
      if (MODE > 0) {       // pass 0 leaves w as it is
        bulk_s2g(c.w + r0, b, 8u * len);
        bulk_commit();
      }
      if (ni < nt) {  // ni = t + NS - 1 reuses the stage of tile t - 1
        bulk_wait_read<1>();
        issue(ni++);
      }
    }
  }
  // an expired wait: the tiles already issued land before anything moves on
  if (threadIdx.x == 0)
    for (; t < ni; ++t) mbar_wait(bar(t), par(t), err0, 1000000000ull);
  return MStreamOut{part, evA, evB};
}

// tiles of a streamed span [qa, qb)
__host__ __device__ __forceinline__ int stream_tiles(int qa, int qb) {
  return (qb - qa + IGM_MGS_T - 1) / IGM_MGS_T;
}

// resident basis buffers: per pass parity IGM_MGS_WMAX rows plus room for
// each cached segment's alignment (a bulk copy starts on a 16-byte boundary
// of the basis vector, up to 3 words before the segment's first row)
#define IGM_MGS_VPAD (12 * IGM_MGS_GCACHE + 8)
// layout of the dynamic shared memory for S resident rows: w (8 S bytes),
// then at a 16-byte boundary two basis buffers of IGM_MGS_VB(S) words
#define IGM_MGS_VOFF(S) (((size_t)(S) * 8 + 15) & ~(size_t)15)
#define IGM_MGS_VB(S) ((((S) + 3) & ~3) + IGM_MGS_VPAD)
#define IGM_MGS_SMEM(S) (IGM_MGS_VOFF(S) + 2 * sizeof(int) * (size_t)IGM_MGS_VB(S))
// ... in ring mode the stages follow at a 128-byte boundary
#define IGM_MGS_RINGOFF(S) ((IGM_MGS_SMEM(S) + 127) & ~(size_t)127)
#define IGM_MGS_SMEM_RING(S) (IGM_MGS_RINGOFF(S) + (size_t)IGM_MGS_RING)

// line 5 (Table 3) for the rows of segment c in the fused kernel: exact
// int128 row sums over the SELL-32 copy of Abar_0 (one term, s = 0), the
// basis vector read from L2 (other CTAs wrote it during this launch), w into
// shared memory for the resident rows and global memory for the others;
// each thread the rows q = threadIdx.x (mod IGM_MGS_GBS), the rows it owns
// in the passes
template <bool NAR>
__device__ __forceinline__ void seg_spmv(const SysDev *s, const MSegC &c, int j, int qw, i64 *ws,
                                         unsigned &ev) {
  const i64 *vj = s->V + (size_t)j * c.n;
  const int *vj32 = s->V32 + (size_t)j * c.n;
  const long long *sptr = s->sptr;
  const i64 *sval = s->sval;
  const int *scol = s->scol;
  for (int q = threadIdx.x; q < c.nrows; q += IGM_MGS_GBS) {
    const int i = c.row0 + q;
    const int sl = i >> 5;
    const long long base = sptr[sl] + (i & 31);
    const int len = (int)((sptr[sl + 1] - sptr[sl]) >> 5);
    i128 acc = 0;
    for (int k0 = 0; k0 < len; k0 += 8) {
      i64 a[8];
      int cc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = k0 + u < len;
        a[u] = ok ? __ldcs(sval + base + 32 * (k0 + u)) : 0;
        cc[u] = ok ? __ldcs(scol + base + 32 * (k0 + u)) : i;
      }
      i64 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        x[u] = !IGM_OK((unsigned)cc[u] < (unsigned)c.n, CHK_SPMV_COL) ? 0
               : NAR ? (i64)__ldcg(vj32 + cc[u]) : __ldcg(vj + cc[u]);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += (i128)mulw(a[u], x[u], ev);
    }
    ev += out64(acc);
    const i64 w = wrap(acc);
    if (q < qw) ws[q] = w;
    else c.w[q] = w;
  }
}

// spin (bounded) until every segment of system `sys` has published tag in
// mvtag; one segment per thread; false (in every thread) when the bound
// expired or a CTA has reported an expired wait
__device__ bool mvtag_wait(const BatchDev &B, int sys, unsigned tag, const unsigned *err0) {
  const int lo = B.sys_seg[sys], hi = B.sys_seg[sys + 1];
  bool ok = true;
  for (int g = lo + threadIdx.x; g < hi && ok; g += blockDim.x)
    for (int it = 0; ld_relaxed_u32(B.mvtag + g) != tag; ++it) {
      if (it > IGM_SPIN_MAX || ((it & 255) == 255 && (ld_relaxed_u32(err0) & ERR_TIMEOUT))) {
        ok = false;
        break;
      }
      if (it > 32) __nanosleep(32);
    }
  return __syncthreads_and(ok) != 0;
}

// Grid mode: every CTA owns the same rows in every pass (a balanced partition
// of all systems' rows, planned on the host).  The first B.mgs_wrows of them
// (in segments among the first IGM_MGS_GCACHE) are resident in shared
// memory: w from pass 0 to line 11, and (while every basis entry of the
// inner solve fits int32) the int32 words of v_{i-1} and v_i in two
// buffers; v_{i+1} is bulk-copied into the buffer of v_{i-1} while the
// pass's sums travel, so a pass over resident rows reads nothing from global
// memory.  Further rows keep w in global memory and read the basis from
// global memory (the next vector prefetched into L2 during the pass).
// There is no grid barrier: each CTA publishes its tagged sum of the pass
// per segment and reads those of its systems' segments, so a CTA waits only
// for the CTAs that share a system with it.  Lines 6-19 of step j (line 5
// ran before).
template <bool RING>
__global__ void __launch_bounds__(IGM_MGS_GBS, 1) k_mgs_step_grid(BatchDev B, int j) {
  constexpr int BS = IGM_MGS_GBS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = B.mgs_wrows;  // resident rows of this CTA
  i64 *sw = reinterpret_cast<i64 *>(smem);                    // w of the resident rows
  int *sv = reinterpret_cast<int *>(smem + IGM_MGS_VOFF(S));  // 2 basis buffers
  const int vb = IGM_MGS_VB(S);                               // words of one
  constexpr bool ring = RING;  // further rows of narrow segments streamed
  __shared__ MSegC s_seg[IGM_MGS_GCACHE + 1];  // + one slot for the others in turn
  __shared__ i64 s_h[IGM_MGS_GCACHE];
  __shared__ __align__(8) u64 s_vbar[2];  // bulk copies into basis buffer 0 / 1
  __shared__ __align__(8) u64 s_full[IGM_MGS_NST];  // ring stages
  __shared__ unsigned s_epoch, s_vbytes;
  __shared__ int s_fail;
  unsigned *err0 = &B.sys[0]->sc->err;
  const int g0 = B.mseg_ptr[blockIdx.x], ns = B.mseg_ptr[blockIdx.x + 1] - g0;
  // descriptors; segments beyond the cache keep their step flags (taken
  // now, before this CTA publishes anything) in mseg_act
  for (int k = threadIdx.x; k < ns; k += BS) {
    if (k < IGM_MGS_GCACHE) {
      mseg_make(B, g0 + k, j, s_seg[k]);
    } else {
      MSegC c;
      mseg_make(B, g0 + k, j, c);
      B.mseg_act[g0 + k] = c.active | (c.narrow << 1);
    }
  }
  if (threadIdx.x == 0) {
    s_epoch = ld_relaxed_u32(B.bar + 2);
    s_fail = 0;
    mbar_init(&s_vbar[0], 1);
    mbar_init(&s_vbar[1], 1);
    for (int q = 0; q < IGM_MGS_NST; ++q) mbar_init(&s_full[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned epoch = s_epoch, e16 = (epoch & 0xffffu) << 16;
  MRing R{smem + IGM_MGS_RINGOFF(S), s_full, 0u};
  // a segment's descriptor with the flags taken at the start (into c)
  auto seg_make = [&](int k, MSegC &c) {
    mseg_make(B, g0 + k, j, c);
    const int f = B.mseg_act[g0 + k];
    c.active = f & 1;
    c.narrow = f >> 1;
  };
  // the descriptor of segment k in shared memory (all threads call it in
  // step): beyond the cache, thread 0 builds it in the spare slot
  auto seg = [&](int k) -> const MSegC & {
    if (k < IGM_MGS_GCACHE) return s_seg[k];
    __syncthreads();
    if (threadIdx.x == 0) seg_make(k, s_seg[IGM_MGS_GCACHE]);
    __syncthreads();
    return s_seg[IGM_MGS_GCACHE];
  };
  // resident rows of segment k: w (res_w) and the basis (res_v: cached
  // segments while narrow)
  auto res_w = [&](const MSegC &c) { return min(max(S - c.off, 0), c.nrows); };
  auto res_v = [&](const MSegC &c, int k) {
    return (k < IGM_MGS_GCACHE && c.narrow) ? res_w(c) : 0;
  };
  // where vector i of cached segment k starts in its basis buffer: at a
  // 16-byte aligned offset, plus the vector's misalignment
  auto vbase = [&](const MSegC &c, int k, int i) -> int * {
    return sv + (size_t)(i & 1) * vb + ((c.off + 3) & ~3) + 12 * k +
           (int)(((size_t)i * c.n + c.row0) & 3);
  };
  // bulk-copy v_i of every resident segment into buffer i & 1 (thread 0,
  // after a block barrier behind the last reads of that buffer)
  auto stage = [&](int i) {
    unsigned bytes = 0;
    for (int k = 0; k < ns && k < IGM_MGS_GCACHE; ++k) {
      const MSegC &c = s_seg[k];
      const int qv = c.active ? res_v(c, k) : 0;
      if (qv == 0) continue;
      const size_t e0 = (size_t)i * c.n + c.row0;
      const int pad = (int)(e0 & 3);
      bytes += 4u * (unsigned)((pad + qv + 3) & ~3);
    }
    s_vbytes = bytes;
    if (bytes == 0) return;
    fence_proxy_async();
    mbar_expect_tx(&s_vbar[i & 1], bytes);
    for (int k = 0; k < ns && k < IGM_MGS_GCACHE; ++k) {
      const MSegC &c = s_seg[k];
      const int qv = c.active ? res_v(c, k) : 0;
      if (qv == 0) continue;
      const size_t e0 = (size_t)i * c.n + c.row0;
      const int pad = (int)(e0 & 3), words = (pad + qv + 3) & ~3;
      if (IGM_OK(vbase(c, k, i) - pad + words <= sv + (size_t)((i & 1) + 1) * vb, CHK_MGS_STAGE))
        bulk_g2s(vbase(c, k, i) - pad, c.V32 + (e0 - pad), 4u * (unsigned)words, &s_vbar[i & 1]);
    }
  };
  if (threadIdx.x == 0) stage(0);
  __syncthreads();
  const bool vst = s_vbytes != 0;  // the same for every vector
  int staged = 0;                  // the last vector copied
  for (int i = 0; i <= j + 1; ++i) {
    const unsigned tag = e16 | ((unsigned)j << 8) | (unsigned)(i + 1);
    // v_i of the resident rows is in place (v_{i-1} already was)
    if (vst && i <= j && !mbar_wait(&s_vbar[i & 1], (unsigned)(i >> 1) & 1u, err0, 1000000000ull))
      s_fail = 1;
    for (int k = 0; k < ns; ++k) {
      const MSegC &c = seg(k);
      if (!c.active) continue;
      MPass P;
      P.nr = c.nrows;
      P.qw = res_w(c);
      P.qv = res_v(c, k);
      P.w0s = false;
      // ring mode: this segment's further rows are streamed
      const bool strm = ring && c.narrow && k < IGM_MGS_GCACHE;
      // pull the global rows of v_{i+1} into L2 while this pass runs
      if (!strm && i + 1 <= j && P.qv < P.nr) {
        const size_t o = (size_t)(i + 1) * c.n + c.row0 + P.qv;
        const char *base = c.narrow ? (const char *)(c.V32 + o) : (const char *)(c.V + o);
        const size_t bytes = (size_t)(P.nr - P.qv) * (c.narrow ? sizeof(int) : sizeof(i64));
        for (size_t a = (size_t)threadIdx.x * 128; a < bytes; a += (size_t)BS * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(base + a));
      }
      P.hs = i == 0 ? 0 : (k < IGM_MGS_GCACHE ? s_h[k] : B.mseg_h[g0 + k]);
      P.wg = c.w;
      P.ws = sw + c.off;
      P.s8 = shc(c.df - c.b8);
      P.sA = i <= j ? shc(c.b7) : shc(c.b10);
      if (P.qv > 0) {
        P.vps = vbase(c, k, i > 0 ? i - 1 : 0);
        P.vis = vbase(c, k, i <= j ? i : 0);
      }
      const bool hs32 = P.hs == (i64)(int)P.hs;
      i128 part = 0;
      unsigned evA = 0, evB = 0;
      auto run = [&](auto mode_tag, auto hs_tag) {
        constexpr int MODE = decltype(mode_tag)::value;
        constexpr bool HS = decltype(hs_tag)::value;
        if (!RING || !strm) {
          pass_seg<MODE, HS>(P, c, i, j, part, evA, evB);
          return;
        }
        pass_res<MODE, HS>(P, part, evA, evB);
        // the streamed span [qa, qb): w 16-byte aligned at qa, an even
        // number of rows; the row before and the row after it (if any) go
        // the per-thread way
        int qa = P.qv;
        if (qa < P.nr && (reinterpret_cast<uintptr_t>(c.w + qa) & 15)) ++qa;
        const int qb = qa + ((P.nr - qa) & ~1);
        const size_t op = (size_t)(i > 0 ? i - 1 : 0) * c.n + c.row0;
        const size_t oi = (size_t)(i <= j ? i : 0) * c.n + c.row0;
        MPass Q = P;
        Q.nr = qa;
        pass_glob<MODE, HS, int>(Q, c.V32 + op, c.V32 + oi, part, evA, evB);
        const MStreamOut so =
            pass_stream<MODE, HS>(P, c, i, qa, qb, R.base, R.full, R.tt, &s_fail, err0);
        R.tt += stream_tiles(qa, qb);
        part += so.part;
        evA += so.evA;
        evB += so.evB;
        Q = P;
        Q.qv = qb;
        pass_glob<MODE, HS, int>(Q, c.V32 + op, c.V32 + oi, part, evA, evB);
      };
      using I0 = std::integral_constant<int, 0>;
      using I1 = std::integral_constant<int, 1>;
      using I2 = std::integral_constant<int, 2>;
      if (i == 0) run(I0{}, std::true_type{});
      else if (i <= j) {
        if (hs32) run(I1{}, std::true_type{});
        else run(I1{}, std::false_type{});
      } else {
        if (hs32) run(I2{}, std::true_type{});
        else run(I2{}, std::false_type{});
      }
      flush_ev(evB, &c.sc->ev[IGM_EV_L8]);
      flush_ev(evA, &c.sc->ev[i <= j ? IGM_EV_L7 : IGM_EV_L10]);
      part = block_sum_i128(part);
      if (threadIdx.x == 0) mslot_put(mslot(B, i & 1, g0 + k), part, tag);
    }
    // every read of pass i is behind the block barriers of the sums: v_{i+1}
    // may overwrite the buffer of v_{i-1}
    __syncthreads();
    if (vst && i + 1 <= j && !s_fail) {
      if (threadIdx.x == 0) stage(i + 1);
      staged = i + 1;
    }
    // each segment's coefficient from its system's total (tagged slots)
    for (int k = 0; k < ns && !s_fail; ++k) {
      const MSegC &c = seg(k);
      if (!c.active) continue;
      i128 tot;
      if (!mseg_total(B, c.sys, i & 1, tag, err0, tot)) {
        if (threadIdx.x == 0) s_fail = 1;
        __syncthreads();
        break;
      }
      if (threadIdx.x == 0) {
        const i64 h = mseg_coef(c, tot, i, j);
        if (k < IGM_MGS_GCACHE) s_h[k] = h;
        else B.mseg_h[g0 + k] = h;
      }
    }
    __syncthreads();
    if (s_fail) break;
  }
  // ring mode: the last pass's w stores have landed and are visible to the
  // plain loads below
  if (ring) {
    if (threadIdx.x == 0) {
      bulk_wait<0>();
      fence_proxy_async_global();
    }
    __syncthreads();
  }
  if (s_fail) {
    // the copy in flight lands before the CTA leaves (bounded again)
    if (vst) mbar_wait(&s_vbar[staged & 1], (unsigned)(staged >> 1) & 1u, err0, 1000000000ull);
    if (threadIdx.x == 0) atomicOr(err0, ERR_TIMEOUT);
  } else {
    // line 11 for every system whose divisor is non-zero
    for (int k = 0; k < ns; ++k) {
      const MSegC &c = seg(k);
      if (!c.active) continue;
      const i64 hn = k < IGM_MGS_GCACHE ? s_h[k] : B.mseg_h[g0 + k];
      if (shr(hn, c.b11b) == 0) continue;
      const int qw = res_w(c);
      i64 *vn = c.V + (size_t)(j + 1) * c.n + c.row0;
      int *vn32 = c.V32 + (size_t)(j + 1) * c.n + c.row0;
      const i64 *wg = c.w, *ws = sw + c.off;
      unsigned ev = 0, evr = 0;
      for (int q0 = threadIdx.x; q0 < c.nrows; q0 += IGM_RPT * BS) {
        i64 wv[IGM_RPT];
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          // (from L2: in ring mode the copy engine wrote these rows)
          wv[u] = q >= c.nrows ? 0 : q < qw ? ws[q] : __ldcg(wg + q);
        }
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          if (q >= c.nrows) continue;
          const i64 v = fx_div(wv[u], hn, c.b11a, c.b11b, c.df, ev);
          evr += (v < INT32_MIN || v > INT32_MAX);
          vn[q] = v;
          vn32[q] = (int)v;
        }
      }
      flush_ev(ev, &c.sc->ev[IGM_EV_L11]);
      // an entry outside int32: the readers of the next steps (SpMV, these
      // passes, the update) switch to the int64 copy for this inner solve
      if (__syncthreads_or(evr != 0) && threadIdx.x == 0) atomicOr(&c.sc->vwide, 1);
      flush_ev(evr, &c.sc->ev[IGM_EV_VRANGE]);
    }
    // lines 10 (store) and 12-19, one thread per system, after line 11: the
    // CTA holding the system's row 0 recorded h_{0..j,j} and has h_{j+1,j}
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += BS) {
      if (k < IGM_MGS_GCACHE) {
        if (s_seg[k].active && s_seg[k].first) givens_tail(B, s_seg[k], j, s_h[k]);
      } else {
        MSegC c;
        seg_make(k, c);
        if (c.active && c.first) givens_tail(B, c, j, B.mseg_h[g0 + k]);
      }
    }
  }
  // the last CTA to finish moves the launch epoch on (every CTA of this
  // launch read it before publishing anything)
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned done = atom_add_acq_rel_u32(B.bar + 3, 1u);
    if (done == gridDim.x - 1) {
      st_relaxed_u32(B.bar + 3, 0u);
      st_relaxed_u32(B.bar + 2, epoch + 1u);
    }
  }
}


// The fused grid-mode kernel: steps j0 .. j1-1 of the Arnoldi process, each
// with line 5 first, for systems without preconditioner and without
// correction terms; the same partition, residency and tagged pass sums as
// k_mgs_step_grid, and w of the resident rows stays in shared memory from
// line 5 to line 11.  After line 11 and lines 12-19 of step j a CTA
// publishes (j, its segments) in mvtag; before line 5 of step j + 1 it waits
// for every segment of its systems, so v_{j+1} is complete.  A system held
// by one CTA alone uses the CTA's pass sums directly.
__global__ void __launch_bounds__(IGM_MGS_GBS, 1) k_mgs_fused(BatchDev B, int j0, int j1) {
  constexpr int BS = IGM_MGS_GBS;
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = B.mgs_wrows;  // resident rows of this CTA
  i64 *sw = reinterpret_cast<i64 *>(smem);                    // w of the resident rows
  int *sv = reinterpret_cast<int *>(smem + IGM_MGS_VOFF(S));  // 2 basis buffers
  const int vb = IGM_MGS_VB(S);                               // words of one
  __shared__ MSegC s_seg[IGM_MGS_GCACHE + 1];  // + one slot for the others in turn
  __shared__ i64 s_h[IGM_MGS_GCACHE];
  __shared__ i128 s_tot[IGM_MGS_GCACHE];  // pass totals of systems held by this CTA alone
  __shared__ __align__(8) u64 s_vbar[2];  // bulk copies into basis buffer 0 / 1
  __shared__ unsigned s_vn[2];            // copies issued into each buffer
  __shared__ unsigned s_epoch;
  __shared__ int s_fail;
  unsigned *err0 = &B.sys[0]->sc->err;
  const int g0 = B.mseg_ptr[blockIdx.x], ns = B.mseg_ptr[blockIdx.x + 1] - g0;
  // descriptors; segments beyond the cache keep their step flags (taken
  // now, before this CTA publishes anything) in mseg_act
  for (int k = threadIdx.x; k < ns; k += BS) {
    if (k < IGM_MGS_GCACHE) {
      mseg_make(B, g0 + k, j0, s_seg[k]);
    } else {
      MSegC c;
      mseg_make(B, g0 + k, j0, c);
      B.mseg_act[g0 + k] = c.active | (c.narrow << 1);
    }
  }
  if (threadIdx.x == 0) {
    s_epoch = ld_relaxed_u32(B.bar + 2);
    s_fail = 0;
    s_vn[0] = s_vn[1] = 0;
    mbar_init(&s_vbar[0], 1);
    mbar_init(&s_vbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned e16 = (s_epoch & 0xffffu) << 16;
  int j = j0;
  // a segment's descriptor with the flags of the current step (into c)
  auto seg_make = [&](int k, MSegC &c) {
    mseg_make(B, g0 + k, j, c);
    const int f = B.mseg_act[g0 + k];
    c.active = f & 1;
    c.narrow = f >> 1;
  };
  // the descriptor of segment k in shared memory (all threads call it in
  // step): beyond the cache, thread 0 builds it in the spare slot
  auto seg = [&](int k) -> const MSegC & {
    if (k < IGM_MGS_GCACHE) return s_seg[k];
    __syncthreads();
    if (threadIdx.x == 0) seg_make(k, s_seg[IGM_MGS_GCACHE]);
    __syncthreads();
    return s_seg[IGM_MGS_GCACHE];
  };
  // a cached segment whose system no other CTA holds
  auto alone = [&](const MSegC &c, int k) {
    return k < IGM_MGS_GCACHE && B.sys_seg[c.sys + 1] - B.sys_seg[c.sys] == 1;
  };
  // resident rows of segment k: w (res_w) and the basis (res_v: cached
  // segments while narrow)
  auto res_w = [&](const MSegC &c) { return min(max(S - c.off, 0), c.nrows); };
  auto res_v = [&](const MSegC &c, int k) {
    return (k < IGM_MGS_GCACHE && c.narrow) ? res_w(c) : 0;
  };
  // where vector i of cached segment k starts in its basis buffer: at a
  // 16-byte aligned offset, plus the vector's misalignment
  auto vbase = [&](const MSegC &c, int k, int i) -> int * {
    return sv + (size_t)(i & 1) * vb + ((c.off + 3) & ~3) + 12 * k +
           (int)(((size_t)i * c.n + c.row0) & 3);
  };
  // thread 0: bulk-copy v_i of every resident segment into buffer i & 1
  // (after a block barrier behind the last reads of that buffer)
  auto stage = [&](int i) {
    unsigned bytes = 0;
    for (int k = 0; k < ns && k < IGM_MGS_GCACHE; ++k) {
      const MSegC &c = s_seg[k];
      const int qv = c.active ? res_v(c, k) : 0;
      if (qv == 0) continue;
      const int pad = (int)(((size_t)i * c.n + c.row0) & 3);
      bytes += 4u * (unsigned)((pad + qv + 3) & ~3);
    }
    if (bytes == 0) return;
    fence_proxy_async();
    mbar_expect_tx(&s_vbar[i & 1], bytes);
    for (int k = 0; k < ns && k < IGM_MGS_GCACHE; ++k) {
      const MSegC &c = s_seg[k];
      const int qv = c.active ? res_v(c, k) : 0;
      if (qv == 0) continue;
      const size_t e0 = (size_t)i * c.n + c.row0;
      const int pad = (int)(e0 & 3), words = (pad + qv + 3) & ~3;
      if (IGM_OK(vbase(c, k, i) - pad + words <= sv + (size_t)((i & 1) + 1) * vb, CHK_MGS_STAGE))
        bulk_g2s(vbase(c, k, i) - pad, c.V32 + (e0 - pad), 4u * (unsigned)words, &s_vbar[i & 1]);
    }
    s_vn[i & 1] += 1;
  };
  // wait for the last copy into buffer b (an expired wait fails the launch)
  auto vwait = [&](int b) {
    const unsigned nb = s_vn[b];
    if (nb > 0 && !mbar_wait(&s_vbar[b], (nb - 1) & 1u, err0, 1000000000ull)) s_fail = 1;
  };
  for (; j < j1 && !s_fail; ++j) {
    {
      if (j > j0) {
        // v_j of every active system: each of its segments published step j - 1
        for (int k = 0; k < ns && !s_fail; ++k) {
          const MSegC &c = seg(k);
          if (!c.active || alone(c, k)) continue;
          if (!mvtag_wait(B, c.sys, e16 | ((unsigned)(j - 1) << 8) | 0xffu, err0)) {
            if (threadIdx.x == 0) s_fail = 1;
            __syncthreads();
          }
        }
        __threadfence();
        __syncthreads();
        if (s_fail) break;
        // the flags of step j (a breakdown or the end of a system's steps
        // at step j - 1, a basis entry outside int32 from line 11)
        for (int k = threadIdx.x; k < ns; k += BS) {
          MSegC c;
          if (k < IGM_MGS_GCACHE) c = s_seg[k];
          else seg_make(k, c);
          const SysDev *s = B.sys[c.sys];
          const int act = c.active && m_step(s, j);
          const int nar = c.narrow && s->sc->vwide == 0;
          if (k < IGM_MGS_GCACHE) {
            s_seg[k].active = act;
            s_seg[k].narrow = nar;
          } else {
            B.mseg_act[g0 + k] = act | (nar << 1);
          }
        }
        __syncthreads();
      }
      // v_0 for pass 0 travels while line 5 runs
      if (threadIdx.x == 0) stage(0);
      // line 5
      for (int k = 0; k < ns; ++k) {
        const MSegC &c = seg(k);
        if (!c.active) continue;
        const SysDev *s = B.sys[c.sys];
        unsigned ev = 0;
        if (c.narrow) seg_spmv<true>(s, c, j, res_w(c), sw + c.off, ev);
        else seg_spmv<false>(s, c, j, res_w(c), sw + c.off, ev);
        flush_ev(ev, &c.sc->ev[IGM_EV_L5]);
      }
      __syncthreads();
    }
    for (int i = 0; i <= j + 1; ++i) {
      const unsigned tag = e16 | ((unsigned)j << 8) | (unsigned)(i + 1);
      // v_i of the resident rows is in place (v_{i-1} already was)
      if (i <= j) vwait(i & 1);
      for (int k = 0; k < ns; ++k) {
        const MSegC &c = seg(k);
        if (!c.active) continue;
        MPass P;
        P.nr = c.nrows;
        P.qw = res_w(c);
        P.qv = res_v(c, k);
        P.w0s = true;
        // pull the global rows of v_{i+1} into L2 while this pass runs
        if (i + 1 <= j && P.qv < P.nr) {
          const size_t o = (size_t)(i + 1) * c.n + c.row0 + P.qv;
          const char *base = c.narrow ? (const char *)(c.V32 + o) : (const char *)(c.V + o);
          const size_t bytes = (size_t)(P.nr - P.qv) * (c.narrow ? sizeof(int) : sizeof(i64));
          for (size_t a = (size_t)threadIdx.x * 128; a < bytes; a += (size_t)BS * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + a));
        }
        P.hs = i == 0 ? 0 : (k < IGM_MGS_GCACHE ? s_h[k] : B.mseg_h[g0 + k]);
        P.wg = c.w;
        P.ws = sw + c.off;
        P.s8 = shc(c.df - c.b8);
        P.sA = i <= j ? shc(c.b7) : shc(c.b10);
        if (P.qv > 0) {
          P.vps = vbase(c, k, i > 0 ? i - 1 : 0);
          P.vis = vbase(c, k, i <= j ? i : 0);
        }
        const bool hs32 = P.hs == (i64)(int)P.hs;
        i128 part = 0;
        unsigned evA = 0, evB = 0;
        if (i == 0) pass_seg<0, true>(P, c, i, j, part, evA, evB);
        else if (i <= j) {
          if (hs32) pass_seg<1, true>(P, c, i, j, part, evA, evB);
          else pass_seg<1, false>(P, c, i, j, part, evA, evB);
        } else {
          if (hs32) pass_seg<2, true>(P, c, i, j, part, evA, evB);
          else pass_seg<2, false>(P, c, i, j, part, evA, evB);
        }
        flush_ev(evB, &c.sc->ev[IGM_EV_L8]);
        flush_ev(evA, &c.sc->ev[i <= j ? IGM_EV_L7 : IGM_EV_L10]);
        part = block_sum_i128(part);
        if (threadIdx.x == 0) {
          if (alone(c, k)) s_tot[k] = part;
          else mslot_put(mslot(B, i & 1, g0 + k), part, tag);
        }
      }
      // every read of pass i is behind the block barriers of the sums: v_{i+1}
      // may overwrite the buffer of v_{i-1}
      __syncthreads();
      if (i + 1 <= j && !s_fail && threadIdx.x == 0) stage(i + 1);
      // each segment's coefficient from its system's total
      for (int k = 0; k < ns && !s_fail; ++k) {
        const MSegC &c = seg(k);
        if (!c.active) continue;
        i128 tot = 0;
        if (alone(c, k)) {
          tot = s_tot[k];
        } else if (!mseg_total(B, c.sys, i & 1, tag, err0, tot)) {
          if (threadIdx.x == 0) s_fail = 1;
          __syncthreads();
          break;
        }
        if (threadIdx.x == 0) {
          const i64 h = mseg_coef(c, tot, i, j);
          if (k < IGM_MGS_GCACHE) s_h[k] = h;
          else B.mseg_h[g0 + k] = h;
        }
      }
      __syncthreads();
      if (s_fail) break;
    }
    if (s_fail) break;
    // line 11 for every system whose divisor is non-zero
    for (int k = 0; k < ns; ++k) {
      const MSegC &c = seg(k);
      if (!c.active) continue;
      const i64 hn = k < IGM_MGS_GCACHE ? s_h[k] : B.mseg_h[g0 + k];
      if (shr(hn, c.b11b) == 0) continue;
      const int qw = res_w(c);
      i64 *vn = c.V + (size_t)(j + 1) * c.n + c.row0;
      int *vn32 = c.V32 + (size_t)(j + 1) * c.n + c.row0;
      const i64 *wg = c.w, *ws = sw + c.off;
      unsigned ev = 0, evr = 0;
      for (int q0 = threadIdx.x; q0 < c.nrows; q0 += IGM_RPT * BS) {
        i64 wv[IGM_RPT];
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          wv[u] = q >= c.nrows ? 0 : q < qw ? ws[q] : wg[q];
        }
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          if (q >= c.nrows) continue;
          const i64 v = fx_div(wv[u], hn, c.b11a, c.b11b, c.df, ev);
          evr += (v < INT32_MIN || v > INT32_MAX);
          vn[q] = v;
          vn32[q] = (int)v;
        }
      }
      flush_ev(ev, &c.sc->ev[IGM_EV_L11]);
      // an entry outside int32: the readers of the next steps (SpMV, these
      // passes, the update) switch to the int64 copy for this inner solve
      if (__syncthreads_or(evr != 0) && threadIdx.x == 0) atomicOr(&c.sc->vwide, 1);
      flush_ev(evr, &c.sc->ev[IGM_EV_VRANGE]);
    }
    // this CTA's basis rows, written through the generic proxy, are read by
    // its later bulk copies
    fence_proxy_async_global();
    // lines 10 (store) and 12-19, one thread per system, after line 11: the
    // CTA holding the system's row 0 recorded h_{0..j,j} and has h_{j+1,j}
    __syncthreads();
    for (int k = threadIdx.x; k < ns; k += BS) {
      if (k < IGM_MGS_GCACHE) {
        if (s_seg[k].active && s_seg[k].first) givens_tail(B, s_seg[k], j, s_h[k]);
      } else {
        MSegC c;
        seg_make(k, c);
        if (c.active && c.first) givens_tail(B, c, j, B.mseg_h[g0 + k]);
      }
    }
    {
      // publish step j: the CTA's basis rows, flags and (first CTA) lines
      // 12-19 before the tags
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        for (int k = 0; k < ns; ++k) {
          const bool act = k < IGM_MGS_GCACHE ? s_seg[k].active : (B.mseg_act[g0 + k] & 1);
          if (act) st_relaxed_u32(B.mvtag + g0 + k, e16 | ((unsigned)j << 8) | 0xffu);
        }
      }
      __syncthreads();
    }
  }
  if (s_fail) {
    // the copies in flight land before the CTA leaves (bounded again)
    vwait(0);
    vwait(1);
    if (threadIdx.x == 0) atomicOr(err0, ERR_TIMEOUT);
  }
  // the last CTA to finish moves the launch epoch on (every CTA of this
  // launch read it before publishing anything)
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned done = atom_add_acq_rel_u32(B.bar + 3, 1u);
    if (done == gridDim.x - 1) {
      st_relaxed_u32(B.bar + 3, 0u);
      st_relaxed_u32(B.bar + 2, s_epoch + 1u);
    }
  }
}


// ---------------------------------------------------------------------------
// The same step for the FP64 comparison solver: per-CTA partial sums per
// system, summed by every CTA in CTA order after the barrier, so the result
// is deterministic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double *cpart_at(const BatchDev &B, int slot, int cta, int sys) {
  return B.cpart + ((size_t)slot * B.maxg + cta) * B.nsys + sys;
}

__device__ __forceinline__ double cpart_sum(const BatchDev &B, int slot, int sys) {
  double t = 0.0;
  for (int c = 0; c < gridDim.x; ++c) t = __dadd_rn(t, __ldcg(cpart_at(B, slot, c, sys)));
  return t;
}

__global__ void __launch_bounds__(IGM_MGS_BLOCK, 1) f_mgs_step(BatchDev B, int j) {
  const int G = gridDim.x;
  unsigned *err0 = &B.sys[0]->sc->err;
  __shared__ double s_part;
  for (int i = 0; i <= j + 1; ++i) {
    const int slot = i % 3;
    // this CTA's partials of every system start at zero
    for (int s = threadIdx.x; s < B.nsys; s += blockDim.x) *cpart_at(B, slot, blockIdx.x, s) = 0.0;
    __syncthreads();
    for (int t = blockIdx.x; t < B.nstiles; t += G) {
      Tile tl = B.stiles[t];
      const SysDev *s = B.sys[tl.sys];
      if (!m_step(s, j)) continue;
      const int n = s->n;
      const double *V = reinterpret_cast<const double *>(s->V);
      double *w = reinterpret_cast<double *>(s->w);
      if (threadIdx.x == 0) s_part = i > 0 ? cpart_sum(B, (i - 1) % 3, tl.sys) : 0.0;
      __syncthreads();
      double h = s_part;
      const double *vp = V + (size_t)(i > 0 ? i - 1 : 0) * n;
      const double *vi = V + (size_t)(i <= j ? i : 0) * n;
      double part = 0.0;
      for (int l = tl.row0 + threadIdx.x; l < tl.row0 + tl.nrows; l += blockDim.x) {
        double wl = w[l];
        if (i > 0) {
          wl = __dsub_rn(wl, __dmul_rn(h, vp[l]));
          w[l] = wl;
        }
        part = __dadd_rn(part, __dmul_rn(wl, i <= j ? vi[l] : wl));
      }
      part = block_sum_d(part);
      if (threadIdx.x == 0) {
        double *cp = cpart_at(B, slot, blockIdx.x, tl.sys);
        *cp = __dadd_rn(*cp, part);
      }
      __syncthreads();
    }
    if (!grid_sync(B.bar, err0)) return;
    if (blockIdx.x == 0)
      for (int sidx = threadIdx.x; sidx < B.nsys; sidx += blockDim.x) {
        const SysDev *s = B.sys[sidx];
        if (!m_step(s, j) || i > j) continue;
        reinterpret_cast<double *>(s->H)[i + j * s->ld] = cpart_sum(B, slot, sidx);
      }
  }
  const int slot = (j + 1) % 3;
  for (int t = blockIdx.x; t < B.nstiles; t += G) {
    Tile tl = B.stiles[t];
    const SysDev *s = B.sys[tl.sys];
    if (!m_step(s, j)) continue;
    __syncthreads();
    if (threadIdx.x == 0) s_part = __dsqrt_rn(cpart_sum(B, slot, tl.sys));
    __syncthreads();
    double hn = s_part;
    if (hn == 0.0) continue;
    double *vn = reinterpret_cast<double *>(s->V) + (size_t)(j + 1) * s->n;
    const double *w = reinterpret_cast<const double *>(s->w);
    for (int l = tl.row0 + threadIdx.x; l < tl.row0 + tl.nrows; l += blockDim.x)
      vn[l] = __ddiv_rn(w[l], hn);
  }
}

// h_{j+1,j} and the Givens rotation of column j (FP64), one thread per system
__global__ void f_givens_step(BatchDev B, int j, int G) {
  int si = blockIdx.x * blockDim.x + threadIdx.x;
  if (si >= B.nsys) return;
  const SysDev *s = B.sys[si];
  SysScal *sc = s->sc;
  if (!m_step(s, j)) return;
  const int ld = s->ld, slot = (j + 1) % 3;
  double t2 = 0.0;
  for (int c = 0; c < G; ++c) t2 = __dadd_rn(t2, cpart_at(B, slot, c, si)[0]);
  double hn = __dsqrt_rn(t2);
  double *H = reinterpret_cast<double *>(s->H);
  double *cs = reinterpret_cast<double *>(s->cs), *sn = reinterpret_cast<double *>(s->sn);
  double *g = reinterpret_cast<double *>(s->g);
  H[j + 1 + j * ld] = hn;
  for (int i = 0; i < j; ++i) {
    double x1 = H[i + j * ld], x2 = H[i + 1 + j * ld];
    H[i + j * ld] = __dadd_rn(__dmul_rn(cs[i], x1), __dmul_rn(sn[i], x2));
    H[i + 1 + j * ld] = __dadd_rn(__dmul_rn(-sn[i], x1), __dmul_rn(cs[i], x2));
  }
  double hjj = H[j + j * ld], hj1 = H[j + 1 + j * ld];
  double t = __dsqrt_rn(__dadd_rn(__dmul_rn(hjj, hjj), __dmul_rn(hj1, hj1)));
  if (t == 0.0) {
    sc->early = 1;
    return;
  }
  double c = __ddiv_rn(hjj, t), sv = __ddiv_rn(hj1, t);
  cs[j] = c;
  sn[j] = sv;
  double gj = g[j];
  g[j + 1] = __dmul_rn(-sv, gj);
  g[j] = __dmul_rn(c, gj);
  H[j + j * ld] = t;
  H[j + 1 + j * ld] = 0.0;
  sc->jeff = j + 1;
  if (hn == 0.0) sc->early = 1;
}

static int g_mgs_blocks_per_sm = -1, g_num_sms = 0;
static std::once_flag g_mgs_once;

int persistent_grid(int ntiles) {
  std::call_once(g_mgs_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    // co-resident CTAs with the most dynamic shared memory a plan may give
    // the integer step (IGM_MGS_WMAX resident rows)
    cudaFuncSetAttribute(k_mgs_step_grid<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)IGM_MGS_SMEM(IGM_MGS_WMAX));
    cudaFuncSetAttribute(k_mgs_step_grid<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)IGM_MGS_SMEM_RING(IGM_MGS_WRING));
    cudaFuncSetAttribute(k_mgs_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)IGM_MGS_SMEM(IGM_MGS_WMAX));
    int a = 0, a2 = 0, b = 0;
    int a3 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mgs_step_grid<false>, IGM_MGS_GBS,
                                                      IGM_MGS_SMEM(IGM_MGS_WMAX)) != cudaSuccess)
      a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a3, k_mgs_step_grid<true>, IGM_MGS_GBS,
                                                      IGM_MGS_SMEM_RING(IGM_MGS_WRING)) !=
        cudaSuccess)
      a3 = 1;
    a = a < a3 ? a : a3;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a2, k_mgs_fused, IGM_MGS_GBS,
                                                      IGM_MGS_SMEM(IGM_MGS_WMAX)) != cudaSuccess)
      a2 = 1;
    a = a < a2 ? a : a2;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f_mgs_step, IGM_MGS_BLOCK, 0) !=
        cudaSuccess)
      b = 1;
    cudaGetLastError();
    g_mgs_blocks_per_sm = a < b ? a : b;
    if (g_mgs_blocks_per_sm < 1) g_mgs_blocks_per_sm = 1;
  });
  int G = g_num_sms * g_mgs_blocks_per_sm;
  if (G > ntiles) G = ntiles;
  return G < 1 ? 1 : G;
}

void launch_fp64_mgs_step(const BatchDev &B, int j, cudaStream_t st) {
  int G = persistent_grid(B.nstiles);
  BatchDev b = B;
  void *args[] = {&b, &j};
  note_launch(cudaLaunchCooperativeKernel((const void *)f_mgs_step, dim3(G), dim3(IGM_MGS_BLOCK),
                                          args, 0, st));
  f_givens_step<<<(B.nsys + 127) / 128, 128, 0, st>>>(B, j, G);
}

// The Arnoldi step's partition: CTA c takes the contiguous global rows
// [b_c, b_{c+1}) of the batch (systems in order), b_c = N c / G (equal
// shares); with snap > 0 a boundary inside a system moves to that system's
// nearer end when it is within snap % of a share, so that more systems lie
// in one CTA whole (no exchange of pass sums) at the price of balance.
// ring_ok: the single-step kernel may stream the rows beyond the resident
// ones (ring mode: fewer resident rows, room for the stages); chosen when
// some CTA has more rows than fit resident without it.
void mgs_plan(const std::vector<int> &n, int max_ctas, int wmax, int snap, bool ring_ok, int &G,
              std::vector<int> &ptr, std::vector<Tile> &seg, int &wrows, int &rows, int &ring,
              std::vector<int> &sys_seg) {
  // rows a CTA may keep resident in shared memory: 0 automatic, -1 none,
  // k > 0 at most k (never above what the kernel reserves)
  const int cap = wmax == 0 ? IGM_MGS_WMAX : wmax < 0 ? 0 : std::min(wmax, IGM_MGS_WMAX);
  long long N = 0;
  for (int v : n) N += v;
  long long g = (N + IGM_MGS_BLOCK - 1) / IGM_MGS_BLOCK;
  if (g > max_ctas) g = max_ctas;
  G = (int)(g < 1 ? 1 : g);
  ptr.assign(G + 1, 0);
  seg.clear();
  // CTA boundaries (snapped to system ends where close enough)
  std::vector<long long> bnd(G + 1);
  {
    std::vector<long long> first(n.size() + 1, 0);
    for (size_t k = 0; k < n.size(); ++k) first[k + 1] = first[k] + n[k];
    const long long share = (N + G - 1) / G, tol = share * (long long)std::max(snap, 0) / 100;
    size_t k = 0;
    for (int c = 0; c <= G; ++c) {
      long long b = N * c / G;
      if (snap > 0 && c > 0 && c < G) {
        while (first[k + 1] <= b) ++k;  // b inside system k: [first[k], first[k+1])
        const long long dlo = b - first[k], dhi = first[k + 1] - b;
        if (dlo > 0 && dlo <= tol && dlo <= dhi) b = first[k];
        else if (dlo > 0 && dhi <= tol) b = first[k + 1];
      }
      bnd[c] = c > 0 ? std::max(b, bnd[c - 1]) : 0;
    }
    bnd[G] = N;
  }
  int s = 0, maxrows = 0;
  long long base = 0;  // first global row of system s
  for (int c = 0; c < G; ++c) {
    const long long lo = bnd[c], hi = bnd[c + 1];
    ptr[c] = (int)seg.size();
    int off = 0;
    for (long long r = lo; r < hi;) {
      while (r >= base + n[s]) base += n[s++];
      const long long e = std::min(hi, base + n[s]);
      seg.push_back(Tile{s, (int)(r - base), (int)(e - r), off});
      off += (int)(e - r);
      r = e;
    }
    maxrows = std::max(maxrows, off);
  }
  ptr[G] = (int)seg.size();
  wrows = std::min(maxrows, cap);
  rows = maxrows;
  ring = ring_ok && maxrows > wrows;
  if (ring) wrows = std::min(wrows, IGM_MGS_WRING);
  // segments run in system order: system s owns [sys_seg[s], sys_seg[s+1])
  sys_seg.assign(n.size() + 1, (int)seg.size());
  for (int g = (int)seg.size() - 1; g >= 0; --g) sys_seg[seg[g].sys] = g;
}

void launch_mgs_step(const BatchDev &B, int j, cudaStream_t st) {
  if (mgs_one_cta(B, B.nsys)) {
    static std::once_flag one_attr;  // basis buffers + w: beyond 48 KB
    std::call_once(one_attr, [] {
      cudaFuncSetAttribute(k_mgs_one, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((IGM_ONE_NBUF + 1) * IGM_MGS_BLOCK * sizeof(i64)));
    });
    k_mgs_one<<<1, IGM_MGS_ONE_BLOCK,
                (size_t)(IGM_ONE_NBUF * IGM_MGS_BLOCK + B.mgs_wrows) * sizeof(i64), st>>>(B, j);
    return;
  }
  persistent_grid(1);  // sets the kernel's shared-memory attribute once
  int G = B.mgs_g;
  BatchDev b = B;
  void *args[] = {&b, &j};
  const size_t sm = B.mgs_ring ? IGM_MGS_SMEM_RING(B.mgs_wrows) : IGM_MGS_SMEM(B.mgs_wrows);
  // cooperative: every CTA resident at once (CTAs wait for each other's sums)
  const void *k = B.mgs_ring ? (const void *)k_mgs_step_grid<true>
                             : (const void *)k_mgs_step_grid<false>;
  note_launch(cudaLaunchCooperativeKernel(k, dim3(G), dim3(IGM_MGS_GBS), args, sm, st));
}

void launch_mgs_fused(const BatchDev &B, int j0, int j1, cudaStream_t st) {
  persistent_grid(1);
  int G = B.mgs_g;
  BatchDev b = B;
  void *args[] = {&b, &j0, &j1};
  note_launch(cudaLaunchCooperativeKernel((const void *)k_mgs_fused, dim3(G),
                                          dim3(IGM_MGS_GBS), args, IGM_MGS_SMEM(B.mgs_wrows),
                                          st));
}

IGM_CHECKS_READER(checks_read_mgs)

}  // namespace igm
