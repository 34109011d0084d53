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

#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

// one CTA per SM: few grid-barrier arrivals, many rows in flight per CTA
#define IGM_MGS_BLOCK 1024
// threads of the one-CTA mode (at most IGM_MGS_BLOCK rows: IGM_RPT per thread)
#define IGM_MGS_ONE_BLOCK 256

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

// a pass's int128 sum over one segment: 2 slots (pass parity) x segments
__device__ __forceinline__ u64 *mpart_at(const BatchDev &B, int i, int g) {
  return B.mpart + 2 * ((size_t)(i & 1) * B.nseg + g);
}

// an int128 {lo, hi} pair (16-byte aligned) read from L2
__device__ __forceinline__ i128 acc_load(const u64 *a) {
  const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(a));
  return (i128)(((u128)v.y << 64) | (u128)v.x);
}

__device__ __forceinline__ bool m_step(const SysDev *s, int j) {
  return s->sc->cyc != 0 && s->sc->early == 0 && j < s->p.m;
}

#define IGM_RPT 4           // rows in flight per thread
#define IGM_MSEG_CACHE 64   // segment descriptors a CTA keeps in shared memory
#define IGM_MGS_WMAX 20480  // rows of w a CTA may keep in shared memory (160 KB)

// the step kernel's one-CTA mode: one CTA holding at most IGM_MGS_BLOCK rows
// in all, each system one segment of it (ns segments), every segment
// descriptor cached in shared memory
__host__ __device__ __forceinline__ bool mgs_one_cta(const BatchDev &B, int ns) {
  return B.mgs_g == 1 && B.mgs_wrows > 0 && B.mgs_wrows <= IGM_MGS_BLOCK && ns <= IGM_MSEG_CACHE;
}

// a segment as the step kernel sees it: its system's arrays and shifts
struct MSegC {
  i64 *V;  // basis of the system
  i64 *w;        // the segment's first row of w
  i64 *H;
  SysScal *sc;
  int n, row0, nrows, off, sys, ld;
  int df, b7, b8, b10, b11a, b11b;
  int first;   // holds row 0 of its system: records h_{i,j} and its events
  int active;  // the system takes this step
};

__device__ __forceinline__ void mseg_make(const BatchDev &B, int g, int j, MSegC &c) {
  const Tile t = B.mseg[g];
  const SysDev *s = B.sys[t.sys];
  const SysParams &P = s->p;
  c.V = s->V;
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

// the exact total of pass i over every segment of c's system, summed by one
// warp from the segments' sums (valid in lane 0)
__device__ __forceinline__ i128 mseg_sum(const BatchDev &B, const MSegC &c, int i) {
  const int lane = threadIdx.x & 31;
  const int lo = B.sys_seg[c.sys], hi = B.sys_seg[c.sys + 1];
  i128 t = 0;
  // up to 256 segments per round, all loads in flight together
  for (int g0 = lo + lane; g0 < hi; g0 += 32 * 8) {
    i128 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int g = g0 + 32 * u;
      v[u] = g < hi ? acc_load(mpart_at(B, i, g)) : (i128)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) t += v[u];
  }
  return warp_sum_i128(t);
}

// Every CTA owns the same rows in every pass (a balanced partition of all
// systems' rows, planned on the host); when they fit, its rows of w stay in
// shared memory from pass 0 to line 11, so a pass reads only the two basis
// vectors it needs (v_i from HBM, v_{i-1} mostly from L2).
template <bool ONE>
__global__ void __launch_bounds__(ONE ? IGM_MGS_ONE_BLOCK : IGM_MGS_BLOCK, 1)
    k_mgs_step(BatchDev B, int j) {
  constexpr int BS = ONE ? IGM_MGS_ONE_BLOCK : IGM_MGS_BLOCK;  // threads
  extern __shared__ i64 sw[];  // this CTA's rows of w (B.mgs_wrows > 0)
  __shared__ MSegC s_seg[IGM_MSEG_CACHE + 1];
  __shared__ i64 s_h[IGM_MSEG_CACHE];
  __shared__ i128 s_tot[ONE ? IGM_MSEG_CACHE : 1];   // pass totals (one-CTA mode)
  __shared__ i64 s_v[ONE ? 3 : 1][ONE ? IGM_MGS_BLOCK : 1];  // v_{i-1}, v_i, v_{i+1}
  unsigned *err0 = &B.sys[0]->sc->err;
  const int g0 = B.mseg_ptr[blockIdx.x], ns = B.mseg_ptr[blockIdx.x + 1] - g0;
  const bool wsm = B.mgs_wrows > 0;
  // ONE: one CTA of IGM_MGS_ONE_BLOCK threads holds every row of every
  // system (small systems, mgs_one_cta): each system is one segment of it,
  // its pass totals stay in shared memory, a block barrier replaces the grid
  // barrier, the basis vectors are staged in shared memory (v_{i+1} copied
  // asynchronously during pass i, so no pass waits on a global load); fewer
  // threads keep the per-pass reductions short
  constexpr bool one = ONE;
  for (int k = threadIdx.x; k < ns && k < IGM_MSEG_CACHE; k += blockDim.x)
    mseg_make(B, g0 + k, j, s_seg[k]);
  __syncthreads();
  // one-CTA mode: stage v_i into s_v[i % 3] (i <= j)
  auto stage = [&](int i) {
    for (int k = 0; k < ns; ++k) {
      const MSegC &c = s_seg[k];
      if (!c.active) continue;
      const i64 *src = c.V + (size_t)i * c.n + c.row0;
      i64 *dst = &s_v[i % 3][c.off];
      for (int q = threadIdx.x; q < c.nrows; q += blockDim.x) mgs_cp_async8(dst + q, src + q);
    }
    mgs_cp_async_commit();
  };
  if (one) {
    stage(0);
    mgs_cp_async_wait_all();
    __syncthreads();
  }
  for (int i = 0; i <= j + 1; ++i) {
    if (one && i + 1 <= j) stage(i + 1);
    // grid mode: pull this CTA's rows of v_{i+1} into L2 while pass i runs
    // and waits at its barrier, so pass i+1 streams them from L2
    if (!one && i + 1 <= j)
      for (int k = 0; k < ns && k < IGM_MSEG_CACHE; ++k) {
        const MSegC &c = s_seg[k];
        if (!c.active) continue;
        const char *base = (const char *)(c.V + (size_t)(i + 1) * c.n + c.row0);
        const size_t bytes = (size_t)c.nrows * sizeof(i64);
        for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(base + o));
      }
    for (int k = 0; k < ns; ++k) {
      if (k >= IGM_MSEG_CACHE) {  // descriptor beyond the cache: one spare slot
        __syncthreads();
        if (threadIdx.x == 0) mseg_make(B, g0 + k, j, s_seg[IGM_MSEG_CACHE]);
        __syncthreads();
      }
      const MSegC &c = s_seg[k < IGM_MSEG_CACHE ? k : IGM_MSEG_CACHE];
      if (!c.active) continue;
      const i64 hs = i == 0 ? 0 : (k < IGM_MSEG_CACHE ? s_h[k] : B.mseg_h[g0 + k]);
      const int nr = c.nrows;
      const i64 *vp = one ? &s_v[(i + 2) % 3][c.off]
                          : c.V + (size_t)(i > 0 ? i - 1 : 0) * c.n + c.row0;
      const i64 *vi = one ? &s_v[i % 3][c.off] : c.V + (size_t)(i <= j ? i : 0) * c.n + c.row0;
      i64 *wg = c.w, *ws = sw + c.off;
      const int s8 = shc(c.df - c.b8), s7 = shc(c.b7), s10 = shc(c.b10);
      // line 8's coefficient as a 32-bit value when it fits: the product
      // with a basis entry that fits too is one 32x32 -> 64-bit multiply,
      // exact and never out of range (same word, no event)
      const bool hs32 = hs == (i64)(int)hs;
      i128 part = 0;
      unsigned evA = 0, evB = 0;
      for (int q0 = threadIdx.x; q0 < nr; q0 += IGM_RPT * BS) {
        // all loads of the thread's rows first (memory-level parallelism)
        i64 wv[IGM_RPT], pv[IGM_RPT], qv[IGM_RPT];
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          const bool ok = q < nr;
          wv[u] = ok ? ((wsm && i > 0) ? ws[q] : wg[q]) : 0;
          pv[u] = (ok && i > 0) ? vp[q] : 0;
          qv[u] = (ok && i <= j) ? vi[q] : 0;
        }
#pragma unroll
        for (int u = 0; u < IGM_RPT; ++u) {
          const int q = q0 + u * BS;
          if (q >= nr) continue;
          i64 wl = wv[u];
          if (i > 0) {
            const i64 pr = (hs32 && pv[u] == (i64)(int)pv[u])
                               ? (i64)(int)hs * (i64)(int)pv[u]
                               : mulw(hs, pv[u], evB);
            wl = subw(wl, pr >> s8, evB);
          }
          if (wsm) ws[q] = wl;
          else if (i > 0) wg[q] = wl;
          // lines 7 / 10: a 32x32 -> 64-bit multiply when both factors fit
          // (exact, never out of range: the same word, no event)
          if (i <= j) {
            const i64 a = wl >> s7, b = qv[u];
            part += (i128)((a == (i64)(int)a && b == (i64)(int)b) ? (i64)(int)a * (i64)(int)b
                                                                  : mulw(a, b, evA));
          } else {
            const i64 a = wl >> s10;
            part += (i128)(a == (i64)(int)a ? (i64)(int)a * (i64)(int)a : mulw(a, a, evA));
          }
        }
      }
      flush_ev(evB, &c.sc->ev[IGM_EV_L8]);
      flush_ev(evA, &c.sc->ev[i <= j ? IGM_EV_L7 : IGM_EV_L10]);
      part = block_sum_i128(part);
      if (threadIdx.x == 0) {
        if (one) {
          s_tot[k] = part;
        } else {  // slot i & 1 was last read before barrier i-1
          u64 *pp = mpart_at(B, i, g0 + k);
          pp[0] = (u64)(u128)part;
          pp[1] = (u64)((u128)part >> 64);
        }
      }
    }
    if constexpr (ONE) {
      __syncthreads();
      for (int k = threadIdx.x; k < ns; k += blockDim.x)
        if (s_seg[k].active) s_h[k] = mseg_coef(s_seg[k], s_tot[k], i, j);
    } else {
      if (!grid_sync(B.bar, err0)) return;
      // one warp per segment: its system's total from all segment sums
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int k = wid; k < ns; k += BS / 32) {
        if (k < IGM_MSEG_CACHE) {
          if (!s_seg[k].active) continue;
          const i128 tot = mseg_sum(B, s_seg[k], i);
          if (lane == 0) s_h[k] = mseg_coef(s_seg[k], tot, i, j);
        } else {
          MSegC c;
          mseg_make(B, g0 + k, j, c);
          if (!c.active) continue;
          const i128 tot = mseg_sum(B, c, i);
          if (lane == 0) B.mseg_h[g0 + k] = mseg_coef(c, tot, i, j);
        }
      }
    }
    if (one) mgs_cp_async_wait_all();  // v_{i+1} is in place for pass i+1
    __syncthreads();
  }
  // line 11 for every system whose divisor is non-zero
  for (int k = 0; k < ns; ++k) {
    if (k >= IGM_MSEG_CACHE) {
      __syncthreads();
      if (threadIdx.x == 0) mseg_make(B, g0 + k, j, s_seg[IGM_MSEG_CACHE]);
      __syncthreads();
    }
    const MSegC &c = s_seg[k < IGM_MSEG_CACHE ? k : IGM_MSEG_CACHE];
    if (!c.active) continue;
    const i64 hn = k < IGM_MSEG_CACHE ? s_h[k] : B.mseg_h[g0 + k];
    if (shr(hn, c.b11b) == 0) continue;
    i64 *vn = c.V + (size_t)(j + 1) * c.n + c.row0;
    const i64 *wg = c.w, *ws = sw + c.off;
    unsigned ev = 0, evr = 0;
    for (int q0 = threadIdx.x; q0 < c.nrows; q0 += IGM_RPT * BS) {
      i64 wv[IGM_RPT];
#pragma unroll
      for (int u = 0; u < IGM_RPT; ++u) {
        const int q = q0 + u * BS;
        wv[u] = q < c.nrows ? (wsm ? ws[q] : wg[q]) : 0;
      }
#pragma unroll
      for (int u = 0; u < IGM_RPT; ++u) {
        const int q = q0 + u * BS;
        if (q >= c.nrows) continue;
        const i64 v = fx_div(wv[u], hn, c.b11a, c.b11b, c.df, ev);
        evr += (v < INT32_MIN || v > INT32_MAX);
        vn[q] = v;
      }
    }
    flush_ev(ev, &c.sc->ev[IGM_EV_L11]);
    flush_ev(evr, &c.sc->ev[IGM_EV_VRANGE]);
  }
  // lines 10 (store) and 12-19, one thread per system, after line 11: the
  // CTA holding the system's row 0 recorded h_{0..j,j} and has h_{j+1,j}
  __syncthreads();
  for (int k = threadIdx.x; k < ns; k += BS) {
    if (k < IGM_MSEG_CACHE) {
      if (s_seg[k].active && s_seg[k].first) givens_tail(B, s_seg[k], j, s_h[k]);
    } else {
      MSegC c;
      mseg_make(B, g0 + k, j, c);
      if (c.active && c.first) givens_tail(B, c, j, B.mseg_h[g0 + k]);
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

int persistent_grid(int ntiles) {
  if (g_mgs_blocks_per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    // co-resident CTAs with the most dynamic shared memory a plan may give
    // the integer step (every row of w in shared memory)
    cudaFuncSetAttribute(k_mgs_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IGM_MGS_WMAX * (int)sizeof(i64));
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mgs_step<false>, IGM_MGS_BLOCK,
                                                      IGM_MGS_WMAX * sizeof(i64)) != cudaSuccess)
      a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f_mgs_step, IGM_MGS_BLOCK, 0) !=
        cudaSuccess)
      b = 1;
    cudaGetLastError();
    g_mgs_blocks_per_sm = a < b ? a : b;
    if (g_mgs_blocks_per_sm < 1) g_mgs_blocks_per_sm = 1;
  }
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

void mgs_plan(const std::vector<int> &n, int max_ctas, int wmax, int &G, std::vector<int> &ptr,
              std::vector<Tile> &seg, int &wrows, std::vector<int> &sys_seg) {
  // rows of w a CTA may keep in shared memory: 0 automatic, -1 none, k > 0
  // at most k (never above what the kernel reserves)
  const int cap = wmax == 0 ? IGM_MGS_WMAX : wmax < 0 ? 0 : std::min(wmax, IGM_MGS_WMAX);
  long long N = 0;
  for (int v : n) N += v;
  long long g = (N + IGM_MGS_BLOCK - 1) / IGM_MGS_BLOCK;
  if (g > max_ctas) g = max_ctas;
  G = (int)(g < 1 ? 1 : g);
  ptr.assign(G + 1, 0);
  seg.clear();
  int s = 0, maxrows = 0;
  long long base = 0;  // first global row of system s
  for (int c = 0; c < G; ++c) {
    const long long lo = N * c / G, hi = N * (c + 1) / G;
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
  wrows = maxrows <= cap ? maxrows : 0;
  // segments run in system order: system s owns [sys_seg[s], sys_seg[s+1])
  sys_seg.assign(n.size() + 1, (int)seg.size());
  for (int g = (int)seg.size() - 1; g >= 0; --g) sys_seg[seg[g].sys] = g;
}

void launch_mgs_step(const BatchDev &B, int j, cudaStream_t st) {
  if (mgs_one_cta(B, B.nsys)) {
    // one CTA, no grid barrier
    k_mgs_step<true><<<1, IGM_MGS_ONE_BLOCK, (size_t)B.mgs_wrows * sizeof(i64), st>>>(B, j);
    return;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mgs_step<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         IGM_MGS_WMAX * (int)sizeof(i64));
    attr = true;
  }
  int G = B.mgs_g;
  BatchDev b = B;
  void *args[] = {&b, &j};
  note_launch(cudaLaunchCooperativeKernel((const void *)k_mgs_step<false>, dim3(G),
                                          dim3(IGM_MGS_BLOCK), args,
                                          (size_t)B.mgs_wrows * sizeof(i64), st));
}

}  // namespace igm
