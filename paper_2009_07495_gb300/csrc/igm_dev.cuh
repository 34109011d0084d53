// igm_dev.cuh -- device arithmetic of the int-GMRES kernels.
//
// Fixed-point words are int64 holding the exact value modulo 2^64 (the
// wrap of the paper's int64 hardware, Sec. VII-B).  Products and sums are
// formed exactly in __int128; an overflow event is counted wherever the
// exact value of an operation leaves [-2^63, 2^63).  Right shifts are the
// arithmetic shift (floor division by 2^beta, Sec. V-A), divisions truncate
// toward zero (Sec. V-B), square roots are floor(sqrt(.)) (Sec. V-B).
#pragma once
#include <cuda_runtime.h>

#include "../../include/igm.h"
#include "igm_internal.h"

typedef __int128 i128;
typedef unsigned __int128 u128;

namespace igm {

// ---- checked builds (-DIGM_CHECKS: build variant "checks") ----------------
// IGM_OK(cond, site) is true in normal builds (cond is not evaluated).  In a
// checked build a false cond records the first failing site in the
// translation unit's igm_chk word, which the host reads after each solve
// (the call then fails with IGM_ECUDA naming the site), and the caller skips
// the access the condition guards.
enum CheckSite : unsigned {
  CHK_BULK_G2S = 1,   // bulk copy global -> shared: 16-byte addresses and size
  CHK_BULK_S2G = 2,   // bulk copy shared -> global: the same
  CHK_SPMV_COL = 3,   // SpMV gather (line 5): column inside the system
  CHK_TRSV_RHS = 4,   // substitution gather (line 5'): right-hand side row
  CHK_MGS_STAGE = 5,  // Arnoldi basis copy inside its shared-memory buffer
};
#ifdef IGM_CHECKS
static __device__ unsigned igm_chk;
#define IGM_OK(cond, site) \
  ((cond) ? true : (atomicCAS(&::igm::igm_chk, 0u, (unsigned)(site)), false))
// host reader of this translation unit's record (0: every check passed)
#define IGM_CHECKS_READER(fn)                                  \
  unsigned fn() {                                              \
    unsigned v = 0;                                            \
    if (cudaMemcpyFromSymbol(&v, igm_chk, sizeof(v)) != cudaSuccess) v = ~0u; \
    return v;                                                  \
  }
#else
#define IGM_OK(cond, site) true
#define IGM_CHECKS_READER(fn)
#endif

__device__ __forceinline__ bool out64(i128 x) { return x != (i128)(i64)(u64)x; }
__device__ __forceinline__ i64 wrap(i128 x) { return (i64)(u64)x; }

// right shift by s bits (floor division by 2^s)
__device__ __forceinline__ i64 shr(i64 x, int s) {
  if (s <= 0) return x;
  if (s > 63) return x < 0 ? -1 : 0;
  return x >> s;
}

// wrapped product of two words; an event when the exact product leaves
// int64, i.e. when its high word is not the sign extension of the low one
__device__ __forceinline__ i64 mulw(i64 a, i64 b, unsigned &ev) {
  const i64 lo = (i64)((u64)a * (u64)b);
  const i64 hi = __mul64hi(a, b);
  ev += (hi != (lo >> 63));
  return lo;
}

// wrapped a - b; an event when the exact difference leaves int64
__device__ __forceinline__ i64 subw(i64 a, i64 b, unsigned &ev) {
  const i64 d = (i64)((u64)a - (u64)b);
  ev += (((a ^ b) & (a ^ d)) < 0);
  return d;
}

// a right-shift amount clamped to [0, 63]: x >> shc(s) is floor(x / 2^s)
// for every s >= 0 (and |x| < 2^63)
__device__ __forceinline__ int shc(int s) { return s < 0 ? 0 : (s > 63 ? 63 : s); }

__device__ __forceinline__ i64 negw(i64 a, unsigned &ev) {
  ev += (a == INT64_MIN);
  return (i64)(0ull - (u64)a);
}

// x * 2^e for e >= 0 (counted if out of range), floor(x / 2^-e) for e < 0
__device__ __forceinline__ i64 scale2(i64 x, int e, unsigned &ev) {
  if (e < 0) return shr(x, -e);
  if (e == 0) return x;
  if (e >= 64) {
    ev += (x != 0);
    return 0;
  }
  i128 p = (i128)x * (i128)((u64)1 << (e > 62 ? 62 : e));
  if (e > 62) p = p * 2;
  ev += out64(p);
  return wrap(p);
}

__device__ __forceinline__ i64 divt(i64 a, i64 b, unsigned &ev) {
  if (b == -1 && a == INT64_MIN) {
    ev += 1;
    return INT64_MIN;
  }
  return a / b;
}

// Division by a run-time invariant divisor without a divide instruction
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the unsigned N-bit method of their Sec. 4):
// for 1 <= d < 2^64 with l = ceil(log2 d) and m = floor(2^64 (2^l - d) / d)
// + 1 (which fits in 64 bits), every 0 <= n < 2^64 has
// floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, n).
__device__ __forceinline__ int ceil_log2_u64(u64 d) { return d <= 1 ? 0 : 64 - __clzll(d - 1); }

// m for the divisor d >= 1 (set-up only: a 128-bit division)
__device__ __forceinline__ u64 magic_u64(u64 d) {
  const int l = ceil_log2_u64(d);
  const u128 num = ((u128)1 << 64) * (((u128)1 << l) - (u128)d);
  return (u64)(num / (u128)d) + 1;
}

__device__ __forceinline__ u64 udiv_magic(u64 n, u64 d, u64 m) {
  const int l = ceil_log2_u64(d);
  const u64 t = __umul64hi(m, n);
  return (t + ((n - t) >> (l < 1 ? l : 1))) >> (l > 1 ? l - 1 : 0);
}

// the same with l = ceil_log2_u64(|d|) given (precomputed with m)
__device__ __forceinline__ u64 udiv_magic_l(u64 n, u64 m, int l) {
  const u64 t = __umul64hi(m, n);
  return (t + ((n - t) >> (l < 1 ? l : 1))) >> (l > 1 ? l - 1 : 0);
}

// a / d truncated toward zero for d != 0, m = magic_u64(|d|), l its shift:
// the same result and events as divt
__device__ __forceinline__ i64 divt_magic_l(i64 a, i64 d, u64 m, int l, unsigned &ev) {
  ev += (a == INT64_MIN && d == -1);
  const u64 ua = a < 0 ? 0ull - (u64)a : (u64)a;
  const u64 uq = udiv_magic_l(ua, m, l);
  return (i64)(((a < 0) != (d < 0)) ? 0ull - uq : uq);
}

// a / d truncated toward zero for d != 0, m = magic_u64(|d|): the same result
// and events as divt
__device__ __forceinline__ i64 divt_magic(i64 a, i64 d, u64 m, unsigned &ev) {
  ev += (a == INT64_MIN && d == -1);
  const u64 ua = a < 0 ? 0ull - (u64)a : (u64)a;
  const u64 ud = d < 0 ? 0ull - (u64)d : (u64)d;
  const u64 uq = udiv_magic(ua, ud, m);
  return (i64)(((a < 0) != (d < 0)) ? 0ull - uq : uq);
}

// floor(sqrt(s)) for s >= 0 (0 for s <= 0): FP64 estimate, then exact
// integer correction.
__device__ __forceinline__ i64 isqrt64(i64 s) {
  if (s <= 0) return 0;
  u64 us = (u64)s;
  u64 r = (u64)__dsqrt_rn((double)us);
  while (r * r > us) --r;
  while ((r + 1) * (r + 1) <= us) ++r;
  return (i64)r;
}

// Sec. V-B square root of a word with dfp fractional bits -> Q(df)
__device__ __forceinline__ i64 fx_sqrt(i64 t, int dfp, int df, unsigned &ev) {
  return scale2(isqrt64(t), df - dfp / 2, ev);
}

// Sec. V-B division ((t1 2^b1) / (t2 >> b2)) 2^(df-b1-b2); caller checks
// that t2 >> b2 != 0.
__device__ __forceinline__ i64 fx_div(i64 t1, i64 t2, int b1, int b2, int df,
                                      unsigned &ev) {
  i64 d = shr(t2, b2);
  return scale2(divt(scale2(t1, b1, ev), d, ev), df - b1 - b2, ev);
}

// ---- reproducible FP64 2-norm pieces ------------------------------------
// trunc(x * 2^96) as an integer, |x| < 4
__device__ __forceinline__ i128 trunc_scaled96(double x) {
  u64 bits = (u64)__double_as_longlong(x);
  int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0) return 0;  // zero or subnormal: |x 2^96| < 1
  u64 man = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  int sh = ex - 1075 + 96;  // x 2^96 = man 2^sh
  u128 v;
  if (sh >= 0) v = (u128)man << sh;
  else if (sh <= -64) v = 0;
  else v = (u128)(man >> (-sh));
  i128 r = (i128)v;
  return (bits >> 63) ? -r : r;
}

// round a non-negative 128-bit integer to the nearest double (ties even)
__device__ __forceinline__ double u128_to_double_rn(u128 u) {
  if (u == 0) return 0.0;
  u64 hi = (u64)(u >> 64), lo = (u64)u;
  int len = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  if (len <= 53) return (double)lo;
  int drop = len - 53;
  u128 m = u >> drop;
  u128 rem = u - (m << drop);
  u128 half = (u128)1 << (drop - 1);
  if (rem > half || (rem == half && (m & 1))) {
    m += 1;
    if (m >> 53) {
      m >>= 1;
      drop += 1;
    }
  }
  return scalbn((double)(u64)m, drop);
}

// exact square of r 2^-e, truncated on the 2^-96 grid
__device__ __forceinline__ i128 sq_term(double r, int e) {
  double t = scalbn(r, -e);
  double p = __dmul_rn(t, t);
  double q = __fma_rn(t, t, -p);
  return trunc_scaled96(p) + trunc_scaled96(q);
}

__device__ __forceinline__ double norm_from_acc(i128 acc, int e) {
  double s = u128_to_double_rn((u128)(acc < 0 ? 0 : acc));
  return scalbn(__dsqrt_rn(scalbn(s, -96)), e);
}

// ---- reductions ------------------------------------------------------------
__device__ __forceinline__ i128 shfl_down_i128(i128 v, int o) {
  u128 u = (u128)v;
  u64 lo = __shfl_down_sync(0xffffffffu, (u64)u, o);
  u64 hi = __shfl_down_sync(0xffffffffu, (u64)(u >> 64), o);
  return (i128)(((u128)hi << 64) | (u128)lo);
}

// shuffle down within groups of `width` lanes
__device__ __forceinline__ i128 shfl_down_i128_w(i128 v, int o, int width) {
  u128 u = (u128)v;
  u64 lo = __shfl_down_sync(0xffffffffu, (u64)u, o, width);
  u64 hi = __shfl_down_sync(0xffffffffu, (u64)(u >> 64), o, width);
  return (i128)(((u128)hi << 64) | (u128)lo);
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_down_i128(v, o);
  return v;
}

// block-wide int128 sum; result valid in thread 0
__device__ __forceinline__ i128 block_sum_i128(i128 v) {
  __shared__ u64 s_lo[32], s_hi[32];
  v = warp_sum_i128(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_lo[wid] = (u64)(u128)v;
    s_hi[wid] = (u64)((u128)v >> 64);
  }
  __syncthreads();
  i128 r = 0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    if (lane < nw) r = (i128)(((u128)s_hi[lane] << 64) | (u128)s_lo[lane]);
    r = warp_sum_i128(r);
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double s[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? s[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double s[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? s[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  __syncthreads();
  return r;
}

// add a per-thread event count to a per-system counter
__device__ __forceinline__ void flush_ev(unsigned ev, u64 *ctr) {
  unsigned s = __reduce_add_sync(0xffffffffu, ev);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (u64)s);
}

// ---- flags with acquire/release, bounded waits ----------------------------
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ u64 ld_acquire64(const u64 *p) {
  u64 v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(u64 *p, u64 v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

#define IGM_SPIN_MAX (1 << 22)

// wait until *flag >= epoch; false (and an error bit) if the bound expires.
// Once any wait of the same system has expired, every other wait gives up
// at its next check, so a failure costs one bound, not one per row.
__device__ __forceinline__ bool wait_flag(const int *flag, int epoch, unsigned *err) {
  if (ld_acquire(flag) >= epoch) return true;
  for (int it = 0; it < IGM_SPIN_MAX; ++it) {
    __nanosleep(32);
    if (ld_acquire(flag) >= epoch) return true;
    if ((it & 255) == 255 && (*(volatile unsigned *)err & ERR_TIMEOUT)) return false;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

// wait until *prog >= target (64-bit progress word), bounded like wait_flag
__device__ __forceinline__ bool wait_prog(const u64 *prog, u64 target, unsigned *err) {
  if (ld_acquire64(prog) >= target) return true;
  for (int it = 0; it < IGM_SPIN_MAX; ++it) {
    if (it > 32) __nanosleep(16);
    if (ld_acquire64(prog) >= target) return true;
    if ((it & 255) == 255 && (*(volatile unsigned *)err & ERR_TIMEOUT)) return false;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ u64 gtime_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The one-time set-up kernels (level schedules, the level-scheduled ILU(0))
// are pipelines whose later parts may legitimately wait long for earlier
// ones on big systems: their waits are bounded by time instead.
#define IGM_SETUP_WAIT_NS 20000000000ull

__device__ __forceinline__ bool wait_flag_setup(const int *flag, int epoch, unsigned *err) {
  if (ld_acquire(flag) >= epoch) return true;
  const u64 t0 = gtime_ns();
  for (long long it = 0; it < (1ll << 34); ++it) {
    __nanosleep(64);
    if (ld_acquire(flag) >= epoch) return true;
    if ((it & 255) == 255 &&
        ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtime_ns() - t0 > IGM_SETUP_WAIT_NS))
      break;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ bool wait_prog_setup(const u64 *prog, u64 target, unsigned *err) {
  if (ld_acquire64(prog) >= target) return true;
  const u64 t0 = gtime_ns();
  for (long long it = 0; it < (1ll << 34); ++it) {
    if (it > 32) __nanosleep(32);
    if (ld_acquire64(prog) >= target) return true;
    if ((it & 255) == 255 &&
        ((*(volatile unsigned *)err & ERR_TIMEOUT) || gtime_ns() - t0 > IGM_SETUP_WAIT_NS))
      break;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

// Last-CTA detection for a per-system reduction over its tiles.  Call from
// all threads after the tile partial is written; returns true in every
// thread of the CTA that arrives last (counter reset for reuse).
__device__ __forceinline__ bool last_tile(unsigned *cnt, int ntiles) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(cnt, 1u);
    s_last = (prev == (unsigned)(ntiles - 1));
    if (s_last) *cnt = 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// v * 2^-sh as a double, built with integer operations (exact for
// |v| < 2^53 and results in the normal range): the same value as
// scalbn((double)v, -sh) without the FP64 pipe
__device__ __forceinline__ double i2d_scaled(i64 v, int sh) {
  if (v == 0) return 0.0;
  u64 sgn = (u64)v & 0x8000000000000000ull;
  u64 a = v < 0 ? (u64)(-v) : (u64)v;
  int lz = __clzll((long long)a);
  int e = 63 - lz;                        // position of the leading one
  u64 man = (a << lz) << 1 >> 12;         // the 52 bits below it
  u64 bits = sgn | ((u64)(1023 + e - sh) << 52) | man;
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ i128 load_part(const long long *part, int t) {
  u64 lo = (u64)__ldcg(part + 2 * t), hi = (u64)__ldcg(part + 2 * t + 1);
  return (i128)(((u128)hi << 64) | (u128)lo);
}
__device__ __forceinline__ void store_part(long long *part, int t, i128 v) {
  part[2 * t] = (long long)(u64)(u128)v;
  part[2 * t + 1] = (long long)(u64)((u128)v >> 64);
}

// Givens rotation update of column j (lines 12-19), one thread
static __device__ __noinline__ void givens_col(const SysDev *s, SysScal *sc, int j, i64 hj1) {
  const SysParams &P = s->p;
  const int ld = s->ld, df = P.df;
  i64 *H = s->H;
  unsigned e13 = 0, e15 = 0, e16 = 0, e17 = 0;
  bool zero = shr(hj1, P.b11b) == 0;
  for (int i = 0; i < j; ++i) {
    i64 a = shr(H[i + j * ld], P.b13), b = shr(H[i + 1 + j * ld], P.b13);
    i64 p1 = mulw(s->cs[i], a, e13), p2 = mulw(s->sn[i], b, e13);
    i128 t1 = (i128)p1 + (i128)p2;
    e13 += out64(t1);
    i64 p3 = mulw(negw(s->sn[i], e13), a, e13), p4 = mulw(s->cs[i], b, e13);
    i128 t2 = (i128)p3 + (i128)p4;
    e13 += out64(t2);
    H[i + j * ld] = shr(wrap(t1), df - P.b13);
    H[i + 1 + j * ld] = shr(wrap(t2), df - P.b13);
  }
  i64 hjj = H[j + j * ld], hn = H[j + 1 + j * ld];
  i64 a15 = shr(hjj, P.b15), b15 = shr(hn, P.b15);
  i128 s15 = (i128)mulw(a15, a15, e15) + (i128)mulw(b15, b15, e15);
  e15 += out64(s15);
  i64 tmp = fx_sqrt(wrap(s15), 2 * df - 2 * P.b15, df, e15);
  if (shr(tmp, P.b16b) == 0) {
    sc->early = 1;  // singular column: the solve uses j columns
  } else {
    i64 c = fx_div(hjj, tmp, P.b16a, P.b16b, df, e16);
    i64 sn = fx_div(hn, tmp, P.b16a, P.b16b, df, e16);
    s->cs[j] = c;
    s->sn[j] = sn;
    i64 gj = s->g[j];
    s->g[j + 1] = shr(mulw(negw(sn, e17), gj, e17), df);
    s->g[j] = shr(mulw(c, gj, e17), df);
    H[j + j * ld] = tmp;
    H[j + 1 + j * ld] = 0;
    sc->jeff = j + 1;
    if (zero) sc->early = 1;
  }
  if (e13) atomicAdd(&sc->ev[IGM_EV_L13], (u64)e13);
  if (e15) atomicAdd(&sc->ev[IGM_EV_L15], (u64)e15);
  if (e16) atomicAdd(&sc->ev[IGM_EV_L16], (u64)e16);
  if (e17) atomicAdd(&sc->ev[IGM_EV_L17], (u64)e17);
}


// ---------------------------------------------------------------------------
// shared-memory addresses, mbarriers and bulk copies (the async proxy)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(u64 *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64 *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64 *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bytes (a multiple of 16) from 16-byte aligned global memory to 16-byte
// aligned shared memory, completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, u64 *bar) {
  if (!IGM_OK(((smem_u32(dst) | (unsigned)(size_t)src | bytes) & 15u) == 0, CHK_BULK_G2S)) return;
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ u64 gtimer() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// orders this thread's earlier generic-proxy accesses of shared memory
// before its later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// bytes (a multiple of 16) from 16-byte aligned shared memory to 16-byte
// aligned global memory, in this thread's current bulk group
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
  if (!IGM_OK((((unsigned)(size_t)dst | smem_u32(src) | bytes) & 15u) == 0, CHK_BULK_S2G)) return;
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                   __cvta_generic_to_global(dst)),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// at most N of this thread's bulk groups still read their shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// at most N of this thread's bulk groups still pending (the others' writes
// are complete)
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// orders this thread's earlier generic-proxy accesses of global memory
// before its later async-proxy (bulk copy) accesses of global memory
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// iteration bound of the time-bounded waits (the time limit ends them first)
#define IGM_WAIT_ITERS (1 << 28)

// wait for the phase of parity `parity` of a bulk-copy barrier; bounded by
// time (a copy always completes, so expiry is an error); false if expired
__device__ __forceinline__ bool mbar_wait(u64 *bar, unsigned parity, unsigned *err,
                                          u64 limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const u64 t0 = gtimer();
  for (int it = 0; it < IGM_WAIT_ITERS; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && gtimer() - t0 > limit_ns) break;
  }
  atomicOr(err, ERR_TIMEOUT);
  return false;
}

}  // namespace igm
