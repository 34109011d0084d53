// igm_internal.h -- device-side data layout shared by the kernels and the
// host driver of the int-GMRES library (not part of the public ABI).
//
// Layout in HBM, per system (one igm_handle):
//   CSR pattern   rowptr int32[n+1], col int32[nnz], diagpos int32[n]
//   ahat f64[nnz] (input values, kept for the unscaled residual),
//   a f64[nnz] (eq. 1), d f64[n] (eq. 3), abar int64[nnz] (Sec. IV-B)
//   ILU: f f64[nnz] (eq. ilu), fac int64[nnz] + ldiag/udiag int64[n]
//        (eq. dldr..ilu2), level orders lorder/uorder int32[n],
//        ready flags lflag/uflag int32[n]
//   vectors: b, bh, xt, r, t, xk f64[n]; w, yv int64[n];
//            V int64[(m+1) n] (row-major by basis vector)
//   scalars: H int64[(m+1) m] column-major, cs, sn int64[m], g int64[m+1],
//            yfp f64[m], SysScal (counters, histories, status)
// A batch is a list of systems plus a tile table: tile t covers rows
// [row0, row0+nrows) of one system (never straddling two), IGM_TILE rows
// per tile; every kernel runs one CTA per tile.
#pragma once
#include <cstdint>

#define IGM_TILE 1024
#define IGM_BLOCK 256
#define IGM_NEV 16

typedef long long i64;
typedef unsigned long long u64;

namespace igm {

struct SysParams {
  int df, alpha_a, m, precond;
  int b7, b8, b10, b11a, b11b, b13, b15, b16a, b16b;
  int inner, max_refine;
  double tol;
  int tune;               // inner solves the shift auto-tuning may discard
  int stall;              // tests: the first substitution chunk never signals
  u64 wait_ns;            // bound of each substitution wait (ns)
};

// error bits of SysScal::err
enum : unsigned {
  ERR_TIMEOUT = 1u, ERR_ZERO_ROW = 2u, ERR_ZERO_PIVOT = 4u, ERR_BADCSR = 8u,
  ERR_CAST = 16u
};

// per-system mutable scalars, in device memory
struct SysScal {
  u64 ev[IGM_NEV];
  int status, active, cyc, jeff, early, refinements, inner_steps, breakdowns;
  int seq;                 // epoch of the ready flags
  unsigned err;
  unsigned cnt[2];         // last-CTA counters of tile reductions
  int mode;                // 0 refinement loop, 1 single inner solve
  int normj;               // step whose line 11 runs (-1: none)
  double nb, nbh, rho, gamma, nu, maxabs, relres_unscaled, pad2;
  i64 hnext;               // h_{j+1,j} before the rotations (line 11)
  double relres_hist[65];
  double gamma_hist[64];
  double rho_ring[4];      // the last residuals (stall test of the loop)
  // shift auto-tuning, per line 7, 8, 10, 13, 15 of Fig. 2 (in this order)
  u64 ev0[5];              // their event counts when the inner solve began
  int retries;             // inner solves discarded so far
  int retry;               // 1: the inner solve that just ran is discarded
  int beta[5];             // their shifts in use (a copy of SysDev::p)
  int vwide;               // a basis entry of this inner solve left int32:
                           // readers use the int64 copy of the basis
};

// Schedule and packed data of one triangular factor.  Positions p = 0..n-1
// run in dependency order (L: row p, U: row n-1-p), are cut into chunks of
// `chunk` positions, and inside each chunk grouped by local level
// (dependency depth counted inside the chunk), a level wider than the
// factor's group cap being split into several consecutive groups.  ord[p]
// is the row at position p; group g = (chunk, local group index) covers
// positions lptr[g]..lptr[g+1]; levb[c] is the first group of chunk c and
// lev[i] the local group index of row i.  Each group's rows are packed into
// one block (layout below): the strict part of every row farthest
// dependency first (L: columns ascending, U: columns descending), each
// dependency as a factor entry and a source code.  need[g]: progress the
// previous chunk must reach before group g runs.  Progress words one
// 128-byte line apart (pollers of different chunks do not share a line).
#define IGM_PROG_STRIDE 16

// Source code of a dependency: the values a chunk reads sit in one
// shared-memory array, [the chunk's own ring of `ring` values | the
// predecessor ring of `pring` values | one zero], so a code >= 0 is the
// value's index there (own values at their chunk-local position mod ring,
// the previous chunk's at their position mod pring, padding at the zero); a
// code -1 - p reads the value at position p from the position-ordered copy
// of the results when the row is computed (after waiting for p's chunk when
// chunks may depend on chunks before their predecessor).
// slots of the substitution kernel: each holds one group's packed block
// (bulk-copied) and its right-hand sides (gathered); as many as fit, up to
// IGM_TRSV_NA_MAX and at least IGM_TRSV_NA_MIN
#define IGM_TRSV_NA_MAX 8
#define IGM_TRSV_NA_MIN 4
#define IGM_TRSV_NB 3              // predecessor-copy barriers (one per group, round robin)
#define IGM_TRSV_PFB 2             // groups ahead of a group the predecessor copy is issued
#define IGM_TRSV_RING_MAX 4096
// dynamic shared memory the substitution kernel uses per CTA
#define IGM_TRSV_SMEM (224 * 1024)

// Packed block of one group of w rows (wp = w rounded up to a multiple of
// 4), everything a row needs but its right-hand side and dependency values,
// each array 16-byte aligned: codes [K][wp] int32, orders [wp] int32, row
// words [wp] int32 (IGM_ROW_*), factors [K][wp] (fb bytes), diagonals [wp]
// (8 bytes), division multipliers [wp] u64.
// A row word: bits 0-6 hold 1 + the exactness bound (0: none), bits 8-14 the
// shift of the division by the diagonal, bit 15 is set when a dependency of
// the row is read late (code < 0).
#define IGM_ROW_BOUND(wd) (((wd) & 0x7f) - 1)
#define IGM_ROW_SHIFT(wd) (((wd) >> 8) & 0x7f)
#define IGM_ROW_LATE 0x8000
__host__ __device__ inline unsigned trsv_wp(int w) { return ((unsigned)(w < 1 ? 1 : w) + 3u) & ~3u; }
__host__ __device__ inline unsigned trsv_blk_bytes(unsigned wp, int K, int fb) {
  const unsigned k = (unsigned)(K < 0 ? 0 : K);
  return wp * (4u * k + 8u + (unsigned)fb * k + 16u);
}

struct Tri {
  const int *ord, *lptr, *levb, *lev, *need;
  // the groups' packed blocks (integer factors, int32 when fac32; FP64
  // factors for the comparison solver in blobd) and each group's byte offset
  const unsigned char *blob, *blobd;
  const long long *boff, *boffd;
  u64 *prog;                    // per chunk (IGM_PROG_STRIDE apart): (epoch << 32) | groups done
  int nchunk, K;
  int maxlev;                   // most groups of one chunk
  int maxw;                     // most rows of one group
  int ring;                     // slots of the chunk's value ring (power of two)
  int pring;                    // slots of the predecessor ring (power of two)
  int fac32;                    // every strict factor entry fits in int32
};

// Shared-memory carve-up of one substitution CTA for a factor with groups of
// at most W rows, K dependencies per row, rings of `ring` and `pring` values,
// `nlev` staged groups and factor entries of fb bytes (byte offsets; the same
// on the host and in the kernel): [values: own ring | predecessor ring |
// zero] [na slots: block | right-hand sides] [group pointers].
struct TrsvLayout {
  unsigned szBlk;               // bytes of the largest block
  unsigned szSlot;              // bytes of a slot (block + W right-hand sides)
  unsigned oSlots, na, oLev, lev, total;
};

__host__ __device__ inline unsigned trsv_r128(unsigned b) { return (b + 127u) & ~127u; }

// na: slots to use (0: as many as fit in IGM_TRSV_SMEM, at least IGM_TRSV_NA_MIN)
__host__ __device__ inline TrsvLayout trsv_layout(int W, int K, int ring, int pring, int nlev,
                                                  int fb, int na = 0) {
  TrsvLayout t;
  t.szBlk = trsv_blk_bytes(trsv_wp(W), K, fb);
  t.szSlot = trsv_r128(t.szBlk + (unsigned)(W < 1 ? 1 : W) * 8u);
  t.oSlots = trsv_r128(((unsigned)ring + (unsigned)pring + 2u) * 8u);
  t.na = na > 0 ? (unsigned)na : IGM_TRSV_NA_MAX;
  while (na <= 0 && t.na > IGM_TRSV_NA_MIN && t.oSlots + t.na * t.szSlot > IGM_TRSV_SMEM) --t.na;
  t.oLev = t.oSlots + t.na * t.szSlot;
  // the chunk's group pointers and requirements, and the previous chunk's
  // group pointers, if they fit
  const unsigned lb = (3u * (unsigned)nlev + 3u) * 4u;
  t.lev = (t.oLev + lb <= IGM_TRSV_SMEM) ? (unsigned)nlev : 0u;
  t.total = t.oLev + (t.lev ? trsv_r128(lb) : 0u);
  return t;
}

struct SysDev {
  int n, nnz, ld;          // ld = m + 1
  int pad;
  SysParams p;             // shifts of lines 7, 8, 10, 13, 15 change while
                           // a solve auto-tunes them
  int beta0[5];            // those shifts as set up
  const int *rowptr, *col, *diagpos;
  const double *ahat, *a, *d;
  const i64 *abar;
  // Ā in SELL-32 (slices of 32 rows, each padded to its longest row and
  // stored column-major: entry k of row 32 s + l at sptr[s] + 32 k + l;
  // padding has value 0) for the line-5 SpMV
  const long long *sptr;
  const i64 *sval;               // (ns + 1) terms, each nnz_sell values
  const int *scol;
  long long nnz_sell;            // slots per term of the SELL-32 copy
  // correction terms of eq. (AA): abar and sval hold ns + 1 terms (term l at
  // l * nnz, resp. l * nnz_sell); alphas[0] = 0
  int ns;
  int alphas[IGM_MAX_S + 1];
  // multicolour order: rows of colour c are [cptr[c], cptr[c+1]) (device),
  // ncolors > 0 selects the colour-by-colour substitutions
  int ncolors;
  const int *cptr;
  const double *f;                       // FP64 ILU(0) factors
  const i64 *fac, *ldiag, *udiag;        // integer factors
  // substitution schedules of the two factors, tri[0] = L, tri[1] = U
  Tri tri[2];
  int chunk;                    // rows per chunk (both factors)
  int single_pred;              // chunk >= bandwidth: every dependency
                                // outside a chunk lies in the previous one
  int *lflag, *uflag;           // per-row ready flags (set-up, line 1' none)
  double *b, *bh, *xt, *r, *t, *xk;
  i64 *w, *yv, *V;
  int *V32;                     // the basis as int32 words (read unless sc->vwide)
  i64 *xbuf;                    // substitution results in position order
  i64 *H, *cs, *sn, *g;
  double *yfp;
  SysScal *sc;
};

struct Tile {
  int sys;     // batch-local system index
  int row0;    // first row (or first position of a level order)
  int nrows;
  int first;   // index of the system's first tile
};

#define IGM_STILE 4096     // rows of a super-tile of the persistent kernels

struct BatchDev {
  int nsys, ntiles;
  int nstiles;             // super-tiles (IGM_STILE rows, one system each)
  const Tile *stiles;
  int nctiles;             // substitution chunks over all systems
  const Tile *ctiles;      // {sys, chunk index, -, first chunk tile}
  SysDev *const *sys;      // device pointers to each system's SysDev
  const Tile *tiles;
  const int *sys_ntiles;   // tiles per system
  long long *part;         // 2 x ntiles int64 (int128 partials, lo/hi)
  double *partd;           // ntiles
  unsigned *ticket;        // 4 dynamic-ticket counters
  int *nact;               // systems still refining
  unsigned *bar;           // grid barrier: [0] arrivals, [1] generation;
                           // integer Arnoldi step: [2] launch epoch, [3]
                           // CTAs finished in this launch
  double *cpart;           // 3 slots x maxG x nsys FP64 per-CTA partials
  int maxg;                // CTAs of the persistent kernels
  // integer Arnoldi step: CTA c sweeps the segments
  // mseg[mseg_ptr[c] .. mseg_ptr[c+1]), contiguous row ranges of one system
  // each ({sys, row0, nrows, offset of the rows in the CTA's copy of w})
  int mgs_g;               // its CTAs
  const int *mseg_ptr;
  const Tile *mseg;
  i64 *mseg_h;             // per segment: the coefficient of the next pass
  int nseg;                // segments in all
  u64 *mpart;              // 2 slots (pass parity) x nseg x 4 words: a
                           // pass's exact sum over each segment, tagged
  int *mseg_act;           // per segment beyond a CTA's descriptor cache:
                           // active | narrow << 1 of the current step
  unsigned *mvtag;         // per segment: the last step whose basis rows
                           // the fused Arnoldi kernel published (tagged)
  int fuse;                // steps per fused Arnoldi launch (0: not fused)
  int max_m;               // Arnoldi steps of the batch's systems (all equal)
  const int *sys_seg;      // system s owns segments [sys_seg[s], sys_seg[s+1])
  int mgs_wrows;           // rows each CTA keeps resident in shared memory
  int mgs_rows;            // most rows of a CTA
  int mgs_ring;            // single-step kernel streams further rows (ring mode)
  int trsv_maxk;           // most strict entries of one factor row
  int max_ns;              // most correction terms of eq. (AA) of a system
  int max_colors;          // most colours of a multicolour-ordered system
};

// vector selectors for the generic max / norm kernels
enum Vec : int { VEC_B = 0, VEC_R = 1, VEC_BH = 2 };
// what the last CTA does with a finished norm
enum NormAct : int { ACT_NB = 0, ACT_RHO = 1, ACT_NU = 2, ACT_NBH = 3, ACT_UNSC = 4 };

// Arnoldi step (lines 6-19): one CTA per SM of IGM_MGS_BLOCK threads in the
// grid mode; the one-CTA mode runs IGM_MGS_ONE_BLOCK threads (IGM_RPT rows
// a thread) over at most IGM_MSEG_CACHE systems
#define IGM_MGS_BLOCK 1024
#define IGM_MGS_ONE_BLOCK 256
#define IGM_MSEG_CACHE 64

// the step's one-CTA mode: one CTA holding at most IGM_MGS_BLOCK rows in
// all, every row of w in shared memory, each system one segment of it (ns
// segments), every segment descriptor cached in shared memory
__host__ __device__ __forceinline__ bool mgs_one_cta(const BatchDev &B, int ns) {
  return B.mgs_g == 1 && B.mgs_rows > 0 && B.mgs_rows <= IGM_MGS_BLOCK &&
         B.mgs_wrows == B.mgs_rows && ns <= IGM_MSEG_CACHE;
}

}  // namespace igm
