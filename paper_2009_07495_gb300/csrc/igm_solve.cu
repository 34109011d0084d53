// igm_solve.cu -- kernels of the refinement loop (Fig. 1) and of one
// int-GMRES(m) inner solve (Fig. 2 with lines 1', 5' of Sec. VI).
//
// Every kernel runs one CTA per tile of a batch (a tile = up to IGM_TILE
// rows of one system) and gates itself on the system's state, so the same
// launch sequence serves one system or many.  Per-system reductions are
// exact (int128 partials, or the reproducible FP64 norm) and finished by
// the last CTA of the system, so every result is independent of the tile
// schedule and of the other systems in the batch.
#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

#define TILE_LOOP(r)                                                           \
  for (int r = tl.row0 + (int)threadIdx.x; r < tl.row0 + tl.nrows; r += blockDim.x)

__device__ __forceinline__ bool g_ir(const SysScal *sc) { return sc->active != 0; }
__device__ __forceinline__ bool g_cyc(const SysScal *sc) { return sc->cyc != 0; }
__device__ __forceinline__ bool g_step(const SysScal *sc) {
  return sc->cyc != 0 && sc->early == 0;
}

__device__ __forceinline__ const double *vec_of(const SysDev *s, int which) {
  return which == VEC_B ? s->b : which == VEC_R ? s->r : s->bh;
}

// ---------------------------------------------------------------------------
// Fig. 1 set-up: b = D^-1 bh (eq. 1), x = 0; scalar state reset
// ---------------------------------------------------------------------------
__global__ void k_init_scal(BatchDev B, int mode) {
  int si = blockIdx.x * blockDim.x + threadIdx.x;
  if (si >= B.nsys) return;
  SysScal *sc = B.sys[si]->sc;
  for (int k = 0; k < IGM_NEV; ++k) sc->ev[k] = 0;
  sc->status = 5;  // IGM_ENOCONV until the test of Fig. 1 passes
  sc->active = mode == 0 ? 1 : 0;
  sc->cyc = mode == 0 ? 0 : 1;
  sc->jeff = 0;
  sc->early = 0;
  sc->refinements = 0;
  sc->inner_steps = 0;
  sc->breakdowns = 0;
  sc->err = 0;
  sc->cnt[0] = sc->cnt[1] = 0;
  sc->mode = mode;
  sc->normj = -1;
  sc->gamma = 1.0;
  sc->rho = 0.0;
  sc->relres_unscaled = 0.0;
  for (int k = 0; k < 65; ++k) sc->relres_hist[k] = 0.0;
  for (int k = 0; k < 64; ++k) sc->gamma_hist[k] = 0.0;
}

__global__ void k_init_ir(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  TILE_LOOP(i) {
    s->b[i] = __ddiv_rn(s->bh[i], s->d[i]);
    s->xt[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// max |v_i| per system (exact)
// ---------------------------------------------------------------------------
__global__ void k_max(BatchDev B, int which, int gate) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (gate == 1 && !g_ir(sc)) return;
  if (gate == 2 && !(g_cyc(sc) && sc->early == 0)) return;
  const double *v = vec_of(s, which);
  double m = 0.0;
  TILE_LOOP(i) m = fmax(m, fabs(v[i]));
  m = block_max(m);
  if (threadIdx.x == 0) B.partd[blockIdx.x] = m;
  if (last_tile(&sc->cnt[0], B.sys_ntiles[tl.sys])) {
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int t = 0; t < B.sys_ntiles[tl.sys]; ++t) mx = fmax(mx, __ldcg(B.partd + tl.first + t));
      sc->maxabs = mx;
    }
  }
}

// ---------------------------------------------------------------------------
// reproducible 2-norm of a per-system vector, then the action of `act`
// ---------------------------------------------------------------------------
__device__ void norm_action(const BatchDev &B, const SysDev *s, SysScal *sc, int act,
                            double nrm) {
  const SysParams &P = s->p;
  switch (act) {
    case ACT_NB: sc->nb = nrm; break;
    case ACT_NBH: sc->nbh = nrm; break;
    case ACT_UNSC:
      sc->relres_unscaled = sc->nbh == 0.0 ? 0.0 : __ddiv_rn(nrm, sc->nbh);
      break;
    case ACT_NU:
      sc->nu = nrm;
      if (nrm == 0.0) sc->early = 2;  // nothing to solve: x^(k) stays 0
      break;
    case ACT_RHO: {
      // the test of Fig. 1 on the scaled system, then eq. (gammak)
      double rho = sc->nb == 0.0 ? 0.0 : __ddiv_rn(nrm, sc->nb);
      int k = sc->refinements;
      if (k < 65) sc->relres_hist[k] = rho;
      sc->rho = rho;
      sc->jeff = 0;
      sc->early = 0;
      sc->normj = -1;
      if (rho < P.tol) {
        sc->active = 0;
        sc->cyc = 0;
        sc->status = 0;
      } else if (k >= P.max_refine) {
        sc->active = 0;
        sc->cyc = 0;
        sc->status = 5;
      } else {
        sc->gamma = sc->maxabs;
        if (k < 64) sc->gamma_hist[k] = sc->maxabs;
        sc->cyc = 1;
        atomicAdd(B.nact, 1);
      }
      break;
    }
  }
}

__global__ void k_norm(BatchDev B, int which, int act, int gate) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (gate == 1 && !g_ir(sc)) return;
  if (gate == 2 && !(g_cyc(sc) && sc->early == 0)) return;
  const double *v = vec_of(s, which);
  double mx = sc->maxabs;
  int e = mx > 0.0 ? ilogb(mx) : 0;
  i128 acc = 0;
  if (mx > 0.0) TILE_LOOP(i) acc += sq_term(v[i], e);
  acc = block_sum_i128(acc);
  if (threadIdx.x == 0) store_part(B.part, blockIdx.x, acc);
  if (last_tile(&sc->cnt[0], B.sys_ntiles[tl.sys])) {
    if (threadIdx.x == 0) {
      i128 tot = 0;
      for (int t = 0; t < B.sys_ntiles[tl.sys]; ++t) tot += load_part(B.part, tl.first + t);
      double nrm = mx > 0.0 ? norm_from_acc(tot, e) : 0.0;
      norm_action(B, s, sc, act, nrm);
    }
  }
}

// ---------------------------------------------------------------------------
// eq. (b): r = b - A x (FP64, CSR order, no FMA) and max |r_i|.
// hat = 1: the same on the original system (bh - Ah x) for the report.
// ---------------------------------------------------------------------------
__global__ void k_resid(BatchDev B, int hat) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && !hat) *B.nact = 0;
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!hat && !g_ir(sc)) return;
  const double *av = hat ? s->ahat : s->a;
  const double *bv = hat ? s->bh : s->b;
  double m = 0.0;
  TILE_LOOP(i) {
    double acc = 0.0;
    for (int k = s->rowptr[i]; k < s->rowptr[i + 1]; ++k)
      acc = __dadd_rn(acc, __dmul_rn(av[k], s->xt[s->col[k]]));
    double r = __dsub_rn(bv[i], acc);
    s->r[i] = r;
    m = fmax(m, fabs(r));
  }
  m = block_max(m);
  if (threadIdx.x == 0) B.partd[blockIdx.x] = m;
  if (last_tile(&sc->cnt[0], B.sys_ntiles[tl.sys])) {
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int t = 0; t < B.sys_ntiles[tl.sys]; ++t) mx = fmax(mx, __ldcg(B.partd + tl.first + t));
      sc->maxabs = mx;
    }
  }
}

// line 1 of Fig. 2 for a given initial guess: r = bk - Abar xk (FP64)
__global__ void k_resid_int(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  if (!g_cyc(s->sc)) return;
  TILE_LOOP(i) {
    double acc = 0.0;
    for (int k = s->rowptr[i]; k < s->rowptr[i + 1]; ++k)
      acc = __dadd_rn(acc, __dmul_rn((double)s->abar[k], s->xk[s->col[k]]));
    s->r[i] = __dsub_rn(s->t[i], acc);
  }
}

// eq. (scale): b^(k) = b' / gamma, x^(k) = 0.  Also arms the ready flags
// and tickets of the substitutions that follow.
__global__ void k_rhs(BatchDev B) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.ticket[0] = 0;
    B.ticket[1] = 0;
  }
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_cyc(sc)) return;
  if (blockIdx.x == tl.first && threadIdx.x == 0) sc->seq += 1;
  double gam = sc->gamma;
  TILE_LOOP(i) s->r[i] = __ddiv_rn(s->r[i], gam);
}

// arms flags and tickets (single inner-solve mode)
__global__ void k_arm(BatchDev B) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.ticket[0] = 0;
    B.ticket[1] = 0;
  }
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  if (!g_cyc(s->sc)) return;
  if (blockIdx.x == tl.first && threadIdx.x == 0) s->sc->seq += 1;
}

// ---------------------------------------------------------------------------
// Sparse triangular substitutions, synchronisation-free: rows are visited in
// level order (dependencies always sit at earlier positions of the same
// system), CTAs take tiles by a dynamic ticket so that every row waited on
// belongs to a CTA that is already running; each row waits (bounded) on
// the ready flags of the rows it reads, then publishes its value with a
// release store of the current epoch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int take_ticket(unsigned *ctr) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  return s_t;
}

// line 1': y = Lbar^-1 z (lower = 1) or w = Ubar^-1 y (lower = 0), FP64 on the
// integer factors; z = r -> t (lower) and t -> r (upper)
__global__ void k_trsv_fp(BatchDev B, int lower) {
  int ti = take_ticket(&B.ticket[lower ? 0 : 1]);
  Tile tl = B.tiles[ti];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!(g_cyc(sc) && sc->early == 0) || !s->p.precond) return;
  const int *ord = lower ? s->lorder : s->uorder;
  int *flag = lower ? s->lflag : s->uflag;
  const double *in = lower ? s->r : s->t;
  double *out = lower ? s->t : s->r;
  int ep = sc->seq;
  TILE_LOOP(p) {
    int i = ord[p];
    double acc = in[i];
    int k0 = lower ? s->rowptr[i] : s->diagpos[i] + 1;
    int k1 = lower ? s->diagpos[i] : s->rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      int j = s->col[k];
      wait_flag(flag + j, ep, &sc->err);
      acc = __dsub_rn(acc, __dmul_rn((double)s->fac[k], __ldcg(out + j)));
    }
    out[i] = __ddiv_rn(acc, (double)(lower ? s->ldiag[i] : s->udiag[i]));
    st_release(flag + i, ep);
  }
}

// line 5': integer substitutions, w -> yv (lower) and yv -> w (upper)
__global__ void k_trsv_int(BatchDev B, int lower) {
  int ti = take_ticket(&B.ticket[lower ? 2 : 3]);
  Tile tl = B.tiles[ti];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_step(sc) || !s->p.precond) return;
  const int *ord = lower ? s->lorder : s->uorder;
  int *flag = lower ? s->lflag : s->uflag;
  const i64 *in = lower ? s->w : s->yv;
  i64 *out = lower ? s->yv : s->w;
  int ep = sc->seq;
  unsigned ev = 0;
  TILE_LOOP(p) {
    int i = ord[p];
    i128 acc = in[i];
    int k0 = lower ? s->rowptr[i] : s->diagpos[i] + 1;
    int k1 = lower ? s->diagpos[i] : s->rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      int j = s->col[k];
      wait_flag(flag + j, ep, &sc->err);
      acc -= (i128)mulw(s->fac[k], (i64)__ldcg((const long long *)out + j), ev);
    }
    ev += out64(acc);
    out[i] = divt(wrap(acc), lower ? s->ldiag[i] : s->udiag[i], ev);
    st_release(flag + i, ep);
  }
  flush_ev(ev, &sc->ev[IGM_EV_L5P]);
}

// ---------------------------------------------------------------------------
// line 1 end and lines 2-3: v1 = r0 / ||r0||, cast to Q(df); g = (2^df, 0..)
// ---------------------------------------------------------------------------
__global__ void k_cast_v1(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_step(sc)) return;
  const int df = s->p.df;
  double nu = sc->nu;
  unsigned ev = 0;
  TILE_LOOP(l) {
    double v = scalbn(__ddiv_rn(s->r[l], nu), df);
    i64 q = 0;
    if (fabs(v) < 9223372036854775808.0) q = __double2ll_rz(v);
    else ev += 1;
    s->V[l] = q;
  }
  if (blockIdx.x == tl.first && threadIdx.x == 0) {
    s->g[0] = (i64)1 << df;
    for (int k = 1; k <= s->p.m; ++k) s->g[k] = 0;
  }
  flush_ev(ev, &sc->ev[IGM_EV_L2]);
}

// ---------------------------------------------------------------------------
// line 5: w = Abar_0 v_j (exact int128 row sums; Table 3 line 5)
// ---------------------------------------------------------------------------
__global__ void k_spmv(BatchDev B, int j) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.ticket[2] = 0;
    B.ticket[3] = 0;
  }
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_step(sc) || j >= s->p.m) return;
  if (blockIdx.x == tl.first && threadIdx.x == 0) sc->seq += 1;
  const i64 *vj = s->V + (size_t)j * s->n;
  unsigned ev = 0;
  TILE_LOOP(i) {
    i128 acc = 0;
    for (int k = s->rowptr[i]; k < s->rowptr[i + 1]; ++k)
      acc += (i128)mulw(s->abar[k], vj[s->col[k]], ev);
    ev += out64(acc);
    s->w[i] = wrap(acc);
  }
  flush_ev(ev, &sc->ev[IGM_EV_L5]);
}

// ---------------------------------------------------------------------------
// lines 6-9, modified Gram-Schmidt, one pass per i: the line-8 update with
// h_{i-1,j} (only h shifted) fused with the line-7 inner product with v_i
// (only w shifted); the last CTA forms h_ij = sum >> (df - beta7).
// ---------------------------------------------------------------------------
__global__ void k_mgs(BatchDev B, int i, int j) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_step(sc) || j >= s->p.m) return;
  const SysParams &P = s->p;
  const int n = s->n, ld = s->ld, df = P.df;
  const i64 *vi = s->V + (size_t)i * n;
  const i64 *vp = s->V + (size_t)(i > 0 ? i - 1 : 0) * n;
  i64 hs = i > 0 ? shr(s->H[(i - 1) + j * ld], P.b8) : 0;
  unsigned ev7 = 0, ev8 = 0;
  i128 acc = 0;
  TILE_LOOP(l) {
    i64 wl = s->w[l];
    if (i > 0) {
      i64 p = shr(mulw(hs, vp[l], ev8), df - P.b8);
      i128 d = (i128)wl - (i128)p;
      ev8 += out64(d);
      wl = wrap(d);
      s->w[l] = wl;
    }
    acc += (i128)mulw(shr(wl, P.b7), vi[l], ev7);
  }
  flush_ev(ev8, &sc->ev[IGM_EV_L8]);
  acc = block_sum_i128(acc);
  if (threadIdx.x == 0) store_part(B.part, blockIdx.x, acc);
  if (last_tile(&sc->cnt[0], B.sys_ntiles[tl.sys])) {
    if (threadIdx.x == 0) {
      i128 tot = 0;
      for (int t = 0; t < B.sys_ntiles[tl.sys]; ++t) tot += load_part(B.part, tl.first + t);
      ev7 += out64(tot);
      s->H[i + j * ld] = shr(wrap(tot), df - P.b7);
    }
  }
  flush_ev(ev7, &sc->ev[IGM_EV_L7]);
}

// Givens rotation update of column j (lines 12-19), one thread
__device__ void givens_col(const SysDev *s, SysScal *sc, int j, i64 hj1) {
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

// last MGS pass (line 8 with h_jj) fused with the line-10 norm; the last
// CTA forms h_{j+1,j} and runs lines 12-19 for column j
__global__ void k_mgs_last(BatchDev B, int j) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_step(sc) || j >= s->p.m) return;
  const SysParams &P = s->p;
  const int n = s->n, ld = s->ld, df = P.df;
  const i64 *vp = s->V + (size_t)j * n;
  i64 hs = shr(s->H[j + j * ld], P.b8);
  unsigned ev10 = 0, ev8 = 0;
  i128 acc = 0;
  TILE_LOOP(l) {
    i64 wl = s->w[l];
    i64 p = shr(mulw(hs, vp[l], ev8), df - P.b8);
    i128 d = (i128)wl - (i128)p;
    ev8 += out64(d);
    wl = wrap(d);
    s->w[l] = wl;
    i64 a = shr(wl, P.b10);
    acc += (i128)mulw(a, a, ev10);
  }
  flush_ev(ev8, &sc->ev[IGM_EV_L8]);
  acc = block_sum_i128(acc);
  if (threadIdx.x == 0) store_part(B.part, blockIdx.x, acc);
  if (last_tile(&sc->cnt[0], B.sys_ntiles[tl.sys])) {
    if (threadIdx.x == 0) {
      i128 tot = 0;
      for (int t = 0; t < B.sys_ntiles[tl.sys]; ++t) tot += load_part(B.part, tl.first + t);
      ev10 += out64(tot);
      i64 hj1 = fx_sqrt(wrap(tot), 2 * df - 2 * P.b10, df, ev10);
      s->H[j + 1 + j * ld] = hj1;
      sc->hnext = hj1;
      // line 11 comes before lines 12-19 in Fig. 2: it runs unless its own
      // divisor is zero, whatever line 16 finds
      sc->normj = shr(hj1, P.b11b) == 0 ? -1 : j;
      givens_col(s, sc, j, hj1);
    }
  }
  flush_ev(ev10, &sc->ev[IGM_EV_L10]);
}

// line 11: v_{j+1} = w / h_{j+1,j} (Sec. V-B division), unless breakdown
__global__ void k_normalize(BatchDev B, int j) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_cyc(sc) || sc->normj != j || j >= s->p.m) return;
  const SysParams &P = s->p;
  i64 hn = sc->hnext;
  i64 *vn = s->V + (size_t)(j + 1) * s->n;
  unsigned ev = 0, evr = 0;
  TILE_LOOP(l) {
    i64 q = fx_div(s->w[l], hn, P.b11a, P.b11b, P.df, ev);
    evr += (q < INT32_MIN || q > INT32_MAX);
    vn[l] = q;
  }
  flush_ev(ev, &sc->ev[IGM_EV_L11]);
  flush_ev(evr, &sc->ev[IGM_EV_VRANGE]);
}

// ---------------------------------------------------------------------------
// lines 21-22: y = ||r0|| H^-1 g in FP64 (one thread per system)
// ---------------------------------------------------------------------------
__global__ void k_backsub(BatchDev B) {
  int si = blockIdx.x * blockDim.x + threadIdx.x;
  if (si >= B.nsys) return;
  const SysDev *s = B.sys[si];
  SysScal *sc = s->sc;
  if (!g_cyc(sc)) return;
  const int jeff = sc->jeff, ld = s->ld, df = s->p.df;
  double *z = s->yfp;
  for (int a = jeff - 1; a >= 0; --a) {
    double acc = scalbn((double)s->g[a], -df);
    for (int b = a + 1; b < jeff; ++b)
      acc = __dsub_rn(acc, __dmul_rn(scalbn((double)s->H[a + b * ld], -df), z[b]));
    z[a] = __ddiv_rn(acc, scalbn((double)s->H[a + a * ld], -df));
  }
  for (int a = 0; a < jeff; ++a) z[a] = __dmul_rn(sc->nu, z[a]);
  sc->refinements += 1;
  sc->inner_steps += jeff;
  if (sc->early == 1) sc->breakdowns += 1;
}

// line 23 and eq. (update): x^(k) = sum_i y_i v_i; refinement mode adds
// gamma x^(k) to x, single-solve mode adds the sum to the caller's guess
__global__ void k_update(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!g_cyc(sc)) return;
  const int jeff = sc->jeff, n = s->n, df = s->p.df;
  const bool ir = sc->mode == 0;
  double gam = sc->gamma;
  TILE_LOOP(l) {
    double acc = ir ? 0.0 : s->xk[l];
    for (int i = 0; i < jeff; ++i)
      acc = __dadd_rn(acc, __dmul_rn(s->yfp[i], scalbn((double)s->V[(size_t)i * n + l], -df)));
    if (ir) s->xt[l] = __dadd_rn(s->xt[l], __dmul_rn(gam, acc));
    else s->xk[l] = acc;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nb_sys(const BatchDev &B) { return (B.nsys + 127) / 128; }

void launch_init_scal(const BatchDev &B, int mode, cudaStream_t st) {
  k_init_scal<<<nb_sys(B), 128, 0, st>>>(B, mode);
}
void launch_init_ir(const BatchDev &B, cudaStream_t st) {
  k_init_ir<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}
void launch_max(const BatchDev &B, int which, int gate, cudaStream_t st) {
  k_max<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, which, gate);
}
void launch_norm(const BatchDev &B, int which, int act, int gate, cudaStream_t st) {
  k_norm<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, which, act, gate);
}
void launch_resid(const BatchDev &B, int hat, cudaStream_t st) {
  k_resid<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, hat);
}
void launch_resid_int(const BatchDev &B, cudaStream_t st) {
  k_resid_int<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}
void launch_rhs(const BatchDev &B, cudaStream_t st) {
  k_rhs<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}
void launch_arm(const BatchDev &B, cudaStream_t st) {
  k_arm<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}
void launch_trsv_fp(const BatchDev &B, int lower, cudaStream_t st) {
  k_trsv_fp<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, lower);
}
void launch_trsv_int(const BatchDev &B, int lower, cudaStream_t st) {
  k_trsv_int<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, lower);
}
void launch_cast_v1(const BatchDev &B, cudaStream_t st) {
  k_cast_v1<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}
void launch_spmv(const BatchDev &B, int j, cudaStream_t st) {
  k_spmv<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, j);
}
void launch_mgs(const BatchDev &B, int i, int j, cudaStream_t st) {
  k_mgs<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, i, j);
}
void launch_mgs_last(const BatchDev &B, int j, cudaStream_t st) {
  k_mgs_last<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, j);
}
void launch_normalize(const BatchDev &B, int j, cudaStream_t st) {
  k_normalize<<<B.ntiles, IGM_BLOCK, 0, st>>>(B, j);
}
void launch_backsub(const BatchDev &B, cudaStream_t st) {
  k_backsub<<<nb_sys(B), 128, 0, st>>>(B);
}
void launch_update(const BatchDev &B, cudaStream_t st) {
  k_update<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}

}  // namespace igm
