// igm_api.cu -- host side of the C ABI declared in include/igm.h: handles,
// device memory arenas, batches (tile tables), and the refinement driver of
// Fig. 1, whose per-refinement launch sequence is captured once into two
// CUDA graphs (the convergence test, and one inner solve of Fig. 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "igm_host.h"

using namespace igm;

thread_local std::string g_err;

igm_status fail(igm_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

std::atomic<long long> g_launches{0};

namespace igm {
namespace {
thread_local cudaError_t t_launch_err = cudaSuccess;
}
void note_launch(cudaError_t e) {
  if (e != cudaSuccess && t_launch_err == cudaSuccess) t_launch_err = e;
}
cudaError_t take_launch_error() {
  const cudaError_t e = t_launch_err;
  t_launch_err = cudaSuccess;
  return e;
}
}  // namespace igm

namespace {

std::mutex g_batches_mu;
std::vector<Batch *> g_batches;  // cached multi-system batches

}  // namespace

// The Arnoldi step's partition of the batch's rows over the persistent CTAs
// (mgs_plan with the given snap), in its own arena, installed in b->bd.
igm_status set_plan(Batch *b, int snap) {
  const int ns = (int)b->hs.size();
  std::vector<int> sysn(ns);
  for (int s = 0; s < ns; ++s) sysn[s] = b->hs[s]->n;
  int G = 1, wrows = 0, rows = 0, ring = 0;
  std::vector<int> mptr, sys_seg;
  std::vector<Tile> mseg;
  // ring mode only where the fused kernel never runs (it keeps every
  // resident row it can)
  mgs_plan(sysn, persistent_grid(1 << 30), b->hs[0]->prm.mgs_wmax, snap, !b->fuse_ok, G, mptr,
           mseg, wrows, rows, ring, sys_seg);
  const int MS = (int)mseg.size();
  Arena a;
  int *d_mptr, *d_sysseg, *d_mact;
  Tile *d_mseg;
  long long *d_mh;
  u64 *d_mpart;
  unsigned *d_mvtag;
  a.want(&d_mptr, G + 1);
  a.want(&d_mseg, MS > 0 ? MS : 1);
  a.want(&d_mh, MS > 0 ? MS : 1);
  a.want(&d_mpart, 8 * (size_t)(MS > 0 ? MS : 1));
  a.want(&d_mact, MS > 0 ? MS : 1);
  a.want(&d_mvtag, MS > 0 ? MS : 1);
  a.want(&d_sysseg, ns + 1);
  if (a.commit() != cudaSuccess) {
    cudaGetLastError();
    return fail(IGM_EOOM, "Arnoldi plan arena");
  }
  CK(cudaMemset(d_mpart, 0, 8 * sizeof(u64) * (size_t)(MS > 0 ? MS : 1)));
  CK(cudaMemset(d_mvtag, 0, sizeof(unsigned) * (size_t)(MS > 0 ? MS : 1)));
  CK(cudaMemcpy(d_mptr, mptr.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice));
  if (MS > 0) CK(cudaMemcpy(d_mseg, mseg.data(), sizeof(Tile) * MS, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_sysseg, sys_seg.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice));
  b->plan_arena.release();
  b->plan_arena = a;
  b->snap = snap;
  BatchDev &B = b->bd;
  B.mgs_g = G;
  B.mseg_ptr = d_mptr;
  B.mseg = d_mseg;
  B.mseg_h = d_mh;
  B.nseg = MS;
  B.mpart = d_mpart;
  B.mseg_act = d_mact;
  B.mvtag = d_mvtag;
  B.sys_seg = d_sysseg;
  B.mgs_wrows = wrows;
  B.mgs_rows = rows;
  B.mgs_ring = ring;
  return IGM_OK;
}

igm_status build_batch(const std::vector<igm_handle> &hs, Batch **out) {
  Batch *b = new Batch();
  b->hs = hs;
  int ns = (int)hs.size();
  std::vector<Tile> tiles, ctiles, stiles;
  std::vector<int> snt(ns);
  std::vector<SysDev *> sp(ns);
  b->m = hs[0]->prm.m;
  b->inner = hs[0]->prm.inner;
  int maxk = 0, max_colors = 0;
  for (int s = 0; s < ns; ++s) {
    igm_handle h = hs[s];
    if (h->prm.m != b->m || h->prm.inner != b->inner) {
      delete b;
      return fail(IGM_EINVAL, "batched handles must share m and the inner solver");
    }
    b->any_ilu |= h->prm.precond;
    int first = (int)tiles.size();
    int nt = (h->n + IGM_TILE - 1) / IGM_TILE;
    for (int t = 0; t < nt; ++t)
      tiles.push_back(Tile{s, t * IGM_TILE, std::min(IGM_TILE, h->n - t * IGM_TILE), first});
    snt[s] = nt;
    sp[s] = h->d_sys;
    for (int r0 = 0; r0 < h->n; r0 += IGM_STILE)
      stiles.push_back(Tile{s, r0, std::min(IGM_STILE, h->n - r0), 0});
    int cfirst = (int)ctiles.size();
    if (h->hs.ncolors == 0)  // multicolour systems use the colour-by-colour substitutions
      for (int c = 0; c < h->hs.tri[0].nchunk; ++c) ctiles.push_back(Tile{s, c, 0, cfirst});
    max_colors = std::max(max_colors, h->hs.ncolors);
    b->max_chunk = std::max(b->max_chunk, h->hs.chunk);
    if (h->prm.precond && h->hs.ncolors == 0)
      for (int tr = 0; tr < 2; ++tr) maxk = std::max(maxk, h->hs.tri[tr].K);
  }
  int CT = (int)ctiles.size(), ST = (int)stiles.size();
  Tile *d_ctiles = nullptr, *d_stiles = nullptr;
  int T = (int)tiles.size();
  Tile *d_tiles;
  int *d_snt, *d_nact;
  SysDev **d_sp;
  long long *d_part;
  double *d_partd;
  unsigned *d_ticket, *d_bar;
  double *d_cpart;
  int maxg = persistent_grid(ST);
  b->arena.want(&d_tiles, T);
  b->arena.want(&d_ctiles, CT > 0 ? CT : 1);
  b->arena.want(&d_stiles, ST);
  b->arena.want(&d_bar, 4);
  b->arena.want(&d_cpart, 3 * (size_t)maxg * ns);
  b->arena.want(&d_snt, ns);
  b->arena.want(&d_sp, ns);
  b->arena.want(&d_part, 2 * (size_t)T);
  b->arena.want(&d_partd, T);
  b->arena.want(&d_ticket, 4);
  b->arena.want(&d_nact, 1);
  if (b->arena.commit() != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(IGM_EOOM, "batch arena");
  }
  CK(cudaMemcpy(d_tiles, tiles.data(), sizeof(Tile) * T, cudaMemcpyHostToDevice));
  if (CT > 0) CK(cudaMemcpy(d_ctiles, ctiles.data(), sizeof(Tile) * CT, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_stiles, stiles.data(), sizeof(Tile) * ST, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_snt, snt.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(d_sp, sp.data(), sizeof(SysDev *) * ns, cudaMemcpyHostToDevice));
  CK(cudaMemset(d_ticket, 0, 4 * sizeof(unsigned)));
  CK(cudaMemset(d_nact, 0, sizeof(int)));
  CK(cudaMemset(d_bar, 0, 4 * sizeof(unsigned)));
  BatchDev &B = b->bd;
  B = BatchDev{};
  B.nsys = ns;
  B.ntiles = T;
  B.nstiles = ST;
  B.stiles = d_stiles;
  B.nctiles = CT;
  B.ctiles = d_ctiles;
  B.sys = d_sp;
  B.tiles = d_tiles;
  B.sys_ntiles = d_snt;
  B.part = d_part;
  B.partd = d_partd;
  B.ticket = d_ticket;
  B.nact = d_nact;
  B.bar = d_bar;
  B.cpart = d_cpart;
  B.maxg = maxg;
  B.max_m = b->m;
  B.trsv_maxk = maxk;
  B.max_colors = max_colors;
  B.max_ns = 0;
  for (auto hh : hs) B.max_ns = std::max(B.max_ns, hh->hs.ns);
  // the fused Arnoldi kernel (line 5 inside): integer systems without
  // preconditioner and without correction terms
  b->fuse_ok = b->inner == 0 && !b->any_ilu && B.max_ns == 0;
  {
    const int snap = hs[0]->prm.plan_snap;
    igm_status st = set_plan(b, snap > 0 ? snap : 0);
    if (st) {
      delete b;
      return st;
    }
  }
  const int fs = hs[0]->prm.fuse_steps;
  B.fuse = (!b->fuse_ok || fs < 0 || mgs_one_cta(B, ns)) ? 0 : fs > 0 ? std::min(fs, b->m) : b->m;
  // launch configuration left to the autotuner (results do not depend on it)
  b->tune = b->fuse_ok && !mgs_one_cta(B, ns) && (fs == 0 || hs[0]->prm.plan_snap == 0);
  CK(cudaMallocHost((void **)&b->h_nact, sizeof(int)));
  CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  *out = b;
  return IGM_OK;
}

namespace {

// lines 1-23 of Fig. 2 after line 1's residual: (line 1') r0 = M^-1 r,
// ||r0||, cast, m Arnoldi steps, back-substitution and update
void enqueue_inner(Batch *b, cudaStream_t st) {
  const BatchDev &B = b->bd;
  if (b->inner == 1) {
    launch_fp64_inner(B, b->m, b->any_ilu, st);
    return;
  }
  if (b->any_ilu) {  // line 1'
    launch_trsv_lv(B, 1, 1, 0, st);
    launch_trsv_lv(B, 1, 0, 0, st);
  }
  launch_max(B, VEC_R, 2, st);
  launch_norm(B, VEC_R, ACT_NU, 2, st);
  launch_cast_v1(B, st);
  if (B.fuse > 0) {  // lines 5-19 of every step in persistent launches of B.fuse steps
    for (int j0 = 0; j0 < b->m; j0 += B.fuse)
      launch_mgs_fused(B, j0, std::min(b->m, j0 + B.fuse), st);
    launch_backsub(B, st);
    launch_update(B, st);
    return;
  }
  for (int j = 0; j < b->m; ++j) {
    launch_spmv(B, j, st);
    if (b->any_ilu) {  // line 5'
      launch_trsv_lv(B, 0, 1, 1, st);
      launch_trsv_lv(B, 0, 0, 1, st);
    }
    launch_mgs_step(B, j, st);
  }
  launch_backsub(B, st);
  launch_update(B, st);
}

igm_status capture_graphs(Batch *b) {
  IGM_RANGE("capture the launch graphs of Fig. 1 and Fig. 2");
  if (b->g_check && b->g_cycle) return IGM_OK;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  launch_resid(b->bd, 0, b->cap);
  launch_norm(b->bd, VEC_R, ACT_RHO, 1, b->cap);
  CK(cudaStreamEndCapture(b->cap, &g));
  CK(cudaGraphInstantiate(&b->g_check, g, 0));
  {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->nodes_check = (long long)nn;
  }
  cudaGraphDestroy(g);
  CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  launch_rhs(b->bd, b->cap);
  enqueue_inner(b, b->cap);
  CK(cudaStreamEndCapture(b->cap, &g));
  CK(cudaGraphInstantiate(&b->g_cycle, g, 0));
  {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    b->nodes_cycle = (long long)nn;
  }
  cudaGraphDestroy(g);
  return IGM_OK;
}

// Multicolour order on the host: greedy colouring of the symmetrised
// pattern (i ~ j when a_ij or a_ji is stored, i != j), rows in natural order,
// each taking the smallest colour none of its coloured neighbours has; the
// new order lists rows colour by colour, ascending within a colour.
static void mc_order_host(int n, const int *rp, const int *cl, std::vector<int> &perm,
                          std::vector<int> &cptr) {
  std::vector<int> deg(n + 1, 0);
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (cl[k] != i) {
        ++deg[i];
        ++deg[cl[k]];
      }
  std::vector<long long> ap(n + 1, 0);
  for (int i = 0; i < n; ++i) ap[i + 1] = ap[i] + deg[i];
  std::vector<int> adj(ap[n] > 0 ? ap[n] : 1), at(n, 0);
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = cl[k];
      if (j == i) continue;
      adj[ap[i] + at[i]++] = j;
      adj[ap[j] + at[j]++] = i;
    }
  std::vector<int> color(n), seen(n + 1, -1);
  int ncol = 0;
  for (int i = 0; i < n; ++i) {
    for (long long k = ap[i]; k < ap[i + 1]; ++k)
      if (adj[k] < i) seen[color[adj[k]]] = i;
    int c = 0;
    while (seen[c] == i) ++c;
    color[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  std::vector<int> start(ncol + 1, 0);
  for (int i = 0; i < n; ++i) ++start[color[i] + 1];
  for (int c = 0; c < ncol; ++c) start[c + 1] += start[c];
  cptr.assign(start.begin(), start.end());
  perm.assign(n, 0);
  for (int i = 0; i < n; ++i) perm[start[color[i]]++] = i;
}

// P A P^T on the host (rows in the new order, columns renumbered, sorted)
static void permute_host(int n, const int *rp, const int *cl, const double *v,
                         const std::vector<int> &perm, std::vector<int> &rp2,
                         std::vector<int> &cl2, std::vector<double> &v2) {
  std::vector<int> inv(n);
  for (int r = 0; r < n; ++r) inv[perm[r]] = r;
  rp2.assign(n + 1, 0);
  cl2.resize(rp[n]);
  v2.resize(rp[n]);
  std::vector<std::pair<int, double>> row;
  for (int r = 0; r < n; ++r) {
    const int o = perm[r];
    row.clear();
    for (int k = rp[o]; k < rp[o + 1]; ++k) row.emplace_back(inv[cl[k]], v[k]);
    std::sort(row.begin(), row.end(),
              [](const std::pair<int, double> &x, const std::pair<int, double> &y) {
                return x.first < y.first;
              });
    rp2[r + 1] = rp2[r] + (int)row.size();
    for (size_t q = 0; q < row.size(); ++q) {
      cl2[rp2[r] + q] = row[q].first;
      v2[rp2[r] + q] = row[q].second;
    }
  }
}

// Rows per substitution chunk.  A multiple of the matrix's row period P (for
// a natural-order stencil the grid plane, N^2 in 3D), so that chunks start
// on plane boundaries: then a chunk's first rows need only early levels of
// the previous chunk and consecutive chunks pipeline; at least 1024 rows.
// The set-up first tries `periods` planes per chunk (2 for rows of up to 8
// dependencies, 1 for longer ones: measured best on 7- and 27-point grids of
// 128^3 and 200^3) and keeps it when every chunk reads only its predecessor;
// otherwise the chunk is at least the factors' bandwidth, which guarantees
// that.  With a bandwidth too large for that (fewer than 8 chunks), about one
// chunk per SM.
// The row period of a banded matrix: among 64 rows spread over the middle
// half, the one with the most dependencies farther than half the lower
// bandwidth gives the median of those far offsets (N^2 for 7- and 27-point 3D
// stencils in natural order, N for 2D ones).  0 if there is none.
int row_period(int n, const int *rp, const int *cl, int bw) {
  if (n < 2 || bw < 2) return 0;
  std::vector<int> best;
  for (int k = 0; k < 64; ++k) {
    const int i = (int)(n / 4 + (long long)k * (n / 2) / 64);
    int ext[2];
    if (cudaMemcpy(ext, rp + i, sizeof(ext), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    std::vector<int> c(ext[1] - ext[0]);
    if (!c.empty() &&
        cudaMemcpy(c.data(), cl + ext[0], sizeof(int) * c.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
      return 0;
    std::vector<int> far;
    for (int j : c)
      if (i - j > bw / 2) far.push_back(i - j);
    if (far.size() > best.size()) best = far;
  }
  if (best.empty()) return 0;
  std::sort(best.begin(), best.end());
  return best[best.size() / 2];
}

// periods: rows per chunk in periods (planes) when the chunks only need to
// read their predecessor (checked by the caller), 0 for the bandwidth rule
int auto_chunk(int n, int bw, int P, int periods) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long r;
  if (P < 1 || P > bw) P = bw;
  if (bw >= 1 && (long long)bw * 8 <= n) {
    if (periods > 0) {
      r = (long long)periods * P;
      while (r < 1024) r += P;
    } else {
      r = P;
      while (r < bw || r < 1024) r += P;
    }
  } else {
    r = ((long long)n + sms - 1) / sms;
    r = (r + 1023) / 1024 * 1024;
  }
  if (r < 1024) r = 1024;
  if (r > (1 << 22)) r = 1 << 22;
  return (int)r;
}

igm_status check_params(const igm_params *p) {
  if (!p) return fail(IGM_EINVAL, "params is NULL");
  if (p->df < 1 || p->df > 62) return fail(IGM_EINVAL, "df out of range");
  if (p->alpha_a < 0 || p->alpha_a > 62) return fail(IGM_EINVAL, "alpha_a out of range");
  if (p->m < 1 || p->m > IGM_MAX_M) return fail(IGM_EINVAL, "m out of range");
  if (p->precond < 0 || p->precond > 2)
    return fail(IGM_EINVAL, "precond must be 0 (none), 1 (ILU(0)) or 2 (Gauss-Seidel)");
  const int b[] = {p->beta7, p->beta8, p->beta10, p->beta11a, p->beta11b, p->beta13,
                   p->beta15, p->beta16a, p->beta16b};
  for (int v : b)
    if (v < 0 || v > 62) return fail(IGM_EINVAL, "shift out of range");
  if (p->max_refine < 0 || p->max_refine > 64) return fail(IGM_EINVAL, "max_refine out of range");
  if (!(p->tol >= 0.0)) return fail(IGM_EINVAL, "tol must be >= 0");
  if (p->inner != 0 && p->inner != 1) return fail(IGM_EINVAL, "inner must be 0 or 1");
  if (p->trsv_chunk < 0) return fail(IGM_EINVAL, "trsv_chunk must be >= 0");
  if (p->s < 0 || p->s > IGM_MAX_S) return fail(IGM_EINVAL, "s must be 0 ... %d", IGM_MAX_S);
  if (p->order != 0 && p->order != 1) return fail(IGM_EINVAL, "order must be 0 or 1");
  if (p->shift_tune < 0 || p->shift_tune > 64) return fail(IGM_EINVAL, "shift_tune must be 0 ... 64");
  if (p->mgs_wmax < -1) return fail(IGM_EINVAL, "mgs_wmax must be -1, 0 or positive");
  if (p->wait_us < 0) return fail(IGM_EINVAL, "wait_us must be >= 0");
  if (p->test_stall != 0 && p->test_stall != 1) return fail(IGM_EINVAL, "test_stall must be 0 or 1");
  if (p->fuse_steps < -1) return fail(IGM_EINVAL, "fuse_steps must be -1, 0 or positive");
  if (p->plan_snap < -1 || p->plan_snap > 100)
    return fail(IGM_EINVAL, "plan_snap must be -1, 0 or 1 ... 100");
  if (!(p->trsv_cluster == 0 || p->trsv_cluster == 1 || p->trsv_cluster == 2 ||
        p->trsv_cluster == 4 || p->trsv_cluster == 8))
    return fail(IGM_EINVAL, "trsv_cluster must be 0, 1, 2, 4 or 8");
  return IGM_OK;
}

igm_status err_status(unsigned e) {
  if (e & ERR_BADCSR) return fail(IGM_EINVAL, "malformed CSR (rowptr/col)");
  if (e & ERR_ZERO_ROW) return fail(IGM_EZERO_ROW, "a row of A is zero (eq. 3)");
  if (e & ERR_ZERO_PIVOT) return fail(IGM_EZERO_PIVOT, "zero or missing ILU(0) pivot");
  if (e & ERR_CAST) return fail(IGM_EINVAL, "value out of int64 range in a cast");
  if (e & ERR_TIMEOUT) return fail(IGM_ETIMEOUT, "a bounded device wait expired");
  return IGM_OK;
}

#ifdef IGM_CHECKS
// checked builds: a failed device check (the first failing site of each
// translation unit, igm_dev.cuh CheckSite)
igm_status device_checks() {
  const unsigned m = checks_read_mgs(), t = checks_read_trsv(), v = checks_read_solve();
  if (m | t | v)
    return fail(IGM_ECUDA, "device check failed (first sites: Arnoldi %u, substitution %u, SpMV %u)",
                m, t, v);
  return IGM_OK;
}
#endif

void fill_report(const SysScal &sc, igm_report *rep) {
  if (!rep) return;
  memset(rep, 0, sizeof(*rep));
  for (int k = 0; k < IGM_EV_COUNT; ++k) rep->ev[k] = (long long)sc.ev[k];
  rep->refinements = sc.refinements;
  rep->inner_steps = sc.inner_steps;
  rep->breakdowns = sc.breakdowns;
  rep->status = sc.status;
  rep->relres = sc.rho;
  rep->relres_unscaled = sc.relres_unscaled;
  memcpy(rep->gamma_hist, sc.gamma_hist, sizeof rep->gamma_hist);
  memcpy(rep->relres_hist, sc.relres_hist, sizeof rep->relres_hist);
  rep->shift_retries = sc.retries;
  for (int t = 0; t < 5; ++t) rep->beta_final[t] = sc.beta[t];
}

}  // namespace

igm_status load_vec(igm_handle h, double *dst, const double *src, cudaStream_t s) {
  if (!h->perm) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * h->n, cudaMemcpyDefault, s));
    return IGM_OK;
  }
  CK(cudaMemcpyAsync(h->ptmp, src, sizeof(double) * h->n, cudaMemcpyDefault, s));
  launch_permute(h->n, h->perm, h->ptmp, dst, 0, s);
  CKL();
  return IGM_OK;
}

igm_status store_vec(igm_handle h, double *dst, const double *src, cudaStream_t s) {
  if (!h->perm) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * h->n, cudaMemcpyDefault, s));
    return IGM_OK;
  }
  launch_permute(h->n, h->perm, src, h->ptmp, 1, s);
  CKL();
  CK(cudaMemcpyAsync(dst, h->ptmp, sizeof(double) * h->n, cudaMemcpyDefault, s));
  return IGM_OK;
}

extern "C" {

const char *igm_last_error(void) { return g_err.c_str(); }
const char *igm_version(void) { return "igm-gb300 0.1 (sm_103a)"; }

igm_status igm_params_default(igm_params *p, int precond, int m) {
  if (!p) return fail(IGM_EINVAL, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->df = 30;
  p->m = m;
  p->precond = precond;
  p->tol = 1e-10;
  p->max_refine = 60;
  if (precond) {  // Table 5
    p->alpha_a = 32;
    p->beta7 = p->beta8 = p->beta10 = 0;
    p->beta11a = 30;
    p->beta11b = 0;
    p->beta13 = p->beta15 = 0;
    p->beta16a = 30;
    p->beta16b = 0;
  } else {  // Table 4
    p->alpha_a = 16;
    p->beta7 = p->beta8 = p->beta10 = 16;
    p->beta11a = 16;
    p->beta11b = 14;
    p->beta13 = p->beta15 = 16;
    p->beta16a = 16;
    p->beta16b = 14;
  }
  return IGM_OK;
}

igm_status int_gmres_setup(int n, int nnz, const int *rowptr, const int *col,
                           const double *val, const igm_params *params, void *stream,
                           igm_handle *out) {
  g_err.clear();
  IGM_RANGE("int_gmres_setup: scaling, cast, ILU(0) (Sec. III, IV-B, VI-A)");
  if (!out) return fail(IGM_EINVAL, "out is NULL");
  *out = nullptr;
  igm_status st = check_params(params);
  if (st) return st;
  if (n < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)))
    return fail(IGM_EINVAL, "bad sizes or NULL arrays");
  cudaStream_t s = (cudaStream_t)stream;
  // multicolour order: the whole set-up works on P A P^T, built on the host
  std::vector<int> mc_perm, mc_cptr, mc_rp, mc_cl;
  std::vector<double> mc_v;
  if (params->order == 1) {
    std::vector<int> hr(n + 1), hc(nnz > 0 ? nnz : 1);
    std::vector<double> hv(nnz > 0 ? nnz : 1);
    if (cudaMemcpy(hr.data(), rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault) != cudaSuccess ||
        (nnz > 0 && (cudaMemcpy(hc.data(), col, sizeof(int) * nnz, cudaMemcpyDefault) !=
                         cudaSuccess ||
                     cudaMemcpy(hv.data(), val, sizeof(double) * nnz, cudaMemcpyDefault) !=
                         cudaSuccess))) {
      cudaGetLastError();
      return fail(IGM_EINVAL, "the CSR arrays are not readable");
    }
    if (hr[0] != 0 || hr[n] != nnz) return fail(IGM_EINVAL, "rowptr[0] must be 0 and rowptr[n] must be nnz");
    for (int i = 0; i < n; ++i) {
      if (hr[i + 1] < hr[i]) return fail(IGM_EINVAL, "rowptr must be non-decreasing");
      for (int k = hr[i]; k < hr[i + 1]; ++k)
        if (hc[k] < 0 || hc[k] >= n) return fail(IGM_EINVAL, "column index out of range");
    }
    mc_order_host(n, hr.data(), hc.data(), mc_perm, mc_cptr);
    permute_host(n, hr.data(), hc.data(), hv.data(), mc_perm, mc_rp, mc_cl, mc_v);
    rowptr = mc_rp.data();
    col = mc_cl.data();
    val = mc_v.data();
  }
  igm_handle h = new igm_handle_s();
  h->n = n;
  h->nnz = nnz;
  h->prm = *params;
  const int m = params->m, ilu = params->precond;
  SysDev &d = h->hs;
  int *rp, *cl, *dp, *lfl = nullptr, *ufl = nullptr;
  double *ahat, *a, *dd, *f = nullptr, *b, *bh, *xt, *r, *t, *xk, *yfp;
  i64 *abar, *fac = nullptr, *ld = nullptr, *ud = nullptr, *w, *yv, *V, *H, *cs, *sn, *g;
  int *V32;
  int *bwd = nullptr;
  size_t nz = nnz > 0 ? nnz : 1;
  // the row pointers on the host: checked here (monotone, 0 .. nnz) and used
  // for the sizes of the SELL-32 slices
  std::vector<int> hrp(n + 1);
  if (cudaMemcpy(hrp.data(), rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(IGM_EINVAL, "rowptr is not readable");
  }
  if (hrp[0] != 0 || hrp[n] != nnz) {
    delete h;
    return fail(IGM_EINVAL, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  }
  const int nsl = (n + 31) / 32;
  std::vector<long long> hsp(nsl + 1, 0);
  for (int sl = 0; sl < nsl; ++sl) {
    int len = 0;
    for (int r = 32 * sl; r < std::min(n, 32 * sl + 32); ++r) {
      if (hrp[r + 1] < hrp[r]) {
        delete h;
        return fail(IGM_EINVAL, "rowptr must be non-decreasing");
      }
      len = std::max(len, hrp[r + 1] - hrp[r]);
    }
    hsp[sl + 1] = hsp[sl] + 32ll * len;
  }
  const size_t nzs = hsp[nsl] > 0 ? (size_t)hsp[nsl] : 1;
  const int S = params->s;  // correction terms requested (eq. AA)
  long long *sptr;
  i64 *sval;
  int *scol;
  double *mtR = nullptr;
  unsigned long long *mtmax = nullptr;
  Arena &A = h->arena;
  A.want(&sptr, nsl + 1);
  A.want(&sval, nzs * (S + 1));
  A.want(&scol, nzs);
  if (S > 0) {
    A.want(&mtR, nz);
    A.want(&mtmax, 1);
  }
  A.want(&rp, n + 1);
  A.want(&cl, nz);
  A.want(&dp, n);
  A.want(&ahat, nz);
  A.want(&a, nz);
  A.want(&dd, n);
  A.want(&abar, nz * (S + 1));
  if (ilu) {
    A.want(&f, nz);
    A.want(&fac, nz);
    A.want(&ld, n);
    A.want(&ud, n);
    A.want(&lfl, n);
    A.want(&ufl, n);
    A.want(&bwd, 4);
  }
  A.want(&b, n);
  A.want(&bh, n);
  A.want(&xt, n);
  A.want(&r, n);
  A.want(&t, n);
  A.want(&xk, n);
  A.want(&w, n);
  A.want(&yv, n);
  A.want(&V, (size_t)(m + 1) * n);
  A.want(&V32, (size_t)(m + 1) * n + 4);  // + the tail of a 16-byte copy
  A.want(&H, (size_t)(m + 1) * m);
  A.want(&cs, m);
  A.want(&sn, m);
  A.want(&g, m + 1);
  A.want(&yfp, m);
  A.want(&h->d_sys, 1);
  A.want(&h->d_sc, 1);
  A.want(&h->d_err, 4);
  int *dcptr = nullptr;
  if (params->order == 1) {
    A.want(&h->perm, n);
    A.want(&h->ptmp, n);
    A.want(&dcptr, mc_cptr.size());
  }
  if (A.commit() != cudaSuccess) {
    cudaGetLastError();
    size_t need = A.total();
    delete h;
    return fail(IGM_EOOM, "device allocation of %zu bytes failed", need);
  }
#define CKH(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      cudaGetLastError();                                                         \
      int_gmres_destroy(h);                                                       \
      return fail(IGM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
    }                                                                             \
  } while (0)
  CKH(cudaMemsetAsync(h->d_err, 0, 4 * sizeof(unsigned), s));
  if (h->perm) {
    CKH(cudaMemcpyAsync(h->perm, mc_perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CKH(cudaMemcpyAsync(dcptr, mc_cptr.data(), sizeof(int) * mc_cptr.size(),
                        cudaMemcpyHostToDevice, s));
  }
  CKH(cudaMemsetAsync(h->d_sc, 0, sizeof(SysScal), s));
  CKH(cudaMemcpyAsync(rp, rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault, s));
  if (nnz > 0) {
    CKH(cudaMemcpyAsync(cl, col, sizeof(int) * nnz, cudaMemcpyDefault, s));
    CKH(cudaMemcpyAsync(ahat, val, sizeof(double) * nnz, cudaMemcpyDefault, s));
  }
  int h_rp[2];
  CKH(cudaMemcpyAsync(h_rp, rp, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKH(cudaMemcpyAsync(h_rp + 1, rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKH(cudaStreamSynchronize(s));
  if (h_rp[0] != 0 || h_rp[1] != nnz) {
    int_gmres_destroy(h);
    return fail(IGM_EINVAL, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  }
  unsigned *err = h->d_err;
  launch_validate(n, nnz, rp, cl, dp, err, s);
  unsigned herr = 0;
  CKH(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CKH(cudaStreamSynchronize(s));
  if (herr) {  // a malformed CSR goes no further
    igm_status e = err_status(herr);
    int_gmres_destroy(h);
    return e;
  }
  launch_scale(n, rp, ahat, params->alpha_a, a, dd, err, s);
  launch_cast(nnz, a, abar, err, s);
  // eq. (alpha1), (A): the correction terms, each from the exact FP64
  // remainder of the previous ones; fewer than S when a remainder is zero
  int ns = 0, alphas[IGM_MAX_S + 1] = {0};
  if (S > 0 && nnz > 0) {
    launch_mt_init(nnz, a, abar, mtR, s);
    for (int l = 1; l <= S; ++l) {
      unsigned long long hmx = 0;
      CKH(cudaMemsetAsync(mtmax, 0, sizeof(unsigned long long), s));
      launch_mt_max(nnz, mtR, mtmax, s);
      CKH(cudaMemcpyAsync(&hmx, mtmax, sizeof(hmx), cudaMemcpyDeviceToHost, s));
      CKH(cudaStreamSynchronize(s));
      double mx;
      std::memcpy(&mx, &hmx, sizeof(mx));
      if (mx == 0.0) break;
      alphas[l] = params->alpha_a - std::ilogb(mx);
      launch_mt_term(nnz, mtR, alphas[l], abar + (size_t)l * nnz, s);
      ns = l;
    }
  }
  CKH(cudaMemcpyAsync(sptr, hsp.data(), sizeof(long long) * (nsl + 1), cudaMemcpyHostToDevice, s));
  for (int l = 0; l <= ns; ++l)
    launch_sell_fill(n, nsl, rp, cl, abar + (size_t)l * nnz, sptr, sval + (size_t)l * nzs, scol, s);
  CKH(cudaGetLastError());
  CKH(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CKH(cudaStreamSynchronize(s));
  if (herr) {
    igm_status e = err_status(herr);
    int_gmres_destroy(h);
    return e;
  }
  int R = 0, nch = 0, single = 0;
  i64 *xbuf = nullptr;
  if (ilu) {
    // a stored diagonal is required by ILU(0)
    std::vector<int> hdp(n);
    CKH(cudaMemcpy(hdp.data(), dp, sizeof(int) * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i)
      if (hdp[i] < 0) {
        int_gmres_destroy(h);
        return fail(IGM_EZERO_PIVOT, "row %d has no stored diagonal (ILU(0))", i);
      }
    // bandwidths and longest strict rows of the two triangles
    int hbw[4] = {0, 0, 0, 0};
    CKH(cudaMemsetAsync(bwd, 0, 4 * sizeof(int), s));
    launch_bandwidth(n, rp, cl, bwd, s);
    CKH(cudaMemcpyAsync(hbw, bwd, sizeof(hbw), cudaMemcpyDeviceToHost, s));
    CKH(cudaStreamSynchronize(s));
    const int bw = std::max(hbw[0], hbw[1]);
    // single: every chunk of both factors reads only itself and its
    // predecessor (exact check over all dependencies)
    auto reads_pred_only = [&](int Rc, int &res) -> igm_status {
      int hcd[2] = {0, 0};
      CK(cudaMemsetAsync(bwd, 0, 2 * sizeof(int), s));
      launch_chunkdist(n, rp, cl, dp, 1, Rc, bwd, s);
      launch_chunkdist(n, rp, cl, dp, 0, Rc, bwd + 1, s);
      CK(cudaMemcpyAsync(hcd, bwd, sizeof(hcd), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      res = std::max(hcd[0], hcd[1]) <= 1 ? 1 : 0;
      return IGM_OK;
    };
    if (params->trsv_chunk > 0) {
      R = params->trsv_chunk;
    } else {
      const int P = row_period(n, rp, cl, hbw[0]);
      R = auto_chunk(n, bw, P, std::max(hbw[2], hbw[3]) > 8 ? 1 : 2);
      int ok = 0;
      if (reads_pred_only(R, ok) != IGM_OK) {
        int_gmres_destroy(h);
        return IGM_ECUDA;
      }
      if (!ok) R = auto_chunk(n, bw, P, 0);
    }
    nch = (n + R - 1) / R;
    if (reads_pred_only(R, single) != IGM_OK) {
      int_gmres_destroy(h);
      return IGM_ECUDA;
    }
    // the predecessor copies read up to one position past the last (their
    // 16-byte rounding)
    const int npad = (n + 4 + 3) & ~3;
    // the schedules of L (t = 0) and U (t = 1)
    const int fp = params->inner == 1;
    Arena &A2 = h->arena2;
    int *ord[2], *lptr[2], *levb[2], *lev[2], *need[2], *posof[2], *chmax, *cnt;
    u64 *prog[2];
    for (int tr = 0; tr < 2; ++tr) {
      A2.want(&ord[tr], n);
      A2.want(&lptr[tr], n + 1);
      A2.want(&levb[tr], nch + 1);
      A2.want(&lev[tr], n);
      A2.want(&need[tr], n + 1);
      A2.want(&posof[tr], n);
      A2.want(&prog[tr], (size_t)nch * IGM_PROG_STRIDE);
    }
    A2.want(&chmax, std::max(nch, 4));  // also two 64-bit maxima
    A2.want(&cnt, n + 1);
    A2.want(&xbuf, npad);
    if (A2.commit() != cudaSuccess) {
      cudaGetLastError();
      size_t need2 = A2.total();
      int_gmres_destroy(h);
      return fail(IGM_EOOM, "device allocation of %zu bytes failed", need2);
    }
    // chunk-local levels and (chunk, level) orders of the two factors, with
    // levels wider than the kernel's slots split into several groups
    unsigned *tick = (unsigned *)(h->d_err + 1);
    int *flg[2] = {lfl, ufl};
    std::vector<int> hmax(nch), hlevb(nch + 1), hlevb2(nch + 1), hl, nl, nb;
    std::vector<int> gw[2];  // the width of every group of each factor
    int pring_ok[2] = {1, 1};
    for (int tr = 0; tr < 2; ++tr) {
      const int lower = tr == 0;
      const int K = hbw[2 + tr];
      CKH(cudaMemsetAsync(flg[tr], 0, sizeof(int) * n, s));
      CKH(cudaMemsetAsync(tick, 0, sizeof(unsigned), s));
      CKH(cudaMemsetAsync(chmax, 0, sizeof(int) * nch, s));
      launch_levels(n, rp, cl, dp, lower, R, lev[tr], flg[tr], 1, tick, chmax, err, s);
      CKH(cudaMemcpyAsync(hmax.data(), chmax, sizeof(int) * nch, cudaMemcpyDeviceToHost, s));
      CKH(cudaStreamSynchronize(s));
      hlevb[0] = 0;
      for (int c = 0; c < nch; ++c) hlevb[c + 1] = hlevb[c] + hmax[c] + 1;
      const int L = hlevb[nch];
      CKH(cudaMemcpyAsync(levb[tr], hlevb.data(), sizeof(int) * (nch + 1),
                          cudaMemcpyHostToDevice, s));
      CKH(cudaMemsetAsync(cnt, 0, sizeof(int) * (L + 1), s));
      launch_level_order(n, lower, R, L, lev[tr], levb[tr], cnt, lptr[tr], ord[tr], s);
      // split the levels wider than the cap into consecutive groups
      hl.resize(L + 1);
      CKH(cudaMemcpyAsync(hl.data(), lptr[tr], sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, s));
      CKH(cudaStreamSynchronize(s));
      const int cap = trsv_group_cap(K);
      nb.assign(L, 0);
      nl.clear();
      int maxw = 1, maxlev = 1;
      for (int c = 0; c < nch; ++c) {
        hlevb2[c] = (int)nl.size();
        for (int g = hlevb[c]; g < hlevb[c + 1]; ++g) {
          nb[g] = (int)nl.size();
          const int w = hl[g + 1] - hl[g];
          for (int t0 = 0; t0 < w; t0 += cap) {
            nl.push_back(hl[g] + t0);
            maxw = std::max(maxw, std::min(cap, w - t0));
          }
        }
        maxlev = std::max(maxlev, (int)nl.size() - hlevb2[c]);
      }
      hlevb2[nch] = (int)nl.size();
      nl.push_back(n);
      const int L2 = hlevb2[nch];
      gw[tr].resize(L2);
      for (int g = 0; g < L2; ++g) gw[tr][g] = nl[g + 1] - nl[g];
      CKH(cudaMemcpyAsync(cnt, nb.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
      CKH(cudaMemcpyAsync(need[tr], hlevb2.data(), sizeof(int) * (nch + 1), cudaMemcpyHostToDevice,
                          s));
      launch_regroup(n, R, ord[tr], lev[tr], levb[tr], lptr[tr], cnt, need[tr], cap, posof[tr], s);
      CKH(cudaMemcpyAsync(lptr[tr], nl.data(), sizeof(int) * (L2 + 1), cudaMemcpyHostToDevice, s));
      CKH(cudaMemcpyAsync(levb[tr], hlevb2.data(), sizeof(int) * (nch + 1), cudaMemcpyHostToDevice,
                          s));
      CKH(cudaMemsetAsync(need[tr], 0, sizeof(int) * (L2 + 1), s));
      launch_need(n, rp, cl, dp, lower, R, ord[tr], levb[tr], lev[tr], need[tr], s);
      // the value ring: the farthest same-chunk dependency; the predecessor
      // ring: the span between the copies' front and the oldest value read
      int hd[2] = {0, 0};
      CKH(cudaMemsetAsync(bwd + 2, 0, 2 * sizeof(int), s));
      launch_ringdist(n, rp, cl, dp, lower, R, ord[tr], posof[tr], lev[tr], levb[tr], lptr[tr],
                      bwd + 2, s);
      std::vector<int> hneed(L2 + 1);
      CKH(cudaMemcpyAsync(hneed.data(), need[tr], sizeof(int) * (L2 + 1), cudaMemcpyDeviceToHost,
                          s));
      CKH(cudaStreamSynchronize(s));
      for (int c = 0; c < nch; ++c)
        for (int g = hlevb2[c] + 1; g < hlevb2[c + 1]; ++g) hneed[g] = std::max(hneed[g], hneed[g - 1]);
      CKH(cudaMemcpyAsync(cnt, hneed.data(), sizeof(int) * L2, cudaMemcpyHostToDevice, s));
      if (single)
        launch_pringdist(n, rp, cl, dp, lower, R, ord[tr], posof[tr], lev[tr], levb[tr], lptr[tr],
                         cnt, bwd + 3, s);
      CKH(cudaMemcpyAsync(hd, bwd + 2, sizeof(hd), cudaMemcpyDeviceToHost, s));
      CKH(cudaMemsetAsync(prog[tr], 0, sizeof(u64) * nch * IGM_PROG_STRIDE, s));
      CKH(cudaStreamSynchronize(s));
      auto pow2 = [](int v) {
        int r = 2;
        while (r < v && r < IGM_TRSV_RING_MAX) r <<= 1;
        return r;
      };
      // farther dependencies are read late (same chunk) or late after the
      // waiter's wait (previous chunk, when its ring would be too large)
      pring_ok[tr] = hd[1] <= IGM_TRSV_RING_MAX;
      Tri &T = d.tri[tr];
      T.ord = ord[tr];
      T.lptr = lptr[tr];
      T.levb = levb[tr];
      T.lev = lev[tr];
      T.need = need[tr];
      T.prog = prog[tr];
      T.nchunk = nch;
      T.K = K;
      T.maxlev = maxlev;
      T.maxw = maxw;
      T.ring = pow2(hd[0]);
      T.pring = pow2(hd[1]);
    }
    // the groups' packed blocks, sized for 8-byte factors (int32 factors,
    // decided after the factorisation, use less), and their offsets
    unsigned char *blob[2], *blobd[2] = {nullptr, nullptr};
    long long *boff[2], *boffd[2] = {nullptr, nullptr};
    {
      Arena &A3 = h->arena3;
      for (int tr = 0; tr < 2; ++tr) {
        size_t tot = 0;
        for (int w : gw[tr]) tot += trsv_blk_bytes(trsv_wp(w), d.tri[tr].K, 8);
        A3.want(&blob[tr], tot + 16);
        A3.want(&boff[tr], gw[tr].size() + 1);
        if (fp) {
          A3.want(&blobd[tr], tot + 16);
          A3.want(&boffd[tr], gw[tr].size() + 1);
        }
      }
      if (A3.commit() != cudaSuccess) {
        cudaGetLastError();
        size_t need3 = A3.total();
        int_gmres_destroy(h);
        return fail(IGM_EOOM, "device allocation of %zu bytes failed", need3);
      }
    }
    // eq. (ilu) on the L schedule (epoch 2), or the Gauss-Seidel factor
    // form; then the integer factors
    if (params->precond == 2) {
      launch_gs_factors(n, rp, cl, dp, a, f, err, s);
    } else {
      CKH(cudaMemcpyAsync(f, a, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
      CKH(cudaMemsetAsync(tick, 0, sizeof(unsigned), s));
      launch_ilu0_lv(n, rp, cl, dp, d.tri[0], R, single, f, tick, 2, err, s);
    }
    launch_ilu_int(n, rp, cl, dp, f, fac, ld, ud, err, s);
    // factors that fit pack as int32 (half the bytes, cheaper products)
    {
      unsigned long long *fmx = reinterpret_cast<unsigned long long *>(chmax);
      unsigned long long hfm[2] = {0, 0};
      CKH(cudaMemsetAsync(fmx, 0, 2 * sizeof(unsigned long long), s));
      launch_facmax(n, rp, dp, 1, fac, fmx, s);
      launch_facmax(n, rp, dp, 0, fac, fmx + 1, s);
      CKH(cudaMemcpyAsync(hfm, fmx, sizeof(hfm), cudaMemcpyDeviceToHost, s));
      CKH(cudaStreamSynchronize(s));
      for (int tr = 0; tr < 2; ++tr) d.tri[tr].fac32 = hfm[tr] < (1ull << 31) ? 1 : 0;
    }
    std::vector<long long> hoff[2];
    for (int tr = 0; tr < 2; ++tr) {
      Tri &T = d.tri[tr];
      const int ng = (int)gw[tr].size();
      hoff[tr].assign(ng + 1, 0);
      for (int g = 0; g < ng; ++g)
        hoff[tr][g + 1] = hoff[tr][g] + trsv_blk_bytes(trsv_wp(gw[tr][g]), T.K, T.fac32 ? 4 : 8);
      CKH(cudaMemcpyAsync(boff[tr], hoff[tr].data(), sizeof(long long) * (ng + 1),
                          cudaMemcpyHostToDevice, s));
      CKH(cudaMemsetAsync(blob[tr], 0, hoff[tr][ng] + 16, s));
      if (fp) {
        std::vector<long long> hd8(ng + 1, 0);
        for (int g = 0; g < ng; ++g) hd8[g + 1] = hd8[g] + trsv_blk_bytes(trsv_wp(gw[tr][g]), T.K, 8);
        CKH(cudaMemcpyAsync(boffd[tr], hd8.data(), sizeof(long long) * (ng + 1),
                            cudaMemcpyHostToDevice, s));
        CKH(cudaMemsetAsync(blobd[tr], 0, hd8[ng] + 16, s));
        CKH(cudaStreamSynchronize(s));  // hd8 leaves scope
      }
      launch_pack(n, rp, cl, dp, tr == 0, T.K, R, single && pring_ok[tr], T.ring, T.pring,
                  T.fac32, ord[tr], posof[tr], lev[tr], levb[tr], lptr[tr], boff[tr], boffd[tr],
                  fac, ld, ud, f, blob[tr], blobd[tr], s);
      T.blob = blob[tr];
      T.blobd = blobd[tr];
      T.boff = boff[tr];
      T.boffd = boffd[tr];
    }
    CKH(cudaGetLastError());
    CKH(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CKH(cudaStreamSynchronize(s));
    if (herr) {
      igm_status e = err_status(herr);
      int_gmres_destroy(h);
      return e;
    }
  }
  d.n = n;
  d.nnz = nnz;
  d.ld = m + 1;
  d.p = SysParams{params->df,     params->alpha_a, m,                params->precond,
                  params->beta7,  params->beta8,   params->beta10,   params->beta11a,
                  params->beta11b, params->beta13, params->beta15,   params->beta16a,
                  params->beta16b, params->inner,  params->max_refine, params->tol,
                  params->shift_tune, params->test_stall,
                  params->wait_us > 0 ? 1000ull * (u64)params->wait_us : 1000000000ull};
  {
    const int b0[5] = {params->beta7, params->beta8, params->beta10, params->beta13,
                       params->beta15};
    for (int t = 0; t < 5; ++t) d.beta0[t] = b0[t];
  }
  d.rowptr = rp;
  d.col = cl;
  d.diagpos = dp;
  d.ahat = ahat;
  d.a = a;
  d.d = dd;
  d.abar = abar;
  d.sptr = sptr;
  d.sval = sval;
  d.scol = scol;
  d.nnz_sell = (long long)nzs;
  d.ncolors = (params->order == 1 && ilu) ? (int)mc_cptr.size() - 1 : 0;
  d.cptr = dcptr;
  d.ns = ns;
  for (int l = 0; l <= IGM_MAX_S; ++l) d.alphas[l] = alphas[l];
  d.f = f;
  d.fac = fac;
  d.ldiag = ld;
  d.udiag = ud;
  d.chunk = R;
  d.xbuf = xbuf;
  d.single_pred = single;
  d.lflag = lfl;
  d.uflag = ufl;
  d.b = b;
  d.bh = bh;
  d.xt = xt;
  d.r = r;
  d.t = t;
  d.xk = xk;
  d.w = w;
  d.yv = yv;
  d.V = V;
  d.V32 = V32;
  d.H = H;
  d.cs = cs;
  d.sn = sn;
  d.g = g;
  d.yfp = yfp;
  d.sc = h->d_sc;
  CKH(cudaMemcpyAsync(h->d_sys, &d, sizeof(SysDev), cudaMemcpyHostToDevice, s));
  // epochs 1 and 2 were used by the level and ILU(0) kernels
  int seq0 = 2;
  CKH(cudaMemcpyAsync(&h->d_sc->seq, &seq0, sizeof(int), cudaMemcpyHostToDevice, s));
  CKH(cudaMemsetAsync(H, 0, sizeof(i64) * (size_t)(m + 1) * m, s));
  CKH(cudaMemsetAsync(V, 0, sizeof(i64) * (size_t)(m + 1) * n, s));
  CKH(cudaMemsetAsync(V32, 0, sizeof(int) * (size_t)(m + 1) * n, s));
  CKH(cudaStreamSynchronize(s));
  igm_status bs = build_batch({h}, &h->solo);
  if (bs) {
    int_gmres_destroy(h);
    return bs;
  }
  *out = h;
  return IGM_OK;
#undef CKH
}

void int_gmres_destroy(igm_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> lk(g_batches_mu);
    for (size_t k = 0; k < g_batches.size();) {
      Batch *b = g_batches[k];
      if (std::find(b->hs.begin(), b->hs.end(), h) != b->hs.end()) {
        delete b;
        g_batches.erase(g_batches.begin() + k);
      } else {
        ++k;
      }
    }
  }
  delete h->solo;
  h->arena.release();
  h->arena2.release();
  h->arena3.release();
  delete h;
}

long long int_gmres_device_bytes(igm_handle h) {
  return h ? (long long)(h->arena.size + h->arena2.size + h->arena3.size) : 0;
}

}  // extern "C"

// ---- helpers shared with the serving runtime ------------------------------

// Fig. 1 set-up of every system of a batch: state reset, b = D^-1 bh, x = 0,
// ||b|| and ||bh||
igm_status ir_init_host(Batch *b, cudaStream_t s) {
  const BatchDev &B = b->bd;
  launch_init_scal(B, 0, s);
  launch_init_ir(B, s);
  launch_max(B, VEC_B, 0, s);
  launch_norm(B, VEC_B, ACT_NB, 0, s);
  launch_max(B, VEC_BH, 0, s);
  launch_norm(B, VEC_BH, ACT_NBH, 0, s);
  CKL();
  g_launches += 6;
  return IGM_OK;
}

// residual of the original system, for the report
igm_status ir_finish_host(Batch *b, cudaStream_t s) {
  launch_resid(b->bd, 1, s);
  launch_norm(b->bd, VEC_R, ACT_UNSC, 0, s);
  CKL();
  g_launches += 2;
  return IGM_OK;
}

void enqueue_inner_host(Batch *b, cudaStream_t st) { enqueue_inner(b, st); }

// device bytes int_gmres_setup will hold for a system (an upper estimate of
// the arena: every buffer rounded up to 256 bytes)
long long handle_bytes_estimate(int n, int nnz, const igm_params *p) {
  long long N = n, Z = nnz > 0 ? nnz : 1, m = p->m, r = 0;
  r += 4 * (N + 1) + 4 * Z + 4 * N;                 // rowptr, col, diagpos
  r += 8 * Z * 3 + 8 * N;                           // ahat, a, abar, d
  r += 12 * Z + 12 * N + N / 4 + 8;                 // SELL-32 copy of abar (estimate)
  r += (long long)p->s * (16 * Z + 8 * N) + (p->s > 0 ? 8 * Z : 0);  // correction terms
  if (p->precond) {
    r += 8 * Z * 2 + 8 * N * 2 + 4 * N * 8 + 16 * N + 8 * N;
    // the substitutions' packed group blocks, both triangles: per row 12
    // bytes a strict entry (row length bounded by the mean, rounded up, plus
    // the padding of the longest rows) and 24 bytes of row data; the FP64
    // comparison solver keeps an FP64 copy
    const long long K = (Z + N - 1) / N + 4;
    r += 2 * N * (12 * K + 24) + (p->inner == 1 ? 2 * N * (8 * K + 8) : 0);
  }
  r += 8 * N * 8 + 12 * N * (m + 1) + 8 * (m + 1) * m + 8 * 4 * (m + 1);
  return r + 64 * 256 + (long long)sizeof(SysScal) + sizeof(SysDev);
}

namespace {

// Fig. 1 over a batch: b = D^-1 bh, norms, then {test, inner solve} until
// every system has converged or reached max_refine.
// device error flags of a batch (the grid kernels report in the first
// system's flags)
igm_status check_errors(Batch *b, cudaStream_t s) {
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, &b->hs[0]->d_sc->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
#ifdef IGM_CHECKS
  if (igm_status c = device_checks()) return c;
#endif
  return e ? err_status(e) : IGM_OK;
}

// The autotuner: for every launch configuration left open (plan snap,
// steps per fused launch), set up the first inner solve of Fig. 1 from the
// loaded right-hand sides (x = 0) and time its m Arnoldi steps (lines 5-19)
// with CUDA events; keep the fastest.  The integer results are the same for
// every configuration, and the refinement loop that follows starts again
// from its own set-up (k_init_scal resets every counter the trial touched).
igm_status tune_batch(Batch *b, cudaStream_t s) {
  if (!b->tune) return IGM_OK;
  IGM_RANGE("autotuner: Arnoldi launch configuration");
  b->tune = false;
  const igm_params &P = b->hs[0]->prm;
  const int m = b->m, ns = (int)b->hs.size();
  std::vector<int> snaps, fuses;
  if (P.plan_snap == 0) snaps = {0, 25, 50};
  else snaps = {P.plan_snap > 0 ? P.plan_snap : 0};
  if (P.fuse_steps == 0) {
    for (int f : {m, (m + 1) / 2, 10, 5, 0})
      if (std::find(fuses.begin(), fuses.end(), std::min(f, m)) == fuses.end())
        fuses.push_back(std::min(f, m));
  } else {
    fuses = {P.fuse_steps < 0 ? 0 : std::min(P.fuse_steps, m)};
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_snap = b->snap, best_fuse = b->bd.fuse;
  igm_status st = IGM_OK;
  for (int snap : snaps) {
    if (snap != b->snap && (st = set_plan(b, snap))) break;
    const BatchDev &B = b->bd;
    if (mgs_one_cta(B, ns)) continue;
    for (int f : fuses) {
      b->bd.fuse = f;
      if ((st = ir_init_host(b, s))) break;
      launch_resid(B, 0, s);
      launch_norm(B, VEC_R, ACT_RHO, 1, s);
      launch_rhs(B, s);
      launch_max(B, VEC_R, 2, s);
      launch_norm(B, VEC_R, ACT_NU, 2, s);
      launch_cast_v1(B, s);
      CK(cudaEventRecord(e0, s));
      if (f > 0) {
        for (int j0 = 0; j0 < m; j0 += f) launch_mgs_fused(B, j0, std::min(m, j0 + f), s);
      } else {
        for (int j = 0; j < m; ++j) {
          launch_spmv(B, j, s);
          launch_mgs_step(B, j, s);
        }
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      CKL();
      if ((st = check_errors(b, s))) break;
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_snap = snap;
        best_fuse = f;
      }
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if (best_snap != b->snap && (st = set_plan(b, best_snap))) return st;
  b->bd.fuse = mgs_one_cta(b->bd, ns) ? 0 : best_fuse;
  // the captured graphs hold the batch descriptor by value
  if (b->g_check) cudaGraphExecDestroy(b->g_check);
  if (b->g_cycle) cudaGraphExecDestroy(b->g_cycle);
  b->g_check = b->g_cycle = nullptr;
  return IGM_OK;
}

igm_status run_ir(Batch *b, cudaStream_t s) {
  const BatchDev &B = b->bd;
  igm_status st = tune_batch(b, s);
  if (st) return st;
  for (igm_handle h : b->hs) {
    h->ran_fuse = B.fuse;
    h->ran_snap = b->snap;
  }
  st = capture_graphs(b);
  if (st) return st;
  st = ir_init_host(b, s);
  if (st) return st;
  int maxr = 0;  // refinements plus the inner solves auto-tuning may discard
  for (auto h : b->hs) maxr = std::max(maxr, h->prm.max_refine + h->prm.shift_tune);
  for (int k = 0; k <= maxr + 1; ++k) {
    IGM_RANGE("refinement: Fig. 1 test, then one Fig. 2 inner solve");
    CK(cudaGraphLaunch(b->g_check, s));
    g_launches += b->nodes_check;
    CK(cudaMemcpyAsync(b->h_nact, B.nact, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*b->h_nact == 0) break;
    CK(cudaGraphLaunch(b->g_cycle, s));
    g_launches += b->nodes_cycle;
  }
  return ir_finish_host(b, s);
}

}  // namespace

igm_status collect_host(igm_handle h, igm_report *rep, cudaStream_t s) {
  SysScal sc;
  unsigned e = 0;
  CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(SysScal), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  e = sc.err;
  fill_report(sc, rep);
  if (rep) {
    rep->fuse_steps = h->ran_fuse;
    rep->plan_snap = h->ran_snap;
  }
#ifdef IGM_CHECKS
  if (igm_status c = device_checks()) {
    if (rep) rep->status = c;
    return c;
  }
#endif
  if (e) {
    igm_status st = err_status(e);
    if (rep) rep->status = st;
    return st;
  }
  if (sc.status == IGM_ENOCONV) return fail(IGM_ENOCONV, "max_refine reached at relres %.3e", sc.rho);
  return IGM_OK;
}

extern "C" {

igm_status ir_solve(igm_handle h, const double *bhat, double *xhat, igm_report *rep,
                    void *stream) {
  g_err.clear();
  IGM_RANGE("ir_solve (Fig. 1)");
  if (!h || !bhat || !xhat) return fail(IGM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  {
    igm_status ls = load_vec(h, h->hs.bh, bhat, s);
    if (ls) return ls;
  }
  igm_status st = run_ir(h->solo, s);
  if (st) return st;
  {
    igm_status ss = store_vec(h, xhat, h->hs.xt, s);
    if (ss) return ss;
  }
  return collect_host(h, rep, s);
}

igm_status ir_solve_batched(int count, igm_handle *hs, const double *const *bhat,
                            double *const *xhat, igm_report *reps, void *stream) {
  g_err.clear();
  IGM_RANGE("ir_solve_batched (Fig. 1 over a batch)");
  if (count < 1 || !hs || !bhat || !xhat) return fail(IGM_EINVAL, "bad batch arguments");
  std::vector<igm_handle> v(hs, hs + count);
  for (int i = 0; i < count; ++i) {
    if (!v[i] || !bhat[i] || !xhat[i]) return fail(IGM_EINVAL, "NULL entry %d", i);
    for (int k = 0; k < i; ++k)
      if (v[k] == v[i]) return fail(IGM_EINVAL, "handle %d repeated", i);
  }
  cudaStream_t s = (cudaStream_t)stream;
  Batch *b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batches_mu);
    for (Batch *c : g_batches)
      if (c->hs == v) b = c;
  }
  if (!b) {
    igm_status st = build_batch(v, &b);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_batches_mu);
    g_batches.push_back(b);
  }
  for (int i = 0; i < count; ++i)
    {
      igm_status ls = load_vec(v[i], v[i]->hs.bh, bhat[i], s);
      if (ls) return ls;
    }
  igm_status st = run_ir(b, s);
  if (st) return st;
  for (int i = 0; i < count; ++i)
    {
      igm_status ss = store_vec(v[i], xhat[i], v[i]->hs.xt, s);
      if (ss) return ss;
    }
  igm_status worst = IGM_OK;
  for (int i = 0; i < count; ++i) {
    igm_status e = collect_host(v[i], reps ? reps + i : nullptr, s);
    if (e && !worst) worst = e;
  }
  return worst;
}

igm_status int_gmres_solve(igm_handle h, const double *bk, double *xk, igm_report *rep,
                           void *stream) {
  g_err.clear();
  IGM_RANGE("int_gmres_solve (Fig. 2)");
  if (!h || !bk || !xk) return fail(IGM_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  Batch *b = h->solo;
  const BatchDev &B = b->bd;
  {
    igm_status ls = load_vec(h, h->hs.t, bk, s);
    if (!ls) ls = load_vec(h, h->hs.xk, xk, s);
    if (ls) return ls;
  }
  launch_init_scal(B, 1, s);
  if (b->inner == 1) launch_fp64_resid_guess(B, s);
  else launch_resid_int(B, s);
  launch_arm(B, s);
  enqueue_inner(b, s);
  CKL();
  h->ran_fuse = B.fuse;
  h->ran_snap = b->snap;
  g_launches += 3 + 5 + (b->any_ilu ? 2 : 0) +
                (B.fuse > 0 ? (long long)(b->m + B.fuse - 1) / B.fuse
                            : (long long)b->m * (4 + (b->any_ilu ? 2 : 0)));
  {
    igm_status ss = store_vec(h, xk, h->hs.xk, s);
    if (ss) return ss;
  }
  igm_status st = collect_host(h, rep, s);
  if (st == IGM_ENOCONV) st = IGM_OK;  // a single inner solve has no test
  if (rep && rep->status == IGM_ENOCONV) rep->status = IGM_OK;
  return st;
}

igm_status int_gmres_get_state(igm_handle h, long long *V, long long *H, long long *cs,
                               long long *sn, long long *g, int *jeff, double *nu) {
  g_err.clear();
  if (!h) return fail(IGM_EINVAL, "NULL handle");
  const int n = h->n, m = h->prm.m;
  CK(cudaDeviceSynchronize());
  if (V) CK(cudaMemcpy(V, h->hs.V, sizeof(i64) * (size_t)(m + 1) * n, cudaMemcpyDefault));
  if (H) CK(cudaMemcpy(H, h->hs.H, sizeof(i64) * (size_t)(m + 1) * m, cudaMemcpyDefault));
  if (cs) CK(cudaMemcpy(cs, h->hs.cs, sizeof(i64) * m, cudaMemcpyDefault));
  if (sn) CK(cudaMemcpy(sn, h->hs.sn, sizeof(i64) * m, cudaMemcpyDefault));
  if (g) CK(cudaMemcpy(g, h->hs.g, sizeof(i64) * (m + 1), cudaMemcpyDefault));
  if (jeff || nu) {
    SysScal sc;
    CK(cudaMemcpy(&sc, h->d_sc, sizeof(SysScal), cudaMemcpyDeviceToHost));
    if (jeff) *jeff = sc.jeff;
    if (nu) *nu = sc.nu;
  }
  return IGM_OK;
}

long long igm_kernel_launches(void) { return g_launches.load(); }

igm_status igm_norm2(const double *x, int n, double *out, void *stream) {
  g_err.clear();
  if (!out || n < 0 || (n > 0 && !x)) return fail(IGM_EINVAL, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  static std::mutex mu;
  static long long *ws = nullptr;
  static double *buf = nullptr;  // [0] max, [1] input staging of size n, ...
  static long long ws_words = 0, buf_len = 0;
  std::lock_guard<std::mutex> lk(mu);
  long long need_ws = 2LL * norm2_grid(n) + 2, need_buf = 2 + (long long)n;
  if (need_ws > ws_words) {
    if (ws) cudaFree(ws);
    ws = nullptr;
    if (cudaMalloc((void **)&ws, sizeof(long long) * need_ws) != cudaSuccess) {
      cudaGetLastError();
      ws_words = 0;
      return fail(IGM_EOOM, "norm workspace");
    }
    CK(cudaMemset(ws, 0, sizeof(long long) * need_ws));
    ws_words = need_ws;
  }
  if (need_buf > buf_len) {
    if (buf) cudaFree(buf);
    buf = nullptr;
    if (cudaMalloc((void **)&buf, sizeof(double) * need_buf) != cudaSuccess) {
      cudaGetLastError();
      buf_len = 0;
      return fail(IGM_EOOM, "norm workspace");
    }
    buf_len = need_buf;
  }
  // the counter words sit right after the partials of this call's grid
  const double *xd = x;
  cudaPointerAttributes pa;
  if (n == 0) {
    xd = buf + 2;
  } else if (cudaPointerGetAttributes(&pa, x) != cudaSuccess || pa.type == cudaMemoryTypeHost ||
             pa.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();
    if (n > 0) CK(cudaMemcpyAsync(buf + 2, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    xd = buf + 2;
  }
  long long g = norm2_grid(n);
  CK(cudaMemsetAsync(ws + 2 * g, 0, 2 * sizeof(long long), s));
  launch_norm2(xd, n, ws, buf, buf + 1, s);
  CKL();
  g_launches += 2;
  CK(cudaMemcpyAsync(out, buf + 1, sizeof(double), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return IGM_OK;
}

igm_status igm_time_kernels(igm_handle h, int reps, double *ms, void *stream) {
  g_err.clear();
  if (!h || !ms || reps < 1) return fail(IGM_EINVAL, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Batch *b = h->solo;
  const BatchDev &B = b->bd;
  const int m = h->prm.m, ilu = h->prm.precond;
  // put the inner-solve gates in the running state; h_{m,m-1} := 2^30 keeps
  // line 11's divisor non-zero
  SysScal sc;
  CK(cudaMemcpyAsync(&sc, h->d_sc, sizeof(SysScal), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  SysScal run = sc;
  run.cyc = 1;
  run.early = 0;
  run.active = 1;
  run.hnext = (i64)1 << 30;
  run.normj = -1;
  CK(cudaMemcpyAsync(h->d_sc, &run, sizeof(SysScal), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int k = 0; k < IGM_K_COUNT; ++k) {
    ms[k] = -1.0;
    if ((k == IGM_K_TRSV_L || k == IGM_K_TRSV_U) && !ilu) continue;
    float tot = 0.f;
    for (int r = 0; r < reps; ++r) {
      if (k == IGM_K_TRSV_L || k == IGM_K_TRSV_U) launch_spmv(B, m / 2, s);  // arms flags
      if (k == IGM_K_TRSV_U) launch_trsv_lv(B, 0, 1, 1, s);
      CK(cudaEventRecord(e0, s));
      switch (k) {
        case IGM_K_SPMV: launch_spmv(B, m / 2, s); break;
        case IGM_K_TRSV_L: launch_trsv_lv(B, 0, 1, 1, s); break;
        case IGM_K_TRSV_U: launch_trsv_lv(B, 0, 0, 1, s); break;
        case IGM_K_ARNOLDI: launch_mgs_step(B, m - 1, s); break;
        case IGM_K_RESID: launch_resid(B, 0, s); break;
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      tot += t;
      if (k == IGM_K_ARNOLDI) {  // the Givens step may end the solve: re-arm
        CK(cudaMemcpyAsync(h->d_sc, &run, sizeof(SysScal), cudaMemcpyHostToDevice, s));
      }
    }
    ms[k] = tot / reps;
  }
  CKL();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the scalars of the last solve (seq keeps increasing)
  SysScal now;
  CK(cudaMemcpyAsync(&now, h->d_sc, sizeof(SysScal), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  sc.seq = now.seq;
  CK(cudaMemcpyAsync(h->d_sc, &sc, sizeof(SysScal), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return IGM_OK;
}

}  // extern "C"
