// igm_fp64.cu -- the comparison solver of Sec. VII ("Double"): standard
// restarted GMRES(m) in FP64 with left ILU(0) preconditioning (the FP64
// factors L (unit), U of eq. (ilu)), modified Gram-Schmidt and Givens
// rotations, inside the same refinement loop (Fig. 1) and on the same
// batch/tile layout as the integer solver.  Its basis, Hessenberg matrix and
// rotations reuse the integer solver's 8-byte arrays.  Lines 6-19 run in the
// persistent step kernel of igm_mgs.cu; its reductions are plain FP64 sums
// in a fixed order, deterministic but not bit-identical to a sequential sum.
#include "igm_dev.cuh"
#include "igm_launch.h"

namespace igm {

#define TILE_LOOP(r)                                                           \
  for (int r = tl.row0 + (int)threadIdx.x; r < tl.row0 + tl.nrows; r += blockDim.x)

__device__ __forceinline__ bool f_step(const SysScal *sc) {
  return sc->cyc != 0 && sc->early == 0;
}
__device__ __forceinline__ double *Vd(const SysDev *s) { return reinterpret_cast<double *>(s->V); }
__device__ __forceinline__ double *Hd(const SysDev *s) { return reinterpret_cast<double *>(s->H); }
__device__ __forceinline__ double *Wd(const SysDev *s) { return reinterpret_cast<double *>(s->w); }
__device__ __forceinline__ double *Yd(const SysDev *s) { return reinterpret_cast<double *>(s->yv); }

__device__ __forceinline__ int f_ticket(unsigned *ctr) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  return s_t;
}

// M^-1 with the FP64 factors: lower: y = L^-1 in (unit diagonal);
// upper: out = U^-1 y.  which: 0 -> r (line 1), 1 -> w (line 5)
__global__ void f_trsv(BatchDev B, int lower, int which) {
  int ti = f_ticket(&B.ticket[lower ? (which ? 2 : 0) : (which ? 3 : 1)]);
  Tile tl = B.tiles[ti];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!f_step(sc) || !s->p.precond) return;
  const int *ord = lower ? s->lorder : s->uorder;
  int *flag = lower ? s->lflag : s->uflag;
  double *vec = which ? Wd(s) : s->r;
  const double *in = lower ? vec : s->t;
  double *out = lower ? s->t : vec;
  int ep = sc->seq;
  TILE_LOOP(p) {
    int i = ord[p];
    double acc = in[i];
    int k0 = lower ? s->rowptr[i] : s->diagpos[i] + 1;
    int k1 = lower ? s->diagpos[i] : s->rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      int j = s->col[k];
      wait_flag(flag + j, ep, &sc->err);
      acc = __dsub_rn(acc, __dmul_rn(s->f[k], __ldcg(out + j)));
    }
    out[i] = lower ? acc : __ddiv_rn(acc, s->f[s->diagpos[i]]);
    st_release(flag + i, ep);
  }
}

// line 5 preconditioner by chunks (same schedule as the integer k_trsv_chunk)
__global__ void __launch_bounds__(256) f_trsv_chunk(BatchDev B, int lower) {
  __shared__ int s_t;
  if (threadIdx.x == 0) s_t = (int)atomicAdd(&B.ticket[lower ? 2 : 3], 1u);
  __syncthreads();
  Tile ct = B.ctiles[s_t];
  const SysDev *s = B.sys[ct.sys];
  SysScal *sc = s->sc;
  if (!f_step(sc) || !s->p.precond) return;
  const int c = ct.row0, n = s->n, R = s->chunk;
  const int first = c * R;
  const int *ord = lower ? s->lorder : s->uorder;
  const int *lptr = lower ? s->llptr : s->ulptr;
  const int *levb = lower ? s->llevb : s->ulevb;
  const int *lev = lower ? s->llev : s->ulev;
  u64 *prog = lower ? s->lprog : s->uprog;
  const double *in = lower ? Wd(s) : s->t;
  double *out = lower ? s->t : Wd(s);
  const u64 ep = (u64)(unsigned)sc->seq << 32;
  const int g0 = levb[c], g1 = levb[c + 1];
  for (int g = g0; g < g1; ++g) {
    for (int p = lptr[g] + threadIdx.x; p < lptr[g + 1]; p += blockDim.x) {
      int i = ord[p];
      double acc = in[i];
      int k0 = lower ? s->rowptr[i] : s->diagpos[i] + 1;
      int k1 = lower ? s->diagpos[i] : s->rowptr[i + 1];
      for (int k = k0; k < k1; ++k) {
        int j = s->col[k];
        int pj = lower ? j : n - 1 - j;
        double yj;
        if (pj >= first) {
          yj = out[j];
        } else {
          wait_prog(prog + pj / R, ep | (u64)(lev[j] + 1), &sc->err);
          yj = __ldcg(out + j);
        }
        acc = __dsub_rn(acc, __dmul_rn(s->f[k], yj));
      }
      out[i] = lower ? acc : __ddiv_rn(acc, s->f[s->diagpos[i]]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release64(prog + c, ep | (u64)(g - g0 + 1));
    }
  }
}

// v_1 = r0 / ||r0||, g = (||r0||, 0, ...)
__global__ void f_v1(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!f_step(sc)) return;
  double nu = sc->nu;
  double *V = Vd(s);
  TILE_LOOP(l) V[l] = __ddiv_rn(s->r[l], nu);
  if (blockIdx.x == tl.first && threadIdx.x == 0) {
    double *g = reinterpret_cast<double *>(s->g);
    g[0] = nu;
    for (int k = 1; k <= s->p.m; ++k) g[k] = 0.0;
  }
}

// w = A v_j (scaled FP64 A); arms the flags of the substitutions
__global__ void f_spmv(BatchDev B, int j) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.ticket[2] = 0;
    B.ticket[3] = 0;
  }
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!f_step(sc) || j >= s->p.m) return;
  if (blockIdx.x == tl.first && threadIdx.x == 0) sc->seq += 1;
  const double *vj = Vd(s) + (size_t)j * s->n;
  double *w = Wd(s);
  TILE_LOOP(i) {
    double acc = 0.0;
    for (int k = s->rowptr[i]; k < s->rowptr[i + 1]; ++k)
      acc = __dadd_rn(acc, __dmul_rn(s->a[k], vj[s->col[k]]));
    w[i] = acc;
  }
}

__global__ void f_backsub(BatchDev B) {
  int si = blockIdx.x * blockDim.x + threadIdx.x;
  if (si >= B.nsys) return;
  const SysDev *s = B.sys[si];
  SysScal *sc = s->sc;
  if (!sc->cyc) return;
  const int jeff = sc->jeff, ld = s->ld;
  const double *H = Hd(s), *g = reinterpret_cast<const double *>(s->g);
  double *z = s->yfp;
  for (int a = jeff - 1; a >= 0; --a) {
    double acc = g[a];
    for (int b = a + 1; b < jeff; ++b) acc = __dsub_rn(acc, __dmul_rn(H[a + b * ld], z[b]));
    z[a] = __ddiv_rn(acc, H[a + a * ld]);
  }
  sc->refinements += 1;
  sc->inner_steps += jeff;
  if (sc->early == 1) sc->breakdowns += 1;
}

__global__ void f_update(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  SysScal *sc = s->sc;
  if (!sc->cyc) return;
  const int jeff = sc->jeff, n = s->n;
  const bool ir = sc->mode == 0;
  const double *V = Vd(s);
  double gam = sc->gamma;
  TILE_LOOP(l) {
    double acc = ir ? 0.0 : s->xk[l];
    for (int i = 0; i < jeff; ++i) acc = __dadd_rn(acc, __dmul_rn(s->yfp[i], V[(size_t)i * n + l]));
    if (ir) s->xt[l] = __dadd_rn(s->xt[l], __dmul_rn(gam, acc));
    else s->xk[l] = acc;
  }
}

// r = bk - A xk for a single inner solve with a given guess (line 1)
__global__ void f_resid_guess(BatchDev B) {
  Tile tl = B.tiles[blockIdx.x];
  const SysDev *s = B.sys[tl.sys];
  if (!s->sc->cyc) return;
  TILE_LOOP(i) {
    double acc = 0.0;
    for (int k = s->rowptr[i]; k < s->rowptr[i + 1]; ++k)
      acc = __dadd_rn(acc, __dmul_rn(s->a[k], s->xk[s->col[k]]));
    s->r[i] = __dsub_rn(s->t[i], acc);
  }
}

void launch_fp64_inner(const BatchDev &B, int m, int any_ilu, cudaStream_t st) {
  const int T = B.ntiles;
  if (any_ilu) {
    f_trsv<<<T, IGM_BLOCK, 0, st>>>(B, 1, 0);
    f_trsv<<<T, IGM_BLOCK, 0, st>>>(B, 0, 0);
  }
  launch_max(B, VEC_R, 2, st);
  launch_norm(B, VEC_R, ACT_NU, 2, st);
  f_v1<<<T, IGM_BLOCK, 0, st>>>(B);
  for (int j = 0; j < m; ++j) {
    f_spmv<<<T, IGM_BLOCK, 0, st>>>(B, j);
    if (any_ilu && B.nctiles > 0) {
      f_trsv_chunk<<<B.nctiles, 256, 0, st>>>(B, 1);
      f_trsv_chunk<<<B.nctiles, 256, 0, st>>>(B, 0);
    }
    launch_fp64_mgs_step(B, j, st);
  }
  f_backsub<<<(B.nsys + 127) / 128, 128, 0, st>>>(B);
  f_update<<<T, IGM_BLOCK, 0, st>>>(B);
}

void launch_fp64_resid_guess(const BatchDev &B, cudaStream_t st) {
  f_resid_guess<<<B.ntiles, IGM_BLOCK, 0, st>>>(B);
}

}  // namespace igm
