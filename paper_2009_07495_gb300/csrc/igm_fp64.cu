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
  if (any_ilu) {  // line 1' with the FP64 factors
    launch_trsv_lv(B, 2, 1, 0, st);
    launch_trsv_lv(B, 2, 0, 0, st);
  }
  launch_max(B, VEC_R, 2, st);
  launch_norm(B, VEC_R, ACT_NU, 2, st);
  f_v1<<<T, IGM_BLOCK, 0, st>>>(B);
  for (int j = 0; j < m; ++j) {
    f_spmv<<<T, IGM_BLOCK, 0, st>>>(B, j);
    if (any_ilu) {  // line 5' with the FP64 factors
      launch_trsv_lv(B, 2, 1, 1, st);
      launch_trsv_lv(B, 2, 0, 1, st);
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
