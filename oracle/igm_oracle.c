/*
 * igm_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * integer-arithmetic GMRES solver with FP64 iterative refinement of
 * Iwashita, Suzuki and Fukaya, "An Integer Arithmetic-Based Sparse Linear
 * Solver Using a GMRES Method and Iterative Refinement" (ScalA'20).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; it exists so the tests, the smoke check and the CPU
 * baseline of the benchmark can check the CUDA library against a plain
 * restatement of the paper.  It shares no code, header or table with the
 * CUDA sources.
 *
 * Every integer quantity behaves as on the paper's hardware: an int64 word
 * holding the exact value modulo 2^64 (two's complement wrap).  Each place
 * where the exact value of an operation leaves [-2^63, 2^63) is counted as
 * an overflow event, per line of Fig. 2 (the paper only avoids overflow and
 * does not define what happens; this counting is this project's reading).
 * A sum counts once if its exact total (of the int64 summands) is out of
 * range, and each product counts once if its exact value is.
 *
 * Readings of the paper that this file fixes:
 *  - "right shift by beta" is floor division by 2^beta (arithmetic shift),
 *    Sec. V-A;
 *  - "cast" from FP to integer truncates toward zero (Sec. IV-B, V-D, VI-A);
 *  - integer division truncates toward zero (C semantics, Sec. V-B);
 *  - the square root is floor(sqrt(.)) reached by the Babylonian iteration,
 *    Sec. V-B;
 *  - line 17 of Fig. 2 updates g_{j+1} and g_j from the old g_j;
 *  - "1" in line 3 of Fig. 2 is the Q(d_f) one, 2^d_f;
 *  - FP64 norms are a reproducible, order-independent 2-norm (below);
 *  - FP64 row sums run in CSR order with no fused multiply-add.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long long i64;
typedef __int128 i128;

/* status codes */
enum {
  OR_OK = 0, OR_EINVAL = 1, OR_EZERO_ROW = 2, OR_EZERO_PIVOT = 3,
  OR_EBREAKDOWN = 4, OR_ENOCONV = 5, OR_ENOMEM = 6
};

/* overflow-event counters, one per line of Fig. 2 */
enum {
  EV_L5 = 0,    /* line 5: integer matrix-vector product            */
  EV_L5P = 1,   /* line 5': integer forward/backward substitution   */
  EV_L7 = 2,    /* line 7: inner product                            */
  EV_L8 = 3,    /* line 8: vector update                            */
  EV_L10 = 4,   /* line 10: norm                                    */
  EV_L11 = 5,   /* line 11: division of a vector by a scalar        */
  EV_L13 = 6,   /* line 13: application of old Givens rotations     */
  EV_L15 = 7,   /* line 15: 2-element norm                          */
  EV_L16 = 8,   /* line 16: c and s divisions                       */
  EV_L17 = 9,   /* line 17: update of g                             */
  EV_VRANGE = 10, /* a basis entry outside the int32 range          */
  EV_L2 = 11,   /* line 2: FP->int cast out of range                */
  EV_COUNT = 16
};

/* Parameters of the method: the paper's names (Sec. II, III, VII). */
#define OR_MAX_S 4

typedef struct {
  int df;        /* fractional bits d_f of the Q(d_m).(d_f) word        */
  int alpha_a;   /* exponent of the initial scaling, eq. (3)            */
  int m;         /* Arnoldi steps per inner solve                       */
  int precond;   /* 0: none, 1: integer ILU(0) (Sec. VI), 2: integer
                    Gauss-Seidel (Sec. VII-D) in the same factor form   */
  int beta7, beta8, beta10, beta11a, beta11b, beta13, beta15, beta16a, beta16b;
  double tol;    /* epsilon of Fig. 1                                   */
  int max_refine;
  int s;         /* correction terms of eq. (AA) used in every refinement,
                    s(k) = s (0 ... OR_MAX_S)                          */
  int order;     /* 0: natural row order (the paper's); 1: multicolour
                    order (or_mc_order), the whole method run on the
                    permuted system P A P^T (P x) = P b                */
  int shift_tune;/* shift auto-tuning (Sec. VII-D): cycles that may be
                    discarded and rerun with raised shifts in one solve
                    (0: the shifts stay as given, as in Tables 4 and 5) */
} or_params;

typedef struct {
  i64 ev[EV_COUNT];
  int refinements;          /* inner solves performed                  */
  int inner_steps;          /* Arnoldi steps over all inner solves     */
  int breakdowns;           /* inner solves that ended early           */
  int status;
  double relres;            /* final ||b - A x|| / ||b|| (scaled)      */
  double relres_unscaled;   /* final ||bh - Ah xh|| / ||bh||           */
  double gamma_hist[64];
  double relres_hist[65];
  int shift_retries;        /* cycles discarded by the shift auto-tuning  */
  int beta_final[5];        /* beta7, beta8, beta10, beta13, beta15 at the
                               end of the solve                           */
} or_report;

/* ------------------------------------------------------------------ */
/* Fixed-point primitives (Sec. V-B)                                   */
/* ------------------------------------------------------------------ */

static const i128 I64MIN_128 = -((i128)1 << 63);
static const i128 I64MAX_128 = ((i128)1 << 63) - 1;

static int out64(i128 x) { return x < I64MIN_128 || x > I64MAX_128; }

/* value modulo 2^64, as the hardware stores it */
static i64 wrap64(i128 x) { return (i64)(uint64_t)x; }

/* right shift by s bits = floor(x / 2^s), written without relying on the
 * compiler's treatment of >> on negative numbers */
static i64 shr(i64 x, int s) {
  if (s <= 0) return x;
  if (s > 63) return x < 0 ? -1 : 0;
  if (x >= 0) return x >> s;
  return ~((~x) >> s);
}

/* product of two int64 words, wrapped, counting an event when the exact
 * product is out of range */
static i64 mul(i64 a, i64 b, i64 *ev) {
  i128 p = (i128)a * (i128)b;
  if (out64(p)) (*ev)++;
  return wrap64(p);
}

static i64 neg(i64 a, i64 *ev) {
  i128 p = -(i128)a;
  if (out64(p)) (*ev)++;
  return wrap64(p);
}

/* multiplication by 2^e (e >= 0) or floor division by 2^-e (e < 0) */
static i64 scale2(i64 x, int e, i64 *ev) {
  if (e >= 0) {
    i128 p = (i128)x;
    for (int k = 0; k < e; ++k) p *= 2;
    if (out64(p)) (*ev)++;
    return wrap64(p);
  }
  return shr(x, -e);
}

/* integer division truncating toward zero (C semantics) */
static i64 divt(i64 a, i64 b, i64 *ev) {
  if (b == -1 && a == INT64_MIN) { (*ev)++; return INT64_MIN; }
  return a / b;
}

/* Babylonian square root on integers (Sec. V-B): start at or above sqrt(s)
 * and iterate x <- (x + s/x)/2 while it decreases.  The fixed point reached
 * is floor(sqrt(s)).  A negative argument only arises after a wrapped
 * overflow; it yields 0. */
static i64 isqrt_bab(i64 s) {
  if (s <= 0) return 0;
  i128 x = s;
  for (;;) {
    i128 y = (x + (i128)s / x) / 2;
    if (y >= x) return (i64)x;
    x = y;
  }
}

/* The fixed-point product of eq. (c1c2): ((t1>>b1)*(t2>>b2))>>(df-b1-b2);
 * a negative final shift is a multiplication by 2^(b1+b2-df). */
i64 or_fx_mul(i64 t1, i64 t2, int b1, int b2, int df, i64 *ev) {
  return scale2(mul(shr(t1, b1), shr(t2, b2), ev), b1 + b2 - df, ev);
}

/* The fixed-point division of Sec. V-B: ((t1*2^b1) / (t2>>b2)) * 2^(df-b1-b2).
 * Returns 0 and sets *zero when the shifted divisor is zero. */
i64 or_fx_div(i64 t1, i64 t2, int b1, int b2, int df, i64 *ev, int *zero) {
  i64 d = shr(t2, b2);
  *zero = (d == 0);
  if (d == 0) return 0;
  return scale2(divt(scale2(t1, b1, ev), d, ev), df - b1 - b2, ev);
}

/* The fixed-point square root of Sec. V-B for an argument with dfp
 * fractional bits: isqrt(t) * 2^(df - dfp/2). */
i64 or_fx_sqrt(i64 t, int dfp, int df, i64 *ev) {
  return scale2(isqrt_bab(t), df - dfp / 2, ev);
}

i64 or_isqrt(i64 s) { return isqrt_bab(s); }
i64 or_shr(i64 x, int s) { return shr(x, s); }

/* ------------------------------------------------------------------ */
/* Reproducible FP64 2-norm                                             */
/* ------------------------------------------------------------------ */
/* ||r||_2 defined independently of summation order: with e = ilogb(max|r|),
 * each t_i = r_i 2^-e is squared exactly as p_i + q_i (p = t*t rounded,
 * q = fma(t,t,-p)); p_i 2^96 and q_i 2^96 are truncated toward zero to
 * integers and summed exactly; the integer total is rounded once to double,
 * scaled by 2^-96, square-rooted and scaled by 2^e. */
double or_norm2(int n, const double *r) {
  double mx = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = fabs(r[i]);
    if (a > mx) mx = a;
  }
  if (mx == 0.0) return 0.0;
  int e = ilogb(mx);
  i128 acc = 0;
  for (int i = 0; i < n; ++i) {
    double t = ldexp(r[i], -e);
    double p = t * t;
    double q = fma(t, t, -p);
    acc += (i128)ldexp(p, 96);
    acc += (i128)ldexp(q, 96);
  }
  double s = (double)acc;
  return ldexp(sqrt(ldexp(s, -96)), e);
}

double or_maxabs(int n, const double *r) {
  double mx = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = fabs(r[i]);
    if (a > mx) mx = a;
  }
  return mx;
}

/* ------------------------------------------------------------------ */
/* Setup: initial scaling (eq. 1, eq. 3), cast (Sec. IV-B), ILU(0)      */
/* ------------------------------------------------------------------ */

/* eq. (3): d_i = max_j |ahat_ij| / 2^alpha_a; eq. (1): A = D^-1 Ahat,
 * b = D^-1 bhat.  A zero row is an error. */
int or_scale(int n, const int *rowptr, const int *col, const double *ahat,
             const double *bhat, int alpha_a, double *a, double *b, double *d) {
  (void)col;
  for (int i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double v = fabs(ahat[k]);
      if (v > mx) mx = v;
    }
    if (mx == 0.0) return OR_EZERO_ROW;
    double di = ldexp(mx, -alpha_a);
    d[i] = di;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) a[k] = ahat[k] / di;
    if (b) b[i] = bhat[i] / di;
  }
  return OR_OK;
}

/* Sec. IV-B: Abar_0 = cast(A), truncation toward zero. */
int or_cast(int nnz, const double *a, i64 *abar) {
  for (int k = 0; k < nnz; ++k) {
    double v = a[k];
    if (!(fabs(v) < 9223372036854775808.0)) return OR_EINVAL;
    abar[k] = (i64)v;
  }
  return OR_OK;
}

/* Sec. IV-C, eq. (alpha1) and (A): Abar_0 = trunc(A); then, for l = 1 ... S,
 * with the FP remainder A_l (A_1 = A - Abar_0), alpha_l = alpha_a -
 * floor(log2 max |A_l|), Abar_l = trunc(A_l 2^alpha_l) and A_(l+1) =
 * A_l - Abar_l 2^-alpha_l (every step exact in FP64).  terms holds
 * (S+1) x nnz values (term 0 first), alphas[l] the exponents (alphas[0] =
 * 0).  Returns the number of correction terms built: fewer than S when a
 * remainder is zero (A is then represented exactly). */
int or_multiterm(int nnz, const double *a, int alpha_a, int S, i64 *terms, int *alphas) {
  double *R = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  int built = 0;
  alphas[0] = 0;
  for (int k = 0; k < nnz; ++k) {
    terms[k] = (i64)a[k];
    R[k] = a[k] - (double)terms[k];
  }
  for (int l = 1; l <= S; ++l) {
    double mx = 0.0;
    for (int k = 0; k < nnz; ++k) mx = fmax(mx, fabs(R[k]));
    if (mx == 0.0) break;
    int al = alpha_a - ilogb(mx);
    alphas[l] = al;
    i64 *T = terms + (size_t)l * nnz;
    for (int k = 0; k < nnz; ++k) {
      double t = ldexp(R[k], al);
      T[k] = (i64)t;
      R[k] = ldexp(t - (double)T[k], -al);
    }
    built = l;
  }
  free(R);
  return built;
}

static int find_diag(int n, const int *rowptr, const int *col, int *diagpos) {
  for (int i = 0; i < n; ++i) {
    diagpos[i] = -1;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) diagpos[i] = k;
    if (diagpos[i] < 0) return OR_EZERO_PIVOT;
  }
  return OR_OK;
}

/* Multicolour ordering, a GPU-motivated reordering of the preconditioned
 * solver (the paper runs ILU(0) and Gauss-Seidel in the natural order):
 * greedy distance-1 colouring of the symmetrised pattern of A (i ~ j when
 * a_ij or a_ji is stored, i != j), rows visited in natural order, each
 * taking the smallest colour that none of its already coloured neighbours
 * has.  The new order lists the rows colour by colour, ascending original
 * index within a colour: perm[new] = old, cptr[c] = first new index of
 * colour c (cptr has n + 1 entries).  Returns the number of colours. */
int or_mc_order(int n, const int *rowptr, const int *col, int *perm, int *cptr) {
  const int nnz = rowptr[n];
  /* symmetrised adjacency: every stored off-diagonal entry in both rows */
  int *deg = (int *)calloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] != i) {
        deg[i]++;
        deg[col[k]]++;
      }
  int *aptr = (int *)malloc(sizeof(int) * ((size_t)n + 1));
  aptr[0] = 0;
  for (int i = 0; i < n; ++i) aptr[i + 1] = aptr[i] + deg[i];
  int *adj = (int *)malloc(sizeof(int) * (size_t)(aptr[n] ? aptr[n] : 1));
  int *fill = (int *)calloc((size_t)n, sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] != i) {
        int j = col[k];
        adj[aptr[i] + fill[i]++] = j;
        adj[aptr[j] + fill[j]++] = i;
      }
  (void)nnz;
  /* greedy colouring */
  int *color = (int *)malloc(sizeof(int) * (size_t)(n ? n : 1));
  int *mark = (int *)malloc(sizeof(int) * ((size_t)n + 1));
  for (int c = 0; c <= n; ++c) mark[c] = -1;
  int ncol = 0;
  for (int i = 0; i < n; ++i) {
    for (int k = aptr[i]; k < aptr[i + 1]; ++k) {
      int j = adj[k];
      if (j < i) mark[color[j]] = i;
    }
    int c = 0;
    while (mark[c] == i) ++c;
    color[i] = c;
    if (c + 1 > ncol) ncol = c + 1;
  }
  /* rows by colour, stable */
  for (int c = 0; c <= ncol; ++c) cptr[c] = 0;
  for (int i = 0; i < n; ++i) cptr[color[i] + 1]++;
  for (int c = 0; c < ncol; ++c) cptr[c + 1] += cptr[c];
  for (int c = ncol + 1; c <= n; ++c) cptr[c] = n;
  int *pos = (int *)malloc(sizeof(int) * ((size_t)ncol + 1));
  for (int c = 0; c < ncol; ++c) pos[c] = cptr[c];
  for (int i = 0; i < n; ++i) perm[pos[color[i]]++] = i;
  free(deg); free(aptr); free(adj); free(fill); free(color); free(mark); free(pos);
  return ncol;
}

/* the permuted system P A P^T: row r of the result is row perm[r] of A with
 * columns renumbered by the inverse permutation and sorted ascending */
void or_permute_csr(int n, const int *rowptr, const int *col, const double *val,
                    const int *perm, int *rowptr2, int *col2, double *val2) {
  int *inv = (int *)malloc(sizeof(int) * (size_t)(n ? n : 1));
  for (int r = 0; r < n; ++r) inv[perm[r]] = r;
  rowptr2[0] = 0;
  for (int r = 0; r < n; ++r) {
    int o = perm[r], k2 = rowptr2[r];
    for (int k = rowptr[o]; k < rowptr[o + 1]; ++k) {
      /* insertion by new column index */
      int c = inv[col[k]], q = k2;
      double v = val[k];
      while (q > rowptr2[r] && col2[q - 1] > c) {
        col2[q] = col2[q - 1];
        val2[q] = val2[q - 1];
        --q;
      }
      col2[q] = c;
      val2[q] = v;
      ++k2;
    }
    rowptr2[r + 1] = k2;
  }
  free(inv);
}

/* eq. (ilu): A ~ L D U by ILU(0), the IKJ row variant restricted to the
 * pattern of A (Saad, Iterative Methods, Alg. 10.4), rows in natural order,
 * k ascending.  On return f holds L_ik (k<i, unit diagonal implied) and the
 * non-unit upper factor (L D U' with U = D U': f holds U_ij = d_i U'_ij for
 * j >= i).  Columns within a row must be ascending. */
int or_ilu0(int n, const int *rowptr, const int *col, const double *a, double *f,
            int *diagpos) {
  int nnz = rowptr[n];
  memcpy(f, a, sizeof(double) * (size_t)nnz);
  int st = find_diag(n, rowptr, col, diagpos);
  if (st) return st;
  for (int i = 0; i < n; ++i) {
    for (int kk = rowptr[i]; kk < rowptr[i + 1] && col[kk] < i; ++kk) {
      int k = col[kk];
      double ukk = f[diagpos[k]];
      if (ukk == 0.0) return OR_EZERO_PIVOT;
      double lik = f[kk] / ukk;
      f[kk] = lik;
      /* a_ij -= l_ik * u_kj for j > k in the pattern of row i */
      int p = diagpos[k] + 1; /* walk row k's upper part */
      for (int jj = kk + 1; jj < rowptr[i + 1]; ++jj) {
        int j = col[jj];
        while (p < rowptr[k + 1] && col[p] < j) ++p;
        if (p < rowptr[k + 1] && col[p] == j) {
          double prod = lik * f[p];
          f[jj] = f[jj] - prod;
        }
      }
    }
    if (f[diagpos[i]] == 0.0) return OR_EZERO_PIVOT;
  }
  return OR_OK;
}

/* The Gauss-Seidel preconditioner M = D + L_A (Sec. VII-D mentions it; the
 * reading here): written as M = (I + L_A D^-1) D it has the form of the
 * ILU factors, with unit lower factor entries a_ij / a_jj (j < i, correctly
 * rounded), pivots a_ii and no strict upper part.  f receives that factor
 * storage, so eq. (dldr)-(ilu2) and the substitutions apply unchanged. */
int or_gs_factors(int n, const int *rowptr, const int *col, const double *a, double *f,
                  int *diagpos) {
  int st = find_diag(n, rowptr, col, diagpos);
  if (st) return st;
  for (int i = 0; i < n; ++i)
    if (a[diagpos[i]] == 0.0) return OR_EZERO_PIVOT;
  for (int i = 0; i < n; ++i)
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = col[k];
      f[k] = j < i ? a[k] / a[diagpos[j]] : (j == i ? a[k] : 0.0);
    }
  return OR_OK;
}

/* eq. (dldr)-(ilu2): with d_i the pivots, D_l = |d|^(1/2),
 * D_u = sgn(d)|d|^(1/2), Ltilde = L D_l, Utilde = D_u U', and the integer
 * factors are their casts (truncation).  fac holds Lbar_ij (j<i) and
 * Ubar_ij (j>i) on the pattern of A; the diagonals go to ldiag, udiag. */
int or_ilu_int(int n, const int *rowptr, const int *col, const double *f,
               const int *diagpos, i64 *fac, i64 *ldiag, i64 *udiag) {
  for (int i = 0; i < n; ++i) {
    double di = f[diagpos[i]];
    double sl = sqrt(fabs(di));
    double su = di < 0 ? -sl : sl;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int j = col[k];
      double v;
      if (j < i) {
        double dj = f[diagpos[j]];
        v = f[k] * sqrt(fabs(dj));
      } else if (j > i) {
        v = su * (f[k] / di);
      } else {
        fac[k] = 0;
        continue;
      }
      if (!(fabs(v) < 9223372036854775808.0)) return OR_EINVAL;
      fac[k] = (i64)v;
    }
    if (!(sl < 9223372036854775808.0)) return OR_EINVAL;
    ldiag[i] = (i64)sl;
    udiag[i] = (i64)su;
    if (ldiag[i] == 0 || udiag[i] == 0) return OR_EZERO_PIVOT;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Integer kernels (Sec. V-C, VI)                                       */
/* ------------------------------------------------------------------ */

/* line 5 / eq. (matvec) with s = 0: w = Abar_0 v, Q0 x Q(df) -> Q(df). */
void or_spmv_int(int n, const int *rowptr, const int *col, const i64 *abar,
                 const i64 *v, i64 *w, i64 *ev) {
  for (int i = 0; i < n; ++i) {
    i128 acc = 0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      acc += (i128)mul(abar[k], v[col[k]], ev);
    if (out64(acc)) (*ev)++;
    w[i] = wrap64(acc);
  }
}

/* line 5 / eq. (matvec) with s correction terms: each Abar_l v is the
 * product of an integer matrix program (exact row sums stored as words,
 * events as in or_spmv_int), divided by 2^alpha_l as a right shift and
 * added to the result; the sum of the s + 1 words is exact, stored as a
 * word (an event when it leaves the range).  terms: (s+1) x nnz. */
void or_spmv_int_s(int n, const int *rowptr, const int *col, int ns, const i64 *terms,
                   const int *alphas, const i64 *v, i64 *w, i64 *ev) {
  const int nnz = rowptr[n];
  for (int i = 0; i < n; ++i) {
    i128 tot = 0;
    for (int l = 0; l <= ns; ++l) {
      const i64 *T = terms + (size_t)l * nnz;
      i128 acc = 0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
        acc += (i128)mul(T[k], v[col[k]], ev);
      if (out64(acc)) (*ev)++;
      i64 u = wrap64(acc);
      tot += (i128)(l == 0 ? u : shr(u, alphas[l]));
    }
    if (out64(tot)) (*ev)++;
    w[i] = wrap64(tot);
  }
}

/* line 5', first half: y = Lbar^-1 z by forward substitution with the data
 * types of an FP program changed to integers (Sec. VI-A):
 * y_i = (z_i - sum_{j<i} Lbar_ij y_j) / Lbar_ii, division truncating. */
void or_lsolve_int(int n, const int *rowptr, const int *col, const i64 *fac,
                   const i64 *ldiag, const i64 *z, i64 *y, i64 *ev) {
  for (int i = 0; i < n; ++i) {
    i128 acc = z[i];
    for (int k = rowptr[i]; k < rowptr[i + 1] && col[k] < i; ++k)
      acc -= (i128)mul(fac[k], y[col[k]], ev);
    if (out64(acc)) (*ev)++;
    y[i] = divt(wrap64(acc), ldiag[i], ev);
  }
}

/* line 5', second half: w = Ubar^-1 y by backward substitution. */
void or_usolve_int(int n, const int *rowptr, const int *col, const i64 *fac,
                   const i64 *udiag, const i64 *y, i64 *w, i64 *ev) {
  for (int i = n - 1; i >= 0; --i) {
    i128 acc = y[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] > i) acc -= (i128)mul(fac[k], w[col[k]], ev);
    if (out64(acc)) (*ev)++;
    w[i] = divt(wrap64(acc), udiag[i], ev);
  }
}

/* line 1': the same substitutions in FP64 on the integer factors (their
 * values converted to double, exact below 2^53), CSR order, no FMA. */
void or_lsolve_fp(int n, const int *rowptr, const int *col, const i64 *fac,
                  const i64 *ldiag, const double *z, double *y) {
  for (int i = 0; i < n; ++i) {
    double acc = z[i];
    for (int k = rowptr[i]; k < rowptr[i + 1] && col[k] < i; ++k) {
      double p = (double)fac[k] * y[col[k]];
      acc = acc - p;
    }
    y[i] = acc / (double)ldiag[i];
  }
}

void or_usolve_fp(int n, const int *rowptr, const int *col, const i64 *fac,
                  const i64 *udiag, const double *y, double *w) {
  for (int i = n - 1; i >= 0; --i) {
    double acc = y[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] > i) {
        double p = (double)fac[k] * w[col[k]];
        acc = acc - p;
      }
    w[i] = acc / (double)udiag[i];
  }
}

/* r = b - A x in FP64: s = sum_k a_k x_col(k) in CSR order, then b - s. */
void or_resid_fp(int n, const int *rowptr, const int *col, const double *a,
                 const double *x, const double *b, double *r) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double p = a[k] * x[col[k]];
      s = s + p;
    }
    r[i] = b[i] - s;
  }
}

/* same with the matrix of eq. (AA) (line 1 of Fig. 2): its FP64 value
 * Abar_0 + sum_l Abar_l 2^-alpha_l is exact (a truncation of A's bits) */
static void resid_fp_int(int n, const int *rowptr, const int *col, int ns, const i64 *terms,
                         const int *alphas, const double *x, const double *b, double *r) {
  const int nnz = rowptr[n];
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double av = (double)terms[k];
      for (int l = 1; l <= ns; ++l) av = av + ldexp((double)terms[(size_t)l * nnz + k], -alphas[l]);
      double p = av * x[col[k]];
      s = s + p;
    }
    r[i] = b[i] - s;
  }
}

/* ------------------------------------------------------------------ */
/* One int-GMRES(m) solve, Fig. 2 (with lines 1', 5' of Sec. VI)        */
/* ------------------------------------------------------------------ */

typedef struct {
  int n;
  const int *rowptr, *col;
  const i64 *abar;                  /* Abar_0 ... Abar_ns, (ns+1) x nnz  */
  const i64 *fac, *ldiag, *udiag;   /* integer ILU factors (precond=1)  */
  int ns;                           /* correction terms of eq. (AA)     */
  const int *alphas;                /* their exponents (alphas[0] = 0)  */
} or_system;

/* Solves Abar x = bk approximately with m steps of Fig. 2 and adds the
 * correction to xk (Table 2: xk is the initial guess on input).
 * Optional outputs (NULL allowed): V ((m+1) x n, row-major by vector),
 * H ((m+1) x m, column-major: H[i + j*(m+1)]) after the Givens rotations,
 * Hraw the same before rotation, cs, sn (m), g (m+1), *jeff the number of
 * Arnoldi columns used, *nu = ||r0||.  Returns 1 if the solve ended early
 * (breakdown), else 0. */
int or_int_gmres(const or_params *P, const or_system *S, const double *bk,
                 double *xk, i64 *V_out, i64 *H_out, i64 *Hraw_out, i64 *cs_out,
                 i64 *sn_out, i64 *g_out, int *jeff_out, double *nu_out, i64 *ev) {
  const int n = S->n, m = P->m, df = P->df, ld = m + 1;
  i64 *V = V_out ? V_out : (i64 *)calloc((size_t)(m + 1) * n, sizeof(i64));
  i64 *H = (i64 *)calloc((size_t)(m + 1) * m, sizeof(i64));
  i64 *cs = (i64 *)calloc((size_t)m, sizeof(i64));
  i64 *sn = (i64 *)calloc((size_t)m, sizeof(i64));
  i64 *g = (i64 *)calloc((size_t)m + 1, sizeof(i64));
  i64 *w = (i64 *)calloc((size_t)n, sizeof(i64));
  i64 *yv = (i64 *)calloc((size_t)n, sizeof(i64));
  double *r = (double *)calloc((size_t)n, sizeof(double));
  double *t = (double *)calloc((size_t)n, sizeof(double));
  if (V_out) memset(V_out, 0, sizeof(i64) * (size_t)(m + 1) * n);
  if (Hraw_out) memset(Hraw_out, 0, sizeof(i64) * (size_t)(m + 1) * m);
  int jeff = 0, early = 0;
  double nu;

  /* line 1 (FP): r0 = bk - Abar xk; line 1': r0 = Mbar^-1 (bk - Abar xk) */
  resid_fp_int(n, S->rowptr, S->col, S->ns, S->abar, S->alphas, xk, bk, r);
  if (P->precond) {
    or_lsolve_fp(n, S->rowptr, S->col, S->fac, S->ldiag, r, t);
    or_usolve_fp(n, S->rowptr, S->col, S->fac, S->udiag, t, r);
  }
  nu = or_norm2(n, r);
  if (nu == 0.0) goto done;

  /* line 1: v1 = r0/||r0||; line 2: cast v1 * 2^df to an integer */
  for (int l = 0; l < n; ++l) {
    double v = ldexp(r[l] / nu, df);
    if (!(fabs(v) < 9223372036854775808.0)) { ev[EV_L2]++; V[l] = 0; continue; }
    V[l] = (i64)v;
  }
  /* line 3: g = (1, 0, ..., 0) in Q(df) */
  g[0] = (i64)1 << df;

  for (int j = 0; j < m; ++j) {
    i64 *vj = V + (size_t)j * n;
    /* line 5: w = Abar v_j;  line 5': w = Ubar^-1 Lbar^-1 Abar v_j */
    if (S->ns > 0)
      or_spmv_int_s(n, S->rowptr, S->col, S->ns, S->abar, S->alphas, vj, w, &ev[EV_L5]);
    else
      or_spmv_int(n, S->rowptr, S->col, S->abar, vj, w, &ev[EV_L5]);
    if (P->precond) {
      or_lsolve_int(n, S->rowptr, S->col, S->fac, S->ldiag, w, yv, &ev[EV_L5P]);
      or_usolve_int(n, S->rowptr, S->col, S->fac, S->udiag, yv, w, &ev[EV_L5P]);
    }
    /* lines 6-9: modified Gram-Schmidt */
    for (int i = 0; i <= j; ++i) {
      const i64 *vi = V + (size_t)i * n;
      /* line 7: h_ij = (w, v_i); only w is shifted (beta2 = 0) */
      i128 cs7 = 0;
      for (int l = 0; l < n; ++l) cs7 += (i128)mul(shr(w[l], P->beta7), vi[l], &ev[EV_L7]);
      if (out64(cs7)) ev[EV_L7]++;
      i64 hij = shr(wrap64(cs7), df - P->beta7);
      H[i + j * ld] = hij;
      /* line 8: w = w - h_ij v_i; only h_ij is shifted */
      i64 hs = shr(hij, P->beta8);
      for (int l = 0; l < n; ++l) {
        i64 p = shr(mul(hs, vi[l], &ev[EV_L8]), df - P->beta8);
        i128 d = (i128)w[l] - (i128)p;
        if (out64(d)) ev[EV_L8]++;
        w[l] = wrap64(d);
      }
    }
    /* line 10: h_{j+1,j} = ||w||, beta1 = beta2 = beta10 */
    i128 s10 = 0;
    for (int l = 0; l < n; ++l) {
      i64 a = shr(w[l], P->beta10);
      s10 += (i128)mul(a, a, &ev[EV_L10]);
    }
    if (out64(s10)) ev[EV_L10]++;
    i64 hnext = or_fx_sqrt(wrap64(s10), 2 * df - 2 * P->beta10, df, &ev[EV_L10]);
    H[j + 1 + j * ld] = hnext;
    if (Hraw_out)
      for (int i = 0; i <= j + 1; ++i) Hraw_out[i + j * ld] = H[i + j * ld];

    /* line 11: v_{j+1} = w / h_{j+1,j}; a zero shifted divisor ends the
     * solve after this column (breakdown) */
    int zero;
    {
      i64 d = shr(hnext, P->beta11b);
      zero = (d == 0);
      if (!zero) {
        i64 *vn = V + (size_t)(j + 1) * n;
        for (int l = 0; l < n; ++l) {
          int zz;
          i64 q = or_fx_div(w[l], hnext, P->beta11a, P->beta11b, df, &ev[EV_L11], &zz);
          if (q < INT32_MIN || q > INT32_MAX) ev[EV_VRANGE]++;
          vn[l] = q;
        }
      }
    }

    /* lines 12-14: apply the previous rotations to column j */
    for (int i = 0; i < j; ++i) {
      i64 a = shr(H[i + j * ld], P->beta13), b = shr(H[i + 1 + j * ld], P->beta13);
      i64 p1 = mul(cs[i], a, &ev[EV_L13]), p2 = mul(sn[i], b, &ev[EV_L13]);
      i128 t1 = (i128)p1 + (i128)p2;
      if (out64(t1)) ev[EV_L13]++;
      i64 p3 = mul(neg(sn[i], &ev[EV_L13]), a, &ev[EV_L13]), p4 = mul(cs[i], b, &ev[EV_L13]);
      i128 t2 = (i128)p3 + (i128)p4;
      if (out64(t2)) ev[EV_L13]++;
      H[i + j * ld] = shr(wrap64(t1), df - P->beta13);
      H[i + 1 + j * ld] = shr(wrap64(t2), df - P->beta13);
    }
    /* line 15: t = sqrt(h_jj^2 + h_{j+1,j}^2) */
    i64 hjj = H[j + j * ld], hj1 = H[j + 1 + j * ld];
    i64 a15 = shr(hjj, P->beta15), b15 = shr(hj1, P->beta15);
    i128 s15 = (i128)mul(a15, a15, &ev[EV_L15]) + (i128)mul(b15, b15, &ev[EV_L15]);
    if (out64(s15)) ev[EV_L15]++;
    i64 tmp = or_fx_sqrt(wrap64(s15), 2 * df - 2 * P->beta15, df, &ev[EV_L15]);
    /* line 16: c_j = h_jj / t, s_j = h_{j+1,j} / t */
    int z16;
    i64 c = or_fx_div(hjj, tmp, P->beta16a, P->beta16b, df, &ev[EV_L16], &z16);
    i64 s = or_fx_div(hj1, tmp, P->beta16a, P->beta16b, df, &ev[EV_L16], &z16);
    if (z16) { early = 1; break; }   /* singular column: use j columns */
    cs[j] = c;
    sn[j] = s;
    /* line 17: g_{j+1} = -s_j g_j, g_j = c_j g_j (both from the old g_j),
     * no operand shift */
    i64 gj = g[j];
    g[j + 1] = shr(mul(neg(s, &ev[EV_L17]), gj, &ev[EV_L17]), df);
    g[j] = shr(mul(c, gj, &ev[EV_L17]), df);
    /* lines 18-19 */
    H[j + j * ld] = tmp;
    H[j + 1 + j * ld] = 0;
    jeff = j + 1;
    if (zero) { early = 1; break; }
  }

  /* lines 21-23 (FP): cast g and H, y = ||r0|| H^-1 g, x += sum y_i v_i */
  if (jeff > 0) {
    double *z = (double *)calloc((size_t)jeff, sizeof(double));
    for (int a = jeff - 1; a >= 0; --a) {
      double acc = ldexp((double)g[a], -df);
      for (int b = a + 1; b < jeff; ++b) {
        double p = ldexp((double)H[a + b * ld], -df) * z[b];
        acc = acc - p;
      }
      z[a] = acc / ldexp((double)H[a + a * ld], -df);
    }
    for (int a = 0; a < jeff; ++a) z[a] = nu * z[a];
    for (int l = 0; l < n; ++l) {
      double acc = xk[l];
      for (int i = 0; i < jeff; ++i) {
        double p = z[i] * ldexp((double)V[(size_t)i * n + l], -df);
        acc = acc + p;
      }
      xk[l] = acc;
    }
    free(z);
  }

done:
  if (H_out) memcpy(H_out, H, sizeof(i64) * (size_t)(m + 1) * m);
  if (cs_out) memcpy(cs_out, cs, sizeof(i64) * (size_t)m);
  if (sn_out) memcpy(sn_out, sn, sizeof(i64) * (size_t)m);
  if (g_out) memcpy(g_out, g, sizeof(i64) * (size_t)(m + 1));
  if (jeff_out) *jeff_out = jeff;
  if (nu_out) *nu_out = nu;
  if (!V_out) free(V);
  free(H); free(cs); free(sn); free(g); free(w); free(yv); free(r); free(t);
  return early;
}

/* ------------------------------------------------------------------ */
/* FP64 GMRES(m), the "Double" solver of Sec. VII                       */
/* ------------------------------------------------------------------ */
/* Standard restarted-GMRES cycle: left ILU(0) preconditioning with the FP64
 * factors (unit L, non-unit U), modified Gram-Schmidt, Givens rotations.
 * Plain sequential sums (this is the comparison solver, not the parity
 * path).  f is the output of or_ilu0.  Adds the correction to xk. */
int or_fp_gmres(int n, const int *rowptr, const int *col, const double *a,
                const double *f, const int *diagpos, int m, int precond,
                const double *bk, double *xk, int *jeff_out) {
  int ld = m + 1, jeff = 0;
  double *V = (double *)calloc((size_t)(m + 1) * n, sizeof(double));
  double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)calloc((size_t)m, sizeof(double));
  double *sn = (double *)calloc((size_t)m, sizeof(double));
  double *g = (double *)calloc((size_t)m + 1, sizeof(double));
  double *w = (double *)calloc((size_t)n, sizeof(double));
  double *t = (double *)calloc((size_t)n, sizeof(double));
  double *r = (double *)calloc((size_t)n, sizeof(double));

  or_resid_fp(n, rowptr, col, a, xk, bk, r);
#define FP_PREC(src, dst)                                                        \
  do {                                                                           \
    for (int i = 0; i < n; ++i) {                                                \
      double acc = (src)[i];                                                     \
      for (int k = rowptr[i]; k < rowptr[i + 1] && col[k] < i; ++k)              \
        acc = acc - f[k] * t[col[k]];                                            \
      t[i] = acc;                                                                \
    }                                                                            \
    for (int i = n - 1; i >= 0; --i) {                                           \
      double acc = t[i];                                                         \
      for (int k = diagpos[i] + 1; k < rowptr[i + 1]; ++k)                       \
        acc = acc - f[k] * (dst)[col[k]];                                        \
      (dst)[i] = acc / f[diagpos[i]];                                            \
    }                                                                            \
  } while (0)
  if (precond) FP_PREC(r, r);
  double beta = 0.0;
  for (int l = 0; l < n; ++l) beta += r[l] * r[l];
  beta = sqrt(beta);
  if (beta == 0.0) goto out;
  for (int l = 0; l < n; ++l) V[l] = r[l] / beta;
  g[0] = beta;
  for (int j = 0; j < m; ++j) {
    double *vj = V + (size_t)j * n;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s = s + a[k] * vj[col[k]];
      w[i] = s;
    }
    if (precond) FP_PREC(w, w);
    for (int i = 0; i <= j; ++i) {
      double *vi = V + (size_t)i * n, h = 0.0;
      for (int l = 0; l < n; ++l) h += w[l] * vi[l];
      H[i + j * ld] = h;
      for (int l = 0; l < n; ++l) w[l] -= h * vi[l];
    }
    double hn = 0.0;
    for (int l = 0; l < n; ++l) hn += w[l] * w[l];
    hn = sqrt(hn);
    H[j + 1 + j * ld] = hn;
    if (hn != 0.0)
      for (int l = 0; l < n; ++l) V[(size_t)(j + 1) * n + l] = w[l] / hn;
    for (int i = 0; i < j; ++i) {
      double x1 = H[i + j * ld], x2 = H[i + 1 + j * ld];
      H[i + j * ld] = cs[i] * x1 + sn[i] * x2;
      H[i + 1 + j * ld] = -sn[i] * x1 + cs[i] * x2;
    }
    double hjj = H[j + j * ld], hj1 = H[j + 1 + j * ld];
    double tmp = sqrt(hjj * hjj + hj1 * hj1);
    if (tmp == 0.0) break;
    cs[j] = hjj / tmp;
    sn[j] = hj1 / tmp;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    H[j + j * ld] = tmp;
    H[j + 1 + j * ld] = 0.0;
    jeff = j + 1;
    if (hn == 0.0) break;
  }
  for (int q = jeff - 1; q >= 0; --q) {
    double acc = g[q];
    for (int b = q + 1; b < jeff; ++b) acc -= H[q + b * ld] * t[b];
    t[q] = acc / H[q + q * ld];
  }
  for (int l = 0; l < n; ++l) {
    double acc = xk[l];
    for (int i = 0; i < jeff; ++i) acc += t[i] * V[(size_t)i * n + l];
    xk[l] = acc;
  }
#undef FP_PREC
out:
  if (jeff_out) *jeff_out = jeff;
  free(V); free(H); free(cs); free(sn); free(g); free(w); free(t); free(r);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Iterative refinement, Fig. 1                                          */
/* ------------------------------------------------------------------ */

/* Solves Ahat xhat = bhat.  inner = 0: int-GMRES (Fig. 2); inner = 1: the
 * FP64 GMRES(m) cycle in the same refinement loop ("Double" solver).
 * xhat (n) receives the solution.  Stops when the scaled relative residual
 * of Fig. 1 is below tol (status OR_OK), or after max_refine inner solves or
 * when the residual has not decreased over the last three refinements
 * (OR_ENOCONV). */
static int ir_solve_natural(const or_params *P, int inner, int n, const int *rowptr,
                            const int *col, const double *ahat, const double *bhat,
                            double *xhat, or_report *rep);

int or_ir_solve(const or_params *P, int inner, int n, const int *rowptr,
                const int *col, const double *ahat, const double *bhat,
                double *xhat, or_report *rep) {
  if (P->order != 1) return ir_solve_natural(P, inner, n, rowptr, col, ahat, bhat, xhat, rep);
  /* multicolour order: the method on P A P^T (P x) = P b */
  const int nnz = rowptr[n];
  int *perm = (int *)malloc(sizeof(int) * (size_t)(n ? n : 1));
  int *cptr = (int *)malloc(sizeof(int) * ((size_t)n + 1));
  int *rp2 = (int *)malloc(sizeof(int) * ((size_t)n + 1));
  int *cl2 = (int *)malloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
  double *av2 = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  double *b2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double *x2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  or_mc_order(n, rowptr, col, perm, cptr);
  or_permute_csr(n, rowptr, col, ahat, perm, rp2, cl2, av2);
  for (int r = 0; r < n; ++r) b2[r] = bhat[perm[r]];
  int st = ir_solve_natural(P, inner, n, rp2, cl2, av2, b2, x2, rep);
  for (int r = 0; r < n; ++r) xhat[perm[r]] = x2[r];
  free(perm); free(cptr); free(rp2); free(cl2); free(av2); free(b2); free(x2);
  return st;
}

/* Shift auto-tuning (Sec. VII-D names it for the solver without
 * preconditioning and gives no rule; this is the reading used here).  The
 * lines whose shift beta divides an operand before a product or a sum of
 * products are 7, 8, 10, 13 and 15 (Table 3): a larger beta makes their
 * words smaller.  After a cycle that raised overflow events at any of them,
 * each such line whose beta is below d_f gets beta + 1; returns 1 if a shift
 * was raised (the cycle is then discarded and run again), else 0. */
static int raise_shifts(or_params *Pk, const i64 *evc) {
  const int line[5] = {EV_L7, EV_L8, EV_L10, EV_L13, EV_L15};
  int *beta[5] = {&Pk->beta7, &Pk->beta8, &Pk->beta10, &Pk->beta13, &Pk->beta15};
  int raised = 0;
  for (int t = 0; t < 5; ++t)
    if (evc[line[t]] > 0 && *beta[t] < Pk->df) {
      *beta[t] += 1;
      raised = 1;
    }
  return raised;
}

static int ir_solve_natural(const or_params *P, int inner, int n, const int *rowptr,
                            const int *col, const double *ahat, const double *bhat,
                            double *xhat, or_report *rep) {
  int nnz = rowptr[n], st;
  memset(rep, 0, sizeof(*rep));
  double *a = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
  double *b = (double *)malloc(sizeof(double) * (size_t)n);
  double *d = (double *)malloc(sizeof(double) * (size_t)n);
  const int S_req = P->s < 0 ? 0 : (P->s > OR_MAX_S ? OR_MAX_S : P->s);
  i64 *abar = (i64 *)malloc(sizeof(i64) * (size_t)(nnz ? nnz : 1) * (size_t)(S_req + 1));
  int alphas[OR_MAX_S + 1] = {0};
  int ns = 0;
  double *f = NULL;
  int *diagpos = NULL;
  i64 *fac = NULL, *ldg = NULL, *udg = NULL;
  double *x = (double *)calloc((size_t)n, sizeof(double));
  double *bp = (double *)malloc(sizeof(double) * (size_t)n);
  double *xk = (double *)malloc(sizeof(double) * (size_t)n);

  st = or_scale(n, rowptr, col, ahat, bhat, P->alpha_a, a, b, d);
  if (st) goto out;
  st = or_cast(nnz, a, abar);
  if (st) goto out;
  if (S_req > 0) ns = or_multiterm(nnz, a, P->alpha_a, S_req, abar, alphas);
  if (P->precond) {
    f = (double *)malloc(sizeof(double) * (size_t)nnz);
    diagpos = (int *)malloc(sizeof(int) * (size_t)n);
    fac = (i64 *)malloc(sizeof(i64) * (size_t)nnz);
    ldg = (i64 *)malloc(sizeof(i64) * (size_t)n);
    udg = (i64 *)malloc(sizeof(i64) * (size_t)n);
    st = P->precond == 2 ? or_gs_factors(n, rowptr, col, a, f, diagpos)
                         : or_ilu0(n, rowptr, col, a, f, diagpos);
    if (st) goto out;
    st = or_ilu_int(n, rowptr, col, f, diagpos, fac, ldg, udg);
    if (st) goto out;
  }
  {
    or_system S = {n, rowptr, col, abar, fac, ldg, udg, ns, alphas};
    double nb = or_norm2(n, b);
    st = OR_ENOCONV;
    double ring[4] = {0.0, 0.0, 0.0, 0.0};   /* the last residuals */
    or_params Pk = *P;                        /* the shifts in use     */
    for (int k = 0;; ++k) {
      /* b' = b - A x (FP) and the test of Fig. 1 */
      or_resid_fp(n, rowptr, col, a, x, b, bp);
      double rho = nb == 0.0 ? 0.0 : or_norm2(n, bp) / nb;
      if (k < 65) rep->relres_hist[k] = rho;
      rep->relres = rho;
      /* stalled: no decrease over the last three refinements */
      int stall = k >= 3 && rho >= ring[(k - 3) & 3];
      ring[k & 3] = rho;
      if (rho < P->tol) { st = OR_OK; break; }
      if (k >= P->max_refine || stall) { st = OR_ENOCONV; break; }
      /* eq. (gammak), eq. (scale) */
      double gam = or_maxabs(n, bp);
      if (k < 64) rep->gamma_hist[k] = gam;
      for (int l = 0; l < n; ++l) bp[l] = bp[l] / gam;
      int jeff = 0;
      if (inner == 0) {
        /* the cycle with the current shifts; with auto-tuning, a cycle that
         * overflowed at a shifted line is discarded (x is not updated, the
         * refinement is not counted) and rerun from the same b^(k) */
        for (;;) {
          i64 evc[EV_COUNT] = {0};
          memset(xk, 0, sizeof(double) * (size_t)n);
          jeff = 0;
          int early = or_int_gmres(&Pk, &S, bp, xk, NULL, NULL, NULL, NULL, NULL, NULL,
                                   &jeff, NULL, evc);
          for (int e = 0; e < EV_COUNT; ++e) rep->ev[e] += evc[e];
          if (rep->shift_retries < P->shift_tune && raise_shifts(&Pk, evc)) {
            rep->shift_retries++;
            continue;
          }
          if (early) rep->breakdowns++;
          break;
        }
      } else {
        memset(xk, 0, sizeof(double) * (size_t)n);
        or_fp_gmres(n, rowptr, col, a, f, diagpos, P->m, P->precond, bp, xk, &jeff);
      }
      rep->refinements++;
      rep->inner_steps += jeff;
      /* eq. (update): x += gamma x^(k) */
      for (int l = 0; l < n; ++l) {
        double p = gam * xk[l];
        x[l] = x[l] + p;
      }
    }
    rep->beta_final[0] = Pk.beta7;
    rep->beta_final[1] = Pk.beta8;
    rep->beta_final[2] = Pk.beta10;
    rep->beta_final[3] = Pk.beta13;
    rep->beta_final[4] = Pk.beta15;
    memcpy(xhat, x, sizeof(double) * (size_t)n);
    /* residual of the original system, for reporting */
    or_resid_fp(n, rowptr, col, ahat, x, bhat, bp);
    double nbh = or_norm2(n, bhat);
    rep->relres_unscaled = nbh == 0.0 ? 0.0 : or_norm2(n, bp) / nbh;
  }
out:
  rep->status = st;
  free(a); free(b); free(d); free(abar); free(f); free(diagpos);
  free(fac); free(ldg); free(udg); free(x); free(bp); free(xk);
  return st;
}

/* entry points that expose or_int_gmres with plain arguments for the
 * Python test harness */
int or_int_gmres_flat(const or_params *P, int n, const int *rowptr, const int *col,
                      const i64 *abar, const i64 *fac, const i64 *ldiag,
                      const i64 *udiag, const double *bk, double *xk, i64 *V,
                      i64 *H, i64 *Hraw, i64 *cs, i64 *sn, i64 *g, int *jeff,
                      double *nu, i64 *ev) {
  static const int a0[1] = {0};
  or_system S = {n, rowptr, col, abar, fac, ldiag, udiag, 0, a0};
  return or_int_gmres(P, &S, bk, xk, V, H, Hraw, cs, sn, g, jeff, nu, ev);
}

/* the same with ns correction terms: terms (ns+1) x nnz, alphas ns+1 */
int or_int_gmres_flat_s(const or_params *P, int n, const int *rowptr, const int *col,
                        int ns, const i64 *terms, const int *alphas, const i64 *fac,
                        const i64 *ldiag, const i64 *udiag, const double *bk, double *xk,
                        i64 *V, i64 *H, i64 *Hraw, i64 *cs, i64 *sn, i64 *g, int *jeff,
                        double *nu, i64 *ev) {
  or_system S = {n, rowptr, col, terms, fac, ldiag, udiag, ns, alphas};
  return or_int_gmres(P, &S, bk, xk, V, H, Hraw, cs, sn, g, jeff, nu, ev);
}

int or_sizeof_params(void) { return (int)sizeof(or_params); }
int or_sizeof_report(void) { return (int)sizeof(or_report); }
