/*
 * igm.h -- C ABI of the GB300 (sm_103a) integer-arithmetic GMRES solver with
 * FP64 iterative refinement.
 *
 * Method: T. Iwashita, K. Suzuki, T. Fukaya, "An Integer Arithmetic-Based
 * Sparse Linear Solver Using a GMRES Method and Iterative Refinement",
 * ScalA'20 (arXiv:2009.07495).  Section, equation, figure and table numbers
 * below refer to that paper.
 *
 * Conventions shared by every entry point
 *  - Matrices are CSR: rowptr int32[n+1] (rowptr[0] = 0), col int32[nnz]
 *    with columns strictly ascending inside each row, val float64[nnz].
 *    With ILU(0) every row must store its diagonal.
 *  - Array arguments may be device pointers or host pointers (pageable or
 *    pinned); the library detects which (cudaPointerGetAttributes) and, for
 *    host memory, copies on `stream` and synchronises before returning.
 *    Device inputs are read in stream order on `stream`.
 *  - Ownership: the library never keeps caller pointers.  Setup copies what
 *    it needs into memory owned by the handle; outputs are written into
 *    caller memory on `stream`.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - Every call returns an igm_status and never throws or aborts.  Device
 *    waits are bounded: an expired wait is reported as IGM_ETIMEOUT, never
 *    as a hang or a trap.  igm_last_error() returns a message for the last
 *    failing call of the calling thread.
 *  - Overflow of a fixed-point word is not an error (the paper's hardware
 *    wraps too): each event is counted per line of Fig. 2 in the report.
 *  - Handles are not thread-safe; one handle may be used by one stream at a
 *    time.  Different handles are independent.
 */
#ifndef IGM_H
#define IGM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct igm_handle_s *igm_handle;
typedef struct igm_server_s *igm_server;

typedef enum {
  IGM_OK = 0,
  IGM_EINVAL = 1,       /* malformed argument or matrix                     */
  IGM_EZERO_ROW = 2,    /* a row of A is zero: eq. (3) has no scale        */
  IGM_EZERO_PIVOT = 3,  /* ILU(0) pivot (or its integer cast) is zero       */
  IGM_EBREAKDOWN = 4,   /* reserved                                         */
  IGM_ENOCONV = 5,      /* Fig. 1 loop reached max_refine above tol         */
  IGM_EOOM = 6,         /* device memory budget or cudaMalloc exhausted     */
  IGM_ETIMEOUT = 7,     /* a bounded device wait expired                    */
  IGM_ECUDA = 8         /* a CUDA runtime call failed (in the library's
                           "checks" build variant also: a device bounds or
                           alignment check failed; igm_last_error names
                           the site)                                        */
} igm_status;

/* Indices of igm_report.ev: overflow events per line of Fig. 2. */
enum {
  IGM_EV_L5 = 0,     /* line 5: integer matrix-vector product              */
  IGM_EV_L5P = 1,    /* line 5': integer forward/backward substitution     */
  IGM_EV_L7 = 2,     /* line 7: inner product                              */
  IGM_EV_L8 = 3,     /* line 8: vector update                              */
  IGM_EV_L10 = 4,    /* line 10: norm                                      */
  IGM_EV_L11 = 5,    /* line 11: vector / scalar                           */
  IGM_EV_L13 = 6,    /* line 13: previous Givens rotations                 */
  IGM_EV_L15 = 7,    /* line 15: 2-element norm                            */
  IGM_EV_L16 = 8,    /* line 16: c, s divisions                            */
  IGM_EV_L17 = 9,    /* line 17: g update                                  */
  IGM_EV_VRANGE = 10,/* a basis entry outside int32 (informational)       */
  IGM_EV_L2 = 11,    /* line 2: FP -> int cast out of range                */
  IGM_EV_COUNT = 16
};

/* Parameters of the method (Sec. II, III, V-D, VII; Tables 3-5). */
typedef struct {
  int df;        /* fractional bits d_f of the Q(d_m).(d_f) int64 word (30)  */
  int alpha_a;   /* initial scaling exponent of eq. (3): 16 none, 32 ILU     */
  int m;         /* Arnoldi steps per inner solve, 1..IGM_MAX_M              */
  int precond;   /* 0: none; 1: integer ILU(0) (Sec. VI-A, lines 1', 5');   
                    2: integer Gauss-Seidel (Sec. VII-D), D + L_A in the
                    factor form of Sec. VI-A (Table 5 shifts by default) */
  int beta7;     /* line 7: shift of w (beta1; beta2 = 0)                    */
  int beta8;     /* line 8: shift of h (beta1)                               */
  int beta10;    /* line 10: beta1 = beta2                                   */
  int beta11a, beta11b; /* line 11: divide, beta1 (x2^) and beta2 (/2^)      */
  int beta13;    /* line 13: shift of h (beta2; beta1 = 0)                   */
  int beta15;    /* line 15: beta1 = beta2                                   */
  int beta16a, beta16b; /* line 16: divide                                   */
  double tol;    /* epsilon of Fig. 1 (relative residual of the scaled system)*/
  int max_refine;/* maximum inner solves in Fig. 1                           */
  int inner;     /* 0: int-GMRES (Fig. 2); 1: FP64 GMRES(m) ("Double")       */
  int trsv_chunk;/* rows per chunk of the line-5' substitutions (0: automatic)*/
  int trsv_cluster;/* kept for layout compatibility: 0, 1, 2, 4 or 8 are
                    accepted and ignored (the substitutions hand values
                    between chunks through global memory, with no
                    thread-block clusters)                                 */
  int s;         /* correction terms of Sec. IV-C, eq. (AA), used in every
                    refinement (s(k) = s, 0 ... IGM_MAX_S): the matrix is
                    Abar_0 + sum_l Abar_l / 2^alpha_l and line 5 adds each
                    term's product shifted right by alpha_l (eq. matvec)  */
  int order;     /* 0: natural row order (the paper's); 1: multicolour order
                    (greedy colouring of the symmetrised pattern, rows by
                    colour): the method runs on P A P^T (P x) = P b, so the
                    substitutions have as many levels as colours (a
                    different preconditioner than the natural order's); b
                    and x stay in the caller's order                      */
  int shift_tune;/* shift auto-tuning (Sec. VII-D), 0 ... 64 (0: off, the
                    shifts stay as given, as in Tables 4 and 5): in the
                    refinement loop, an inner solve that raised overflow
                    events at lines 7, 8, 10, 13 or 15 of Fig. 2 raises the
                    shift of each such line by one (up to d_f), is
                    discarded (x is not updated, the refinement is not
                    counted) and runs again from the same b^(k); at most
                    shift_tune inner solves are discarded per solve, and
                    every solve starts from the shifts given here.  Not
                    used by int_gmres_solve.                              */
  /* Launch-configuration knobs (the results do not depend on them; tests use
     them to reach every code path on small systems). */
  int mgs_wmax;  /* rows one CTA of the Arnoldi step (lines 5/6-11) may keep
                    resident in shared memory (w and the int32 basis words):
                    0 automatic (13,952; 3,584 when the step streams the
                    CTA's further rows through the copy engine, which it
                    does for preconditioned systems with more rows a CTA
                    than that), -1 none, k > 0 at most k rows; a CTA's
                    further rows keep w in global memory.  In a batch the
                    first system's value applies.                         */
  int wait_us;   /* bound of each device wait of the line-1'/5' substitutions
                    in microseconds (0: 1 s); an expired wait ends the call
                    with IGM_ETIMEOUT                                      */
  int test_stall;/* tests of the bounded waits only: 1 = the first chunk of
                    every substitution never signals its progress, so the
                    next chunk's wait expires and the call returns
                    IGM_ETIMEOUT (0 in normal use)                         */
  int fuse_steps;/* integer systems without preconditioner and correction
                    terms: Arnoldi steps (lines 5-19 each) per persistent
                    launch; 0 chosen by the autotuner, -1 one SpMV launch
                    and one Arnoldi launch per step, k > 0 k steps         */
  int plan_snap; /* partition of the rows over the Arnoldi CTAs: 0 chosen
                    by the autotuner, -1 equal shares, k in 1..100 a share
                    boundary inside a system moves to the system's nearer
                    end when within k % of a share.  The autotuner (fused
                    systems only; the first refinement call of a batch or
                    handle) times the m steps of one inner solve for each
                    choice left to it and keeps the fastest; the results do
                    not depend on either knob.  In a batch the first
                    system's values apply.                                 */
  int reserved[2];
} igm_params;

#define IGM_MAX_M 128
#define IGM_MAX_S 4

/* Per-solve report.  Histories are indexed by refinement k (Fig. 1). */
typedef struct {
  long long ev[IGM_EV_COUNT]; /* overflow events per line of Fig. 2         */
  int refinements;            /* inner solves performed                     */
  int inner_steps;            /* Arnoldi steps over all inner solves        */
  int breakdowns;             /* inner solves that ended before m steps     */
  int status;                 /* igm_status of the solve                    */
  double relres;              /* final ||b - A x|| / ||b||, scaled system   */
  double relres_unscaled;     /* final ||bh - Ah xh|| / ||bh||              */
  double gamma_hist[64];      /* gamma^(k) of eq. (gammak)                  */
  double relres_hist[65];     /* relative residual before refinement k      */
  int shift_retries;          /* inner solves discarded by shift_tune       */
  int beta_final[5];          /* beta7, beta8, beta10, beta13, beta15 at the
                                 end of the solve                           */
  int fuse_steps;             /* launch configuration the solve ran with:
                                 Arnoldi steps per fused launch (0 none)    */
  int plan_snap;              /* ... and the partition's snap (0 equal)     */
} igm_report;

/* Fills p with the paper's settings: d_f = 30 (Sec. VII-B); precond = 0:
 * alpha_a = 16 and the shifts of Table 4; precond = 1: alpha_a = 32 and the
 * shifts of Table 5; tol = 1e-10, max_refine = 60, inner = 0. */
igm_status igm_params_default(igm_params *p, int precond, int m);

/* Setup of Fig. 1 on the device (steps before the refinement loop):
 * the initial row scaling of eq. (1)/(3), the cast of Sec. IV-B
 * (Abar_0 = trunc(A), s = 0), and with precond = 1 the FP64 ILU(0) of
 * eq. (ilu) and its integer factors Lbar, Ubar of eq. (dldr)-(ilu2).
 * n >= 1 rows, nnz entries; rowptr/col/val as in the conventions above.
 * On success *out owns all device state of the system: about 40 bytes per
 * stored entry (the scaled, cast and SELL-32 copies of A) plus
 * 12 (m + 1) + 92 bytes per row (the basis as int64 and int32 words, work
 * vectors); precond = 1 adds about 16 bytes per entry and 24 K + 120 bytes
 * per row (factors, schedules and packed substitution blocks; K the
 * longest strict row of a factor).  int_gmres_device_bytes gives the exact
 * figure.  Errors: IGM_EINVAL, IGM_EZERO_ROW, IGM_EZERO_PIVOT, IGM_EOOM,
 * IGM_ECUDA. */
igm_status int_gmres_setup(int n, int nnz, const int *rowptr, const int *col,
                           const double *val, const igm_params *params,
                           void *stream, igm_handle *out);

/* One inner solve of Fig. 2 (lines 1-23; lines 1', 5' with precond = 1) on
 * the SCALED system of the handle, with the argument types of Table 2:
 * bk (n doubles, input) is b^(k), xk (n doubles, input/output) is the
 * initial guess on entry and the guess plus the int-GMRES correction on
 * return.  rep may be NULL; if given, ev/inner_steps/breakdowns describe
 * this solve. */
igm_status int_gmres_solve(igm_handle h, const double *bk, double *xk,
                           igm_report *rep, void *stream);

/* The refinement loop of Fig. 1 for the ORIGINAL system Ah xh = bh:
 * b = D^-1 bh, then repeat { r = b - A x; stop if ||r||/||b|| < tol;
 * gamma = max|r_i|; inner solve of A x^(k) = r/gamma; x += gamma x^(k) },
 * xh = x (eq. 1 leaves x unscaled).  bhat, xhat: n doubles.  rep may be
 * NULL.  Returns IGM_ENOCONV when max_refine is reached first, or when
 * ||r||/||b|| has not decreased over the last three refinements (a stall). */
igm_status ir_solve(igm_handle h, const double *bhat, double *xhat,
                    igm_report *rep, void *stream);

/* ir_solve for `count` independent systems in one launch sequence: every
 * kernel covers all systems at once (block-diagonal tiling), each system
 * keeps its own refinement state and stops independently, and each result
 * is bit-identical to ir_solve on that handle alone.  hs[i], bhat[i],
 * xhat[i] (device or host), reps[i] (may be NULL as a whole).  The handles
 * must be distinct and share one m. */
igm_status ir_solve_batched(int count, igm_handle *hs, const double *const *bhat,
                            double *const *xhat, igm_report *reps, void *stream);

/* Copies the integer state of the last inner solve to caller memory (host
 * or device), for inspection and tests; any pointer may be NULL.
 * V: (m+1)*n int64 (basis, row-major by vector), H: (m+1)*m int64
 * (column-major, after the Givens rotations of lines 12-19), cs, sn: m,
 * g: m+1, jeff: Arnoldi columns used, nu: ||r0|| of line 1. */
igm_status int_gmres_get_state(igm_handle h, long long *V, long long *H,
                               long long *cs, long long *sn, long long *g,
                               int *jeff, double *nu);

/* The reproducible FP64 2-norm used by the test of Fig. 1: with
 * e = ilogb(max|x_i|), each (x_i 2^-e)^2 is formed exactly (product plus its
 * FMA error), both parts are truncated to multiples of 2^-96 and summed
 * exactly in integers, the total is rounded once to double, scaled back and
 * square-rooted.  The result does not depend on the order of the elements or
 * of the reduction, and is within one ulp of the exact norm.  x: n doubles
 * (device or host); out: one double (device or host).  Device scratch is
 * taken from a library-owned workspace, allocated on the first call for the
 * largest n seen.  Errors: IGM_EINVAL, IGM_EOOM, IGM_ECUDA. */
igm_status igm_norm2(const double *x, int n, double *out, void *stream);

/* igm_norm2 for callers that cannot allocate device memory (a stream being
 * captured into a CUDA graph, a process whose device memory belongs to
 * another allocator, a latency-critical loop).  The paper has no
 * counterpart: this is an operational variant of the same computation.
 * Scratch (per-CTA partial sums and counters, 32 KB) lives in a static
 * device array held by every GPU that loads the library until the process
 * exits; the call allocates nothing.  x: n doubles and out: one double,
 * both already in device (or managed) memory of the current device (memory
 * of another device is refused with IGM_EINVAL); 0 <= n <= 8,388,608,
 * larger n is rejected with IGM_EINVAL.  The first call on each device resolves the
 * array's device address; make that first call before any stream capture.
 * All calls share the array: calls whose GPU work overlaps (other streams
 * or threads on the same device) race; calls on one stream are ordered.
 * The result is written on `stream` (no synchronisation). */
igm_status igm_norm2_noalloc(const double *x, int n, double *out, void *stream);

/* Kernels that igm_time_kernels can time (one launch each, on the handle's
 * current state, in the launch configuration of the solver). */
enum {
  IGM_K_SPMV = 0,       /* line 5, step j = m/2                            */
  IGM_K_TRSV_L = 1,     /* line 5' forward substitution                    */
  IGM_K_TRSV_U = 2,     /* line 5' backward substitution                   */
  IGM_K_ARNOLDI = 3,    /* lines 6-19 of the last step j = m-1 (m+1 MGS
                           passes, norm, line 11, Givens)                  */
  IGM_K_RESID = 4,      /* eq. (b), FP64 residual of Fig. 1                */
  IGM_K_COUNT = 5
};

/* Average device time per launch (ms) of each kernel kind above, measured
 * with CUDA events around `reps` back-to-back launches on `stream` after a
 * solve has been run on the handle (the launches overwrite the solver's
 * scratch state, not the matrix or the last solution).  ms: IGM_K_COUNT
 * doubles (host), -1 for kinds that do not apply (substitutions without
 * ILU).  Errors: IGM_EINVAL, IGM_ECUDA. */
igm_status igm_time_kernels(igm_handle h, int reps, double *ms, void *stream);

/* Number of kernels the library has launched in this process (a graph
 * launch counts its kernel nodes). */
long long igm_kernel_launches(void);

/* ---- Serving: continuous batching of independent solves ---------------
 * A server owns two threads, each with its CUDA stream.  Submitted requests
 * (host arrays, copied at submission) wait in a FIFO queue; the admission
 * thread admits them in order while the device memory of admitted systems
 * stays within budget_bytes (and at most max_active are admitted; the
 * footprint is estimated before set-up and corrected after it), sets each
 * one up on the device (int_gmres_setup) while rounds run, and keeps its
 * matrix, factors, basis and refinement state resident until it finishes.
 * The round thread's work proceeds in rounds:
 * one convergence test (Fig. 1) and one inner solve (Fig. 2) for every
 * active system in the same kernels; requests that arrive meanwhile join
 * at the next round, finished ones leave.  Each result is bit-identical to
 * ir_solve on the same system alone.  All requests of a server share m and
 * the inner solver (the config's m and inner). */
typedef struct {
  long long budget_bytes; /* device memory for admitted systems (> 0)         */
  int max_active;         /* systems in flight at once (0: no limit)        */
  int m;                  /* restart length every request must use          */
  int inner;              /* 0 int-GMRES, 1 FP64 GMRES                      */
  int reserved[5];
} igm_server_config;

typedef struct {
  long long submitted, completed, failed, rounds;
  long long peak_bytes;        /* largest admitted device memory            */
  double busy_s;               /* worker time spent in rounds               */
} igm_server_stats;

igm_status igm_server_create(const igm_server_config *cfg, igm_server *out);

/* Queues one solve of Ah xh = bh (host CSR arrays and right-hand side,
 * copied before return; params->m and inner must match the server's).
 * *id receives the request id.  Errors: IGM_EINVAL, IGM_EOOM (the system
 * alone exceeds the budget). */
igm_status igm_server_submit(igm_server s, int n, int nnz, const int *rowptr,
                             const int *col, const double *val, const double *bhat,
                             const igm_params *params, long long *id);

/* Waits up to wait_ms (0: no wait, -1: forever) for request id.  *done = 1
 * when finished: xhat (host, n doubles, may be NULL) receives the solution
 * and rep (may be NULL) the report; the request is then forgotten.  The
 * return value is the solve's status once done, IGM_OK while pending.
 * lat_s (may be NULL) receives submit-to-completion seconds. */
igm_status igm_server_poll(igm_server s, long long id, int wait_ms, double *xhat,
                           igm_report *rep, double *lat_s, int *done);

igm_status igm_server_get_stats(igm_server s, igm_server_stats *st);

/* Stops the worker after the current round; pending requests are dropped. */
void igm_server_destroy(igm_server s);

/* Bytes of device memory the handle holds. */
long long int_gmres_device_bytes(igm_handle h);

/* Releases everything the handle owns.  NULL is ignored. */
void int_gmres_destroy(igm_handle h);

/* Message for the last failing call on this thread ("" if none). */
const char *igm_last_error(void);

/* Library version string. */
const char *igm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IGM_H */
