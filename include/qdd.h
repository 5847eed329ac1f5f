/*
 * qdd.h -- C ABI of the GB300 Wilson-clover quark solver with the restricted
 * additive Schwarz (RAS) preconditioner.
 *
 * Method: Osaki & Ishikawa, "Domain Decomposition method on GPU cluster",
 * Lattice 2010.  The library solves the quark equation D phi = eta (Eq. 1)
 * for the O(a)-improved Wilson (Wilson-clover) operator
 *
 *     D = A - kappa H,
 *     (H psi)(x) = sum_mu [ b (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + b (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *     A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x),
 *
 * (kappa and c_SW as in Sec. 5; gamma matrices in the DeGrand-Rossi basis,
 * b = the boundary sign of a hop that wraps around the lattice), with the
 * mixed-precision nested BiCGStab of Sec. 3 whose inner solve is right-
 * preconditioned (Eq. 3) by the RAS iteration of Alg. 1 / Eq. 2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: dims = (Lx, Ly, Lz, Lt), site index i = x + Lx(y + Ly(z + Lz t)),
 * mu = 0..3 <-> x, y, z, t.  bc[mu] = +1 periodic, -1 antiperiodic; the sign
 * multiplies fermion hops that wrap around direction mu.  Gauge links are
 * always periodic.
 *
 * Canonical layouts (all FP64, interleaved complex: re, im):
 *   spinor  double[n_rhs][V][4 spin][3 colour][2] (24 doubles per site and
 *           right-hand side; n_rhs as given to qdd_create_lattice)
 *   gauge   double[V][4 mu][3 row][3 col][2]      (72 doubles per site)
 * Every double* argument may be a DEVICE pointer (cudaMalloc, torch CUDA
 * tensor) or a HOST pointer (pinned or pageable); the library detects which.
 * Host buffers are copied to and from the device inside the call, on the
 * lattice's stream, and a call that writes a host buffer returns only after
 * the data has arrived.  Calls with device buffers are stream-ordered on the
 * stream given to qdd_create_lattice and may return before the GPU is done,
 * except qdd_solve / qdd_solve_batch, which read residual norms on the host
 * and so return after the solve completes.
 *
 * Ownership: the caller owns every buffer it passes; the library never keeps
 * a caller pointer after a call returns.  The library owns the lattice, its
 * internal copies of the links (FP64, FP32 and FP16, 12-real compressed for
 * the reduced precisions), the clover cache keyed by (kappa, c_sw), the
 * solver work vectors and the reduction scratch.
 *
 * Errors: every call returns a qdd_status and never aborts the process.
 * qdd_last_error() returns a description of the last failure on the calling
 * thread.  A call that fails leaves the lattice usable.
 *
 * Threading: a lattice may be used by one host thread at a time.
 */
#ifndef QDD_H
#define QDD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QDD_OK = 0,
    QDD_ERR_ARG = 1,            /* invalid argument (sizes, blocking, null pointer, non-SU(3) link) */
    QDD_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    QDD_ERR_NOMEM = 3,          /* device allocation failed */
    QDD_ERR_NOT_CONVERGED = 4,  /* iteration budget exhausted; phi holds the best iterate */
    QDD_ERR_BREAKDOWN = 5,      /* BiCGStab broke down twice (after one restart) */
    QDD_ERR_NONFINITE = 6,      /* NaN or Inf in a residual norm */
    QDD_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up (a RAS sweep waiting for its
                                   bulk-copied domain data); the results of the call are undefined */
    QDD_ERR_STATE = 8           /* call out of order (e.g. no gauge field loaded) */
} qdd_status;

typedef enum { QDD_F64 = 0, QDD_F32 = 1, QDD_F16 = 2 } qdd_prec;

/* Right-hand sides a lattice can hold (qdd_create_lattice n_rhs). */
#define QDD_MAX_RHS 64
/* Largest lattice volume: every device field plane index (at most 36 planes
 * of V sites) fits in 32 bits. */
#define QDD_MAX_SITES 119304647LL

/* Opaque lattice: geometry, boundary signs, links, clover cache, stream. */
typedef struct qdd_lattice qdd_lattice;

/* Opaque spinor field in the library's internal GPU layout (for repeated
 * application without layout conversion, e.g. throughput measurement). */
typedef struct qdd_field qdd_field;

/* Solver parameters (Sec. 2 and Sec. 5 name block shape, overlap depth
 * d = 2 s, N_dominv and NRAS). */
typedef struct {
    int block[4];       /* bulk block Omega_i (each divides the lattice), default 4,4,4,4 */
    int overlap;        /* s: extension of Omega'_i on each side, d = 2 s; default 0 */
    int n_dominv;       /* MR iterations per domain solve, default 4 */
    int n_ras;          /* NRAS sweeps per preconditioner application, default 3 */
    int inner_prec;     /* qdd_prec of the inner solve: QDD_F32 (default) or QDD_F16;
                           QDD_F64 runs the plain FP64 BiCGStab (no nesting, no RAS) */
    double inner_tol;   /* relative residual of each inner solve, default 1e-3 */
    int max_inner;      /* inner BiCGStab iterations per outer step, default 2000 */
    int max_outer;      /* outer defect-correction steps, default 50 */
    int use_ras;        /* 1: right-precondition the inner solve with K_RAS (default 1) */
    int outer_mode;     /* outer level of the nested solver (Sec. 3): 0 FP64 defect
                           correction, phi += |r| inner(r / |r|) (default); 1 the paper's
                           FP64 outer BiCGStab with the inner solve (to inner_tol) as a
                           flexible preconditioner, restarted from the true residual until
                           tol is met; max_outer then bounds its iterations */
    int autotune;       /* reserved, 0 */
    int ras_kernel;     /* RAS sweep staging: 0 auto (TMA bulk tensor copies for overlap-free
                           256-site blocks with x extents divisible by 4, else per-thread
                           loads), 1 compact per-thread staging (links and clover in the
                           field's storage format), 2 expanded (FP32 18-real links and FP32
                           clover, domains of at most 256 sites), 3 the general kernel
                           (global scratch, one CTA per domain) for every extended domain
                           above 512 sites; auto uses for those one thread-block cluster
                           per domain (one CTA per t-slice) when the domain has 2 to 8
                           t-slices of at most 512 sites, else, when domains x n_rhs is
                           below 304, the phased sweep (each domain over many CTAs, one
                           launch per MR step), else the general kernel */
    int schwarz;        /* member of the Schwarz family used as K (Sec. 1, Sec. 2), a
                           qdd_schwarz: QDD_SCHWARZ_RAS (default, Alg. 1), QDD_SCHWARZ_SAP or
                           QDD_SCHWARZ_AS; n_ras counts cycles for each */
} qdd_solver_params;

/* The Schwarz iteration run by K.  Every variant starts from phi = 0, r = eta
 * and ends each sweep with phi += v, r -= D v (Alg. 1 line 9); they differ in
 * which domains a sweep solves and where their solutions go:
 *   RAS  one sweep per cycle over every domain, solution restricted to the
 *        bulk block (R_i), Alg. 1;
 *   SAP  the multiplicative Schwarz alternating procedure: two sweeps per
 *        cycle, first the domains whose block coordinates have an even sum
 *        (red), then the odd ones (black), each restricted to its bulk block,
 *        with the residual updated in between;
 *   AS   plain additive Schwarz: one sweep per cycle over every domain, the
 *        solution prolonged onto the whole extended domain and the
 *        overlapping copies summed (identical to RAS when overlap = 0; with
 *        overlap the sum is formed with FP32 atomic additions, so its
 *        rounding depends on their order). */
typedef enum { QDD_SCHWARZ_RAS = 0, QDD_SCHWARZ_SAP = 1, QDD_SCHWARZ_AS = 2 } qdd_schwarz;

typedef struct {
    int outer_iters;            /* defect-correction steps (outer_mode 0) or outer BiCGStab
                                   iterations (outer_mode 1) */
    int inner_iters;            /* inner BiCGStab iterations, summed */
    int dv_count;               /* global D applications (the paper's "Dv count", Table 1) */
    int ras_sweeps;             /* block-solve sweeps of K (SAP: two per cycle, one per colour) */
    int status;                 /* qdd_status of the solve */
    double true_rel_residual;   /* |eta - D phi| / |eta| with the FP64 D */
    double t_total_ms;          /* wall time of the call */
    double t_outer_ms;          /* FP64 residuals, conversions and accumulation (outer level, Sec. 3) */
    double t_inner_ms;          /* inner solves (inner level, Sec. 3) */
    /* Time per kernel class (D, RAS sweeps, BLAS) is not kept here: with
     * qdd_set_profiling on, qdd_profile_read returns it, measured with CUDA
     * events on the lattice's stream. */
} qdd_solve_info;

/* Library version string. */
const char *qdd_version(void);

/* Description of the last error on the calling thread ("" if none).  The
 * paper defines no error reporting; every failure of the calls below, which
 * implement Eq. 1, Alg. 1 and Sec. 3, is described here. */
const char *qdd_last_error(void);

/* Fills *p with the defaults listed in qdd_solver_params. */
void qdd_default_params(qdd_solver_params *p);

/* Creates a lattice of dims[4] = (Lx, Ly, Lz, Lt) sites with boundary signs
 * bc[4] (+1 / -1) on the current CUDA device: the four-dimensional lattice
 * on which Eq. 1 acts and which Sec. 4 decomposes into domains (the paper's
 * workload of Sec. 5 is 32^4; its fermion boundary is not stated, the
 * benchmark takes antiperiodic time, bc = {1, 1, 1, -1}).  Every spinor the lattice
 * works on holds n_rhs (1..QDD_MAX_RHS) right-hand sides, processed together
 * by every kernel (links and clover are read once per site block for all of
 * them).  cuda_stream is a cudaStream_t (NULL: the legacy default stream);
 * every kernel of this lattice runs on it, and solves can be captured into
 * CUDA graphs only on a non-default stream.  Allocates the lattice's device
 * memory (about 2.2 KB per site).  Errors: QDD_ERR_ARG for extents outside
 * 1..4096, a volume above QDD_MAX_SITES, bc not +-1, n_rhs out of range;
 * QDD_ERR_NOMEM. */
qdd_status qdd_create_lattice(qdd_lattice **out, const int dims[4], const int bc[4], int n_rhs,
                              void *cuda_stream);

/* Frees the lattice of qdd_create_lattice (the lattice of Eq. 1 and Sec. 4)
 * and everything it owns (fields created from it must be destroyed first).
 * NULL is accepted. */
qdd_status qdd_destroy_lattice(qdd_lattice *lat);

/* Loads the gauge field U (canonical FP64, host or device) and derives the
 * internal FP64 (18-real), FP32 and FP16 (12-real, third row rebuilt as the
 * conjugated cross product of the first two) copies; invalidates the clover
 * cache.  The links enter D through the hopping term of Eq. 1 and the clover
 * leaves.  Rejects with QDD_ERR_ARG a field with any max|U^dag U - 1| or
 * |det U - 1| above 1e-10 (the compression needs SU(3)).  A host U goes
 * through a device staging buffer (576 B per site) allocated by the first
 * such call and kept until the lattice is destroyed.  Synchronous. */
qdd_status qdd_load_gauge(qdd_lattice *lat, const double *U);

/* qdd_load_gauge followed by the clover term for (kappa, c_sw) (the O(a)
 * improvement of Sec. 5), in one pass: for host U with Lt a multiple of 8
 * and at least 16, the links are copied in 8 groups of t-slices and the
 * clover of each group is built as soon as its two neighbouring groups are
 * converted, so that the build overlaps the copy of the remaining links;
 * otherwise it is built after the conversion.  The clover cache then holds (kappa, c_sw), and calls with
 * these parameters need no build.  Errors as qdd_load_gauge; QDD_ERR_ARG
 * also for a non-finite kappa or c_sw.  Synchronous. */
qdd_status qdd_load_gauge_clover(qdd_lattice *lat, const double *U, double kappa, double c_sw);

/* out = D in (Eq. 1), computed in precision prec (QDD_F64: FP64 throughout;
 * QDD_F32: FP32 fields and arithmetic; QDD_F16: FP16 storage with per-site
 * norms, FP32 arithmetic).  in/out canonical FP64 spinors, host or device,
 * must not overlap.  Builds the clover term for (kappa, c_sw) on first use. */
qdd_status qdd_dslash(qdd_lattice *lat, double *out, const double *in, double kappa, double c_sw,
                      qdd_prec prec);

/* out = K_RAS in (Alg. 1): NRAS sweeps of projection onto every extended
 * domain Omega'_i, n_dominv MR iterations of the Dirichlet-restricted D on
 * it, restriction to the bulk block and summation, then phi += v,
 * r -= D v.  Uses params->block, overlap, n_dominv, n_ras, inner_prec
 * (QDD_F32 or QDD_F16) and schwarz (SAP and AS in place of RAS, see
 * qdd_schwarz).  in/out canonical FP64 spinors, host or device.
 * Errors: QDD_ERR_ARG if a block does not divide the lattice or
 * block + 2*overlap exceeds it; QDD_ERR_TIMEOUT if a sweep gave up waiting
 * for its staged data (out is then undefined). */
qdd_status qdd_ras_apply(qdd_lattice *lat, double *out, const double *in, double kappa, double c_sw,
                         const qdd_solver_params *params);

/* Solves D phi = eta to |eta - D phi| / |eta| <= tol (the stopping rule of
 * Sec. 5) for every right-hand side, with the FP64 outer defect correction
 * around the right-preconditioned inner BiCGStab (Sec. 3, Eq. 3), or with the
 * plain FP64 BiCGStab when params->inner_prec == QDD_F64.  params NULL:
 * defaults.  phi is overwritten (no initial guess).  info may be NULL, else
 * it receives n_rhs entries.  The inner iterations run as a CUDA graph when
 * the lattice has a non-default stream.  Returns QDD_OK,
 * QDD_ERR_NOT_CONVERGED (phi = best iterate), QDD_ERR_BREAKDOWN,
 * QDD_ERR_NONFINITE or QDD_ERR_TIMEOUT (the first failure over the
 * right-hand sides). */
qdd_status qdd_solve(qdd_lattice *lat, double *phi, const double *eta, double kappa, double c_sw,
                     double tol, const qdd_solver_params *params, qdd_solve_info *info);

/* Solves n independent systems, one per lattice (lattices of any shapes and
 * right-hand-side counts, each with its own kappa[i] and c_sw[i], all to tol
 * with the same params), in lockstep: the inner iterations of all lattices
 * are captured into one CUDA graph forked across their streams (the lattices
 * must then have distinct non-default streams; otherwise the same work is
 * launched eagerly) and replayed until every right-hand side has converged.
 * phi[i] and eta[i] are canonical spinors of lattice i (host or device);
 * info (may be NULL) receives the entries of lattice 0's right-hand sides,
 * then lattice 1's, and so on.  A lattice may appear only once. */
qdd_status qdd_solve_batch(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                           const double *kappa, const double *c_sw, double tol,
                           const qdd_solver_params *params, qdd_solve_info *info);

/* qdd_solve_batch with parameters per lattice: params[i] (params may be NULL,
 * and so may params[i]) for lattice i; a NULL entry takes the tuning cache's
 * parameters for lattice i's shape (qdd_tuned_params), else the defaults.
 * The lattices may differ in RAS blocking, overlap, n_dominv, n_ras, Schwarz
 * variant, sweep kernel, inner precision (QDD_F32 or QDD_F16), inner
 * tolerance and iteration budgets -- each size gets the parameters the
 * paper's survey (Sec. 5) finds best for it; they must agree on the plain
 * FP64 solver (inner_prec QDD_F64) against the nested one and on
 * outer_mode (QDD_ERR_ARG otherwise).  Otherwise as qdd_solve_batch. */
qdd_status qdd_solve_batch_each(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                                const double *kappa, const double *c_sw, double tol,
                                const qdd_solver_params *const *params, qdd_solve_info *info);

/* Work lists for batches (qdd_solve_batch, qdd_solve_batch_each), on (1) by
 * default.  The paper has no counterpart (it solves one system at a time);
 * this is an execution choice.  While on, the lattices of a batch with FP16 inner storage
 * (inner_prec QDD_F16) that share n_ras and the number of sites per RAS
 * domain (128 or 256, overlap 0, x extents divisible by 4), with one
 * right-hand side each and the RAS Schwarz variant, run each step of their
 * inner iteration as one launch over all of them, in groups of up to 16
 * lattices: every sweep of K_RAS is one launch over the (lattice, domain)
 * items of the group (Alg. 1 lines 4-8 for all domains of all its
 * lattices), every D one launch over the concatenated site ranges, and the
 * closing BiCGStab update one launch.  Their blockings, n_dominv, kappa,
 * tolerances and sizes may differ.  Other lattices, and every lattice while
 * off, launch their own kernels (forked across their streams in the graph).
 * The choice changes the launches, not the arithmetic of a site or a
 * domain; the dot products of a lattice are summed over a different number
 * of blocks, so its iterates agree to rounding.  Process-wide; the previous
 * setting is returned in *previous when it is not NULL. */
qdd_status qdd_set_batch_lists(int on, int *previous);

/* The tuning cache: the parameters the last qdd_autotune in this process
 * chose for a lattice of the same extents, boundary signs and right-hand-side
 * count (the paper's parameter survey of Sec. 5, kept per lattice shape).
 * QDD_ERR_STATE if that shape was never tuned. */
qdd_status qdd_tuned_params(const qdd_lattice *lat, qdd_solver_params *params);

/* Chooses the RAS parameters that minimise the time of a whole solve of
 * D phi = eta (the paper's parameter survey of Sec. 5, done by timing):
 * coordinate search over (n_dominv, n_ras), block shapes of 16 to 256 sites,
 * overlap 1, the sweep kernel's staging variant, the inner precision and
 * tighter inner tolerances (3e-4 with FP16 storage, 1e-4 and 1e-5 with
 * FP32 storage); at most max_trials solves.  params is the starting point
 * (inner_prec QDD_F32 or QDD_F16, use_ras = 1) and receives the best
 * parameters, which are also kept in the tuning cache for the lattice's shape
 * (qdd_tuned_params); best_ms (may be NULL) receives the best solve time.
 * eta is a canonical FP64 spinor, host or device.  Runs synchronously. */
qdd_status qdd_autotune(qdd_lattice *lat, const double *eta, double kappa, double c_sw, double tol,
                        qdd_solver_params *params, int max_trials, double *best_ms);

/* -- internal-layout fields ------------------------------------------------ */

/* Creates a spinor field of precision prec in the internal layout. */
qdd_status qdd_field_create(qdd_lattice *lat, qdd_prec prec, qdd_field **out);
qdd_status qdd_field_destroy(qdd_field *f);
/* Canonical FP64 spinor (host or device) -> field (rounded to its precision). */
qdd_status qdd_field_import(qdd_field *f, const double *src);
/* Field -> canonical FP64 spinor (host or device). */
qdd_status qdd_field_export(const qdd_field *f, double *dst);
/* out = D in on internal fields of one precision (the dslash kernel alone:
 * one launch, stream-ordered, nothing else). */
qdd_status qdd_dslash_field(qdd_lattice *lat, qdd_field *out, const qdd_field *in, double kappa,
                            double c_sw);

/* K_RAS of qdd_ras_apply on caller-owned fields, with no device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library call cudaMalloc when the preconditioner runs --
 * programs that own all device memory through their own pool or arena, and
 * loops where an allocation (or the synchronisation of a cudaFree) would
 * stall the GPU.
 * out = K_RAS in with params->block, overlap, n_dominv, n_ras and schwarz
 * (RAS or SAP; AS with overlap > 0 needs a summation buffer and is rejected
 * with QDD_ERR_ARG); out, in, rho and v are four different fields of this
 * lattice in one precision (QDD_F32 or QDD_F16); rho and v are work vectors
 * whose contents are overwritten.
 * Every sweep runs the general domain kernel, whose scratch is a fixed
 * 16 MiB device array inside the library (present on every GPU that loads
 * it, until the process exits): an extended domain may have at most 58254
 * sites (36 * 8 bytes each), and larger ones are rejected with QDD_ERR_ARG.
 * The lattice's device must be the current device (QDD_ERR_STATE otherwise).
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make it before any stream capture begins.  All
 * calls share the array, so calls whose kernels overlap on the GPU race and
 * give wrong results.  Stream-ordered on the lattice's stream; needs a gauge
 * field (QDD_ERR_STATE otherwise); builds the clover term for (kappa, c_sw)
 * if it is not cached, which launches a kernel but allocates nothing; if
 * that build is due while the lattice's stream is being captured, the call
 * returns QDD_ERR_STATE and does nothing. */
qdd_status qdd_ras_field_noalloc(qdd_lattice *lat, qdd_field *out, const qdd_field *in, qdd_field *rho,
                                 qdd_field *v, double kappa, double c_sw, const qdd_solver_params *params);

/* -- measurement ------------------------------------------------------------ */

/* Kernel classes of the per-class GPU timers. */
enum {
    QDD_K_DSLASH = 0,      /* D in FP32 / FP16 (inner solve, RAS residual updates) */
    QDD_K_DSLASH_F64 = 1,  /* D in FP64 (plain solver, outer true residual) */
    QDD_K_RAS = 2,         /* RAS sweeps (projection + domain solves + restriction) */
    QDD_K_BLAS = 3,        /* Krylov vector kernels and reductions */
    QDD_K_CONVERT = 4,     /* layout and precision conversions */
    QDD_K_CLOVER = 5,      /* clover-term build and gauge conversion */
    QDD_NKCLASS = 6
};

typedef struct {
    double ms[QDD_NKCLASS];            /* summed GPU time of each class */
    long long launches[QDD_NKCLASS];   /* timed launches of each class */
} qdd_profile;

/* Process-wide count of kernel launches made by this library. */
unsigned long long qdd_kernel_launches(void);

/* Turns per-class GPU timing on or off for this lattice: while on, every
 * launch is bracketed by CUDA events on the lattice's stream (inside a
 * solve's captured graph, as event-record nodes read after each replay). */
qdd_status qdd_set_profiling(qdd_lattice *lat, int on);

/* Synchronises the lattice's stream and returns the per-class totals since
 * the last reset; reset != 0 clears them. */
qdd_status qdd_profile_read(qdd_lattice *lat, qdd_profile *out, int reset);

/* Measures the FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA): fp64 != 0 for FP64, else FP32.  Runs a few short kernels on the
 * legacy default stream. */
qdd_status qdd_measure_fma_peak(int fp64, double *tflops);

/* Test support, with no counterpart in the paper.  The TMA-staged RAS sweep
 * waits for its bulk copies on an mbarrier for at most max_polls polls
 * (<= 0: the default, 2000 polls that each suspend the thread for at most
 * 0.5 ms) and then gives up: the call that ran it returns QDD_ERR_TIMEOUT
 * and its results are undefined, while the CUDA context stays usable.  extra_bytes > 0 makes every such sweep announce that many
 * bytes more than its copies deliver, so that its wait runs out; this is
 * how the tests exercise the timeout path.  Process-wide; (0, 0) restores
 * the defaults.  Never fails. */
qdd_status qdd_test_ras_wait(unsigned extra_bytes, long max_polls);

#ifdef __cplusplus
}
#endif

#endif /* QDD_H */
