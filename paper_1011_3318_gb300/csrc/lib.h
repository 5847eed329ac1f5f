// lib.h -- host-side structures and kernel launchers of the library.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "qdd_internal.h"

namespace qdd {

// Counts kernel launches of this library (qdd_kernel_launches()); graph
// replays add the launches their capture recorded.
void note_launch(unsigned n = 1);
void note_launch_adjust(long long n);
unsigned long long launch_count();

// Per-kernel-class GPU time, measured with CUDA events on the lattice stream
// around every launch while profiling is on (qdd_set_profiling).
struct Profiler {
    struct Pair {
        int cls;
        cudaEvent_t a, b;
        int graph;  // which captured graph holds the pair (0 or 1)
    };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Pair> pending;
    // pairs recorded while a CUDA graph is captured: event-record nodes of
    // the graph, read after each replay and kept until the graph is released
    bool capturing = false;
    int capture_graph = 0;  // the id given to the pairs of the graph being captured
    std::vector<Pair> graph_pairs;
    int graph_replays[2] = {0, 0};  // replays of each graph since its pairs were last read
    double ms[QDD_NKCLASS] = {};
    long long n[QDD_NKCLASS] = {};
    ~Profiler();
    cudaEvent_t get();
    void drain();          // after the stream has passed every pending event and replay
    void release_graph();  // the graph holding graph_pairs is destroyed
};

// Dslash epilogues.
enum Epi {
    EPI_D = 0,         // out = D in
    EPI_XMY = 1,       // out = y - D in
    EPI_XMY_NORM = 2,  // out = y - D in, |out|^2 -> sc->aux[aux_slot]
    EPI_RV = 3,        // out = D in, alpha = rho / <y, out>   (BiCGStab, y = rhat)
    EPI_TS = 4,        // out = D in, omega = <out, y> / |out|^2 (BiCGStab, y = s)
};

// Every kernel works on nrhs right-hand sides at once: fields hold nrhs
// vectors one after the other, sc points at nrhs Scalars, and the grid covers
// (site block x right-hand side) with the right-hand side fastest, so that
// consecutive CTAs read the same links and clover (served from L2).
struct DslashArgs {
    Geom g;
    SpinorView out, in, y;
    LinkView U;
    CloverView A;
    double kappa;
    ReduceScratch rs;
    Scalars *sc;
    int aux_slot;
    int nrhs;
};

cudaError_t launch_dslash(int prec, int epi, const DslashArgs &a, cudaStream_t st);
// FP16 D on two right-hand sides per thread (links and clover decoded once
// for both); nrhs >= 2.  launch_dslash uses it for FP16 lattices with
// several right-hand sides.
cudaError_t launch_dslash_mrhs_f16(int epi, const DslashArgs &a, cudaStream_t st);

// Field conversions between the canonical FP64 layout and internal layouts.
// Canonical multi-RHS layout: double[nrhs][V][4][3][2].
cudaError_t launch_import_spinor(const Geom &g, int prec, SpinorView dst, const double *src, int nrhs,
                                 cudaStream_t st);
cudaError_t launch_export_spinor(const Geom &g, int prec, double *dst, SpinorView src, int nrhs, cudaStream_t st);

// Gauge conversion of the links of sites [site0, site1) (site1 < 0: up to
// V); writes max(|U^dag U - 1|, |det U - 1|) as the bit pattern of a
// non-negative double into *maxdev (device, zeroed first; a running max).
cudaError_t launch_gauge_convert(const Geom &g, const double *U, void *U64, void *U32, void *U16, void *Udf,
                                 unsigned long long *maxdev, cudaStream_t st, long long site0 = 0,
                                 long long site1 = -1);

// Clover term from the double-float links, stored in all three precisions,
// for the sites [site0, site1) (site1 < 0: up to V); it reads the links of
// the sites within one step in two directions of them.
cudaError_t launch_clover_build(const Geom &g, const void *Udf, double kappa, double csw, void *A64, void *A32,
                                void *A16, float *A16n, cudaStream_t st, long long site0 = 0, long long site1 = -1);

// BLAS of the Krylov solvers (K-B4 in the design notes).
struct BlasArgs {
    long long V;
    SpinorView f[8];
    Scalars *sc;
    ReduceScratch rs;
    int aux_slot;
    double tol2_rel;   // bicg_init: tol^2
    int nrhs;
    unsigned long long active;  // B_INIT: bit r set = right-hand side r is solved (others start converged)
};

enum BlasOp {
    B_INIT = 0,       // f0 = b: r(f1) = b, rhat(f2) = b, x(f3) = p(f4) = v(f5) = 0; scalars reset
    B_P = 1,          // p(f0) = r(f1) + beta (p - omega v(f2))
    B_S = 2,          // s(f0) = r(f1) - alpha v(f2)
    B_XR = 3,         // x(f0) += alpha phat(f1) + omega shat(f2); r(f3) = s(f4) - omega t(f5); <rhat(f6), r>, |r|^2
    B_NORM = 4,       // |f0|^2 -> aux[aux_slot]
    B_COPY = 5,       // f0 = f1 (same precision)
    B_ZERO = 6,       // f0 = 0
    B_RESTART = 7,    // rhat(f0) = r(f1); p(f2) = v(f3) = 0; rho = <r, r>; alpha = omega = 1
    B_AXPY = 8,       // f0 += f1 (same precision)
};

cudaError_t launch_blas(int prec, int op, const BlasArgs &a, cudaStream_t st);

// Precision changes around the inner solve (outer defect correction).
// dst(prec) = src64 / sqrt(aux[slot]) of each right-hand side
cudaError_t launch_convert_scaled(long long V, int prec, SpinorView dst, SpinorView src64, const Scalars *sc,
                                  int slot, int nrhs, cudaStream_t st);
// phi64 += sqrt(aux[slot]) * x(prec) of each right-hand side
cudaError_t launch_accum_scaled(long long V, int prec, SpinorView phi64, SpinorView x, const Scalars *sc, int slot,
                                int nrhs, cudaStream_t st);
// dst(pd) = src(ps)
cudaError_t launch_convert(long long V, int pd, SpinorView dst, int ps, SpinorView src, int nrhs, cudaStream_t st);

// RAS block solve (Alg. 1 lines 4-8) over every domain.
struct RasArgs {
    Geom g;
    DomainGeom dg;
    SpinorView in;     // residual rho (projected per domain)
    SpinorView vout;   // v on bulk sites (d == nullptr: not written)
    SpinorView acc;    // phi: acc = v (accumulate = 0) or acc += v (accumulate = 1)
    int accumulate;
    LinkView U;
    CloverView A;
    float kappa;
    int n_iter;
    const Scalars *sc;  // may be null; a non-running solver status skips the work
    float2 *scratch;    // general kernel: per-slot rho, q, v
    int slots;
    int nrhs;
    int variant;        // qdd_solver_params::ras_kernel
    // Fused BiCGStab update (shared-memory kernel only): instead of reading
    // `in`, the sweep stages in = fr + b fy + c fz with the coefficients of
    // the solver scalars, and writes that vector to `in` on its bulk sites.
    //   RAS_FUSE_P: p = r + beta (p - omega v)  (fr = r, fy = p = in, fz = v)
    //   RAS_FUSE_S: s = r - alpha v             (fr = r, fz = v)
    int fuse;
    SpinorView fr, fz;
    unsigned *err;  // may be null: set to 1 when a bounded wait for staged data gives up
    // Schwarz variants (qdd_schwarz).  color = 0: every domain; color = 1 + c:
    // only the domains whose block coordinates sum to parity c are solved,
    // the others write zero to vout and (accumulate = 0) acc on their bulk
    // sites.  asum non-null
    // (additive Schwarz with overlap): instead of writing outputs, every
    // domain adds its solution on all its extended sites to asum, FP32
    // float4[nrhs][6][V], and launch_as_finish writes vout and acc from it.
    int color;
    float4 *asum;
};

enum { RAS_FUSE_NONE = 0, RAS_FUSE_P = 1, RAS_FUSE_S = 2 };

// Sites of an extended domain up to which the shared-memory kernel is used.
constexpr int RAS_SMEM_MAX_SITES = 512;
// Whether larger extended domains fit the cluster kernel (one CTA per
// t-slice of at most 512 sites, at most 8 slices).
bool ras_cluster_shape(const DomainGeom &dg);
// Whether the domains (times right-hand sides) are too few for one CTA each:
// then every domain is spread over many CTAs (the phased sweep), which needs
// ras_phased_scratch_bytes of scratch.
bool ras_use_phased(const DomainGeom &dg, int nrhs);
size_t ras_phased_scratch_bytes(const DomainGeom &dg, int nrhs);

cudaError_t launch_ras_block(int prec, const RasArgs &a, cudaStream_t st);
// vout = asum, acc = asum or acc += asum (the additive-Schwarz sum of a sweep)
cudaError_t launch_as_finish(int prec, const RasArgs &a, cudaStream_t st);
// Which sweeps K runs: the effective variant (AS without overlap is RAS),
// sweeps per cycle, and whether the additive sum needs asum.
struct SchwarzPlan {
    int variant;  // qdd_schwarz
    int colors;   // 2 for SAP, else 1
    bool sum;     // additive Schwarz over overlapping domains
};
SchwarzPlan schwarz_plan(int schwarz, const DomainGeom &dg);
inline bool valid_schwarz(int s) { return s == QDD_SCHWARZ_RAS || s == QDD_SCHWARZ_SAP || s == QDD_SCHWARZ_AS; }
// The general (global-scratch) sweep kernel for any domain size, with the
// scratch and slot count given in a (FP32 and FP16 only).
cudaError_t launch_ras_block_gmem(int prec, const RasArgs &a, cudaStream_t st);
size_t ras_scratch_bytes(const DomainGeom &dg, int slots, int nrhs);
// Test support for the TMA sweep's bounded wait (qdd_test_ras_wait).
void ras_set_wait_test(unsigned extra_bytes, long max_polls);
int ras_default_slots();

bool domain_geom(const Geom &g, const int block[4], int s, DomainGeom *dg, std::string *why);

// ---------------------------------------------------------------- work lists
// One launch over several lattices of a batch: lattice i of a list owns the
// blocks first[i] .. first[i+1]-1 of the grid, and the per-lattice arguments
// travel as one kernel parameter.  Every lattice of a list has one
// right-hand side and a solver status (sc); the blocks of a lattice whose
// solver no longer runs return at once.
constexpr int LIST_MAX = 16;
// Lists exist for FP16 storage only.
// Whether sweep `a` can be an item of launch_ras_list: FP16 storage, a domain
// of 128 or 256 sites without overlap, staged by TMA (the same test as the
// one-lattice launch), one right-hand side.
bool ras_list_ok(int prec, const RasArgs &a);
// One RAS sweep (launch_ras_block) of n <= LIST_MAX lattices whose domains
// all have the same number of sites.
cudaError_t launch_ras_list(int prec, const RasArgs *a, int n, cudaStream_t st);
// D with epilogue EPI_XMY, EPI_RV or EPI_TS on n <= LIST_MAX lattices.
cudaError_t launch_dslash_list(int prec, int epi, const DslashArgs *a, int n, cudaStream_t st);
// The BiCGStab update B_XR on n <= LIST_MAX lattices.
cudaError_t launch_blas_list(int prec, int op, const BlasArgs *a, int n, cudaStream_t st);

}  // namespace qdd

struct qdd_field {
    qdd_lattice *lat;
    int prec;
    void *d;
    float *n;
    qdd::SpinorView view() const { return qdd::SpinorView{d, n}; }
};

// Solver workspace (allocated on first use, kept with the lattice).
struct qdd_work;

struct qdd_lattice {
    qdd::Geom g;
    int nrhs;  // right-hand sides held by every spinor field of this lattice
    int device;
    cudaStream_t stream;
    // links (Udf: double-float copy, float4 (re.hi, re.lo, im.hi, im.lo) [4][9][V])
    void *U64, *U32, *U16, *Udf;
    bool has_gauge;
    // clover cache
    bool clover_valid;
    double kappa_c, csw_c;
    void *A64, *A32, *A16;
    float *A16n;
    // reductions and device scalars
    qdd::ReduceScratch rs;
    qdd::Scalars *sc;       // device
    qdd::Scalars *sc_host;  // pinned mirror
    unsigned long long *maxdev;
    unsigned *ras_err;  // device word: a RAS sweep's bounded wait gave up
    // canonical staging buffers for host pointers (spinors, and the links)
    double *stage_a, *stage_b;
    double *gauge_stage;
    // host-to-device copies that overlap the lattice stream's work
    cudaStream_t copy_stream;
    cudaEvent_t copy_ev[2];
    // RAS scratch, and the additive-Schwarz sum (FP32 float4[nrhs][6][V])
    float2 *ras_scratch;
    size_t ras_scratch_bytes;
    float4 *as_sum;
    // in/out fields of the canonical-layout entry points, per precision
    void *io_d[3][2];
    float *io_n[3][2];
    qdd_work *work;
    qdd::Profiler *prof;
};

// Helpers shared by api.cu and solver.cu.
namespace qdd {
// Records events around the launches in its lifetime when profiling is on.
struct ProfScope {
    Profiler *prof;
    int cls;
    cudaStream_t st;
    cudaEvent_t a;
    ProfScope(qdd_lattice *lat, int cls);
    ~ProfScope();
};
void set_error(const std::string &msg);
qdd_status cuda_fail(cudaError_t e, const char *what);
qdd_status ensure_clover(qdd_lattice *lat, double kappa, double csw);
size_t spinor_bytes(long long V, int prec);
qdd_status field_alloc(long long V, int prec, void **d, float **n);
void field_free(void *d, float *n);
LinkView links_of(const qdd_lattice *lat, int prec);
CloverView clover_of(const qdd_lattice *lat, int prec);
// sc: the scalars the epilogue reads and writes (null: the lattice's own)
qdd_status run_dslash(qdd_lattice *lat, int prec, int epi, SpinorView out, SpinorView in, SpinorView y, double kappa,
                      int aux_slot, Scalars *sc = nullptr);
qdd_status ras_apply_fields(qdd_lattice *lat, int prec, const qdd_solver_params *p, const DomainGeom &dg,
                            SpinorView out, SpinorView in, SpinorView rho, SpinorView v, double kappa, int *dv,
                            const Scalars *sc,
                            int fuse = RAS_FUSE_NONE, SpinorView fr = SpinorView{nullptr, nullptr},
                            SpinorView fz = SpinorView{nullptr, nullptr});
// Whether the first sweep of ras_apply_fields can form the BiCGStab update
// `fuse` while staging (shared-memory kernel; the in-place p update also
// needs domains without overlap, whose halo would read p after another
// domain has written it; RAS only: a SAP sweep skips half of the domains).
bool ras_can_fuse(int prec, const DomainGeom &dg, int fuse, int schwarz = QDD_SCHWARZ_RAS);
qdd_status solve_impl(qdd_lattice *lat, double *phi_dev, const double *eta_dev, double kappa, double csw, double tol,
                      const qdd_solver_params *p, qdd_solve_info *info);
// A batch of n lattices, lattice i solved with the parameters *ps[i] (they
// must agree on the plain FP64 solver against the nested one, and on
// outer_mode).
qdd_status solve_batch_impl(qdd_lattice *const *lats, double *const *phi_dev, const double *const *eta_dev, int n,
                            const double *kappa, const double *csw, double tol, const qdd_solver_params *const *ps,
                            qdd_solve_info *const *infos);
void work_free(qdd_work *w);
// Whether batches run compatible lattices as work-list groups (process-wide).
void set_batch_lists(bool on);
bool batch_lists();
// The tuning cache: the parameters qdd_autotune chose, per lattice shape
// (extents, boundary signs, right-hand-side count), for the process.
void tuned_store(const qdd_lattice *lat, const qdd_solver_params &p);
bool tuned_lookup(const qdd_lattice *lat, qdd_solver_params *p);
qdd_status autotune_impl(qdd_lattice *lat, double *phi_dev, const double *eta_dev, double kappa, double csw,
                         double tol, qdd_solver_params *p, int max_trials, double *best_ms);
}  // namespace qdd
