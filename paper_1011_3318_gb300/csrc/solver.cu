// solver.cu -- host orchestration of the nested solver (Sec. 3): an FP64
// outer level around an inner BiCGStab in FP32 or FP16 storage, right-
// preconditioned by K_RAS (Eq. 3, Alg. 1); and the plain FP64 BiCGStab.  The
// outer level is FP64 defect correction (outer_mode 0) or the paper's FP64
// outer BiCGStab with the inner solve as a flexible preconditioner (outer_mode
// 1), restarted from the true residual by the same defect-correction loop.
//
// A solve is a lockstep batch: one or more lattices, each with nrhs right-
// hand sides, each lattice on its own stream with its own device scalars and
// reduction scratch.  Every vector operation runs in a kernel of this
// library; the host enqueues work and reads the solver status and residual
// norms (a few dozen bytes per right-hand side) to decide when to stop.
//
// The inner iterations of all lattices are captured once into a CUDA graph
// (forked across the lattices' streams) and replayed; kernels of a right-hand
// side that has converged return at once, so the host can run several
// iterations between status reads.  Per-kernel profiling records its event
// pairs as nodes of the graph.  When a lattice uses the legacy default
// stream, the same work is launched eagerly.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "lib.h"

struct qdd_work {
    // FP64 outer vectors: eta, phi, r (nrhs each)
    void *o_d[3] = {nullptr, nullptr, nullptr};
    // FP64 vectors of the outer BiCGStab (outer_mode 1): e r rhat p v s t phat
    // shat, and its scalars (device, and a pinned host mirror)
    static constexpr int NNEST = 9;
    void *n_d[NNEST] = {};
    qdd::Scalars *osc = nullptr, *osc_host = nullptr;
    // inner vectors per precision: b x r rhat p v s t phat shat rho_ras v_ras
    static constexpr int NIN = 12;
    void *in_d[3][NIN] = {};
    float *in_n[3][NIN] = {};
    bool in_ok[3] = {false, false, false};
};

namespace qdd {

enum { W_B, W_X, W_R, W_RHAT, W_P, W_V, W_S, W_T, W_PHAT, W_SHAT, W_RHO, W_VR };
// vectors of the outer BiCGStab
enum { N_E, N_R, N_RHAT, N_P, N_V, N_S, N_T, N_PHAT, N_SHAT };

// aux slots of the device scalars (AUX_TOL2 is also read by B_INIT)
enum { AUX_ETA2 = 0, AUX_R2 = 1, AUX_Y2 = 2, AUX_S2 = 3, AUX_TOL2 = 7 };

void work_free(qdd_work *w)
{
    if (!w) return;
    for (int k = 0; k < qdd_work::NNEST; k++) cudaFree(w->n_d[k]);
    cudaFree(w->osc);
    if (w->osc_host) cudaFreeHost(w->osc_host);
    for (int k = 0; k < 3; k++) cudaFree(w->o_d[k]);
    for (int p = 0; p < 3; p++)
        for (int k = 0; k < qdd_work::NIN; k++) field_free(w->in_d[p][k], w->in_n[p][k]);
    delete w;
}

static long long nsites(const qdd_lattice *lat) { return lat->g.V * lat->nrhs; }

static qdd_status ensure_outer(qdd_lattice *lat)
{
    if (!lat->work) lat->work = new qdd_work();
    qdd_work *w = lat->work;
    for (int k = 0; k < 3; k++)
        if (!w->o_d[k]) {
            float *n = nullptr;
            qdd_status st = field_alloc(nsites(lat), P64, &w->o_d[k], &n);
            if (st != QDD_OK) return st;
        }
    return QDD_OK;
}

static qdd_status ensure_inner(qdd_lattice *lat, int prec)
{
    if (!lat->work) lat->work = new qdd_work();
    qdd_work *w = lat->work;
    if (w->in_ok[prec]) return QDD_OK;
    for (int k = 0; k < qdd_work::NIN; k++) {
        qdd_status st = field_alloc(nsites(lat), prec, &w->in_d[prec][k], &w->in_n[prec][k]);
        if (st != QDD_OK) return st;
    }
    w->in_ok[prec] = true;
    return QDD_OK;
}

static qdd_status ensure_nested(qdd_lattice *lat)
{
    qdd_work *w = lat->work;
    for (int k = 0; k < qdd_work::NNEST; k++)
        if (!w->n_d[k]) {
            float *n = nullptr;
            qdd_status st = field_alloc(nsites(lat), P64, &w->n_d[k], &n);
            if (st != QDD_OK) return st;
        }
    if (!w->osc) {
        if (cudaMalloc(&w->osc, sizeof(Scalars) * lat->nrhs) != cudaSuccess ||
            cudaMemset(w->osc, 0, sizeof(Scalars) * lat->nrhs) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(w->osc);
            w->osc = nullptr;
            set_error("cudaMalloc of the outer solver scalars failed");
            return QDD_ERR_NOMEM;
        }
    }
    if (!w->osc_host) {
        if (cudaMallocHost(&w->osc_host, sizeof(Scalars) * lat->nrhs) != cudaSuccess) {
            cudaGetLastError();
            w->osc_host = nullptr;
            set_error("cudaMallocHost of the outer solver scalars failed");
            return QDD_ERR_NOMEM;
        }
        memset(w->osc_host, 0, sizeof(Scalars) * lat->nrhs);
    }
    return QDD_OK;
}

static SpinorView nested(qdd_lattice *lat, int k) { return SpinorView{lat->work->n_d[k], nullptr}; }

static SpinorView inner(qdd_lattice *lat, int prec, int k)
{
    return SpinorView{lat->work->in_d[prec][k], lat->work->in_n[prec][k]};
}

static SpinorView outer(qdd_lattice *lat, int k) { return SpinorView{lat->work->o_d[k], nullptr}; }

static BlasArgs blas_args(qdd_lattice *lat, std::initializer_list<SpinorView> fs, int aux_slot = 0, double tol2 = 0.0,
                          unsigned long long active = ~0ull, Scalars *sc = nullptr)
{
    BlasArgs a;
    memset(&a, 0, sizeof(a));
    a.V = lat->g.V;
    int i = 0;
    for (const SpinorView &f : fs) a.f[i++] = f;
    a.sc = sc ? sc : lat->sc;
    a.rs = lat->rs;
    a.aux_slot = aux_slot;
    a.tol2_rel = tol2;
    a.nrhs = lat->nrhs;
    a.active = active;
    return a;
}

static qdd_status blas(qdd_lattice *lat, int prec, int op, std::initializer_list<SpinorView> fs, int aux_slot = 0,
                       double tol2 = 0.0, unsigned long long active = ~0ull, Scalars *sc = nullptr)
{
    const BlasArgs a = blas_args(lat, fs, aux_slot, tol2, active, sc);
    ProfScope ps(lat, QDD_K_BLAS);
    cudaError_t e = launch_blas(prec, op, a, lat->stream);
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "blas kernel");
}

// Copies the device scalars of every lattice (with outer = true: those of
// the outer BiCGStab) to the host and waits.
static qdd_status read_scalars(const std::vector<qdd_lattice *> &lats, bool outer = false)
{
    for (qdd_lattice *lat : lats) {
        cudaError_t e = outer ? cudaMemcpyAsync(lat->work->osc_host, lat->work->osc, sizeof(Scalars) * lat->nrhs,
                                                cudaMemcpyDeviceToHost, lat->stream)
                              : cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(Scalars) * lat->nrhs,
                                                cudaMemcpyDeviceToHost, lat->stream);
        if (e != cudaSuccess) return cuda_fail(e, "reading solver scalars");
    }
    for (qdd_lattice *lat : lats) {
        cudaError_t e = cudaStreamSynchronize(lat->stream);
        if (e != cudaSuccess) return cuda_fail(e, "reading solver scalars");
        if (lat->prof) lat->prof->drain();
    }
    return QDD_OK;
}

static DslashArgs dslash_args(qdd_lattice *lat, int prec, SpinorView out, SpinorView in, SpinorView y, double kappa,
                              int aux_slot, Scalars *sc)
{
    DslashArgs a;
    memset(&a, 0, sizeof(a));
    a.g = lat->g;
    a.out = out;
    a.in = in;
    a.y = y;
    a.U = links_of(lat, prec);
    a.A = clover_of(lat, prec);
    a.kappa = kappa;
    a.rs = lat->rs;
    a.sc = sc ? sc : lat->sc;
    a.aux_slot = aux_slot;
    a.nrhs = lat->nrhs;
    return a;
}

qdd_status run_dslash(qdd_lattice *lat, int prec, int epi, SpinorView out, SpinorView in, SpinorView y, double kappa,
                      int aux_slot, Scalars *sc)
{
    const DslashArgs a = dslash_args(lat, prec, out, in, y, kappa, aux_slot, sc);
    ProfScope ps(lat, prec == P64 ? QDD_K_DSLASH_F64 : QDD_K_DSLASH);
    cudaError_t e = launch_dslash(prec, epi, a, lat->stream);
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "dslash kernel");
}

static qdd_status ensure_ras_scratch(qdd_lattice *lat, const DomainGeom &dg)
{
    const size_t need = ras_scratch_bytes(dg, ras_default_slots(), lat->nrhs);
    if (need <= lat->ras_scratch_bytes) return QDD_OK;
    cudaFree(lat->ras_scratch);
    lat->ras_scratch = nullptr;
    lat->ras_scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&lat->ras_scratch, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of RAS scratch failed");
        return QDD_ERR_NOMEM;
    }
    lat->ras_scratch_bytes = need;
    return QDD_OK;
}

SchwarzPlan schwarz_plan(int schwarz, const DomainGeom &dg)
{
    bool overlap = false;
    for (int mu = 0; mu < 4; mu++) overlap |= dg.e[mu] != dg.b[mu];
    SchwarzPlan sp;
    sp.variant = schwarz == QDD_SCHWARZ_AS && !overlap ? QDD_SCHWARZ_RAS : schwarz;
    sp.colors = sp.variant == QDD_SCHWARZ_SAP ? 2 : 1;
    sp.sum = sp.variant == QDD_SCHWARZ_AS;
    return sp;
}

bool ras_can_fuse(int prec, const DomainGeom &dg, int fuse, int schwarz)
{
    if (prec == P64 || dg.nloc > RAS_SMEM_MAX_SITES) return false;
    if (schwarz_plan(schwarz, dg).variant != QDD_SCHWARZ_RAS) return false;
    if (fuse == RAS_FUSE_P)
        for (int mu = 0; mu < 4; mu++)
            if (dg.e[mu] != dg.b[mu]) return false;
    return true;
}

static qdd_status ensure_as_sum(qdd_lattice *lat)
{
    if (lat->as_sum) return QDD_OK;
    cudaError_t e = cudaMalloc(&lat->as_sum, (size_t)lat->nrhs * 6 * (size_t)lat->g.V * sizeof(float4));
    if (e != cudaSuccess) {
        cudaGetLastError();
        lat->as_sum = nullptr;
        set_error("cudaMalloc of the additive-Schwarz sum failed");
        return QDD_ERR_NOMEM;
    }
    return QDD_OK;
}

// out = K in for the Schwarz variant of p (Alg. 1 for RAS): sweep q projects,
// solves and restricts on its domains (one launch; SAP alternates the two
// colours), accumulates phi += v, and updates rho = rho - D v except after
// the last sweep, where phi no longer depends on rho.
qdd_status ras_apply_fields(qdd_lattice *lat, int prec, const qdd_solver_params *p, const DomainGeom &dg,
                            SpinorView out, SpinorView in, SpinorView rho, SpinorView v, double kappa, int *dv,
                            const Scalars *sc, int fuse, SpinorView fr, SpinorView fz)
{
    qdd_status st = ensure_ras_scratch(lat, dg);
    if (st != QDD_OK) return st;
    const SchwarzPlan sp = schwarz_plan(p->schwarz, dg);
    if (sp.sum && (st = ensure_as_sum(lat)) != QDD_OK) return st;
    RasArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.g = lat->g;
    ra.dg = dg;
    ra.U = links_of(lat, prec);
    ra.A = clover_of(lat, prec);
    ra.kappa = (float)kappa;
    ra.n_iter = p->n_dominv;
    ra.sc = sc;
    ra.scratch = lat->ras_scratch;
    ra.slots = ras_default_slots();
    ra.nrhs = lat->nrhs;
    ra.variant = p->ras_kernel;
    ra.err = lat->ras_err;
    ra.asum = sp.sum ? lat->as_sum : nullptr;
    const int nsweep = p->n_ras * sp.colors;
    for (int q = 0; q < nsweep; q++) {
        const bool last = q == nsweep - 1;
        ra.in = q == 0 ? in : rho;
        ra.vout = last ? SpinorView{nullptr, nullptr} : v;
        ra.acc = out;
        ra.accumulate = q > 0;
        ra.color = sp.colors == 2 ? 1 + q % 2 : 0;
        // the first sweep may form its input (written to `in`) from fr, in, fz
        ra.fuse = q == 0 ? fuse : RAS_FUSE_NONE;
        ra.fr = fr;
        ra.fz = fz;
        cudaError_t e;
        {
            ProfScope ps(lat, QDD_K_RAS);
            e = cudaSuccess;
            if (sp.sum)
                e = cudaMemsetAsync(ra.asum, 0, (size_t)lat->nrhs * 6 * (size_t)lat->g.V * sizeof(float4),
                                    lat->stream);
            if (e == cudaSuccess) e = launch_ras_block(prec, ra, lat->stream);
            if (e == cudaSuccess && sp.sum) e = launch_as_finish(prec, ra, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "RAS block kernel");
        if (!last) {
            st = run_dslash(lat, prec, EPI_XMY, rho, v, ra.in, kappa, 0);
            if (st != QDD_OK) return st;
            if (dv) (*dv)++;
        }
    }
    return QDD_OK;
}

// ----------------------------------------------------------------- batch solve

namespace {

struct Member {
    qdd_lattice *lat;
    double *phi_dev;
    const double *eta_dev;
    double kappa, csw;
    qdd_solve_info *info;  // nrhs entries (may be null)
    qdd_solver_params prm; // this lattice's solver parameters
    int prec;              // its inner precision
    bool use_ras;
    DomainGeom dg;
    std::vector<double> eta2, rr, best;
    std::vector<int> stalls, restarted, done, result;
    std::vector<int> oit;  // outer BiCGStab iterations (outer_mode 1)
    // the last |r|^2 and iteration count seen by the host, per right-hand
    // side, to estimate how many iterations an inner solve still needs
    std::vector<double> seen_rr;
    std::vector<int> seen_it;
};

// Whether one more iteration is likely to end right-hand side r of m: the
// reduction of |r|^2 per iteration since the host last looked, extrapolated
// to the tolerance (BiCGStab's residual is not monotonic, so this is only an
// estimate: a wrong guess costs one more replay, not a wrong result).  Then
// records what it saw.
bool one_more_suffices(Member &m, int r, const Scalars &h)
{
    bool one = false;
    if (m.seen_it[r] >= 0 && h.iter > m.seen_it[r] && h.rr > 0.0 && m.seen_rr[r] > h.rr && h.tol2 > 0.0) {
        const double per = std::log(h.rr / m.seen_rr[r]) / (h.iter - m.seen_it[r]);  // < 0
        one = std::log(h.tol2 / h.rr) >= per;  // the next iteration reaches tol2
    }
    m.seen_rr[r] = h.rr;
    m.seen_it[r] = h.iter;
    return one;
}

// One BiCGStab iteration (van der Vorst) of every right-hand side of a
// lattice, right-preconditioned by K_RAS when use_ras: D K chi = b,
// x = K chi (Eq. 3).
qdd_status enqueue_iteration(Member &m)
{
    qdd_lattice *lat = m.lat;
    const int prec = m.prec;
    const qdd_solver_params *p = &m.prm;
    auto F = [&](int k) { return inner(lat, prec, k); };
    const SpinorView phat = m.use_ras ? F(W_PHAT) : F(W_P);
    const SpinorView shat = m.use_ras ? F(W_SHAT) : F(W_S);
    // with RAS, the updates p = r + beta (p - omega v) and s = r - alpha v are
    // formed by the sweeps that precondition them, while they stage their
    // input, instead of by separate passes over memory
    const bool fuse_p = m.use_ras && ras_can_fuse(prec, m.dg, RAS_FUSE_P, p->schwarz);
    const bool fuse_s = m.use_ras && ras_can_fuse(prec, m.dg, RAS_FUSE_S, p->schwarz);
    qdd_status st;
    if (!fuse_p && (st = blas(lat, prec, B_P, {F(W_P), F(W_R), F(W_V)})) != QDD_OK) return st;
    if (m.use_ras && (st = ras_apply_fields(lat, prec, p, m.dg, phat, F(W_P), F(W_RHO), F(W_VR), m.kappa, nullptr,
                                            lat->sc, fuse_p ? RAS_FUSE_P : RAS_FUSE_NONE, F(W_R), F(W_V))) != QDD_OK)
        return st;
    if ((st = run_dslash(lat, prec, EPI_RV, F(W_V), phat, F(W_RHAT), m.kappa, 0)) != QDD_OK) return st;
    if (!fuse_s && (st = blas(lat, prec, B_S, {F(W_S), F(W_R), F(W_V)})) != QDD_OK) return st;
    if (m.use_ras && (st = ras_apply_fields(lat, prec, p, m.dg, shat, F(W_S), F(W_RHO), F(W_VR), m.kappa, nullptr,
                                            lat->sc, fuse_s ? RAS_FUSE_S : RAS_FUSE_NONE, F(W_R), F(W_V))) != QDD_OK)
        return st;
    if ((st = run_dslash(lat, prec, EPI_TS, F(W_T), shat, F(W_S), m.kappa, 0)) != QDD_OK) return st;
    return blas(lat, prec, B_XR, {F(W_X), phat, shat, F(W_R), F(W_S), F(W_T), F(W_RHAT)});
}

// ----------------------------------------------------------- work-list groups
// Lattices of a batch whose inner iterations share work-list launches: each
// step of the iteration (every RAS sweep, every D, the closing update) is one
// launch over the (lattice, domain) or (lattice, site block) items of all
// members, instead of one launch per lattice.  Members have FP16 inner
// storage and share NRAS and the number of sites per domain (128 or 256,
// without overlap, staged by TMA); blockings, N_dominv, kappa, tolerances and
// lattice sizes are free.  Each has one right-hand side.
struct Group {
    std::vector<int> idx;          // members (indices into the batch)
    std::vector<cudaEvent_t> ev;   // ordering between the first member's stream and the others'
    Group() = default;
    Group(const Group &) = delete;  // owns its events
    Group &operator=(const Group &) = delete;
    ~Group()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};
typedef std::vector<std::unique_ptr<Group>> Groups;

std::atomic<int> g_batch_lists{1};

// The arguments of sweep q of the preconditioner application k (0: phat =
// K p, 1: shat = K s) of one BiCGStab iteration, as ras_apply_fields sets
// them for the fused updates.
RasArgs sweep_args(const Member &m, int k, int q)
{
    qdd_lattice *lat = m.lat;
    const int prec = m.prec;
    auto F = [&](int w) { return inner(lat, prec, w); };
    RasArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.g = lat->g;
    ra.dg = m.dg;
    ra.U = links_of(lat, prec);
    ra.A = clover_of(lat, prec);
    ra.kappa = (float)m.kappa;
    ra.n_iter = m.prm.n_dominv;
    ra.sc = lat->sc;
    ra.scratch = lat->ras_scratch;
    ra.slots = ras_default_slots();
    ra.nrhs = lat->nrhs;
    ra.variant = m.prm.ras_kernel;
    ra.err = lat->ras_err;
    const bool last = q == m.prm.n_ras - 1;
    ra.in = q > 0 ? F(W_RHO) : k == 0 ? F(W_P) : F(W_S);
    ra.vout = last ? SpinorView{nullptr, nullptr} : F(W_VR);
    ra.acc = k == 0 ? F(W_PHAT) : F(W_SHAT);
    ra.accumulate = q > 0;
    ra.fuse = q > 0 ? RAS_FUSE_NONE : k == 0 ? RAS_FUSE_P : RAS_FUSE_S;
    ra.fr = F(W_R);
    ra.fz = F(W_V);
    return ra;
}

bool list_eligible(const Member &m)
{
    if (!m.use_ras || m.prec != P16 || m.lat->nrhs != 1) return false;
    const SchwarzPlan sp = schwarz_plan(m.prm.schwarz, m.dg);
    if (sp.variant != QDD_SCHWARZ_RAS || sp.colors != 1 || sp.sum) return false;
    if (!ras_can_fuse(m.prec, m.dg, RAS_FUSE_P, m.prm.schwarz) ||
        !ras_can_fuse(m.prec, m.dg, RAS_FUSE_S, m.prm.schwarz))
        return false;
    for (int k = 0; k < 2; k++)
        for (int q = 0; q < m.prm.n_ras; q++)
            if (!ras_list_ok(m.prec, sweep_args(m, k, q))) return false;
    return true;
}

// Splits the batch into groups of at most LIST_MAX compatible lattices;
// lattices without a partner keep their own launches (solo).
qdd_status form_groups(const std::vector<Member> &ms, bool enable, Groups &groups, std::vector<int> &solo)
{
    std::vector<int> cand;
    for (size_t i = 0; i < ms.size(); i++) {
        if (enable && list_eligible(ms[i])) cand.push_back((int)i);
        else solo.push_back((int)i);
    }
    std::vector<int> used(ms.size(), 0);
    for (size_t a = 0; a < cand.size(); a++) {
        const int i = cand[a];
        if (used[i]) continue;
        std::vector<int> idx{i};
        used[i] = 1;
        for (size_t b = a + 1; b < cand.size() && (int)idx.size() < LIST_MAX; b++) {
            const int j = cand[b];
            if (used[j] || ms[j].prec != ms[i].prec || ms[j].prm.n_ras != ms[i].prm.n_ras ||
                ms[j].dg.nloc != ms[i].dg.nloc)
                continue;
            idx.push_back(j);
            used[j] = 1;
        }
        if (idx.size() == 1) {
            solo.push_back(i);
            continue;
        }
        groups.emplace_back(new Group());
        Group &g = *groups.back();
        g.idx = idx;
        g.ev.assign(idx.size(), nullptr);
        for (auto &e : g.ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "event");
    }
    std::sort(solo.begin(), solo.end());
    return QDD_OK;
}

// One BiCGStab iteration (as enqueue_iteration, with both fused updates) of
// every member of a group, on the first member's stream, ordered after the
// work queued on the other members' streams and before their next work.
qdd_status enqueue_group(Group &g, std::vector<Member> &ms)
{
    const int n = (int)g.idx.size();
    Member &m0 = ms[g.idx[0]];
    qdd_lattice *lat0 = m0.lat;
    cudaStream_t st = lat0->stream;
    const int prec = m0.prec, nras = m0.prm.n_ras;
    for (int i = 1; i < n; i++) {
        cudaEventRecord(g.ev[i], ms[g.idx[i]].lat->stream);
        cudaStreamWaitEvent(st, g.ev[i], 0);
    }
    RasArgs ra[LIST_MAX];
    DslashArgs da[LIST_MAX];
    BlasArgs ba[LIST_MAX];
    auto F = [&](int i, int w) { return inner(ms[g.idx[i]].lat, prec, w); };
    for (int k = 0; k < 2; k++) {
        for (int q = 0; q < nras; q++) {
            for (int i = 0; i < n; i++) ra[i] = sweep_args(ms[g.idx[i]], k, q);
            cudaError_t e;
            {
                ProfScope ps(lat0, QDD_K_RAS);
                e = launch_ras_list(prec, ra, n, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "RAS work-list kernel");
            if (q == nras - 1) break;
            // rho = in - D v
            for (int i = 0; i < n; i++)
                da[i] = dslash_args(ms[g.idx[i]].lat, prec, F(i, W_RHO), F(i, W_VR), ra[i].in, ms[g.idx[i]].kappa, 0,
                                    nullptr);
            {
                ProfScope ps(lat0, QDD_K_DSLASH);
                e = launch_dslash_list(prec, EPI_XMY, da, n, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "dslash work-list kernel");
        }
        // v = D phat with alpha, or t = D shat with omega
        for (int i = 0; i < n; i++)
            da[i] = k == 0 ? dslash_args(ms[g.idx[i]].lat, prec, F(i, W_V), F(i, W_PHAT), F(i, W_RHAT),
                                         ms[g.idx[i]].kappa, 0, nullptr)
                           : dslash_args(ms[g.idx[i]].lat, prec, F(i, W_T), F(i, W_SHAT), F(i, W_S),
                                         ms[g.idx[i]].kappa, 0, nullptr);
        cudaError_t e;
        {
            ProfScope ps(lat0, QDD_K_DSLASH);
            e = launch_dslash_list(prec, k == 0 ? EPI_RV : EPI_TS, da, n, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "dslash work-list kernel");
    }
    for (int i = 0; i < n; i++)
        ba[i] = blas_args(ms[g.idx[i]].lat, {F(i, W_X), F(i, W_PHAT), F(i, W_SHAT), F(i, W_R), F(i, W_S), F(i, W_T),
                                             F(i, W_RHAT)});
    cudaError_t e;
    {
        ProfScope ps(lat0, QDD_K_BLAS);
        e = launch_blas_list(prec, B_XR, ba, n, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "update work-list kernel");
    cudaEventRecord(g.ev[0], st);
    for (int i = 1; i < n; i++) cudaStreamWaitEvent(ms[g.idx[i]].lat->stream, g.ev[0], 0);
    return QDD_OK;
}

// One iteration of every lattice: the groups' list launches and the solo
// lattices' own launches.
qdd_status enqueue_all(std::vector<Member> &ms, Groups &groups, const std::vector<int> &solo)
{
    qdd_status st;
    for (auto &g : groups)
        if ((st = enqueue_group(*g, ms)) != QDD_OK) return st;
    for (int i : solo)
        if ((st = enqueue_iteration(ms[i])) != QDD_OK) return st;
    return QDD_OK;
}

bool graph_capable(const std::vector<Member> &ms)
{
    for (size_t i = 0; i < ms.size(); i++) {
        if (!ms[i].lat->stream) return false;
        for (size_t j = 0; j < i; j++)
            if (ms[j].lat->stream == ms[i].lat->stream) return false;
    }
    return true;
}

// Enqueues `chunk` iterations of every member, eagerly or as one graph launch.
struct IterGraph {
    int id = 0;  // 0: the chunk graph, 1: the one-iteration graph (per-kernel profiling tells them apart)
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;
    std::vector<cudaEvent_t> events;  // fork/join inside the capture
    std::vector<cudaEvent_t> pre;     // member streams -> launch stream, before each launch
    cudaEvent_t post = nullptr;       // launch stream -> member streams, after each launch
    std::vector<qdd_lattice *> lats;  // whose profilers hold event pairs recorded in the graph
    ~IterGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (qdd_lattice *lat : lats)
            if (lat->prof) lat->prof->release_graph();
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        for (cudaEvent_t e : pre) cudaEventDestroy(e);
        if (post) cudaEventDestroy(post);
    }
};

qdd_status build_graph(std::vector<Member> &ms, Groups &groups, const std::vector<int> &solo, int chunk, IterGraph &g)
{
    cudaStream_t s0 = ms[0].lat->stream;
    g.events.resize(ms.size() + 1, nullptr);
    g.pre.resize(ms.size(), nullptr);
    for (auto &e : g.events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "event");
    for (auto &e : g.pre)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "event");
    if (cudaEventCreateWithFlags(&g.post, cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "event");
    for (Member &m : ms) g.lats.push_back(m.lat);
    const unsigned long long c0 = launch_count();
    cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    for (Member &m : ms)
        if (m.lat->prof && m.lat->prof->on) {
            m.lat->prof->capturing = true;
            m.lat->prof->capture_graph = g.id;
        }
    qdd_status st = QDD_OK;
    cudaEventRecord(g.events[0], s0);
    for (size_t i = 1; i < ms.size(); i++) cudaStreamWaitEvent(ms[i].lat->stream, g.events[0], 0);
    for (int c = 0; c < chunk && st == QDD_OK; c++) st = enqueue_all(ms, groups, solo);
    for (size_t i = 1; i < ms.size(); i++) {
        cudaEventRecord(g.events[i], ms[i].lat->stream);
        cudaStreamWaitEvent(s0, g.events[i], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s0, &graph);
    for (Member &m : ms)
        if (m.lat->prof) m.lat->prof->capturing = false;
    g.launches = launch_count() - c0;
    note_launch_adjust(-(long long)g.launches);  // counted again on every replay
    if (st != QDD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiation");
    return QDD_OK;
}

}  // namespace

void set_batch_lists(bool on) { g_batch_lists.store(on ? 1 : 0); }
bool batch_lists() { return g_batch_lists.load() != 0; }

qdd_status solve_batch_impl(qdd_lattice *const *lats, double *const *phi_dev, const double *const *eta_dev, int n,
                            const double *kappa, const double *csw, double tol, const qdd_solver_params *const *ps,
                            qdd_solve_info *const *infos)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    double t_inner = 0.0;
    // plain FP64 BiCGStab or nested solve, and the outer level, are common to
    // the batch; everything else is per lattice
    const bool plain = ps[0]->inner_prec == P64;
    for (int i = 1; i < n; i++)
        if ((ps[i]->inner_prec == P64) != plain || ps[i]->outer_mode != ps[0]->outer_mode) {
            set_error("the lattices of a batch must share the plain FP64 solver or the nested one, and outer_mode");
            return QDD_ERR_ARG;
        }
    std::vector<Member> ms(n);
    std::vector<qdd_lattice *> L(n);
    qdd_status st;
    for (int i = 0; i < n; i++) {
        Member &m = ms[i];
        m.lat = L[i] = lats[i];
        m.phi_dev = phi_dev[i];
        m.eta_dev = eta_dev[i];
        m.kappa = kappa[i];
        m.csw = csw[i];
        m.info = infos ? infos[i] : nullptr;
        m.prm = *ps[i];
        m.prec = m.prm.inner_prec;
        m.use_ras = !plain && m.prm.use_ras;
        if (m.use_ras) {
            std::string why;
            if (!domain_geom(m.lat->g, m.prm.block, m.prm.overlap, &m.dg, &why)) {
                set_error("invalid RAS blocking: " + why);
                return QDD_ERR_ARG;
            }
        }
        const int R = m.lat->nrhs;
        m.eta2.assign(R, 0.0);
        m.rr.assign(R, 0.0);
        m.best.assign(R, 0.0);
        m.stalls.assign(R, 0);
        m.restarted.assign(R, 0);
        m.done.assign(R, 0);
        m.result.assign(R, QDD_ERR_NOT_CONVERGED);
        m.oit.assign(R, 0);
        m.seen_rr.assign(R, 0.0);
        m.seen_it.assign(R, -1);
        if (m.info) memset(m.info, 0, sizeof(qdd_solve_info) * R);
        for (int j = 0; j < i; j++)
            if (L[j] == L[i]) {
                set_error("a lattice appears twice in one batch");
                return QDD_ERR_ARG;
            }
    }
    for (Member &m : ms) {
        qdd_lattice *lat = m.lat;
        if ((st = ensure_clover(lat, m.kappa, m.csw)) != QDD_OK) return st;
        if ((st = ensure_outer(lat)) != QDD_OK) return st;
        if ((st = ensure_inner(lat, m.prec)) != QDD_OK) return st;
        SpinorView eta = outer(lat, 0), phi = outer(lat, 1), r = outer(lat, 2);
        cudaError_t e;
        {
            ProfScope ps(lat, QDD_K_CONVERT);
            e = launch_import_spinor(lat->g, P64, eta, m.eta_dev, lat->nrhs, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "import");
        if ((st = blas(lat, P64, B_NORM, {eta}, AUX_ETA2)) != QDD_OK) return st;
        if ((st = blas(lat, P64, B_COPY, {r, eta})) != QDD_OK) return st;
        if ((st = blas(lat, P64, B_ZERO, {phi})) != QDD_OK) return st;
        if ((st = blas(lat, P64, B_NORM, {r}, AUX_R2)) != QDD_OK) return st;
    }
    if ((st = read_scalars(L)) != QDD_OK) return st;
    for (Member &m : ms)
        for (int r = 0; r < m.lat->nrhs; r++) {
            m.eta2[r] = m.lat->sc_host[r].aux[AUX_ETA2];
            m.rr[r] = m.best[r] = m.lat->sc_host[r].aux[AUX_R2];
            if (!std::isfinite(m.eta2[r])) {
                m.done[r] = 1;
                m.result[r] = QDD_ERR_NONFINITE;
            }
        }

    const bool graphs = graph_capable(ms);
    long long vmax = 0;
    for (Member &m : ms) vmax = std::max(vmax, m.lat->g.V);
    const int chunk = vmax >= (1 << 18) ? 2 : 4;
    // work-list groups need the lattices on distinct streams (as the graph
    // does) and their inner fields, allocated above
    Groups groups;
    std::vector<int> solo;
    if ((st = form_groups(ms, graphs && !plain && g_batch_lists.load() != 0, groups, solo)) != QDD_OK) return st;
    // the graph of `chunk` iterations, and one of a single iteration for the
    // replay that the residuals say ends the inner solve (a chunk there would
    // run iterations whose kernels return at once)
    IterGraph graph, graph1;
    graph1.id = 1;
    bool have_graph = false, have_graph1 = false;
    const bool nested_outer = !plain && ps[0]->outer_mode == 1;

    // One inner solve of every lattice: right-hand side r of lattice m is
    // src(m) / sqrt(nsc[r].aux[slot]), solved to the relative tolerance
    // sqrt(sc_host[r].aux[AUX_TOL2]) (set by the caller) for the right-hand
    // sides whose bit is set in active[m]; the solution is left in W_X.
    auto inner_solve = [&](const std::vector<SpinorView> &src, const std::vector<Scalars *> &nsc, int slot,
                           const std::vector<unsigned long long> &active) -> qdd_status {
        const auto ti = clk::now();
        qdd_status st;
        for (size_t i = 0; i < ms.size(); i++) {
            Member &m = ms[i];
            qdd_lattice *lat = m.lat;
            const int prec = m.prec;
            const int R = lat->nrhs;
            for (int r = 0; r < R; r++) {
                m.restarted[r] = 0;
                cudaError_t e = cudaMemcpyAsync(&lat->sc[r].aux[AUX_TOL2], &lat->sc_host[r].aux[AUX_TOL2],
                                                sizeof(double), cudaMemcpyHostToDevice, lat->stream);
                if (e != cudaSuccess) return cuda_fail(e, "scalar upload");
            }
            cudaError_t e;
            {
                ProfScope ps(lat, QDD_K_CONVERT);
                e = launch_convert_scaled(lat->g.V, prec, inner(lat, prec, W_B), src[i], nsc[i], slot, R, lat->stream);
            }
            if (e != cudaSuccess) return cuda_fail(e, "convert");
            auto F = [&](int k) { return inner(lat, prec, k); };
            if ((st = blas(lat, prec, B_INIT, {F(W_B), F(W_R), F(W_RHAT), F(W_X), F(W_P), F(W_V)}, 0, -1.0,
                           active[i])) != QDD_OK)
                return st;
            for (int r = 0; r < R; r++) m.seen_it[r] = -1;
        }
        // inner iterations of every lattice until no right-hand side runs
        bool one = false;  // the next replay runs a single iteration
        for (;;) {
            if (graphs) {
                if (!have_graph) {
                    // one eager iteration first: it sets kernel attributes and
                    // allocates scratch outside the capture
                    if ((st = enqueue_all(ms, groups, solo)) != QDD_OK) return st;
                    if ((st = build_graph(ms, groups, solo, chunk, graph)) != QDD_OK) return st;
                    have_graph = true;
                } else {
                    if (one && !have_graph1) {
                        if ((st = build_graph(ms, groups, solo, 1, graph1)) != QDD_OK) return st;
                        have_graph1 = true;
                    }
                    IterGraph &g = one ? graph1 : graph;
                    // the graph runs on the first lattice's stream: order it after
                    // the work already queued on the other lattices' streams, and
                    // their next work after it
                    cudaStream_t s0 = ms[0].lat->stream;
                    for (size_t i = 1; i < ms.size(); i++) {
                        cudaEventRecord(g.pre[i], ms[i].lat->stream);
                        cudaStreamWaitEvent(s0, g.pre[i], 0);
                    }
                    cudaError_t e = cudaGraphLaunch(g.exec, s0);
                    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
                    note_launch_adjust((long long)g.launches);
                    for (Member &m : ms)
                        if (m.lat->prof && !m.lat->prof->graph_pairs.empty()) m.lat->prof->graph_replays[g.id]++;
                    cudaEventRecord(g.post, s0);
                    for (size_t i = 1; i < ms.size(); i++) cudaStreamWaitEvent(ms[i].lat->stream, g.post, 0);
                }
            } else {
                for (int c = 0; c < (one ? 1 : chunk); c++)
                    if ((st = enqueue_all(ms, groups, solo)) != QDD_OK) return st;
            }
            if ((st = read_scalars(L)) != QDD_OK) return st;
            bool running = false;
            one = true;
            for (Member &m : ms) {
                qdd_lattice *lat = m.lat;
                bool restart = false;
                for (int r = 0; r < lat->nrhs; r++) {
                    const Scalars &h = lat->sc_host[r];
                    if (h.status == S_RUN && !one_more_suffices(m, r, h)) one = false;
                    if (h.status == S_RUN) {
                        if (h.iter >= m.prm.max_inner) {
                            // out of inner iterations: stop this right-hand side
                            const int conv = S_CONVERGED;
                            cudaMemcpyAsync(&lat->sc[r].status, &conv, sizeof(int), cudaMemcpyHostToDevice,
                                            lat->stream);
                            cudaStreamSynchronize(lat->stream);
                        } else {
                            running = true;
                        }
                    } else if (h.status == S_BREAK_RV || h.status == S_BREAK_TT) {
                        if (!m.restarted[r]) {
                            m.restarted[r] = 1;
                            restart = true;
                            running = true;
                        }
                    }
                }
                if (restart) {
                    const int prec = m.prec;
                    auto F = [&](int k) { return inner(lat, prec, k); };
                    if ((st = blas(lat, prec, B_RESTART, {F(W_RHAT), F(W_R), F(W_P), F(W_V)})) != QDD_OK) return st;
                }
            }
            if (!running) break;
        }
        // counts, and failures that end a right-hand side
        for (size_t i = 0; i < ms.size(); i++) {
            Member &m = ms[i];
            for (int r = 0; r < m.lat->nrhs; r++) {
                if (!((active[i] >> r) & 1ull) || m.done[r]) continue;
                const Scalars &h = m.lat->sc_host[r];
                if (m.info) {
                    m.info[r].inner_iters += h.iter;
                    const int nsweep = m.prm.n_ras * schwarz_plan(m.prm.schwarz, m.dg).colors;
                    m.info[r].dv_count += 2 * h.iter + (m.use_ras ? 2 * h.iter * (nsweep - 1) : 0);
                    m.info[r].ras_sweeps += m.use_ras ? 2 * h.iter * nsweep : 0;
                }
                if (h.status == S_NONFINITE) {
                    m.done[r] = 1;
                    m.result[r] = QDD_ERR_NONFINITE;
                } else if (h.status == S_TIMEOUT) {
                    m.done[r] = 1;
                    m.result[r] = QDD_ERR_TIMEOUT;
                }
            }
        }
        t_inner += std::chrono::duration<double, std::milli>(clk::now() - ti).count();
        return QDD_OK;
    };

    // Uploads the host copy of the outer scalars of right-hand side r.
    auto put_osc = [&](qdd_lattice *lat, int r) -> qdd_status {
        cudaError_t e = cudaMemcpyAsync(&lat->work->osc[r], &lat->work->osc_host[r], sizeof(Scalars),
                                        cudaMemcpyHostToDevice, lat->stream);
        return e == cudaSuccess ? QDD_OK : cuda_fail(e, "scalar upload");
    };

    // One pass of the outer BiCGStab (outer_mode 1) on D e = r from e = 0,
    // the inner solve as its flexible preconditioner M(y) = |y| inner(y/|y|):
    //   p = r + beta (p - omega v); phat = M(p); v = D phat; alpha = rho / <rhat, v>;
    //   s = r - alpha v; shat = M(s); t = D shat; omega = <t, s> / |t|^2;
    //   e += alpha phat + omega shat; r = s - omega t
    // until |r| <= 0.5 tol |eta| (or |s| is: then e += alpha phat), then phi += e.
    auto nested_pass = [&]() -> qdd_status {
        qdd_status st;
        std::vector<unsigned long long> active(ms.size(), 0);
        std::vector<SpinorView> src(ms.size());
        std::vector<Scalars *> nsc(ms.size());
        for (size_t i = 0; i < ms.size(); i++) {
            Member &m = ms[i];
            qdd_lattice *lat = m.lat;
            if ((st = ensure_nested(lat)) != QDD_OK) return st;
            Scalars *oh = lat->work->osc_host;
            for (int r = 0; r < lat->nrhs; r++) {
                oh[r].aux[AUX_TOL2] = m.rr[r] > 0 ? 0.25 * tol * tol * m.eta2[r] / m.rr[r] : 1.0;
                cudaError_t e = cudaMemcpyAsync(&lat->work->osc[r].aux[AUX_TOL2], &oh[r].aux[AUX_TOL2],
                                                sizeof(double), cudaMemcpyHostToDevice, lat->stream);
                if (e != cudaSuccess) return cuda_fail(e, "scalar upload");
                if (!m.done[r]) active[i] |= 1ull << r;
            }
            auto N = [&](int k) { return nested(lat, k); };
            if ((st = blas(lat, P64, B_INIT, {outer(lat, 2), N(N_R), N(N_RHAT), N(N_E), N(N_P), N(N_V)}, 0, -1.0,
                           active[i], lat->work->osc)) != QDD_OK)
                return st;
            nsc[i] = lat->work->osc;
        }
        if ((st = read_scalars(L, true)) != QDD_OK) return st;
        std::vector<std::vector<int>> sdone(ms.size());
        for (;;) {
            // the right-hand sides whose outer BiCGStab runs
            bool any = false;
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                active[i] = 0;
                sdone[i].assign(m.lat->nrhs, 0);
                for (int r = 0; r < m.lat->nrhs; r++) {
                    const bool budget = m.oit[r] < m.prm.max_outer;
                    if (m.lat->work->osc_host[r].status == S_RUN && !m.done[r] && budget) {
                        active[i] |= 1ull << r;
                        any = true;
                    } else if (m.lat->work->osc_host[r].status == S_RUN) {
                        // out of outer iterations: stop it
                        m.lat->work->osc_host[r].status = S_CONVERGED;
                        if ((st = put_osc(m.lat, r)) != QDD_OK) return st;
                    }
                }
            }
            if (!any) break;
            // p, phat = M(p), v = D phat with alpha, s, |s|^2
            for (size_t i = 0; i < ms.size(); i++) {
                const Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                auto N = [&](int k) { return nested(lat, k); };
                Scalars *osc = lat->work->osc;
                if ((st = blas(lat, P64, B_P, {N(N_P), N(N_R), N(N_V)}, 0, 0.0, ~0ull, osc)) != QDD_OK) return st;
                if ((st = blas(lat, P64, B_NORM, {N(N_P)}, AUX_Y2, 0.0, ~0ull, osc)) != QDD_OK) return st;
                if ((st = blas(lat, P64, B_ZERO, {N(N_PHAT)})) != QDD_OK) return st;
                src[i] = N(N_P);
                for (int r = 0; r < lat->nrhs; r++) lat->sc_host[r].aux[AUX_TOL2] = m.prm.inner_tol * m.prm.inner_tol;
            }
            if ((st = inner_solve(src, nsc, AUX_Y2, active)) != QDD_OK) return st;
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                auto N = [&](int k) { return nested(lat, k); };
                Scalars *osc = lat->work->osc;
                cudaError_t e;
                {
                    ProfScope ps(lat, QDD_K_CONVERT);
                    e = launch_accum_scaled(lat->g.V, m.prec, N(N_PHAT), inner(lat, m.prec, W_X), osc, AUX_Y2, lat->nrhs,
                                            lat->stream);
                }
                if (e != cudaSuccess) return cuda_fail(e, "accumulate");
                if ((st = run_dslash(lat, P64, EPI_RV, N(N_V), N(N_PHAT), N(N_RHAT), m.kappa, 0, osc)) != QDD_OK)
                    return st;
                if ((st = blas(lat, P64, B_S, {N(N_S), N(N_R), N(N_V)}, 0, 0.0, ~0ull, osc)) != QDD_OK) return st;
                if ((st = blas(lat, P64, B_NORM, {N(N_S)}, AUX_S2, 0.0, ~0ull, osc)) != QDD_OK) return st;
                if ((st = blas(lat, P64, B_ZERO, {N(N_SHAT)})) != QDD_OK) return st;
            }
            if ((st = read_scalars(L, true)) != QDD_OK) return st;
            // a right-hand side whose |s| already meets the target skips M(s)
            // and t: it is parked (status not running) until e += alpha phat
            for (size_t i = 0; i < ms.size(); i++) {
                const Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                Scalars *oh = lat->work->osc_host;
                for (int r = 0; r < lat->nrhs; r++) {
                    if (!((active[i] >> r) & 1ull)) continue;
                    if (oh[r].status != S_RUN) {
                        active[i] &= ~(1ull << r);
                    } else if (oh[r].aux[AUX_S2] <= oh[r].tol2) {
                        sdone[i][r] = 1;
                        active[i] &= ~(1ull << r);
                        oh[r].status = S_CONVERGED;
                        if ((st = put_osc(lat, r)) != QDD_OK) return st;
                    }
                }
                src[i] = nested(lat, N_S);
                for (int r = 0; r < lat->nrhs; r++) lat->sc_host[r].aux[AUX_TOL2] = m.prm.inner_tol * m.prm.inner_tol;
            }
            if ((st = inner_solve(src, nsc, AUX_S2, active)) != QDD_OK) return st;
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                auto N = [&](int k) { return nested(lat, k); };
                Scalars *osc = lat->work->osc;
                Scalars *oh = lat->work->osc_host;
                cudaError_t e;
                {
                    ProfScope ps(lat, QDD_K_CONVERT);
                    e = launch_accum_scaled(lat->g.V, m.prec, N(N_SHAT), inner(lat, m.prec, W_X), osc, AUX_S2, lat->nrhs,
                                            lat->stream);
                }
                if (e != cudaSuccess) return cuda_fail(e, "accumulate");
                if ((st = run_dslash(lat, P64, EPI_TS, N(N_T), N(N_SHAT), N(N_S), m.kappa, 0, osc)) != QDD_OK)
                    return st;
                for (int r = 0; r < lat->nrhs; r++)
                    if (sdone[i][r]) {  // omega = 0: e += alpha phat, r = s
                        oh[r].status = S_RUN;
                        oh[r].omega = make_double2(0.0, 0.0);
                        if ((st = put_osc(lat, r)) != QDD_OK) return st;
                    }
                if ((st = blas(lat, P64, B_XR,
                               {N(N_E), N(N_PHAT), N(N_SHAT), N(N_R), N(N_S), N(N_T), N(N_RHAT)}, 0, 0.0, ~0ull,
                               osc)) != QDD_OK)
                    return st;
            }
            if ((st = read_scalars(L, true)) != QDD_OK) return st;
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                for (int r = 0; r < m.lat->nrhs; r++) {
                    if (!((active[i] >> r) & 1ull) && !sdone[i][r]) continue;
                    m.oit[r]++;
                    if (m.info) m.info[r].outer_iters++;
                    const int os = m.lat->work->osc_host[r].status;
                    if (os == S_NONFINITE) {
                        m.done[r] = 1;
                        m.result[r] = QDD_ERR_NONFINITE;
                    }
                    // a breakdown ends the pass; the defect-correction loop
                    // restarts from the true residual
                }
            }
        }
        for (Member &m : ms)
            if ((st = blas(m.lat, P64, B_AXPY, {outer(m.lat, 1), nested(m.lat, N_E)})) != QDD_OK) return st;
        return QDD_OK;
    };

    for (int outer_it = 0;; outer_it++) {
        // which right-hand sides still need a correction
        bool any = false;
        for (Member &m : ms)
            for (int r = 0; r < m.lat->nrhs; r++) {
                if (m.done[r]) continue;
                const double rel = m.eta2[r] > 0 ? std::sqrt(m.rr[r] / m.eta2[r]) : 0.0;
                const bool budget = nested_outer ? m.oit[r] < m.prm.max_outer : outer_it < m.prm.max_outer;
                if (!std::isfinite(rel)) {
                    m.done[r] = 1;
                    m.result[r] = QDD_ERR_NONFINITE;
                } else if (rel <= tol) {
                    m.done[r] = 1;
                    m.result[r] = QDD_OK;
                } else if (!budget || (nested_outer && outer_it >= m.prm.max_outer)) {
                    m.done[r] = 1;
                } else {
                    any = true;
                }
            }
        if (!any) break;
        if (nested_outer) {
            if ((st = nested_pass()) != QDD_OK) return st;
        } else {
            // one inner solve of r / |r|, then phi += |r| x
            std::vector<unsigned long long> active(ms.size(), 0);
            std::vector<SpinorView> src(ms.size());
            std::vector<Scalars *> nsc(ms.size());
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                for (int r = 0; r < lat->nrhs; r++) {
                    // tolerance of this inner solve relative to |r|: no further than
                    // the outer target needs, with a margin for the gap between the
                    // recursive and the true residual
                    double tol_in = m.rr[r] > 0 ? 0.5 * tol * std::sqrt(m.eta2[r] / m.rr[r]) : 1.0;
                    if (!plain && m.prm.inner_tol > tol_in) tol_in = m.prm.inner_tol;
                    lat->sc_host[r].aux[AUX_TOL2] = tol_in * tol_in;
                    if (!m.done[r]) active[i] |= 1ull << r;
                }
                src[i] = outer(lat, 2);
                nsc[i] = lat->sc;
            }
            if ((st = inner_solve(src, nsc, AUX_R2, active)) != QDD_OK) return st;
            for (size_t i = 0; i < ms.size(); i++) {
                Member &m = ms[i];
                qdd_lattice *lat = m.lat;
                if (m.info)
                    for (int r = 0; r < lat->nrhs; r++)
                        if ((active[i] >> r) & 1ull) m.info[r].outer_iters++;
                cudaError_t e;
                {
                    ProfScope ps(lat, QDD_K_CONVERT);
                    e = launch_accum_scaled(lat->g.V, m.prec, outer(lat, 1), inner(lat, m.prec, W_X), lat->sc, AUX_R2,
                                            lat->nrhs, lat->stream);
                }
                if (e != cudaSuccess) return cuda_fail(e, "accumulate");
            }
        }
        // r = eta - D phi ; |r|^2
        for (Member &m : ms) {
            qdd_lattice *lat = m.lat;
            if ((st = run_dslash(lat, P64, EPI_XMY_NORM, outer(lat, 2), outer(lat, 1), outer(lat, 0), m.kappa,
                                 AUX_R2)) != QDD_OK)
                return st;
        }
        if ((st = read_scalars(L)) != QDD_OK) return st;
        for (Member &m : ms)
            for (int r = 0; r < m.lat->nrhs; r++) {
                if (m.done[r]) continue;
                m.rr[r] = m.lat->sc_host[r].aux[AUX_R2];
                if (m.rr[r] < 0.5 * m.best[r]) {
                    m.best[r] = m.rr[r];
                    m.stalls[r] = 0;
                } else if (++m.stalls[r] >= 3) {
                    m.done[r] = 1;
                    const int s = m.lat->sc_host[r].status;
                    m.result[r] = (s == S_BREAK_RV || s == S_BREAK_TT) ? QDD_ERR_BREAKDOWN : QDD_ERR_NOT_CONVERGED;
                }
            }
    }
    qdd_status result = QDD_OK;
    for (Member &m : ms) {
        qdd_lattice *lat = m.lat;
        cudaError_t e;
        {
            ProfScope ps(lat, QDD_K_CONVERT);
            e = launch_export_spinor(lat->g, P64, m.phi_dev, outer(lat, 1), lat->nrhs, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "export");
    }
    for (Member &m : ms) {
        cudaError_t e = cudaStreamSynchronize(m.lat->stream);
        if (e != cudaSuccess) return cuda_fail(e, "solve");
    }
    const double total = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    for (Member &m : ms)
        for (int r = 0; r < m.lat->nrhs; r++) {
            if (m.result[r] != QDD_OK && result == QDD_OK) result = (qdd_status)m.result[r];
            if (m.info) {
                m.info[r].status = m.result[r];
                m.info[r].true_rel_residual = m.eta2[r] > 0 ? std::sqrt(m.rr[r] / m.eta2[r]) : 0.0;
                m.info[r].t_total_ms = total;
                m.info[r].t_inner_ms = t_inner;
                m.info[r].t_outer_ms = total - t_inner;
            }
        }
    if (result == QDD_ERR_NOT_CONVERGED) set_error("solve did not reach the tolerance");
    else if (result == QDD_ERR_BREAKDOWN) set_error("BiCGStab broke down");
    else if (result == QDD_ERR_NONFINITE) set_error("non-finite residual");
    else if (result == QDD_ERR_TIMEOUT) set_error("a RAS sweep gave up waiting for its staged data");
    return result;
}

qdd_status solve_impl(qdd_lattice *lat, double *phi_dev, const double *eta_dev, double kappa, double csw, double tol,
                      const qdd_solver_params *p, qdd_solve_info *info)
{
    qdd_lattice *lats[1] = {lat};
    double *phis[1] = {phi_dev};
    const double *etas[1] = {eta_dev};
    qdd_solve_info *infos[1] = {info};
    const qdd_solver_params *ps[1] = {p};
    return solve_batch_impl(lats, phis, etas, 1, &kappa, &csw, tol, ps, info ? infos : nullptr);
}

}  // namespace qdd
