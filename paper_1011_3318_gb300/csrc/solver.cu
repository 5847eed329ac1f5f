// solver.cu -- host orchestration of the nested solver (Sec. 3): FP64 outer
// defect correction around an inner BiCGStab in FP32 or FP16 storage, right-
// preconditioned by K_RAS (Eq. 3, Alg. 1); and the plain FP64 BiCGStab.
//
// Every vector operation runs in a kernel of this library; the host only
// enqueues launches on the lattice's stream and reads the solver status and
// residual norms (a few dozen bytes) to decide when to stop.
#include <chrono>
#include <cmath>
#include <cstring>

#include "lib.h"

struct qdd_work {
    // FP64 outer vectors: eta, phi, r
    void *o_d[3] = {nullptr, nullptr, nullptr};
    // inner vectors per precision: b x r rhat p v s t phat shat rho_ras v_ras
    static constexpr int NIN = 12;
    void *in_d[3][NIN] = {};
    float *in_n[3][NIN] = {};
    bool in_ok[3] = {false, false, false};
};

namespace qdd {

enum { W_B, W_X, W_R, W_RHAT, W_P, W_V, W_S, W_T, W_PHAT, W_SHAT, W_RHO, W_VR };

void work_free(qdd_work *w)
{
    if (!w) return;
    for (int k = 0; k < 3; k++) cudaFree(w->o_d[k]);
    for (int p = 0; p < 3; p++)
        for (int k = 0; k < qdd_work::NIN; k++) field_free(w->in_d[p][k], w->in_n[p][k]);
    delete w;
}

static qdd_status ensure_outer(qdd_lattice *lat)
{
    if (!lat->work) lat->work = new qdd_work();
    qdd_work *w = lat->work;
    for (int k = 0; k < 3; k++)
        if (!w->o_d[k]) {
            float *n = nullptr;
            qdd_status st = field_alloc(lat->g.V, P64, &w->o_d[k], &n);
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
        qdd_status st = field_alloc(lat->g.V, prec, &w->in_d[prec][k], &w->in_n[prec][k]);
        if (st != QDD_OK) return st;
    }
    w->in_ok[prec] = true;
    return QDD_OK;
}

static SpinorView inner(qdd_lattice *lat, int prec, int k)
{
    return SpinorView{lat->work->in_d[prec][k], lat->work->in_n[prec][k]};
}

static SpinorView outer(qdd_lattice *lat, int k) { return SpinorView{lat->work->o_d[k], nullptr}; }

static qdd_status blas(qdd_lattice *lat, int prec, int op, std::initializer_list<SpinorView> fs, int aux_slot = 0,
                       double tol2 = 0.0)
{
    BlasArgs a;
    memset(&a, 0, sizeof(a));
    a.V = lat->g.V;
    int i = 0;
    for (const SpinorView &f : fs) a.f[i++] = f;
    a.sc = lat->sc;
    a.rs = lat->rs;
    a.aux_slot = aux_slot;
    a.tol2_rel = tol2;
    ProfScope ps(lat, QDD_K_BLAS);
    cudaError_t e = launch_blas(prec, op, a, lat->stream);
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "blas kernel");
}

static qdd_status read_scalars(qdd_lattice *lat)
{
    cudaError_t e = cudaMemcpyAsync(lat->sc_host, lat->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e == cudaSuccess && lat->prof) lat->prof->drain();
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "reading solver scalars");
}

qdd_status run_dslash(qdd_lattice *lat, int prec, int epi, SpinorView out, SpinorView in, SpinorView y, double kappa,
                      int aux_slot)
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
    a.sc = lat->sc;
    a.aux_slot = aux_slot;
    ProfScope ps(lat, prec == P64 ? QDD_K_DSLASH_F64 : QDD_K_DSLASH);
    cudaError_t e = launch_dslash(prec, epi, a, lat->stream);
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "dslash kernel");
}

static qdd_status ensure_ras_scratch(qdd_lattice *lat, const DomainGeom &dg)
{
    const size_t need = ras_scratch_bytes(dg, ras_default_slots());
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

// out = K_RAS in (Alg. 1): sweep j projects, solves and restricts on every
// domain (one launch), accumulates phi += v, and updates rho = rho - D v
// except after the last sweep, where phi no longer depends on rho.
qdd_status ras_apply_fields(qdd_lattice *lat, int prec, const qdd_solver_params *p, const DomainGeom &dg,
                            SpinorView out, SpinorView in, SpinorView rho, SpinorView v, double kappa, int *dv,
                            const Scalars *sc)
{
    qdd_status st = ensure_ras_scratch(lat, dg);
    if (st != QDD_OK) return st;
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
    for (int j = 0; j < p->n_ras; j++) {
        const bool last = j == p->n_ras - 1;
        ra.in = j == 0 ? in : rho;
        ra.vout = last ? SpinorView{nullptr, nullptr} : v;
        ra.acc = out;
        ra.accumulate = j > 0;
        cudaError_t e;
        {
            ProfScope ps(lat, QDD_K_RAS);
            e = launch_ras_block(prec, ra, lat->stream);
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

struct InnerResult {
    int iters = 0;
    int dv = 0;
    int sweeps = 0;
    int status = S_RUN;
};

// BiCGStab (van der Vorst) on D x = b, right-preconditioned by K_RAS when
// use_ras: D K chi = b, x = K chi (Eq. 3).  b is inner(W_B); x is inner(W_X).
static qdd_status inner_bicgstab(qdd_lattice *lat, int prec, const qdd_solver_params *p, const DomainGeom *dg,
                                 double kappa, double tol, int maxit, InnerResult *res)
{
    auto F = [&](int k) { return inner(lat, prec, k); };
    qdd_status st = blas(lat, prec, B_INIT, {F(W_B), F(W_R), F(W_RHAT), F(W_X), F(W_P), F(W_V)}, 0, tol * tol);
    if (st != QDD_OK) return st;
    const bool ras = dg != nullptr;
    const SpinorView phat = ras ? F(W_PHAT) : F(W_P);
    const SpinorView shat = ras ? F(W_SHAT) : F(W_S);
    const int chunk = lat->g.V >= (1 << 18) ? 2 : 6;
    bool restarted = false;
    int dv_ras = 0;
    for (;;) {
        for (int c = 0; c < chunk; c++) {
            if ((st = blas(lat, prec, B_P, {F(W_P), F(W_R), F(W_V)})) != QDD_OK) return st;
            if (ras && (st = ras_apply_fields(lat, prec, p, *dg, phat, F(W_P), F(W_RHO), F(W_VR), kappa, &dv_ras,
                                              lat->sc)) != QDD_OK)
                return st;
            if ((st = run_dslash(lat, prec, EPI_RV, F(W_V), phat, F(W_RHAT), kappa, 0)) != QDD_OK) return st;
            if ((st = blas(lat, prec, B_S, {F(W_S), F(W_R), F(W_V)})) != QDD_OK) return st;
            if (ras && (st = ras_apply_fields(lat, prec, p, *dg, shat, F(W_S), F(W_RHO), F(W_VR), kappa, &dv_ras,
                                              lat->sc)) != QDD_OK)
                return st;
            if ((st = run_dslash(lat, prec, EPI_TS, F(W_T), shat, F(W_S), kappa, 0)) != QDD_OK) return st;
            if ((st = blas(lat, prec, B_XR, {F(W_X), phat, shat, F(W_R), F(W_S), F(W_T), F(W_RHAT)})) != QDD_OK)
                return st;
        }
        if ((st = read_scalars(lat)) != QDD_OK) return st;
        const Scalars &h = *lat->sc_host;
        res->iters = h.iter;
        if (h.status == S_CONVERGED || h.status == S_NONFINITE) break;
        if (h.status == S_BREAK_RV || h.status == S_BREAK_TT) {
            if (restarted) break;
            restarted = true;
            if ((st = blas(lat, prec, B_RESTART, {F(W_RHAT), F(W_R), F(W_P), F(W_V)})) != QDD_OK) return st;
            continue;
        }
        if (h.iter >= maxit) break;
    }
    res->status = lat->sc_host->status;
    res->dv = 2 * res->iters + (ras ? 2 * res->iters * (p->n_ras - 1) : 0);
    res->sweeps = ras ? 2 * res->iters * p->n_ras : 0;
    return QDD_OK;
}

qdd_status solve_impl(qdd_lattice *lat, double *phi_dev, const double *eta_dev, double kappa, double csw, double tol,
                      const qdd_solver_params *p, qdd_solve_info *info)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    double t_inner = 0.0;
    qdd_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    const int prec = p->inner_prec;
    const bool plain = prec == P64;
    const bool use_ras = !plain && p->use_ras;
    DomainGeom dg;
    if (use_ras) {
        std::string why;
        if (!domain_geom(lat->g, p->block, p->overlap, &dg, &why)) {
            set_error("invalid RAS blocking: " + why);
            return QDD_ERR_ARG;
        }
    }
    qdd_status st;
    if ((st = ensure_clover(lat, kappa, csw)) != QDD_OK) return st;
    if ((st = ensure_outer(lat)) != QDD_OK) return st;
    if ((st = ensure_inner(lat, prec)) != QDD_OK) return st;

    const Geom &g = lat->g;
    SpinorView eta = outer(lat, 0), phi = outer(lat, 1), r = outer(lat, 2);
    cudaError_t e;
    {
        ProfScope ps(lat, QDD_K_CONVERT);
        e = launch_import_spinor(g, P64, eta, eta_dev, lat->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "import");
    if ((st = blas(lat, P64, B_NORM, {eta}, 0)) != QDD_OK) return st;   // |eta|^2 -> aux[0]
    if ((st = blas(lat, P64, B_COPY, {r, eta})) != QDD_OK) return st;
    if ((st = blas(lat, P64, B_ZERO, {phi})) != QDD_OK) return st;
    if ((st = blas(lat, P64, B_NORM, {r}, 1)) != QDD_OK) return st;     // |r|^2 -> aux[1]
    if ((st = read_scalars(lat)) != QDD_OK) return st;
    const double eta2 = lat->sc_host->aux[0];
    double rr = lat->sc_host->aux[1];
    if (!std::isfinite(eta2)) {
        set_error("source has non-finite entries");
        return QDD_ERR_NONFINITE;
    }
    qdd_status result = QDD_ERR_NOT_CONVERGED;
    int stalls = 0;
    double best = rr;
    for (;;) {
        const double rel = eta2 > 0 ? std::sqrt(rr / eta2) : 0.0;
        inf.true_rel_residual = rel;
        if (!std::isfinite(rel)) { result = QDD_ERR_NONFINITE; break; }
        if (rel <= tol) { result = QDD_OK; break; }
        if (inf.outer_iters >= p->max_outer) break;
        // tolerance of this inner solve relative to |r|: do not solve further
        // than the outer target needs, with a margin for the gap between the
        // recursive and the true residual
        double tol_in = 0.5 * tol * std::sqrt(eta2 / rr);
        if (!plain && p->inner_tol > tol_in) tol_in = p->inner_tol;
        const auto ti = clk::now();
        {
            ProfScope ps(lat, QDD_K_CONVERT);
            e = launch_convert_scaled(g.V, prec, inner(lat, prec, W_B), r, lat->sc, 1, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "convert");
        InnerResult ir;
        if ((st = inner_bicgstab(lat, prec, p, use_ras ? &dg : nullptr, kappa, tol_in, p->max_inner, &ir)) !=
            QDD_OK)
            return st;
        t_inner += std::chrono::duration<double, std::milli>(clk::now() - ti).count();
        inf.inner_iters += ir.iters;
        inf.dv_count += ir.dv;
        inf.ras_sweeps += ir.sweeps;
        inf.outer_iters++;
        if (ir.status == S_NONFINITE) { result = QDD_ERR_NONFINITE; break; }
        // phi += |r| x ; r = eta - D phi ; |r|^2 -> aux[1]
        {
            ProfScope ps(lat, QDD_K_CONVERT);
            e = launch_accum_scaled(g.V, prec, phi, inner(lat, prec, W_X), lat->sc, 1, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "accumulate");
        if ((st = run_dslash(lat, P64, EPI_XMY_NORM, r, phi, eta, kappa, 1)) != QDD_OK) return st;
        if ((st = read_scalars(lat)) != QDD_OK) return st;
        rr = lat->sc_host->aux[1];
        if (rr < 0.5 * best) { best = rr; stalls = 0; }
        else if (++stalls >= 3) {
            result = (ir.status == S_BREAK_RV || ir.status == S_BREAK_TT) ? QDD_ERR_BREAKDOWN : QDD_ERR_NOT_CONVERGED;
            inf.true_rel_residual = eta2 > 0 ? std::sqrt(rr / eta2) : 0.0;
            break;
        }
    }
    {
        ProfScope ps(lat, QDD_K_CONVERT);
        e = launch_export_spinor(g, P64, phi_dev, phi, lat->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "export");
    e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "solve");
    inf.status = result;
    inf.t_total_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    inf.t_inner_ms = t_inner;
    inf.t_outer_ms = inf.t_total_ms - t_inner;
    if (info) *info = inf;
    if (result != QDD_OK) {
        if (result == QDD_ERR_NOT_CONVERGED) set_error("solve did not reach the tolerance");
        else if (result == QDD_ERR_BREAKDOWN) set_error("BiCGStab broke down");
        else set_error("non-finite residual");
    }
    return result;
}

}  // namespace qdd
