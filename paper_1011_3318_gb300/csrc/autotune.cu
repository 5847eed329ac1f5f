// autotune.cu -- picks the RAS parameters that minimise time to solution.
//
// The paper surveys NRAS = 1..10, N_dominv = 1..20 and d = 0, 2, 4 on its
// cluster and keeps the fastest (Sec. 5); this survey adds the sweep
// kernel's staging variant and the inner precision.  The best point depends on the
// machine: there the global D was dominated by GigE communication, here it is
// an HBM-bound kernel, so the balance between domain work and Krylov
// iterations moves.  This tuner times whole solves of the caller's system
// and searches coordinate-wise:
//   1. (N_dominv, NRAS) on the starting block shape,
//   2. the block shape (16 .. 256-site blocks, one orientation per shape),
//   3. (N_dominv, NRAS) again around the best point of each of the two best
//      shapes,
//   4. overlap s = 1 on the best shape when its extended domain stays small,
//   5. the staging variant of the sweep kernel, then the other inner precision,
//   6. tighter inner tolerances (fewer outer steps): 3e-4 with FP16 storage,
//      1e-4 and 1e-5 with FP32 storage;
//   7. the three fastest candidates timed three more times each, ranked by
//      the median of their four timings.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "lib.h"

namespace qdd {

namespace {

struct Trial {
    qdd_solver_params p;
    double ms;
};

bool same_ras(const qdd_solver_params &a, const qdd_solver_params &b)
{
    return memcmp(a.block, b.block, sizeof(a.block)) == 0 && a.overlap == b.overlap && a.n_dominv == b.n_dominv &&
           a.n_ras == b.n_ras && a.ras_kernel == b.ras_kernel && a.inner_prec == b.inner_prec &&
           a.inner_tol == b.inner_tol && a.schwarz == b.schwarz && a.outer_mode == b.outer_mode;
}

// Tuning cache, keyed by the lattice's extents, boundary signs and
// right-hand-side count.
struct ShapeKey {
    int L[4], bc[4], nrhs;
    bool operator<(const ShapeKey &o) const { return memcmp(this, &o, sizeof(ShapeKey)) < 0; }
};

std::mutex g_tuned_mu;
std::map<ShapeKey, qdd_solver_params> g_tuned;

ShapeKey shape_key(const qdd_lattice *lat)
{
    ShapeKey k;
    memset(&k, 0, sizeof(k));
    for (int mu = 0; mu < 4; mu++) {
        k.L[mu] = lat->g.L[mu];
        k.bc[mu] = lat->g.bc[mu];
    }
    k.nrhs = lat->nrhs;
    return k;
}

}  // namespace

void tuned_store(const qdd_lattice *lat, const qdd_solver_params &p)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[shape_key(lat)] = p;
}

bool tuned_lookup(const qdd_lattice *lat, qdd_solver_params *p)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(shape_key(lat));
    if (it == g_tuned.end()) return false;
    *p = it->second;
    return true;
}

qdd_status autotune_impl(qdd_lattice *lat, double *phi_dev, const double *eta_dev, double kappa, double csw,
                         double tol, qdd_solver_params *p, int max_trials, double *best_ms)
{
    using clk = std::chrono::steady_clock;
    std::vector<Trial> done;
    Trial best{*p, 1e300};
    qdd_status st = QDD_OK;

    auto trial = [&](qdd_solver_params q) -> void {
        if ((int)done.size() >= max_trials) return;
        for (const Trial &t : done)
            if (same_ras(t.p, q)) return;
        DomainGeom dg;
        if (!domain_geom(lat->g, q.block, q.overlap, &dg, nullptr)) return;
        // the general kernel is never the fastest
        if (dg.nloc > RAS_SMEM_MAX_SITES && !ras_cluster_shape(dg)) return;
        std::vector<qdd_solve_info> info(lat->nrhs);
        const auto t0 = clk::now();
        qdd_status s = solve_impl(lat, phi_dev, eta_dev, kappa, csw, tol, &q, info.data());
        const double ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
        if (s != QDD_OK && s != QDD_ERR_NOT_CONVERGED && s != QDD_ERR_BREAKDOWN && s != QDD_ERR_NONFINITE) {
            st = s;  // a CUDA or allocation failure ends the search
            return;
        }
        const double score = s == QDD_OK ? ms : 1e299;
        done.push_back(Trial{q, score});
        if (score < best.ms) best = Trial{q, score};
    };

    // warm the clover cache and the work vectors so the first trial is not penalised
    {
        std::vector<qdd_solve_info> info(lat->nrhs);
        qdd_solver_params q = *p;
        solve_impl(lat, phi_dev, eta_dev, kappa, csw, tol, &q, info.data());
    }
    const int nds[] = {1, 2, 3, 4, 6};
    const int nrs[] = {1, 2, 3};
    for (int nd : nds)
        for (int nr : nrs) {
            qdd_solver_params q = *p;
            q.n_dominv = nd;
            q.n_ras = nr;
            trial(q);
            if (st != QDD_OK) return st;
        }
    const int shapes[][4] = {{2, 2, 2, 2}, {4, 2, 2, 2}, {4, 4, 2, 2}, {4, 4, 4, 2}, {4, 4, 4, 4}, {8, 4, 4, 4}};
    const qdd_solver_params base = best.p;
    for (const auto &sh : shapes) {
        qdd_solver_params q = base;
        for (int mu = 0; mu < 4; mu++) q.block[mu] = sh[mu];
        q.overlap = 0;
        trial(q);
        if (st != QDD_OK) return st;
    }
    // refine (N_dominv, NRAS) around the two fastest block shapes: the best
    // (N_dominv, NRAS) of one shape need not be the best of another, so a
    // shape that loses at the first point can still win after refinement
    std::vector<qdd_solver_params> arounds;
    {
        std::vector<Trial> by = done;
        std::sort(by.begin(), by.end(), [](const Trial &a, const Trial &b) { return a.ms < b.ms; });
        for (const Trial &t : by) {
            bool seen = false;
            for (const qdd_solver_params &a : arounds) seen |= memcmp(a.block, t.p.block, sizeof(a.block)) == 0;
            if (!seen && t.ms < 1e299) arounds.push_back(t.p);
            if (arounds.size() == 2) break;
        }
    }
    for (const qdd_solver_params &around : arounds)
        for (int dnd = -1; dnd <= 1; dnd++)
            for (int nr : nrs) {
                qdd_solver_params q = around;
                q.n_dominv = around.n_dominv + dnd;
                q.n_ras = nr;
                if (q.n_dominv < 1) continue;
                trial(q);
                if (st != QDD_OK) return st;
            }
    {
        qdd_solver_params q = best.p;
        q.overlap = 1;
        trial(q);
        if (st != QDD_OK) return st;
    }
    // the staging variant of the sweep kernel, then the other inner precision
    for (int v = 1; v <= 2; v++) {
        qdd_solver_params q = best.p;
        q.ras_kernel = v;
        trial(q);
        if (st != QDD_OK) return st;
    }
    {
        qdd_solver_params q = best.p;
        q.inner_prec = q.inner_prec == QDD_F16 ? QDD_F32 : QDD_F16;
        trial(q);
        if (st != QDD_OK) return st;
    }
    // a tighter inner tolerance trades inner iterations for fewer outer
    // steps (each one an FP64 D): FP16 storage resolves residuals only a
    // little below 1e-3 (its 2^-11 rounding), FP32 storage far below
    {
        const qdd_solver_params base_t = best.p;
        const struct {
            int prec;
            double tol;
        } cands[] = {{QDD_F16, 3e-4}, {QDD_F32, 1e-4}, {QDD_F32, 1e-5}};
        for (const auto &c : cands) {
            qdd_solver_params q = base_t;
            q.inner_prec = c.prec;
            if (c.tol >= q.inner_tol) continue;
            q.inner_tol = c.tol;
            trial(q);
            if (st != QDD_OK) return st;
        }
    }
    if (best.ms >= 1e299) {
        set_error("autotune: no candidate converged");
        return QDD_ERR_NOT_CONVERGED;
    }
    // one timed solve per candidate is noisy at the few-percent level that
    // separates the leading candidates: the best three are timed three more
    // times each and ranked by their median
    {
        std::vector<Trial> top = done;
        std::sort(top.begin(), top.end(), [](const Trial &a, const Trial &b) { return a.ms < b.ms; });
        if (top.size() > 3) top.resize(3);
        double best_med = 1e300;
        for (const Trial &t : top) {
            if (t.ms >= 1e299) continue;
            double r[4] = {t.ms, 0, 0, 0};
            for (int k = 1; k < 4; k++) {
                std::vector<qdd_solve_info> info(lat->nrhs);
                qdd_solver_params q = t.p;
                const auto t0 = clk::now();
                qdd_status s = solve_impl(lat, phi_dev, eta_dev, kappa, csw, tol, &q, info.data());
                r[k] = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
                if (s != QDD_OK) r[k] = 1e299;
            }
            std::sort(r, r + 4);
            const double med = 0.5 * (r[1] + r[2]);
            if (med < best_med) {
                best_med = med;
                best = Trial{t.p, med};
            }
        }
    }
    *p = best.p;
    if (best_ms) *best_ms = best.ms;
    return QDD_OK;
}

}  // namespace qdd
