// api.cu -- the C ABI declared in include/qdd.h.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lib.h"

namespace qdd {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

qdd_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a non-sticky error
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QDD_ERR_NOMEM : QDD_ERR_CUDA;
}

size_t spinor_bytes(long long V, int prec)
{
    return prec == P64 ? (size_t)V * 192 : prec == P32 ? (size_t)V * 96 : (size_t)V * 48;
}

qdd_status field_alloc(long long V, int prec, void **d, float **n)
{
    *d = nullptr;
    *n = nullptr;
    cudaError_t e = cudaMalloc(d, spinor_bytes(V, prec));
    if (e == cudaSuccess && prec == P16) e = cudaMalloc((void **)n, (size_t)V * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(*d);
        *d = nullptr;
        *n = nullptr;
        set_error("device allocation of a spinor field failed");
        return QDD_ERR_NOMEM;
    }
    return QDD_OK;
}

void field_free(void *d, float *n)
{
    cudaFree(d);
    cudaFree(n);
}

LinkView links_of(const qdd_lattice *lat, int prec)
{
    return LinkView{prec == P64 ? lat->U64 : prec == P32 ? lat->U32 : lat->U16};
}

CloverView clover_of(const qdd_lattice *lat, int prec)
{
    if (prec == P64) return CloverView{lat->A64, nullptr};
    if (prec == P32) return CloverView{lat->A32, nullptr};
    return CloverView{lat->A16, lat->A16n};
}

qdd_status ensure_clover(qdd_lattice *lat, double kappa, double csw)
{
    if (!lat->has_gauge) {
        set_error("no gauge field loaded");
        return QDD_ERR_STATE;
    }
    if (lat->clover_valid && lat->kappa_c == kappa && lat->csw_c == csw) return QDD_OK;
    ProfScope ps(lat, QDD_K_CLOVER);
    cudaError_t e = launch_clover_build(lat->g, lat->Udf, kappa, csw, lat->A64, lat->A32, lat->A16, lat->A16n,
                                        lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clover build");
    lat->clover_valid = true;
    lat->kappa_c = kappa;
    lat->csw_c = csw;
    return QDD_OK;
}

}  // namespace qdd

using namespace qdd;

namespace {

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t canon_bytes(const qdd_lattice *lat) { return (size_t)lat->g.V * lat->nrhs * 24 * sizeof(double); }

qdd_status ensure_stage(qdd_lattice *lat, double **buf)
{
    if (*buf) return QDD_OK;
    cudaError_t e = cudaMalloc((void **)buf, canon_bytes(lat));
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(e, "staging buffer");
    }
    return QDD_OK;
}

// A device pointer holding the canonical spinor `src` (staged if on the host).
qdd_status stage_in(qdd_lattice *lat, const double *src, double **buf, const double **dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return QDD_OK;
    }
    qdd_status st = ensure_stage(lat, buf);
    if (st != QDD_OK) return st;
    cudaError_t e = cudaMemcpyAsync(*buf, src, canon_bytes(lat), cudaMemcpyHostToDevice, lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    *dev = *buf;
    return QDD_OK;
}

// Where to write the canonical spinor destined for `dst`.
qdd_status stage_out(qdd_lattice *lat, double *dst, double **buf, double **dev, bool *host)
{
    *host = !is_device_ptr(dst);
    if (!*host) {
        *dev = dst;
        return QDD_OK;
    }
    qdd_status st = ensure_stage(lat, buf);
    if (st != QDD_OK) return st;
    *dev = *buf;
    return QDD_OK;
}

qdd_status finish_out(qdd_lattice *lat, double *dst, const double *dev, bool host)
{
    if (!host) return QDD_OK;
    cudaError_t e = cudaMemcpyAsync(dst, dev, canon_bytes(lat), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return QDD_OK;
}

bool valid_prec(int p) { return p == QDD_F64 || p == QDD_F32 || p == QDD_F16; }

bool valid_params(const qdd_solver_params &p)
{
    return valid_prec(p.inner_prec) && p.max_inner >= 1 && p.max_outer >= 1 && p.n_ras >= 1 && p.n_dominv >= 0 &&
           valid_schwarz(p.schwarz) && (p.outer_mode == 0 || p.outer_mode == 1) &&
           (p.inner_prec == QDD_F64 || (p.inner_tol > 0 && p.inner_tol < 1));
}

qdd_status solve_batch_common(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                              const double *kappa, const double *c_sw, double tol,
                              const qdd_solver_params *const *ps, qdd_solve_info *info);

// The in/out field pair of precision prec of the canonical-layout entry points.
qdd_status io_fields(qdd_lattice *lat, int prec, SpinorView *fin, SpinorView *fout)
{
    for (int k = 0; k < 2; k++)
        if (!lat->io_d[prec][k]) {
            qdd_status st = field_alloc(lat->g.V * lat->nrhs, prec, &lat->io_d[prec][k], &lat->io_n[prec][k]);
            if (st != QDD_OK) return st;
        }
    *fin = SpinorView{lat->io_d[prec][0], lat->io_n[prec][0]};
    *fout = SpinorView{lat->io_d[prec][1], lat->io_n[prec][1]};
    return QDD_OK;
}

}  // namespace

namespace {

qdd_status solve_batch_common(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                              const double *kappa, const double *c_sw, double tol,
                              const qdd_solver_params *const *ps, qdd_solve_info *info)
{
    std::vector<const double *> deta(n);
    std::vector<double *> dphi(n);
    std::vector<bool> host(n);
    std::vector<qdd_solve_info *> infos(n, nullptr);
    size_t off = 0;
    qdd_status st;
    for (int i = 0; i < n; i++) {
        if (!lats[i] || !phi[i] || !eta[i]) {
            set_error("null lattice or buffer in the batch");
            return QDD_ERR_ARG;
        }
        bool h = false;
        if ((st = stage_in(lats[i], eta[i], &lats[i]->stage_a, &deta[i])) != QDD_OK) return st;
        if ((st = stage_out(lats[i], phi[i], &lats[i]->stage_b, &dphi[i], &h)) != QDD_OK) return st;
        host[i] = h;
        if (info) infos[i] = info + off;
        off += lats[i]->nrhs;
    }
    qdd_status res = solve_batch_impl(lats, dphi.data(), deta.data(), n, kappa, c_sw, tol, ps,
                                      info ? infos.data() : nullptr);
    if (res != QDD_OK && res != QDD_ERR_NOT_CONVERGED && res != QDD_ERR_BREAKDOWN && res != QDD_ERR_NONFINITE)
        return res;
    std::string keep = g_err;
    for (int i = 0; i < n; i++)
        if ((st = finish_out(lats[i], phi[i], dphi[i], host[i])) != QDD_OK) return st;
    g_err = keep;
    return res;
}

}  // namespace

extern "C" {

const char *qdd_version(void) { return "qdd 0.1 (sm_103a)"; }

const char *qdd_last_error(void) { return g_err.c_str(); }

void qdd_default_params(qdd_solver_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    for (int mu = 0; mu < 4; mu++) p->block[mu] = 4;
    p->overlap = 0;
    p->n_dominv = 4;
    p->n_ras = 3;
    p->inner_prec = QDD_F32;
    p->inner_tol = 1e-3;
    p->max_inner = 2000;
    p->max_outer = 50;
    p->use_ras = 1;
    p->outer_mode = 0;
    p->autotune = 0;
    p->ras_kernel = 0;
    p->schwarz = QDD_SCHWARZ_RAS;
}

qdd_status qdd_create_lattice(qdd_lattice **out, const int dims[4], const int bc[4], int n_rhs, void *cuda_stream)
{
    g_err.clear();
    if (!out || !dims || !bc) {
        set_error("null argument");
        return QDD_ERR_ARG;
    }
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (dims[mu] < 1 || dims[mu] > 4096) {
            set_error("lattice extents must be in 1..4096");
            return QDD_ERR_ARG;
        }
        if (bc[mu] != 1 && bc[mu] != -1) {
            set_error("boundary signs must be +1 or -1");
            return QDD_ERR_ARG;
        }
        V *= dims[mu];
    }
    if (V > QDD_MAX_SITES) {
        set_error("lattice volume above 119304647 sites (device field planes are indexed in 32 bits)");
        return QDD_ERR_ARG;
    }
    if (n_rhs < 1 || n_rhs > QDD_MAX_RHS) {
        set_error("n_rhs must be in 1..64");
        return QDD_ERR_ARG;
    }
    qdd_lattice *lat = new qdd_lattice();
    memset(lat, 0, sizeof(*lat));
    for (int mu = 0; mu < 4; mu++) {
        lat->g.L[mu] = dims[mu];
        lat->g.bc[mu] = bc[mu];
    }
    lat->g.stride[0] = 1;
    for (int mu = 1; mu < 4; mu++) lat->g.stride[mu] = lat->g.stride[mu - 1] * dims[mu - 1];
    lat->g.V = V;
    lat->nrhs = n_rhs;
    lat->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&lat->device);
    const int max_blocks = (int)(V / 64 + 4096);
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {&lat->U64, (size_t)V * 4 * 9 * 16}, {&lat->Udf, (size_t)V * 4 * 9 * 16}, {&lat->U32, (size_t)V * 4 * 3 * 16}, {&lat->U16, (size_t)V * 4 * 3 * 8},
        {&lat->A64, (size_t)V * 36 * 16},    {&lat->A32, (size_t)V * 18 * 16},    {&lat->A16, (size_t)V * 9 * 16},
        {(void **)&lat->A16n, (size_t)V * 4}, {(void **)&lat->rs.partials, (size_t)max_blocks * 4 * sizeof(double) * n_rhs},
        {(void **)&lat->rs.counter, (size_t)64 * n_rhs},     {(void **)&lat->sc, sizeof(Scalars) * n_rhs},
        {(void **)&lat->maxdev, 64},         {(void **)&lat->ras_err, 64},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            qdd_destroy_lattice(lat);
            return cuda_fail(e, "lattice allocation");
        }
    }
    lat->rs.max_blocks = max_blocks;
    cudaError_t e = cudaMemset(lat->rs.counter, 0, (size_t)64 * n_rhs);
    if (e == cudaSuccess) e = cudaMemset(lat->sc, 0, sizeof(Scalars) * n_rhs);
    if (e == cudaSuccess) e = cudaMemset(lat->ras_err, 0, 64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&lat->sc_host, sizeof(Scalars) * n_rhs);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&lat->copy_stream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaEventCreateWithFlags(&lat->copy_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        qdd_destroy_lattice(lat);
        return cuda_fail(e, "lattice initialisation");
    }
    *out = lat;
    return QDD_OK;
}

qdd_status qdd_destroy_lattice(qdd_lattice *lat)
{
    if (!lat) return QDD_OK;
    cudaStreamSynchronize(lat->stream);
    void *ptrs[] = {lat->U64, lat->Udf, lat->U32, lat->U16, lat->A64, lat->A32, lat->A16, lat->A16n, lat->rs.partials,
                    lat->rs.counter, lat->sc, lat->maxdev, lat->ras_err, lat->stage_a, lat->stage_b,
                    lat->ras_scratch, lat->gauge_stage, lat->as_sum};
    for (void *p : ptrs) cudaFree(p);
    if (lat->sc_host) cudaFreeHost(lat->sc_host);
    if (lat->copy_stream) {
        cudaStreamSynchronize(lat->copy_stream);
        cudaStreamDestroy(lat->copy_stream);
    }
    for (int k = 0; k < 2; k++)
        if (lat->copy_ev[k]) cudaEventDestroy(lat->copy_ev[k]);
    work_free(lat->work);
    for (int p = 0; p < 3; p++)
        for (int k = 0; k < 2; k++) field_free(lat->io_d[p][k], lat->io_n[p][k]);
    delete lat->prof;
    delete lat;
    return QDD_OK;
}

namespace {

// Loads the links (and, with_clover, builds the clover term for (kappa, csw)
// in the same pass).  Host links go through a device staging buffer kept for
// later loads, in chunks: the copy of chunk c + 1 (copy stream) overlaps the
// conversion of chunk c (lattice stream).  With the clover, the chunks are
// groups of t-slices and the clover of chunk c is built as soon as chunks
// c - 1, c and c + 1 are converted (the clover at a site reads links one
// step away in two directions), so that the build also hides behind the copy.
qdd_status load_gauge_impl(qdd_lattice *lat, const double *U, bool with_clover, double kappa, double csw)
{
    const size_t bytes = (size_t)lat->g.V * 72 * sizeof(double);
    const long long V = lat->g.V, per_site = 72;
    const int Lt = lat->g.L[3];
    const long long slice = lat->g.stride[3];
    // clover chunks: 8 groups of Lt / 8 >= 2 t-slices (a group's clover needs
    // its two neighbouring groups), else one build at the end; 32 groups of
    // one slice measured slower at 32^4 (6.7 against 6.2 ms: the small clover
    // launches lose their tails)
    const int T = Lt / 8;
    const int tchunks = 8;
    const bool clover_chunks = with_clover && Lt % 8 == 0 && T >= 2;
    auto build = [&](long long s0, long long s1) -> cudaError_t {
        ProfScope ps(lat, QDD_K_CLOVER);
        return launch_clover_build(lat->g, lat->Udf, kappa, csw, lat->A64, lat->A32, lat->A16, lat->A16n, lat->stream,
                                   s0, s1);
    };
    lat->clover_valid = false;
    cudaError_t e = cudaMemsetAsync(lat->maxdev, 0, sizeof(unsigned long long), lat->stream);
    bool built = false;
    if (e == cudaSuccess && !is_device_ptr(U)) {
        if (!lat->gauge_stage) {
            e = cudaMalloc((void **)&lat->gauge_stage, bytes);
            if (e != cudaSuccess) {
                lat->gauge_stage = nullptr;
                return cuda_fail(e, "gauge staging");
            }
        }
        const int chunks = clover_chunks ? tchunks : (V >= 65536 ? 8 : 1);
        auto lo = [&](int c) { return clover_chunks ? (long long)T * c * slice : V * c / chunks; };
        // the staging buffer is free once the lattice stream's earlier work is done
        e = cudaEventRecord(lat->copy_ev[0], lat->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->copy_stream, lat->copy_ev[0], 0);
        for (int c = 0; c < chunks && e == cudaSuccess; c++) {
            const long long s0 = lo(c), s1 = c + 1 < chunks ? lo(c + 1) : V;
            e = cudaMemcpyAsync(lat->gauge_stage + s0 * per_site, U + s0 * per_site,
                                (size_t)(s1 - s0) * per_site * sizeof(double), cudaMemcpyHostToDevice,
                                lat->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(lat->copy_ev[1], lat->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->stream, lat->copy_ev[1], 0);
            if (e == cudaSuccess) {
                ProfScope ps(lat, QDD_K_CLOVER);
                e = launch_gauge_convert(lat->g, lat->gauge_stage, lat->U64, lat->U32, lat->U16, lat->Udf,
                                         lat->maxdev, lat->stream, s0, s1);
            }
            // chunk c - 1 has both neighbours converted now
            if (e == cudaSuccess && clover_chunks && c >= 2) e = build(lo(c - 1), lo(c));
        }
        if (e == cudaSuccess && clover_chunks) {  // the last chunk and the first (which wraps to the last)
            e = build(lo(chunks - 1), V);
            if (e == cudaSuccess) e = build(0, lo(1));
            built = true;
        }
    } else if (e == cudaSuccess) {
        ProfScope ps(lat, QDD_K_CLOVER);
        e = launch_gauge_convert(lat->g, U, lat->U64, lat->U32, lat->U16, lat->Udf, lat->maxdev, lat->stream);
    }
    if (e == cudaSuccess && with_clover && !built) e = build(0, V);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, lat->maxdev, sizeof(bits), cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gauge conversion");
    double dev;
    memcpy(&dev, &bits, sizeof(dev));
    if (!(dev <= 1e-10)) {
        lat->has_gauge = false;
        set_error("gauge field is not SU(3): max deviation " + std::to_string(dev));
        return QDD_ERR_ARG;
    }
    lat->has_gauge = true;
    if (with_clover) {
        lat->clover_valid = true;
        lat->kappa_c = kappa;
        lat->csw_c = csw;
    }
    return QDD_OK;
}

}  // namespace

qdd_status qdd_load_gauge(qdd_lattice *lat, const double *U)
{
    g_err.clear();
    if (!lat || !U) {
        set_error("null argument");
        return QDD_ERR_ARG;
    }
    return load_gauge_impl(lat, U, false, 0.0, 0.0);
}

qdd_status qdd_load_gauge_clover(qdd_lattice *lat, const double *U, double kappa, double c_sw)
{
    g_err.clear();
    if (!lat || !U || !std::isfinite(kappa) || !std::isfinite(c_sw)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    return load_gauge_impl(lat, U, true, kappa, c_sw);
}

qdd_status qdd_dslash(qdd_lattice *lat, double *out, const double *in, double kappa, double c_sw, qdd_prec prec)
{
    g_err.clear();
    if (!lat || !out || !in || !valid_prec(prec)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_status st = ensure_clover(lat, kappa, c_sw);
    if (st != QDD_OK) return st;
    SpinorView fin, fout;
    if ((st = io_fields(lat, prec, &fin, &fout)) != QDD_OK) return st;
    const double *din;
    if ((st = stage_in(lat, in, &lat->stage_a, &din)) != QDD_OK) return st;
    cudaError_t e = launch_import_spinor(lat->g, prec, fin, din, lat->nrhs, lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "import");
    if ((st = run_dslash(lat, prec, EPI_D, fout, fin, SpinorView{nullptr, nullptr}, kappa, 0)) != QDD_OK) return st;
    double *dout;
    bool host;
    if ((st = stage_out(lat, out, &lat->stage_b, &dout, &host)) != QDD_OK) return st;
    e = launch_export_spinor(lat->g, prec, dout, fout, lat->nrhs, lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return finish_out(lat, out, dout, host);
}

// Reads (and clears) the lattice's RAS wait-timeout word; the stream must be idle.
static qdd_status check_ras_err(qdd_lattice *lat)
{
    unsigned flag = 0;
    cudaError_t e = cudaMemcpy(&flag, lat->ras_err, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the RAS status word");
    if (!flag) return QDD_OK;
    cudaMemset(lat->ras_err, 0, sizeof(flag));
    set_error("a RAS sweep gave up waiting for its staged data; the output is undefined");
    return QDD_ERR_TIMEOUT;
}

qdd_status qdd_ras_apply(qdd_lattice *lat, double *out, const double *in, double kappa, double c_sw,
                         const qdd_solver_params *params)
{
    g_err.clear();
    if (!lat || !out || !in || !params) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    const int prec = params->inner_prec;
    if (prec != QDD_F32 && prec != QDD_F16) {
        set_error("qdd_ras_apply needs inner_prec QDD_F32 or QDD_F16");
        return QDD_ERR_ARG;
    }
    if (params->n_ras < 1 || params->n_dominv < 0 || !valid_schwarz(params->schwarz)) {
        set_error("n_ras must be >= 1, n_dominv >= 0 and schwarz a qdd_schwarz");
        return QDD_ERR_ARG;
    }
    DomainGeom dg;
    std::string why;
    if (!domain_geom(lat->g, params->block, params->overlap, &dg, &why)) {
        set_error("invalid RAS blocking: " + why);
        return QDD_ERR_ARG;
    }
    qdd_status st = ensure_clover(lat, kappa, c_sw);
    if (st != QDD_OK) return st;
    SpinorView fin, fout;
    if ((st = io_fields(lat, prec, &fin, &fout)) != QDD_OK) return st;
    void *wd[2] = {nullptr, nullptr};
    float *wn[2] = {nullptr, nullptr};
    for (int k = 0; k < 2; k++)
        if ((st = field_alloc(lat->g.V * lat->nrhs, prec, &wd[k], &wn[k])) != QDD_OK) {
            for (int j = 0; j < 2; j++) field_free(wd[j], wn[j]);
            return st;
        }
    const double *din;
    double *dout = nullptr;
    bool host = false;
    cudaError_t e = cudaSuccess;
    if ((st = stage_in(lat, in, &lat->stage_a, &din)) == QDD_OK) {
        e = launch_import_spinor(lat->g, prec, fin, din, lat->nrhs, lat->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "import");
    }
    if (st == QDD_OK)
        st = ras_apply_fields(lat, prec, params, dg, fout, fin, SpinorView{wd[0], wn[0]}, SpinorView{wd[1], wn[1]},
                              kappa, nullptr, nullptr);
    if (st == QDD_OK) st = stage_out(lat, out, &lat->stage_b, &dout, &host);
    if (st == QDD_OK) {
        e = launch_export_spinor(lat->g, prec, dout, fout, lat->nrhs, lat->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "export");
    }
    if (st == QDD_OK) st = finish_out(lat, out, dout, host);
    cudaStreamSynchronize(lat->stream);
    for (int j = 0; j < 2; j++) field_free(wd[j], wn[j]);
    if (st == QDD_OK) st = check_ras_err(lat);
    return st;
}

qdd_status qdd_solve(qdd_lattice *lat, double *phi, const double *eta, double kappa, double c_sw, double tol,
                     const qdd_solver_params *params, qdd_solve_info *info)
{
    g_err.clear();
    if (!lat || !phi || !eta || !(tol > 0)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_solver_params p;
    if (params) p = *params;
    else qdd_default_params(&p);
    if (!valid_params(p)) {
        set_error("invalid solver parameters");
        return QDD_ERR_ARG;
    }
    qdd_status st;
    const double *deta;
    if (!is_device_ptr(eta)) {
        // the host source is copied on the copy stream while the clover term
        // is built on the lattice stream
        if ((st = ensure_stage(lat, &lat->stage_a)) != QDD_OK) return st;
        cudaError_t e = cudaEventRecord(lat->copy_ev[0], lat->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->copy_stream, lat->copy_ev[0], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(lat->stage_a, eta, canon_bytes(lat), cudaMemcpyHostToDevice, lat->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(lat->copy_ev[1], lat->copy_stream);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
        if ((st = ensure_clover(lat, kappa, c_sw)) != QDD_OK) return st;
        e = cudaStreamWaitEvent(lat->stream, lat->copy_ev[1], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
        deta = lat->stage_a;
    } else if ((st = stage_in(lat, eta, &lat->stage_a, &deta)) != QDD_OK) {
        return st;
    }
    double *dphi;
    bool host;
    if ((st = stage_out(lat, phi, &lat->stage_b, &dphi, &host)) != QDD_OK) return st;
    qdd_status res = solve_impl(lat, dphi, deta, kappa, c_sw, tol, &p, info);
    if (res != QDD_OK && res != QDD_ERR_NOT_CONVERGED && res != QDD_ERR_BREAKDOWN && res != QDD_ERR_NONFINITE)
        return res;
    std::string keep = g_err;
    st = finish_out(lat, phi, dphi, host);
    if (st != QDD_OK) return st;
    g_err = keep;
    return res;
}

qdd_status qdd_solve_batch(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                           const double *kappa, const double *c_sw, double tol, const qdd_solver_params *params,
                           qdd_solve_info *info)
{
    g_err.clear();
    if (!lats || !phi || !eta || !kappa || !c_sw || n < 1 || !(tol > 0)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_solver_params p;
    if (params) p = *params;
    else qdd_default_params(&p);
    if (!valid_params(p)) {
        set_error("invalid solver parameters");
        return QDD_ERR_ARG;
    }
    std::vector<const qdd_solver_params *> ps(n, &p);
    return solve_batch_common(lats, phi, eta, n, kappa, c_sw, tol, ps.data(), info);
}

qdd_status qdd_set_batch_lists(int on, int *previous)
{
    g_err.clear();
    if (previous) *previous = batch_lists() ? 1 : 0;
    set_batch_lists(on != 0);
    return QDD_OK;
}

qdd_status qdd_solve_batch_each(qdd_lattice *const *lats, double *const *phi, const double *const *eta, int n,
                                const double *kappa, const double *c_sw, double tol,
                                const qdd_solver_params *const *params, qdd_solve_info *info)
{
    g_err.clear();
    if (!lats || !phi || !eta || !kappa || !c_sw || n < 1 || !(tol > 0)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    std::vector<qdd_solver_params> own(n);
    std::vector<const qdd_solver_params *> ps(n);
    for (int i = 0; i < n; i++) {
        if (!lats[i]) {
            set_error("null lattice in the batch");
            return QDD_ERR_ARG;
        }
        if (params && params[i]) own[i] = *params[i];
        else if (!tuned_lookup(lats[i], &own[i])) qdd_default_params(&own[i]);
        if (!valid_params(own[i])) {
            set_error("invalid solver parameters for lattice " + std::to_string(i));
            return QDD_ERR_ARG;
        }
        ps[i] = &own[i];
    }
    return solve_batch_common(lats, phi, eta, n, kappa, c_sw, tol, ps.data(), info);
}

qdd_status qdd_tuned_params(const qdd_lattice *lat, qdd_solver_params *params)
{
    g_err.clear();
    if (!lat || !params) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    if (!tuned_lookup(lat, params)) {
        set_error("no tuned parameters for this lattice shape (run qdd_autotune first)");
        return QDD_ERR_STATE;
    }
    return QDD_OK;
}

qdd_status qdd_autotune(qdd_lattice *lat, const double *eta, double kappa, double c_sw, double tol,
                        qdd_solver_params *params, int max_trials, double *best_ms)
{
    g_err.clear();
    if (!lat || !eta || !params || !(tol > 0) || max_trials < 1) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    if ((params->inner_prec != QDD_F32 && params->inner_prec != QDD_F16) || !params->use_ras) {
        set_error("qdd_autotune tunes the RAS parameters of an FP32 or FP16 inner solve (use_ras = 1)");
        return QDD_ERR_ARG;
    }
    qdd_status st;
    const double *deta;
    if ((st = stage_in(lat, eta, &lat->stage_a, &deta)) != QDD_OK) return st;
    double *dphi = nullptr;
    if ((st = ensure_stage(lat, &lat->stage_b)) != QDD_OK) return st;
    dphi = lat->stage_b;
    if ((st = autotune_impl(lat, dphi, deta, kappa, c_sw, tol, params, max_trials, best_ms)) != QDD_OK) return st;
    tuned_store(lat, *params);
    return QDD_OK;
}

qdd_status qdd_field_create(qdd_lattice *lat, qdd_prec prec, qdd_field **out)
{
    g_err.clear();
    if (!lat || !out || !valid_prec(prec)) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_field *f = new qdd_field();
    f->lat = lat;
    f->prec = prec;
    qdd_status st = field_alloc(lat->g.V * lat->nrhs, prec, &f->d, &f->n);
    if (st != QDD_OK) {
        delete f;
        return st;
    }
    *out = f;
    return QDD_OK;
}

qdd_status qdd_field_destroy(qdd_field *f)
{
    if (!f) return QDD_OK;
    cudaStreamSynchronize(f->lat->stream);
    field_free(f->d, f->n);
    delete f;
    return QDD_OK;
}

qdd_status qdd_field_import(qdd_field *f, const double *src)
{
    g_err.clear();
    if (!f || !src) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_lattice *lat = f->lat;
    const double *d;
    qdd_status st = stage_in(lat, src, &lat->stage_a, &d);
    if (st != QDD_OK) return st;
    cudaError_t e = launch_import_spinor(lat->g, f->prec, f->view(), d, lat->nrhs, lat->stream);
    return e == cudaSuccess ? QDD_OK : cuda_fail(e, "import");
}

qdd_status qdd_field_export(const qdd_field *f, double *dst)
{
    g_err.clear();
    if (!f || !dst) {
        set_error("invalid argument");
        return QDD_ERR_ARG;
    }
    qdd_lattice *lat = f->lat;
    double *d;
    bool host;
    qdd_status st = stage_out(lat, dst, &lat->stage_b, &d, &host);
    if (st != QDD_OK) return st;
    cudaError_t e = launch_export_spinor(lat->g, f->prec, d, f->view(), lat->nrhs, lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return finish_out(lat, dst, d, host);
}

qdd_status qdd_dslash_field(qdd_lattice *lat, qdd_field *out, const qdd_field *in, double kappa, double c_sw)
{
    g_err.clear();
    if (!lat || !out || !in || out == in || out->prec != in->prec || out->lat != lat || in->lat != lat) {
        set_error("invalid argument (fields must differ, share the lattice and the precision)");
        return QDD_ERR_ARG;
    }
    qdd_status st = ensure_clover(lat, kappa, c_sw);
    if (st != QDD_OK) return st;
    return run_dslash(lat, out->prec, EPI_D, out->view(), in->view(), SpinorView{nullptr, nullptr}, kappa, 0);
}

}  // extern "C"
