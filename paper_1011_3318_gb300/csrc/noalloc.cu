// noalloc.cu -- K_RAS on caller-owned fields without any device allocation.
//
// Who needs it: callers that must not let a library allocate device memory
// when it applies the preconditioner -- host programs that manage all device
// memory in their own pool or arena and forbid libraries from calling
// cudaMalloc behind their back, and latency-critical loops where an
// allocation (and the implicit synchronisation of cudaFree) would stall the
// device.  qdd_ras_apply allocates its general-kernel scratch on first use
// with a given blocking; this entry point instead takes the scratch from a
// fixed array compiled into the library.
//
// The scratch is the file-scope array below: QDD_NOALLOC_SCRATCH_BYTES (16 MiB)
// on every GPU that loads this library, held until the process exits.  Host
// code must not pass the array's name to a kernel (on the host it names a
// host-side stand-in, not device memory); the device address is obtained once
// per device with cudaGetSymbolAddress, with that device current, on the
// first call made on that device.  Make that first call before any stream
// capture begins.  The call must be made with the lattice's device current.
//
// Every call shares the one array and overwrites it; the kernel initialises
// all the scratch it reads (residual and solution of each domain) before
// reading it, so nothing carries over between calls.  Calls whose kernels
// overlap on the GPU (different streams, or different lattices on the same
// device at the same time) race on the array and give wrong results.
#include <cstring>
#include <mutex>

#include "lib.h"

namespace {

constexpr size_t QDD_NOALLOC_SCRATCH_BYTES = 16u << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[QDD_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_dev[MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the lattice's device, which must be
// the current device (set up once per device).
qdd_status scratch_address(int lat_device, void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return qdd::cuda_fail(e, "cudaGetDevice");
    if (dev != lat_device) {
        qdd::set_error("the current device is not the lattice's device: make device " + std::to_string(lat_device) +
                       " current before calling");
        return QDD_ERR_STATE;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        qdd::set_error("device index out of range for the no-allocation scratch");
        return QDD_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return qdd::cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return QDD_OK;
}

}  // namespace

using namespace qdd;

extern "C" qdd_status qdd_ras_field_noalloc(qdd_lattice *lat, qdd_field *out, const qdd_field *in, qdd_field *rho,
                                            qdd_field *v, double kappa, double c_sw, const qdd_solver_params *params)
{
    set_error("");
    if (!lat || !out || !in || !rho || !v || !params) {
        set_error("null argument");
        return QDD_ERR_ARG;
    }
    const qdd_field *fs[4] = {out, in, rho, v};
    for (int i = 0; i < 4; i++) {
        if (fs[i]->lat != lat || fs[i]->prec != fs[0]->prec) {
            set_error("fields must belong to this lattice and share one precision");
            return QDD_ERR_ARG;
        }
        for (int j = 0; j < i; j++)
            if (fs[i] == fs[j]) {
                set_error("out, in, rho and v must be four different fields");
                return QDD_ERR_ARG;
            }
    }
    const int prec = out->prec;
    if (prec != QDD_F32 && prec != QDD_F16) {
        set_error("the no-allocation K_RAS needs QDD_F32 or QDD_F16 fields");
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
    const SchwarzPlan sp = schwarz_plan(params->schwarz, dg);
    if (sp.sum) {
        set_error("additive Schwarz with overlap needs a summation buffer: use qdd_ras_apply");
        return QDD_ERR_ARG;
    }
    const size_t per_slot = (size_t)36 * (size_t)dg.nloc * sizeof(float2);
    const size_t fit = QDD_NOALLOC_SCRATCH_BYTES / per_slot;
    if (fit < 1) {
        set_error("extended domain of " + std::to_string(dg.nloc) + " sites needs " + std::to_string(per_slot) +
                  " bytes of scratch; the no-allocation entry point holds " +
                  std::to_string(QDD_NOALLOC_SCRATCH_BYTES) + " bytes (at most " +
                  std::to_string(QDD_NOALLOC_SCRATCH_BYTES / (36 * sizeof(float2))) + " sites per domain)");
        return QDD_ERR_ARG;
    }
    void *scratch = nullptr;
    qdd_status st = scratch_address(lat->device, &scratch);
    if (st != QDD_OK) return st;
    if (lat->has_gauge && !(lat->clover_valid && lat->kappa_c == kappa && lat->csw_c == c_sw)) {
        // the clover build below would only be recorded, not run, while the
        // stream is captured, yet the cache would be marked as built
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(lat->stream, &cs);
        if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            if (e != cudaSuccess) cudaGetLastError();
            set_error("the clover term for this kappa and c_sw is not built and the lattice's stream is being "
                      "captured: make one call with these parameters before the capture");
            return QDD_ERR_STATE;
        }
    }
    if ((st = ensure_clover(lat, kappa, c_sw)) != QDD_OK) return st;  // a kernel launch, no allocation

    RasArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.g = lat->g;
    ra.dg = dg;
    ra.U = links_of(lat, prec);
    ra.A = clover_of(lat, prec);
    ra.kappa = (float)kappa;
    ra.n_iter = params->n_dominv;
    ra.sc = nullptr;
    ra.scratch = reinterpret_cast<float2 *>(scratch);
    ra.nrhs = lat->nrhs;
    const size_t items = (size_t)dg.ndom * (size_t)lat->nrhs;
    ra.slots = (int)(fit < items ? fit : items);

    DslashArgs da;
    memset(&da, 0, sizeof(da));
    da.g = lat->g;
    da.U = links_of(lat, prec);
    da.A = clover_of(lat, prec);
    da.kappa = kappa;
    da.rs = lat->rs;
    da.sc = lat->sc;
    da.nrhs = lat->nrhs;

    const int nsweep = params->n_ras * sp.colors;
    for (int j = 0; j < nsweep; j++) {
        const bool last = j == nsweep - 1;
        ra.in = j == 0 ? in->view() : rho->view();
        ra.vout = last ? SpinorView{nullptr, nullptr} : v->view();
        ra.acc = out->view();
        ra.accumulate = j > 0;
        ra.color = sp.colors == 2 ? 1 + j % 2 : 0;
        cudaError_t e;
        {
            ProfScope ps(lat, QDD_K_RAS);
            e = launch_ras_block_gmem(prec, ra, lat->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "RAS block kernel");
        if (!last) {
            // rho = rho_in - D v (no reduction, so no scratch)
            da.out = rho->view();
            da.in = v->view();
            da.y = ra.in;
            {
                ProfScope ps(lat, QDD_K_DSLASH);
                e = launch_dslash(prec, EPI_XMY, da, lat->stream);
            }
            if (e != cudaSuccess) return cuda_fail(e, "dslash kernel");
        }
    }
    return QDD_OK;
}
