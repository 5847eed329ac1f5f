// diag.cu -- launch counting, per-kernel-class GPU timing and an FMA
// throughput probe (measurement support for the roofline of each kernel).
#include <atomic>
#include <cstring>

#include "lib.h"

namespace qdd {

static std::atomic<unsigned long long> g_launches{0};

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void note_launch_adjust(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

unsigned long long launch_count() { return g_launches.load(); }

Profiler::~Profiler()
{
    for (auto &p : pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto &p : graph_pairs) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

void Profiler::release_graph()
{
    for (auto &p : graph_pairs) {
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    graph_pairs.clear();
    graph_replays[0] = graph_replays[1] = 0;
}

cudaEvent_t Profiler::get()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void Profiler::drain()
{
    // each replay of a captured graph re-records its pairs; one replay runs
    // between two reads, so the pairs hold the last replay's times
    for (auto &p : graph_pairs) {
        const int reps = graph_replays[p.graph];
        if (reps <= 0) continue;
        float ms_ = 0.f;
        if (cudaEventElapsedTime(&ms_, p.a, p.b) == cudaSuccess) {
            ms[p.cls] += ms_ * reps;
            n[p.cls] += reps;
        } else {
            cudaGetLastError();
        }
    }
    graph_replays[0] = graph_replays[1] = 0;
    for (auto &p : pending) {
        float ms_ = 0.f;
        if (cudaEventElapsedTime(&ms_, p.a, p.b) == cudaSuccess) {
            ms[p.cls] += ms_;
            n[p.cls] += 1;
        } else {
            cudaGetLastError();
        }
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}

ProfScope::ProfScope(qdd_lattice *lat, int cls) : prof(lat->prof), cls(cls), st(lat->stream), a(nullptr)
{
    if (!prof || !prof->on) return;
    a = prof->get();
    // inside a stream capture only an "external" record becomes an event
    // node that records a time stamp when the graph runs
    if (a) cudaEventRecordWithFlags(a, st, prof->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEvent_t b = prof->get();
    if (!b) {
        prof->pool.push_back(a);
        return;
    }
    cudaEventRecordWithFlags(b, st, prof->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    if (prof->capturing) {  // the records are nodes of the graph being captured
        prof->graph_pairs.push_back(Profiler::Pair{cls, a, b, prof->capture_graph});
        return;
    }
    prof->pending.push_back(Profiler::Pair{cls, a, b, 0});
    // bound the number of outstanding pairs: drain (which waits) when many
    if (prof->pending.size() >= 4096) {
        cudaEventSynchronize(b);
        prof->drain();
    }
}

// ---------------------------------------------------------------- FMA probe
template <typename T>
__global__ void fma_probe_kernel(T *sink, int iters, T seed)
{
    T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
      a7 = a0 + 7;
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 16; k++) {
            a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
            a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
        }
    }
    const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == (T)-1.2345) sink[threadIdx.x] = s;  // never true; keeps the chains alive
}

template <typename T>
static qdd_status fma_probe(double *tflops)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 1024 * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "probe allocation");
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 256 : 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fma_probe_kernel<T><<<blocks, threads>>>(sink, iters, (T)1);  // warm-up
    cudaEventRecord(a);
    const int reps = 5;
    for (int r = 0; r < reps; r++) fma_probe_kernel<T><<<blocks, threads>>>(sink, iters, (T)1);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    note_launch(reps + 1);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "probe");
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return QDD_OK;
}

}  // namespace qdd

using namespace qdd;

extern "C" {

unsigned long long qdd_kernel_launches(void) { return g_launches.load(); }

qdd_status qdd_set_profiling(qdd_lattice *lat, int on)
{
    if (!lat) {
        set_error("null lattice");
        return QDD_ERR_ARG;
    }
    if (!lat->prof) lat->prof = new Profiler();
    lat->prof->on = on != 0;
    return QDD_OK;
}

qdd_status qdd_profile_read(qdd_lattice *lat, qdd_profile *out, int reset)
{
    if (!lat || !out) {
        set_error("null argument");
        return QDD_ERR_ARG;
    }
    memset(out, 0, sizeof(*out));
    if (!lat->prof) return QDD_OK;
    cudaError_t e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "profile read");
    lat->prof->drain();
    for (int k = 0; k < QDD_NKCLASS; k++) {
        out->ms[k] = lat->prof->ms[k];
        out->launches[k] = lat->prof->n[k];
    }
    if (reset) {
        memset(lat->prof->ms, 0, sizeof(lat->prof->ms));
        memset(lat->prof->n, 0, sizeof(lat->prof->n));
    }
    return QDD_OK;
}

qdd_status qdd_measure_fma_peak(int fp64, double *tflops)
{
    if (!tflops) {
        set_error("null argument");
        return QDD_ERR_ARG;
    }
    return fp64 ? fma_probe<double>(tflops) : fma_probe<float>(tflops);
}

qdd_status qdd_test_ras_wait(unsigned extra_bytes, long max_polls)
{
    ras_set_wait_test(extra_bytes, max_polls);
    return QDD_OK;
}

}  // extern "C"
