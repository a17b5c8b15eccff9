// Batched assembly of many patches (uneven size, degree, map and coefficient)
// as one CUDA graph launch.
//
// The first call with a given batch creates the matrices eagerly.  Later calls
// with the same batch (same descriptions, the same matrix handles, dtype and
// contraction arithmetic) replay a cached graph: every patch's kernel chain
// (tables, coefficient field, quadrature stages, interpolation, fill; with their
// stream-ordered scratch allocations) captured on B concurrent branches, patches
// assigned to branches longest-first by their stencil slot count.  B is picked
// by an autotuner on the first graph call: it captures B = 1, 2, 4, ..., 32
// (up to the batch size), times two replays of each and keeps the fastest.
// Replays add the graph's kernel count to iga_launch_count.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "iga_internal.cuh"

namespace iga {
namespace {

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    int branches = 0;
    float ms = 0.f;
    std::vector<iga_matrix_t> mats;      // the matrices the graph writes into
};

std::mutex g_batch_mu;
std::unordered_map<uint64_t, GraphEntry> g_graphs;
constexpr int kMaxBranches = 32;
struct Streams {
    int device = -1;
    cudaStream_t cap = nullptr;
    cudaStream_t br[kMaxBranches] = {};
    cudaEvent_t fork = nullptr, join[kMaxBranches] = {}, t0 = nullptr, t1 = nullptr;
};
Streams g_streams[16];

thread_local int t_branches = 0;
thread_local int64_t t_kernels = 0;
thread_local int t_cached = 0;
thread_local float t_ms = 0.f;

uint64_t fnv(uint64_t h, const void* data, size_t n)
{
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

cudaError_t get_streams(int dev, Streams*& S)
{
    if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
    S = &g_streams[dev];
    if (S->device == dev) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking);
    for (int b = 0; b < kMaxBranches && e == cudaSuccess; ++b) {
        e = cudaStreamCreateWithFlags(&S->br[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->join[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&S->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&S->t1);
    if (e == cudaSuccess) S->device = dev;
    return e;
}

int64_t item_work(const iga_batch_item_t& it)
{
    int64_t N = 1, S = 1;
    for (int d = 0; d < it.patch.dim && d < 3; ++d) {
        N *= (int64_t)it.patch.n_el[d] + it.p;
        S *= 2 * it.p + 1;
    }
    return N * S;
}

// Capture the whole batch on B branches of the capture stream into an executable graph.
int capture(Streams& S, int n, const iga_batch_item_t* items, int dtype, iga_matrix_t* A, int B,
            const std::vector<int>& order, GraphEntry& out)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(S.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return report_error(IGA_ECUDA, "begin graph capture failed");
    set_capture(true);
    const int64_t l0 = launch_count();
    int rc = IGA_OK;
    e = cudaEventRecord(S.fork, S.cap);
    for (int b = 0; b < B && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(S.br[b], S.fork, 0);
    // longest patches first, each to the branch with the least work so far
    std::vector<int64_t> load(B, 0);
    for (size_t k = 0; k < order.size() && e == cudaSuccess && rc == IGA_OK; ++k) {
        const int i = order[k];
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += item_work(items[i]);
        const iga_batch_item_t& it = items[i];
        iga_matrix_t h = A[i];
        rc = assemble_patch(&it.patch, it.p, &it.map, &it.kappa, it.M >= 1, it.M >= 1 ? it.M : 1, it.q,
                            it.domains, dtype, S.br[b], &h);
    }
    for (int b = 0; b < B && e == cudaSuccess; ++b) {
        e = cudaEventRecord(S.join[b], S.br[b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(S.cap, S.join[b], 0);
    }
    const int64_t captured = launch_count() - l0;
    add_launches(-captured);                 // nothing ran yet; replays add the count
    cudaError_t ee = cudaStreamEndCapture(S.cap, &graph);
    set_capture(false);
    if (rc != IGA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&out.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return report_error(IGA_ECUDA, cudaGetErrorString(e));
    out.kernels = captured;
    out.branches = B;
    (void)n;
    return IGA_OK;
}

}  // namespace

void batch_forget(iga_matrix_t A)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        const auto& m = it->second.mats;
        if (std::find(m.begin(), m.end(), A) != m.end()) {
            // a graph that may still run on some stream: wait for the device before destroying it
            cudaDeviceSynchronize();
            if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace iga

using namespace iga;

extern "C" {

int iga_assemble_batch(int n, const iga_batch_item_t* items, int dtype, void* stream, iga_matrix_t* A)
{
    if (n < 1 || !items || !A) return report_error(IGA_EINVAL, "batch needs n >= 1 items and n matrix handles");
    if (dtype != IGA_F64 && dtype != IGA_F32) return report_error(IGA_EINVAL, "dtype must be IGA_F64 or IGA_F32");
    cudaStream_t st = (cudaStream_t)stream;
    bool all = true;
    for (int i = 0; i < n; ++i) all = all && A[i] != nullptr;
    t_cached = 0;
    if (!all) {
        // first call: create every matrix with an eager assembly on the caller's stream
        const int64_t l0 = launch_count();
        for (int i = 0; i < n; ++i) {
            const iga_batch_item_t& it = items[i];
            const int rc = assemble_patch(&it.patch, it.p, &it.map, &it.kappa, it.M >= 1, it.M >= 1 ? it.M : 1, it.q,
                                          it.domains, dtype, stream, &A[i]);
            if (rc != IGA_OK) return rc;
        }
        t_branches = 0;
        t_kernels = launch_count() - l0;
        t_ms = 0.f;
        return IGA_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(IGA_ECUDA, "cudaGetDevice failed");
    uint64_t key = 1469598103934665603ull;
    key = fnv(key, &n, sizeof(n));
    key = fnv(key, items, sizeof(iga_batch_item_t) * (size_t)n);
    key = fnv(key, A, sizeof(iga_matrix_t) * (size_t)n);
    key = fnv(key, &dtype, sizeof(dtype));
    const int arith = current_arith(dtype);
    key = fnv(key, &arith, sizeof(arith));
    key = fnv(key, &dev, sizeof(dev));

    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto hit = g_graphs.find(key);
    if (hit != g_graphs.end()) {
        e = cudaGraphLaunch(hit->second.exec, st);
        if (e != cudaSuccess) return report_error(IGA_ECUDA, cudaGetErrorString(e));
        add_launches(hit->second.kernels);
        t_branches = hit->second.branches;
        t_kernels = hit->second.kernels;
        t_ms = hit->second.ms;
        t_cached = 1;
        return IGA_OK;
    }
    Streams* S = nullptr;
    if ((e = get_streams(dev, S)) != cudaSuccess) return report_error(IGA_ECUDA, cudaGetErrorString(e));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return item_work(items[a]) > item_work(items[b]); });
    // the capture stream follows the caller's stream
    cudaEvent_t in_ev = S->join[0];
    if ((e = cudaEventRecord(in_ev, st)) != cudaSuccess || (e = cudaStreamWaitEvent(S->cap, in_ev, 0)) != cudaSuccess)
        return report_error(IGA_ECUDA, cudaGetErrorString(e));
    GraphEntry best;
    for (int B = 1; B <= kMaxBranches && B <= std::max(1, n); B *= 2) {
        GraphEntry cand;
        const int rc = capture(*S, n, items, dtype, A, B, order, cand);
        if (rc != IGA_OK) {
            if (best.exec) cudaGraphExecDestroy(best.exec);
            return rc;
        }
        // one warm replay, then two timed ones
        e = cudaGraphLaunch(cand.exec, S->cap);
        if (e == cudaSuccess) e = cudaEventRecord(S->t0, S->cap);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = cudaGraphLaunch(cand.exec, S->cap);
        if (e == cudaSuccess) e = cudaEventRecord(S->t1, S->cap);
        if (e == cudaSuccess) e = cudaEventSynchronize(S->t1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, S->t0, S->t1);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(cand.exec);
            if (best.exec) cudaGraphExecDestroy(best.exec);
            return report_error(IGA_ECUDA, cudaGetErrorString(e));
        }
        add_launches(3 * cand.kernels);
        cand.ms = ms / 2.f;
        if (!best.exec || cand.ms < best.ms) {
            if (best.exec) cudaGraphExecDestroy(best.exec);
            best = cand;
        } else {
            cudaGraphExecDestroy(cand.exec);
        }
    }
    // the caller's stream follows the replays
    if ((e = cudaEventRecord(in_ev, S->cap)) != cudaSuccess || (e = cudaStreamWaitEvent(st, in_ev, 0)) != cudaSuccess)
        return report_error(IGA_ECUDA, cudaGetErrorString(e));
    best.mats.assign(A, A + n);
    g_graphs[key] = best;
    t_branches = best.branches;
    t_kernels = best.kernels;
    t_ms = best.ms;
    return IGA_OK;
}

int iga_batch_info(int* branches, int64_t* kernels, int* cached, float* tuned_ms)
{
    if (branches) *branches = t_branches;
    if (kernels) *kernels = t_kernels;
    if (cached) *cached = t_cached;
    if (tuned_ms) *tuned_ms = t_ms;
    return IGA_OK;
}

int iga_batch_release(void)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& kv : g_graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g_graphs.clear();
    return IGA_OK;
}

}  // extern "C"
