// Batches of independent slices (one plan each, any mix of geometries):
// a largest-first (LPT) schedule of the slices over a pool of CUDA streams,
// fork/join against the caller's stream, and each plan's captured iteration
// graph replayed on its stream, so that small slices run side by side and
// fill the GPU.  The same host scheduler splits a batch across processes.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <set>
#include <vector>

#include "internal.cuh"

namespace dgct {

constexpr int kMaxDevices = 64;

// Lazily created non-blocking streams, per device, shared by every batch call.
static std::mutex g_pool_mu;
static std::vector<cudaStream_t> g_pool[kMaxDevices];

static int stream_pool(int device, int count, std::vector<cudaStream_t>& out) {
    if (device < 0 || device >= kMaxDevices) return DGAMP_CT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto& pool = g_pool[device];
    while ((int)pool.size() < count) {
        cudaStream_t s;
        DGCT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        pool.push_back(s);
    }
    out.assign(pool.begin(), pool.begin() + count);
    return DGAMP_CT_OK;
}

}  // namespace dgct

using namespace dgct;

extern "C" {

int dgamp_ct_schedule_lpt(int32_t n, const int64_t* work, int32_t queues, int32_t* queue_of, int64_t* load) {
    if (n < 0 || queues < 1 || (n > 0 && (!work || !queue_of))) return DGAMP_CT_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n; ++i)
        if (work[i] < 0) return DGAMP_CT_ERR_INVALID_ARG;
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    // largest first; equal work keeps the input order
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    std::vector<int64_t> acc(queues, 0);
    for (int32_t i : order) {
        int32_t best = 0;
        for (int32_t q = 1; q < queues; ++q)
            if (acc[q] < acc[best]) best = q;   // least loaded; ties to the lowest index
        queue_of[i] = best;
        acc[best] += work[i];
    }
    if (load)
        for (int32_t q = 0; q < queues; ++q) load[q] = acc[q];
    return DGAMP_CT_OK;
}

int dgamp_ct_solve_batched(int32_t n, const dgamp_ct_plan_t* plans, const float* const* d_counts, const double* I0,
                           int32_t iters, float* const* d_mu_out, dgamp_ct_stats* stats, void* stream) {
    if (n < 0 || (n > 0 && (!plans || !d_counts || !I0 || !d_mu_out))) return DGAMP_CT_ERR_INVALID_ARG;
    if (n == 0) return DGAMP_CT_OK;
    if (iters < 1 || iters > kMaxIters) return DGAMP_CT_ERR_INVALID_ARG;
    int device = 0;
    DGCT_CUDA(cudaGetDevice(&device));
    std::set<dgamp_ct_plan_t> seen;
    std::set<const dgamp_ct_cnn_s*> nets;   // a network's workspace serves one solve at a time
    std::vector<int64_t> work(n);
    for (int32_t i = 0; i < n; ++i) {
        const dgamp_ct_plan_t pl = plans[i];
        if (!pl || !d_counts[i] || !d_mu_out[i] || !(I0[i] > 0) || !std::isfinite(I0[i])) return DGAMP_CT_ERR_INVALID_ARG;
        if (pl->device != device) return DGAMP_CT_ERR_INVALID_ARG;
        if (pl->opt.denoiser == 1 && !pl->cnn) return DGAMP_CT_ERR_INVALID_ARG;
        if (!seen.insert(pl).second) return DGAMP_CT_ERR_INVALID_ARG;   // a plan holds one slice's state
        if (pl->opt.denoiser == 1 && !nets.insert(pl->cnn).second) return DGAMP_CT_ERR_INVALID_ARG;
        work[i] = (int64_t)pl->nv * pl->nd * pl->n;                   // Joseph steps of one projection
    }
    const int32_t queues = std::min<int32_t>(n, kBatchStreams);
    std::vector<int32_t> queue_of(n);
    DGCT_TRY(dgamp_ct_schedule_lpt(n, work.data(), queues, queue_of.data(), nullptr));
    std::vector<cudaStream_t> qs;
    DGCT_TRY(stream_pool(device, queues, qs));

    cudaStream_t st = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(queues + 1, nullptr);
    for (auto& e : ev) DGCT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int rc = DGAMP_CT_OK;
    cudaError_t ce = cudaEventRecord(ev[queues], st);                  // fork
    for (int32_t q = 0; q < queues && ce == cudaSuccess; ++q) ce = cudaStreamWaitEvent(qs[q], ev[queues], 0);
    if (ce != cudaSuccess) rc = cuda_fail(ce);
    // enqueue in schedule order (largest first) so the big slices start first
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    for (int32_t k = 0; k < n && rc == DGAMP_CT_OK; ++k) {
        const int32_t i = order[k];
        rc = dgamp_ct_solve(plans[i], d_counts[i], I0[i], iters, d_mu_out[i], nullptr, nullptr, qs[queue_of[i]]);
    }
    // join every queue that was forked, whatever happened above
    for (int32_t q = 0; q < queues; ++q) {
        ce = cudaEventRecord(ev[q], qs[q]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ev[q], 0);
        if (ce != cudaSuccess && rc == DGAMP_CT_OK) rc = cuda_fail(ce);
    }
    for (auto& e : ev) cudaEventDestroy(e);   // destruction is deferred until the events complete
    if (rc != DGAMP_CT_OK || !stats) return rc;
    DGCT_CUDA(cudaStreamSynchronize(st));
    int out = DGAMP_CT_OK;
    for (int32_t i = 0; i < n; ++i) {
        const int r = fill_stats(plans[i], iters, &stats[i]);
        if (r != DGAMP_CT_OK && out == DGAMP_CT_OK) out = r;
    }
    return out;
}

}  // extern "C"
