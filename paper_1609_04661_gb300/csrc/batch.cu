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
        const bool cnn = pl->opt.denoiser == 1 || pl->opt.denoiser == 2;
        if (cnn && !pl->cnn) return DGAMP_CT_ERR_INVALID_ARG;
        if (!seen.insert(pl).second) return DGAMP_CT_ERR_INVALID_ARG;   // a plan holds one slice's state
        if (cnn && !nets.insert(pl->cnn).second) return DGAMP_CT_ERR_INVALID_ARG;
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

// ===================================================================== //
// One launch per phase over all slices (dgamp_ct_batch_*).  The stream-pool
// path above replays one graph per slice, about seven launches per slice and
// iteration; a batch object instead runs each phase of an iteration as ONE
// launch over a work list that covers every slice -- the projector, the
// cluster sinogram step, the tile back-projection, the probe and the two TV
// launches -- so an iteration of a 64-slice batch is 6 launches, captured
// once as a graph.  Every block finds its slice in the phase's block ->
// slice table and runs the same block body as the single-slice kernel, so a
// slice's result is bit-identical to its own solve with the batch's
// implementation choices (pj_seg 16, tile back-projection, the cluster
// sinogram form, 10 TV steps per launch over 64-row regions).
#include "fft_device.cuh"
#include "output_device.cuh"

namespace dgct {

// Algorithm 1 initialisation of every slice: y = counts, x = 0, s_prev = 0,
// the staged images of x = 0 (zeros, guards included) and the scalars.
__global__ void __launch_bounds__(256) k_batch_begin(const BatchSlice* __restrict__ sl,
                                                     const uint16_t* __restrict__ map) {
    const BatchSlice& B = sl[map[blockIdx.x]];
    const long long e = (long long)((int)blockIdx.x - B.off[kPhBegin]) * blockDim.x + threadIdx.x;
    if (e < B.M) {
        B.y[e] = B.counts[e];
        reinterpret_cast<float*>(B.s)[e] = 0.f;   // zero bits: zero in either storage type
    }
    if (e < B.N) B.x[e] = 0.f;
    if (e < (long long)B.n * B.ldp) {
        reinterpret_cast<float*>(B.XR)[e] = 0.f;
        reinterpret_cast<float*>(B.XC)[e] = 0.f;
    }
    if (e == 0) {
        DevScalars s;
        memset(&s, 0, sizeof(s));
        s.tau_x = B.tau_x0;
        s.frob2 = B.frob2;
        s.logI0 = B.logI0;
        s.t = 1u;
        *B.S = s;
    }
}

// After the last iteration: each slice's pending divergence (one warp per slice).
__global__ void k_batch_finish(const BatchSlice* __restrict__ sl) {
    const BatchSlice& B = sl[blockIdx.x];
    pending_tau_x(B.S, B.partial_div, (double)B.N, B.tau_x_floor, B.log, true);
    __syncwarp();
    if (threadIdx.x == 0) B.S->div_pending = 0u;
}

// mu = V^-1 x of every slice, the three passes of the image filter (fft.cu):
// rows of x -> spectrum rows, columns with the gain, inverse rows -> mu.
__global__ void __launch_bounds__(512) k_batch_vinv_rows(const BatchSlice* __restrict__ sl,
                                                         const uint16_t* __restrict__ map) {
    extern __shared__ float2 smem[];
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int iy = (int)blockIdx.x - B.off[kPhRow], n = B.n, m = B.m2;
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        a[fpad(i)] = make_float2(i < n ? B.x[(size_t)iy * n + i] : 0.f, 0.f);
    __syncthreads();
    float2* r = fft_stockham(a, b, m, B.tw2, -1.f);
    for (int i = threadIdx.x; i < m; i += blockDim.x) B.fft2d[(size_t)iy * m + i] = r[fpad(i)];
}

__global__ void __launch_bounds__(512) k_batch_vinv_cols(const BatchSlice* __restrict__ sl,
                                                         const uint16_t* __restrict__ map) {
    extern __shared__ float2 smem[];
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int kx = (int)blockIdx.x - B.off[kPhCol], n = B.n, m = B.m2;
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    float2* C = B.fft2d;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        a[fpad(i)] = i < n ? C[(size_t)i * m + kx] : make_float2(0.f, 0.f);
    __syncthreads();
    float2* r = fft_stockham(a, b, m, B.tw2, -1.f);
    float2* o = (r == a) ? b : a;
    const float f0 = 1.0f / (2.0f * (float)B.P);
    const float fx = (float)(kx <= m / 2 ? kx : kx - m) / (float)m;
    for (int ky = threadIdx.x; ky < m; ky += blockDim.x) {
        const float fy = (float)(ky <= m / 2 ? ky : ky - m) / (float)m;
        const float g = sqrtf(fmaxf(sqrtf(fx * fx + fy * fy), f0));
        const float2 v = r[fpad(ky)];
        r[fpad(ky)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    r = fft_stockham(r, o, m, B.tw2, 1.f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) C[(size_t)i * m + kx] = r[fpad(i)];
}

__global__ void __launch_bounds__(512) k_batch_vinv_rows_inv(const BatchSlice* __restrict__ sl,
                                                             const uint16_t* __restrict__ map) {
    extern __shared__ float2 smem[];
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int iy = (int)blockIdx.x - B.off[kPhRow], n = B.n, m = B.m2;
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[fpad(i)] = B.fft2d[(size_t)iy * m + i];
    __syncthreads();
    float2* r = fft_stockham(a, b, m, B.tw2, 1.f);
    const float sc = 1.0f / ((float)m * (float)m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) B.mu_out[(size_t)iy * n + i] = r[fpad(i)].x * sc;
}

}  // namespace dgct

struct dgamp_ct_batch_s {
    int device = 0;
    std::vector<dgamp_ct_plan_t> plans;
    std::vector<BatchSlice> h;          // host copy of the descriptors
    BatchExec E;                        // the whole batch: begin, finish and V^-1 tables
    std::vector<BatchExec> grp;         // per group: the tables of the iteration's phases
    cudaGraphExec_t graph = nullptr;    // one iteration: 6 launches per group, groups on parallel branches
    cudaGraphExec_t graph_k = nullptr;  // kBatchGraphIters iterations, one after the other
    int tv_launches = 0;
};

namespace dgct {

static void batch_free(dgamp_ct_batch_s* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_k) cudaGraphExecDestroy(b->graph_k);
    if (b->E.sl) cudaFree(b->E.sl);
    for (int p = 0; p < kPhases; ++p)
        if (b->E.map[p]) cudaFree(b->E.map[p]);
    for (auto& g : b->grp)
        for (int p = 0; p < kPhases; ++p)
            if (g.map[p]) cudaFree(g.map[p]);
    b->graph = b->graph_k = nullptr;
    b->E = BatchExec{};
    b->grp.clear();
}

static int batch_vinv_threads(int m) { return m / 8 < 32 ? 32 : (m / 8 > 512 ? 512 : m / 8); }

// One iteration of every slice of a group: the six batched launches.
static int batch_iteration(dgamp_ct_batch_s* b, const BatchExec& E, cudaStream_t st) {
    DGCT_TRY(launch_project_batch(E, st));                         // Step 1: A x
    DGCT_TRY(launch_sino_batch(E, st));                            //         H A x, Step 2, H s
    DGCT_TRY(launch_backproject_batch(E, st));                     // Step 3: r = x + tau_r A^T H s
    DGCT_TRY(launch_probe_batch(E, st));                           // Step 4: r + eps b
    for (int i = 0; i < b->tv_launches; ++i)                       //         D(r), D(r + eps b), x, D'
        DGCT_TRY(launch_tv_batch(E, i, i == b->tv_launches - 1, st));
    return DGAMP_CT_OK;
}

// Iterations per launch of the longer batch graph.
constexpr int kBatchGraphIters = 5;

// The graph of `iters` iterations: in each, group k's six launches on branch
// k, forked from and joined back into the capture stream (one branch when
// there is one group).
static int batch_graph_iters(dgamp_ct_batch_s* b, int iters, cudaGraphExec_t* out) {
    const int G = (int)b->grp.size();
    std::vector<cudaStream_t> br(G, nullptr);
    std::vector<cudaEvent_t> ev(G + 1, nullptr);
    cudaStream_t cs;
    DGCT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < G && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking);
    for (int k = 0; k <= G && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    auto cleanup = [&]() {
        for (auto s_ : br)
            if (s_) cudaStreamDestroy(s_);
        for (auto v : ev)
            if (v) cudaEventDestroy(v);
        cudaStreamDestroy(cs);
    };
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e);
    }
    int rc = DGAMP_CT_OK;
    for (int it = 0; it < iters && rc == DGAMP_CT_OK; ++it) {
        if (G == 1) {
            rc = batch_iteration(b, b->grp[0], cs);
        } else {
            cudaError_t ce = cudaEventRecord(ev[G], cs);                              // fork
            for (int k = 0; k < G && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(br[k], ev[G], 0);
            if (ce != cudaSuccess) rc = cuda_fail(ce);
            for (int k = 0; k < G && rc == DGAMP_CT_OK; ++k) rc = batch_iteration(b, b->grp[k], br[k]);
            for (int k = 0; k < G; ++k) {                                              // join every branch
                ce = cudaEventRecord(ev[k], br[k]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, ev[k], 0);
                if (ce != cudaSuccess && rc == DGAMP_CT_OK) rc = cuda_fail(ce);
            }
        }
    }
    e = cudaStreamEndCapture(cs, &g);
    cleanup();
    if (rc != DGAMP_CT_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(e);
    }
    return DGAMP_CT_OK;
}

static int batch_graph(dgamp_ct_batch_s* b) {
    if (!b->graph) DGCT_TRY(batch_graph_iters(b, 1, &b->graph));
    if (!b->graph_k) DGCT_TRY(batch_graph_iters(b, kBatchGraphIters, &b->graph_k));
    return DGAMP_CT_OK;
}

}  // namespace dgct

extern "C" {

int dgamp_ct_batch_create(int32_t n, const dgamp_ct_plan_t* plans, int32_t groups, dgamp_ct_batch_t* out) {
    if (!out || n < 1 || n > 65535 || !plans || groups < 1) return DGAMP_CT_ERR_INVALID_ARG;
    *out = nullptr;
    int device = 0;
    DGCT_CUDA(cudaGetDevice(&device));
    std::set<dgamp_ct_plan_t> seen;
    const dgamp_ct_plan_s* p0 = plans[0];
    if (!p0) return DGAMP_CT_ERR_INVALID_ARG;
    int max_nd = 0;
    for (int32_t i = 0; i < n; ++i) {
        const dgamp_ct_plan_s* pl = plans[i];
        if (!pl || !seen.insert(plans[i]).second || pl->device != device) return DGAMP_CT_ERR_INVALID_ARG;
        const dgamp_ct_options& o = pl->opt;
        // the batched kernels: parallel beam, prox-TV (l2), Laplace's output step,
        // one storage type and one step count for all slices
        if (pl->fan || o.denoiser != 0 || o.tv_metric || o.output_moments) return DGAMP_CT_ERR_INVALID_ARG;
        if (o.storage != p0->opt.storage || o.k_tv != p0->opt.k_tv) return DGAMP_CT_ERR_INVALID_ARG;
        if (o.k_tv < kBatchTvKb || o.k_tv % kBatchTvKb != 0 || !(o.c_tv > 0)) return DGAMP_CT_ERR_INVALID_ARG;
        if (sino_ct_config(pl->nd, nullptr) == 0 || pl->nv > pl->max_partials) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
        max_nd = std::max(max_nd, pl->nd);
    }
    dgamp_ct_batch_s* b = new (std::nothrow) dgamp_ct_batch_s();
    if (!b) return DGAMP_CT_ERR_OOM;
    b->device = device;
    b->plans.assign(plans, plans + n);
    b->tv_launches = p0->opt.k_tv / kBatchTvKb;
    BatchExec& E = b->E;
    E.ns = n;
    E.bf = p0->opt.storage;
    E.R = sino_ct_config(max_nd, &E.cl);
    // descriptors and the block -> slice tables, largest slices first in
    // each grid (the work list order of the LPT scheduler); the iteration's
    // phases get one set of tables per group (slices split largest-first
    // over the groups), the once-per-solve phases one for the whole batch
    std::vector<int64_t> work(n);
    for (int32_t i = 0; i < n; ++i) work[i] = (int64_t)plans[i]->nv * plans[i]->nd * plans[i]->n;
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return work[a] > work[c]; });
    const int G = std::min<int32_t>(groups, n);
    std::vector<int32_t> group_of(n);
    if (dgamp_ct_schedule_lpt(n, work.data(), G, group_of.data(), nullptr) != DGAMP_CT_OK) {
        delete b;
        return DGAMP_CT_ERR_INVALID_ARG;
    }
    b->grp.resize(G);
    std::vector<int> gmax_nd(G, 0);
    b->h.resize(n);
    std::vector<std::vector<uint16_t>> maps(kPhases);
    std::vector<std::vector<std::vector<uint16_t>>> gmaps(G, std::vector<std::vector<uint16_t>>(kPhases));
    for (int32_t k = 0; k < n; ++k) {
        const int32_t i = order[k];
        const dgamp_ct_plan_s* pl = plans[i];
        const Workspace& w = pl->ws;
        BatchSlice& d = b->h[i];
        memset(&d, 0, sizeof(d));
        d.n = pl->n; d.nv = pl->nv; d.nd = pl->nd; d.ldp = pl->ldp; d.m2 = pl->m2; d.P = pl->P;
        d.N = pl->N; d.M = pl->M;
        d.XR = w.XR; d.XC = w.XC; d.zraw = w.zraw; d.s = w.s; d.hs = w.hs;
        d.x = w.x; d.r = w.r; d.b = w.b; d.y = w.y; d.p = w.p; d.fft2d = w.fft2d;
        d.partial = w.partial; d.partial_div = w.partial_div; d.S = w.S; d.log = w.log;
        d.vc = w.vc; d.hx = w.hx; d.tw2 = w.tw2;
        d.c_tv = (float)pl->opt.c_tv; d.eps_rel = (float)pl->opt.eps_rel;
        d.damp_x = (float)pl->opt.damp_x; d.damp_s = (float)pl->opt.damp_s;
        d.tau_x_floor = pl->opt.tau_x_floor; d.frob2 = pl->frob2; d.tau_x0 = pl->opt.tau_x0;
        d.onsager = pl->opt.onsager; d.truncate = pl->opt.truncate_z;
        d.key = make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
        d.slice_id = (unsigned)pl->opt.slice_id;
        const long long begin_elems = std::max<long long>(std::max<long long>(pl->M, pl->N), (long long)pl->n * pl->ldp);
        const int cnt[kPhases] = {batch_grid_project(pl->nv, pl->nd), pl->nv, batch_grid_backproject(pl->n),
                                  batch_grid_probe(pl->N), batch_grid_tv(pl->n, 0), batch_grid_tv(pl->n, 1),
                                  pl->n, pl->m2, (int)((begin_elems + 255) / 256)};
        const int gk = group_of[i];
        for (int ph = 0; ph < kPhases; ++ph) {
            auto& mp = (ph == kPhRow || ph == kPhCol || ph == kPhBegin) ? maps[ph] : gmaps[gk][ph];
            d.off[ph] = (int)mp.size();
            mp.insert(mp.end(), (size_t)cnt[ph], (uint16_t)i);
        }
        E.max_m2 = std::max(E.max_m2, pl->m2);
        gmax_nd[gk] = std::max(gmax_nd[gk], pl->nd);
    }
    for (int ph = 0; ph < kPhases; ++ph) E.nblk[ph] = (int)maps[ph].size();
    E.ct_smem = sino_ct_smem_bytes(max_nd, E.R, E.cl);
    int rc = DGAMP_CT_OK;
    cudaError_t e = cudaMalloc((void**)&E.sl, (size_t)n * sizeof(BatchSlice));
    auto upload = [&](uint16_t** dst, const std::vector<uint16_t>& v) {
        if (v.empty() || e != cudaSuccess) return;
        e = cudaMalloc((void**)dst, v.size() * sizeof(uint16_t));
        if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    };
    for (int ph : {kPhRow, kPhCol, kPhBegin}) upload(&E.map[ph], maps[ph]);
    for (int k = 0; k < G; ++k) {
        BatchExec& X = b->grp[k];
        X.ns = n;
        X.bf = E.bf;
        X.R = sino_ct_config(gmax_nd[k], &X.cl);
        X.ct_smem = sino_ct_smem_bytes(gmax_nd[k], X.R, X.cl);
        X.max_m2 = E.max_m2;
        for (int ph = 0; ph < kPhases; ++ph) {
            X.nblk[ph] = (int)gmaps[k][ph].size();
            if (ph != kPhRow && ph != kPhCol && ph != kPhBegin) upload(&X.map[ph], gmaps[k][ph]);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(E.sl, b->h.data(), (size_t)n * sizeof(BatchSlice), cudaMemcpyHostToDevice);
    for (auto& X : b->grp) X.sl = E.sl;
    if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? DGAMP_CT_ERR_OOM : cuda_fail(e);
    if (rc == DGAMP_CT_OK) {
        const int fsm = 2 * fft_buf_len(E.max_m2) * (int)sizeof(float2);
        const int lim = fsm > 48 * 1024 ? fsm : 48 * 1024;
        rc = raise_smem_limit((const void*)k_batch_vinv_rows, lim);
        if (rc == DGAMP_CT_OK) rc = raise_smem_limit((const void*)k_batch_vinv_cols, lim);
        if (rc == DGAMP_CT_OK) rc = raise_smem_limit((const void*)k_batch_vinv_rows_inv, lim);
    }
    if (rc == DGAMP_CT_OK) rc = batch_graph(b);
    if (rc != DGAMP_CT_OK) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return DGAMP_CT_OK;
}

void dgamp_ct_batch_destroy(dgamp_ct_batch_t b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

int64_t dgamp_ct_batch_launches(dgamp_ct_batch_t b, int32_t iters) {
    if (!b || iters < 0) return -1;
    // the begin kernel, per iteration and group the projector, sinogram step,
    // back-projection, probe and TV launches, then the finish and V^-1 (3)
    return 1 + (int64_t)iters * (int64_t)b->grp.size() * (4 + b->tv_launches) + 4;
}

int dgamp_ct_batch_solve(dgamp_ct_batch_t b, const float* const* d_counts, const double* I0, int32_t iters,
                         float* const* d_mu_out, dgamp_ct_stats* stats, void* stream) {
    if (!b || !d_counts || !I0 || !d_mu_out) return DGAMP_CT_ERR_INVALID_ARG;
    if (iters < 1 || iters > kMaxIters) return DGAMP_CT_ERR_INVALID_ARG;
    int device = 0;
    DGCT_CUDA(cudaGetDevice(&device));
    if (device != b->device) return DGAMP_CT_ERR_INVALID_ARG;
    const int n = b->E.ns;
    for (int i = 0; i < n; ++i) {
        if (!d_counts[i] || !d_mu_out[i] || !(I0[i] > 0) || !std::isfinite(I0[i])) return DGAMP_CT_ERR_INVALID_ARG;
        b->h[i].counts = d_counts[i];
        b->h[i].mu_out = d_mu_out[i];
        b->h[i].logI0 = std::log(I0[i]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const BatchExec& E = b->E;
    DGCT_CUDA(cudaMemcpyAsync(E.sl, b->h.data(), (size_t)n * sizeof(BatchSlice), cudaMemcpyHostToDevice, st));
    k_batch_begin<<<E.nblk[kPhBegin], 256, 0, st>>>(E.sl, E.map[kPhBegin]);
    DGCT_LAUNCH_CHECK();
    int t = 0;
    for (; t + kBatchGraphIters <= iters; t += kBatchGraphIters) DGCT_CUDA(cudaGraphLaunch(b->graph_k, st));
    for (; t < iters; ++t) DGCT_CUDA(cudaGraphLaunch(b->graph, st));
    k_batch_finish<<<n, 32, 0, st>>>(E.sl);
    DGCT_LAUNCH_CHECK();
    const int thr = batch_vinv_threads(E.max_m2);
    const size_t fsm = (size_t)2 * fft_buf_len(E.max_m2) * sizeof(float2);
    k_batch_vinv_rows<<<E.nblk[kPhRow], thr, fsm, st>>>(E.sl, E.map[kPhRow]);
    DGCT_LAUNCH_CHECK();
    k_batch_vinv_cols<<<E.nblk[kPhCol], thr, fsm, st>>>(E.sl, E.map[kPhCol]);
    DGCT_LAUNCH_CHECK();
    k_batch_vinv_rows_inv<<<E.nblk[kPhRow], thr, fsm, st>>>(E.sl, E.map[kPhRow]);
    DGCT_LAUNCH_CHECK();
    if (!stats) return DGAMP_CT_OK;
    DGCT_CUDA(cudaStreamSynchronize(st));
    int rc = DGAMP_CT_OK;
    for (int i = 0; i < n; ++i) {
        const int r = fill_stats(b->plans[i], iters, &stats[i]);
        if (r != DGAMP_CT_OK && rc == DGAMP_CT_OK) rc = r;
    }
    return rc;
}

}  // extern "C"
