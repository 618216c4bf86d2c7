// Host side of the C ABI declared in include/dgamp_ct.h: plan construction,
// the single-step entry points, and the D-GAMP-CT loop (Algorithm 1) with its
// per-iteration kernel sequence captured once into a CUDA graph.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_device.cuh"
#include "output_device.cuh"

namespace dgct {

static thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda = (int)e;
    return DGAMP_CT_ERR_CUDA;
}

static void free_ws(Workspace& w) {
    void* ptrs[] = {w.XR, w.XC, w.x, w.r, w.b, w.p, w.zraw, w.z, w.s, w.hs, w.y, w.fft2d, w.partial,
                    w.partial_div, w.S, w.log, w.vc, w.gain, w.tw, w.tw2, w.scratch_d, w.hx, w.zraw2,
                    w.fan_rays, w.fan_views, w.pj_order, w.pj_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    w = Workspace{};
}

template <typename T>
static int dalloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        *p = nullptr;
        return DGAMP_CT_ERR_OOM;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return DGAMP_CT_OK;
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static bool options_ok(const dgamp_ct_options* o) {
    if (o->denoiser < 0 || o->denoiser > 2) return false;
    if (o->k_tv < 0 || o->k_tv > 100000) return false;
    if (!std::isfinite(o->c_tv) || o->c_tv < 0) return false;
    if (!std::isfinite(o->eps_rel) || o->eps_rel <= 0) return false;
    if (!(o->damp_x > 0 && o->damp_x <= 1) || !(o->damp_s > 0 && o->damp_s <= 1)) return false;
    if (!(o->tau_x_floor >= 0) || !std::isfinite(o->tau_x_floor)) return false;
    if (!(o->tau_x0 > 0) || !std::isfinite(o->tau_x0)) return false;
    if (o->cnn_scale != 0 && o->cnn_scale != 1) return false;
    if (o->truncate_z != 0 && o->truncate_z != 1) return false;
    if (o->storage != 0 && o->storage != 1) return false;
    if (o->output_moments != 0 && o->output_moments != 1) return false;
    if (o->output_moments == 1 && o->truncate_z) return false;
    if (o->tv_metric != 0 && o->tv_metric != 1) return false;
    return true;
}

// Per-view Joseph constants (see ViewConst), computed in FP64 and rounded.
static void view_constants(int n, int nd, const std::vector<double>& ang, std::vector<ViewConst>& out) {
    const double c = 0.5 * (n - 1), cd = 0.5 * (nd - 1);
    out.resize(ang.size());
    for (size_t k = 0; k < ang.size(); ++k) {
        const double st = std::sin(ang[k]), ct = std::cos(ang[k]);
        ViewConst v{};
        if (std::fabs(st) >= std::fabs(ct)) {
            // fractional row at column s: c - (u_d - (s - c) cos)/sin, u_d = d - cd
            v.col = 1;
            v.a0 = (float)(c + cd / st - c * ct / st);
            v.a_step = (float)(ct / st);
            v.a_det = (float)(-1.0 / st);
            v.w = (float)(1.0 / std::fabs(st));
        } else {
            // fractional column at row s: (u_d - (c - s) sin)/cos + c
            v.col = 0;
            v.a0 = (float)(c - cd / ct - c * st / ct);
            v.a_step = (float)(st / ct);
            v.a_det = (float)(1.0 / ct);
            v.w = (float)(1.0 / std::fabs(ct));
        }
        // 32.32 fixed point from the FP64 values (not from the rounded floats)
        const double a0 = v.col ? (c + cd / st - c * ct / st) : (c - cd / ct - c * st / ct);
        const double as = v.col ? ct / st : st / ct;
        const double ad = v.col ? -1.0 / st : 1.0 / ct;
        const double q = 4294967296.0;
        v.inv_adet = (float)(1.0 / ad);
        v.inv_astep = as != 0.0 ? (float)(1.0 / as) : 0.f;
        v.P0 = (long long)std::llround(a0 * q);
        v.PSTEP = (long long)std::llround(as * q);
        v.PDET = (long long)std::llround(ad * q);
        v.AP = v.PDET > 0 ? v.PDET : -v.PDET;
        v.sg = v.PDET > 0 ? 1 : -1;
        out[k] = v;
    }
}

static int plan_alloc(dgamp_ct_plan_s* pl, const std::vector<double>& ang) {
    Workspace& w = pl->ws;
    const size_t N = (size_t)pl->N, M = (size_t)pl->M;
    const size_t img_staged = (size_t)pl->n * pl->ldp;
    DGCT_TRY(dalloc(&w.XR, img_staged));
    DGCT_TRY(dalloc(&w.XC, img_staged));
    DGCT_TRY(dalloc(&w.x, N));
    DGCT_TRY(dalloc(&w.r, 2 * N));
    DGCT_TRY(dalloc(&w.b, N));
    DGCT_TRY(dalloc(&w.p, 4 * N));
    DGCT_TRY(dalloc(&w.zraw, M));
    DGCT_TRY(dalloc(&w.z, M));
    DGCT_TRY(dalloc(&w.s, M));
    DGCT_TRY(dalloc(&w.hs, M));
    DGCT_TRY(dalloc(&w.y, M));
    DGCT_TRY(dalloc(&w.fft2d, (size_t)pl->m2 * pl->m2));
    const size_t tiles32 = (size_t)((pl->n + 31) / 32) * ((pl->n + 31) / 32);
    pl->max_partials = 1024;
    // blocks of the last blocked-TV launch, smallest tiles (43 x 11 pixels), two images
    const size_t tv_parts = 2 * (size_t)((pl->n + 42) / 43) * ((pl->n + 10) / 11);
    size_t nparts = tiles32 > (size_t)pl->max_partials ? tiles32 : (size_t)pl->max_partials;
    if (tv_parts > nparts) nparts = tv_parts;
    DGCT_TRY(dalloc(&w.partial, nparts));
    DGCT_TRY(dalloc(&w.partial_div, nparts));
    DGCT_TRY(dalloc(&w.S, 1));
    DGCT_TRY(dalloc(&w.log, (size_t)kMaxIters));
    DGCT_TRY(dalloc(&w.vc, (size_t)pl->nv));
    DGCT_TRY(dalloc(&w.gain, (size_t)pl->P));
    DGCT_TRY(dalloc(&w.tw, (size_t)fft_twiddle_count(pl->P) + 1));
    DGCT_TRY(dalloc(&w.tw2, (size_t)fft_twiddle_count(pl->m2) + 1));
    DGCT_TRY(dalloc(&w.hx, (size_t)2 * pl->nd));
    DGCT_TRY(dalloc(&w.zraw2, M));
    DGCT_TRY(dalloc(&w.scratch_d, (size_t)(pl->nd + 1) + 2 * pl->nd + pl->nv + (size_t)pl->nv * pl->nd));

    DGCT_CUDA(cudaMemset(w.XR, 0, img_staged * sizeof(float)));
    DGCT_CUDA(cudaMemset(w.XC, 0, img_staged * sizeof(float)));
    // blocked-TV steps per launch: timed on this geometry (uses the workspace
    // before the scalar block below is initialised)
    DGCT_TRY(tv_set_smem_limits());
    DGCT_TRY(tv_autotune(pl));
    {
        DevScalars s0;
        std::memset(&s0, 0, sizeof(s0));
        s0.tau_x = 1.0;
        s0.t = 1u;
        s0.logI0 = std::log(1e4);
        DGCT_CUDA(cudaMemcpy(w.S, &s0, sizeof(s0), cudaMemcpyHostToDevice));
    }

    std::vector<ViewConst> vc;
    view_constants(pl->n, pl->nd, ang, vc);
    DGCT_CUDA(cudaMemcpy(w.vc, vc.data(), vc.size() * sizeof(ViewConst), cudaMemcpyHostToDevice));
    // banded A: the views in orientation order, and its partial sums where a
    // band of 16 lines fits the shared memory the plan allows
    {
        std::vector<int> order;
        for (int pass = 0; pass < 2; ++pass)
            for (int v = 0; v < pl->nv; ++v)
                if (vc[v].col == pass) order.push_back(v);
        pl->pj_n0 = 0;
        for (int v = 0; v < pl->nv; ++v) pl->pj_n0 += vc[v].col == 0;
        DGCT_TRY(dalloc(&w.pj_order, (size_t)pl->nv));
        DGCT_CUDA(cudaMemcpy(w.pj_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
        const size_t nb16 = (size_t)((pl->n + 15) / 16), part = nb16 * M;
        if (16 * pl->ldp * (int)sizeof(float) <= 100 * 1024 && part * sizeof(float) <= ((size_t)512 << 20)) {
            DGCT_TRY(dalloc(&w.pj_part, part));
            DGCT_CUDA(cudaMemset(w.pj_part, 0, part * sizeof(float)));
        }
    }

    const int P = pl->P;
    std::vector<float> g(P);
    for (int k = 0; k < P; ++k) {
        const int kk = k <= P / 2 ? k : P - k;
        g[k] = (float)std::sqrt(std::fmax((double)kk / P, 1.0 / (2.0 * P)));
    }
    DGCT_CUDA(cudaMemcpy(w.gain, g.data(), P * sizeof(float), cudaMemcpyHostToDevice));
    const double two_pi = 6.283185307179586476925286766559;
    // the FFT's stage-by-stage twiddle table (fft_device.cuh), from FP64
    auto twiddles = [&](int L, float2* dst) -> int {
        std::vector<float2> t;
        for (int Ns = 1, R = fft_stage_radix(L, 1); R > 1; Ns *= R, R = fft_stage_radix(L, Ns)) {
            if (Ns == 1) continue;
            for (int r = 1; r < R; ++r)
                for (int k = 0; k < Ns; ++k) {
                    const double a = two_pi * (double)r * (double)k / ((double)Ns * R);
                    t.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
                }
        }
        if (t.empty()) return DGAMP_CT_OK;
        DGCT_CUDA(cudaMemcpy(dst, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice));
        return DGAMP_CT_OK;
    };
    DGCT_TRY(twiddles(P, w.tw));
    DGCT_TRY(twiddles(pl->m2, w.tw2));

    // ||Phi~||_F^2 on the device in FP64
    double* ang_dev = w.scratch_d + (pl->nd + 1) + 2 * pl->nd;
    DGCT_CUDA(cudaMemcpy(ang_dev, ang.data(), ang.size() * sizeof(double), cudaMemcpyHostToDevice));
    DGCT_TRY(launch_frobenius(pl));
    std::vector<double> terms((size_t)pl->nv * pl->nd);
    DGCT_CUDA(cudaMemcpy(terms.data(), ang_dev + pl->nv, terms.size() * sizeof(double),
                         cudaMemcpyDeviceToHost));
    double tot = 0.0;
    for (double v : terms) tot += v;
    pl->frob2 = tot;
    DGCT_CUDA(cudaMemcpy(&w.S->frob2, &tot, sizeof(double), cudaMemcpyHostToDevice));
    // H's kernel h[0..nd] (FP64, computed on the device above) -> hx for the Toeplitz form
    {
        const int nd = pl->nd;
        std::vector<double> h(nd + 1);
        DGCT_CUDA(cudaMemcpy(h.data(), w.scratch_d, (nd + 1) * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<float> hx(2 * nd - 1);
        for (int m = -(nd - 1); m <= nd - 1; ++m) hx[m + nd - 1] = (float)h[m < 0 ? -m : m];
        DGCT_CUDA(cudaMemcpy(w.hx, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    const int smem_need = 2 * fft_buf_len(P > pl->m2 ? P : pl->m2) * (int)sizeof(float2);
    DGCT_TRY(fft_set_smem_limits(smem_need > 48 * 1024 ? smem_need : 48 * 1024));
    DGCT_TRY(tvm_set_smem_limits(smem_need > 48 * 1024 ? smem_need : 48 * 1024));
    DGCT_TRY(toeplitz_set_smem_limit(pl->nd));
    DGCT_TRY(sino_step_set_smem_limit(pl));
    DGCT_TRY(filter_autotune(pl));
    DGCT_TRY(backproject_autotune(pl));
    DGCT_TRY(project_autotune(pl));
    DGCT_TRY(sino_autotune(pl));
    return DGAMP_CT_OK;
}

int raise_smem_limit(const void* kernel, int bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    DGCT_CUDA(cudaFuncGetAttributes(&fa, kernel));
    if (fa.maxDynamicSharedSizeBytes >= bytes) return DGAMP_CT_OK;
    DGCT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return DGAMP_CT_OK;
}

// -------------------------------------------------------------- solve ----
// The solve runs the fused sinogram kernel when the tuning asks for it and the
// output step is Laplace's (the exact moments take the three-kernel form,
// whose output-step kernel spreads the heavier per-measurement work over
// every SM).
static bool fused_sino_now(const dgamp_ct_plan_s* pl) { return pl->sino_fused && !pl->opt.output_moments; }

// denoiser 1 (the CNN) and 2 (the CNN judged by prox-TV) run the network
static bool uses_cnn(const dgamp_ct_plan_s* pl) { return pl->opt.denoiser == 1 || pl->opt.denoiser == 2; }

// One iteration of Algorithm 1 (Steps 1-4); every scalar it needs lives in
// DevScalars, so the same launch sequence serves every iteration.
// With `ev` non-NULL, ev[i] is recorded before kernel i and ev[count] after
// the last one (kernel-level timing on the launching stream).
static int enqueue_iteration(dgamp_ct_plan_s* pl, cudaStream_t st, cudaEvent_t* ev = nullptr) {
    Workspace& w = pl->ws;
    int k = 0;
    auto mark = [&]() -> int {
        if (ev) DGCT_CUDA(cudaEventRecord(ev[k], st));
        ++k;
        return DGAMP_CT_OK;
    };
    DGCT_TRY(mark());
    const int bf = pl->opt.storage;                                      // BF16 sinograms / staged image
    if (pl->fan) {
        // fan beam: Phi~ = A V^-1 with the image-domain filter, FP32 storage
        DGCT_TRY(launch_precond_image(pl, w.x, w.r, 1, st));             // Step 1: V^-1 x (3 kernels)
        DGCT_TRY(launch_stage_image(pl, w.r, st, 0));
        DGCT_TRY(launch_fan_project(pl, w.z, st));                       //         z = A V^-1 x
        DGCT_TRY(mark());
        DGCT_TRY(launch_output_step(pl, w.z, w.y, w.s, 1, 1, 0.0, 0.0, nullptr, st, 0));  // Step 2
        DGCT_TRY(mark());
        DGCT_TRY(launch_fan_backproject(pl, w.s, w.r, st));              // Step 3: A^T s
        DGCT_TRY(mark());
        DGCT_TRY(launch_precond_image_update(pl, w.r, w.x, w.r, st));    //         r = x + tau_r V^-1 A^T s
    } else {
    DGCT_TRY(launch_project(pl, w.zraw, st, bf, !project_sum_in_sino(pl)));   // Step 1: A x
    DGCT_TRY(mark());
    if (fused_sino_now(pl)) {
        DGCT_TRY(launch_sino_step(pl, st, bf));                         // H A x, Step 2, H s
        DGCT_TRY(mark());
    } else {
        DGCT_TRY(launch_filter(pl, w.zraw, w.z, st, bf));               //         H A x
        DGCT_TRY(mark());
        DGCT_TRY(launch_output_step(pl, w.z, w.y, w.s, 1, 1, 0.0, 0.0, nullptr, st, bf));  // Step 2
        DGCT_TRY(mark());
        DGCT_TRY(launch_filter(pl, w.s, w.hs, st, bf));                 // Step 3: H s
        DGCT_TRY(mark());
    }
    DGCT_TRY(launch_backproject(pl, w.hs, w.x, w.r, 1, st, bf,          //         r = x + tau_r A^T H s
                                fused_sino_now(pl) ? sino_step_partials(pl) : 0));
    }
    DGCT_TRY(mark());
    // Step 4: the probe b (learned denoiser) or r + eps b (prox-TV) beside r
    DGCT_TRY(launch_probe_input(pl, 0, st, uses_cnn(pl) ? 1 : 0));
    if (pl->opt.denoiser == 2) {
        // both denoisers on r, each with its divergence: the CNN and its
        // forward-mode derivative along b, then r + eps b beside r (the same
        // b) for prox-TV, written to dn[2] with its divergence in S; the lower
        // SURE risk estimate decides x, D' and tau_x
        const size_t N = (size_t)pl->N;
        DGCT_TRY(mark());
        DGCT_TRY(cnn_denoise_jvp(pl->cnn, w.r, w.S, pl->n, pl->dn, pl->opt.cnn_scale, st));
        DGCT_TRY(mark());
        DGCT_TRY(launch_probe_input(pl, 0, st, 0));
        const int ntv = tv_num_launches(pl, 1, 0.0);
        for (int i = 0; i < ntv; ++i) {
            DGCT_TRY(mark());
            DGCT_TRY(launch_tv_chunk(pl, 2, 1, 0.0, i, pl->dn + 2 * N, 0, 0, &w.S->div_plain, st));
        }
        DGCT_TRY(mark());
        DGCT_TRY(launch_select(pl, 0, st));
        DGCT_TRY(mark());
        DGCT_TRY(launch_select(pl, 1, st));
    } else if (pl->opt.denoiser == 1) {
        // learned denoiser: D(r) and its forward-mode derivative J_D(r) b, then x, D', tau_x
        DGCT_TRY(mark());
        DGCT_TRY(cnn_denoise_jvp(pl->cnn, w.r, w.S, pl->n, pl->dn, pl->opt.cnn_scale, st));
        DGCT_TRY(mark());
        DGCT_TRY(launch_denoise_final(pl, pl->dn, w.x, 1, 0, nullptr, st));
    } else {
        // D(r), D(r + eps b), x, D', tau_x: the blocked TV launches, the last one final
        const int ntv = tv_num_launches(pl, 1, 0.0);
        for (int i = 0; i < ntv; ++i) {
            DGCT_TRY(mark());
            DGCT_TRY(launch_tv_chunk(pl, 2, 1, 0.0, i, w.x, 1, 0, nullptr, st));
        }
    }
    DGCT_TRY(mark());
    return DGAMP_CT_OK;
}

// Steps 1-3 of one iteration: kernels and timed segments.  Parallel beam:
// A x, the sinogram step (1 or 3 kernels), the back-projection.  Fan beam:
// V^-1 x (3) with the staging and A (one segment), the output step, A^T,
// and V^-1 with the update (3, one segment).
static int front_kernels(const dgamp_ct_plan_s* pl) {
    if (pl->fan) return 10;
    return (fused_sino_now(pl) ? 1 : 3) + 2 + (pl->pj_band && !project_sum_in_sino(pl) ? 1 : 0);
}
static int front_segments(const dgamp_ct_plan_s* pl) {
    if (pl->fan) return 4;
    return (fused_sino_now(pl) ? 1 : 3) + 2;
}

// kernels one iteration launches: Steps 1-3, the probe, the denoiser
static int kernels_per_iteration(const dgamp_ct_plan_s* pl) {
    if (pl->opt.denoiser == 2 && pl->cnn)
        return front_kernels(pl) + 1 + cnn_launches_per_pair(pl->cnn) + 1 + tv_num_launches(pl, 1, 0.0) + 2;
    if (pl->opt.denoiser == 1 && pl->cnn) return front_kernels(pl) + 1 + cnn_launches_per_pair(pl->cnn) + 1;
    return front_kernels(pl) + 1 + tv_num_launches(pl, 1, 0.0);
}

// timed segments of one iteration (dgamp_ct_profile_iteration): as above,
// except that the learned denoiser's launches form one segment
static int segments_per_iteration(const dgamp_ct_plan_s* pl) {
    // denoiser 2: the probe, the CNN pair, the second probe, the TV launches, the two selection kernels
    if (pl->opt.denoiser == 2 && pl->cnn) return front_segments(pl) + 3 + tv_num_launches(pl, 1, 0.0) + 2;
    if (pl->opt.denoiser == 1 && pl->cnn) return front_segments(pl) + 3;
    return front_segments(pl) + 1 + tv_num_launches(pl, 1, 0.0);
}

static void drop_graph(dgamp_ct_plan_s* pl) {
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    if (pl->graph_k) cudaGraphExecDestroy(pl->graph_k);
    pl->graph = pl->graph_k = nullptr;
}

// Iterations per launch of the longer graph: consecutive iterations in one
// graph run back to back with no graph-launch boundary between them.
constexpr int kGraphIters = 5;

// k iterations captured as one graph into *out
static int capture_iterations(dgamp_ct_plan_s* pl, int k, cudaGraphExec_t* out) {
    cudaStream_t cs;
    DGCT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e);
    }
    int rc = DGAMP_CT_OK;
    for (int i = 0; i < k && rc == DGAMP_CT_OK; ++i) rc = enqueue_iteration(pl, cs);
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
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

// the one-iteration graph, and the kGraphIters one when `iters` can use it
static int ensure_graph(dgamp_ct_plan_s* pl, int iters) {
    if (!pl->graph) {
        DGCT_TRY(capture_iterations(pl, 1, &pl->graph));
        pl->graph_cnn_gen = pl->cnn ? cnn_ws_generation(pl->cnn) : 0;
    }
    if (iters >= kGraphIters && !pl->graph_k) DGCT_TRY(capture_iterations(pl, kGraphIters, &pl->graph_k));
    return DGAMP_CT_OK;
}

// `iters` iterations through the captured graphs
static int launch_graphs(dgamp_ct_plan_s* pl, int iters, cudaStream_t st) {
    DGCT_TRY(ensure_graph(pl, iters));
    int t = 0;
    for (; t + kGraphIters <= iters; t += kGraphIters) DGCT_CUDA(cudaGraphLaunch(pl->graph_k, st));
    for (; t < iters; ++t) DGCT_CUDA(cudaGraphLaunch(pl->graph, st));
    return DGAMP_CT_OK;
}

}  // namespace dgct

using namespace dgct;

extern "C" {

int dgamp_ct_default_options(dgamp_ct_options* o) {
    if (!o) return DGAMP_CT_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->denoiser = 0;
    o->k_tv = 20;
    o->c_tv = 3.0;
    o->eps_rel = 1e-3;
    o->seed = 12345;
    o->slice_id = 0;
    o->onsager = 1;
    o->damp_x = 1.0;
    o->damp_s = 1.0;
    o->tau_x_floor = 1e-6;
    o->use_graph = 1;
    o->cnn_scale = 0;
    o->tau_x0 = 1.0;
    o->truncate_z = 0;
    o->storage = 0;
    o->output_moments = 0;
    o->tv_metric = 0;
    return DGAMP_CT_OK;
}

int dgamp_ct_plan(const dgamp_ct_geometry* g, const dgamp_ct_options* opt, dgamp_ct_plan_t* out) {
    if (!g || !out) return DGAMP_CT_ERR_INVALID_ARG;
    *out = nullptr;
    if (g->n < 2 || g->n > DGAMP_CT_MAX_N || g->n_views < 1 || g->n_views > DGAMP_CT_MAX_VIEWS ||
        g->n_det < 2)
        return DGAMP_CT_ERR_INVALID_ARG;
    dgamp_ct_options o;
    if (opt) o = *opt; else dgamp_ct_default_options(&o);
    if (!options_ok(&o)) return DGAMP_CT_ERR_INVALID_ARG;
    const int P = 1 << ilog2(2 * g->n_det);
    if (P > DGAMP_CT_MAX_P) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    std::vector<double> ang(g->n_views);
    for (int k = 0; k < g->n_views; ++k) {
        ang[k] = g->angles ? g->angles[k] : (double)k * (3.14159265358979323846 / g->n_views);
        if (!std::isfinite(ang[k])) return DGAMP_CT_ERR_INVALID_ARG;
    }
    dgamp_ct_plan_s* pl = new (std::nothrow) dgamp_ct_plan_s();
    if (!pl) return DGAMP_CT_ERR_OOM;
    cudaGetDevice(&pl->device);
    pl->n = g->n;
    pl->nv = g->n_views;
    pl->nd = g->n_det;
    pl->P = P;
    pl->logP = ilog2(P);
    pl->m2 = 1 << ilog2(2 * g->n);
    pl->logm2 = ilog2(pl->m2);
    pl->ldp = ((g->n + 2 * kPad + 3) / 4) * 4;
    pl->N = (int64_t)g->n * g->n;
    pl->M = (int64_t)g->n_views * g->n_det;
    pl->opt = o;
    int rc = plan_alloc(pl, ang);
    if (rc != DGAMP_CT_OK) {
        free_ws(pl->ws);
        delete pl;
        return rc;
    }
    *out = pl;
    return DGAMP_CT_OK;
}

int dgamp_ct_plan_fan(const dgamp_ct_fan_geometry* g, const dgamp_ct_options* opt, dgamp_ct_plan_t* out) {
    if (!g || !out) return DGAMP_CT_ERR_INVALID_ARG;
    *out = nullptr;
    const dgamp_ct_geometry& b = g->base;
    if (b.n < 2 || b.n > DGAMP_CT_MAX_N || b.n_views < 1 || b.n_views > DGAMP_CT_MAX_VIEWS || b.n_det < 2)
        return DGAMP_CT_ERR_INVALID_ARG;
    // source and detector outside the image's circumscribed circle with a
    // margin of two pixels (the back-projector projects points one pixel
    // outside the image through the source), and not so far that the 32.32
    // positions overflow
    const double rmin = b.n / std::sqrt(2.0) + 2.0;
    if (!(g->src_dist > rmin && g->src_dist <= 1e8) || !(g->det_dist > rmin && g->det_dist <= 1e8) ||
        !(g->det_spacing > 0 && g->det_spacing <= 1e4))
        return DGAMP_CT_ERR_INVALID_ARG;
    std::vector<double> ang(b.n_views);
    for (int k = 0; k < b.n_views; ++k) {
        ang[k] = b.angles ? b.angles[k] : (double)k * (2.0 * 3.14159265358979323846 / b.n_views);
        if (!std::isfinite(ang[k])) return DGAMP_CT_ERR_INVALID_ARG;
    }
    // the parallel plan of the same sizes provides the workspace, the image
    // filter and the single-step entry points; the fan rays replace its views
    dgamp_ct_geometry pg = b;
    pg.angles = ang.data();
    dgamp_ct_plan_t pl = nullptr;
    int rc = dgamp_ct_plan(&pg, opt, &pl);
    if (rc != DGAMP_CT_OK) return rc;
    rc = fan_setup(pl, ang, g->src_dist, g->det_dist, g->det_spacing);
    if (rc != DGAMP_CT_OK) {
        dgamp_ct_plan_destroy(pl);
        return rc;
    }
    *out = pl;
    return DGAMP_CT_OK;
}

void dgamp_ct_plan_destroy(dgamp_ct_plan_t pl) {
    if (!pl) return;
    cudaDeviceSynchronize();
    drop_graph(pl);
    free_ws(pl->ws);
    if (pl->dn) cudaFree(pl->dn);
    delete pl;
}

int dgamp_ct_plan_set_cnn(dgamp_ct_plan_t pl, dgamp_ct_cnn_t net) {
    if (!pl) return DGAMP_CT_ERR_INVALID_ARG;
    drop_graph(pl);
    pl->cnn = net;
    if (!net) return DGAMP_CT_OK;
    if (!pl->dn) {
        // D(r) and J_D(r) b of the CNN, and prox-TV's D(r) when it judges the CNN (denoiser 2)
        cudaError_t e = cudaMalloc(&pl->dn, 3 * (size_t)pl->N * sizeof(float));
        if (e != cudaSuccess) {
            pl->dn = nullptr;
            pl->cnn = nullptr;
            if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return DGAMP_CT_ERR_OOM; }
            return cuda_fail(e);
        }
    }
    const int rc = cnn_prepare_pair(net, pl->n);
    if (rc != DGAMP_CT_OK) pl->cnn = nullptr;
    return rc;
}

int dgamp_ct_set_options(dgamp_ct_plan_t pl, const dgamp_ct_options* opt) {
    if (!pl || !opt || !options_ok(opt)) return DGAMP_CT_ERR_INVALID_ARG;
    pl->opt = *opt;
    drop_graph(pl);
    return DGAMP_CT_OK;
}

int dgamp_ct_plan_info(dgamp_ct_plan_t pl, double* frob_sq, int32_t* fft_len) {
    if (!pl) return DGAMP_CT_ERR_INVALID_ARG;
    if (frob_sq) *frob_sq = pl->frob2;
    if (fft_len) *fft_len = pl->P;
    return DGAMP_CT_OK;
}

int dgamp_ct_get_tuning(dgamp_ct_plan_t pl, dgamp_ct_tuning* out) {
    if (!pl || !out) return DGAMP_CT_ERR_INVALID_ARG;
    out->filter_mode = pl->filter_mode;
    out->tv_kb = pl->tv_kb;
    out->tv_rows = pl->tv_rows;
    out->sino_fused = pl->sino_fused;
    out->bp_mode = pl->bp_mode;
    out->pj_seg = pl->pj_seg;
    out->tv_vrows = pl->tv_vrows;
    out->pj_band = pl->pj_band;
    out->pj_waves = pl->pj_waves;
    return DGAMP_CT_OK;
}

int dgamp_ct_set_tuning(dgamp_ct_plan_t pl, const dgamp_ct_tuning* t) {
    if (!pl || !t || t->filter_mode > 1 || t->tv_kb > 10 || t->tv_kb == 0 || t->sino_fused > 2 || t->bp_mode > 1)
        return DGAMP_CT_ERR_INVALID_ARG;
    if (t->pj_seg >= 0 && t->pj_seg != 8 && t->pj_seg != 16 && t->pj_seg != 32) return DGAMP_CT_ERR_INVALID_ARG;
    if (t->tv_rows >= 0 && t->tv_rows != 32 && t->tv_rows != 64 && t->tv_rows != 128) return DGAMP_CT_ERR_INVALID_ARG;
    if (t->tv_vrows >= 0 && t->tv_vrows != 2 && t->tv_vrows != 4 && t->tv_vrows != 8) return DGAMP_CT_ERR_INVALID_ARG;
    if (t->pj_band >= 0 && t->pj_band != 0 && t->pj_band != 16 && t->pj_band != 32) return DGAMP_CT_ERR_INVALID_ARG;
    if (t->pj_waves >= 0 && t->pj_waves != 1 && t->pj_waves != 2) return DGAMP_CT_ERR_INVALID_ARG;
    if (t->pj_band > 0 && (pl->fan || !project_band_smem(pl, t->pj_band))) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    if (t->sino_fused == 1 && !sino_step_eligible(pl)) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    if (t->sino_fused == 2 && !sino_toeplitz_eligible(pl)) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    if (pl->fan && t->bp_mode == 1 && pl->fan_stride <= 0) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    if (t->filter_mode >= 0) pl->filter_mode = t->filter_mode;
    if (t->tv_kb > 0) pl->tv_kb = t->tv_kb;
    if (t->tv_rows > 0) pl->tv_rows = t->tv_rows;
    if (t->sino_fused >= 0) pl->sino_fused = t->sino_fused;
    if (t->bp_mode >= 0) pl->bp_mode = t->bp_mode;
    if (t->pj_seg > 0) pl->pj_seg = t->pj_seg;
    if (t->pj_seg > 0 && t->pj_band < 0) pl->pj_band = 0;     // a segment count picks the ray-group form
    if (t->pj_band >= 0) pl->pj_band = t->pj_band;
    if (t->pj_waves > 0) pl->pj_waves = t->pj_waves;
    if (int rc = project_band_chunks(pl)) return rc;       // checked above: fits
    if (t->tv_vrows > 0) pl->tv_vrows = t->tv_vrows;
    drop_graph(pl);
    return DGAMP_CT_OK;
}

int dgamp_ct_project(dgamp_ct_plan_t pl, const float* d_img, float* d_sino, int precond, void* stream) {
    if (!pl || !d_img || !d_sino) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (pl->fan) {   // Phi~ x = A (V^-1 x), V^-1 x in ws.r
        const float* src = d_img;
        if (precond) {
            DGCT_TRY(launch_precond_image(pl, d_img, pl->ws.r, 1, st));
            src = pl->ws.r;
        }
        DGCT_TRY(launch_stage_image(pl, src, st));
        return launch_fan_project(pl, d_sino, st);
    }
    DGCT_TRY(launch_stage_image(pl, d_img, st));
    if (!precond) return launch_project(pl, d_sino, st);
    DGCT_TRY(launch_project(pl, pl->ws.zraw, st));
    return launch_filter(pl, pl->ws.zraw, d_sino, st);
}

int dgamp_ct_backproject(dgamp_ct_plan_t pl, const float* d_sino, float* d_img, int precond, void* stream) {
    if (!pl || !d_sino || !d_img) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (pl->fan) {   // Phi~^T s = V^-1 (A^T s), A^T s in ws.r
        if (!precond) return launch_fan_backproject(pl, d_sino, d_img, st);
        DGCT_TRY(launch_fan_backproject(pl, d_sino, pl->ws.r, st));
        return launch_precond_image(pl, pl->ws.r, d_img, 1, st);
    }
    const float* src = d_sino;
    if (precond) {
        DGCT_TRY(launch_filter(pl, d_sino, pl->ws.hs, st));
        src = pl->ws.hs;
    }
    return launch_backproject(pl, src, nullptr, d_img, 0, st);
}

int dgamp_ct_filter(dgamp_ct_plan_t pl, const float* d_in, float* d_out, void* stream) {
    if (!pl || !d_in || !d_out) return DGAMP_CT_ERR_INVALID_ARG;
    if (pl->fan) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;   // H is the parallel-beam form of V^-1
    return launch_filter(pl, d_in, d_out, (cudaStream_t)stream);
}

int dgamp_ct_output_step(dgamp_ct_plan_t pl, const float* d_z, const float* d_y, const float* d_s_prev,
                         double I0, double tau_p, float* d_s, double* d_tau_s, void* stream) {
    if (!pl || !d_z || !d_y || !d_s || !d_tau_s) return DGAMP_CT_ERR_INVALID_ARG;
    if (!(I0 > 0) || !std::isfinite(I0) || !(tau_p > 0) || !std::isfinite(tau_p))
        return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int use_prev = 0;
    if (d_s_prev) {
        if (d_s_prev != d_s)
            DGCT_CUDA(cudaMemcpyAsync(d_s, d_s_prev, (size_t)pl->M * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st));
        use_prev = 1;
    }
    return launch_output_step(pl, d_z, d_y, d_s, use_prev, 0, tau_p, std::log(I0), d_tau_s, st);
}

int dgamp_ct_denoise_tv(dgamp_ct_plan_t pl, const float* d_r, double lambda, float* d_x, void* stream) {
    if (!pl || !d_r || !d_x || !(lambda >= 0) || !std::isfinite(lambda)) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    DGCT_CUDA(cudaMemcpyAsync(pl->ws.r, d_r, (size_t)pl->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return launch_tv(pl, 1, 0, lambda, d_x, 0, 0, nullptr, st);
}

int dgamp_ct_denoise_div(dgamp_ct_plan_t pl, const float* d_r, double tau_r, int32_t t, float* d_x,
                         double* d_div, void* stream) {
    if (!pl || !d_r || !d_x || !d_div || !(tau_r > 0) || !std::isfinite(tau_r) || t < 1)
        return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    DGCT_CUDA(cudaMemcpyAsync(pl->ws.r, d_r, (size_t)pl->N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    DGCT_TRY(launch_absmax(pl, pl->ws.r, st));
    DGCT_TRY(launch_probe_input(pl, t, st));
    const double lambda = pl->opt.c_tv * std::sqrt(tau_r);
    return launch_tv(pl, 2, 0, lambda, d_x, 0, t, d_div, st);
}

int dgamp_ct_probe(dgamp_ct_plan_t pl, int32_t t, int64_t n, float* d_b, uint32_t* d_words, void* stream) {
    if (!pl || n < 0 || (!d_b && !d_words)) return DGAMP_CT_ERR_INVALID_ARG;
    if (n == 0) return DGAMP_CT_OK;
    return launch_probe(pl, (unsigned)t, n, d_b, d_words, (cudaStream_t)stream);
}

int dgamp_ct_precond_image(dgamp_ct_plan_t pl, const float* d_in, float* d_out, int inverse, void* stream) {
    if (!pl || !d_in || !d_out) return DGAMP_CT_ERR_INVALID_ARG;
    return launch_precond_image(pl, d_in, d_out, inverse, (cudaStream_t)stream);
}

int dgamp_ct_profile_iteration(dgamp_ct_plan_t pl, int32_t reps, double* h_ms, int32_t cap,
                               int32_t* count, void* stream) {
    if (!pl || reps < 1 || !h_ms || !count) return DGAMP_CT_ERR_INVALID_ARG;
    if (uses_cnn(pl) && !pl->cnn) return DGAMP_CT_ERR_INVALID_ARG;
    const int nk = segments_per_iteration(pl);
    *count = nk;
    if (cap < nk) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(nk + 1, nullptr);
    for (auto& e : ev) DGCT_CUDA(cudaEventCreate(&e));
    std::vector<double> acc(nk, 0.0);
    int rc = DGAMP_CT_OK;
    for (int r = 0; r < reps && rc == DGAMP_CT_OK; ++r) {
        rc = enqueue_iteration(pl, st, ev.data());
        if (rc != DGAMP_CT_OK) break;
        cudaError_t e = cudaEventSynchronize(ev[nk]);
        if (e != cudaSuccess) { rc = cuda_fail(e); break; }
        for (int i = 0; i < nk; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            acc[i] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int i = 0; i < nk; ++i) h_ms[i] = acc[i] / reps;
    return rc;
}

int64_t dgamp_ct_solve_launches(dgamp_ct_plan_t pl, int32_t iters) {
    if (!pl || iters < 0) return -1;
    // per iteration, plus the image staging and scalar init before, and the
    // pending-divergence finish and the three V^-1 passes after
    return (int64_t)iters * kernels_per_iteration(pl) + 6;
}

}  // extern "C"

namespace dgct {

// After a solve's last iteration: the divergence its TV step left in partials
// (the next iteration's output step would have finished it).
__global__ void k_finish_pending(DevScalars* S, const double* partial_div, double N, double floor_rel,
                                 IterLog* log) {
    pending_tau_x(S, partial_div, N, floor_rel, log, true);
    __syncwarp();
    if (threadIdx.x == 0) S->div_pending = 0u;
}

static int solve_end(dgamp_ct_plan_s* pl, cudaStream_t st) {
    k_finish_pending<<<1, 32, 0, st>>>(pl->ws.S, pl->ws.partial_div, (double)pl->N, pl->opt.tau_x_floor, pl->ws.log);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

__global__ void k_init_scalars(DevScalars* S, double frob2, double logI0, double tau_x0) {
    DevScalars s;
    memset(&s, 0, sizeof(s));
    s.tau_x = tau_x0;              // Algorithm 1 initialisation (1 by default)
    s.frob2 = frob2;
    s.logI0 = logI0;
    s.t = 1u;
    *S = s;
}

// Algorithm 1 initialisation (x = 0, tau_x = tau_x0, s_prev = 0) and the counts.
static int solve_begin(dgamp_ct_plan_s* pl, const float* d_counts, double I0, cudaStream_t st) {
    Workspace& w = pl->ws;
    const size_t N = (size_t)pl->N, M = (size_t)pl->M;
    DGCT_CUDA(cudaMemcpyAsync(w.y, d_counts, M * sizeof(float), cudaMemcpyDeviceToDevice, st));
    DGCT_CUDA(cudaMemsetAsync(w.x, 0, N * sizeof(float), st));
    DGCT_CUDA(cudaMemsetAsync(w.s, 0, M * sizeof(float), st));
    DGCT_TRY(launch_stage_image(pl, w.x, st, pl->opt.storage));
    if (uses_cnn(pl)) {
        // the network may have been used (and its workspace regrown) since the
        // graph was captured: make room again and re-capture if it moved
        DGCT_TRY(cnn_prepare_pair(pl->cnn, pl->n));
        if ((pl->graph || pl->graph_k) && pl->graph_cnn_gen != cnn_ws_generation(pl->cnn)) drop_graph(pl);
    }
    k_init_scalars<<<1, 1, 0, st>>>(w.S, pl->frob2, std::log(I0), pl->opt.tau_x0);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct

extern "C" {

int dgamp_ct_solve_trace(dgamp_ct_plan_t pl, const float* d_counts, double I0, int32_t iters, float* d_mu_out,
                         float* d_r_trace, double* h_tau_r, void* stream) {
    if (!pl || !d_counts || !d_mu_out) return DGAMP_CT_ERR_INVALID_ARG;
    if (iters < 1 || iters > kMaxIters || !(I0 > 0) || !std::isfinite(I0)) return DGAMP_CT_ERR_INVALID_ARG;
    if (uses_cnn(pl) && !pl->cnn) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)pl->N;
    DGCT_TRY(solve_begin(pl, d_counts, I0, st));
    for (int t = 0; t < iters; ++t) {
        DGCT_TRY(enqueue_iteration(pl, st));
        if (d_r_trace)   // r^t: the denoiser input of iteration t+1 (ws.r image 0)
            DGCT_CUDA(cudaMemcpyAsync(d_r_trace + (size_t)t * N, pl->ws.r, N * sizeof(float),
                                      cudaMemcpyDeviceToDevice, st));
    }
    DGCT_TRY(solve_end(pl, st));
    DGCT_TRY(launch_precond_image(pl, pl->ws.x, d_mu_out, 1, st));
    if (h_tau_r) {
        std::vector<IterLog> lg(iters);
        DGCT_CUDA(cudaMemcpyAsync(lg.data(), pl->ws.log, iters * sizeof(IterLog), cudaMemcpyDeviceToHost, st));
        DGCT_CUDA(cudaStreamSynchronize(st));
        for (int t = 0; t < iters; ++t) h_tau_r[t] = lg[t].tau_r;
    }
    return DGAMP_CT_OK;
}

int dgamp_ct_solve(dgamp_ct_plan_t pl, const float* d_counts, double I0, int32_t iters, float* d_mu_out,
                   float* d_x_out, dgamp_ct_stats* stats, void* stream) {
    if (!pl || !d_counts || !d_mu_out) return DGAMP_CT_ERR_INVALID_ARG;
    if (iters < 1 || iters > kMaxIters || !(I0 > 0) || !std::isfinite(I0)) return DGAMP_CT_ERR_INVALID_ARG;
    if (uses_cnn(pl) && !pl->cnn) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace& w = pl->ws;
    const size_t N = (size_t)pl->N;
    DGCT_TRY(solve_begin(pl, d_counts, I0, st));
    if (pl->opt.use_graph) {
        DGCT_TRY(launch_graphs(pl, iters, st));
    } else {
        for (int t = 0; t < iters; ++t) DGCT_TRY(enqueue_iteration(pl, st));
    }
    DGCT_TRY(solve_end(pl, st));
    DGCT_TRY(launch_precond_image(pl, w.x, d_mu_out, 1, st));           // mu = V^-1 x
    if (d_x_out) DGCT_CUDA(cudaMemcpyAsync(d_x_out, w.x, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (!stats) return DGAMP_CT_OK;
    DGCT_CUDA(cudaStreamSynchronize(st));
    return fill_stats(pl, iters, stats);
}

}  // extern "C"

namespace dgct {

// Per-iteration log and counters of the plan's last solve (the solve's work
// must be complete).
int fill_stats(const dgamp_ct_plan_s* pl, int iters, dgamp_ct_stats* stats) {
    const Workspace& w = pl->ws;
    DevScalars hs;
    DGCT_CUDA(cudaMemcpy(&hs, w.S, sizeof(hs), cudaMemcpyDeviceToHost));
    std::vector<IterLog> lg(iters);
    DGCT_CUDA(cudaMemcpy(lg.data(), w.log, iters * sizeof(IterLog), cudaMemcpyDeviceToHost));
    for (int t = 0; t < iters; ++t) {
        if (stats->tau_x) stats->tau_x[t] = lg[t].tau_x;
        if (stats->tau_p) stats->tau_p[t] = lg[t].tau_p;
        if (stats->tau_s) stats->tau_s[t] = lg[t].tau_s;
        if (stats->tau_r) stats->tau_r[t] = lg[t].tau_r;
        if (stats->div) stats->div[t] = lg[t].div;
        const bool judged = pl->opt.denoiser == 2;
        if (stats->risk_plain) stats->risk_plain[t] = judged ? lg[t].risk_plain : NAN;
        if (stats->risk_learned) stats->risk_learned[t] = judged ? lg[t].risk_learned : NAN;
        if (stats->kept_learned) stats->kept_learned[t] = judged ? lg[t].keep_learned : 0;
    }
    stats->learned_kept = (int32_t)hs.learned_kept;
    stats->iters_done = (int32_t)(hs.t - 1u);
    stats->newton_capped = (int32_t)hs.newton_capped;
    stats->tau_x_floored = (int32_t)hs.floored;
    // a tensor-core convolution of the learned denoiser whose bounded wait ran out
    if (uses_cnn(pl) && pl->cnn) DGCT_TRY(cnn_take_timeout(pl->cnn));
    if (hs.nonfinite) return DGAMP_CT_ERR_NONFINITE;
    return DGAMP_CT_OK;
}

}  // namespace dgct

extern "C" {

int dgamp_ct_solve_host(dgamp_ct_plan_t pl, const float* h_counts, double I0, int32_t iters, float* h_mu_out,
                        dgamp_ct_stats* stats, void* stream) {
    if (!pl || !h_counts || !h_mu_out) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)pl->N, M = (size_t)pl->M;
    // counts land in the hs buffer (free until the first filter of s), mu in r
    DGCT_CUDA(cudaMemcpyAsync(pl->ws.hs, h_counts, M * sizeof(float), cudaMemcpyHostToDevice, st));
    int rc = dgamp_ct_solve(pl, pl->ws.hs, I0, iters, pl->ws.r, nullptr, stats, stream);
    if (rc != DGAMP_CT_OK && rc != DGAMP_CT_ERR_NONFINITE) return rc;
    DGCT_CUDA(cudaMemcpyAsync(h_mu_out, pl->ws.r, N * sizeof(float), cudaMemcpyDeviceToHost, st));
    DGCT_CUDA(cudaStreamSynchronize(st));
    if (!stats && uses_cnn(pl) && pl->cnn) DGCT_TRY(cnn_take_timeout(pl->cnn));
    return rc;
}

const char* dgamp_ct_strerror(int code) {
    switch (code) {
        case DGAMP_CT_OK: return "ok";
        case DGAMP_CT_ERR_INVALID_ARG: return "invalid argument";
        case DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY: return "unsupported geometry";
        case DGAMP_CT_ERR_OOM: return "out of device memory";
        case DGAMP_CT_ERR_CUDA: return "CUDA error (see dgamp_ct_last_cuda_error)";
        case DGAMP_CT_ERR_TIMEOUT: return "device wait timed out";
        case DGAMP_CT_ERR_NONFINITE: return "non-finite scalar in the iteration";
        default: return "unknown error";
    }
}

int dgamp_ct_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
