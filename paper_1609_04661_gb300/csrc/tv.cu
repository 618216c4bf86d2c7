// Denoiser and divergence, Algorithm 1 Step 4 (Section 4.3, Section 6.3).
//
// D is the l2 proximal map of isotropic TV, solved by Chambolle's 2004 dual
// projection (forward differences, Neumann boundary, step 1/8, a fixed
// number of iterations from a zero dual).  The MC divergence of Eq. MC_SURE
// with one probe needs D at r and at r + eps b; both images are denoised by
// the same blocks, and the last launch forms x = D(r), b^T (D(r+eps b) - D(r))
// in FP64 and -- inside a solve -- tau_x = max(tau_r D', floor tau_r).
//
// Temporal blocking.  One Chambolle step updates p at a pixel from p within
// one pixel of it:
//   q = div p - r/lambda,  div p = px(i,j) - px(i,j-1) + py(i,j) - py(i-1,j)
//   p <- (p + tau grad q) / (1 + tau |grad q|),  grad q uses q(i,j+1), q(i+1,j)
// so a block that holds a 32 x 32 tile plus a halo of H = KB + 1 pixels in
// shared memory runs KB steps with no global traffic (the valid region
// shrinks by one pixel per side per step) and can still form div p on its
// tile for the final x = r - lambda div p.  Duals outside the image stay
// zero, and grad q is zero on the last row/column (Neumann), which
// reproduces the boundary rules exactly.  Successive launches exchange the
// tile's duals through ping-pong global buffers [image][n][n] of float2.
// KB is a template parameter chosen per plan by timing (tv_autotune).
#include <vector>

#include "internal.cuh"

namespace dgct {

constexpr int TB = 32;             // interior tile edge
constexpr int kTvThreads = 1024;
constexpr int kTvMaxKb = 10;       // most Chambolle steps one launch may run
constexpr float kTau = 0.125f;

__device__ __forceinline__ float solve_lambda(const DevScalars* S, float c_tv, int from_scalars,
                                              float lambda_arg) {
    return from_scalars ? c_tv * sqrtf((float)S->tau_r) : lambda_arg;
}

// --------------------------------------------------------- probe input ----
// r2 = r + eps b, eps = eps_rel max(max|r|, 1e-6), or r2 = b itself
// (write_b = 1: the direction of a forward-mode divergence).  One thread per
// block of four probe elements (one Philox call).
__global__ void k_probe_input(const float* __restrict__ r, float* __restrict__ r2, long long N,
                              float eps_rel, int t_arg, unsigned slice, uint2 key,
                              DevScalars* S, int write_b) {
    const float rmax = __uint_as_float(S->rmax_bits);
    const float eps = eps_rel * fmaxf(rmax, 1e-6f);
    const unsigned t = t_arg > 0 ? (unsigned)t_arg : S->t;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) S->eps = (double)eps;
    const long long i0 = 4 * g;
    if (i0 >= N) return;
    const float4 b = probe4((unsigned)g, t, slice, key);
    const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < N) r2[i0 + k] = write_b ? bb[k] : fmaf(eps, bb[k], r[i0 + k]);
}

static uint2 probe_key(const dgamp_ct_plan_s* pl) {
    return make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
}

int launch_probe_input(const dgamp_ct_plan_s* pl, int t_arg, cudaStream_t st, int write_b) {
    const long long N = pl->N;
    const long long groups = (N + 3) / 4;
    k_probe_input<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(
        pl->ws.r, pl->ws.r + N, N, (float)pl->opt.eps_rel, t_arg, (unsigned)pl->opt.slice_id,
        probe_key(pl), pl->ws.S, write_b);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// max |r| into S->rmax_bits (standalone divergence call; inside a solve the
// back-projection produces it).
__global__ void k_absmax(const float* __restrict__ r, long long N, DevScalars* S) {
    unsigned m = 0u;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(r[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&S->rmax_bits, m);
}

int launch_absmax(const dgamp_ct_plan_s* pl, const float* r, cudaStream_t st) {
    DGCT_CUDA(cudaMemsetAsync(&pl->ws.S->rmax_bits, 0, sizeof(unsigned), st));
    k_absmax<<<256, 256, 0, st>>>(r, pl->N, pl->ws.S);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// --------------------------------------------------- blocked Chambolle ----
struct TvFinal {
    float* x_out;          // D(r) (with damping against the old x in a solve)
    float* XR;             // staged copies for the next projection (nullable)
    float* XC;
    int ldp;
    float damp_x;
    int t_arg;             // probe iteration (0: from S)
    unsigned slice;
    uint2 key;
    double tau_x_floor;
    double* partial;
    IterLog* log;
    double* div_out;       // nullable
    int solve_mode;        // 1: update tau_x, the log and t in S
    int jvp;               // learned denoiser: dn[1] is J_D b (divergence b^T J_D b / N)
};

// KB Chambolle steps on the block's region in shared memory.  BORDER = false
// is the fast path for blocks whose whole region lies inside the image and
// away from its last row/column, where no boundary rule applies.
template <int NIMG, int KB, bool BORDER>
__device__ __forceinline__ void tv_steps(float* __restrict__ spx, float* __restrict__ spy,
                                         float* __restrict__ sq, const float* __restrict__ sr, int n,
                                         int gi0, int gj0, float inv_lam) {
    constexpr int H = KB + 1, R = TB + 2 * H, RR = R * R;
    const int tid = threadIdx.x;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int lo = k + 1;
        const int W = R - 2 * k - 1;            // a constant once the loop is unrolled
        // q on rows/cols [k+1, R-k)
#pragma unroll
        for (int im = 0; im < NIMG; ++im) {
            for (int e = tid; e < W * W; e += kTvThreads) {
                const int a = lo + e / W, b = lo + (e - (e / W) * W);
                const int idx = im * RR + a * R + b;
                float q = (spx[idx] - spx[idx - 1] + spy[idx] - spy[idx - R]) - sr[idx] * inv_lam;
                if (BORDER) {
                    const int gi = gi0 + a, gj = gj0 + b;
                    if (!(gi >= 0 && gi < n && gj >= 0 && gj < n)) q = 0.f;
                }
                sq[idx] = q;
            }
        }
        __syncthreads();
        // p on rows/cols [k+1, R-k-1)
        const int W2 = W - 1;
#pragma unroll
        for (int im = 0; im < NIMG; ++im) {
            for (int e = tid; e < W2 * W2; e += kTvThreads) {
                const int a = lo + e / W2, b = lo + (e - (e / W2) * W2);
                const int idx = im * RR + a * R + b;
                const float qc = sq[idx];
                float gx = sq[idx + 1] - qc;
                float gy = sq[idx + R] - qc;
                if (BORDER) {
                    const int gi = gi0 + a, gj = gj0 + b;
                    if (gi < 0 || gi >= n || gj < 0 || gj >= n) continue;
                    if (gj >= n - 1) gx = 0.f;
                    if (gi >= n - 1) gy = 0.f;
                }
                const float g2 = fmaf(gx, gx, gy * gy);
                const float nrm = g2 > 0.f ? g2 * rsqrtf(g2) : 0.f;
                const float inv = __frcp_rn(fmaf(kTau, nrm, 1.f));
                spx[idx] = fmaf(kTau, gx, spx[idx]) * inv;
                spy[idx] = fmaf(kTau, gy, spy[idx]) * inv;
            }
        }
        __syncthreads();
    }
}

template <int NIMG, int KB>
__global__ void __launch_bounds__(kTvThreads)
k_tv_block(const float* __restrict__ rbase, const float2* __restrict__ pin, float2* __restrict__ pout,
           int n, int first, int final_step, float c_tv, int from_scalars, float lambda_arg,
           DevScalars* S, TvFinal F) {
    constexpr int H = KB + 1, R = TB + 2 * H, RR = R * R;
    extern __shared__ float sm[];
    float* __restrict__ spx = sm;
    float* __restrict__ spy = sm + NIMG * RR;
    float* __restrict__ sq = sm + 2 * NIMG * RR;
    float* __restrict__ sr = sm + 3 * NIMG * RR;
    const size_t N = (size_t)n * n;
    const int gi0 = blockIdx.y * TB - H, gj0 = blockIdx.x * TB - H;
    const int tid = threadIdx.x;
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const float inv_lam = lam > 0.f ? 1.0f / lam : 0.f;

    for (int e = tid; e < NIMG * RR; e += kTvThreads) {
        const int im = e / RR, c = e - im * RR;
        const int a = c / R, b = c - a * R;
        const int gi = gi0 + a, gj = gj0 + b;
        const bool in = gi >= 0 && gi < n && gj >= 0 && gj < n;
        const size_t o = im * N + (size_t)gi * n + gj;
        sr[e] = in ? rbase[o] : 0.f;
        float2 p = make_float2(0.f, 0.f);
        if (in && !first) p = pin[o];
        spx[e] = p.x;
        spy[e] = p.y;
    }
    __syncthreads();

    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + R < n && gj0 + R < n;
    if (interior)
        tv_steps<NIMG, KB, false>(spx, spy, sq, sr, n, gi0, gj0, inv_lam);
    else
        tv_steps<NIMG, KB, true>(spx, spy, sq, sr, n, gi0, gj0, inv_lam);

    if (!final_step) {
        for (int e = tid; e < NIMG * TB * TB; e += kTvThreads) {
            const int im = e / (TB * TB), c = e - im * (TB * TB);
            const int a = H + c / TB, b = H + (c & (TB - 1));
            const int gi = gi0 + a, gj = gj0 + b;
            if (gi >= n || gj >= n) continue;
            const int idx = im * RR + a * R + b;
            pout[im * N + (size_t)gi * n + gj] = make_float2(spx[idx], spy[idx]);
        }
        return;
    }

    // ---- final: x = r - lambda div p on the tile, staging, divergence ----
    __shared__ double red[32];
    __shared__ bool am_last;
    const unsigned t = F.t_arg > 0 ? (unsigned)F.t_arg : S->t;
    double acc = 0.0;
    float* tile = sq;                  // [TB][TB+1] staging tile for the transposed copy
    {
        const int ta = tid >> 5, tb = tid & 31;     // one tile pixel per thread
        const int a = H + ta, b = H + tb;
        const int gi = gi0 + a, gj = gj0 + b;
        float xv = 0.f;
        if (gi < n && gj < n) {
            float xs[NIMG];
#pragma unroll
            for (int im = 0; im < NIMG; ++im) {
                const int idx = im * RR + a * R + b;
                const float dv = spx[idx] - spx[idx - 1] + spy[idx] - spy[idx - R];
                xs[im] = sr[idx] - lam * dv;
            }
            const size_t o = (size_t)gi * n + gj;
            xv = xs[0];
            if (NIMG == 2) {
                const float4 b4 = probe4((unsigned)(o >> 2), t, F.slice, F.key);
                const int kk = (int)(o & 3);
                const float bv = kk == 0 ? b4.x : (kk == 1 ? b4.y : (kk == 2 ? b4.z : b4.w));
                acc += (double)bv * (double)(xs[NIMG - 1] - xs[0]);
            }
            if (F.solve_mode && F.damp_x != 1.f) xv = F.damp_x * xv + (1.f - F.damp_x) * F.x_out[o];
            F.x_out[o] = xv;
            if (F.XR) F.XR[(size_t)gi * F.ldp + kPad + gj] = xv;
        }
        tile[ta * (TB + 1) + tb] = xv;
    }
    if (F.XC) {
        __syncthreads();
        const int ta = tid >> 5, tb = tid & 31;     // ta: tile column, tb: tile row
        const int gj = gj0 + H + ta, gi = gi0 + H + tb;
        if (gi < n && gj < n) F.XC[(size_t)gj * F.ldp + kPad + gi] = tile[tb * (TB + 1) + ta];
    }
    if (NIMG < 2) return;
    acc = block_sum(acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) {
        F.partial[bid] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_div, 1u);
        am_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double tot = 0.0;
    for (int b = tid; b < nblk; b += kTvThreads) tot += ((volatile double*)F.partial)[b];
    tot = block_sum(tot, red);
    if (tid == 0) {
        const double div = tot / ((double)N * S->eps);
        if (F.div_out) *F.div_out = div;
        if (F.solve_mode) {
            const double tau_r = S->tau_r;
            double tx = tau_r * div;
            const double fl = F.tau_x_floor * tau_r;
            if (!(tx >= fl)) { tx = fl; S->floored += 1u; }
            if (!isfinite(tx)) S->nonfinite += 1u;
            S->div = div;
            S->tau_x = tx;
            const unsigned tt = S->t;
            if (tt >= 1u && tt <= (unsigned)kMaxIters) {
                IterLog L;
                L.tau_x = tx; L.tau_p = S->tau_p; L.tau_s = S->tau_s; L.tau_r = tau_r;
                L.div = div; L.eps = S->eps;
                F.log[tt - 1] = L;
            }
            S->t = tt + 1u;
        }
        S->done_div = 0u;
    }
}

// Steps per launch the autotuner may choose.
static const int kTvKbChoices[] = {3, 4, 5, 6, 8, 10};

bool tv_active(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (pl->opt.k_tv <= 0) return false;
    return from_scalars ? pl->opt.c_tv > 0.0 : lambda_arg > 0.0;
}

int tv_num_launches(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (!tv_active(pl, from_scalars, lambda_arg)) return 1;
    return (pl->opt.k_tv + pl->tv_kb - 1) / pl->tv_kb;
}

static constexpr size_t tv_smem_bytes(int nimg, int kb) {
    const int R = TB + 2 * (kb + 1);
    return (size_t)4 * nimg * R * R * sizeof(float);
}

template <int NIMG, int KB>
static void launch_kb(dim3 grd, cudaStream_t st, const float* r, const float2* pin, float2* pout, int n,
                      int first, int fin, float c_tv, int fs, float lam, DevScalars* S, const TvFinal& F) {
    k_tv_block<NIMG, KB><<<grd, kTvThreads, tv_smem_bytes(NIMG, KB), st>>>(r, pin, pout, n, first, fin, c_tv,
                                                                           fs, lam, S, F);
}

// One launch running exactly `steps` Chambolle steps (0..kTvMaxKb).
template <int NIMG>
static int launch_dispatch(int steps, dim3 grd, cudaStream_t st, const float* r, const float2* pin,
                           float2* pout, int n, int first, int fin, float c_tv, int fs, float lam,
                           DevScalars* S, const TvFinal& F) {
#define DGCT_TV_CASE(KB) \
    case KB: launch_kb<NIMG, KB>(grd, st, r, pin, pout, n, first, fin, c_tv, fs, lam, S, F); break;
    switch (steps) {
        DGCT_TV_CASE(0) DGCT_TV_CASE(1) DGCT_TV_CASE(2) DGCT_TV_CASE(3) DGCT_TV_CASE(4) DGCT_TV_CASE(5)
        DGCT_TV_CASE(6) DGCT_TV_CASE(7) DGCT_TV_CASE(8) DGCT_TV_CASE(9) DGCT_TV_CASE(10)
        default: return DGAMP_CT_ERR_INVALID_ARG;
    }
#undef DGCT_TV_CASE
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// Launch i (0-based) of the blocked denoiser on nimg images of ws.r; the last
// launch (i = tv_num_launches - 1) performs the final step.
int launch_tv_chunk(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                    float* x_out, int solve_mode, int t_arg, double* div_out, cudaStream_t st) {
    const int n = pl->n;
    const size_t N = (size_t)pl->N;
    const int KB = pl->tv_kb;
    const bool active = tv_active(pl, from_scalars, lambda_arg);
    const int nl = tv_num_launches(pl, from_scalars, lambda_arg);
    const int K = active ? pl->opt.k_tv : 0;
    const int iters = active ? ((i + 1) * KB <= K ? KB : K - i * KB) : 0;
    float2* buf[2] = {pl->ws.p, pl->ws.p + 2 * N};
    const float2* pin = buf[(i + 1) & 1];
    float2* pout = buf[i & 1];
    TvFinal F;
    F.x_out = x_out;
    F.XR = solve_mode ? pl->ws.XR : nullptr;
    F.XC = solve_mode ? pl->ws.XC : nullptr;
    F.ldp = pl->ldp;
    F.damp_x = (float)pl->opt.damp_x;
    F.t_arg = t_arg;
    F.slice = (unsigned)pl->opt.slice_id;
    F.key = probe_key(pl);
    F.tau_x_floor = pl->opt.tau_x_floor;
    F.partial = pl->ws.partial;
    F.log = pl->ws.log;
    F.div_out = div_out;
    F.solve_mode = solve_mode;
    F.jvp = 0;
    dim3 grd((n + TB - 1) / TB, (n + TB - 1) / TB);
    const float c_tv = (float)pl->opt.c_tv, lam = (float)lambda_arg;
    if (nimg == 2)
        return launch_dispatch<2>(iters, grd, st, pl->ws.r, pin, pout, n, i == 0, i == nl - 1, c_tv,
                                  from_scalars, lam, pl->ws.S, F);
    return launch_dispatch<1>(iters, grd, st, pl->ws.r, pin, pout, n, i == 0, i == nl - 1, c_tv,
                              from_scalars, lam, pl->ws.S, F);
}

// The whole denoiser (and, for nimg = 2, the divergence): tv_num_launches launches.
int launch_tv(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, float* x_out,
              int solve_mode, int t_arg, double* div_out, cudaStream_t st) {
    const int nl = tv_num_launches(pl, from_scalars, lambda_arg);
    for (int i = 0; i < nl; ++i) {
        const int rc = launch_tv_chunk(pl, nimg, from_scalars, lambda_arg, i, x_out, solve_mode, t_arg,
                                       div_out, st);
        if (rc != DGAMP_CT_OK) return rc;
    }
    return DGAMP_CT_OK;
}

template <int NIMG, int KB>
static int set_attr_range() {
    DGCT_CUDA(cudaFuncSetAttribute(k_tv_block<NIMG, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tv_smem_bytes(NIMG, KB)));
    if constexpr (KB > 0) return set_attr_range<NIMG, KB - 1>();
    return DGAMP_CT_OK;
}

int tv_set_smem_limits() {
    const int rc = set_attr_range<1, kTvMaxKb>();
    return rc != DGAMP_CT_OK ? rc : set_attr_range<2, kTvMaxKb>();
}

// Plan-time choice of the steps per launch: time the two-image denoiser of
// the plan's geometry (K = opt.k_tv) for every choice and keep the fastest.
// Runs on zeroed workspace; the timing does not depend on the values.
int tv_autotune(dgamp_ct_plan_s* pl) {
    if (pl->opt.k_tv <= 0) return DGAMP_CT_OK;
    const size_t N = (size_t)pl->N;
    DGCT_CUDA(cudaMemset(pl->ws.r, 0, 2 * N * sizeof(float)));
    DGCT_CUDA(cudaMemset(pl->ws.S, 0, sizeof(DevScalars)));
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_kb = pl->tv_kb;
    for (int kb : kTvKbChoices) {
        pl->tv_kb = kb;
        int rc = DGAMP_CT_OK;
        for (int rep = 0; rep < 4 && rc == DGAMP_CT_OK; ++rep) {      // first rep warms up
            if (rep == 1) cudaEventRecord(e0, 0);
            rc = launch_tv(pl, 2, 0, 1.0, pl->ws.x, 0, 1, nullptr, 0);
        }
        cudaEventRecord(e1, 0);
        cudaError_t e = cudaEventSynchronize(e1);
        if (rc != DGAMP_CT_OK || e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc != DGAMP_CT_OK ? rc : cuda_fail(e);
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_kb = kb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->tv_kb = best_kb;
    return DGAMP_CT_OK;
}

// ------------------------------------- final step for a learned denoiser --
// x = D(r) (damped in a solve), staged copies, the divergence and tau_x from
// dn[0] = D(r) and dn[1] = J_D(r) b ([2][n][n]): D' = b^T J_D b / N, the
// eps -> 0 limit of Eq. MC_SURE (F.jvp = 1), or from dn[1] = D(r + eps b):
// D' = b^T (dn[1] - dn[0]) / (N eps).  32 x 32 tiles as in the blocked TV's
// final launch.
__global__ void __launch_bounds__(1024)
k_denoise_final(const float* __restrict__ dn, int n, DevScalars* S, TvFinal F) {
    __shared__ float tile[TB][TB + 1];
    __shared__ double red[32];
    __shared__ bool am_last;
    const size_t N = (size_t)n * n;
    const int tid = threadIdx.x, ta = tid >> 5, tb = tid & 31;
    const int gi = blockIdx.y * TB + ta, gj = blockIdx.x * TB + tb;
    const unsigned t = F.t_arg > 0 ? (unsigned)F.t_arg : S->t;
    double acc = 0.0;
    float xv = 0.f;
    if (gi < n && gj < n) {
        const size_t o = (size_t)gi * n + gj;
        const float x1 = dn[o], x2 = dn[N + o];
        const float4 b4 = probe4((unsigned)(o >> 2), t, F.slice, F.key);
        const int kk = (int)(o & 3);
        const float bv = kk == 0 ? b4.x : (kk == 1 ? b4.y : (kk == 2 ? b4.z : b4.w));
        acc = (double)bv * (double)(F.jvp ? x2 : x2 - x1);
        xv = x1;
        if (F.solve_mode && F.damp_x != 1.f) xv = F.damp_x * xv + (1.f - F.damp_x) * F.x_out[o];
        F.x_out[o] = xv;
        if (F.XR) F.XR[(size_t)gi * F.ldp + kPad + gj] = xv;
    }
    tile[ta][tb] = xv;
    if (F.XC) {
        __syncthreads();
        const int gj2 = blockIdx.x * TB + ta, gi2 = blockIdx.y * TB + tb;
        if (gi2 < n && gj2 < n) F.XC[(size_t)gj2 * F.ldp + kPad + gi2] = tile[tb][ta];
    }
    acc = block_sum(acc, red);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) {
        F.partial[bid] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_div, 1u);
        am_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double tot = 0.0;
    for (int b = tid; b < nblk; b += blockDim.x) tot += ((volatile double*)F.partial)[b];
    tot = block_sum(tot, red);
    if (tid == 0) {
        const double div = F.jvp ? tot / (double)N : tot / ((double)N * S->eps);
        if (F.div_out) *F.div_out = div;
        if (F.solve_mode) {
            const double tau_r = S->tau_r;
            double tx = tau_r * div;
            const double fl = F.tau_x_floor * tau_r;
            if (!(tx >= fl)) { tx = fl; S->floored += 1u; }
            if (!isfinite(tx)) S->nonfinite += 1u;
            S->div = div;
            S->tau_x = tx;
            const unsigned tt = S->t;
            if (tt >= 1u && tt <= (unsigned)kMaxIters) {
                IterLog L;
                L.tau_x = tx; L.tau_p = S->tau_p; L.tau_s = S->tau_s; L.tau_r = tau_r;
                L.div = div; L.eps = S->eps;
                F.log[tt - 1] = L;
            }
            S->t = tt + 1u;
        }
        S->done_div = 0u;
    }
}

int launch_denoise_final(const dgamp_ct_plan_s* pl, const float* dn, float* x_out, int solve_mode, int t_arg,
                         double* div_out, cudaStream_t st) {
    TvFinal F;
    F.x_out = x_out;
    F.XR = solve_mode ? pl->ws.XR : nullptr;
    F.XC = solve_mode ? pl->ws.XC : nullptr;
    F.ldp = pl->ldp;
    F.damp_x = (float)pl->opt.damp_x;
    F.t_arg = t_arg;
    F.slice = (unsigned)pl->opt.slice_id;
    F.key = probe_key(pl);
    F.tau_x_floor = pl->opt.tau_x_floor;
    F.partial = pl->ws.partial;
    F.log = pl->ws.log;
    F.div_out = div_out;
    F.solve_mode = solve_mode;
    F.jvp = 1;
    const int n = pl->n;
    dim3 grd((n + TB - 1) / TB, (n + TB - 1) / TB);
    k_denoise_final<<<grd, 1024, 0, st>>>(dn, n, pl->ws.S, F);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// ------------------------------------------------------------ probe -----
__global__ void k_probe(long long n, unsigned t, unsigned slice, uint2 key, float* __restrict__ b,
                        uint32_t* __restrict__ words) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long i0 = 4 * g;
    if (i0 >= n) return;
    if (b) {
        const float4 v = probe4((unsigned)g, t, slice, key);
        const float vv[4] = {v.x, v.y, v.z, v.w};
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) b[i0 + k] = vv[k];
    }
    if (words) {
        const uint4 w = philox4x32_10(make_uint4((unsigned)g, t, slice, 0u), key);
        const unsigned ww[4] = {w.x, w.y, w.z, w.w};
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) words[i0 + k] = ww[k];
    }
}

int launch_probe(const dgamp_ct_plan_s* pl, unsigned t, int64_t n, float* b, uint32_t* words,
                 cudaStream_t st) {
    const long long groups = (n + 3) / 4;
    k_probe<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(n, t, (unsigned)pl->opt.slice_id,
                                                              probe_key(pl), b, words);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
