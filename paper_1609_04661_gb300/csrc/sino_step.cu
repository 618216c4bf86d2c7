// The sinogram part of one iteration as one kernel (Algorithm 1, Steps 1-3
// between the projector and the back-projector):
//   z = H (A x)            detector-axis preconditioner, Section 2.4
//   s, tau_s_i             Poisson output step, Section 4.2 / Appendix A
//   H s                    the adjoint side, H being symmetric
// One block takes two views packed as the real and imaginary parts of one
// complex line (the gain is real and even, so one FFT pair filters both), as
// the stand-alone filter kernel does.  z stays in shared memory; the twiddle
// table is staged there once for the four transforms; s is written for the
// next iteration and, rounded as stored, filtered in place.
//
// Reductions.  Each block stores its FP64 partial sum of tau_s_i; the
// back-projection that follows adds the partials in a fixed order and forms
// tau_s and tau_r, so no block here waits for the others.  Before the output
// step the kernel needs tau_x, whose TV divergence (Step 4 of the previous
// iteration) may still be in partial sums: every block adds those in a fixed
// order, and block 0 records D', tau_x, the iteration's log and the next t
// (pending_tau_x).  This replaces three launches, two round trips of a
// sinogram through L2 and two grid-wide reduction tails.
#include <cooperative_groups.h>

#include "fft_device.cuh"
#include "output_device.cuh"

namespace cg = cooperative_groups;

namespace dgct {

constexpr int kSinoThreads = 512;
constexpr int kSinoMaxP = 8192;       // two padded buffers and the twiddles: 213 KB of shared memory

// elements of the output step one thread keeps in registers from the start
// (s_prev and y are loaded before the first transform, which hides their
// latency); beyond 2 n_det = kSinoPre * kSinoThreads they are loaded in place
constexpr int kSinoPre = 4;
// TV divergence partials each lane of warp 0 prefetches (10 x 32 covers the
// 288 blocks of the 512 x 512 denoiser launch)
constexpr int kDivPre = 10;

// the value a store of v into T and a load back give
__device__ __forceinline__ float as_stored(float v, const float*) { return v; }
__device__ __forceinline__ float as_stored(float v, const bf16s*) { return __bfloat162float(__float2bfloat16_rn(v)); }

template <typename T>
__global__ void __launch_bounds__(kSinoThreads)
k_sino_step(const T* __restrict__ zraw, const float* __restrict__ y, T* s, T* __restrict__ hs, int nv, int nd,
            int P, const float* __restrict__ gain, const float2* __restrict__ tw_g, long long M,
            int onsager, float damp_s, int truncate, DevScalars* S, double* __restrict__ partial,
            const double* __restrict__ partial_div, double N, double floor_rel, IterLog* log) {
    extern __shared__ float2 smem[];
    const int BL = fft_buf_len(P), TC = fft_twiddle_count(P);
    float2* a = smem;                 // [BL], padded layout
    float2* b = smem + BL;            // [BL]
    float2* tw = smem + 2 * BL;       // [TC], stage by stage
    __shared__ double sm[32];
    __shared__ float s_tp, s_inv, s_logI0;
    const int va = 2 * blockIdx.x, vb = va + 1;
    const bool hasb = vb < nv;
    const int ne = hasb ? 2 * nd : nd;
    // tau_x of the previous iteration may still be in the TV step's partial
    // sums: warp 0 loads its lanes' first kDivPre of them now and finishes
    // the sum after the first transform pair, which hides the loads
    double div_pre[kDivPre];
    if (threadIdx.x < 32) {
        const unsigned np = S->div_pending;
#pragma unroll
        for (int k = 0; k < kDivPre; ++k) {
            const unsigned i = threadIdx.x + 32u * k;
            div_pre[k] = i < np ? partial_div[i] : 0.0;
        }
        if (threadIdx.x == 0 && blockIdx.x == 0) S->rmax_bits = 0u;   // refilled by the back-projection
    }
    // s_prev and y of this thread's first kSinoPre elements
    float pre_sp[kSinoPre], pre_y[kSinoPre];
#pragma unroll
    for (int j = 0; j < kSinoPre; ++j) {
        const int e = threadIdx.x + j * kSinoThreads;
        pre_sp[j] = pre_y[j] = 0.f;
        if (e < ne) {
            const int d = e >= nd ? e - nd : e;
            const size_t gi = (size_t)(e >= nd ? vb : va) * nd + d;
            pre_sp[j] = ldf(s + gi);
            pre_y[j] = y[gi];
        }
    }
    for (int i = threadIdx.x; i < TC; i += blockDim.x) tw[i] = tw_g[i];
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (i < nd) {
            v.x = ldf(zraw + (size_t)va * nd + i);
            if (hasb) v.y = ldf(zraw + (size_t)vb * nd + i);
        }
        a[fpad(i)] = v;
    }
    __syncthreads();
    // z = H A x; the 1/P of the inverse transform is folded into the gain
    // (a power of two: the same rounding as scaling afterwards)
    const float invP = 1.0f / (float)P;
    float2* r = fft_stockham(a, b, P, tw, -1.f);
    float2* o = (r == a) ? b : a;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float g = __ldg(gain + i) * invP;
        const float2 v = r[fpad(i)];
        r[fpad(i)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    r = fft_stockham(r, o, P, tw, 1.f);
    o = (r == a) ? b : a;

    if (threadIdx.x < 32) {
        const double tx = pending_tau_x(S, partial_div, N, floor_rel, log, blockIdx.x == 0, div_pre, kDivPre);
        if (threadIdx.x == 0) {
            const double tp = S->frob2 * tx / (double)M;          // Step 2: tau_p
            s_tp = (float)tp;
            s_inv = (float)(1.0 / tp);
            s_logI0 = (float)S->logI0;
        }
    }
    __syncthreads();
    // output step on both views; s (as stored) goes into o, zero-padded
    const float tau_p = s_tp, inv_tp = s_inv, logI0 = s_logI0;
    for (int i = nd + threadIdx.x; i < P; i += blockDim.x) o[fpad(i)] = make_float2(0.f, 0.f);
    double acc = 0.0;
    unsigned capped = 0;
#pragma unroll 1
    for (int j = 0, e = threadIdx.x; e < ne; ++j, e += kSinoThreads) {
        const bool isb = e >= nd;
        const int d = isb ? e - nd : e;
        const size_t gi = (size_t)(isb ? vb : va) * nd + d;
        float sp, yv;
        if (j < kSinoPre) {
            sp = pre_sp[0];
            yv = pre_y[0];
#pragma unroll
            for (int u = 1; u < kSinoPre; ++u)
                if (j == u) {
                    sp = pre_sp[u];
                    yv = pre_y[u];
                }
        } else {
            sp = ldf(s + gi);
            yv = y[gi];
        }
        float sv;
        acc += (double)output_element(isb ? r[fpad(d)].y : r[fpad(d)].x, sp, yv, tau_p, inv_tp, logI0, onsager,
                                      damp_s, truncate, capped, sv);
        stf(s + gi, sv);
        const float sq = as_stored(sv, s);
        if (!hasb)
            o[fpad(d)] = make_float2(sq, 0.f);
        else if (isb)
            o[fpad(d)].y = sq;
        else
            o[fpad(d)].x = sq;
    }
    __syncthreads();
    // H s
    float2* q = fft_stockham(o, r, P, tw, -1.f);
    float2* q2 = (q == o) ? r : o;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float g = __ldg(gain + i) * invP;
        const float2 v = q[fpad(i)];
        q[fpad(i)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    q = fft_stockham(q, q2, P, tw, 1.f);
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        const float2 v = q[fpad(i)];
        stf(hs + (size_t)va * nd + i, v.x);
        if (hasb) stf(hs + (size_t)vb * nd + i, v.y);
    }
    capped = warp_sum(capped);
    if ((threadIdx.x & 31) == 0 && capped) atomicAdd(&S->newton_capped, capped);
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// ---------------------------------------------- cluster Toeplitz form ----
// The same step with H as its Toeplitz product, (H z)[d] = sum_d' h[|d - d'|]
// z[d'] (the FFT form's operator, fft.cu), spread over a cluster of CL
// CTAs per view instead of one block per pair of views: the FFT form's four
// transforms are a serial chain that leaves most SMs idle, while the direct
// products split freely over output bins.  CTA `rank` of the cluster of view
// v owns bins [rank per, (rank + 1) per), per = ceil(n_det / CL):
//   1. it loads the whole row of A x and the kernel hx;
//   2. W warps split the d' range of z = H A x for its bins, each lane
//      R consecutive bins with a sliding window of hx in registers (R odd:
//      the lanes' window loads fall on distinct banks), partial sums added
//      in a fixed order; meanwhile one more warp finishes tau_x (the
//      previous iteration's divergence) and tau_p;
//   3. the output step on its bins; s goes to global memory and, as stored,
//      into the s row of every CTA of the cluster (distributed shared memory);
//      the block's tau_s_i sum goes to rank 0;
//   4. one cluster barrier; rank 0 stores the view's tau_s partial (a fixed
//      order over the ranks); every CTA forms H s for its bins.
// No CTA reads another's shared memory after the barrier, so there is no
// second one.  The back-projection adds the n_views partials.
// Two shapes, chosen by the number of bins: up to 896 bins, a cluster of 4
// CTAs per view with 8 product warps and up to 7 bins per lane (more
// multiply-adds per shared-memory load, shorter serial chains); beyond that, 8
// CTAs with 4 product warps (up to 1792 bins).
constexpr int kCtMaxCL = 8;
constexpr int kCtPre = 2;              // s_prev and y prefetched per thread (covers 2 x 160 >= 224 bins)
constexpr int kCtMaxR = 7;             // bins per lane at most
constexpr int kCtSmallNd = 4 * 32 * kCtMaxR;   // 896: the 4-CTA shape up to here

__host__ __device__ constexpr int ct_threads(int W) { return 32 * (W + 1); }
__host__ __device__ __forceinline__ int ct_hs_len(int nd, int R) { return 2 * nd + R + 1; }

// acc[k] = sum over d' in [p0, p1) of hs[dl + k - d' + nd] z[d'] (hs = hx shifted by one)
template <int R>
__device__ __forceinline__ void ct_product(const float* __restrict__ z, const float* __restrict__ hs, int nd,
                                           int dl, int p0, int p1, float (&acc)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = 0.f;
    if (p0 >= p1) return;
    int base = dl - p0 + nd;
    float h[R];
#pragma unroll
    for (int k = 0; k < R; ++k) h[k] = hs[base + k];
    // unrolled by R, the window's shift becomes a rotation of registers
#pragma unroll R
    for (int dp = p0; dp < p1; ++dp) {
        const float zv = z[dp];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = fmaf(h[k], zv, acc[k]);
#pragma unroll
        for (int k = R - 1; k > 0; --k) h[k] = h[k - 1];
        --base;
        h[0] = hs[base];
    }
}

struct CtShared {
    double sm[32];
    double tsum[kCtMaxCL];
    float s_tp, s_inv, s_logI0;
};

// View v's cluster (CL CTAs, W product warps each), this CTA's part;
// record: the slice's first CTA (it records the previous iteration's tau_x
// and log, and resets max |r|).
template <typename T, int R, int CL, int W>
__device__ __forceinline__ void sino_ct_block(const T* __restrict__ zraw, const float* __restrict__ y, T* s,
                                              T* __restrict__ hsout, int nd, const float* __restrict__ hx,
                                              long long M, int onsager, float damp_s, int truncate, DevScalars* S,
                                              double* __restrict__ partial, const double* __restrict__ partial_div,
                                              double N, double floor_rel, IterLog* log, int v, bool record,
                                              float* smf, CtShared& shd, const float* __restrict__ part = nullptr,
                                              int nb = 0, float wv = 0.f) {
    constexpr int OUT = 32 * R;
    constexpr int TH = ct_threads(W);
    auto& sm = shd.sm;
    auto& tsum = shd.tsum;
    auto& s_tp = shd.s_tp;
    auto& s_inv = shd.s_inv;
    auto& s_logI0 = shd.s_logI0;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int per = (nd + CL - 1) / CL;
    const int d_lo = min(nd, rank * per), d_hi = min(nd, d_lo + per), nown = d_hi - d_lo;
    const int HL = ct_hs_len(nd, R);
    float* zs = smf;            // [nd]  A x of the view
    float* sf = zs + nd;        // [nd]  s of the view, filled by every CTA of the cluster
    float* hs = sf + nd;        // [HL]  hs[i] = hx[i - 1], zero outside
    float* red = hs + HL;       // [W][OUT]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const size_t row0 = (size_t)v * nd;
    // the filter is constant over a solve: staged before waiting on the
    // previous kernel, whose output (A x) and scalars everything else reads
    for (int i = tid; i < HL; i += TH) {
        const int m = i - 1;
        hs[i] = (m >= 0 && m < 2 * nd - 1) ? hx[m] : 0.f;
    }
    // every CTA of the cluster has started before the first write into another's
    // shared memory: arrive now, wait just before that write
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
    pdl_wait();
    // the tau_x warp issues its loads of the divergence partials first, so
    // that their latency overlaps the loads and the first product
    double div_pre[kDivPre];
    if (w == W) {
        const unsigned np = S->div_pending;
#pragma unroll
        for (int k = 0; k < kDivPre; ++k) {
            const unsigned i = (unsigned)lane + 32u * k;
            div_pre[k] = i < np ? partial_div[i] : 0.0;
        }
    }
    // this thread's bins of the output step: s_prev and y now, used after the first product
    float pre_sp[kCtPre], pre_y[kCtPre];
#pragma unroll
    for (int j = 0; j < kCtPre; ++j) {
        const int o = tid + j * TH;
        pre_sp[j] = pre_y[j] = 0.f;
        if (o < nown) {
            pre_sp[j] = ldf(s + row0 + d_lo + o);
            pre_y[j] = y[row0 + d_lo + o];
        }
    }
    if (part) {
        // A x from the banded projector's partial sums (nb bands, added in
        // band order, times the path length per step, rounded as the storage
        // type would store it): each CTA its own bins, then to every CTA
        for (int o = tid; o < nown; o += TH) {
            const float* __restrict__ pp = part + row0 + d_lo + o;
            float t = 0.f;
            int b = 0;
            for (; b + 16 <= nb; b += 16) {
                float pv[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) pv[k] = pp[(size_t)(b + k) * M];
#pragma unroll
                for (int k = 0; k < 16; ++k) t += pv[k];
            }
            for (; b < nb; ++b) t += pp[(size_t)b * M];
            zs[d_lo + o] = as_stored(t * wv, zraw);
        }
        asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
        __syncthreads();
        for (int o = tid; o < nown; o += TH) {
            const float z = zs[d_lo + o];
#pragma unroll
            for (int r = 0; r < CL; ++r)
                if (r != rank) *cluster.map_shared_rank(zs + d_lo + o, r) = z;
        }
        cluster.sync();         // every bin of zs is in every CTA
    } else {
        for (int i = tid; i < nd; i += TH) zs[i] = ldf(zraw + row0 + i);
        asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
    }
    __syncthreads();
    const int len = (nd + W - 1) / W;
    const int dl = d_lo + R * lane;
    if (w < W) {
        // z = H A x for this CTA's bins, warp w's share of d'
        float acc[R];
        if (dl < d_hi) ct_product<R>(zs, hs, nd, dl, w * len, min(nd, w * len + len), acc);
        else
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) red[w * OUT + R * lane + k] = acc[k];
    } else {
        // tau_x of the previous iteration (its divergence may still be in
        // partial sums; every CTA adds them in the same order), then tau_p
        const double tx = pending_tau_x(S, partial_div, N, floor_rel, log, record, div_pre, kDivPre);
        if (lane == 0) {
            const double tp = S->frob2 * tx / (double)M;
            s_tp = (float)tp;
            s_inv = (float)(1.0 / tp);
            s_logI0 = (float)S->logI0;
            if (record) S->rmax_bits = 0u;   // refilled by the back-projection
        }
    }
    __syncthreads();
    // output step on this CTA's bins; s as stored into every CTA's s row
    const float tau_p = s_tp, inv_tp = s_inv, logI0 = s_logI0;
    double acc = 0.0;
    unsigned capped = 0;
#pragma unroll
    for (int j = 0; j < kCtPre; ++j) {
        const int o = tid + j * TH;
        if (o < nown) {
            float zi = 0.f;
#pragma unroll
            for (int k = 0; k < W; ++k) zi += red[k * OUT + o];
            float sv;
            acc += (double)output_element(zi, pre_sp[j], pre_y[j], tau_p, inv_tp, logI0, onsager, damp_s, truncate,
                                          capped, sv);
            stf(s + row0 + d_lo + o, sv);
            const float sq = as_stored(sv, s);
#pragma unroll
            for (int r = 0; r < CL; ++r) *cluster.map_shared_rank(sf + d_lo + o, r) = sq;
        }
    }
    capped = warp_sum(capped);
    if (lane == 0 && capped) atomicAdd(&S->newton_capped, capped);
    acc = block_sum(acc, sm);
    if (tid == 0) *cluster.map_shared_rank(&tsum[rank], 0) = acc;
    cluster.sync();             // every s of the view is in sf; tau_s sums are at rank 0
    if (rank == 0 && tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int r = 0; r < CL; ++r) t += tsum[r];
        partial[v] = t;
    }
    // H s for this CTA's bins
    if (w < W) {
        float a2[R];
        if (dl < d_hi) ct_product<R>(sf, hs, nd, dl, w * len, min(nd, w * len + len), a2);
        else
#pragma unroll
            for (int k = 0; k < R; ++k) a2[k] = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) red[w * OUT + R * lane + k] = a2[k];
    }
    __syncthreads();
    for (int o = tid; o < nown; o += TH) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < W; ++k) t += red[k * OUT + o];
        stf(hsout + row0 + d_lo + o, t);
    }
}

template <typename T, int R, int CL, int W>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(ct_threads(W), 2)
k_sino_toeplitz(const T* __restrict__ zraw, const float* __restrict__ y, T* s, T* __restrict__ hsout, int nd,
                const float* __restrict__ hx, long long M, int onsager, float damp_s, int truncate, DevScalars* S,
                double* __restrict__ partial, const double* __restrict__ partial_div, double N, double floor_rel,
                IterLog* log, const float* __restrict__ part, int nb, const ViewConst* __restrict__ vcs) {
    extern __shared__ float smf[];
    __shared__ CtShared shd;
    const int v = (int)blockIdx.x / CL;
    sino_ct_block<T, R, CL, W>(zraw, y, s, hsout, nd, hx, M, onsager, damp_s, truncate, S, partial, partial_div, N,
                               floor_rel, log, v, blockIdx.x == 0, smf, shd, part, nb, part ? vcs[v].w : 0.f);
}

// The sinogram step of every slice of a batch in one launch: cluster c
// (CL CTAs) -> (slice, view); the slices' bins may differ (the shape, R and
// the shared memory are those of the largest).
template <typename T, int R, int CL, int W>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(ct_threads(W))
k_sino_toeplitz_batch(const BatchSlice* __restrict__ sl, const uint16_t* __restrict__ map) {
    extern __shared__ float smf[];
    __shared__ CtShared shd;
    const int c = (int)blockIdx.x / CL;
    const BatchSlice& B = sl[map[c]];
    const int v = c - B.off[kPhView];
    sino_ct_block<T, R, CL, W>((const T*)B.zraw, B.y, (T*)B.s, (T*)B.hs, B.nd, B.hx, B.M, B.onsager, B.damp_s,
                               B.truncate, B.S, B.partial, B.partial_div, (double)B.N, B.tau_x_floor, B.log, v,
                               blockIdx.x == (unsigned)(B.off[kPhView] * CL), smf, shd);
}

// Shape for n_det bins: returns R (bins per lane; 0 = too many bins) and the
// cluster size in *cl (4 or 8, with 8 or 4 product warps).
int sino_ct_config(int nd, int* cl) {
    const int c = nd <= kCtSmallNd ? 4 : 8;
    const int per = (nd + c - 1) / c;
    if (cl) *cl = c;
    for (int R = 3; R <= kCtMaxR; R += 2)
        if (32 * R >= per) return R;
    return 0;
}

static int ct_warps(int cl) { return cl == 4 ? 8 : 4; }

static int ct_smem(int nd, int R, int cl) {
    return (2 * nd + ct_hs_len(nd, R) + ct_warps(cl) * 32 * R) * (int)sizeof(float);
}

int sino_ct_smem_bytes(int nd, int R, int cl) { return ct_smem(nd, R, cl); }

// one instantiation per (R, shape); F(kernel pointer, threads, cluster size)
template <typename T, bool BATCH, typename Fn>
static int ct_dispatch(int R, int cl, Fn&& f) {
#define DGCT_CT_K(RR, CC, WW)                                                                         \
    if (R == RR && cl == CC) {                                                                        \
        if (BATCH) return f((const void*)k_sino_toeplitz_batch<T, RR, CC, WW>, ct_threads(WW), CC);   \
        return f((const void*)k_sino_toeplitz<T, RR, CC, WW>, ct_threads(WW), CC);                    \
    }
    DGCT_CT_K(3, 4, 8) DGCT_CT_K(5, 4, 8) DGCT_CT_K(7, 4, 8)
    DGCT_CT_K(3, 8, 4) DGCT_CT_K(5, 8, 4) DGCT_CT_K(7, 8, 4)
#undef DGCT_CT_K
    return DGAMP_CT_ERR_INVALID_ARG;
}

template <typename T>
static int launch_ct_batch(const BatchExec& E, cudaStream_t st) {
    const size_t sm = (size_t)E.ct_smem;
    void* args[] = {(void*)&E.sl, (void*)&E.map[kPhView]};
    return ct_dispatch<T, true>(E.R, E.cl, [&](const void* k, int threads, int cl) -> int {
        DGCT_TRY(raise_smem_limit(k, (int)sm));
        DGCT_CUDA(launch_pdl_c(k, dim3((unsigned)(E.nblk[kPhView] * cl)), dim3(threads), sm, st, args));
        return DGAMP_CT_OK;
    });
}

int launch_sino_batch(const BatchExec& E, cudaStream_t st) {
    return E.bf ? launch_ct_batch<bf16s>(E, st) : launch_ct_batch<float>(E, st);
}

bool sino_toeplitz_eligible(const dgamp_ct_plan_s* pl) {
    int cl = 0;
    const int R = sino_ct_config(pl->nd, &cl);
    return R > 0 && pl->nv <= pl->max_partials && ct_smem(pl->nd, R, cl) <= 200 * 1024;
}

template <typename T>
static int launch_ct(const dgamp_ct_plan_s* pl, cudaStream_t st, const T* zraw, T* s, T* hs) {
    const Workspace& w = pl->ws;
    int cl = 0;
    const int R = sino_ct_config(pl->nd, &cl);
    const size_t sm = (size_t)ct_smem(pl->nd, R, cl);
    int nd = pl->nd, onsager = pl->opt.onsager, truncate = pl->opt.truncate_z;
    long long M = pl->M;
    float damp_s = (float)pl->opt.damp_s;
    double N = (double)pl->N, floor_rel = pl->opt.tau_x_floor;
    const float* y = w.y;
    const float* hx = w.hx;
    DevScalars* S = w.S;
    double* partial = w.partial;
    const double* partial_div = w.partial_div;
    IterLog* log = w.log;
    // with the banded projector the kernel adds its band partials itself
    const float* part = project_sum_in_sino(pl) ? w.pj_part : nullptr;
    int nb = part ? (pl->n + pl->pj_band - 1) / pl->pj_band : 0;
    const ViewConst* vcs = w.vc;
    void* args[] = {(void*)&zraw, (void*)&y, (void*)&s, (void*)&hs, (void*)&nd, (void*)&hx, (void*)&M,
                    (void*)&onsager, (void*)&damp_s, (void*)&truncate, (void*)&S, (void*)&partial,
                    (void*)&partial_div, (void*)&N, (void*)&floor_rel, (void*)&log, (void*)&part, (void*)&nb,
                    (void*)&vcs};
    return ct_dispatch<T, false>(R, cl, [&](const void* k, int threads, int c) -> int {
        DGCT_CUDA(launch_pdl_c(k, dim3((unsigned)(pl->nv * c)), dim3(threads), sm, st, args));
        return DGAMP_CT_OK;
    });
}

template <typename T>
static int ct_set_limits(int bytes, int R, int cl) {
    return ct_dispatch<T, false>(R, cl, [&](const void* k, int, int) -> int { return raise_smem_limit(k, bytes); });
}

static int sino_step_smem(int P) {
    return (2 * fft_buf_len(P) + fft_twiddle_count(P)) * (int)sizeof(float2);
}

// FP64 tau_s partials the current form leaves in ws.partial: one per block
// of the FFT form (two views each), one per view of the cluster form
int sino_step_partials(const dgamp_ct_plan_s* pl) { return pl->sino_fused == 2 ? pl->nv : (pl->nv + 1) / 2; }

bool sino_step_eligible(const dgamp_ct_plan_s* pl) {
    return pl->P <= kSinoMaxP && (pl->nv + 1) / 2 <= pl->max_partials;
}

int sino_step_set_smem_limit(const dgamp_ct_plan_s* pl) {
    if (sino_toeplitz_eligible(pl)) {
        int cl = 0;
        const int R = sino_ct_config(pl->nd, &cl);
        const int bytes = ct_smem(pl->nd, R, cl);
        DGCT_TRY(ct_set_limits<float>(bytes, R, cl));
        DGCT_TRY(ct_set_limits<bf16s>(bytes, R, cl));
    }
    if (!sino_step_eligible(pl)) return DGAMP_CT_OK;
    // set even at or below 48 KB: the static shared memory of the reduction
    // comes on top of the dynamic part
    const int bytes = sino_step_smem(pl->P);
    DGCT_TRY(raise_smem_limit((const void*)k_sino_step<float>, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_sino_step<bf16s>, bytes));
    return DGAMP_CT_OK;
}

// z = H zraw, the output step into s (s_prev in, damped s out), hs = H s;
// bf = 1: the three sinograms in BF16 (counts stay FP32).  The plan's
// sino_fused picks the form: 1 the FFT form, 2 the cluster Toeplitz form.
int launch_sino_step(const dgamp_ct_plan_s* pl, cudaStream_t st, int bf) {
    const Workspace& w = pl->ws;
    if (pl->sino_fused == 2) {
        if (!sino_toeplitz_eligible(pl)) return DGAMP_CT_ERR_INVALID_ARG;
        if (bf) return launch_ct<bf16s>(pl, st, (const bf16s*)w.zraw, (bf16s*)w.s, (bf16s*)w.hs);
        return launch_ct<float>(pl, st, w.zraw, w.s, w.hs);
    }
    if (!sino_step_eligible(pl)) return DGAMP_CT_ERR_INVALID_ARG;
    const int grid = (pl->nv + 1) / 2;
    const size_t sm = (size_t)sino_step_smem(pl->P);
    const float damp_s = (float)pl->opt.damp_s;
    if (bf)
        k_sino_step<bf16s><<<grid, kSinoThreads, sm, st>>>((const bf16s*)w.zraw, w.y, (bf16s*)w.s, (bf16s*)w.hs,
                                                           pl->nv, pl->nd, pl->P, w.gain, w.tw, pl->M,
                                                           pl->opt.onsager, damp_s, pl->opt.truncate_z, w.S,
                                                           w.partial, w.partial_div, (double)pl->N,
                                                           pl->opt.tau_x_floor, w.log);
    else
        k_sino_step<float><<<grid, kSinoThreads, sm, st>>>(w.zraw, w.y, w.s, w.hs, pl->nv, pl->nd, pl->P, w.gain,
                                                           w.tw, pl->M, pl->opt.onsager, damp_s, pl->opt.truncate_z,
                                                           w.S, w.partial, w.partial_div, (double)pl->N,
                                                           pl->opt.tau_x_floor, w.log);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// Plan-time choice of the fused form (sino_fused 1: FFT, 2: cluster Toeplitz)
// by timing both on the plan's geometry; 0 when neither applies.  Runs on
// zero counts and a zero sinogram (solve_begin resets every buffer and scalar
// it touches).
int sino_autotune(dgamp_ct_plan_s* pl) {
    const bool fft = sino_step_eligible(pl), ct = sino_toeplitz_eligible(pl);
    pl->sino_fused = fft ? 1 : (ct ? 2 : 0);
    if (!(fft && ct)) return DGAMP_CT_OK;
    const Workspace& w = pl->ws;
    const size_t M = (size_t)pl->M;
    DGCT_CUDA(cudaMemset(w.zraw, 0, M * sizeof(float)));
    DGCT_CUDA(cudaMemset(w.y, 0, M * sizeof(float)));
    DGCT_CUDA(cudaMemset(w.s, 0, M * sizeof(float)));
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 0.f;
    int pick = 1, rc = DGAMP_CT_OK;
    for (int mode = 1; mode <= 2 && rc == DGAMP_CT_OK; ++mode) {
        pl->sino_fused = mode;
        for (int i = 0; i < 3 && rc == DGAMP_CT_OK; ++i) rc = launch_sino_step(pl, 0, 0);
        if (rc != DGAMP_CT_OK) break;
        cudaEventRecord(e0, 0);
        for (int i = 0; i < 20 && rc == DGAMP_CT_OK; ++i) rc = launch_sino_step(pl, 0, 0);
        cudaEventRecord(e1, 0);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (mode == 1 || ms < best) {
            best = ms;
            pick = mode;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->sino_fused = pick;
    return rc;
}

}  // namespace dgct
