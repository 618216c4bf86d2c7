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
#include "fft_device.cuh"
#include "output_device.cuh"

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

static int sino_step_smem(int P) {
    return (2 * fft_buf_len(P) + fft_twiddle_count(P)) * (int)sizeof(float2);
}

int sino_step_partials(const dgamp_ct_plan_s* pl) { return (pl->nv + 1) / 2; }

bool sino_step_eligible(const dgamp_ct_plan_s* pl) {
    return pl->P <= kSinoMaxP && (pl->nv + 1) / 2 <= pl->max_partials;
}

int sino_step_set_smem_limit(const dgamp_ct_plan_s* pl) {
    if (!sino_step_eligible(pl)) return DGAMP_CT_OK;
    // set even at or below 48 KB: the static shared memory of the reduction
    // comes on top of the dynamic part
    const int bytes = sino_step_smem(pl->P);
    DGCT_TRY(raise_smem_limit((const void*)k_sino_step<float>, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_sino_step<bf16s>, bytes));
    return DGAMP_CT_OK;
}

// z = H zraw, the output step into s (s_prev in, damped s out), hs = H s;
// bf = 1: the three sinograms in BF16 (counts stay FP32)
int launch_sino_step(const dgamp_ct_plan_s* pl, cudaStream_t st, int bf) {
    if (!sino_step_eligible(pl)) return DGAMP_CT_ERR_INVALID_ARG;
    const Workspace& w = pl->ws;
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

}  // namespace dgct
