// Poisson output step, Algorithm 1 Step 2 (Section 4.2, Appendix A).
//
// Per measurement: p = z - tau_p s_prev, the Laplace mode z0 of
// N(z; p, tau_p) x Poisson(y; I0 e^{-z}), s = (z0 - p)/tau_p and
// tau_s_i = w/(1 + tau_p w), w = I0 e^{-z0}.  The mode is found for
// delta = z0 - p as the root of psi(delta) = delta/tau_p + y - e^{log I0 - p - delta}
// (strictly increasing) by Newton's method safeguarded with bisection on a
// bracket where psi changes sign:
//   y > 0:  [min(0, L - p), max(0, L - p)], L = log(I0 / y)
//   y = 0:  [0, m - p + tau_p e^{log I0 - m}], m = max(p, log I0).
// With truncate = 1 the posterior is restricted to z >= 0: where z0 < 0 the
// mode is 0, s = -p/tau_p and tau_s_i = 1/tau_p (the mode no longer moves with p).
// Arithmetic is FP32; tau_s = mean(tau_s_i) is accumulated in FP64 and
// finished by the last block to arrive, which (inside a solve) also forms
// tau_r = N / (||Phi~||_F^2 tau_s) for Step 3.
#include "internal.cuh"

namespace dgct {

__device__ __forceinline__ float mode_delta(float p, float y, float tau_p, float inv_tp,
                                            float logI0, unsigned& capped) {
    const float e0 = logI0 - p;                  // log of I0 e^{-p}
    float lo, hi;
    if (y > 0.f) {
        const float Lp = logI0 - logf(y) - p;    // L - p
        lo = fminf(0.f, Lp);
        hi = fmaxf(0.f, Lp);
    } else {
        const float m = fmaxf(p, logI0);
        lo = 0.f;
        hi = m - p + tau_p * expf(logI0 - m);
    }
    float d = lo, dxold = hi - lo;
    int it = 0;
    for (; it < kNewtonCap; ++it) {
        const float w = expf(e0 - d);
        const float f = d * inv_tp + y - w;
        // converged to rounding: |psi| within a few ulps of its largest term
        if (fabsf(f) <= 4.0e-7f * (fabsf(d * inv_tp) + y + w)) break;
        if (f < 0.f) lo = d; else hi = d;
        const float df = inv_tp + w;
        const float nt = d - __fdividef(f, df);     // an iterate: a fast quotient is enough
        const bool bad = !(nt > lo && nt < hi) || fabsf(2.f * f) > fabsf(dxold * df);
        const float nx = bad ? 0.5f * (lo + hi) : nt;
        dxold = fabsf(nx - d);
        d = nx;
        if (dxold <= 1.2e-7f * fabsf(d)) break;
    }
    if (it == kNewtonCap) ++capped;
    return d;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_output_step(const T* z, const float* y, T* s, long long M, int use_prev,
              int from_scalars, double tau_p_arg, double logI0_arg, int onsager, float damp_s,
              int truncate, double N, DevScalars* S, double* partial, double* tau_s_out) {
    __shared__ double sm[32];
    __shared__ float s_tp, s_inv, s_logI0;
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        double tp = from_scalars ? S->frob2 * S->tau_x / (double)M : tau_p_arg;
        s_tp = (float)tp;
        s_inv = (float)(1.0 / tp);
        s_logI0 = (float)(from_scalars ? S->logI0 : logI0_arg);
    }
    __syncthreads();
    const float tau_p = s_tp, inv_tp = s_inv, logI0 = s_logI0;
    double acc = 0.0;
    unsigned capped = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (long long)gridDim.x * blockDim.x) {
        const float sp = use_prev ? ldf(s + i) : 0.f;
        const float zi = ldf(z + i);
        const float p = onsager ? fmaf(-tau_p, sp, zi) : zi;
        const float yv = y[i];
        float d = mode_delta(p, yv, tau_p, inv_tp, logI0, capped);
        const bool clamp = truncate && p + d < 0.f;
        if (clamp) d = -p;
        float sv = d * inv_tp;
        if (damp_s != 1.f) sv = damp_s * sv + (1.f - damp_s) * sp;
        stf(s + i, sv);
        const float w = expf(logI0 - p - d);
        const float tsi = (clamp || isinf(w)) ? inv_tp : w / fmaf(tau_p, w, 1.f);
        acc += (double)tsi;
    }
    capped = warp_sum(capped);
    if ((threadIdx.x & 31) == 0 && capped) atomicAdd(&S->newton_capped, capped);
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_out, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    // last block: fixed-order sum of the partials
    __threadfence();
    double tot = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) tot += ((volatile double*)partial)[b];
    tot = block_sum(tot, sm);
    if (threadIdx.x == 0) {
        const double tau_s = tot / (double)M;
        if (tau_s_out) *tau_s_out = tau_s;
        if (from_scalars) {
            const double tp = S->frob2 * S->tau_x / (double)M;
            S->tau_p = tp;
            S->tau_s = tau_s;
            S->tau_r = N / (S->frob2 * tau_s);
            if (!isfinite(S->tau_r)) S->nonfinite += 1u;
            S->rmax_bits = 0u;             // the back-projection that follows refills it
        }
        S->done_out = 0u;
    }
}

int launch_output_step(const dgamp_ct_plan_s* pl, const float* z, const float* y, float* s,
                       int use_prev, int from_scalars, double tau_p_arg, double logI0_arg,
                       double* tau_s_out, cudaStream_t st, int bf) {
    const long long M = pl->M;
    int blocks = (int)((M + 127) / 128);          // one element per thread, 128-thread blocks
    if (blocks > pl->max_partials) blocks = pl->max_partials;
    const int onsager = from_scalars ? pl->opt.onsager : 1;
    const float damp_s = from_scalars ? (float)pl->opt.damp_s : 1.f;
    if (bf)   // z and s in BF16 (a solve with storage = 1); the counts stay FP32
        k_output_step<bf16s><<<blocks, 128, 0, st>>>((const bf16s*)z, y, (bf16s*)s, M, use_prev, from_scalars,
                                                     tau_p_arg, logI0_arg, onsager, damp_s, pl->opt.truncate_z,
                                                     (double)pl->N, pl->ws.S, pl->ws.partial, tau_s_out);
    else
        k_output_step<float><<<blocks, 128, 0, st>>>(z, y, s, M, use_prev, from_scalars, tau_p_arg, logI0_arg,
                                                     onsager, damp_s, pl->opt.truncate_z, (double)pl->N, pl->ws.S,
                                                     pl->ws.partial, tau_s_out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// The same kernel on caller-supplied scratch (no plan): S holds the arrival
// counter and the Newton-cap counter, partial[] one FP64 sum per block
// (at most max_blocks blocks).
int launch_output_step_scratch(const float* z, const float* y, float* s, long long M, int use_prev,
                               double tau_p, double logI0, double* tau_s_out, DevScalars* S,
                               double* partial, int max_blocks, cudaStream_t st) {
    long long blocks = (M + 255) / 256;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    k_output_step<float><<<(int)blocks, 256, 0, st>>>(z, y, s, M, use_prev, 0, tau_p, logI0, 1, 1.f, 0, 0.0, S,
                                                      partial, tau_s_out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
