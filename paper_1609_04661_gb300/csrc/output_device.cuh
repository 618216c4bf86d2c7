// Poisson output step, Algorithm 1 Step 2 (Section 4.2, Appendix A): the
// per-measurement arithmetic and the reduction of tau_s, shared by the
// stand-alone output-step kernel and the fused sinogram kernel.
//
// Per measurement: p = z - tau_p s_prev, the Laplace mode z0 of
// N(z; p, tau_p) x Poisson(y; I0 e^{-z}), s = (z0 - p)/tau_p and
// tau_s_i = w/(1 + tau_p w), w = I0 e^{-z0}.  The mode is found for
// delta = z0 - p as the root of psi(delta) = delta/tau_p + y - e^{log I0 - p - delta}
// (strictly increasing) by Newton's method safeguarded with bisection on a
// bracket where psi changes sign:
//   y > 0:  [min(0, L - p), max(0, L - p)], L = log(I0 / y)
//   y = 0:  [0, m - p + tau_p e^{log I0 - m}], m = max(p, log I0).
// Starting point.  psi is concave, so Newton from any point lands on or left
// of the root and then climbs to it monotonically; a start near the root is
// what matters.  For y > 0 it is the root of psi with I0 e^{-z} replaced by
// its tangent at z = L (a lower bound of the convex exponential, so the start
// is left of the root): delta0 = (L - p) y tau_p / (1 + y tau_p).  For y = 0
// the root solves delta e^delta = tau_p I0 e^{-p} = a, i.e. delta = W(a)
// (Lambert W), and delta0 = log(1 + a) >= W(a) lies just right of it.  Both
// lie inside the bracket.  A start at the bracket end instead takes about one
// step per unit of log(I0 e^{-p} / y) while the exponential dominates.
// With truncate = 1 the posterior is restricted to z >= 0: where z0 < 0 the
// mode is 0, s = -p/tau_p and tau_s_i = 1/tau_p (the mode no longer moves with p).
// Arithmetic is FP32; tau_s = mean(tau_s_i) is accumulated in FP64 and
// finished by the last block to arrive, which (inside a solve) also forms
// tau_r = N / (||Phi~||_F^2 tau_s) for Step 3.
#pragma once
#include "internal.cuh"

namespace dgct {

__device__ __forceinline__ float mode_delta(float p, float y, float tau_p, float inv_tp,
                                            float logI0, unsigned& capped) {
    const float e0 = logI0 - p;                  // log of I0 e^{-p}
    float lo, hi, d;
    if (y > 0.f) {
        const float Lp = logI0 - logf(y) - p;    // L - p
        const float a = y * tau_p;
        lo = fminf(0.f, Lp);
        hi = fmaxf(0.f, Lp);
        d = Lp * (a / (1.f + a));
    } else {
        const float m = fmaxf(p, logI0);
        const float la = e0 + logf(tau_p);       // log a
        lo = 0.f;
        hi = m - p + tau_p * expf(logI0 - m);
        d = la > 15.f ? la : log1pf(expf(la));
    }
    d = fminf(fmaxf(d, lo), hi);
    float dxold = hi - lo;
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

// The end of Step 4 of the previous iteration when the blocked TV denoiser
// left its divergence as FP64 partial sums (S->div_pending of them in
// partial_div; Eq. MC_SURE): D' = sum / (N eps), tau_x = max(tau_r D',
// floor tau_r).  Run by one warp of every block of the output step that
// needs tau_x: the partials are added in one fixed order (lane-strided, then
// the warp's shuffle tree), so every block gets the same tau_x; the block
// with record = true also stores D', tau_x, the iteration's log record and
// the next t.  Returns tau_x (S->tau_x when nothing is pending).  The
// back-projection that follows clears div_pending.
// pre / npre: the lane's first partials (i = lane, lane + 32, ...), loaded
// earlier by the caller to hide their latency (npre = 0: none).
__device__ __forceinline__ double pending_tau_x(DevScalars* S, const double* __restrict__ partial_div, double N,
                                               double floor_rel, IterLog* log, bool record,
                                               const double* pre = nullptr, int npre = 0) {
    const unsigned np = S->div_pending;
    if (np == 0u) return S->tau_x;
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    for (int k = 0; k < npre; ++k) a += pre[k];
    for (unsigned i = lane + 32u * (unsigned)npre; i < np; i += 32u) a += partial_div[i];
    a = warp_sum(a);
    const double div = a / (N * S->eps);
    const double tau_r = S->tau_r;
    double tx = tau_r * div;
    const double fl = floor_rel * tau_r;
    const bool floored = !(tx >= fl);
    if (floored) tx = fl;
    if (record && lane == 0) {
        if (floored) S->floored += 1u;
        if (!isfinite(tx)) S->nonfinite += 1u;
        S->div = div;
        S->tau_x = tx;
        const unsigned tt = S->t;
        if (tt >= 1u && tt <= (unsigned)kMaxIters) {
            IterLog L;
            L.tau_x = tx;
            L.tau_p = S->tau_p;
            L.tau_s = S->tau_s;
            L.tau_r = tau_r;
            L.div = div;
            L.eps = S->eps;
            log[tt - 1] = L;
        }
        S->t = tt + 1u;
    }
    return tx;
}

// One measurement: s (damped against s_prev = sp) into sv; returns tau_s_i.
__device__ __forceinline__ float output_element(float zi, float sp, float yv, float tau_p, float inv_tp,
                                                float logI0, int onsager, float damp_s, int truncate,
                                                unsigned& capped, float& sv) {
    const float p = onsager ? fmaf(-tau_p, sp, zi) : zi;
    float d = mode_delta(p, yv, tau_p, inv_tp, logI0, capped);
    const bool clamp = truncate && p + d < 0.f;
    if (clamp) d = -p;
    sv = d * inv_tp;
    if (damp_s != 1.f) sv = damp_s * sv + (1.f - damp_s) * sp;
    const float w = expf(logI0 - p - d);
    return (clamp || isinf(w)) ? inv_tp : w / fmaf(tau_p, w, 1.f);
}

// The same measurement with the exact posterior moments of z instead of
// Laplace's (option output_moments = 1).  Relative to the mode z0 = p + d the
// log posterior is l(t) = -t^2 / (2 tau_p) - w0 (e^{-t} - 1 + t), w0 =
// I0 e^{-z0} (the mode condition cancels the linear terms): concave, l(0) =
// 0, l(t) <= -t^2 / (2 tau_p).  The window [t_lo, t_hi] where l >=
// -kExactLogCut on each side is found by bisection inside [0, +-sqrt(2 cut
// tau_p)]; mean and variance of t follow from the trapezoid rule on
// kExactPts points (the density is smooth, so the rule converges fast, and
// the window holds all but e^-50 of the mass whatever the skew).  Then
// s = (d + E[t]) / tau_p and tau_s_i = (1/tau_p)(1 - Var/tau_p).  The
// Poisson term is w0 (expm1(-t) + t) near the mode (|t| < 1) and
// exp(log w0 - t) + w0 (t - 1) away from it, which stays finite where w0
// underflows.
constexpr float kExactLogCut = 50.f;
constexpr int kExactPts = 257;

__device__ __forceinline__ float exact_logpost(float t, float inv_tp, float w0, float lw0) {
    const float poi = fabsf(t) < 1.f ? w0 * (expm1f(-t) + t) : expf(lw0 - t) + w0 * (t - 1.f);
    return -0.5f * t * t * inv_tp - poi;
}

__device__ __forceinline__ float exact_edge(float sign, float tau_p, float inv_tp, float w0, float lw0) {
    float lo = 0.f, hi = sign * sqrtf(2.f * kExactLogCut * tau_p);
    for (int k = 0; k < 40; ++k) {
        const float mid = 0.5f * (lo + hi);
        if (exact_logpost(mid, inv_tp, w0, lw0) > -kExactLogCut)
            lo = mid;
        else
            hi = mid;
    }
    return hi;
}

__device__ __forceinline__ float output_element_exact(float zi, float sp, float yv, float tau_p, float inv_tp,
                                                      float logI0, int onsager, float damp_s, unsigned& capped,
                                                      float& sv) {
    const float p = onsager ? fmaf(-tau_p, sp, zi) : zi;
    const float d = mode_delta(p, yv, tau_p, inv_tp, logI0, capped);
    const float lw0 = logI0 - p - d;                 // log of w0 = I0 e^{-z0}
    const float w0 = expf(lw0);
    const float t_lo = exact_edge(-1.f, tau_p, inv_tp, w0, lw0), t_hi = exact_edge(1.f, tau_p, inv_tp, w0, lw0);
    const float h = (t_hi - t_lo) / (float)(kExactPts - 1);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int k = 0; k < kExactPts; ++k) {
        const float t = fmaf((float)k, h, t_lo);
        float w = expf(exact_logpost(t, inv_tp, w0, lw0));
        if (k == 0 || k == kExactPts - 1) w *= 0.5f;
        s0 += w;
        s1 = fmaf(w, t, s1);
        s2 = fmaf(w * t, t, s2);
    }
    const float m1 = s1 / s0;
    const float var = fmaxf(s2 / s0 - m1 * m1, 0.f);
    sv = (d + m1) * inv_tp;
    if (damp_s != 1.f) sv = damp_s * sv + (1.f - damp_s) * sp;
    return inv_tp * (1.f - var * inv_tp);
}

// End of a grid that summed tau_s_i: each block stores its FP64 partial, the
// last block to arrive adds the partials in a fixed order, forms
// tau_s = sum / M and (inside a solve) tau_p, tau_s and tau_r = N /
// (||Phi~||_F^2 tau_s) for Step 3.  Every thread of the block must call it.
__device__ __forceinline__ void finish_tau_s(double acc, unsigned capped, long long M, double N,
                                             int from_scalars, DevScalars* S, double* partial,
                                             double* tau_s_out, double* sm) {
    __shared__ bool am_last;
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

}  // namespace dgct
