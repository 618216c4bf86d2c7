// Poisson output step, Algorithm 1 Step 2 (Section 4.2, Appendix A), as a
// stand-alone kernel over a whole sinogram; the arithmetic is in
// output_device.cuh.
#include "output_device.cuh"

namespace dgct {

template <typename T>
__global__ void __launch_bounds__(256)
k_output_step(const T* z, const float* y, T* s, long long M, int use_prev,
              int from_scalars, double tau_p_arg, double logI0_arg, int onsager, float damp_s,
              int truncate, double N, DevScalars* S, double* partial, double* tau_s_out,
              const double* partial_div, double floor_rel, IterLog* log, int exact) {
    __shared__ double sm[32];
    __shared__ float s_tp, s_inv, s_logI0;
    if (threadIdx.x < 32) {
        const double tx = from_scalars ? pending_tau_x(S, partial_div, N, floor_rel, log, blockIdx.x == 0) : 0.0;
        if (threadIdx.x == 0) {
            const double tp = from_scalars ? S->frob2 * tx / (double)M : tau_p_arg;
            s_tp = (float)tp;
            s_inv = (float)(1.0 / tp);
            s_logI0 = (float)(from_scalars ? S->logI0 : logI0_arg);
        }
    }
    __syncthreads();
    const float tau_p = s_tp, inv_tp = s_inv, logI0 = s_logI0;
    double acc = 0.0;
    unsigned capped = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (long long)gridDim.x * blockDim.x) {
        const float sp = use_prev ? ldf(s + i) : 0.f;
        float sv;
        acc += exact ? (double)output_element_exact(ldf(z + i), sp, y[i], tau_p, inv_tp, logI0, onsager, damp_s,
                                                    capped, sv)
                     : (double)output_element(ldf(z + i), sp, y[i], tau_p, inv_tp, logI0, onsager, damp_s, truncate,
                                              capped, sv);
        stf(s + i, sv);
    }
    finish_tau_s(acc, capped, M, N, from_scalars, S, partial, tau_s_out, sm);
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
                                                     (double)pl->N, pl->ws.S, pl->ws.partial, tau_s_out,
                                                     pl->ws.partial_div, pl->opt.tau_x_floor, pl->ws.log,
                                                     pl->opt.output_moments);
    else
        k_output_step<float><<<blocks, 128, 0, st>>>(z, y, s, M, use_prev, from_scalars, tau_p_arg, logI0_arg,
                                                     onsager, damp_s, pl->opt.truncate_z, (double)pl->N, pl->ws.S,
                                                     pl->ws.partial, tau_s_out, pl->ws.partial_div,
                                                     pl->opt.tau_x_floor, pl->ws.log, pl->opt.output_moments);
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
                                                      partial, tau_s_out, nullptr, 0.0, nullptr, 0);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
