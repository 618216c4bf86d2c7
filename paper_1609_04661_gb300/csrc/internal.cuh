// Internal declarations of the GB300 D-GAMP-CT library: plan layout, device
// scalar block, and the small device helpers that several kernels share.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dgamp_ct.h"

namespace dgct {

constexpr int kPad = 4;            // zero guard cells on each side of a staged image line
constexpr int kMaxIters = 1 << 16; // bound on one solve's iteration count (log size)
constexpr int kNewtonCap = 64;     // output-step iteration cap
constexpr int kBatchStreams = 16;  // streams a batched solve spreads its slices over

// Joseph constants of one view.  The ray of bin d meets march line s (a
// column for col = 1, a row for col = 0) at fractional index
//   pos(d, s) = a0 + d a_det + s a_step
// across that line.  Positions are carried in 32.32 fixed point
// (P0 + d PDET + s PSTEP, 64-bit integers), so stepping along a ray is exact
// and the projector and the back-projector obtain bit-identical taps and
// weights however they evaluate the sum.  The float copies serve only to
// bound loops.
struct ViewConst {
    long long P0, PSTEP, PDET;    // a0, a_step, a_det scaled by 2^32
    long long AP;                 // |PDET|: ray spacing on a march line (>= 2^32)
    float a0, a_step, a_det, w;   // w = path length per step (1/|sin| or 1/|cos|)
    float inv_adet;               // 1 / a_det
    int col;                      // 1: march over columns, interpolate along rows
    int sg;                       // sign of PDET: +1 if position grows with d
    float inv_astep;              // 1 / a_step (0 when a_step is 0)
};

// Scalars of Algorithm 1 that live on the device for the whole solve.
struct DevScalars {
    double tau_x;       // tau_x^t (Step 4 of the previous iteration; 1 at start)
    double tau_p;       // Step 1
    double tau_s;       // Step 2
    double tau_r;       // Step 3
    double div;         // Step 4, D'
    double eps;         // MC step of Step 4
    double frob2;       // ||Phi~||_F^2
    double logI0;
    unsigned int rmax_bits;     // max |r| (float bits; |r| >= 0 so integer order works)
    unsigned int t;             // current iteration, 1-based
    unsigned int done_out;      // last-block counters
    unsigned int done_div;
    unsigned int newton_capped;
    unsigned int floored;
    unsigned int nonfinite;
    unsigned int div_pending;   // TV divergence partial sums left for the next output step (0: none)
    // denoiser 2 (learned, judged by prox-TV): the candidates' divergences
    // and SURE risk estimates of the current iteration, the kept one
    double div_plain, div_learned;
    double risk_plain, risk_learned;
    unsigned int keep_learned;  // 1: this iteration keeps the CNN's output
    unsigned int learned_kept;  // iterations of the solve that kept it
};

// The TV weight: lambda = c_tv sqrt(tau_r) inside a solve, the caller's lambda otherwise.
__device__ __forceinline__ float solve_lambda(const DevScalars* S, float c_tv, int from_scalars,
                                              float lambda_arg) {
    return from_scalars ? c_tv * sqrtf((float)S->tau_r) : lambda_arg;
}

// One fan-beam ray's Joseph constants (fanbeam.cu): its position on the
// interpolated axis at step s is pos = P0 + s PSTEP in 32.32 fixed point
// (the fractional row in column s when col = 1, the fractional column in row
// s otherwise), |PSTEP| <= 2^32; w is the path length per step.
struct FanRay {
    long long P0, PSTEP;
    float a0, a_step, w;
    int col;
};

// One fan-beam view: the detector axis e_u, the central direction e_c (the
// source sits at -dso e_c), the source-detector distance and the bin map
// bin(p) = dsd (p . e_u) / ((p . e_c + dso) du) + half.
struct FanView {
    float eux, euy, ecx, ecy, dso, dsd, du, half;
};

// Per-iteration log record (what dgamp_ct_stats exposes).
struct IterLog {
    double tau_x, tau_p, tau_s, tau_r, div, eps;
    double risk_plain = 0.0, risk_learned = 0.0;   // denoiser 2 only
    int keep_learned = 0;
};

// One slice of a batch (dgamp_ct_batch_*): its geometry, the device
// workspace of its plan, its options, the per-solve inputs and outputs, and
// where its blocks start in each phase's grid.  A batch runs every phase of
// an iteration as one launch over all slices; a block finds its slice in the
// phase's block -> slice table and its own block index from the offsets.
enum BatchPhase { kPhProj, kPhView, kPhBp, kPhProbe, kPhTv0, kPhTv1, kPhRow, kPhCol, kPhBegin, kPhases };
struct BatchSlice {
    int n, nv, nd, ldp, m2, P;
    long long N, M;
    void* XR;                  // staged image (FP32, or BF16 with storage = 1)
    void* XC;
    void* zraw;                // A x, s, H s (the storage type)
    void* s;
    void* hs;
    float* x;
    float* r;                  // r and r + eps b
    float* b;
    float* y;
    float2* p;                 // TV duals, ping-pong
    float2* fft2d;
    double* partial;
    double* partial_div;
    DevScalars* S;
    IterLog* log;
    const ViewConst* vc;
    const float* hx;
    const float2* tw2;
    float c_tv, eps_rel, damp_x, damp_s;
    double tau_x_floor, frob2, tau_x0;
    int onsager, truncate;
    uint2 key;
    unsigned slice_id;
    const float* counts;       // per solve
    float* mu_out;
    double logI0;
    int off[kPhases];          // first block of the slice in each phase's grid
};

struct Workspace {
    float* XR = nullptr;     // staged image, rows padded:  [n][ldp]
    float* XC = nullptr;     // staged transpose:            [n][ldp]
    float* x = nullptr;      // current x  [n][n]
    float* r = nullptr;      // r and r + eps b  [2][n][n]
    float2* p = nullptr;     // TV duals, ping-pong: [2 buffers][2 images][n][n]
    float* zraw = nullptr;   // A x           [M]
    float* z = nullptr;      // H A x         [M]
    float* s = nullptr;      // s (in place over s_prev) [M]
    float* hs = nullptr;     // H s           [M]
    float* y = nullptr;      // counts        [M]
    float2* fft2d = nullptr; // [2n][2n] complex scratch for V / V^-1
    double* partial = nullptr;     // block partial sums
    double* partial_div = nullptr; // the TV divergence's block partial sums inside a solve
    DevScalars* S = nullptr;
    IterLog* log = nullptr;        // [kMaxIters]
    ViewConst* vc = nullptr;       // [n_views]
    float* gain = nullptr;         // [P]
    float* hx = nullptr;           // [2 n_det - 1]  H's kernel h[|m|], m = -(n_det-1)..n_det-1
    float* zraw2 = nullptr;        // [M]  copy for in-place Toeplitz filtering
    float2* tw = nullptr;          // FFT twiddles for length P, stage by stage (fft_device.cuh)
    float2* tw2 = nullptr;         // the same for length m2
    double* scratch_d = nullptr;   // plan-time FP64 scratch
    float* b = nullptr;            // the iteration's probe b (Eq. MC_SURE) [n][n]
    FanRay* fan_rays = nullptr;    // fan-beam plans: [n_views][n_det]
    FanView* fan_views = nullptr;  // fan-beam plans: [n_views]
    int* pj_order = nullptr;       // banded A: views marching over rows, then over columns [n_views]
    float* pj_part = nullptr;      // banded A: per-band partial sums [ceil(n / 16)][n_views][n_det]
};

}  // namespace dgct

struct dgamp_ct_cnn_s;

struct dgamp_ct_plan_s {
    dgamp_ct_cnn_s* cnn = nullptr;         // learned denoiser (not owned), used when opt.denoiser is 1 or 2
    float* dn = nullptr;                   // [3][n][n]: its D(r), J_D(r) b; prox-TV's D(r) (denoiser 2)
    int device = 0;
    int n = 0, nv = 0, nd = 0, P = 0, logP = 0, m2 = 0, logm2 = 0, ldp = 0;
    int64_t N = 0, M = 0;
    double frob2 = 0.0;
    dgamp_ct_options opt{};
    dgct::Workspace ws;
    int max_partials = 0;
    int tv_kb = 5;                         // Chambolle steps per blocked TV launch
    int tv_rows = 64;                      // rows of a blocked TV region (32, 64 or 128)
    int tv_vrows = 4;                      // rows per thread of a TV region (4, or 8 with 64-row regions)
    int filter_mode = 0;                   // H by 0: FFT, 1: Toeplitz product (plan-time choice)
    int sino_fused = 0;                    // solve: H A x, output step, H s in one kernel (k_sino_step)
    int bp_mode = 0;                       // A^T: 0 pixel-driven gather, 1 ray-driven tiles (plan-time choice)
    int pj_seg = 8;                        // A: step segments (warps) per ray group, 8/16/32 (plan-time choice)
    int pj_band = 0;                       // A: 0 ray-group form; 16 or 32: lines per shared-memory band
    int pj_waves = 1;                      // A, banded form: full waves of blocks (1 or 2)
    int pj_c0 = 0, pj_c1 = 0;              // A, banded form: ray chunks per band of each orientation
    int pj_n0 = 0;                         // views that march over rows (the first pj_n0 of ws.pj_order)
    int fan = 0;                           // 1: flat-detector fan beam (dgamp_ct_plan_fan)
    int fan_stride = 0;                    // fan A^T tiles: ray stride of one pass (0: tiles not applicable)
    // captured iteration graph
    cudaGraphExec_t graph = nullptr;       // one iteration
    cudaGraphExec_t graph_k = nullptr;     // kGraphIters iterations (captured when a solve is that long)
    cudaStream_t graph_stream = nullptr;   // stream the graph was captured for (identity only)
    uint64_t graph_cnn_gen = 0;            // network workspace generation the graph was captured with
    int kernels_per_iter = 0;
};

namespace dgct {

// ---------------------------------------------------------------- helpers --
// Storage of the solve's sinograms and staged images: float, or BF16 with
// every sum in FP32 (option storage = 1).
typedef __nv_bfloat16 bf16s;
__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const bf16s* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(bf16s* p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ long long joseph_pos(const ViewConst& c, int d, int s) {
    return c.P0 + (long long)d * c.PDET + (long long)s * c.PSTEP;
}

// Steps of a ray (position `base` at s = 0, `a_step` per step) whose taps can
// touch the image: pos in [-1, n) widened by one step each way (|a_step| <= 1,
// so the taps of the extra steps stay inside the zero guard cells).
__device__ __forceinline__ void step_range(float base, float a_step, int n, int& s0, int& s1) {
    if (fabsf(a_step) < 1e-12f) {
        if (base >= -1.f && base < (float)n) { s0 = 0; s1 = n - 1; } else { s0 = 1; s1 = 0; }
        return;
    }
    float t0 = (-1.f - base) / a_step, t1 = ((float)n - base) / a_step;
    float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
    lo = fmaxf(lo, -1.f);
    hi = fminf(hi, (float)n);
    s0 = max(0, (int)floorf(lo) - 1);
    s1 = min(n - 1, (int)ceilf(hi) + 1);
}

// step_range with the reciprocal of a_step in place of two divisions.  The
// bounds may move by a rounding error of the reciprocal, well inside the
// one-step widening, so the range still holds every step with a tap in the
// image, and any extra step's taps fall in the zero guard cells (adding an
// exact 0).
__device__ __forceinline__ void step_range_rcp(float base, float a_step, float inv_astep, int n, int& s0, int& s1) {
    if (fabsf(a_step) < 1e-12f) {
        if (base >= -1.f && base < (float)n) { s0 = 0; s1 = n - 1; } else { s0 = 1; s1 = 0; }
        return;
    }
    float t0 = (-1.f - base) * inv_astep, t1 = ((float)n - base) * inv_astep;
    float lo = fminf(t0, t1), hi = fmaxf(t0, t1);
    lo = fmaxf(lo, -1.f);
    hi = fminf(hi, (float)n);
    s0 = max(0, (int)floorf(lo) - 1);
    s1 = min(n - 1, (int)ceilf(hi) + 1);
}

// Split a 32.32 position into its left tap (floor) and the fraction in [0, 1):
// the fraction's top 23 bits become the mantissa of a float in [1, 2), so no
// int-to-float conversion is needed (truncation error < 2^-23).
__device__ __forceinline__ void joseph_tap(long long pos, int& i0, float& f) {
    i0 = (int)(pos >> 32);
    f = __uint_as_float(0x3F800000u | ((unsigned)pos >> 9)) - 1.0f;
}

// Nearest integer of |x| < 2^22 without a float-to-int conversion.
__device__ __forceinline__ int round_magic(float x) {
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block (any size that is a multiple of 32, <= 1024); result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem32) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int l = tid & 31, w = tid >> 5;
    v = warp_sum(v);
    if (l == 0) smem32[w] = v;
    __syncthreads();
    T out = T(0);
    if (w == 0) {
        out = (l < nw) ? smem32[l] : T(0);
        out = warp_sum(out);
    }
    __syncthreads();
    return out;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Four probe normals of block g for iteration t (Box-Muller on word pairs).
__device__ __forceinline__ float4 probe4(unsigned g, unsigned t, unsigned slice, uint2 key) {
    uint4 w = philox4x32_10(make_uint4(g, t, slice, 0u), key);
    const float s32 = 2.3283064365386963e-10f;  // 2^-32
    float u0 = fmaf(__uint2float_rn(w.x), s32, 0.5f * s32);
    float u1 = fmaf(__uint2float_rn(w.y), s32, 0.5f * s32);
    float u2 = fmaf(__uint2float_rn(w.z), s32, 0.5f * s32);
    float u3 = fmaf(__uint2float_rn(w.w), s32, 0.5f * s32);
    u0 = fminf(u0, 1.0f);
    u2 = fminf(u2, 1.0f);
    float r01 = sqrtf(-2.0f * logf(u0));
    float r23 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    return make_float4(r01 * c1, r01 * s1, r23 * c3, r23 * s3);
}

// Launch-error check used by every launcher.
int cuda_fail(cudaError_t e);
#define DGCT_LAUNCH_CHECK()                                        \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::dgct::cuda_fail(_e);       \
    } while (0)
#define DGCT_TRY(x)                                                \
    do {                                                           \
        int _rc = (x);                                             \
        if (_rc != DGAMP_CT_OK) return _rc;                        \
    } while (0)
#define DGCT_CUDA(call)                                            \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::dgct::cuda_fail(_e);       \
    } while (0)

// Programmatic dependent launch of the iteration's kernels.  A kernel
// launched this way is set up by the hardware while the kernel before it in
// the stream is still finishing; its blocks may load what no kernel of the
// iteration writes (launch parameters, view constants, batch descriptors,
// the filter), and pdl_wait() returns once every earlier kernel of the
// stream has completed and its writes are visible.  Nothing the iteration
// writes is read or written before that.  No kernel signals its dependents
// early (griddepcontrol.launch_dependents): letting the next kernel's blocks
// onto the SMs during a kernel's last wave made the iteration 7% slower,
// while the launch at completion gains about 1%.  pdl_wait() is a no-op for
// a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

inline cudaError_t launch_pdl_c(const void* kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                void** args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

// typed form: launch_pdl(kernel, grid, block, smem, stream, kernel arguments...)
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// api.cu: copy the last solve's log and counters to *stats (work must be complete)
int fill_stats(const dgamp_ct_plan_s* pl, int iters, dgamp_ct_stats* stats);

// ----------------------------------------------------------- launchers ----
// joseph.cu
// bf = 1: the staged image XR/XC and the sinogram `sino` hold BF16 (solve with storage = 1)
int launch_stage_image(const dgamp_ct_plan_s* pl, const float* img, cudaStream_t st, int bf = 0);
// sum = false (banded form only): leave A x as band partials in ws.pj_part
// for the cluster sinogram kernel, which adds them itself
int launch_project(const dgamp_ct_plan_s* pl, float* sino, cudaStream_t st, int bf = 0, bool sum = true);
// inside a solve the cluster sinogram kernel adds the banded projector's partials
inline bool project_sum_in_sino(const dgamp_ct_plan_s* pl) {
    return pl->pj_band && pl->sino_fused == 2 && !pl->opt.output_moments && !pl->fan;
}
int backproject_autotune(dgamp_ct_plan_s* pl);
int project_autotune(dgamp_ct_plan_s* pl);
int project_band_smem(const dgamp_ct_plan_s* pl, int BR);
int project_band_chunks(dgamp_ct_plan_s* pl);
int launch_backproject(const dgamp_ct_plan_s* pl, const float* sino, const float* x_in,
                       float* out, int update, cudaStream_t st, int bf = 0, int nparts = 0);
int launch_frobenius(dgamp_ct_plan_s* pl);
// fft.cu
int launch_filter(const dgamp_ct_plan_s* pl, const float* in, float* out, cudaStream_t st, int bf = 0);
// Raises a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowering it: the limit belongs to the kernel in the whole context, and a
// plan made earlier may launch it with more.
int raise_smem_limit(const void* kernel, int bytes);
bool sino_step_eligible(const dgamp_ct_plan_s* pl);      // the FFT form (sino_fused = 1) applies
bool sino_toeplitz_eligible(const dgamp_ct_plan_s* pl);  // the cluster Toeplitz form (sino_fused = 2) applies
int sino_autotune(dgamp_ct_plan_s* pl);
int sino_step_set_smem_limit(const dgamp_ct_plan_s* pl);
int launch_sino_step(const dgamp_ct_plan_s* pl, cudaStream_t st, int bf);
int sino_step_partials(const dgamp_ct_plan_s* pl);   // FP64 partial sums of tau_s_i it leaves in ws.partial
int launch_precond_image(const dgamp_ct_plan_s* pl, const float* in, float* out, int inverse,
                         cudaStream_t st);
// the same on nimg images at once ([nimg][n][n]) through the caller's scratch C ([nimg][n][m2] complex)
int launch_precond_images(const dgamp_ct_plan_s* pl, const float* in, float* out, float2* C, int nimg, int inverse,
                          cudaStream_t st);
int fft_set_smem_limits(int bytes);
// r = x + tau_r V^-1 in (tau_r from S), max |r| into S (a fan-beam solve's Step 3)
int launch_precond_image_update(const dgamp_ct_plan_s* pl, const float* in, const float* x, float* out,
                                cudaStream_t st);
int filter_autotune(dgamp_ct_plan_s* pl);
int toeplitz_set_smem_limit(int nd);
// output_step.cu
int launch_output_step(const dgamp_ct_plan_s* pl, const float* z, const float* y, float* s,
                       int use_prev, int from_scalars, double tau_p_arg, double logI0_arg,
                       double* tau_s_out, cudaStream_t st, int bf = 0);
// tv.cu
int launch_probe_input(const dgamp_ct_plan_s* pl, int t_arg, cudaStream_t st, int write_b = 0);
int launch_absmax(const dgamp_ct_plan_s* pl, const float* r, cudaStream_t st);
bool tv_active(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg);
int tv_num_launches(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg);
int tv_set_smem_limits();
int tv_autotune(dgamp_ct_plan_s* pl);
int launch_tv_chunk(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                    float* x_out, int solve_mode, int t_arg, double* div_out, cudaStream_t st);
int launch_tv(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, float* x_out,
              int solve_mode, int t_arg, double* div_out, cudaStream_t st);
int launch_probe(const dgamp_ct_plan_s* pl, unsigned t, int64_t n, float* b, uint32_t* words,
                 cudaStream_t st);
// the TV final step on images the caller has already formed (xbase, nimg of them, [n][n]
// each): x of image 0 (damped in a solve) to x_out, staged copies, divergence, tau_x
int launch_tv_final_x(const dgamp_ct_plan_s* pl, int nimg, const float* xbase, float* x_out, int solve_mode,
                      int t_arg, double* div_out, cudaStream_t st);
// tv_metric.cu: prox-TV in the (V^T V)^{-1} norm (option tv_metric)
int tvm_num_launches(const dgamp_ct_plan_s* pl);
int launch_tvm_chunk(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                     float* x_out, int solve_mode, int t_arg, double* div_out, cudaStream_t st);
int tvm_set_smem_limits(int bytes);
// fanbeam.cu: flat-detector fan-beam A, A^T and ||A V^-1||_F^2
int fan_setup(dgamp_ct_plan_s* pl, const std::vector<double>& ang, double src_dist, double det_dist,
              double det_spacing);
int launch_fan_project(const dgamp_ct_plan_s* pl, float* sino, cudaStream_t st);
int launch_fan_backproject(const dgamp_ct_plan_s* pl, const float* sino, float* img, cudaStream_t st);
// x, staging, divergence and tau_x from D(r) and J_D(r) b (learned denoiser)
int launch_denoise_final(const dgamp_ct_plan_s* pl, const float* dn, float* x_out, int solve_mode, int t_arg,
                         double* div_out, cudaStream_t st);
// denoiser 2: part 0 forms both candidates' SURE risk estimates and keeps one,
// part 1 writes the kept output as x, the staged copies, tau_x and the log
int launch_select(const dgamp_ct_plan_s* pl, int part, cudaStream_t st);
// Batched execution (batch.cu): device descriptors and tables of a batch,
// and the grid of each phase (blocks; clusters for kPhView)
struct BatchExec {
    BatchSlice* sl = nullptr;                    // device [ns]
    uint16_t* map[kPhases] = {};                 // device: block -> slice
    int nblk[kPhases] = {};
    int ns = 0;
    int bf = 0;                                  // BF16 storage
    int R = 3;                                   // bins per lane of the cluster sinogram kernel
    int cl = 8;                                  // its CTAs per view (4 or 8)
    int ct_smem = 0;                             // its dynamic shared memory (largest slice)
    int max_m2 = 0;                              // largest V^-1 FFT length
};
// joseph.cu (pj_seg 16, tile back-projection)
constexpr int kBatchPjSeg = 16;
constexpr int kBatchTvKb = 10;                   // Chambolle steps per batched TV launch
int batch_grid_project(int nv, int nd);
int batch_grid_backproject(int n);
int launch_project_batch(const BatchExec& E, cudaStream_t st);
int launch_backproject_batch(const BatchExec& E, cudaStream_t st);
// sino_step.cu (cluster Toeplitz form)
int sino_ct_config(int nd, int* cl);             // bins per lane (0: n_det too large), CTAs per view
int sino_ct_smem_bytes(int nd, int R, int cl);
int launch_sino_batch(const BatchExec& E, cudaStream_t st);
// tv.cu (64-row regions, kBatchTvKb steps per launch; `launch` counts from 0)
int batch_grid_tv(int n, int final_launch);
int batch_grid_probe(long long N);
int launch_probe_batch(const BatchExec& E, cudaStream_t st);
int launch_tv_batch(const BatchExec& E, int launch, bool final_launch, cudaStream_t st);

// cnn.cu
int cnn_prepare_pair(dgamp_ct_cnn_s* c, int n);
int cnn_denoise_jvp(dgamp_ct_cnn_s* c, const float* rb, const DevScalars* S, int n, float* out, int scaled,
                    cudaStream_t st);
int cnn_launches_per_pair(const dgamp_ct_cnn_s* c);
// conv_tc.cu: hidden 64 -> 64 layers on tcgen05 (mode 0: bias + ReLU, mode 1: masked linear)
int conv64_tc_init();
// stall_ns > 0: the timeout test (the kernel waits that long on a barrier nothing
// arrives at, sets *err and computes nothing)
int launch_conv64_tc(int mode, const void* in, const void* wk_all, int layers, int layer, const float* bias,
                     const void* mask, void* out, int B, int H, int W, int grid_cap, unsigned* err, cudaStream_t st,
                     unsigned long long stall_ns = 0);
// weight gradient of a hidden layer on tcgen05: partial[groups][9][ci][co]
int launch_wgrad64_tc(const void* a, const void* g, int B, int H, int W, int groups, float* partial, unsigned* err,
                      cudaStream_t st, unsigned long long stall_ns = 0);
// after the network's work is complete: DGAMP_CT_ERR_TIMEOUT (and the flag cleared)
// if a tensor-core convolution's bounded wait ran out since the last check
int cnn_take_timeout(dgamp_ct_cnn_s* c);
// changes whenever the network's workspace is reallocated (captured graphs hold its pointers)
uint64_t cnn_ws_generation(const dgamp_ct_cnn_s* c);

}  // namespace dgct
