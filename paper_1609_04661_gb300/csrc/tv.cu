// Denoiser and divergence, Algorithm 1 Step 4 (Section 4.3, Section 6.3).
//
// D is the l2 proximal map of isotropic TV, solved by Chambolle's 2004 dual
// projection (forward differences, Neumann boundary, step 1/8, a fixed
// number of iterations from a zero dual).  The MC divergence of Eq. MC_SURE
// with one probe needs D at r and at r + eps b; both images are denoised by
// the same blocks, and the last launch forms x = D(r) and b^T (D(r+eps b) - D(r))
// in FP64; tau_x = max(tau_r D', floor tau_r) follows from it (inside a solve
// in the next iteration's output step, see output_device.cuh).
//
// Temporal blocking.  One Chambolle step updates p at a pixel from p within
// one pixel of it:
//   q = div p - r/lambda,  div p = px(i,j) - px(i,j-1) + py(i,j) - py(i-1,j)
//   p <- (p + tau grad q) / (1 + tau |grad q|),  grad q uses q(i,j+1), q(i+1,j)
// so a block that holds a region of the image runs KB steps with no global
// traffic while the valid part shrinks by one pixel per side per step, and
// writes back the region minus KB pixels on each side.  The region lives in
// registers (see k_tv_steps).  Duals outside the image stay zero, and
// grad q is zero on the last row/column (Neumann), which reproduces the
// boundary rules exactly.  Successive launches exchange duals through
// ping-pong global buffers [image][n][n] of float2; a last launch forms
// x = r - lambda div p and the divergence.  KB and the region height are
// chosen per plan by timing (tv_autotune).
#include <vector>

#include "internal.cuh"

namespace dgct {

constexpr int TB = 32;             // pixel tile edge of the final step
constexpr int kTvMaxKb = 10;       // most Chambolle steps one launch may run
constexpr float kTau = 0.125f;

// --------------------------------------------------------- probe input ----
// r2 = r + eps b, eps = eps_rel max(max|r|, 1e-6), or r2 = b itself
// (write_b = 1: the direction of a forward-mode divergence); b itself also
// to bout for the divergence sum.  One thread per group of four probe
// elements (one Philox call): group g below.
__device__ __forceinline__ void probe_group(const float* __restrict__ r, float* __restrict__ r2,
                                            float* __restrict__ bout, long long N, float eps_rel, int t_arg,
                                            unsigned slice, uint2 key, DevScalars* S, int write_b, long long g) {
    pdl_wait();      // r and the scalars are the previous kernels' output
    const float rmax = __uint_as_float(S->rmax_bits);
    const float eps = eps_rel * fmaxf(rmax, 1e-6f);
    const unsigned t = t_arg > 0 ? (unsigned)t_arg : S->t;
    if (g == 0) S->eps = (double)eps;
    const long long i0 = 4 * g;
    if (i0 >= N) return;
    const float4 b = probe4((unsigned)g, t, slice, key);
    const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < N) {
            r2[i0 + k] = write_b ? bb[k] : fmaf(eps, bb[k], r[i0 + k]);
            bout[i0 + k] = bb[k];
        }
}

__global__ void k_probe_input(const float* __restrict__ r, float* __restrict__ r2, float* __restrict__ bout,
                              long long N, float eps_rel, int t_arg, unsigned slice, uint2 key,
                              DevScalars* S, int write_b) {
    probe_group(r, r2, bout, N, eps_rel, t_arg, slice, key, S, write_b,
                (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// r + eps b beside r for every slice of a batch (prox-TV), 256 groups per block.
__global__ void __launch_bounds__(256) k_probe_input_batch(const BatchSlice* __restrict__ sl,
                                                           const uint16_t* __restrict__ map) {
    const BatchSlice& B = sl[map[blockIdx.x]];
    const long long g = (long long)((int)blockIdx.x - B.off[kPhProbe]) * blockDim.x + threadIdx.x;
    probe_group(B.r, B.r + B.N, B.b, B.N, B.eps_rel, 0, B.slice_id, B.key, B.S, 0, g);
}

static uint2 probe_key(const dgamp_ct_plan_s* pl) {
    return make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
}

int launch_probe_input(const dgamp_ct_plan_s* pl, int t_arg, cudaStream_t st, int write_b) {
    const long long N = pl->N;
    const long long groups = (N + 3) / 4;
    DGCT_CUDA(launch_pdl(k_probe_input, dim3((unsigned)((groups + 255) / 256)), dim3(256), 0, st,
                         (const float*)pl->ws.r, pl->ws.r + N, pl->ws.b, N, (float)pl->opt.eps_rel, t_arg,
                         (unsigned)pl->opt.slice_id, probe_key(pl), pl->ws.S, write_b));
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

// ------------------------------------------- register-blocked Chambolle ----
struct TvFinal;
__device__ __forceinline__ void stage_store(float* base, int xbf, size_t idx, float v) {
    if (xbf)
        stf(reinterpret_cast<bf16s*>(base) + idx, v);
    else
        base[idx] = v;
}

struct TvFinal {
    float* x_out;          // D(r) (with damping against the old x in a solve)
    float* XR;             // staged copies for the next projection (nullable)
    float* XC;
    int ldp;
    int xbf;               // staged copies in BF16 (a solve with storage = 1)
    float damp_x;
    int t_arg;             // probe iteration (0: from S)
    unsigned slice;
    uint2 key;
    double tau_x_floor;
    double* partial;
    double* partial_div;   // a solve's divergence partials, finished by the next output step
    IterLog* log;
    double* div_out;       // nullable
    int solve_mode;        // 1: update tau_x, the log and t in S
    int jvp;               // learned denoiser: dn[1] is J_D b (divergence b^T J_D b / N)
};

// A block holds a region of kTvRW = 64 columns by RH = 4 WY rows of one image
// in registers: thread (warp w, lane l) owns rows 4w..4w+3 of the adjacent
// columns 2l and 2l + 1.  A horizontal neighbour is the thread's own other
// column or, once per row and direction, a warp shuffle from the next lane;
// vertical neighbours come from the thread's own registers except across
// warps, where the first row's q and the last row's py pass through shared
// memory (two barriers per step).  After KB steps the
// region minus KB pixels on each side holds exact duals and is written back.
constexpr int kTvU = 2;            // columns per thread
constexpr int kTvV = 4;            // rows per thread
constexpr int kTvRW = 32 * kTvU;   // region width
constexpr int kTvRowsBatch = 64;   // region height of the batched launches

// PTX sqrt.approx / rcp.approx (flush-to-zero): one special-function
// instruction each, accurate to a few ulp, well inside the 1e-5 the TV
// parity tests hold against the FP64 oracle.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int WY, int KB, bool BORDER, int V = kTvV>
__device__ __forceinline__ void tv_region_steps(float (&px)[V][kTvU], float (&py)[V][kTvU],
                                                const float (&rl)[V][kTvU], unsigned inside, unsigned lastc,
                                                unsigned lastr, float (*e_py)[kTvU][32], float (*e_q)[kTvU][32]) {
    constexpr int U = kTvU;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float q[V][U];
#pragma unroll
    for (int u = 0; u < U; ++u) e_py[w][u][lane] = py[V - 1][u];
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < KB; ++k) {
        // q = div p - r / lambda  (zero outside the image)
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float pxl;
                if (u > 0) {
                    pxl = px[v][u - 1];
                } else {
                    const float t = __shfl_up_sync(0xffffffffu, px[v][U - 1], 1);
                    pxl = lane > 0 ? t : 0.f;
                }
                const float pyu = v > 0 ? py[v - 1][u] : (w > 0 ? e_py[w - 1][u][lane] : 0.f);
                float qq = (px[v][u] - pxl + py[v][u] - pyu) - rl[v][u];
                if (BORDER && !((inside >> (v * U + u)) & 1u)) qq = 0.f;
                q[v][u] = qq;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) e_q[w][u][lane] = q[0][u];
        __syncthreads();
        // p <- (p + tau grad q) / (1 + tau |grad q|)  (grad q = 0 across the last row/column)
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float qr;
                if (u + 1 < U) {
                    qr = q[v][u + 1];
                } else {
                    const float t = __shfl_down_sync(0xffffffffu, q[v][0], 1);
                    qr = lane < 31 ? t : 0.f;
                }
                const float qd = v + 1 < V ? q[v + 1][u] : (w + 1 < WY ? e_q[w + 1][u][lane] : 0.f);
                float gx = qr - q[v][u];
                float gy = qd - q[v][u];
                bool upd = true;
                if (BORDER) {
                    const int bit = v * U + u;
                    upd = (inside >> bit) & 1u;
                    if ((lastc >> bit) & 1u) gx = 0.f;
                    if ((lastr >> bit) & 1u) gy = 0.f;
                }
                if (upd) {
                    // |grad q| and 1 / (1 + tau |grad q|) by the hardware's approximate
                    // square root and reciprocal (sqrt(0) = 0; the denominator is >= 1)
                    const float g2 = fmaf(gx, gx, gy * gy);
                    const float nrm = sqrt_approx(g2);
                    const float inv = rcp_approx(fmaf(kTau, nrm, 1.f));
                    px[v][u] = fmaf(kTau, gx, px[v][u]) * inv;
                    py[v][u] = fmaf(kTau, gy, py[v][u]) * inv;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) e_py[w][u][lane] = py[V - 1][u];
        __syncthreads();
    }
}

// Divergence sum of one block (FP64, any image) -> partial[bid]; the last
// block to arrive forms D' = (sum of partials) / (N eps) and, in a solve,
// tau_x = max(tau_r D', floor tau_r), the log record and the next t.
__device__ __forceinline__ void tv_divergence_finish(double acc, int nblk, int bid, size_t N, DevScalars* S,
                                                     const TvFinal& F, double* red, bool* am_last) {
    const int tid = threadIdx.x;
    acc = block_sum(acc, red);
    if (tid == 0) {
        F.partial[bid] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_div, 1u);
        *am_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!*am_last) return;
    __threadfence();
    double tot = 0.0;
    for (int b = tid; b < nblk; b += blockDim.x) tot += ((volatile double*)F.partial)[b];
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

// KB Chambolle steps of image blockIdx.z (of nimg) from the duals pin (zero
// when first).  Not FINAL: the region minus KB pixels per side goes to pout.
// FINAL: x = r - lambda div p on the region minus KB + 1 pixels at the top
// and left (div p reads the left and upper neighbours) and KB at the bottom
// and right; image 0's x (damped in a solve) to x_out and the staged
// copies; for nimg = 2 the divergence b^T (x_1 - x_0) / (N eps), summed as
// +b^T x_1 and -b^T x_0 over the blocks of the two images -- inside a solve
// left as FP64 block partials that the next output step adds (it needs tau_x
// first), elsewhere finished by the last block.
template <int WY>
struct TvShared {
    float e_py[WY][kTvU][32];
    float e_q[WY][kTvU][32];
    double red[32];
    bool am_last;
};

// Region (bx, by) of image bz of a launch whose grid is gx x gy x gz.
template <int WY, int KB, bool FINAL, int V = kTvV>
__device__ __forceinline__ void tv_steps_block(const float* __restrict__ rbase, const float2* __restrict__ pin,
                                               float2* __restrict__ pout, int n, int first, float c_tv,
                                               int from_scalars, float lambda_arg, DevScalars* S,
                                               const float* __restrict__ bprobe, const TvFinal& F, int bx, int by,
                                               int bz, int gx, int gy, int gz, TvShared<WY>& sh) {
    constexpr int U = kTvU, RW = kTvRW, RH = V * WY;
    constexpr int E = FINAL ? KB + 1 : KB;      // top/left margin of the tile
    constexpr int TW = RW - KB - E, TH = RH - KB - E;
    auto& e_py = sh.e_py;
    auto& e_q = sh.e_q;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t N = (size_t)n * n;
    const int im = bz;
    const size_t img = (size_t)im * N;
    const int gi0 = by * TH - E, gj0 = bx * TW - E;
    pdl_wait();      // r, the duals and the scalars are earlier kernels' output
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const float inv_lam = lam > 0.f ? 1.0f / lam : 0.f;
    float px[V][U], py[V][U], rl[V][U];
    unsigned inside = 0u, lastc = 0u, lastr = 0u;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int gi = gi0 + w * V + v;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int gj = gj0 + U * lane + u;
            const bool in = gi >= 0 && gi < n && gj >= 0 && gj < n;
            float rv = 0.f;
            float2 p = make_float2(0.f, 0.f);
            if (in) {
                const size_t o = img + (size_t)gi * n + gj;
                rv = rbase[o];
                if (!first) p = pin[o];
            }
            rl[v][u] = rv * inv_lam;
            px[v][u] = p.x;
            py[v][u] = p.y;
            const unsigned bit = 1u << (v * U + u);
            if (in) inside |= bit;
            if (gj == n - 1) lastc |= bit;
            if (gi == n - 1) lastr |= bit;
        }
    }
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + RH < n && gj0 + RW < n;
    if (interior)
        tv_region_steps<WY, KB, false, V>(px, py, rl, inside, lastc, lastr, e_py, e_q);
    else
        tv_region_steps<WY, KB, true, V>(px, py, rl, inside, lastc, lastr, e_py, e_q);
    if (!FINAL) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr = w * V + v;
            if (rr < KB || rr >= RH - KB) continue;
            const int gi = gi0 + rr;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int cc = U * lane + u;
                const int gj = gj0 + cc;
                if (cc < KB || cc >= RW - KB || gi >= n || gj >= n) continue;
                pout[img + (size_t)gi * n + gj] = make_float2(px[v][u], py[v][u]);
            }
        }
        return;
    }
    // ---- final: x = r - lambda div p (e_py holds the last rows' py) ----
    auto& red = sh.red;
    auto& am_last = sh.am_last;
    const int nimg = gz;
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int rr = w * V + v;
        const int gi = gi0 + rr;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float pxl;
            if (u > 0) {
                pxl = px[v][u - 1];
            } else {
                const float t = __shfl_up_sync(0xffffffffu, px[v][U - 1], 1);
                pxl = lane > 0 ? t : 0.f;
            }
            const float pyu = v > 0 ? py[v - 1][u] : (w > 0 ? e_py[w - 1][u][lane] : 0.f);
            const int cc = U * lane + u;
            const int gj = gj0 + cc;
            if (rr < E || rr >= RH - KB || cc < E || cc >= RW - KB || gi >= n || gj >= n) continue;
            const size_t o = (size_t)gi * n + gj;
            const float dv = px[v][u] - pxl + py[v][u] - pyu;
            const float xv = rbase[img + o] - lam * dv;
            if (nimg == 2) acc += (double)bprobe[o] * (double)(im == 1 ? xv : -xv);
            if (im == 0) {
                float xo = xv;
                if (F.solve_mode && F.damp_x != 1.f) xo = F.damp_x * xo + (1.f - F.damp_x) * F.x_out[o];
                F.x_out[o] = xo;
                if (F.XR) stage_store(F.XR, F.xbf, (size_t)gi * F.ldp + kPad + gj, xo);
                if (F.XC) stage_store(F.XC, F.xbf, (size_t)gj * F.ldp + kPad + gi, xo);
            }
        }
    }
    if (nimg < 2) return;
    const int nblk = gx * gy * gz;
    const int bid = (bz * gy + by) * gx + bx;
    if (F.solve_mode) {
        // inside a solve the next output step adds the partials (it needs
        // tau_x first): no grid-wide tail here
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) {
            F.partial_div[bid] = acc;
            if (bid == 0) S->div_pending = (unsigned)nblk;
        }
        return;
    }
    tv_divergence_finish(acc, nblk, bid, N, S, F, red, &am_last);
}

template <int WY, int KB, bool FINAL, int V = kTvV>
__global__ void __launch_bounds__(32 * WY)
k_tv_steps(const float* __restrict__ rbase, const float2* __restrict__ pin, float2* __restrict__ pout, int n,
           int first, float c_tv, int from_scalars, float lambda_arg, DevScalars* S,
           const float* __restrict__ bprobe, TvFinal F) {
    __shared__ TvShared<WY> sh;
    tv_steps_block<WY, KB, FINAL, V>(rbase, pin, pout, n, first, c_tv, from_scalars, lambda_arg, S, bprobe, F,
                                     blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z, sh);
}

// ---------------------------------------- both images in one thread ----
// The two images of the MC pair (r and r + eps b) take the same steps on
// the same pixels, so one thread can hold both: every value is a pair
// (image 0, image 1) and the dual step's additions and multiplications run
// as packed FP32 pairs (one instruction for both images, sm_100 and later).
// Each lane of a pair is rounded exactly as the one-image kernel rounds it
// (a - b as fma(b, -1, a) is the same correctly rounded difference), so the
// duals and x are bit-identical to the one-image form; only the FP64
// divergence sum, b (x_1 - x_0) per pixel here, adds in another order.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 shfl_up2(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

template <int WY>
struct TvShared2 {
    float2 e_py[WY][kTvU][32];
    float2 e_q[WY][kTvU][32];
    double red[32];
    bool am_last;
};

template <int WY, int KB, bool BORDER, int V>
__device__ __forceinline__ void tv_region_steps2(float2 (&px)[V][kTvU], float2 (&py)[V][kTvU],
                                                 const float2 (&rl)[V][kTvU], unsigned inside, unsigned lastc,
                                                 unsigned lastr, float2 (*e_py)[kTvU][32], float2 (*e_q)[kTvU][32]) {
    constexpr int U = kTvU;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float2 zero = make_float2(0.f, 0.f), tau = make_float2(kTau, kTau), one = make_float2(1.f, 1.f);
    float2 q[V][U];
#pragma unroll
    for (int u = 0; u < U; ++u) e_py[w][u][lane] = py[V - 1][u];
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < KB; ++k) {
        // q = div p - r / lambda  (zero outside the image)
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float2 pxl;
                if (u > 0) {
                    pxl = px[v][u - 1];
                } else {
                    const float2 t = shfl_up2(px[v][U - 1], 1);
                    pxl = lane > 0 ? t : zero;
                }
                const float2 pyu = v > 0 ? py[v - 1][u] : (w > 0 ? e_py[w - 1][u][lane] : zero);
                float2 qq = sub2(sub2(add2(sub2(px[v][u], pxl), py[v][u]), pyu), rl[v][u]);
                if (BORDER && !((inside >> (v * U + u)) & 1u)) qq = zero;
                q[v][u] = qq;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) e_q[w][u][lane] = q[0][u];
        __syncthreads();
        // p <- (p + tau grad q) / (1 + tau |grad q|)  (grad q = 0 across the last row/column)
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float2 qr;
                if (u + 1 < U) {
                    qr = q[v][u + 1];
                } else {
                    const float2 t = shfl_down2(q[v][0], 1);
                    qr = lane < 31 ? t : zero;
                }
                const float2 qd = v + 1 < V ? q[v + 1][u] : (w + 1 < WY ? e_q[w + 1][u][lane] : zero);
                float2 gx = sub2(qr, q[v][u]);
                float2 gy = sub2(qd, q[v][u]);
                bool upd = true;
                if (BORDER) {
                    const int bit = v * U + u;
                    upd = (inside >> bit) & 1u;
                    if ((lastc >> bit) & 1u) gx = zero;
                    if ((lastr >> bit) & 1u) gy = zero;
                }
                if (upd) {
                    const float2 g2 = fma2(gx, gx, mul2(gy, gy));
                    const float2 nrm = make_float2(sqrt_approx(g2.x), sqrt_approx(g2.y));
                    const float2 den = fma2(tau, nrm, one);
                    const float2 inv = make_float2(rcp_approx(den.x), rcp_approx(den.y));
                    px[v][u] = mul2(fma2(tau, gx, px[v][u]), inv);
                    py[v][u] = mul2(fma2(tau, gy, py[v][u]), inv);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) e_py[w][u][lane] = py[V - 1][u];
        __syncthreads();
    }
}

// Region (bx, by) of both images (a launch of gx x gy blocks); as
// tv_steps_block with nimg = 2, the divergence summed as b (x_1 - x_0).
template <int WY, int KB, bool FINAL, int V>
__device__ __forceinline__ void tv_steps_block2(const float* __restrict__ rbase, const float2* __restrict__ pin,
                                                float2* __restrict__ pout, int n, int first, float c_tv,
                                                int from_scalars, float lambda_arg, DevScalars* S,
                                                const float* __restrict__ bprobe, const TvFinal& F, int bx, int by,
                                                int gx, int gy, TvShared2<WY>& sh) {
    constexpr int U = kTvU, RW = kTvRW, RH = V * WY;
    constexpr int E = FINAL ? KB + 1 : KB;
    constexpr int TW = RW - KB - E, TH = RH - KB - E;
    auto& e_py = sh.e_py;
    auto& e_q = sh.e_q;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t N = (size_t)n * n;
    const int gi0 = by * TH - E, gj0 = bx * TW - E;
    pdl_wait();      // r, the duals and the scalars are earlier kernels' output
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const float inv_lam = lam > 0.f ? 1.0f / lam : 0.f;
    float2 px[V][U], py[V][U], rl[V][U];
    unsigned inside = 0u, lastc = 0u, lastr = 0u;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int gi = gi0 + w * V + v;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int gj = gj0 + U * lane + u;
            const bool in = gi >= 0 && gi < n && gj >= 0 && gj < n;
            float r0 = 0.f, r1 = 0.f;
            float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
            if (in) {
                const size_t o = (size_t)gi * n + gj;
                r0 = rbase[o];
                r1 = rbase[N + o];
                if (!first) {
                    p0 = pin[o];
                    p1 = pin[N + o];
                }
            }
            rl[v][u] = make_float2(r0 * inv_lam, r1 * inv_lam);
            px[v][u] = make_float2(p0.x, p1.x);
            py[v][u] = make_float2(p0.y, p1.y);
            const unsigned bit = 1u << (v * U + u);
            if (in) inside |= bit;
            if (gj == n - 1) lastc |= bit;
            if (gi == n - 1) lastr |= bit;
        }
    }
    const bool interior = gi0 >= 0 && gj0 >= 0 && gi0 + RH < n && gj0 + RW < n;
    if (interior)
        tv_region_steps2<WY, KB, false, V>(px, py, rl, inside, lastc, lastr, e_py, e_q);
    else
        tv_region_steps2<WY, KB, true, V>(px, py, rl, inside, lastc, lastr, e_py, e_q);
    if (!FINAL) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int rr = w * V + v;
            if (rr < KB || rr >= RH - KB) continue;
            const int gi = gi0 + rr;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int cc = U * lane + u;
                const int gj = gj0 + cc;
                if (cc < KB || cc >= RW - KB || gi >= n || gj >= n) continue;
                const size_t o = (size_t)gi * n + gj;
                pout[o] = make_float2(px[v][u].x, py[v][u].x);
                pout[N + o] = make_float2(px[v][u].y, py[v][u].y);
            }
        }
        return;
    }
    // ---- final: x = r - lambda div p for both images (e_py holds the last rows' py) ----
    auto& red = sh.red;
    auto& am_last = sh.am_last;
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int rr = w * V + v;
        const int gi = gi0 + rr;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float2 pxl;
            if (u > 0) {
                pxl = px[v][u - 1];
            } else {
                const float2 t = shfl_up2(px[v][U - 1], 1);
                pxl = lane > 0 ? t : make_float2(0.f, 0.f);
            }
            const float2 pyu = v > 0 ? py[v - 1][u] : (w > 0 ? e_py[w - 1][u][lane] : make_float2(0.f, 0.f));
            const int cc = U * lane + u;
            const int gj = gj0 + cc;
            if (rr < E || rr >= RH - KB || cc < E || cc >= RW - KB || gi >= n || gj >= n) continue;
            const size_t o = (size_t)gi * n + gj;
            const float dv0 = px[v][u].x - pxl.x + py[v][u].x - pyu.x;
            const float dv1 = px[v][u].y - pxl.y + py[v][u].y - pyu.y;
            const float x0 = rbase[o] - lam * dv0;
            const float x1 = rbase[N + o] - lam * dv1;
            acc += (double)bprobe[o] * ((double)x1 - (double)x0);
            float xo = x0;
            if (F.solve_mode && F.damp_x != 1.f) xo = F.damp_x * xo + (1.f - F.damp_x) * F.x_out[o];
            F.x_out[o] = xo;
            if (F.XR) stage_store(F.XR, F.xbf, (size_t)gi * F.ldp + kPad + gj, xo);
            if (F.XC) stage_store(F.XC, F.xbf, (size_t)gj * F.ldp + kPad + gi, xo);
        }
    }
    const int nblk = gx * gy;
    const int bid = by * gx + bx;
    if (F.solve_mode) {
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) {
            F.partial_div[bid] = acc;
            if (bid == 0) S->div_pending = (unsigned)nblk;
        }
        return;
    }
    tv_divergence_finish(acc, nblk, bid, N, S, F, red, &am_last);
}

template <int WY, int KB, bool FINAL, int V>
__global__ void __launch_bounds__(32 * WY)
k_tv_steps2(const float* __restrict__ rbase, const float2* __restrict__ pin, float2* __restrict__ pout, int n,
            int first, float c_tv, int from_scalars, float lambda_arg, DevScalars* S,
            const float* __restrict__ bprobe, TvFinal F) {
    __shared__ TvShared2<WY> sh;
    tv_steps_block2<WY, KB, FINAL, V>(rbase, pin, pout, n, first, c_tv, from_scalars, lambda_arg, S, bprobe, F,
                                      blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, sh);
}

// TV region dims of a launch: tile width and height of the valid part
template <int WY, int KB, bool FINAL>
__host__ __device__ constexpr int tv_tile_w() { return kTvRW - KB - (FINAL ? KB + 1 : KB); }
template <int WY, int KB, bool FINAL>
__host__ __device__ constexpr int tv_tile_h() { return kTvV * WY - KB - (FINAL ? KB + 1 : KB); }

// The final-step fields of a solve on batch slice B (as make_tv_final gives
// them for a plan inside a solve)
__device__ __forceinline__ TvFinal tv_final_of(const BatchSlice& B, int xbf) {
    TvFinal F;
    F.x_out = B.x;
    F.XR = (float*)B.XR;
    F.XC = (float*)B.XC;
    F.ldp = B.ldp;
    F.xbf = xbf;
    F.damp_x = B.damp_x;
    F.t_arg = 0;
    F.slice = B.slice_id;
    F.key = B.key;
    F.tau_x_floor = B.tau_x_floor;
    F.partial = B.partial;
    F.partial_div = B.partial_div;
    F.log = B.log;
    F.div_out = nullptr;
    F.solve_mode = 1;
    F.jvp = 0;
    return F;
}

// KB Chambolle steps of both images (r and r + eps b) of every slice of a
// batch in one launch; first: the duals start at zero; the final launch
// forms x, the staged copies and the divergence partials as in a solve.
// Ping-pong dual buffers as in launch_tv_chunk: launch i reads buffer
// (i + 1) & 1 and writes i & 1.
template <int WY, int KB, bool FINAL>
__global__ void __launch_bounds__(32 * WY)
k_tv_steps_batch(const BatchSlice* __restrict__ sl, const uint16_t* __restrict__ map, int phase, int launch,
                 int xbf) {
    __shared__ TvShared2<WY> sh;
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int l = (int)blockIdx.x - B.off[phase];
    const int n = B.n;
    const int gx = (n + tv_tile_w<WY, KB, FINAL>() - 1) / tv_tile_w<WY, KB, FINAL>();
    const int gy = (n + tv_tile_h<WY, KB, FINAL>() - 1) / tv_tile_h<WY, KB, FINAL>();
    const int bx = l % gx, by = l / gx;
    const size_t N = (size_t)B.N;
    const float2* pin = B.p + ((launch + 1) & 1) * 2 * N;
    float2* pout = B.p + (launch & 1) * 2 * N;
    const TvFinal F = tv_final_of(B, xbf);
    tv_steps_block2<WY, KB, FINAL, kTvV>(B.r, pin, pout, n, launch == 0, B.c_tv, 1, 0.f, B.S, B.b, F, bx, by, gx,
                                         gy, sh);
}

int batch_grid_tv(int n, int final_launch) {
    constexpr int WY = kTvRowsBatch / kTvV;
    const int tw = final_launch ? tv_tile_w<WY, kBatchTvKb, true>() : tv_tile_w<WY, kBatchTvKb, false>();
    const int th = final_launch ? tv_tile_h<WY, kBatchTvKb, true>() : tv_tile_h<WY, kBatchTvKb, false>();
    return ((n + tw - 1) / tw) * ((n + th - 1) / th);   // both images of a region in one block
}

int batch_grid_probe(long long N) { return (int)(((N + 3) / 4 + 255) / 256); }

int launch_probe_batch(const BatchExec& E, cudaStream_t st) {
    const BatchSlice* sl = E.sl;
    const uint16_t* map = E.map[kPhProbe];
    DGCT_CUDA(launch_pdl(k_probe_input_batch, dim3(E.nblk[kPhProbe]), dim3(256), 0, st, sl, map));
    return DGAMP_CT_OK;
}

int launch_tv_batch(const BatchExec& E, int launch, bool final_launch, cudaStream_t st) {
    constexpr int WY = kTvRowsBatch / kTvV;
    const BatchSlice* sl = E.sl;
    if (final_launch)
        DGCT_CUDA(launch_pdl(k_tv_steps_batch<WY, kBatchTvKb, true>, dim3(E.nblk[kPhTv1]), dim3(32 * WY), 0, st, sl,
                             (const uint16_t*)E.map[kPhTv1], (int)kPhTv1, launch, E.bf));
    else
        DGCT_CUDA(launch_pdl(k_tv_steps_batch<WY, kBatchTvKb, false>, dim3(E.nblk[kPhTv0]), dim3(32 * WY), 0, st, sl,
                             (const uint16_t*)E.map[kPhTv0], (int)kPhTv0, launch, E.bf));
    return DGAMP_CT_OK;
}

// Final step: x = r - lambda div p for NIMG images (p = 0 when pfin is NULL),
// x of image 0 (damped in a solve) to x_out and the staged copies, and for
// NIMG = 2 the divergence b^T (x_1 - x_0) / (N eps) (b as k_probe_input
// stored it) and, in a solve, tau_x.  32 x 32 pixel tiles, one pixel per thread.
template <int NIMG>
__global__ void __launch_bounds__(1024)
k_tv_final(const float* __restrict__ rbase, const float2* __restrict__ pfin, const float* __restrict__ bprobe, int n,
           float c_tv, int from_scalars, float lambda_arg, DevScalars* S, TvFinal F) {
    __shared__ float tile[TB][TB + 1];
    __shared__ double red[32];
    __shared__ bool am_last;
    const size_t N = (size_t)n * n;
    const int tid = threadIdx.x, ta = tid >> 5, tb = tid & 31;
    const int gi = blockIdx.y * TB + ta, gj = blockIdx.x * TB + tb;
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    double acc = 0.0;
    float xv = 0.f;
    if (gi < n && gj < n) {
        const size_t o = (size_t)gi * n + gj;
        float xs[NIMG];
#pragma unroll
        for (int im = 0; im < NIMG; ++im) {
            float dv = 0.f;
            if (pfin) {
                const float2* p = pfin + im * N;
                const float2 pc = p[o];
                const float pxl = gj > 0 ? p[o - 1].x : 0.f;
                const float pyu = gi > 0 ? p[o - n].y : 0.f;
                dv = pc.x - pxl + pc.y - pyu;
            }
            xs[im] = rbase[im * N + o] - lam * dv;
        }
        xv = xs[0];
        if (NIMG == 2) acc = (double)bprobe[o] * (double)(xs[NIMG - 1] - xs[0]);
        if (F.solve_mode && F.damp_x != 1.f) xv = F.damp_x * xv + (1.f - F.damp_x) * F.x_out[o];
        F.x_out[o] = xv;
        if (F.XR) stage_store(F.XR, F.xbf, (size_t)gi * F.ldp + kPad + gj, xv);
    }
    tile[ta][tb] = xv;
    if (F.XC) {
        __syncthreads();
        const int gj2 = blockIdx.x * TB + ta, gi2 = blockIdx.y * TB + tb;
        if (gi2 < n && gj2 < n) stage_store(F.XC, F.xbf, (size_t)gj2 * F.ldp + kPad + gi2, tile[tb][ta]);
    }
    if (NIMG < 2) return;
    tv_divergence_finish(acc, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x, N, S, F, red, &am_last);
}

// Steps per launch and region heights the autotuner may choose.
static const int kTvKbChoices[] = {3, 4, 5, 6, 8, 10};
static const int kTvRowChoices[] = {32, 64, 128};

bool tv_active(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (pl->opt.k_tv <= 0) return false;
    return from_scalars ? pl->opt.c_tv > 0.0 : lambda_arg > 0.0;
}

static int tv_step_launches(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (!tv_active(pl, from_scalars, lambda_arg)) return 0;
    return (pl->opt.k_tv + pl->tv_kb - 1) / pl->tv_kb;
}

// the step launches, the last of them forming x (or one final launch when
// the denoiser is the identity: no steps or lambda = 0); the metric form
// (option tv_metric) has its own sequence, see tv_metric.cu
int tv_num_launches(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (pl->opt.tv_metric && tv_active(pl, from_scalars, lambda_arg)) return tvm_num_launches(pl);
    const int ns = tv_step_launches(pl, from_scalars, lambda_arg);
    return ns > 0 ? ns : 1;
}

struct TvLaunch {
    int n, nimg, first;
    const float* r;
    const float2* pin;
    float2* pout;
    float c_tv, lam;
    int fs;
    DevScalars* S;
    const float* b;
};

// The MC pair's launches take the two-image kernel in 32- and 64-row regions
// of 4-row threads (about 100 registers a thread) and in 64-row regions of
// 2-row threads (1024 threads); the 128-row and 8-row shapes would spill
// there and keep the one-image kernel.
template <int WY, int V>
constexpr bool tv_paired_shape() { return (V == 4 && (WY == 8 || WY == 16)) || (V == 2 && WY == 32); }

template <int WY, int KB, bool FIN, int V>
static cudaError_t launch_steps_kb(const TvLaunch& L, cudaStream_t st, const TvFinal& F) {
    constexpr int E = FIN ? KB + 1 : KB;
    constexpr int TW = kTvRW - KB - E, TH = V * WY - KB - E;
    if constexpr (tv_paired_shape<WY, V>()) if (L.nimg == 2) {   // the MC pair: both images in one thread
        const dim3 grd((L.n + TW - 1) / TW, (L.n + TH - 1) / TH);
        return launch_pdl(k_tv_steps2<WY, KB, FIN, V>, grd, dim3(32 * WY), 0, st, L.r, L.pin, L.pout, L.n,
                          L.first, L.c_tv, L.fs, L.lam, L.S, L.b, F);
    }
    const dim3 grd((L.n + TW - 1) / TW, (L.n + TH - 1) / TH, L.nimg);
    return launch_pdl(k_tv_steps<WY, KB, FIN, V>, grd, dim3(32 * WY), 0, st, L.r, L.pin, L.pout, L.n, L.first,
                      L.c_tv, L.fs, L.lam, L.S, L.b, F);
}

template <int WY, bool FIN, int V = kTvV>
static int launch_steps_wy(int steps, const TvLaunch& L, cudaStream_t st, const TvFinal& F) {
    cudaError_t e = cudaSuccess;
#define DGCT_TV_CASE(KB) \
    case KB: e = launch_steps_kb<WY, KB, FIN, V>(L, st, F); break;
    switch (steps) {
        DGCT_TV_CASE(1) DGCT_TV_CASE(2) DGCT_TV_CASE(3) DGCT_TV_CASE(4) DGCT_TV_CASE(5)
        DGCT_TV_CASE(6) DGCT_TV_CASE(7) DGCT_TV_CASE(8) DGCT_TV_CASE(9) DGCT_TV_CASE(10)
        default: return DGAMP_CT_ERR_INVALID_ARG;
    }
#undef DGCT_TV_CASE
    DGCT_CUDA(e);
    return DGAMP_CT_OK;
}

// rows: region height; vrows: rows per thread (4, or 8 with 64-row regions only)
template <bool FIN>
static int launch_steps(int rows, int vrows, int steps, const TvLaunch& L, cudaStream_t st, const TvFinal& F) {
    if (vrows == 8) return launch_steps_wy<8, FIN, 8>(steps, L, st, F);
    if (vrows == 2) return launch_steps_wy<32, FIN, 2>(steps, L, st, F);
    if (rows == 128) return launch_steps_wy<32, FIN>(steps, L, st, F);
    if (rows == 32) return launch_steps_wy<8, FIN>(steps, L, st, F);
    return launch_steps_wy<16, FIN>(steps, L, st, F);
}

static TvFinal make_tv_final(const dgamp_ct_plan_s* pl, float* x_out, int solve_mode, int t_arg,
                             double* div_out) {
    TvFinal F;
    F.x_out = x_out;
    F.XR = solve_mode ? pl->ws.XR : nullptr;
    F.XC = solve_mode ? pl->ws.XC : nullptr;
    F.ldp = pl->ldp;
    F.xbf = solve_mode ? pl->opt.storage : 0;
    F.damp_x = (float)pl->opt.damp_x;
    F.t_arg = t_arg;
    F.slice = (unsigned)pl->opt.slice_id;
    F.key = probe_key(pl);
    F.tau_x_floor = pl->opt.tau_x_floor;
    F.partial = pl->ws.partial;
    F.partial_div = pl->ws.partial_div;
    F.log = pl->ws.log;
    F.div_out = div_out;
    F.solve_mode = solve_mode;
    F.jvp = 0;
    return F;
}

int launch_tv_final_x(const dgamp_ct_plan_s* pl, int nimg, const float* xbase, float* x_out, int solve_mode,
                      int t_arg, double* div_out, cudaStream_t st) {
    const int n = pl->n;
    const TvFinal F = make_tv_final(pl, x_out, solve_mode, t_arg, div_out);
    dim3 grd((n + TB - 1) / TB, (n + TB - 1) / TB);
    // no duals: the final step takes xbase as the denoised images
    if (nimg == 2)
        k_tv_final<2><<<grd, 1024, 0, st>>>(xbase, nullptr, pl->ws.b, n, 0.f, 0, 0.f, pl->ws.S, F);
    else
        k_tv_final<1><<<grd, 1024, 0, st>>>(xbase, nullptr, pl->ws.b, n, 0.f, 0, 0.f, pl->ws.S, F);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// Launch i (0-based) of the denoiser on nimg images of ws.r.
int launch_tv_chunk(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                    float* x_out, int solve_mode, int t_arg, double* div_out, cudaStream_t st) {
    if (pl->opt.tv_metric && tv_active(pl, from_scalars, lambda_arg))
        return launch_tvm_chunk(pl, nimg, from_scalars, lambda_arg, i, x_out, solve_mode, t_arg, div_out, st);
    const int n = pl->n;
    const size_t N = (size_t)pl->N;
    const int KB = pl->tv_kb;
    const int ns = tv_step_launches(pl, from_scalars, lambda_arg);
    float2* buf[2] = {pl->ws.p, pl->ws.p + 2 * N};
    const float c_tv = (float)pl->opt.c_tv, lam = (float)lambda_arg;
    if (ns == 0)   // identity denoiser: x = r
        return launch_tv_final_x(pl, nimg, pl->ws.r, x_out, solve_mode, t_arg, div_out, st);
    const TvFinal F = make_tv_final(pl, x_out, solve_mode, t_arg, div_out);
    const int steps = (i + 1) * KB <= pl->opt.k_tv ? KB : pl->opt.k_tv - i * KB;
    TvLaunch L{n, nimg, i == 0, pl->ws.r, buf[(i + 1) & 1], buf[i & 1], c_tv, lam, from_scalars, pl->ws.S,
               pl->ws.b};
    if (i == ns - 1) return launch_steps<true>(pl->tv_rows, pl->tv_vrows, steps, L, st, F);
    return launch_steps<false>(pl->tv_rows, pl->tv_vrows, steps, L, st, F);
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

// Shared memory is static (at most 16 KiB): nothing to raise.
int tv_set_smem_limits() { return DGAMP_CT_OK; }

// Plan-time choice of the steps per launch and the region height: time the
// two-image denoiser of the plan's geometry (K = opt.k_tv) for every pair
// and keep the fastest.  Runs on zeroed workspace; the timing does not
// depend on the values.
int tv_autotune(dgamp_ct_plan_s* pl) {
    if (pl->opt.k_tv <= 0) return DGAMP_CT_OK;
    const size_t N = (size_t)pl->N;
    DGCT_CUDA(cudaMemset(pl->ws.r, 0, 2 * N * sizeof(float)));
    DGCT_CUDA(cudaMemset(pl->ws.S, 0, sizeof(DevScalars)));
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_kb = pl->tv_kb, best_rows = pl->tv_rows, best_v = pl->tv_vrows;
    // (region rows, rows per thread): the 4-row threads at three heights, and
    // 64-row regions of 8-row threads (half the threads, each with twice the
    // pixels) and of 2-row threads (twice the threads, half the pixels each)
    const int shapes[][2] = {{kTvRowChoices[0], 4}, {kTvRowChoices[1], 4}, {kTvRowChoices[2], 4}, {64, 8}, {64, 2}};
    for (const auto& sh : shapes) {
        const int rows = sh[0];
        for (int kb : kTvKbChoices) {
            pl->tv_kb = kb;
            pl->tv_rows = rows;
            pl->tv_vrows = sh[1];
            int rc = DGAMP_CT_OK;
            for (int rep = 0; rep < 4 && rc == DGAMP_CT_OK; ++rep) {      // first rep warms up
                if (rep == 1) cudaEventRecord(e0, 0);
                // as inside a solve (staged copies, divergence partials), lambda = 1
                rc = launch_tv(pl, 2, 0, 1.0, pl->ws.x, 1, 1, nullptr, 0);
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
            if (ms < best) {
                best = ms;
                best_kb = kb;
                best_rows = rows;
                best_v = sh[1];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->tv_kb = best_kb;
    pl->tv_rows = best_rows;
    pl->tv_vrows = best_v;
    return DGAMP_CT_OK;
}

// ------------------------------------- final step for a learned denoiser --
// x = D(r) (damped in a solve), staged copies, the divergence and tau_x from
// dn[0] = D(r) and dn[1] = J_D(r) b ([2][n][n]): D' = b^T J_D b / N, the
// eps -> 0 limit of Eq. MC_SURE (F.jvp = 1), or from dn[1] = D(r + eps b):
// D' = b^T (dn[1] - dn[0]) / (N eps).  32 x 32 tiles as in the blocked TV's
// final launch.
__global__ void __launch_bounds__(1024)
k_denoise_final(const float* __restrict__ dn, const float* __restrict__ bprobe, int n, DevScalars* S, TvFinal F) {
    __shared__ float tile[TB][TB + 1];
    __shared__ double red[32];
    __shared__ bool am_last;
    const size_t N = (size_t)n * n;
    const int tid = threadIdx.x, ta = tid >> 5, tb = tid & 31;
    const int gi = blockIdx.y * TB + ta, gj = blockIdx.x * TB + tb;
    double acc = 0.0;
    float xv = 0.f;
    if (gi < n && gj < n) {
        const size_t o = (size_t)gi * n + gj;
        const float x1 = dn[o], x2 = dn[N + o];
        acc = (double)bprobe[o] * (double)(F.jvp ? x2 : x2 - x1);
        xv = x1;
        if (F.solve_mode && F.damp_x != 1.f) xv = F.damp_x * xv + (1.f - F.damp_x) * F.x_out[o];
        F.x_out[o] = xv;
        if (F.XR) stage_store(F.XR, F.xbf, (size_t)gi * F.ldp + kPad + gj, xv);
    }
    tile[ta][tb] = xv;
    if (F.XC) {
        __syncthreads();
        const int gj2 = blockIdx.x * TB + ta, gi2 = blockIdx.y * TB + tb;
        if (gi2 < n && gj2 < n) stage_store(F.XC, F.xbf, (size_t)gj2 * F.ldp + kPad + gi2, tile[tb][ta]);
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
    F.xbf = solve_mode ? pl->opt.storage : 0;
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
    k_denoise_final<<<grd, 1024, 0, st>>>(dn, pl->ws.b, n, pl->ws.S, F);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// ------------------------- denoiser 2: the CNN judged by prox-TV -----
// Both denoisers have run on r: dn[0] = D_cnn(r), dn[1] = J_cnn(r) b,
// dn[2] = D_tv(r), and S->div_plain holds prox-TV's divergence (Eq. MC_SURE).
// k_select_sums adds, over the pixels, (D_cnn(r) - r)^2, b J_cnn b and
// (D_tv(r) - r)^2 (FP32 per thread, FP64 per block and across blocks, in a
// fixed order); its last block forms each candidate's SURE risk estimate
//   ||D(r) - r||^2 / N - tau_r + 2 tau_r D'(r)
// and keeps the CNN where its estimate is strictly lower and its divergence
// lies in (0, M/N).  (tau_x = tau_r D' is a variance, so D' <= 0 estimates
// nothing; and with a large tau_p the output step gives tau_s near 1/tau_p,
// so tau_r^{t+1} is about tau_r^t D'/(M/N): a denoiser with D' >= M/N makes
// tau_r grow, and SURE, which takes tau_r as the noise level of r, cannot be
// trusted then.)  k_select_final
// then writes the kept output as x (damped), the staged copies, tau_x, the
// log record and the next t.
constexpr int kSelBlocks = 256;

__global__ void __launch_bounds__(256)
k_select_sums(const float* __restrict__ r, const float* __restrict__ dn, const float* __restrict__ bprobe,
              long long N, double max_div, DevScalars* S, double* __restrict__ partial) {
    __shared__ double red[32];
    __shared__ bool am_last;
    pdl_wait();
    float s_cnn = 0.f, s_jb = 0.f, s_tv = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const float rv = r[i];
        const float dc = dn[i] - rv, dt = dn[2 * N + i] - rv;
        s_cnn = fmaf(dc, dc, s_cnn);
        s_jb = fmaf(bprobe[i], dn[N + i], s_jb);
        s_tv = fmaf(dt, dt, s_tv);
    }
    const double a = block_sum((double)s_cnn, red);
    const double b = block_sum((double)s_jb, red);
    const double c = block_sum((double)s_tv, red);
    const int nblk = gridDim.x, bid = blockIdx.x;
    if (threadIdx.x == 0) {
        partial[3 * bid] = a;
        partial[3 * bid + 1] = b;
        partial[3 * bid + 2] = c;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_div, 1u);
        am_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double pa = 0.0, pb = 0.0, pc = 0.0;
    const volatile double* P = partial;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
        pa += P[3 * k];
        pb += P[3 * k + 1];
        pc += P[3 * k + 2];
    }
    const double ta = block_sum(pa, red), tb = block_sum(pb, red), tc = block_sum(pc, red);
    if (threadIdx.x != 0) return;
    const double Nd = (double)N, tau_r = S->tau_r;
    const double div_l = tb / Nd, div_p = S->div_plain;
    const double risk_l = ta / Nd - tau_r + 2.0 * tau_r * div_l;
    const double risk_p = tc / Nd - tau_r + 2.0 * tau_r * div_p;
    const unsigned keep = (risk_l < risk_p && div_l > 0.0 && div_l < max_div) ? 1u : 0u;
    S->div_learned = div_l;
    S->risk_learned = risk_l;
    S->risk_plain = risk_p;
    S->keep_learned = keep;
    S->div = keep ? div_l : div_p;
    S->done_div = 0u;
}

__global__ void __launch_bounds__(1024)
k_select_final(const float* __restrict__ dn, int n, DevScalars* S, TvFinal F) {
    __shared__ float tile[TB][TB + 1];
    pdl_wait();
    const size_t N = (size_t)n * n;
    const int tid = threadIdx.x, ta = tid >> 5, tb = tid & 31;
    const int gi = blockIdx.y * TB + ta, gj = blockIdx.x * TB + tb;
    const float* __restrict__ src = S->keep_learned ? dn : dn + 2 * N;
    float xv = 0.f;
    if (gi < n && gj < n) {
        const size_t o = (size_t)gi * n + gj;
        xv = src[o];
        if (F.damp_x != 1.f) xv = F.damp_x * xv + (1.f - F.damp_x) * F.x_out[o];
        F.x_out[o] = xv;
        stage_store(F.XR, F.xbf, (size_t)gi * F.ldp + kPad + gj, xv);
    }
    tile[ta][tb] = xv;
    __syncthreads();
    const int gj2 = blockIdx.x * TB + ta, gi2 = blockIdx.y * TB + tb;
    if (gi2 < n && gj2 < n) stage_store(F.XC, F.xbf, (size_t)gj2 * F.ldp + kPad + gi2, tile[tb][ta]);
    if (blockIdx.x != 0 || blockIdx.y != 0 || tid != 0) return;
    // tau_x from the kept divergence, the log record and the next t (one thread)
    const double tau_r = S->tau_r, div = S->div;
    double tx = tau_r * div;
    const double fl = F.tau_x_floor * tau_r;
    if (!(tx >= fl)) { tx = fl; S->floored += 1u; }
    if (!isfinite(tx)) S->nonfinite += 1u;
    S->tau_x = tx;
    S->learned_kept += S->keep_learned;
    const unsigned tt = S->t;
    if (tt >= 1u && tt <= (unsigned)kMaxIters) {
        IterLog L;
        L.tau_x = tx; L.tau_p = S->tau_p; L.tau_s = S->tau_s; L.tau_r = tau_r;
        L.div = div; L.eps = S->eps;
        L.risk_plain = S->risk_plain;
        L.risk_learned = S->risk_learned;
        L.keep_learned = (int)S->keep_learned;
        F.log[tt - 1] = L;
    }
    S->t = tt + 1u;
}

int launch_select(const dgamp_ct_plan_s* pl, int part, cudaStream_t st) {
    const int n = pl->n;
    const long long N = pl->N;
    if (part == 0) {
        const double max_div = (double)pl->M / (double)pl->N;
        DGCT_CUDA(launch_pdl(k_select_sums, dim3(kSelBlocks), dim3(256), 0, st, (const float*)pl->ws.r,
                             (const float*)pl->dn, (const float*)pl->ws.b, N, max_div, pl->ws.S, pl->ws.partial));
        return DGAMP_CT_OK;
    }
    TvFinal F = make_tv_final(pl, pl->ws.x, 1, 0, nullptr);
    dim3 grd((n + TB - 1) / TB, (n + TB - 1) / TB);
    DGCT_CUDA(launch_pdl(k_select_final, grd, dim3(1024), 0, st, (const float*)pl->dn, n, pl->ws.S, F));
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
