// Shared-memory FFTs for the Radon preconditioner (Section 2.4, Eq. Aprecon).
//
//  * H on sinograms: one block filters two views at once, packed as the real
//    and imaginary parts of one complex line.  Because the gain g is real and
//    even, filtering a + i b gives H a + i H b, so one forward and one inverse
//    complex FFT of length P serve two views.
//  * V^-1 / V on images: a 2-D zero-padded FFT done as row FFTs, column FFTs
//    with the radial gain applied between the forward and inverse column
//    transforms, and inverse row FFTs.  It runs once per solve.
//
// The transform (fft_device.cuh) is a Stockham autosort FFT with radix-8
// stages, in shared memory.
#include "fft_device.cuh"

namespace dgct {

// one thread per radix-8 butterfly, 32 to 512 threads
static int fft_threads(int P) { return P / 8 < 32 ? 32 : (P / 8 > 512 ? 512 : P / 8); }

// ------------------------------------------------------------ H on views --
template <typename T>
__global__ void __launch_bounds__(512)
k_filter_views(const T* in, T* out, int nv, int nd, int P,
               const float* __restrict__ gain, const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(P);
    const int va = 2 * blockIdx.x, vb = va + 1;
    const bool hasb = vb < nv;
    const T* ra = in + (size_t)va * nd;
    const T* rb = in + (size_t)vb * nd;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (i < nd) {
            v.x = ldf(ra + i);
            if (hasb) v.y = ldf(rb + i);
        }
        a[fpad(i)] = v;
    }
    __syncthreads();
    float2* r = fft_stockham(a, b, P, tw, -1.f);
    float2* o = (r == a) ? b : a;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const float g = __ldg(gain + i);
        const float2 v = r[fpad(i)];
        r[fpad(i)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    r = fft_stockham(r, o, P, tw, 1.f);
    const float sc = 1.0f / (float)P;
    T* wa = out + (size_t)va * nd;
    T* wb = out + (size_t)vb * nd;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        const float2 v = r[fpad(i)];
        stf(wa + i, v.x * sc);
        if (hasb) stf(wb + i, v.y * sc);
    }
}

// ------------------------------------------------- H as a Toeplitz product --
// The same operator without an FFT: with zero padding to P >= 2 n_det there
// is no wrap-around, so (H z)[d] = sum_d' h[|d - d'|] z[d'] with
// h = IFFT_P(g) (real and even), computed in FP64 at plan time and stored as
// hx[m + n_det - 1] = h[|m|] for m in (-n_det, n_det).  Block = one view x
// 128 outputs; each lane keeps 4 consecutive outputs (a sliding window of
// hx in registers) and the 8 warps split the d' range, their partial sums
// added in a fixed order.
constexpr int kTzOut = 128, kTzWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kTzWarps)
k_filter_toeplitz(const T* in, T* out, int nd, const float* __restrict__ hx) {
    extern __shared__ float sm[];
    float* zs = sm;                       // [nd]
    float* hs = sm + nd;                  // [2 nd - 1]
    float* red = hs + 2 * nd - 1;         // [kTzWarps][kTzOut]
    const int v = blockIdx.y;
    const int d0 = blockIdx.x * kTzOut;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const T* row = in + (size_t)v * nd;
    for (int i = tid; i < nd; i += blockDim.x) zs[i] = ldf(row + i);
    for (int i = tid; i < 2 * nd - 1; i += blockDim.x) hs[i] = hx[i];
    __syncthreads();
    const int dl = d0 + 4 * lane;          // this lane's first output
    const int len = (nd + kTzWarps - 1) / kTzWarps;
    const int p0 = w * len, p1 = min(nd, p0 + len);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (dl < nd && p0 < p1) {
        // output dl + i at input d' uses hs[dl + i - d' + nd - 1]
        int base = dl - p0 + nd - 1;
        float h0 = hs[base], h1 = hs[min(base + 1, 2 * nd - 2)], h2 = hs[min(base + 2, 2 * nd - 2)],
              h3 = hs[min(base + 3, 2 * nd - 2)];
        for (int dp = p0; dp < p1; ++dp) {
            const float zv = zs[dp];
            a0 = fmaf(h0, zv, a0);
            a1 = fmaf(h1, zv, a1);
            a2 = fmaf(h2, zv, a2);
            a3 = fmaf(h3, zv, a3);
            // next d' shifts every index down by one
            h3 = h2;
            h2 = h1;
            h1 = h0;
            --base;
            h0 = base >= 0 ? hs[base] : 0.f;
        }
    }
    red[w * kTzOut + 4 * lane + 0] = a0;
    red[w * kTzOut + 4 * lane + 1] = a1;
    red[w * kTzOut + 4 * lane + 2] = a2;
    red[w * kTzOut + 4 * lane + 3] = a3;
    __syncthreads();
    for (int o = tid; o < kTzOut; o += blockDim.x) {
        const int d = d0 + o;
        if (d >= nd) continue;
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kTzWarps; ++k) t += red[k * kTzOut + o];
        stf(out + (size_t)v * nd + d, t);
    }
}

static size_t toeplitz_smem(int nd) {
    return ((size_t)nd + 2 * nd - 1 + kTzWarps * kTzOut) * sizeof(float);
}

// bf = 1: in and out hold BF16 (a solve with storage = 1); sums in FP32 either way
int launch_filter(const dgamp_ct_plan_s* pl, const float* in, float* out, cudaStream_t st, int bf) {
    if (pl->filter_mode == 1) {
        // the block reads its whole input row first, so in == out needs a copy
        const float* src = in;
        if (in == out) {
            DGCT_CUDA(cudaMemcpyAsync(pl->ws.zraw2, in, (size_t)pl->M * (bf ? 2 : 4), cudaMemcpyDeviceToDevice, st));
            src = pl->ws.zraw2;
        }
        dim3 grd((pl->nd + kTzOut - 1) / kTzOut, pl->nv);
        if (bf)
            k_filter_toeplitz<bf16s><<<grd, 32 * kTzWarps, toeplitz_smem(pl->nd), st>>>((const bf16s*)src, (bf16s*)out,
                                                                                        pl->nd, pl->ws.hx);
        else
            k_filter_toeplitz<float><<<grd, 32 * kTzWarps, toeplitz_smem(pl->nd), st>>>(src, out, pl->nd, pl->ws.hx);
        DGCT_LAUNCH_CHECK();
        return DGAMP_CT_OK;
    }
    const int P = pl->P;
    const size_t sm = (size_t)2 * fft_buf_len(P) * sizeof(float2);
    const int thr = fft_threads(P);
    if (bf)
        k_filter_views<bf16s><<<(pl->nv + 1) / 2, thr, sm, st>>>((const bf16s*)in, (bf16s*)out, pl->nv, pl->nd, P,
                                                                 pl->ws.gain, pl->ws.tw);
    else
        k_filter_views<float><<<(pl->nv + 1) / 2, thr, sm, st>>>(in, out, pl->nv, pl->nd, P, pl->ws.gain,
                                                                 pl->ws.tw);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// Plan-time choice between the FFT and the Toeplitz form of H (same operator):
// time both on the plan's geometry and keep the faster.
int filter_autotune(dgamp_ct_plan_s* pl) {
    DGCT_CUDA(cudaMemset(pl->ws.zraw, 0, (size_t)pl->M * sizeof(float)));
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_mode = 0;
    for (int mode = 0; mode < 2; ++mode) {
        pl->filter_mode = mode;
        int rc = DGAMP_CT_OK;
        for (int rep = 0; rep < 6 && rc == DGAMP_CT_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, 0);
            rc = launch_filter(pl, pl->ws.zraw, pl->ws.z, 0);
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
        if (ms < best) { best = ms; best_mode = mode; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->filter_mode = best_mode;
    return DGAMP_CT_OK;
}

int toeplitz_set_smem_limit(int nd) {
    const size_t need = toeplitz_smem(nd);
    DGCT_TRY(raise_smem_limit((const void*)k_filter_toeplitz<float>, (int)need));
    DGCT_TRY(raise_smem_limit((const void*)k_filter_toeplitz<bf16s>, (int)need));
    return DGAMP_CT_OK;
}

// ------------------------------------------------------- V^-1 / V image --
// Image blockIdx.y of a batch (img and out [nimg][n][n], C [nimg][n][m]); a
// single image is the batch of one.
// pass 1: rows iy < n of the m x m padded image -> C[iy][:]
__global__ void __launch_bounds__(512)
k_img_rows_fwd(const float* __restrict__ img, int n, int m, const float2* __restrict__ tw,
               float2* __restrict__ C) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int iy = blockIdx.x;
    img += (size_t)blockIdx.y * n * n;
    C += (size_t)blockIdx.y * n * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        a[fpad(i)] = make_float2(i < n ? img[(size_t)iy * n + i] : 0.f, 0.f);
    __syncthreads();
    float2* r = fft_stockham(a, b, m, tw, -1.f);
    for (int i = threadIdx.x; i < m; i += blockDim.x) C[(size_t)iy * m + i] = r[fpad(i)];
}

// pass 2: every column kx: forward FFT over rows (rows >= n are zero),
// radial gain, inverse FFT; rows < n are stored back.
__global__ void __launch_bounds__(512)
k_img_cols(float2* __restrict__ C, int n, int m, const float2* __restrict__ tw, float f0,
           int inverse_gain) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int kx = blockIdx.x;
    C += (size_t)blockIdx.y * n * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        a[fpad(i)] = i < n ? C[(size_t)i * m + kx] : make_float2(0.f, 0.f);
    __syncthreads();
    float2* r = fft_stockham(a, b, m, tw, -1.f);
    float2* o = (r == a) ? b : a;
    const float fx = (float)(kx <= m / 2 ? kx : kx - m) / (float)m;
    for (int ky = threadIdx.x; ky < m; ky += blockDim.x) {
        const float fy = (float)(ky <= m / 2 ? ky : ky - m) / (float)m;
        const float rho = sqrtf(fx * fx + fy * fy);
        float g = sqrtf(fmaxf(rho, f0));
        if (inverse_gain) g = 1.0f / g;
        const float2 v = r[fpad(ky)];
        r[fpad(ky)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    r = fft_stockham(r, o, m, tw, 1.f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) C[(size_t)i * m + kx] = r[fpad(i)];
}

// pass 3: inverse row FFTs, real part of the first n columns, scaled by 1/m^2.
__global__ void __launch_bounds__(512)
k_img_rows_inv(const float2* __restrict__ C, int n, int m, const float2* __restrict__ tw,
               float* __restrict__ out) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int iy = blockIdx.x;
    C += (size_t)blockIdx.y * n * m;
    out += (size_t)blockIdx.y * n * n;
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[fpad(i)] = C[(size_t)iy * m + i];
    __syncthreads();
    float2* r = fft_stockham(a, b, m, tw, 1.f);
    const float sc = 1.0f / ((float)m * (float)m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[(size_t)iy * n + i] = r[fpad(i)].x * sc;
}

// pass 3 of V^-1 inside a fan-beam solve (Algorithm 1, Step 3 with
// Phi~^T = V^-1 A^T): r = x + tau_r Re(.) / m^2 with tau_r from the device
// scalars (the output step formed it), max |r| into S->rmax_bits (the output
// step reset it), and the consumed divergence flag cleared, as the
// parallel-beam back-projection does.
__global__ void __launch_bounds__(512)
k_img_rows_inv_update(const float2* __restrict__ C, int n, int m, const float2* __restrict__ tw,
                      const float* __restrict__ x, DevScalars* __restrict__ S, float* __restrict__ out) {
    extern __shared__ float2 smem[];
    __shared__ unsigned s_max;
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int iy = blockIdx.x;
    if (threadIdx.x == 0) {
        s_max = 0u;
        if (iy == 0) S->div_pending = 0u;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[fpad(i)] = C[(size_t)iy * m + i];
    __syncthreads();
    const float2* r = fft_stockham(a, b, m, tw, 1.f);
    const float sc = (float)S->tau_r / ((float)m * (float)m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t o = (size_t)iy * n + i;
        const float rv = fmaf(sc, r[fpad(i)].x, x[o]);
        out[o] = rv;
        atomicMax(&s_max, __float_as_uint(fabsf(rv)));   // |r| >= 0: bit order is value order
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&S->rmax_bits, s_max);
}

int launch_precond_image_update(const dgamp_ct_plan_s* pl, const float* in, const float* x, float* out,
                                cudaStream_t st) {
    const int n = pl->n, m = pl->m2;
    const size_t sm = (size_t)2 * fft_buf_len(m) * sizeof(float2);
    const int thr = fft_threads(m);
    const float f0 = 1.0f / (2.0f * (float)pl->P);
    k_img_rows_fwd<<<n, thr, sm, st>>>(in, n, m, pl->ws.tw2, pl->ws.fft2d);
    DGCT_LAUNCH_CHECK();
    k_img_cols<<<m, thr, sm, st>>>(pl->ws.fft2d, n, m, pl->ws.tw2, f0, 0);
    DGCT_LAUNCH_CHECK();
    k_img_rows_inv_update<<<n, thr, sm, st>>>(pl->ws.fft2d, n, m, pl->ws.tw2, x, pl->ws.S, out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

int launch_precond_image(const dgamp_ct_plan_s* pl, const float* in, float* out, int inverse,
                         cudaStream_t st) {
    const int n = pl->n, m = pl->m2;
    const size_t sm = (size_t)2 * fft_buf_len(m) * sizeof(float2);
    const int thr = fft_threads(m);
    const float f0 = 1.0f / (2.0f * (float)pl->P);
    k_img_rows_fwd<<<n, thr, sm, st>>>(in, n, m, pl->ws.tw2, pl->ws.fft2d);
    DGCT_LAUNCH_CHECK();
    // V^-1 applies sqrt(max(rho, f0)); V applies its reciprocal
    k_img_cols<<<m, thr, sm, st>>>(pl->ws.fft2d, n, m, pl->ws.tw2, f0, inverse ? 0 : 1);
    DGCT_LAUNCH_CHECK();
    k_img_rows_inv<<<n, thr, sm, st>>>(pl->ws.fft2d, n, m, pl->ws.tw2, out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// nimg images at once ([nimg][n][n] in and out) through the scratch C
// ([nimg][n][m] complex, the caller's); the same kernels and arithmetic per
// image as launch_precond_image
int launch_precond_images(const dgamp_ct_plan_s* pl, const float* in, float* out, float2* C, int nimg, int inverse,
                          cudaStream_t st) {
    if (nimg < 1) return DGAMP_CT_ERR_INVALID_ARG;
    const int n = pl->n, m = pl->m2;
    const size_t sm = (size_t)2 * fft_buf_len(m) * sizeof(float2);
    const int thr = fft_threads(m);
    const float f0 = 1.0f / (2.0f * (float)pl->P);
    k_img_rows_fwd<<<dim3(n, nimg), thr, sm, st>>>(in, n, m, pl->ws.tw2, C);
    DGCT_LAUNCH_CHECK();
    k_img_cols<<<dim3(m, nimg), thr, sm, st>>>(C, n, m, pl->ws.tw2, f0, inverse ? 0 : 1);
    DGCT_LAUNCH_CHECK();
    k_img_rows_inv<<<dim3(n, nimg), thr, sm, st>>>(C, n, m, pl->ws.tw2, out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

int fft_set_smem_limits(int bytes) {
    DGCT_TRY(raise_smem_limit((const void*)k_filter_views<float>, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_filter_views<bf16s>, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_img_rows_fwd, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_img_cols, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_img_rows_inv, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_img_rows_inv_update, bytes));
    return DGAMP_CT_OK;
}

}  // namespace dgct
