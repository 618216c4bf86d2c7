// Prox-TV in the norm of the preconditioned space (Section 6.3, option
// tv_metric): Section 4.3 lets the denoiser act with the norm of the space
// that x = V mu lives in, and Section 6.3 compares the l2 prox-TV with the one
// in the (V^T V)^{-1} norm.  The norm is read as the Mahalanobis distance of
// the covariance Q = (V^T V)^{-1} (the covariance white noise takes on
// through V^-1, Eq. r_input):
//
//     D(r) = argmin_x 1/2 (x - r)^T Q^{-1} (x - r) + lambda TV(x).
//
// On the paper's Fourier grid Q = F^-1 C^-1 F, the radial gain |rho|; it is
// realised like V^-1 (fft.cu): the gain max(rho, f0), f0 = 1/(2P), on the
// m x m zero-padded grid, cropped to n x n.  Only Q is ever applied.  Writing
// lambda |grad x|_i as the largest lambda p_i . (grad x)_i over |p_i| <= 1 and
// minimising over x first gives x(p) = r + lambda Q div p, and the dual is
// solved by projected gradient ascent (Chambolle 2005; Beck and Teboulle
// 2009 for the dual TV problem):
//
//     x_k = r + lambda Q div p_k,
//     p_{k+1} = Proj_{|p_i| <= 1}(p_k + theta / lambda grad x_k),
//     theta = 1 / (8 q_max)  (||grad||^2 <= 8, ||Q|| <= q_max),
//
// from p_0 = 0 for k_tv steps, returning x(p_{k_tv}).  grad, div and the
// Neumann boundary are those of the l2 prox (tv.cu): forward differences,
// the last difference in each direction zero, so duals on the last column
// (x part) and last row (y part) stay zero and div p needs no special case.
//
// The gain max(rho, f0) is real and even, so the filter maps real images to
// real images: the two images of the MC pair (D(r) and D(r + eps b)) travel
// as the real and imaginary parts of one complex image through the three
// FFT passes, which halves their work (a single image has a zero imaginary
// part).  Launch sequence for K = k_tv >= 1 (4K + 1 launches):
//   0                      dual step from p = 0 with x_0 = r
//   4s-3, 4s-2, 4s-1       x_s = r + lambda Q div p_s     (s = 1 .. K)
//                          (rows: div p and row FFTs; columns: FFT, gain,
//                          inverse FFT; rows: inverse FFTs and r + lambda .)
//   4s    (s < K)          dual step
//   4K                     the TV final step on x_K (tv.cu): damping, the
//                          staged copies, the divergence and tau_x.
// Buffers (no allocation of their own): the duals use the first 2 N float2
// of the l2 prox's dual buffer ws.p and x(p) its second half as floats; the
// row spectra use the first n m entries of ws.fft2d (m x m).
#include <cmath>

#include "fft_device.cuh"

namespace dgct {

static int tvm_threads(int m) { return m / 8 < 32 ? 32 : (m / 8 > 512 ? 512 : m / 8); }

static float tvm_theta(const dgamp_ct_plan_s* pl) {
    // the largest gain on the m x m grid: rho at (-1/2, -1/2) = sqrt(1/2)
    // (m >= 4 is even), or the floor if that were larger
    const double f0 = 1.0 / (2.0 * pl->P);
    const double qmax = std::sqrt(0.5) > f0 ? std::sqrt(0.5) : f0;
    return (float)(1.0 / (8.0 * qmax));
}

// div p at (iy, i) of one image's duals (zero duals on the last column and row).
__device__ __forceinline__ float tvm_div(const float2* __restrict__ prow, int iy, int i, int n) {
    const float2 pc = prow[i];
    float d = pc.x + pc.y;
    if (i > 0) d -= prow[i - 1].x;
    if (iy > 0) d -= prow[i - n].y;     // p_y of the row above
    return d;
}

// Row iy < n: div p of image 0 (real part) and image 1 (imaginary part, or
// zero when nimg = 1), zero-padded to m, forward FFT -> C[iy][0..m).
__global__ void __launch_bounds__(512)
k_tvm_rows_fwd(const float2* __restrict__ p, int nimg, int n, int m, const float2* __restrict__ tw,
               float2* __restrict__ C) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int iy = blockIdx.x;
    const size_t N = (size_t)n * n;
    const float2* prow0 = p + (size_t)iy * n;
    const float2* prow1 = prow0 + N;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        float d0 = 0.f, d1 = 0.f;
        if (i < n) {
            d0 = tvm_div(prow0, iy, i, n);
            if (nimg == 2) d1 = tvm_div(prow1, iy, i, n);
        }
        a[fpad(i)] = make_float2(d0, d1);
    }
    __syncthreads();
    const float2* r = fft_stockham(a, b, m, tw, -1.f);
    float2* crow = C + (size_t)iy * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) crow[i] = r[fpad(i)];
}

// Column kx: forward FFT over the rows (rows >= n are zero), times
// max(rho, f0), inverse FFT; rows < n are stored back.
__global__ void __launch_bounds__(512)
k_tvm_cols(float2* __restrict__ C, int n, int m, const float2* __restrict__ tw, float f0) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int kx = blockIdx.x;
    float2* Ci = C;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        a[fpad(i)] = i < n ? Ci[(size_t)i * m + kx] : make_float2(0.f, 0.f);
    __syncthreads();
    float2* r = fft_stockham(a, b, m, tw, -1.f);
    float2* o = (r == a) ? b : a;
    const float fx = (float)(kx <= m / 2 ? kx : kx - m) / (float)m;
    for (int ky = threadIdx.x; ky < m; ky += blockDim.x) {
        const float fy = (float)(ky <= m / 2 ? ky : ky - m) / (float)m;
        const float g = fmaxf(sqrtf(fx * fx + fy * fy), f0);
        const float2 v = r[fpad(ky)];
        r[fpad(ky)] = make_float2(v.x * g, v.y * g);
    }
    __syncthreads();
    r = fft_stockham(r, o, m, tw, 1.f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) Ci[(size_t)i * m + kx] = r[fpad(i)];
}

// Row iy: inverse FFT; on the first n columns X_0 = r_0 + lambda Re(.) / m^2
// and (nimg = 2) X_1 = r_1 + lambda Im(.) / m^2.
__global__ void __launch_bounds__(512)
k_tvm_rows_inv(const float2* __restrict__ C, int nimg, int n, int m, const float2* __restrict__ tw,
               const float* __restrict__ rimg, float* __restrict__ X, const DevScalars* S, float c_tv,
               int from_scalars, float lambda_arg) {
    extern __shared__ float2 smem[];
    float2* a = smem;
    float2* b = smem + fft_buf_len(m);
    const int iy = blockIdx.x;
    const float2* crow = C + (size_t)iy * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[fpad(i)] = crow[i];
    __syncthreads();
    const float2* r = fft_stockham(a, b, m, tw, 1.f);
    const float sc = solve_lambda(S, c_tv, from_scalars, lambda_arg) / ((float)m * (float)m);
    const size_t N = (size_t)n * n, row = (size_t)iy * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float2 v = r[fpad(i)];
        X[row + i] = fmaf(sc, v.x, rimg[row + i]);
        if (nimg == 2) X[N + row + i] = fmaf(sc, v.y, rimg[N + row + i]);
    }
}

// One dual step on image blockIdx.y, one pixel per thread:
// p <- Proj_{|p| <= 1}(p + theta / lambda grad X), p = 0 before the first.
__global__ void __launch_bounds__(256)
k_tvm_dual(const float* __restrict__ X, float2* __restrict__ p, int n, int first, float theta,
           const DevScalars* S, float c_tv, int from_scalars, float lambda_arg) {
    const size_t N = (size_t)n * n;
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= N) return;
    const int iy = (int)(o / (size_t)n), ix = (int)(o - (size_t)iy * n);
    const float* Xi = X + (size_t)blockIdx.y * N;
    float2* pi = p + (size_t)blockIdx.y * N;
    const float xc = Xi[o];
    const float gx = ix < n - 1 ? Xi[o + 1] - xc : 0.f;
    const float gy = iy < n - 1 ? Xi[o + n] - xc : 0.f;
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const float step = lam > 0.f ? theta / lam : 0.f;
    float2 q = first ? make_float2(0.f, 0.f) : pi[o];
    q.x = fmaf(step, gx, q.x);
    q.y = fmaf(step, gy, q.y);
    const float nrm = fmaxf(sqrtf(q.x * q.x + q.y * q.y), 1.f);
    pi[o] = make_float2(q.x / nrm, q.y / nrm);
}

int tvm_num_launches(const dgamp_ct_plan_s* pl) { return 4 * pl->opt.k_tv + 1; }

// Launch i of the sequence above on nimg images of ws.r (the caller has
// checked that the denoiser is active: k_tv >= 1 and lambda > 0).
int launch_tvm_chunk(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                     float* x_out, int solve_mode, int t_arg, double* div_out, cudaStream_t st) {
    const int n = pl->n, m = pl->m2, K = pl->opt.k_tv;
    const size_t N = (size_t)pl->N;
    if (nimg < 1 || nimg > 2 || K < 1 || i < 0 || i > 4 * K || (size_t)n * m > (size_t)m * m)
        return DGAMP_CT_ERR_INVALID_ARG;
    float2* p = pl->ws.p;                                        // [nimg][n][n] float2
    float* X = reinterpret_cast<float*>(pl->ws.p + 2 * N);       // [nimg][n][n] float
    const float c_tv = (float)pl->opt.c_tv, lam = (float)lambda_arg;
    const int phase = i == 0 ? 3 : (i - 1) % 4;
    if (i == 4 * K) return launch_tv_final_x(pl, nimg, X, x_out, solve_mode, t_arg, div_out, st);
    if (phase == 3) {
        const dim3 grd((unsigned)((N + 255) / 256), (unsigned)nimg);
        k_tvm_dual<<<grd, 256, 0, st>>>(i == 0 ? pl->ws.r : X, p, n, i == 0 ? 1 : 0, tvm_theta(pl), pl->ws.S,
                                        c_tv, from_scalars, lam);
        DGCT_LAUNCH_CHECK();
        return DGAMP_CT_OK;
    }
    const size_t sm = (size_t)2 * fft_buf_len(m) * sizeof(float2);
    const int thr = tvm_threads(m);
    if (phase == 0)
        k_tvm_rows_fwd<<<n, thr, sm, st>>>(p, nimg, n, m, pl->ws.tw2, pl->ws.fft2d);
    else if (phase == 1)
        k_tvm_cols<<<m, thr, sm, st>>>(pl->ws.fft2d, n, m, pl->ws.tw2, (float)(1.0 / (2.0 * pl->P)));
    else
        k_tvm_rows_inv<<<n, thr, sm, st>>>(pl->ws.fft2d, nimg, n, m, pl->ws.tw2, pl->ws.r, X, pl->ws.S, c_tv,
                                           from_scalars, lam);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

int tvm_set_smem_limits(int bytes) {
    DGCT_TRY(raise_smem_limit((const void*)k_tvm_rows_fwd, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_tvm_cols, bytes));
    DGCT_TRY(raise_smem_limit((const void*)k_tvm_rows_inv, bytes));
    return DGAMP_CT_OK;
}

}  // namespace dgct
