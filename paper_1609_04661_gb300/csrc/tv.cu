// Denoiser and divergence, Algorithm 1 Step 4 (Section 4.3, Section 6.3).
//
// D is the l2 proximal map of isotropic TV, solved by Chambolle's 2004 dual
// projection (forward differences, Neumann boundary, step 1/8, fixed
// iteration count from a zero dual).  The MC divergence of Eq. MC_SURE with
// one probe needs D at r and at r + eps b; both images are denoised by the
// same launches (blockIdx.z selects the image), and the final kernel forms
// x = D(r), b^T (D(r + eps b) - D(r)) in FP64, and -- inside a solve --
// tau_x = max(tau_r D', floor tau_r) for the next iteration.
//
// Dual layout: float2 (px, py) per pixel, [image][n][n], ping-pong buffers.
// px is the dual of the horizontal difference, py of the vertical one; px in
// the last column and py in the last row stay zero (their differences are
// zero), so div p = px(i,j) - px(i,j-1) + py(i,j) - py(i-1,j) with the
// out-of-image terms taken as zero reproduces the Neumann divergence.
#include "internal.cuh"

namespace dgct {

constexpr int TX = 32, TY = 8;
constexpr float kTau = 0.125f;

__device__ __forceinline__ float solve_lambda(const DevScalars* S, float c_tv, int from_scalars,
                                              float lambda_arg) {
    return from_scalars ? c_tv * sqrtf((float)S->tau_r) : lambda_arg;
}

// --------------------------------------------------------- probe input ----
// r2 = r + eps b, eps = eps_rel max(max|r|, 1e-6).  One thread per block of
// four probe elements (one Philox call).
__global__ void k_probe_input(const float* __restrict__ r, float* __restrict__ r2, long long N,
                              float eps_rel, int t_arg, unsigned slice, uint2 key,
                              DevScalars* S) {
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
        if (i0 + k < N) r2[i0 + k] = fmaf(eps, bb[k], r[i0 + k]);
}

int launch_probe_input(const dgamp_ct_plan_s* pl, int t_arg, cudaStream_t st) {
    const long long N = pl->N;
    const long long groups = (N + 3) / 4;
    const uint2 key = make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
    k_probe_input<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(
        pl->ws.r, pl->ws.r + N, N, (float)pl->opt.eps_rel, t_arg, (unsigned)pl->opt.slice_id, key,
        pl->ws.S);
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

// ------------------------------------------------------ Chambolle step ----
// One iteration p <- (p + tau grad q) / (1 + tau |grad q|), q = div p - r/lambda.
// Tile TX x TY pixels; q is formed in shared memory on the tile plus one
// column to the right and one row below; p is read with a one-pixel halo
// above and to the left.
template <bool FIRST>
__global__ void __launch_bounds__(TX * TY)
k_tv_iter(const float* __restrict__ rbase, const float2* __restrict__ pin, float2* __restrict__ pout,
          int n, float c_tv, int from_scalars, float lambda_arg, const DevScalars* __restrict__ S) {
    __shared__ float2 sp[TY + 2][TX + 2];   // p at rows i0-1..i0+TY, cols j0-1..j0+TX
    __shared__ float sq[TY + 1][TX + 1];    // q at rows i0..i0+TY, cols j0..j0+TX
    const size_t N = (size_t)n * n;
    const int img = blockIdx.z;
    const float* __restrict__ r = rbase + img * N;
    const float2* __restrict__ P = pin + img * N;
    float2* __restrict__ Q = pout + img * N;
    const int i0 = blockIdx.y * TY, j0 = blockIdx.x * TX;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const float inv_lam = 1.0f / lam;
    if (!FIRST) {
        for (int e = tid; e < (TY + 2) * (TX + 2); e += TX * TY) {
            const int a = e / (TX + 2), b = e % (TX + 2);
            const int gi = i0 - 1 + a, gj = j0 - 1 + b;
            sp[a][b] = (gi >= 0 && gi < n && gj >= 0 && gj < n) ? P[(size_t)gi * n + gj]
                                                                 : make_float2(0.f, 0.f);
        }
        __syncthreads();
    }
    for (int e = tid; e < (TY + 1) * (TX + 1); e += TX * TY) {
        const int a = e / (TX + 1), b = e % (TX + 1);
        const int gi = i0 + a, gj = j0 + b;
        float q = 0.f;
        if (gi < n && gj < n) {
            float dv = 0.f;
            if (!FIRST) dv = sp[a + 1][b + 1].x - sp[a + 1][b].x + sp[a + 1][b + 1].y - sp[a][b + 1].y;
            q = dv - r[(size_t)gi * n + gj] * inv_lam;
        }
        sq[a][b] = q;
    }
    __syncthreads();
    const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
    if (i >= n || j >= n) return;
    const float qc = sq[threadIdx.y][threadIdx.x];
    const float gx = (j < n - 1) ? sq[threadIdx.y][threadIdx.x + 1] - qc : 0.f;
    const float gy = (i < n - 1) ? sq[threadIdx.y + 1][threadIdx.x] - qc : 0.f;
    const float den = 1.f + kTau * sqrtf(gx * gx + gy * gy);
    float2 pv = FIRST ? make_float2(0.f, 0.f) : sp[threadIdx.y + 1][threadIdx.x + 1];
    pv.x = (pv.x + kTau * gx) / den;
    pv.y = (pv.y + kTau * gy) / den;
    Q[(size_t)i * n + j] = pv;
}

bool tv_active(const dgamp_ct_plan_s* pl, int from_scalars, double lambda_arg) {
    if (pl->opt.k_tv <= 0) return false;
    return from_scalars ? pl->opt.c_tv > 0.0 : lambda_arg > 0.0;
}

// Chambolle iteration i (0-based) on nimg images of ws.r: iteration i writes
// dual buffer i & 1 and reads buffer (i - 1) & 1; *final_buf names the buffer
// written.
int launch_tv_step(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg, int i,
                   cudaStream_t st, int* final_buf) {
    const int n = pl->n;
    const size_t N = (size_t)pl->N;
    float2* buf[2] = {pl->ws.p, pl->ws.p + 2 * N};
    dim3 blk(TX, TY), grd((n + TX - 1) / TX, (n + TY - 1) / TY, nimg);
    const float c_tv = (float)pl->opt.c_tv;
    if (i == 0)
        k_tv_iter<true><<<grd, blk, 0, st>>>(pl->ws.r, buf[0], buf[0], n, c_tv, from_scalars,
                                              (float)lambda_arg, pl->ws.S);
    else
        k_tv_iter<false><<<grd, blk, 0, st>>>(pl->ws.r, buf[(i - 1) & 1], buf[i & 1], n, c_tv,
                                               from_scalars, (float)lambda_arg, pl->ws.S);
    DGCT_LAUNCH_CHECK();
    *final_buf = i & 1;
    return DGAMP_CT_OK;
}

// k_tv iterations (none when lambda would be 0); *final_buf = -1 means x = r.
int launch_tv_iters(const dgamp_ct_plan_s* pl, int nimg, int from_scalars, double lambda_arg,
                    cudaStream_t st, int* final_buf) {
    *final_buf = -1;
    if (!tv_active(pl, from_scalars, lambda_arg)) return DGAMP_CT_OK;
    for (int i = 0; i < pl->opt.k_tv; ++i) {
        const int rc = launch_tv_step(pl, nimg, from_scalars, lambda_arg, i, st, final_buf);
        if (rc != DGAMP_CT_OK) return rc;
    }
    return DGAMP_CT_OK;
}

// ------------------------------------------------------- final step -----
// x = r - lambda div p for each image; optional staging of x for the next
// projection; divergence b^T (x2 - x1) / (N eps) and, in a solve, tau_x.
// Tiles of 32 x 32 pixels so that the transposed staging write is coalesced.
__global__ void __launch_bounds__(TX * TY)
k_tv_final(const float* __restrict__ rbase, const float2* __restrict__ pbase, int have_p, int n,
           int nimg, float c_tv, int from_scalars, float lambda_arg, float* x_out,
           float* __restrict__ XR, float* __restrict__ XC, int ldp, float damp_x, int t_arg,
           unsigned slice, uint2 key, double tau_r_arg, double tau_x_floor, DevScalars* S,
           double* partial, IterLog* log, double* div_out, int solve_mode) {
    __shared__ float tile[32][33];
    __shared__ double sm[32];
    __shared__ bool am_last;
    const size_t N = (size_t)n * n;
    const float lam = solve_lambda(S, c_tv, from_scalars, lambda_arg);
    const unsigned t = t_arg > 0 ? (unsigned)t_arg : S->t;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    double acc = 0.0;
    for (int jj = threadIdx.y; jj < 32; jj += TY) {
        const int i = by + jj, j = bx + threadIdx.x;
        float xv = 0.f;
        if (i < n && j < n) {
            const size_t o = (size_t)i * n + j;
            float xs[2];
            for (int im = 0; im < nimg; ++im) {
                float dv = 0.f;
                if (have_p) {
                    const float2* P = pbase + im * N;
                    const float2 pc = P[o];
                    dv = pc.x + pc.y;
                    if (j > 0) dv -= P[o - 1].x;
                    if (i > 0) dv -= P[o - n].y;
                }
                xs[im] = rbase[im * N + o] - lam * dv;
            }
            xv = xs[0];
            if (nimg == 2) {
                const float4 b4 = probe4((unsigned)(o >> 2), t, slice, key);
                const int k = (int)(o & 3);
                const float b = k == 0 ? b4.x : (k == 1 ? b4.y : (k == 2 ? b4.z : b4.w));
                acc += (double)b * (double)(xs[1] - xs[0]);
            }
            if (solve_mode && damp_x != 1.f) xv = damp_x * xv + (1.f - damp_x) * x_out[o];
            x_out[o] = xv;
            if (XR) XR[(size_t)i * ldp + kPad + j] = xv;
        }
        tile[jj][threadIdx.x] = xv;
    }
    if (XC) {
        __syncthreads();
        for (int jj = threadIdx.y; jj < 32; jj += TY) {
            const int j = bx + jj, i = by + threadIdx.x;
            if (i < n && j < n) XC[(size_t)j * ldp + kPad + i] = tile[threadIdx.x][jj];
        }
    }
    if (nimg < 2) return;
    acc = block_sum(acc, sm);
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        partial[bid] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&S->done_div, 1u);
        am_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int tid = threadIdx.y * TX + threadIdx.x;
    double tot = 0.0;
    for (int b = tid; b < nblk; b += TX * TY) tot += ((volatile double*)partial)[b];
    tot = block_sum(tot, sm);
    if (tid == 0) {
        const double div = tot / ((double)N * S->eps);
        if (div_out) *div_out = div;
        if (solve_mode) {
            const double tau_r = S->tau_r;
            double tx = tau_r * div;
            const double fl = tau_x_floor * tau_r;
            if (!(tx >= fl)) { tx = fl; S->floored += 1u; }
            if (!isfinite(tx)) S->nonfinite += 1u;
            S->div = div;
            S->tau_x = tx;
            const unsigned tt = S->t;
            if (tt >= 1u && tt <= (unsigned)kMaxIters) {
                IterLog L;
                L.tau_x = tx; L.tau_p = S->tau_p; L.tau_s = S->tau_s; L.tau_r = tau_r;
                L.div = div; L.eps = S->eps;
                log[tt - 1] = L;
            }
            S->t = tt + 1u;
        }
        (void)tau_r_arg;
        S->done_div = 0u;
    }
}

int launch_tv_final(const dgamp_ct_plan_s* pl, int nimg, int final_buf, int from_scalars,
                    double lambda_arg, float* x_out, int solve_mode, int t_arg, double* div_out,
                    cudaStream_t st) {
    const int n = pl->n;
    const size_t N = (size_t)pl->N;
    const float2* pb = final_buf < 0 ? pl->ws.p : pl->ws.p + (size_t)final_buf * 2 * N;
    dim3 blk(TX, TY), grd((n + 31) / 32, (n + 31) / 32);
    const uint2 key = make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
    k_tv_final<<<grd, blk, 0, st>>>(pl->ws.r, pb, final_buf >= 0, n, nimg, (float)pl->opt.c_tv,
                                    from_scalars, (float)lambda_arg, x_out,
                                    solve_mode ? pl->ws.XR : nullptr, solve_mode ? pl->ws.XC : nullptr,
                                    pl->ldp, (float)pl->opt.damp_x, t_arg, (unsigned)pl->opt.slice_id,
                                    key, 0.0, pl->opt.tau_x_floor, pl->ws.S, pl->ws.partial,
                                    pl->ws.log, div_out, solve_mode);
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
    const uint2 key = make_uint2((unsigned)(pl->opt.seed & 0xffffffffu), (unsigned)(pl->opt.seed >> 32));
    k_probe<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(n, t, (unsigned)pl->opt.slice_id, key, b,
                                                              words);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
