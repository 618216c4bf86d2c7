// Learned denoiser of Step 4 (Section 4.3 black-box denoiser; the residual
// CNN the paper points to in Section 1): forward, backward and Adam on the GPU.
//
//   f: 17 layers of 3x3 same-padded convolutions, 1 -> 64 -> ... -> 64 -> 1,
//      bias per output channel, ReLU after layers 1..16;
//   D_sigma(r) = r - sigma f(r / sigma)   (residual form, scale-normalised).
//
// Layout.  Images FP32 [B][H][W]; hidden activations BF16 channels-last
// [B][H][W][64]; master parameters FP32 in the flat order of the reference
// (per layer W[ky][kx][ci][co] then b[co]); compute copies of the 15 hidden
// weight tensors in BF16 as [co][k] (k = tap*64 + ci) for the forward pass and
// as [ci][k'] (k' = (8 - tap)*64 + co) for the input gradient, which is then
// a forward convolution of the output gradient with the flipped, transposed
// kernel.
//
// The 64 -> 64 layers (forward, input gradient and forward-mode tangent) are
// implicit GEMMs on the tcgen05 tensor cores with TMEM accumulators
// (conv_tc.cu), and so is their weight gradient (M = 64 co, N = 64 ci per
// tap, K = pixels), which writes per-CTA FP32 partials that a second kernel
// adds in a fixed order.  The first (1 -> 64) and last
// (64 -> 1) layers are small and run on the CUDA cores.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"

namespace dgct {

constexpr int CH = 64;          // hidden channels
constexpr int KW = 9 * CH;      // GEMM K of a hidden layer (576)
constexpr int PSTR = 72;        // shared-memory stride (bf16) of one pixel's 64 channels

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------- first layer --
// a1 = relu(b0 + conv(u, W0)), u = r / sigma; also stores u for the weight gradient.
// Tangent form (b0 == nullptr, mask != nullptr): a1 = conv(u, W0) where the
// primal layer-1 activation `mask` is positive, else 0.
//
// Activations are [pixel][64] BF16, 128 bytes per pixel, so the 32 pixels of
// a warp touch 32 rows: a warp's output rows (and mask rows) pass through
// shared memory and reach global memory as whole rows, contiguous across the
// warp.  In shared memory a row takes PSTR = 72 BF16 (144 bytes), so the
// eight lanes of one 16-byte access phase that touch the same chunk of eight
// consecutive rows hit distinct banks, while every lane works on the same
// chunk and the weights it reads are broadcasts.
constexpr int kC1Threads = 128;

__global__ void __launch_bounds__(kC1Threads)
k_conv_first(const float* __restrict__ r, const float* __restrict__ sigma, int B, int H, int W,
             const float* __restrict__ w0, const float* __restrict__ b0,
             const bf16* __restrict__ mask, bf16* __restrict__ a1, float* __restrict__ u_out) {
    __shared__ float sw[9 * CH + CH];
    __shared__ __align__(16) bf16 stage[kC1Threads / 32][32 * PSTR];   // one warp's 32 rows
    for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w0[i];
    for (int i = threadIdx.x; i < CH; i += blockDim.x) sw[9 * CH + i] = b0 ? b0[i] : 0.f;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long HW = (long long)H * W, total = (long long)B * HW;
    const long long p0 = (long long)blockIdx.x * kC1Threads + wp * 32, p = p0 + lane;
    bf16* S = stage[wp];
    if (mask) {   // the warp's mask rows, contiguous loads
        for (int i = lane; i < 32 * 8; i += 32) {
            const long long pp = p0 + (i >> 3);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (pp < total) v = *reinterpret_cast<const uint4*>(mask + pp * CH + (i & 7) * 8);
            *reinterpret_cast<uint4*>(S + (i >> 3) * PSTR + (i & 7) * 8) = v;
        }
    }
    __syncthreads();
    const bool live = p < total;
    const int b = live ? (int)(p / HW) : 0;
    const int y = live ? (int)((p - b * HW) / W) : 0, x = live ? (int)(p - b * HW - (long long)y * W) : 0;
    const float inv = 1.0f / sigma[b];
    const float* img = r + b * HW;
    float u[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        u[t] = (live && yy >= 0 && yy < H && xx >= 0 && xx < W) ? img[(long long)yy * W + xx] * inv : 0.f;
    }
    if (u_out && live) u_out[p] = u[4];
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int c0 = k * 8;
        bf16* row = S + lane * PSTR + c0;
        __align__(16) bf16 v[8];
        __align__(16) bf16 mk[8];
        if (mask) *reinterpret_cast<uint4*>(mk) = *reinterpret_cast<const uint4*>(row);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float acc = sw[9 * CH + c0 + j];
#pragma unroll
            for (int t = 0; t < 9; ++t) acc = fmaf(u[t], sw[t * CH + c0 + j], acc);
            if (mask)
                v[j] = __float2bfloat16_rn(__bfloat162float(mk[j]) > 0.f ? acc : 0.f);
            else
                v[j] = __float2bfloat16_rn(fmaxf(acc, 0.f));
        }
        *reinterpret_cast<uint4*>(row) = *reinterpret_cast<const uint4*>(v);
    }
    __syncwarp();
    for (int i = lane; i < 32 * 8; i += 32) {   // the warp's rows, contiguous stores
        const long long pp = p0 + (i >> 3);
        if (pp < total)
            *reinterpret_cast<uint4*>(a1 + pp * CH + (i & 7) * 8) =
                *reinterpret_cast<const uint4*>(S + (i >> 3) * PSTR + (i & 7) * 8);
    }
}

// ------------------------------------------------------ hidden 64 -> 64 --
// On the tcgen05 tensor cores, conv_tc.cu (launch_conv64_tc): mode 0 is the
// forward layer relu(bias + conv(in, Wk)); mode 1 the masked linear layer
// conv(in, Wk) * (mask > 0).  With Wk = the flipped/transposed kernel, `in`
// = the output gradient and mask = this layer's input activation, mode 1 is
// the input gradient; with Wk = the forward kernel, `in` = a tangent and mask
// = the primal output activation of this layer, it is the forward-mode
// derivative.

// ------------------------------------------------------------ last layer --
// f = b16 + conv(a16, W16) (W16 as [tap][ci]); D = r - sigma f.  b16 == nullptr
// drops the bias (tangent form: r = the direction b, D = b - sigma J_f (b / sigma)).
// A block computes kCLRows x kCLCols pixels (warp = one row, lane = one
// pixel) from the tile of input rows with its one-pixel halo, staged in shared
// memory by contiguous 16-byte loads (rows PSTR apart, as in k_conv_first);
// each lane reads its nine 128-byte taps there.
constexpr int kCLRows = 4, kCLCols = 32;
constexpr int kCLTile = (kCLRows + 2) * (kCLCols + 2);      // staged pixels

__global__ void __launch_bounds__(32 * kCLRows)
k_conv_last(const bf16* __restrict__ a16, const float* __restrict__ w16, const float* __restrict__ b16,
            const float* __restrict__ r, const float* __restrict__ sigma, int B, int H, int W,
            float* __restrict__ f_out, float* __restrict__ d_out) {
    __shared__ __align__(16) float sw[9 * CH];
    __shared__ __align__(16) bf16 tile[kCLTile * PSTR];
    for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w16[i];
    const int bz = blockIdx.z, x0 = blockIdx.x * kCLCols, y0 = blockIdx.y * kCLRows;
    for (int i = threadIdx.x; i < kCLTile * 8; i += blockDim.x) {
        const int pix = i >> 3, ch = (i & 7) * 8;
        const int yy = y0 - 1 + pix / (kCLCols + 2), xx = x0 - 1 + pix % (kCLCols + 2);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (yy >= 0 && yy < H && xx >= 0 && xx < W)
            v = *reinterpret_cast<const uint4*>(a16 + (((long long)bz * H + yy) * W + xx) * CH + ch);
        *reinterpret_cast<uint4*>(tile + pix * PSTR + ch) = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int y = y0 + wp, x = x0 + lane;
    float acc = b16 ? b16[0] : 0.f;
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
        const bf16* src = tile + ((wp + t / 3) * (kCLCols + 2) + lane + t % 3) * PSTR;
        const float* wt = sw + t * CH;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c0 = k * 8;
            const uint4 raw = *reinterpret_cast<const uint4*>(src + c0);
            const float4 wa = *reinterpret_cast<const float4*>(wt + c0);
            const float4 wb = *reinterpret_cast<const float4*>(wt + c0 + 4);
            const __nv_bfloat162* v2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
            const float2 f0 = __bfloat1622float2(v2[0]), f1 = __bfloat1622float2(v2[1]);
            const float2 f2 = __bfloat1622float2(v2[2]), f3 = __bfloat1622float2(v2[3]);
            acc = fmaf(f0.x, wa.x, acc);
            acc = fmaf(f0.y, wa.y, acc);
            acc = fmaf(f1.x, wa.z, acc);
            acc = fmaf(f1.y, wa.w, acc);
            acc = fmaf(f2.x, wb.x, acc);
            acc = fmaf(f2.y, wb.y, acc);
            acc = fmaf(f3.x, wb.z, acc);
            acc = fmaf(f3.y, wb.w, acc);
        }
    }
    if (y >= H || x >= W) return;
    const long long p = ((long long)bz * H + y) * W + x;
    if (f_out) f_out[p] = acc;
    if (d_out) d_out[p] = r[p] - sigma[bz] * acc;
}

static dim3 conv_last_grid(int B, int H, int W) {
    return dim3((unsigned)((W + kCLCols - 1) / kCLCols), (unsigned)((H + kCLRows - 1) / kCLRows), (unsigned)B);
}

// g16 = (sum_tap gout[p - off(tap)] W16[tap][ci]) * (a16 > 0)
__global__ void k_dgrad_last(const float* __restrict__ gout, const float* __restrict__ w16,
                             const bf16* __restrict__ a16, bf16* __restrict__ g16, int B, int H, int W) {
    __shared__ float sw[9 * CH];
    for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w16[i];
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long HW = (long long)H * W;
    if (p >= (long long)B * HW) return;
    const int b = (int)(p / HW);
    const int y = (int)((p - b * HW) / W), x = (int)(p - b * HW - (long long)y * W);
    float gv[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
        gv[t] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? gout[b * HW + (long long)yy * W + xx] : 0.f;
    }
    const bf16* a = a16 + p * CH;
    bf16* g = g16 + p * CH;
    for (int c0 = 0; c0 < CH; c0 += 8) {
        const uint4 raw = *reinterpret_cast<const uint4*>(a + c0);
        const bf16* av = reinterpret_cast<const bf16*>(&raw);
        __align__(16) bf16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) acc = fmaf(gv[t], sw[t * CH + c0 + k], acc);
            o[k] = __float2bfloat16_rn(__bfloat162float(av[k]) > 0.f ? acc : 0.f);
        }
        *reinterpret_cast<uint4*>(g + c0) = *reinterpret_cast<const uint4*>(o);
    }
}

// ----------------------------------------------------- weight gradients --
// All parameter gradients are sums over the batch's pixels.  Each kernel below
// sums a fixed range of pixels per block in FP32 (a thread's pixels, then the
// block's threads in a fixed tree) and writes one row of FP32 partials; a
// second kernel adds the rows in a fixed order.  Nothing depends on timing, so
// the gradients are reproducible run to run.

// grad W (reference layout [tap][ci][co]) = sum over groups of
// partial[group][tap][ci][co] (the tensor-core kernel's layout)
__global__ void k_reduce_wgrad64(const float* __restrict__ partial, int ngroups, float* __restrict__ gw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;     // index in [tap][ci][co]
    if (i >= 9 * CH * CH) return;
    float s = 0.f;
    for (int gq = 0; gq < ngroups; ++gq) s += partial[(size_t)gq * 9 * CH * CH + i];
    gw[i] = s;
}

// out[col] = sum over rows of partial[row][col]: one warp per column, the
// lanes' strided sums then a butterfly (the same order every run)
__global__ void k_reduce_cols(const float* __restrict__ partial, int nrows, int width, float* __restrict__ out) {
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (col >= width) return;
    float s = 0.f;
    for (int r = lane; r < nrows; r += 32) s += partial[(size_t)r * width + col];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[col] = s;
}

// Blocks of the pixel-sum kernels: about 256 pixels each, at most kColBlocks.
constexpr int kColBlocks = 1024;
static int col_blocks(long long npix) {
    const long long b = (npix + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), kColBlocks);
}

// Thread layout of the pixel-sum kernels (256 threads): thread t takes the
// 8 channels 8 (t % 8) .. + 7 of every 32nd pixel of the block's range,
// starting at pixel t / 8; a warp holds 4 pixel lanes, summed by shuffles
// across lanes 8 and 16 apart, then the 8 warps through shared memory.
template <int NV>
__device__ __forceinline__ void block_colsum(float (&s)[NV][8], float (*sm)[NV * CH], float* __restrict__ out) {
    const int cg = threadIdx.x & 7, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s[v][k] += __shfl_xor_sync(0xffffffffu, s[v][k], 8);
            s[v][k] += __shfl_xor_sync(0xffffffffu, s[v][k], 16);
        }
    if (lane < 8)
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int k = 0; k < 8; ++k) sm[warp][v * CH + cg * 8 + k] = s[v][k];
    __syncthreads();
    for (int i = threadIdx.x; i < NV * CH; i += blockDim.x) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += sm[w][i];
        out[i] = t;
    }
}

__device__ __forceinline__ void unpack8(const uint4& v, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

// bias gradient: partial[block][c] = sum over the block's pixels of g[p][c]
__global__ void __launch_bounds__(256) k_bias_partial(const bf16* __restrict__ g, long long npix, long long per,
                                                      float* __restrict__ partial) {
    __shared__ float sm[8][CH];
    const int cg = threadIdx.x & 7, pl = threadIdx.x >> 3;
    const long long p0 = (long long)blockIdx.x * per, p1 = std::min(p0 + per, npix);
    float s[1][8] = {};
    for (long long p = p0 + pl; p < p1; p += 32) {
        float f[8];
        unpack8(*reinterpret_cast<const uint4*>(g + p * CH + cg * 8), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[0][k] += f[k];
    }
    block_colsum<1>(s, sm, partial + (size_t)blockIdx.x * CH);
}

// First layer: partial[block][tap*64 + co] = sum_p u[p + off(tap)] g1[p][co];
// partial[block][9*64 + co] = sum_p g1[p][co].  u is the scaled input r/sigma.
__global__ void __launch_bounds__(256) k_wgrad_first(const float* __restrict__ r, const float* __restrict__ sigma,
                                                     const bf16* __restrict__ g1, int B, int H, int W, long long per,
                                                     float* __restrict__ partial) {
    __shared__ float sm[8][10 * CH];
    const int cg = threadIdx.x & 7, pl = threadIdx.x >> 3;
    const long long HW = (long long)H * W, npix = B * HW;
    const long long p0 = (long long)blockIdx.x * per, p1 = std::min(p0 + per, npix);
    float s[10][8] = {};
    for (long long p = p0 + pl; p < p1; p += 32) {
        const int b = (int)(p / HW);
        const int y = (int)((p - b * HW) / W), x = (int)(p - b * HW - (long long)y * W);
        const float inv = 1.0f / sigma[b];
        float gv[8];
        unpack8(*reinterpret_cast<const uint4*>(g1 + p * CH + cg * 8), gv);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            const float u = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? r[b * HW + (long long)yy * W + xx] * inv : 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) s[t][k] = fmaf(u, gv[k], s[t][k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) s[9][k] += gv[k];
    }
    block_colsum<10>(s, sm, partial + (size_t)blockIdx.x * 10 * CH);
}

// Last layer: partial[block][tap*64 + ci] = sum_p a16[p + off(tap)][ci] gout[p];
// partial[block][9*64] = sum_p gout[p] (columns 9*64 + 1 .. 10*64 - 1 are zero).
__global__ void __launch_bounds__(256) k_wgrad_last(const bf16* __restrict__ a16, const float* __restrict__ gout,
                                                    int B, int H, int W, long long per, float* __restrict__ partial) {
    __shared__ float sm[8][10 * CH];
    const int cg = threadIdx.x & 7, pl = threadIdx.x >> 3;
    const long long HW = (long long)H * W, npix = B * HW;
    const long long p0 = (long long)blockIdx.x * per, p1 = std::min(p0 + per, npix);
    float s[10][8] = {};
    for (long long p = p0 + pl; p < p1; p += 32) {
        const int b = (int)(p / HW);
        const int y = (int)((p - b * HW) / W), x = (int)(p - b * HW - (long long)y * W);
        const float gv = gout[p];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                float f[8];
                unpack8(*reinterpret_cast<const uint4*>(a16 + (((long long)b * H + yy) * W + xx) * CH + cg * 8), f);
#pragma unroll
                for (int k = 0; k < 8; ++k) s[t][k] = fmaf(f[k], gv, s[t][k]);
            }
        }
        if (cg == 0) s[9][0] += gv;
    }
    block_colsum<10>(s, sm, partial + (size_t)blockIdx.x * 10 * CH);
}

// e = (r - sigma f) - x_true; loss partials sum e^2; gout = -2 sigma e / count
__global__ void k_loss(const float* __restrict__ r, const float* __restrict__ sigma, const float* __restrict__ f,
                       const float* __restrict__ xt, long long HW, long long npix, float* __restrict__ gout,
                       double* __restrict__ partial) {
    __shared__ double red[32];
    double s = 0.0;
    const double inv_count = 1.0 / (double)npix;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        // noise-normalised residual e / sigma = (r - x) / sigma - f
        const float sg = sigma[p / HW];
        const float e = ((r[p] - sg * f[p]) - xt[p]) / sg;
        s += (double)e * e;
        gout[p] = (float)(-2.0 * e * inv_count);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_loss_final(const double* __restrict__ partial, int n, long long npix, double* __restrict__ loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *loss = s / (double)npix;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// master (reference layout) -> compute copies.  Hidden weights are rounded to
// BF16 (round to nearest even) into [co][tap*64+ci] and the flipped
// transpose [ci][(8-tap)*64+co]; first/last layer weights are rounded to
// BF16 values and kept in FP32 [tap][c].
__global__ void k_pack(const float* __restrict__ master, int nhidden, long long off_first, long long off_hidden,
                       long long stride_hidden, long long off_last, bf16* __restrict__ wh, bf16* __restrict__ wt,
                       float* __restrict__ w0, float* __restrict__ w16) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long hid = (long long)nhidden * 9 * CH * CH;
    if (i < hid) {
        const int l = (int)(i / (9 * CH * CH));
        const int rem = (int)(i - (long long)l * 9 * CH * CH);
        const int tap = rem / (CH * CH), ci = (rem / CH) % CH, co = rem % CH;
        const bf16 v = __float2bfloat16_rn(master[off_hidden + l * stride_hidden + rem]);
        wh[((size_t)l * CH + co) * KW + tap * CH + ci] = v;
        wt[((size_t)l * CH + ci) * KW + (8 - tap) * CH + co] = v;
        return;
    }
    const long long k = i - hid;
    if (k < 9 * CH) {
        w0[k] = __bfloat162float(__float2bfloat16_rn(master[off_first + k]));    // [tap][co]
    } else if (k < 18 * CH) {
        const long long kk = k - 9 * CH;                                           // [tap][ci] (cout = 1)
        w16[kk] = __bfloat162float(__float2bfloat16_rn(master[off_last + kk]));
    }
}

}  // namespace dgct

// ======================================================================
//                               C ABI
// ======================================================================
using namespace dgct;

struct dgamp_ct_cnn_s {
    int L = 17;
    int64_t nparam = 0;
    std::vector<int64_t> w_off, b_off;
    float* master = nullptr;
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t step = 0;
    bf16* wh = nullptr;   // [15][64][576]
    bf16* wt = nullptr;   // [15][64][576]
    float* w0 = nullptr;  // [9][64]
    float* w16 = nullptr; // [9][64]
    // shape-dependent workspace
    int64_t cap_pix = 0;
    int cap_store = 0;    // activations kept for all layers (training), 2 (inference) or 4 (with tangent)
    bf16* act = nullptr;  // [cap_store][cap_pix][64]
    bf16* g0 = nullptr;   // [cap_pix][64]
    bf16* g1 = nullptr;
    float* f = nullptr;   // [cap_pix]
    float* gout = nullptr;
    float* partial = nullptr;   // wgrad partials
    double* dpart = nullptr;
    double* loss = nullptr;
    float* sig_buf = nullptr;   // per-image sigma (device) [cap_batch]
    int cap_batch = 0;
    int sm_count = 0;           // persistent grid of the tensor-core convolutions
    unsigned* tc_err = nullptr; // set by a tensor-core convolution whose bounded wait timed out
    unsigned long long stall_ns = 0;  // timeout test (dgamp_ct_cnn_test_timeout): 0 = off
    uint64_t ws_gen = 0;        // bumped whenever the workspace is reallocated or captured launches change
};

constexpr int kWgGroupsMax = 64;   // most CTA groups of the tensor-core weight gradient

static void cnn_free_ws(dgamp_ct_cnn_s* c) {
    void* ptrs[] = {c->act, c->g0, c->g1, c->f, c->gout, c->partial, c->dpart, c->loss, c->sig_buf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->act = c->g0 = c->g1 = nullptr;
    c->f = c->gout = c->partial = c->sig_buf = nullptr;
    c->dpart = c->loss = nullptr;
    c->cap_pix = 0;
    c->cap_store = 0;
    c->cap_batch = 0;
}

static int cnn_ensure_ws(dgamp_ct_cnn_s* c, int64_t npix, int nstore, int batch) {
    if (npix <= c->cap_pix && nstore <= c->cap_store && batch <= c->cap_batch) return DGAMP_CT_OK;
    const int64_t cap = npix > c->cap_pix ? npix : c->cap_pix;
    const int ns = nstore > c->cap_store ? nstore : c->cap_store;
    const int cb = batch > c->cap_batch ? batch : c->cap_batch;
    cnn_free_ws(c);
    auto A = [](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return DGAMP_CT_ERR_OOM; }
        return e == cudaSuccess ? DGAMP_CT_OK : cuda_fail(e);
    };
    int rc;
    if ((rc = A((void**)&c->act, (size_t)ns * cap * CH * sizeof(bf16))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->g0, (size_t)cap * CH * sizeof(bf16))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->g1, (size_t)cap * CH * sizeof(bf16))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->f, (size_t)cap * sizeof(float))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->gout, (size_t)cap * sizeof(float))) != DGAMP_CT_OK) return rc;
    // the larger of the tensor-core weight gradient's partials and the pixel sums' (+ their reduction)
    const size_t n_part = std::max((size_t)kWgGroupsMax * 9 * CH * CH, (size_t)(kColBlocks + 1) * 10 * CH);
    if ((rc = A((void**)&c->partial, n_part * sizeof(float))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->dpart, 1024 * sizeof(double))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->loss, sizeof(double))) != DGAMP_CT_OK) return rc;
    if ((rc = A((void**)&c->sig_buf, (size_t)cb * sizeof(float))) != DGAMP_CT_OK) return rc;
    c->cap_pix = cap;
    c->cap_store = ns;
    c->cap_batch = cb;
    c->ws_gen += 1;
    return DGAMP_CT_OK;
}


static int cnn_pack(dgamp_ct_cnn_s* c, cudaStream_t st) {
    const long long tot = (long long)(c->L - 2) * 9 * CH * CH + 18 * CH;
    const long long stride_hidden = 9LL * CH * CH + CH;
    k_pack<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c->master, c->L - 2, c->w_off[0], c->w_off[1], stride_hidden,
                                                         c->w_off[c->L - 1], c->wh, c->wt, c->w0, c->w16);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// forward over a batch; store_all keeps every activation (for the backward pass)
static int cnn_forward(dgamp_ct_cnn_s* c, const float* r, const float* sig, int B, int H, int W, float* d_out,
                       int store_all, cudaStream_t st) {
    const int64_t npix = (int64_t)B * H * W;
    const int L = c->L;
    auto act = [&](int l) -> bf16* {   // activation a_l, l = 1..L-1
        const int slot = store_all ? (l - 1) : ((l - 1) & 1);
        return c->act + (size_t)slot * c->cap_pix * CH;
    };
    const unsigned blocks = (unsigned)((npix + 127) / 128);
    k_conv_first<<<blocks, 128, 0, st>>>(r, sig, B, H, W, c->w0, c->master + c->b_off[0], nullptr, act(1), nullptr);
    DGCT_LAUNCH_CHECK();
    for (int l = 1; l <= L - 2; ++l)
        DGCT_TRY(launch_conv64_tc(0, act(l), c->wh, L - 2, l - 1, c->master + c->b_off[l], nullptr, act(l + 1), B, H,
                                  W, c->sm_count, c->tc_err, st, c->stall_ns));
    k_conv_last<<<conv_last_grid(B, H, W), 32 * kCLRows, 0, st>>>(act(L - 1), c->w16, c->master + c->b_off[L - 1], r, sig, B,
                                                                H, W, c->f, d_out);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// backward of sum(gout * f) after a store_all forward; writes c->grad (reference layout)
static int cnn_backward(dgamp_ct_cnn_s* c, const float* r, const float* sig, int B, int H, int W, cudaStream_t st) {
    const int64_t npix = (int64_t)B * H * W;
    const int L = c->L;
    auto act = [&](int l) -> bf16* { return c->act + (size_t)(l - 1) * c->cap_pix * CH; };
    const unsigned blocks = (unsigned)((npix + 127) / 128);
    // blocks of the pixel sums and the pixels each takes
    const int nb = col_blocks(npix);
    const long long per = (npix + nb - 1) / nb;
    const unsigned rgrid = (unsigned)((10 * CH + 7) / 8);   // k_reduce_cols: 8 columns per 256 threads
    // CTA groups of the hidden layers' weight gradient: 3 CTAs (one per tap
    // row) per group, about one CTA per SM
    const int Gw = std::max(1, std::min(kWgGroupsMax, c->sm_count / 3));
    // last layer weights and bias
    k_wgrad_last<<<nb, 256, 0, st>>>(act(L - 1), c->gout, B, H, W, per, c->partial);
    DGCT_LAUNCH_CHECK();
    float* red = c->partial + (size_t)nb * 10 * CH;
    k_reduce_cols<<<rgrid, 256, 0, st>>>(c->partial, nb, 10 * CH, red);
    DGCT_LAUNCH_CHECK();
    // scatter [tap*64+ci] -> grad W[L-1] ([tap][ci][1]) and [9*64] -> b
    DGCT_CUDA(cudaMemcpyAsync(c->grad + c->w_off[L - 1], red, 9 * CH * sizeof(float), cudaMemcpyDeviceToDevice, st));
    DGCT_CUDA(cudaMemcpyAsync(c->grad + c->b_off[L - 1], red + 9 * CH, sizeof(float), cudaMemcpyDeviceToDevice, st));
    bf16* gcur = c->g0;
    bf16* gnext = c->g1;
    k_dgrad_last<<<blocks, 128, 0, st>>>(c->gout, c->w16, act(L - 1), gcur, B, H, W);
    DGCT_LAUNCH_CHECK();
    for (int l = L - 2; l >= 1; --l) {
        // layer l maps a_l -> z_{l+1}; gcur = dL/dz_{l+1}
        DGCT_TRY(launch_wgrad64_tc(act(l), gcur, B, H, W, Gw, c->partial, c->tc_err, st, c->stall_ns));
        k_reduce_wgrad64<<<(9 * CH * CH + 255) / 256, 256, 0, st>>>(c->partial, Gw, c->grad + c->w_off[l]);
        DGCT_LAUNCH_CHECK();
        k_bias_partial<<<nb, 256, 0, st>>>(gcur, npix, per, c->partial);
        DGCT_LAUNCH_CHECK();
        k_reduce_cols<<<(CH + 7) / 8, 256, 0, st>>>(c->partial, nb, CH, c->grad + c->b_off[l]);
        DGCT_LAUNCH_CHECK();
        DGCT_TRY(launch_conv64_tc(1, gcur, c->wt, L - 2, l - 1, nullptr, act(l), gnext, B, H, W, c->sm_count,
                                  c->tc_err, st, c->stall_ns));
        bf16* t = gcur;
        gcur = gnext;
        gnext = t;
    }
    // first layer: gcur = dL/dz_1
    k_wgrad_first<<<nb, 256, 0, st>>>(r, sig, gcur, B, H, W, per, c->partial);
    DGCT_LAUNCH_CHECK();
    k_reduce_cols<<<rgrid, 256, 0, st>>>(c->partial, nb, 10 * CH, c->grad + c->w_off[0]);
    DGCT_LAUNCH_CHECK();   // w_off[0] .. +9*64 are W0 [tap][0][co]; the next 64 are b0 (b_off[0] == w_off[0] + 576)
    return DGAMP_CT_OK;
}

// ------------------------------------------------- use inside a solve ----
// scaled = 1: sigma = sqrt(tau_r) (read on the device); 0: blind network, sigma = 1
__global__ void k_sigma_from_tau(const DevScalars* __restrict__ S, float* __restrict__ sig, int n, int scaled) {
    if (threadIdx.x < n) sig[threadIdx.x] = scaled ? sqrtf((float)S->tau_r) : 1.0f;
}

namespace dgct {
// Workspace for one n x n image and its tangent (two activation slots each);
// call before any capture.
int cnn_prepare_pair(dgamp_ct_cnn_s* c, int n) { return cnn_ensure_ws(c, (int64_t)n * n, 4, 2); }

// out[0] = D_sigma(rb[0]) and out[1] = J_D(rb[0]) rb[1] = b - sigma J_f(r / sigma)(b / sigma)
// for rb = [r; b] ([2][n][n]); sigma = sqrt(tau_r) read on the device
// (scaled = 1) or 1 (blind network).  Layer by layer, the primal pass is
// followed by the tangent pass masked with the primal's fresh activation.
static int jvp_passes(dgamp_ct_cnn_s* c, const float* r, const float* b, int H, int W, float* d_out, float* d_jb,
                      cudaStream_t st);

int cnn_denoise_jvp(dgamp_ct_cnn_s* c, const float* rb, const DevScalars* S, int n, float* out, int scaled,
                    cudaStream_t st) {
    k_sigma_from_tau<<<1, 32, 0, st>>>(S, c->sig_buf, 1, scaled);
    DGCT_LAUNCH_CHECK();
    return jvp_passes(c, rb, rb + (int64_t)n * n, n, n, out, out + (int64_t)n * n, st);
}

// D_sigma(r) -> d_out and J_D(r) b -> d_jb for one H x W image, sigma = c->sig_buf[0].
static int jvp_passes(dgamp_ct_cnn_s* c, const float* r, const float* b, int H, int W, float* d_out, float* d_jb,
                      cudaStream_t st) {
    const int64_t npix = (int64_t)H * W;
    const int L = c->L;
    auto prim = [&](int l) -> bf16* { return c->act + (size_t)((l - 1) & 1) * c->cap_pix * CH; };
    auto tang = [&](int l) -> bf16* { return c->act + (size_t)(2 + ((l - 1) & 1)) * c->cap_pix * CH; };
    const unsigned blocks = (unsigned)((npix + 127) / 128);
    k_conv_first<<<blocks, 128, 0, st>>>(r, c->sig_buf, 1, H, W, c->w0, c->master + c->b_off[0], nullptr, prim(1),
                                         nullptr);
    DGCT_LAUNCH_CHECK();
    k_conv_first<<<blocks, 128, 0, st>>>(b, c->sig_buf, 1, H, W, c->w0, nullptr, prim(1), tang(1), nullptr);
    DGCT_LAUNCH_CHECK();
    for (int l = 1; l <= L - 2; ++l) {
        DGCT_TRY(launch_conv64_tc(0, prim(l), c->wh, L - 2, l - 1, c->master + c->b_off[l], nullptr, prim(l + 1), 1,
                                  H, W, c->sm_count, c->tc_err, st, c->stall_ns));
        DGCT_TRY(launch_conv64_tc(1, tang(l), c->wh, L - 2, l - 1, nullptr, prim(l + 1), tang(l + 1), 1, H, W,
                                  c->sm_count, c->tc_err, st, c->stall_ns));
    }
    k_conv_last<<<conv_last_grid(1, H, W), 32 * kCLRows, 0, st>>>(prim(L - 1), c->w16, c->master + c->b_off[L - 1], r,
                                                                c->sig_buf, 1, H, W,
                                        nullptr, d_out);
    DGCT_LAUNCH_CHECK();
    k_conv_last<<<conv_last_grid(1, H, W), 32 * kCLRows, 0, st>>>(tang(L - 1), c->w16, nullptr, b, c->sig_buf, 1, H, W,
                                                                nullptr, d_jb);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

int cnn_launches_per_pair(const dgamp_ct_cnn_s* c) { return 1 + 2 * c->L; }

uint64_t cnn_ws_generation(const dgamp_ct_cnn_s* c) { return c->ws_gen; }
}  // namespace dgct

// a tensor-core convolution whose bounded wait ran out sets c->tc_err; read
// (and cleared) once the network's work is complete
namespace dgct {
int cnn_take_timeout(dgamp_ct_cnn_s* c) {
    unsigned flag = 0;
    DGCT_CUDA(cudaMemcpy(&flag, c->tc_err, sizeof(flag), cudaMemcpyDeviceToHost));
    if (!flag) return DGAMP_CT_OK;
    DGCT_CUDA(cudaMemset(c->tc_err, 0, sizeof(flag)));
    return DGAMP_CT_ERR_TIMEOUT;
}
}  // namespace dgct
static int cnn_check_timeout(dgamp_ct_cnn_s* c) { return cnn_take_timeout(c); }

// finish a single-step call: wait for its work, then report a timed-out wait
static int cnn_finish(dgamp_ct_cnn_s* c, int rc, cudaStream_t st) {
    if (rc != DGAMP_CT_OK) return rc;
    DGCT_CUDA(cudaStreamSynchronize(st));
    return cnn_check_timeout(c);
}

static int upload_sigma(dgamp_ct_cnn_s* c, const float* h_sigma, int B, cudaStream_t st) {
    DGCT_CUDA(cudaMemcpyAsync(c->sig_buf, h_sigma, (size_t)B * sizeof(float), cudaMemcpyHostToDevice, st));
    DGCT_CUDA(cudaStreamSynchronize(st));
    return DGAMP_CT_OK;
}

extern "C" {

int dgamp_ct_cnn_create(int32_t layers, uint64_t seed, dgamp_ct_cnn_t* out) {
    if (!out || layers < 3 || layers > 64) return DGAMP_CT_ERR_INVALID_ARG;
    *out = nullptr;
    dgamp_ct_cnn_s* c = new (std::nothrow) dgamp_ct_cnn_s();
    if (!c) return DGAMP_CT_ERR_OOM;
    c->L = layers;
    int64_t off = 0;
    for (int l = 0; l < layers; ++l) {
        const int cin = l == 0 ? 1 : CH, cout = l == layers - 1 ? 1 : CH;
        c->w_off.push_back(off);
        off += 9LL * cin * cout;
        c->b_off.push_back(off);
        off += cout;
    }
    c->nparam = off;
    // He initialisation (std sqrt(2/(9 cin)), last layer x0.1), zero biases, weights rounded to BF16
    std::vector<float> h(off, 0.f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 1;
    auto nextu = [&]() {
        s ^= s << 13; s ^= s >> 7; s ^= s << 17;
        return (double)((s >> 11) + 0.5) / 9007199254740992.0;
    };
    for (int l = 0; l < layers; ++l) {
        const int cin = l == 0 ? 1 : CH, cout = l == layers - 1 ? 1 : CH;
        const double sd = std::sqrt(2.0 / (9.0 * cin)) * (l == layers - 1 ? 0.1 : 1.0);
        for (int64_t i = 0; i < 9LL * cin * cout; ++i) {
            const double u1 = nextu(), u2 = nextu();
            const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
            h[c->w_off[l] + i] = (float)(g * sd);
        }
    }
    const size_t hid = (size_t)(layers - 2) * CH * KW;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&c->master, off * sizeof(float));
    e = e ? e : cudaMalloc(&c->grad, off * sizeof(float));
    e = e ? e : cudaMalloc(&c->adam_m, off * sizeof(float));
    e = e ? e : cudaMalloc(&c->adam_v, off * sizeof(float));
    e = e ? e : cudaMalloc(&c->wh, hid * sizeof(bf16));
    e = e ? e : cudaMalloc(&c->wt, hid * sizeof(bf16));
    e = e ? e : cudaMalloc(&c->w0, 9 * CH * sizeof(float));
    e = e ? e : cudaMalloc(&c->w16, 9 * CH * sizeof(float));
    e = e ? e : cudaMemcpy(c->master, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemset(c->adam_m, 0, off * sizeof(float));
    e = e ? e : cudaMemset(c->adam_v, 0, off * sizeof(float));
    e = e ? e : cudaMemset(c->grad, 0, off * sizeof(float));
    e = e ? e : cudaMalloc(&c->tc_err, sizeof(unsigned));
    e = e ? e : cudaMemset(c->tc_err, 0, sizeof(unsigned));
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    c->sm_count = nsm > 0 ? nsm : 152;
    if (e != cudaSuccess) {
        dgamp_ct_cnn_destroy(c);
        return e == cudaErrorMemoryAllocation ? DGAMP_CT_ERR_OOM : cuda_fail(e);
    }
    int rc = conv64_tc_init();
    if (rc == DGAMP_CT_OK) rc = cnn_pack(c, 0);
    if (rc == DGAMP_CT_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    if (rc != DGAMP_CT_OK) {
        dgamp_ct_cnn_destroy(c);
        return rc;
    }
    *out = c;
    return DGAMP_CT_OK;
}

void dgamp_ct_cnn_destroy(dgamp_ct_cnn_t c) {
    if (!c) return;
    cudaDeviceSynchronize();
    cnn_free_ws(c);
    void* ptrs[] = {c->master, c->grad, c->adam_m, c->adam_v, c->wh, c->wt, c->w0, c->w16, c->tc_err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

int64_t dgamp_ct_cnn_num_params(dgamp_ct_cnn_t c) { return c ? c->nparam : -1; }

int dgamp_ct_cnn_set_params(dgamp_ct_cnn_t c, const float* h_params, int64_t count) {
    if (!c || !h_params || count != c->nparam) return DGAMP_CT_ERR_INVALID_ARG;
    DGCT_CUDA(cudaMemcpy(c->master, h_params, count * sizeof(float), cudaMemcpyHostToDevice));
    DGCT_CUDA(cudaMemset(c->adam_m, 0, count * sizeof(float)));
    DGCT_CUDA(cudaMemset(c->adam_v, 0, count * sizeof(float)));
    c->step = 0;
    int rc = cnn_pack(c, 0);
    if (rc != DGAMP_CT_OK) return rc;
    DGCT_CUDA(cudaDeviceSynchronize());
    return DGAMP_CT_OK;
}

int dgamp_ct_cnn_get_params(dgamp_ct_cnn_t c, float* h_params, int64_t count) {
    if (!c || !h_params || count != c->nparam) return DGAMP_CT_ERR_INVALID_ARG;
    DGCT_CUDA(cudaDeviceSynchronize());
    DGCT_CUDA(cudaMemcpy(h_params, c->master, count * sizeof(float), cudaMemcpyDeviceToHost));
    return DGAMP_CT_OK;
}

int dgamp_ct_cnn_denoise(dgamp_ct_cnn_t c, const float* d_r, const float* h_sigma, int32_t batch, int32_t H,
                         int32_t W, float* d_out, void* stream) {
    if (!c || !d_r || !h_sigma || !d_out || batch < 1 || H < 1 || W < 1) return DGAMP_CT_ERR_INVALID_ARG;
    for (int b = 0; b < batch; ++b)
        if (!(h_sigma[b] > 0.f) || !std::isfinite(h_sigma[b])) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npix = (int64_t)batch * H * W;
    int rc = cnn_ensure_ws(c, npix, 2, batch);
    if (rc != DGAMP_CT_OK) return rc;
    if ((rc = upload_sigma(c, h_sigma, batch, st)) != DGAMP_CT_OK) return rc;
    return cnn_finish(c, cnn_forward(c, d_r, c->sig_buf, batch, H, W, d_out, 0, st), st);
}

int dgamp_ct_cnn_denoise_jvp(dgamp_ct_cnn_t c, const float* d_r, const float* d_b, float sigma, int32_t H,
                             int32_t W, float* d_out, float* d_jb, void* stream) {
    if (!c || !d_r || !d_b || !d_out || !d_jb || H < 1 || W < 1) return DGAMP_CT_ERR_INVALID_ARG;
    if (!(sigma > 0.f) || !std::isfinite(sigma)) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cnn_ensure_ws(c, (int64_t)H * W, 4, 1);
    if (rc != DGAMP_CT_OK) return rc;
    if ((rc = upload_sigma(c, &sigma, 1, st)) != DGAMP_CT_OK) return rc;
    return cnn_finish(c, jvp_passes(c, d_r, d_b, H, W, d_out, d_jb, st), st);
}

int dgamp_ct_cnn_test_timeout(dgamp_ct_cnn_t c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return DGAMP_CT_ERR_INVALID_ARG;
    const unsigned long long ns = on ? 1000000ull : 0ull;   // 1 ms
    if (ns != c->stall_ns) {
        DGCT_CUDA(cudaDeviceSynchronize());   // no launch of this network in flight changes its behaviour
        c->stall_ns = ns;
        c->ws_gen += 1;                       // captured solve graphs hold the old launch arguments
    }
    return DGAMP_CT_OK;
}

int dgamp_ct_cnn_gradients(dgamp_ct_cnn_t c, const float* d_r, const float* d_x, const float* h_sigma, int32_t batch,
                           int32_t H, int32_t W, double* h_loss, float* h_grad, void* stream) {
    if (!c || !d_r || !d_x || !h_sigma || batch < 1 || H < 1 || W < 1) return DGAMP_CT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npix = (int64_t)batch * H * W;
    int rc = cnn_ensure_ws(c, npix, c->L - 1, batch);
    if (rc != DGAMP_CT_OK) return rc;
    if ((rc = upload_sigma(c, h_sigma, batch, st)) != DGAMP_CT_OK) return rc;
    if ((rc = cnn_forward(c, d_r, c->sig_buf, batch, H, W, nullptr, 1, st)) != DGAMP_CT_OK) return rc;
    const int lb = 256;
    k_loss<<<lb, 256, 0, st>>>(d_r, c->sig_buf, c->f, d_x, (long long)H * W, npix, c->gout, c->dpart);
    DGCT_LAUNCH_CHECK();
    k_loss_final<<<1, 256, 0, st>>>(c->dpart, lb, npix, c->loss);
    DGCT_LAUNCH_CHECK();
    if ((rc = cnn_backward(c, d_r, c->sig_buf, batch, H, W, st)) != DGAMP_CT_OK) return rc;
    if (h_loss) DGCT_CUDA(cudaMemcpyAsync(h_loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (h_grad) DGCT_CUDA(cudaMemcpyAsync(h_grad, c->grad, c->nparam * sizeof(float), cudaMemcpyDeviceToHost, st));
    DGCT_CUDA(cudaStreamSynchronize(st));
    return cnn_check_timeout(c);
}

int dgamp_ct_cnn_train_step(dgamp_ct_cnn_t c, const float* d_r, const float* d_x, const float* h_sigma, int32_t batch,
                            int32_t H, int32_t W, float lr, double* h_loss, void* stream) {
    if (!(lr > 0.f)) return DGAMP_CT_ERR_INVALID_ARG;
    int rc = dgamp_ct_cnn_gradients(c, d_r, d_x, h_sigma, batch, H, W, h_loss, nullptr, stream);
    if (rc != DGAMP_CT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)c->step), c2 = 1.f - std::pow(b2, (float)c->step);
    k_adam<<<(unsigned)((c->nparam + 255) / 256), 256, 0, st>>>(c->master, c->grad, c->adam_m, c->adam_v, c->nparam, lr,
                                                                b1, b2, 1e-8f, c1, c2);
    DGCT_LAUNCH_CHECK();
    return cnn_pack(c, st);
}

}  // extern "C"
