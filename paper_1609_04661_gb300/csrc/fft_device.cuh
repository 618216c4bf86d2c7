// Shared-memory FFT used by the detector-axis preconditioner H (Section 2.4,
// Eq. Aprecon) and the image-domain V^-1 (Algorithm 1, last step).
//
// The transform is a Stockham autosort FFT (natural order in and out,
// ping-pong between two shared-memory buffers) with radix-8 stages and one
// final radix-4 or radix-2 stage when log2 P is not a multiple of 3.  With
// Ns = the product of the radices already applied, butterfly j (of P/R)
// reads a[j + r P/R], r < R, multiplies input r by w^(r k) with k = j mod Ns
// and w = exp(-+ 2 pi i / (Ns R)), takes the R-point DFT in registers and
// writes output q to b[(j - k) R + k + q Ns].
//
// Shared-memory layout.  Element i of a buffer lives at fpad(i) = i + i/8
// (a buffer of P elements takes fft_buf_len(P) = P + P/8 slots): the first
// stage's stores b[8 j + q] and the second's fall on distinct banks for the
// 16 lanes of a 64-bit access, which without the padding collide 8- and
// 4-fold.  Twiddles are stored stage by stage (fft_twiddle_count(P) values):
// for every stage with Ns > 1, the (R - 1) Ns values exp(2 pi i r k / (Ns R))
// at [(r - 1) Ns + k], so the lanes of a warp read consecutive words.
#pragma once
#include "internal.cuh"

namespace dgct {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// c * (dir i)
__device__ __forceinline__ float2 cmul_i(float2 c, float dir) { return make_float2(-dir * c.y, dir * c.x); }

// In-place R-point DFT X_q = sum_r v_r exp(dir 2 pi i r q / R), R = 2, 4, 8,
// by radix-2 splitting (even / odd inputs).
template <int R> __device__ __forceinline__ void dft_small(float2* v, float dir);

template <> __device__ __forceinline__ void dft_small<2>(float2* v, float) {
    const float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
}

__device__ __forceinline__ void dft4(float2 a0, float2 a1, float2 a2, float2 a3, float dir, float2* X) {
    const float2 e0 = cadd(a0, a2), e1 = csub(a0, a2);
    const float2 o0 = cadd(a1, a3), o1 = cmul_i(csub(a1, a3), dir);
    X[0] = cadd(e0, o0);
    X[1] = cadd(e1, o1);
    X[2] = csub(e0, o0);
    X[3] = csub(e1, o1);
}

template <> __device__ __forceinline__ void dft_small<4>(float2* v, float dir) {
    float2 X[4];
    dft4(v[0], v[1], v[2], v[3], dir, X);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = X[q];
}

template <> __device__ __forceinline__ void dft_small<8>(float2* v, float dir) {
    float2 E[4], O[4];
    dft4(v[0], v[2], v[4], v[6], dir, E);
    dft4(v[1], v[3], v[5], v[7], dir, O);
    const float s = 0.70710678118654752f;   // 1/sqrt(2)
    // W^q O_q with W = exp(dir 2 pi i / 8): W = (1 + dir i)/sqrt2, W^2 = dir i, W^3 = (-1 + dir i)/sqrt2
    const float2 t1 = make_float2(s * (O[1].x - dir * O[1].y), s * (dir * O[1].x + O[1].y));
    const float2 t2 = cmul_i(O[2], dir);
    const float2 t3 = make_float2(s * (-O[3].x - dir * O[3].y), s * (dir * O[3].x - O[3].y));
    v[0] = cadd(E[0], O[0]);
    v[4] = csub(E[0], O[0]);
    v[1] = cadd(E[1], t1);
    v[5] = csub(E[1], t1);
    v[2] = cadd(E[2], t2);
    v[6] = csub(E[2], t2);
    v[3] = cadd(E[3], t3);
    v[7] = csub(E[3], t3);
}

__host__ __device__ __forceinline__ int fpad(int i) { return i + (i >> 3); }
__host__ __device__ __forceinline__ int fft_buf_len(int P) { return P + P / 8 + 1; }

// Radices of the stages: 8 while Ns * 8 <= P, then 4 or 2 for the rest.
__host__ __device__ __forceinline__ int fft_stage_radix(int P, int Ns) {
    return Ns * 8 <= P ? 8 : (Ns * 4 == P ? 4 : (Ns * 2 == P ? 2 : 1));
}
__host__ __device__ __forceinline__ int fft_twiddle_count(int P) {
    int cnt = 0;
    for (int Ns = 1, R = fft_stage_radix(P, 1); R > 1; Ns *= R, R = fft_stage_radix(P, Ns))
        if (Ns > 1) cnt += (R - 1) * Ns;
    return cnt;
}

// One stage; tws = this stage's twiddles; dir = -1 forward, +1 inverse.
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* a, float2* b, int P, int Ns,
                                               const float2* tws, float dir) {
    const int nb = P / R;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int k = j & (Ns - 1);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = a[fpad(j + r * nb)];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tws[(r - 1) * Ns + k];
                w.y *= dir;
                v[r] = cmul(v[r], w);
            }
        }
        dft_small<R>(v, dir);
        const int o = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) b[fpad(o + q * Ns)] = v[q];
    }
}

// Transforms a[0..P) (P a power of two, padded layout); returns the buffer
// holding the result.  Every thread of the block takes part; tw (the
// stage-by-stage table) may point to global or shared memory.
__device__ __forceinline__ float2* fft_stockham(float2* a, float2* b, int P, const float2* tw, float dir) {
    int off = 0;
    for (int Ns = 1, R = fft_stage_radix(P, 1); R > 1; Ns *= R, R = fft_stage_radix(P, Ns)) {
        if (R == 8)
            stockham_stage<8>(a, b, P, Ns, tw + off, dir);
        else if (R == 4)
            stockham_stage<4>(a, b, P, Ns, tw + off, dir);
        else
            stockham_stage<2>(a, b, P, Ns, tw + off, dir);
        if (Ns > 1) off += (R - 1) * Ns;
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace dgct
