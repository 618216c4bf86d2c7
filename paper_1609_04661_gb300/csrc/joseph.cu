// Joseph ray-driven projector A, its exact transpose A^T, and the plan-time
// FP64 evaluation of ||Phi~||_F^2 (Eq. linCT; Algorithm 1, Steps 1 and 3).
//
// Layout.  Before a projection the image is staged twice in row-padded form:
// XR[iy][kPad + ix] (rows) and XC[ix][kPad + iy] (the transpose), each line
// with kPad zero cells on both sides.  A view that marches over rows reads
// XR, one that marches over columns reads XC, so in both cases a warp of
// adjacent rays reads adjacent floats of one line per step, and taps that
// fall just outside the image read zeros instead of being bounds-checked.
#include "internal.cuh"

namespace dgct {

// ------------------------------------------------------------- staging ----
template <typename T>
__global__ void k_stage_image(const float* __restrict__ img, int n, int ldp,
                              T* __restrict__ XR, T* __restrict__ XC) {
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int iy = by + j, ix = bx + threadIdx.x;
        float v = 0.f;
        if (iy < n && ix < n) {
            v = img[(size_t)iy * n + ix];
            stf(XR + (size_t)iy * ldp + kPad + ix, v);
        }
        tile[j][threadIdx.x] = v;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int ix = bx + j, iy = by + threadIdx.x;
        if (iy < n && ix < n) stf(XC + (size_t)ix * ldp + kPad + iy, tile[threadIdx.x][j]);
    }
    // Guard cells of the lines that start or end in this block.  An FP32 and
    // a BF16 staging share the same bytes, so the guards are rewritten each
    // time rather than left from the allocation's zero fill.
    const int gr = ldp - kPad - n;   // 4..7 cells on the right
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int t = threadIdx.x, iy = by + j, ix = bx + j;
        if (iy < n) {
            if (blockIdx.x == 0 && t < kPad) stf(XR + (size_t)iy * ldp + t, 0.f);
            if (blockIdx.x == gridDim.x - 1 && t < gr) stf(XR + (size_t)iy * ldp + kPad + n + t, 0.f);
        }
        if (ix < n) {
            if (blockIdx.y == 0 && t < kPad) stf(XC + (size_t)ix * ldp + t, 0.f);
            if (blockIdx.y == gridDim.y - 1 && t < gr) stf(XC + (size_t)ix * ldp + kPad + n + t, 0.f);
        }
    }
}

int launch_stage_image(const dgamp_ct_plan_s* pl, const float* img, cudaStream_t st, int bf) {
    dim3 blk(32, 8), grd((pl->n + 31) / 32, (pl->n + 31) / 32);
    if (bf)
        k_stage_image<bf16s><<<grd, blk, 0, st>>>(img, pl->n, pl->ldp, (bf16s*)pl->ws.XR, (bf16s*)pl->ws.XC);
    else
        k_stage_image<float><<<grd, blk, 0, st>>>(img, pl->n, pl->ldp, pl->ws.XR, pl->ws.XC);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// --------------------------------------------------------- projection ----
// One block = 32 adjacent rays of one view; its SEG warps (8, 16 or 32,
// chosen at plan time) march disjoint parts of the step range of those rays
// and the partial sums are added in a fixed order, so the result does not
// depend on scheduling.  A warp's 32 rays read ~32-46 adjacent floats of one
// staged line per step; the gathers wait on L2, so more warps per ray group
// hide more of that latency, up to the point where the segments get short.
constexpr int kPjRays = 32;

// The rays of ray group gx of view v (one block's work).
template <typename T, int kPjSeg>
__device__ __forceinline__ void project_block(const T* __restrict__ XR, const T* __restrict__ XC, int ldp, int n,
                                              int nd, const ViewConst* __restrict__ vcs, T* __restrict__ sino,
                                              int gx, int v, float (*red)[kPjRays]) {
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int d = gx * kPjRays + lane;
    const ViewConst c = vcs[v];
    pdl_wait();      // the staged image is the previous kernel's output
    float acc = 0.f;
    if (d < nd) {
        const T* __restrict__ B = c.col ? XC : XR;
        const float base = fmaf((float)d, c.a_det, c.a0);
        int s0, s1;
        step_range(base, c.a_step, n, s0, s1);
        const int len = (n + kPjSeg - 1) / kPjSeg;
        s0 = max(s0, seg * len);
        s1 = min(s1, seg * len + len - 1);
        if (s0 <= s1) {
            long long pos = joseph_pos(c, d, s0);
            const T* __restrict__ line = B + (size_t)s0 * ldp + kPad;
#pragma unroll 4
            for (int s = s0; s <= s1; ++s, pos += c.PSTEP, line += ldp) {
                int i0;
                float f;
                joseph_tap(pos, i0, f);
                const float x0 = ldf(line + i0), x1 = ldf(line + i0 + 1);
                acc += fmaf(f, x1 - x0, x0);
            }
        }
    }
    red[seg][lane] = acc;
    __syncthreads();
    if (seg == 0 && d < nd) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kPjSeg; ++k) t += red[k][lane];
        stf(sino + (size_t)v * nd + d, t * c.w);
    }
}

template <typename T, int kPjSeg>
__global__ void __launch_bounds__(kPjRays * kPjSeg)
k_project(const T* __restrict__ XR, const T* __restrict__ XC, int ldp, int n, int nd,
          const ViewConst* __restrict__ vcs, T* __restrict__ sino) {
    __shared__ float red[kPjSeg][kPjRays];
    project_block<T, kPjSeg>(XR, XC, ldp, n, nd, vcs, sino, blockIdx.x, blockIdx.y, red);
}

// A x of every slice of a batch in one launch: block -> (slice, ray group, view).
template <typename T, int kPjSeg>
__global__ void __launch_bounds__(kPjRays * kPjSeg)
k_project_batch(const BatchSlice* __restrict__ sl, const uint16_t* __restrict__ map) {
    __shared__ float red[kPjSeg][kPjRays];
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int l = (int)blockIdx.x - B.off[kPhProj];
    const int ngx = (B.nd + kPjRays - 1) / kPjRays;
    project_block<T, kPjSeg>((const T*)B.XR, (const T*)B.XC, B.ldp, B.n, B.nd, B.vc, (T*)B.zraw, l % ngx, l / ngx,
                             red);
}

// ------------------------------------------------ banded projection ----
// The same sums as project_block, organised around the image instead of the
// rays.  A block copies BR consecutive march lines of the staged image
// (lines b*BR .. b*BR + BR - 1 of XR for the views that march over rows, of
// XC for the others; they are contiguous) into shared memory once, and takes
// the steps inside that band of a contiguous chunk of rays from there.  The
// gathers then wait on shared memory instead of L2, and a staged line is
// read from L2 once per chunk instead of once per ray group that crosses it.
// Rays are listed per orientation, view by view in `order` (the n0 views
// that march over rows, then the rest); each orientation's list is cut into
// C0 or C1 equal chunks, so the views of a block share one orientation, and
// the plan picks the chunk counts that fill whole waves of the GPU.  The
// block writes the band's partial sum of each of its rays to part[b][v][d]
// (0 where the ray has no step in the band); k_band_sum then adds the bands
// in order and applies the path length per step.  Each partial sums its
// steps in order from 0, like one segment of project_block, so with BR equal
// to the segment length of the ray-group form (n = 512, BR = 32 and 16
// segments) the two forms give identical bits.
constexpr int kBandThreads = 512;
constexpr int kBandMaxViews = 8;            // a chunk spans at most this many views
constexpr int kBandSmemMax = 100 * 1024;    // largest band the plan considers (bytes)

template <typename T>
__global__ void __launch_bounds__(kBandThreads, 3)
k_project_band(const T* __restrict__ XR, const T* __restrict__ XC, int ldp, int n, int nd, int nv,
               const ViewConst* __restrict__ vcs, const int* __restrict__ order, int n0, int BR, int C0, int C1,
               float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char band_raw[];
    __shared__ ViewConst svc[kBandMaxViews];
    __shared__ int sv[kBandMaxViews];
    T* band = reinterpret_cast<T*>(band_raw);
    const int b = blockIdx.x, c = blockIdx.y;
    const int col = c >= C0 ? 1 : 0;
    const int C = col ? C1 : C0, ci = col ? c - C0 : c;
    const long long tot = (long long)(col ? nv - n0 : n0) * nd;     // rays of this orientation
    const int lo = (int)(tot * ci / C), hi = (int)(tot * (ci + 1) / C);
    const int vfirst = lo / nd, nvb = (hi - 1) / nd - vfirst + 1;   // views of the chunk (<= kBandMaxViews)
    const int r0 = b * BR, rows = min(BR, n - r0);
    if (threadIdx.x < nvb) {                         // plan constants: read before the wait
        const int v = order[(col ? n0 : 0) + vfirst + threadIdx.x];
        sv[threadIdx.x] = v;
        svc[threadIdx.x] = vcs[v];
    }
    pdl_wait();      // the staged image is the previous kernel's output
    {
        const T* __restrict__ src = (col ? XC : XR) + (size_t)r0 * ldp;
        const int bytes = rows * ldp * (int)sizeof(T);      // a multiple of 8 (ldp % 4 == 0)
        const uint4* __restrict__ s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(band);
        const int n16 = bytes >> 4;
#pragma unroll 4
        for (int i = threadIdx.x; i < n16; i += kBandThreads) d4[i] = s4[i];
        if ((bytes & 15) && threadIdx.x == 0)
            reinterpret_cast<uint2*>(band)[bytes / 8 - 1] = reinterpret_cast<const uint2*>(src)[bytes / 8 - 1];
    }
    __syncthreads();
    // this thread's rays lo + tid, lo + tid + kBandThreads, ...: the view and
    // bin of the first by one division, then stepped
    int g = lo + threadIdx.x;
    int j = g / nd, d = g - j * nd;
    j -= vfirst;
    for (; g < hi; g += kBandThreads) {
        const ViewConst& cv = svc[j];
        float acc = 0.f;
        const float base = fmaf((float)d, cv.a_det, cv.a0);
        int s0, s1;
        step_range_rcp(base, cv.a_step, cv.inv_astep, n, s0, s1);
        s0 = max(s0, r0);
        s1 = min(s1, r0 + rows - 1);
        if (s0 <= s1) {
            long long pos = joseph_pos(cv, d, s0);
            const long long pstep = cv.PSTEP;
            const T* line = band + (s0 - r0) * ldp + kPad;
#pragma unroll 4
            for (int s = s0; s <= s1; ++s, pos += pstep, line += ldp) {
                int i0;
                float f;
                joseph_tap(pos, i0, f);
                const float x0 = ldf(line + i0), x1 = ldf(line + i0 + 1);
                acc += fmaf(f, x1 - x0, x0);
            }
        }
        part[((size_t)b * nv + sv[j]) * nd + d] = acc;
        for (d += kBandThreads; d >= nd; d -= nd) ++j;
    }
}

// sino[v][d] = w_v * sum over bands b = 0, 1, ... of part[b][v][d]; the loads
// of 16 bands are issued before their adds.
constexpr int kBandSumThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kBandSumThreads)
k_band_sum(const float* __restrict__ part, int nb, int M, int nd, const ViewConst* __restrict__ vcs,
           T* __restrict__ sino) {
    const int i = blockIdx.x * kBandSumThreads + threadIdx.x;
    const float w = i < M ? vcs[i / nd].w : 0.f;
    pdl_wait();
    if (i >= M) return;
    float t = 0.f;
    int b = 0;
    for (; b + 16 <= nb; b += 16) {
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = part[(size_t)(b + k) * M + i];
#pragma unroll
        for (int k = 0; k < 16; ++k) t += v[k];
    }
    for (; b < nb; ++b) t += part[(size_t)b * M + i];
    stf(sino + i, t * w);
}

// Shared memory of a band of BR lines; 0 if the plan cannot take the form.
int project_band_smem(const dgamp_ct_plan_s* pl, int BR) {
    if (!pl->ws.pj_part || (BR != 16 && BR != 32)) return 0;
    const int bytes = BR * pl->ldp * (int)sizeof(float);
    return bytes <= kBandSmemMax ? bytes : 0;
}

// Chunks per band of each orientation for bands of pj_band lines: pj_waves
// full waves of resident blocks over the bands, split between the two
// orientations by their views, each chunk at most kBandMaxViews - 1 views
// long (so it touches at most kBandMaxViews) and at least one ray.
int project_band_chunks(dgamp_ct_plan_s* pl) {
    pl->pj_c0 = pl->pj_c1 = 0;
    if (!pl->pj_band) return DGAMP_CT_OK;
    const int smem = project_band_smem(pl, pl->pj_band);
    if (!smem) return DGAMP_CT_ERR_UNSUPPORTED_GEOMETRY;
    int bps = 0, sms = 0;
    DGCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_project_band<float>, kBandThreads, smem));
    DGCT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device));
    const int nb = (pl->n + pl->pj_band - 1) / pl->pj_band;
    const int total = std::max(2, pl->pj_waves * std::max(bps, 1) * sms / nb);
    const int n0 = pl->pj_n0, n1 = pl->nv - n0;
    auto fit = [&](int want, int nvo) {
        if (nvo == 0) return 0;
        want = std::max(want, (nvo + kBandMaxViews - 2) / (kBandMaxViews - 1));
        return (int)std::min<long long>(std::max(want, 1), (long long)nvo * pl->nd);
    };
    pl->pj_c0 = fit((int)std::lround((double)total * n0 / pl->nv), n0);
    pl->pj_c1 = fit(total - pl->pj_c0, n1);
    return DGAMP_CT_OK;
}

template <typename T>
static cudaError_t launch_project_band(const dgamp_ct_plan_s* pl, T* sino, cudaStream_t st, bool sum) {
    const int BR = pl->pj_band;
    const int nb = (pl->n + BR - 1) / BR;
    const dim3 grd(nb, pl->pj_c0 + pl->pj_c1);
    const size_t smem = (size_t)BR * pl->ldp * sizeof(T);
    cudaError_t e = launch_pdl(k_project_band<T>, grd, dim3(kBandThreads), smem, st, (const T*)pl->ws.XR,
                               (const T*)pl->ws.XC, pl->ldp, pl->n, pl->nd, pl->nv, (const ViewConst*)pl->ws.vc,
                               (const int*)pl->ws.pj_order, pl->pj_n0, BR, pl->pj_c0, pl->pj_c1, pl->ws.pj_part);
    if (e != cudaSuccess || !sum) return e;
    const int M = (int)pl->M;
    return launch_pdl(k_band_sum<T>, dim3((M + kBandSumThreads - 1) / kBandSumThreads), dim3(kBandSumThreads), 0, st,
                      (const float*)pl->ws.pj_part, nb, M, pl->nd, (const ViewConst*)pl->ws.vc, sino);
}

template <int SEG>
static cudaError_t launch_project_seg(const dgamp_ct_plan_s* pl, float* sino, cudaStream_t st, int bf) {
    dim3 blk(kPjRays * SEG), grd((pl->nd + kPjRays - 1) / kPjRays, pl->nv);
    if (bf)
        return launch_pdl(k_project<bf16s, SEG>, grd, blk, 0, st, (const bf16s*)pl->ws.XR, (const bf16s*)pl->ws.XC,
                          pl->ldp, pl->n, pl->nd, (const ViewConst*)pl->ws.vc, (bf16s*)sino);
    return launch_pdl(k_project<float, SEG>, grd, blk, 0, st, (const float*)pl->ws.XR, (const float*)pl->ws.XC,
                      pl->ldp, pl->n, pl->nd, (const ViewConst*)pl->ws.vc, sino);
}

int launch_project(const dgamp_ct_plan_s* pl, float* sino, cudaStream_t st, int bf, bool sum) {
    if (pl->pj_band) {
        if (bf)
            DGCT_CUDA(launch_project_band<bf16s>(pl, (bf16s*)sino, st, sum));
        else
            DGCT_CUDA(launch_project_band<float>(pl, sino, st, sum));
        return DGAMP_CT_OK;
    }
    if (pl->pj_seg == 32)
        DGCT_CUDA(launch_project_seg<32>(pl, sino, st, bf));
    else if (pl->pj_seg == 16)
        DGCT_CUDA(launch_project_seg<16>(pl, sino, st, bf));
    else
        DGCT_CUDA(launch_project_seg<8>(pl, sino, st, bf));
    return DGAMP_CT_OK;
}

// ---------------------------------------------------- back-projection ----
// Pixel-driven gather of the exact transpose: for every view, the rays whose
// interpolation taps include this pixel are found from the same pos(d, s)
// expression the projector uses, so each weight equals the projector's.
// With update = 1 the kernel also forms r = x + tau_r A^T s (Algorithm 1,
// Step 3) and the running max |r| used by the MC step of Step 4.
constexpr int kBpViews = 256;

// tau_r of the update r = x + tau_r A^T H s (Algorithm 1, Step 3), by warp 0
// of a block into *s_tau_r.  nparts > 0: the fused sinogram kernel left
// nparts FP64 partial sums of tau_s_i; every block adds them in the same
// fixed order (lane-strided, then the warp's shuffle tree), forms
// tau_s = sum / M and tau_r = N / (||Phi~||_F^2 tau_s) in FP64, and the
// slice's first block (`first`) records tau_p, tau_s and tau_r in S for the
// kernels after it.  nparts == 0: tau_r is already in S.
__device__ __forceinline__ void bp_tau_r(DevScalars* __restrict__ S, const double* __restrict__ partial,
                                         int nparts, double M, double N, float* s_tau_r, bool first) {
    const int lane = threadIdx.x & 31;
    // the divergence partials of the previous TV step have been consumed
    if (lane == 0 && first) S->div_pending = 0u;
    if (nparts == 0) {
        if (lane == 0) *s_tau_r = (float)S->tau_r;
        return;
    }
    double a = 0.0;
    for (int i = lane; i < nparts; i += 32) a += partial[i];
    a = warp_sum(a);
    if (lane == 0) {
        const double tau_s = a / M, tau_r = N / (S->frob2 * tau_s);
        *s_tau_r = (float)tau_r;
        if (first) {
            S->tau_p = S->frob2 * S->tau_x / M;
            S->tau_s = tau_s;
            S->tau_r = tau_r;
            if (!isfinite(tau_r)) S->nonfinite += 1u;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_backproject(const T* __restrict__ sino, int nv, int nd, int n,
              const ViewConst* __restrict__ vcs, const float* __restrict__ x_in,
              float* __restrict__ out, int update, DevScalars* __restrict__ S,
              const double* __restrict__ partial, int nparts, double M) {
    __shared__ ViewConst svc[kBpViews];
    __shared__ unsigned s_max;
    __shared__ float s_tau_r;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const bool live = ix < n && iy < n;
    const float fx = (float)ix, fy = (float)iy, fx1 = fx + 1.f, fy1 = fy + 1.f;
    if (tid == 0) s_max = 0u;
    if (update && tid < 32) bp_tau_r(S, partial, nparts, M, (double)n * n, &s_tau_r, blockIdx.x == 0 && blockIdx.y == 0);
    float acc = 0.f;
    for (int v0 = 0; v0 < nv; v0 += kBpViews) {
        const int cnt = min(kBpViews, nv - v0);
        __syncthreads();
        for (int i = tid; i < cnt; i += blockDim.x * blockDim.y) svc[i] = vcs[v0 + i];
        __syncthreads();
        if (!live) continue;
        for (int vi = 0; vi < cnt; ++vi) {
            const ViewConst c = svc[vi];
            const int s = c.col ? ix : iy;        // march line of this pixel
            const int k = c.col ? iy : ix;        // index across the line
            // Rays of one view are >= 1 pixel apart on a march line, so pixel k
            // is tapped by at most two rays: the last ray (in position order)
            // with pos < k + 1, d1, and the one before it, d2.  d1 is estimated
            // in float from pos ~= t + d a_det and corrected by at most one ray
            // with exact fixed-point positions.
            const float t = fmaf(c.col ? fx : fy, c.a_step, c.a0);
            float df = ((c.col ? fy1 : fx1) - t) * c.inv_adet;     // where pos == k + 1
            df = fminf(fmaxf(df, -4.f), (float)nd + 4.f);
            // the last ray below k + 1 is ceil(df) - 1 (or floor(df) + 1 when the
            // position falls with d); rounding df - sg/2 lands within one ray of
            // it, which the exact correction below absorbs
            int d1 = round_magic(df - 0.5f * (float)c.sg);
            long long pos1 = joseph_pos(c, d1, s);
            if ((int)(pos1 >> 32) > k) {
                pos1 -= c.AP;
                d1 -= c.sg;
            } else if ((int)((pos1 + c.AP) >> 32) <= k) {
                pos1 += c.AP;
                d1 += c.sg;
            }
            int i1, i2;
            float f1, f2;
            joseph_tap(pos1, i1, f1);
            joseph_tap(pos1 - c.AP, i2, f2);
            const int d2 = d1 - c.sg;
            const float w1 = (i1 == k) ? (1.f - f1) : ((i1 == k - 1) ? f1 : 0.f);
            const float w2 = (i1 == k && i2 == k - 1) ? f2 : 0.f;
            const T* __restrict__ row = sino + (size_t)(v0 + vi) * nd;
            const float v1 = (d1 >= 0 && d1 < nd) ? ldf(row + d1) : 0.f;
            const float v2 = (d2 >= 0 && d2 < nd) ? ldf(row + d2) : 0.f;
            acc = fmaf(fmaf(w1, v1, w2 * v2), c.w, acc);
        }
    }
    const size_t o = (size_t)iy * n + ix;
    if (update && live) {
        const float rv = fmaf(s_tau_r, acc, x_in[o]);
        out[o] = rv;
        // |r| >= 0, so its float bit pattern orders like the value
        atomicMax(&s_max, __float_as_uint(fabsf(rv)));
    }
    if (!update) {
        if (live) out[o] = acc;
        return;
    }
    __syncthreads();
    if (tid == 0) atomicMax(&S->rmax_bits, s_max);
}

// Ray-driven form of the same transpose (bp_mode 1).  One block = one
// kBtS x kBtS image tile; warp w takes views w, w + 8, ...  For each view it
// marches the rays that have a tap in the tile, 32 rays at a time, over the
// tile's steps with the projector's own fixed-point positions, and adds
// (1 - f) v w at the left tap into one accumulator tile and f v w at the
// right tap into a second one (both the warp's own).  On one march line the
// rays' left taps are distinct (rays are >= 1 apart), and so are their right
// taps, so no two lanes of a warp ever add to the same word of one
// accumulator in the same step.  The warps' tiles are summed in a fixed
// order, so the result does not depend on scheduling.
constexpr int kBtS = 16, kBtLd = kBtS + 1, kBtWarps = 8;

// One view's rays over the tile.  COL = 1: the view marches over columns
// (step k = column s0 + k, taps along rows), else over rows.
template <int COL, typename T>
__device__ __forceinline__ void bp_tile_view(const ViewConst& c, const T* __restrict__ row, int nd, int n,
                                             int tx0, int ty0, float* __restrict__ AL, float* __restrict__ AR) {
    constexpr int as = COL ? 1 : kBtLd, ac = COL ? kBtLd : 1;     // accumulator strides: step, tap
    const int lane = threadIdx.x & 31;
    const int s0 = COL ? tx0 : ty0, c0 = COL ? ty0 : tx0;
    const int ns = min(kBtS, n - s0), nc = min(kBtS, n - c0);
    // rays with a left tap in [c0 - 1, c0 + nc) at a step of [s0, s0 + ns),
    // i.e. a0 + d a_det + s a_step in [c0 - 1, c0 + nc): solved for d in
    // float and widened by one ray on each side
    const float e0 = (float)s0 * c.a_step, e1 = (float)(s0 + ns - 1) * c.a_step;
    const float dA = ((float)(c0 - 1) - fmaxf(e0, e1) - c.a0) * c.inv_adet;
    const float dB = ((float)(c0 + nc) - fminf(e0, e1) - c.a0) * c.inv_adet;
    const int dlo = max(0, (int)floorf(fminf(dA, dB)) - 1);
    const int dhi = min(nd - 1, (int)ceilf(fmaxf(dA, dB)) + 1);
    for (int d0 = dlo; d0 <= dhi; d0 += 32) {
        const int d = d0 + lane;
        const float vw = d <= dhi ? ldf(row + d) * c.w : 0.f;        // rays past dhi add zeros
        // positions relative to the tile: the left tap's index in the tile is the high word
        long long pos = joseph_pos(c, d, s0) - ((long long)c0 << 32);
        auto step = [&](int k) {
            const int rel = (int)(pos >> 32);
            const float f = __uint_as_float(0x3F800000u | ((unsigned)pos >> 9)) - 1.0f;
            const int at = k * as + rel * ac;
            if ((unsigned)rel < (unsigned)nc) AL[at] += (1.f - f) * vw;
            if ((unsigned)(rel + 1) < (unsigned)nc) AR[at + ac] += f * vw;
            pos += c.PSTEP;
        };
        if (ns == kBtS) {
#pragma unroll
            for (int k = 0; k < kBtS; ++k) step(k);
        } else {
            for (int k = 0; k < ns; ++k) step(k);
        }
    }
}

struct BtShared {
    float accL[kBtWarps][kBtS * kBtLd], accR[kBtWarps][kBtS * kBtLd];
    unsigned s_max;
    float s_tau_r;
};

// Tile (bx, by) of the image; `first` marks the block that records the
// scalars (bp_tau_r) -- block (0, 0) of the slice.
template <typename T>
__device__ __forceinline__ void backproject_tile_block(const T* __restrict__ sino, int nv, int nd, int n,
                                                       const ViewConst* __restrict__ vcs,
                                                       const float* __restrict__ x_in, float* __restrict__ out,
                                                       int update, DevScalars* __restrict__ S,
                                                       const double* __restrict__ partial, int nparts, double M,
                                                       int bx, int by, bool first, BtShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int tx0 = bx * kBtS, ty0 = by * kBtS;
    auto& accL = sh.accL;
    auto& accR = sh.accR;
    auto& s_max = sh.s_max;
    auto& s_tau_r = sh.s_tau_r;
    float* AL = accL[wp];
    float* AR = accR[wp];
    for (int i = lane; i < kBtS * kBtLd; i += 32) AL[i] = AR[i] = 0.f;
    if (tid == 0) s_max = 0u;
    pdl_wait();      // H s and the tau_s partials are the previous kernel's output
    if (update && wp == 0) bp_tau_r(S, partial, nparts, M, (double)n * n, &s_tau_r, first);
    __syncwarp();
    for (int v = wp; v < nv; v += kBtWarps) {
        const ViewConst c = vcs[v];
        const T* row = sino + (size_t)v * nd;
        if (c.col)
            bp_tile_view<1>(c, row, nd, n, tx0, ty0, AL, AR);
        else
            bp_tile_view<0>(c, row, nd, n, tx0, ty0, AL, AR);
        __syncwarp();
    }
    __syncthreads();
    for (int p = tid; p < kBtS * kBtS; p += blockDim.x) {
        const int ly = p / kBtS, lx = p % kBtS;
        const int ix = tx0 + lx, iy = ty0 + ly;
        if (ix >= n || iy >= n) continue;
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kBtWarps; ++w) t += accL[w][ly * kBtLd + lx] + accR[w][ly * kBtLd + lx];
        const size_t o = (size_t)iy * n + ix;
        if (update) {
            const float rv = fmaf(s_tau_r, t, x_in[o]);
            out[o] = rv;
            atomicMax(&s_max, __float_as_uint(fabsf(rv)));
        } else {
            out[o] = t;
        }
    }
    if (!update) return;
    __syncthreads();
    if (tid == 0) atomicMax(&S->rmax_bits, s_max);
}

template <typename T>
__global__ void __launch_bounds__(kBtWarps * 32, 5)    // 48 registers: 5 blocks per SM, no spills
k_backproject_tile(const T* __restrict__ sino, int nv, int nd, int n, const ViewConst* __restrict__ vcs,
                   const float* __restrict__ x_in, float* __restrict__ out, int update,
                   DevScalars* __restrict__ S, const double* __restrict__ partial, int nparts, double M) {
    __shared__ BtShared sh;
    backproject_tile_block<T>(sino, nv, nd, n, vcs, x_in, out, update, S, partial, nparts, M, blockIdx.x, blockIdx.y,
                              blockIdx.x == 0 && blockIdx.y == 0, sh);
}

// r = x + tau_r A^T H s of every slice of a batch in one launch (after the
// cluster sinogram kernel: one tau_s partial per view).
template <typename T>
__global__ void __launch_bounds__(kBtWarps * 32, 5)
k_backproject_tile_batch(const BatchSlice* __restrict__ sl, const uint16_t* __restrict__ map) {
    __shared__ BtShared sh;
    const BatchSlice& B = sl[map[blockIdx.x]];
    const int l = (int)blockIdx.x - B.off[kPhBp];
    const int ntx = (B.n + kBtS - 1) / kBtS;
    backproject_tile_block<T>((const T*)B.hs, B.nv, B.nd, B.n, B.vc, B.x, B.r, 1, B.S, B.partial, B.nv, (double)B.M,
                              l % ntx, l / ntx, l == 0, sh);
}

// nparts > 0 (update = 1 after the fused sinogram kernel): tau_r from the
// nparts partial sums in ws.partial; else from S.
int launch_backproject(const dgamp_ct_plan_s* pl, const float* sino, const float* x_in,
                       float* out, int update, cudaStream_t st, int bf, int nparts) {
    const double M = (double)pl->M;
    const double* part = pl->ws.partial;
    if (pl->bp_mode == 1) {
        dim3 grd((pl->n + kBtS - 1) / kBtS, (pl->n + kBtS - 1) / kBtS);
        const ViewConst* vc = pl->ws.vc;
        if (bf)
            DGCT_CUDA(launch_pdl(k_backproject_tile<bf16s>, grd, dim3(kBtWarps * 32), 0, st, (const bf16s*)sino,
                                 pl->nv, pl->nd, pl->n, vc, x_in, out, update, pl->ws.S, part, nparts, M));
        else
            DGCT_CUDA(launch_pdl(k_backproject_tile<float>, grd, dim3(kBtWarps * 32), 0, st, sino, pl->nv, pl->nd,
                                 pl->n, vc, x_in, out, update, pl->ws.S, part, nparts, M));
        return DGAMP_CT_OK;
    }
    dim3 blk(32, 8), grd((pl->n + 31) / 32, (pl->n + 7) / 8);
    if (bf)
        k_backproject<bf16s><<<grd, blk, 0, st>>>((const bf16s*)sino, pl->nv, pl->nd, pl->n, pl->ws.vc, x_in, out,
                                                  update, pl->ws.S, part, nparts, M);
    else
        k_backproject<float><<<grd, blk, 0, st>>>(sino, pl->nv, pl->nd, pl->n, pl->ws.vc, x_in, out, update,
                                                  pl->ws.S, part, nparts, M);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// ------------------------------------------------------------ batches ----
int batch_grid_project(int nv, int nd) { return ((nd + kPjRays - 1) / kPjRays) * nv; }
int batch_grid_backproject(int n) { return ((n + kBtS - 1) / kBtS) * ((n + kBtS - 1) / kBtS); }

int launch_project_batch(const BatchExec& E, cudaStream_t st) {
    const BatchSlice* sl = E.sl;
    const uint16_t* map = E.map[kPhProj];
    const dim3 grd(E.nblk[kPhProj]), blk(kPjRays * kBatchPjSeg);
    if (E.bf)
        DGCT_CUDA(launch_pdl(k_project_batch<bf16s, kBatchPjSeg>, grd, blk, 0, st, sl, map));
    else
        DGCT_CUDA(launch_pdl(k_project_batch<float, kBatchPjSeg>, grd, blk, 0, st, sl, map));
    return DGAMP_CT_OK;
}

int launch_backproject_batch(const BatchExec& E, cudaStream_t st) {
    const BatchSlice* sl = E.sl;
    const uint16_t* map = E.map[kPhBp];
    const dim3 grd(E.nblk[kPhBp]), blk(kBtWarps * 32);
    if (E.bf)
        DGCT_CUDA(launch_pdl(k_backproject_tile_batch<bf16s>, grd, blk, 0, st, sl, map));
    else
        DGCT_CUDA(launch_pdl(k_backproject_tile_batch<float>, grd, blk, 0, st, sl, map));
    return DGAMP_CT_OK;
}

// Plan-time choice between the two forms of A^T (same operator): time both
// on the plan's geometry (a zero sinogram; the work does not depend on the
// values) and keep the faster.
int backproject_autotune(dgamp_ct_plan_s* pl) {
    DGCT_CUDA(cudaMemset(pl->ws.hs, 0, (size_t)pl->M * sizeof(float)));
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_mode = 0, rc = DGAMP_CT_OK;
    for (int mode = 0; mode < 2 && rc == DGAMP_CT_OK; ++mode) {
        pl->bp_mode = mode;
        for (int rep = 0; rep < 6 && rc == DGAMP_CT_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, 0);
            rc = launch_backproject(pl, pl->ws.hs, nullptr, pl->ws.r, 0, 0);
        }
        cudaEventRecord(e1, 0);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (rc == DGAMP_CT_OK && e != cudaSuccess) rc = cuda_fail(e);
        float ms = 0.f;
        if (rc == DGAMP_CT_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (rc == DGAMP_CT_OK && ms < best) {
            best = ms;
            best_mode = mode;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->bp_mode = best_mode;
    return rc;
}

// Plan-time choice of the form of A (same sums in another order): the ray-
// group form with 8, 16 and 32 step segments, and where the plan allows it
// the banded form with 16- or 32-line bands in one or two waves; each
// is timed on the plan's geometry (the staged image buffers' contents do not
// change the work) and the fastest is kept.
int project_autotune(dgamp_ct_plan_s* pl) {
    const int big = project_band_smem(pl, 32) ? project_band_smem(pl, 32) : project_band_smem(pl, 16);
    if (big > 48 * 1024) {
        DGCT_TRY(raise_smem_limit((const void*)k_project_band<float>, big));
        DGCT_TRY(raise_smem_limit((const void*)k_project_band<bf16s>, big));
    }
    cudaEvent_t e0, e1;
    DGCT_CUDA(cudaEventCreate(&e0));
    DGCT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_seg = 8, best_band = 0, best_waves = 1, rc = DGAMP_CT_OK;
    // {pj_seg, pj_band, pj_waves}
    const int forms[7][3] = {{8, 0, 1}, {16, 0, 1}, {32, 0, 1}, {16, 16, 1}, {16, 16, 2}, {16, 32, 1}, {16, 32, 2}};
    for (int k = 0; k < 7 && rc == DGAMP_CT_OK; ++k) {
        if (forms[k][1] && !project_band_smem(pl, forms[k][1])) continue;
        pl->pj_seg = forms[k][0];
        pl->pj_band = forms[k][1];
        pl->pj_waves = forms[k][2];
        rc = project_band_chunks(pl);
        for (int rep = 0; rep < 6 && rc == DGAMP_CT_OK; ++rep) {
            if (rep == 1) cudaEventRecord(e0, 0);
            rc = launch_project(pl, pl->ws.zraw, 0, 0);
        }
        cudaEventRecord(e1, 0);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (rc == DGAMP_CT_OK && e != cudaSuccess) rc = cuda_fail(e);
        float ms = 0.f;
        if (rc == DGAMP_CT_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (rc == DGAMP_CT_OK && ms < best) {
            best = ms;
            best_seg = pl->pj_seg;
            best_band = pl->pj_band;
            best_waves = pl->pj_waves;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->pj_seg = best_seg;
    pl->pj_band = best_band;
    pl->pj_waves = best_waves;
    if (rc == DGAMP_CT_OK) rc = project_band_chunks(pl);
    return rc;
}

// ---------------------------------------------- ||Phi~||_F^2 in FP64 ----
// ||H A||_F^2 = sum_k trace(T^T T G_k) with T[i,j] = h[(i-j) mod P] the matrix
// of H and G_k = A_k A_k^T, which is tridiagonal for Joseph weights (two
// rays of one view share a pixel only if |d - d'| <= 1).  Everything here is
// FP64 and runs once per plan.

// h[m] = (1/P) sum_k g_k cos(2 pi k m / P), m = 0..nd (h is even).
__global__ void k_filter_kernel_fp64(int P, int nd, double* __restrict__ h) {
    const int m = blockIdx.x;
    if (m > nd) return;
    double acc = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int kk = (k <= P / 2) ? k : P - k;
        const double f = (double)kk / (double)P;
        const double g = sqrt(fmax(f, 1.0 / (2.0 * P)));
        const long long arg = ((long long)k * m) % P;       // exact argument reduction
        acc += g * cospi(2.0 * (double)arg / (double)P);
    }
    __shared__ double sm[32];
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) h[m] = acc / (double)P;
}

// TT0[i] = (T^T T)[i,i], TT1[i] = (T^T T)[i,i+1]
__global__ void k_tt_band(const double* __restrict__ h, int nd, double* __restrict__ tt0,
                          double* __restrict__ tt1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nd) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nd; ++k) {
        const double hi = h[abs(k - i)];
        a += hi * hi;
        if (i + 1 < nd) b += hi * h[abs(k - i - 1)];
    }
    tt0[i] = a;
    tt1[i] = (i + 1 < nd) ? b : 0.0;
}

// One (view, ray) per thread: G_k[d,d] and G_k[d,d+1] from FP64 Joseph
// weights, weighted by the T^T T band.
__global__ void k_frob_terms(int n, int nv, int nd, const double* __restrict__ ang,
                             const double* __restrict__ tt0, const double* __restrict__ tt1,
                             double* __restrict__ term) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (d >= nd) return;
    const double th = ang[v];
    double st, ct;
    sincos(th, &st, &ct);
    const double c = 0.5 * (n - 1), cd = 0.5 * (nd - 1);
    const bool col = fabs(st) >= fabs(ct);
    const double w = col ? 1.0 / fabs(st) : 1.0 / fabs(ct);
    const double u0 = d - cd, u1 = d + 1 - cd;
    double g0 = 0.0, g1 = 0.0;
    for (int s = 0; s < n; ++s) {
        double p0, p1;
        if (col) {
            const double X = s - c;
            p0 = c - (u0 - X * ct) / st;
            p1 = c - (u1 - X * ct) / st;
        } else {
            const double Y = c - s;
            p0 = (u0 - Y * st) / ct + c;
            p1 = (u1 - Y * st) / ct + c;
        }
        const double f0 = floor(p0), f1 = floor(p1);
        const int a0 = (int)f0, b0 = (int)f1;
        const double wa[2] = {(1.0 - (p0 - f0)) * w, (p0 - f0) * w};
        const double wb[2] = {(1.0 - (p1 - f1)) * w, (p1 - f1) * w};
        for (int i = 0; i < 2; ++i) {
            const int ia = a0 + i;
            if (ia < 0 || ia > n - 1) continue;
            g0 += wa[i] * wa[i];
            if (d + 1 < nd)
                for (int j = 0; j < 2; ++j)
                    if (b0 + j == ia) g1 += wa[i] * wb[j];
        }
    }
    term[(size_t)v * nd + d] = tt0[d] * g0 + 2.0 * tt1[d] * g1;
}

int launch_frobenius(dgamp_ct_plan_s* pl) {
    const int nd = pl->nd, nv = pl->nv;
    double* h = pl->ws.scratch_d;               // [nd+1]
    double* tt0 = h + (nd + 1);                 // [nd]
    double* tt1 = tt0 + nd;                     // [nd]
    double* ang = tt1 + nd;                     // [nv]
    double* term = ang + nv;                    // [nv*nd]
    k_filter_kernel_fp64<<<nd + 1, 256>>>(pl->P, nd, h);
    DGCT_LAUNCH_CHECK();
    k_tt_band<<<(nd + 127) / 128, 128>>>(h, nd, tt0, tt1);
    DGCT_LAUNCH_CHECK();
    dim3 grd((nd + 127) / 128, nv);
    k_frob_terms<<<grd, 128>>>(pl->n, nv, nd, ang, tt0, tt1, term);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
