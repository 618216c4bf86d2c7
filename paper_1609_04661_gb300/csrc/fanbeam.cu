// Flat-detector fan beam (Section 6; option of the plan, dgamp_ct_plan_fan):
// the Joseph projector A along each ray's own direction, its exact
// transpose, and ||Phi~||_F^2 for Phi~ = A V^-1 (Eq. precondAMP_op with the
// image-domain cone filter; the detector-axis form H A is a parallel-beam
// identity and does not apply).
//
// Geometry (pixel units, pixel centres as for parallel beam): at view angle
// theta the source sits at S = -dso e_c with e_c = (-sin, cos), the detector
// centre at ddo e_c, and bin d at the detector centre plus u_d e_u with
// e_u = (cos, sin), u_d = (d - (n_det-1)/2) du.  Ray d runs along
// v = T_d - S.  A ray with |v_x| >= |v_y| is marched by columns: in column s
// it sits at the fractional row a0 + s a_step, a_step = -v_y / v_x, and the
// linear interpolation between the two nearest rows is weighted by
// w = |v| / |v_x|; any other ray is marched by rows with the fractional
// column a0 + s a_step, a_step = -v_x / v_y, w = |v| / |v_y|.  Positions are
// 32.32 fixed point computed once per ray in FP64, so the projector and the
// back-projector take bit-identical taps.
//
// A: one block = 32 adjacent rays of one view; 8 warps march disjoint parts
// of the step range and add their partial sums in a fixed order.  A ray
// marched by columns reads the staged transpose XC (line s = column s), one
// marched by rows the staged rows XR, as in joseph.cu; taps just outside the
// image read the zero guard cells.
//
// A^T, ray-driven tiles (bp_mode 1, the default where it applies): one
// block = one 16 x 16 image tile, warp w takes views w, w + 8, ...  The rays
// of a view that can put a tap in the tile are those whose bins lie between
// the bins of the corners of the tile grown by one pixel (the bin map is
// monotone along any segment in front of the source, so its extremes over
// the square are at the corners), widened by one bin each way.  A warp's 32
// lanes take rays S apart, S the plan's stride, and march them over the
// tile's 16 steps with the projector's own integer positions, adding
// (1 - f) s w at the left tap into one accumulator tile and f s w at the
// right tap into another -- rays marched by columns in one pass, rays
// marched by rows in another.  The two half-warps take the even and the odd
// bin offsets of a pass, each with its own pair of accumulator tiles, so a
// stride of 2 costs no second pass.  S is the smallest stride for which any two
// rays of a view marched the same way and S or more bins apart are at least
// one pixel apart on every march line through the image (checked at plan
// time from the integer positions), so no two lanes add to the same word of
// an accumulator in the same step.  The warps' tiles are summed in a fixed
// order.  Where no stride up to kFtMaxStride suffices (a source very close
// to the image with fine bins), the gather below is used.
//
// A^T, pixel-driven gather (bp_mode 0): one thread per pixel, views in order.  The rays
// of view k that can put a tap on pixel (X, Y) through column X are those
// crossing the segment (X, Y-1)-(X, Y+1); their bins lie between the
// projections of its end points through the source (bin(p) is monotone
// along a segment in front of the source), widened by one bin each way.
// Each candidate is then tested with the projector's own integer position,
// so the gather applies exactly the projector's taps.  Rays marched by rows
// are found through the segment (X-1, Y)-(X+1, Y) likewise.
//
// ||Phi~||_F^2 = sum over rays of ||V^-1 a_i||^2: plan-time, one ray at a
// time (its taps scattered into an image, V^-1 by the image filter of
// fft.cu, the sum of squares in FP64).
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace dgct {

constexpr int kFanSeg = 8;

// ------------------------------------------------------------ projector ----
template <typename T>
__global__ void __launch_bounds__(32 * kFanSeg)
k_fan_project(const T* __restrict__ XR, const T* __restrict__ XC, int ldp, int n, int nd,
              const FanRay* __restrict__ rays, float* __restrict__ sino) {
    __shared__ float red[kFanSeg][32];
    const int v = blockIdx.y;
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int d = blockIdx.x * 32 + lane;
    float acc = 0.f, w = 0.f;
    if (d < nd) {
        const FanRay R = rays[(size_t)v * nd + d];
        w = R.w;
        const T* __restrict__ B = R.col ? XC : XR;
        int s0, s1;
        step_range(R.a0, R.a_step, n, s0, s1);
        const int len = (n + kFanSeg - 1) / kFanSeg;
        s0 = max(s0, seg * len);
        s1 = min(s1, seg * len + len - 1);
        if (s0 <= s1) {
            long long pos = R.P0 + (long long)s0 * R.PSTEP;
            const T* __restrict__ line = B + (size_t)s0 * ldp + kPad;
            for (int s = s0; s <= s1; ++s, pos += R.PSTEP, line += ldp) {
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
        for (int k = 0; k < kFanSeg; ++k) t += red[k][lane];
        sino[(size_t)v * nd + d] = t * w;
    }
}

// ------------------------------------------------------- back-projector ----
__device__ __forceinline__ float fan_bin(const FanView& V, float x, float y) {
    const float along = fmaf(x, V.ecx, fmaf(y, V.ecy, V.dso));   // > 0: in front of the source
    const float across = fmaf(x, V.eux, y * V.euy);
    return V.dsd * across / (along * V.du) + V.half;
}

__device__ __forceinline__ void fan_candidates(const FanView& V, float x1, float y1, float x2, float y2,
                                               int nd, int& lo, int& hi) {
    const float b1 = fan_bin(V, x1, y1), b2 = fan_bin(V, x2, y2);
    // both ends clamped to [-2, nd + 1] before the conversion to int
    const float bl = fminf(fmaxf(fminf(b1, b2), -2.f), (float)nd + 1.f);
    const float bh = fmaxf(fminf(fmaxf(b1, b2), (float)nd + 1.f), -2.f);
    lo = max(0, (int)floorf(bl) - 1);
    hi = min(nd - 1, (int)ceilf(bh) + 1);
}

__global__ void __launch_bounds__(256)
k_fan_backproject(const float* __restrict__ sino, const FanRay* __restrict__ rays,
                  const FanView* __restrict__ views, int n, int nv, int nd, float* __restrict__ img) {
    const int ix = blockIdx.x * 16 + (threadIdx.x & 15), iy = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (ix >= n || iy >= n) return;
    const float c = 0.5f * (float)(n - 1);
    const float X = (float)ix - c, Y = c - (float)iy;
    float acc = 0.f;
    for (int k = 0; k < nv; ++k) {
        const FanView V = views[k];
        const FanRay* __restrict__ R = rays + (size_t)k * nd;
        const float* __restrict__ sk = sino + (size_t)k * nd;
        int lo, hi;
        // rays marched by columns that cross column X within one row of Y
        fan_candidates(V, X, Y - 1.f, X, Y + 1.f, nd, lo, hi);
        for (int d = lo; d <= hi; ++d) {
            const FanRay r = R[d];
            if (!r.col) continue;
            int i0;
            float f;
            joseph_tap(r.P0 + (long long)ix * r.PSTEP, i0, f);
            if (i0 == iy) acc = fmaf((1.f - f) * r.w, sk[d], acc);
            else if (i0 == iy - 1) acc = fmaf(f * r.w, sk[d], acc);
        }
        // rays marched by rows that cross row Y within one column of X
        fan_candidates(V, X - 1.f, Y, X + 1.f, Y, nd, lo, hi);
        for (int d = lo; d <= hi; ++d) {
            const FanRay r = R[d];
            if (r.col) continue;
            int i0;
            float f;
            joseph_tap(r.P0 + (long long)iy * r.PSTEP, i0, f);
            if (i0 == ix) acc = fmaf((1.f - f) * r.w, sk[d], acc);
            else if (i0 == ix - 1) acc = fmaf(f * r.w, sk[d], acc);
        }
    }
    img[(size_t)iy * n + ix] = acc;
}

constexpr int kFtS = 16, kFtLd = kFtS + 1, kFtWarps = 8, kFtMaxStride = 8;

// two accumulator pairs per warp: the two half-warps of a pass take rays of
// neighbouring bins, each half into its own pair
struct FtShared {
    float accL[kFtWarps][2][kFtS * kFtLd], accR[kFtWarps][2][kFtS * kFtLd];
};

// One pass of a warp over the tile: the lanes whose rays are marched by
// columns (COL = 1: step k = column tx0 + k, taps along rows) or by rows.
template <int COL>
__device__ __forceinline__ void fan_tile_pass(const FanRay& r, float sw, bool on, int tx0, int ty0, int ncol,
                                              int nrow, float* __restrict__ AL, float* __restrict__ AR) {
    constexpr int as = COL ? 1 : kFtLd, ac = COL ? kFtLd : 1;     // accumulator strides: step, tap
    if (!on) return;
    const int s0 = COL ? tx0 : ty0, c0 = COL ? ty0 : tx0;
    const int ns = COL ? ncol : nrow, nc = COL ? nrow : ncol;
    // position relative to the tile: the left tap's index in the tile is the high word
    long long pos = r.P0 + (long long)s0 * r.PSTEP - ((long long)c0 << 32);
    auto step = [&](int k) {
        const int rel = (int)(pos >> 32);
        const float f = __uint_as_float(0x3F800000u | ((unsigned)pos >> 9)) - 1.0f;
        const int at = k * as + rel * ac;
        if ((unsigned)rel < (unsigned)nc) AL[at] += (1.f - f) * sw;
        if ((unsigned)(rel + 1) < (unsigned)nc) AR[at + ac] += f * sw;
        pos += r.PSTEP;
    };
    if (ns == kFtS) {
#pragma unroll
        for (int k = 0; k < kFtS; ++k) step(k);
    } else {
        for (int k = 0; k < ns; ++k) step(k);
    }
}

__global__ void __launch_bounds__(kFtWarps * 32, 4)
k_fan_backproject_tile(const float* __restrict__ sino, const FanRay* __restrict__ rays,
                       const FanView* __restrict__ views, int n, int nv, int nd, int stride,
                       float* __restrict__ img) {
    __shared__ FtShared sh;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int tx0 = blockIdx.x * kFtS, ty0 = blockIdx.y * kFtS;
    const int ncol = min(kFtS, n - tx0), nrow = min(kFtS, n - ty0);
    const int half = lane >> 4, hl = lane & 15;
    float* AL = sh.accL[wp][half];
    float* AR = sh.accR[wp][half];
    for (int i = hl; i < kFtS * kFtLd; i += 16) AL[i] = AR[i] = 0.f;
    __syncwarp();
    // lane stride rounded up to even: pass p gives bin offset 2p + half to each
    // half-warp, whose 16 lanes then take rays `st` bins apart
    const int st = stride + (stride & 1);
    // the tile grown by one pixel each way, centred coordinates (x right, y up)
    const float c = 0.5f * (float)(n - 1);
    const float xa = (float)(tx0 - 1) - c, xb = (float)(tx0 + ncol) - c;
    const float ya = c - (float)(ty0 - 1), yb = c - (float)(ty0 + nrow);
    for (int v = wp; v < nv; v += kFtWarps) {
        const FanView V = views[v];
        const float b0 = fan_bin(V, xa, ya), b1 = fan_bin(V, xa, yb), b2 = fan_bin(V, xb, ya), b3 = fan_bin(V, xb, yb);
        const float bl = fminf(fmaxf(fminf(fminf(b0, b1), fminf(b2, b3)), -2.f), (float)nd + 1.f);
        const float bh = fmaxf(fminf(fmaxf(fmaxf(b0, b1), fmaxf(b2, b3)), (float)nd + 1.f), -2.f);
        const int lo = max(0, (int)floorf(bl) - 1), hi = min(nd - 1, (int)ceilf(bh) + 1);
        const FanRay* __restrict__ R = rays + (size_t)v * nd;
        const float* __restrict__ sk = sino + (size_t)v * nd;
        for (int base = lo; base <= hi; base += 16 * st) {
            for (int p = 0; 2 * p < st; ++p) {
                const int d = base + 2 * p + half + st * hl;
                const bool valid = d <= hi;
                FanRay r{};
                float sw = 0.f;
                if (valid) {
                    r = R[d];
                    sw = sk[d] * r.w;
                }
                const bool by_col = valid && r.col, by_row = valid && !r.col;
                if (__any_sync(0xffffffffu, by_col)) fan_tile_pass<1>(r, sw, by_col, tx0, ty0, ncol, nrow, AL, AR);
                __syncwarp();
                if (__any_sync(0xffffffffu, by_row)) fan_tile_pass<0>(r, sw, by_row, tx0, ty0, ncol, nrow, AL, AR);
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int p = tid; p < kFtS * kFtS; p += blockDim.x) {
        const int ly = p / kFtS, lx = p % kFtS;
        if (lx >= ncol || ly >= nrow) continue;
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kFtWarps; ++w)
#pragma unroll
            for (int h = 0; h < 2; ++h) t += sh.accL[w][h][ly * kFtLd + lx] + sh.accR[w][h][ly * kFtLd + lx];
        img[(size_t)(ty0 + ly) * n + tx0 + lx] = t;
    }
}

// ------------------------------------------------------- ||Phi~||_F^2 ----
// Ray ray0 + b's taps scattered into zeroed image b of a batch ([nimg][n][n],
// one block per image; a ray puts at most one tap on a pixel, so the writes
// do not collide).  Rays past the last (nrays) leave their image zero.
__global__ void __launch_bounds__(1024)
k_fan_ray_image(const FanRay* __restrict__ rays, long long ray0, long long nrays, int n, float* __restrict__ img) {
    const size_t N = (size_t)n * n;
    img += (size_t)blockIdx.x * N;
    for (size_t i = threadIdx.x; i < N; i += blockDim.x) img[i] = 0.f;
    __syncthreads();
    const long long ray = ray0 + blockIdx.x;
    if (ray >= nrays) return;
    const FanRay R = rays[ray];
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        int i0;
        float f;
        joseph_tap(R.P0 + (long long)s * R.PSTEP, i0, f);
        const float t[2] = {(1.f - f) * R.w, f * R.w};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int q = i0 + j;
            if (q < 0 || q >= n) continue;
            const size_t o = R.col ? (size_t)q * n + s : (size_t)s * n + q;
            img[o] = t[j];
        }
    }
}

// out[slot0 + b] = sum of squares of image b (FP64, one block per image,
// fixed order), for the images of rays before nrays.
__global__ void __launch_bounds__(1024)
k_sum_squares(const float* __restrict__ img, long long N, double* __restrict__ out, long long slot0,
              long long nrays) {
    __shared__ double red[32];
    if (slot0 + blockIdx.x >= nrays) return;
    img += (size_t)blockIdx.x * N;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        const double v = img[i];
        acc += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) out[slot0 + blockIdx.x] = t;
    }
}

// ----------------------------------------------------------------- host ----
static void fan_constants(int n, int nd, const std::vector<double>& ang, double dso, double ddo, double du,
                          std::vector<FanRay>& rays, std::vector<FanView>& views) {
    const double c = 0.5 * (n - 1), half = 0.5 * (nd - 1), q = 4294967296.0;
    rays.resize(ang.size() * (size_t)nd);
    views.resize(ang.size());
    for (size_t k = 0; k < ang.size(); ++k) {
        const double st = std::sin(ang[k]), ct = std::cos(ang[k]);
        const double sx = dso * st, sy = -dso * ct;
        views[k] = FanView{(float)ct, (float)st, (float)-st, (float)ct, (float)dso, (float)(dso + ddo),
                           (float)du, (float)half};
        for (int d = 0; d < nd; ++d) {
            const double u = (d - half) * du;
            const double vx = -ddo * st + u * ct - sx, vy = ddo * ct + u * st - sy;
            const double L = std::hypot(vx, vy);
            FanRay R{};
            double a0, as, w;
            if (std::fabs(vx) >= std::fabs(vy)) {       // by columns: row c - (S_y + (X - S_x) v_y / v_x)
                const double t = vy / vx;
                a0 = c - sy + (sx + c) * t;
                as = -t;
                w = L / std::fabs(vx);
                R.col = 1;
            } else {                                     // by rows: column S_x + (Y - S_y) v_x / v_y + c
                const double t = vx / vy;
                a0 = sx + c + (c - sy) * t;
                as = -t;
                w = L / std::fabs(vy);
                R.col = 0;
            }
            R.P0 = std::llround(a0 * q);
            R.PSTEP = std::llround(as * q);
            R.a0 = (float)a0;
            R.a_step = (float)as;
            R.w = (float)w;
            rays[k * (size_t)nd + d] = R;
        }
    }
}

int launch_fan_project(const dgamp_ct_plan_s* pl, float* sino, cudaStream_t st) {
    const dim3 grd((unsigned)((pl->nd + 31) / 32), (unsigned)pl->nv);
    k_fan_project<float><<<grd, 32 * kFanSeg, 0, st>>>(pl->ws.XR, pl->ws.XC, pl->ldp, pl->n, pl->nd,
                                                       pl->ws.fan_rays, sino);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

int launch_fan_backproject(const dgamp_ct_plan_s* pl, const float* sino, float* img, cudaStream_t st) {
    const dim3 grd((unsigned)((pl->n + 15) / 16), (unsigned)((pl->n + 15) / 16));
    if (pl->bp_mode == 1 && pl->fan_stride > 0)
        k_fan_backproject_tile<<<grd, kFtWarps * 32, 0, st>>>(sino, pl->ws.fan_rays, pl->ws.fan_views, pl->n, pl->nv,
                                                              pl->nd, pl->fan_stride, img);
    else
        k_fan_backproject<<<grd, 256, 0, st>>>(sino, pl->ws.fan_rays, pl->ws.fan_views, pl->n, pl->nv, pl->nd, img);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// Smallest lane stride S of the tile back-projection: for every view and
// every bin d, the next ray d + kS (k >= 1) marched the same way is at least
// one pixel away from ray d at both ends of the march (s = 0 and s = n - 1,
// the same side at both, so everywhere between: the gap is linear in s).
// Positions along a march line are monotone in the bin, so rays further
// apart are further apart still.  0 when no S <= kFtMaxStride works.
static int fan_tile_stride(const std::vector<FanRay>& rays, int nv, int nd, int n) {
    const double one = 4294967296.0;
    for (int S = 1; S <= kFtMaxStride; ++S) {
        bool ok = true;
        for (int v = 0; v < nv && ok; ++v) {
            const FanRay* R = rays.data() + (size_t)v * nd;
            for (int d = 0; d < nd && ok; ++d) {
                int e = d + S;
                while (e < nd && R[e].col != R[d].col) e += S;
                if (e >= nd) continue;
                const double g0 = (double)(R[e].P0 - R[d].P0);
                const double g1 = g0 + (double)(n - 1) * (double)(R[e].PSTEP - R[d].PSTEP);
                if (!(g0 * g1 > 0.0) || std::fabs(g0) < one || std::fabs(g1) < one) ok = false;
            }
        }
        if (ok) return S;
    }
    return 0;
}

int fan_setup(dgamp_ct_plan_s* pl, const std::vector<double>& ang, double src_dist, double det_dist,
              double det_spacing) {
    std::vector<FanRay> rays;
    std::vector<FanView> views;
    fan_constants(pl->n, pl->nd, ang, src_dist, det_dist, det_spacing, rays, views);
    if (cudaMalloc((void**)&pl->ws.fan_rays, rays.size() * sizeof(FanRay)) != cudaSuccess ||
        cudaMalloc((void**)&pl->ws.fan_views, views.size() * sizeof(FanView)) != cudaSuccess) {
        cudaGetLastError();
        return DGAMP_CT_ERR_OOM;
    }
    DGCT_CUDA(cudaMemcpy(pl->ws.fan_rays, rays.data(), rays.size() * sizeof(FanRay), cudaMemcpyHostToDevice));
    DGCT_CUDA(cudaMemcpy(pl->ws.fan_views, views.data(), views.size() * sizeof(FanView), cudaMemcpyHostToDevice));
    pl->fan = 1;
    pl->fan_stride = fan_tile_stride(rays, pl->nv, pl->nd, pl->n);
    pl->bp_mode = pl->fan_stride > 0 ? 1 : 0;
    // ||Phi~||_F^2: batches of B rays -- their tap images, V^-1 of them (the
    // image filter, batched), one FP64 sum of squares per ray into `sums` --
    // added on the host in ray order.  Each ray's arithmetic is that of the
    // single-image filter.  B keeps the scratch near 512 MB.
    const int64_t M = pl->M, N = pl->N;
    const size_t per_img = (size_t)N * 2 * sizeof(float) + (size_t)pl->n * pl->m2 * sizeof(float2);
    const int B = (int)std::max<size_t>(1, std::min<size_t>(64, ((size_t)512 << 20) / per_img));
    double* sums = nullptr;
    float* imgs = nullptr;
    float2* C = nullptr;
    if (cudaMalloc((void**)&sums, (size_t)M * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&imgs, (size_t)B * N * 2 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&C, (size_t)B * pl->n * pl->m2 * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sums);
        cudaFree(imgs);
        cudaFree(C);
        return DGAMP_CT_ERR_OOM;
    }
    int rc = DGAMP_CT_OK;
    for (int64_t i = 0; i < M && rc == DGAMP_CT_OK; i += B) {
        k_fan_ray_image<<<B, 1024>>>(pl->ws.fan_rays, i, M, pl->n, imgs);
        rc = launch_precond_images(pl, imgs, imgs + (size_t)B * N, C, B, 1, 0);
        if (rc == DGAMP_CT_OK) k_sum_squares<<<B, 1024>>>(imgs + (size_t)B * N, N, sums, i, M);
        const cudaError_t e = cudaGetLastError();
        if (rc == DGAMP_CT_OK && e != cudaSuccess) rc = cuda_fail(e);
    }
    cudaFree(imgs);
    cudaFree(C);
    std::vector<double> h((size_t)M);
    if (rc == DGAMP_CT_OK) {
        const cudaError_t e = cudaMemcpy(h.data(), sums, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    cudaFree(sums);
    if (rc != DGAMP_CT_OK) return rc;
    double tot = 0.0;
    for (double v : h) tot += v;
    pl->frob2 = tot;
    DGCT_CUDA(cudaMemcpy(&pl->ws.S->frob2, &tot, sizeof(double), cudaMemcpyHostToDevice));
    return DGAMP_CT_OK;
}

}  // namespace dgct

using namespace dgct;

extern "C" int dgamp_ct_fan_ray_constants(const dgamp_ct_fan_geometry* g, int64_t* p0, int64_t* pstep, float* w,
                                          int32_t* col) {
    if (!g || !p0 || !pstep || !w || !col) return DGAMP_CT_ERR_INVALID_ARG;
    const dgamp_ct_geometry& b = g->base;
    if (b.n < 2 || b.n_views < 1 || b.n_det < 2 || !(g->det_spacing > 0) || !std::isfinite(g->src_dist) ||
        !std::isfinite(g->det_dist))
        return DGAMP_CT_ERR_INVALID_ARG;
    std::vector<double> ang(b.n_views);
    for (int k = 0; k < b.n_views; ++k)
        ang[k] = b.angles ? b.angles[k] : (double)k * (2.0 * 3.14159265358979323846 / b.n_views);
    std::vector<FanRay> rays;
    std::vector<FanView> views;
    fan_constants(b.n, b.n_det, ang, g->src_dist, g->det_dist, g->det_spacing, rays, views);
    for (size_t i = 0; i < rays.size(); ++i) {
        p0[i] = rays[i].P0;
        pstep[i] = rays[i].PSTEP;
        w[i] = rays[i].w;
        col[i] = rays[i].col;
    }
    return DGAMP_CT_OK;
}
