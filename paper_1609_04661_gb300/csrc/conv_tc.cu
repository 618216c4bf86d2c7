// Hidden 64 -> 64 layers of the learned denoiser on the 5th-generation
// tensor cores (tcgen05, sm_103a): an implicit GEMM per strip of 128 pixels,
//   D[m][co] = sum_{tap, ci} A_tap[m][ci] W[co][tap*64 + ci],
// M = 128 pixels of one image row, N = 64 output channels, K = 9 x 64.
//
// Operands are K-major with the 128-byte swizzle: a pixel's 64 channels are
// one 128-byte row, exactly as the activations lie in global memory
// ([B][H][W][64] BF16), so one TMA copy (box 64 channels x 130 pixels, zero
// fill outside the image = the convolution's zero padding) brings a whole
// halo row, and the operand of tap (dy, dx) is the row slot of input row
// y + dy - 1 started dx rows later.  Weights are staged once per CTA, one 64 x 64
// block per tap.  A CTA takes a contiguous range of strips, consecutive rows
// of one 128-column band, so each strip needs one new input row: a ring of
// NI + 4 row slots keeps the NI + 2 rows that the NI issuing warps' strips
// read and two loading ahead.  The FP32 accumulators live in tensor memory,
// two per issuing warp (64 columns each), so the epilogue of one strip
// (tcgen05.ld, bias + ReLU or the mask, BF16 store) overlaps the MMAs of the
// next.
//
// One elected thread per issuing warp issues the 36 MMAs of a strip and commits them to an
// mbarrier; every wait on it is bounded and reports a timeout through
// *err instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "internal.cuh"

namespace dgct {
namespace tc {

constexpr int CH = 64;
constexpr int M = 128;                    // pixels per strip (MMA M)
constexpr int HWL = M + 2;                // halo pixels loaded per row
constexpr int HWP = 136;                  // row slot: 136 pixels x 128 B = 17 x 1024 B
constexpr int A_ROW = HWP * 128;          // bytes of one row slot (pixel-major, 128-byte swizzle)
constexpr int NI = 4;                     // MMA-issuing warps (strip k goes to warp 1 + k % NI)
constexpr int RING = NI + 4;              // row slots: NI + 2 rows in use, two loading ahead
constexpr int A_BYTES = RING * A_ROW;     // the ring
constexpr int ROW_BYTES = HWL * 128;      // bytes one row load delivers (130 pixels x 64 channels)
constexpr int B_TAP = 64 * 128;           // one tap of the weights: 64 co x 64 ci, 128-byte swizzle
constexpr int B_BYTES = 9 * B_TAP;
constexpr int SMEM = 1024 + B_BYTES + A_BYTES;       // + alignment slack
constexpr int EPI_WARP0 = 8;              // warps 8..15: epilogue; warp 0: TMA; warps 1..NI: MMA
                                          // (the epilogue warps start at a multiple of 4: warp % 4 is
                                          // the TMEM lane quarter a warp may read)
constexpr int THREADS = 32 * (EPI_WARP0 + 8);
constexpr int EPI_THREADS = 32 * 8;
constexpr unsigned TMEM_COLS = 128 * NI;  // 2 NI 64-column FP32 accumulators, two per MMA warp
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bound of every mbarrier wait (2 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major operand with 128-byte swizzle (rows of 64 BF16 = 128 B, 8-row groups
// 1024 B apart): start address and SBO = 1024.  The swizzle follows the
// absolute shared-memory address (the TMA wrote with the same rule), so a
// start moved by whole 128-byte rows or by 32 bytes within a row needs no
// base offset.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                           ((uint32_t)(M >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the mbarrier; false once `bound_ns` has
// passed.  The clock is read only when the first try fails.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          unsigned long long bound_ns = WAIT_NS) {
    if (mbar_try(mbar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(mbar, parity)) return true;
        if (global_ns() - t0 > bound_ns) return false;
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// TMA tiled loads (zero fill outside the tensor), completion counted on mbar
__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                       uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

typedef __nv_bfloat16 bf16;

// Strip s of the batch (row fastest): band = s / H is a 128-column band of
// image b = band / nx at x0 = (band % nx) * 128, row y = s % H.  A CTA takes a
// contiguous range of strips, so its consecutive strips are consecutive rows
// of one band and share two of their three input rows.
struct Strip {
    int b, y, x0;
};
__device__ __forceinline__ Strip strip_of(int s, int H, int nx) {
    const int band = s / H;
    Strip t;
    t.b = band / nx;
    t.y = s - band * H;
    t.x0 = (band - t.b * nx) * M;
    return t;
}

// Input rows in the order the CTA's strips need them: a run of strips of one
// band needs rows y_first - 1 .. y_last + 1 (rows -1 and H load as zeros);
// row number q of the sequence goes to ring slot q % RING.
struct RowCursor {
    int s_a, s_e;   // current run of strips [s_a, s_e]
    int y, q;       // next row to load and its sequence number
    bool done;
};

__device__ __forceinline__ int run_end(int s_a, int s1, int H) {
    const int e = (s_a / H + 1) * H;
    return (e < s1 ? e : s1) - 1;
}

// one input row (130 pixels x 64 channels) -> its ring slot: one TMA copy
__device__ __forceinline__ void load_row(const CUtensorMap* map, RowCursor& c, int H, int nx, int s1, uint32_t sA,
                                         uint64_t* row_bar) {
    const int band = c.s_a / H;
    const int b = band / nx, x0 = (band - b * nx) * M;
    const int slot = c.q % RING;
    const uint32_t bar = smem_u32(&row_bar[slot]);
    mbar_expect_tx(bar, ROW_BYTES);
    tma_4d(sA + (uint32_t)(slot * A_ROW), map, 0, x0 - 1, c.y, b, bar);
    ++c.q;
    if (++c.y > c.s_e - band * H + 1) {   // past the run's last row + 1: next run
        c.s_a = c.s_e + 1;
        if (c.s_a >= s1) {
            c.done = true;
        } else {
            c.s_e = run_end(c.s_a, s1, H);
            c.y = c.s_a - (c.s_a / H) * H - 1;
        }
    }
}

// accumulator of a strip (TMEM columns tcol .. tcol + 63) -> out, with bias +
// ReLU (MODE 0) or the mask (MODE 1).  Epilogue warp e (warp e + 4) reads TMEM
// lanes 32 (e % 4) .. +31 (pixels of the strip) and columns 32 (e / 4) .. +31
// (output channels).
template <int MODE>
__device__ __forceinline__ void epilogue(uint32_t tcol, const Strip& s, int H, int W, const float* __restrict__ bias,
                                         const bf16* __restrict__ mask, bf16* __restrict__ out, uint32_t empty_bar) {
    const int ew = (threadIdx.x >> 5) - EPI_WARP0, lane = threadIdx.x & 31;
    const int quad = ew & 3, c0 = (ew >> 2) * 32;   // quad == warp % 4: the TMEM lanes this warp may read
    const int x = s.x0 + quad * 32 + lane;
    const bool live = x < W;
    const size_t o = (((size_t)s.b * H + s.y) * W + (live ? x : 0)) * CH + c0;
    const uint32_t taddr = tcol + (uint32_t)c0 + ((uint32_t)(quad * 32) << 16);
    float v[32];
    tmem_ld16(taddr, v);          // warp-collective: every lane takes part
    tmem_ld16(taddr + 16, v + 16);
    fence_before();               // the reads are complete: the accumulator may be reused
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(empty_bar) : "memory");
    if (!live) return;
    if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i] + __ldg(bias + c0 + i), 0.f);
    } else {
        __align__(16) bf16 mk[32];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(mk + 8 * q) = *reinterpret_cast<const uint4*>(mask + o + 8 * q);
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (!(__bfloat162float(mk[i]) > 0.f)) v[i] = 0.f;
    }
    __align__(16) __nv_bfloat162 pk[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) pk[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(out + o + 8 * q) = *reinterpret_cast<const uint4*>(pk + 4 * q);
}

// first input-row number of a CTA's strip k given that of strip k - 1: +1
// inside a band, +3 when strip s starts a new band
__device__ __forceinline__ int next_q(int Q, int s, int H) { return Q + ((s % H == 0) ? 3 : 1); }

// accumulator of a CTA's strip k: MMA warp k % NI, its own buffer (k / NI) % 2
__device__ __forceinline__ int acc_of(int k) { return 2 * (k % NI) + ((k / NI) & 1); }

// MODE 0: out = relu(bias + conv(in, Wk)); MODE 1: out = conv(in, Wk) * (mask > 0).
// stall_ns > 0 is the timeout test: before any copy or MMA is issued, thread 0
// waits at most stall_ns on an mbarrier that nothing arrives at, records the
// timeout in *err and the CTA returns without computing (after freeing its
// tensor memory), exactly as a wait that ran out in the loop reports it.
// Wk = layer `layer` of a [layers][co][tap*64 + ci] BF16 array (map_w); the
// input is [B][H][W][64] BF16 (map_in).  CTA k takes strips [k per, (k+1) per).
// Warp-specialised, with no block barrier inside the loop:
//   warp 0 (one lane): TMA producer -- weights, then input rows into the ring,
//     a slot refilled once every MMA warp has released its previous row;
//   warps 1..NI (one lane each): MMA issuers, warp 1 + X for the strips k
//     with k % NI == X -- one issuing thread cannot feed the tensor core
//     with N = 64 instructions.  Each waits for its strip's three rows and a
//     free accumulator of its own, issues 9 taps x 4 channel steps, commits
//     acc_full, and commits row_empty for every row below its next strip's
//     first row (each row gets one release from each MMA warp, so a slot is
//     refilled only after all the MMAs reading it are done);
//   warps 8..15: epilogue -- wait acc_full, read TMEM, free the accumulator
//     (acc_empty), then bias + ReLU or mask and the BF16 store.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_conv64_tc(const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_w, int layer,
            const float* __restrict__ bias, const bf16* __restrict__ mask, bf16* __restrict__ out, int B, int H,
            int W, int per, unsigned* err, unsigned long long stall_ns) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t row_full[RING];
    __shared__ __align__(8) uint64_t row_empty[RING];
    __shared__ __align__(8) uint64_t acc_full[2 * NI];
    __shared__ __align__(8) uint64_t acc_empty[2 * NI];
    __shared__ __align__(8) uint64_t w_bar;
    __shared__ __align__(8) uint64_t never_bar;   // the timeout test's barrier: nothing arrives
    __shared__ uint32_t tmem_slot;
    __shared__ int stalled;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sB = (raw + 1023u) & ~1023u, sA = sB + B_BYTES;
    const int nx = (W + M - 1) / M;
    const int nstrips = B * H * nx;
    const int s0 = (int)blockIdx.x * per;
    const int s1 = s0 + per < nstrips ? s0 + per : nstrips;
    if (s0 >= s1) return;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int r = 0; r < RING; ++r) {
            mbar_init(smem_u32(&row_full[r]), 1);
            mbar_init(smem_u32(&row_empty[r]), NI);
        }
        for (int b = 0; b < 2 * NI; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), EPI_THREADS);
        }
        mbar_init(smem_u32(&w_bar), 1);
        mbar_init(smem_u32(&never_bar), 1);
        stalled = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    bool ok = true;
    if (stall_ns) {
        if (tid == 0 && !mbar_wait(smem_u32(&never_bar), 0u, stall_ns)) stalled = 1;
        __syncthreads();
        ok = stalled == 0;
    }
    if (!ok) {
        // timeout test: nothing was issued, so nothing is in flight
    } else if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            mbar_expect_tx(smem_u32(&w_bar), B_BYTES);
#pragma unroll 1
            for (int t = 0; t < 9; ++t) tma_3d(sB + (uint32_t)(t * B_TAP), &map_w, 64 * t, 0, layer, smem_u32(&w_bar));
            RowCursor cur;
            cur.s_a = s0;
            cur.s_e = run_end(s0, s1, H);
            cur.y = s0 - (s0 / H) * H - 1;
            cur.q = 0;
            cur.done = false;
            while (!cur.done) {
                const int slot = cur.q % RING;
                if (cur.q >= RING && !mbar_wait(smem_u32(&row_empty[slot]), (uint32_t)((cur.q / RING - 1) & 1)))
                    ok = false;
                load_row(&map_in, cur, H, nx, s1, sA, row_full);
            }
        }
    } else if (warp >= 1 && warp <= NI) {
        if (lane == 0) {
            // ---- MMA issuer X for strips k with k % NI == X ----
            const int X = warp - 1;
            int q_total = 0;   // input rows of the CTA: first row of the last strip + 3
            for (int s = s0 + 1; s < s1; ++s) q_total = next_q(q_total, s, H);
            q_total += 3;
            if (!mbar_wait(smem_u32(&w_bar), 0u)) ok = false;
            const uint64_t bdesc0 = sdesc_sw128(sB);
            int Q = 0, fx = 0;   // first row of strip k; rows below fx released by this warp
            int k = 0;
            for (int s = s0; s < s1; ++s, ++k) {
                if (k > 0) Q = next_q(Q, s, H);
                if (k % NI != X) continue;
                for (; fx < Q; ++fx) mma_commit(smem_u32(&row_empty[fx % RING]));   // rows this warp skips
                const int a = acc_of(k);
                if (k >= 2 * NI && !mbar_wait(smem_u32(&acc_empty[a]), (uint32_t)(((k - 2 * NI) / (2 * NI)) & 1)))
                    ok = false;
#pragma unroll 1
                for (int dy = 0; dy < 3; ++dy) {
                    const int q = Q + dy;
                    if (!mbar_wait(smem_u32(&row_full[q % RING]), (uint32_t)((q / RING) & 1))) ok = false;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(a * 64);
                // descriptors advance by (byte offset >> 4) in their address field
                uint64_t arow[3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) arow[dy] = sdesc_sw128(sA + (uint32_t)(((Q + dy) % RING) * A_ROW));
#pragma unroll
                for (int t = 0; t < 9; ++t) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        // pixel m of the strip reads halo pixel m + dx (dx = t % 3 rows later);
                        // 16 channels (32 bytes of each row) per MMA
                        const uint64_t ad = arow[t / 3] + (uint64_t)(((t % 3) * 128 + kk * 32) >> 4);
                        const uint64_t bd = bdesc0 + (uint64_t)((t * B_TAP + kk * 32) >> 4);
                        mma_bf16(d, ad, bd, (t | kk) != 0 ? 1u : 0u);
                    }
                }
                mma_commit(smem_u32(&acc_full[a]));
                // release the rows below this warp's next strip (strip k + NI)
                int bound = q_total;
                if (s + NI < s1) {
                    bound = Q;
                    for (int j = 1; j <= NI; ++j) bound = next_q(bound, s + j, H);
                }
                for (; fx < bound; ++fx) mma_commit(smem_u32(&row_empty[fx % RING]));
            }
            for (; fx < q_total; ++fx) mma_commit(smem_u32(&row_empty[fx % RING]));
        }
    } else if (warp >= EPI_WARP0) {
        // ---- epilogue ----
        int k = 0;
        for (int s = s0; s < s1; ++s, ++k) {
            const int a = acc_of(k);
            if (!mbar_wait(smem_u32(&acc_full[a]), (uint32_t)((k / (2 * NI)) & 1))) ok = false;
            fence_after();
            epilogue<MODE>(tmem + (uint32_t)(a * 64), strip_of(s, H, nx), H, W, bias, mask, out,
                           smem_u32(&acc_empty[a]));
        }
    }
    if (!ok && (!stall_ns || tid == 0)) atomicOr(err, 1u);
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------- weight gradient ----
// partial[group][tap][ci][co] = sum over the group's pixels p of
//   g[p][co] a[p + (dy - 1, dx - 1)][ci],   tap = 3 dy + dx,
// a GEMM per tap with M = 64 output channels, N = 64 input channels and the
// pixels as K.  Both operands lie pixel-major in global memory (one pixel's
// 64 channels = one 128-byte row), which read with pixels as K is the
// MN-major operand layout with the 128-byte swizzle: the same TMA copies as
// the forward kernel's (a strip of 128 gradient pixels, a halo row of 130
// activation pixels) feed the MMAs with no transposition, and the three dx
// taps of a row start 0, 1 and 2 pixel rows into the halo row.
//
// CTA (group, dy) takes a contiguous range of strips and accumulates taps
// (dy, 0..2) over all of them in tensor memory: three 64-column FP32
// accumulators.  With M = 64 the accumulator's row m lies in TMEM lane
// 32 (m / 16) + m % 16 (the first 16 lanes of each quarter); the four
// warps read their quarters once, at the end.  Warp 0 (one lane) loads
// strips into a ring of WG_STAGES stages, warp 1 (one lane) issues 3 x 8
// MMAs per strip and releases the stage with a commit.
constexpr int WG_G_BYTES = M * 128;                    // 128 gradient pixels
constexpr int WG_STAGE = WG_G_BYTES + A_ROW;           // + one halo row slot (136 pixels)
constexpr int WG_STAGES = 5;
constexpr int WG_SMEM = 1024 + WG_STAGES * WG_STAGE;
constexpr int WG_THREADS = 128;
constexpr unsigned WG_TMEM_COLS = 256;                 // three 64-column accumulators
// kind::f16 instruction descriptor: D FP32, A and B BF16, both MN-major, N = 64, M = 64
constexpr uint32_t IDESC_WG = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(64 >> 4) << 24);

__device__ __forceinline__ void mma_bf16_wg(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC_WG), "r"(accumulate));
}

// MN-major operand, 128-byte swizzle, 64 elements along M or N (one swizzle
// atom, so the leading-dimension offset is not used): rows of 128 bytes are
// successive K (pixels), 8-row groups 1024 bytes apart.  The swizzle follows
// the absolute shared-memory address, as the TMA wrote it, so the start may
// move by whole rows.
__device__ __forceinline__ uint64_t sdesc_sw128_mn(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

__global__ void __launch_bounds__(WG_THREADS, 1)
k_wgrad64_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_g, int B, int H,
             int W, int per, float* __restrict__ partial, unsigned* err, unsigned long long stall_ns) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[WG_STAGES];
    __shared__ __align__(8) uint64_t empty[WG_STAGES];
    __shared__ __align__(8) uint64_t acc_full;
    __shared__ __align__(8) uint64_t never_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int stalled;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int group = blockIdx.x, dy = blockIdx.y;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t s_base = (raw + 1023u) & ~1023u;
    const int nx = (W + M - 1) / M;
    const int nstrips = B * H * nx;
    const int s0 = group * per;
    const int s1 = s0 + per < nstrips ? s0 + per : nstrips;
    float* out = partial + ((size_t)group * 9 + 3 * dy) * CH * CH;
    if (s0 >= s1) {   // no strips: zero partials
        for (int i = tid; i < 3 * CH * CH; i += WG_THREADS) out[i] = 0.f;
        return;
    }
    const int nk = s1 - s0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(WG_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&acc_full), 1);
        mbar_init(smem_u32(&never_bar), 1);
        stalled = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    bool run = true;   // false only in the timeout test: nothing is issued
    if (stall_ns) {
        if (tid == 0 && !mbar_wait(smem_u32(&never_bar), 0u, stall_ns)) stalled = 1;
        __syncthreads();
        run = stalled == 0;
    }
    bool ok = run;
    if (run && warp == 0 && lane == 0) {
        // ---- TMA producer ----
        int k = 0;
        for (; k < nk; ++k) {
            const int st = k % WG_STAGES;
            if (k >= WG_STAGES && !mbar_wait(smem_u32(&empty[st]), (uint32_t)((k / WG_STAGES - 1) & 1))) {
                ok = false;
                break;
            }
            const Strip t = strip_of(s0 + k, H, nx);
            const uint32_t sg = s_base + (uint32_t)(st * WG_STAGE), sa = sg + WG_G_BYTES;
            const uint32_t bar = smem_u32(&full[st]);
            mbar_expect_tx(bar, WG_G_BYTES + ROW_BYTES);
            tma_4d(sg, &map_g, 0, t.x0, t.y, t.b, bar);
            tma_4d(sa, &map_a, 0, t.x0 - 1, t.y + dy - 1, t.b, bar);
        }
        // every copy issued has landed before the CTA may exit (bounded)
        for (int j = (k > WG_STAGES ? k - WG_STAGES : 0); j < k; ++j)
            if (!mbar_wait(smem_u32(&full[j % WG_STAGES]), (uint32_t)((j / WG_STAGES) & 1))) ok = false;
    } else if (run && warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        for (int k = 0; k < nk; ++k) {
            const int st = k % WG_STAGES;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((k / WG_STAGES) & 1))) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t sg = s_base + (uint32_t)(st * WG_STAGE), sa = sg + WG_G_BYTES;
            const uint64_t gd = sdesc_sw128_mn(sg), ad = sdesc_sw128_mn(sa);
#pragma unroll
            for (int ks = 0; ks < M / 16; ++ks) {
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    // 16 pixels (rows) per MMA; tap dx reads the halo row dx rows later
                    mma_bf16_wg(tmem + (uint32_t)(dx * 64), gd + (uint64_t)((ks * 16 * 128) >> 4),
                                ad + (uint64_t)(((ks * 16 + dx) * 128) >> 4), (k | ks) != 0 ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&empty[st]));
        }
        // arrives once every MMA issued above has completed
        mma_commit(smem_u32(&acc_full));
    }
    __syncwarp();
    // ---- epilogue: all four warps, once ----
    if (run) {
        int got = 0;
        if (lane == 0) got = mbar_wait(smem_u32(&acc_full), 0u) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
            ok = false;
        } else {
            fence_after();
            const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
            const int co = warp * 16 + lane;     // lanes 0..15 hold rows 16 warp .. + 15
#pragma unroll 1
            for (int c = 0; c < 3 * 64; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)c, v);   // warp-collective
                if (lane < 16) {   // 16 output channels of one warp: 64 contiguous bytes per ci
                    const int tap = c >> 6, ci = c & 63;
                    float* dst = out + ((size_t)tap * CH + ci) * CH + co;
#pragma unroll
                    for (int j = 0; j < 16; ++j) dst[(size_t)j * CH] = v[j];
                }
            }
        }
    }
    if (!ok && (run || tid == 0)) atomicOr(err, 1u);
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(WG_TMEM_COLS)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace dgct

namespace dgct {

int conv64_tc_init() {
    DGCT_CUDA(cudaFuncSetAttribute(tc::k_conv64_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM));
    DGCT_CUDA(cudaFuncSetAttribute(tc::k_conv64_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM));
    DGCT_CUDA(cudaFuncSetAttribute(tc::k_wgrad64_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::WG_SMEM));
    return DGAMP_CT_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

static int encode(CUtensorMap* map, cuuint32_t rank, const void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn) return cuda_fail(cudaErrorNotSupported);
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims, strides, box,
                          es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DGAMP_CT_OK : cuda_fail(cudaErrorInvalidValue);
}

// in: [B][H][W][64] BF16; wk_all: [layers][64][576] BF16 (layer `layer` used);
// out (mode 0: bias + ReLU, mode 1: times mask > 0) like in.
int launch_conv64_tc(int mode, const void* in, const void* wk_all, int layers, int layer, const float* bias,
                     const void* mask, void* out, int B, int H, int W, int grid_cap, unsigned* err, cudaStream_t st,
                     unsigned long long stall_ns) {
    const long long nstrips = (long long)B * H * ((W + tc::M - 1) / tc::M);
    if (nstrips <= 0) return DGAMP_CT_OK;
    if (layer < 0 || layer >= layers) return DGAMP_CT_ERR_INVALID_ARG;
    CUtensorMap map_in, map_w;
    {
        const cuuint64_t dims[4] = {64, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {128, (cuuint64_t)W * 128, (cuuint64_t)H * W * 128};
        const cuuint32_t box[4] = {64, (cuuint32_t)tc::HWL, 1, 1};
        DGCT_TRY(encode(&map_in, 4, in, dims, strides, box));
    }
    {
        const cuuint64_t dims[3] = {576, 64, (cuuint64_t)layers};
        const cuuint64_t strides[2] = {1152, 1152 * 64};
        const cuuint32_t box[3] = {64, 64, 1};
        DGCT_TRY(encode(&map_w, 3, wk_all, dims, strides, box));
    }
    // contiguous ranges of strips, one per CTA, at most grid_cap CTAs
    const int cap = grid_cap > 0 ? grid_cap : 1;
    const int per = (int)((nstrips + cap - 1) / cap);
    const int grid = (int)((nstrips + per - 1) / per);
    typedef __nv_bfloat16 bf16;
    if (mode == 0)
        tc::k_conv64_tc<0><<<grid, tc::THREADS, tc::SMEM, st>>>(map_in, map_w, layer, bias, (const bf16*)mask,
                                                                (bf16*)out, B, H, W, per, err, stall_ns);
    else
        tc::k_conv64_tc<1><<<grid, tc::THREADS, tc::SMEM, st>>>(map_in, map_w, layer, bias, (const bf16*)mask,
                                                                (bf16*)out, B, H, W, per, err, stall_ns);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

// a: the layer's input activations, g: the gradient at its output, both
// [B][H][W][64] BF16; partial: [groups][9][64 ci][64 co] FP32, every group
// written (zeros for a group without strips).
int launch_wgrad64_tc(const void* a, const void* g, int B, int H, int W, int groups, float* partial, unsigned* err,
                      cudaStream_t st, unsigned long long stall_ns) {
    if (groups < 1) return DGAMP_CT_ERR_INVALID_ARG;
    const long long nstrips = (long long)B * H * ((W + tc::M - 1) / tc::M);
    if (nstrips <= 0) {
        DGCT_CUDA(cudaMemsetAsync(partial, 0, (size_t)groups * 9 * 64 * 64 * sizeof(float), st));
        return DGAMP_CT_OK;
    }
    CUtensorMap map_a, map_g;
    const cuuint64_t dims[4] = {64, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {128, (cuuint64_t)W * 128, (cuuint64_t)H * W * 128};
    {
        const cuuint32_t box[4] = {64, (cuuint32_t)tc::HWL, 1, 1};
        DGCT_TRY(encode(&map_a, 4, a, dims, strides, box));
    }
    {
        const cuuint32_t box[4] = {64, (cuuint32_t)tc::M, 1, 1};
        DGCT_TRY(encode(&map_g, 4, g, dims, strides, box));
    }
    const int per = (int)((nstrips + groups - 1) / groups);
    tc::k_wgrad64_tc<<<dim3(groups, 3), tc::WG_THREADS, tc::WG_SMEM, st>>>(map_a, map_g, B, H, W, per, partial, err,
                                                                          stall_ns);
    DGCT_LAUNCH_CHECK();
    return DGAMP_CT_OK;
}

}  // namespace dgct
