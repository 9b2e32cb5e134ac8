// 3x3 periodic convolution of the surrogate on the 5th-generation tensor
// cores: tcgen05.mma (kind::f16: BF16 operands in shared memory, FP32
// accumulators in tensor memory), completion tracked by tcgen05.commit on an
// mbarrier (every wait bounded in time).
//
// Work: the output is cut into rows of TC_TW = 128 pixels (one MMA M); the
// rows of all (image, 128-pixel strip) columns are dealt out to the CTAs in
// contiguous runs, so a CTA walks down a strip and loads each input row once,
// into a ring of TC_NSLOT halo'd input rows in shared memory filled by
// cp.async copies issued TC_NSLOT - 2 rows ahead of their use (ReLU, where
// the layer wants it, is applied in place by the thread that copied the
// vector).
//
// The MMAs are input-stationary: input row li of a run (image row y0 - 1 +
// li) feeds output rows t = li - 2, li - 1 and li of the run through taps
// dy = +1, 0 and -1; the weights of the three dy taps sit side by side in
// N, so one MMA (M = 128 pixels, N = 3 COUT, K = 16) applies one (dx,
// 16-channel) step of input row li to all three output rows at once.
// Output row t accumulates in block t % TC_NBLK of tensor memory (COUT
// columns each); where the blocks of the rows wrap around, or where a row
// starts its accumulator (its first step, accumulate flag off), the step is
// split into two or three MMAs over adjacent blocks. Per output row this
// reads the input operand 3 CIN / 16 times instead of 9 CIN / 16 and issues
// about 3 CIN / 16 + 1 MMAs instead of 9 CIN / 16; every output still sums
// its 9 CIN / 16 K-steps in the order (dy, dx, channel chunk).
//
// Roles: warps 0 .. TC_EPI_WARPS - 1 copy, apply ReLU and run the epilogue;
// the last warp only issues the MMAs (one elected lane), so the next input
// row's MMAs never wait for an epilogue. The epilogue of output row t runs
// once input row t + 2 is done, while the MMAs of input row t + 3 run: it
// reads the row out with tcgen05.ld (warp w reads lanes 32 (w % 4) .. + 31
// = pixels, a share of the columns), adds the bias and stages FP32 values in
// one of two shared tiles (16-byte chunks XOR-swizzled by pixel, no bank
// conflicts); in the next iteration the tile leaves in coalesced 16-byte
// stores, where the mask and the residual (loaded a row ahead) are applied,
// while the other tile takes the next row.
//
// Shared-memory operand layouts (K-major). With CIN = 64 both operands use
// the tensor core's 128-byte swizzle: one 128-byte row of 64 channels per
// pixel (A) or per N row (B), the 16-byte chunk c of a row stored at chunk
// c ^ (row address bits 7-9), 1024-byte atoms of 8 rows (SBO); the K step
// of 16 channels moves the descriptor start 32 bytes along the rows.
//   input row slot [TC_TW + 2 pixels][128 B] (1024-byte aligned): the window
//     of tap dx is the same operand started dx + 1 rows in.
//   weights [3 dx][3 blocks: dy = +1, 0, -1][COUT][128 B].
// With CIN = 16 (the lift layer), no swizzle; a core matrix is 8 rows of 16
// bytes:
//   input row slot [CIN/8 channel groups][TC_TW + 2 pixels, stride 16 B],
//     channel-group stride GS = (TC_TW + 3) * 16 B (LBO), SBO = 128; the
//     window of tap dx starts (1 + dx) * 16 B in.
//   weights [3 dx][CIN/8][3 blocks][COUT][8 channels]: LBO = 3 COUT * 16,
//     SBO = 128.
// The block of tap dy for output row t and input row li is t - li + 2, so
// adjacent output rows take adjacent blocks in N, as they take adjacent
// blocks of tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_conv.h"
#include "lbm_ptx.cuh"

namespace lbm {
namespace {

constexpr int TC_TW = 128;          // pixels per output row segment (MMA M)
constexpr int TC_EPI_WARPS = 16;    // warps 0 .. TC_EPI_WARPS - 1: copies and epilogue
constexpr int TC_EPI_THREADS = 32 * TC_EPI_WARPS;
constexpr int TC_THREADS = TC_EPI_THREADS + 32;  // + one warp: MMA issue
constexpr int TC_NSLOT = 5;         // input-row ring: 1 row in use, 1 ready, the rest in flight
constexpr int TC_NBLK = 8;          // accumulator blocks in tensor memory (output rows in flight)

template <int CIN, int COUT>
struct TcCfg {
    static constexpr int KG = CIN / 8;                  // 8-channel groups
    static constexpr int PIX = TC_TW + 2;               // halo'd pixels per row
    static constexpr int GS = (TC_TW + 3) * 16;         // bytes between channel groups
    // input rows: with CIN = 64, one 128-byte row per pixel, 16-byte chunks
    // swizzled by the pixel's address (the tensor core's 128-byte swizzle);
    // otherwise no swizzle, channel groups GS bytes apart
    static constexpr bool ASW = CIN == 64;
    static constexpr int SLOT_BYTES = ASW ? (PIX * 128 + 1023) / 1024 * 1024 : KG * GS;
    // weights: with CIN = 64, one 128-byte row of channels per N row, 16-byte
    // chunks swizzled by the row (the tensor core's 128-byte swizzle);
    // otherwise no swizzle, channel groups WGS bytes apart
    static constexpr bool WSW = CIN == 64;
    static constexpr int WGS = 3 * COUT * 16;
    static constexpr int WDX = WSW ? 3 * COUT * 128 : KG * WGS;  // bytes per tap dx
    static constexpr int W_BYTES = 3 * WDX;
    static constexpr int TILE = TC_TW * COUT;            // FP32 values of one output row
    static constexpr int OUT_BYTES = 2 * TILE * 4;      // two staging tiles (rows t and t - 1)
    static constexpr int BYTES = W_BYTES + TC_NSLOT * SLOT_BYTES + OUT_BYTES + 1024;  // + alignment slack
    static constexpr int ROW_VECS = KG * PIX;           // 16-byte vectors per halo'd row
    static constexpr int VPT = (ROW_VECS + TC_EPI_THREADS - 1) / TC_EPI_THREADS;
    static constexpr int TMEM_COLS = TC_NBLK * COUT < 32 ? 32 : TC_NBLK * COUT;  // power of two
    // warps reading the accumulator (4 per lane quarter group, >= 8 columns each)
    static constexpr int TW_WARPS = TC_EPI_WARPS < COUT / 2 ? TC_EPI_WARPS : COUT / 2;
    static constexpr int EPI_COLS = COUT / (TW_WARPS / 4);  // accumulator columns per reading warp
    static constexpr int NC = EPI_COLS < 16 ? EPI_COLS : 16;        // columns per tcgen05.ld
    static constexpr int EPI_CH = EPI_COLS / NC;        // tcgen05.ld per thread and row
    static constexpr int CPP = COUT / 4;                // 16-byte FP32 chunks per pixel in the tile
    static constexpr int SWZ = (CPP < 8 ? CPP : 8) - 1; // chunk swizzle mask
    static constexpr int N16 = TC_TW * COUT / 8, N32 = TC_TW * COUT / 4;  // 16-byte output chunks of a row
    static constexpr int O16 = (N16 + TC_EPI_THREADS - 1) / TC_EPI_THREADS;  // BF16 chunks per thread
    static constexpr int O32 = (N32 + TC_EPI_THREADS - 1) / TC_EPI_THREADS;  // FP32 chunks per thread
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && 3 * COUT <= 256, "tcgen05 f16 shape");
    static_assert((TMEM_COLS & (TMEM_COLS - 1)) == 0 && TC_NBLK >= 4, "accumulator blocks");
    static_assert(WDX % 1024 == 0, "swizzle atoms of the weights start on 1024-byte boundaries");
    static_assert(TW_WARPS % 4 == 0 && COUT % (TW_WARPS / 4) == 0 && (NC == 8 || NC == 16), "tile split");
    static_assert(TMEM_COLS <= 512, "tensor memory");
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), fixed version 0b001 (46-48), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// the same for a K-major operand in 128-byte swizzled rows: 8-row atoms of
// 1024 bytes (SBO), LBO unused (16), swizzle mode 2 (bits 61-63)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// N consecutive FP32 columns (N = 8 or 16) of this thread's tensor-memory lane
template <int N>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float* v) {
    uint32_t r[16];
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// barrier of the epilogue threads only (the issue warp does not wait)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(TC_EPI_THREADS) : "memory"); }

// bounded wait on an mbarrier phase; true when it completed in time
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint4 relu8(uint4 v) {
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __hmax2(h[j], z);
    return v;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
              int N, int H, int W, int in_relu, const __nv_bfloat16* __restrict__ mask,
              const __nv_bfloat16* __restrict__ res16, const float* __restrict__ res32, int res32_c,
              __nv_bfloat16* __restrict__ out16, float* __restrict__ out32, int* __restrict__ status) {
    using Cf = TcCfg<CIN, COUT>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(16) float s_bias[COUT];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* s_w = smem;
    unsigned char* s_in = s_w + Cf::W_BYTES;
    unsigned char* s_out = s_in + TC_NSLOT * Cf::SLOT_BYTES;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const bool is_epi = tid < TC_EPI_THREADS;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)Cf::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int c = tid; c < COUT; c += TC_THREADS) s_bias[c] = bias ? bias[c] : 0.f;
    // weights [9 taps (dy, dx)][COUT][CIN] -> per dx, N rows n = block (dy = +1,
    // 0, -1) * COUT + co: [3 dx][n][64 channels, chunk kg at kg ^ (n % 8)]
    // (CIN = 64) or [3 dx][CIN/8][n][8 channels]
    for (int e = tid; e < 9 * COUT * Cf::KG; e += TC_THREADS) {
        const int kg = e % Cf::KG, co = (e / Cf::KG) % COUT, tap = e / (Cf::KG * COUT);
        const int dyi = tap / 3, dxi = tap % 3, n = (2 - dyi) * COUT + co;
        const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)tap * COUT + co) * CIN + kg * 8);
        const int off = Cf::WSW ? dxi * Cf::WDX + n * 128 + ((kg ^ (n & 7)) * 16)
                                : (dxi * Cf::KG + kg) * Cf::WGS + n * 16;
        *reinterpret_cast<uint4*>(s_w + off) = v;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    // instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
    // 10-12 = 1), both K-major (bits 15, 16 = 0), M >> 4 (bits 24-28); N >> 3
    // (bits 17-22) is added per MMA
    const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_TW >> 4) << 24);
    const uint32_t s_in_addr = smem_u32(s_in), s_w_addr = smem_u32(s_w);
    // descriptors of the weights and of ring slot 0; an operand inside them is
    // the same descriptor with its start moved by a constant (the 14-bit
    // start field stays below 2^14 for any shared-memory address)
    const uint64_t b_desc0 = Cf::WSW ? sdesc_sw128(s_w_addr) : sdesc(s_w_addr, Cf::WGS, 128);
    const uint64_t a_desc0 = Cf::ASW ? sdesc_sw128(s_in_addr) : sdesc(s_in_addr, Cf::GS, 128);
    const int tiles_x = (W + TC_TW - 1) / TC_TW;
    const long long rows_total = (long long)N * tiles_x * H;
    const long long r_begin = rows_total * blockIdx.x / gridDim.x;
    const long long r_end = rows_total * (blockIdx.x + 1) / gridDim.x;
    uint32_t parity = 0;   // bit b: phase parity awaited next on bar[b]
    uint32_t pending = 0;  // bit b: a commit to bar[b] not yet waited for
    bool ok = true;

    // epilogue geometry of this thread: pixel = TMEM lane, a share of the columns
    const int pix = 32 * (warp % 4) + lane;
    const int col0 = (warp / 4) * Cf::EPI_COLS;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (warp % 4)) << 16);
    float* tiles = reinterpret_cast<float*>(s_out);

    for (long long r = r_begin; r < r_end && ok;) {
        const int y0 = (int)(r % H);
        const long long strip = r / H;
        const int x0 = (int)(strip % tiles_x) * TC_TW, n = (int)(strip / tiles_x);
        const int L = (int)((long long)(H - y0) < r_end - r ? (long long)(H - y0) : r_end - r);
        const int nvalid = W - x0 < TC_TW ? W - x0 : TC_TW;  // output pixels of this strip
        r += L;
        const __nv_bfloat16* img = in + (size_t)n * H * W * CIN;
        // this thread's vectors of a halo'd row: global element offset within
        // an input row (periodic in x) and byte offset within a slot, fixed
        // for the run
        int src_off[Cf::VPT], dst_off[Cf::VPT];
#pragma unroll
        for (int i = 0; i < Cf::VPT; ++i) {
            const int e = tid + i * TC_EPI_THREADS;
            const int kg = e % Cf::KG, px = e / Cf::KG;
            int gx = x0 - 1 + px;
            gx = gx < 0 ? gx + W : gx;
            gx = gx >= W ? gx % W : gx;
            src_off[i] = gx * CIN + kg * 8;
            dst_off[i] = Cf::ASW ? px * 128 + ((kg ^ (px & 7)) * 16) : kg * Cf::GS + px * 16;
        }
        // halo'd input row li of this run (input row y0 - 1 + li, periodic)
        // into ring slot li % TC_NSLOT; one commit group per row, empty for
        // rows the run does not need, so that group counts stay uniform
        auto copy_row = [&](int li) {
            if (li <= L + 1) {
                int gy = y0 - 1 + li;
                gy = gy < 0 ? gy + H : (gy >= H ? gy - H : gy);
                const __nv_bfloat16* row = img + (size_t)gy * W * CIN;
                unsigned char* slot = s_in + (li % TC_NSLOT) * Cf::SLOT_BYTES;
#pragma unroll
                for (int i = 0; i < Cf::VPT; ++i)
                    if (tid + i * TC_EPI_THREADS < Cf::ROW_VECS) cp_async16(slot + dst_off[i], row + src_off[i]);
            }
            cp_async_commit();
        };
        // ReLU in place on the vectors this thread copied (after they landed)
        auto relu_row = [&](int li) {
            if (!in_relu || li > L + 1) return;
            unsigned char* slot = s_in + (li % TC_NSLOT) * Cf::SLOT_BYTES;
#pragma unroll
            for (int i = 0; i < Cf::VPT; ++i) {
                if (tid + i * TC_EPI_THREADS < Cf::ROW_VECS) {
                    uint4* v = reinterpret_cast<uint4*>(slot + dst_off[i]);
                    *v = relu8(*v);
                }
            }
        };
        // MMAs of input row li (in ring slot li % TC_NSLOT): it feeds output rows
        // li - 2 (tap dy = +1), li - 1 (dy = 0) and li (dy = -1), those of them in
        // the run. One MMA per (dx, channel chunk) step covers the rows whose
        // accumulator blocks are adjacent; the first step starts row li's
        // accumulator in an MMA of its own.
        auto issue = [&](int li) {
            const int tlo = li - 2 > 0 ? li - 2 : 0, thi = li < L - 1 ? li : L - 1;
            // The cut of the rows into MMA segments is the same for every step but
            // the first, so it is worked out once per row and the steps only add
            // constant offsets (worked out per MMA, the issuing thread's scalar
            // code took longer than the MMAs). Cut points in (tlo, thi], thi + 1
            // where there is none: wr, the row whose block index wraps to 0 (at
            // most one in three rows); sp, row li where it starts its accumulator
            // after other rows of the step.
            int wr = thi + 1;
            for (int t = tlo + 1; t <= thi; ++t)
                if ((t & (TC_NBLK - 1)) == 0) wr = t;
            const int sp = li > tlo && li <= thi ? li : thi + 1;
            const int q1 = wr < sp ? wr : sp, q2 = wr < sp ? sp : (sp < wr ? wr : thi + 1);
            // one MMA segment, output rows a .. b: tensor-memory column, offset of
            // the weight block (16-byte units) and instruction descriptor
            auto seg = [&](int a, int b, uint32_t& d, uint32_t& bo, uint32_t& id) {
                d = tmem + (uint32_t)((a & (TC_NBLK - 1)) * COUT);
                bo = (uint32_t)(((a - li + 2) * COUT * (Cf::WSW ? 128 : 16)) >> 4);
                id = idesc0 | ((uint32_t)(((b - a + 1) * COUT) >> 3) << 17);
            };
            uint32_t f0d, f0b, f0i, f1d = 0, f1b = 0, f1i = 0, f2d = 0, f2b = 0, f2i = 0;  // first step
            uint32_t g0d, g0b, g0i, g1d = 0, g1b = 0, g1i = 0;                           // the others
            seg(tlo, q1 - 1, f0d, f0b, f0i);
            if (q1 <= thi) seg(q1, q2 - 1, f1d, f1b, f1i);
            if (q2 <= thi) seg(q2, thi, f2d, f2b, f2i);
            seg(tlo, wr - 1, g0d, g0b, g0i);
            if (wr <= thi) seg(wr, thi, g1d, g1b, g1i);
            const uint64_t a_row = a_desc0 + (uint64_t)(((li % TC_NSLOT) * Cf::SLOT_BYTES) >> 4);
#pragma unroll
            for (int dxi = 0; dxi < 3; ++dxi) {
#pragma unroll
                for (int kc = 0; kc < CIN / 16; ++kc) {
                    // swizzled: the window of tap dx starts dx + 1 pixels (128-byte rows)
                    // in and the K step moves the start 32 bytes along the rows; the
                    // swizzle follows the address bits, so the base offset stays 0
                    const uint64_t ad = a_row + (uint64_t)((Cf::ASW ? dxi * 128 + kc * 32
                                                                    : dxi * 16 + 2 * kc * Cf::GS) >> 4);
                    // swizzled: the K step moves the start 32 bytes along the 128-byte rows
                    const uint64_t bs = b_desc0 + (uint64_t)((Cf::WSW ? dxi * Cf::WDX + kc * 32
                                                                      : (dxi * Cf::KG + 2 * kc) * Cf::WGS) >> 4);
                    if (dxi == 0 && kc == 0) {
                        tc_mma(f0d, ad, bs + f0b, f0i, tlo == li ? 0u : 1u);
                        if (q1 <= thi) tc_mma(f1d, ad, bs + f1b, f1i, q1 == li ? 0u : 1u);
                        if (q2 <= thi) tc_mma(f2d, ad, bs + f2b, f2i, q2 == li ? 0u : 1u);
                    } else {
                        tc_mma(g0d, ad, bs + g0b, g0i, 1u);
                        if (wr <= thi) tc_mma(g1d, ad, bs + g1b, g1i, 1u);
                    }
                }
            }
            tc_commit(&bar[li & 1]);
        };
        // the mask and residual chunks of output row t this thread stores
        uint4 mreg[Cf::O16], rreg[Cf::O16];
        auto prefetch_epi = [&](int t) {
            if (!out16 || t >= L) return;
            const size_t row0 = ((size_t)n * H + y0 + t) * W + x0;
#pragma unroll
            for (int j = 0; j < Cf::O16; ++j) {
                const int i = tid + j * TC_EPI_THREADS;
                const int p = i / (COUT / 8), g8 = i % (COUT / 8);
                if (i < Cf::N16 && p < nvalid) {
                    const size_t o = (row0 + p) * COUT + g8 * 8;
                    if (mask) mreg[j] = *reinterpret_cast<const uint4*>(mask + o);
                    if (res16) rreg[j] = *reinterpret_cast<const uint4*>(res16 + o);
                }
            }
        };

        // staging tile -> global, coalesced 16-byte chunks of output row tr
        // of the run, applying mask and residual (loaded by prefetch_epi(tr))
        auto copy_out = [&](int tr, const float* tile) {
            const int y = y0 + tr;
            const size_t row0 = ((size_t)n * H + y) * W + x0;
            if (out16) {
#pragma unroll
                for (int j = 0; j < Cf::O16; ++j) {
                    const int i = tid + j * TC_EPI_THREADS;
                    const int p = i / (COUT / 8), g8 = i % (COUT / 8);
                    if (i >= Cf::N16 || p >= nvalid) continue;
                    // the two FP32 chunks 2 g8 and 2 g8 + 1, read first the one that puts the
                    // 8 threads of a shared-memory phase on 8 different bank groups
                    const int c1 = 2 * g8 + (g8 >> 2) % 2, c2 = 2 * g8 + 1 - (g8 >> 2) % 2;
                    const float4 q1 = *reinterpret_cast<const float4*>(tile + p * COUT + 4 * (c1 ^ (p & Cf::SWZ)));
                    const float4 q2 = *reinterpret_cast<const float4*>(tile + p * COUT + 4 * (c2 ^ (p & Cf::SWZ)));
                    const float4 lo = c1 < c2 ? q1 : q2, hi = c1 < c2 ? q2 : q1;
                    float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                    if (mask) {
                        const __nv_bfloat16* mh = reinterpret_cast<const __nv_bfloat16*>(&mreg[j]);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (!(__bfloat162float(mh[q]) > 0.f)) v[q] = 0.f;
                    }
                    if (res16) {
                        const __nv_bfloat16* rh = reinterpret_cast<const __nv_bfloat16*>(&rreg[j]);
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[q] += __bfloat162float(rh[q]);
                    }
                    if (res32) {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (g8 * 8 + q < res32_c) v[q] += res32[(row0 + p) * res32_c + g8 * 8 + q];
                    }
                    uint4 ov;
                    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&ov);
#pragma unroll
                    for (int q = 0; q < 4; ++q) oh[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    *reinterpret_cast<uint4*>(out16 + (row0 + p) * COUT + g8 * 8) = ov;
                }
            } else {
#pragma unroll
                for (int j = 0; j < Cf::O32; ++j) {
                    const int i = tid + j * TC_EPI_THREADS;
                    const int p = i / (COUT / 4), k = i % (COUT / 4);
                    if (i >= Cf::N32 || p >= nvalid) continue;
                    float4 v = *reinterpret_cast<const float4*>(tile + p * COUT + 4 * (k ^ (p & Cf::SWZ)));
                    if (res32) {
                        if (4 * k + 0 < res32_c) v.x += res32[(row0 + p) * res32_c + 4 * k + 0];
                        if (4 * k + 1 < res32_c) v.y += res32[(row0 + p) * res32_c + 4 * k + 1];
                        if (4 * k + 2 < res32_c) v.z += res32[(row0 + p) * res32_c + 4 * k + 2];
                        if (4 * k + 3 < res32_c) v.w += res32[(row0 + p) * res32_c + 4 * k + 3];
                    }
                    *reinterpret_cast<float4*>(out32 + (row0 + p) * COUT + 4 * k) = v;
                }
            }
        };

        if (is_epi) {
            // prologue: every slot's row in flight; input row 0 in place for its MMAs
#pragma unroll 1
            for (int li = 0; li < TC_NSLOT; ++li) copy_row(li);
            cp_async_wait<TC_NSLOT - 1>();
            relu_row(0);
            fence_proxy_async();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == TC_EPI_THREADS) issue(0);
        pending |= 1u;
        bool timed_out = false;
        // iteration j: issue input row j + 1, then (epilogue) wait for input row
        // j, whose MMAs complete output row j - 2, and write that row out
        for (int j = 0; j < L + 2; ++j) {
            if (j + 1 < L + 2) {
                if (is_epi) {
                    cp_async_wait<TC_NSLOT - 2>();
                    relu_row(j + 1);
                    fence_proxy_async();
                }
                tc_fence_before();
                // also: every thread has left the staging tile that row j - 2 takes
                // (and tensor-memory blocks of rows read out are free long before
                // they come round again)
                if (__syncthreads_or(timed_out)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (tid == TC_EPI_THREADS) issue(j + 1);
                pending |= 1u << ((j + 1) & 1);
            }
            if (!is_epi) continue;
            const uint32_t b = (uint32_t)(j & 1);
            if (!bar_wait(&bar[b], (parity >> b) & 1u)) timed_out = true;
            parity ^= 1u << b;
            pending &= ~(1u << b);
            tc_fence_after();
            // input row j's MMAs are done: its slot takes row j + TC_NSLOT
            copy_row(j + TC_NSLOT);
            const int t = j - 2;
            if (t < 0) continue;
            // accumulator + bias -> FP32 staging tile t & 1 (on the run's last row
            // no block barrier has separated this from the tile's previous readers)
            if (j + 1 >= L + 2) epi_sync();
            float* tile = tiles + (t & 1) * Cf::TILE;
            const uint32_t blk = (uint32_t)((t % TC_NBLK) * COUT);
#pragma unroll
            for (int ch = 0; ch < Cf::EPI_CH; ++ch) {
                if (warp >= Cf::TW_WARPS) break;
                const int c = col0 + Cf::NC * ch;
                float v[16];
                tc_ld<Cf::NC>(t_lane + blk + (uint32_t)c, v);
#pragma unroll
                for (int q = 0; q < Cf::NC / 4; ++q) {
                    const int k = c / 4 + q;
                    const float4 bb = *reinterpret_cast<const float4*>(s_bias + 4 * k);
                    *reinterpret_cast<float4*>(tile + pix * COUT + 4 * (k ^ (pix & Cf::SWZ))) =
                        make_float4(v[4 * q] + bb.x, v[4 * q + 1] + bb.y, v[4 * q + 2] + bb.z, v[4 * q + 3] + bb.w);
                }
            }
            // row t - 1 leaves from the other tile (written in the previous
            // iteration, one block barrier ago)
            if (t >= 1) copy_out(t - 1, tiles + ((t - 1) & 1) * Cf::TILE);
            prefetch_epi(t);  // row t's mask and residual, for its copy-out
        }
        // the run's last row (after a timeout every thread has left the loop together)
        if (ok && is_epi) {
            epi_sync();
            copy_out(L - 1, tiles + ((L - 1) & 1) * Cf::TILE);
        }
        // copies still in flight (rows the run does not need) land before the slots are reused
        if (is_epi) cp_async_wait<0>();
        tc_fence_before();
        if (__syncthreads_or(timed_out)) ok = false;
        tc_fence_after();
    }
    if (!ok) {
        // let MMAs still in flight finish (bounded) before the memory is released
        if (is_epi)
            for (uint32_t b = 0; b < 2; ++b)
                if (pending & (1u << b)) bar_wait(&bar[b], (parity >> b) & 1u);
        if (tid == 0) atomicOr(status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cf::TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of a 64 -> 64 convolution on the tensor cores:
// dW[tap (dy, dx)][co][ci] = sum over pixels p of dOut[p][co] In[p + (dy, dx)][ci]
// (In after the ReLU the forward applied). Block (x, y): filter row dy =
// y - 1, a share x of the (image, row, 128-pixel strip) chunks. Per chunk
// the dOut row segment [128 pixels][64 co] and the input row segment
// [130 pixels][64 ci] (one pixel of halo each side, periodic) land by
// cp.async in one of WG_NS stages (the next chunk in flight while one is
// multiplied), both as 128-byte rows per pixel with the tensor core's
// 128-byte swizzle. The contraction runs over pixels, so both
// operands are MN-major (the pixel index is the K index of their rows):
//   D1[(dx, ci)][co], dx = -1, 0:  A = the input rows from pixel k (dx = -1)
//       and the same rows one pixel on (dx = 0) as the two 64-row halves
//       of M = 128 (leading byte offset 128: the second half starts one
//       pixel row later), B = the dOut rows (N = 64);
//   D2[(dx, ci)][co], dx = 0, +1: the same from one pixel on (its first
//       half repeats dx = 0 and is not read).
// One K step is 16 pixels (2048 bytes); 8 steps and 2 MMAs per chunk. The
// accumulators live in tensor memory (128 lanes x 128 columns) for all of
// the block's chunks; at the end they are read with tcgen05.ld and written
// as the block's partial sums [block][dy][dx][co][ci], which
// k_wgrad_sum adds in block order. The MMAs of chunk i are committed to
// the mbarrier of its stage, which is refilled only after they completed.
constexpr int WG_THREADS = 256;
constexpr int WG_PIX = 128;
constexpr int WG_D_BYTES = WG_PIX * 128;                        // 16 KB
constexpr int WG_X_BYTES = ((WG_PIX + 2) * 128 + 1023) / 1024 * 1024;  // 17 KB
constexpr int WG_STAGE = WG_D_BYTES + WG_X_BYTES;
constexpr int WG_NS = 2;     // stages (three, loading one or two chunks ahead, measured the same)
constexpr int WG_AHEAD = 1;  // chunks loaded ahead: the stage refilled is that of chunk
                             // it + WG_AHEAD - WG_NS
constexpr int WG_BYTES = WG_NS * WG_STAGE + 1024;

__device__ __forceinline__ void wg_cp16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// MN-major operand in 128-byte swizzled rows (one row per K index): atoms of
// 8 K rows (SBO = 1024 bytes); lbo: byte offset between the 64-wide halves
// along M or N; swizzle mode 2 (bits 61-63)
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad_tc(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dout, int N, int H, int W,
               int in_relu, float* __restrict__ part, int* __restrict__ status) {
    constexpr int C = 64;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[WG_NS];
    __shared__ uint32_t tmem_base;
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int dy = (int)blockIdx.y - 1;
    const int tiles_x = (W + WG_PIX - 1) / WG_PIX;
    const int nchunks = N * H * tiles_x;  // below 2^31 (checked by the launcher)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < WG_NS; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both
    // MN-major (bits 15, 16 = 1), N = 64 (N >> 3 at bits 17-22), M = 128
    // (M >> 4 at bits 24-28)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((64u >> 3) << 17) |
                           ((128u >> 4) << 24);

    // chunk ch into stage st: dOut row segment and halo'd input row segment
    // (32-bit index arithmetic: every thread works out the chunk's position)
    auto load = [&](int ch, int st) {
        if (ch < nchunks) {
            const unsigned ry = (unsigned)ch / (unsigned)tiles_x;  // n * H + y
            const int x0 = (ch - (int)ry * tiles_x) * WG_PIX;
            const unsigned n = ry / (unsigned)H;
            const int y = (int)(ry - n * (unsigned)H);
            int yy = y + dy;
            yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
            const uint32_t sd = sbase + st * WG_STAGE, sx = sd + WG_D_BYTES;
            const __nv_bfloat16* drow = dout + (size_t)ry * W * C;
            const __nv_bfloat16* xrow = in + ((size_t)n * H + yy) * W * C;
            for (int e = tid; e < WG_PIX * 8; e += WG_THREADS) {
                const int px = e / 8, kg = e % 8;
                const int x = x0 + px;
                wg_cp16(sd + px * 128 + ((kg ^ (px & 7)) * 16), drow + (size_t)(x < W ? x : 0) * C + kg * 8,
                        x < W ? 16 : 0);  // pixels past the image contribute nothing
            }
            for (int e = tid; e < (WG_PIX + 2) * 8; e += WG_THREADS) {
                const int px = e / 8, kg = e % 8;
                int x = x0 - 1 + px;
                x = x < 0 ? x + W : (x >= W ? x % W : x);
                wg_cp16(sx + px * 128 + ((kg ^ (px & 7)) * 16), xrow + (size_t)x * C + kg * 8, 16);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto relu_stage = [&](int st) {
        unsigned char* sx = smem + st * WG_STAGE + WG_D_BYTES;
        for (int e = tid; e < (WG_PIX + 2) * 8; e += WG_THREADS) {
            uint4* v = reinterpret_cast<uint4*>(sx + e * 16);
            *v = relu8(*v);
        }
    };

    // thread 0 waits for the tensor core, the block learns the outcome at a
    // barrier (every thread takes the same branch)
    bool ok = true;
    uint32_t pending = 0;  // bit b: a commit to bar[b] not yet waited for
    int it = 0;
    int ch = blockIdx.x;
    for (int j = 0; j < WG_AHEAD; ++j) load(ch + j * (int)gridDim.x, j);
    for (; ch < nchunks; ch += gridDim.x, ++it) {
        const int st = it % WG_NS;
        const int sp = (it + WG_AHEAD) % WG_NS;  // refilled with chunk it + WG_AHEAD
        const int prev = it + WG_AHEAD - WG_NS;  // the chunk that stage held
        // it is refilled once the MMAs of that chunk have read it
        if (prev >= 0) {
            const int late = tid == 0 && !bar_wait(&bar[sp], (uint32_t)(prev / WG_NS) & 1u);
            if (__syncthreads_or(late)) { ok = false; break; }
            pending &= ~(1u << sp);
        }
        load(ch + WG_AHEAD * (int)gridDim.x, sp);
        // one commit group per load: all but the newest WG_AHEAD have landed
        asm volatile("cp.async.wait_group %0;" ::"n"(WG_AHEAD) : "memory");
        if (in_relu) {
            __syncthreads();  // every thread's copies have landed
            relu_stage(st);
        }
        fence_proxy_async();  // the copies and the ReLU, for the tensor core's reads
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sd = sbase + st * WG_STAGE, sx = sd + WG_D_BYTES;
#pragma unroll
            for (int kk = 0; kk < WG_PIX / 16; ++kk) {
                const uint64_t b = sdesc_mn_sw128(sd + kk * 16 * 128, 16);
                const uint64_t a1 = sdesc_mn_sw128(sx + kk * 16 * 128, 128);
                const uint64_t a2 = sdesc_mn_sw128(sx + (kk * 16 + 1) * 128, 128);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                tc_mma(tmem, a1, b, idesc, acc);
                tc_mma(tmem + 64, a2, b, idesc, acc);
            }
            tc_commit(&bar[st]);
        }
        pending |= 1u << st;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last commits: every MMA done before the accumulators are read
    int late = 0;
    if (tid == 0)
        for (int b = 0; b < WG_NS; ++b)
            if (pending & (1u << b)) {
                const int last = b + WG_NS * ((it - 1 - b) / WG_NS);  // the last chunk in stage b
                if (!bar_wait(&bar[b], (uint32_t)(last / WG_NS) & 1u)) late = 1;
            }
    if (__syncthreads_or(late)) ok = false;
    tc_fence_after();
    float* pb = part + ((size_t)blockIdx.x * 3 + blockIdx.y) * 3 * C * C;
    if (warp < 4) {
        // lane m = 32 warp + lane of D: (dx, ci) = (m / 64, m % 64) for D1 (dx = -1, 0)
        // and (m / 64 + 1, m % 64) for D2 (dx = 0, +1: its upper half only)
        const int m = 32 * warp + lane;
        const int ci = m % 64;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && m < 64) continue;
            const int dxi = m / 64 + h;  // 0, 1, 2 for dx = -1, 0, +1
#pragma unroll
            for (int c16 = 0; c16 < 4; ++c16) {
                float v[16];
                if (it > 0 && ok) tc_ld<16>(tl + h * 64 + c16 * 16, v);
                else
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
#pragma unroll
                for (int j = 0; j < 16; ++j) pb[((size_t)dxi * C + c16 * 16 + j) * C + ci] = v[j];
            }
        }
    }
    if (!ok && tid == 0) atomicOr(status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
    }
}

template <int CIN, int COUT>
cudaError_t conv_tc_t(const ConvArgs& a, cudaStream_t s, int sms, int* status) {
    using Cf = TcCfg<CIN, COUT>;
    static bool set = false;
    if (!set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::BYTES);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const long long rows = (long long)a.N * a.H * ((a.W + TC_TW - 1) / TC_TW);
    const int grid = rows < sms ? (int)rows : sms;
    k_conv_tc<CIN, COUT><<<grid, TC_THREADS, Cf::BYTES, s>>>(a.in, a.w, a.bias, a.N, a.H, a.W, a.in_relu, a.mask,
                                                             a.res16, a.res32, a.res32_c, a.out16, a.out32, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wgrad_tc(int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W,
                            int in_relu, float* dw, float* part, cudaStream_t s, int sms, int* status) {
    if (cin != 64 || cout != 64 || N < 1 || H < 1 || W < 16 || W % 16 != 0 || !status || sms < 1)
        return cudaErrorInvalidValue;
    static bool set = false;
    if (!set) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_BYTES);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const long long chunks = (long long)N * H * ((W + WG_PIX - 1) / WG_PIX);
    if (chunks + (long long)WG_NS * (2 * sms + 2) / 3 >= (1ll << 31)) return cudaErrorInvalidValue;  // 32-bit chunk indices
    // with the three filter rows: two blocks per SM, all in one wave (the
    // mma.sync weight gradient splits the pixels the same way, so the two
    // paths sum the same partials in the same order)
    long long gx = (2 * sms) / 3;
    if (gx < 1) gx = 1;
    if (gx > chunks) gx = chunks;
    k_wgrad_tc<<<dim3((unsigned)gx, 3), WG_THREADS, WG_BYTES, s>>>(in, dout, N, H, W, in_relu, part, status);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_wgrad_sum(part, (int)gx, cout * cin, dw, s);
}

cudaError_t launch_conv_tc(int cin, int cout, const ConvArgs& a, cudaStream_t s, int sms, int* status) {
    if (a.N < 1 || a.H < 1 || a.W < 16 || a.W % 16 != 0 || !status || sms < 1) return cudaErrorInvalidValue;
    if (cin == 16 && cout == 64) return conv_tc_t<16, 64>(a, s, sms, status);
    if (cin == 64 && cout == 64) return conv_tc_t<64, 64>(a, s, sms, status);
    if (cin == 64 && cout == 16) return conv_tc_t<64, 16>(a, s, sms, status);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
