// 3x3 periodic convolution of the surrogate on the 5th-generation tensor
// cores: tcgen05.mma (kind::f16: BF16 operands in shared memory, FP32
// accumulators in tensor memory), issued by one thread, completion tracked by
// tcgen05.commit on an mbarrier (every wait bounded in time).
//
// Work: the output is cut into rows of TC_TW = 128 pixels (one MMA M); the
// rows of all (image, 128-pixel strip) columns are dealt out to the CTAs in
// contiguous runs, so a CTA walks down a strip and loads each input row once
// (a ring of 4 halo'd input rows in shared memory: 3 in use, 1 filling).
// Two accumulators in tensor memory let the MMAs of row t + 1 run while the
// epilogue of row t reads row t out with tcgen05.ld.
//
// Shared-memory operand layouts (K-major, no swizzle; a core matrix is 8
// rows of 16 bytes):
//   input row slot [CIN/8 channel groups][TC_TW + 2 pixels, stride 16 B]
//     with the channel-group stride GS = (TC_TW + 3) * 16 B (an odd number
//     of 16-byte units, so the staging stores spread over the banks). An
//     8-pixel run of one group is one core matrix: the window of tap dx is
//     the same operand with its start moved by (1 + dx) * 16 B.
//     Descriptor: LBO (next channel group, K) = GS, SBO (next 8 pixels, M) = 128.
//   weights [9 taps][CIN/8][COUT][8 channels]: LBO = COUT * 16, SBO = 128.
// One output row = 9 taps x CIN/16 MMAs of M = 128, N = COUT, K = 16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_conv.h"
#include "lbm_ptx.cuh"

namespace lbm {
namespace {

constexpr int TC_TW = 128;       // pixels per output row segment (MMA M)
constexpr int TC_THREADS = 256;  // 8 warps; warp w reads TMEM lanes 32 (w % 4) .. + 31
constexpr int TC_NSLOT = 4;      // input-row ring

template <int CIN, int COUT>
struct TcCfg {
    static constexpr int KG = CIN / 8;                  // 8-channel groups
    static constexpr int PIX = TC_TW + 2;               // halo'd pixels per row
    static constexpr int GS = (TC_TW + 3) * 16;         // bytes between channel groups
    static constexpr int SLOT_BYTES = KG * GS;
    static constexpr int W_BYTES = 9 * KG * COUT * 16;
    static constexpr int BYTES = TC_NSLOT * SLOT_BYTES + W_BYTES + 128;  // + alignment slack
    static constexpr int ROW_VECS = KG * PIX;           // 16-byte vectors per halo'd row
    static constexpr int VPT = (ROW_VECS + TC_THREADS - 1) / TC_THREADS;
    static constexpr int TMEM_COLS = 2 * COUT < 32 ? 32 : 2 * COUT;  // two accumulators, power of two
    static constexpr int EPI_WARPS = COUT >= 32 ? 8 : 4;
    static constexpr int EPI_COLS = COUT >= 32 ? COUT / 2 : COUT;    // accumulator columns per epilogue warp
    static constexpr int EPI_CH = EPI_COLS / 16;                      // 16-column chunks per epilogue thread
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "tcgen05 f16 shape");
    static_assert(TMEM_COLS <= 512, "tensor memory");
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
// SBO >> 4 (32-45), fixed version 0b001 (46-48), no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
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

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// all threads: make this thread's shared-memory stores visible to the tensor
// cores, then a block barrier that also orders tensor-core work around it
__device__ __forceinline__ void tc_sync_stores() {
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// bounded wait on an mbarrier phase; true when it completed in time
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > WAIT_NS) return false;
    return true;
}

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
    __shared__ float s_bias[COUT];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    unsigned char* s_in = smem;
    unsigned char* s_w = smem + TC_NSLOT * Cf::SLOT_BYTES;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

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
    // weights [9][COUT][CIN] -> [9][CIN/8][COUT][8]
    for (int e = tid; e < 9 * COUT * Cf::KG; e += TC_THREADS) {
        const int kg = e % Cf::KG, co = (e / Cf::KG) % COUT, tap = e / (Cf::KG * COUT);
        const uint4 v = *reinterpret_cast<const uint4*>(w + ((size_t)tap * COUT + co) * CIN + kg * 8);
        *reinterpret_cast<uint4*>(s_w + ((tap * Cf::KG + kg) * COUT + co) * 16) = v;
    }
    tc_sync_stores();
    const uint32_t tmem = tmem_base;
    // instruction descriptor: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
    // 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
    // M >> 4 (bits 24-28)
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) |
                           ((uint32_t)(TC_TW >> 4) << 24);
    const uint32_t s_in_addr = smem_u32(s_in), s_w_addr = smem_u32(s_w);
    const int tiles_x = (W + TC_TW - 1) / TC_TW;
    const long long rows_total = (long long)N * tiles_x * H;
    const long long r_begin = rows_total * blockIdx.x / gridDim.x;
    const long long r_end = rows_total * (blockIdx.x + 1) / gridDim.x;
    uint32_t parity = 0;   // bit b: phase parity awaited next on bar[b]
    uint32_t pending = 0;  // bit b: a commit to bar[b] not yet waited for
    bool ok = true;

    // epilogue geometry of this thread: pixel = TMEM lane, a range of columns
    const bool epi = warp < Cf::EPI_WARPS;
    const int pix = 32 * (warp % 4) + lane;
    const int col0 = (warp / 4) * Cf::EPI_COLS;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (warp % 4)) << 16);

    for (long long r = r_begin; r < r_end && ok;) {
        const int y0 = (int)(r % H);
        const long long strip = r / H;
        const int x0 = (int)(strip % tiles_x) * TC_TW, n = (int)(strip / tiles_x);
        const int L = (int)((long long)(H - y0) < r_end - r ? (long long)(H - y0) : r_end - r);
        r += L;
        const __nv_bfloat16* img = in + (size_t)n * H * W * CIN;
        uint4 rv[Cf::VPT];
        // halo'd input row li of this run (input row y0 - 1 + li, periodic)
        auto load_row = [&](int li) {
            const int gy = ((y0 - 1 + li) % H + H) % H;
            const __nv_bfloat16* row = img + (size_t)gy * W * CIN;
#pragma unroll
            for (int i = 0; i < Cf::VPT; ++i) {
                const int e = tid + i * TC_THREADS;
                if (e < Cf::ROW_VECS) {
                    const int kg = e % Cf::KG, px = e / Cf::KG;
                    const int gx = ((x0 - 1 + px) % W + W) % W;
                    rv[i] = *reinterpret_cast<const uint4*>(row + (size_t)gx * CIN + kg * 8);
                }
            }
        };
        auto store_row = [&](int li) {
            unsigned char* slot = s_in + (li % TC_NSLOT) * Cf::SLOT_BYTES;
#pragma unroll
            for (int i = 0; i < Cf::VPT; ++i) {
                const int e = tid + i * TC_THREADS;
                if (e < Cf::ROW_VECS) {
                    const int kg = e % Cf::KG, px = e / Cf::KG;
                    *reinterpret_cast<uint4*>(slot + kg * Cf::GS + px * 16) = in_relu ? relu8(rv[i]) : rv[i];
                }
            }
        };
        // MMAs of output row t (input rows li = t, t + 1, t + 2) into accumulator t & 1
        auto issue = [&](int t) {
            if (tid == 0) {
                const uint32_t d = tmem + (uint32_t)((t & 1) * COUT);
                uint32_t accum = 0;
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                    const uint32_t a_tap =
                        s_in_addr + (uint32_t)(((t + dy + 1) % TC_NSLOT) * Cf::SLOT_BYTES + (1 + dx) * 16);
                    const uint32_t b_tap = s_w_addr + (uint32_t)(tap * Cf::KG * COUT * 16);
#pragma unroll
                    for (int kc = 0; kc < CIN / 16; ++kc) {
                        const uint64_t ad = sdesc(a_tap + (uint32_t)(2 * kc * Cf::GS), Cf::GS, 128);
                        const uint64_t bd = sdesc(b_tap + (uint32_t)(2 * kc * COUT * 16), COUT * 16, 128);
                        tc_mma(d, ad, bd, idesc, accum);
                        accum = 1;
                    }
                }
                tc_commit(&bar[t & 1]);
            }
            pending |= 1u << (t & 1);
        };

        load_row(0);
        store_row(0);
        load_row(1);
        store_row(1);
        load_row(2);
        store_row(2);
        if (L > 1) load_row(3);
        tc_sync_stores();
        issue(0);
        for (int t = 0; t < L; ++t) {
            const int y = y0 + t;
            if (t + 1 < L) {
                // the slot of row li = t + 3 last served output row t - 1, whose MMAs were waited for
                store_row(t + 3);
                tc_sync_stores();  // also: the epilogue of row t - 1 has read accumulator (t + 1) & 1
                issue(t + 1);
                if (t + 2 < L) load_row(t + 4);
            }
            // prefetch the epilogue's operands of row t
            const bool valid = epi && x0 + pix < W;
            const size_t p = ((size_t)n * H + y) * W + (valid ? x0 + pix : 0);
            uint4 mreg[Cf::EPI_CH][2], rreg[Cf::EPI_CH][2];
            if (valid) {
#pragma unroll
                for (int ch = 0; ch < Cf::EPI_CH; ++ch) {
                    const int c = col0 + 16 * ch;
                    if (mask) {
                        mreg[ch][0] = *reinterpret_cast<const uint4*>(mask + p * COUT + c);
                        mreg[ch][1] = *reinterpret_cast<const uint4*>(mask + p * COUT + c + 8);
                    }
                    if (res16) {
                        rreg[ch][0] = *reinterpret_cast<const uint4*>(res16 + p * COUT + c);
                        rreg[ch][1] = *reinterpret_cast<const uint4*>(res16 + p * COUT + c + 8);
                    }
                }
            }
            const uint32_t b = (uint32_t)(t & 1);
            const bool done = bar_wait(&bar[b], (parity >> b) & 1u);
            if (__syncthreads_or(!done)) {
                ok = false;
                break;
            }
            parity ^= 1u << b;
            pending &= ~(1u << b);
            tc_fence_after();
            if (epi) {
#pragma unroll
                for (int ch = 0; ch < Cf::EPI_CH; ++ch) {
                    const int c = col0 + 16 * ch;
                    float v[16];
                    tc_ld16(t_lane + b * COUT + (uint32_t)c, v);
                    if (!valid) continue;
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += s_bias[c + j];
                    if (mask) {
                        const __nv_bfloat16* mh = reinterpret_cast<const __nv_bfloat16*>(mreg[ch]);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (!(__bfloat162float(mh[j]) > 0.f)) v[j] = 0.f;
                    }
                    if (res16) {
                        const __nv_bfloat16* rh = reinterpret_cast<const __nv_bfloat16*>(rreg[ch]);
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] += __bfloat162float(rh[j]);
                    }
                    if (res32) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c + j < res32_c) v[j] += res32[p * res32_c + c + j];
                    }
                    if (out32) {
                        float4* o = reinterpret_cast<float4*>(out32 + p * COUT + c);
#pragma unroll
                        for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    } else {
                        uint4 o[2];
                        __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(o);
#pragma unroll
                        for (int j = 0; j < 8; ++j) oh[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        uint4* dst = reinterpret_cast<uint4*>(out16 + p * COUT + c);
                        dst[0] = o[0];
                        dst[1] = o[1];
                    }
                }
            }
        }
        // the next run reuses the slots and accumulator 0
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok) {
        // let MMAs still in flight finish (bounded) before the memory is released
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

cudaError_t launch_conv_tc(int cin, int cout, const ConvArgs& a, cudaStream_t s, int sms, int* status) {
    if (a.N < 1 || a.H < 1 || a.W < 16 || a.W % 16 != 0 || !status || sms < 1) return cudaErrorInvalidValue;
    if (cin == 16 && cout == 64) return conv_tc_t<16, 64>(a, s, sms, status);
    if (cin == 64 && cout == 64) return conv_tc_t<64, 64>(a, s, sms, status);
    if (cin == 64 && cout == 16) return conv_tc_t<64, 16>(a, s, sms, status);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
