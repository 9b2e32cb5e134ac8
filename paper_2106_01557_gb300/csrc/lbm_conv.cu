// BF16 tensor-core kernels of the learned surrogate (a 3x3 convolutional
// neural operator that advances (rho, u_x, u_y, T) by K lattice steps), with
// FP32 accumulation:
//   k_conv       implicit-GEMM 3x3 convolution, periodic padding, NHWC BF16
//                activations; the whole weight tensor and a halo'd input tile
//                sit in shared memory; fused epilogue: bias, ReLU mask of
//                another tensor, residual add (BF16 or FP32), BF16 or FP32
//                output. Also serves the input gradient (flipped weights).
//   k_wgrad      weight gradient: per (tap, 16 output channels) a GEMM over
//                pixels, warps splitting the pixels; each block writes its
//                partial sums, which k_wgrad_sum adds in block order (the
//                64 -> 64 layers have a tcgen05 version in lbm_conv_tc.cu).
//   k_bgrad      bias gradient (per-block partials, summed in block order).
// No reduction uses atomics: the order of every sum is fixed, so training
// is bit-for-bit reproducible.
//   k_mse        loss and its gradient.
//   k_adam       optimiser step on FP32 master weights, refreshing the BF16
//                forward and flipped copies.
//   k_pack / k_unpack  fields <-> normalised network tensors.
// The MMA is mma.sync m16n8k16 (BF16 in, FP32 accumulate).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_conv.h"

namespace lbm {
namespace {

__device__ __forceinline__ void mma_bf16(float& c0, float& c1, float& c2, float& c3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ __nv_bfloat16 relu_bf(__nv_bfloat16 v) {
    return __hgt(v, __float2bfloat16(0.f)) ? v : __float2bfloat16(0.f);
}

constexpr int TW = 128;          // output pixels along x per tile
constexpr int TH = 2;            // output rows per tile
constexpr int CT = 512;          // threads: 16 warps, one 16-pixel m-tile each

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int PS = CIN + 8;                       // padded pixel stride (bank spread)
    static constexpr int IN_ELEMS = (TH + 2) * (TW + 2) * PS;
    static constexpr int W_ELEMS = 9 * COUT * PS;
    static constexpr int BYTES = 2 * (IN_ELEMS + W_ELEMS);
};

// Persistent: each CTA stages all weights once, then walks tiles of TH rows x
// TW pixels of one image.
template <int CIN, int COUT>
__global__ void __launch_bounds__(CT, 1)
    k_conv(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
           int N, int H, int W, int in_relu, const __nv_bfloat16* __restrict__ mask,
           const __nv_bfloat16* __restrict__ res16, const float* __restrict__ res32, int res32_c,
           __nv_bfloat16* __restrict__ out16, float* __restrict__ out32) {
    using SMc = ConvSmem<CIN, COUT>;
    constexpr int PS = SMc::PS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* s_in = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* s_w = s_in + SMc::IN_ELEMS;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int g = lane / 4, t = lane % 4;

    // weights [9][COUT][CIN] -> shared [9][COUT][PS], 8 channels per copy
    for (int e = tid; e < 9 * COUT * (CIN / 8); e += CT) {
        const int row = e / (CIN / 8), c8 = e % (CIN / 8);
        *reinterpret_cast<uint4*>(s_w + row * PS + c8 * 8) = *reinterpret_cast<const uint4*>(w + row * CIN + c8 * 8);
    }
    const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
    const int ntiles = N * tiles_y * tiles_x;
    constexpr int NT8 = COUT / 8;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, n = tile / (tiles_x * tiles_y);
        const int x0 = tx * TW, y0 = ty * TH;
        __syncthreads();  // previous tile's reads of s_in done (and weights staged)
        // halo'd input tile: rows y0-1 .. y0+TH, pixels x0-1 .. x0+TW (periodic)
        for (int e = tid; e < (TH + 2) * (TW + 2) * (CIN / 8); e += CT) {
            const int c8 = e % (CIN / 8), px = (e / (CIN / 8)) % (TW + 2), r = e / ((CIN / 8) * (TW + 2));
            int gy = y0 - 1 + r, gx = x0 - 1 + px;
            gy = (gy % H + H) % H;
            gx = (gx % W + W) % W;
            uint4 v = *reinterpret_cast<const uint4*>(in + (((size_t)n * H + gy) * W + gx) * CIN + c8 * 8);
            if (in_relu) {
                __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = relu_bf(h[j]);
            }
            *reinterpret_cast<uint4*>(s_in + (r * (TW + 2) + px) * PS + c8 * 8) = v;
        }
        __syncthreads();
        const int orow = warp / (TW / 16), px0 = (warp % (TW / 16)) * 16;
        float acc[NT8][4];
#pragma unroll
        for (int j = 0; j < NT8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const __nv_bfloat16* arow = s_in + ((orow + 1 + dy) * (TW + 2) + px0 + 1 + dx) * PS;
            const __nv_bfloat16* wt = s_w + tap * COUT * PS;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                const __nv_bfloat16* a = arow + kc * 16 + 2 * t;
                const uint32_t a0 = ld32(a + g * PS), a1 = ld32(a + (g + 8) * PS);
                const uint32_t a2 = ld32(a + g * PS + 8), a3 = ld32(a + (g + 8) * PS + 8);
#pragma unroll
                for (int j = 0; j < NT8; ++j) {
                    const __nv_bfloat16* b = wt + (j * 8 + g) * PS + kc * 16 + 2 * t;
                    mma_bf16(acc[j][0], acc[j][1], acc[j][2], acc[j][3], a0, a1, a2, a3, ld32(b), ld32(b + 8));
                }
            }
        }
        // epilogue
        const int oy = y0 + orow;
        if (oy < H) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int ox = x0 + px0 + g + 8 * half;
                if (ox >= W) continue;
                const size_t p = ((size_t)n * H + oy) * W + ox;
#pragma unroll
                for (int j = 0; j < NT8; ++j) {
                    const int co = j * 8 + 2 * t;
                    float v0 = acc[j][2 * half], v1 = acc[j][2 * half + 1];
                    if (bias) { v0 += bias[co]; v1 += bias[co + 1]; }
                    if (mask) {
                        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask + p * COUT + co);
                        if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
                    }
                    if (res16) {
                        const __nv_bfloat162 r = *reinterpret_cast<const __nv_bfloat162*>(res16 + p * COUT + co);
                        v0 += __bfloat162float(r.x);
                        v1 += __bfloat162float(r.y);
                    }
                    if (res32) {
                        if (co < res32_c) v0 += res32[p * res32_c + co];
                        if (co + 1 < res32_c) v1 += res32[p * res32_c + co + 1];
                    }
                    if (out32) {
                        out32[p * COUT + co] = v0;
                        out32[p * COUT + co + 1] = v1;
                    } else {
                        *reinterpret_cast<__nv_bfloat162*>(out16 + p * COUT + co) = __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
        }
    }
}

// Weight gradient dW[tap][co][ci] += sum_p dOut[p][co] * act(in[p + off(tap)][ci]).
// A CTA owns one filter row dy (its three taps dx = -1, 0, 1) and every
// output and input channel, over a run of 128-pixel row chunks: the chunk's
// dOut row [128 px][COUT] and the input row y + dy [130 px][CIN] (periodic
// halo) are copied with cp.async into padded shared tiles (two stages), and
// ldmatrix.trans forms the MMA fragments straight from these pixel-major
// tiles: A = dOut^T (co x pixels), B = input (pixels x ci, shifted by dx).
// One A fragment serves the three taps. Warp w owns the 16-channel output
// block w % (COUT/16) and a contiguous group of 8-channel input blocks; its
// FP32 sums are added to dw once at the end (atomics).
constexpr int WT = 256;      // threads (8 warps)
constexpr int WCH = 128;     // pixels per chunk

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
// 16-byte async copy; src_bytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

template <int CIN, int COUT>
struct WgCfg {
    static constexpr int RSD = COUT * 2 + 16;          // padded row bytes of the dOut tile (ldmatrix: no conflicts)
    static constexpr int RSX = CIN * 2 + 16;           // padded row bytes of the input tile
    static constexpr int D_BYTES = WCH * RSD;
    static constexpr int X_BYTES = (WCH + 2) * RSX;
    static constexpr int STAGE = D_BYTES + X_BYTES;
    static constexpr int MT = COUT / 16;               // 16-channel output blocks
    static constexpr int NG = 8 / MT;                  // warps per output block
    static constexpr int NPW = (CIN / 8) / NG;         // 8-channel input blocks per warp
    static_assert(COUT % 16 == 0 && COUT <= 128 && 8 % MT == 0 && (CIN / 8) % NG == 0 && NPW >= 1, "warp split");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(WT)
    k_wgrad(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dout, int N, int H, int W,
            int in_relu, float* __restrict__ part) {
    using Cf = WgCfg<CIN, COUT>;
    extern __shared__ __align__(16) unsigned char wg_smem[];
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int g = lane / 4, t = lane % 4;
    const int dy = (int)blockIdx.y - 1;
    const int tiles_x = (W + WCH - 1) / WCH;
    const long long nchunks = (long long)N * H * tiles_x;
    const int mt = warp % Cf::MT, nt0 = (warp / Cf::MT) * Cf::NPW;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(wg_smem);
    float acc[3][Cf::NPW][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < Cf::NPW; ++j) acc[a][j][0] = acc[a][j][1] = acc[a][j][2] = acc[a][j][3] = 0.f;

    // copy chunk ch into stage st (one commit group per call, empty past the end)
    auto load = [&](long long ch, int st) {
        if (ch < nchunks) {
            const int x0 = (int)(ch % tiles_x) * WCH;
            const long long ry = ch / tiles_x;  // n * H + y
            const int y = (int)(ry % H), n = (int)(ry / H);
            int yy = y + dy;
            yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
            const uint32_t sd = sbase + st * Cf::STAGE, sx = sd + Cf::D_BYTES;
            const __nv_bfloat16* drow = dout + (size_t)ry * W * COUT;
            const __nv_bfloat16* xrow = in + ((size_t)n * H + yy) * W * CIN;
            for (int e = tid; e < WCH * (COUT / 8); e += WT) {
                const int px = e / (COUT / 8), c8 = e % (COUT / 8);
                const int x = x0 + px;
                cp16(sd + px * Cf::RSD + c8 * 16, drow + (size_t)(x < W ? x : 0) * COUT + c8 * 8, x < W ? 16 : 0);
            }
            for (int e = tid; e < (WCH + 2) * (CIN / 8); e += WT) {
                const int px = e / (CIN / 8), c8 = e % (CIN / 8);
                int x = x0 - 1 + px;
                x = x < 0 ? x + W : (x >= W ? x % W : x);
                cp16(sx + px * Cf::RSX + c8 * 16, xrow + (size_t)x * CIN + c8 * 8, 16);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // ReLU in place on the input vectors this thread copied
    auto relu_tile = [&](int st) {
        unsigned char* sx = wg_smem + st * Cf::STAGE + Cf::D_BYTES;
        for (int e = tid; e < (WCH + 2) * (CIN / 8); e += WT) {
            const int px = e / (CIN / 8), c8 = e % (CIN / 8);
            uint4* v = reinterpret_cast<uint4*>(sx + px * Cf::RSX + c8 * 16);
            uint4 u = *v;
            __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(&u);
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = relu_bf(h[q]);
            *v = u;
        }
    };

    long long ch = blockIdx.x;
    load(ch, 0);
    for (int it = 0; ch < nchunks; ch += gridDim.x, ++it) {
        const int st = it & 1;
        load(ch + gridDim.x, st ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        if (in_relu) relu_tile(st);
        __syncthreads();
        const uint32_t sd = sbase + st * Cf::STAGE, sx = sd + Cf::D_BYTES;
#pragma unroll 2
        for (int k0 = 0; k0 < WCH; k0 += 16) {
            // A = dOut^T: rows co (mt*16 ..), columns pixels k0 .. k0+15
            const int q = lane / 8;
            uint32_t a0, a1, a2, a3;
            ldsm_x4_t(sd + (k0 + (q >= 2 ? 8 : 0) + lane % 8) * Cf::RSD + (mt * 16 + (q & 1) * 8) * 2, a0, a1, a2, a3);
#pragma unroll
            for (int tap = 0; tap < 3; ++tap) {
                // B = input pixels k0 + dx .. (tile pixel index + 1 for the halo)
#pragma unroll
                for (int j = 0; j < Cf::NPW; ++j) {
                    uint32_t b0, b1;
                    const int l = lane % 16;
                    ldsm_x2_t(sx + (k0 + tap + (l >= 8 ? 8 : 0) + l % 8) * Cf::RSX + (nt0 + j) * 16, b0, b1);
                    mma_bf16(acc[tap][j][0], acc[tap][j][1], acc[tap][j][2], acc[tap][j][3], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        __syncthreads();  // the stage is refilled by the next iteration's load
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // accumulator (row co, column ci) of filter column dx = tap - 1 -> this
    // block's partial [blockIdx.x][dy + 1][tap][co][ci]
    float* pb = part + ((size_t)blockIdx.x * 3 + blockIdx.y) * 3 * COUT * CIN;
#pragma unroll
    for (int tap = 0; tap < 3; ++tap) {
#pragma unroll
        for (int j = 0; j < Cf::NPW; ++j) {
            const int co = mt * 16 + g, ci = (nt0 + j) * 8 + 2 * t;
            float* d = pb + ((size_t)tap * COUT + co) * CIN + ci;
            d[0] = acc[tap][j][0];
            d[1] = acc[tap][j][1];
            d[8 * CIN] = acc[tap][j][2];
            d[8 * CIN + 1] = acc[tap][j][3];
        }
    }
}

// dw[tp][co][ci] += sum over blocks b = 0, 1, ... of the partials, tap
// tp = 3 (dy + 1) + dx + 1 (the order of the sum is fixed)
__global__ void k_wgrad_sum(const float* __restrict__ part, int nblk, int cc, float* __restrict__ dw) {
    const int n = 9 * cc;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int tp = e / cc, rem = e % cc;
        const int by = tp / 3, tl = tp % 3;
        float s = 0.f;
#pragma unroll 8
        for (int b = 0; b < nblk; ++b) s += part[(((size_t)b * 3 + by) * 3 + tl) * cc + rem];
        dw[e] += s;
    }
}

// Bias gradient db[c] += sum_p dOut[p][c] (C a multiple of 8, C <= 256):
// thread = one 8-channel group of a pixel (16-byte loads, coalesced across
// the block), per-thread sums reduced per channel group in shared memory.
__global__ void k_bgrad(const __nv_bfloat16* __restrict__ dout, long long P, int C, float* __restrict__ part) {
    __shared__ float s[256][9];
    const int G8 = C / 8;
    const int per = blockDim.x / G8;  // pixels per block sweep
    const int c8 = threadIdx.x % G8, sub = threadIdx.x / G8;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (sub < per) {
        for (long long p = (long long)blockIdx.x * per + sub; p < P; p += (long long)gridDim.x * per) {
            const uint4 v = *reinterpret_cast<const uint4*>(dout + p * C + c8 * 8);
            const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] += __bfloat162float(h[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int g8 = c / 8, q = c % 8;
        float t = 0.f;
        for (int k = 0; k < per; ++k) t += s[k * G8 + g8][q];
        part[(size_t)blockIdx.x * C + c] = t;
    }
}

// db[c] += sum over blocks b = 0, 1, ... of part[b][c]
// One warp per channel: lane l adds the partials of blocks l, l + 32, ...
// in that order, then a butterfly over the lanes; lane 0's result is the
// same on every run (a fixed order, not a sequential one)
__global__ void k_bgrad_sum(const float* __restrict__ part, int nblk, int C, float* __restrict__ db) {
    const int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
    if (c >= C) return;
    float t = 0.f;
    for (int b = lane; b < nblk; b += 32) t += part[(size_t)b * C + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) db[c] += t;
}

// *out += sum over i = 0 .. n-1 of part[i], by one warp in a fixed order
// (lane l: i = l, l + 32, ...; then a butterfly)
__global__ void k_sum_in_order(const double* __restrict__ part, int n, double* __restrict__ out) {
    const int lane = threadIdx.x;
    if (blockIdx.x != 0 || lane >= 32) return;
    double t = 0.0;
    for (int i = lane; i < n; i += 32) t += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) *out += t;
}

// loss = mean over P pixels and 4 channels of (out - target)^2; dout = d loss / d out.
// With the mass-conserving output layer (csum not null) the density gradient
// is projected: minus its per-image mean, which equals
// 2 (mean(x_rho) - mean(target_rho)) / (4 P); csum[n] = sum over image n of
// (x_rho - target_rho), HW pixels per image.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, long long P,
                      __nv_bfloat16* __restrict__ dout, double* __restrict__ part, const double* __restrict__ csum,
                      long long HW) {
    __shared__ double s[256];
    double acc = 0.0;
    const float scale = 2.0f / (float)(P * 4);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float shift = csum ? (float)(csum[p / HW] / (double)HW) : 0.f;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float d = 0.f;
            if (c < 4) {
                d = out[p * 16 + c] - target[p * 4 + c];
                acc += (double)d * d;
            }
            dout[p * 16 + c] = __float2bfloat16(c < 4 ? scale * (c == 0 ? d - shift : d) : 0.f);
        }
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0] / (double)(P * 4);
}

// Adam on FP32 master weights of one convolution ([9][COUT][CIN] and bias),
// then the BF16 forward copy and the flipped, transposed copy used for the
// input gradient: wf[8 - tap][ci][co] = w[tap][co][ci].
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ gw, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = gw[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_refresh(const float* __restrict__ w, int cin, int cout, int cin_real, int cout_real,
                          __nv_bfloat16* __restrict__ w16, __nv_bfloat16* __restrict__ wflip) {
    const int n = 9 * cout * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cin, co = (i / cin) % cout, tap = i / (cin * cout);
        const float val = (ci < cin_real && co < cout_real) ? w[i] : 0.f;  // padding stays zero
        const __nv_bfloat16 b = __float2bfloat16(val);
        w16[i] = b;
        if (wflip) wflip[((size_t)(8 - tap) * cin + ci) * cout + co] = b;
    }
}

// fields -> normalised network input: 16 BF16 channels (4 used) and an FP32
// copy of the 4 channels for the output residual
__global__ void k_pack(const double* __restrict__ rho, const double* __restrict__ ux, const double* __restrict__ uy,
                       const double* __restrict__ T, long long P, NormConsts nc, __nv_bfloat16* __restrict__ x16,
                       float* __restrict__ x32) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float v[4] = {(float)((rho[p] - nc.off[0]) * nc.inv_scale[0]), (float)((ux[p] - nc.off[1]) * nc.inv_scale[1]),
                            (float)((uy[p] - nc.off[2]) * nc.inv_scale[2]), (float)((T[p] - nc.off[3]) * nc.inv_scale[3])};
#pragma unroll
        for (int c = 0; c < 16; ++c) x16[p * 16 + c] = __float2bfloat16(c < 4 ? v[c] : 0.f);
        if (x32)
#pragma unroll
            for (int c = 0; c < 4; ++c) x32[p * 4 + c] = v[c];
    }
}

__global__ void k_unpack(const float* __restrict__ y, long long P, NormConsts nc, double* __restrict__ rho,
                         double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        rho[p] = nc.off[0] + (double)y[p * 16 + 0] * nc.scale[0];
        ux[p] = nc.off[1] + (double)y[p * 16 + 1] * nc.scale[1];
        uy[p] = nc.off[2] + (double)y[p * 16 + 2] * nc.scale[2];
        T[p] = nc.off[3] + (double)y[p * 16 + 3] * nc.scale[3];
    }
}

// Mass-conserving output layer: per image n, sums[n] = sum of
// (y_rho - x_rho) and, with a target, sums[N + n] = sum of (x_rho - t_rho);
// then y_rho -= sums[n] / HW. y: [P][16], x, t: [P][4]; grid y = images.
// Each block writes its two partial sums to part[n][block][2];
// k_mass_sums adds them in block order.
__global__ void k_mass_stats(const float* __restrict__ y, const float* __restrict__ x, const float* __restrict__ t,
                             int N, long long HW, double* __restrict__ part) {
    __shared__ double s[2][256];
    const int n = blockIdx.y;
    double a = 0.0, b = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < HW; q += (long long)gridDim.x * blockDim.x) {
        const long long p = n * HW + q;
        a += (double)y[p * 16] - (double)x[p * 4];
        if (t) b += (double)x[p * 4] - (double)t[p * 4];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* pp = part + ((size_t)n * gridDim.x + blockIdx.x) * 2;
        pp[0] = s[0][0];
        pp[1] = s[1][0];
    }
}

// one warp per image: lane l adds blocks l, l + 32, ..., then a butterfly
// (a fixed order)
__global__ void k_mass_sums(const double* __restrict__ part, int N, int nblk, int with_t, double* __restrict__ sums) {
    const int n = (int)((blockIdx.x * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
    if (n >= N) return;
    double a = 0.0, b = 0.0;
    for (int k = lane; k < nblk; k += 32) {
        a += part[((size_t)n * nblk + k) * 2];
        b += part[((size_t)n * nblk + k) * 2 + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sums[n] = a;
        if (with_t) sums[N + n] = b;
    }
}

__global__ void k_mass_apply(float* __restrict__ y, long long P, long long HW, const double* __restrict__ sums) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x)
        y[p * 16] = (float)((double)y[p * 16] - sums[p / HW] / (double)HW);
}

// counts over a field set [4][P] of one W-wide periodic image: cnt[0] nodes
// with rho > mid (liquid), cnt[1] nodes that are non-finite or have rho <= 0
// or T <= 0, cnt[2] liquid-vapour edges between x- and y-neighbours (the
// interface length on the lattice's staircase), cnt[3] nodes whose phase
// differs from that in the field set prev (if not null)
__global__ void k_field_check(const double* __restrict__ f, const double* __restrict__ prev, long long P, int W,
                              double mid, unsigned long long* __restrict__ cnt) {
    unsigned long long liq = 0, bad = 0, edge = 0, flip = 0;
    const long long H = P / W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const double r = f[p], u = f[P + p], v = f[2 * P + p], T = f[3 * P + p];
        const bool l = r > mid;
        liq += l;
        bad += !(isfinite(r) && isfinite(u) && isfinite(v) && isfinite(T) && r > 0.0 && T > 0.0);
        const long long yy = p / W, xx = p % W;
        const long long px = yy * W + (xx + 1 == W ? 0 : xx + 1);
        const long long py = (yy + 1 == H ? 0 : yy + 1) * W + xx;
        edge += (l != (f[px] > mid)) + (l != (f[py] > mid));
        if (prev) flip += l != (prev[p] > mid);
    }
    for (int o = 16; o > 0; o >>= 1) {
        liq += __shfl_down_sync(0xffffffffu, liq, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
        edge += __shfl_down_sync(0xffffffffu, edge, o);
        flip += __shfl_down_sync(0xffffffffu, flip, o);
    }
    if (threadIdx.x % 32 == 0) {
        atomicAdd(&cnt[0], liq);
        atomicAdd(&cnt[1], bad);
        atomicAdd(&cnt[2], edge);
        atomicAdd(&cnt[3], flip);
    }
}

// Largest per-node change between two field sets [4][P] (a, b) for the
// density (plane 0) and the temperature (plane 3), and the largest |b| of
// each: out[0] max |a_rho - b_rho|, out[1] max |b_rho|, out[2], out[3] the
// same for T, as the bit patterns of non-negative doubles (their order is the
// order of the values, so an integer maximum is exact and independent of the
// order of the nodes; a NaN difference compares above every number).
__global__ void k_field_change(const double* __restrict__ a, const double* __restrict__ b, long long P,
                               unsigned long long* __restrict__ out) {
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const long long q = (k == 0 ? 0 : 3) * P + p;
            const double d = fabs(a[q] - b[q]), v = fabs(b[q]);
            m[2 * k] = (d > m[2 * k] || d != d) ? d : m[2 * k];
            m[2 * k + 1] = (v > m[2 * k + 1] || v != v) ? v : m[2 * k + 1];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long u = (unsigned long long)__double_as_longlong(m[k]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_down_sync(0xffffffffu, u, o);
            u = w > u ? w : u;
        }
        if (threadIdx.x % 32 == 0) atomicMax(&out[k], u);
    }
}

template <int CIN, int COUT>
cudaError_t conv_t(const ConvArgs& a, cudaStream_t s, int sms) {
    using SMc = ConvSmem<CIN, COUT>;
    static bool set = false;
    if (!set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMc::BYTES);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const int tiles = a.N * ((a.H + TH - 1) / TH) * ((a.W + TW - 1) / TW);
    const int grid = tiles < sms ? tiles : sms;
    k_conv<CIN, COUT><<<grid, CT, SMc::BYTES, s>>>(a.in, a.w, a.bias, a.N, a.H, a.W, a.in_relu, a.mask, a.res16,
                                                   a.res32, a.res32_c, a.out16, a.out32);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad_t(const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W, int in_relu, float* dw,
                    float* part, cudaStream_t s, int sms) {
    using Cf = WgCfg<CIN, COUT>;
    static bool set = false;
    if (!set) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * Cf::STAGE);
        if (e != cudaSuccess) return e;
        set = true;
    }
    const long long chunks = (long long)N * H * ((W + WCH - 1) / WCH);
    long long gx = (2 * sms) / 3;  // with the three filter rows: two CTAs per SM, as in the tcgen05 path
    if (gx > chunks) gx = chunks;
    if (gx < 1) gx = 1;
    k_wgrad<CIN, COUT><<<dim3((unsigned)gx, 3), WT, 2 * Cf::STAGE, s>>>(in, dout, N, H, W, in_relu, part);
    k_wgrad_sum<<<(9 * COUT * CIN + 255) / 256, 256, 0, s>>>(part, (int)gx, COUT * CIN, dw);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_field_check(const double* f, const double* prev, long long P, int W, double mid,
                               unsigned long long* cnt, cudaStream_t s) {
    if (W < 1 || P % W != 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long g = (P + 255) / 256;
    if (g > 2048) g = 2048;
    k_field_check<<<(unsigned)g, 256, 0, s>>>(f, prev, P, W, mid, cnt);
    return cudaGetLastError();
}

cudaError_t launch_field_change(const double* a, const double* b, long long P, unsigned long long* out,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long g = (P + 255) / 256;
    if (g > 2048) g = 2048;
    k_field_change<<<(unsigned)g, 256, 0, s>>>(a, b, P, out);
    return cudaGetLastError();
}

cudaError_t launch_mass_layer(float* y, const float* x, const float* t, int N, long long HW, double* sums,
                              double* part, cudaStream_t s) {
    if (N < 1 || HW < 1) return cudaErrorInvalidValue;
    long long gx = (HW + 255) / 256;
    if (gx > MASS_BLOCKS) gx = MASS_BLOCKS;
    k_mass_stats<<<dim3((unsigned)gx, (unsigned)N), 256, 0, s>>>(y, x, t, N, HW, part);
    k_mass_sums<<<(32 * N + 127) / 128, 128, 0, s>>>(part, N, (int)gx, t != nullptr, sums);
    const long long P = (long long)N * HW;
    long long g = (P + 255) / 256;
    if (g > 2048) g = 2048;
    k_mass_apply<<<(unsigned)g, 256, 0, s>>>(y, P, HW, sums);
    return cudaGetLastError();
}

size_t conv_smem_bytes(int cin, int cout) {
    if (cin == 16 && cout == 64) return ConvSmem<16, 64>::BYTES;
    if (cin == 64 && cout == 64) return ConvSmem<64, 64>::BYTES;
    if (cin == 64 && cout == 16) return ConvSmem<64, 16>::BYTES;
    return 0;
}

cudaError_t launch_conv(int cin, int cout, const ConvArgs& a, cudaStream_t s, int sms) {
    if (a.W % 16 != 0) return cudaErrorInvalidValue;
    if (cin == 16 && cout == 64) return conv_t<16, 64>(a, s, sms);
    if (cin == 64 && cout == 64) return conv_t<64, 64>(a, s, sms);
    if (cin == 64 && cout == 16) return conv_t<64, 16>(a, s, sms);
    return cudaErrorInvalidValue;
}

size_t grad_scratch_floats(int sms) {
    const size_t gx = (size_t)(2 * sms + 2) / 3;
    const size_t w = gx * 9 * 64 * 64, b = (size_t)608 * 256;
    return w > b ? w : b;
}

cudaError_t launch_wgrad(int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W,
                         int in_relu, float* dw, float* part, cudaStream_t s, int sms) {
    if (cin == 16 && cout == 64) return wgrad_t<16, 64>(in, dout, N, H, W, in_relu, dw, part, s, sms);
    if (cin == 64 && cout == 64) return wgrad_t<64, 64>(in, dout, N, H, W, in_relu, dw, part, s, sms);
    if (cin == 64 && cout == 16) return wgrad_t<64, 16>(in, dout, N, H, W, in_relu, dw, part, s, sms);
    return cudaErrorInvalidValue;
}

cudaError_t launch_wgrad_sum(const float* part, int nblk, int cc, float* dw, cudaStream_t s) {
    if (nblk < 1 || cc < 1) return cudaErrorInvalidValue;
    k_wgrad_sum<<<(9 * cc + 255) / 256, 256, 0, s>>>(part, nblk, cc, dw);
    return cudaGetLastError();
}

cudaError_t launch_bgrad(const __nv_bfloat16* dout, long long P, int C, float* db, float* part, cudaStream_t s) {
    if (C < 8 || C % 8 != 0 || C > 256) return cudaErrorInvalidValue;
    const int per = 256 / (C / 8);
    long long g = (P + per - 1) / per;
    if (g > 608) g = 608;
    k_bgrad<<<(unsigned)g, 256, 0, s>>>(dout, P, C, part);
    k_bgrad_sum<<<(C * 32 + 255) / 256, 256, 0, s>>>(part, (int)g, C, db);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float* out, const float* target, long long P, __nv_bfloat16* dout, double* loss,
                       const double* csum, long long HW, double* part, cudaStream_t s) {
    if (csum && HW < 1) return cudaErrorInvalidValue;
    long long g = (P + 255) / 256;
    if (g > MSE_BLOCKS) g = MSE_BLOCKS;
    k_mse<<<(unsigned)g, 256, 0, s>>>(out, target, P, dout, part, csum, HW);
    k_sum_in_order<<<1, 32, 0, s>>>(part, (int)g, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* w, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s) {
    k_adam<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(w, m, v, g, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const float* w, int cin, int cout, int cin_real, int cout_real, __nv_bfloat16* w16,
                           __nv_bfloat16* wflip, cudaStream_t s) {
    const int n = 9 * cin * cout;
    k_refresh<<<(n + 255) / 256, 256, 0, s>>>(w, cin, cout, cin_real, cout_real, w16, wflip);
    return cudaGetLastError();
}

cudaError_t launch_pack(const double* rho, const double* ux, const double* uy, const double* T, long long P,
                        const NormConsts& nc, __nv_bfloat16* x16, float* x32, cudaStream_t s) {
    long long g = (P + 255) / 256;
    if (g > 4096) g = 4096;
    k_pack<<<(unsigned)g, 256, 0, s>>>(rho, ux, uy, T, P, nc, x16, x32);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const float* y, long long P, const NormConsts& nc, double* rho, double* ux, double* uy,
                          double* T, cudaStream_t s) {
    long long g = (P + 255) / 256;
    if (g > 4096) g = 4096;
    k_unpack<<<(unsigned)g, 256, 0, s>>>(y, P, nc, rho, ux, uy, T);
    return cudaGetLastError();
}

}  // namespace lbm
