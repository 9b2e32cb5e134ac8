// BF16 tensor-core kernels of the learned surrogate (a 3x3 convolutional
// neural operator that advances (rho, u_x, u_y, T) by K lattice steps), with
// FP32 accumulation:
//   k_conv       implicit-GEMM 3x3 convolution, periodic padding, NHWC BF16
//                activations; the whole weight tensor and a halo'd input tile
//                sit in shared memory; fused epilogue: bias, ReLU mask of
//                another tensor, residual add (BF16 or FP32), BF16 or FP32
//                output. Also serves the input gradient (flipped weights).
//   k_wgrad      weight gradient: per (tap, 16 output channels) a GEMM over
//                pixels, warps splitting the pixels, FP32 atomics at the end.
//   k_bgrad      bias gradient.
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
// Grid: x = 9 taps * COUT/16 output-channel tiles, y = pixel partitions.
constexpr int WT = 256;      // threads (8 warps)
constexpr int WCH = 128;     // pixels per chunk: 8 warps x one k16 step

template <int CIN, int COUT>
__global__ void __launch_bounds__(WT)
    k_wgrad(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dout, int N, int H, int W,
            int in_relu, float* __restrict__ dw) {
    constexpr int PP = WCH + 8;  // padded pixel stride of the transposed tiles
    constexpr int TILE_BYTES = 2 * (16 + CIN) * PP;
    constexpr int RED_BYTES = 4 * 8 * 16 * (CIN + 1);
    // the transposed tiles and, after the pixel loop, the cross-warp sums share one buffer
    __shared__ __align__(16) unsigned char s_buf[TILE_BYTES > RED_BYTES ? TILE_BYTES : RED_BYTES];
    __nv_bfloat16* s_d = reinterpret_cast<__nv_bfloat16*>(s_buf);            // [co][p]
    __nv_bfloat16* s_x = s_d + 16 * PP;                                       // [ci][p]
    float (*s_red)[16][CIN + 1] = reinterpret_cast<float (*)[16][CIN + 1]>(s_buf);
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    const int g = lane / 4, t = lane % 4;
    const int tap = blockIdx.x / (COUT / 16), cot = blockIdx.x % (COUT / 16);
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long P = (long long)N * H * W;
    const long long nchunks = (P + WCH - 1) / WCH;
    constexpr int NT8 = CIN / 8;
    float acc[NT8][4];
#pragma unroll
    for (int j = 0; j < NT8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (long long ch = blockIdx.y; ch < nchunks; ch += gridDim.y) {
        const long long p0 = ch * WCH;
        __syncthreads();
        // 16-byte coalesced loads (8 channels of one pixel), scattered into
        // the transposed [channel][pixel] tiles
        constexpr int C8 = (16 + CIN) / 8;  // 8-channel groups per pixel: 2 of dOut, CIN/8 of input
        for (int e = tid; e < WCH * C8; e += WT) {
            const int grp = e % C8, px = e / C8;
            const long long p = p0 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (p < P) {
                if (grp < 2) {
                    v = *reinterpret_cast<const uint4*>(dout + p * COUT + cot * 16 + grp * 8);
                } else {
                    const int n = (int)(p / ((long long)H * W));
                    const int rem = (int)(p % ((long long)H * W));
                    int yy = rem / W + dy, xx = rem % W + dx;
                    yy = (yy % H + H) % H;
                    xx = (xx % W + W) % W;
                    v = *reinterpret_cast<const uint4*>(in + (((size_t)n * H + yy) * W + xx) * CIN + (grp - 2) * 8);
                    if (in_relu) {
                        __nv_bfloat16* hh = reinterpret_cast<__nv_bfloat16*>(&v);
#pragma unroll
                        for (int j = 0; j < 8; ++j) hh[j] = relu_bf(hh[j]);
                    }
                }
            }
            const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v);
            __nv_bfloat16* dst = grp < 2 ? s_d + (grp * 8) * PP + px : s_x + ((grp - 2) * 8) * PP + px;
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j * PP] = hv[j];
        }
        __syncthreads();
        // warp w: pixels [16 w, 16 w + 16) as the k16 step; A = dOut^T (co x p), B = in (p x ci)
        const int k0 = warp * 16;
        const __nv_bfloat16* a = s_d + k0 + 2 * t;
        const uint32_t a0 = ld32(a + g * PP), a1 = ld32(a + (g + 8) * PP);
        const uint32_t a2 = ld32(a + g * PP + 8), a3 = ld32(a + (g + 8) * PP + 8);
#pragma unroll
        for (int j = 0; j < NT8; ++j) {
            const __nv_bfloat16* b = s_x + (j * 8 + g) * PP + k0 + 2 * t;
            mma_bf16(acc[j][0], acc[j][1], acc[j][2], acc[j][3], a0, a1, a2, a3, ld32(b), ld32(b + 8));
        }
    }
    // reduce the 8 warps' partial sums, then one atomic per element
    __syncthreads();  // last chunk's tile reads done before the buffer is reused
#pragma unroll
    for (int j = 0; j < NT8; ++j) {
        s_red[warp][g][j * 8 + 2 * t] = acc[j][0];
        s_red[warp][g][j * 8 + 2 * t + 1] = acc[j][1];
        s_red[warp][g + 8][j * 8 + 2 * t] = acc[j][2];
        s_red[warp][g + 8][j * 8 + 2 * t + 1] = acc[j][3];
    }
    __syncthreads();
    for (int e = tid; e < 16 * CIN; e += WT) {
        const int co = e / CIN, ci = e % CIN;
        float s = 0.f;
#pragma unroll
        for (int w8 = 0; w8 < 8; ++w8) s += s_red[w8][co][ci];
        atomicAdd(&dw[((size_t)tap * COUT + cot * 16 + co) * CIN + ci], s);
    }
}

__global__ void k_bgrad(const __nv_bfloat16* __restrict__ dout, long long P, int C, float* __restrict__ db) {
    __shared__ float s[256];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (long long p = blockIdx.y * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.y * blockDim.x)
        acc += __bfloat162float(dout[p * C + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&db[c], s[0]);
}

// loss = mean over P pixels and 4 channels of (out - target)^2; dout = d loss / d out.
// With the mass-conserving output layer (csum not null) the density gradient
// is projected: minus its per-image mean, which equals
// 2 (mean(x_rho) - mean(target_rho)) / (4 P); csum[n] = sum over image n of
// (x_rho - target_rho), HW pixels per image.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, long long P,
                      __nv_bfloat16* __restrict__ dout, double* __restrict__ loss, const double* __restrict__ csum,
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
    if (threadIdx.x == 0) atomicAdd(loss, s[0] / (double)(P * 4));
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
__global__ void k_mass_stats(const float* __restrict__ y, const float* __restrict__ x, const float* __restrict__ t,
                             int N, long long HW, double* __restrict__ sums) {
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
        atomicAdd(&sums[n], s[0][0]);
        if (t) atomicAdd(&sums[N + n], s[1][0]);
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
                    cudaStream_t s, int sms) {
    const long long P = (long long)N * H * W;
    long long chunks = (P + WCH - 1) / WCH;
    const int gx = 9 * (COUT / 16);
    long long gy = (2 * sms + gx - 1) / gx * 4;
    if (gy > chunks) gy = chunks;
    if (gy < 1) gy = 1;
    k_wgrad<CIN, COUT><<<dim3(gx, (unsigned)gy), WT, 0, s>>>(in, dout, N, H, W, in_relu, dw);
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

cudaError_t launch_mass_layer(float* y, const float* x, const float* t, int N, long long HW, double* sums,
                              cudaStream_t s) {
    if (N < 1 || HW < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * (size_t)N * sizeof(double), s);
    if (e != cudaSuccess) return e;
    long long gx = (HW + 255) / 256;
    if (gx > 256) gx = 256;
    k_mass_stats<<<dim3((unsigned)gx, (unsigned)N), 256, 0, s>>>(y, x, t, N, HW, sums);
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

cudaError_t launch_wgrad(int cin, int cout, const __nv_bfloat16* in, const __nv_bfloat16* dout, int N, int H, int W,
                         int in_relu, float* dw, cudaStream_t s, int sms) {
    if (cin == 16 && cout == 64) return wgrad_t<16, 64>(in, dout, N, H, W, in_relu, dw, s, sms);
    if (cin == 64 && cout == 64) return wgrad_t<64, 64>(in, dout, N, H, W, in_relu, dw, s, sms);
    if (cin == 64 && cout == 16) return wgrad_t<64, 16>(in, dout, N, H, W, in_relu, dw, s, sms);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bgrad(const __nv_bfloat16* dout, long long P, int C, float* db, cudaStream_t s) {
    long long gy = (P + 255) / 256;
    if (gy > 64) gy = 64;
    k_bgrad<<<dim3(C, (unsigned)gy), 256, 0, s>>>(dout, P, C, db);
    return cudaGetLastError();
}

cudaError_t launch_mse(const float* out, const float* target, long long P, __nv_bfloat16* dout, double* loss,
                       const double* csum, long long HW, cudaStream_t s) {
    if (csum && HW < 1) return cudaErrorInvalidValue;
    long long g = (P + 255) / 256;
    if (g > 1024) g = 1024;
    k_mse<<<(unsigned)g, 256, 0, s>>>(out, target, P, dout, loss, csum, HW);
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
