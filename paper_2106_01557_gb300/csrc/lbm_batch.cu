// Batched time step: many independent cases of different size and
// temperature advance together, one persistent launch per time step.
//
// The work list holds (case, tile) items in an order the autotuner picks;
// one CTA per SM walks the list with the same two-stage TMA pipeline as the
// single-case step (per-case tensor maps live in a device table). Each
// case's constants (temperature-dependent c, dt, c_s, G^2/c, rho_v/rho_l,
// C_ref, shift) sit in a device table too; the constants of the next item are
// copied into shared memory one item ahead, so the compute of an item reads
// them from shared memory and a tile still needs one block barrier.
// Per-item FP32 partial sums of the conservation record are written to a
// table from which per-case records are reduced on demand.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_batch.h"
#include "lbm_device.cuh"
#include "lbm_ptx.cuh"

namespace lbm {

namespace {

__host__ __device__ constexpr int bex(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int bey(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }

template <class S, int BX_, int BY_, int NT_>
struct BTile {
    static constexpr int BX = BX_, BY = BY_, NT = NT_;
    static constexpr int HX = 16 / (int)sizeof(S);
    static constexpr int WX = BX + 2 * HX;
    static constexpr int FR = BY + 4, GR = BY + 2;
    static constexpr int F_BYTES = 9 * FR * WX * (int)sizeof(S);
    static constexpr int G_BYTES = 9 * GR * WX * (int)sizeof(S);
    static constexpr int G_OFF = ((F_BYTES + 127) / 128) * 128;
    static constexpr int STAGE = G_OFF + ((G_BYTES + 127) / 128) * 128;
    static constexpr int RX = BX + 2, RY = BY + 2;
    static constexpr int R_BYTES = ((4 * RX * RY + 127) / 128) * 128;
    static constexpr int K_BYTES = ((int)((sizeof(KC<float>) + 127) / 128)) * 128;
    static constexpr int C_BYTES = ((int)((sizeof(BatchCase) + 127) / 128)) * 128;
    static constexpr int R_OFF = 2 * STAGE;
    static constexpr int K_OFF = R_OFF + 2 * R_BYTES;
    static constexpr int C_OFF = K_OFF + 2 * K_BYTES;
    static constexpr int BYTES = C_OFF + 2 * C_BYTES + 128;
    static_assert(NT % BX == 0, "whole tile rows per thread sweep");
};

template <class S, class T>
__global__ void __launch_bounds__(T::NT, 1)
    k_batch_step(const BatchItem* __restrict__ items, int nitems, const BatchCase* __restrict__ cases,
                 const KC<float>* __restrict__ kcs, const CUtensorMap* __restrict__ maps, int from,
                 S* __restrict__ arena_out, float* __restrict__ partials, int* __restrict__ status,
                 double* __restrict__ steps, unsigned* __restrict__ done, int rounding,
                 unsigned long long tile_wait_ns) {
    using C = float;
    constexpr int BX = T::BX, BY = T::BY, HX = T::HX, WX = T::WX, NT = T::NT;
    constexpr int FR = T::FR, GR = T::GR, RX = T::RX, RY = T::RY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[2][NT / 32][8];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int tid = threadIdx.x;

    auto item_of = [&](int it) { return (int)blockIdx.x + it * (int)gridDim.x; };
    auto issue = [&](int item, int stage) {
        const BatchItem w = items[item];
        const BatchCase& cs = cases[w.c];
        const int tx0 = (w.tile % cs.ntx) * BX, ty0 = (w.tile / cs.ntx) * BY;
        const CUtensorMap* mf = maps + ((size_t)w.c * 2 + from) * 2;
        unsigned char* st = smem + stage * T::STAGE;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(T::F_BYTES + T::G_BYTES));
        tma_load_3d(st, mf, tx0, ty0, 0, &bar[stage]);
        tma_load_3d(st + T::G_OFF, mf + 1, tx0, ty0 + 1, 9, &bar[stage]);
    };
    // copy the constants and geometry of `item` into shared slot `slot`
    auto stage_consts = [&](int item, int slot) {
        const int c = items[item].c;
        const uint32_t* ks = reinterpret_cast<const uint32_t*>(kcs + c);
        uint32_t* kd = reinterpret_cast<uint32_t*>(smem + T::K_OFF + slot * T::K_BYTES);
        for (int j = tid; j < (int)(sizeof(KC<float>) / 4); j += NT) kd[j] = ks[j];
        const uint32_t* cs = reinterpret_cast<const uint32_t*>(cases + c);
        uint32_t* cd = reinterpret_cast<uint32_t*>(smem + T::C_OFF + slot * T::C_BYTES);
        for (int j = tid; j < (int)(sizeof(BatchCase) / 4); j += NT) cd[j] = cs[j];
    };
    auto flush = [&](int item, int slot) {
        if (tid < 8) {
            float t = 0.f;
            for (int w = 0; w < NT / 32; ++w) t = (tid == 5) ? fmaxf(t, red[slot][w][tid]) : t + red[slot][w][tid];
            partials[(size_t)item * 8 + tid] = t;
        }
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (item_of(0) < nitems) stage_consts(item_of(0), 0);
    if (item_of(1) < nitems) stage_consts(item_of(1), 1);
    __syncthreads();
    if (tid == 0) {
        if (item_of(0) < nitems) issue(item_of(0), 0);
        if (item_of(1) < nitems) issue(item_of(1), 1);
    }

    // stochastic rounding of 16-bit storage, keyed as for a single case by
    // (node, step): the batch's step count is kept on the device by the last
    // block of each launch
    const bool sr = Store<S, C>::SHIFTED && rounding;
    const uint32_t step_key = sr ? fmix32((uint32_t)(long long)__ldcg(steps) * 0x9e3779b9u + 0x7f4a7c15u) : 0u;
    bool ok = true;
    int it = 0;
    for (; item_of(it) < nitems; ++it) {
        const int item = item_of(it);
        const int stage = it & 1;
        bool timed_out = false;
        {
            const uint32_t parity = (it >> 1) & 1;
            if (tile_wait_ns == 0) {
                timed_out = !mbar_test_wait(&bar[stage], parity);  // no waiting at all
            } else {
                const uint64_t t0 = globaltimer_ns();
                while (!mbar_try_wait(&bar[stage], parity)) {
                    if (globaltimer_ns() - t0 > tile_wait_ns) { timed_out = true; break; }
                }
            }
        }
        const S* sf = reinterpret_cast<const S*>(smem + stage * T::STAGE);
        const S* sg = reinterpret_cast<const S*>(smem + stage * T::STAGE + T::G_OFF);
        float* srho = reinterpret_cast<float*>(smem + T::R_OFF + stage * T::R_BYTES);
        // the density pass reads the item's geometry from the global tables
        // (its shared copy is only guaranteed visible after the barrier)
        const BatchItem w = items[item];
        const int c_ntx = cases[w.c].ntx;
        const float rest_sum = cases[w.c].rest_sum;
        const int tx0 = (w.tile % c_ntx) * BX, ty0 = (w.tile / c_ntx) * BY;
#pragma unroll 1
        for (int idx = tid; idx < RX * RY; idx += NT) {
            const int rx = idx % RX, ry = idx / RX;
            const S* p = sf + (ry + 1) * WX + rx - 1 + HX;
            float r = rest_sum;
#pragma unroll
            for (int i = 0; i < 9; ++i) r += Store<S, C>::ld(p[i * FR * WX - bey(i) * WX - bex(i)], 0.f);
            srho[idx] = r;
        }
        if (__syncthreads_or(timed_out)) { ok = false; break; }
        {
            const int ahead = item_of(it + 1);
            if (it > 0 && ahead < nitems) {
                if (tid == 0) issue(ahead, stage ^ 1);
                stage_consts(ahead, stage ^ 1);
            }
            if (it > 0) flush(item_of(it - 1), stage ^ 1);
        }
        const KC<float>& k = *reinterpret_cast<const KC<float>*>(smem + T::K_OFF + stage * T::K_BYTES);
        const BatchCase& cs = *reinterpret_cast<const BatchCase*>(smem + T::C_OFF + stage * T::C_BYTES);
        const Geometry& G = cs.geo;
        S* out = arena_out + cs.off;
        float a_mass = 0.f, a_mx = 0.f, a_my = 0.f, a_ek = 0.f, a_et = 0.f, a_u2 = 0.f, a_bad = 0.f;

        const int lx = tid % BX;
        const int x = tx0 + lx;
#pragma unroll 1
        for (int ly = tid / BX; ly < BY; ly += NT / BX) {
            const int y = ty0 + ly;
            if (x >= G.nx || y >= G.ny) continue;
            float f[9], g[9], rn[9];
            const S* pf = sf + (ly + 2) * WX + lx + HX;
            const S* pg = sg + (ly + 1) * WX + lx + HX;
            const float* pr = srho + (ly + 1) * RX + lx + 1;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = Store<S, C>::raw(pf[i * FR * WX - bey(i) * WX - bex(i)]);
                g[i] = Store<S, C>::raw(pg[i * GR * WX - bey(i) * WX - bex(i)]);
                rn[i] = pr[bey(i) * RX + bex(i)];
            }
            NodeMacro<float> s;
            node_macro<Store<S, C>::SHIFTED>(k, f, g, rn, s);
            {
                const float rho = s.rho;
                a_mass += rho;
                a_mx += rho * s.uhx;
                a_my += rho * s.uhy;
                a_ek += s.rek;
                const float lap = 2.f * ((1.f / 3.f) * ((rn[1] + rn[2]) + (rn[3] + rn[4])) +
                                         (1.f / 12.f) * ((rn[5] + rn[6]) + (rn[7] + rn[8])) - (5.f / 3.f) * rho);
                a_et += s.rek - k.a * rho * rho - k.half_kappa * rho * lap;
                const float u2 = s.uhx * s.uhx + s.uhy * s.uhy;
                a_u2 = fmaxf(a_u2, u2);
                // as for a single case: density, temperature, velocity (NaN included)
                if (!(rho > 0.f && rho < 1e30f && s.T > 0.f && s.T < 1e30f && u2 < 1e30f)) a_bad += 1.f;
            }
            // shifted formats: f and g leave the collision as deviations from the rest populations
            collide<Store<S, C>::SHIFTED>(k, f, g, s);
            S sf[9], sg[9];
            if (sr) {
                cvt_sr_node<S, C>(f, g, fmix32((uint32_t)(y * G.nx + x) ^ step_key), sf, sg);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    sf[i] = Store<S, C>::cvt(f[i]);
                    sg[i] = Store<S, C>::cvt(g[i]);
                }
            }
            const bool interior = x >= GHOST_COLS && x < G.nx - GHOST_COLS && y >= 2 && y < G.ny - 2;
            if (interior) {
                S* o = out + (long long)(y + 2) * G.pitch + G.PX + x;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    o[i * G.plane] = sf[i];
                    o[(9 + i) * G.plane] = sg[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    put<S>(out, G, i, x, y, sf[i]);
                    put<S>(out, G, 9 + i, x, y, sg[i]);
                }
            }
        }
        // per-item partial sums: warp shuffles, then one slot per warp
        float v[8] = {a_mass, a_mx * k.c, a_my * k.c, a_ek, a_et, a_u2 * k.c2, a_bad, 0.f};
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float wv = __shfl_down_sync(0xffffffffu, v[q], o);
                v[q] = (q == 5) ? fmaxf(v[q], wv) : v[q] + wv;
            }
        if (tid % 32 == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) red[stage][tid / 32][q] = v[q];
            if (v[6] > 0.f) atomicOr(status, ST_NONFINITE);
        }
    }
    __syncthreads();
    if (ok && it > 0) flush(item_of(it - 1), (it - 1) & 1);
    if (!ok && tid == 0) {
        atomicOr(status, ST_TIMEOUT);
        // the copies issued and not yet consumed: items it and, at it = 0, 1
        // (item it + 1 is issued only after iteration it's barrier); each
        // drained within the full default bound
        const int jend = it == 0 ? 1 : it;
        for (int j = it; j <= jend; ++j) {
            if (item_of(j) >= nitems) break;
            const uint64_t t0 = globaltimer_ns();
            while (!mbar_try_wait(&bar[j & 1], (j >> 1) & 1) && globaltimer_ns() - t0 < WAIT_NS) {}
        }
    }
    // the last block to finish counts the step (every block read the count
    // at its start, before any block could reach this point)
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == gridDim.x - 1) {
            *steps = *steps + 1.0;
            *done = 0u;
        }
    }
}

// Per-case conservation record from the per-item partials, FP64, items in
// list order (deterministic).
__global__ void k_batch_case_record(const BatchItem* __restrict__ items, int nitems, int c,
                                    const float* __restrict__ partials, double* __restrict__ out) {
    __shared__ double red[8][256];
    double t[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
        if (items[i].c != c) continue;
        for (int q = 0; q < 7; ++q) {
            const double v = (double)partials[(size_t)i * 8 + q];
            t[q] = (q == 5) ? fmax(t[q], v) : t[q] + v;
        }
    }
    for (int q = 0; q < 7; ++q) red[q][threadIdx.x] = t[q];
    __syncthreads();
    if (threadIdx.x < 7) {
        const int q = threadIdx.x;
        double s = 0.0;
        for (int j = 0; j < (int)blockDim.x; ++j) s = (q == 5) ? fmax(s, red[q][j]) : s + red[q][j];
        out[q] = (q == 5) ? sqrt(s) : s;
    }
}

using T16a = BTile<__half, 64, 32, 512>;
using T16b = BTile<__half, 32, 16, 256>;
using Tb16a = BTile<__nv_bfloat16, 64, 32, 512>;
using Tb16b = BTile<__nv_bfloat16, 32, 16, 256>;
using T32a = BTile<float, 64, 16, 512>;
using T32b = BTile<float, 32, 16, 256>;

template <class S, class T>
cudaError_t launch_bt(const BatchLaunch& B, int from, void* out, cudaStream_t s) {
    const int grid = B.nitems < B.sms ? B.nitems : B.sms;
    k_batch_step<S, T><<<grid, T::NT, T::BYTES, s>>>(B.items, B.nitems, B.cases, B.kcs, B.maps, from,
                                                     static_cast<S*>(out), B.partials, B.status, B.steps,
                                                     B.done, B.rounding, B.tile_wait_ns);
    return cudaGetLastError();
}

template <class S, class T>
cudaError_t attr_bt() {
    return cudaFuncSetAttribute(k_batch_step<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::BYTES);
}

}  // namespace

void batch_tile(int storage, int variant, int* bx, int* by) {
    const bool a = variant == 0;
    if (storage == S_F32) { *bx = a ? T32a::BX : T32b::BX; *by = a ? T32a::BY : T32b::BY; }
    else { *bx = a ? T16a::BX : T16b::BX; *by = a ? T16a::BY : T16b::BY; }
}

cudaError_t batch_prepare(int storage) {
    cudaError_t e = cudaSuccess;
    switch (storage) {
        case S_F16: if ((e = attr_bt<__half, T16a>())) return e; return attr_bt<__half, T16b>();
        case S_BF16: if ((e = attr_bt<__nv_bfloat16, Tb16a>())) return e; return attr_bt<__nv_bfloat16, Tb16b>();
        case S_F32: if ((e = attr_bt<float, T32a>())) return e; return attr_bt<float, T32b>();
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_step(int storage, int variant, const BatchLaunch& B, int from, void* out,
                              cudaStream_t s) {
    const bool a = variant == 0;
    switch (storage) {
        case S_F16: return a ? launch_bt<__half, T16a>(B, from, out, s) : launch_bt<__half, T16b>(B, from, out, s);
        case S_BF16:
            return a ? launch_bt<__nv_bfloat16, Tb16a>(B, from, out, s) : launch_bt<__nv_bfloat16, Tb16b>(B, from, out, s);
        case S_F32: return a ? launch_bt<float, T32a>(B, from, out, s) : launch_bt<float, T32b>(B, from, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_case_record(const BatchLaunch& B, int c, double* out, cudaStream_t s) {
    k_batch_case_record<<<1, 256, 0, s>>>(B.items, B.nitems, c, B.partials, out);
    return cudaGetLastError();
}

}  // namespace lbm
