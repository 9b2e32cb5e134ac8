// Kernels around the time step: initial populations from macroscopic fields,
// population import/export, and the macroscopic fields / conservation record
// of the current state. They compute in FP64 and convert to the storage type
// at the end; k_init, k_rho and k_moments also come in an FP32 form for
// 32- and 16-bit storage (per-node arithmetic in FP32, sums in FP64), which
// the surrogate rollout uses. None is on the per-step path.
//
// Addressing: the stored state holds post-collision populations; the
// post-streaming population l_i(x) sits at x - e_i (pull streaming,
// Eq. 12a). Ghost columns and rows always hold valid copies (or, next to a
// wall, the reflected value), so a read at x - e_i needs no wrap.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

namespace {

constexpr int AUX_NT = 256;

template <class S>
__device__ __forceinline__ double load_d(const S* buf, const Geometry& G, int p, int x, int y, double rest) {
    const S v = buf[(long long)p * G.plane + (long long)(y + 2) * G.pitch + G.PX + x];
    if constexpr (sizeof(S) == 2) return rest + (double)Store<S, float>::ld(v, 0.0f);
    else return (double)v;
}

template <class S>
__device__ __forceinline__ S to_store(double v, double rest) {
    if constexpr (sizeof(S) == 2) return Store<S, float>::st((float)(v - rest), 0.0f);
    else return (S)v;
}

// load_d / to_store in the compute type C (identical to them for C = double)
template <class S, class C>
__device__ __forceinline__ C load_c(const S* buf, const Geometry& G, int p, int x, int y, C rest) {
    const S v = buf[(long long)p * G.plane + (long long)(y + 2) * G.pitch + G.PX + x];
    if constexpr (sizeof(S) == 2) return rest + (C)Store<S, float>::ld(v, 0.0f);
    else return (C)v;
}
template <class S, class C>
__device__ __forceinline__ S to_store_c(C v, C rest) {
    if constexpr (sizeof(S) == 2) return Store<S, float>::st((float)(v - rest), 0.0f);
    else return (S)v;
}

__device__ __forceinline__ int ex_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ int ey_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Write post-streaming population l_i(x, y) so that the next pull finds it:
// at x - e_i (wrapped in x unless the left and right sides are open; wrapped
// in y when periodic; a ghost row or column at a wall or an open side).
template <class S>
__device__ __forceinline__ void scatter(S* buf, const Geometry& G, int p, int i, int x, int y, S v) {
    int xs = x - ex_of(i), ys = y - ey_of(i);
    if (!(G.open & 12)) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
    if (!G.walls) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
    put<S>(buf, G, p, xs, ys, v);
}

// density at (x, y) as the pair force sees it: the open sides' fixed
// density beyond them, the adjacent fluid node's beyond a wall, periodic
// images elsewhere
__device__ __forceinline__ double rho_nb(const double* rho, const Geometry& G, double rho_open, int x, int y) {
    if (G.open && beyond_open(G, x, y)) return rho_open;
    x = x < 0 ? x + G.nx : (x >= G.nx ? x - G.nx : x);
    if (G.walls) y = y < 0 ? 0 : (y >= G.ny ? G.ny - 1 : y);
    else y = y < 0 ? y + G.ny : (y >= G.ny ? y - G.ny : y);
    return rho[(long long)y * G.nx + x];
}

template <class S, class C>
__global__ void k_init(const Launch L, const double* __restrict__ rho, const double* __restrict__ ux,
                       const double* __restrict__ uy, const double* __restrict__ T, S* __restrict__ buf) {
    const Geometry& G = L.geo;
    const KC<C>& k = kc<C>(L);
    const long long n = (long long)G.nx * G.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
        NodeMacro<C> s;
        C rn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) rn[i] = (C)rho_nb(rho, G, (double)L.kd.rho_open, x + ex_of(i), y + ey_of(i));
        const C r = (C)rho[idx], vx = (C)ux[idx], vy = (C)uy[idx];
        s.rho = r;
        s.inv_rho = C(1) / r;
        s.gx = (rn[1] - rn[3]) / C(3) + ((rn[5] - rn[7]) + (rn[8] - rn[6])) / C(12);
        s.gy = (rn[2] - rn[4]) / C(3) + ((rn[5] - rn[7]) + (rn[6] - rn[8])) / C(12);
        s.Fhx = k.G2c * r * s.gx + r * k.axc;
        s.Fhy = k.G2c * r * s.gy + r * k.ayc;
        s.uhx = vx / k.c;
        s.uhy = vy / k.c;
        s.q = k.c2 * (s.Fhx * s.uhx + s.Fhy * s.uhy);
        s.T = (C)T[idx];
        s.rek = r * k.cv * s.T + C(0.5) * r * (vx * vx + vy * vy);
        C meq[9], Fm[9], neq[9], qm[9], m[9], nn[9], f[9], g[9];
        equilibria(k, s, meq, Fm, neq, qm, L.cubic != 0);
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            m[j] = meq[j] - k.half_dt * Fm[j];
            nn[j] = neq[j] - k.half_dt * qm[j];
        }
        populations9(m, f);
        populations9(nn, g);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            scatter<S>(buf, G, i, i, x, y, to_store_c<S, C>(f[i], (C)L.kf.rest[i]));
            scatter<S>(buf, G, 9 + i, i, x, y, to_store_c<S, C>(g[i], (C)L.kf.rest[9 + i]));
        }
    }
}

template <class S>
__global__ void k_set_pops(const Launch L, const double* __restrict__ f, const double* __restrict__ g,
                           S* __restrict__ buf) {
    const Geometry& G = L.geo;
    const long long n = (long long)G.nx * G.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            scatter<S>(buf, G, i, i, x, y, to_store<S>(f[i * n + idx], (double)L.kf.rest[i]));
            scatter<S>(buf, G, 9 + i, i, x, y, to_store<S>(g[i * n + idx], (double)L.kf.rest[9 + i]));
        }
    }
}

template <class S>
__global__ void k_get_pops(const Launch L, const S* __restrict__ buf, double* __restrict__ f,
                           double* __restrict__ g) {
    const Geometry& G = L.geo;
    const long long n = (long long)G.nx * G.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i * n + idx] = load_d<S>(buf, G, i, x - ex_of(i), y - ey_of(i), (double)L.kf.rest[i]);
            g[i * n + idx] = load_d<S>(buf, G, 9 + i, x - ex_of(i), y - ey_of(i), (double)L.kf.rest[9 + i]);
        }
    }
}

template <class S, class C>
__global__ void k_rho(const Launch L, const S* __restrict__ buf, double* __restrict__ rho) {
    const Geometry& G = L.geo;
    const long long n = (long long)G.nx * G.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
        C r = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) r += load_c<S, C>(buf, G, i, x - ex_of(i), y - ey_of(i), (C)L.kf.rest[i]);
        rho[idx] = (double)r;
    }
}

// rho u_x^3 and rho u_y^3 (u over c) of every node, phi [2][ny][nx], for
// the cubic-term elimination; rho_f: the density field (k_rho). Periodic
// boxes only.
template <class S, class C>
__global__ void k_phi(const Launch L, const S* __restrict__ buf, const double* __restrict__ rho_f,
                      double* __restrict__ phi) {
    const Geometry& G = L.geo;
    const KC<C>& k = kc<C>(L);
    const long long n = (long long)G.nx * G.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
        C f[9], g[9], rn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = load_c<S, C>(buf, G, i, x - ex_of(i), y - ey_of(i), (C)L.kf.rest[i]);
            g[i] = C(0);
            rn[i] = (C)rho_nb(rho_f, G, (double)L.kd.rho_open, x + ex_of(i), y + ey_of(i));
        }
        NodeMacro<C> s;
        node_macro(k, f, g, rn, s);
        phi[idx] = (double)(s.rho * s.uhx * s.uhx * s.uhx);
        phi[n + idx] = (double)(s.rho * s.uhy * s.uhy * s.uhy);
    }
}

// Macroscopic fields (Eq. 13, 14) and, if partials != NULL, the FP64
// conservation record reduced deterministically into stats[0..6].
template <class S, class C>
__global__ void __launch_bounds__(AUX_NT) k_moments(const Launch L, const S* __restrict__ buf,
                                                    const double* __restrict__ rho_f, double* __restrict__ o_rho,
                                                    double* __restrict__ o_ux, double* __restrict__ o_uy,
                                                    double* __restrict__ o_T, double* __restrict__ partials,
                                                    double* __restrict__ stats, unsigned* __restrict__ counter) {
    const Geometry& G = L.geo;
    const KC<C>& k = kc<C>(L);
    const long long n = (long long)G.nx * G.ny;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
        C f[9], g[9], rn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = load_c<S, C>(buf, G, i, x - ex_of(i), y - ey_of(i), (C)L.kf.rest[i]);
            g[i] = load_c<S, C>(buf, G, 9 + i, x - ex_of(i), y - ey_of(i), (C)L.kf.rest[9 + i]);
            rn[i] = (C)rho_nb(rho_f, G, (double)L.kd.rho_open, x + ex_of(i), y + ey_of(i));
        }
        NodeMacro<C> s;
        node_macro(k, f, g, rn, s);
        if (o_rho) o_rho[idx] = (double)s.rho;
        if (o_ux) o_ux[idx] = (double)(s.uhx * k.c);
        if (o_uy) o_uy[idx] = (double)(s.uhy * k.c);
        if (o_T) o_T[idx] = (double)s.T;
        const C lap = C(2) * (((rn[1] + rn[2]) + (rn[3] + rn[4])) / C(3) +
                              ((rn[5] + rn[6]) + (rn[7] + rn[8])) / C(12) - (C(5) / C(3)) * s.rho);
        acc[0] += (double)s.rho;
        acc[1] += (double)(s.rho * s.uhx * k.c);
        acc[2] += (double)(s.rho * s.uhy * k.c);
        acc[3] += (double)s.rek;
        acc[4] += (double)(s.rek - k.a * s.rho * s.rho - k.half_kappa * s.rho * lap);
        acc[5] = fmax(acc[5], (double)(k.c2 * (s.uhx * s.uhx + s.uhy * s.uhy)));
        // as the step kernel counts them: density, temperature, velocity (NaN included)
        if (!(s.rho > C(0) && s.rho < C(1e30) && s.T > C(0) && s.T < C(1e30) &&
              s.uhx * s.uhx + s.uhy * s.uhy < C(1e30)))
            acc[6] += 1.0;
    }
    if (!partials) return;
    __shared__ double red[AUX_NT / 32][7];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, acc[q], o);
            acc[q] = (q == 5) ? fmax(acc[q], w) : acc[q] + w;
        }
    if (lane == 0)
        for (int q = 0; q < 7; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (tid == 0) {
        double t[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < AUX_NT / 32; ++w)
            for (int q = 0; q < 7; ++q) t[q] = (q == 5) ? fmax(t[q], red[w][q]) : t[q] + red[w][q];
        for (int q = 0; q < 7; ++q) partials[(size_t)blockIdx.x * NQ + q] = t[q];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every thread combines the blocks tid, tid + AUX_NT, ... (independent L2
    // loads), then a fixed-order tree over the threads: the same record on
    // every run
    double t[7] = {0, 0, 0, 0, 0, 0, 0};
    for (unsigned b = tid; b < gridDim.x; b += AUX_NT)
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const double pv = __ldcg(partials + (size_t)b * NQ + q);
            t[q] = (q == 5) ? fmax(t[q], pv) : t[q] + pv;
        }
#pragma unroll
    for (int q = 0; q < 7; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, t[q], o);
            t[q] = (q == 5) ? fmax(t[q], w) : t[q] + w;
        }
    __syncthreads();  // red[] of the block pass is no longer needed
    if (lane == 0)
        for (int q = 0; q < 7; ++q) red[warp][q] = t[q];
    __syncthreads();
    if (tid == 0) {
        double u[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < AUX_NT / 32; ++w)
            for (int q = 0; q < 7; ++q) u[q] = (q == 5) ? fmax(u[q], red[w][q]) : u[q] + red[w][q];
        for (int q = 0; q < 7; ++q) stats[q] = (q == 5) ? sqrt(u[q]) : u[q];
        *counter = 0u;
    }
}

int aux_blocks(const Geometry& g) {
    const long long n = (long long)g.nx * g.ny;
    long long b = (n + AUX_NT - 1) / AUX_NT;
    return (int)(b < 4096 ? b : 4096);
}

template <class S>
struct AuxT {
    // fast: FP32 per-node arithmetic (32- and 16-bit storage only)
    static cudaError_t init(const Launch& L, const double* rho, const double* ux, const double* uy, const double* T,
                            void* buf, cudaStream_t s, bool fast) {
        if constexpr (sizeof(S) < 8) {
            if (fast) {
                k_init<S, float><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, rho, ux, uy, T, static_cast<S*>(buf));
                return cudaGetLastError();
            }
        }
        k_init<S, double><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, rho, ux, uy, T, static_cast<S*>(buf));
        return cudaGetLastError();
    }
    // in the step's compute type: FP64 for FP64 storage, FP32 otherwise
    static cudaError_t phi(const Launch& L, const void* buf, double* rho_scratch, double* out, cudaStream_t s) {
        using C = typename std::conditional<sizeof(S) == 8, double, float>::type;
        k_rho<S, C><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch);
        k_phi<S, C><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch, out);
        return cudaGetLastError();
    }
    static cudaError_t set(const Launch& L, const double* f, const double* g, void* buf, cudaStream_t s) {
        k_set_pops<S><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, f, g, static_cast<S*>(buf));
        return cudaGetLastError();
    }
    static cudaError_t get(const Launch& L, const void* buf, double* f, double* g, cudaStream_t s) {
        k_get_pops<S><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), f, g);
        return cudaGetLastError();
    }
    static cudaError_t moments(const Launch& L, const void* buf, double* rho_scratch, double* rho, double* ux,
                               double* uy, double* T, double* partials, double* stats, unsigned* counter,
                               cudaStream_t s, bool fast) {
        if constexpr (sizeof(S) < 8) {
            if (fast) {
                k_rho<S, float><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch);
                k_moments<S, float><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch,
                                                                        rho, ux, uy, T, partials, stats, counter);
                return cudaGetLastError();
            }
        }
        k_rho<S, double><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch);
        k_moments<S, double><<<aux_blocks(L.geo), AUX_NT, 0, s>>>(L, static_cast<const S*>(buf), rho_scratch, rho, ux,
                                                                 uy, T, partials, stats, counter);
        return cudaGetLastError();
    }
};

}  // namespace

int moments_blocks(const Geometry& g) { return aux_blocks(g); }

#define LBM_DISPATCH(storage, call)                                  \
    switch (storage) {                                               \
        case S_F64: return AuxT<double>::call;                       \
        case S_F32: return AuxT<float>::call;                        \
        case S_F16: return AuxT<__half>::call;                       \
        case S_BF16: return AuxT<__nv_bfloat16>::call;               \
    }                                                                \
    return cudaErrorInvalidValue;

cudaError_t launch_init(int storage, const Launch& L, const double* rho, const double* ux, const double* uy,
                        const double* T, void* buf, cudaStream_t s, bool fast) {
    LBM_DISPATCH(storage, init(L, rho, ux, uy, T, buf, s, fast))
}
cudaError_t launch_cubic_phi(int storage, const Launch& L, const void* buf, double* rho_scratch, double* phi,
                             cudaStream_t s) {
    LBM_DISPATCH(storage, phi(L, buf, rho_scratch, phi, s))
}
cudaError_t launch_set_pops(int storage, const Launch& L, const double* f, const double* g, void* buf,
                            cudaStream_t s) {
    LBM_DISPATCH(storage, set(L, f, g, buf, s))
}
cudaError_t launch_get_pops(int storage, const Launch& L, const void* buf, double* f, double* g, cudaStream_t s) {
    LBM_DISPATCH(storage, get(L, buf, f, g, s))
}
cudaError_t launch_moments(int storage, const Launch& L, const void* buf, double* rho_scratch, double* rho,
                           double* ux, double* uy, double* T, double* partials, double* stats, unsigned* counter,
                           cudaStream_t s, bool fast) {
    LBM_DISPATCH(storage, moments(L, buf, rho_scratch, rho, ux, uy, T, partials, stats, counter, s, fast))
}

}  // namespace lbm
