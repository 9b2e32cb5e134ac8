// Conservation record of a caller-owned population state, computed without
// allocating any memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// framework owns the device memory pool, code that must not allocate on a
// latency-critical path, or code that runs where an allocation would break
// a memory budget. This file serves them with one variant of the
// conservation reduction (the density-field pass followed by the moments
// pass with a last-block FP64 reduction) whose scratch memory -- the
// density field, the per-block partial sums and the completion counter --
// lives in one file-scope device array of fixed size instead of in buffers
// a handle allocates. Every GPU that loads the library holds this array
// (about 8.3 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm_device.cuh"

namespace lbm {

namespace {

constexpr long long NA_MAX_NODES = 1ll << 20;  // largest lattice (nx * ny) served
constexpr int NA_NT = 256;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr size_t NA_RHO_BYTES = NA_MAX_NODES * sizeof(double);
constexpr size_t NA_PART_BYTES = (size_t)NA_MAX_BLOCKS * NQ * sizeof(double);
constexpr size_t NA_BYTES = NA_RHO_BYTES + NA_PART_BYTES + 256;  // + completion counter

// The scratch. In host code this name is only a stand-in for the device
// symbol: its address must come from cudaGetSymbolAddress on each device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};

__device__ __forceinline__ int na_ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ int na_ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

__device__ __forceinline__ long long na_wrap(const Geometry& G, int x, int y) {
    x = x < 0 ? x + G.nx : (x >= G.nx ? x - G.nx : x);
    if (G.walls) y = y < 0 ? 0 : (y >= G.ny ? G.ny - 1 : y);
    else y = y < 0 ? y + G.ny : (y >= G.ny ? y - G.ny : y);
    return (long long)y * G.nx + x;
}

// rho = sum_i f_i (Eq. 14) of caller populations [9][ny][nx] into the scratch
__global__ void k_na_rho(const Launch L, const double* __restrict__ f, double* __restrict__ rho) {
    const long long n = (long long)L.geo.nx * L.geo.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) r += f[i * n + idx];
        rho[idx] = r;
    }
}

// Moments (Eq. 13, 14) and the FP64 record, reduced deterministically:
// per-block partials in the scratch, the last block to finish sums them in
// block order into out[0..6] and resets the counter.
__global__ void __launch_bounds__(NA_NT) k_na_record(const Launch L, const double* __restrict__ f,
                                                     const double* __restrict__ g,
                                                     const double* __restrict__ rho_f,
                                                     double* __restrict__ partials, unsigned* __restrict__ counter,
                                                     double* __restrict__ out) {
    const Geometry& G = L.geo;
    const KC<double>& k = L.kd;
    const long long n = (long long)G.nx * G.ny;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % G.nx), y = (int)(idx / G.nx);
        double fl[9], gl[9], rn[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fl[i] = f[i * n + idx];
            gl[i] = g[i * n + idx];
            // beyond an open side the pair force sees the open sides' density
            rn[i] = (G.open && beyond_open(G, x + na_ex(i), y + na_ey(i)))
                        ? k.rho_open
                        : rho_f[na_wrap(G, x + na_ex(i), y + na_ey(i))];
        }
        NodeMacro<double> s;
        node_macro(k, fl, gl, rn, s);
        const double lap = 2.0 * (((rn[1] + rn[2]) + (rn[3] + rn[4])) / 3.0 +
                                  ((rn[5] + rn[6]) + (rn[7] + rn[8])) / 12.0 - (5.0 / 3.0) * s.rho);
        acc[0] += s.rho;
        acc[1] += s.rho * s.uhx * k.c;
        acc[2] += s.rho * s.uhy * k.c;
        acc[3] += s.rek;
        acc[4] += s.rek - k.a * s.rho * s.rho - k.half_kappa * s.rho * lap;
        acc[5] = fmax(acc[5], k.c2 * (s.uhx * s.uhx + s.uhy * s.uhy));
        // as the step kernel counts them: density, temperature, velocity (NaN included)
        if (!(s.rho > 0.0 && s.rho < 1e30 && s.T > 0.0 && s.T < 1e30 && s.uhx * s.uhx + s.uhy * s.uhy < 1e30))
            acc[6] += 1.0;
    }
    __shared__ double red[NA_NT / 32][7];
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
        for (int w = 0; w < NA_NT / 32; ++w)
            for (int q = 0; q < 7; ++q) t[q] = (q == 5) ? fmax(t[q], red[w][q]) : t[q] + red[w][q];
        for (int q = 0; q < 7; ++q) partials[(size_t)blockIdx.x * NQ + q] = t[q];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid == 0) {
        double t[7] = {0, 0, 0, 0, 0, 0, 0};
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const volatile double* pp = partials + (size_t)b * NQ;
            for (int q = 0; q < 7; ++q) t[q] = (q == 5) ? fmax(t[q], pp[q]) : t[q] + pp[q];
        }
        for (int q = 0; q < 7; ++q) out[q] = (q == 5) ? sqrt(t[q]) : t[q];
        *counter = 0u;
    }
}

}  // namespace

long long noalloc_max_nodes() { return NA_MAX_NODES; }

// Launch the record on the calling thread's current device. The first call
// on each device looks up the scratch symbol's device address there
// (cudaGetSymbolAddress) and keeps it; that first call should therefore be
// made before any stream capture begins.
cudaError_t launch_record_noalloc(const Launch& L, const double* f, const double* g, double* out, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    double* rho = reinterpret_cast<double*>(b);
    double* partials = reinterpret_cast<double*>(b + NA_RHO_BYTES);
    unsigned* counter = reinterpret_cast<unsigned*>(b + NA_RHO_BYTES + NA_PART_BYTES);
    // the array keeps the previous call's contents: the counter must start at 0
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)L.geo.nx * L.geo.ny;
    long long blocks = (n + NA_NT - 1) / NA_NT;
    if (blocks > NA_MAX_BLOCKS) blocks = NA_MAX_BLOCKS;
    k_na_rho<<<(int)blocks, NA_NT, 0, s>>>(L, f, rho);
    k_na_record<<<(int)blocks, NA_NT, 0, s>>>(L, f, g, rho, partials, counter, out);
    return cudaGetLastError();
}

}  // namespace lbm
