// Internal declarations shared by the host runtime and the kernels of liblbm.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Device status word bits (set by kernels, read and cleared by the host).
enum : int { ST_TIMEOUT = 1, ST_NONFINITE = 2 };

// Number of FP64 quantities in one conservation record.
constexpr int NQ = 8;

// Physical and model scalars in the kernel's compute type. Everything the
// collision needs is precomputed here so that a node update does no
// parameter arithmetic.
template <class C>
struct KC {
    C c, c2, dt, half_dt;
    C G2c;           // G^2 / c   (F^ = F / c)
    C axc, ayc;      // a / c
    C a, half_kappa; // Eq. 16 a and kappa / 2 (total-energy diagnostic)
    C cs2_inv;       // 1 / c_s^2
    C RK, aK_eff, b4;   // p_BE = RK rho T Z(b4 rho) + aK_eff rho^2
    C inv_cv, cv, Cref;
    C g1, g2, beta, kS, hS, bS;
    C se, seps, sq, sp, sige, sigeps, sigp;
    C tauj_v, dtauj, rho_v, inv_drho;
    C qc;            // G^2 dt^2 / 12 of SM Eq. S6a (dx = 1)
    // products of the constants above, formed once on the host
    C we_kS_seps;    // (s_e/2 - 1) k s_eps
    C we_hS;         // (s_e/2 - 1) h
    C wp_bS;         // (s_p/2 - 1) b
    C six_qc;        // 6 qc
    C dt_g1, dt_g2, hdt_g1, hdt_g2;  // dt gamma_1, dt gamma_2, dt/2 gamma_1, dt/2 gamma_2
    C c4g1_Cref, c4g2_Cref;          // (4 + gamma_1) C_ref, (4 - gamma_2) C_ref
    C c2_third;      // c^2 / 3
    C T_bottom, T_top, T_hot;
    C rho_open, T_open;  // state of the open sides
    C rest[18];      // shifted-storage rest populations (f 0..8, g 9..17)
    C mrest[3], nrest[3];  // moments 0-2 of the f and g rest populations (the others vanish)
};

// Ghost columns that hold periodic copies: a pull reads one column beyond
// the lattice and the density of the step's one-node ring pulls from a
// second; the other columns of the HX-wide ghost block exist only to keep
// the tile copies 16-byte aligned and are never read.
constexpr int GHOST_COLS = 2;

struct Geometry {
    int nx, ny, walls, HX;  // HX: ghost columns on each side (16 bytes)
    int PX;          // elements before column x = 0 of a row (128 bytes), so
                     // that row stores start on a cache line
    int pitch;       // padded row length in elements (a multiple of 128 bytes)
    int nyp;         // padded number of rows (ny + 4 at least)
    long long plane; // elements per plane
    int hot_x0, hot_len;
    int sms;         // persistent grid size (one CTA per SM)
    int open;        // open sides: 1 bottom, 2 top, 4 left, 8 right (left and right only together with all)
};

// Is lattice point (x, y) beyond an open side? (x is periodic unless the
// left and right sides are open.)
__host__ __device__ __forceinline__ bool beyond_open(const Geometry& G, int x, int y) {
    return ((G.open & 1) && y < 0) || ((G.open & 2) && y >= G.ny) || ((G.open & 4) && x < 0) ||
           ((G.open & 8) && x >= G.nx);
}

struct Launch {
    Geometry geo;
    KC<float> kf;
    KC<double> kd;
    int rounding;  // 16-bit storage: 0 nearest, 1 stochastic
    // bound in ns on each wait of the step kernel for a tile's copies; 0: the
    // copies must already have landed when the tile's turn comes (no waiting)
    unsigned long long tile_wait_ns;
    int cubic;  // eliminate the cubic velocity terms (periodic single cases)
};

// default tile-wait bound: 2 s
constexpr unsigned long long TILE_WAIT_NS_DEFAULT = 2000000000ull;

// Storage kinds
enum { S_F64 = 0, S_F32 = 1, S_F16 = 2, S_BF16 = 3 };

// Host-side launchers (lbm_kernels.cu). All return cudaError_t of the launch.
// phi: with L.cubic, [2][ny][nx] rho u_x^3 and rho u_y^3 (u over c) of the
// state entering the step (launch_cubic_phi); otherwise unused
cudaError_t launch_step(int storage, const Launch& L, const CUtensorMap* tmf, const CUtensorMap* tmg,
                        void* out, double* partials, double* stats, unsigned* counter, int* status,
                        cudaStream_t s, const double* phi = nullptr);
// rho u_x^3 and rho u_y^3 of every node of a state (for the cubic-term
// elimination): the density field into rho_scratch, then phi [2][ny][nx]
cudaError_t launch_cubic_phi(int storage, const Launch& L, const void* buf, double* rho_scratch, double* phi,
                             cudaStream_t s);
void step_tile(int storage, int* bx, int* by, int* hx);
int step_blocks(int storage, const Geometry& g);
size_t step_smem_bytes(int storage);
cudaError_t prepare_step(int storage);  // per-device kernel attributes; call before capture

// fast: FP32 per-node arithmetic for 32- and 16-bit storage (sums in FP64);
// FP64 storage always computes in FP64
cudaError_t launch_init(int storage, const Launch& L, const double* rho, const double* ux,
                        const double* uy, const double* T, void* buf, cudaStream_t s, bool fast = false);
cudaError_t launch_set_pops(int storage, const Launch& L, const double* f, const double* g, void* buf,
                            cudaStream_t s);
cudaError_t launch_get_pops(int storage, const Launch& L, const void* buf, double* f, double* g,
                            cudaStream_t s);
cudaError_t launch_moments(int storage, const Launch& L, const void* buf, double* rho_scratch,
                           double* rho, double* ux, double* uy, double* T, double* partials,
                           double* stats, unsigned* counter, cudaStream_t s, bool fast = false);
int moments_blocks(const Geometry& g);

// Conservation record of caller-owned [9][ny][nx] FP64 populations with all
// scratch in a fixed device array (lbm_noalloc.cu); allocates nothing.
long long noalloc_max_nodes();
cudaError_t launch_record_noalloc(const Launch& L, const double* f, const double* g, double* out,
                                  cudaStream_t s);

}  // namespace lbm

// Access the surrogate's host code needs to a single-case handle (lbm_host.cpp).
struct lbm_handle;
int lbm_internal_fail(int code, const char* msg);
size_t lbm_internal_state_bytes(const lbm_handle* h);
int lbm_internal_snapshot(lbm_handle* h, void* dst);       // device copy of the current state
int lbm_internal_restore(lbm_handle* h, const void* src);  // and back
// lbm_set_fields from device fields [4][n] with FP32 per-node arithmetic
// (32- and 16-bit storage), synchronous
int lbm_internal_set_fields_fast(lbm_handle* h, const double* fields);
// the fields [4][n] (device, may be null) and the conservation record of the
// current state in one FP32 pass (sums in FP64), synchronous
int lbm_internal_read_fast(lbm_handle* h, double* fields, double out[6]);
cudaStream_t lbm_internal_stream(const lbm_handle* h);
// the handle's step count, host and device copies (the device copy keys the
// stochastic rounding of 16-bit storage); synchronous
int lbm_internal_set_steps(lbm_handle* h, int64_t steps);
void lbm_internal_rho_bounds(const lbm_handle* h, double* rho_v, double* rho_l, int* nx, int* ny);
