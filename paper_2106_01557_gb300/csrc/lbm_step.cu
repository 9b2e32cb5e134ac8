// Fused f+g time step of the liquid-vapor LB model (Eq. 12a-c, 13, 14):
// one persistent CTA per SM walks BX x BY tiles of the lattice.
//
//  1. One elected thread issues two 3-D TMA tile loads (all nine f planes of
//     the tile plus a 2-row / HX-column halo; all nine g planes plus a
//     1-row / HX-column halo) from the ghost-padded state into shared
//     memory, completing on an mbarrier (bounded wait). NS stages: the
//     copies of the next NS - 1 tiles are in flight while one computes.
//  2. The density of the tile and its one-node ring is formed from the
//     pulled f populations in shared memory (pull streaming, Eq. 12a).
//  3. Each node pulls its 18 populations, evaluates the pair force on the
//     shared density tile (Eq. 13), the moments (Eq. 14), the EOS (Eq. 17),
//     collides f and g (Eq. 12b, 12c), and stores the post-collision
//     populations at its own node: coalesced row stores, plus copies into
//     the periodic ghost cells or the reflected value into a wall ghost row.
//  4. The conservation sums of the state entering the step are reduced in
//     FP64 (warp shuffles, then a fixed-order last-block pass), so the
//     result is deterministic.
//
// With 16-bit storage the common case (no open sides, no cubic terms) runs
// the pair form: 384 threads, each updating two neighbouring nodes (x, x + 1)
// with the packed FP32 instructions (lbm_f2.cuh) and storing each population
// of the pair as one 32-bit word. It issues a third fewer instructions per
// node; the packed instructions take the FMA pipe for two cycles each, so
// the step, bound by its FP32 arithmetic, gains only a few per cent.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_f2.cuh"
#include "lbm_ptx.cuh"

namespace lbm {

namespace {

// one persistent CTA per SM; its thread count is a per-precision trait (Tile::NT)

// D2Q9 directions (SM Eq. S1), e_i / c
__host__ __device__ constexpr int EXf(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int EYf(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }


// Tile shape per storage type: BX x BY nodes, HX staged halo columns (16
// bytes), NT threads, NS staging buffers per CTA, CPS resident CTAs per SM;
// NTP: threads of the pair form (16-bit storage; 0: not used).
// With NS >= 2 the copies of the next NS - 1 tiles land while this one
// computes; with NS = 1 and CPS = 2 the two CTAs of an SM cover each
// other's waits.
template <class S>
struct Tile;
template <>
struct Tile<double> { static constexpr int BX = 32, BY = 16, HX = 2, NT = 512, NS = 2, CPS = 1, NTP = 0; };
template <>
struct Tile<float> { static constexpr int BX = 64, BY = 16, HX = 4, NT = 512, NS = 2, CPS = 1, NTP = 0; };
template <>
struct Tile<__half> { static constexpr int BX = 64, BY = 32, HX = 8, NT = 512, NS = 2, CPS = 1, NTP = 384; };
template <>
struct Tile<__nv_bfloat16> { static constexpr int BX = 64, BY = 32, HX = 8, NT = 512, NS = 2, CPS = 1, NTP = 384; };

template <class S, class C>
struct Smem {
    static constexpr int BX = Tile<S>::BX, BY = Tile<S>::BY, HX = Tile<S>::HX;
    static constexpr int WX = BX + 2 * HX;       // row width of a staged plane
    static constexpr int FR = BY + 4;            // staged f rows
    static constexpr int GR = BY + 2;            // staged g rows
    static constexpr int F_BYTES = 9 * FR * WX * (int)sizeof(S);
    static constexpr int G_BYTES = 9 * GR * WX * (int)sizeof(S);
    static constexpr int STAGE = ((F_BYTES + 127) / 128) * 128 + ((G_BYTES + 127) / 128) * 128;
    static constexpr int G_OFF = ((F_BYTES + 127) / 128) * 128;  // within a stage
    static constexpr int NS = Tile<S>::NS;                      // staging buffers
    static constexpr int NR = NS == 1 ? 1 : 2;                   // density tiles
    static constexpr int RX = BX + 2, RY = BY + 2;               // density tile with ring
    static constexpr int R_OFF = NS * STAGE;
    static constexpr int R_BYTES = (((int)sizeof(C) * RX * RY + 127) / 128) * 128;
    static constexpr int BYTES = R_OFF + NR * R_BYTES + 128;     // + alignment slack
    static_assert(NS >= 1 && NS <= 4, "one to four staging buffers");
};

// Wall ghost-row stores of a node next to a wall: the populations leaving
// through the wall come back reversed at the next pull (half-way bounce-back
// of f; of g adiabatic, or anti-bounce-back on a fixed-temperature segment).
// fo[j], go[j] are the post-collision populations of the three directions
// that leave through the wall: (4, 7, 8) at the bottom, (2, 5, 6) at the top.
template <class S, class C, bool OPEN>
__device__ __noinline__ void wall_store(S* __restrict__ out, const Geometry& G, const KC<C>& k, int x, int y,
                                        C fo0, C fo1, C fo2, C go0, C go1, C go2, C rho) {
    const bool bottom = (y == 0);
    const int yg = bottom ? -1 : G.ny;
    const C Tw = bottom ? k.T_bottom : k.T_top;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int opp = bottom ? (j == 0 ? 2 : (j == 1 ? 5 : 6)) : (j == 0 ? 4 : (j == 1 ? 7 : 8));
        // x step of the leaving direction: 0 for 4/2; 7 and 6 go left, 8 and 5 right
        const int ex = j == 0 ? 0 : (bottom ? (j == 1 ? -1 : 1) : (j == 1 ? 1 : -1));
        const C fv = j == 0 ? fo0 : (j == 1 ? fo1 : fo2);
        C gv = j == 0 ? go0 : (j == 1 ? go1 : go2);
        int xg = x + ex;
        xg = xg < 0 ? xg + G.nx : (xg >= G.nx ? xg - G.nx : xg);
        C T_link = Tw;
        if (bottom && G.hot_len > 0) {
            int dxh = (xg - G.hot_x0) % G.nx;
            if (dxh < 0) dxh += G.nx;
            if (dxh < G.hot_len) T_link = k.T_hot;
        }
        if (T_link > C(0)) {
            C ga, gd;
            g_rest_wall(k, rho, T_link, ga, gd);
            gv = C(2) * (j == 0 ? ga : gd) - gv;
        }
        put<S, OPEN>(out, G, opp, xg, yg, Store<S, C>::st(fv, k.rest[opp]));
        put<S, OPEN>(out, G, 9 + opp, xg, yg, Store<S, C>::st(gv, k.rest[9 + opp]));
    }
}

// Per-thread partial sums stay in the compute type (FP64 is a narrow pipe on
// this GPU); they are widened to FP64 once per CTA.
template <class C>
struct Acc {
    C mass, mx, my, ek, et, u2max, bad;
};

// Post-collision populations of node (x, y) into its own slot of the output
// state (pull scheme), with the periodic ghost copies near the edges and the
// wall reflections in the rows next to a wall, or, with OPEN, the ghosts
// beyond the open sides. For shifted formats f and g already hold the
// deviations from the rest populations.
template <class S, class C, bool OPEN>
__device__ __forceinline__ void store_node(S* __restrict__ out, const Geometry& G, const KC<C>& k, int x, int y,
                                           const C f[9], const C g[9], const NodeMacro<C>& s, bool sr, uint32_t seed) {
    const C rho = s.rho;
    const C* rest = k.rest;
    constexpr bool SH = Store<S, C>::SHIFTED;
    const bool interior = x >= GHOST_COLS && x < G.nx - GHOST_COLS && y >= 2 && y < G.ny - 2;
    // the values as stored: 16-bit storage rounds stochastically (sr, from
    // the node's seed), else to nearest
    S sf[9], sg[9];
    if (SH && sr) {
        cvt_sr_node<S, C>(f, g, seed, sf, sg);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            sf[i] = Store<S, C>::cvt(f[i]);
            sg[i] = Store<S, C>::cvt(g[i]);
        }
    }
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
            put<S, OPEN>(out, G, i, x, y, sf[i]);
            put<S, OPEN>(out, G, 9 + i, x, y, sg[i]);
        }
    }
    if (G.walls && (y == 0 || y == G.ny - 1)) {
        // the reflections work on the populations themselves
        auto a = [&](const C* v, int i, int off) { return SH ? v[i] + rest[off + i] : v[i]; };
        // (a side that is open has its own ghosts, below)
        if (y == 0 && !(OPEN && (G.open & 1)))
            wall_store<S, C, OPEN>(out, G, k, x, y, a(f, 4, 0), a(f, 7, 0), a(f, 8, 0), a(g, 4, 9), a(g, 7, 9), a(g, 8, 9), rho);
        if (y == G.ny - 1 && !(OPEN && (G.open & 2)))
            wall_store<S, C, OPEN>(out, G, k, x, y, a(f, 2, 0), a(f, 5, 0), a(f, 6, 0), a(g, 2, 9), a(g, 5, 9), a(g, 6, 9), rho);
    }
    if constexpr (OPEN) {
        if (((G.open & 1) && y == 0) || ((G.open & 2) && y == G.ny - 1) || ((G.open & 4) && x == 0) ||
            ((G.open & 8) && x == G.nx - 1)) {
            Pops9<C> pf, pg;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                pf.v[i] = f[i];
                pg.v[i] = g[i];
            }
            open_store<S, C>(out, G, k, x, y, pf, pg, s.rho, s.uhx, s.uhy, s.T);
        }
    }
}

// One population of a node pair (x even, x + 1) as stored: a 64-bit word of
// two FP32 values, or a 32-bit word of two 16-bit values with node x in the
// low half; nearest rounding (rn) or stochastic (sr, 32 random bits: the
// upper 16 drive node x + 1, the lower 16 node x).
template <class S>
struct PairWord;
template <>
struct PairWord<float> {
    using W = float2;
    static __device__ __forceinline__ W rn(F2 v) { return v.v; }
    static __device__ __forceinline__ W sr(F2 v, uint32_t) { return v.v; }
};
template <>
struct PairWord<__half> {
    using W = uint32_t;
    static __device__ __forceinline__ W rn(F2 v) {
        uint32_t d;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x));
        return d;
    }
    static __device__ __forceinline__ W sr(F2 v, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        return d;
    }
};
template <>
struct PairWord<__nv_bfloat16> {
    using W = uint32_t;
    static __device__ __forceinline__ W rn(F2 v) {
        uint32_t d;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x));
        return d;
    }
    static __device__ __forceinline__ W sr(F2 v, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.v.y), "f"(v.v.x), "r"(r));
        return d;
    }
};

// Two neighbouring staged values as FP32, p at an even element index: one
// 32-bit (16-bit storage) or 64-bit (FP32) shared-memory load
template <class S>
__device__ __forceinline__ F2 ld_pair(const S* p);
template <>
__device__ __forceinline__ F2 ld_pair<float>(const float* p) { return F2(*reinterpret_cast<const float2*>(p)); }
template <>
__device__ __forceinline__ F2 ld_pair<__half>(const __half* p) {
    return F2(__half22float2(*reinterpret_cast<const __half2*>(p)));
}
template <>
__device__ __forceinline__ F2 ld_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
    return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
}
// the same where the index parity is known at compile time: odd indices
// take two loads
template <class S, bool EVEN>
__device__ __forceinline__ F2 ld_pair_at(const S* p) {
    if constexpr (EVEN) return ld_pair<S>(p);
    else return F2(Store<S, float>::raw(p[0]), Store<S, float>::raw(p[1]));
}

// Post-collision populations of the pair (x, x + 1) at row y. Pairs whose
// nodes and ghost copies all lie inside the interior band store each
// population as one word; the others (next to the edges of the lattice, or
// with x + 1 outside it: v1 false) go node by node through store_node. With
// stochastic rounding the interior pair draws its 18 words from one seed h
// (multiplicative hashing with 18 fixed odd constants), the node-by-node
// path from each node's own seed.
template <class S>
__device__ __forceinline__ void store_pair(S* __restrict__ out, const Geometry& G, const KC<float>& k, int x, int y,
                                           bool v1, const F2 f[9], const F2 g[9], F2 rho, bool sr,
                                           uint32_t step_key) {
    const bool interior = v1 && x >= GHOST_COLS && x + 1 < G.nx - GHOST_COLS && y >= 2 && y < G.ny - 2;
    if (interior) {
        using PW = PairWord<S>;
        using W = typename PW::W;
        S* o = out + (long long)(y + 2) * G.pitch + G.PX + x;
        if (Store<S, float>::SHIFTED && sr) {
            const uint32_t h = fmix32((uint32_t)(y * G.nx + x) ^ step_key);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                *reinterpret_cast<W*>(o + i * G.plane) = PW::sr(f[i], h * (0x9e3779b9u * (2u * i + 1u)));
                *reinterpret_cast<W*>(o + (9 + i) * G.plane) = PW::sr(g[i], h * (0x9e3779b9u * (2u * i + 19u)));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                *reinterpret_cast<W*>(o + i * G.plane) = PW::rn(f[i]);
                *reinterpret_cast<W*>(o + (9 + i) * G.plane) = PW::rn(g[i]);
            }
        }
        return;
    }
    float fl[9], gl[9];
    NodeMacro<float> s;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fl[i] = f[i].v.x;
        gl[i] = g[i].v.x;
    }
    s.rho = rho.v.x;
    store_node<S, float, false>(out, G, k, x, y, fl, gl, s, sr, fmix32((uint32_t)(y * G.nx + x) ^ step_key));
    if (v1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fl[i] = f[i].v.y;
            gl[i] = g[i].v.y;
        }
        s.rho = rho.v.y;
        store_node<S, float, false>(out, G, k, x + 1, y, fl, gl, s, sr,
                                    fmix32((uint32_t)(y * G.nx + x + 1) ^ step_key));
    }
}

// threads of a step CTA: the pair form takes half
template <class S, bool PAIR>
__host__ __device__ constexpr int step_threads() { return PAIR ? Tile<S>::NTP : Tile<S>::NT; }

// OPEN: the case has open sides; CUBIC: the cubic-term elimination, with
// phi = rho u_x^3, rho u_y^3 of the entering state (separate instantiations,
// so that the common path carries none of their code)
template <class S, class C, bool OPEN, bool CUBIC, bool PAIR>
__global__ void __launch_bounds__(step_threads<S, PAIR>(), Tile<S>::CPS)
    k_step(const __grid_constant__ CUtensorMap tmf, const __grid_constant__ CUtensorMap tmg,
           S* __restrict__ out, const __grid_constant__ Launch L, double* __restrict__ partials,
           double* __restrict__ stats, unsigned* __restrict__ counter, int* __restrict__ status,
           const double* __restrict__ phi) {
    using SM = Smem<S, C>;
    constexpr int BX = SM::BX, BY = SM::BY, HX = SM::HX, WX = SM::WX;
    constexpr int FR = SM::FR, GR = SM::GR, RX = SM::RX, RY = SM::RY;
    constexpr int NT = step_threads<S, PAIR>(), NS = SM::NS;
    constexpr int TPR = PAIR ? BX / 2 : BX;  // threads per tile row
    static_assert(NT % TPR == 0 && BX % 2 == 0, "whole tile rows per thread sweep");
    static_assert(!PAIR || (std::is_same<C, float>::value && !OPEN && !CUBIC), "pair form: FP32 arithmetic, common case");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[SM::NS];
    __shared__ C red[NT / 32][7];
    __shared__ bool last;
    // TMA destinations start on a 128-byte boundary (the launch adds 128 bytes)
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);

    const Geometry& G = L.geo;
    const KC<C>& k = kc<C>(L);
    const int tid = threadIdx.x;
    const int ntx = (G.nx + BX - 1) / BX, nty = (G.ny + BY - 1) / BY;
    const int ntiles = ntx * nty;

    auto issue = [&](int tile, int stage) {
        const int tx0 = (tile % ntx) * BX, ty0 = (tile / ntx) * BY;
        unsigned char* st = smem + stage * SM::STAGE;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(SM::F_BYTES + SM::G_BYTES));
        // padded coordinates: x_p = x + HX, y_p = y + 2
        tma_load_3d(st, &tmf, tx0, ty0, 0, &bar[stage]);                 // rows ty0-2 .. ty0+BY+1
        tma_load_3d(st + SM::G_OFF, &tmg, tx0, ty0 + 1, 9, &bar[stage]);  // rows ty0-1 .. ty0+BY
    };

    if (tid == 0) {
        for (int j = 0; j < NS; ++j) mbar_init(&bar[j], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < NS; ++j)
            if ((int)blockIdx.x + j * (int)gridDim.x < ntiles) issue(blockIdx.x + j * gridDim.x, j);
    }

    Acc<C> acc = {0, 0, 0, 0, 0, 0, 0};
    Acc<F2> acc2 = {0, 0, 0, 0, 0, 0, 0};  // pair form: one lane per node of the pair
    bool ok = true;
    int it = 0;
    // stochastic rounding of 16-bit storage: the step count (kept in the
    // record by the last block of the previous launch) keys the dither
    const bool sr = Store<S, C>::SHIFTED && L.rounding;
    const uint32_t step_key = sr ? fmix32((uint32_t)(long long)__ldcg(&stats[7]) * 0x9e3779b9u + 0x7f4a7c15u) : 0u;
    // NS >= 2: one block barrier per tile. At the barrier after the density
    // pass of tile `it`, every thread has finished tile it-1, so its stage is
    // refilled with tile it+NS-1 and the other density buffer is free.
    // NS = 1: a second barrier after the compute pass frees the one stage.
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int stage = it % NS;
        bool timed_out = false;
        {
            const uint32_t parity = (uint32_t)(it / NS) & 1u;
            if (L.tile_wait_ns == 0) {
                timed_out = !mbar_test_wait(&bar[stage], parity);  // no waiting at all
            } else {
                const uint64_t t0 = globaltimer_ns();
                while (!mbar_try_wait(&bar[stage], parity)) {
                    if (globaltimer_ns() - t0 > L.tile_wait_ns) { timed_out = true; break; }
                }
            }
        }
        const S* sf = reinterpret_cast<const S*>(smem + stage * SM::STAGE);
        const S* sg = reinterpret_cast<const S*>(smem + stage * SM::STAGE + SM::G_OFF);
        C* srho = reinterpret_cast<C*>(smem + SM::R_OFF + (it % SM::NR) * SM::R_BYTES);
        const int tx0 = (tile % ntx) * BX, ty0 = (tile / ntx) * BY;

        // ---- density on tile + ring (pull sums from staged f) --------------
        // (after a timed-out wait these reads see stale data; the pass is
        // discarded at the barrier below)
        if constexpr (PAIR) {
            // node pairs (rx, rx + 1) of the ring-extended tile (RX even); the
            // staged column of node rx - 1 + HX - e_x is even for e_x = +-1
            static_assert(RX % 2 == 0 && HX % 2 == 0 && WX % 2 == 0, "pair alignment");
#pragma unroll 1
            for (int idx = tid; idx < (RX / 2) * RY; idx += NT) {
                const int rx = 2 * (idx % (RX / 2)), ry = idx / (RX / 2);
                const int gy = ty0 + ry - 1;
                int sy = ry + 1;
                if (G.walls) {
                    if (gy < 0) sy -= gy;
                    else if (gy >= G.ny) sy -= gy - (G.ny - 1);
                }
                const S* p = sf + sy * WX + rx - 1 + HX;
                F2 r = F2(Store<S, C>::SHIFTED ? (float)k.mrest[0] : 0.f);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int o = i * FR * WX - EYf(i) * WX - EXf(i);
                    if (EXf(i) != 0) r += ld_pair_at<S, true>(p + o);
                    else r += ld_pair_at<S, false>(p + o);
                }
                *reinterpret_cast<float2*>(reinterpret_cast<float*>(srho) + ry * RX + rx) = r.v;
            }
        } else {
#pragma unroll 1
        for (int idx = tid; idx < RX * RY; idx += NT) {
            const int rx = idx % RX, ry = idx / RX;
            const int gy = ty0 + ry - 1;
            if (OPEN && beyond_open(G, tx0 + rx - 1, gy)) {  // the open sides' fixed density
                srho[idx] = k.rho_open;
                continue;
            }
            int sy = ry + 1;  // staged row of this node: y - (ty0 - 2)
            if (G.walls) {    // density beyond a wall = adjacent fluid node's
                if (gy < 0) sy -= gy;
                else if (gy >= G.ny) sy -= gy - (G.ny - 1);
            }
            const S* p = sf + sy * WX + rx - 1 + HX;
            // shifted formats: the rest populations sum to mrest[0]
            C r = Store<S, C>::SHIFTED ? k.mrest[0] : C(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) r += Store<S, C>::raw(p[i * FR * WX - EYf(i) * WX - EXf(i)]);
            srho[idx] = r;
        }
        }
        if (__syncthreads_or(timed_out)) { ok = false; break; }
        if (NS >= 2 && tid == 0) {
            const int ahead = tile + (NS - 1) * gridDim.x;  // tile it+NS-1 goes into the stage tile it-1 used
            if (it > 0 && ahead < ntiles) issue(ahead, (it - 1) % NS);
        }

        if constexpr (PAIR) {
            const int lx = 2 * (tid % TPR);
            const int x = tx0 + lx;
#pragma unroll 1
            for (int ly = tid / TPR; ly < BY; ly += NT / TPR) {
                const int y = ty0 + ly;
                if (x >= G.nx || y >= G.ny) continue;
                const bool v1 = x + 1 < G.nx;  // the pair's second node is in the lattice
                F2 f[9], g[9], rn[9];
                const S* pf = sf + (ly + 2) * WX + lx + HX;
                const S* pg = sg + (ly + 1) * WX + lx + HX;
                const float* pr = reinterpret_cast<const float*>(srho) + (ly + 1) * RX + lx + 1;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int of = i * FR * WX - EYf(i) * WX - EXf(i), og = i * GR * WX - EYf(i) * WX - EXf(i);
                    // the staged column lx + HX - e_x is even for e_x = 0
                    if (EXf(i) == 0) {
                        f[i] = ld_pair_at<S, true>(pf + of);
                        g[i] = ld_pair_at<S, true>(pg + og);
                    } else {
                        f[i] = ld_pair_at<S, false>(pf + of);
                        g[i] = ld_pair_at<S, false>(pg + og);
                    }
                    // the density tile's pairs start on 8 bytes where x - 1 + e_x is even
                    const int orr = EYf(i) * RX + EXf(i);
                    if (EXf(i) != 0)
                        rn[i] = F2(*reinterpret_cast<const float2*>(pr + orr));
                    else
                        rn[i] = F2(pr[orr], pr[orr + 1]);
                }
                NodeMacro<F2> s;
                node_macro<Store<S, C>::SHIFTED>(k, f, g, rn, s);
                {   // conservation record of the entering state (lane 1 only where v1)
                    const F2 rho = s.rho;
                    const F2 third = F2(1.0 / 3.0), twelfth = F2(1.0 / 12.0);
                    const F2 lap = F2(2.0f) * (third * ((rn[1] + rn[2]) + (rn[3] + rn[4])) +
                                               twelfth * ((rn[5] + rn[6]) + (rn[7] + rn[8])) - F2(5.0 / 3.0) * rho);
                    F2 cm = rho, cx = rho * s.uhx, cy = rho * s.uhy, ce = s.rek;
                    F2 et = s.rek - k.a * rho * rho - k.half_kappa * rho * lap;
                    F2 u2 = s.uhx * s.uhx + s.uhy * s.uhy;
                    const float r0 = rho.v.x, r1 = rho.v.y, T0 = s.T.v.x, T1 = s.T.v.y;
                    F2 bad = F2(!(r0 > 0.f && r0 < 1e30f && T0 > 0.f && T0 < 1e30f && u2.v.x < 1e30f) ? 1.f : 0.f,
                                !(r1 > 0.f && r1 < 1e30f && T1 > 0.f && T1 < 1e30f && u2.v.y < 1e30f) ? 1.f : 0.f);
                    if (!v1) {
                        cm.v.y = cx.v.y = cy.v.y = ce.v.y = et.v.y = u2.v.y = bad.v.y = 0.f;
                    }
                    acc2.mass += cm;
                    acc2.mx += cx;
                    acc2.my += cy;
                    acc2.ek += ce;
                    acc2.et += et;
                    acc2.u2max = F2(u2.v.x > acc2.u2max.v.x ? u2.v.x : acc2.u2max.v.x,
                                    u2.v.y > acc2.u2max.v.y ? u2.v.y : acc2.u2max.v.y);
                    acc2.bad += bad;
                }
                collide<Store<S, C>::SHIFTED, false>(k, f, g, s, F2(0.f));
                store_pair<S>(out, G, k, x, y, v1, f, g, s.rho, sr, step_key);
            }
        } else {
        const int lx = tid % BX;
        const int x = tx0 + lx;
#pragma unroll 1
        for (int ly = tid / BX; ly < BY; ly += NT / BX) {
            const int y = ty0 + ly;
            if (x >= G.nx || y >= G.ny) continue;
            C f[9], g[9], rn[9];
            const S* pf = sf + (ly + 2) * WX + lx + HX;
            const S* pg = sg + (ly + 1) * WX + lx + HX;
            const C* pr = srho + (ly + 1) * RX + lx + 1;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = Store<S, C>::raw(pf[i * FR * WX - EYf(i) * WX - EXf(i)]);
                g[i] = Store<S, C>::raw(pg[i * GR * WX - EYf(i) * WX - EXf(i)]);
                rn[i] = pr[EYf(i) * RX + EXf(i)];
            }
            NodeMacro<C> s;
            node_macro<Store<S, C>::SHIFTED>(k, f, g, rn, s);
            {   // conservation record of the entering state
                const C rho = s.rho;
                acc.mass += rho;
                acc.mx += rho * s.uhx;
                acc.my += rho * s.uhy;
                acc.ek += s.rek;
                const C third = C(1.0 / 3.0), twelfth = C(1.0 / 12.0);
                const C lap = C(2) * (third * ((rn[1] + rn[2]) + (rn[3] + rn[4])) +
                                      twelfth * ((rn[5] + rn[6]) + (rn[7] + rn[8])) - C(5.0 / 3.0) * s.rho);
                acc.et += s.rek - k.a * s.rho * s.rho - k.half_kappa * s.rho * lap;
                const C u2 = s.uhx * s.uhx + s.uhy * s.uhy;
                acc.u2max = u2 > acc.u2max ? u2 : acc.u2max;
                // a non-positive or non-finite density or temperature, or a
                // runaway velocity (the comparisons also catch NaN)
                if (!(rho > C(0) && rho < C(1e30) && s.T > C(0) && s.T < C(1e30) && u2 < C(1e30))) acc.bad += C(1);
            }
            C R7 = C(0);
            if constexpr (CUBIC) {
                // -c (d_x(rho u_x^3) - d_y(rho u_y^3)), periodic central differences
                const long long n = (long long)G.nx * G.ny;
                const int xm = x == 0 ? G.nx - 1 : x - 1, xp = x == G.nx - 1 ? 0 : x + 1;
                const int ym = y == 0 ? G.ny - 1 : y - 1, yp = y == G.ny - 1 ? 0 : y + 1;
                const double dpx = 0.5 * (__ldg(phi + (long long)y * G.nx + xp) - __ldg(phi + (long long)y * G.nx + xm));
                const double dpy = 0.5 * (__ldg(phi + n + (long long)yp * G.nx + x) - __ldg(phi + n + (long long)ym * G.nx + x));
                R7 = -k.c * ((C)dpx - (C)dpy);
            }
            collide<Store<S, C>::SHIFTED, CUBIC>(k, f, g, s, R7);
            store_node<S, C, OPEN>(out, G, k, x, y, f, g, s, sr, fmix32((uint32_t)(y * G.nx + x) ^ step_key));
        }
        }
        if (NS == 1) {
            __syncthreads();  // every thread is done with the stage: refill it
            if (tid == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, 0);
        }
    }
    if (!ok && tid == 0) {
        atomicOr(status, ST_TIMEOUT);
        // give the copies in flight (this iteration's and those of the next
        // NS - 1 tiles) a bounded chance to land before exiting; this drain
        // keeps the full default bound whatever the tile-wait limit
        const int jend = it == 0 ? NS : it + NS - 1;  // tiles issued so far: 0 .. jend - 1
        for (int j = it; j < jend; ++j) {
            if ((int)blockIdx.x + j * (int)gridDim.x >= ntiles) break;
            const uint64_t t0 = globaltimer_ns();
            while (!mbar_try_wait(&bar[j % NS], (uint32_t)(j / NS) & 1u) && globaltimer_ns() - t0 < WAIT_NS) {}
        }
    }

    if constexpr (PAIR) {  // the pair lanes into the scalar record
        acc.mass = acc2.mass.v.x + acc2.mass.v.y;
        acc.mx = acc2.mx.v.x + acc2.mx.v.y;
        acc.my = acc2.my.v.x + acc2.my.v.y;
        acc.ek = acc2.ek.v.x + acc2.ek.v.y;
        acc.et = acc2.et.v.x + acc2.et.v.y;
        acc.u2max = acc2.u2max.v.x > acc2.u2max.v.y ? acc2.u2max.v.x : acc2.u2max.v.y;
        acc.bad = acc2.bad.v.x + acc2.bad.v.y;
    }

    // ---- block reduction: compute type within warps, FP64 across warps -----
    C v[7] = {acc.mass, acc.mx, acc.my, acc.ek, acc.et, acc.u2max, acc.bad};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const C w = __shfl_down_sync(0xffffffffu, v[q], o);
            v[q] = (q == 5) ? (w > v[q] ? w : v[q]) : v[q] + w;
        }
    }
    const int warp = tid / 32, lane = tid % 32;
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) red[warp][q] = v[q];
    }
    __syncthreads();
    const unsigned nblocks = gridDim.x;
    if (tid < 7) {
        const int q = tid;
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t = (q == 5) ? fmax(t, (double)red[w][q]) : t + (double)red[w][q];
        const double cc = (double)k.c;
        if (q == 1 || q == 2) t *= cc;
        if (q == 5) t *= cc * cc;
        partials[(size_t)blockIdx.x * NQ + q] = t;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        last = (atomicAdd(counter, 1u) == nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // warp q < 7 combines quantity q: lane l takes blocks l, l + 32, ...
    // (independent L2 loads), then a butterfly; a fixed order, so the
    // record is the same on every run
    if (warp < 7) {
        const int q = warp;
        double t = 0.0;
        for (unsigned b = lane; b < nblocks; b += 32) {
            const double pv = __ldcg(partials + (size_t)b * NQ + q);
            t = (q == 5) ? fmax(t, pv) : t + pv;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, t, o);
            t = (q == 5) ? fmax(t, w) : t + w;
        }
        if (lane == 0) {
            stats[q] = (q == 5) ? sqrt(t) : t;
            if (q == 6 && t > 0.0) atomicOr(status, ST_NONFINITE);
        }
    }
    __syncthreads();
    if (tid == 0) {
        stats[7] = stats[7] + 1.0;  // fused steps executed so far
        *counter = 0u;
    }
}

template <class S, class C>
cudaError_t launch_t(const Launch& L, const CUtensorMap* tmf, const CUtensorMap* tmg, void* out,
                     double* partials, double* stats, unsigned* counter, int* status, cudaStream_t s,
                     const double* phi) {
    using SM = Smem<S, C>;
    const int ntiles = ((L.geo.nx + SM::BX - 1) / SM::BX) * ((L.geo.ny + SM::BY - 1) / SM::BY);
    const int slots = Tile<S>::CPS * L.geo.sms;
    const int grid = ntiles < slots ? ntiles : slots;
    constexpr bool P = Tile<S>::NTP > 0;  // the pair form for 16-bit storage
    if (L.geo.open)
        k_step<S, C, true, false, false><<<grid, Tile<S>::NT, SM::BYTES, s>>>(*tmf, *tmg, static_cast<S*>(out), L,
                                                                              partials, stats, counter, status, phi);
    else if (L.cubic)
        k_step<S, C, false, true, false><<<grid, Tile<S>::NT, SM::BYTES, s>>>(*tmf, *tmg, static_cast<S*>(out), L,
                                                                              partials, stats, counter, status, phi);
    else
        k_step<S, C, false, false, P><<<grid, step_threads<S, P>(), SM::BYTES, s>>>(
            *tmf, *tmg, static_cast<S*>(out), L, partials, stats, counter, status, phi);
    return cudaGetLastError();
}

}  // namespace

void step_tile(int storage, int* bx, int* by, int* hx) {
    switch (storage) {
        case S_F64: *bx = Tile<double>::BX; *by = Tile<double>::BY; *hx = Tile<double>::HX; break;
        case S_F32: *bx = Tile<float>::BX; *by = Tile<float>::BY; *hx = Tile<float>::HX; break;
        default: *bx = Tile<__half>::BX; *by = Tile<__half>::BY; *hx = Tile<__half>::HX; break;
    }
}

int step_blocks(int storage, const Geometry& g) {
    int bx, by, hx;
    step_tile(storage, &bx, &by, &hx);
    const int cps = storage == S_F64 ? Tile<double>::CPS : (storage == S_F32 ? Tile<float>::CPS : Tile<__half>::CPS);
    const int ntiles = ((g.nx + bx - 1) / bx) * ((g.ny + by - 1) / by);
    return ntiles < cps * g.sms ? ntiles : cps * g.sms;
}

size_t step_smem_bytes(int storage) {
    switch (storage) {
        case S_F64: return Smem<double, double>::BYTES;
        case S_F32: return Smem<float, float>::BYTES;
        case S_F16: return Smem<__half, float>::BYTES;
        default: return Smem<__nv_bfloat16, float>::BYTES;
    }
}

template <class S, class C>
cudaError_t attr_t(int smem) {
    constexpr bool P = Tile<S>::NTP > 0;
    cudaError_t e =
        cudaFuncSetAttribute(k_step<S, C, false, false, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step<S, C, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_step<S, C, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t prepare_step(int storage) {
    const int smem = (int)step_smem_bytes(storage);
    switch (storage) {
        case S_F64: return attr_t<double, double>(smem);
        case S_F32: return attr_t<float, float>(smem);
        case S_F16: return attr_t<__half, float>(smem);
        case S_BF16: return attr_t<__nv_bfloat16, float>(smem);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(int storage, const Launch& L, const CUtensorMap* tmf, const CUtensorMap* tmg, void* out,
                        double* partials, double* stats, unsigned* counter, int* status, cudaStream_t s,
                        const double* phi) {
    if (L.cubic && !phi) return cudaErrorInvalidValue;
    switch (storage) {
        case S_F64: return launch_t<double, double>(L, tmf, tmg, out, partials, stats, counter, status, s, phi);
        case S_F32: return launch_t<float, float>(L, tmf, tmg, out, partials, stats, counter, status, s, phi);
        case S_F16: return launch_t<__half, float>(L, tmf, tmg, out, partials, stats, counter, status, s, phi);
        case S_BF16:
            return launch_t<__nv_bfloat16, float>(L, tmf, tmg, out, partials, stats, counter, status, s, phi);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
