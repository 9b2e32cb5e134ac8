// Device-side pieces of the liquid-vapor LB model shared by the kernels:
// storage conversion, the D2Q9 moment transforms and the per-node collision
// (Eq. 12b, 12c with SM Eq. S3-S6), written as fixed add/sub trees.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// ---- storage <-> compute ---------------------------------------------------
template <class S, class C>
struct Store;
// ld / st convert a stored population to / from its value; raw / cvt only
// convert, leaving the rest population to the caller (shifted formats add it
// in moment space, where it touches three moments instead of nine values).
// SHIFTED marks the formats that store deviations from the rest state.
template <>
struct Store<double, double> {
    static constexpr bool SHIFTED = false;
    static __device__ __forceinline__ double ld(double v, double) { return v; }
    static __device__ __forceinline__ double st(double v, double) { return v; }
    static __device__ __forceinline__ double raw(double v) { return v; }
    static __device__ __forceinline__ double cvt(double v) { return v; }
    static __device__ __forceinline__ void cvt_sr2(double a, double b, uint32_t, double& sa, double& sb) {
        sa = a;
        sb = b;
    }
};
template <>
struct Store<float, float> {
    static constexpr bool SHIFTED = false;
    static __device__ __forceinline__ float ld(float v, float) { return v; }
    static __device__ __forceinline__ float st(float v, float) { return v; }
    static __device__ __forceinline__ float raw(float v) { return v; }
    static __device__ __forceinline__ float cvt(float v) { return v; }
    static __device__ __forceinline__ void cvt_sr2(float a, float b, uint32_t, float& sa, float& sb) {
        sa = a;
        sb = b;
    }
};
template <>
struct Store<__half, float> {
    static constexpr bool SHIFTED = true;
    static __device__ __forceinline__ float ld(__half v, float rest) { return rest + __half2float(v); }
    static __device__ __forceinline__ __half st(float v, float rest) { return __float2half_rn(v - rest); }
    static __device__ __forceinline__ float raw(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half cvt(float v) { return __float2half_rn(v); }
    // a and b rounded stochastically (up with probability equal to the
    // discarded fraction, subnormals included) by the stochastic-rounding
    // conversion; the upper 16 bits of r drive a, the lower 16 bits b
    static __device__ __forceinline__ void cvt_sr2(float a, float b, uint32_t r, __half& sa, __half& sb) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
        sa = __ushort_as_half((unsigned short)(d >> 16));
        sb = __ushort_as_half((unsigned short)(d & 0xffffu));
    }
};
template <>
struct Store<__nv_bfloat16, float> {
    static constexpr bool SHIFTED = true;
    static __device__ __forceinline__ float ld(__nv_bfloat16 v, float rest) { return rest + __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 st(float v, float rest) { return __float2bfloat16_rn(v - rest); }
    static __device__ __forceinline__ float raw(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 cvt(float v) { return __float2bfloat16_rn(v); }
    // as for half precision: the upper 16 bits of r drive a, the lower b
    static __device__ __forceinline__ void cvt_sr2(float a, float b, uint32_t r, __nv_bfloat16& sa,
                                                   __nv_bfloat16& sb) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
        sa = __ushort_as_bfloat16((unsigned short)(d >> 16));
        sb = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
    }
};

// Dither of the stochastic rounding: the 32-bit finaliser of MurmurHash3
// (A. Appleby) mixes (node, step) into a seed h per node, uniform on 32 bits;
// pair i of stored populations takes h K_i mod 2^32 with a fixed odd K_i
// (multiplicative hashing, Knuth): a bijection of h, so each pair's 32 bits
// are uniform too, at one multiply per pair.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// The nine (f_i, g_i) pairs of a node converted with stochastic rounding
// from the node's seed h (cvt_sr2: the upper 16 bits round f_i, the lower
// 16 bits g_i).
template <class S, class C>
__device__ __forceinline__ void cvt_sr_node(const C f[9], const C g[9], uint32_t h, S sf[9], S sg[9]) {
    constexpr uint32_t K[9] = {0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du, 0x27d4eb2fu, 0x165667b1u,
                               0xd3a2646du, 0xfd7046c5u, 0xb55a4f09u, 0x61c88647u};
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<S, C>::cvt_sr2(f[i], g[i], h * K[i], sf[i], sg[i]);
}

// Reciprocal: IEEE in FP64; in FP32 the hardware approximation (relative
// error ~1e-7, far below the FP32 path's 1e-5 parity bound).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }

// clamp to [0, 1]
__device__ __forceinline__ double clamp01(double w) { return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w); }
__device__ __forceinline__ float clamp01(float w) { return w < 0.f ? 0.f : (w > 1.f ? 1.f : w); }

template <class C>
__device__ __forceinline__ const KC<C>& kc(const Launch& L);
template <>
__device__ __forceinline__ const KC<float>& kc<float>(const Launch& L) { return L.kf; }
template <>
__device__ __forceinline__ const KC<double>& kc<double>(const Launch& L) { return L.kd; }

// m = M l (SM Eq. S2)
template <class C>
__device__ __forceinline__ void moments9(const C l[9], C m[9]) {
    const C ax = l[1] + l[2] + l[3] + l[4];
    const C dg = l[5] + l[6] + l[7] + l[8];
    m[0] = l[0] + ax + dg;
    m[1] = C(-4) * l[0] - ax + C(2) * dg;
    m[2] = C(4) * l[0] - C(2) * ax + dg;
    const C dx = l[5] - l[6] - l[7] + l[8];
    const C dy = l[5] + l[6] - l[7] - l[8];
    m[3] = l[1] - l[3] + dx;
    m[4] = C(-2) * (l[1] - l[3]) + dx;
    m[5] = l[2] - l[4] + dy;
    m[6] = C(-2) * (l[2] - l[4]) + dy;
    m[7] = l[1] - l[2] + l[3] - l[4];
    m[8] = l[5] - l[6] + l[7] - l[8];
}

// m0 / 9, the weight of moment 0 in every population. Each column of M^-1
// but the first sums to zero over the nine populations, so the populations
// sum to 9 (m0 / 9) whatever the other moments: a relative error e of this
// one product is a gain of 9 e per step in mass (f) and energy (g). In FP32,
// m0 * fl(1/9) has e = 9 fl(1/9) - 1 = +7.45e-9 at every node, a drift the
// bulk phases cannot average out; the constant split into a rounded part
// and its remainder (hi + lo = 1/9 to 48 bits in FP32, to 110 bits in FP64)
// gives a correctly rounded quotient in all but rare ties. In FP64 the same
// split removes e = -5.6e-17 per step (3e-12 of the mass over 60,000 steps).
__device__ __forceinline__ double ninth(double m) {
    constexpr double hi = 1.0 / 9.0;
    constexpr double lo = 6.1679056923619804e-18;  // 1/9 - hi, rounded
    return __fma_rn(m, hi, m * lo);
}
__device__ __forceinline__ float ninth(float m) {
    constexpr float hi = (float)(1.0 / 9.0);
    constexpr float lo = (float)(1.0 / 9.0 - (double)(float)(1.0 / 9.0));
    return __fmaf_rn(m, hi, m * lo);
}

// With FP32 populations the rest population is taken as the complement of
// the other eight, l_0 = m_0 - sum_{i >= 1} l_i: the nine then sum to m_0 up
// to the rounding of that sum, where the back-transform's own roundings,
// correlated across the nine values, leave a small bias in mass (f) and
// energy (g) from step to step.
template <class C>
__device__ __forceinline__ void rest_as_complement(C m0, C l[9]) {
    if constexpr (sizeof(C) == 4) l[0] = m0 - (((l[1] + l[2]) + (l[3] + l[4])) + ((l[5] + l[6]) + (l[7] + l[8])));
}

// l = M^-1 m = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m
template <class C>
__device__ __forceinline__ void populations9(const C m[9], C l[9]) {
    const C a0 = ninth(m[0]), a1 = m[1] * C(1.0 / 36.0), a2 = m[2] * C(1.0 / 36.0);
    const C a3 = m[3] * C(1.0 / 6.0), a4 = m[4] * C(1.0 / 12.0);
    const C a5 = m[5] * C(1.0 / 6.0), a6 = m[6] * C(1.0 / 12.0);
    const C a7 = m[7] * C(0.25), a8 = m[8] * C(0.25);
    l[0] = a0 - C(4) * a1 + C(4) * a2;
    const C axis = a0 - a1 - C(2) * a2;
    const C px = a3 - C(2) * a4, py = a5 - C(2) * a6;
    l[1] = axis + px + a7;
    l[2] = axis + py - a7;
    l[3] = axis - px + a7;
    l[4] = axis - py - a7;
    const C diag = a0 + C(2) * a1 + a2;
    const C qx = a3 + a4, qy = a5 + a6;
    l[5] = diag + qx + qy + a8;
    l[6] = diag - qx + qy - a8;
    l[7] = diag - qx - qy + a8;
    l[8] = diag + qx - qy - a8;
}

// Per-node macroscopic state (Eq. 13, 14) from the pulled populations and
// the density field around the node: rn[i] = rho(x + e_i), rn[0] = rho(x),
// which every caller has already formed as sum_i f_i (Eq. 14). The moments
// m = M f and n = M g are kept for the collision.
template <class C>
struct NodeMacro {
    C rho, inv_rho;
    C gx, gy;      // sum_i omega_i rho(x+e_i) e_i = grad rho (F_pair = G^2 rho grad rho)
    C Fhx, Fhy;    // F / c
    C uhx, uhy;    // u / c
    C q, rek, T;
    C m[9], n[9];
};

// SH: f and g hold deviations from the rest populations; their moments get
// the rest moments added back (moments 0-2, the others vanish).
template <bool SH = false, class C, class K>
__device__ __forceinline__ void node_macro(const K& k, const C f[9], const C g[9], const C rn[9],
                                           NodeMacro<C>& s) {
    moments9(f, s.m);
    moments9(g, s.n);
    if constexpr (SH) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            s.m[q] += k.mrest[q];
            s.n[q] += k.nrest[q];
        }
    }
    const C rho = rn[0];
    // Eq. 13 weights: 1/3 on the axes, 1/12 on the diagonals
    const C third = C(1.0 / 3.0), twelfth = C(1.0 / 12.0);
    s.gx = third * (rn[1] - rn[3]) + twelfth * ((rn[5] - rn[7]) + (rn[8] - rn[6]));
    s.gy = third * (rn[2] - rn[4]) + twelfth * ((rn[5] - rn[7]) + (rn[6] - rn[8]));
    s.rho = rho;
    s.inv_rho = recip(rho);
    s.Fhx = k.G2c * rho * s.gx + rho * k.axc;
    s.Fhy = k.G2c * rho * s.gy + rho * k.ayc;
    // Eq. 14: rho u = sum e_i f_i + dt/2 F  ->  rho u^ = m_3,5 + dt/2 F^
    s.uhx = (s.m[3] + k.half_dt * s.Fhx) * s.inv_rho;
    s.uhy = (s.m[5] + k.half_dt * s.Fhy) * s.inv_rho;
    // q = F . u = c^2 F^ . u^
    s.q = k.c2 * (s.Fhx * s.uhx + s.Fhy * s.uhy);
    s.rek = s.n[0] + k.half_dt * s.q;
    const C ke = C(0.5) * k.c2 * (s.uhx * s.uhx + s.uhy * s.uhy);
    s.T = (s.rek * s.inv_rho - ke) * k.inv_cv;
}

// p_BE = p_EOS + a rho^2 with Eq. 17
template <class C, class K>
__device__ __forceinline__ C p_BE(const K& k, C rho, C T) {
    const C th = k.b4 * rho;
    const C om = C(1) - th;
    const C z = (C(1) + th * (C(1) + th * (C(1) - th))) * recip(om * om * om);
    return k.RK * rho * T * z + k.aK_eff * rho * rho;
}

// Equilibria of f and g at one node, used by initialisation:
// m^eq (SM Eq. S3a), F_m (S3b), n^eq (S4a), q_m (S4b). cubic: the q_x, q_y
// equilibria carry the cubic terms 3 rho u_x u_y^2, 3 rho u_y u_x^2.
template <class C>
__device__ __forceinline__ void equilibria(const KC<C>& k, const NodeMacro<C>& s, C meq[9], C Fm[9],
                                           C neq[9], C qm[9], bool cubic = false) {
    const C rho = s.rho, ux = s.uhx, uy = s.uhy;
    const C u2 = ux * ux + uy * uy;
    const C pbe = p_BE(k, rho, s.T);
    const C eta = pbe * k.cs2_inv - rho;
    const C rhk = s.rek + pbe;
    meq[0] = rho;
    meq[1] = C(-2) * rho + C(2) * eta + C(3) * rho * u2;
    meq[2] = rho + k.beta * eta - C(3) * rho * u2;
    meq[3] = rho * ux;
    meq[4] = -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * ux * uy;
    if (cubic) {
        meq[4] += C(3) * rho * ux * uy * uy;
        meq[6] += C(3) * rho * uy * ux * ux;
    }
    const C Fx = s.Fhx, Fy = s.Fhy;
    const C FU = Fx * ux + Fy * uy;
    Fm[0] = C(0);
    Fm[1] = C(6) * FU;
    Fm[2] = C(-6) * FU;
    Fm[3] = Fx;
    Fm[4] = -Fx;
    Fm[5] = Fy;
    Fm[6] = -Fy;
    Fm[7] = C(2) * (Fx * ux - Fy * uy);
    Fm[8] = Fx * uy + Fy * ux;
    const C E = s.rek, CT = k.Cref * s.T;
    neq[0] = E;
    neq[1] = C(-4) * E + (C(4) + k.g1) * CT;
    neq[2] = C(4) * E - (C(4) - k.g2) * CT;
    neq[3] = rhk * ux;
    neq[4] = -rhk * ux;
    neq[5] = rhk * uy;
    neq[6] = -rhk * uy;
    neq[7] = C(0);
    neq[8] = C(0);
    qm[0] = s.q;
    qm[1] = k.g1 * s.q;
    qm[2] = k.g2 * s.q;
    qm[3] = s.q * ux;
    qm[4] = -s.q * ux;
    qm[5] = s.q * uy;
    qm[6] = -s.q * uy;
    qm[7] = C(0);
    qm[8] = C(0);
}

// The collision of both DFs at one node (Eq. 12b, 12c). On entry s holds
// the moments of the pulled populations; on exit f, g hold the post-
// collision populations. Rows 0, 3, 5 of m - m^eq + dt/2 F_m and row 0 of
// n - n^eq + dt/2 q_m vanish by Eq. 14, so s_0, s_j and sigma_0 never act
// and are not applied.
// SH: on exit f and g hold the post-collision deviations from the rest
// populations (the rest moments are taken off before the back-transform).
// CUBIC: the cubic-term elimination: q_x, q_y equilibria with 3 rho u_x u_y^2,
// 3 rho u_y u_x^2, and the source R7 = -c (d_x(rho u_x^3) - d_y(rho u_y^3))
// in the p_xx row as dt (1 - s_p/2) R7 (R has no other component, and no
// other row of S reads column p_xx).
template <bool SH = false, bool CUBIC = false, class C, class K>
__device__ __forceinline__ void collide(const K& k, C f[9], C g[9], const NodeMacro<C>& s, C R7 = C(0)) {
    const C rho = s.rho, ux = s.uhx, uy = s.uhy;
    const C u2 = ux * ux + uy * uy;
    const C pbe = p_BE(k, rho, s.T);
    const C eta = pbe * k.cs2_inv - rho;
    const C rhk = s.rek + pbe;
    const C Fx = s.Fhx, Fy = s.Fhy;
    const C FU = Fx * ux + Fy * uy;
    const C* m = s.m;
    const C* n = s.n;

    // ---- f: m_bar = m + dt F_m - S (m - m^eq + dt/2 F_m - Q_m) -----------
    const C r3u2 = C(3) * rho * u2;
    const C meq1 = C(-2) * rho + C(2) * eta + r3u2;
    const C meq2 = rho + k.beta * eta - r3u2;
    const C meq7 = rho * (ux * ux - uy * uy);
    const C meq8 = rho * ux * uy;
    const C Fm1 = C(6) * FU, Fm7 = C(2) * (Fx * ux - Fy * uy), Fm8 = Fx * uy + Fy * ux;
    // Q_m of SM Eq. S6a with grad rho = F_pair / (G^2 rho)
    const C Q1 = k.six_qc * (s.gx * s.gx + s.gy * s.gy);
    const C Q7 = k.qc * (s.gx * s.gx - s.gy * s.gy);
    const C Q8 = k.qc * s.gx * s.gy;
    const C w1 = m[1] - meq1 + k.half_dt * Fm1 - Q1;
    const C w2 = m[2] - meq2 - k.half_dt * Fm1 + Q1;
    C w4 = m[4] + rho * ux - k.half_dt * Fx;
    C w6 = m[6] + rho * uy - k.half_dt * Fy;
    if constexpr (CUBIC) {
        w4 -= C(3) * rho * ux * uy * uy;
        w6 -= C(3) * rho * uy * ux * ux;
    }
    const C w7 = m[7] - meq7 + k.half_dt * Fm7 - Q7;
    const C w8 = m[8] - meq8 + k.half_dt * Fm8 - Q8;
    // S of SM Eq. S5a; omega_e = s_e/2 - 1, omega_p = s_p/2 - 1
    const C sqw4 = k.sq * w4, sqw6 = k.sq * w6;
    const C Sw1 = k.se * w1 + k.we_kS_seps * w2 + k.we_hS * (ux * sqw4 + uy * sqw6);
    const C Sw7 = k.sp * w7 + k.wp_bS * (C(2) * (ux * sqw4 - uy * sqw6));
    const C Sw8 = k.sp * w8 + k.wp_bS * (uy * sqw4 + ux * sqw6);
    C mb[9];
    mb[0] = m[0];
    mb[1] = m[1] + k.dt * Fm1 - Sw1;
    mb[2] = m[2] - k.dt * Fm1 - k.seps * w2;
    mb[3] = m[3] + k.dt * Fx;
    mb[4] = m[4] - k.dt * Fx - sqw4;
    mb[5] = m[5] + k.dt * Fy;
    mb[6] = m[6] - k.dt * Fy - sqw6;
    mb[7] = m[7] + k.dt * Fm7 - Sw7;
    if constexpr (CUBIC) mb[7] += k.dt * (R7 - C(0.5) * k.sp * R7);
    mb[8] = m[8] + k.dt * Fm8 - Sw8;
    // viscous-dissipation input of Eq. 12c: (m + m_bar)/2 - m^eq, columns e, pxx, pxy
    const C d1 = C(0.5) * (m[1] + mb[1]) - meq1;
    const C d7 = C(0.5) * (m[7] + mb[7]) - meq7;
    const C d8 = C(0.5) * (m[8] + mb[8]) - meq8;
    if constexpr (SH) {
#pragma unroll
        for (int q = 0; q < 3; ++q) mb[q] -= k.mrest[q];
    }
    populations9(mb, f);
    if constexpr (!SH) rest_as_complement(mb[0], f);

    // ---- g: n_bar = n + dt q_m - L (n - n^eq + dt/2 q_m) + c^2 Y d -------
    const C E = s.rek, T = s.T, q = s.q;
    const C z1 = n[1] + C(4) * E - k.c4g1_Cref * T + k.hdt_g1 * q;
    const C z2 = n[2] - C(4) * E + k.c4g2_Cref * T + k.hdt_g2 * q;
    const C qux = q * ux, quy = q * uy;
    const C z3 = n[3] - rhk * ux + k.half_dt * qux;
    const C z4 = n[4] + rhk * ux - k.half_dt * qux;
    const C z5 = n[5] - rhk * uy + k.half_dt * quy;
    const C z6 = n[6] + rhk * uy - k.half_dt * quy;
    // sigma_j(rho): tau_j linear in rho between rho_v and rho_l; sigma_q = sigma_j
    const C wl = clamp01((rho - k.rho_v) * k.inv_drho);
    const C sj = recip(k.tauj_v + k.dtauj * wl + C(0.5));
    const C sjwj = sj * (C(0.5) * sj - C(1));   // sigma_q omega_j with sigma_q = sigma_j
    // c^2 Y d of SM Eq. S6b
    const C yx = k.c2_third * ux * d1 + k.c2 * (ux * d7 + C(2) * uy * d8);
    const C yy = k.c2_third * uy * d1 + k.c2 * (C(2) * ux * d8 - uy * d7);
    C nb[9];
    nb[0] = n[0] + k.dt * q;
    nb[1] = n[1] + k.dt_g1 * q - k.sige * z1;
    nb[2] = n[2] + k.dt_g2 * q - k.sigeps * z2;
    nb[3] = n[3] + k.dt * qux - (sj * z3 + sjwj * z4) + yx;
    nb[4] = n[4] - k.dt * qux - sj * z4 - yx;
    nb[5] = n[5] + k.dt * quy - (sj * z5 + sjwj * z6) + yy;
    nb[6] = n[6] - k.dt * quy - sj * z6 - yy;
    nb[7] = n[7] - k.sigp * n[7];
    nb[8] = n[8] - k.sigp * n[8];
    if constexpr (SH) {
#pragma unroll
        for (int q = 0; q < 3; ++q) nb[q] -= k.nrest[q];
    }
    populations9(nb, g);
    if constexpr (!SH) rest_as_complement(nb[0], g);
}

// Rest equilibrium of g for a fixed-temperature wall: M^-1 n^eq(rho_w c_v T_w,
// T_w, u = 0); returns the axis and diagonal populations (equal by symmetry).
template <class C>
__device__ __forceinline__ void g_rest_wall(const KC<C>& k, C rho_w, C T_w, C& g_axis, C& g_diag) {
    const C E = rho_w * k.cv * T_w, CT = k.Cref * T_w;
    const C n1 = C(-4) * E + (C(4) + k.g1) * CT;
    const C n2 = C(4) * E - (C(4) - k.g2) * CT;
    const C a0 = E * C(1.0 / 9.0), a1 = n1 * C(1.0 / 36.0), a2 = n2 * C(1.0 / 36.0);
    g_axis = a0 - a1 - C(2) * a2;
    g_diag = a0 + C(2) * a1 + a2;
}

// Store one post-collision value at physical (x, y) of plane p, with the
// copies the periodic ghost cells need. y may be -1 or ny for a wall ghost,
// and, with open left and right sides, x may be -1 or nx. XOPEN = false:
// the caller knows that x is periodic.
template <class S, bool XOPEN = true>
__device__ __forceinline__ void put(S* __restrict__ out, const Geometry& G, int p, int x, int y, S v) {
    S* base = out + (long long)p * G.plane;
    int rows[2];
    int nr = 1;
    rows[0] = y;
    if (!G.walls) {
        if (y < 2) rows[nr++] = y + G.ny;
        else if (y >= G.ny - 2) rows[nr++] = y - G.ny;
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r >= nr) break;
        S* row = base + (long long)(rows[r] + 2) * G.pitch + G.PX;
        row[x] = v;
        if (!(XOPEN && (G.open & 12))) {
            if (x < GHOST_COLS) row[x + G.nx] = v;
            if (x >= G.nx - GHOST_COLS) row[x - G.nx] = v;
        }
    }
}

// Equilibrium populations M^-1 m^eq and M^-1 n^eq (SM Eq. S3a, S4a) of the
// force-free state (rho, u^ = u / c, T), with rho e_k = rho c_v T +
// rho |u|^2 / 2.
template <class C>
__device__ __forceinline__ void eq_pops(const KC<C>& k, C rho, C ux, C uy, C T, C fe[9], C ge[9]) {
    const C u2 = ux * ux + uy * uy;
    const C pbe = p_BE(k, rho, T);
    const C eta = pbe * k.cs2_inv - rho;
    const C E = rho * k.cv * T + C(0.5) * k.c2 * rho * u2;
    const C rhk = E + pbe;
    const C CT = k.Cref * T;
    C m[9], n[9];
    m[0] = rho;
    m[1] = C(-2) * rho + C(2) * eta + C(3) * rho * u2;
    m[2] = rho + k.beta * eta - C(3) * rho * u2;
    m[3] = rho * ux;
    m[4] = -rho * ux;
    m[5] = rho * uy;
    m[6] = -rho * uy;
    m[7] = rho * (ux * ux - uy * uy);
    m[8] = rho * ux * uy;
    n[0] = E;
    n[1] = C(-4) * E + (C(4) + k.g1) * CT;
    n[2] = C(4) * E - (C(4) - k.g2) * CT;
    n[3] = rhk * ux;
    n[4] = -rhk * ux;
    n[5] = rhk * uy;
    n[6] = -rhk * uy;
    n[7] = C(0);
    n[8] = C(0);
    populations9(m, fe);
    populations9(n, ge);
}

// Ghost populations beyond the open sides next to node (x, y): every ghost
// node whose nearest fluid node is (x, y) -- the one across each open side
// the node touches, and the corner between two -- carries the node's
// post-collision populations f, g (for shifted formats, their deviations
// from the rest populations) with the equilibrium part moved from the
// node's state (rho, u^, T) to the open state (rho_open, u^, T_open)
// (non-equilibrium extrapolation), and streams into the lattice the
// directions that point back across the open sides.
// (f and g come as the nine values each so that the caller's arrays stay in
// registers on the path that does not call this.)
template <class C>
struct Pops9 {
    C v[9];
};
template <class S, class C>
__device__ __noinline__ void open_store(S* __restrict__ out, const Geometry& G, const KC<C>& k, int x, int y,
                                        const Pops9<C> f, const Pops9<C> g, C rho, C ux, C uy, C T) {
    C fe[9], ge[9], fo[9], go[9];
    eq_pops(k, rho, ux, uy, T, fe, ge);
    eq_pops(k, k.rho_open, ux, uy, k.T_open, fo, go);
    // e_i / c of D2Q9 (SM Eq. S1); the loops are unrolled so that the choice of
    // directions per ghost is made at compile time and the arrays stay in
    // registers
    constexpr int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;  // the node itself is not a ghost
            const int gx = x + dx, gy = y + dy;
            const bool ox = beyond_open(G, gx, y), oy = beyond_open(G, x, gy);
            if (!(ox || oy) || (dx != 0 && !ox) || (dy != 0 && !oy)) continue;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if ((dx != 0 && ex[i] != -dx) || (dy != 0 && ey[i] != -dy)) continue;
                if (beyond_open(G, gx + ex[i], gy + ey[i])) continue;
                put<S>(out, G, i, gx, gy, Store<S, C>::cvt(f.v[i] + fo[i] - fe[i]));
                put<S>(out, G, 9 + i, gx, gy, Store<S, C>::cvt(g.v[i] + go[i] - ge[i]));
            }
        }
}

}  // namespace lbm
