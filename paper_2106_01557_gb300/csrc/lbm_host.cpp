// Host runtime of liblbm: configuration checks, parameter derivation
// (Eq. 16-19 and the Maxwell coexistence of Eq. 17), device buffers and
// TMA descriptors, the step loop (CUDA graphs of step pairs), and the C ABI
// declared in include/lbm.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_batch.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Thermodynamics of Eq. 17 (per unit K_EOS): p(rho) and the chemical
// potential mu(rho) = d psi / d rho of the Carnahan-Starling free energy.
// ---------------------------------------------------------------------------
struct Eos {
    double a, b, R, T;
    double p(double r) const {
        const double t = 0.25 * b * r, o = 1.0 - t;
        return r * R * T * (1.0 + t + t * t - t * t * t) / (o * o * o) - a * r * r;
    }
    double dp(double r) const {
        const double t = 0.25 * b * r, o = 1.0 - t;
        return R * T * (1.0 + 4.0 * t + 4.0 * t * t - 4.0 * t * t * t + t * t * t * t) / (o * o * o * o) - 2.0 * a * r;
    }
    double mu(double r) const {
        const double t = 0.25 * b * r, o = 1.0 - t;
        return R * T * (std::log(r) + (4.0 * t - 3.0 * t * t) / (o * o) + t * (4.0 - 2.0 * t) / (o * o * o)) -
               2.0 * a * r;
    }
};

template <class F>
double bisect(F fn, double lo, double hi, int iters = 200) {
    double flo = fn(lo);
    for (int k = 0; k < iters; ++k) {
        const double mid = 0.5 * (lo + hi);
        const double fm = fn(mid);
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; }
        else hi = mid;
        if (hi - lo <= 1e-17 * std::fabs(hi)) break;
    }
    return 0.5 * (lo + hi);
}

// Coexistence by a different route from a pressure bisection: bisect on the
// vapour density rho_v in (0, spinodal_v); for each candidate the liquid
// branch density with the same pressure is found and the chemical-potential
// mismatch is the bisection function. Then two Newton polish steps on the
// 2x2 system p(rl) = p(rv), mu(rl) = mu(rv).
bool maxwell(const Eos& e, double* rv_out, double* rl_out, double* ps_out) {
    const double rmax = 4.0 / e.b;
    // spinodals: dp = 0 on either side of the minimum of dp
    double rmin = 0.0, dmin = 1e300;
    for (int k = 1; k < 4000; ++k) {
        const double r = rmax * k / 4000.0;
        const double d = e.dp(r);
        if (d < dmin) { dmin = d; rmin = r; }
    }
    if (!(dmin < 0.0)) return false;
    const double s1 = bisect([&](double r) { return e.dp(r); }, 1e-12 * rmax, rmin);
    const double s2 = bisect([&](double r) { return e.dp(r); }, rmin, rmax * 0.9999);
    const double p_s2 = e.p(s2);
    auto liquid_at = [&](double ps) {
        double hi = s2;
        while (e.p(hi) < ps) hi = hi + 0.5 * (rmax - hi);
        return bisect([&](double r) { return e.p(r) - ps; }, s2, hi);
    };
    // lowest admissible vapour density: its pressure must reach the liquid branch
    double lo_v = 1e-14 * rmax;
    if (p_s2 > 0.0) lo_v = bisect([&](double r) { return e.p(r) - p_s2; }, 1e-14 * rmax, s1);
    auto mismatch = [&](double rv) { return e.mu(liquid_at(e.p(rv))) - e.mu(rv); };
    const double lo = lo_v * (1.0 + 1e-12), hi = s1 * (1.0 - 1e-12);
    if ((mismatch(lo) > 0) == (mismatch(hi) > 0)) return false;
    double rv = bisect(mismatch, lo, hi, 300);
    double rl = liquid_at(e.p(rv));
    for (int it = 0; it < 2; ++it) {
        // Newton: unknowns (rv, rl); F1 = p(rl) - p(rv), F2 = mu(rl) - mu(rv);
        // d mu / d rho = (dp / d rho) / rho
        const double F1 = e.p(rl) - e.p(rv), F2 = e.mu(rl) - e.mu(rv);
        const double a11 = -e.dp(rv), a12 = e.dp(rl);
        const double a21 = -e.dp(rv) / rv, a22 = e.dp(rl) / rl;
        const double det = a11 * a22 - a12 * a21;
        if (!(std::fabs(det) > 0)) break;
        const double dv = (-F1 * a22 + F2 * a12) / det;
        const double dl = (-a11 * F2 + a21 * F1) / det;
        if (!std::isfinite(dv) || !std::isfinite(dl)) break;
        rv += dv;
        rl += dl;
    }
    *rv_out = rv;
    *rl_out = rl;
    *ps_out = e.p(rv);
    return rv > 0 && rl > rv;
}

// Coexistence across a curved interface at temperature T: mu(rho_v) =
// mu(rho_l) and K_EOS (p(rho_l) - p(rho_v)) = dp (Laplace's law, dp = sigma
// / R in 2-D), by Newton's method from the flat (Maxwell) pair.
bool shifted_coexistence(const Eos& e, double K, double dp, double* rv, double* rl, double* pv) {
    double ps;
    if (!maxwell(e, rv, rl, &ps)) return false;
    for (int it = 0; it < 50 && dp != 0.0; ++it) {
        const double F1 = K * (e.p(*rl) - e.p(*rv)) - dp, F2 = e.mu(*rl) - e.mu(*rv);
        const double a11 = -K * e.dp(*rv), a12 = K * e.dp(*rl);
        const double a21 = -e.dp(*rv) / *rv, a22 = e.dp(*rl) / *rl;
        const double det = a11 * a22 - a12 * a21;
        if (!(std::fabs(det) > 0)) return false;
        const double dv = (-F1 * a22 + F2 * a12) / det;
        const double dl = (-a11 * F2 + a21 * F1) / det;
        if (!std::isfinite(dv) || !std::isfinite(dl)) return false;
        *rv += dv;
        *rl += dl;
        if (std::fabs(dv) <= 1e-15 * *rv && std::fabs(dl) <= 1e-15 * *rl) break;
    }
    *pv = K * e.p(*rv);
    return *rv > 0 && *rl > *rv;
}

int storage_of(int precision) {
    switch (precision) {
        case LBM_F64: return S_F64;
        case LBM_F32: return S_F32;
        case LBM_F16S: return S_F16;
        case LBM_BF16S: return S_BF16;
    }
    return -1;
}

size_t elem_size(int storage) { return storage == S_F64 ? 8 : (storage == S_F32 ? 4 : 2); }

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

}  // namespace

struct lbm_handle {
    lbm_config cfg;
    lbm_params prm;
    Launch L;
    int storage;
    size_t esize;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;  // index of the buffer holding the current state
    CUtensorMap tmf[2], tmg[2];
    double* partials = nullptr;  // step_blocks x NQ
    double* stats = nullptr;     // NQ (step) + NQ (moments)
    unsigned* counter = nullptr; // 2 counters
    int* status = nullptr;
    double* scratch = nullptr;   // 9 * 2 * n doubles (populations / fields)
    size_t scratch_elems = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;  // GRAPH_STEPS steps starting from buffer 0
    int64_t steps = 0;
    static constexpr int GRAPH_STEPS = 20;  // even: the graph returns to buffer 0
};

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

void lbm_default_config(lbm_config* c, int32_t nx, int32_t ny) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->nx = nx;
    c->ny = ny;
    c->precision = LBM_F32;
    c->walls = 0;
    c->a_t = 1.0;
    c->b_t = 4.0;
    c->R = 1.0;
    c->K_EOS = 0.479820;
    c->K_INT = 2.294922;
    c->Tr0 = 0.8;
    c->varpi = 1.0 / 6.0;
    c->gamma1 = -2.0;
    c->gamma2 = 2.0;
    c->s_p = 1.0;
    c->s_eps = 1.0;
    c->sig_e = 1.0;
    c->sig_eps = 1.0;
    c->sig_p = 1.0;
    c->tau_j_v = 0.25;
    c->tau_j_l = 2.5;
    c->c_v = 1.5;
    c->C_ref = 0.0;
    c->rho_ref = 0.0;
    c->stream = nullptr;
    c->device = 0;
    c->rounding = 1;
}

static int derive(const lbm_config& c, lbm_params& p, Launch& L) {
    auto in01 = [](double s) { return s > 0.0 && s < 2.0; };
    if (c.nx < 8 || c.ny < 8) return fail(LBM_ERR_ARG, "nx and ny must be >= 8");
    if ((long long)c.nx * c.ny > (1ll << 31)) return fail(LBM_ERR_ARG, "lattice too large");
    if (storage_of(c.precision) < 0) return fail(LBM_ERR_ARG, "unknown precision");
    if (c.walls != 0 && c.walls != 1) return fail(LBM_ERR_ARG, "walls must be 0 or 1");
    if (c.rounding != 0 && c.rounding != 1) return fail(LBM_ERR_ARG, "rounding must be 0 or 1");
    L.rounding = c.rounding;
    L.tile_wait_ns = TILE_WAIT_NS_DEFAULT;
    if (!(c.a_t > 0 && c.b_t > 0 && c.R > 0 && c.K_EOS > 0 && c.K_INT > 0))
        return fail(LBM_ERR_ARG, "a~, b~, R, K_EOS, K_INT must be positive");
    if (!(c.Tr0 > 0.3 && c.Tr0 < 1.0)) return fail(LBM_ERR_ARG, "Tr0 must lie in (0.3, 1)");
    if (!(c.varpi > 0 && c.varpi < 1.0 / 3.0)) return fail(LBM_ERR_ARG, "varpi must lie in (0, 1/3)");
    if (!in01(c.s_p) || !in01(c.s_eps) || !in01(c.sig_e) || !in01(c.sig_eps) || !in01(c.sig_p))
        return fail(LBM_ERR_ARG, "relaxation rates must lie in (0, 2)");
    if (!(c.tau_j_v > 0 && c.tau_j_l > 0)) return fail(LBM_ERR_ARG, "tau_j must be positive");
    if (!(c.c_v > 0)) return fail(LBM_ERR_ARG, "c_v must be positive");
    if (c.hot_len < 0 || c.hot_len > c.nx) return fail(LBM_ERR_ARG, "hot_len out of range");
    if (!std::isfinite(c.accel_x) || !std::isfinite(c.accel_y)) return fail(LBM_ERR_ARG, "non-finite acceleration");
    if (c.open_sides < 0 || c.open_sides > 15) return fail(LBM_ERR_ARG, "open_sides must lie in 0..15");
    if ((c.open_sides & 3) && c.walls != 1) return fail(LBM_ERR_ARG, "an open bottom or top needs walls = 1");
    if ((c.open_sides & 12) && c.open_sides != 15)
        return fail(LBM_ERR_ARG, "open left and right sides come only with all four sides open");
    if (c.open_sides && !(c.Tr_open > 0)) return fail(LBM_ERR_ARG, "open sides need Tr_open > 0");
    if (c.cubic != 0 && c.cubic != 1) return fail(LBM_ERR_ARG, "cubic must be 0 or 1");
    if (c.cubic && (c.walls || c.open_sides))
        return fail(LBM_ERR_ARG, "the cubic-term elimination is built for periodic boxes only");
    L.cubic = c.cubic;

    // Eq. 17: a~ = A R^2 Tc^2 / pc, b~ = B R Tc / pc
    const double A = 0.4963880577294099, B = 0.1872945669467330;
    p.Tc = (B / A) * c.a_t / (c.b_t * c.R);
    p.pc = B * c.R * p.Tc / c.b_t;
    p.T0 = c.Tr0 * p.Tc;
    Eos e{c.a_t, c.b_t, c.R, p.T0};
    double ps;
    if (!maxwell(e, &p.rho_v, &p.rho_l, &ps)) return fail(LBM_ERR_ARG, "no liquid-vapour coexistence at Tr0");
    p.p_s = c.K_EOS * ps;
    // the open sides' density: the vapour branch of Eq. 17 at their own
    // temperature and the saturation pressure at Tr0
    double rho_open = c.rho_open;
    if (c.open_sides && !(rho_open > 0)) {
        Eos eo{c.a_t, c.b_t, c.R, c.Tr_open * p.Tc};
        const double rmax = 4.0 / c.b_t;
        // the vapour branch ends at the first maximum of p (or, above the
        // critical temperature, p is monotonic): scan for where dp turns negative
        double hi = rmax * 0.9999;
        for (int k = 1; k < 4000; ++k) {
            const double r = rmax * k / 4000.0;
            if (eo.dp(r) < 0.0) { hi = r; break; }
        }
        hi = bisect([&](double r) { return eo.dp(r); }, 1e-12 * rmax, hi);
        if (!(eo.p(hi) > ps)) return fail(LBM_ERR_ARG, "no vapour at Tr_open with the saturation pressure at Tr0");
        rho_open = bisect([&](double r) { return eo.p(r) - ps; }, 1e-14 * rmax, hi);
    }
    p.rho_open = c.open_sides ? rho_open : 0.0;
    p.T_open = c.open_sides ? c.Tr_open * p.Tc : 0.0;
    // Eq. 18, 19 (dx = 1): c_s^2 = K_INT^2 (dp_EOS/drho + 2 K_EOS a~ rho) at rho_l
    p.G2 = c.K_INT * c.K_INT * 2.0 * c.K_EOS * c.a_t;
    const double cs2 = c.K_INT * c.K_INT * (c.K_EOS * e.dp(p.rho_l) + 2.0 * c.K_EOS * c.a_t * p.rho_l);
    if (!(cs2 > 0)) return fail(LBM_ERR_ARG, "non-positive sound speed");
    p.cs = std::sqrt(cs2);
    p.c = std::sqrt(3.0) * p.cs;
    p.dt = 1.0 / p.c;
    p.a = 0.5 * p.G2;      // Eq. 16
    p.kappa = 0.25 * p.G2;
    p.cv = c.c_v * c.R;
    p.Cref = c.C_ref > 0 ? c.C_ref : p.rho_v * p.cv;
    const double w = c.varpi;
    p.kS = 1.0 - w;
    p.hS = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w);
    p.bS = (1.0 - w) / (1.0 - 3.0 * w);
    p.beta = -2.0 / (1.0 - w);
    const double tau_p = 1.0 / c.s_p - 0.5;
    const double tau_q = 1.0 / (12.0 * tau_p);
    const double tau_e = tau_p / (p.kS + 1.0);
    p.sq = 1.0 / (tau_q + 0.5);
    p.se = 1.0 / (tau_e + 0.5);
    if (!in01(p.sq) || !in01(p.se)) return fail(LBM_ERR_ARG, "s_p gives s_q or s_e outside (0, 2)");

    Geometry& G = L.geo;
    const int storage = storage_of(c.precision);
    int bx, by, hx;
    step_tile(storage, &bx, &by, &hx);
    G.nx = c.nx;
    G.ny = c.ny;
    G.walls = c.walls;
    G.HX = hx;
    const int line = 128 / (int)elem_size(storage);  // elements per 128 bytes
    G.PX = line;
    int pitch = G.PX + (c.nx > bx ? c.nx : bx) + hx;
    pitch = ((pitch + line - 1) / line) * line;
    G.pitch = pitch;
    G.nyp = c.ny + 4 > by + 4 ? c.ny + 4 : by + 4;
    G.plane = (long long)G.pitch * G.nyp;
    G.hot_x0 = ((c.hot_x0 % c.nx) + c.nx) % c.nx;
    G.hot_len = c.hot_len;
    G.open = c.open_sides;

    auto fill = [&](auto& k, auto cast) {
        k.c = cast(p.c);
        k.c2 = cast(p.c * p.c);
        k.dt = cast(p.dt);
        k.half_dt = cast(0.5 * p.dt);
        k.G2c = cast(p.G2 / p.c);
        k.axc = cast(c.accel_x / p.c);
        k.ayc = cast(c.accel_y / p.c);
        k.a = cast(p.a);
        k.half_kappa = cast(0.5 * p.kappa);
        k.cs2_inv = cast(1.0 / cs2);
        k.RK = cast(c.R * c.K_EOS);
        k.aK_eff = cast(p.a - c.a_t * c.K_EOS);
        k.b4 = cast(0.25 * c.b_t);
        k.inv_cv = cast(1.0 / p.cv);
        k.cv = cast(p.cv);
        k.Cref = cast(p.Cref);
        k.g1 = cast(c.gamma1);
        k.g2 = cast(c.gamma2);
        k.beta = cast(p.beta);
        k.kS = cast(p.kS);
        k.hS = cast(p.hS);
        k.bS = cast(p.bS);
        k.se = cast(p.se);
        k.seps = cast(c.s_eps);
        k.sq = cast(p.sq);
        k.sp = cast(c.s_p);
        k.sige = cast(c.sig_e);
        k.sigeps = cast(c.sig_eps);
        k.sigp = cast(c.sig_p);
        k.tauj_v = cast(c.tau_j_v);
        k.dtauj = cast(c.tau_j_l - c.tau_j_v);
        k.rho_v = cast(p.rho_v);
        k.inv_drho = cast(1.0 / (p.rho_l - p.rho_v));
        k.qc = cast(p.G2 * p.dt * p.dt / 12.0);
        k.we_kS_seps = cast((0.5 * p.se - 1.0) * p.kS * c.s_eps);
        k.we_hS = cast((0.5 * p.se - 1.0) * p.hS);
        k.wp_bS = cast((0.5 * c.s_p - 1.0) * p.bS);
        k.six_qc = cast(6.0 * p.G2 * p.dt * p.dt / 12.0);
        k.dt_g1 = cast(p.dt * c.gamma1);
        k.dt_g2 = cast(p.dt * c.gamma2);
        k.hdt_g1 = cast(0.5 * p.dt * c.gamma1);
        k.hdt_g2 = cast(0.5 * p.dt * c.gamma2);
        k.c4g1_Cref = cast((4.0 + c.gamma1) * p.Cref);
        k.c4g2_Cref = cast((4.0 - c.gamma2) * p.Cref);
        k.c2_third = cast(p.c * p.c / 3.0);
        k.T_bottom = cast(c.Tr_bottom > 0 ? c.Tr_bottom * p.Tc : 0.0);
        k.T_top = cast(c.Tr_top > 0 ? c.Tr_top * p.Tc : 0.0);
        k.T_hot = cast(c.Tr_hot > 0 ? c.Tr_hot * p.Tc : 0.0);
        k.rho_open = cast(c.open_sides ? rho_open : 0.0);
        k.T_open = cast(c.open_sides ? c.Tr_open * p.Tc : 0.0);
    };
    fill(L.kd, [](double v) { return v; });
    fill(L.kf, [](double v) { return (float)v; });
    if (c.hot_len > 0 && !(c.Tr_hot > 0)) return fail(LBM_ERR_ARG, "hot segment needs Tr_hot > 0");

    // Rest populations of the shifted formats: M^-1 m^eq and M^-1 n^eq at
    // (rho_ref, T0, u = 0), evaluated in FP64 then rounded to FP32 once. The
    // default rho_ref = rho_v keeps the stored deviations of vapour nodes
    // near zero; liquid nodes then carry deviations of their own size, so
    // both phases keep the format's relative precision.
    for (int i = 0; i < 18; ++i) { L.kf.rest[i] = 0.0f; L.kd.rest[i] = 0.0; }
    for (int q = 0; q < 3; ++q) { L.kf.mrest[q] = L.kf.nrest[q] = 0.0f; L.kd.mrest[q] = L.kd.nrest[q] = 0.0; }
    if (storage == S_F16 || storage == S_BF16) {
        const double rho = c.rho_ref > 0 ? c.rho_ref : p.rho_v;
        const double T = p.T0;
        const double th = 0.25 * c.b_t * rho, om = 1.0 - th;
        const double pbe = c.R * c.K_EOS * rho * T * (1.0 + th + th * th - th * th * th) / (om * om * om) +
                           (p.a - c.a_t * c.K_EOS) * rho * rho;
        const double eta = pbe / cs2 - rho;
        const double m0 = rho, m1 = -2.0 * rho + 2.0 * eta, m2 = rho + p.beta * eta;
        const double E = rho * p.cv * T, CT = p.Cref * T;
        const double n0 = E, n1 = -4.0 * E + (4.0 + c.gamma1) * CT, n2 = 4.0 * E - (4.0 - c.gamma2) * CT;
        auto rest = [](double a, double b, double cc, double* out) {
            const double a0 = a / 9.0, a1 = b / 36.0, a2 = cc / 36.0;
            out[0] = a0 - 4 * a1 + 4 * a2;
            for (int i = 1; i <= 4; ++i) out[i] = a0 - a1 - 2 * a2;
            for (int i = 5; i <= 8; ++i) out[i] = a0 + 2 * a1 + a2;
        };
        double rf[9], rg[9];
        rest(m0, m1, m2, rf);
        rest(n0, n1, n2, rg);
        for (int i = 0; i < 9; ++i) {
            L.kf.rest[i] = (float)rf[i];
            L.kf.rest[9 + i] = (float)rg[i];
            L.kd.rest[i] = (double)L.kf.rest[i];
            L.kd.rest[9 + i] = (double)L.kf.rest[9 + i];
        }
        // moments 0-2 of the rounded rest populations (M of SM Eq. S2); the
        // rest state has u = 0, so moments 3-8 vanish exactly (equal axis and
        // equal diagonal populations)
        auto m012 = [](const float* r, double* m) {
            const double ax = (double)r[1] + r[2] + r[3] + r[4], dg = (double)r[5] + r[6] + r[7] + r[8];
            m[0] = r[0] + ax + dg;
            m[1] = -4.0 * r[0] - ax + 2.0 * dg;
            m[2] = 4.0 * r[0] - 2.0 * ax + dg;
        };
        double mf[3], mg[3];
        m012(L.kf.rest, mf);
        m012(L.kf.rest + 9, mg);
        for (int q = 0; q < 3; ++q) {
            L.kf.mrest[q] = (float)mf[q];
            L.kf.nrest[q] = (float)mg[q];
            L.kd.mrest[q] = mf[q];
            L.kd.nrest[q] = mg[q];
        }
    }
    return LBM_OK;
}

static int make_maps(lbm_handle* h) {
    EncodeTiled enc = get_encoder();
    if (!enc) return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    const Geometry& G = h->L.geo;
    int bx, by, hx;
    step_tile(h->storage, &bx, &by, &hx);
    CUtensorMapDataType dt = h->storage == S_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                             : h->storage == S_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : h->storage == S_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // map x = 0 is the first ghost column (row element PX - HX, 16-byte aligned);
    // the map ends after the right ghost block, so that a box reaching into
    // the row padding reads the out-of-bounds fill instead of memory
    const int x0 = G.PX - G.HX;
    cuuint64_t dims[3] = {(cuuint64_t)((G.nx > bx ? G.nx : bx) + 2 * G.HX), (cuuint64_t)G.nyp, 18};
    cuuint64_t strides[2] = {(cuuint64_t)G.pitch * h->esize, (cuuint64_t)G.plane * h->esize};
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t boxf[3] = {(cuuint32_t)(bx + 2 * hx), (cuuint32_t)(by + 4), 9};
    cuuint32_t boxg[3] = {(cuuint32_t)(bx + 2 * hx), (cuuint32_t)(by + 2), 9};
    for (int b = 0; b < 2; ++b) {
        void* base = static_cast<unsigned char*>(h->buf[b]) + (size_t)x0 * h->esize;
        CUresult r1 = enc(&h->tmf[b], dt, 3, base, dims, strides, boxf, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r2 = enc(&h->tmg[b], dt, 3, base, dims, strides, boxg, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS)
            return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r1) + "/" +
                                          std::to_string((int)r2) + ")");
    }
    return LBM_OK;
}

static void release(lbm_handle* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    if (h->partials) cudaFree(h->partials);
    if (h->stats) cudaFree(h->stats);
    if (h->counter) cudaFree(h->counter);
    if (h->status) cudaFree(h->status);
    if (h->scratch) cudaFree(h->scratch);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int lbm_init(const lbm_config* cfg, lbm_handle** out) {
    if (!cfg || !out) return fail(LBM_ERR_ARG, "null argument");
    *out = nullptr;
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
    h->cfg = *cfg;
    int rc = derive(h->cfg, h->prm, h->L);
    if (rc) { delete h; return rc; }
    h->storage = storage_of(cfg->precision);
    h->esize = elem_size(h->storage);
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaSetDevice"); }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e != cudaSuccess || sms <= 0) { delete h; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    h->L.geo.sms = sms;
    if (cfg->stream) {
        h->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
        h->own_stream = true;
    }
    const Geometry& G = h->L.geo;
    const size_t bytes = (size_t)18 * G.plane * h->esize;
    const size_t n = (size_t)G.nx * G.ny;
    const int nb = std::max(step_blocks(h->storage, G), moments_blocks(G));
    h->scratch_elems = 18 * n;
    bool ok = cudaMalloc(&h->buf[0], bytes) == cudaSuccess && cudaMalloc(&h->buf[1], bytes) == cudaSuccess &&
              cudaMalloc(&h->partials, (size_t)nb * NQ * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->stats, 2 * NQ * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&h->counter, 2 * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&h->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->scratch, h->scratch_elems * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(h);
        delete h;
        return fail(LBM_ERR_OOM, "device allocation failed");
    }
    ok = cudaMemsetAsync(h->buf[0], 0, bytes, h->stream) == cudaSuccess &&
         cudaMemsetAsync(h->buf[1], 0, bytes, h->stream) == cudaSuccess &&
         cudaMemsetAsync(h->stats, 0, 2 * NQ * sizeof(double), h->stream) == cudaSuccess &&
         cudaMemsetAsync(h->counter, 0, 2 * sizeof(unsigned), h->stream) == cudaSuccess &&
         cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) == cudaSuccess &&
         cudaStreamSynchronize(h->stream) == cudaSuccess;
    if (!ok) { release(h); delete h; return fail(LBM_ERR_CUDA, "device initialisation failed"); }
    rc = make_maps(h);
    if (rc) { release(h); delete h; return rc; }
    e = prepare_step(h->storage);
    if (e != cudaSuccess) { release(h); delete h; return cuda_fail(e, "cudaFuncSetAttribute"); }
    *out = h;
    return LBM_OK;
}

int lbm_get_params(const lbm_handle* h, lbm_params* out) {
    if (!h || !out) return fail(LBM_ERR_ARG, "null argument");
    *out = h->prm;
    return LBM_OK;
}

int lbm_coexistence(const lbm_config* cfg, double Tr, double dp, double out[3]) {
    if (!cfg || !out) return fail(LBM_ERR_ARG, "null argument");
    if (!(Tr > 0.3 && Tr < 1.0)) return fail(LBM_ERR_ARG, "Tr must lie in (0.3, 1)");
    if (!std::isfinite(dp)) return fail(LBM_ERR_ARG, "non-finite pressure jump");
    const double A = 0.4963880577294099, B = 0.1872945669467330;
    const double Tc = (B / A) * cfg->a_t / (cfg->b_t * cfg->R);
    Eos e{cfg->a_t, cfg->b_t, cfg->R, Tr * Tc};
    if (!shifted_coexistence(e, cfg->K_EOS, dp, &out[0], &out[1], &out[2]))
        return fail(LBM_ERR_ARG, "no coexistence with this pressure jump at this temperature");
    return LBM_OK;
}

int lbm_surface_tension(const lbm_config* cfg, double Tr, double* sigma) {
    if (!cfg || !sigma) return fail(LBM_ERR_ARG, "null argument");
    if (!(Tr > 0.3 && Tr < 1.0)) return fail(LBM_ERR_ARG, "Tr must lie in (0.3, 1)");
    const double A = 0.4963880577294099, B = 0.1872945669467330;
    const double Tc = (B / A) * cfg->a_t / (cfg->b_t * cfg->R);
    const double T = Tr * Tc;
    Eos e{cfg->a_t, cfg->b_t, cfg->R, T};
    double rv, rl, ps;
    if (!maxwell(e, &rv, &rl, &ps)) return fail(LBM_ERR_ARG, "no coexistence at this temperature");
    // free energy density per unit K_EOS whose pressure rho psi' - psi is Eq.
    // 17's: psi = rho mu - p, mu from Eos::mu; the grand-potential excess
    // Omega = psi - mu_s rho + p_s vanishes at both coexistence densities
    const double mus = e.mu(rv);
    auto omega = [&](double r) {
        const double om = r * e.mu(r) - e.p(r) - mus * r + ps;
        return om > 0.0 ? om : 0.0;
    };
    // square-gradient coefficient of Eq. 11 and 16: kappa = G^2 / 4 (dx = 1)
    const double kappa = 0.25 * cfg->K_INT * cfg->K_INT * 2.0 * cfg->K_EOS * cfg->a_t;
    // sigma = int sqrt(2 kappa K_EOS Omega) drho over [rho_v, rho_l]:
    // 8-point Gauss-Legendre on 1,000 cells spaced closer at both ends
    static const double gx[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double gw[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    const int ncell = 1000;
    const double pi = 3.14159265358979323846;
    double s = 0.0;
    for (int j = 0; j < ncell; ++j) {
        const double lo = rv + (rl - rv) * 0.5 * (1.0 - std::cos(pi * j / ncell));
        const double hi = rv + (rl - rv) * 0.5 * (1.0 - std::cos(pi * (j + 1) / ncell));
        const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
        for (int q = 0; q < 4; ++q)
            s += half * gw[q] * (std::sqrt(2.0 * kappa * cfg->K_EOS * omega(mid - half * gx[q])) +
                                 std::sqrt(2.0 * kappa * cfg->K_EOS * omega(mid + half * gx[q])));
    }
    *sigma = s;
    return LBM_OK;
}

int lbm_eos_pressure(const lbm_config* cfg, double rho, double T, double* p) {
    if (!cfg || !p) return fail(LBM_ERR_ARG, "null argument");
    if (!(rho > 0.0 && rho < 4.0 / cfg->b_t) || !std::isfinite(T))
        return fail(LBM_ERR_ARG, "density outside (0, 4 / b) or non-finite temperature");
    Eos e{cfg->a_t, cfg->b_t, cfg->R, T};
    *p = cfg->K_EOS * e.p(rho);
    return LBM_OK;
}

int lbm_maxwell(const lbm_config* cfg, double Tr, double out[3]) {
    if (!cfg || !out) return fail(LBM_ERR_ARG, "null argument");
    if (!(Tr > 0.3 && Tr < 1.0)) return fail(LBM_ERR_ARG, "Tr must lie in (0.3, 1)");
    const double A = 0.4963880577294099, B = 0.1872945669467330;
    const double Tc = (B / A) * cfg->a_t / (cfg->b_t * cfg->R);
    Eos e{cfg->a_t, cfg->b_t, cfg->R, Tr * Tc};
    double ps;
    if (!maxwell(e, &out[0], &out[1], &ps)) return fail(LBM_ERR_ARG, "no coexistence at this temperature");
    out[2] = cfg->K_EOS * ps;
    return LBM_OK;
}

static int check_status(lbm_handle* h) {
    CK(cudaStreamSynchronize(h->stream));
    int st = 0;
    CK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(h->status, 0, sizeof(int)));
        if (st & ST_TIMEOUT) return fail(LBM_ERR_TIMEOUT, "a device-side wait exceeded its bound");
        if (st & ST_NONFINITE) return fail(LBM_ERR_DIVERGED, "non-finite or non-positive density or temperature");
    }
    return LBM_OK;
}

int lbm_synchronize(lbm_handle* h) {
    if (!h) return fail(LBM_ERR_ARG, "null handle");
    return check_status(h);
}

// Copy n doubles of a caller field into the scratch area (device), or
// use the caller's device pointer directly.
static const double* stage_in(lbm_handle* h, const double* src, size_t off, size_t n, int on_device,
                              cudaError_t* e) {
    if (on_device) return src;
    double* dst = h->scratch + off;
    *e = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    return dst;
}

int lbm_set_fields(lbm_handle* h, const double* rho, const double* ux, const double* uy, const double* T,
                   int on_device) {
    if (!h || !rho || !ux || !uy || !T) return fail(LBM_ERR_ARG, "null argument");
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    cudaError_t e = cudaSuccess;
    const double* d[4];
    const double* src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k) {
        d[k] = stage_in(h, src[k], k * n, n, on_device, &e);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    // The scatter writes every stored entry that a pull reads (including
    // ghost copies); clear first so the unread corners are defined too.
    const size_t bytes = (size_t)18 * h->L.geo.plane * h->esize;
    CK(cudaMemsetAsync(h->buf[0], 0, bytes, h->stream));
    // per-node arithmetic in the storage's compute type: FP64 for FP64
    // storage, FP32 otherwise (the stored values are FP32 or narrower)
    CK(launch_init(h->storage, h->L, d[0], d[1], d[2], d[3], h->buf[0], h->stream, h->storage != S_F64));
    h->cur = 0;
    return check_status(h);
}

int lbm_set_populations(lbm_handle* h, const double* f, const double* g) {
    if (!h || !f || !g) return fail(LBM_ERR_ARG, "null argument");
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    CK(cudaMemcpyAsync(h->scratch, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->scratch + 9 * n, g, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const size_t bytes = (size_t)18 * h->L.geo.plane * h->esize;
    CK(cudaMemsetAsync(h->buf[0], 0, bytes, h->stream));
    CK(launch_set_pops(h->storage, h->L, h->scratch, h->scratch + 9 * n, h->buf[0], h->stream));
    h->cur = 0;
    return check_status(h);
}

int lbm_get_populations(lbm_handle* h, double* f, double* g) {
    if (!h || !f || !g) return fail(LBM_ERR_ARG, "null argument");
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    CK(launch_get_pops(h->storage, h->L, h->buf[h->cur], h->scratch, h->scratch + 9 * n, h->stream));
    CK(cudaMemcpyAsync(f, h->scratch, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(g, h->scratch + 9 * n, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
}

static cudaError_t step_once(lbm_handle* h, int from) {
    const double* phi = nullptr;
    if (h->L.cubic) {
        // rho u^3 of the entering state, for the cubic-term source
        const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
        cudaError_t e = launch_cubic_phi(h->storage, h->L, h->buf[from], h->scratch, h->scratch + n, h->stream);
        if (e != cudaSuccess) return e;
        phi = h->scratch + n;
    }
    return launch_step(h->storage, h->L, &h->tmf[from], &h->tmg[from], h->buf[1 - from], h->partials, h->stats,
                       h->counter, h->status, h->stream, phi);
}

static int build_graph(lbm_handle* h) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < lbm_handle::GRAPH_STEPS && e == cudaSuccess; ++k) e = step_once(h, k & 1);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "step launch during capture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int n) {
    if (!h) return fail(LBM_ERR_ARG, "null handle");
    if (n < 0) return fail(LBM_ERR_ARG, "negative step count");
    while (n > 0) {
        if (h->cur == 0 && n >= lbm_handle::GRAPH_STEPS) {
            if (!h->graph) {
                int rc = build_graph(h);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(h->graph, h->stream));
            h->steps += lbm_handle::GRAPH_STEPS;
            n -= lbm_handle::GRAPH_STEPS;
            continue;
        }
        CK(step_once(h, h->cur));
        h->cur = 1 - h->cur;
        h->steps += 1;
        n -= 1;
    }
    return LBM_OK;
}

int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, double* T, int on_device) {
    if (!h) return fail(LBM_ERR_ARG, "null handle");
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    double* outs[4] = {rho, ux, uy, T};
    double* d[4];
    for (int k = 0; k < 4; ++k) d[k] = outs[k] ? (on_device ? outs[k] : h->scratch + (1 + k) * n) : nullptr;
    CK(launch_moments(h->storage, h->L, h->buf[h->cur], h->scratch, d[0], d[1], d[2], d[3], nullptr, nullptr,
                      nullptr, h->stream, h->storage != S_F64));
    if (!on_device)
        for (int k = 0; k < 4; ++k)
            if (outs[k]) CK(cudaMemcpyAsync(outs[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
}

int lbm_conservation(lbm_handle* h, double out[6]) {
    if (!h || !out) return fail(LBM_ERR_ARG, "null argument");
    CK(launch_moments(h->storage, h->L, h->buf[h->cur], h->scratch, nullptr, nullptr, nullptr, nullptr,
                      h->partials, h->stats + NQ, h->counter + 1, h->stream));
    double s[NQ];
    CK(cudaMemcpyAsync(s, h->stats + NQ, NQ * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int rc = check_status(h);
    if (rc) return rc;
    for (int k = 0; k < 6; ++k) out[k] = s[k];
    if (s[6] > 0) return fail(LBM_ERR_DIVERGED, "non-finite or non-positive density or temperature");
    return LBM_OK;
}

int lbm_step_stats(lbm_handle* h, double out[8]) {
    if (!h || !out) return fail(LBM_ERR_ARG, "null argument");
    double s[NQ];
    CK(cudaMemcpyAsync(s, h->stats, NQ * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int rc = check_status(h);
    for (int k = 0; k < 8; ++k) out[k] = s[k];
    return rc;
}

int64_t lbm_step_count(const lbm_handle* h) { return h ? h->steps : -1; }

int lbm_set_tile_wait(lbm_handle* h, int64_t ns) {
    if (!h) return fail(LBM_ERR_ARG, "null handle");
    if (ns < 0) return fail(LBM_ERR_ARG, "negative wait bound");
    if (h->L.tile_wait_ns == (unsigned long long)ns) return LBM_OK;
    // the captured graph holds the launch parameters: capture anew
    CK(cudaStreamSynchronize(h->stream));
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->L.tile_wait_ns = (unsigned long long)ns;
    return LBM_OK;
}

double lbm_bytes_per_step(const lbm_handle* h) {
    if (!h) return 0.0;
    return 2.0 * 18.0 * (double)h->esize * (double)h->cfg.nx * (double)h->cfg.ny;
}

// Checkpoint layout: magic, nx, ny, precision, walls, a hash of the whole
// configuration, steps, then the raw stored buffer (18 ghost-padded planes).
static const uint64_t CK_MAGIC = 0x4c424d4c56434b32ull;  // "LBMLVCK2"

// FNV-1a (Fowler, Noll, Vo) over every field of the configuration that
// defines the case -- all but the stream and the device -- field by field
// (so that struct padding never enters).
static uint64_t config_hash(const lbm_config& c) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    };
    const int32_t ints[] = {c.nx, c.ny, c.precision, c.walls, c.hot_x0, c.hot_len, c.rounding, c.open_sides,
                            c.cubic};
    const double dbl[] = {c.a_t, c.b_t, c.R, c.K_EOS, c.K_INT, c.Tr0, c.varpi, c.gamma1, c.gamma2,
                          c.s_p, c.s_eps, c.sig_e, c.sig_eps, c.sig_p, c.tau_j_v, c.tau_j_l, c.c_v,
                          c.C_ref, c.accel_x, c.accel_y, c.Tr_bottom, c.Tr_top, c.Tr_hot, c.rho_ref,
                          c.Tr_open, c.rho_open};
    mix(ints, sizeof ints);
    mix(dbl, sizeof dbl);
    return h;
}

int lbm_save(lbm_handle* h, const char* path) {
    if (!h || !path) return fail(LBM_ERR_ARG, "null argument");
    int rc = check_status(h);
    if (rc) return rc;
    const size_t bytes = (size_t)18 * h->L.geo.plane * h->esize;
    std::vector<unsigned char> host(bytes);
    CK(cudaMemcpy(host.data(), h->buf[h->cur], bytes, cudaMemcpyDeviceToHost));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    int32_t hdr[4] = {h->cfg.nx, h->cfg.ny, h->cfg.precision, h->cfg.walls};
    const uint64_t ch = config_hash(h->cfg);
    bool ok = std::fwrite(&CK_MAGIC, 8, 1, fp) == 1 && std::fwrite(hdr, sizeof hdr, 1, fp) == 1 &&
              std::fwrite(&ch, 8, 1, fp) == 1 && std::fwrite(&h->steps, 8, 1, fp) == 1 &&
              std::fwrite(host.data(), 1, bytes, fp) == bytes;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(LBM_ERR_IO, std::string("write failed: ") + path);
}

int lbm_load(lbm_handle* h, const char* path) {
    if (!h || !path) return fail(LBM_ERR_ARG, "null argument");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    uint64_t magic = 0, ch = 0;
    int32_t hdr[4];
    int64_t steps = 0;
    const size_t bytes = (size_t)18 * h->L.geo.plane * h->esize;
    std::vector<unsigned char> host(bytes);
    bool ok = std::fread(&magic, 8, 1, fp) == 1 && std::fread(hdr, sizeof hdr, 1, fp) == 1 &&
              std::fread(&ch, 8, 1, fp) == 1 && std::fread(&steps, 8, 1, fp) == 1;
    if (ok && (magic != CK_MAGIC || hdr[0] != h->cfg.nx || hdr[1] != h->cfg.ny || hdr[2] != h->cfg.precision ||
               hdr[3] != h->cfg.walls)) {
        std::fclose(fp);
        return fail(LBM_ERR_ARG, "checkpoint does not match this handle's lattice");
    }
    if (ok && ch != config_hash(h->cfg)) {
        std::fclose(fp);
        return fail(LBM_ERR_ARG, "checkpoint was written under another configuration (EOS, rates, forces, "
                                 "walls or rounding differ)");
    }
    ok = ok && std::fread(host.data(), 1, bytes, fp) == bytes;
    std::fclose(fp);
    if (!ok) return fail(LBM_ERR_IO, std::string("read failed: ") + path);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(h->buf[0], host.data(), bytes, cudaMemcpyHostToDevice));
    // the device copy of the step count keys the stochastic rounding of
    // 16-bit storage: a resumed run continues with the same dither
    const double st = (double)steps;
    CK(cudaMemcpy(h->stats + 7, &st, sizeof st, cudaMemcpyHostToDevice));
    h->cur = 0;
    h->steps = steps;
    return LBM_OK;
}

int lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return LBM_OK;
}


// ---------------------------------------------------------------------------
// Batched cases
// ---------------------------------------------------------------------------
struct lbm_batch {
    int n = 0;
    int storage = 0;
    size_t esize = 0;
    std::vector<lbm_config> cfg;
    std::vector<lbm_params> prm;
    std::vector<Launch> L;
    std::vector<long long> off;  // element offsets of each case in an arena buffer
    long long arena_elems = 0;
    void* arena[2] = {nullptr, nullptr};
    int cur = 0;
    BatchCase* d_cases[2] = {nullptr, nullptr};  // per tile shape (ntx differs)
    KC<float>* d_kcs = nullptr;
    CUtensorMap* d_maps[2] = {nullptr, nullptr};
    BatchItem* d_items = nullptr;
    int max_items = 0;
    std::vector<BatchItem> items[2][3];  // [shape][order]
    float* d_partials = nullptr;
    int* d_status = nullptr;
    double* d_steps = nullptr;   // step count (device copy, keys stochastic rounding)
    unsigned* d_done = nullptr;  // finished blocks of the current launch
    double* d_rec = nullptr;     // 8 (case record) + 8 (conservation)
    double* scratch = nullptr;   // 18 x largest case
    double* aux_partials = nullptr;
    unsigned* aux_counter = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int shape = 0, order = 1;
    int sms = 0;
    unsigned long long tile_wait_ns = TILE_WAIT_NS_DEFAULT;
    cudaGraphExec_t graph = nullptr;
    int64_t steps = 0;
    static constexpr int GRAPH_STEPS = 20;
};

static BatchLaunch batch_launch(lbm_batch* b) {
    BatchLaunch B;
    B.items = b->d_items;
    B.nitems = (int)b->items[b->shape][b->order].size();
    B.cases = b->d_cases[b->shape];
    B.kcs = b->d_kcs;
    B.maps = b->d_maps[b->shape];
    B.partials = b->d_partials;
    B.status = b->d_status;
    B.sms = b->sms;
    B.steps = b->d_steps;
    B.done = b->d_done;
    B.rounding = b->cfg[0].rounding;
    B.tile_wait_ns = b->tile_wait_ns;
    return B;
}

static void batch_release(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void* ptrs[] = {b->arena[0], b->arena[1], b->d_cases[0], b->d_cases[1], b->d_kcs, b->d_maps[0], b->d_maps[1],
                    b->d_items, b->d_partials, b->d_status, b->d_rec, b->scratch, b->aux_partials, b->aux_counter,
                    b->d_steps, b->d_done};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

static int batch_upload_items(lbm_batch* b) {
    const std::vector<BatchItem>& v = b->items[b->shape][b->order];
    CK(cudaMemcpyAsync(b->d_items, v.data(), v.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return LBM_OK;
}

int lbm_batch_init(const lbm_config* cfgs, int32_t ncases, lbm_batch** out) {
    if (!cfgs || !out || ncases <= 0) return fail(LBM_ERR_ARG, "null argument or no cases");
    *out = nullptr;
    const int prec = cfgs[0].precision;
    if (prec != LBM_F32 && prec != LBM_F16S && prec != LBM_BF16S)
        return fail(LBM_ERR_ARG, "batch precision must be LBM_F32, LBM_F16S or LBM_BF16S");
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ERR_OOM, "host allocation failed");
    b->n = ncases;
    b->storage = storage_of(prec);
    b->esize = elem_size(b->storage);
    b->cfg.assign(cfgs, cfgs + ncases);
    b->prm.resize(ncases);
    b->L.resize(ncases);
    b->off.resize(ncases);
    long long total = 0;
    size_t max_n = 0;
    for (int i = 0; i < ncases; ++i) {
        if (cfgs[i].precision != prec) { delete b; return fail(LBM_ERR_ARG, "all batch cases need one precision"); }
        if (cfgs[i].walls != 0 || cfgs[i].open_sides != 0) {
            delete b;
            return fail(LBM_ERR_ARG, "batch cases must be periodic (walls = 0, no open sides)");
        }
        if (cfgs[i].rounding != cfgs[0].rounding) { delete b; return fail(LBM_ERR_ARG, "all batch cases need one rounding"); }
        if (cfgs[i].cubic) { delete b; return fail(LBM_ERR_ARG, "the cubic-term elimination is built for single cases"); }
        std::memset(&b->L[i], 0, sizeof(Launch));
        int rc = derive(cfgs[i], b->prm[i], b->L[i]);
        if (rc) { delete b; return rc; }
        b->off[i] = total;
        total += ((18 * b->L[i].geo.plane + 127) / 128) * 128;  // 256-byte aligned case starts
        max_n = std::max(max_n, (size_t)cfgs[i].nx * cfgs[i].ny);
    }
    b->arena_elems = total;
    cudaError_t e = cudaSetDevice(cfgs[0].device);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaSetDevice"); }
    e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, cfgs[0].device);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    for (int i = 0; i < ncases; ++i) b->L[i].geo.sms = b->sms;
    if (cfgs[0].stream) {
        b->stream = static_cast<cudaStream_t>(cfgs[0].stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    // work lists for both tile shapes and the three orders
    std::vector<int> by_size(ncases);
    for (int i = 0; i < ncases; ++i) by_size[i] = i;
    std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int c) {
        return (long long)cfgs[a].nx * cfgs[a].ny > (long long)cfgs[c].nx * cfgs[c].ny;
    });
    std::vector<BatchCase> hc[2];
    for (int v = 0; v < 2; ++v) {
        int bx, by;
        batch_tile(b->storage, v, &bx, &by);
        hc[v].resize(ncases);
        std::vector<int> nt(ncases);
        for (int i = 0; i < ncases; ++i) {
            BatchCase& c = hc[v][i];
            std::memset(&c, 0, sizeof c);
            c.geo = b->L[i].geo;
            c.off = b->off[i];
            c.ntx = (cfgs[i].nx + bx - 1) / bx;
            c.ntiles = c.ntx * ((cfgs[i].ny + by - 1) / by);
            float rs = 0.f;
            for (int q = 0; q < 9; ++q) rs += b->L[i].kf.rest[q];
            c.rest_sum = rs;
            nt[i] = c.ntiles;
        }
        for (int i = 0; i < ncases; ++i)
            for (int t = 0; t < nt[i]; ++t) b->items[v][0].push_back({i, t});
        for (int i : by_size)
            for (int t = 0; t < nt[i]; ++t) b->items[v][1].push_back({i, t});
        int maxt = *std::max_element(nt.begin(), nt.end());
        for (int t = 0; t < maxt; ++t)
            for (int i = 0; i < ncases; ++i)
                if (t < nt[i]) b->items[v][2].push_back({i, t});
        b->max_items = std::max(b->max_items, (int)b->items[v][0].size());
    }
    const size_t abytes = (size_t)total * b->esize;
    const size_t nb_aux = 4096;
    bool ok = cudaMalloc(&b->arena[0], abytes) == cudaSuccess && cudaMalloc(&b->arena[1], abytes) == cudaSuccess &&
              cudaMalloc(&b->d_cases[0], ncases * sizeof(BatchCase)) == cudaSuccess &&
              cudaMalloc(&b->d_cases[1], ncases * sizeof(BatchCase)) == cudaSuccess &&
              cudaMalloc(&b->d_kcs, ncases * sizeof(KC<float>)) == cudaSuccess &&
              cudaMalloc(&b->d_maps[0], (size_t)ncases * 4 * sizeof(CUtensorMap)) == cudaSuccess &&
              cudaMalloc(&b->d_maps[1], (size_t)ncases * 4 * sizeof(CUtensorMap)) == cudaSuccess &&
              cudaMalloc(&b->d_items, (size_t)b->max_items * sizeof(BatchItem)) == cudaSuccess &&
              cudaMalloc(&b->d_partials, (size_t)b->max_items * 8 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_rec, 16 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->scratch, 18 * max_n * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->aux_partials, nb_aux * NQ * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->aux_counter, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&b->d_steps, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&b->d_done, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_release(b);
        delete b;
        return fail(LBM_ERR_OOM, "device allocation failed");
    }
    // tensor maps: [case][buffer][f, g] per tile shape
    EncodeTiled enc = get_encoder();
    if (!enc) { batch_release(b); delete b; return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"); }
    CUtensorMapDataType dt = b->storage == S_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : b->storage == S_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                   : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    for (int v = 0; v < 2; ++v) {
        int bx, by;
        batch_tile(b->storage, v, &bx, &by);
        std::vector<CUtensorMap> maps((size_t)ncases * 4);
        for (int i = 0; i < ncases; ++i) {
            const Geometry& G = b->L[i].geo;
            const int x0 = G.PX - G.HX;  // map x = 0: the first ghost column
            // up to the right ghost block: boxes of ragged tiles read the
            // out-of-bounds fill, not the row padding
            cuuint64_t dims[3] = {(cuuint64_t)((G.nx > bx ? G.nx : bx) + 2 * G.HX), (cuuint64_t)G.nyp, 18};
            cuuint64_t strides[2] = {(cuuint64_t)G.pitch * b->esize, (cuuint64_t)G.plane * b->esize};
            cuuint32_t estr[3] = {1, 1, 1};
            cuuint32_t boxf[3] = {(cuuint32_t)(bx + 2 * G.HX), (cuuint32_t)(by + 4), 9};
            cuuint32_t boxg[3] = {(cuuint32_t)(bx + 2 * G.HX), (cuuint32_t)(by + 2), 9};
            for (int buf = 0; buf < 2; ++buf) {
                void* base = static_cast<unsigned char*>(b->arena[buf]) + ((size_t)b->off[i] + x0) * b->esize;
                CUresult r1 = enc(&maps[(i * 2 + buf) * 2], dt, 3, base, dims, strides, boxf, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                CUresult r2 = enc(&maps[(i * 2 + buf) * 2 + 1], dt, 3, base, dims, strides, boxg, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
                    batch_release(b);
                    delete b;
                    return fail(LBM_ERR_CUDA, "cuTensorMapEncodeTiled failed for a batch case");
                }
            }
        }
        e = cudaMemcpy(b->d_maps[v], maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_cases[v], hc[v].data(), ncases * sizeof(BatchCase), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { batch_release(b); delete b; return cuda_fail(e, "cudaMemcpy"); }
    }
    std::vector<KC<float>> kk(ncases);
    for (int i = 0; i < ncases; ++i) kk[i] = b->L[i].kf;
    ok = cudaMemcpy(b->d_kcs, kk.data(), ncases * sizeof(KC<float>), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(b->arena[0], 0, abytes) == cudaSuccess && cudaMemset(b->arena[1], 0, abytes) == cudaSuccess &&
         cudaMemset(b->d_status, 0, sizeof(int)) == cudaSuccess &&
         cudaMemset(b->d_partials, 0, (size_t)b->max_items * 8 * sizeof(float)) == cudaSuccess &&
         cudaMemset(b->aux_counter, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(b->d_steps, 0, sizeof(double)) == cudaSuccess &&
         cudaMemset(b->d_done, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) { batch_release(b); delete b; return fail(LBM_ERR_CUDA, "device initialisation failed"); }
    e = batch_prepare(b->storage);
    if (e == cudaSuccess) e = prepare_step(b->storage);
    if (e != cudaSuccess) { batch_release(b); delete b; return cuda_fail(e, "cudaFuncSetAttribute"); }
    int rc = batch_upload_items(b);
    if (rc) { batch_release(b); delete b; return rc; }
    *out = b;
    return LBM_OK;
}

static int batch_check(lbm_batch* b) {
    CK(cudaStreamSynchronize(b->stream));
    int st = 0;
    CK(cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        CK(cudaMemset(b->d_status, 0, sizeof(int)));
        if (st & ST_TIMEOUT) return fail(LBM_ERR_TIMEOUT, "a device-side wait exceeded its bound");
        if (st & ST_NONFINITE) return fail(LBM_ERR_DIVERGED, "non-finite or non-positive density in a batch case");
    }
    return LBM_OK;
}

static void* case_buf(lbm_batch* b, int i, int which) {
    return static_cast<unsigned char*>(b->arena[which]) + (size_t)b->off[i] * b->esize;
}

int lbm_batch_set_fields(lbm_batch* b, int32_t i, const double* rho, const double* ux, const double* uy,
                         const double* T, int on_device) {
    if (!b || i < 0 || i >= b->n || !rho || !ux || !uy || !T) return fail(LBM_ERR_ARG, "bad argument");
    const size_t n = (size_t)b->cfg[i].nx * b->cfg[i].ny;
    const double* src[4] = {rho, ux, uy, T};
    const double* d[4];
    for (int k = 0; k < 4; ++k) {
        if (on_device) { d[k] = src[k]; continue; }
        CK(cudaMemcpyAsync(b->scratch + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        d[k] = b->scratch + k * n;
    }
    CK(cudaMemsetAsync(case_buf(b, i, b->cur), 0, (size_t)18 * b->L[i].geo.plane * b->esize, b->stream));
    CK(launch_init(b->storage, b->L[i], d[0], d[1], d[2], d[3], case_buf(b, i, b->cur), b->stream));
    return batch_check(b);
}

static int batch_build_graph(lbm_batch* b) {
    cudaGraph_t g;
    const BatchLaunch B = batch_launch(b);
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < lbm_batch::GRAPH_STEPS && e == cudaSuccess; ++k)
        e = launch_batch_step(b->storage, b->shape, B, k & 1, b->arena[1 - (k & 1)], b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "batch step launch during capture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
    if (!b || n < 0) return fail(LBM_ERR_ARG, "bad argument");
    const BatchLaunch B = batch_launch(b);
    while (n > 0) {
        if (b->cur == 0 && n >= lbm_batch::GRAPH_STEPS) {
            if (!b->graph) {
                int rc = batch_build_graph(b);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(b->graph, b->stream));
            b->steps += lbm_batch::GRAPH_STEPS;
            n -= lbm_batch::GRAPH_STEPS;
            continue;
        }
        CK(launch_batch_step(b->storage, b->shape, B, b->cur, b->arena[1 - b->cur], b->stream));
        b->cur = 1 - b->cur;
        b->steps += 1;
        n -= 1;
    }
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, int32_t i, double* rho, double* ux, double* uy, double* T, int on_device) {
    if (!b || i < 0 || i >= b->n) return fail(LBM_ERR_ARG, "bad argument");
    const size_t n = (size_t)b->cfg[i].nx * b->cfg[i].ny;
    double* outs[4] = {rho, ux, uy, T};
    double* d[4];
    for (int k = 0; k < 4; ++k) d[k] = outs[k] ? (on_device ? outs[k] : b->scratch + (1 + k) * n) : nullptr;
    CK(launch_moments(b->storage, b->L[i], case_buf(b, i, b->cur), b->scratch, d[0], d[1], d[2], d[3], nullptr,
                      nullptr, nullptr, b->stream));
    if (!on_device)
        for (int k = 0; k < 4; ++k)
            if (outs[k]) CK(cudaMemcpyAsync(outs[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return batch_check(b);
}

int lbm_batch_conservation(lbm_batch* b, int32_t i, double out[6]) {
    if (!b || i < 0 || i >= b->n || !out) return fail(LBM_ERR_ARG, "bad argument");
    CK(launch_moments(b->storage, b->L[i], case_buf(b, i, b->cur), b->scratch, nullptr, nullptr, nullptr, nullptr,
                      b->aux_partials, b->d_rec + 8, b->aux_counter, b->stream));
    double s[8];
    CK(cudaMemcpyAsync(s, b->d_rec + 8, 8 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    int rc = batch_check(b);
    if (rc) return rc;
    for (int k = 0; k < 6; ++k) out[k] = s[k];
    return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch* b, int32_t i, double* f, double* g) {
    if (!b || i < 0 || i >= b->n || !f || !g) return fail(LBM_ERR_ARG, "bad argument");
    const size_t n = (size_t)b->cfg[i].nx * b->cfg[i].ny;
    CK(launch_get_pops(b->storage, b->L[i], case_buf(b, i, b->cur), b->scratch, b->scratch + 9 * n, b->stream));
    CK(cudaMemcpyAsync(f, b->scratch, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(g, b->scratch + 9 * n, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return batch_check(b);
}

int lbm_batch_step_stats(lbm_batch* b, int32_t i, double out[8]) {
    if (!b || i < 0 || i >= b->n || !out) return fail(LBM_ERR_ARG, "bad argument");
    CK(launch_batch_case_record(batch_launch(b), i, b->d_rec, b->stream));
    double s[8], steps = 0.0;
    CK(cudaMemcpyAsync(s, b->d_rec, 8 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(&steps, b->d_steps, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    int rc = batch_check(b);
    for (int k = 0; k < 7; ++k) out[k] = s[k];
    out[7] = steps;
    return rc;
}

int64_t lbm_batch_step_count(const lbm_batch* b) { return b ? b->steps : -1; }

int lbm_batch_set_tile_wait(lbm_batch* b, int64_t ns) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    if (ns < 0) return fail(LBM_ERR_ARG, "negative wait bound");
    if (b->tile_wait_ns == (unsigned long long)ns) return LBM_OK;
    CK(cudaStreamSynchronize(b->stream));
    if (b->graph) {  // the captured graph holds the launch parameters
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->tile_wait_ns = (unsigned long long)ns;
    return LBM_OK;
}

int lbm_batch_select(lbm_batch* b, int32_t shape, int32_t order) {
    if (!b || shape < 0 || shape > 1 || order < 0 || order > 2) return fail(LBM_ERR_ARG, "bad candidate");
    b->shape = shape;
    b->order = order;
    return batch_upload_items(b);
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, int32_t choice[2], double* ms) {
    if (!b || trial_steps < 2) return fail(LBM_ERR_ARG, "need at least 2 trial steps");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int bs = 0, bo = 0;
    for (int v = 0; v < 2; ++v)
        for (int o = 0; o < 3; ++o) {
            int rc = lbm_batch_select(b, v, o);
            if (rc) return rc;
            const BatchLaunch B = batch_launch(b);
            CK(launch_batch_step(b->storage, b->shape, B, b->cur, b->arena[1 - b->cur], b->stream));  // warm-up
            b->cur = 1 - b->cur;
            CK(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < trial_steps; ++k) {
                CK(launch_batch_step(b->storage, b->shape, B, b->cur, b->arena[1 - b->cur], b->stream));
                b->cur = 1 - b->cur;
            }
            CK(cudaEventRecord(e1, b->stream));
            CK(cudaEventSynchronize(e1));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e0, e1));
            const double per = t / trial_steps;
            if (ms) ms[3 * v + o] = per;
            b->steps += trial_steps + 1;
            if (per < best) { best = per; bs = v; bo = o; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (choice) { choice[0] = bs; choice[1] = bo; }
    int rc = lbm_batch_select(b, bs, bo);
    if (rc) return rc;
    return batch_check(b);
}

int lbm_batch_get_params(const lbm_batch* b, int32_t i, lbm_params* out) {
    if (!b || !out || i < 0 || i >= b->n) return fail(LBM_ERR_ARG, "bad argument");
    *out = b->prm[i];
    return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch* b) {
    if (!b) return fail(LBM_ERR_ARG, "null batch");
    return batch_check(b);
}

int64_t lbm_batch_nodes(const lbm_batch* b) {
    if (!b) return 0;
    int64_t s = 0;
    for (int i = 0; i < b->n; ++i) s += (int64_t)b->cfg[i].nx * b->cfg[i].ny;
    return s;
}

double lbm_batch_bytes_per_step(const lbm_batch* b) {
    return b ? 2.0 * 18.0 * (double)b->esize * (double)lbm_batch_nodes(b) : 0.0;
}

int lbm_batch_destroy(lbm_batch* b) {
    if (!b) return LBM_OK;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
    return LBM_OK;
}

}  // extern "C"

int lbm_internal_fail(int code, const char* msg) { return fail(code, msg); }

size_t lbm_internal_state_bytes(const lbm_handle* h) { return (size_t)18 * h->L.geo.plane * h->esize; }

int lbm_internal_snapshot(lbm_handle* h, void* dst) {
    CK(cudaMemcpyAsync(dst, h->buf[h->cur], lbm_internal_state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    return LBM_OK;
}

int lbm_internal_set_fields_fast(lbm_handle* h, const double* fields) {
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    const size_t bytes = (size_t)18 * h->L.geo.plane * h->esize;
    CK(cudaMemsetAsync(h->buf[0], 0, bytes, h->stream));
    CK(launch_init(h->storage, h->L, fields, fields + n, fields + 2 * n, fields + 3 * n, h->buf[0], h->stream, true));
    h->cur = 0;
    return check_status(h);
}

int lbm_internal_read_fast(lbm_handle* h, double* fields, double out[6]) {
    const size_t n = (size_t)h->cfg.nx * h->cfg.ny;
    double* d[4] = {nullptr, nullptr, nullptr, nullptr};
    if (fields)
        for (int k = 0; k < 4; ++k) d[k] = fields + k * n;
    CK(launch_moments(h->storage, h->L, h->buf[h->cur], h->scratch, d[0], d[1], d[2], d[3], h->partials,
                      h->stats + NQ, h->counter + 1, h->stream, true));
    double st[NQ];
    CK(cudaMemcpyAsync(st, h->stats + NQ, NQ * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int rc = check_status(h);
    if (rc) return rc;
    for (int k = 0; k < 6; ++k) out[k] = st[k];
    if (st[6] > 0) return fail(LBM_ERR_DIVERGED, "non-finite or non-positive density or temperature");
    return LBM_OK;
}

int lbm_internal_restore(lbm_handle* h, const void* src) {
    CK(cudaMemcpyAsync(h->buf[h->cur], src, lbm_internal_state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    return LBM_OK;
}

cudaStream_t lbm_internal_stream(const lbm_handle* h) { return h->stream; }

int lbm_internal_set_steps(lbm_handle* h, int64_t steps) {
    CK(cudaStreamSynchronize(h->stream));
    const double st = (double)steps;
    CK(cudaMemcpy(h->stats + 7, &st, sizeof st, cudaMemcpyHostToDevice));
    h->steps = steps;
    return LBM_OK;
}

void lbm_internal_rho_bounds(const lbm_handle* h, double* rho_v, double* rho_l, int* nx, int* ny) {
    *rho_v = h->prm.rho_v;
    *rho_l = h->prm.rho_l;
    *nx = h->cfg.nx;
    *ny = h->cfg.ny;
}

extern "C" {

int lbm_conservation_noalloc(const lbm_config* cfg, const double* f, const double* g, double* out,
                             void* stream) {
    if (!cfg || !f || !g || !out) return fail(LBM_ERR_ARG, "null argument");
    const long long n = (long long)cfg->nx * (long long)cfg->ny;
    if (n > noalloc_max_nodes())
        return fail(LBM_ERR_ARG, "lattice of " + std::to_string(n) +
                                     " nodes exceeds LBM_NOALLOC_MAX_NODES = " +
                                     std::to_string(noalloc_max_nodes()) + " of the no-allocation scratch");
    lbm_params prm;
    Launch L;
    std::memset(&L, 0, sizeof L);
    int rc = derive(*cfg, prm, L);
    if (rc) return rc;
    cudaError_t e = launch_record_noalloc(L, f, g, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "conservation record without allocation");
    return LBM_OK;
}

}  // extern "C"
