"""Oracle thermodynamics and parameter derivation (FP64, CPU).

TEST INFRASTRUCTURE ONLY. This module belongs to the oracle: only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it. The product library derives its own parameters in its own
host code and never calls anything here.

What it computes, in the paper's notation (Huang, Wu & Adams, PRL 2021,
"Mesoscopic lattice Boltzmann modeling of the liquid-vapor phase transition"):

* the full dense-gas EOS, Carnahan-Starling hard spheres plus an attractive
  term (Eq. 17), with the critical constants that define a~ and b~;
* the chemical potential that belongs to it and the Maxwell (equal chemical
  potential, equal pressure) coexistence densities rho_v, rho_l -- the
  thermodynamic-consistency statement under Eq. 11 and Eq. 16;
* the interaction strength G (Eq. 18), the lattice sound speed c_s (Eq. 19),
  c = sqrt(3) c_s, dt = dx / c, a and kappa (Eq. 16);
* the collision-model coefficients k, h, b, beta and the relaxation-rate
  constraint tau_p tau_q = (k+1) tau_e tau_q = 1/12 (Supplemental Material,
  text under Eq. S5);
* surface tension and interface width of a planar interface from square-
  gradient theory with the pressure tensor of Eq. 11 (free energy density
  psi + kappa/2 |grad rho|^2), used to pin K_EOS, K_INT against the paper's
  sigma = 0.01, W = 10 at T_r = 0.8 (Sec. "simulations", after Eq. 19).

Readings where the paper is silent:
* c_v = 3R/2 (the Maxwellian of Eq. 3 is three-dimensional);
* C_ref = rho_v(T_r0) c_v (C_ref / (rho c_v) above about 2 makes the heat-
  conduction part linearly unstable, so the smallest bulk capacity is used);
* W is the 5%-95% width of the planar equilibrium profile;
* relaxation rates not given in the paper use parameter set "P0"
  (s_p = 1, s_eps = 1, sigma_e = sigma_eps = sigma_p = 1, tau_j linear in
  rho from 0.25 at rho_v to 2.5 at rho_l so that lambda_l = 10 lambda_v,
  sigma_q = sigma_j).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

from scipy.integrate import quad
from scipy.optimize import brentq

# Eq. 17: a~ = A R^2 Tc^2 / pc, b~ = B R Tc / pc
A_CS = 0.4963880577294099
B_CS = 0.1872945669467330


# --------------------------------------------------------------------------
# Eq. 17 and its thermodynamics (per unit K_EOS unless stated)
# --------------------------------------------------------------------------
def critical_point(a_t: float, b_t: float, R: float):
    """Critical temperature and pressure implied by a~, b~ (Eq. 17)."""
    Tc = B_CS * a_t / (A_CS * b_t * R)
    pc = B_CS * R * Tc / b_t
    return Tc, pc


def p_cs(rho, T, b_t, R):
    """Carnahan-Starling hard-sphere pressure rho R T (1+t+t^2-t^3)/(1-t)^3."""
    t = b_t * rho / 4.0
    return rho * R * T * (1.0 + t + t * t - t ** 3) / (1.0 - t) ** 3


def dp_cs_drho(rho, T, b_t, R):
    """d p_CS / d rho at constant T (closed form of the derivative)."""
    t = b_t * rho / 4.0
    return R * T * (1.0 + 4.0 * t + 4.0 * t * t - 4.0 * t ** 3 + t ** 4) / (1.0 - t) ** 4


def p_eos(rho, T, a_t, b_t, R, K_EOS=1.0):
    """Full EOS, Eq. 17."""
    return K_EOS * (p_cs(rho, T, b_t, R) - a_t * rho * rho)


def dp_eos_drho(rho, T, a_t, b_t, R, K_EOS=1.0):
    return K_EOS * (dp_cs_drho(rho, T, b_t, R) - 2.0 * a_t * rho)


def psi(rho, T, a_t, b_t, R):
    """Helmholtz free energy density whose pressure rho psi' - psi is Eq. 17
    (per unit K_EOS, up to a term linear in rho)."""
    t = b_t * rho / 4.0
    return (rho * R * T * (math.log(rho) - 1.0)
            + rho * R * T * (4.0 * t - 3.0 * t * t) / (1.0 - t) ** 2
            - a_t * rho * rho)


def mu(rho, T, a_t, b_t, R):
    """Chemical potential d psi / d rho (per unit K_EOS)."""
    t = b_t * rho / 4.0
    phi = (4.0 * t - 3.0 * t * t) / (1.0 - t) ** 2
    return R * T * (math.log(rho) + phi + t * (4.0 - 2.0 * t) / (1.0 - t) ** 3) - 2.0 * a_t * rho


def critical_density(a_t, b_t, R):
    """rho_c where dp/drho and d2p/drho2 vanish at T_c (Eq. 17)."""
    Tc, _ = critical_point(a_t, b_t, R)
    # at T_c the inflection of p(rho): solve d2p/drho2 = 0 numerically
    h = 1e-6

    def d2p(r):
        return (dp_eos_drho(r + h, Tc, a_t, b_t, R) - dp_eos_drho(r - h, Tc, a_t, b_t, R)) / (2 * h)

    return brentq(d2p, 0.05 * 4.0 / b_t, 0.9 * 4.0 / b_t, xtol=1e-15)


def spinodals(T, a_t, b_t, R):
    """The two roots of dp/drho = 0 below T_c (vapour and liquid spinodal)."""
    rho_max = 4.0 / b_t
    # dp/drho has one interior minimum between the spinodals; locate it first
    grid = [rho_max * k / 4000.0 for k in range(1, 4000)]
    vals = [dp_eos_drho(r, T, a_t, b_t, R) for r in grid]
    kmin = min(range(len(vals)), key=lambda k: vals[k])
    if vals[kmin] >= 0.0:
        raise ValueError("temperature at or above critical: no spinodals")
    r_min = grid[kmin]
    f = lambda r: dp_eos_drho(r, T, a_t, b_t, R)
    r1 = brentq(f, 1e-12, r_min, xtol=1e-16, rtol=1e-15)
    r2 = brentq(f, r_min, grid[-1], xtol=1e-16, rtol=1e-15)
    return r1, r2


def maxwell(T, a_t, b_t, R):
    """Coexistence densities (rho_v, rho_l) and saturation pressure p_s
    (per unit K_EOS) from mu(rho_v) = mu(rho_l), p(rho_v) = p(rho_l)."""
    s1, s2 = spinodals(T, a_t, b_t, R)
    p = lambda r: p_eos(r, T, a_t, b_t, R)
    p_lo = max(p(s2), 0.0)
    p_hi = p(s1)
    rho_top = 4.0 / b_t

    def branch_v(ps):
        lo = 1e-3 * ps / (R * T)   # ideal-gas bound: p(lo) < ps there
        return brentq(lambda r: p(r) - ps, lo, s1, xtol=1e-18, rtol=1e-15)

    def branch_l(ps):
        hi = s2
        while p(hi) < ps:
            hi = hi + 0.5 * (rho_top - hi)
        return brentq(lambda r: p(r) - ps, s2, hi, xtol=1e-18, rtol=1e-15)

    def dmu(ps):
        return mu(branch_l(ps), T, a_t, b_t, R) - mu(branch_v(ps), T, a_t, b_t, R)

    eps = 1e-14 * p_hi
    ps = brentq(dmu, p_lo + eps, p_hi - eps, xtol=1e-20, rtol=1e-15)
    return branch_v(ps), branch_l(ps), ps


def equal_area_residual(T, rho_v, rho_l, ps, a_t, b_t, R):
    """Maxwell's equal-area statement in the specific-volume plane:
    int_{v_l}^{v_v} (p(v) - p_s) dv = 0 with v = 1/rho."""
    val, _ = quad(lambda r: (p_eos(r, T, a_t, b_t, R) - ps) / (r * r), rho_v, rho_l,
                  epsabs=1e-16, epsrel=1e-13, limit=400)
    return val


def latent_heat(T, a_t, b_t, R, K_EOS=1.0):
    """Latent heat of vaporisation per unit mass on the coexistence curve of
    Eq. 17 at temperature T. The internal energy per unit mass of the EOS
    fluid is c_v T - K_EOS a~ rho (the repulsive part of Eq. 17 is linear in
    T and stores no energy), and T, p are equal across coexistence, so
    h_v - h_l = K_EOS a~ (rho_l - rho_v) + p_s (1/rho_v - 1/rho_l)."""
    rv, rl, ps = maxwell(T, a_t, b_t, R)
    return K_EOS * (a_t * (rl - rv) + ps * (1.0 / rv - 1.0 / rl))


def stefan_number(Tr0, Tr1, cv, a_t, b_t, R, K_EOS):
    """The Stefan number of the one-dimensional Stefan problem (text after
    Eq. 21): rho_v c_v T_c (T_r1 - T_r0) / (rho_l h_lv), with the coexistence
    densities at T_r0 and h_lv the EOS's latent heat there (`latent_heat`);
    cv is the heat capacity per unit mass. The model's own energy balance
    carries a larger latent heat when K_INT != 1, so which h_lv the paper
    means is a reading."""
    Tc, _ = critical_point(a_t, b_t, R)
    rv, rl, _ = maxwell(Tr0 * Tc, a_t, b_t, R)
    return rv * cv * Tc * (Tr1 - Tr0) / (rl * latent_heat(Tr0 * Tc, a_t, b_t, R, K_EOS))


def stefan_root(Ste):
    """k > 0 with Ste / (exp(k^2) erf(k)) = k sqrt(pi) (Eq. 21): the interface
    of the one-phase Stefan problem is at X = 2 k sqrt(alpha_v t) (Eq. 20)."""
    f = lambda k: k * math.sqrt(math.pi) * math.exp(k * k) * math.erf(k) - Ste
    hi = 1.0
    while f(hi) < 0:
        hi *= 2.0
    return brentq(f, 1e-300, hi, xtol=1e-16, rtol=1e-15)


# --------------------------------------------------------------------------
# Square-gradient interface (pressure tensor of Eq. 11, kappa of Eq. 16)
# --------------------------------------------------------------------------
def _omega(rho, T, a_t, b_t, R, rv, rl, ps):
    """Grand-potential excess psi - mu_s rho + p_s (per unit K_EOS)."""
    mus = mu(rv, T, a_t, b_t, R)
    return max(psi(rho, T, a_t, b_t, R) - mus * rho + ps, 0.0)


def surface_tension_and_width(T, a_t, b_t, R, K_EOS, K_INT, dx=1.0):
    """sigma = int sqrt(2 kappa K_EOS Omega) drho and the 5%-95% width
    W = int_{rho_5}^{rho_95} sqrt(kappa / (2 K_EOS Omega)) drho, with
    kappa = G^2 dx^4 / 4 and G from Eq. 18."""
    rv, rl, ps = maxwell(T, a_t, b_t, R)
    G2 = K_INT ** 2 * 2.0 * K_EOS * a_t / dx ** 2
    kappa = G2 * dx ** 4 / 4.0
    om = lambda r: _omega(r, T, a_t, b_t, R, rv, rl, ps)
    sig, _ = quad(lambda r: math.sqrt(2.0 * kappa * K_EOS * om(r)), rv, rl,
                  epsabs=1e-15, epsrel=1e-12, limit=400)
    d = rl - rv
    r5, r95 = rv + 0.05 * d, rv + 0.95 * d
    W, _ = quad(lambda r: math.sqrt(kappa / (2.0 * K_EOS * om(r))), r5, r95,
                epsabs=1e-13, epsrel=1e-12, limit=400)
    return sig, W


def planar_profile(T, a_t, b_t, R, K_EOS, K_INT, z, dx=1.0):
    """Equilibrium planar profile rho(z) of square-gradient theory, centred
    where rho = (rho_v + rho_l)/2, rho increasing with z: z(rho) integrated
    on a density grid, then inverted by interpolation."""
    import numpy as np
    rv, rl, ps = maxwell(T, a_t, b_t, R)
    G2 = K_INT ** 2 * 2.0 * K_EOS * a_t / dx ** 2
    kappa = G2 * dx ** 4 / 4.0
    om = lambda r: _omega(r, T, a_t, b_t, R, rv, rl, ps)
    d = rl - rv
    grid = rv + d * (0.5 - 0.5 * np.cos(np.linspace(0.0, math.pi, 2001)))[1:-1]
    # Gauss-Legendre on each (short, smooth) cell of the grid
    xg, wg = np.polynomial.legendre.leggauss(8)
    integrand = lambda s: math.sqrt(kappa / (2.0 * K_EOS * om(s)))
    dz = []
    for k in range(len(grid) - 1):
        lo, hi = grid[k], grid[k + 1]
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        dz.append(half * sum(w * integrand(mid + half * t) for t, w in zip(xg, wg)))
    zg = np.concatenate([[0.0], np.cumsum(dz)])
    zg -= np.interp(0.5 * (rv + rl), grid, zg)
    return np.interp(np.asarray(z, dtype=np.float64), zg, grid, left=grid[0], right=grid[-1])


# --------------------------------------------------------------------------
# Model parameters (Eq. 16, 18, 19; Supplemental Material, Eq. S3-S5)
# --------------------------------------------------------------------------
@dataclass
class Config:
    """Physical and model inputs of one case."""
    nx: int = 128
    ny: int = 128
    walls: int = 0                 # 0 periodic; 1 half-way bounce-back at y=0 and y=ny-1
    a_t: float = 1.0
    b_t: float = 4.0
    R: float = 1.0
    K_EOS: float = 0.479820
    K_INT: float = 2.294922
    Tr0: float = 0.8               # reference temperature: c_s, C_ref, tau_j ends
    varpi: float = 1.0 / 6.0
    gamma1: float = -2.0
    gamma2: float = 2.0
    s_p: float = 1.0
    s_eps: float = 1.0
    s_0: float = 1.0
    s_j: float = 1.0
    sig_0: float = 1.0
    sig_e: float = 1.0
    sig_eps: float = 1.0
    sig_p: float = 1.0
    tau_j_v: float = 0.25
    tau_j_l: float = 2.5
    c_v: float = 1.5               # in units of R
    C_ref: float = 0.0             # 0 -> rho_v(Tr0) c_v R
    accel_x: float = 0.0
    accel_y: float = 0.0
    Tr_bottom: float = 0.0         # fixed bottom-wall reduced T (<= 0: adiabatic)
    Tr_top: float = 0.0            # fixed top-wall reduced T (<= 0: adiabatic)
    Tr_hot: float = 0.0            # hot-spot reduced T on the bottom wall
    hot_x0: int = 0
    hot_len: int = 0
    open_sides: int = 0            # open, heated sides: 1 bottom, 2 top (with walls), 15 all four
    Tr_open: float = 0.0           # reduced T of the open sides
    cubic: int = 0                 # eliminate the cubic velocity terms (periodic boxes only)


@dataclass
class Params:
    """Derived scalars the oracle step consumes."""
    nx: int
    ny: int
    walls: int
    Tc: float
    pc: float
    rho_v: float
    rho_l: float
    T0: float
    cs: float
    c: float
    dt: float
    G2: float
    a: float
    kappa: float
    R: float
    a_t: float
    b_t: float
    K_EOS: float
    cv: float
    Cref: float
    varpi: float
    gamma1: float
    gamma2: float
    beta: float
    kS: float
    hS: float
    bS: float
    s0: float
    se: float
    seps: float
    sj: float
    sq: float
    sp: float
    sig0: float
    sige: float
    sigeps: float
    sigp: float
    tauj_v: float
    tauj_l: float
    ax: float
    ay: float
    T_bottom: float
    T_top: float
    T_hot: float
    hot_x0: int
    hot_len: int
    open_sides: int
    rho_out: float
    T_open: float
    cubic: int


def _outflow_density(cfg: Config, T0, rv):
    """Density of the open sides: the vapour at T_open and at the saturation
    pressure of the liquid at T0 (the vapour branch of Eq. 17)."""
    if not cfg.open_sides:
        return 0.0
    if cfg.open_sides & 3 and not cfg.walls:
        raise ValueError("an open bottom or top needs walls = 1")
    if cfg.open_sides & 12 and cfg.open_sides != 15:
        raise ValueError("open left and right sides come only with all four sides open")
    Tc, _ = critical_point(cfg.a_t, cfg.b_t, cfg.R)
    Tb = cfg.Tr_open * Tc
    if not Tb > 0:
        raise ValueError("open sides need Tr_open > 0")
    ps = maxwell(T0, cfg.a_t, cfg.b_t, cfg.R)[2]
    return brentq(lambda r: p_eos(r, Tb, cfg.a_t, cfg.b_t, cfg.R) - ps, 1e-6 * rv, rv * T0 / Tb * 1.5)


def _cubic_flag(cfg: Config) -> int:
    if cfg.cubic and (cfg.walls or cfg.open_sides):
        raise ValueError("the cubic-term elimination is built for periodic boxes only")
    return 1 if cfg.cubic else 0


def derive_params(cfg: Config) -> Params:
    """Derivation of every scalar the collision uses from the case inputs."""
    Tc, pc = critical_point(cfg.a_t, cfg.b_t, cfg.R)
    T0 = cfg.Tr0 * Tc
    rv, rl, _ = maxwell(T0, cfg.a_t, cfg.b_t, cfg.R)
    dx = 1.0
    G2 = cfg.K_INT ** 2 * 2.0 * cfg.K_EOS * cfg.a_t / dx ** 2        # Eq. 18
    # Eq. 19: c_s^2 = K_INT^2 (dp_EOS/drho + 2 K_EOS a~ rho) at rho_l
    cs2 = cfg.K_INT ** 2 * (dp_eos_drho(rl, T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS)
                            + 2.0 * cfg.K_EOS * cfg.a_t * rl)
    cs = math.sqrt(cs2)
    c = math.sqrt(3.0) * cs                                           # c_s = c / sqrt(3)
    dt = dx / c
    a = G2 * dx ** 2 / 2.0                                            # Eq. 16
    kappa = G2 * dx ** 4 / 4.0
    w = cfg.varpi
    kS = 1.0 - w                                                      # Eq. S5 text
    hS = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w)
    bS = (1.0 - w) / (1.0 - 3.0 * w)
    beta = -2.0 / (1.0 - w)                                           # Eq. S3 text
    tau_p = 1.0 / cfg.s_p - 0.5
    tau_q = 1.0 / (12.0 * tau_p)                                      # tau_p tau_q = 1/12
    tau_e = tau_p / (kS + 1.0)                                        # (k+1) tau_e = tau_p
    cv = cfg.c_v * cfg.R
    Cref = cfg.C_ref if cfg.C_ref > 0 else rv * cv
    return Params(
        nx=cfg.nx, ny=cfg.ny, walls=cfg.walls, Tc=Tc, pc=pc, rho_v=rv, rho_l=rl, T0=T0,
        cs=cs, c=c, dt=dt, G2=G2, a=a, kappa=kappa, R=cfg.R, a_t=cfg.a_t, b_t=cfg.b_t,
        K_EOS=cfg.K_EOS, cv=cv, Cref=Cref, varpi=w, gamma1=cfg.gamma1, gamma2=cfg.gamma2,
        beta=beta, kS=kS, hS=hS, bS=bS, s0=cfg.s_0, se=1.0 / (tau_e + 0.5),
        seps=cfg.s_eps, sj=cfg.s_j, sq=1.0 / (tau_q + 0.5), sp=cfg.s_p,
        sig0=cfg.sig_0, sige=cfg.sig_e, sigeps=cfg.sig_eps, sigp=cfg.sig_p,
        tauj_v=cfg.tau_j_v, tauj_l=cfg.tau_j_l, ax=cfg.accel_x, ay=cfg.accel_y,
        T_bottom=cfg.Tr_bottom * Tc, T_top=cfg.Tr_top * Tc, T_hot=cfg.Tr_hot * Tc,
        hot_x0=cfg.hot_x0, hot_len=cfg.hot_len,
        open_sides=cfg.open_sides, rho_out=_outflow_density(cfg, T0, rv), T_open=cfg.Tr_open * Tc,
        cubic=_cubic_flag(cfg))


def params_dict(p: Params) -> dict:
    return asdict(p)
