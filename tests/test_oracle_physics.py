"""Physics pins of the oracle: the paper's thermodynamic-consistency claim
(text after Eq. 16: coexistence densities and the interface given by the
pressure tensor of Eq. 11) and Laplace's law for a static droplet (the
equilibrium-droplet run described after Eq. 19)."""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, thermo

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _width_5_95(prof, x, rv, rl):
    lvl = lambda fr: np.interp(rv + fr * (rl - rv), prof, x)
    return lvl(0.95) - lvl(0.05)


def test_flat_interface_coexistence_and_width():
    # A periodic liquid slab started from the square-gradient equilibrium
    # profile must stay at the Maxwell densities (within 1%) and keep the
    # interface width W = 10 that K_INT prescribes (the paper measured
    # 9.961104 for its droplet); 10,000 steps at T_r = 0.8.
    N = 128
    cfg = thermo.Config(nx=N, ny=4)
    o = Oracle(cfg)
    p = o.p
    x = np.arange(N, dtype=float)
    z = np.minimum(x - N / 4, 3 * N / 4 - x)
    r1 = thermo.planar_profile(p.T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS, cfg.K_INT, z)
    rho = np.repeat(r1[None, :], 4, axis=0)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    c0 = o.conservation()
    o.step(10000)
    m = o.moments()
    r, T = m["rho"][0], m["T"][0]
    rv, rl = r[0], r[N // 2]
    Mv, _, _ = thermo.maxwell(T[0], cfg.a_t, cfg.b_t, cfg.R)
    _, Ml, _ = thermo.maxwell(T[N // 2], cfg.a_t, cfg.b_t, cfg.R)
    assert abs(rv / Mv - 1) < 0.01
    assert abs(rl / Ml - 1) < 0.01
    xs = np.arange(N // 4 - 20, N // 4 + 20)
    assert _width_5_95(r[xs], xs, rv, rl) == pytest.approx(10.0, rel=0.02)
    # temperature stays uniform to 0.1% of T_c, velocities die out
    assert np.abs(T / p.Tc - 0.8).max() < 1e-3
    assert np.abs(m["ux"]).max() < 1e-5 * p.c
    c1 = o.conservation()
    assert c1[0] == pytest.approx(c0[0], rel=1e-12)
    # total energy including rho eps_p: bounded drift (not a discrete invariant)
    assert abs(c1[4] / c0[4] - 1) < 1e-3


def test_tanh_slab_relaxes_to_coexistence():
    # The benchmark's initial state: tanh edges of width 4 between the
    # Maxwell densities. The interface relaxes to width 10, moving mass and
    # latent heat; the bulks equilibrate thermally on the heat-conduction
    # time scale. After 60,000 steps each bulk density is within 1% of the
    # Maxwell density at its own measured temperature (at 10,000 steps the
    # vapour is still 6% off, at 30,000 steps 1.1%).
    from paper_2106_01557_gb300 import inputs
    N = 128
    cfg = thermo.Config(nx=N, ny=4)
    o = Oracle(cfg)
    p = o.p
    rho = inputs.slab(N, 4, p.rho_v, p.rho_l, N / 4, 3 * N / 4, 4.0)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    o.step(60000)
    m = o.moments()
    r, T = m["rho"][0], m["T"][0]
    Mv, _, _ = thermo.maxwell(T[0], cfg.a_t, cfg.b_t, cfg.R)
    _, Ml, _ = thermo.maxwell(T[N // 2], cfg.a_t, cfg.b_t, cfg.R)
    assert abs(r[0] / Mv - 1) < 0.01
    assert abs(r[N // 2] / Ml - 1) < 0.01


@pytest.mark.slow
def test_laplace_law_static_droplets():
    # Pressure jump across static droplets against 1/R (R the equimolar
    # radius); the slope is the surface tension. Prescribed sigma = 0.01; the
    # paper's own run measured 0.0101676 (with a cubic-velocity correction
    # from another paper, not part of this model). Here the droplets are
    # small (R/W = 2..4) and after 10,000 steps their interiors are still
    # about 0.5% warmer than the vapour, which the liquid EOS turns into a
    # visible pressure error, so the bound is loose: 20% (measured 0.0116).
    N = 128
    res = []
    for R in (20.0, 30.0, 40.0):
        cfg = thermo.Config(nx=N, ny=N)
        o = Oracle(cfg)
        p = o.p
        yy, xx = np.meshgrid(np.arange(N) + 0.0, np.arange(N) + 0.0, indexing="ij")
        rr = np.hypot(xx - N / 2, yy - N / 2)
        rho = thermo.planar_profile(p.T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS, cfg.K_INT, R - rr)
        o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
        o.step(10000)
        m = o.moments()
        r, T = m["rho"], m["T"]
        c = N // 2
        dp = (thermo.p_eos(r[c, c], T[c, c], cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS)
              - thermo.p_eos(r[0, 0], T[0, 0], cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS))
        area = ((r - r[0, 0]) / (r[c, c] - r[0, 0])).sum()
        res.append((1.0 / np.sqrt(area / np.pi), dp))
        # spurious currents stay small against the lattice speed
        assert np.hypot(m["ux"], m["uy"]).max() < 1e-3 * p.c
    x = np.array([a for a, _ in res])
    y = np.array([b for _, b in res])
    slope, icpt = np.polyfit(x, y, 1)
    sigma = GOLD["simulation_parameters"]["sigma_prescribed"]
    assert slope == pytest.approx(sigma, rel=0.20)
    assert abs(icpt) < 0.2 * y.min()



def test_viscous_dissipation_term_gives_the_viscous_work():
    # pins the Y term of Eq. 12c (SM Eq. S6b) with its input (m + m_bar)/2 - m^eq:
    # measured 0.989 (0.006 with the term removed, 1.955 with m - m^eq as input)
    from gpu_common import shear_wave_viscous_work_factor

    class _Lat:
        def __init__(self, nx, ny):
            self.o = Oracle(thermo.Config(nx=nx, ny=ny))
            p = self.o.p
            self.p = {"cs": p.cs, "rho_v": p.rho_v, "T0": p.T0}
            self.moments, self.step, self.set_fields = self.o.moments, self.o.step, self.o.init_fields

    assert shear_wave_viscous_work_factor(_Lat) == pytest.approx(1.0, abs=0.05)


def test_density_wave_leaves_a_uniform_cross_flow_uniform():
    # Galilean invariance of the shear stress: pins the velocity couplings of
    # S in row pxy (SM Eq. S5a), b u_y s_q omega_p (wave along x, flow along
    # y) and b u_x s_q omega_p (wave along y, flow along x). The residual is
    # the D2Q9 lattice's own (its equilibria lack the cubic velocity
    # moments), measured 3.4e-5 in the liquid at 0.03 c_s and 7.8e-4 in the
    # vapour at 0.1 c_s; dropping either coupling gives 3.2e-3 and 2.3e-2,
    # flipping its sign twice that. The liquid moves below its stability
    # limit (test_moving_liquid_stability_limit).
    from gpu_common import cross_flow_residual
    for along_x in (True, False):
        assert cross_flow_residual(_OracleLattice, "l", 0.03, along_x) < 5e-4, along_x
        assert cross_flow_residual(_OracleLattice, "v", 0.1, along_x) < 3e-3, along_x


class _OracleLattice:
    """The oracle behind the interface of the shared physics checks."""

    def __init__(self, nx, ny, **cfg):
        c = thermo.Config(nx=nx, ny=ny, **cfg)
        self.o = Oracle(c)
        p = self.o.p
        self.p = {"cs": p.cs, "dt": p.dt, "rho_v": p.rho_v, "rho_l": p.rho_l, "T0": p.T0, "Tc": p.Tc}
        self.s_p = c.s_p
        self.moments, self.step, self.set_fields = self.o.moments, self.o.step, self.o.init_fields


def test_poiseuille_flow_between_bounce_back_walls():
    # the wall treatment (not in the paper: half-way bounce-back) against the
    # textbook parabola with the walls half a node outside the wall rows:
    # measured 0.22% of the peak at 16 rows (0.054% at 32: second order)
    from gpu_common import poiseuille_deviation
    assert poiseuille_deviation(_OracleLattice) < 0.01


def test_steady_conduction_between_fixed_temperature_walls():
    # fixed-temperature walls (anti-bounce-back of g): the steady temperature
    # is a straight line that reaches the wall values half a node outside
    # the wall rows; measured 0.07% and 0.25% of the difference, and 0.2%
    # from straight (the vapour's density follows the pressure balance)
    from gpu_common import conduction_wall_errors
    eb, et, dev = conduction_wall_errors(_OracleLattice)
    assert eb < 0.01 and et < 0.01 and dev < 0.01


def test_heated_poiseuille_temperature_shape():
    # Force-driven vapour between adiabatic bounce-back walls heats up: by
    # Eq. 6c the body-force work goes into the flow and leaves it as viscous
    # dissipation mu u'^2, which conduction spreads. Once the temperature
    # rises uniformly, T - mean(T) has the shape fixed by
    # lambda theta'' = <mu u'^2> - mu u'^2 with theta' = 0 at the walls:
    # y'^2 H^2 / 24 - y'^4 / 12 (y' from the centre line), whatever lambda is;
    # measured within 0.26% of the peak
    ny = 32
    o = Oracle(thermo.Config(nx=4, ny=ny, walls=1, accel_x=2e-5))
    p = o.p
    one = np.ones((ny, 4))
    o.init_fields(p.rho_v * one, 0 * one, 0 * one, p.T0 * one)
    o.step(22000)
    T = o.moments()["T"].mean(axis=1)
    theta = T - T.mean()
    yp = np.arange(ny) + 0.5 - ny / 2
    shape = yp ** 2 * ny ** 2 / 24 - yp ** 4 / 12
    shape -= shape.mean()
    amp = (theta * shape).sum() / (shape * shape).sum()
    assert amp > 0
    assert np.abs(theta - amp * shape).max() < 0.02 * np.abs(amp * shape).max()


def test_closed_box_heating_carries_the_models_latent_heat():
    # A flat slab in a closed periodic box, heated uniformly by 0.005 T_c,
    # evaporates part of its liquid and settles at a slightly higher
    # temperature. The total energy of Eq. 8 (rho e_k + rho eps_p) stays
    # conserved through the phase change (1.6e-7), so the final temperature
    # follows the lever rule with the model's attraction energy a = G^2 / 2
    # (rise 0.00032 T_c against 0.00042 predicted; the interfaces' own energy
    # makes the rest), not with the EOS's K_EOS a~ (0.0016). With K_INT != 1
    # the model's latent heat a (rho_l - rho_v) + p_s (1/rho_v - 1/rho_l) is
    # 4.6 times the one Clausius-Clapeyron gives for Eq. 17 at T_r = 0.8.
    from scipy.optimize import brentq
    ny, nx = 128, 4
    cfg = thermo.Config(nx=nx, ny=ny)
    o = Oracle(cfg)
    p = o.p
    y = np.arange(ny, dtype=float)
    r1 = thermo.planar_profile(p.T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS, cfg.K_INT,
                               np.minimum(y - ny / 4, 3 * ny / 4 - y))
    rho = np.repeat(r1[:, None], nx, axis=1)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    o.step(10000)
    m = o.moments()
    T_before = m["T"].mean()
    c0 = o.conservation()
    o.init_fields(m["rho"], m["ux"], m["uy"], m["T"] + 0.005 * p.Tc)
    c1 = o.conservation()
    o.step(60000)
    c2 = o.conservation()
    rise = o.moments()["T"].mean() - T_before
    assert abs(c2[4] / c1[4] - 1) < 1e-5
    mass, heat = c0[0] / nx, (c1[4] - c0[4]) / nx

    def energy(T, a):
        rv, rl, _ = thermo.maxwell(T, cfg.a_t, cfg.b_t, cfg.R)
        Ll = (mass - rv * ny) / (rl - rv)
        return (ny - Ll) * (rv * p.cv * T - a * rv * rv) + Ll * (rl * p.cv * T - a * rl * rl)

    def predicted_rise(a):
        e0 = energy(T_before, a)
        return brentq(lambda T: energy(T, a) - e0 - heat, T_before, T_before + 0.005 * p.Tc) - T_before

    assert rise == pytest.approx(predicted_rise(p.a), rel=0.35)
    assert rise < 0.5 * predicted_rise(cfg.K_EOS * cfg.a_t)
    assert thermo.latent_heat(p.T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS) * 4.5 < (
        p.a * (p.rho_l - p.rho_v)
        + cfg.K_EOS * thermo.maxwell(p.T0, cfg.a_t, cfg.b_t, cfg.R)[2] * (1 / p.rho_v - 1 / p.rho_l))


def test_open_heated_bottom_keeps_its_own_state_at_rest():
    # a uniform vapour at the open bottom's own state (rho_out, T_open),
    # at rest under an adiabatic top wall, is a fixed point: the ghost row
    # then carries exactly the bottom row's populations
    o = Oracle(thermo.Config(nx=4, ny=32, walls=1, Tr_open=0.85, open_sides=1))
    p = o.p
    one = np.ones((32, 4))
    o.init_fields(p.rho_out * one, 0 * one, 0 * one, p.T_open * one)
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(500)
    assert np.abs(o.f - f0).max() < 1e-14 * np.abs(f0).max()
    assert np.abs(o.g - g0).max() < 1e-14 * np.abs(g0).max()
    # the open bottom's density: the vapour branch of Eq. 17 at T_open
    # and the liquid's saturation pressure
    ps = thermo.maxwell(p.T0, p.a_t, p.b_t, p.R)[2]
    assert thermo.p_eos(p.rho_out, p.T_open, p.a_t, p.b_t, p.R) == pytest.approx(ps, rel=1e-12)
    assert p.rho_out < p.rho_v


def test_box_open_on_all_four_sides_keeps_its_own_state_and_symmetry():
    # With all four sides open (the evaporating droplet's box): a uniform
    # vapour at the open state (rho_out, T_open) at rest is a fixed point --
    # every ghost, corners included, then carries its nearest node's own
    # populations -- and a centred droplet stays symmetric under the quarter
    # turn and the mirror of the box, which a corner ghost taken from the
    # wrong node, or a side missed, would break.
    n = 16
    o = Oracle(thermo.Config(nx=n, ny=n, walls=1, Tr_open=0.85, open_sides=15))
    p = o.p
    one = np.ones((n, n))
    o.init_fields(p.rho_out * one, 0 * one, 0 * one, p.T_open * one)
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(300)
    assert np.abs(o.f - f0).max() < 1e-13 * np.abs(f0).max()
    assert np.abs(o.g - g0).max() < 1e-13 * np.abs(g0).max()
    from paper_2106_01557_gb300 import inputs
    n = 24
    o = Oracle(thermo.Config(nx=n, ny=n, walls=1, Tr_open=0.85, open_sides=15))
    p = o.p
    rho = inputs.droplets(n, n, p.rho_v, p.rho_l, [(n / 2 - 0.5, n / 2 - 0.5)], [6.0], 4.0)
    o.init_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
    o.step(200)
    m = o.moments()
    for f in ("rho", "T"):
        a = m[f]
        assert np.abs(a - np.rot90(a)).max() < 1e-12 * np.abs(a).max(), f
        assert np.abs(a - a[:, ::-1]).max() < 1e-12 * np.abs(a).max(), f
    assert np.abs(m["ux"] + m["ux"][:, ::-1]).max() < 1e-12 * p.c


def test_stefan_front_with_an_open_heated_bottom():
    # The one-dimensional Stefan problem (Eq. 20, 21; text after Eq. 21):
    # vapour between an open bottom at T_r 0.85 (the outflow at the liquid's
    # saturation pressure) and liquid at T_r 0.8 that stays at rest, Ste =
    # 0.005 with the model's latent heat and c_v = 11.2 R. X^2 grows at
    # 4 k^2 alpha_v. Over 200,000 steps the start-up transient still shows
    # (measured 1.17); a 2.5-million-step run on 256 rows settles to 1.03.
    # With the EOS's latent heat the front would run about 4.5 times faster.
    ny, nx = 128, 4
    paper = GOLD["stefan_problem"]
    cfg = thermo.Config(nx=nx, ny=ny, walls=1, Tr_open=paper["Tr1"], open_sides=1, c_v=11.2)
    o = Oracle(cfg)
    p = o.p
    T0, T1 = p.T0, paper["Tr1"] * p.Tc
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    rho = thermo.planar_profile(T0, cfg.a_t, cfg.b_t, cfg.R, cfg.K_EOS, cfg.K_INT, y - 20.0)
    T = np.where(y < 20.0, T1 + (T0 - T1) * (y + 0.5) / 20.5, T0)
    o.init_fields(rho, 0 * rho, 0 * rho, T)

    def front():
        m = o.moments()
        r = m["rho"].mean(axis=1)
        mid = 0.5 * (p.rho_v + p.rho_l)
        j = int(np.argmax(r > mid))
        return j - 0.5 + (mid - r[j - 1]) / (r[j] - r[j - 1]), m   # from the boundary at y = -1/2

    o.step(100000)
    X1, _ = front()
    o.step(100000)
    X2, m = front()
    ps0 = thermo.maxwell(T0, cfg.a_t, cfg.b_t, cfg.R)[2]
    h_lv = p.a * (p.rho_l - p.rho_v) + cfg.K_EOS * ps0 * (1 / p.rho_v - 1 / p.rho_l)
    Ste = p.rho_v * p.cv * (T1 - T0) / (p.rho_l * h_lv)
    assert Ste == pytest.approx(paper["Ste"], rel=0.01)     # c_v = 11.2 R sets the paper's Ste
    k = thermo.stefan_root(Ste)
    # lambda_v (text after Eq. 15) over rho_v c_v
    alpha_v = (4 + 3 * p.gamma1 + 2 * p.gamma2) / 6 * p.Cref * p.c * p.tauj_v / (p.rho_v * p.cv)
    ratio = (X2 ** 2 - X1 ** 2) / (100000 * p.dt) / (4 * k * k * alpha_v)
    assert 0.85 < ratio < 1.3, ratio
    assert np.abs(m["uy"][ny // 2:]).max() < 1e-5 * p.c           # the liquid stays at rest
