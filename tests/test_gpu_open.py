"""The open, heated sides (the outflow and constant-pressure condition of the
paper's phase-change runs, paragraph after Eq. 19) on the GPU path: parity
with the oracle for an open bottom (the Stefan problem's boundary) and for a
box open on all four sides (the evaporating droplet's), and the Stefan front
of Eq. 20 on the GPU. Tolerances as in the other parity tests: FP64 storage
1e-12 and FP32 storage 1e-5 of max |gpu - oracle| / max |oracle|."""
import json
import os

import numpy as np
import pytest

from gpu_common import gpu_case, oracle_case, rel_err
from paper_2106_01557_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _vapour_below_liquid(o, seed):
    """Vapour in the lower quarter of the box, liquid above (tanh edge of
    width 4), with seeded perturbations of rho, u and T."""
    p = o.p
    nx, ny = o.nx, o.ny
    rho = p.rho_l + p.rho_v - inputs.layer(nx, ny, p.rho_v, p.rho_l, 0.25 * ny, 4.0)
    rho = inputs.perturbed(rho, 0.02, seed)
    ux, uy = inputs.random_velocity((ny, nx), 0.01 * p.c, seed + 1)
    T = inputs.perturbed(np.full((ny, nx), p.T0), 0.02, seed + 2)
    return rho, ux, uy, T


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_open_bottom_matches_oracle(gpu_lib, prec):
    # 40 x 36: ragged tiles in both directions; the open bottom at T_r 0.85
    # below the vapour, a bounce-back top wall above the liquid
    kw = dict(walls=1, open_sides=1, Tr_open=0.85)
    o = oracle_case(40, 36, **kw)
    g = gpu_case(40, 36, prec, **kw)
    assert g.params()["rho_open"] == pytest.approx(o.p.rho_out, rel=1e-12)
    assert g.params()["T_open"] == pytest.approx(o.p.T_open, rel=1e-14)
    fields = _vapour_below_liquid(o, seed=31)
    o.init_fields(*fields)
    g.set_fields(*fields)
    f0, g0 = g.get_populations()
    assert rel_err(f0, o.f) < TOL[prec] and rel_err(g0, o.g) < TOL[prec]
    for n in (1, 49):
        o.step(n)
        g.step(n)
        f, gg = g.get_populations()
        assert rel_err(f, o.f) < TOL[prec], (n, rel_err(f, o.f))
        assert rel_err(gg, o.g) < TOL[prec], (n, rel_err(gg, o.g))
    m, mo = g.moments(), o.moments()
    assert rel_err(m["rho"], mo["rho"]) < TOL[prec] and rel_err(m["T"], mo["T"]) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_box_open_on_all_four_sides_matches_oracle(gpu_lib, prec):
    # a perturbed droplet off the centre of a 40 x 36 box whose four sides
    # (corners included) are open at T_r 0.85
    kw = dict(walls=1, open_sides=15, Tr_open=0.85)
    o = oracle_case(40, 36, **kw)
    g = gpu_case(40, 36, prec, **kw)
    p = o.p
    rho = inputs.droplets(40, 36, p.rho_v, p.rho_l, [(17.0, 19.5)], [9.0], 4.0)
    rho = inputs.perturbed(rho, 0.02, 41)
    ux, uy = inputs.random_velocity((36, 40), 0.01 * p.c, 42)
    T = inputs.perturbed(np.full((36, 40), p.T0), 0.02, 43)
    o.init_fields(rho, ux, uy, T)
    g.set_fields(rho, ux, uy, T)
    for n in (1, 49):
        o.step(n)
        g.step(n)
        f, gg = g.get_populations()
        assert rel_err(f, o.f) < TOL[prec], (n, rel_err(f, o.f))
        assert rel_err(gg, o.g) < TOL[prec], (n, rel_err(gg, o.g))


def test_open_sides_keep_their_own_state_on_gpu(gpu_lib):
    # the open state itself, at rest, is a fixed point of the GPU step
    for sides, shape in ((1, (8, 32)), (15, (16, 16))):
        g = gpu_case(*shape, "f64", walls=1, open_sides=sides, Tr_open=0.85)
        p = g.params()
        one = np.ones(shape[::-1])
        g.set_fields(p["rho_open"] * one, 0 * one, 0 * one, p["T_open"] * one)
        f0, g0 = g.get_populations()
        g.step(300)
        f1, g1 = g.get_populations()
        assert rel_err(f1, f0) < 1e-13 and rel_err(g1, g0) < 1e-13


def test_open_side_configurations_are_checked(gpu_lib):
    from paper_2106_01557_gb300 import lbm
    for kw in (dict(walls=0, open_sides=1, Tr_open=0.85), dict(walls=1, open_sides=4, Tr_open=0.85),
               dict(walls=1, open_sides=1, Tr_open=0.0), dict(walls=1, open_sides=16, Tr_open=0.85)):
        with pytest.raises(lbm.LbmError) as e:
            gpu_case(16, 16, "f32", **kw)
        assert e.value.code == -1


def test_stefan_front_on_gpu(gpu_lib):
    # The one-dimensional Stefan problem of Eq. 20, 21 on the GPU path, as the
    # oracle's pin sets it up (open bottom at T_r 0.85 below vapour, liquid
    # at T_r 0.8 above, c_v = 11.2 R so that Ste = 0.005 with the model's
    # latent heat) on 8 x 256 nodes, FP32 storage, 2.5 million steps: X^2
    # grows at 4 k^2 alpha_v (the oracle measured 1.03 of it over 2.5
    # million steps on 4 x 256).
    from oracle import thermo
    paper = GOLD["stefan_problem"]
    nx, ny = 8, 256
    kw = dict(walls=1, open_sides=1, Tr_open=paper["Tr1"], c_v=11.2)
    o = oracle_case(nx, ny, **kw)
    p = o.p
    g = gpu_case(nx, ny, "f32", **kw)
    T0, T1 = p.T0, paper["Tr1"] * p.Tc
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    rho = thermo.planar_profile(T0, 1.0, 4.0, 1.0, o.cfg.K_EOS, o.cfg.K_INT, y - 20.0)
    T = np.where(y < 20.0, T1 + (T0 - T1) * (y + 0.5) / 20.5, T0)
    g.set_fields(rho, 0 * rho, 0 * rho, T)

    def front():
        r = g.moments()["rho"].mean(axis=1)
        mid = 0.5 * (p.rho_v + p.rho_l)
        j = int(np.argmax(r > mid))
        return j - 0.5 + (mid - r[j - 1]) / (r[j] - r[j - 1])

    g.step(1_000_000)
    X1 = front()
    g.step(1_500_000)
    X2 = front()
    k = thermo.stefan_root(paper["Ste"])
    alpha_v = (4 + 3 * p.gamma1 + 2 * p.gamma2) / 6 * p.Cref * p.c * p.tauj_v / (p.rho_v * p.cv)
    ratio = (X2 ** 2 - X1 ** 2) / (1_500_000 * p.dt) / (4 * k * k * alpha_v)
    print("Stefan front", X1, X2, "growth of X^2 over 4 k^2 alpha_v:", ratio)
    assert 0.9 < ratio < 1.15, ratio


def test_droplet_heated_from_all_sides_follows_the_d2_law(gpu_lib):
    # N2, the evaporating droplet of the text after Eq. 21, scaled down: a
    # droplet of diameter D0 = 32 in a 128 x 128 box open and heated on all
    # four sides (T_r 0.85 at the liquid's saturation pressure), droplet at
    # T_r 0.8, c_v = 11.2 R (Ste = 0.005 with the model's latent heat), FP32
    # storage. (D / D0)^2, D from the liquid area, falls on a straight line
    # in time (the D^2 law) over 0.8 > (D/D0)^2 > 0.2 (measured r^2 =
    # 0.99989), and its slope is of the size the quasi-steady conduction
    # through the vapour gives, d(D^2)/dt = -8 alpha_v Ste / ln(R_inf / R)
    # with R_inf = 1.08 x the half-width of the square: an estimate for a
    # sharp interface without the outward Stefan flow (measured 1.29 of it
    # here, where the interface width W = 10 is a third of D0, and 0.65 at
    # D0 = 64). Over that window the droplet stays near T_r 0.8
    # (evaporative cooling of a few percent).
    import math
    n, D0 = 128, 32.0
    kw = dict(walls=1, open_sides=15, Tr_open=0.85, c_v=11.2)
    g = gpu_case(n, n, "f32", **kw)
    p = g.params()
    rho = inputs.droplets(n, n, p["rho_v"], p["rho_l"], [(n / 2 - 0.5, n / 2 - 0.5)], [D0 / 2], 4.0)
    g.set_fields(rho, 0 * rho, 0 * rho, 0 * rho + p["T0"])
    cv, Tc = p["cv"], p["Tc"]
    h_lv = p["a"] * (p["rho_l"] - p["rho_v"]) + p["p_s"] * (1 / p["rho_v"] - 1 / p["rho_l"])
    ste = p["rho_v"] * cv * (0.85 * Tc - p["T0"]) / (p["rho_l"] * h_lv)
    assert ste == pytest.approx(0.005, rel=0.01)
    alpha_v = (4 + 3 * -2.0 + 2 * 2.0) / 6 * p["Cref"] * p["c"] * 0.25 / (p["rho_v"] * cv)
    ts, d2, Tcen = [], [], []
    steps, every = 0, 25000
    while True:
        m = g.moments()
        area = float(((m["rho"] - p["rho_v"]) / (p["rho_l"] - p["rho_v"])).clip(0, None).sum())
        ts.append(alpha_v * steps * p["dt"] / D0 ** 2)
        d2.append(4 * area / math.pi / D0 ** 2)
        Tcen.append(m["T"][n // 2, n // 2] / Tc)
        if d2[-1] < 0.15 or steps > 3_000_000:
            break
        g.step(every)
        steps += every
    ts, d2, Tcen = np.array(ts), np.array(d2), np.array(Tcen)
    sel = (d2 < 0.8) & (d2 > 0.2)
    assert sel.sum() >= 8
    k, c = np.polyfit(ts[sel], d2[sel], 1)
    r2 = 1 - ((d2[sel] - (k * ts[sel] + c)) ** 2).sum() / ((d2[sel] - d2[sel].mean()) ** 2).sum()
    qs = 8 * ste / math.log(1.08 * (n / 2) / (0.5 * D0 * math.sqrt(0.5)))
    print(f"D^2 law: slope {k:.4e} per t*, r2 {r2:.6f}, quasi-steady {-qs:.4e}, ratio {-k / qs:.3f}, "
          f"droplet T/Tc {Tcen[sel].min():.4f}..{Tcen[sel].max():.4f}")
    assert r2 > 0.995
    assert 0.4 < -k / qs < 1.6
    assert np.all((Tcen[sel] > 0.75) & (Tcen[sel] < 0.801))


def test_droplet_pair_attracts_when_slow_and_repels_when_fast(gpu_lib):
    # The paper's large-small droplet pair (text after Eq. 21, Fig. 3) at half
    # its size: 512^2 heated from all four sides, diameters 80 and 48, centres
    # 128 apart, Ste set through c_v. At Ste = 0.005 the evaporation is slow
    # and the two droplets attract each other and coalesce (measured: the
    # centres close from 128 to 86 and merge at t* = 11); at Ste = 0.5 it is
    # fast, the vapour streaming out of the two facing surfaces pushes them
    # apart (measured: 128 to 166) and the pair has evaporated by t* = 2.5,
    # against t* = 264 at Ste = 0.005.
    import bench
    slow = bench.droplet_pair_study(n=512, stes=(0.005,), samples=400, max_steps=700_000)["results"][0]
    assert slow["error"] is None
    assert slow["coalesced_at_t_star"] is not None and slow["coalesced_at_t_star"] < 20
    assert slow["distance_min"] < 0.8 * slow["distance_initial"]
    fast = bench.droplet_pair_study(n=512, stes=(0.5,))["results"][0]
    assert fast["error"] is None
    assert fast["coalesced_at_t_star"] is None
    assert fast["distance_max"] > 1.15 * fast["distance_initial"]
    assert fast["samples"][-1]["V_over_V0"] < 0.05 and fast["t_star_end"] < 5
    print(f"pair: Ste 0.005 closes to {slow['distance_min']:.1f} and merges at t* {slow['coalesced_at_t_star']:.2f}; "
          f"Ste 0.5 opens to {fast['distance_max']:.1f}, gone at t* {fast['t_star_end']:.2f}")
