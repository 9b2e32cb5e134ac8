"""Shared helpers of the GPU parity tests: seeded cases built once from the
input generators and run on both the oracle and the CUDA library."""
import numpy as np

from oracle import Oracle, thermo
from paper_2106_01557_gb300 import inputs

OPTS = ("walls", "accel_x", "accel_y", "Tr_bottom", "Tr_top", "Tr_hot", "hot_x0", "hot_len", "Tr0")


def oracle_case(nx, ny, **kw):
    cfg = thermo.Config(nx=nx, ny=ny, **{k: v for k, v in kw.items() if k in OPTS})
    return Oracle(cfg)


def gpu_case(nx, ny, precision, **kw):
    from paper_2106_01557_gb300 import lbm
    return lbm.Lattice.create(nx, ny, precision=precision, **{k: v for k, v in kw.items() if k in OPTS})


def slab_fields(o, seed=0, eps=0.02, uamp=0.01):
    """Tanh slab (width 4) between the oracle's Maxwell densities, with seeded
    perturbations of rho, u, T so that every term of the collision is active."""
    p = o.p
    nx, ny = o.nx, o.ny
    rho = inputs.slab(nx, ny, p.rho_v, p.rho_l, nx / 4, 3 * nx / 4, 4.0)
    rho = inputs.perturbed(rho, eps, seed)
    ux, uy = inputs.random_velocity((ny, nx), uamp * p.c, seed + 1)
    T = inputs.perturbed(np.full((ny, nx), p.T0), eps, seed + 2)
    return rho, ux, uy, T


def rel_err(a, b):
    """max |a - b| / max |b| (per field: the error relative to the field's scale)."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def shear_wave_viscous_work_factor(make, nx=4, N=128, amp=0.1):
    """A decaying shear wave u_x = A(t) sin(ky) in a uniform vapour, on a
    lattice make(nx, N) with .p (cs, rho_v, T0), set_fields, step and
    moments. The energy equation (Eq. 6c) carries the viscous work flux
    u . Pi, whose divergence feeds the cos(2ky) mode of rho e_k at
    lambda rho nu k^2 A^2 with lambda = 1, while the cos(2ky) mode of the
    macroscopic kinetic energy rho u^2 / 2 grows at rho nu k^2 A^2 / 2 (the
    wave's own decay). Their ratio over a short window (steps 5 to 10, before
    conduction and sound act) is 2 lambda, whatever the transport
    coefficients. Returns lambda: without the Y term of Eq. 12c it is 0,
    with m - m^eq in place of (m + m_bar)/2 - m^eq it is 2."""
    lat = make(nx, N)
    p = lat.p
    y = np.arange(N) + 0.0
    cos2 = np.cos(4 * np.pi * y / N)
    ux = np.repeat((amp * p["cs"] * np.sin(2 * np.pi * y / N))[:, None], nx, axis=1)
    lat.set_fields(np.full((N, nx), p["rho_v"]), ux, 0 * ux, 0 * ux + p["T0"])

    def coefficients():
        m = lat.moments()
        r, u, v, T = (m[f].mean(axis=1) for f in ("rho", "ux", "uy", "T"))
        ek = r * 1.5 * T + 0.5 * r * (u * u + v * v)  # rho e_k = rho c_v T + rho |u|^2 / 2, c_v = 3/2 R
        return (2 / N) * (ek * cos2).sum(), (2 / N) * (0.5 * r * u * u * cos2).sum()

    lat.step(5)
    e0, k0 = coefficients()
    lat.step(5)
    e1, k1 = coefficients()
    return (e1 - e0) / (2 * (k1 - k0))


def poiseuille_deviation(make, nx=4, ny=16, g=1e-5, steps=6000):
    """Force-driven flow of the uniform vapour between the half-way
    bounce-back walls (y = -1/2 and ny - 1/2, periodic in x), run to its
    steady state: the largest deviation of u_x from the parabola
    g / (2 nu) (y + 1/2) (ny - 1/2 - y), nu = c_s^2 (1/s_p - 1/2) dt, over
    the parabola's peak. make(nx, ny, **cfg) returns a lattice with .p (cs,
    dt, rho_v, T0), .s_p, set_fields, step and moments."""
    lat = make(nx, ny, walls=1, accel_x=g)
    p = lat.p
    one = np.ones((ny, nx))
    lat.set_fields(p["rho_v"] * one, 0 * one, 0 * one, p["T0"] * one)
    lat.step(steps)
    u = lat.moments()["ux"].mean(axis=1)
    nu = p["cs"] ** 2 * (1 / lat.s_p - 0.5) * p["dt"]
    y = np.arange(ny) + 0.0
    ref = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    return float(np.abs(u - ref).max() / ref.max())


def conduction_wall_errors(make, nx=4, ny=16, tb=0.81, tt=0.79, steps=10000):
    """Steady conduction through the vapour between fixed-temperature walls
    (reduced temperatures tb at the bottom, tt at the top, half-way between
    the wall rows and their ghosts), no flow: the straight line fitted to the
    interior temperature extrapolated to y = -1/2 and y = ny - 1/2, and the
    largest deviation from that line, each over tb - tt."""
    lat = make(nx, ny, walls=1, Tr_bottom=tb, Tr_top=tt)
    p = lat.p
    one = np.ones((ny, nx))
    lat.set_fields(p["rho_v"] * one, 0 * one, 0 * one, p["T0"] * one)
    lat.step(steps)
    T = lat.moments()["T"].mean(axis=1) / p["Tc"]
    y = np.arange(ny) + 0.0
    a, b = np.polyfit(y[3:-3], T[3:-3], 1)
    dT = tb - tt
    return (abs(a * -0.5 + b - tb) / dT, abs(a * (ny - 0.5) + b - tt) / dT,
            float(np.abs(T - (a * y + b)).max() / dT))
