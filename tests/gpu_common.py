"""Shared helpers of the GPU parity tests: seeded cases built once from the
input generators and run on both the oracle and the CUDA library."""
import numpy as np

from oracle import Oracle, thermo
from paper_2106_01557_gb300 import inputs

OPTS = ("walls", "accel_x", "accel_y", "Tr_bottom", "Tr_top", "Tr_hot", "hot_x0", "hot_len", "Tr0",
        "varpi", "gamma1", "gamma2", "s_p", "s_eps", "sig_e", "sig_eps", "sig_p", "tau_j_v", "tau_j_l",
        "c_v", "C_ref", "open_sides", "Tr_open", "cubic")


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


def cross_flow_residual(make, phase, U, along_x, n=64, width=8, amp=1e-3, steps=400):
    """A density wave of relative amplitude amp along one axis of a periodic
    lattice (n nodes along the wave, `width` across) whose fluid, the bulk
    liquid or vapour (phase "l" or "v"), moves uniformly at U c_s along the
    other axis. With nothing varying along the flow, the Navier-Stokes
    momentum equation along the flow (Eq. 6b) reduces to
    d(rho u_par)/dt = U c_s d(rho)/dt, so the flow velocity stays exactly
    U c_s everywhere. make(nx, ny) returns a lattice with .p (cs, rho_v,
    rho_l, T0), set_fields, step and moments. Returns
    max |u_par - U c_s| / (amp c_s) after `steps` steps."""
    shape = (width, n) if along_x else (n, width)
    lat = make(shape[1], shape[0])
    p = lat.p
    rho0 = p["rho_l"] if phase == "l" else p["rho_v"]
    wave = np.sin(2 * np.pi * np.arange(n) / n)
    rho = rho0 * (1 + amp * (wave[None, :] if along_x else wave[:, None])) * np.ones(shape)
    flow = np.full(shape, U * p["cs"])
    if along_x:
        lat.set_fields(rho, 0 * rho, flow, 0 * rho + p["T0"])
    else:
        lat.set_fields(rho, flow, 0 * rho, 0 * rho + p["T0"])
    lat.step(steps)
    u_par = lat.moments()["uy" if along_x else "ux"]
    return float(np.abs(u_par - U * p["cs"]).max() / (amp * p["cs"]))


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


def strip_reference(fields, cfg, x0, w, margin, steps):
    """The oracle's state after `steps` steps on columns x0 .. x0 + w - 1 (all
    rows) of a lattice periodic in x, from a strip of the initial fields
    `margin` columns wider on each side (periodic crop). A node's update
    reads the previous state within two nodes, so with margin > 2 steps the
    strip's centre is exact; walls (in y) are kept whole, and the hot wall
    segment is cut to the strip (the parts beyond the margin cannot reach the
    centre). cfg: the thermo.Config keyword arguments of the full lattice
    (nx, ny, walls, accel_*, Tr_*, hot_x0, hot_len). Returns the strip's
    centre moments {rho, ux, uy, T}, each (ny, w)."""
    assert margin > 2 * steps
    nx, ny = cfg["nx"], cfg["ny"]
    n = w + 2 * margin
    lo = x0 - margin
    crop = [np.roll(a, -lo, axis=1)[:, :n] for a in fields]
    c = dict(cfg)
    c["nx"] = n
    if cfg.get("hot_len", 0) > 0:
        # the hot segment in strip coordinates, clipped to the strip
        a = (cfg["hot_x0"] - lo) % nx
        b = a + cfg["hot_len"]
        if a >= n:   # starts beyond the strip: maybe wraps into it from the left
            a, b = a - nx, b - nx
        a, b = max(a, 0), min(b, n)
        if b > a:
            c["hot_x0"], c["hot_len"] = a, b - a
        else:
            c["hot_x0"], c["hot_len"] = 0, 0
            c["Tr_hot"] = 0.0
    o = Oracle(thermo.Config(**c))
    o.init_fields(*crop)
    o.step(steps)
    mo = o.moments()
    return {k: mo[k][:, margin:margin + w] for k in ("rho", "ux", "uy", "T")}


def boiling_fields(nx, ny, p, seed):
    """The boiling layout's initial state (liquid below 3 ny / 4, vapour above,
    tanh edge of width 4) with seeded perturbations of rho, u and T so that
    every term of the step is active."""
    rho = inputs.layer(nx, ny, p.rho_v, p.rho_l, 0.75 * ny, 4.0)
    rho = inputs.perturbed(rho, 0.02, seed)
    ux, uy = inputs.random_velocity((ny, nx), 0.01 * p.c, seed + 1)
    T = inputs.perturbed(np.full((ny, nx), p.T0), 0.02, seed + 2)
    return rho, ux, uy, T
