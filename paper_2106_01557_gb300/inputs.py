"""Seeded synthetic input fields shaped like the paper's test problems.

Shared by the oracle tests and the CUDA-path tests and benchmark. It holds
none of the model's arithmetic: coexistence densities, temperatures and
every other physical number come in as arguments, computed by whichever
side (oracle or library) is under test.

Recipes:
* ``slab``: rho(x) = rho_v + (rho_l - rho_v)/2 [tanh(2(x - x1)/w) - tanh(2(x - x2)/w)]
  on a periodic box, evaluated with the periodic images of both edges.
* ``droplets``: sum of tanh-edged discs rho_v + (rho_l - rho_v)/2 [1 - tanh(2(r - R)/w)],
  distances periodic.
* ``layer``: liquid below y_int, vapour above, tanh edge of width w.
* ``perturbed``: a smooth field plus seeded uniform noise of relative size eps.
"""
from __future__ import annotations

import math

import numpy as np


def _periodic_delta(a, b, n):
    d = (a - b) % n
    return np.where(d > n / 2, d - n, d)


def slab(nx, ny, rho_v, rho_l, x1, x2, width=4.0):
    """Flat liquid slab between x1 and x2 in vapour (periodic in x)."""
    x = np.arange(nx, dtype=np.float64)
    prof = np.zeros(nx)
    for shift in (-nx, 0, nx):
        prof += 0.5 * (np.tanh(2.0 * (x - x1 - shift) / width) - np.tanh(2.0 * (x - x2 - shift) / width))
    prof = np.clip(prof, 0.0, 1.0)
    rho = rho_v + (rho_l - rho_v) * prof
    return np.repeat(rho[None, :], ny, axis=0)


def droplets(nx, ny, rho_v, rho_l, centers, radii, width=4.0):
    """Liquid discs in vapour, periodic distances, tanh edges."""
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    phase = np.zeros((ny, nx))
    for (cx, cy), R in zip(centers, radii):
        dx = _periodic_delta(xx, cx, nx)
        dy = _periodic_delta(yy, cy, ny)
        r = np.sqrt(dx * dx + dy * dy)
        phase = np.maximum(phase, 0.5 * (1.0 - np.tanh(2.0 * (r - R) / width)))
    return rho_v + (rho_l - rho_v) * phase


def place_droplets(nx, ny, n, r_lo, r_hi, gap, seed, max_tries=100000):
    """Seeded non-overlapping droplet centres and radii: R ~ U[r_lo, r_hi],
    centres by rejection sampling with periodic gap >= R1 + R2 + gap."""
    rng = np.random.default_rng(seed)
    centers, radii = [], []
    tries = 0
    while len(radii) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place droplets")
        R = rng.uniform(r_lo, r_hi)
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        ok = True
        for (ox, oy), oR in zip(centers, radii):
            dx = _periodic_delta(cx, ox, nx)
            dy = _periodic_delta(cy, oy, ny)
            if math.hypot(dx, dy) < R + oR + gap:
                ok = False
                break
        if ok and 2 * R + gap < min(nx, ny):
            centers.append((cx, cy))
            radii.append(R)
    return centers, radii


def layer(nx, ny, rho_v, rho_l, y_int, width=4.0):
    """Liquid for y < y_int, vapour above."""
    y = np.arange(ny, dtype=np.float64)
    prof = 0.5 * (1.0 - np.tanh(2.0 * (y - y_int) / width))
    rho = rho_v + (rho_l - rho_v) * prof
    return np.repeat(rho[:, None], nx, axis=1)


def perturbed(base, eps, seed):
    """base * (1 + eps * U[-1, 1]) with a seeded generator."""
    rng = np.random.default_rng(seed)
    return base * (1.0 + eps * rng.uniform(-1.0, 1.0, size=base.shape))


def uniform(shape, value):
    return np.full(shape, float(value))


def random_velocity(shape, amp, seed):
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1.0, 1.0, size=shape), amp * rng.uniform(-1.0, 1.0, size=shape)


def hot_spot_x0(nx, length, seed):
    """Seeded start abscissa of a hot-spot segment of the bottom wall."""
    rng = np.random.default_rng(seed)
    return int(rng.integers(0, nx - length + 1))


def batch_cases(n, seed, lo=64, hi=512, multiple=8, tr_lo=0.6, tr_hi=0.95):
    """Seeded heterogeneous sweep: (nx, ny) log-uniform in [lo, hi] rounded
    to a multiple of `multiple`, droplet radius U[8, 0.3 min(nx, ny)],
    reduced temperature U[tr_lo, tr_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / multiple) * multiple)
        ny = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))) / multiple) * multiple)
        nx = min(max(nx, lo), hi)
        ny = min(max(ny, lo), hi)
        R = float(rng.uniform(8.0, 0.3 * min(nx, ny)))
        Tr = float(rng.uniform(tr_lo, tr_hi))
        out.append({"nx": nx, "ny": ny, "R": R, "Tr": Tr})
    return out
