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
