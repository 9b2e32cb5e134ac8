"""GPU parity at the size limits: the smallest lattice the library accepts
(8 x 8, and a ragged 8 x 13), and a 8192 x 4096 lattice (33.5 M nodes, far
larger than any tile schedule the small tests reach) checked on windows.
The update at a node reads the previous state within two nodes (pulled
populations one node away, the pair force's densities one node further),
so after n steps a node depends on the initial state within 2 n nodes: the
oracle run on a periodic crop of the initial fields with a margin wider
than that reproduces the crop's centre exactly."""
import numpy as np
import pytest

from gpu_common import boiling_fields, gpu_case, oracle_case, rel_err, slab_fields, strip_reference

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
# 16-bit shifted storage after 10 steps: each step rounds every stored
# deviation to 11 (FP16) significant bits; the bounds of the 100-step tests
# (test_gpu_precision) hold with room
TOL16 = {"rho": 5e-3, "T": 8e-3, "u": 5e-4}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(8, 8), (8, 13), (9, 13)])
def test_smallest_lattices_match_oracle(gpu_lib, prec, shape):
    nx, ny = shape
    o = oracle_case(nx, ny)
    fields = slab_fields(o, seed=5)
    o.init_fields(*fields)
    g = gpu_case(nx, ny, prec)
    g.set_fields(*fields)
    o.step(20)
    g.step(20)
    f, gg = g.get_populations()
    assert rel_err(f, o.f) < TOL[prec]
    assert rel_err(gg, o.g) < TOL[prec]


def test_large_lattice_windows_match_oracle(gpu_lib):
    from paper_2106_01557_gb300 import inputs
    nx, ny, steps, margin, w = 8192, 4096, 10, 24, 48
    probe = oracle_case(64, 64)
    p = probe.p
    rng = np.random.default_rng(11)
    # slabs with seeded perturbations: interfaces, velocity and temperature
    # structure everywhere
    rho = inputs.slab(nx, ny, p.rho_v, p.rho_l, nx / 4, 3 * nx / 4, 4.0)
    rho = rho + (p.rho_l - p.rho_v) * 0.05 * np.sin(2 * np.pi * np.arange(ny) / 97.0)[:, None] ** 2
    rho = inputs.perturbed(rho, 0.02, 12)
    ux, uy = inputs.random_velocity((ny, nx), 0.01 * p.c, 13)
    T = inputs.perturbed(np.full((ny, nx), p.T0), 0.02, 14)
    g = gpu_case(nx, ny, "f32")
    g.set_fields(rho, ux, uy, T)
    g.step(steps)
    m = g.moments()
    n = w + 2 * margin
    windows = [(0, 0), (ny // 2 + 7, nx // 4 - 20), (int(rng.integers(0, ny)), int(rng.integers(0, nx)))]
    for (y0, x0) in windows:
        crop = [np.roll(a, (margin - y0, margin - x0), axis=(0, 1))[:n, :n] for a in (rho, ux, uy, T)]
        o = oracle_case(n, n)
        o.init_fields(*crop)
        o.step(steps)
        mo = o.moments()
        for k in ("rho", "T"):
            got = np.roll(m[k], (-y0, -x0), axis=(0, 1))[:w, :w]
            ref = mo[k][margin:margin + w, margin:margin + w]
            assert rel_err(got, ref) < TOL["f32"], (y0, x0, k)
        for k in ("ux", "uy"):
            got = np.roll(m[k], (-y0, -x0), axis=(0, 1))[:w, :w]
            ref = mo[k][margin:margin + w, margin:margin + w]
            assert np.abs(got - ref).max() < TOL["f32"] * p.c, (y0, x0, k)


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_boiling_workload_full_size_strips_match_oracle(gpu_lib, prec):
    # the benchmark's own configuration at its full size (4096 x 1024, walls,
    # body force, a 32-cell hot wall segment at the benchmark's seeded place),
    # FP32 storage and the 16-bit form (node pairs, stochastic rounding), from
    # a perturbed boiling layout so every term acts: after 10 steps, three
    # full-height strips of 48 columns (one over the hot segment's start, one
    # across the periodic seam, one seeded) against the oracle run on the
    # periodic crops (tests/gpu_common.strip_reference)
    from paper_2106_01557_gb300 import inputs
    nx, ny, steps = 4096, 1024, 10
    hot_x0 = inputs.hot_spot_x0(nx, 32, seed=3)
    cfg = dict(nx=nx, ny=ny, walls=1, accel_y=-1e-5, Tr_bottom=0.8, Tr_hot=0.95, hot_x0=hot_x0, hot_len=32)
    p = oracle_case(64, 64).p
    fields = boiling_fields(nx, ny, p, seed=31)
    g = gpu_case(nx, ny, prec, **{k: v for k, v in cfg.items() if k not in ("nx", "ny")})
    g.set_fields(*fields)
    g.step(steps)
    m = g.moments()
    rng = np.random.default_rng(32)
    tol = {"rho": TOL["f32"], "T": TOL["f32"], "u": TOL["f32"]} if prec == "f32" else TOL16
    for x0 in ((hot_x0 - 20) % nx, nx - 24, int(rng.integers(0, nx))):
        ref = strip_reference(fields, cfg, x0, 48, 24, steps)
        for k in ("rho", "T"):
            got = np.roll(m[k], -x0, axis=1)[:, :48]
            assert rel_err(got, ref[k]) < tol[k], (x0, k)
        for k in ("ux", "uy"):
            got = np.roll(m[k], -x0, axis=1)[:, :48]
            assert np.abs(got - ref[k]).max() < tol["u"] * p.c, (x0, k)
