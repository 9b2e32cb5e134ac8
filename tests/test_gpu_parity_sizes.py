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

from gpu_common import gpu_case, oracle_case, rel_err, slab_fields

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(8, 8), (8, 13)])
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
