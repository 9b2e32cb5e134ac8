"""Laplace's law on the GPU path at the sizes the oracle cannot reach: one
static droplet per periodic 512 x 512 box (radii 40 to 100, R/W = 3 to 13),
started from the planar square-gradient profile of the EOS, at three reduced
temperatures. After 60,000 steps the pressure jump, from the EOS (Eq. 17) at
each bulk's measured density and temperature, against 1/R (R the equimolar
radius) has the slope of the surface tension that gradient theory gives for
the configured K_EOS and K_INT (the paragraph after Eq. 19 prescribes
sigma = 0.01 at T_r = 0.8 and reports 0.0101676 measured). Measured excess:
+9.3% at T_r 0.7 (wider rates), +6.7% at 0.8, +8.4% at 0.9, +6.6% at 0.8 with
the cubic-term elimination (the droplets are at rest, so the u^3 terms it
removes are negligible here). The bound is 12%: the droplets end slightly
warmer than the vapour (the total-energy drift of the scheme), and the
liquid's stiff EOS turns that into a pressure excess; the oracle's
small-droplet pin is looser (20%)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


# T_r = 0.7 with the wider rates sigma_eps = 1.4, sigma_p = 1.8: with the
# default rates the liquid is linearly unstable below T_r = 0.75; the last
# case switches on the cubic-term elimination, as the paper's own runs do
# (paragraph after Eq. 19)
LAPLACE_CASES = [(0.7, dict(sig_eps=1.4, sig_p=1.8)), (0.8, {}), (0.9, {}), (0.8, dict(cubic=1))]


@pytest.mark.parametrize("tr,opts", LAPLACE_CASES)
def test_laplace_law_large_droplets(gpu_lib, tr, opts):
    from oracle import thermo
    from gpu_common import gpu_case, oracle_case
    N, steps = 512, 60000
    o = oracle_case(N, N, Tr0=tr, **opts)
    p = o.p
    K_EOS, K_INT = o.cfg.K_EOS, o.cfg.K_INT
    sigma, _ = thermo.surface_tension_and_width(p.T0, 1.0, 4.0, 1.0, K_EOS, K_INT)
    yy, xx = np.meshgrid(np.arange(N) + 0.0, np.arange(N) + 0.0, indexing="ij")
    rr = np.hypot(xx - N / 2, yy - N / 2)
    c = N // 2
    inv_r, dp = [], []
    for R in (40.0, 60.0, 80.0, 100.0):
        rho = thermo.planar_profile(p.T0, 1.0, 4.0, 1.0, K_EOS, K_INT, R - rr)
        g = gpu_case(N, N, "f32", Tr0=tr, **opts)
        g.set_fields(rho, 0 * rho, 0 * rho, 0 * rho + p.T0)
        g.step(steps)
        m = g.moments()
        g.close()
        r, T = m["rho"], m["T"]
        dp.append(thermo.p_eos(r[c, c], T[c, c], 1.0, 4.0, 1.0, K_EOS)
                  - thermo.p_eos(r[0, 0], T[0, 0], 1.0, 4.0, 1.0, K_EOS))
        area = ((r - r[0, 0]) / (r[c, c] - r[0, 0])).sum()
        inv_r.append(1.0 / np.sqrt(area / np.pi))
        # spurious currents stay small against the lattice speed
        assert np.hypot(m["ux"], m["uy"]).max() < 1e-2 * p.c
    slope, icpt = np.polyfit(np.array(inv_r), np.array(dp), 1)
    print(f"T_r {tr} {opts}: Laplace slope / sigma - 1 = {slope / sigma - 1:+.4f}, intercept / dp_min = {icpt / min(dp):+.3f}")
    assert slope == pytest.approx(sigma, rel=0.12)
    assert abs(icpt) < 0.2 * min(dp)


def test_viscous_work_on_gpu(gpu_lib):
    # the oracle's pin of the Y term (Eq. 12c, SM Eq. S6b), on the FP64 GPU path
    from gpu_common import gpu_case, shear_wave_viscous_work_factor

    class _Lat:
        def __init__(self, nx, ny):
            self.g = gpu_case(nx, ny, "f64")
            self.p = self.g.params()
            self.moments, self.step, self.set_fields = self.g.moments, self.g.step, self.g.set_fields

    assert shear_wave_viscous_work_factor(_Lat, nx=8) == pytest.approx(1.0, abs=0.05)


class _GpuLattice:
    """An FP64 GPU lattice behind the interface of the shared physics checks."""

    def __init__(self, nx, ny, **cfg):
        from gpu_common import gpu_case
        self.g = gpu_case(nx, ny, "f64", **cfg)
        self.p = self.g.params()
        from paper_2106_01557_gb300 import lbm
        self.s_p = lbm.default_config(nx, ny).s_p
        self.moments, self.step, self.set_fields = self.g.moments, self.g.step, self.g.set_fields


def test_cross_flow_pin_on_gpu(gpu_lib):
    # the oracle's Galilean-invariance pin of S's row-pxy velocity couplings
    # (a density wave leaves a uniform cross-flow uniform) on the FP64 GPU path
    from gpu_common import cross_flow_residual
    for along_x in (True, False):
        assert cross_flow_residual(_GpuLattice, "l", 0.03, along_x) < 5e-4, along_x
        assert cross_flow_residual(_GpuLattice, "v", 0.1, along_x) < 3e-3, along_x


def test_wall_pins_on_gpu(gpu_lib):
    # the oracle's pins of the walls (Poiseuille parabola, steady conduction)
    # on the FP64 GPU path
    from gpu_common import conduction_wall_errors, poiseuille_deviation
    assert poiseuille_deviation(_GpuLattice, nx=8) < 0.01
    eb, et, dev = conduction_wall_errors(_GpuLattice, nx=8)
    assert eb < 0.01 and et < 0.01 and dev < 0.01
