"""Batched heterogeneous cases: every case in a batch must evolve as the same
case on its own handle (same precision, agreement to FP32 rounding: the two
kernels are compiled separately and may contract multiply-adds
differently), for every tile shape and work-list order the autotuner can
pick, and match the FP64 oracle within the FP32 tolerance."""
import numpy as np
import pytest

from gpu_common import rel_err

pytestmark = pytest.mark.gpu


def _cases():
    # uneven sizes (multiples of 8, ragged against both tile shapes), one
    # droplet each, different temperatures
    return [(72, 64, 0.8, 14.0), (96, 136, 0.7, 20.0), (64, 64, 0.9, 12.0), (200, 88, 0.85, 18.0)]


def _fields(nx, ny, p, R, seed):
    from paper_2106_01557_gb300 import inputs
    rho = inputs.droplets(nx, ny, p["rho_v"], p["rho_l"], [(nx / 2, ny / 2)], [R], 4.0)
    rho = inputs.perturbed(rho, 0.01, seed)
    ux, uy = inputs.random_velocity((ny, nx), 0.005 * p["c"], seed + 1)
    T = np.full((ny, nx), p["T0"])
    return rho, ux, uy, T


@pytest.mark.parametrize("prec", ["f32", "f16s"])
def test_batch_equals_single_cases(gpu_lib, prec):
    from paper_2106_01557_gb300 import lbm
    cfgs = [lbm.default_config(nx, ny, precision=prec, Tr0=tr) for nx, ny, tr, _ in _cases()]
    # 16-bit storage rounded to nearest: the single-lattice kernel draws the
    # stochastic-rounding dither per node pair, the batch per node, so with
    # stochastic rounding the two are compared through the oracle instead
    # (test_batch_fp16_storage_matches_oracle, test_gpu_precision)
    for c in cfgs:
        c.rounding = 0
    singles = [lbm.Lattice(c) for c in cfgs]
    fields = []
    for k, (s, (nx, ny, tr, R)) in enumerate(zip(singles, _cases())):
        fields.append(_fields(nx, ny, s.params(), R, 40 + k))
        s.set_fields(*fields[-1])
        s.step(30)
    for shape in (0, 1):
        for order in (0, 1, 2):
            b = lbm.Batch(cfgs)
            b.select(shape, order)
            for i, fl in enumerate(fields):
                b.set_fields(i, *fl)
            b.step(30)
            for i, s in enumerate(singles):
                fb, gb = b.get_populations(i)
                fs, gs = s.get_populations()
                # FP16 storage rounds every population to 11 bits each step,
                # so a difference in the last FP32 bit (the kernels fuse their
                # products differently) shows at that level where it flips a
                # rounding
                tol = 1e-5 if prec == "f32" else 1e-2
                assert rel_err(fb, fs) < tol and rel_err(gb, gs) < tol, (shape, order, i)
            b.close()


# per-case model coefficients and relaxation rates, so that a batch kernel
# that took one from another case's parameter block would fail
CASE_RATES = [{}, dict(sig_eps=1.4, sig_p=1.8), dict(s_p=1.2, varpi=0.2, gamma1=-1.5, gamma2=2.5),
              dict(tau_j_v=0.3, tau_j_l=2.0, sig_e=0.9, s_eps=1.3, c_v=2.0)]


def test_batch_matches_oracle_and_records(gpu_lib):
    from oracle import Oracle, thermo
    from paper_2106_01557_gb300 import lbm
    cases = _cases()
    cfgs = [lbm.default_config(nx, ny, precision="f32", Tr0=tr, **r) for (nx, ny, tr, _), r in zip(cases, CASE_RATES)]
    b = lbm.Batch(cfgs)
    ors = []
    for i, (nx, ny, tr, R) in enumerate(cases):
        o = Oracle(thermo.Config(nx=nx, ny=ny, Tr0=tr, **CASE_RATES[i]))
        p = {"rho_v": o.p.rho_v, "rho_l": o.p.rho_l, "c": o.p.c, "T0": o.p.T0}
        fl = _fields(nx, ny, p, R, 60 + i)
        o.init_fields(*fl)
        b.set_fields(i, *fl)
        ors.append(o)
    b.step(20)
    for o in ors:
        o.step(20)
    for i, o in enumerate(ors):
        f, g = b.get_populations(i)
        assert rel_err(f, o.f) < 1e-5 and rel_err(g, o.g) < 1e-5, i
    # the fused per-case record of the last step equals the state record
    # entering it (FP32 partials, so at FP32 precision)
    before = [b.conservation(i) for i in range(len(cases))]
    b.step(1)
    for i in range(len(cases)):
        s = b.step_stats(i)
        assert s[0] == pytest.approx(before[i][0], rel=1e-5)
        assert s[3] == pytest.approx(before[i][3], rel=1e-5)
        assert s[6] == 0


def test_batch_autotune_picks_a_candidate(gpu_lib):
    from paper_2106_01557_gb300 import lbm
    cfgs = [lbm.default_config(nx, ny, precision="f16s", Tr0=tr) for nx, ny, tr, _ in _cases()]
    b = lbm.Batch(cfgs)
    for i, (nx, ny, tr, R) in enumerate(_cases()):
        p = lbm.Lattice(cfgs[i]).params()
        b.set_fields(i, *_fields(nx, ny, p, R, 80 + i))
    (shape, order), ms = b.autotune(3)
    assert shape in (0, 1) and order in (0, 1, 2)
    assert np.all(ms > 0) and ms[3 * shape + order] == ms.min()
    b.step(25)
    b.synchronize()


def test_batch_fp16_storage_matches_oracle(gpu_lib):
    # FP16 shifted storage in the batch, stochastic rounding (the default),
    # against the FP64 oracle at the single-lattice FP16 bounds after 100
    # steps (rho 5e-3, T 8e-3 of the field's largest value, u 5e-4 of c): a
    # perturbed slab on 100 x 37 and a droplet case at another temperature;
    # the device's step count, which keys the rounding, follows the steps
    from oracle import Oracle, thermo
    from paper_2106_01557_gb300 import inputs, lbm
    shapes = [(100, 37, 0.8), (72, 64, 0.85)]
    cfgs = [lbm.default_config(nx, ny, precision="f16s", Tr0=tr) for nx, ny, tr in shapes]
    assert all(c.rounding == 1 for c in cfgs)
    b = lbm.Batch(cfgs)
    ors = []
    for i, (nx, ny, tr) in enumerate(shapes):
        o = Oracle(thermo.Config(nx=nx, ny=ny, Tr0=tr))
        p = o.p
        if i == 0:
            rho = inputs.slab(nx, ny, p.rho_v, p.rho_l, nx / 4, 3 * nx / 4, 4.0)
        else:
            rho = inputs.droplets(nx, ny, p.rho_v, p.rho_l, [(nx / 2, ny / 2)], [14.0], 4.0)
        rho = inputs.perturbed(rho, 0.02, 90 + i)
        ux, uy = inputs.random_velocity((ny, nx), 0.01 * p.c, 92 + i)
        T = inputs.perturbed(np.full((ny, nx), p.T0), 0.02, 94 + i)
        o.init_fields(rho, ux, uy, T)
        b.set_fields(i, rho, ux, uy, T)
        ors.append(o)
    b.step(100)
    for o in ors:
        o.step(100)
    for i, o in enumerate(ors):
        m, mo = b.moments(i), o.moments()
        e_rho = rel_err(m["rho"], mo["rho"])
        e_T = rel_err(m["T"], mo["T"])
        e_u = max(np.abs(m["ux"] - mo["ux"]).max(), np.abs(m["uy"] - mo["uy"]).max()) / o.p.c
        print(f"batch f16s case {i}: rho {e_rho:.3e} T {e_T:.3e} u/c {e_u:.3e}")
        assert e_rho < 5e-3 and e_T < 8e-3 and e_u < 5e-4, (i, e_rho, e_T, e_u)
    assert b.steps == 100 and b.step_stats(0)[7] == 100


def test_batch_tile_wait_that_runs_out_is_reported(gpu_lib):
    # as for a single case: with no time to wait, the first item of every
    # block times out, the launch ends after the copies in flight have
    # landed, LBM_ERR_TIMEOUT is reported, and the batch then steps as a
    # fresh one does, bit for bit
    from paper_2106_01557_gb300 import lbm
    cases = _cases()
    cfgs = [lbm.default_config(nx, ny, precision="f32", Tr0=tr) for nx, ny, tr, _ in cases]
    fields = [_fields(nx, ny, lbm.Lattice(c).params(), R, 70 + i) for i, (c, (nx, ny, tr, R)) in enumerate(zip(cfgs, cases))]
    a = lbm.Batch(cfgs)
    for i, fl in enumerate(fields):
        a.set_fields(i, *fl)
    a.set_tile_wait(0)
    a.step(2)
    with pytest.raises(lbm.LbmError) as e:
        a.synchronize()
    assert e.value.code == -5
    a.set_tile_wait(2_000_000_000)
    for i, fl in enumerate(fields):
        a.set_fields(i, *fl)
    a.step(25)
    b = lbm.Batch(cfgs)
    for i, fl in enumerate(fields):
        b.set_fields(i, *fl)
    b.step(25)
    for i in range(len(cases)):
        fa, ga = a.get_populations(i)
        fb, gb = b.get_populations(i)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), i
