"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs. Tolerances: FP64 storage 1e-12 and FP32 storage 1e-5,
both as max |gpu - oracle| / max |oracle| per distribution function or
field; velocity errors are measured against the lattice speed c."""
import numpy as np
import pytest

from gpu_common import gpu_case, oracle_case, rel_err, slab_fields

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _pair(nx, ny, prec, seed=0, **kw):
    o = oracle_case(nx, ny, **kw)
    fields = slab_fields(o, seed=seed)
    o.init_fields(*fields)
    g = gpu_case(nx, ny, prec, **kw)
    g.set_fields(*fields)
    return o, g


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_derived_parameters_match_oracle(gpu_lib, prec):
    o = oracle_case(64, 64)
    g = gpu_case(64, 64, prec)
    p = g.params()
    for k in ("Tc", "pc", "T0", "rho_v", "rho_l", "cs", "c", "dt", "G2", "a", "kappa", "Cref", "beta",
              "kS", "hS", "bS", "se", "sq"):
        assert p[k] == pytest.approx(getattr(o.p, k), rel=1e-13), k


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_init_populations_match_oracle(gpu_lib, prec):
    o, g = _pair(100, 37, prec)
    f, gg = g.get_populations()
    # FP32 storage: the set-up computes in FP32 (a few ulps of the largest
    # population); FP64 storage in FP64
    tol = 1e-14 if prec == "f64" else 5e-7
    print(prec, "init error", rel_err(f, o.f), rel_err(gg, o.g))
    assert rel_err(f, o.f) < tol
    assert rel_err(gg, o.g) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nsteps", [1, 10, 100])
def test_periodic_steps_match_oracle(gpu_lib, prec, nsteps):
    # 100 x 37: two tiles across (ragged tail), three tile rows (ragged)
    o, g = _pair(100, 37, prec, seed=3)
    o.step(nsteps)
    g.step(nsteps)
    f, gg = g.get_populations()
    assert rel_err(f, o.f) < TOL[prec]
    assert rel_err(gg, o.g) < TOL[prec]
    m = g.moments()
    mo = o.moments()
    assert rel_err(m["rho"], mo["rho"]) < TOL[prec]
    assert rel_err(m["T"], mo["T"]) < TOL[prec]
    assert np.abs(m["ux"] - mo["ux"]).max() < TOL[prec] * o.p.c
    assert np.abs(m["uy"] - mo["uy"]).max() < TOL[prec] * o.p.c


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_walls_body_force_hot_spot_match_oracle(gpu_lib, prec):
    kw = dict(walls=1, accel_y=-1e-4, Tr_bottom=0.8, Tr_hot=0.95, hot_x0=90, hot_len=20, Tr_top=0.0)
    o, g = _pair(100, 40, prec, seed=5, **kw)
    o.step(25)
    g.step(25)
    f, gg = g.get_populations()
    assert rel_err(f, o.f) < TOL[prec]
    assert rel_err(gg, o.g) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_walled_case_stays_with_the_oracle_over_1000_steps(gpu_lib, prec):
    # the walled case (walls, body force, hot wall segment across the
    # periodic seam) on 100 x 37, errors at 1, 10, 100 and 1,000 steps; the
    # 1,000-step error stays within the parity bound
    kw = dict(walls=1, accel_y=-1e-4, Tr_bottom=0.8, Tr_hot=0.95, hot_x0=90, hot_len=20, Tr_top=0.0)
    o, g = _pair(100, 37, prec, seed=5, **kw)
    errs, done = [], 0
    for n in (1, 10, 100, 1000):
        o.step(n - done)
        g.step(n - done)
        done = n
        f, gg = g.get_populations()
        errs.append(max(rel_err(f, o.f), rel_err(gg, o.g)))
    print(prec, "error after 1, 10, 100, 1000 steps:", ["%.2e" % e for e in errs])
    assert errs[-1] < TOL[prec], errs


# every model coefficient and relaxation rate away from its default, so that
# a kernel that kept one fixed, or took one from the wrong slot, fails
RATES = dict(Tr0=0.85, varpi=0.2, gamma1=-1.5, gamma2=2.5, s_p=1.2, s_eps=1.3, sig_e=0.9, sig_eps=1.4,
             sig_p=1.8, tau_j_v=0.3, tau_j_l=2.0, c_v=2.0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_non_default_rates_match_oracle(gpu_lib, prec):
    o, g = _pair(100, 37, prec, seed=7, **RATES)
    p = g.params()
    for k in ("T0", "rho_v", "rho_l", "cs", "Cref", "beta", "kS", "hS", "bS", "se", "sq"):
        assert p[k] == pytest.approx(getattr(o.p, k), rel=1e-13), k
    o.step(10)
    g.step(10)
    f, gg = g.get_populations()
    assert rel_err(f, o.f) < TOL[prec]
    assert rel_err(gg, o.g) < TOL[prec]


def test_rest_state_stays_at_rest(gpu_lib):
    g = gpu_case(64, 64, "f64")
    p = g.params()
    n = (64, 64)
    g.set_fields(np.full(n, p["rho_l"]), np.zeros(n), np.zeros(n), np.full(n, p["T0"]))
    f0, g0 = g.get_populations()
    g.step(40)
    f1, g1 = g.get_populations()
    assert rel_err(f1, f0) < 1e-14 and rel_err(g1, g0) < 1e-14


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_conservation_record_matches_oracle(gpu_lib, prec):
    o, g = _pair(128, 64, prec, seed=7)
    o.step(5)
    g.step(5)
    co = o.conservation()
    cg = g.conservation()
    tol = TOL[prec]
    assert cg[0] == pytest.approx(co[0], rel=tol)
    scale = co[0] * o.p.c
    assert abs(cg[1] - co[1]) < tol * scale and abs(cg[2] - co[2]) < tol * scale
    assert cg[3] == pytest.approx(co[3], rel=tol)
    assert cg[4] == pytest.approx(co[4], rel=10 * tol)
    assert cg[5] == pytest.approx(co[5], rel=1e-3)


def test_fused_step_reduction_equals_state_record(gpu_lib):
    # the in-kernel reduction of step n is the record of the state entering it
    o, g = _pair(128, 64, "f64", seed=8)
    g.step(3)
    before = g.conservation()
    g.step(1)
    s = g.step_stats()
    assert s[0] == pytest.approx(before[0], rel=1e-13)
    assert s[3] == pytest.approx(before[3], rel=1e-13)
    assert s[4] == pytest.approx(before[4], rel=1e-12)
    assert s[6] == 0 and s[7] == 4


def test_exact_conservation_on_gpu(gpu_lib):
    o, g = _pair(128, 64, "f64", seed=9)
    c0 = g.conservation()
    g.step(200)
    c1 = g.conservation()
    assert c1[0] == pytest.approx(c0[0], rel=1e-13)
    assert abs(c1[1] - c0[1]) < 1e-13 * c0[0] * o.p.c


def test_checkpoint_resume_is_bitwise(gpu_lib, tmp_path):
    for prec in ("f64", "f32", "f16s"):
        o = oracle_case(72, 40)
        fields = slab_fields(o, seed=11)
        a = gpu_case(72, 40, prec)
        a.set_fields(*fields)
        a.step(7)
        path = str(tmp_path / f"ck_{prec}.bin")
        a.save(path)
        a.step(13)
        fa, ga = a.get_populations()
        b = gpu_case(72, 40, prec)
        b.load(path)
        assert b.steps == 7
        b.step(13)
        fb, gb = b.get_populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_checkpoint_of_another_lattice_or_a_short_file_is_refused(gpu_lib, tmp_path):
    # the header names the lattice (nx, ny, precision, walls): a checkpoint
    # of another one is refused with LBM_ERR_ARG, a short or missing file
    # with LBM_ERR_IO, before any device copy, and the handle stays usable
    from paper_2106_01557_gb300 import lbm
    o = oracle_case(72, 40)
    fields = slab_fields(o, seed=13)
    a = gpu_case(72, 40, "f32")
    a.set_fields(*fields)
    a.step(3)
    path = tmp_path / "ck.bin"
    a.save(str(path))
    short = tmp_path / "short.bin"
    short.write_bytes(path.read_bytes()[: path.stat().st_size // 2])
    # the header also carries a hash of the configuration: the same lattice
    # under another temperature or body force is refused too
    for other, code in ((gpu_case(72, 48, "f32"), -1), (gpu_case(72, 40, "f16s"), -1),
                        (gpu_case(72, 40, "f32", walls=1), -1), (gpu_case(72, 40, "f32", Tr0=0.85), -1),
                        (gpu_case(72, 40, "f32", accel_x=1e-6), -1)):
        with pytest.raises(lbm.LbmError) as e:
            other.load(str(path))
        assert e.value.code == code
    b = gpu_case(72, 40, "f32")
    b.set_fields(*fields)
    for bad in (short, tmp_path / "missing.bin"):
        with pytest.raises(lbm.LbmError) as e:
            b.load(str(bad))
        assert e.value.code == -7
    assert b.steps == 0
    b.step(3)
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_divergence_is_reported(gpu_lib):
    from paper_2106_01557_gb300 import lbm
    o = oracle_case(64, 64)
    fields = slab_fields(o, seed=12)
    g = gpu_case(64, 64, "f32")
    g.set_fields(*fields)
    f, gg = g.get_populations()
    f[:, 10, 10] = -1.0  # negative density at one node: a host-made fault
    g.set_populations(f, gg)
    g.step(1)
    with pytest.raises(lbm.LbmError) as e:
        g.synchronize()
    assert e.value.code == -4


@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_negative_temperature_is_reported(gpu_lib, prec):
    # a host-made fault in the energy field alone: one node's g populations
    # set to minus their value (rho e_k < 0, so T < 0), the density untouched;
    # the step's record counts it (out[6]) and the synchronising call reports
    # divergence. The separate record of the state counts it too.
    from paper_2106_01557_gb300 import lbm
    o = oracle_case(64, 64)
    fields = slab_fields(o, seed=13)
    g = gpu_case(64, 64, prec)
    g.set_fields(*fields)
    f, gg = g.get_populations()
    gg[:, 20, 30] = -gg[:, 20, 30]
    g.set_populations(f, gg)
    g.step(1)
    with pytest.raises(lbm.LbmError) as e:
        g.synchronize()
    assert e.value.code == -4
    assert g.step_stats()[6] >= 1


def test_tile_wait_that_runs_out_is_reported(gpu_lib):
    # Failure detection of the step kernel's bounded waits, without a fault:
    # with a zero bound a tile whose copies have not landed when its turn
    # comes times out (the first tile of every block always does), the
    # block ends its launch after its copies in flight have landed, and the
    # next synchronising call reports LBM_ERR_TIMEOUT. The handle stays
    # usable: with the default bound and the state set again it steps as a
    # fresh handle does, bit for bit.
    from paper_2106_01557_gb300 import lbm
    o = oracle_case(256, 128)
    fields = slab_fields(o, seed=21)
    a = gpu_case(256, 128, "f32")
    a.set_fields(*fields)
    a.set_tile_wait(0)
    a.step(3)
    with pytest.raises(lbm.LbmError) as e:
        a.synchronize()
    assert e.value.code == -5
    a.set_tile_wait(2_000_000_000)
    a.set_fields(*fields)
    a.step(25)                     # a captured graph of 20 steps and 5 single launches
    a.synchronize()
    b = gpu_case(256, 128, "f32")
    b.set_fields(*fields)
    b.step(25)
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    with pytest.raises(lbm.LbmError) as e:
        a.set_tile_wait(-1)
    assert e.value.code == -1


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cubic_term_elimination_matches_oracle(gpu_lib, prec):
    # the cubic-term elimination (oracle reading pinned by the sound-decay
    # asymmetry of a moving vapour) on the GPU path: a perturbed slab with
    # a flow of 0.1 c along a diagonal, so that every cubic term acts
    from paper_2106_01557_gb300 import inputs
    o = oracle_case(100, 37, cubic=1)
    p = o.p
    rho, ux, uy, T = slab_fields(o, seed=17)
    ux = ux + 0.07 * p.c
    uy = uy - 0.07 * p.c
    o.init_fields(rho, ux, uy, T)
    g = gpu_case(100, 37, prec, cubic=1)
    g.set_fields(rho, ux, uy, T)
    f0, g0 = g.get_populations()
    assert rel_err(f0, o.f) < (1e-14 if prec == "f64" else 5e-7)
    for n in (1, 49):
        o.step(n)
        g.step(n)
        f, gg = g.get_populations()
        assert rel_err(f, o.f) < TOL[prec], (n, rel_err(f, o.f))
        assert rel_err(gg, o.g) < TOL[prec], (n, rel_err(gg, o.g))
    # and the terms act: the same case without them differs well above the bound
    q = gpu_case(100, 37, prec)
    q.set_fields(rho, ux, uy, T)
    q.step(50)
    fq, _ = q.get_populations()
    assert rel_err(fq, o.f) > 10 * TOL[prec]
