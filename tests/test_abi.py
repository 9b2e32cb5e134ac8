"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/lbm.h declares, and its
ctypes structures match the header's layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lbm_[A-Za-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_01557_gb300 import build
    path = build.build()
    return ctypes.CDLL(path), path


def test_library_exports_every_declared_function(lib):
    l, path = lib
    names = declared_functions()
    assert "lbm_init" in names and "lbm_step" in names and "lbm_moments" in names
    for n in names:
        assert hasattr(l, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header(lib):
    from paper_2106_01557_gb300 import lbm
    for n in declared_functions():
        if n.startswith("lbm_batch") or n.startswith("lbm_surrogate"):
            continue
        assert n in lbm.SIGNATURES, n


def test_struct_layout_matches_header():
    # compile a tiny C program against the header and compare offsets
    from paper_2106_01557_gb300 import lbm
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "lbm.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbm_config), offsetof(lbm_config, Tr_hot),
             offsetof(lbm_config, rho_ref), offsetof(lbm_config, stream), sizeof(lbm_params),
             offsetof(lbm_params, sq), offsetof(lbm_config, open_sides), offsetof(lbm_config, rho_open),
             offsetof(lbm_config, cubic));
      return 0;
    }'''
    tmp = os.path.join(ROOT, "paper_2106_01557_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "layout.c")
    exe = os.path.join(tmp, "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    C, P = lbm.LbmConfig, lbm.LbmParams
    assert got == [ctypes.sizeof(C), C.Tr_hot.offset, C.rho_ref.offset, C.stream.offset,
                   ctypes.sizeof(P), P.sq.offset, C.open_sides.offset, C.rho_open.offset, C.cubic.offset]


def test_default_config_and_argument_errors_without_gpu(lib):
    from paper_2106_01557_gb300 import lbm
    cfg = lbm.default_config(64, 32)
    assert cfg.K_EOS == pytest.approx(0.479820) and cfg.K_INT == pytest.approx(2.294922)
    assert cfg.varpi == pytest.approx(1 / 6) and cfg.gamma1 == -2 and cfg.gamma2 == 2
    l = lbm.load()
    bad = lbm.default_config(4, 32)
    h = ctypes.c_void_p()
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert b"nx" in l.lbm_last_error()
    bad = lbm.default_config(64, 32, s_p=2.5)
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = lbm.default_config(64, 32, Tr0=1.2)
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    # size limits: at least 8 x 8 nodes, at most 2^31 nodes (rejected before any device call)
    bad = lbm.default_config(64, 7)
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = lbm.default_config(65536, 32769)
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert b"too large" in l.lbm_last_error()
    # 16-bit storage rounds stochastically by default; only 0 and 1 are valid
    assert lbm.default_config(64, 32).rounding == 1
    bad = lbm.default_config(64, 32, precision="f16s", rounding=2)
    assert l.lbm_init(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert b"rounding" in l.lbm_last_error()


def test_library_maxwell_matches_oracle_on_host(lib):
    # the library's own coexistence solver (host code, no GPU) against the
    # oracle's, over the benchmark temperature range
    from oracle import thermo
    from paper_2106_01557_gb300 import lbm
    cfg = lbm.default_config(64, 64)
    Tc, _ = thermo.critical_point(1.0, 4.0, 1.0)
    for Tr in (0.6, 0.7, 0.8, 0.85, 0.9, 0.95):
        rv, rl, ps = lbm.maxwell(cfg, Tr)
        ov, ol, ops = thermo.maxwell(Tr * Tc, 1.0, 4.0, 1.0)
        assert rv == pytest.approx(ov, rel=1e-12)
        assert rl == pytest.approx(ol, rel=1e-12)
        assert ps == pytest.approx(cfg.K_EOS * ops, rel=1e-12)
    with pytest.raises(lbm.LbmError):
        lbm.maxwell(cfg, 1.1)


def test_library_laplace_coexistence_and_surface_tension_on_host(lib):
    # the library's host solvers for the curved-interface reference of the
    # batched sweep, against the oracle's thermodynamics: its surface
    # tension (square-gradient theory, the paper's sigma = 0.01 at T_r 0.8),
    # and coexistence with a pressure jump, which must keep the chemical
    # potentials equal and carry the jump
    from oracle import thermo
    from paper_2106_01557_gb300 import lbm
    cfg = lbm.default_config(64, 64)
    Tc, _ = thermo.critical_point(1.0, 4.0, 1.0)
    for Tr in (0.65, 0.8, 0.9):
        sig = lbm.surface_tension(cfg, Tr)
        osig, _ = thermo.surface_tension_and_width(Tr * Tc, 1.0, 4.0, 1.0, cfg.K_EOS, cfg.K_INT)
        assert sig == pytest.approx(osig, rel=1e-8), Tr
        for R in (10.0, 40.0):
            rv, rl, pv = lbm.coexistence(cfg, Tr, sig / R)
            T = Tr * Tc
            assert thermo.mu(rv, T, 1.0, 4.0, 1.0) == pytest.approx(thermo.mu(rl, T, 1.0, 4.0, 1.0), rel=1e-12)
            assert (thermo.p_eos(rl, T, 1.0, 4.0, 1.0, cfg.K_EOS) - thermo.p_eos(rv, T, 1.0, 4.0, 1.0, cfg.K_EOS)
                    == pytest.approx(sig / R, rel=1e-9))
            mv, ml, _ = thermo.maxwell(T, 1.0, 4.0, 1.0)
            assert rv > mv and rl > ml        # a droplet's vapour and liquid are both denser
    assert lbm.surface_tension(cfg, 0.8) == pytest.approx(0.01, rel=1e-5)
    assert lbm.coexistence(cfg, 0.8, 0.0)[:2] == pytest.approx(lbm.maxwell(cfg, 0.8)[:2], rel=1e-14)


def test_library_eos_pressure_on_host(lib):
    # the library's Eq. 17 against the oracle's, on both branches and in the
    # spinodal region, with K_EOS away from 1; it equals the saturation
    # pressure at both Maxwell densities; out-of-range densities are refused
    from oracle import thermo
    from paper_2106_01557_gb300 import lbm
    cfg = lbm.default_config(64, 64)
    cfg.K_EOS = 0.7
    Tc, _ = thermo.critical_point(1.0, 4.0, 1.0)
    for Tr in (0.65, 0.8, 0.95):
        T = Tr * Tc
        for rho in (0.01, 0.1, 0.3, 0.6, 0.9):
            assert lbm.eos_pressure(cfg, rho, T) == pytest.approx(thermo.p_eos(rho, T, 1.0, 4.0, 1.0, 0.7), rel=1e-13)
        rv, rl, ps = lbm.maxwell(cfg, Tr)
        assert lbm.eos_pressure(cfg, rv, T) == pytest.approx(ps, rel=1e-10)
        assert lbm.eos_pressure(cfg, rl, T) == pytest.approx(ps, rel=1e-9)
    for bad in (0.0, -0.1, 1.0, 2.0):
        with pytest.raises(lbm.LbmError):
            lbm.eos_pressure(cfg, bad, 0.1)


def test_null_arguments_are_rejected_without_gpu(lib):
    # every entry point checks its handle and required pointers before any
    # device work: LBM_ERR_ARG, a no-op for the destroy calls, -1 or 0 for the
    # count queries, and lbm_default_config(NULL) returns without writing
    from paper_2106_01557_gb300 import lbm
    l = lbm.load()
    skip = {"lbm_last_error"}
    noop = {"lbm_destroy", "lbm_batch_destroy", "lbm_surrogate_destroy"}
    queries = {"lbm_step_count": -1, "lbm_batch_step_count": -1, "lbm_bytes_per_step": 0.0, "lbm_batch_nodes": 0,
               "lbm_batch_bytes_per_step": 0.0, "lbm_surrogate_num_params": 0}
    for name, (args, res) in lbm.SIGNATURES.items():
        if name in skip:
            continue
        vals = []
        for a in args:
            if a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64):
                vals.append(0)
            elif a is ctypes.c_double:
                vals.append(0.8)
            else:
                vals.append(None)
        got = getattr(l, name)(*vals)
        if name == "lbm_default_config":
            assert got is None
        elif name in noop:
            assert got == 0, name
        elif name in queries:
            assert got == queries[name], name
        else:
            assert got == -1, name
            assert l.lbm_last_error(), name
