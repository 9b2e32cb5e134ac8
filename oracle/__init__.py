"""FP64 CPU oracle of the liquid-vapor lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

``thermo`` holds the thermodynamics and parameter derivation (Python, FP64);
``lbm_oracle.c`` holds one time step, initialisation and moments (plain C,
FP64), built here with gcc and called through ctypes.

Parity status of each function is stated in its docstring. The g source
q_m (SM Eq. S4b) is pinned against the moments of the textbook second-order
scalar source (rows 0, 1 and 3-8; row eps, gamma2 q, is a literal reading).
The coefficient k s_eps omega_e of S
(row e, column eps; SM Eq. S5a) is pinned only through the linear stability
of the moving vapour, the walls (not in the paper) only through textbook
flows (Poiseuille, steady conduction), and the open heated sides (not in the
paper) through the Stefan problem (Eq. 20, 21) and the quasi-steady
evaporation of a droplet.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import thermo

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, strict IEEE: no -ffast-math, no FMA
    contraction so that the oracle's rounding is the textbook one). OpenMP
    splits the independent per-node loops across host cores; results do not
    depend on the thread count."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("walls", ctypes.c_int),
        ("c", ctypes.c_double), ("dt", ctypes.c_double), ("G2", ctypes.c_double),
        ("a", ctypes.c_double), ("kappa", ctypes.c_double), ("cs2", ctypes.c_double),
        ("R", ctypes.c_double), ("a_t", ctypes.c_double), ("b_t", ctypes.c_double),
        ("K_EOS", ctypes.c_double), ("cv", ctypes.c_double), ("Cref", ctypes.c_double),
        ("varpi", ctypes.c_double), ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
        ("beta", ctypes.c_double), ("kS", ctypes.c_double), ("hS", ctypes.c_double),
        ("bS", ctypes.c_double),
        ("s0", ctypes.c_double), ("se", ctypes.c_double), ("seps", ctypes.c_double),
        ("sj", ctypes.c_double), ("sq", ctypes.c_double), ("sp", ctypes.c_double),
        ("sig0", ctypes.c_double), ("sige", ctypes.c_double), ("sigeps", ctypes.c_double),
        ("sigp", ctypes.c_double),
        ("tauj_v", ctypes.c_double), ("tauj_l", ctypes.c_double),
        ("rho_v", ctypes.c_double), ("rho_l", ctypes.c_double),
        ("ax", ctypes.c_double), ("ay", ctypes.c_double),
        ("T_bottom", ctypes.c_double), ("T_top", ctypes.c_double), ("T_hot", ctypes.c_double),
        ("hot_x0", ctypes.c_int), ("hot_len", ctypes.c_int),
        ("open_sides", ctypes.c_int), ("rho_out", ctypes.c_double), ("T_open", ctypes.c_double),
        ("cubic", ctypes.c_int),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(OrcParams)
            lib.orc_step.argtypes = [pp, dp, dp, ctypes.c_int]
            lib.orc_step.restype = ctypes.c_int
            lib.orc_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            lib.orc_init.restype = ctypes.c_int
            lib.orc_moments.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_moments.restype = ctypes.c_int
            lib.orc_collide_node.argtypes = [pp, dp, dp, dp, dp, dp, dp]
            lib.orc_collide_node.restype = None
            lib.orc_collide_node_r.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
            lib.orc_collide_node_r.restype = None
            lib.orc_get_M.argtypes = [dp, dp]
            lib.orc_get_M.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def c_params(p: thermo.Params) -> OrcParams:
    o = OrcParams()
    for name, _ in OrcParams._fields_:
        if name == "cs2":
            o.cs2 = p.cs * p.cs
        else:
            setattr(o, name, getattr(p, name))
    return o


def M_and_inverse():
    """M of SM Eq. S2 and its Gauss-Jordan inverse as the oracle uses them."""
    lib = _load()
    M = np.zeros((9, 9))
    Mi = np.zeros((9, 9))
    lib.orc_get_M(_ptr(M), _ptr(Mi))
    return M, Mi


class Oracle:
    """One case of the FP64 oracle: populations f, g of shape (9, ny, nx)
    holding the post-streaming state whose moments Eq. 14 defines."""

    def __init__(self, cfg: thermo.Config, params: thermo.Params | None = None):
        self.cfg = cfg
        self.p = params if params is not None else thermo.derive_params(cfg)
        self.cp = c_params(self.p)
        self.lib = _load()
        self.nx, self.ny = cfg.nx, cfg.ny
        self.f = np.zeros((9, self.ny, self.nx))
        self.g = np.zeros((9, self.ny, self.nx))

    def init_fields(self, rho, ux, uy, T):
        rho, ux, uy, T = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T))
        self.lib.orc_init(ctypes.byref(self.cp), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T),
                          _ptr(self.f), _ptr(self.g))

    def set_populations(self, f, g):
        self.f = np.ascontiguousarray(f, dtype=np.float64).copy()
        self.g = np.ascontiguousarray(g, dtype=np.float64).copy()

    def step(self, n: int = 1):
        rc = self.lib.orc_step(ctypes.byref(self.cp), _ptr(self.f), _ptr(self.g), int(n))
        if rc != 0:
            raise MemoryError("oracle step allocation failed")

    def moments(self):
        """dict of (ny, nx) fields: rho, ux, uy, T, Fpx, Fpy, q, rek."""
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "T", "Fpx", "Fpy", "q", "rek")}
        self.lib.orc_moments(ctypes.byref(self.cp), _ptr(self.f), _ptr(self.g),
                             *(_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "Fpx", "Fpy", "q", "rek")))
        return out

    def conservation(self):
        """[mass, sum rho u_x, sum rho u_y, sum rho e_k, total energy, max |u|] of
        the current state (Eq. 6 quantities; rho e = rho e_k + rho eps_p with
        rho eps_p = rho V_mean / 2, V_mean = -2 a rho - kappa lap rho, Eq. 8)."""
        m = self.moments()
        rho = m["rho"]
        lap = laplacian9(rho, self.p.walls)
        e_tot = m["rek"] - self.p.a * rho * rho - 0.5 * self.p.kappa * rho * lap
        return np.array([rho.sum(), (rho * m["ux"]).sum(), (rho * m["uy"]).sum(),
                         m["rek"].sum(), e_tot.sum(),
                         np.sqrt(m["ux"] ** 2 + m["uy"] ** 2).max()])

    def collide_node(self, fl, gl, rho_nb, dphi=None):
        """One node's collision; dphi = the central differences (d_x(rho
        u_x^3), d_y(rho u_y^3)) at the node, u over c, from which the
        cubic-term source is formed (None: no source)."""
        fl, gl, rho_nb = (np.ascontiguousarray(a, dtype=np.float64) for a in (fl, gl, rho_nb))
        fb = np.zeros(9)
        gb = np.zeros(9)
        macro = np.zeros(8)
        if dphi is None:
            self.lib.orc_collide_node(ctypes.byref(self.cp), _ptr(fl), _ptr(gl), _ptr(rho_nb),
                                      _ptr(fb), _ptr(gb), _ptr(macro))
        else:
            r = np.ascontiguousarray(dphi, dtype=np.float64)
            self.lib.orc_collide_node_r(ctypes.byref(self.cp), _ptr(fl), _ptr(gl), _ptr(rho_nb), _ptr(r),
                                        _ptr(fb), _ptr(gb), _ptr(macro))
        return fb, gb, macro


def laplacian9(rho, walls=0):
    """Isotropic 9-point Laplacian with the pair-force weights (1/3, 1/12):
    lap rho = 2 sum_i omega_i (rho(x + e_i) - rho(x)), dx = 1."""
    ex = [1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 1, 0, -1, 1, 1, -1, -1]
    w = [1 / 3] * 4 + [1 / 12] * 4
    if walls:
        padded = np.pad(rho, ((1, 1), (0, 0)), mode="edge")
    else:
        padded = np.pad(rho, ((1, 1), (0, 0)), mode="wrap")
    out = np.zeros_like(rho)
    for k in range(8):
        nb = np.roll(padded, (-ey[k], -ex[k]), axis=(0, 1))[1:-1]
        out += 2.0 * w[k] * (nb - rho)
    return out
