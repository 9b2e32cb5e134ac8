"""Thin ctypes binding of liblbm (include/lbm.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
converts numpy arrays and torch tensors to pointers and status codes to
exceptions. There is no fallback: if the shared library or a CUDA device is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S = 0, 1, 2, 3
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16s": LBM_BF16S}
ERRORS = {-1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM", -4: "LBM_ERR_DIVERGED",
          -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE", -7: "LBM_ERR_IO"}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class LbmConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("walls", ctypes.c_int32),
        ("a_t", ctypes.c_double), ("b_t", ctypes.c_double), ("R", ctypes.c_double),
        ("K_EOS", ctypes.c_double), ("K_INT", ctypes.c_double), ("Tr0", ctypes.c_double),
        ("varpi", ctypes.c_double), ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
        ("s_p", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("sig_e", ctypes.c_double), ("sig_eps", ctypes.c_double), ("sig_p", ctypes.c_double),
        ("tau_j_v", ctypes.c_double), ("tau_j_l", ctypes.c_double),
        ("c_v", ctypes.c_double), ("C_ref", ctypes.c_double),
        ("accel_x", ctypes.c_double), ("accel_y", ctypes.c_double),
        ("Tr_bottom", ctypes.c_double), ("Tr_top", ctypes.c_double), ("Tr_hot", ctypes.c_double),
        ("hot_x0", ctypes.c_int32), ("hot_len", ctypes.c_int32),
        ("rho_ref", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int32), ("rounding", ctypes.c_int32),
        ("open_sides", ctypes.c_int32), ("Tr_open", ctypes.c_double), ("rho_open", ctypes.c_double),
        ("cubic", ctypes.c_int32),
    ]


class LbmParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "Tc", "pc", "T0", "rho_v", "rho_l", "p_s", "cs", "c", "dt", "G2", "a", "kappa",
        "cv", "Cref", "beta", "kS", "hS", "bS", "se", "sq", "rho_open", "T_open")]


_lib = None
_lock = threading.Lock()

_DP = ctypes.POINTER(ctypes.c_double)
_H = ctypes.c_void_p

SIGNATURES = {
    "lbm_last_error": ([], ctypes.c_char_p),
    "lbm_default_config": ([ctypes.POINTER(LbmConfig), ctypes.c_int32, ctypes.c_int32], None),
    "lbm_init": ([ctypes.POINTER(LbmConfig), ctypes.POINTER(_H)], ctypes.c_int),
    "lbm_get_params": ([_H, ctypes.POINTER(LbmParams)], ctypes.c_int),
    "lbm_set_fields": ([_H, _DP, _DP, _DP, _DP, ctypes.c_int], ctypes.c_int),
    "lbm_step": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_moments": ([_H, _DP, _DP, _DP, _DP, ctypes.c_int], ctypes.c_int),
    "lbm_conservation": ([_H, _DP], ctypes.c_int),
    "lbm_step_stats": ([_H, _DP], ctypes.c_int),
    "lbm_get_populations": ([_H, _DP, _DP], ctypes.c_int),
    "lbm_set_populations": ([_H, _DP, _DP], ctypes.c_int),
    "lbm_save": ([_H, ctypes.c_char_p], ctypes.c_int),
    "lbm_load": ([_H, ctypes.c_char_p], ctypes.c_int),
    "lbm_synchronize": ([_H], ctypes.c_int),
    "lbm_step_count": ([_H], ctypes.c_int64),
    "lbm_bytes_per_step": ([_H], ctypes.c_double),
    "lbm_destroy": ([_H], ctypes.c_int),
    "lbm_batch_init": ([ctypes.POINTER(LbmConfig), ctypes.c_int32, ctypes.POINTER(_H)], ctypes.c_int),
    "lbm_batch_set_fields": ([_H, ctypes.c_int32, _DP, _DP, _DP, _DP, ctypes.c_int], ctypes.c_int),
    "lbm_batch_step": ([_H, ctypes.c_int], ctypes.c_int),
    "lbm_batch_moments": ([_H, ctypes.c_int32, _DP, _DP, _DP, _DP, ctypes.c_int], ctypes.c_int),
    "lbm_batch_conservation": ([_H, ctypes.c_int32, _DP], ctypes.c_int),
    "lbm_batch_get_populations": ([_H, ctypes.c_int32, _DP, _DP], ctypes.c_int),
    "lbm_batch_step_stats": ([_H, ctypes.c_int32, _DP], ctypes.c_int),
    "lbm_batch_autotune": ([_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), _DP], ctypes.c_int),
    "lbm_batch_select": ([_H, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    "lbm_batch_synchronize": ([_H], ctypes.c_int),
    "lbm_batch_get_params": ([_H, ctypes.c_int32, ctypes.POINTER(LbmParams)], ctypes.c_int),
    "lbm_maxwell": ([ctypes.POINTER(LbmConfig), ctypes.c_double, _DP], ctypes.c_int),
    "lbm_coexistence": ([ctypes.POINTER(LbmConfig), ctypes.c_double, ctypes.c_double, _DP], ctypes.c_int),
    "lbm_surface_tension": ([ctypes.POINTER(LbmConfig), ctypes.c_double, _DP], ctypes.c_int),
    "lbm_eos_pressure": ([ctypes.POINTER(LbmConfig), ctypes.c_double, ctypes.c_double, _DP], ctypes.c_int),
    "lbm_batch_nodes": ([_H], ctypes.c_int64),
    "lbm_batch_step_count": ([_H], ctypes.c_int64),
    "lbm_batch_set_tile_wait": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm_batch_bytes_per_step": ([_H], ctypes.c_double),
    "lbm_batch_destroy": ([_H], ctypes.c_int),
    "lbm_surrogate_create": ([ctypes.c_void_p, ctypes.POINTER(_H)], ctypes.c_int),
    "lbm_surrogate_num_params": ([_H], ctypes.c_int64),
    "lbm_surrogate_set_params": ([_H, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "lbm_surrogate_get_params": ([_H, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "lbm_surrogate_forward": ([_H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p],
                              ctypes.c_int),
    "lbm_surrogate_loss_grad": ([_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 _DP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "lbm_surrogate_train_step": ([_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_double, _DP], ctypes.c_int),
    "lbm_surrogate_rollout": ([_H, _H, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, _DP], ctypes.c_int),
    "lbm_set_tile_wait": ([_H, ctypes.c_int64], ctypes.c_int),
    "lbm_surrogate_destroy": ([_H], ctypes.c_int),
    "lbm_conservation_noalloc": ([ctypes.POINTER(LbmConfig), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p], ctypes.c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it in-tree with nvcc if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library not built: {path}")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise LbmError(rc, _lib.lbm_last_error().decode())


def _host_ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _dev_ptr(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), _DP)


def default_config(nx: int, ny: int, **overrides) -> LbmConfig:
    lib = load()
    cfg = LbmConfig()
    lib.lbm_default_config(ctypes.byref(cfg), int(nx), int(ny))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(cfg, k, v)
    return cfg


def maxwell(cfg: LbmConfig, Tr: float):
    """Coexistence densities (rho_v, rho_l) and saturation pressure of the
    EOS of cfg at reduced temperature Tr, from the library's host solver."""
    out = np.zeros(3)
    _check(load().lbm_maxwell(ctypes.byref(cfg), float(Tr), _host_ptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def coexistence(cfg: LbmConfig, Tr: float, dp: float = 0.0):
    """Densities (rho_v, rho_l) with equal chemical potential whose pressures
    differ by dp (Laplace's law: sigma / R), and the vapour's pressure, from
    the library's host solver."""
    out = np.zeros(3)
    _check(load().lbm_coexistence(ctypes.byref(cfg), float(Tr), float(dp), _host_ptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def surface_tension(cfg: LbmConfig, Tr: float) -> float:
    """Planar surface tension at Tr from square-gradient theory (library host code)."""
    out = np.zeros(1)
    _check(load().lbm_surface_tension(ctypes.byref(cfg), float(Tr), _host_ptr(out)))
    return float(out[0])


def eos_pressure(cfg: LbmConfig, rho: float, T: float) -> float:
    """The full EOS (Eq. 17) at density rho and temperature T (library host code)."""
    out = np.zeros(1)
    _check(load().lbm_eos_pressure(ctypes.byref(cfg), float(rho), float(T), _host_ptr(out)))
    return float(out[0])


NOALLOC_MAX_NODES = 1 << 20


def conservation_noalloc(cfg: LbmConfig, f, g, out, stream=None):
    """lbm_conservation_noalloc: f, g CUDA float64 tensors (9, ny, nx), out a
    CUDA float64 tensor of >= 7 entries; asynchronous on `stream` (a
    torch.cuda.Stream or None for the legacy default stream). Allocates
    nothing, for callers that cannot allocate device memory."""
    lib = load()
    for t in (f, g, out):
        assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"
    import torch
    if stream is None:
        torch.cuda.current_stream().synchronize()
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib.lbm_conservation_noalloc(ctypes.byref(cfg), ctypes.c_void_p(f.data_ptr()),
                                        ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()), s))


class Lattice:
    """One case on the GPU. Fields are numpy (host) arrays or CUDA torch
    tensors of float64, shape (ny, nx); populations (9, ny, nx)."""

    def __init__(self, cfg: LbmConfig):
        self.lib = load()
        self.cfg = cfg
        h = _H()
        _check(self.lib.lbm_init(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.nx, self.ny = cfg.nx, cfg.ny

    @classmethod
    def create(cls, nx, ny, **overrides):
        return cls(default_config(nx, ny, **overrides))

    def close(self):
        if self.h:
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> dict:
        p = LbmParams()
        _check(self.lib.lbm_get_params(self.h, ctypes.byref(p)))
        return {n: getattr(p, n) for n, _ in LbmParams._fields_}

    def set_fields(self, rho, ux, uy, T):
        arrs = (rho, ux, uy, T)
        if hasattr(rho, "data_ptr"):
            import torch
            for a in arrs:
                assert a.is_cuda and a.is_contiguous() and str(a.dtype) == "torch.float64"
            # the handle's stream is not ordered after torch's: finish the producers
            torch.cuda.current_stream().synchronize()
            _check(self.lib.lbm_set_fields(self.h, *(_dev_ptr(a) for a in arrs), 1))
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
            _check(self.lib.lbm_set_fields(self.h, *(_host_ptr(a) for a in arrs), 0))

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self.h, int(n)))

    def synchronize(self):
        _check(self.lib.lbm_synchronize(self.h))

    def moments(self, out=None):
        """dict rho, ux, uy, T as (ny, nx) float64 host arrays; with out = a
        dict of CUDA float64 tensors, filled on the device; with out = a dict
        of C-contiguous float64 numpy arrays (e.g. pinned host memory),
        filled in place."""
        if out is not None:
            keys = ("rho", "ux", "uy", "T")
            if isinstance(out["rho"], np.ndarray):
                _check(self.lib.lbm_moments(self.h, *(_host_ptr(out[k]) for k in keys), 0))
                return out
            import torch
            torch.cuda.current_stream().synchronize()
            _check(self.lib.lbm_moments(self.h, *(_dev_ptr(out[k]) for k in keys), 1))
            return out
        res = {k: np.empty((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T")}
        _check(self.lib.lbm_moments(self.h, *(_host_ptr(res[k]) for k in ("rho", "ux", "uy", "T")), 0))
        return res

    def conservation(self, allow_diverged=False) -> np.ndarray:
        """Mass, momentum, sum rho e_k, total energy, max |u| of the current
        state; raises LbmError (LBM_ERR_DIVERGED) if a node has a
        non-positive or non-finite density or temperature, unless
        allow_diverged (the record is then returned all the same)."""
        out = np.zeros(6)
        rc = self.lib.lbm_conservation(self.h, _host_ptr(out))
        if not (allow_diverged and rc == -4):
            _check(rc)
        return out

    def step_stats(self) -> np.ndarray:
        out = np.zeros(8)
        _check(self.lib.lbm_step_stats(self.h, _host_ptr(out)))
        return out

    def get_populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        _check(self.lib.lbm_get_populations(self.h, _host_ptr(f), _host_ptr(g)))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        _check(self.lib.lbm_set_populations(self.h, _host_ptr(f), _host_ptr(g)))

    def save(self, path: str):
        _check(self.lib.lbm_save(self.h, path.encode()))

    def load(self, path: str):
        _check(self.lib.lbm_load(self.h, path.encode()))

    @property
    def steps(self) -> int:
        return int(self.lib.lbm_step_count(self.h))

    def set_tile_wait(self, ns: int):
        """Bound (ns) on each wait of the step kernel for a tile's copies;
        0: no waiting. A wait that runs out is reported by the next
        synchronising call as LBM_ERR_TIMEOUT."""
        _check(self.lib.lbm_set_tile_wait(self.h, int(ns)))

    def bytes_per_step(self) -> float:
        return float(self.lib.lbm_bytes_per_step(self.h))


class Batch:
    """Many independent periodic cases advanced together (lbm_batch_*).
    cfgs: list of LbmConfig, one precision for all (f32, f16s or bf16s)."""

    ORDERS = ("case-major", "largest-first", "round-robin")

    def __init__(self, cfgs):
        self.lib = load()
        self.cfgs = list(cfgs)
        arr = (LbmConfig * len(self.cfgs))(*self.cfgs)
        h = _H()
        _check(self.lib.lbm_batch_init(arr, len(self.cfgs), ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.cfgs)

    def set_fields(self, i, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, T)]
        _check(self.lib.lbm_batch_set_fields(self.h, int(i), *(_host_ptr(a) for a in arrs), 0))

    def step(self, n=1):
        _check(self.lib.lbm_batch_step(self.h, int(n)))

    def synchronize(self):
        _check(self.lib.lbm_batch_synchronize(self.h))

    def moments(self, i):
        c = self.cfgs[i]
        res = {k: np.empty((c.ny, c.nx)) for k in ("rho", "ux", "uy", "T")}
        _check(self.lib.lbm_batch_moments(self.h, int(i), *(_host_ptr(res[k]) for k in ("rho", "ux", "uy", "T")), 0))
        return res

    def conservation(self, i):
        out = np.zeros(6)
        _check(self.lib.lbm_batch_conservation(self.h, int(i), _host_ptr(out)))
        return out

    def get_populations(self, i):
        c = self.cfgs[i]
        f = np.empty((9, c.ny, c.nx))
        g = np.empty((9, c.ny, c.nx))
        _check(self.lib.lbm_batch_get_populations(self.h, int(i), _host_ptr(f), _host_ptr(g)))
        return f, g

    def step_stats(self, i):
        out = np.zeros(8)
        _check(self.lib.lbm_batch_step_stats(self.h, int(i), _host_ptr(out)))
        return out

    @property
    def steps(self) -> int:
        return int(self.lib.lbm_batch_step_count(self.h))

    def set_tile_wait(self, ns: int):
        """Bound (ns) on each wait of the batch kernel for an item's copies; 0: no waiting."""
        _check(self.lib.lbm_batch_set_tile_wait(self.h, int(ns)))

    def autotune(self, trial_steps=10):
        choice = (ctypes.c_int32 * 2)()
        ms = np.zeros(6)
        _check(self.lib.lbm_batch_autotune(self.h, int(trial_steps), choice, _host_ptr(ms)))
        return (int(choice[0]), int(choice[1])), ms

    def params(self, i) -> dict:
        p = LbmParams()
        _check(self.lib.lbm_batch_get_params(self.h, int(i), ctypes.byref(p)))
        return {n: getattr(p, n) for n, _ in LbmParams._fields_}

    def select(self, shape, order):
        _check(self.lib.lbm_batch_select(self.h, int(shape), int(order)))

    @property
    def nodes(self):
        return int(self.lib.lbm_batch_nodes(self.h))

    def bytes_per_step(self):
        return float(self.lib.lbm_batch_bytes_per_step(self.h))


class SurrogateConfig(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int32), ("blocks", ctypes.c_int32), ("K", ctypes.c_int32),
                ("conv_path", ctypes.c_int32), ("norm_off", ctypes.c_double * 4),
                ("norm_scale", ctypes.c_double * 4), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("conserve_mass", ctypes.c_int32)]


class Surrogate:
    """The learned surrogate (lbm_surrogate_*). Fields are CUDA float64
    tensors of shape (4, N, H, W) = (rho, u_x, u_y, T); parameters are a flat
    float32 numpy array in the library's order."""

    def __init__(self, norm_off, norm_scale, K=50, channels=64, blocks=6, stream=None, conv_path="tcgen05",
                 conserve_mass=True):
        """stream: a torch.cuda.Stream to issue the work on (None: a stream of
        the library's own). Every call first waits for torch's current
        stream, so that the tensors it reads are complete. conv_path:
        "tcgen05" (tensor-memory accumulators) or "mma" (warp-level MMAs) for
        the 3x3 convolutions. conserve_mass: the output layer that keeps each
        image's mass."""
        self.lib = load()
        cfg = SurrogateConfig()
        cfg.channels, cfg.blocks, cfg.K = channels, blocks, K
        if conv_path not in ("tcgen05", "mma"):
            raise ValueError("conv_path must be 'tcgen05' or 'mma'")
        cfg.conv_path = 0 if conv_path == "tcgen05" else 1
        cfg.conserve_mass = 1 if conserve_mass else 0
        self.conserve_mass = bool(conserve_mass)
        for i in range(4):
            cfg.norm_off[i] = float(norm_off[i])
            cfg.norm_scale[i] = float(norm_scale[i])
        cfg.stream = None if stream is None else stream.cuda_stream
        self.cfg = cfg
        self.norm_off = [float(v) for v in norm_off]
        self.norm_scale = [float(v) for v in norm_scale]
        h = _H()
        _check(self.lib.lbm_surrogate_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.K = K
        self.channels, self.blocks = channels, blocks

    def close(self):
        if self.h:
            self.lib.lbm_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(self.lib.lbm_surrogate_num_params(self.h))

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params
        _check(self.lib.lbm_surrogate_set_params(self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self):
        out = np.empty(self.num_params, dtype=np.float32)
        _check(self.lib.lbm_surrogate_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    @staticmethod
    def _dims(t):
        import torch
        assert t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64" and t.shape[0] == 4
        # the library's stream is not ordered after torch's: finish the producers
        torch.cuda.current_stream().synchronize()
        return int(t.shape[1]), int(t.shape[2]), int(t.shape[3])

    def forward(self, fields, out):
        N, H, W = self._dims(fields)
        _check(self.lib.lbm_surrogate_forward(self.h, ctypes.c_void_p(fields.data_ptr()), N, H, W,
                                              ctypes.c_void_p(out.data_ptr())))
        return out

    def loss_grad(self, fields, target, grads=True):
        N, H, W = self._dims(fields)
        loss = ctypes.c_double()
        g = np.empty(self.num_params, dtype=np.float32) if grads else None
        _check(self.lib.lbm_surrogate_loss_grad(self.h, ctypes.c_void_p(fields.data_ptr()),
                                                ctypes.c_void_p(target.data_ptr()), N, H, W, ctypes.byref(loss),
                                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if grads else None))
        return loss.value, g

    def train_step(self, fields, target, lr):
        N, H, W = self._dims(fields)
        loss = ctypes.c_double()
        _check(self.lib.lbm_surrogate_train_step(self.h, ctypes.c_void_p(fields.data_ptr()),
                                                 ctypes.c_void_p(target.data_ptr()), N, H, W, float(lr),
                                                 ctypes.byref(loss)))
        return loss.value

    def rollout(self, lattice, njumps, drift_tol=1e-3, iface_tol=0.5, verify_steps=None, field_tol=0.2):
        """drift_tol: largest relative change of mass and of total energy per
        jump; iface_tol: largest mean interface displacement per jump, in
        lattice units; verify_steps: LB steps run from each surrogate state
        before it is checked (default K / 10); field_tol: largest change of a
        node's density or temperature over those steps, relative to the
        field's largest value. Every jump advances the lattice by
        K + verify_steps steps."""
        import torch
        torch.cuda.current_stream().synchronize()
        if verify_steps is None:
            verify_steps = max(1, self.K // 10)
        self.verify_steps = int(verify_steps)
        stats = np.zeros(17)
        _check(self.lib.lbm_surrogate_rollout(self.h, lattice.h, int(njumps), int(verify_steps), float(drift_tol),
                                              float(iface_tol), float(field_tol), _host_ptr(stats)))
        return {"accepted": int(stats[0]), "fallbacks": int(stats[1]), "ms_surrogate": stats[2],
                "ms_fallback_lb": stats[3], "max_mass_drift": stats[4], "max_energy_drift": stats[5],
                "max_mass_drift_all": stats[6], "max_energy_drift_all": stats[7],
                "max_iface_displacement_all": stats[8], "unphysical": int(stats[9]),
                "verify_diverged": int(stats[10]), "verify_steps": int(verify_steps),
                "ms_read_state": stats[11], "ms_network": stats[12], "ms_check_reinit": stats[13],
                "ms_verify": stats[14], "max_local_change_rho_all": stats[15],
                "max_local_change_T_all": stats[16], "field_tol": float(field_tol)}


def surrogate_params_from_oracle_layout(p):
    """Flatten a parameter dict laid out as {'lift': (w, b), 'blocks': [((w1, b1), (w2, b2)), ...],
    'proj': (w, b)} with weights (9, Cout, Cin) into the library's order."""
    parts = [p["lift"][0], p["lift"][1]]
    for (w1, b1), (w2, b2) in p["blocks"]:
        parts += [w1, b1, w2, b2]
    parts += [p["proj"][0], p["proj"][1]]
    return np.concatenate([np.asarray(a, dtype=np.float32).reshape(-1) for a in parts])
