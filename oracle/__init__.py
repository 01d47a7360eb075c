"""FP64 CPU oracle of the LBfoam free-surface foaming step.

TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
baseline leg of ``bench.py`` may import this package; the product path
(``paper_1908_04262_gb300``) never does.  The C source next to this file
shares no code with the CUDA path.

``build()`` compiles ``lbf_oracle.c`` with gcc (``-ffp-contract=off`` so
that every expression rounds exactly as written, on x86 and on Arm alike);
``OracleSim`` wraps the C entry points with numpy arrays.

Parity: every oracle function is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or library routines, except
the two-bubble coalescence timing of Sec. 3.3, which is qualitative in the
paper ("parity unpinned" for that experiment only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbf_oracle.so")

GAS, LIQ, IFC, WALL = 0, 1, 2, 3
FIELDS = {"rho": 0, "u": 1, "alpha": 2, "mass": 3, "conc": 4, "kappa": 5,
          "pi": 6, "normal": 7, "dstar": 8, "fpop": 9, "gpop": 10}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "lbf_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double), ("accel", ctypes.c_double * 3),
        ("rheo", ctypes.c_int),
        ("rheo_n", ctypes.c_double), ("rheo_k", ctypes.c_double),
        ("rheo_lambda", ctypes.c_double), ("rheo_a", ctypes.c_double),
        ("tau0", ctypes.c_double), ("tau_inf", ctypes.c_double),
        ("tau_min", ctypes.c_double), ("tau_max", ctypes.c_double),
        ("sigma", ctypes.c_double), ("k_pi", ctypes.c_double), ("d_max", ctypes.c_double),
        ("D", ctypes.c_double), ("kH", ctypes.c_double), ("RT", ctypes.c_double),
        ("c0", ctypes.c_double), ("q", ctypes.c_double), ("p0", ctypes.c_double),
        ("fill_height", ctypes.c_double),
        ("walls", ctypes.c_int), ("wall_u", ctypes.c_double * 3),
        ("atmosphere", ctypes.c_int), ("eps", ctypes.c_double),
        ("bubble_capacity", ctypes.c_int),
        ("collision", ctypes.c_int), ("trt_magic", ctypes.c_double),
        ("kappa", ctypes.c_int), ("mrt_rates", ctypes.c_double * 4),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.POINTER(_Config)]
        lib.or_destroy.argtypes = [P]
        lib.or_error.argtypes = [P]
        lib.or_set_cells.argtypes = [P, P, P, P, P, P]
        lib.or_nucleate.argtypes = [P, ctypes.c_int, P, P]
        lib.or_step.argtypes = [P, ctypes.c_int]
        lib.or_get.argtypes = [P, ctypes.c_int, P]
        lib.or_get_type.argtypes = [P, P]
        lib.or_get_label.argtypes = [P, P]
        lib.or_num_bubbles.argtypes = [P]
        lib.or_bubbles.argtypes = [P, P, P, P, P, P, P]
        lib.or_ledger.argtypes = [P, P]
        lib.or_debug_set_types.argtypes = [P, P]
        lib.or_debug_relabel.argtypes = [P]
        lib.or_plic_liquid_fraction.restype = ctypes.c_double
        lib.or_plic_liquid_fraction.argtypes = [ctypes.c_int, dp, ctypes.c_double]
        lib.or_hf_curvature.argtypes = [P, P]
        lib.or_plic_offset.restype = ctypes.c_double
        lib.or_plic_offset.argtypes = [ctypes.c_int, dp, ctypes.c_double]
        lib.or_lsq_kappa.restype = ctypes.c_double
        lib.or_lsq_kappa.argtypes = [ctypes.c_int, P, ctypes.c_int]
        lib.or_mrt_basis.argtypes = [ctypes.c_int, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_config(d: dict) -> _Config:
    c = _Config()
    for name, _ in _Config._fields_:
        if name in ("accel", "wall_u"):
            v = d.get(name, (0.0, 0.0, 0.0))
            getattr(c, name)[:] = [float(x) for x in v]
        elif name == "mrt_rates":
            getattr(c, name)[:] = [float(x) for x in d.get(name, (0.0, 0.0, 0.0, 0.0))]
        elif name in d:
            setattr(c, name, d[name])
    return c


def mrt_basis(dim: int):
    """The MRT moment basis (rows over the oracle's velocity order) and the
    group id of each row (``or_mrt_basis``)."""
    q = 9 if dim == 2 else 19
    M = np.zeros((q, q))
    g = np.zeros(q, np.int32)
    _load().or_mrt_basis(dim, _ptr(M), _ptr(g))
    return M, g


class OracleSim:
    """One oracle lattice.  ``cfg`` is a workload dictionary."""

    def __init__(self, cfg: dict):
        self.lib = _load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.nx, self.ny, self.nz = cfg["nx"], cfg["ny"], cfg["nz"]
        self.dim = 2 if self.nz == 1 else 3
        self.N = self.nx * self.ny * self.nz
        self.Q, self.QA = (9, 5) if self.dim == 2 else (19, 7)
        self.h = self.lib.or_create(ctypes.byref(self._c))
        if not self.h:
            raise RuntimeError("or_create failed")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle error %d" % rc)

    def step(self, n: int = 1):
        self._check(self.lib.or_step(self.h, int(n)))

    def nucleate(self, centres, radii):
        c = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(-1, 3))
        r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
        self._check(self.lib.or_nucleate(self.h, len(r), _ptr(c), _ptr(r)))

    def set_cells(self, types, rho, u, alpha, conc):
        t = np.ascontiguousarray(np.asarray(types, dtype=np.uint8).reshape(-1))
        r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
        uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
        c = np.ascontiguousarray(np.asarray(conc, dtype=np.float64).reshape(-1))
        assert t.size == self.N and r.size == self.N and uu.size == 3 * self.N
        self._check(self.lib.or_set_cells(self.h, _ptr(t), _ptr(r), _ptr(uu), _ptr(a), _ptr(c)))

    def get(self, name: str) -> np.ndarray:
        width = {"u": 3, "normal": 3, "fpop": self.Q, "gpop": self.QA}.get(name, 1)
        out = np.zeros(self.N * width, dtype=np.float64)
        self._check(self.lib.or_get(self.h, FIELDS[name], _ptr(out)))
        return out.reshape(self.N, width) if width > 1 else out

    def hf_curvature(self) -> np.ndarray:
        """Height-function curvature of the interface cells (0 elsewhere,
        NaN where a column meets a wall)."""
        out = np.zeros(self.N, dtype=np.float64)
        self._check(self.lib.or_hf_curvature(self.h, _ptr(out)))
        return out

    def types(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint8)
        self.lib.or_get_type(self.h, _ptr(out))
        return out

    def labels(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int32)
        self.lib.or_get_label(self.h, _ptr(out))
        return out

    def bubbles(self) -> dict:
        nb = self.lib.or_num_bubbles(self.h)
        k = max(nb, 1)
        d = dict(id=np.zeros(k, np.int32), root=np.zeros(k, np.int64), volume=np.zeros(k),
                 mass=np.zeros(k), pressure=np.zeros(k), atm=np.zeros(k, np.int32))
        self.lib.or_bubbles(self.h, _ptr(d["id"]), _ptr(d["root"]), _ptr(d["volume"]),
                            _ptr(d["mass"]), _ptr(d["pressure"]), _ptr(d["atm"]))
        return {key: v[:nb] for key, v in d.items()}

    def debug_set_types(self, types):
        t = np.ascontiguousarray(np.asarray(types, dtype=np.uint8).reshape(-1))
        self.lib.or_debug_set_types(self.h, _ptr(t))

    def debug_relabel(self):
        self._check(self.lib.or_debug_relabel(self.h))

    def ledger(self) -> np.ndarray:
        out = np.zeros(8)
        self.lib.or_ledger(self.h, _ptr(out))
        return out


def plic_liquid_fraction(dim: int, n, s: float) -> float:
    lib = _load()
    a = (ctypes.c_double * 3)(*[float(x) for x in (list(n) + [0.0] * 3)[:3]])
    return lib.or_plic_liquid_fraction(dim, a, float(s))


def plic_offset(dim: int, n, alpha: float) -> float:
    lib = _load()
    a = (ctypes.c_double * 3)(*[float(x) for x in (list(n) + [0.0] * 3)[:3]])
    return lib.or_plic_offset(dim, a, float(alpha))


def lsq_kappa(dim: int, pts) -> float:
    """Least-squares curvature of the given points (n x 3, local frame)."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    return lib.or_lsq_kappa(dim, _ptr(a), a.shape[0])
