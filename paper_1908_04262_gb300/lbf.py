"""Python binding of the C ABI in ``include/lbf.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/liblbf.so``; this module
converts numpy arrays / torch tensors to pointers and error codes to
exceptions.  There is no CPU fallback: without the library or a GPU the
constructor raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbf.so")

STORAGE = {"fp64": 0, "fp32": 1, "fp16s": 2, "bf16s": 3}
FIELD_BITS = {"rho": 0, "u": 1, "alpha": 2, "mass": 3, "flags": 4, "conc": 5, "kappa": 6,
              "label": 7, "pi": 8, "normal": 9, "dstar": 10}
VECTOR_FIELDS = ("u", "normal")
INT_FIELDS = ("flags", "label")
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOTCONV", -5: "ENONFINITE",
          -6: "ECAPACITY"}


class LbfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("storage", ctypes.c_int),
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
        ("stream", ctypes.c_void_p),
    ]


class Bubble(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("atm", ctypes.c_int32), ("label", ctypes.c_int64),
                ("volume", ctypes.c_double), ("gas_mass", ctypes.c_double),
                ("pressure", ctypes.c_double)]


EXPORTS = ("lbf_create", "lbf_destroy", "lbf_nucleate", "lbf_set_cells", "lbf_step",
           "lbf_bubbles", "lbf_fields", "lbf_ledger", "lbf_timing_enable", "lbf_timing_read",
           "lbf_timing_name", "lbf_cell_counts", "lbf_step_count", "lbf_last_error",
           "lbf_label_gas_noalloc")

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run __graft_entry__.build() "
                           "(nvcc, sm_103a) first" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.lbf_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(P)]
    lib.lbf_destroy.argtypes = [P]
    lib.lbf_destroy.restype = None
    lib.lbf_nucleate.argtypes = [P, ctypes.c_int, P, P, P]
    lib.lbf_set_cells.argtypes = [P, P, P, P, P, P]
    lib.lbf_step.argtypes = [P, ctypes.c_int]
    lib.lbf_bubbles.argtypes = [P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.lbf_fields.argtypes = [P, ctypes.c_uint, P, ctypes.c_int, ctypes.c_int]
    lib.lbf_ledger.argtypes = [P, P]
    lib.lbf_timing_enable.argtypes = [P, ctypes.c_int]
    lib.lbf_timing_read.argtypes = [P, P, P, ctypes.c_int]
    lib.lbf_timing_name.argtypes = [ctypes.c_int]
    lib.lbf_timing_name.restype = ctypes.c_char_p
    lib.lbf_cell_counts.argtypes = [P, P]
    lib.lbf_step_count.argtypes = [P]
    lib.lbf_step_count.restype = ctypes.c_longlong
    lib.lbf_last_error.restype = ctypes.c_char_p
    lib.lbf_label_gas_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
    _lib = lib
    return lib


def make_config(d: dict, stream: int | None = None) -> Config:
    c = Config()
    for name, _ in Config._fields_:
        if name in ("accel", "wall_u"):
            getattr(c, name)[:] = [float(x) for x in d.get(name, (0.0, 0.0, 0.0))]
        elif name == "storage":
            s = d.get("storage", "fp32")
            c.storage = STORAGE[s] if isinstance(s, str) else int(s)
        elif name == "stream":
            c.stream = stream
        elif name in d:
            setattr(c, name, d[name])
    return c


def label_gas_noalloc(types, nx: int, ny: int, nz: int, labels, count, stream: int | None = None):
    """Bubble labels of a device cell-type field without any allocation
    (``lbf_label_gas_noalloc``): ``types`` uint8, ``labels`` int32 (N) and
    ``count`` int32 (1) are caller-owned device tensors."""
    lib = load()
    rc = lib.lbf_label_gas_noalloc(types.data_ptr(), nx, ny, nz, labels.data_ptr(), count.data_ptr(), stream)
    if rc != 0:
        raise LbfError(rc, lib.lbf_last_error().decode(errors="replace"))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Sim:
    """One GPU lattice (``lbf_create``).  ``cfg`` is a workload dictionary;
    ``stream`` an optional cudaStream_t handle (int)."""

    def __init__(self, cfg: dict, stream: int | None = None):
        self.lib = load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg, stream)
        self.nx, self.ny, self.nz = cfg["nx"], cfg["ny"], cfg["nz"]
        self.dim = 2 if self.nz == 1 else 3
        self.N = self.nx * self.ny * self.nz
        h = ctypes.c_void_p()
        self._check(self.lib.lbf_create(ctypes.byref(self._c), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise LbfError(rc, self.lib.lbf_last_error().decode(errors="replace"))

    # --- the boundary -----------------------------------------------------
    def nucleate(self, centres, radii, at_step=None):
        c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1, 3))
        r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
        s = None if at_step is None else np.ascontiguousarray(np.asarray(at_step, np.int64).reshape(-1))
        self._check(self.lib.lbf_nucleate(self.h, len(r), _p(c), _p(r), None if s is None else _p(s)))

    def set_cells(self, types, rho, u, alpha, conc):
        t = np.ascontiguousarray(np.asarray(types, np.uint8).reshape(-1))
        a = [np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1)) for x in (rho, u, alpha, conc)]
        assert t.size == self.N and a[1].size == 3 * self.N
        self._check(self.lib.lbf_set_cells(self.h, _p(t), *[_p(x) for x in a]))

    def step(self, n: int = 1):
        self._check(self.lib.lbf_step(self.h, int(n)))

    def step_count(self) -> int:
        return int(self.lib.lbf_step_count(self.h))

    def bubbles(self) -> dict:
        cnt = ctypes.c_int()
        self._check(self.lib.lbf_bubbles(self.h, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        arr = (Bubble * max(n, 1))()
        self._check(self.lib.lbf_bubbles(self.h, ctypes.cast(arr, ctypes.c_void_p), n, ctypes.byref(cnt)))
        rows = arr[:n]
        return dict(id=np.array([b.id for b in rows], np.int32),
                    atm=np.array([b.atm for b in rows], np.int32),
                    root=np.array([b.label for b in rows], np.int64),
                    volume=np.array([b.volume for b in rows]),
                    mass=np.array([b.gas_mass for b in rows]),
                    pressure=np.array([b.pressure for b in rows]))

    def fields(self, names, dtype=np.float64) -> dict:
        """Host copies of the named fields (``FIELD_BITS`` keys)."""
        names = sorted(set(names), key=lambda k: FIELD_BITS[k])
        outs = {}
        ptrs = (ctypes.c_void_p * len(names))()
        mask = 0
        for i, k in enumerate(names):
            width = 3 if k in VECTOR_FIELDS else 1
            dt = np.int32 if k in INT_FIELDS else dtype
            a = np.zeros(self.N * width, dt)
            outs[k] = a
            ptrs[i] = a.ctypes.data
            mask |= 1 << FIELD_BITS[k]
        self._check(self.lib.lbf_fields(self.h, mask, ctypes.cast(ptrs, ctypes.c_void_p), 0,
                                        1 if dtype == np.float64 else 0))
        return {k: (v.reshape(self.N, 3) if k in VECTOR_FIELDS else v) for k, v in outs.items()}

    def fields_device(self, tensors: dict, dtype_code: int = 0):
        """Write fields straight into caller-owned device buffers (torch
        tensors on this GPU, float32 for dtype_code 0, float64 for 1, int32
        for flags/label)."""
        names = sorted(tensors, key=lambda k: FIELD_BITS[k])
        ptrs = (ctypes.c_void_p * len(names))()
        mask = 0
        for i, k in enumerate(names):
            ptrs[i] = tensors[k].data_ptr()
            mask |= 1 << FIELD_BITS[k]
        self._check(self.lib.lbf_fields(self.h, mask, ctypes.cast(ptrs, ctypes.c_void_p), 1, dtype_code))

    def ledger(self) -> np.ndarray:
        out = np.zeros(8)
        rc = self.lib.lbf_ledger(self.h, _p(out))
        if rc not in (0, -5):
            self._check(rc)
        return out

    def cell_counts(self) -> np.ndarray:
        out = np.zeros(4, np.int64)
        self._check(self.lib.lbf_cell_counts(self.h, _p(out)))
        return out

    def timing_enable(self, on: bool = True):
        self._check(self.lib.lbf_timing_enable(self.h, 1 if on else 0))

    def timing_read(self) -> dict:
        ms = np.zeros(16)
        n = np.zeros(16, np.int64)
        k = self.lib.lbf_timing_read(self.h, _p(ms), _p(n), 16)
        if k < 0:
            self._check(k)
        return {self.lib.lbf_timing_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(k)}
