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
        ("collision", ctypes.c_int), ("trt_magic", ctypes.c_double),
        ("kappa", ctypes.c_int), ("mrt_rates", ctypes.c_double * 4),
    ]


class Bubble(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("atm", ctypes.c_int32), ("label", ctypes.c_int64),
                ("volume", ctypes.c_double), ("gas_mass", ctypes.c_double),
                ("pressure", ctypes.c_double)]


class MlpTrainCfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_ulonglong), ("n_samples", ctypes.c_int), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("lr", ctypes.c_double), ("rmin", ctypes.c_double),
                ("rmax", ctypes.c_double), ("noise", ctypes.c_double), ("x_extra", ctypes.c_void_p),
                ("y_extra", ctypes.c_void_p), ("n_extra", ctypes.c_int), ("stream", ctypes.c_void_p)]


EXPORTS = ("lbf_create", "lbf_destroy", "lbf_nucleate", "lbf_set_cells", "lbf_step",
           "lbf_bubbles", "lbf_fields", "lbf_ledger", "lbf_timing_enable", "lbf_timing_read",
           "lbf_timing_name", "lbf_cell_counts", "lbf_step_count", "lbf_last_error",
           "lbf_label_gas_noalloc", "lbf_mlp_forward", "lbf_mlp_loss_grad", "lbf_mlp_generate",
           "lbf_mlp_stencils_from_params", "lbf_mlp_train", "lbf_mlp_harvest", "lbf_mlp_attach",
           "lbf_checkpoint_bytes", "lbf_checkpoint_save", "lbf_checkpoint_load")

MLP_NPARAM = 6017

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
    lib.lbf_mlp_forward.argtypes = [P, P, ctypes.c_int, P, P]
    lib.lbf_mlp_loss_grad.argtypes = [P, P, P, ctypes.c_int, P, P, P]
    lib.lbf_mlp_generate.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P, P]
    lib.lbf_mlp_stencils_from_params.argtypes = [P, ctypes.c_int, P, P, P]
    lib.lbf_mlp_train.argtypes = [ctypes.POINTER(MlpTrainCfg), P, P]
    lib.lbf_mlp_attach.argtypes = [P, P]
    lib.lbf_mlp_harvest.argtypes = [P, P, P, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.lbf_checkpoint_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.lbf_checkpoint_save.argtypes = [P, P, ctypes.c_size_t]
    lib.lbf_checkpoint_load.argtypes = [P, P, ctypes.c_size_t]
    _lib = lib
    return lib


def make_config(d: dict, stream: int | None = None) -> Config:
    c = Config()
    for name, _ in Config._fields_:
        if name in ("accel", "wall_u"):
            getattr(c, name)[:] = [float(x) for x in d.get(name, (0.0, 0.0, 0.0))]
        elif name == "mrt_rates":
            getattr(c, name)[:] = [float(x) for x in d.get(name, (0.0, 0.0, 0.0, 0.0))]
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


def _raise(rc: int):
    if rc != 0:
        raise LbfError(rc, load().lbf_last_error().decode(errors="replace"))


# --- learned curvature (device tensors in, device tensors out) -------------


def mlp_forward(theta, x, y, stream: int | None = None):
    """y (n) = network(x (n x 27)); float32 device tensors."""
    _raise(load().lbf_mlp_forward(theta.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr(), stream))


def mlp_loss_grad(theta, x, t, grad, loss, stream: int | None = None):
    """grad (6017 float32) and loss (1 float64) of 0.5 mean((y - t)^2)."""
    _raise(load().lbf_mlp_loss_grad(theta.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0],
                                    grad.data_ptr(), loss.data_ptr(), stream))


def mlp_generate(seed: int, x, y, rmin: float = 2.0, rmax: float = 40.0, stream: int | None = None):
    """Synthetic canonical stencils x (n x 27) and targets y = 4 kappa (n)."""
    _raise(load().lbf_mlp_generate(int(seed), x.shape[0], rmin, rmax, x.data_ptr(), y.data_ptr(), stream))


def mlp_stencils_from_params(params, x, y, stream: int | None = None):
    """Stencils of explicit shapes: params host (n x 20) float64."""
    p = np.ascontiguousarray(np.asarray(params, np.float64).reshape(-1, 20))
    _raise(load().lbf_mlp_stencils_from_params(_p(p), p.shape[0], x.data_ptr(), y.data_ptr(), stream))


def mlp_train(theta0, n_samples: int = 1 << 22, epochs: int = 20, batch: int = 2048, lr: float = 3e-3,
              rmin: float = 2.0, rmax: float = 40.0, seed: int = 1, noise: float = 0.0,
              x_extra=None, y_extra=None, stream: int | None = None):
    """Train on the device from theta0 (host, 6017) on ``n_samples``
    generated stencils plus optional extra device tensors (n x 27, n);
    returns (theta, mean loss per epoch)."""
    th = np.ascontiguousarray(np.asarray(theta0, np.float32).reshape(-1).copy())
    assert th.size == MLP_NPARAM
    curve = np.zeros(epochs, np.float32)
    ne = 0 if x_extra is None else int(x_extra.shape[0])
    c = MlpTrainCfg(int(seed), int(n_samples), int(epochs), int(batch), float(lr), float(rmin),
                    float(rmax), float(noise), None if ne == 0 else x_extra.data_ptr(),
                    None if ne == 0 else y_extra.data_ptr(), ne, stream)
    _raise(load().lbf_mlp_train(ctypes.byref(c), _p(th), _p(curve)))
    return th, curve


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
        """The bubble table (one library call: rows up to the capacity)."""
        if getattr(self, "_bub", None) is None:
            self._bub = (Bubble * max(int(self.cfg.get("bubble_capacity", 4096)), 1))()
        cnt = ctypes.c_int()
        self._check(self.lib.lbf_bubbles(self.h, ctypes.cast(self._bub, ctypes.c_void_p), len(self._bub),
                                         ctypes.byref(cnt)))
        n = min(cnt.value, len(self._bub))
        rows = self._bub[:n]
        return dict(id=np.array([b.id for b in rows], np.int32),
                    atm=np.array([b.atm for b in rows], np.int32),
                    root=np.array([b.label for b in rows], np.int64),
                    volume=np.array([b.volume for b in rows]),
                    mass=np.array([b.gas_mass for b in rows]),
                    pressure=np.array([b.pressure for b in rows]))

    def fields(self, names, dtype=np.float64, out=None) -> dict:
        """Host copies of the named fields (``FIELD_BITS`` keys).  ``out``
        optionally maps names to caller-owned contiguous host arrays of the
        right size and dtype (page-locked ones are filled by one direct
        copy each)."""
        names = sorted(set(names), key=lambda k: FIELD_BITS[k])
        outs = {}
        ptrs = (ctypes.c_void_p * len(names))()
        mask = 0
        for i, k in enumerate(names):
            width = 3 if k in VECTOR_FIELDS else 1
            dt = np.int32 if k in INT_FIELDS else dtype
            if out is not None and k in out:
                a = out[k]
                if a.dtype != dt or a.size != self.N * width or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("out[%r] must be a contiguous %s array of %d values" % (k, np.dtype(dt), self.N * width))
                a = a.reshape(-1)
            else:
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

    def checkpoint(self) -> np.ndarray:
        """The whole simulation state as a host byte array (``lbf_checkpoint_save``)."""
        n = ctypes.c_size_t()
        self._check(self.lib.lbf_checkpoint_bytes(self.h, ctypes.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._check(self.lib.lbf_checkpoint_save(self.h, _p(buf), buf.nbytes))
        return buf

    def restore(self, buf: np.ndarray):
        """Resume from a checkpoint of a sim with the same configuration
        (``lbf_checkpoint_load``)."""
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self.lib.lbf_checkpoint_load(self.h, _p(buf), buf.nbytes))

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

    def mlp_attach(self, theta=None):
        """Learned curvature from the next step on (3D); None detaches."""
        if theta is None:
            self._check(self.lib.lbf_mlp_attach(self.h, None))
            return
        th = np.ascontiguousarray(np.asarray(theta, np.float32).reshape(-1))
        assert th.size == MLP_NPARAM
        self._check(self.lib.lbf_mlp_attach(self.h, _p(th)))

    def mlp_harvest(self, x, y, cells=None) -> int:
        """Training pairs of the current interface cells into the device
        tensors x (cap x 27) and y (cap), float32, and optionally their cell
        indices (cap int32); returns how many."""
        cnt = ctypes.c_int()
        self._check(self.lib.lbf_mlp_harvest(self.h, x.data_ptr(), y.data_ptr(),
                                             None if cells is None else cells.data_ptr(),
                                             int(x.shape[0]), ctypes.byref(cnt)))
        return cnt.value

    def timing_enable(self, on: bool = True):
        self._check(self.lib.lbf_timing_enable(self.h, 1 if on else 0))

    def timing_read(self) -> dict:
        ms = np.zeros(16)
        n = np.zeros(16, np.int64)
        k = self.lib.lbf_timing_read(self.h, _p(ms), _p(n), 16)
        if k < 0:
            self._check(k)
        return {self.lib.lbf_timing_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(k)}
