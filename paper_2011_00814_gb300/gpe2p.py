"""ctypes binding of ``libgpe2p.so`` (the C ABI of include/gpe2p.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing the
import of :func:`lib` raises.

Parameters are a plain ``dict`` (see :mod:`paper_2011_00814_gb300.inputs`)
plus the solver keys ``precision`` (32 | 64), ``check_stability`` (0 | 1),
``diag_every`` (int) and ``axisym`` (0 | 1, the axisymmetric (r, z) form).  Fields are numpy float64 arrays of shape ``(ny, nx)``
or ``(nz, ny, nx)``; the library copies them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpe2p.so")

OK, EINVAL, EUNSTABLE, ENOMEM, ECUDA, EDIVERGED, ETIMEOUT, ESTATE = range(8)
STATUS = {0: "OK", 1: "EINVAL", 2: "EUNSTABLE", 3: "ENOMEM", 4: "ECUDA", 5: "EDIVERGED", 6: "ETIMEOUT",
          7: "ESTATE"}
BC = {"periodic": 0, "noslip": 1, "freeslip": 2}
FIELD = {"p": 0, "u": 1, "v": 2, "w": 3, "phi": 4, "mu": 5, "phi_lo": 6}


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("cs", ctypes.c_double),
        ("rhoL", ctypes.c_double), ("rhoG", ctypes.c_double), ("etaL", ctypes.c_double),
        ("etaG", ctypes.c_double), ("rho_ref", ctypes.c_double), ("sigma", ctypes.c_double),
        ("M", ctypes.c_double), ("W", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("bc", ctypes.c_int * 3), ("precision", ctypes.c_int), ("ch_scheme", ctypes.c_int),
        ("iso", ctypes.c_int), ("bulk_visc", ctypes.c_int), ("p_average", ctypes.c_int),
        ("ch_advection", ctypes.c_int), ("check_stability", ctypes.c_int), ("diag_every", ctypes.c_int),
        ("axisym", ctypes.c_int),
    ]


class Diag(ctypes.Structure):
    _fields_ = [("int_phi", ctypes.c_double), ("kinetic", ctypes.c_double), ("umax", ctypes.c_double),
                ("nan_flag", ctypes.c_int), ("step", ctypes.c_longlong), ("t", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GPE2PError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2011_00814_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.gpe2p_stability_limits.argtypes = [ctypes.POINTER(Params), dp]
        L.gpe2p_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
        L.gpe2p_init_fields.argtypes = [vp] + [dp] * 5
        L.gpe2p_step.argtypes = [vp]
        L.gpe2p_advance.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(Diag)]
        L.gpe2p_read_fields.argtypes = [vp] + [dp] * 6
        L.gpe2p_diagnostics.argtypes = [vp, ctypes.POINTER(Diag)]
        L.gpe2p_eval_rates.argtypes = [vp] + [dp] * 5
        L.gpe2p_field_ptr.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_longlong)]
        L.gpe2p_profile_steps.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_char_p, ctypes.c_int]
        L.gpe2p_diagnostics_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp,
                                                ctypes.c_longlong, vp, vp]
        L.gpe2p_diagnostics_noalloc.restype = ctypes.c_int
        L.gpe2p_create_batch.argtypes = [ctypes.POINTER(Params), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.gpe2p_init_instance.argtypes = [vp, ctypes.c_int] + [dp] * 5
        L.gpe2p_read_instance.argtypes = [vp, ctypes.c_int] + [dp] * 6
        L.gpe2p_diagnostics_instance.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Diag)]
        L.gpe2p_batch_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), dp]
        L.gpe2p_set_fault_injection.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
        for nm in ("gpe2p_create_batch", "gpe2p_init_instance", "gpe2p_read_instance",
                   "gpe2p_diagnostics_instance", "gpe2p_batch_config", "gpe2p_set_fault_injection"):
            getattr(L, nm).restype = ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        L.gpe2p_net_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, vp,
                                       ctypes.POINTER(vp)]
        L.gpe2p_net_num_params.argtypes = [vp]
        L.gpe2p_net_num_params.restype = ctypes.c_longlong
        L.gpe2p_net_get_params.argtypes = [vp, fp, ctypes.c_longlong]
        L.gpe2p_net_set_params.argtypes = [vp, fp, ctypes.c_longlong]
        L.gpe2p_net_forward.argtypes = [vp, vp, vp, ctypes.c_int]
        L.gpe2p_net_set_normalization.argtypes = [vp, fp, fp, fp, ctypes.c_int]
        L.gpe2p_net_set_backend.argtypes = [vp, ctypes.c_int]
        L.gpe2p_net_fault.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.gpe2p_net_fault.restype = ctypes.c_int
        L.gpe2p_net_sync.argtypes = [vp]
        L.gpe2p_net_gradients.argtypes = [vp, vp, vp, ctypes.c_int, fp, fp]
        L.gpe2p_net_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, fp]
        L.gpe2p_net_flops.argtypes = [vp, ctypes.c_int]
        L.gpe2p_net_flops.restype = ctypes.c_double
        L.gpe2p_net_last_error.argtypes = [vp]
        L.gpe2p_net_last_error.restype = ctypes.c_char_p
        L.gpe2p_net_destroy.argtypes = [vp]
        L.gpe2p_net_destroy.restype = None
        for nm in ("gpe2p_net_create", "gpe2p_net_get_params", "gpe2p_net_set_params", "gpe2p_net_forward",
                   "gpe2p_net_gradients", "gpe2p_net_train_step"):
            getattr(L, nm).restype = ctypes.c_int
        for nm in ("gpe2p_pack_state", "gpe2p_unpack_state"):
            getattr(L, nm).argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, fp, fp]
            getattr(L, nm).restype = ctypes.c_int
        L.gpe2p_state_distance.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, fp, fp,
                                           ctypes.POINTER(ctypes.c_double)]
        L.gpe2p_state_distance.restype = ctypes.c_int
        L.gpe2p_interface_distance.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, fp, fp,
                                               ctypes.POINTER(ctypes.c_double)]
        L.gpe2p_interface_distance.restype = ctypes.c_int
        L.gpe2p_set_phi_accumulation.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        L.gpe2p_phi_accumulation.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
        L.gpe2p_fma_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     vp]
        L.gpe2p_fma_rate.restype = ctypes.c_int
        L.gpe2p_mma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.gpe2p_mma_rate.restype = ctypes.c_int
        L.gpe2p_last_error.argtypes = [vp]
        L.gpe2p_last_error.restype = ctypes.c_char_p
        L.gpe2p_destroy.argtypes = [vp]
        L.gpe2p_destroy.restype = None
        for nm in ("gpe2p_stability_limits", "gpe2p_create", "gpe2p_init_fields", "gpe2p_step",
                   "gpe2p_advance", "gpe2p_read_fields", "gpe2p_diagnostics", "gpe2p_eval_rates",
                   "gpe2p_field_ptr", "gpe2p_profile_steps"):
            getattr(L, nm).restype = ctypes.c_int
        _lib = L
    return _lib


def fma_rate(precision: int, stream: int | None = None) -> dict:
    """Measured multiply-add rate of the current device (gpe2p_fma_rate):
    {"flops_per_s": ..., "ms": ...} in the given precision (32 or 64)."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    rc = lib().gpe2p_fma_rate(int(precision), ctypes.byref(f), ctypes.byref(ms), stream)
    if rc != OK:
        raise GPE2PError(rc, "gpe2p_fma_rate failed")
    return {"flops_per_s": f.value, "ms": ms.value}


def mma_rate(n: int, issuers: int = 1, stream: int | None = None) -> float:
    """SM clock cycles per tcgen05.mma (M = 128, N = n, K = 16, BF16) of one
    SM with `issuers` issuing threads (gpe2p_mma_rate)."""
    c = ctypes.c_double()
    rc = lib().gpe2p_mma_rate(int(n), int(issuers), ctypes.byref(c), stream)
    if rc != OK:
        raise GPE2PError(rc, "gpe2p_mma_rate failed")
    return c.value


def params(prm: dict) -> Params:
    q = Params()
    dim = int(prm["dim"])
    q.dim, q.nx, q.ny = dim, int(prm["nx"]), int(prm["ny"])
    q.nz = int(prm.get("nz", 1)) if dim == 3 else 1
    for k in ("dx", "dt", "cs", "rhoL", "rhoG", "etaL", "etaG", "sigma", "M", "W"):
        setattr(q, k, float(prm[k]))
    q.rho_ref = float(prm.get("rho_ref", 0.0))
    g = list(prm.get("g", (0.0, 0.0, 0.0))) + [0.0] * 3
    bc = list(prm.get("bc", ("periodic",) * 3)) + ["periodic"] * 3
    for a in range(3):
        q.g[a] = float(g[a])
        q.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
    q.precision = int(prm.get("precision", 64))
    q.ch_scheme = int(prm.get("ch_scheme", 2 if dim == 2 else 4))
    q.iso = int(prm.get("iso", 9 if dim == 2 else 15))
    q.bulk_visc = int(prm.get("bulk_visc", 1))
    q.p_average = int(prm.get("p_average", 1))
    q.ch_advection = int(prm.get("ch_advection", 0))
    q.check_stability = int(prm.get("check_stability", 0))
    q.diag_every = int(prm.get("diag_every", 0))
    q.axisym = int(prm.get("axisym", 0))
    return q


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def stability_limits(prm: dict):
    out = (ctypes.c_double * 3)()
    rc = lib().gpe2p_stability_limits(ctypes.byref(params(prm)), out)
    if rc != OK:
        raise GPE2PError(rc, lib().gpe2p_last_error(None).decode())
    return tuple(out)


def _tensor_call(obj, op, inst, tensor, mean, scale):
    """Marshal one call of the state <-> tensor family; ``tensor`` is a
    contiguous CUDA float32 tensor [ny, nx, nch] (or a raw device pointer
    with ``nch`` taken from ``mean``)."""
    if isinstance(tensor, int):
        ptr, nch = tensor, len(mean) if mean is not None else 4
    else:
        if tensor.dtype != __import__("torch").float32 or not tensor.is_contiguous() or not tensor.is_cuda:
            raise ValueError("tensor must be a contiguous CUDA float32 tensor")
        ptr, nch = tensor.data_ptr(), int(tensor.shape[-1])
    m = None if mean is None else (ctypes.c_float * nch)(*[float(x) for x in mean])
    s = None if scale is None else (ctypes.c_float * nch)(*[float(x) for x in scale])
    L = lib()
    if op == "pack":
        obj._check(L.gpe2p_pack_state(obj.h, int(inst), ctypes.c_void_p(ptr), nch, m, s))
    elif op == "unpack":
        obj._check(L.gpe2p_unpack_state(obj.h, int(inst), ctypes.c_void_p(ptr), nch, m, s))
    elif op == "interface":
        out = (ctypes.c_double * 3)()
        obj._check(L.gpe2p_interface_distance(obj.h, int(inst), ctypes.c_void_p(ptr), nch, m, s, out))
        return list(out)
    else:
        out = (ctypes.c_double * 8)()
        obj._check(L.gpe2p_state_distance(obj.h, int(inst), ctypes.c_void_p(ptr), nch, m, s, out))
        return list(out)


PHI_ACC_FP32, PHI_ACC_COMPENSATED, PHI_ACC_AUTO = 0, 1, 2


class Solver:
    """One problem on the current CUDA device (``gpe2p_create`` ... ``gpe2p_destroy``)."""

    def __init__(self, prm: dict, stream: int | None = None):
        self.prm = dict(prm)
        self.dim = int(prm["dim"])
        self.shape = ((int(prm["nz"]), int(prm["ny"]), int(prm["nx"])) if self.dim == 3
                      else (int(prm["ny"]), int(prm["nx"])))
        self._p = params(prm)
        h = ctypes.c_void_p()
        rc = lib().gpe2p_create(ctypes.byref(self._p), ctypes.c_void_p(stream) if stream else None,
                                ctypes.byref(h))
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_last_error(self.h).decode())

    def _arr(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != self.shape:
            raise ValueError(f"field shape {a.shape} != {self.shape}")
        return a

    def init_fields(self, f: dict):
        a = {k: self._arr(f[k]) for k in ("phi", "u", "v", "p")}
        a["w"] = self._arr(f["w"]) if self.dim == 3 else None
        self._check(lib().gpe2p_init_fields(self.h, _dptr(a["phi"]), _dptr(a["u"]), _dptr(a["v"]),
                                            _dptr(a["w"]), _dptr(a["p"])))

    def step(self):
        self._check(lib().gpe2p_step(self.h))

    def advance(self, nsteps: int) -> dict:
        d = Diag()
        self._check(lib().gpe2p_advance(self.h, int(nsteps), ctypes.byref(d)))
        return d.as_dict()

    def diagnostics(self) -> dict:
        d = Diag()
        self._check(lib().gpe2p_diagnostics(self.h, ctypes.byref(d)))
        return d.as_dict()

    def read_fields(self) -> dict:
        names = ["phi", "u", "v", "w", "p", "mu"]
        out = {k: np.empty(self.shape) for k in names}
        if self.dim == 2:
            out["w"] = None
        self._check(lib().gpe2p_read_fields(self.h, *[_dptr(out[k]) for k in names]))
        if self.dim == 2:
            out.pop("w")
        return out

    def eval_rates(self) -> dict:
        names = ["Lp", "Lu", "Lv", "Lw", "Lphi"]
        out = {k: np.empty(self.shape) for k in names}
        if self.dim == 2:
            out["Lw"] = None
        self._check(lib().gpe2p_eval_rates(self.h, *[_dptr(out[k]) for k in names]))
        if self.dim == 2:
            out.pop("Lw")
        return out

    def profile_steps(self, nsteps: int):
        """[(kernel name, mean ms per launch)] for the launches of one step."""
        ms = (ctypes.c_double * 64)()
        n = ctypes.c_int()
        names = ctypes.create_string_buffer(2048)
        self._check(lib().gpe2p_profile_steps(self.h, int(nsteps), ms, 64, ctypes.byref(n), names, 2048))
        nm = names.value.decode().split(",")
        return [(nm[i], ms[i]) for i in range(n.value)]

    def set_phi_accumulation(self, mode: int, threshold: float = 1e-10):
        """PHI_ACC_FP32, PHI_ACC_COMPENSATED or PHI_ACC_AUTO (see gpe2p_set_phi_accumulation)."""
        self._check(lib().gpe2p_set_phi_accumulation(self.h, int(mode), float(threshold)))

    def phi_accumulation(self) -> dict:
        m, a, d, sw = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_longlong()
        self._check(lib().gpe2p_phi_accumulation(self.h, ctypes.byref(m), ctypes.byref(a), ctypes.byref(d),
                                                 ctypes.byref(sw)))
        return {"mode": m.value, "active": bool(a.value), "drift": d.value, "switched_at": sw.value}

    def pack(self, tensor, mean=None, scale=None):
        """State -> tensor [ny, nx, nch] (phi, u, v, p[, rho/rho_L]), normalised."""
        _tensor_call(self, "pack", 0, tensor, mean, scale)

    def unpack(self, tensor, mean=None, scale=None):
        """Tensor -> state (mu recomputed)."""
        _tensor_call(self, "unpack", 0, tensor, mean, scale)

    def distance(self, tensor, mean=None, scale=None):
        """[sum (f_c - t_c)^2, sum f_c^2] for c = phi, u, v, p (8 floats)."""
        return _tensor_call(self, "distance", 0, tensor, mean, scale)

    def interface_distance(self, tensor, mean=None, scale=None):
        """[max, mean] displacement in cells of the tensor's phi = 0 interface
        from the state's, and the cells of the interface band."""
        return _tensor_call(self, "interface", 0, tensor, mean, scale)

    def fault(self, what: int, value: int = 0):
        """Host-side test switch of the kernels' timeout paths (gpe2p_set_fault_injection)."""
        self._check(lib().gpe2p_set_fault_injection(self.h, int(what), int(value)))

    def field_ptr(self, name: str):
        """(device pointer, row pitch in elements) of a field of the current state."""
        p = ctypes.c_void_p()
        pitch = ctypes.c_longlong()
        self._check(lib().gpe2p_field_ptr(self.h, FIELD[name], ctypes.byref(p), ctypes.byref(pitch)))
        return p.value, pitch.value

    def close(self):
        if getattr(self, "h", None):
            lib().gpe2p_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FAULT_SKIP_BARRIER, FAULT_WAIT_LIMIT, FAULT_FORCE_PERSISTENT, FAULT_CLEAR, FAULT_LOSE_COPY = 1, 2, 3, 4, 5
LOSE_FLOW_RING, LOSE_CH_RING, LOSE_MU_RING, LOSE_CH_POINTS = 1, 2, 4, 8


class Batch:
    """Many independent 2D problems advanced together (``gpe2p_create_batch``)."""

    def __init__(self, prms, stream: int | None = None):
        self.prms = [dict(p) for p in prms]
        n = len(self.prms)
        arr = (Params * n)(*[params(p) for p in self.prms])
        self._arr = arr
        h = ctypes.c_void_p()
        rc = lib().gpe2p_create_batch(arr, n, ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_last_error(None).decode())
        self.h = h
        self.shapes = [(int(p["ny"]), int(p["nx"])) for p in self.prms]

    def _check(self, rc):
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_last_error(self.h).decode())

    def init_instance(self, k: int, f: dict):
        a = {key: np.ascontiguousarray(f[key], dtype=np.float64) for key in ("phi", "u", "v", "p")}
        for key, v in a.items():
            if v.shape != self.shapes[k]:
                raise ValueError(f"instance {k}: field {key} shape {v.shape} != {self.shapes[k]}")
        self._check(lib().gpe2p_init_instance(self.h, int(k), _dptr(a["phi"]), _dptr(a["u"]), _dptr(a["v"]),
                                              None, _dptr(a["p"])))

    def read_instance(self, k: int) -> dict:
        out = {key: np.empty(self.shapes[k]) for key in ("phi", "u", "v", "p", "mu")}
        self._check(lib().gpe2p_read_instance(self.h, int(k), _dptr(out["phi"]), _dptr(out["u"]),
                                              _dptr(out["v"]), None, _dptr(out["p"]), _dptr(out["mu"])))
        return out

    def step(self):
        self._check(lib().gpe2p_step(self.h))

    def advance(self, nsteps: int) -> dict:
        d = Diag()
        self._check(lib().gpe2p_advance(self.h, int(nsteps), ctypes.byref(d)))
        return d.as_dict()

    def diagnostics(self, k: int | None = None) -> dict:
        d = Diag()
        if k is None:
            self._check(lib().gpe2p_diagnostics(self.h, ctypes.byref(d)))
        else:
            self._check(lib().gpe2p_diagnostics_instance(self.h, int(k), ctypes.byref(d)))
        return d.as_dict()

    def pack(self, k: int, tensor, mean=None, scale=None):
        _tensor_call(self, "pack", k, tensor, mean, scale)

    def unpack(self, k: int, tensor, mean=None, scale=None):
        _tensor_call(self, "unpack", k, tensor, mean, scale)

    def distance(self, k: int, tensor, mean=None, scale=None):
        return _tensor_call(self, "distance", k, tensor, mean, scale)

    def interface_distance(self, k: int, tensor, mean=None, scale=None):
        return _tensor_call(self, "interface", k, tensor, mean, scale)

    def config(self) -> dict:
        tx, ty, pers = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        self._check(lib().gpe2p_batch_config(self.h, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(pers),
                                             ctypes.byref(ms)))
        return {"tile": (tx.value, ty.value), "persistent": bool(pers.value), "tuned_ms_per_step": ms.value}

    def fault(self, what: int, value: int = 0):
        self._check(lib().gpe2p_set_fault_injection(self.h, int(what), int(value)))

    def close(self):
        if getattr(self, "h", None):
            lib().gpe2p_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The surrogate U-Net (``gpe2p_net_*``).  Tensors are torch CUDA float32
    tensors (or raw device pointers) in NHWC order."""

    def __init__(self, levels, channels, in_ch, out_ch, H, W, max_batch, seed=0, stream: int | None = None):
        self.levels, self.channels = int(levels), [int(c) for c in channels]
        self.in_ch, self.out_ch, self.H, self.W, self.max_batch = in_ch, out_ch, H, W, max_batch
        ch = (ctypes.c_int * len(channels))(*channels)
        h = ctypes.c_void_p()
        rc = lib().gpe2p_net_create(levels, ch, in_ch, out_ch, H, W, max_batch, ctypes.c_ulonglong(seed),
                                    ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_net_last_error(None).decode())
        self.h = h
        self.nparam = int(lib().gpe2p_net_num_params(h))

    def _check(self, rc):
        if rc != OK:
            raise GPE2PError(rc, lib().gpe2p_net_last_error(self.h).decode())

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparam, dtype=np.float32)
        self._check(lib().gpe2p_net_get_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               self.nparam))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().gpe2p_net_set_params(self.h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               self.nparam))

    def set_normalization(self, in_mean=None, in_scale=None, out_scale=None, residual: bool = False):
        """Input normalisation and output map (see gpe2p_net_set_normalization)."""
        def arr(v, n):
            return None if v is None else (ctypes.c_float * n)(*[float(a) for a in v])
        self._check(lib().gpe2p_net_set_normalization(self.h, arr(in_mean, self.in_ch), arr(in_scale, self.in_ch),
                                                      arr(out_scale, self.out_ch), int(bool(residual))))

    def set_backend(self, tcgen05: bool):
        """3x3 convolutions on tcgen05 (True, default) or on mma.sync (False)."""
        self._check(lib().gpe2p_net_set_backend(self.h, int(bool(tcgen05))))

    def fault(self, what: int, value: int = 0):
        """Host-side test switch of the tcgen05 convolutions (gpe2p_net_fault):
        FAULT_LOSE_COPY (value 1 on, 0 off) or FAULT_CLEAR."""
        self._check(lib().gpe2p_net_fault(self.h, int(what), int(value)))

    def sync(self):
        self._check(lib().gpe2p_net_sync(self.h))

    def forward(self, x, y, batch: int):
        self._check(lib().gpe2p_net_forward(self.h, self._ptr(x), self._ptr(y), int(batch)))

    def gradients(self, x, t, batch: int):
        g = np.empty(self.nparam, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(lib().gpe2p_net_gradients(self.h, self._ptr(x), self._ptr(t), int(batch),
                                              g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              ctypes.byref(loss)))
        return float(loss.value), g

    def train_step(self, x, t, batch: int, lr: float, want_loss: bool = True):
        loss = ctypes.c_float()
        self._check(lib().gpe2p_net_train_step(self.h, self._ptr(x), self._ptr(t), int(batch), float(lr),
                                               ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def flops(self, batch: int) -> float:
        return float(lib().gpe2p_net_flops(self.h, int(batch)))

    def close(self):
        if getattr(self, "h", None):
            lib().gpe2p_net_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
