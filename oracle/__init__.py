"""CPU FP64 oracle of the two-phase GPE method (Huang, arXiv 2011.00814).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may load it; the product library never does.

This module is a thin ctypes wrapper around ``gpe2p_oracle.c`` (plain loops,
double precision, built with ``-ffp-contract=off``).  Arrays are numpy float64
of shape ``(ny, nx)`` in 2D and ``(nz, ny, nx)`` in 3D (x fastest).  Parameters
are a plain ``dict`` with the keys of :data:`PARAM_KEYS` (the same physical
names the product binding takes); this module does no arithmetic of the method
itself beyond marshalling.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpe2p_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"periodic": 0, "noslip": 1, "freeslip": 2}


class _Par(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("cs", ctypes.c_double),
        ("rhoL", ctypes.c_double), ("rhoG", ctypes.c_double), ("etaL", ctypes.c_double),
        ("etaG", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("sigma", ctypes.c_double), ("M", ctypes.c_double), ("W", ctypes.c_double),
        ("g", ctypes.c_double * 3), ("bc", ctypes.c_int * 3),
        ("ch_scheme", ctypes.c_int), ("iso", ctypes.c_int), ("bulk_visc", ctypes.c_int),
        ("p_average", ctypes.c_int), ("ch_advection", ctypes.c_int), ("axisym", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, -O2, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                   "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Par)
        lib.orc_flow_rhs.argtypes = [pp] + [dp] * 10
        lib.orc_ch_rhs.argtypes = [pp] + [dp] * 6
        lib.orc_mu.argtypes = [pp, dp, dp]
        lib.orc_lap_iso.argtypes = [pp, dp, dp]
        lib.orc_grad_iso.argtypes = [pp, dp, dp, dp, dp]
        lib.orc_step.argtypes = [pp] + [dp] * 6 + [ctypes.c_longlong]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_diag.argtypes = [pp] + [dp] * 5 + [dp]
        lib.orc_lattice_table.argtypes = [pp, ctypes.POINTER(ctypes.c_int), dp]
        lib.orc_lattice_table.restype = ctypes.c_int
        _lib = lib
    return _lib


def _par(prm: dict) -> _Par:
    q = _Par()
    dim = int(prm["dim"])
    q.dim = dim
    q.nx, q.ny = int(prm["nx"]), int(prm["ny"])
    q.nz = int(prm.get("nz", 1)) if dim == 3 else 1
    for k in ("dx", "dt", "cs", "rhoL", "rhoG", "etaL", "etaG", "sigma", "M", "W"):
        setattr(q, k, float(prm[k]))
    q.rho_ref = float(prm.get("rho_ref", 0.0))
    g = list(prm.get("g", (0.0, 0.0, 0.0))) + [0.0] * 3
    for a in range(3):
        q.g[a] = float(g[a])
    bc = prm.get("bc", ("periodic",) * 3)
    for a in range(3):
        b = bc[a] if a < len(bc) else "periodic"
        q.bc[a] = BC[b] if isinstance(b, str) else int(b)
    q.ch_scheme = int(prm.get("ch_scheme", 2 if dim == 2 else 4))
    q.iso = int(prm.get("iso", 9 if dim == 2 else 15))
    q.bulk_visc = int(prm.get("bulk_visc", 1))
    q.p_average = int(prm.get("p_average", 1))
    q.ch_advection = int(prm.get("ch_advection", 0))
    q.axisym = int(prm.get("axisym", 0))
    return q


def _shape(prm: dict):
    if int(prm["dim"]) == 3:
        return (int(prm["nz"]), int(prm["ny"]), int(prm["nx"]))
    return (int(prm["ny"]), int(prm["nx"]))


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(prm, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == _shape(prm), (a.shape, _shape(prm))
    return a


def mu(prm: dict, phi) -> np.ndarray:
    """Chemical potential (Eq. chem-pot) of ``phi``."""
    lib = _load()
    phi = _arr(prm, phi)
    out = np.empty_like(phi)
    q = _par(prm)
    lib.orc_mu(ctypes.byref(q), _ptr(phi), _ptr(out))
    return out


def lap_iso(prm: dict, f) -> np.ndarray:
    """Isotropic Laplacian (Eq. laplacian-iso)."""
    lib = _load()
    f = _arr(prm, f)
    out = np.empty_like(f)
    lib.orc_lap_iso(ctypes.byref(_par(prm)), _ptr(f), _ptr(out))
    return out


def grad_iso(prm: dict, f):
    """Isotropic gradient (Eq. 1st-der-iso): list of dim arrays."""
    lib = _load()
    f = _arr(prm, f)
    g = [np.zeros_like(f) for _ in range(3)]
    lib.orc_grad_iso(ctypes.byref(_par(prm)), _ptr(f), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]))
    return g[: int(prm["dim"])]


def flow_rhs(prm: dict, st: dict):
    """Semi-discrete flow rates (L_p, L_u, L_v[, L_w]) of Eq. p-u-v-semidiscrete-2d."""
    lib = _load()
    dim = int(prm["dim"])
    a = {k: _arr(prm, st[k]) for k in ("p", "u", "v", "phi", "mu")}
    a["w"] = _arr(prm, st["w"]) if dim == 3 else None
    out = [np.zeros(_shape(prm)) for _ in range(4)]
    lib.orc_flow_rhs(ctypes.byref(_par(prm)), _ptr(a["p"]), _ptr(a["u"]), _ptr(a["v"]), _ptr(a["w"]),
                     _ptr(a["phi"]), _ptr(a["mu"]), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                     _ptr(out[3]) if dim == 3 else None)
    return out[: 1 + dim]


def ch_rhs(prm: dict, phi, mu_, uh):
    """CH rate (Eq. che) with the cell-centre velocity ``uh`` (list of dim arrays)."""
    lib = _load()
    dim = int(prm["dim"])
    phi, mu_ = _arr(prm, phi), _arr(prm, mu_)
    u3 = [_arr(prm, x) for x in uh] + [None] * (3 - dim)
    out = np.empty_like(phi)
    lib.orc_ch_rhs(ctypes.byref(_par(prm)), _ptr(phi), _ptr(mu_), _ptr(u3[0]), _ptr(u3[1]),
                   _ptr(u3[2]), _ptr(out))
    return out


def step(prm: dict, st: dict, nsteps: int = 1) -> dict:
    """Advance a copy of the state ``st`` (keys p,u,v[,w],phi,mu) by ``nsteps`` full steps."""
    lib = _load()
    dim = int(prm["dim"])
    s = {k: _arr(prm, st[k]).copy() for k in ("p", "u", "v", "phi", "mu")}
    s["w"] = _arr(prm, st["w"]).copy() if dim == 3 else None
    rc = lib.orc_step(ctypes.byref(_par(prm)), _ptr(s["p"]), _ptr(s["u"]), _ptr(s["v"]), _ptr(s["w"]),
                      _ptr(s["phi"]), _ptr(s["mu"]), ctypes.c_longlong(int(nsteps)))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    if dim == 2:
        s.pop("w")
    return s


def init_state(prm: dict, phi, p=None, u=None, v=None, w=None) -> dict:
    """State at t=0: the given fields (zeros where omitted) and mu = mu(phi)."""
    shp = _shape(prm)
    z = lambda a: np.zeros(shp) if a is None else _arr(prm, a).copy()
    st = {"phi": _arr(prm, phi).copy(), "p": z(p), "u": z(u), "v": z(v)}
    if int(prm["dim"]) == 3:
        st["w"] = z(w)
    st["mu"] = mu(prm, st["phi"])
    return st


def diag(prm: dict, st: dict):
    """(sum phi dV, kinetic energy, max |u|, nan flag)."""
    lib = _load()
    dim = int(prm["dim"])
    a = {k: _arr(prm, st[k]) for k in ("p", "u", "v", "phi")}
    w = _arr(prm, st["w"]) if dim == 3 else None
    out = np.zeros(4)
    lib.orc_diag(ctypes.byref(_par(prm)), _ptr(a["p"]), _ptr(a["u"]), _ptr(a["v"]), _ptr(w),
                 _ptr(a["phi"]), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2]), bool(out[3])


def lattice_table(prm: dict):
    """(e, w) of the lattice the oracle's isotropic stencils use."""
    lib = _load()
    e = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    n = lib.orc_lattice_table(ctypes.byref(_par(prm)), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              _ptr(w))
    return e[:n].copy(), w[:n].copy()
