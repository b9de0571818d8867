"""ctypes binding of the oracle library (test infrastructure only).

Marshals workloads.System objects into the oracle's C structs; all arithmetic
is in hsref.c.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

_LIB = None
_LOCK = threading.Lock()
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Type(C.Structure):
    _fields_ = [("lmax", C.c_int), ("rmt", C.c_double),
                ("u", _dp), ("du", _dp), ("udot", _dp), ("dudot", _dp),
                ("udot_norm2", _dp), ("e_l", _dp),
                ("I_uu", _dp), ("I_uud", _dp), ("I_udu", _dp), ("I_udud", _dp),
                ("T_override", _dp), ("lmax_nonsph", C.c_int), ("wronskian", _dp)]


class _System(C.Structure):
    _fields_ = [("omega", C.c_double), ("n_types", C.c_int), ("types", C.POINTER(_Type)),
                ("n_atoms", C.c_int), ("type_of_atom", _ip), ("pos", _dp), ("rot", _dp)]


def _bind(path: str):
    lib = C.CDLL(path)
    lib.hsref_sbessel.argtypes = [C.c_int, C.c_double, _dp, _dp]
    lib.hsref_ylm.argtypes = [C.c_int, _dp, _dp]
    lib.hsref_wigner3j.argtypes = [C.c_int] * 6
    lib.hsref_wigner3j.restype = C.c_double
    lib.hsref_gaunt.argtypes = [C.c_int] * 6
    lib.hsref_gaunt.restype = C.c_double
    lib.hsref_T.argtypes = [C.POINTER(_Type), _dp]
    lib.hsref_cholesky.argtypes = [C.c_int, _dp, C.c_longlong, _dp]
    lib.hsref_coefficients.argtypes = [C.POINTER(_System), C.c_int, C.c_int, _dp, _dp]
    lib.hsref_build_HS.argtypes = [C.POINTER(_System), C.c_int, _dp, _dp, _dp, C.c_longlong, C.c_int, C.c_int]
    lib.hsref_HS_entries.argtypes = [C.POINTER(_System), C.c_int, _dp, C.c_int, _ip, _ip, _dp, _dp, C.c_int]
    lib.hsref_HS_columns.argtypes = [C.POINTER(_System), C.c_int, _dp, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp]
    lib.hsref_HS_brute.argtypes = [C.POINTER(_System), C.c_int, _dp, _dp, _dp, C.c_longlong]
    lib.hsref_threads.restype = C.c_int
    return lib


def load():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _bind(_build.build())
    return _LIB


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call through another build of hsref.c
    (used by the tests that plant mistakes in a copy of the oracle)."""
    global _LIB
    prev = load()
    _LIB = _bind(path)
    try:
        yield
    finally:
        _LIB = prev


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


class _Marshal:
    """Keeps the numpy arrays alive while the C structs point at them."""

    def __init__(self, sysm):
        self.keep = []
        types = (_Type * len(sysm.types))()
        for i, t in enumerate(sysm.types):
            arrs = {k: _f64(getattr(t, k)) for k in
                    ("u", "du", "udot", "dudot", "udot_norm2", "e_l", "I_uu", "I_uud", "I_udu", "I_udud")}
            self.keep.extend(arrs.values())
            types[i].lmax = int(t.lmax)
            types[i].rmt = float(t.rmt)
            lns = getattr(t, "lmax_nonsph", None)
            types[i].lmax_nonsph = int(t.lmax) if lns is None else int(lns)
            for k, v in arrs.items():
                setattr(types[i], k, _d(v))
            if t.T_override is not None:
                tov = _c128(np.asfortranarray(t.T_override)).reshape(-1, order="F").view(np.float64).copy()
                self.keep.append(tov)
                types[i].T_override = _d(tov)
            else:
                types[i].T_override = None
            wr = getattr(t, "wronskian", None)
            if wr is not None:
                wa = _f64(wr).copy()
                self.keep.append(wa)
                types[i].wronskian = _d(wa)
            else:
                types[i].wronskian = None
        self.types = types
        self.toa = np.ascontiguousarray(sysm.type_of_atom, dtype=np.int32)
        self.pos = _f64(sysm.pos).reshape(-1).copy()
        self.rot = _f64(sysm.rot).reshape(-1).copy()
        self.sys = _System(float(sysm.omega), len(sysm.types), types, int(self.toa.shape[0]),
                           self.toa.ctypes.data_as(_ip), _d(self.pos), _d(self.rot))

    @property
    def ptr(self):
        return C.byref(self.sys)


def threads() -> int:
    return int(load().hsref_threads())


def sbessel(lmax: int, x: float):
    j = np.zeros(lmax + 1)
    dj = np.zeros(lmax + 1)
    if load().hsref_sbessel(int(lmax), float(x), _d(j), _d(dj)) != 0:
        raise ValueError("sbessel: bad lmax")
    return j, dj


def ylm(lmax: int, v) -> np.ndarray:
    vv = _f64(v)
    out = np.zeros(2 * (lmax + 1) ** 2)
    if load().hsref_ylm(int(lmax), _d(vv), _d(out)) != 0:
        raise ValueError("ylm: bad lmax")
    return out.view(np.complex128)


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    return float(load().hsref_wigner3j(j1, j2, j3, m1, m2, m3))


def gaunt(l, m, lp, mp, lpp, mpp) -> float:
    return float(load().hsref_gaunt(l, m, lp, mp, lpp, mpp))


def T_matrix(atom_type) -> np.ndarray:
    """(2N_L, 2N_L) complex T for one species."""
    from types import SimpleNamespace
    m = _Marshal(SimpleNamespace(types=[atom_type], type_of_atom=np.zeros(1, np.int32), pos=np.zeros(3),
                                 rot=np.eye(3), omega=1.0))
    n = 2 * (atom_type.lmax + 1) ** 2
    out = np.zeros(2 * n * n)
    if load().hsref_T(C.byref(m.types[0]), _d(out)) != 0:
        raise RuntimeError("hsref_T failed")
    return out.view(np.complex128).reshape(n, n, order="F")


def cholesky(T: np.ndarray):
    """(info, C): the Cholesky factor C (lower, C C^H = T) of a Hermitian T
    and the potrf-style status (0: HPD; k > 0: the leading minor of order k
    is not positive definite, C then holds the first k - 1 columns)."""
    A = _c128(T)
    n = A.shape[0]
    buf = _c128(A.reshape(-1, order="F")).view(np.float64).copy()
    out = np.zeros(2 * n * n)
    info = load().hsref_cholesky(n, _d(buf), max(n, 1), _d(out))
    if info < 0:
        raise MemoryError("hsref_cholesky")
    return int(info), out.view(np.complex128).reshape(n, n, order="F")


def T_hpd_info(atom_type) -> int:
    """Sec. 4.6.3: the status of the Cholesky factorisation of the species'
    T (0: HPD, the species takes the H = Y^H Y route)."""
    return cholesky(T_matrix(atom_type))[0]


def coefficients(sysm, atom: int, kvec: np.ndarray) -> np.ndarray:
    """W_a = [A_a; B_a] as (2N_L, N_G) complex (column t = plane wave t)."""
    m = _Marshal(sysm)
    kv = _f64(kvec).reshape(-1).copy()
    n_g = kv.shape[0] // 3
    nl2 = 2 * (sysm.types[int(sysm.type_of_atom[atom])].lmax + 1) ** 2
    out = np.zeros(2 * nl2 * n_g)
    if load().hsref_coefficients(m.ptr, int(atom), n_g, _d(kv), _d(out)) != 0:
        raise RuntimeError("hsref_coefficients failed")
    return out.view(np.complex128).reshape(n_g, nl2).T


def build_HS(sysm, kvec: np.ndarray, full: bool = False, compensated: bool = False):
    """H, S (N_G x N_G complex). full=False: upper triangle only (rest zero)."""
    m = _Marshal(sysm)
    kv = _f64(kvec).reshape(-1).copy()
    n_g = kv.shape[0] // 3
    H = np.zeros(2 * n_g * n_g)
    S = np.zeros(2 * n_g * n_g)
    rc = load().hsref_build_HS(m.ptr, n_g, _d(kv), _d(H), _d(S), max(n_g, 1), int(full), int(compensated))
    if rc != 0:
        raise RuntimeError(f"hsref_build_HS failed ({rc})")
    return (H.view(np.complex128).reshape(n_g, n_g, order="F"),
            S.view(np.complex128).reshape(n_g, n_g, order="F"))


def HS_entries(sysm, kvec: np.ndarray, rows, cols, compensated: bool = False):
    m = _Marshal(sysm)
    kv = _f64(kvec).reshape(-1).copy()
    n_g = kv.shape[0] // 3
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    H = np.zeros(2 * r.shape[0])
    S = np.zeros(2 * r.shape[0])
    rc = load().hsref_HS_entries(m.ptr, n_g, _d(kv), int(r.shape[0]), r.ctypes.data_as(_ip),
                                 c.ctypes.data_as(_ip), _d(H), _d(S), int(compensated))
    if rc != 0:
        raise RuntimeError(f"hsref_HS_entries failed ({rc})")
    return H.view(np.complex128), S.view(np.complex128)


def HS_columns(sysm, kvec: np.ndarray, cols, norms: bool = False):
    """Whole columns H[:, cols], S[:, cols] (N_G x len(cols) complex), every row.
    norms=True also returns (||w_t|| for every row, ||T w|| and ||U w|| of the columns)."""
    m = _Marshal(sysm)
    kv = _f64(kvec).reshape(-1).copy()
    n_g = kv.shape[0] // 3
    c = np.ascontiguousarray(cols, dtype=np.int32)
    H = np.zeros(2 * n_g * c.shape[0])
    S = np.zeros(2 * n_g * c.shape[0])
    wn, xn, yn = np.zeros(n_g), np.zeros(c.shape[0]), np.zeros(c.shape[0])
    rc = load().hsref_HS_columns(m.ptr, n_g, _d(kv), int(c.shape[0]), c.ctypes.data_as(_ip), _d(H), _d(S),
                                 _d(wn), _d(xn), _d(yn))
    if rc != 0:
        raise RuntimeError(f"hsref_HS_columns failed ({rc})")
    Hc = H.view(np.complex128).reshape(n_g, c.shape[0], order="F")
    Sc = S.view(np.complex128).reshape(n_g, c.shape[0], order="F")
    return (Hc, Sc, (wn, xn, yn)) if norms else (Hc, Sc)


def HS_brute(sysm, kvec: np.ndarray):
    m = _Marshal(sysm)
    kv = _f64(kvec).reshape(-1).copy()
    n_g = kv.shape[0] // 3
    H = np.zeros(2 * n_g * n_g)
    S = np.zeros(2 * n_g * n_g)
    if load().hsref_HS_brute(m.ptr, n_g, _d(kv), _d(H), _d(S), max(n_g, 1)) != 0:
        raise RuntimeError("hsref_HS_brute failed")
    return (H.view(np.complex128).reshape(n_g, n_g, order="F"),
            S.view(np.complex128).reshape(n_g, n_g, order="F"))
