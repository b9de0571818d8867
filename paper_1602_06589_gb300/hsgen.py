"""Thin ctypes binding of the C ABI in include/hsgen.h (argument marshalling only).

Each ``hsgen_*`` function here calls the entry point of the same name in
libhsgen.so; every step of the computation runs in that library's CUDA
kernels. torch is used only for device buffers and streams. If the library is
missing, loading raises: there is no fallback path.

``Generator`` wraps a context for a ``workloads.System``-like object (any
object with lattice, omega, types, type_of_atom, pos, rot attributes).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsgen.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP, ENUMERIC = range(7)
FP64, SPLIT = 0, 1
S_CONTRACTION, S_LEGENDRE = 0, 1
SCHEME_AUTO, SCHEME_SLICES, SCHEME_MODULI = 0, 1, 2
H_TW, H_HPD = 0, 1
STATUS_NAMES = {0: "HSGEN_OK", 1: "HSGEN_EINVAL", 2: "HSGEN_ENOMEM", 3: "HSGEN_ECUDA", 4: "HSGEN_ETIMEOUT",
                5: "HSGEN_ENOTSUP", 6: "HSGEN_ENUMERIC"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("target_rel_err", C.c_double), ("slices", C.c_int), ("uplo", C.c_int),
                ("fill_full", C.c_int), ("atom_chunk", C.c_int), ("wait_timeout_ns", C.c_longlong),
                ("s_form", C.c_int), ("scheme", C.c_int), ("moduli", C.c_int), ("h_form", C.c_int)]


class TypeDesc(C.Structure):
    _fields_ = [("lmax", C.c_int), ("rmt", C.c_double), ("u", _dp), ("du", _dp), ("udot", _dp), ("dudot", _dp),
                ("wronskian", _dp), ("udot_norm2", _dp), ("e_l", _dp), ("I_uu", _dp), ("I_uud", _dp),
                ("I_udu", _dp), ("I_udud", _dp), ("T_override", _dp), ("lmax_nonsph", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("ms_coefficients", C.c_double), ("ms_tapply", C.c_double), ("ms_slice", C.c_double),
                ("ms_contract", C.c_double), ("ms_total", C.c_double), ("flops_algorithmic", C.c_double),
                ("precision", C.c_int), ("slices", C.c_int), ("n_kpoints", C.c_int),
                ("workspace_bytes", C.c_longlong), ("kernel_launches", C.c_longlong), ("s_form", C.c_int),
                ("ms_s", C.c_double), ("kseg_blocks", C.c_int), ("tile_band", C.c_int),
                ("ms_upload", C.c_double), ("ms_download", C.c_double), ("scheme", C.c_int), ("moduli", C.c_int),
                ("bits", C.c_int), ("products", C.c_int), ("atom_chunks", C.c_int), ("tuned_rel_err", C.c_double),
                ("stage_geometry", C.c_int), ("unit_order", C.c_int),
                ("l2_hint", C.c_int), ("hpd_species", C.c_int)]


EXPORTS = ["hsgen_default_options", "hsgen_create", "hsgen_set_atoms", "hsgen_build_HS", "hsgen_build_HS_blocks",
           "hsgen_build_HS_batched",
           "hsgen_coefficients", "hsgen_coefficients_noalloc", "hsgen_T_matrix", "hsgen_T_factor", "hsgen_depth_layout",
           "hsgen_autotune",
           "hsgen_reduce_generalized", "hsgen_get_stats", "hsgen_synchronize", "hsgen_last_error",
           "hsgen_destroy"]

_LIB = None
_LOCK = threading.Lock()


class HsgenError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: Optional[str] = None):
    """Loads libhsgen.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None and path is None:
            return _LIB
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1602_06589_gb300.build.build() "
                               "(there is no non-CUDA fallback)")
        lib = C.CDLL(p)
        vp = C.c_void_p
        lib.hsgen_default_options.argtypes = [C.POINTER(Options)]
        lib.hsgen_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Options)]
        lib.hsgen_set_atoms.argtypes = [vp, _dp, C.c_double, C.c_int, C.POINTER(TypeDesc), C.c_int, _ip, _dp, _dp]
        lib.hsgen_build_HS.argtypes = [vp, C.c_int, vp, vp, vp, C.c_longlong, vp]
        lib.hsgen_build_HS_blocks.argtypes = [vp, C.c_int, vp, vp, vp, C.c_longlong, C.c_int, C.c_int, C.c_int,
                                              C.c_int, C.c_int, vp]
        lib.hsgen_build_HS_batched.argtypes = [vp, C.c_int, _ip, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                               C.POINTER(C.c_longlong), vp]
        lib.hsgen_coefficients.argtypes = [vp, C.c_int, vp, vp, C.c_longlong, vp]
        lib.hsgen_coefficients_noalloc.argtypes = [vp, C.c_int, vp, vp, C.c_longlong, vp]
        lib.hsgen_T_matrix.argtypes = [vp, C.c_int, _dp]
        lib.hsgen_T_factor.argtypes = [vp, C.c_int, _dp, _ip]
        lib.hsgen_depth_layout.argtypes = [vp, _ip, C.c_int]
        lib.hsgen_autotune.argtypes = [vp, C.c_int, vp, vp, vp, C.c_longlong, vp]
        lib.hsgen_reduce_generalized.argtypes = [vp, C.c_int, vp, vp, C.c_longlong, vp]
        lib.hsgen_get_stats.argtypes = [vp, C.POINTER(Stats)]
        lib.hsgen_synchronize.argtypes = [vp, vp]
        lib.hsgen_last_error.argtypes = [vp]
        lib.hsgen_last_error.restype = C.c_char_p
        lib.hsgen_destroy.argtypes = [vp]
        lib.hsgen_destroy.restype = None
        for name in EXPORTS:
            if name not in ("hsgen_last_error", "hsgen_destroy"):
                getattr(lib, name).restype = C.c_int
        if path is None:
            _LIB = lib
        return lib


# ---- C-ABI functions under their own names ----------------------------------

def hsgen_default_options() -> Options:
    o = Options()
    load().hsgen_default_options(C.byref(o))
    return o


def hsgen_create(device: int = 0, opt: Optional[Options] = None) -> C.c_void_p:
    h = C.c_void_p()
    st = load().hsgen_create(C.byref(h), int(device), C.byref(opt) if opt is not None else None)
    if st != OK:
        raise HsgenError(st, "hsgen_create failed (needs an sm_103 GPU)")
    return h


def hsgen_last_error(ctx) -> str:
    r = load().hsgen_last_error(ctx)
    return r.decode() if r else ""


def _check(ctx, st: int, what: str):
    if st != OK:
        raise HsgenError(st, f"{what}: {hsgen_last_error(ctx)}")


class _TypeArrays:
    def __init__(self, types):
        self.keep = []
        self.arr = (TypeDesc * len(types))()
        for i, t in enumerate(types):
            d = self.arr[i]
            d.lmax = int(t.lmax)
            d.rmt = float(t.rmt)
            lns = getattr(t, "lmax_nonsph", None)
            d.lmax_nonsph = -1 if lns is None else int(lns)
            for k in ("u", "du", "udot", "dudot", "udot_norm2", "e_l", "I_uu", "I_uud", "I_udu", "I_udud"):
                a = np.ascontiguousarray(getattr(t, k), dtype=np.float64)
                self.keep.append(a)
                setattr(d, k, a.ctypes.data_as(_dp))
            w = getattr(t, "wronskian", None)
            if w is not None:
                a = np.ascontiguousarray(w, dtype=np.float64)
                self.keep.append(a)
                d.wronskian = a.ctypes.data_as(_dp)
            tov = getattr(t, "T_override", None)
            if tov is not None:
                a = np.ascontiguousarray(np.asfortranarray(tov, dtype=np.complex128).reshape(-1, order="F"))
                a = a.view(np.float64).copy()
                self.keep.append(a)
                d.T_override = a.ctypes.data_as(_dp)


def hsgen_set_atoms(ctx, lattice, omega: float, types, type_of_atom, pos, rot):
    ta = _TypeArrays(types)
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
    toa = np.ascontiguousarray(type_of_atom, dtype=np.int32)
    p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    r = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1)
    st = load().hsgen_set_atoms(ctx, lat.ctypes.data_as(_dp), float(omega), len(types), ta.arr, int(toa.shape[0]),
                                toa.ctypes.data_as(_ip), p.ctypes.data_as(_dp), r.ctypes.data_as(_dp))
    _check(ctx, st, "hsgen_set_atoms")


def hsgen_build_HS(ctx, n_g: int, kvec_ptr: int, H_ptr: int, S_ptr: int, ld: int, stream: int = 0):
    st = load().hsgen_build_HS(ctx, int(n_g), C.c_void_p(kvec_ptr), C.c_void_p(H_ptr), C.c_void_p(S_ptr),
                               int(ld), C.c_void_p(stream))
    _check(ctx, st, "hsgen_build_HS")


def hsgen_build_HS_blocks(ctx, n_g: int, kvec_ptr: int, H_ptr: int, S_ptr: int, ld: int, block: int, nprow: int,
                          npcol: int, myrow: int, mycol: int, stream: int = 0):
    st = load().hsgen_build_HS_blocks(ctx, int(n_g), C.c_void_p(kvec_ptr), C.c_void_p(H_ptr), C.c_void_p(S_ptr),
                                      int(ld), int(block), int(nprow), int(npcol), int(myrow), int(mycol),
                                      C.c_void_p(stream))
    _check(ctx, st, "hsgen_build_HS_blocks")


def hsgen_build_HS_batched(ctx, n_g: Sequence[int], kvec_ptrs, H_ptrs, S_ptrs, lds, stream: int = 0):
    n = len(n_g)
    ng = (C.c_int * n)(*[int(x) for x in n_g])
    kv = (C.c_void_p * n)(*[C.c_void_p(int(p)) for p in kvec_ptrs])
    hp = (C.c_void_p * n)(*[C.c_void_p(int(p)) for p in H_ptrs])
    sp = (C.c_void_p * n)(*[C.c_void_p(int(p)) for p in S_ptrs])
    ld = (C.c_longlong * n)(*[int(x) for x in lds])
    st = load().hsgen_build_HS_batched(ctx, n, ng, kv, hp, sp, ld, C.c_void_p(stream))
    _check(ctx, st, "hsgen_build_HS_batched")


def hsgen_coefficients(ctx, n_g: int, kvec_ptr: int, W_ptr: int, ldw: int, stream: int = 0):
    st = load().hsgen_coefficients(ctx, int(n_g), C.c_void_p(kvec_ptr), C.c_void_p(W_ptr), int(ldw),
                                   C.c_void_p(stream))
    _check(ctx, st, "hsgen_coefficients")


def hsgen_coefficients_noalloc(ctx, n_g: int, kvec_ptr: int, W_ptr: int, ldw: int, stream: int = 0):
    """Like hsgen_coefficients but with no device allocation (fixed library scratch;
    kvec and W on the device; n_types * n_g <= 95325)."""
    st = load().hsgen_coefficients_noalloc(ctx, int(n_g), C.c_void_p(kvec_ptr), C.c_void_p(W_ptr), int(ldw),
                                           C.c_void_p(stream))
    _check(ctx, st, "hsgen_coefficients_noalloc")


def hsgen_T_matrix(ctx, type_index: int, nl: int) -> np.ndarray:
    n = 2 * nl
    out = np.zeros(2 * n * n)
    _check(ctx, load().hsgen_T_matrix(ctx, int(type_index), out.ctypes.data_as(_dp)), "hsgen_T_matrix")
    return out.view(np.complex128).reshape(n, n, order="F")


def hsgen_T_factor(ctx, type_index: int, n: int):
    """(info, C): the Cholesky status of the species' T (0: HPD) and its lower
    factor C (n x n, n = 2 N_L of the contraction's rows)."""
    out = np.zeros(2 * n * n)
    info = C.c_int(-1)
    _check(ctx, load().hsgen_T_factor(ctx, int(type_index), out.ctypes.data_as(_dp), C.byref(info)), "hsgen_T_factor")
    return int(info.value), out.view(np.complex128).reshape(n, n, order="F")


def hsgen_depth_layout(ctx, n_atoms: int) -> np.ndarray:
    out = np.zeros(n_atoms + 1, dtype=np.int32)
    _check(ctx, load().hsgen_depth_layout(ctx, out.ctypes.data_as(_ip), n_atoms + 1), "hsgen_depth_layout")
    return out


def hsgen_autotune(ctx, n_g: int, kvec_ptr: int, H_ptr: int, S_ptr: int, ld: int, stream: int = 0):
    st = load().hsgen_autotune(ctx, int(n_g), C.c_void_p(kvec_ptr), C.c_void_p(H_ptr), C.c_void_p(S_ptr), int(ld),
                               C.c_void_p(stream))
    _check(ctx, st, "hsgen_autotune")


def hsgen_reduce_generalized(ctx, n: int, H_ptr: int, S_ptr: int, ld: int, stream: int = 0):
    st = load().hsgen_reduce_generalized(ctx, int(n), C.c_void_p(H_ptr), C.c_void_p(S_ptr), int(ld),
                                         C.c_void_p(stream))
    _check(ctx, st, "hsgen_reduce_generalized")


def hsgen_get_stats(ctx) -> dict:
    s = Stats()
    _check(ctx, load().hsgen_get_stats(ctx, C.byref(s)), "hsgen_get_stats")
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def hsgen_synchronize(ctx, stream: int = 0):
    """Waits for `stream`; raises HsgenError(ETIMEOUT) if a bounded device wait expired."""
    _check(ctx, load().hsgen_synchronize(ctx, C.c_void_p(stream)), "hsgen_synchronize")


def hsgen_destroy(ctx):
    if ctx:
        load().hsgen_destroy(ctx)


# ---- convenience wrapper ------------------------------------------------------

class Generator:
    """One context bound to one crystal; builds H and S into torch tensors."""

    def __init__(self, system, device: int = 0, precision: int = FP64, slices: int = 0,
                 target_rel_err: float = 1e-12, uplo: str = "U", fill_full: bool = False, atom_chunk: int = 0,
                 wait_timeout_ns: int = 2_000_000_000, s_form: int = S_CONTRACTION, scheme: int = SCHEME_AUTO,
                 moduli: int = 0, h_form: int = H_TW):
        o = hsgen_default_options()
        o.precision = precision
        o.slices = slices
        o.target_rel_err = target_rel_err
        o.uplo = ord(uplo)
        o.fill_full = int(fill_full)
        o.atom_chunk = atom_chunk
        o.wait_timeout_ns = wait_timeout_ns
        o.s_form = s_form
        o.scheme = scheme
        o.moduli = moduli
        o.h_form = h_form
        self.device = device
        self.system = system
        self.ctx = hsgen_create(device, o)
        try:
            hsgen_set_atoms(self.ctx, system.lattice, system.omega, system.types, system.type_of_atom,
                            system.pos, system.rot)
        except Exception:
            hsgen_destroy(self.ctx)
            self.ctx = None
            raise

    def close(self):
        if self.ctx:
            hsgen_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def depth_offsets(self) -> np.ndarray:
        return hsgen_depth_layout(self.ctx, len(self.system.type_of_atom))

    def build(self, kvec, H=None, S=None, stream=None):
        """kvec: (N_G, 3) float64 torch tensor (cuda or cpu) or numpy array.
        Returns (H, S) as complex128 cuda tensors (column-major: H[:, j] is column j,
        i.e. the tensor is the transpose view of a row-major buffer)."""
        import torch
        dev = torch.device("cuda", self.device)
        kv = kvec if isinstance(kvec, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(kvec))
        kv = kv.to(dtype=torch.float64).contiguous()
        n_g = int(kv.shape[0])
        if H is None:
            H = torch.zeros((n_g, n_g), dtype=torch.complex128, device=dev)
        if S is None:
            S = torch.zeros((n_g, n_g), dtype=torch.complex128, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        # column-major n_g x n_g with ld = n_g is a row-major tensor read transposed
        hsgen_build_HS(self.ctx, n_g, kv.data_ptr(), H.data_ptr(), S.data_ptr(), n_g, st.cuda_stream)
        return H.mT, S.mT

    def autotune(self, kvec, H=None, S=None, stream=None):
        """Picks the split form's depth segment and tile band by timing builds
        of this k-point (hsgen_autotune); returns (H, S) built with the choice."""
        import torch
        dev = torch.device("cuda", self.device)
        kv = kvec if isinstance(kvec, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(kvec))
        kv = kv.to(dtype=torch.float64).contiguous()
        n_g = int(kv.shape[0])
        if H is None:
            H = torch.zeros((n_g, n_g), dtype=torch.complex128, device=dev)
        if S is None:
            S = torch.zeros((n_g, n_g), dtype=torch.complex128, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        hsgen_autotune(self.ctx, n_g, kv.data_ptr(), H.data_ptr(), S.data_ptr(), n_g, st.cuda_stream)
        return H.mT, S.mT

    def reduce(self, H, S, stream=None):
        """Reduces H c = eps S c to standard form in place (hsgen_reduce_generalized).
        H, S: the (column-major) complex128 cuda tensors build() returns, or any
        n x n ones in that layout; returns (H~, factor) as the same views."""
        import torch
        n = int(H.shape[0])
        Hr, Sr = H.mT, S.mT  # the row-major buffers the library sees column-major
        assert Hr.is_contiguous() and Sr.is_contiguous(), "H, S must be column-major views of contiguous buffers"
        st = stream if stream is not None else torch.cuda.current_stream(H.device)
        hsgen_reduce_generalized(self.ctx, n, Hr.data_ptr(), Sr.data_ptr(), n, st.cuda_stream)
        return H, S

    def coefficients(self, kvec, stream=None):
        import torch
        dev = torch.device("cuda", self.device)
        kv = kvec if isinstance(kvec, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(kvec))
        kv = kv.to(device=dev, dtype=torch.float64).contiguous()
        n_g = int(kv.shape[0])
        depth = int(self.depth_offsets[-1])
        W = torch.zeros((n_g, depth), dtype=torch.complex128, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        hsgen_coefficients(self.ctx, n_g, kv.data_ptr(), W.data_ptr(), depth, st.cuda_stream)
        return W.mT  # (depth, N_G)

    def T_matrix(self, type_index: int) -> np.ndarray:
        return hsgen_T_matrix(self.ctx, type_index, self.system.types[type_index].nl)

    def T_factor(self, type_index: int, nl: Optional[int] = None):
        """(info, C) of hsgen_T_factor; nl: N_L of the contraction's rows (default the species' N_L)."""
        return hsgen_T_factor(self.ctx, type_index, 2 * (nl or self.system.types[type_index].nl))

    def stats(self) -> dict:
        return hsgen_get_stats(self.ctx)

    def synchronize(self, stream=None):
        """Waits for the stream and reports an expired bounded wait (HSGEN_ETIMEOUT)."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", self.device))
        hsgen_synchronize(self.ctx, st.cuda_stream)
