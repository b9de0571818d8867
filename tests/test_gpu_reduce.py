"""GPU parity of the generalized-eigenproblem hand-off (Sec. 2.3, Eq.
matrix_kohnsham) through the C ABI: S = U^H U (or L L^H) in place and
H~ = U^-H H U^-1 in full, blocked, in this library's kernels only: FP64
tile kernels for the diagonal blocks (Cholesky and inverse), the products
as FP64 DMMA (FP64 form) or 7-slice BF16 products (split form, to
FP64-level accuracy).

Inputs: the oracle's muffin-tin H, S plus a stand-in for the interstitial
part (S + I, H + diag(|K_t|^2)) so that S is positive definite, uploaded in
the layout hsgen_build_HS writes (one triangle, column-major). Tolerance: both
sides are FP64 Cholesky + triangular solves in different orders, so they
agree to a few n eps cond(S); the test derives the bound from cond(S).
At the 16-atom / N_G 3000 size the library's own H, S are reduced and checked
through properties that hold at any size (U^H U = S and U^H H~ U = H on
sampled columns, exact Hermitian symmetry).
"""
import re

import numpy as np
import pytest

import oracle
from workloads import kpoint_list, make_config, make_system

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def pd_problem(seed, n_g):
    lat = np.array([[9.0, 0.3, 0.0], [0.0, 9.9, 0.2], [0.1, 0.0, 8.6]])
    sysm = make_system(seed, lat, [(2, 1.5), (4, 1.6), (0, 1.7)], [2, 1, 2])
    kv = kpoint_list(sysm.lattice, (0.13, -0.07, 0.21), n_g)
    H, S = oracle.build_HS(sysm, kv, full=True)
    return sysm, H + np.diag(np.sum(kv * kv, axis=1)), S + np.eye(n_g)


def to_device(M, uplo):
    """One triangle, column-major: the row-major buffer holds M^T."""
    import torch

    T = np.triu(M) if uplo == "U" else np.tril(M)
    return torch.from_numpy(np.ascontiguousarray(T.T)).cuda()


@pytest.mark.parametrize("precision,uplo,n_g", [("FP64", "U", 90), ("FP64", "L", 90), ("FP64", "U", 600),
                                                ("FP64", "L", 600), ("SPLIT", "U", 90), ("SPLIT", "U", 600),
                                                ("SPLIT", "U", 1300), ("SPLIT", "L", 600)])
def test_reduce_matches_oracle(hs, precision, uplo, n_g):
    """Blocks of 128 rows (1, 5 and 11 blocks here), diagonal blocks in FP64
    tile kernels; products in FP64 DMMA (FP64) or as 7-slice BF16 products on
    the tensor cores (SPLIT); the lower layout through a transposed copy."""
    import torch

    sysm, H, S = pd_problem(seed=3 + n_g, n_g=n_g)
    Hd, Sd = to_device(H, uplo), to_device(S, uplo)
    with hs.Generator(sysm, precision=getattr(hs, precision), uplo=uplo) as g:
        hs.hsgen_reduce_generalized(g.ctx, n_g, Hd.data_ptr(), Sd.data_ptr(), n_g, 0)
        torch.cuda.synchronize()
    Hr = Hd.cpu().numpy().T
    F = Sd.cpu().numpy().T
    Ho, Fo = oracle.reduce_generalized(H, S, uplo)
    ev = np.linalg.eigvalsh(S)
    tol = 8 * n_g * EPS * ev[-1] / ev[0]
    assert np.linalg.norm(Hr - Ho) <= tol * np.linalg.norm(Ho)
    assert np.array_equal(Hr, Hr.conj().T)  # exactly Hermitian, real diagonal
    tri = np.triu if uplo == "U" else np.tril
    assert np.linalg.norm(tri(F) - Fo) <= tol * np.linalg.norm(Fo)
    # the other triangle of S is left as it was (zeros here)
    other = np.tril(F, -1) if uplo == "U" else np.triu(F, 1)
    assert np.all(other == 0)
    # and the eigenvalues are LAPACK's generalized ones
    import scipy.linalg as sla

    ref = sla.eigh(H, S, eigvals_only=True)
    # |d lambda| <= ||dH~||_2 <= ||dH~||_F <= tol ||H~||_F <= tol sqrt(n) max |lambda|
    assert np.max(np.abs(np.linalg.eigvalsh(Hr) - ref)) <= tol * np.sqrt(n_g) * np.max(np.abs(ref))


def test_reduce_properties_at_3000(hs):
    """16 atoms, N_G 3000: the library's H, S (+ the interstitial stand-in)."""
    import torch

    w = make_config(1)
    kv = w.kvecs[0]
    n = kv.shape[0]
    with hs.Generator(w.system, precision=hs.SPLIT) as g:
        H, S = g.build(torch.from_numpy(kv).cuda())  # column-major views
        H += torch.diag(torch.from_numpy(np.sum(kv * kv, axis=1)).to(H)).triu()
        S += torch.eye(n, dtype=S.dtype, device=S.device)
        torch.cuda.synchronize()
        Hin = H.cpu().numpy()
        Sin = S.cpu().numpy()
        g.reduce(H, S)
        torch.cuda.synchronize()
        Hr = H.cpu().numpy()
        U = np.triu(S.cpu().numpy())
    Hf = oracle.hermitian_from_triangle(Hin, "U")
    Sf = oracle.hermitian_from_triangle(Sin, "U")
    ev = np.linalg.eigvalsh(Sf)
    assert ev[0] > 0
    tol_s = 8 * n * EPS
    tol_h = tol_s * ev[-1] / ev[0]
    assert np.array_equal(Hr, Hr.conj().T)
    assert np.all(np.diag(U).imag == 0) and np.all(np.diag(U).real > 0)
    cols = np.unique(np.r_[0, np.random.default_rng(4).choice(n, 10, replace=False), n - 1])
    # U^H U = S and U^H H~ U = H on sampled columns
    rec_s = U.conj().T @ U[:, cols]
    assert np.linalg.norm(rec_s - Sf[:, cols]) <= tol_s * np.linalg.norm(Sf[:, cols])
    rec_h = U.conj().T @ (Hr @ U[:, cols])
    assert np.linalg.norm(rec_h - Hf[:, cols]) <= tol_h * np.linalg.norm(Hf[:, cols])


@pytest.mark.parametrize("precision,n_g", [("FP64", 64), ("SPLIT", 64), ("SPLIT", 700)])
def test_reduce_rejects_non_positive_definite(hs, precision, n_g):
    """S indefinite (SPLIT at N_G 700: the failure is in the third block of 256)."""
    import torch

    sysm, H, S = pd_problem(seed=5, n_g=n_g)
    S[600:, 600:] -= 2.0 * np.eye(n_g - 600) * np.max(np.abs(S)) if n_g > 600 else 0.0
    if n_g <= 600:
        S = S - 2.0 * np.eye(n_g) * np.max(np.abs(S))  # negative definite
    Hd, Sd = to_device(H, "U"), to_device(S, "U")
    with hs.Generator(sysm, precision=getattr(hs, precision)) as g:
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_reduce_generalized(g.ctx, n_g, Hd.data_ptr(), Sd.data_ptr(), n_g, 0)
        assert ei.value.status == hs.ENUMERIC
        # the failing leading minor is reported: inside the shifted block (N_G 700) or the first row
        minor = int(re.search(r"leading minor (\d+)", str(ei.value)).group(1))
        assert (600 < minor <= n_g) if n_g > 600 else minor == 1, minor
        # the context stays usable
        sysm2, H2, S2 = pd_problem(seed=6, n_g=64)
        Hd2, Sd2 = to_device(H2, "U"), to_device(S2, "U")
        hs.hsgen_reduce_generalized(g.ctx, 64, Hd2.data_ptr(), Sd2.data_ptr(), 64, 0)
        torch.cuda.synchronize()
        Ho, _ = oracle.reduce_generalized(H2, S2, "U")
        assert np.linalg.norm(Hd2.cpu().numpy().T - Ho) <= 1e-12 * np.linalg.norm(Ho)


def test_reduce_rejects_host_pointers_and_aliasing(hs):
    import torch

    sysm, H, S = pd_problem(seed=7, n_g=32)
    Hh = np.ascontiguousarray(H.T)
    Sh = np.ascontiguousarray(S.T)
    with hs.Generator(sysm, precision=hs.FP64) as g:
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_reduce_generalized(g.ctx, 32, Hh.ctypes.data, Sh.ctypes.data, 32, 0)
        assert ei.value.status == hs.EINVAL
        Hd = to_device(H, "U")
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_reduce_generalized(g.ctx, 32, Hd.data_ptr(), Hd.data_ptr(), 32, 0)
        assert ei.value.status == hs.EINVAL
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_reduce_generalized(g.ctx, 32, Hd.data_ptr(), to_device(S, "U").data_ptr(), 16, 0)
        assert ei.value.status == hs.EINVAL
        torch.cuda.synchronize()
