"""Pins of the oracle's reduction of the generalized eigenproblem (Sec. 2.3,
Eq. matrix_kohnsham) to standard form, against the mathematics (CPU only).

Inputs are the oracle's muffin-tin H, S plus a stand-in for the interstitial
part that the hot path does not compute: S + I and H + diag(|K_t|^2) (the
plane waves' own overlap and kinetic energy with unit weight), which makes S
positive definite as the full problem's S is.

Pins: the eigenvalues of H~ equal LAPACK's generalized eigenvalues of (H, S)
(scipy.linalg.eigh(H, S), a different routine); eigenvectors c = U^-1 y
satisfy H c = eps S c; the factor reproduces S and is triangular with a
positive real diagonal; S = I and S = diag(d) reduce to closed forms; both
triangles give the same H~; a planted mistake (the factor on the wrong side)
fails the eigenvalue pin.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from workloads import kpoint_list, make_system


def pd_problem(seed=3, n_g=90, uplo="U"):
    lat = np.array([[9.0, 0.3, 0.0], [0.0, 9.9, 0.2], [0.1, 0.0, 8.6]])
    sysm = make_system(seed, lat, [(2, 1.5), (4, 1.6), (0, 1.7)], [2, 1, 2])
    kv = kpoint_list(sysm.lattice, (0.13, -0.07, 0.21), n_g)
    H, S = oracle.build_HS(sysm, kv, full=True)
    H = H + np.diag(np.sum(kv * kv, axis=1))
    S = S + np.eye(n_g)
    keep = np.triu if uplo == "U" else np.tril
    return keep(H), keep(S), H, S


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_eigenvalues_match_lapack_generalized(uplo):
    Ht, Hs, Hf, Sf = pd_problem(uplo=uplo)
    Hr, F = oracle.reduce_generalized(Ht, Hs, uplo)
    ours = np.linalg.eigvalsh(Hr)
    ref = sla.eigh(Hf, Sf, eigvals_only=True)
    assert np.max(np.abs(ours - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_factor_reproduces_S_and_is_triangular(uplo):
    Ht, Hs, Hf, Sf = pd_problem(seed=5, uplo=uplo)
    _, F = oracle.reduce_generalized(Ht, Hs, uplo)
    rec = F.conj().T @ F if uplo == "U" else F @ F.conj().T
    assert np.linalg.norm(rec - Sf) <= 1e-14 * np.linalg.norm(Sf)
    other = np.tril(F, -1) if uplo == "U" else np.triu(F, 1)
    assert np.all(other == 0)
    d = np.diag(F)
    assert np.all(d.imag == 0) and np.all(d.real > 0)


def test_eigenvectors_solve_the_generalized_problem():
    Ht, Hs, Hf, Sf = pd_problem(seed=7, n_g=120)
    Hr, U = oracle.reduce_generalized(Ht, Hs, "U")
    eps, Y = np.linalg.eigh(Hr)
    C = sla.solve_triangular(U, Y, lower=False)
    R = Hf @ C - (Sf @ C) * eps
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(Hf) * np.linalg.norm(C)


def test_both_triangles_give_the_same_reduction():
    Ht, Hs, _, _ = pd_problem(seed=9, uplo="U")
    Hl, Sl, _, _ = pd_problem(seed=9, uplo="L")
    Ru, _ = oracle.reduce_generalized(Ht, Hs, "U")
    Rl, _ = oracle.reduce_generalized(Hl, Sl, "L")
    assert np.linalg.norm(Ru - Rl) <= 1e-14 * np.linalg.norm(Ru)


def test_identity_and_diagonal_S_closed_forms():
    rng = np.random.default_rng(1)
    n = 40
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    H = A + A.conj().T
    Hr, F = oracle.reduce_generalized(np.triu(H), np.eye(n), "U")
    assert np.allclose(F, np.eye(n), rtol=0, atol=0)
    assert np.linalg.norm(Hr - H) <= 1e-15 * np.linalg.norm(H)
    d = rng.uniform(0.5, 4.0, size=n)
    Hr, F = oracle.reduce_generalized(np.triu(H), np.diag(d), "U")
    want = H / np.sqrt(np.outer(d, d))
    assert np.linalg.norm(Hr - want) <= 1e-15 * np.linalg.norm(want)
    assert np.allclose(np.diag(F).real, np.sqrt(d), rtol=1e-15, atol=0)


def test_hermitian_from_triangle():
    rng = np.random.default_rng(2)
    M = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    F = oracle.hermitian_from_triangle(M, "U")
    assert np.array_equal(np.triu(F, 1), np.triu(M, 1))
    assert np.array_equal(F, F.conj().T)
    assert np.array_equal(np.diag(F).imag, np.zeros(6))


def test_planted_wrong_side_fails_the_eigenvalue_pin():
    """U^-1 H U^-H (factor on the wrong side) is not similar to the pencil."""
    _, _, Hf, Sf = pd_problem(seed=11)
    U = np.linalg.cholesky(Sf).conj().T
    A = sla.solve_triangular(U, Hf, lower=False)
    wrong = sla.solve_triangular(U, A.conj().T, lower=False)
    ref = sla.eigh(Hf, Sf, eigvals_only=True)
    bad = np.linalg.eigvalsh(0.5 * (wrong + wrong.conj().T))
    assert np.max(np.abs(bad - ref)) > 1e-6 * np.max(np.abs(ref))
