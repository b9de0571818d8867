"""ORACLE -- test infrastructure only (tests/, the smoke check and the
benchmark's CPU-baseline leg may use it; the CUDA library never does).

Reduction of the generalized eigenproblem of Sec. 2.3 (Eq. matrix_kohnsham,
H c = eps S c, H and S Hermitian, S positive definite) to a standard one,
written from its textbook definition; the paper only says the problem is
solved numerically. With the Cholesky factor of S,

    S = U^H U  (U upper triangular, real positive diagonal)   -> H~ = U^-H H U^-1
    S = L L^H  (L = U^H lower triangular)                      -> H~ = L^-1 H L^-H

and H~ y = eps y holds with c = U^-1 y (= L^-H y). The factor is unique, so H~
is the same for both triangles. FP64 throughout; a Cholesky and triangular
solves from numpy / scipy are the library steps.
"""
from __future__ import annotations

import numpy as np


def hermitian_from_triangle(M: np.ndarray, uplo: str = "U") -> np.ndarray:
    """The Hermitian matrix whose `uplo` triangle (diagonal included) is M's."""
    M = np.asarray(M, dtype=np.complex128)
    T = np.triu(M) if uplo == "U" else np.tril(M)
    F = T + T.conj().T
    F[np.diag_indices_from(F)] = np.diag(T).real
    return F


def reduce_generalized(H: np.ndarray, S: np.ndarray, uplo: str = "U"):
    """(H~, factor): H~ = U^-H H U^-1 (full, Hermitian) and the Cholesky factor
    of S in the `uplo` triangle (U for 'U', L for 'L'; zeros elsewhere). Only
    the `uplo` triangles of H and S are read. Raises numpy.linalg.LinAlgError
    when S is not positive definite."""
    from scipy.linalg import solve_triangular

    Hf = hermitian_from_triangle(H, uplo)
    Sf = hermitian_from_triangle(S, uplo)
    L = np.linalg.cholesky(Sf)  # S = L L^H
    A = solve_triangular(L, Hf, lower=True)  # L^-1 H
    Ht = solve_triangular(L, A.conj().T, lower=True)  # L^-1 (L^-1 H)^H = L^-1 H L^-H
    Ht = 0.5 * (Ht + Ht.conj().T)
    factor = L.conj().T if uplo == "U" else L
    return Ht, factor
