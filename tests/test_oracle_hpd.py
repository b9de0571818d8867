"""Pins of the oracle's HPD test (Sec. 4.6.2-4.6.3): the Cholesky status that
routes a species' H contribution through Y = C^H W.

What fixes the answer independently of the oracle's own loop: a Hermitian
matrix is positive definite exactly when its smallest eigenvalue is positive
(numpy's eigvalsh), the factor is unique (C C^H = T with a positive diagonal,
so it equals numpy's cholesky), and the potrf status k is the order of the
first leading minor that is not positive definite (eigenvalues of the
leading minors, brute force). CPU only.
"""
import numpy as np
import pytest

import oracle
from workloads import make_config, shift_energies


def _rand_hpd(rng, n, shift=0.1):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return M @ M.conj().T + shift * np.eye(n)


def _first_bad_minor(T):
    for k in range(1, T.shape[0] + 1):
        if np.linalg.eigvalsh(T[:k, :k]).min() <= 0.0:
            return k
    return 0


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_factor_of_hpd_matrix(n):
    rng = np.random.default_rng(100 + n)
    T = _rand_hpd(rng, n)
    info, C = oracle.cholesky(T)
    assert info == 0
    assert np.allclose(np.triu(C, 1), 0.0)
    d = np.diag(C)
    assert np.all(d.real > 0) and np.all(d.imag == 0)
    assert np.abs(C @ C.conj().T - T).max() <= 1e-13 * np.abs(T).max()
    assert np.abs(C - np.linalg.cholesky(T)).max() <= 1e-12 * np.abs(C).max()


def test_factor_reads_the_lower_triangle_only():
    rng = np.random.default_rng(7)
    T = _rand_hpd(rng, 9)
    junk = np.triu(rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9)), 1)
    info0, C0 = oracle.cholesky(T)
    info1, C1 = oracle.cholesky(np.tril(T) + junk)
    assert info0 == info1 == 0
    assert np.array_equal(C0, C1)


@pytest.mark.parametrize("seed", range(6))
def test_status_is_the_first_indefinite_leading_minor(seed):
    rng = np.random.default_rng(200 + seed)
    n = 12
    T = _rand_hpd(rng, n)
    T = T - np.linalg.eigvalsh(T)[2 + seed] * np.eye(n)  # a few eigenvalues below zero
    want = _first_bad_minor(T)
    assert want > 0
    assert oracle.cholesky(T)[0] == want


def test_special_cases():
    # diagonal: the first non-positive entry
    assert oracle.cholesky(np.diag([2.0, 1.0, -1.0, 3.0]).astype(complex))[0] == 3
    assert oracle.cholesky(np.diag([2.0, 0.0, 1.0]).astype(complex))[0] == 2
    # zero matrix: the first pivot
    assert oracle.cholesky(np.zeros((5, 5), complex))[0] == 1
    # complex 2 x 2 just inside / outside the cone: [[1, z], [z*, |z|^2 +- d]]
    z, d = 0.9j, 1e-3
    assert oracle.cholesky(np.array([[1, z], [np.conj(z), abs(z) ** 2 + d]]))[0] == 0
    assert oracle.cholesky(np.array([[1, z], [np.conj(z), abs(z) ** 2 - d]]))[0] == 2
    # NaN on the diagonal: not positive definite
    assert oracle.cholesky(np.diag([1.0, np.nan]).astype(complex))[0] == 2


def test_energy_shift_adds_sigma_D_and_makes_T_hpd():
    """Raising every E_l by sigma adds sigma * diag(1 on A rows, ||u_dot_l||^2
    on B rows) to T (Eq. t_matrices: E_l enters the spherical diagonal only);
    the stand-in species are not HPD as drawn and are with sigma = 12."""
    for cfg in (1, 2):
        w = make_config(cfg, n_g_override=10)
        sh = shift_energies(w.system, 12.0)
        for ty, ty2 in zip(w.system.types, sh.types):
            T0, T1 = oracle.T_matrix(ty), oracle.T_matrix(ty2)
            nl = ty.nl
            D = np.concatenate([np.ones(nl), np.repeat(ty.udot_norm2, [2 * l + 1 for l in range(ty.lmax + 1)])])
            assert np.abs(T1 - T0 - 12.0 * np.diag(D)).max() <= 1e-12
            assert np.linalg.eigvalsh(T0).min() < 0 and oracle.T_hpd_info(ty) == _first_bad_minor(T0) > 0
            assert np.linalg.eigvalsh(T1).min() > 0 and oracle.T_hpd_info(ty2) == 0


def test_Y_route_reproduces_H_contribution():
    """With T = C C^H, W^H T W = (C^H W)^H (C^H W) (Sec. 4.6.2): the oracle's
    factor of a stand-in species' shifted T gives the same per-atom H as T
    itself."""
    w = make_config(1, n_g_override=40)
    ty = shift_energies(w.system, 12.0).types[0]
    T = oracle.T_matrix(ty)
    info, C = oracle.cholesky(T)
    assert info == 0
    Wa = oracle.coefficients(shift_energies(w.system, 12.0), 0, w.kvecs[0])
    Y = C.conj().T @ Wa
    Ha = Wa.conj().T @ T @ Wa
    assert np.abs(Y.conj().T @ Y - Ha).max() <= 1e-12 * np.abs(Ha).max()
