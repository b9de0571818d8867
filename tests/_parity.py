"""Helpers shared by the GPU parity tests: oracle-side reference values and the
normwise per-entry scale ||w_i|| ||x_j|| (reading: the Cauchy-Schwarz scale
of any dot-product error, used for the per-entry tolerance)."""
import numpy as np

import oracle


def oracle_columns(system, kvec):
    """W (depth_unpadded x N_G) stacked over atoms, X = T_a W_a, Y = U W (oracle)."""
    Ws, Xs, Ys = [], [], []
    Ts = [oracle.T_matrix(t) for t in system.types]
    for a in range(system.n_atoms):
        ty = system.types[system.type_of_atom[a]]
        Wa = oracle.coefficients(system, a, kvec)
        Ws.append(Wa)
        Xs.append(Ts[system.type_of_atom[a]] @ Wa)
        lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
        u = np.concatenate([np.ones(ty.nl), ty.udot_norm2[lvec]])
        Ys.append(u[:, None] * Wa)
    return np.vstack(Ws), np.vstack(Xs), np.vstack(Ys)


def normwise_scales(system, kvec):
    W, X, Y = oracle_columns(system, kvec)
    return np.linalg.norm(W, axis=0), np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0)


def compare(A, B, wn, xn, mask):
    """Relative Frobenius error over `mask` and max per-entry normwise error."""
    d = np.abs(A - B)[mask]
    rel_f = np.linalg.norm((A - B)[mask]) / max(np.linalg.norm(B[mask]), 1e-300)
    scale = np.outer(wn, xn)[mask]
    per = np.max(d / np.maximum(scale, 1e-300)) if d.size else 0.0
    return rel_f, per


def tri_mask(n, uplo="U"):
    m = np.zeros((n, n), bool)
    if uplo == "U":
        m[np.triu_indices(n)] = True
    else:
        m[np.tril_indices(n)] = True
    return m
