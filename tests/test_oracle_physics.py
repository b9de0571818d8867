"""Pins of the oracle's A, B, T, H and S against what the mathematics fixes.

None of these re-types the oracle's own formulas; each checks a different
route to the same quantity:
  * A, B (Eqs. def_a_tensor / def_b_tensor): the MT expansion must reproduce
    the Rayleigh expansion of the plane wave on the sphere, value and radial
    derivative (the C^1 matching of App. A.1), with scipy's Y_lm, j_l and
    Legendre polynomials; for large l_max, the plane wave itself.
  * S (Eq. def_overlap): the Legendre closed form obtained by summing over m
    (Sec. 3.1 m-sum identity, with the prefactor 4 pi / Omega), N_G = 1 case,
    Hermitian and positive semidefinite.
  * T (Eq. t_matrices) and H (Eq. def_hamilton): spherical-only T gives a
    Legendre closed form; the non-spherical part equals the angular quadrature
    of Phi^* V Phi, independent of the Gaunt table; H = S when T is
    blockdiag(1, U); a rank-one T gives a rank-<=N_A PSD H; brute-force
    quadruple sum agrees with the matrix form.
  * Invariances: atom permutation, lattice shift of one atom, global
    translation (H -> P H P^H), rotation of atoms under a spherical potential.
  * The oracle's own rounding: compensated (Dot2) vs plain summation.
"""
import copy
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle
from workloads import make_config, make_system, kpoint_list


def f_ab(ty, kn):
    """Radial matching factors f_A, f_B (from App. A.1) with scipy's j_l."""
    ls = np.arange(ty.lmax + 1)
    x = kn * ty.rmt
    j = sp.spherical_jn(ls, x)
    dj = sp.spherical_jn(ls, x, derivative=True)
    fa = ty.udot * kn * dj - ty.dudot * j
    fb = -ty.u * kn * dj + ty.du * j
    W = ty.udot * ty.du - ty.u * ty.dudot
    return fa, fb, W


def _angles(v):
    r = np.linalg.norm(v, axis=-1)
    th = np.arccos(np.clip(v[..., 2] / r, -1, 1))
    ph = np.arctan2(v[..., 1], v[..., 0]) % (2 * np.pi)
    return th, ph


def _ylm_scipy(lmax, pts):
    th, ph = _angles(pts)
    out = np.zeros(pts.shape[:-1] + ((lmax + 1) ** 2,), complex)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            out[..., l * l + l + m] = sp.sph_harm_y(l, m, th, ph)
    return out


def small_system(lmax=3, n_atoms=2, seed=5, identity_rot=False, cell=9.0):
    lat = np.diag([cell, cell * 1.1, cell * 1.2])
    species = [(lmax, 1.8), (max(lmax - 1, 0), 1.6)]
    counts = [n_atoms - n_atoms // 2, n_atoms // 2]
    return make_system(seed, lat, species, counts, identity_rot=identity_rot)


@pytest.mark.parametrize("cfg", ["c0", "small"])
def test_rayleigh_matching(cfg):
    if cfg == "c0":
        w = make_config(0)
        sysm, kv = w.system, w.kvecs[0][::17]
    else:
        sysm = small_system(lmax=5, n_atoms=3)
        kv = kpoint_list(sysm.lattice, (0.13, -0.21, 0.4), 40)[::5]
    rng = np.random.default_rng(2)
    rh = rng.normal(size=(12, 3))
    rh /= np.linalg.norm(rh, axis=1)[:, None]
    for a in range(sysm.n_atoms):
        ty = sysm.types[sysm.type_of_atom[a]]
        nl = ty.nl
        W = oracle.coefficients(sysm, a, kv)  # (2NL, NG)
        Yr = _ylm_scipy(ty.lmax, rh @ sysm.rot[a].T)  # Y_L(R_a r^)
        lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
        for t in range(kv.shape[0]):
            K = kv[t]
            kn = np.linalg.norm(K)
            A, B = W[:nl, t], W[nl:, t]
            val = (A * ty.u[lvec] + B * ty.udot[lvec]) @ Yr.T
            der = (A * ty.du[lvec] + B * ty.dudot[lvec]) @ Yr.T
            kh = K / kn if kn > 0 else np.array([0, 0, 1.0])
            ls = np.arange(ty.lmax + 1)
            jl = sp.spherical_jn(ls, kn * ty.rmt)
            djl = sp.spherical_jn(ls, kn * ty.rmt, derivative=True)
            P = np.array([sp.eval_legendre(l, rh @ kh) for l in ls])  # (l, npts)
            c = np.exp(1j * K @ sysm.pos[a]) / math.sqrt(sysm.omega)
            il = 1j ** ls
            ref_v = c * ((2 * ls + 1) * il * jl) @ P
            ref_d = c * ((2 * ls + 1) * il * kn * djl) @ P
            assert np.max(np.abs(val - ref_v)) < 1e-13 * max(1.0, np.max(np.abs(ref_v)))
            assert np.max(np.abs(der - ref_d)) < 1e-13 * max(1.0, np.max(np.abs(ref_d)))


def test_rayleigh_plane_wave_limit():
    sysm = small_system(lmax=20, n_atoms=1, seed=8)
    kv = kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 12)
    ty = sysm.types[0]
    rng = np.random.default_rng(4)
    rh = rng.normal(size=(6, 3))
    rh /= np.linalg.norm(rh, axis=1)[:, None]
    W = oracle.coefficients(sysm, 0, kv)
    Yr = _ylm_scipy(ty.lmax, rh @ sysm.rot[0].T)
    lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
    for t in range(kv.shape[0]):
        K = kv[t]
        assert np.linalg.norm(K) * ty.rmt + 12 <= ty.lmax
        val = (W[:ty.nl, t] * ty.u[lvec] + W[ty.nl:, t] * ty.udot[lvec]) @ Yr.T
        exact = np.exp(1j * (sysm.pos[0] + ty.rmt * rh) @ K) / math.sqrt(sysm.omega)
        assert np.max(np.abs(val - exact)) < 1e-12


def legendre_form(sysm, kv, diag):
    """sum over atoms and l of the m-summed product (Sec. 3.1 identity):
    (4 pi / Omega) sum_a e^{i(K_t - K_t').x_a} sum_l (2l+1) P_l(K^_t.K^_t') d_l(t', t) / W_l^2,
    with d_l built from f_A, f_B by `diag(ty, l, faL, fbL, faR, fbR)`."""
    n = kv.shape[0]
    kn = np.linalg.norm(kv, axis=1)
    kh = np.where(kn[:, None] > 0, kv / np.maximum(kn, 1e-300)[:, None], np.array([0, 0, 1.0]))
    cosg = np.clip(kh @ kh.T, -1, 1)
    out = np.zeros((n, n), complex)
    for a in range(sysm.n_atoms):
        ty = sysm.types[sysm.type_of_atom[a]]
        fa = np.zeros((n, ty.lmax + 1))
        fb = np.zeros((n, ty.lmax + 1))
        for t in range(n):
            fa[t], fb[t], W = f_ab(ty, kn[t])
        ph = np.exp(1j * kv @ sysm.pos[a])
        phase = np.conj(ph)[:, None] * ph[None, :]
        acc = np.zeros((n, n))
        for l in range(ty.lmax + 1):
            d = diag(ty, l, fa[:, l][:, None], fb[:, l][:, None], fa[:, l][None, :], fb[:, l][None, :])
            acc += (2 * l + 1) * sp.eval_legendre(l, cosg) * d / W[l] ** 2
        out += 4 * math.pi / sysm.omega * phase * acc
    return out


def s_diag(ty, l, faL, fbL, faR, fbR):
    return faL * faR + ty.udot_norm2[l] * fbL * fbR


def h_sph_diag(ty, l, faL, fbL, faR, fbR):
    return ty.e_l[l] * faL * faR + 0.5 * faL * fbR + 0.5 * fbL * faR + ty.e_l[l] * ty.udot_norm2[l] * fbL * fbR


def test_S_legendre_closed_form_c0():
    w = make_config(0)
    kv = w.kvecs[0]
    H, S = oracle.build_HS(w.system, kv, full=True)
    ref = legendre_form(w.system, kv, s_diag)
    assert np.max(np.abs(S - ref)) < 1e-13 * np.max(np.abs(ref))


def test_S_legendre_closed_form_c1_sampled():
    w = make_config(1)
    kv = w.kvecs[0]
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(kv.shape[0], 24, replace=False))
    rows, cols = np.meshgrid(idx, idx, indexing="ij")
    H, S = oracle.HS_entries(w.system, kv, rows.ravel(), cols.ravel())
    ref = legendre_form(w.system, kv[idx], s_diag).ravel()
    assert np.max(np.abs(S - ref)) < 1e-13 * np.max(np.abs(ref))


def test_S_single_plane_wave():
    sysm = small_system(lmax=4, n_atoms=3, seed=21)
    kv = kpoint_list(sysm.lattice, (0.3, 0.1, 0.2), 1)
    _, S = oracle.build_HS(sysm, kv)
    kn = np.linalg.norm(kv[0])
    ref = 0.0
    for a in range(sysm.n_atoms):
        ty = sysm.types[sysm.type_of_atom[a]]
        fa, fb, W = f_ab(ty, kn)
        ls = np.arange(ty.lmax + 1)
        ref += 4 * math.pi / sysm.omega * np.sum((2 * ls + 1) * (fa ** 2 + ty.udot_norm2 * fb ** 2) / W ** 2)
    assert S[0, 0].real == pytest.approx(ref, rel=1e-14)
    assert abs(S[0, 0].imag) < 1e-16


def test_H_spherical_only_closed_form():
    w = make_config(0)
    sysm = copy.deepcopy(w.system)
    for ty in sysm.types:
        for k in ("I_uu", "I_uud", "I_udu", "I_udud"):
            setattr(ty, k, np.zeros_like(getattr(ty, k)))
    kv = w.kvecs[0][:80]
    H, _ = oracle.build_HS(sysm, kv, full=True)
    ref = legendre_form(sysm, kv, h_sph_diag)
    assert np.max(np.abs(H - ref)) < 1e-13 * np.max(np.abs(ref))


def _sphere_grid(nth, nph):
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    X, P = np.meshgrid(x, ph, indexing="ij")
    W = np.outer(w, np.full(nph, 2 * np.pi / nph))
    st = np.sqrt(1 - X ** 2)
    pts = np.stack([st * np.cos(P), st * np.sin(P), X], axis=-1).reshape(-1, 3)
    return pts, W.reshape(-1)


@pytest.mark.parametrize("cfg", ["c0", "small", "small-lns"])
def test_H_quadrature_form(cfg):
    """Non-spherical H from the angular integral of Phi^{x*}_{l',t'} V_{l''} Phi^y_{l,t}
    on an exact product grid (no Gaunt table), plus the spherical Legendre part.
    "small-lns": l_nonsph = 1 (Sec. 3.1, Fig. Tmat_structure): the non-spherical
    integral only couples l, l' <= 1, the spherical part runs to l_max."""
    lns = None
    if cfg == "c0":
        w = make_config(0)
        sysm, kv = w.system, w.kvecs[0][::10]
    else:
        sysm = small_system(lmax=3, n_atoms=2, seed=13)
        kv = kpoint_list(sysm.lattice, (0.05, 0.3, -0.2), 60)[::4]
        if cfg == "small-lns":
            lns = 1
            for ty in sysm.types:
                ty.lmax_nonsph = lns
    n = kv.shape[0]
    H, _ = oracle.build_HS(sysm, kv, full=True)
    ref = legendre_form(sysm, kv, h_sph_diag)
    for a in range(sysm.n_atoms):
        ty = sysm.types[sysm.type_of_atom[a]]
        lm = ty.lmax
        pts, wq = _sphere_grid(2 * lm + 2, 4 * lm + 2)
        Y = _ylm_scipy(2 * lm, pts)  # (npts, (2lm+1)^2)
        Wc = oracle.coefficients(sysm, a, kv)
        nl = ty.nl
        # Phi^{A/B}_{l,t}(Omega) = sum_m coef_{lm,t} Y_lm(Omega)
        phi = {}
        for key, off in (("A", 0), ("B", nl)):
            arr = np.zeros((lm + 1, len(wq), n), complex)
            for l in range(lm + 1):
                sl = slice(l * l, (l + 1) ** 2)
                arr[l] = Y[:, sl] @ Wc[off + l * l: off + (l + 1) ** 2, :]
            phi[key] = arr
        V = np.zeros((2 * lm + 1, len(wq)), complex)
        for l2 in range(2 * lm + 1):
            for m2 in range(-l2, l2 + 1):
                c = 1.0 if m2 >= 0 else (-1.0) ** m2
                V[l2] += c * Y[:, l2 * l2 + l2 + m2]
        Ixy = {("A", "A"): ty.I_uu, ("A", "B"): ty.I_uud, ("B", "A"): ty.I_udu, ("B", "B"): ty.I_udud}
        lcut = lm if lns is None else min(lns, lm)
        for (x, y), I in Ixy.items():
            for l in range(lcut + 1):
                for lp in range(lcut + 1):
                    for l2 in range(2 * lm + 1):
                        if I[l, lp, l2] == 0.0:
                            continue
                        f = (wq * V[l2])[:, None] * phi[y][l]
                        ref += I[l, lp, l2] * (phi[x][lp].conj().T @ f)
    assert np.max(np.abs(H - ref)) < 1e-12 * np.max(np.abs(ref))


def test_H_equals_S_for_U_weighted_identity():
    sysm = small_system(lmax=3, n_atoms=3, seed=17)
    for ty in sysm.types:
        T = np.zeros((2 * ty.nl, 2 * ty.nl), complex)
        lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
        T[:ty.nl, :ty.nl] = np.eye(ty.nl)
        T[ty.nl:, ty.nl:] = np.diag(ty.udot_norm2[lvec])
        ty.T_override = T
    kv = kpoint_list(sysm.lattice, (0.2, 0.1, 0.0), 50)
    H, S = oracle.build_HS(sysm, kv, full=True)
    assert np.max(np.abs(H - S)) <= 1e-15 * np.max(np.abs(S))


def test_H_rank_one_T():
    sysm = small_system(lmax=2, n_atoms=3, seed=19)
    rng = np.random.default_rng(5)
    vs = []
    for ty in sysm.types:
        v = rng.normal(size=2 * ty.nl) + 1j * rng.normal(size=2 * ty.nl)
        ty.T_override = np.outer(v, v.conj())
        vs.append(v)
    kv = kpoint_list(sysm.lattice, (0.1, 0.1, 0.1), 30)
    H, _ = oracle.build_HS(sysm, kv, full=True)
    ref = np.zeros_like(H)
    for a in range(sysm.n_atoms):
        c = vs[sysm.type_of_atom[a]].conj() @ oracle.coefficients(sysm, a, kv)  # c(t) = v^H w_t
        ref += np.outer(c.conj(), c)
    assert np.max(np.abs(H - ref)) < 1e-13 * np.max(np.abs(ref))
    ev = np.linalg.eigvalsh(0.5 * (H + H.conj().T))
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(ev > 1e-10 * ev.max()) <= sysm.n_atoms


def test_hermitian_psd_and_brute_force_c0():
    w = make_config(0)
    H, S = oracle.build_HS(w.system, w.kvecs[0], full=True)
    assert np.max(np.abs(H - H.conj().T)) < 1e-14 * np.max(np.abs(H))
    assert np.max(np.abs(S - S.conj().T)) < 1e-14 * np.max(np.abs(S))
    ev = np.linalg.eigvalsh(S)
    assert ev.min() > -1e-13 * ev.max()
    Hb, Sb = oracle.HS_brute(w.system, w.kvecs[0])
    assert np.max(np.abs(H - Hb)) < 1e-13 * np.max(np.abs(H))
    assert np.max(np.abs(S - Sb)) < 1e-13 * np.max(np.abs(S))


def test_upper_triangle_matches_full():
    sysm = small_system(lmax=3, n_atoms=2, seed=23)
    kv = kpoint_list(sysm.lattice, (0.2, 0.3, 0.1), 40)
    Hf, Sf = oracle.build_HS(sysm, kv, full=True)
    Hu, Su = oracle.build_HS(sysm, kv, full=False)
    iu = np.triu_indices(40)
    assert np.array_equal(Hu[iu], Hf[iu]) and np.array_equal(Su[iu], Sf[iu])
    il = np.tril_indices(40, -1)
    assert np.all(Hu[il] == 0) and np.all(Su[il] == 0)
    rows, cols = np.triu_indices(40)
    He, Se = oracle.HS_entries(sysm, kv, rows, cols)
    assert np.array_equal(He, Hf[rows, cols]) and np.array_equal(Se, Sf[rows, cols])


def test_whole_columns_match_full_matrix():
    """Whole columns (every row) equal the same columns of the full matrix."""
    sysm = small_system(lmax=3, n_atoms=3, seed=37)
    kv = kpoint_list(sysm.lattice, (0.17, -0.05, 0.29), 50)
    Hf, Sf = oracle.build_HS(sysm, kv, full=True)
    cols = [0, 17, 49]
    Hc, Sc = oracle.HS_columns(sysm, kv, cols)
    assert np.array_equal(Hc, Hf[:, cols]) and np.array_equal(Sc, Sf[:, cols])


def test_caller_wronskian():
    """App. A.1 divides A and B by W_l: a caller's W_l equal to
    u_dot u' - u u_dot' changes nothing, and W_l scaled by c_l scales the A
    and B rows of that l by 1 / c_l."""
    sysm = small_system(lmax=4, n_atoms=3, seed=31)
    kv = kpoint_list(sysm.lattice, (0.11, 0.23, -0.17), 30)
    W0 = [oracle.coefficients(sysm, a, kv) for a in range(sysm.n_atoms)]
    same = copy.deepcopy(sysm)
    for ty in same.types:
        ty.wronskian = ty.udot * ty.du - ty.u * ty.dudot
    for a in range(sysm.n_atoms):
        assert np.array_equal(oracle.coefficients(same, a, kv), W0[a])
    scaled = copy.deepcopy(sysm)
    rng = np.random.default_rng(7)
    cs = []
    for ty in scaled.types:
        c = rng.uniform(0.5, 2.0, ty.lmax + 1)
        ty.wronskian = c * (ty.udot * ty.du - ty.u * ty.dudot)
        cs.append(c)
    for a in range(sysm.n_atoms):
        t = int(sysm.type_of_atom[a])
        ty = sysm.types[t]
        lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
        inv = np.concatenate([1.0 / cs[t][lvec], 1.0 / cs[t][lvec]])
        W1 = oracle.coefficients(scaled, a, kv)
        assert np.max(np.abs(W1 - W0[a] * inv[:, None])) <= 1e-14 * np.max(np.abs(W0[a]))
        assert not np.allclose(W1, W0[a])


def test_invariances():
    sysm = small_system(lmax=3, n_atoms=4, seed=29)
    kv = kpoint_list(sysm.lattice, (0.1, -0.2, 0.35), 45)
    H, S = oracle.build_HS(sysm, kv, full=True)
    sc = max(np.max(np.abs(H)), np.max(np.abs(S)))
    # atom permutation
    perm = np.array([2, 0, 3, 1])
    p = copy.deepcopy(sysm)
    p.type_of_atom, p.pos, p.rot = sysm.type_of_atom[perm], sysm.pos[perm], sysm.rot[perm]
    H2, S2 = oracle.build_HS(p, kv, full=True)
    assert np.max(np.abs(H2 - H)) < 1e-14 * sc and np.max(np.abs(S2 - S)) < 1e-14 * sc
    # lattice-vector shift of one atom
    q = copy.deepcopy(sysm)
    q.pos = sysm.pos.copy()
    q.pos[1] += sysm.lattice[0] - 2 * sysm.lattice[2]
    H3, S3 = oracle.build_HS(q, kv, full=True)
    assert np.max(np.abs(H3 - H)) < 1e-13 * sc and np.max(np.abs(S3 - S)) < 1e-13 * sc
    # global translation: H -> P H P^H with P = diag(e^{-i K_t . d}) on the conjugated side
    d = np.array([0.37, -1.2, 0.5])
    r = copy.deepcopy(sysm)
    r.pos = sysm.pos + d
    H4, S4 = oracle.build_HS(r, kv, full=True)
    ph = np.exp(1j * kv @ d)
    assert np.max(np.abs(H4 - np.conj(ph)[:, None] * H * ph[None, :])) < 1e-13 * sc
    assert np.max(np.abs(S4 - np.conj(ph)[:, None] * S * ph[None, :])) < 1e-13 * sc


def test_rotation_invariance_spherical_potential():
    sysm = small_system(lmax=3, n_atoms=2, seed=31)
    for ty in sysm.types:
        for k in ("I_uu", "I_uud", "I_udu", "I_udud"):
            arr = getattr(ty, k).copy()
            arr[:, :, 1:] = 0.0
            setattr(ty, k, arr)
    kv = kpoint_list(sysm.lattice, (0.3, 0.1, 0.2), 30)
    H, S = oracle.build_HS(sysm, kv, full=True)
    r = copy.deepcopy(sysm)
    r.rot = np.tile(np.eye(3), (sysm.n_atoms, 1, 1))
    H2, S2 = oracle.build_HS(r, kv, full=True)
    assert np.max(np.abs(H2 - H)) < 1e-13 * np.max(np.abs(H))
    assert np.max(np.abs(S2 - S)) < 1e-13 * np.max(np.abs(S))


def test_T_hermitian_and_structure():
    w = make_config(1)
    for ty in w.system.types:
        T = oracle.T_matrix(ty)
        nl = ty.nl
        assert np.max(np.abs(T - T.conj().T)) < 1e-14 * np.max(np.abs(T))
        assert np.max(np.abs(T[nl:, :nl] - T[:nl, nl:].conj().T)) < 1e-14  # T^BA = (T^AB)^H


def test_T_nonsph_block_structure():
    """l_nonsph < l_max (Fig. Tmat_structure): inside the dense block T equals the
    full T; outside it only the spherical diagonal of App. A.2 remains (E_l,
    E_l ||u_dot_l||^2, and 1/2 on AB and BA, reading R1)."""
    sysm = small_system(lmax=4, n_atoms=2, seed=23)
    for ty in sysm.types:
        full = oracle.T_matrix(ty)
        for lns in range(0, ty.lmax):
            t2 = copy.deepcopy(ty)
            t2.lmax_nonsph = lns
            T = oracle.T_matrix(t2)
            nl = ty.nl
            lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
            inner = np.tile(lvec <= lns, 2)
            blk = np.outer(inner, inner)
            assert np.array_equal(T[blk], full[blk])
            sph = np.zeros_like(full)
            for L, l in enumerate(lvec):
                sph[L, L] = ty.e_l[l]
                sph[nl + L, nl + L] = ty.e_l[l] * ty.udot_norm2[l]
                sph[L, nl + L] = sph[nl + L, L] = 0.5
            assert np.max(np.abs(T[~blk] - sph[~blk])) < 1e-15
            assert np.max(np.abs(T - T.conj().T)) < 1e-14 * np.max(np.abs(T))


def test_compensated_vs_plain():
    w = make_config(1)
    kv = w.kvecs[0]
    rng = np.random.default_rng(1)
    idx = rng.choice(kv.shape[0], 16, replace=False)
    rows, cols = np.meshgrid(idx, idx, indexing="ij")
    H, S = oracle.HS_entries(w.system, kv, rows.ravel(), cols.ravel())
    Hc, Sc = oracle.HS_entries(w.system, kv, rows.ravel(), cols.ravel(), compensated=True)
    assert np.max(np.abs(H - Hc)) < 1e-14 * np.max(np.abs(Hc))
    assert np.max(np.abs(S - Sc)) < 1e-14 * np.max(np.abs(Sc))


def test_gamma_point_plane_wave():
    """K = 0 (k = 0, G = 0): only l = 0 survives (j_l(0) = delta_l0)."""
    sysm = small_system(lmax=4, n_atoms=2, seed=37)
    kv = kpoint_list(sysm.lattice, (0.0, 0.0, 0.0), 7)
    assert np.linalg.norm(kv[0]) == 0.0
    W = oracle.coefficients(sysm, 0, kv)
    ty = sysm.types[0]
    assert np.all(W[1:ty.nl, 0] == 0) and np.all(W[ty.nl + 1:, 0] == 0)
    fa, fb, Wr = f_ab(ty, 0.0)
    y00 = 0.5 / math.sqrt(math.pi)
    pre = 4 * math.pi / (Wr[0] * math.sqrt(sysm.omega)) * np.exp(1j * 0.0)
    assert W[0, 0] == pytest.approx(pre * y00 * fa[0], rel=1e-14)
    assert W[ty.nl, 0] == pytest.approx(pre * y00 * fb[0], rel=1e-14)
