"""Pins of the oracle's special functions against the mathematics (CPU only).

j_l (App. A.1): closed forms of j_0, j_1, scipy's spherical_jn, the sum rule
sum_l (2l+1) j_l(x)^2 = 1, and the derivative identity.
Y_lm: closed forms for l <= 2, scipy's sph_harm_y, Unsoeld's theorem and
orthonormality by exact product quadrature.
Gaunt (Eq. gaunt): sympy's exact values, the selection rules, and a direct
quadrature of Y*_{L'} Y_L Y_{L''} with scipy's harmonics.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle


XS = [1e-7, 5e-4, 0.01, 0.3, 1.0, 2.5, 4.4, 7.7, 9.0, 11.3, 15.0, 24.0, 40.0]


def test_bessel_closed_forms():
    for x in XS:
        j, dj = oracle.sbessel(1, x)
        assert j[0] == pytest.approx(math.sin(x) / x, rel=1e-14, abs=1e-300)
        if x > 0.5:
            j1 = math.sin(x) / x ** 2 - math.cos(x) / x
        else:  # Taylor series of the same closed form, no cancellation
            j1 = sum((-1) ** k * x ** (2 * k + 1) * 2.0 * (k + 1) / math.factorial(2 * k + 3) for k in range(12))
        assert j[1] == pytest.approx(j1, rel=1e-12, abs=1e-18)
        assert dj[0] == pytest.approx(-j[1], rel=1e-14, abs=1e-300)


def test_bessel_vs_scipy():
    ls = np.arange(13)
    for x in XS:
        j, dj = oracle.sbessel(12, x)
        ref = sp.spherical_jn(ls, x)
        dref = sp.spherical_jn(ls, x, derivative=True)
        scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
        assert np.max(np.abs(j - ref) / scale) < 5e-14, x
        dscale = np.maximum(np.abs(dref), 1e-3 * np.max(np.abs(dref)))
        assert np.max(np.abs(dj - dref) / dscale) < 5e-13, x


def test_bessel_zero_argument():
    j, dj = oracle.sbessel(10, 0.0)
    assert j[0] == 1.0 and np.all(j[1:] == 0.0)
    assert dj[1] == pytest.approx(1.0 / 3.0) and dj[0] == 0.0 and np.all(dj[2:] == 0.0)


@pytest.mark.parametrize("x", [0.2, 3.3, 8.1, 17.0])
def test_bessel_sum_rule(x):
    j, _ = oracle.sbessel(60, x)
    s = np.sum((2 * np.arange(61) + 1) * j ** 2)
    assert s == pytest.approx(1.0, abs=1e-14)


def _angles(v):
    v = np.asarray(v, float)
    r = np.linalg.norm(v)
    return np.arccos(v[2] / r), np.arctan2(v[1], v[0]) % (2 * np.pi)


def test_ylm_closed_forms():
    rng = np.random.default_rng(7)
    for _ in range(20):
        v = rng.normal(size=3)
        th, ph = _angles(v)
        Y = oracle.ylm(2, v)
        ct, st, e = math.cos(th), math.sin(th), np.exp(1j * ph)
        ref = {
            (0, 0): 0.5 / math.sqrt(math.pi),
            (1, 0): math.sqrt(3 / (4 * math.pi)) * ct,
            (1, 1): -math.sqrt(3 / (8 * math.pi)) * st * e,
            (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * ct * ct - 1),
            (2, 1): -math.sqrt(15 / (8 * math.pi)) * st * ct * e,
            (2, 2): math.sqrt(15 / (32 * math.pi)) * st * st * e * e,
        }
        for (l, m), val in ref.items():
            assert abs(Y[l * l + l + m] - val) < 1e-15
            assert abs(Y[l * l + l - m] - (-1) ** m * np.conj(val)) < 1e-15


def test_ylm_vs_scipy_and_unsoeld():
    rng = np.random.default_rng(11)
    for _ in range(30):
        v = rng.normal(size=3)
        th, ph = _angles(v)
        Y = oracle.ylm(10, v)
        for l in range(11):
            ms = np.arange(-l, l + 1)
            ref = sp.sph_harm_y(l, ms, th, ph)
            assert np.max(np.abs(Y[l * l: (l + 1) ** 2] - ref)) < 2e-14
            assert np.sum(np.abs(Y[l * l:(l + 1) ** 2]) ** 2) == pytest.approx((2 * l + 1) / (4 * math.pi), rel=1e-13)


def test_ylm_poles():
    Y = oracle.ylm(6, [0.0, 0.0, 2.0])
    for l in range(7):
        assert Y[l * l + l] == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), rel=1e-14)
        for m in range(1, l + 1):
            assert abs(Y[l * l + l + m]) < 1e-15 and abs(Y[l * l + l - m]) < 1e-15


def _sphere_grid(nth, nph):
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = 2 * np.pi * np.arange(nph) / nph
    X, P = np.meshgrid(x, ph, indexing="ij")
    W = np.outer(w, np.full(nph, 2 * np.pi / nph))
    st = np.sqrt(1 - X ** 2)
    pts = np.stack([st * np.cos(P), st * np.sin(P), X], axis=-1).reshape(-1, 3)
    return pts, W.reshape(-1)


def test_ylm_orthonormal_quadrature():
    lmax = 8
    pts, w = _sphere_grid(lmax + 2, 2 * lmax + 2)
    Y = np.array([oracle.ylm(lmax, p) for p in pts])  # (npts, NL)
    G = (Y.conj() * w[:, None]).T @ Y
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-13


def test_gaunt_vs_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    rng = np.random.default_rng(3)
    count = 0
    while count < 60:
        l, lp = rng.integers(0, 11, size=2)
        lpp = int(rng.integers(abs(l - lp), l + lp + 1))
        m = int(rng.integers(-l, l + 1))
        mp = int(rng.integers(-lp, lp + 1))
        mpp = mp - m
        if abs(mpp) > lpp:
            continue
        count += 1
        # G_{L,L',L''} = int Y*_{L'} Y_L Y_{L''} = (-1)^{m'} int Y_{l,m} Y_{l'',m''} Y_{l',-m'}
        ref = float((-1) ** (mp % 2) * wig.gaunt(int(l), lpp, int(lp), m, mpp, -mp))
        assert oracle.gaunt(int(l), m, int(lp), mp, lpp, mpp) == pytest.approx(ref, rel=1e-13, abs=1e-16)


def test_gaunt_selection_rules():
    for l in range(5):
        for lp in range(5):
            for lpp in range(0, 10):
                for m in range(-l, l + 1):
                    for mp in range(-lp, lp + 1):
                        for mpp in range(-lpp, lpp + 1):
                            g = oracle.gaunt(l, m, lp, mp, lpp, mpp)
                            allowed = (mp == m + mpp) and ((l + lp + lpp) % 2 == 0) and abs(l - lp) <= lpp <= l + lp
                            if not allowed:
                                assert g == 0.0


def test_gaunt_quadrature():
    lmax = 4
    pts, w = _sphere_grid(3 * lmax + 2, 6 * lmax + 2)
    th = np.arccos(np.clip(pts[:, 2], -1, 1))
    ph = np.arctan2(pts[:, 1], pts[:, 0]) % (2 * np.pi)

    def Y(l, m):
        return sp.sph_harm_y(l, m, th, ph)

    for (l, m, lp, mp, lpp) in [(1, 0, 1, 1, 2), (2, -1, 3, 1, 3), (4, 2, 2, -1, 4), (3, 3, 4, 4, 1),
                                (2, 0, 2, 0, 0), (4, -4, 4, 2, 8)]:
        mpp = mp - m
        if abs(mpp) > lpp:
            continue
        q = np.sum(w * np.conj(Y(lp, mp)) * Y(l, m) * Y(lpp, mpp))
        assert abs(q.imag) < 1e-14
        assert oracle.gaunt(l, m, lp, mp, lpp, mpp) == pytest.approx(q.real, abs=1e-14)
