"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle source (a
dropped factor, a flipped sign, a transposed index, the paper's literal but
non-Hermitian spherical diagonal, ...), builds it, routes the oracle through
that build and requires that at least one pin of test_oracle_special /
test_oracle_physics fails. Runs on the CPU only; nothing here touches a GPU.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
from oracle import hsref as _hsref

import test_oracle_hpd as Hp
import test_oracle_physics as P
import test_oracle_special as Sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "hsref.c")

MUTATIONS = {
    "paper-literal AB/BA diagonal (1 and 0)": (
        "acc[0][1] += 0.5;\n            acc[1][0] += 0.5;",
        "acc[0][1] += 1.0;\n            acc[1][0] += 0.0;"),
    "BB diagonal without ||u_dot||^2": (
        "acc[1][1] += ty->e_l[l] * ty->udot_norm2[l];", "acc[1][1] += ty->e_l[l];"),
    "sign of u K j' in B": (
        "double fb = -ty->u[l] * kn * djl[l] + ty->du[l] * jl[l];",
        "double fb = ty->u[l] * kn * djl[l] + ty->du[l] * jl[l];"),
    "Y_L instead of Y_L^*": (
        "double complex yc = Y[2 * L] - I * Y[2 * L + 1];", "double complex yc = Y[2 * L] + I * Y[2 * L + 1];"),
    "I indices l and l' swapped": (
        "acc[x][y] += Ixy[x][y][((size_t)l * (lmax + 1) + lp) * n3 + lpp] * g;",
        "acc[x][y] += Ixy[x][y][((size_t)lp * (lmax + 1) + l) * n3 + lpp] * g;"),
    "complex potential coefficients": (
        "static double cpot(int mpp) { return (mpp >= 0) ? 1.0 : ((mpp & 1) ? -1.0 : 1.0); }",
        "static double cpot(int mpp) { (void)mpp; return 1.0; }"),
    "structure phase sign": (
        "double complex phase = cos(kx) + I * sin(kx);", "double complex phase = cos(kx) - I * sin(kx);"),
    "i^l dropped": (
        "double complex il = (l % 4 == 0) ? 1.0 : (l % 4 == 1) ? I : (l % 4 == 2) ? -1.0 : -I;",
        "double complex il = 1.0;"),
    "Condon-Shortley phase dropped": (
        "long double plm = ((m & 1) ? -1.0L : 1.0L) * sm * s / powl(2.0L, l);",
        "long double plm = sm * s / powl(2.0L, l);"),
    "Bessel derivative index": (
        "dj[l] = (double)l / x * jj[l] - jj[l + 1];", "dj[l] = (double)(l + 1) / x * jj[l] - jj[l + 1];"),
    "S without ||u_dot||^2": (
        "ya[nl + L] = ty->udot_norm2[l] * wa[nl + L];", "ya[nl + L] = wa[nl + L];"),
    "T transposed in T w": (
        "for (int c = 0; c < n; ++c) s += T[r + (size_t)c * n] * wa[c];",
        "for (int c = 0; c < n; ++c) s += T[c + (size_t)r * n] * wa[c];"),
    "Gaunt (-1)^{m'} dropped": (
        "double sg = (mp & 1) ? -1.0 : 1.0;\n  return sg * pre * w0 * w;", "return pre * w0 * w;"),
    "1/Omega instead of 1/sqrt(Omega)": (
        "4.0 * M_PI / (W * sqrt(sys->omega))", "4.0 * M_PI / (W * sys->omega)"),
    "Wronskian sign": (
        ": ty->udot[l] * ty->du[l] - ty->u[l] * ty->dudot[l];",
        ": ty->u[l] * ty->dudot[l] - ty->udot[l] * ty->du[l];"),
    "caller's Wronskian ignored": (
        "double W = ty->wronskian ? ty->wronskian[l] :", "double W = 0 ? ty->wronskian[l] :"),
    "whole columns: S column from X": (
        "Sc[e] = cdot(w + (size_t)tp * D, y + (size_t)c * D, D, 0);",
        "Sc[e] = cdot(w + (size_t)tp * D, x + (size_t)c * D, D, 0);"),
    "l_nonsph cutoff on one index only": (
        "lpp <= l + lp && l <= lns && lp <= lns; ++lpp", "lpp <= l + lp && l <= lns; ++lpp"),
    "Cholesky pivot with c^2 instead of |c|^2": (
        "d -= creal(c) * creal(c) + cimag(c) * cimag(c);", "d -= creal(c * c);"),
    "Cholesky conjugate on the wrong factor": (
        "v -= L[i + (size_t)k * n] * conj(L[j + (size_t)k * n]);",
        "v -= conj(L[i + (size_t)k * n]) * L[j + (size_t)k * n];"),
    "Cholesky pivot test admits zero": (
        "if (!(d > 0.0) || !isfinite(d)) {", "if (!(d >= 0.0) || !isfinite(d)) {"),
    "conjugate on the wrong side of the dot": (
        "sr += pr * qr + pi * qi;\n      si += pr * qi - pi * qr;",
        "sr += pr * qr + pi * qi;\n      si += pi * qr - pr * qi;"),
}

PINS = [
    lambda: Sp.test_bessel_closed_forms(),
    lambda: Sp.test_bessel_vs_scipy(),
    lambda: Sp.test_ylm_closed_forms(),
    lambda: Sp.test_gaunt_quadrature(),
    lambda: P.test_rayleigh_matching("small"),
    lambda: P.test_S_legendre_closed_form_c0(),
    lambda: P.test_S_single_plane_wave(),
    lambda: P.test_H_spherical_only_closed_form(),
    lambda: P.test_H_quadrature_form("small"),
    lambda: P.test_H_quadrature_form("small-lns"),
    lambda: P.test_H_rank_one_T(),
    lambda: P.test_hermitian_psd_and_brute_force_c0(),
    lambda: P.test_invariances(),
    lambda: P.test_caller_wronskian(),
    lambda: P.test_whole_columns_match_full_matrix(),
    lambda: Hp.test_factor_of_hpd_matrix(7),
    lambda: Hp.test_special_cases(),
    lambda: [Hp.test_status_is_the_first_indefinite_leading_minor(k) for k in range(6)],
    lambda: Hp.test_energy_shift_adds_sigma_D_and_makes_T_hpd(),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    mut = tmp_path / "hsref_mut.c"
    mut.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(SRC), "hsref.h")
    lib = tmp_path / "libhsref_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-D_GNU_SOURCE",
                    "-I", os.path.dirname(hdr), "-o", str(lib), str(mut), "-lm"], check=True)
    caught = None
    with _hsref.use_library(str(lib)):
        for i, pin in enumerate(PINS):
            try:
                pin()
            except AssertionError:
                caught = i
                break
    assert caught is not None, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_all_pins():
    for pin in PINS:
        pin()
