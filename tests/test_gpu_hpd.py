"""GPU parity of the HPD route of H (Sec. 4.6.2-4.6.3, Listings alg:H_AA_HPD
and alg:H_AA_dynamic), option h_form HSGEN_H_HPD, through the C ABI.

hsgen_set_atoms factors each species' T as C C^H on the device; the status of
that factorization (LAPACK potrf's: 0, or the order of the first leading minor
that is not positive definite) must equal the oracle's, and so must the factor.
A species that passes takes Y_a = C^H W_a and H += Y_a^H Y_a; H is the same
matrix as by X = T W, so the oracle's H (Eq. def_hamilton) is the reference,
with the tolerances of the form that builds it. The stand-in radial data draw
E_l from [-1, 1], which leaves no species' T positive definite; raising every
E_l by 12 (a shift of the energy reference, workloads.shift_energies) makes
the species of the 16- and 64-atom workloads HPD.
"""
import numpy as np
import pytest

import oracle
from workloads import make_config, shift_energies

from test_gpu_split import check as check_split, run_gpu

pytestmark = pytest.mark.gpu

SIGMA = 12.0


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def check_fp64(system, kv, H, S):
    from test_gpu_fp64 import check as check_f

    check_f(system, kv, H, S)


def form_kw(hs, form):
    if form == "fp64":
        return {"precision": hs.FP64}
    return {"precision": hs.SPLIT,
            "scheme": hs.SCHEME_MODULI if form == "moduli" else hs.SCHEME_SLICES, "target_rel_err": 1e-12}


def check(form, system, kv, H, S):
    (check_fp64 if form == "fp64" else check_split)(system, kv, H, S)


@pytest.mark.parametrize("shift", [0.0, SIGMA])
def test_T_factor_matches_the_oracle(hs, shift):
    w = make_config(2, n_g_override=16)
    sysm = shift_energies(w.system, shift) if shift else w.system
    with hs.Generator(sysm, precision=hs.FP64, h_form=hs.H_HPD) as g:
        routed = 0
        for t, ty in enumerate(sysm.types):
            info_o, C_o = oracle.cholesky(oracle.T_matrix(ty))
            info, C = g.T_factor(t)
            assert info == info_o, (t, info, info_o)
            k = C.shape[0] if info == 0 else info - 1
            if k:
                assert np.abs(C[:, :k] - C_o[:, :k]).max() <= 1e-12 * np.abs(C_o).max(), t
            assert np.all(C[:, k:] == 0) and np.all(np.triu(C, 1) == 0)
            routed += info == 0
        assert g.stats()["hpd_species"] == routed
        assert routed == (len(sysm.types) if shift else 0)


def test_T_factor_needs_the_hpd_form(hs):
    w = make_config(0)
    with hs.Generator(w.system, precision=hs.FP64) as g:
        with pytest.raises(hs.HsgenError):
            g.T_factor(0)


@pytest.mark.parametrize("form", ["fp64", "moduli", "slices"])
def test_hpd_route_parity(hs, form):
    """Every species routed: H = sum_a (C^H W_a)^H (C^H W_a), S unchanged."""
    w = make_config(1)
    sysm = shift_energies(w.system, SIGMA)
    kv = w.kvecs[0]
    H, S, st = run_gpu(hs, sysm, kv, h_form=hs.H_HPD, **form_kw(hs, form))
    assert st["hpd_species"] == 2
    check(form, sysm, kv, H, S)


@pytest.mark.parametrize("form", ["fp64", "moduli"])
def test_hpd_route_mixed_species(hs, form):
    """Only species 0 is HPD: its atoms take Y = C^H W, species 1's X = T W;
    the passes over the atoms split where the route changes."""
    w = make_config(1)
    sysm = shift_energies(w.system, SIGMA, types=[0])
    kv = w.kvecs[0]
    H, S, st = run_gpu(hs, sysm, kv, h_form=hs.H_HPD, **form_kw(hs, form))
    assert st["hpd_species"] == 1 and st["atom_chunks"] == 2
    check(form, sysm, kv, H, S)


@pytest.mark.parametrize("form", ["fp64", "moduli", "slices"])
def test_hpd_route_with_legendre_S(hs, form):
    """S in the Legendre form: the contraction builds H only, as Y^H Y (the
    moduli scheme then forms no residues of W)."""
    w = make_config(1)
    sysm = shift_energies(w.system, SIGMA)
    kv = w.kvecs[0]
    H, S, st = run_gpu(hs, sysm, kv, h_form=hs.H_HPD, s_form=hs.S_LEGENDRE, **form_kw(hs, form))
    assert st["hpd_species"] == 2 and st["s_form"] == hs.S_LEGENDRE
    check(form, sysm, kv, H, S)


def test_not_hpd_takes_the_T_route_bit_for_bit(hs):
    """A species whose factorization fails keeps X = T W: the HPD option then
    changes nothing."""
    w = make_config(1)
    kv = w.kvecs[0]
    H0, S0, _ = run_gpu(hs, w.system, kv, scheme=hs.SCHEME_MODULI)
    H1, S1, st = run_gpu(hs, w.system, kv, scheme=hs.SCHEME_MODULI, h_form=hs.H_HPD)
    assert st["hpd_species"] == 0
    assert np.array_equal(H0, H1) and np.array_equal(S0, S1)


def test_hpd_route_batched_equals_sequential(hs):
    """Batched k-points with every species routed: the grouped launch takes
    the same route, bit for bit the k-point-by-k-point result."""
    import torch

    w = make_config(3)
    sysm = shift_energies(w.system, SIGMA)
    with hs.Generator(sysm, precision=hs.SPLIT, h_form=hs.H_HPD) as g:
        assert g.stats()["hpd_species"] == len(sysm.types)
        kvs = [np.ascontiguousarray(k[:700]) for k in w.kvecs[:3]]
        n_gs = [k.shape[0] for k in kvs]
        Hb = [torch.zeros((n, n), dtype=torch.complex128, device="cuda") for n in n_gs]
        Sb = [torch.zeros_like(h) for h in Hb]
        hs.hsgen_build_HS_batched(g.ctx, n_gs, [k.ctypes.data for k in kvs], [h.data_ptr() for h in Hb],
                                  [s.data_ptr() for s in Sb], n_gs, 0)
        torch.cuda.synchronize()
        for k, n in enumerate(n_gs):
            H1, S1 = g.build(torch.from_numpy(kvs[k]).cuda())
            torch.cuda.synchronize()
            assert torch.equal(H1.mT, Hb[k]) and torch.equal(S1.mT, Sb[k]), k
        check_split(sysm, kvs[0], Hb[0].mT.cpu().numpy(), Sb[0].mT.cpu().numpy())
