"""GPU parity with l_nonsph < l_max (Sec. 3.1, Fig. Tmat_structure): the Gaunt
part of T is dense for l, l' <= l_nonsph only, the spherical diagonal runs to
l_max. With S in the Legendre form the contraction covers the rows
l <= l_nonsph and H's spherical tail comes from the Legendre kernel; with the
S contraction the whole T (with that structure) is contracted. Both are
compared with the oracle, which builds T with the same cutoff.
"""
import numpy as np
import pytest

import oracle
from workloads import make_config, make_system, kpoint_list

from _parity import compare, normwise_scales, tri_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def nonsph_system(seed=5, lmaxes=(4, 3, 2), lns=(2, 1, 0), counts=(2, 2, 1), cell=10.0):
    lat = np.array([[cell, 0.2, 0.0], [0.0, cell * 1.05, 0.3], [0.2, 0.0, cell * 0.9]])
    sysm = make_system(seed, lat, [(lm, 1.5 + 0.1 * i) for i, lm in enumerate(lmaxes)], list(counts))
    for ty, l in zip(sysm.types, lns):
        ty.lmax_nonsph = l
    return sysm


def build(hs, system, kv, **kw):
    import torch

    with hs.Generator(system, **kw) as g:
        H, S = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        return H.cpu().numpy(), S.cpu().numpy(), g.stats(), g.depth_offsets


def check(system, kv, H, S, tol_h, tol_s=1e-12):
    Ho, So = oracle.build_HS(system, kv, full=True)
    wn, xn, yn = normwise_scales(system, kv)
    m = tri_mask(kv.shape[0])
    hf, hp = compare(H, Ho, wn, xn, m)
    sf, sp = compare(S, So, wn, yn, m)
    assert hf <= tol_h and hp <= 1e-10, (hf, hp)
    assert sf <= tol_s and sp <= 1e-10, (sf, sp)
    assert np.all(H[~m] == 0) and np.all(S[~m] == 0)


@pytest.mark.parametrize("precision,tol_h", [("SPLIT", 1e-11), ("FP64", 1e-12)])
def test_nonsph_legendre_tail(hs, precision, tol_h):
    sysm = nonsph_system()
    kv = kpoint_list(sysm.lattice, (0.11, -0.05, 0.17), 260)
    H, S, st, off = build(hs, sysm, kv, precision=getattr(hs, precision), s_form=hs.S_LEGENDRE)
    assert st["s_form"] == hs.S_LEGENDRE
    # the contraction covers l <= l_nonsph only
    rows = np.diff(off)
    want = [2 * (sysm.types[t].lmax_nonsph + 1) ** 2 for t in sysm.type_of_atom]
    if precision == "SPLIT":
        assert list(rows) == want
    else:
        assert all(r >= w_ and r < w_ + 8 for r, w_ in zip(rows, want))
    check(sysm, kv, H, S, tol_h)


@pytest.mark.parametrize("precision,tol_h", [("SPLIT", 1e-11), ("FP64", 1e-12)])
def test_nonsph_full_contraction(hs, precision, tol_h):
    """S contraction: T with the l_nonsph structure, contracted over all rows."""
    sysm = nonsph_system(seed=7)
    kv = kpoint_list(sysm.lattice, (0.2, 0.1, -0.1), 200)
    H, S, st, _ = build(hs, sysm, kv, precision=getattr(hs, precision))
    assert st["s_form"] == hs.S_CONTRACTION
    check(sysm, kv, H, S, tol_h, tol_s=1e-11 if precision == "SPLIT" else 1e-12)


@pytest.mark.parametrize("s_form", ["S_CONTRACTION", "S_LEGENDRE"])
def test_nonsph_T_matrix(hs, s_form):
    sysm = nonsph_system(seed=9)
    with hs.Generator(sysm, precision=hs.SPLIT, s_form=getattr(hs, s_form)) as g:
        for t, ty in enumerate(sysm.types):
            Tg = g.T_matrix(t)
            To = oracle.T_matrix(ty)
            assert np.max(np.abs(Tg - To)) <= 1e-14 * np.max(np.abs(To))


def test_nonsph_gamma_and_lower(hs):
    sysm = nonsph_system(seed=11, counts=(1, 2, 2))
    kv = kpoint_list(sysm.lattice, (0.0, 0.0, 0.0), 150)
    H, S, _, _ = build(hs, sysm, kv, precision=hs.SPLIT, s_form=hs.S_LEGENDRE, uplo="L")
    Ho, So = oracle.build_HS(sysm, kv, full=True)
    wn, xn, yn = normwise_scales(sysm, kv)
    m = tri_mask(kv.shape[0], "L")
    assert compare(H, Ho, wn, xn, m)[0] <= 1e-11
    assert compare(S, So, wn, yn, m)[0] <= 1e-12


def test_nonsph_off_lattice_is_refused(hs):
    import torch

    sysm = nonsph_system(seed=13)
    kv = kpoint_list(sysm.lattice, (0.1, 0.0, 0.2), 80).copy()
    kv[3] += np.array([0.0, 2e-3, 0.0])
    with hs.Generator(sysm, precision=hs.SPLIT, s_form=hs.S_LEGENDRE) as g:
        with pytest.raises(hs.HsgenError) as ei:
            g.build(torch.from_numpy(kv).cuda())
        assert ei.value.status == hs.ENOTSUP


def test_nonsph_batched_graph_matches_single(hs):
    import torch

    w = make_config(3)
    sysm = w.system
    for ty in sysm.types:
        ty.lmax_nonsph = max(0, ty.lmax - 3)
    ks = [np.ascontiguousarray(w.kvecs[i]) for i in (2, 9, 30)]
    with hs.Generator(sysm, precision=hs.SPLIT, s_form=hs.S_LEGENDRE) as g:
        singles = [tuple(x.clone() for x in g.build(torch.from_numpy(k).cuda())) for k in ks]
        Hs = [torch.zeros((k.shape[0],) * 2, dtype=torch.complex128, device="cuda") for k in ks]
        Ss = [torch.zeros_like(h) for h in Hs]
        hs.hsgen_build_HS_batched(g.ctx, [k.shape[0] for k in ks], [k.ctypes.data for k in ks],
                                  [h.data_ptr() for h in Hs], [s.data_ptr() for s in Ss], [k.shape[0] for k in ks])
        torch.cuda.synchronize()
        for (H1, S1), H2, S2 in zip(singles, Hs, Ss):
            assert torch.equal(H1, H2.mT) and torch.equal(S1, S2.mT)
    # one k-point against the oracle (sampled)
    kv = ks[0]
    n = kv.shape[0]
    idx = np.unique(np.r_[0, np.sort(np.random.default_rng(1).choice(n, 10, replace=False)), n - 1])
    r, c = np.meshgrid(idx, idx, indexing="ij")
    sel = r <= c
    H1, S1 = singles[0]
    Hg = H1[torch.from_numpy(r[sel]).cuda(), torch.from_numpy(c[sel]).cuda()].cpu().numpy()
    Sg = S1[torch.from_numpy(r[sel]).cuda(), torch.from_numpy(c[sel]).cuda()].cpu().numpy()
    Ho, So = oracle.HS_entries(sysm, kv, r[sel], c[sel])
    assert np.linalg.norm(Hg - Ho) <= 1e-11 * np.linalg.norm(Ho)
    assert np.linalg.norm(Sg - So) <= 1e-12 * np.linalg.norm(So)
