"""GPU parity of the split-precision form (BF16 products on tcgen05) against
the oracle, through the C ABI, in both of its schemes: slices (Ozaki scheme
I, s(s+1)/2 products of s BF16 slices per operand) and moduli (Ozaki scheme
II, one product per modulus of b-bit integer operands, exact by the Chinese
remainder theorem).

Tolerances (split form): relative Frobenius error <= 1e-11 over
the written triangle and <= 1e-10 per entry relative to ||w_i|| ||x_j||.
Full-size configurations are checked on sampled entries that the oracle
computes one by one, in the launch configuration bench.py times.
"""
import numpy as np
import pytest

import oracle
from workloads import make_config, make_system, kpoint_list

from _parity import compare, normwise_scales, tri_mask

pytestmark = pytest.mark.gpu

REL_F = 1e-11
PER_ENTRY = 1e-10


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def mixed_system(seed=3, lmaxes=(2, 4, 0), counts=(2, 1, 2), cell=10.0):
    lat = np.array([[cell, 0.3, 0.0], [0.0, cell * 1.1, 0.2], [0.1, 0.0, cell * 0.95]])
    species = [(lm, 1.5 + 0.1 * i) for i, lm in enumerate(lmaxes)]
    return make_system(seed, lat, species, list(counts))


SCHEMES = ["slices", "moduli"]


def scheme_kw(hs, scheme):
    return {"scheme": hs.SCHEME_SLICES if scheme == "slices" else hs.SCHEME_MODULI}


def run_gpu(hs, system, kv, **kw):
    import torch

    kw.setdefault("precision", hs.SPLIT)
    with hs.Generator(system, **kw) as g:
        H, S = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        return H.cpu().numpy(), S.cpu().numpy(), g.stats()


def errors(system, kv, H, S, uplo="U", full=False):
    Ho, So = oracle.build_HS(system, kv, full=True)
    wn, xn, yn = normwise_scales(system, kv)
    n = kv.shape[0]
    mask = np.ones((n, n), bool) if full else tri_mask(n, uplo)
    return compare(H, Ho, wn, xn, mask), compare(S, So, wn, yn, mask), mask


def check(system, kv, H, S, uplo="U", full=False):
    (hf, hp), (sf, sp), mask = errors(system, kv, H, S, uplo, full)
    assert hf <= REL_F and hp <= PER_ENTRY, (hf, hp)
    assert sf <= REL_F and sp <= PER_ENTRY, (sf, sp)
    if not full:
        assert np.all(H[~mask] == 0) and np.all(S[~mask] == 0)
    assert np.all(np.diag(H).imag == 0.0) and np.all(np.diag(S).imag == 0.0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_config0(hs, scheme):
    w = make_config(0)
    H, S, st = run_gpu(hs, w.system, w.kvecs[0], **scheme_kw(hs, scheme))
    check(w.system, w.kvecs[0], H, S)
    assert st["precision"] == hs.SPLIT and st["slices"] == 6
    if scheme == "slices":
        assert st["scheme"] == hs.SCHEME_SLICES and st["products"] == 21
    else:
        assert st["scheme"] == hs.SCHEME_MODULI and st["products"] == st["moduli"] and 10 <= st["moduli"] <= 14


def test_default_scheme_is_moduli_when_they_meet_the_target(hs):
    w = make_config(0)
    _, _, st = run_gpu(hs, w.system, w.kvecs[0])
    assert st["scheme"] == hs.SCHEME_MODULI and st["products"] < 21
    _, _, st = run_gpu(hs, w.system, w.kvecs[0], slices=6)  # a slice count forces the slices scheme
    assert st["scheme"] == hs.SCHEME_SLICES
    _, _, st = run_gpu(hs, w.system, w.kvecs[0], target_rel_err=1e-15)  # beyond 14 moduli
    assert st["scheme"] == hs.SCHEME_SLICES and st["slices"] == 7


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n_g", [1, 7, 129, 300])
def test_split_ragged_sizes_mixed_lmax(hs, n_g, scheme):
    sysm = mixed_system()
    kv = kpoint_list(sysm.lattice, (0.13, -0.07, 0.21), n_g)
    H, S, _ = run_gpu(hs, sysm, kv, **scheme_kw(hs, scheme))
    check(sysm, kv, H, S)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_gamma_point(hs, scheme):
    sysm = mixed_system(seed=9)
    kv = kpoint_list(sysm.lattice, (0.0, 0.0, 0.0), 70)
    H, S, _ = run_gpu(hs, sysm, kv, **scheme_kw(hs, scheme))
    check(sysm, kv, H, S)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_lower_full_and_chunked(hs, scheme):
    sysm = mixed_system(seed=11, counts=(3, 2, 2))
    kv = kpoint_list(sysm.lattice, (0.2, 0.1, -0.3), 250)
    kw = scheme_kw(hs, scheme)
    H, S, _ = run_gpu(hs, sysm, kv, uplo="L", **kw)
    check(sysm, kv, H, S, uplo="L")
    H, S, _ = run_gpu(hs, sysm, kv, fill_full=True, **kw)
    check(sysm, kv, H, S, full=True)
    H, S, st = run_gpu(hs, sysm, kv, atom_chunk=3, **kw)
    assert st["atom_chunks"] == 3
    check(sysm, kv, H, S)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_host_pointers(hs, scheme):
    sysm = mixed_system(seed=13)
    kv = np.ascontiguousarray(kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 90))
    n = kv.shape[0]
    H = np.zeros((n, n), np.complex128)
    S = np.zeros((n, n), np.complex128)
    with hs.Generator(sysm, precision=hs.SPLIT, **scheme_kw(hs, scheme)) as g:
        hs.hsgen_build_HS(g.ctx, n, kv.ctypes.data, H.ctypes.data, S.ctypes.data, n, 0)
    check(sysm, kv, H.T, S.T)


def test_moduli_error_follows_the_bits(hs):
    """Moduli form: the integer product is exact, so the error is that of
    rounding the operands' columns to integers of 2-norm at most 2^B: it
    falls by about 2^-(added bits) (B = 39, 43, 46 for 10, 11, 12 moduli; 47,
    the cap, from 13 on, where X = T W's own rounding, about 1e-13, takes
    over) and stays below the library's a-priori model 3 sqrt(2K) 2^-B,
    which chooses the count."""
    w = make_config(0)
    kv = w.kvecs[0]
    depth = sum(2 * w.system.types[t].nl for t in w.system.type_of_atom)
    errs = []
    for n in (10, 11, 12, 13, 14):
        H, S, st = run_gpu(hs, w.system, kv, scheme=hs.SCHEME_MODULI, moduli=n)
        assert st["moduli"] == n and st["products"] == n
        (hf, _), (sf, _), _ = errors(w.system, kv, H, S)
        err = max(hf, sf)
        assert err <= 3.0 * np.sqrt(2 * depth) * 2.0 ** -st["bits"] + 2e-13, (n, st["bits"], err)
        errs.append((st["bits"], err))
    assert [b for b, _ in errs] == [39, 43, 46, 47, 47], errs
    assert errs[1][1] < errs[0][1] / 8, errs  # 39 -> 43 bits
    assert max(e for _, e in errs[2:]) < 3e-13, errs  # the floor of X = T W


def test_moduli_stage_geometries_and_unit_orders_agree_bitwise(hs, monkeypatch):
    """The moduli kernel's two stage geometries (3 stages of 2 k-blocks with
    chunks of 8, 2 stages of 3 with chunks of 6), its two orders of
    (tile, modulus) units and its L2 priorities sum the same exact integers,
    and the reconstruction inside the contraction or in a kernel of its own
    is the same arithmetic, so H and S agree bit for bit."""
    w = make_config(1)
    out = []
    for geom, order, hint, recon in (("0", "0", "0", "1"), ("1", "0", "8", "0"), ("0", "1", "0", "0"),
                                     ("1", "1", "8", "1")):
        monkeypatch.setenv("HSGEN_CRT_GEOMETRY", geom)
        monkeypatch.setenv("HSGEN_CRT_ORDER", order)
        monkeypatch.setenv("HSGEN_L2_HINT", hint)
        monkeypatch.setenv("HSGEN_CRT_RECON", recon)
        H, S, st = run_gpu(hs, w.system, w.kvecs[0], scheme=hs.SCHEME_MODULI)
        assert st["stage_geometry"] == int(geom) and st["unit_order"] == int(order) and st["l2_hint"] == int(hint)
        out.append((H, S))
    for H, S in out[1:]:
        assert np.array_equal(out[0][0], H) and np.array_equal(out[0][1], S)
    check(w.system, w.kvecs[0], *out[-1])


@pytest.mark.parametrize("order", ["0", "1"])
def test_moduli_across_many_depth_segments(hs, monkeypatch, order):
    """One depth segment of 64 rows per launch (41 launches at 16 atoms /
    N_G 3000): the residues of every segment add up modulo each m_i in the
    residue store, and only the last launch writes H and S."""
    monkeypatch.setenv("HSGEN_KSEG_BLOCKS", "1")
    monkeypatch.setenv("HSGEN_CRT_ORDER", order)
    w = make_config(1)
    H, S, st = run_gpu(hs, w.system, w.kvecs[0], scheme=hs.SCHEME_MODULI)
    assert st["kseg_blocks"] == 1 and st["scheme"] == hs.SCHEME_MODULI and st["unit_order"] == int(order)
    check(w.system, w.kvecs[0], H, S)


@pytest.mark.parametrize("uplo,s_form,chunk", [("U", "S_CONTRACTION", 0), ("L", "S_CONTRACTION", 0),
                                              ("U", "S_LEGENDRE", 0), ("L", "S_LEGENDRE", 0),
                                              ("U", "S_CONTRACTION", 40)])
def test_pinned_host_outputs_match_device(hs, uplo, s_form, chunk):
    """Pinned host outputs: the H/S launches run group by group of column
    bands and each group's finished columns are copied to the host while later
    groups compute (several groups at N_G 6000; S in the Legendre form in
    column groups of its own kernel for the upper triangle). The host result
    equals the build into device buffers bit for bit, and the other triangle
    is overwritten with zeros."""
    import torch

    w = make_config(2, n_g_override=6000)
    kv = np.ascontiguousarray(w.kvecs[0])
    n = kv.shape[0]
    with hs.Generator(w.system, precision=hs.SPLIT, uplo=uplo, s_form=getattr(hs, s_form), atom_chunk=chunk) as g:
        Hd, Sd = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        Hd, Sd = Hd.mT.cpu(), Sd.mT.cpu()  # the raw column-major buffers
        kh = torch.from_numpy(kv.copy()).pin_memory()
        Hh = torch.full((n, n), complex(7.0, -7.0), dtype=torch.complex128).pin_memory()
        Sh = torch.full((n, n), complex(-3.0, 3.0), dtype=torch.complex128).pin_memory()
        for _ in range(2):
            hs.hsgen_build_HS(g.ctx, n, kh.data_ptr(), Hh.data_ptr(), Sh.data_ptr(), n, 0)
            assert torch.equal(Hh, Hd) and torch.equal(Sh, Sd)
            Hh.fill_(complex(1.0, 1.0))
            Sh.fill_(complex(1.0, 1.0))
    # and the device build itself against the oracle on sampled entries
    idx = np.unique(np.r_[0, np.sort(np.random.default_rng(5).choice(n, 12, replace=False)), n - 1])
    r, c = np.meshgrid(idx, idx, indexing="ij")
    sel = (r <= c) if uplo == "U" else (r >= c)
    Ho, So = oracle.HS_entries(w.system, kv, r[sel], c[sel])
    Hg = Hd.numpy().T[r[sel], c[sel]]  # H(i, j) sits at buffer[j, i]
    Sg = Sd.numpy().T[r[sel], c[sel]]
    assert np.linalg.norm(Hg - Ho) <= REL_F * np.linalg.norm(Ho)
    assert np.linalg.norm(Sg - So) <= REL_F * np.linalg.norm(So)


def test_two_uneven_passes_host_and_device(hs, monkeypatch):
    """A workspace budget that holds about 60 % of the atoms: the library
    makes two passes, the last as large as the budget allows (the first
    takes the rest), and pinned host outputs leave the device during the last
    pass. Host and device outputs agree bit for bit and match the oracle."""
    import torch

    w = make_config(2, n_g_override=3000)
    kv = np.ascontiguousarray(w.kvecs[0])
    n = kv.shape[0]
    monkeypatch.setenv("HSGEN_WS_BYTES", "6e9")
    with hs.Generator(w.system, precision=hs.SPLIT, scheme=hs.SCHEME_MODULI, target_rel_err=1e-11) as g:
        Hd, Sd = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        st = g.stats()
        assert st["atom_chunks"] == 2, st["atom_chunks"]
        Hd, Sd = Hd.mT.cpu(), Sd.mT.cpu()
        kh = torch.from_numpy(kv.copy()).pin_memory()
        Hh = torch.full((n, n), complex(7.0, -7.0), dtype=torch.complex128).pin_memory()
        Sh = torch.full((n, n), complex(-3.0, 3.0), dtype=torch.complex128).pin_memory()
        hs.hsgen_build_HS(g.ctx, n, kh.data_ptr(), Hh.data_ptr(), Sh.data_ptr(), n, 0)
        assert torch.equal(Hh, Hd) and torch.equal(Sh, Sd)
    check(w.system, kv, Hd.numpy().T, Sd.numpy().T)


def test_split_error_falls_with_slices(hs):
    """About 8 bits per slice; 7 slices reach FP64-level agreement, which also
    shows that every FP32 tensor-core chunk accumulated exactly."""
    w = make_config(0)
    kv = w.kvecs[0]
    errs = []
    for s in (3, 4, 5, 6, 7):
        H, S, st = run_gpu(hs, w.system, kv, slices=s)
        assert st["slices"] == s
        (hf, _), (sf, _), _ = errors(w.system, kv, H, S)
        errs.append(max(hf, sf))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 50, errs
    assert errs[-1] < 2e-14, errs


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_complex_T_override(hs, scheme):
    """A genuinely complex Hermitian T exercises the imaginary half of X = T W."""
    sysm = mixed_system(seed=21)
    rng = np.random.default_rng(3)
    for ty in sysm.types:
        n = 2 * ty.nl
        A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        ty.T_override = 0.5 * (A + A.conj().T)
    kv = kpoint_list(sysm.lattice, (0.1, 0.0, 0.2), 140)
    H, S, _ = run_gpu(hs, sysm, kv, **scheme_kw(hs, scheme))
    check(sysm, kv, H, S)


@pytest.mark.parametrize("n_moduli", [10, 14])
def test_moduli_at_the_cauchy_schwarz_bound(hs, n_moduli):
    """The moduli form's integer product is exact because every operand
    column is rounded to integers of 2-norm <= 2^B with 2^(2B+1) < M, and
    |P'^H Q'| <= ||P'|| ||Q'|| (Cauchy-Schwarz). With T = 1 the diagonal of
    H = W^H W reaches that bound (H_jj = ||w_j||^2, both factors the same
    column), so a bound one bit too loose would wrap H's diagonal modulo M;
    S = W^H U W has its diagonal near it as well."""
    w = make_config(1)
    sysm = w.system
    for ty in sysm.types:
        ty.T_override = np.eye(2 * ty.nl, dtype=complex)
    kv = w.kvecs[0][:1500]
    H, S, st = run_gpu(hs, sysm, kv, scheme=hs.SCHEME_MODULI, moduli=n_moduli)
    assert st["moduli"] == n_moduli
    Ho, So = oracle.build_HS(sysm, kv, full=True)
    d, do = np.diag(H).real, np.diag(Ho).real
    assert np.all(do > 0)
    assert np.max(np.abs(d - do) / do) <= 1e-9, np.max(np.abs(d - do) / do)  # a wrap would be off by ~M
    # the rounding error itself, within the a-priori model 3 sqrt(2K) 2^-B
    depth = sum(2 * sysm.types[t].nl for t in sysm.type_of_atom)
    (hf, _), (sf, _), _ = errors(sysm, kv, H, S)
    assert max(hf, sf) <= 3.0 * np.sqrt(2 * depth) * 2.0 ** -st["bits"] + 2e-13, (hf, sf, st["bits"])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_config1(hs, scheme):
    w = make_config(1)
    H, S, _ = run_gpu(hs, w.system, w.kvecs[0], **scheme_kw(hs, scheme))
    check(w.system, w.kvecs[0], H, S)


def test_split_matches_fp64_form(hs):
    sysm = mixed_system(seed=25, counts=(4, 3, 2))
    kv = kpoint_list(sysm.lattice, (0.31, 0.1, 0.05), 400)
    Hs, Ss, _ = run_gpu(hs, sysm, kv)
    Hd, Sd, _ = run_gpu(hs, sysm, kv, precision=hs.FP64)
    m = tri_mask(400)
    assert np.linalg.norm((Hs - Hd)[m]) <= 1e-11 * np.linalg.norm(Hd[m])
    assert np.linalg.norm((Ss - Sd)[m]) <= 1e-11 * np.linalg.norm(Sd[m])


def sampled_check(hs, cfg, kidx=0, n_samp=14, seed=0, **kw):
    import torch

    w = make_config(cfg)
    kv = w.kvecs[kidx]
    n = kv.shape[0]
    with hs.Generator(w.system, precision=hs.SPLIT, **kw) as g:
        H, S = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(n, n_samp, replace=False))
        idx[0], idx[-1] = 0, n - 1  # first and last column (ragged tail)
        idx = np.unique(idx)
        r, c = np.meshgrid(idx, idx, indexing="ij")
        sel = r <= c
        ti = torch.from_numpy(r[sel]).cuda(), torch.from_numpy(c[sel]).cuda()
        Hg = H[ti].cpu().numpy()
        Sg = S[ti].cpu().numpy()
    Ho, So = oracle.HS_entries(w.system, kv, r[sel], c[sel])
    # normwise per-entry scale from the oracle's columns of W, X, U W
    import _parity

    Wc, Xc, Yc = _parity.oracle_columns(w.system, kv[idx])
    pos = {v: i for i, v in enumerate(idx)}
    ri = np.array([pos[v] for v in r[sel]])
    ci = np.array([pos[v] for v in c[sel]])
    wn, xn, yn = (np.linalg.norm(M, axis=0) for M in (Wc, Xc, Yc))
    rel_h = np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho)
    rel_s = np.linalg.norm(Sg - So) / np.linalg.norm(So)
    per_h = np.max(np.abs(Hg - Ho) / (wn[ri] * xn[ci]))
    per_s = np.max(np.abs(Sg - So) / (wn[ri] * yn[ci]))
    assert rel_h <= REL_F and rel_s <= REL_F, (rel_h, rel_s)
    assert per_h <= PER_ENTRY and per_s <= PER_ENTRY, (per_h, per_s)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_split_config2_sampled(hs, scheme):
    sampled_check(hs, 2, **scheme_kw(hs, scheme))


def test_split_config3_one_kpoint_sampled(hs):
    sampled_check(hs, 3, kidx=5)


def test_split_autotune_choice_and_parity(hs):
    """The autotuner picks a candidate schedule, keeps it for later builds and
    its output is a correct H and S."""
    import torch

    w = make_config(2, n_g_override=3000)
    kv = w.kvecs[0]
    kd = torch.from_numpy(kv).cuda()
    with hs.Generator(w.system, precision=hs.SPLIT) as g:
        H, S = g.autotune(kd)
        torch.cuda.synchronize()
        st = g.stats()
        assert st["kseg_blocks"] in (16, 24, 32, 48, 64, 96, 128, 192, 256) and st["tile_band"] in (8, 16, 32)
        assert st["unit_order"] in (0, 1)
        H2, S2 = g.build(kd)
        torch.cuda.synchronize()
        assert torch.equal(H, H2) and torch.equal(S, S2)
        assert g.stats()["kseg_blocks"] == st["kseg_blocks"]
    check(w.system, kv, H.cpu().numpy(), S.cpu().numpy())


@pytest.mark.parametrize("target", [1e-11, 1e-14])
def test_autotune_picks_the_form_by_measured_error(hs, target):
    """The autotuner measures candidate forms against a 7-slice build over
    the whole triangle, takes each scheme's smallest count within half the
    target and keeps the faster of the two; only 7 slices reach 1e-14 (the
    moduli form stops near 1e-13, where X = T W's own rounding lies)."""
    import torch

    w = make_config(2, n_g_override=1200)
    kd = torch.from_numpy(w.kvecs[0]).cuda()
    with hs.Generator(w.system, precision=hs.SPLIT, target_rel_err=target) as g:
        H, S = g.autotune(kd)
        g.synchronize()
        st = g.stats()
        H2, S2 = g.build(kd)  # the choice stays in the context
        g.synchronize()
        assert torch.equal(H, H2) and torch.equal(S, S2)
        st2 = g.stats()
    assert st2["scheme"] == st["scheme"] and st2["products"] == st["products"]
    # (7 slices are the reference itself: measured 0)
    assert 0.0 <= st["tuned_rel_err"] <= 0.5 * target and (st["tuned_rel_err"] > 0.0) == (target == 1e-11)
    if target == 1e-11:
        assert (st["scheme"] == hs.SCHEME_MODULI and st["products"] <= 13) or \
            (st["scheme"] == hs.SCHEME_SLICES and st["slices"] <= 6)
    else:
        assert st["scheme"] == hs.SCHEME_SLICES and st["slices"] == 7
    # the measured figure is the real error (to the reference's ~1e-15)
    (hf, _), (sf, _), _ = errors(w.system, w.kvecs[0], H.cpu().numpy(), S.cpu().numpy())
    assert max(hf, sf) <= 2.0 * st["tuned_rel_err"] + 1e-13


def test_split_timeout_is_reported_and_context_recovers(hs):
    """A wait limit far below the kernel's latency makes bounded device waits
    expire. The build returns without waiting for the device (device buffers),
    so the expiry is reported afterwards by hsgen_synchronize as
    HSGEN_ETIMEOUT (no trap), once; the GPU and the context stay usable."""
    import torch

    w = make_config(1)
    kv = torch.from_numpy(w.kvecs[0]).cuda()
    with hs.Generator(w.system, precision=hs.SPLIT, wait_timeout_ns=1) as g:
        g.build(kv)
        with pytest.raises(hs.HsgenError) as ei:
            g.synchronize()
        assert ei.value.status == hs.ETIMEOUT
        g.synchronize()  # reported once, then cleared
        # the next call finds an expiry of an earlier call whose work has finished
        g.build(kv)
        torch.cuda.synchronize()
        with pytest.raises(hs.HsgenError) as ei:
            g.build(kv)
        assert ei.value.status == hs.ETIMEOUT
        torch.cuda.synchronize()
    H, S, _ = run_gpu(hs, w.system, w.kvecs[0])
    check(w.system, w.kvecs[0], H, S)


def test_split_build_returns_before_the_device_finishes(hs):
    """With device buffers the split build is asynchronous on its stream: the
    host gets control back while the kernels still run (64 atoms, N_G 12000:
    about 0.2 s of device work)."""
    import torch

    w = make_config(2)
    kv = torch.from_numpy(w.kvecs[0]).cuda()
    n = kv.shape[0]
    H = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    S = torch.zeros_like(H)
    stream = torch.cuda.current_stream()
    with hs.Generator(w.system, precision=hs.SPLIT) as g:
        g.build(kv, H, S)  # sets up the workspaces
        g.synchronize()
        hs.hsgen_build_HS(g.ctx, n, kv.data_ptr(), H.data_ptr(), S.data_ptr(), n, stream.cuda_stream)
        done = torch.cuda.Event()
        done.record(stream)
        assert not done.query(), "the build waited for the device"
        g.synchronize()
        assert done.query()


def test_allocation_failure_is_reported_and_context_recovers(hs, monkeypatch):
    """Fault injection on the host: with HSGEN_FAIL_ALLOC=1 the workspace
    allocation fails as an out-of-memory cudaMalloc would; the call returns
    HSGEN_ENOMEM and, with the variable unset, the same context builds a
    correct H and S."""
    import torch

    sysm = mixed_system(seed=29)
    kv = kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 120)
    with hs.Generator(sysm, precision=hs.SPLIT) as g:
        monkeypatch.setenv("HSGEN_FAIL_ALLOC", "1")
        with pytest.raises(hs.HsgenError) as ei:
            g.build(torch.from_numpy(kv).cuda())
        assert ei.value.status == hs.ENOMEM
        monkeypatch.delenv("HSGEN_FAIL_ALLOC")
        H, S = g.build(torch.from_numpy(kv).cuda())
        g.synchronize()
        H, S = H.cpu().numpy(), S.cpu().numpy()
    check(sysm, kv, H, S)
