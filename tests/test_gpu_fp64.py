"""GPU parity of the FP64 form against the oracle, through the C ABI.

Tolerances (FP64 form): relative Frobenius error <= 1e-12 over the
written triangle, and per entry |dH_ij| <= 1e-10 ||w_i|| ||x_j|| (the
Cauchy-Schwarz scale of a dot product; S uses ||y_j||).
"""
import copy

import numpy as np
import pytest

import oracle
from workloads import make_config, make_system, kpoint_list

from _parity import compare, normwise_scales, tri_mask

pytestmark = pytest.mark.gpu

REL_F = 1e-12
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


def run_gpu(hs, system, kv, **kw):
    import torch

    with hs.Generator(system, **kw) as g:
        H, S = g.build(torch.from_numpy(kv).cuda())
        torch.cuda.synchronize()
        return H.cpu().numpy(), S.cpu().numpy(), g.stats()


def check(system, kv, H, S, uplo="U", full=False, rel_f=REL_F, per=PER_ENTRY):
    Ho, So = oracle.build_HS(system, kv, full=True)
    wn, xn, yn = normwise_scales(system, kv)
    n = kv.shape[0]
    mask = np.ones((n, n), bool) if full else tri_mask(n, uplo)
    for A, B, sc, name in ((H, Ho, xn, "H"), (S, So, yn, "S")):
        rf, pe = compare(A, B, wn, sc, mask)
        assert rf <= rel_f, f"{name}: relative Frobenius {rf:.3e}"
        assert pe <= per, f"{name}: per-entry {pe:.3e}"
        if not full:
            assert np.all(A[~mask] == 0), f"{name}: other triangle written"
        assert np.all(np.diag(A).imag == 0.0)


def test_T_matrix_vs_oracle(hs):
    for lm in range(0, 11):
        sysm = make_system(100 + lm, np.eye(3) * 9.0, [(lm, 1.7)], [1])
        with hs.Generator(sysm) as g:
            Tg = g.T_matrix(0)
        To = oracle.T_matrix(sysm.types[0])
        assert np.max(np.abs(Tg - To)) <= 1e-14 * max(1.0, np.max(np.abs(To))), lm


def test_coefficients_vs_oracle(hs):
    import torch

    for sysm, kv in ((make_config(0).system, make_config(0).kvecs[0]),
                     (mixed_system(), kpoint_list(mixed_system().lattice, (0.0, 0.0, 0.0), 129))):
        with hs.Generator(sysm) as g:
            Wg = g.coefficients(torch.from_numpy(kv).cuda()).cpu().numpy()
            off = g.depth_offsets
        for a in range(sysm.n_atoms):
            Wo = oracle.coefficients(sysm, a, kv)
            blk = Wg[off[a]:off[a] + Wo.shape[0]]
            assert np.max(np.abs(blk - Wo)) <= 2e-14 * np.max(np.abs(Wo)), a
            assert np.all(Wg[off[a] + Wo.shape[0]:off[a + 1]] == 0)


def test_fp64_config0(hs):
    w = make_config(0)
    H, S, st = run_gpu(hs, w.system, w.kvecs[0])
    check(w.system, w.kvecs[0], H, S)
    assert st["precision"] == hs.FP64 and st["flops_algorithmic"] > 0


@pytest.mark.parametrize("n_g", [1, 7, 129])
def test_fp64_ragged_sizes_mixed_lmax(hs, n_g):
    sysm = mixed_system()
    kv = kpoint_list(sysm.lattice, (0.13, -0.07, 0.21), n_g)
    H, S, _ = run_gpu(hs, sysm, kv)
    check(sysm, kv, H, S)


def test_fp64_gamma_point(hs):
    sysm = mixed_system(seed=9)
    kv = kpoint_list(sysm.lattice, (0.0, 0.0, 0.0), 70)
    assert np.linalg.norm(kv[0]) == 0.0
    H, S, _ = run_gpu(hs, sysm, kv)
    check(sysm, kv, H, S)


def test_fp64_lower_full_and_chunked(hs):
    sysm = mixed_system(seed=11, counts=(3, 2, 2))
    kv = kpoint_list(sysm.lattice, (0.2, 0.1, -0.3), 150)
    H, S, _ = run_gpu(hs, sysm, kv, uplo="L")
    check(sysm, kv, H, S, uplo="L")
    H, S, _ = run_gpu(hs, sysm, kv, fill_full=True)
    check(sysm, kv, H, S, full=True)
    Hc, Sc, _ = run_gpu(hs, sysm, kv, atom_chunk=3)
    check(sysm, kv, Hc, Sc)


def test_fp64_host_pointers(hs):
    sysm = mixed_system(seed=13)
    kv = np.ascontiguousarray(kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 90))
    n = kv.shape[0]
    H = np.zeros((n, n), np.complex128)
    S = np.zeros((n, n), np.complex128)
    with hs.Generator(sysm) as g:
        hs.hsgen_build_HS(g.ctx, n, kv.ctypes.data, H.ctypes.data, S.ctypes.data, n, 0)
    check(sysm, kv, H.T, S.T)


def test_fp64_T_override_reduces_to_S(hs):
    sysm = mixed_system(seed=17)
    for ty in sysm.types:
        lvec = np.repeat(np.arange(ty.lmax + 1), 2 * np.arange(ty.lmax + 1) + 1)
        T = np.zeros((2 * ty.nl, 2 * ty.nl), complex)
        T[:ty.nl, :ty.nl] = np.eye(ty.nl)
        T[ty.nl:, ty.nl:] = np.diag(ty.udot_norm2[lvec])
        ty.T_override = T
    kv = kpoint_list(sysm.lattice, (0.1, 0.0, 0.2), 80)
    H, S, _ = run_gpu(hs, sysm, kv)
    m = tri_mask(80)
    assert np.max(np.abs(H - S)[m]) <= 1e-14 * np.max(np.abs(S))


def test_fp64_config1(hs):
    w = make_config(1)
    H, S, _ = run_gpu(hs, w.system, w.kvecs[0])
    check(w.system, w.kvecs[0], H, S)


def test_fp64_zero_plane_waves(hs):
    sysm = mixed_system()
    with hs.Generator(sysm) as g:
        hs.hsgen_build_HS(g.ctx, 0, 0, 0, 0, 1, 0)


def test_fp64_invalid_arguments(hs):
    import torch

    sysm = mixed_system()
    kv = torch.from_numpy(kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 10)).cuda()
    H = torch.zeros((10, 10), dtype=torch.complex128, device="cuda")
    S = torch.zeros_like(H)
    with hs.Generator(sysm) as g:
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_build_HS(g.ctx, 10, kv.data_ptr(), H.data_ptr(), S.data_ptr(), 5, 0)
        assert ei.value.status == hs.EINVAL
        with pytest.raises(hs.HsgenError) as ei:
            hs.hsgen_build_HS(g.ctx, 10, kv.data_ptr(), H.data_ptr(), H.data_ptr(), 10, 0)
        assert ei.value.status == hs.EINVAL
    bad = copy.deepcopy(sysm)
    bad.types[0].udot = bad.types[0].u * bad.types[0].dudot / bad.types[0].du  # W_l = 0
    with pytest.raises(hs.HsgenError) as ei:
        hs.Generator(bad)
    assert ei.value.status == hs.ENUMERIC
    bad2 = copy.deepcopy(sysm)
    bad2.types[0].lmax = 11
    with pytest.raises(hs.HsgenError) as ei:
        hs.Generator(bad2)
    assert ei.value.status == hs.EINVAL
