"""Many k-points in one call (one H, S per k-point, Sec. 2.3), through
hsgen_build_HS_batched: uneven N_G and mixed l_max in one grouped launch,
captured as a CUDA graph. The batched result must equal the k-point-by-k-point
result bit for bit (same slices, same tile schedule), match the oracle on
sampled entries, and a replay of the captured graph must reproduce it."""
import numpy as np
import pytest

import oracle
from workloads import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def alloc(n_gs, pad=0):
    import torch

    Hs = [torch.zeros((n, n + pad), dtype=torch.complex128, device="cuda") for n in n_gs]
    Ss = [torch.zeros_like(h) for h in Hs]
    return Hs, Ss


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_batched_equals_sequential(hs, precision):
    import torch

    w = make_config(3)
    kvs = w.kvecs[:6]
    n_gs = [k.shape[0] for k in kvs]
    prec = hs.SPLIT if precision == "split" else hs.FP64
    kv_host = [np.ascontiguousarray(k) for k in kvs]
    with hs.Generator(w.system, precision=prec) as g:
        Hb, Sb = alloc(n_gs, pad=3)  # ld = n_g + 3
        hs.hsgen_build_HS_batched(g.ctx, n_gs, [k.ctypes.data for k in kv_host], [h.data_ptr() for h in Hb],
                                  [s.data_ptr() for s in Sb], [n + 3 for n in n_gs], 0)
        torch.cuda.synchronize()
        st = g.stats()
        assert st["n_kpoints"] == 6
        for k, n in enumerate(n_gs):
            H1 = torch.zeros((n, n + 3), dtype=torch.complex128, device="cuda")
            S1 = torch.zeros_like(H1)
            hs.hsgen_build_HS(g.ctx, n, torch.from_numpy(kv_host[k]).cuda().data_ptr(), H1.data_ptr(),
                              S1.data_ptr(), n + 3, 0)
            torch.cuda.synchronize()
            assert torch.equal(H1, Hb[k]) and torch.equal(S1, Sb[k]), k
        if prec == hs.SPLIT:
            # replay of the captured graph (same sizes and pointers) gives the same result
            Hc = [h.clone() for h in Hb]
            for h in Hb:
                h.zero_()
            hs.hsgen_build_HS_batched(g.ctx, n_gs, [k.ctypes.data for k in kv_host], [h.data_ptr() for h in Hb],
                                      [s.data_ptr() for s in Sb], [n + 3 for n in n_gs], 0)
            torch.cuda.synchronize()
            assert all(torch.equal(a, b) for a, b in zip(Hc, Hb))


def test_batched_config3_sampled_parity(hs):
    import torch

    import _parity

    w = make_config(3)
    n_gs = w.n_g
    kv_host = [np.ascontiguousarray(k) for k in w.kvecs]
    with hs.Generator(w.system, precision=hs.SPLIT) as g:
        Hb, Sb = alloc(n_gs)
        hs.hsgen_build_HS_batched(g.ctx, n_gs, [k.ctypes.data for k in kv_host], [h.data_ptr() for h in Hb],
                                  [s.data_ptr() for s in Sb], n_gs, 0)
        torch.cuda.synchronize()
        rng = np.random.default_rng(4)
        for k in (0, 17, 47):
            n = n_gs[k]
            idx = np.unique(np.concatenate([[0, n - 1], rng.choice(n, 8, replace=False)]))
            r, c = np.meshgrid(idx, idx, indexing="ij")
            sel = r <= c
            ti = torch.from_numpy(r[sel]).cuda(), torch.from_numpy(c[sel]).cuda()
            Hg = Hb[k].mT[ti].cpu().numpy()
            Sg = Sb[k].mT[ti].cpu().numpy()
            Ho, So = oracle.HS_entries(w.system, kv_host[k], r[sel], c[sel])
            Wc, Xc, Yc = _parity.oracle_columns(w.system, kv_host[k][idx])
            pos = {v: i for i, v in enumerate(idx)}
            ri = np.array([pos[v] for v in r[sel]])
            ci = np.array([pos[v] for v in c[sel]])
            wn, xn, yn = (np.linalg.norm(M, axis=0) for M in (Wc, Xc, Yc))
            assert np.linalg.norm(Hg - Ho) <= 1e-11 * np.linalg.norm(Ho)
            assert np.linalg.norm(Sg - So) <= 1e-11 * np.linalg.norm(So)
            assert np.max(np.abs(Hg - Ho) / (wn[ri] * xn[ci])) <= 1e-10
            assert np.max(np.abs(Sg - So) / (wn[ri] * yn[ci])) <= 1e-10
