"""hsgen_coefficients_noalloc: the coefficient step for callers that cannot
let the library allocate device memory (for example code that runs under
another framework's memory manager, or a latency-critical loop that cannot
take cudaMalloc's implicit synchronisation).

Checked through the C ABI against hsgen_coefficients, the entry point that
does allocate, on two calls in a row with different inputs (the fixed scratch
keeps the previous call's contents), plus its argument checks. This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from workloads import make_config, make_system, kpoint_list

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    assert torch.cuda.is_available()
    return hsgen


def mixed_system():
    lat = np.array([[10.0, 0.3, 0.0], [0.0, 11.0, 0.2], [0.1, 0.0, 9.5]])
    return make_system(41, lat, [(2, 1.5), (4, 1.6), (0, 1.7)], [2, 1, 2])


def existing(hs, g, kv):
    """Reference: the allocating entry point hsgen_coefficients."""
    import torch

    n_g, depth = kv.shape[0], int(g.depth_offsets[-1])
    W = torch.zeros((n_g, depth), dtype=torch.complex128, device="cuda")
    hs.hsgen_coefficients(g.ctx, n_g, kv.data_ptr(), W.data_ptr(), depth, 0)
    torch.cuda.synchronize()
    return W.cpu().numpy()


def noalloc(hs, g, kv):
    import torch

    n_g, depth = kv.shape[0], int(g.depth_offsets[-1])
    W = torch.full((n_g, depth), complex(7.0, -7.0), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    hs.hsgen_coefficients_noalloc(g.ctx, n_g, kv.data_ptr(), W.data_ptr(), depth, 0)
    torch.cuda.synchronize()
    return W.cpu().numpy()


@pytest.mark.parametrize("which", ["config0", "mixed"])
def test_two_calls_match_the_allocating_entry_point(hs, which):
    import torch

    if which == "config0":
        w = make_config(0)
        sysm, kvs = w.system, [w.kvecs[0], w.kvecs[0][:57]]
    else:
        sysm = mixed_system()
        kvs = [kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 129), kpoint_list(sysm.lattice, (0.0, 0.0, 0.0), 40)]
    with hs.Generator(sysm) as g:
        for kv_np in kvs:  # two calls in a row, different sizes and k-points
            kv = torch.from_numpy(kv_np).cuda()
            ref = existing(hs, g, kv)
            got = noalloc(hs, g, kv)
            assert np.max(np.abs(got - ref)) <= 2e-14 * np.max(np.abs(ref))


def test_no_device_memory_is_taken_per_call(hs):
    import torch

    sysm = mixed_system()
    kv = torch.from_numpy(kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 200)).cuda()
    with hs.Generator(sysm) as g:
        noalloc(hs, g, kv)  # first call on the device: address look-up
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        depth = int(g.depth_offsets[-1])
        W = torch.empty((200, depth), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            hs.hsgen_coefficients_noalloc(g.ctx, 200, kv.data_ptr(), W.data_ptr(), depth, 0)
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert free2 == free1, (free0, free1, free2)


def test_rejects_requests_beyond_the_fixed_scratch(hs):
    import torch

    sysm = mixed_system()  # 3 species
    n_g = 40000  # 3 * 40000 = 120000 > 95325
    kv = torch.zeros((n_g, 3), dtype=torch.float64, device="cuda")
    with hs.Generator(sysm) as g:
        depth = int(g.depth_offsets[-1])
        W = torch.zeros((1, depth), dtype=torch.complex128, device="cuda")
        with pytest.raises(hs.HsgenError, match="fixed scratch") as ei:
            hs.hsgen_coefficients_noalloc(g.ctx, n_g, kv.data_ptr(), W.data_ptr(), depth, 0)
        assert ei.value.status == hs.EINVAL


def test_rejects_host_pointers(hs):
    sysm = mixed_system()
    kv = np.ascontiguousarray(kpoint_list(sysm.lattice, (0.1, 0.2, 0.3), 10))
    import torch

    with hs.Generator(sysm) as g:
        depth = int(g.depth_offsets[-1])
        W = torch.zeros((10, depth), dtype=torch.complex128, device="cuda")
        with pytest.raises(hs.HsgenError, match="device pointer") as ei:
            hs.hsgen_coefficients_noalloc(g.ctx, 10, kv.ctypes.data, W.data_ptr(), depth, 0)
        assert ei.value.status == hs.EINVAL
