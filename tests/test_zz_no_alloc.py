"""blco_cpals_update_noalloc: the CP-ALS factor update for callers that
cannot let the library allocate device memory (a process whose memory is all
reserved for its own pool, or a loop that cannot afford cudaFree's
synchronization). It must give the same result as blco_cpals_update, call
after call, although every call reuses one fixed scratch array, and it must
take no device memory: neither from the device (cudaMalloc) nor from the
default stream-ordered pool (cudaMallocAsync)."""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

blco = pytest.importorskip("paper_2201_12523_gb300.blco")

cudaMemPoolAttrUsedMemHigh = 8  # enum cudaMemPoolAttr (driver_types.h)


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found")


def _problem(seed, R, dims, n, tie=False):
    rng = np.random.default_rng(seed)
    hosts = [rng.standard_normal((d, R)).astype(np.float32) for d in dims]
    if tie:  # two equal columns in every factor: V is singular
        for a in hosts:
            a[:, 1] = a[:, 0]
    A = [torch.from_numpy(a).cuda() for a in hosts]
    G = [torch.empty((R, R), dtype=torch.float64, device="cuda") for _ in dims]
    for a, g in zip(A, G):
        blco.blco_gram(a, blco.BLCO_F32, a.shape[0], R, g)
    M = torch.from_numpy(rng.standard_normal((dims[n], R)).astype(np.float32)).cuda()
    return G, M


def _update(fn, G, M, n, R):
    A = torch.empty_like(M)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    Gn = torch.empty((R, R), dtype=torch.float64, device="cuda")
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    fn(G, len(G), n, R, M, M.shape[0], A, lam, Gn, info)
    torch.cuda.synchronize()
    return A.cpu().numpy(), lam.cpu().numpy(), Gn.cpu().numpy(), int(info.item())


def _compare(G, M, n, R, expect_info):
    A0, l0, G0, i0 = _update(blco.blco_cpals_update, G, M, n, R)
    A1, l1, G1, i1 = _update(blco.blco_cpals_update_noalloc, G, M, n, R)
    assert i0 == i1 == expect_info
    np.testing.assert_allclose(l1, l0, rtol=1e-5)
    np.testing.assert_allclose(A1, A0, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(G1, G0, rtol=1e-5, atol=1e-8 * max(1.0, np.abs(G0).max()))


def test_noalloc_update_matches_allocating_update_twice():
    R = 32
    cases = [(11, (500, 300, 200), 0), (12, (400, 350, 600), 2)]  # two calls in a row, different inputs
    for seed, dims, n in cases:
        G, M = _problem(seed, R, dims, n)
        _compare(G, M, n, R, 0)


def test_noalloc_update_at_its_rank_limit_and_on_a_singular_v():
    # R = 64, the largest rank the fixed scratch holds, twice in a row
    for seed, n in ((21, 1), (22, 0)):
        G, M = _problem(seed, 64, (700, 500, 300), n)
        _compare(G, M, n, 64, 0)
    # V singular (two equal columns in every factor): the pseudo-inverse path
    G, M = _problem(23, 8, (60, 50, 40), 1, tie=True)
    _compare(G, M, 1, 8, 1)


def test_noalloc_update_takes_no_device_memory():
    rt = _cudart()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    R = 64
    G, M = _problem(31, R, (4000, 3000, 2000), 0)
    A = torch.empty_like(M)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    Gn = torch.empty((R, R), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (G, 3, 0, R, M, M.shape[0], A, lam, Gn, info)
    blco.blco_cpals_update_noalloc(*args)  # the first call in this context may load the module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, ctypes.byref(zero)) == 0
    for _ in range(3):
        blco.blco_cpals_update_noalloc(*args)
    torch.cuda.synchronize()
    high = ctypes.c_uint64(1)
    assert rt.cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, ctypes.byref(high)) == 0
    free1, _ = torch.cuda.mem_get_info()
    assert high.value == 0, f"the default pool handed out {high.value} bytes during the calls"
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    # the allocating variant, for contrast, does draw on the pool
    blco.blco_cpals_update(*args)
    torch.cuda.synchronize()
    assert rt.cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, ctypes.byref(high)) == 0
    assert high.value > 0


def test_noalloc_update_rejects_rank_beyond_its_scratch():
    Gbig = [torch.zeros((128, 128), dtype=torch.float64, device="cuda") for _ in range(3)]
    Mbig = torch.zeros((50, 128), device="cuda")
    A = torch.empty_like(Mbig)
    lam = torch.empty(128, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_cpals_update_noalloc(Gbig, 3, 0, 128, Mbig, 50, A, lam, None, info)
    assert ei.value.status == blco.BLCO_ERR_ARG and "R <= 64" in str(ei.value)
