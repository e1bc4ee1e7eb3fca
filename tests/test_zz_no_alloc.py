"""blco_cpals_update_noalloc: the CP-ALS factor update for callers that
cannot let the library allocate device memory (a process whose memory is all
reserved for its own pool, or a loop that cannot afford cudaFree's
synchronization). It must give the same result as blco_cpals_update, call
after call, although every call reuses one fixed scratch array."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

blco = pytest.importorskip("paper_2201_12523_gb300.blco")


def _problem(seed, R, dims, n):
    rng = np.random.default_rng(seed)
    A = [torch.from_numpy(rng.standard_normal((d, R)).astype(np.float32)).cuda() for d in dims]
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


def test_noalloc_update_matches_allocating_update_twice():
    R = 32
    cases = [(11, (500, 300, 200), 0), (12, (400, 350, 600), 2)]  # two calls in a row, different inputs
    for seed, dims, n in cases:
        G, M = _problem(seed, R, dims, n)
        A0, l0, G0, i0 = _update(blco.blco_cpals_update, G, M, n, R)
        A1, l1, G1, i1 = _update(blco.blco_cpals_update_noalloc, G, M, n, R)
        assert i0 == i1 == 0
        np.testing.assert_allclose(l1, l0, rtol=1e-5)
        np.testing.assert_allclose(A1, A0, rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(G1, G0, rtol=1e-5, atol=1e-8)


def test_noalloc_update_rejects_rank_beyond_its_scratch():
    G, M = _problem(13, 8, (50, 40, 30), 0)
    Gbig = [torch.zeros((128, 128), dtype=torch.float64, device="cuda") for _ in range(3)]
    Mbig = torch.zeros((50, 128), device="cuda")
    A = torch.empty_like(Mbig)
    lam = torch.empty(128, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_cpals_update_noalloc(Gbig, 3, 0, 128, Mbig, 50, A, lam, None, info)
    assert ei.value.status == blco.BLCO_ERR_ARG and "R <= 64" in str(ei.value)
