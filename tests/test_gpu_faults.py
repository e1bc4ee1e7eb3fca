"""Failure handling, with every failure made on the host (blco_inject_fault):
a device allocation that reports out-of-memory at each allocation point of a
streamed build (through device queues, or read in host memory), and a batch
copy of a streamed MTTKRP that fails mid-call. No GPU fault is raised; the
library must report the error, release what it had, and leave the GPU and
later handles working."""

import numpy as np
import pytest
import torch

import oracle
from paper_2201_12523_gb300 import synth
from tests._util import FP32_TOL, check_mttkrp_all, make, to_np64

pytestmark = pytest.mark.gpu

blco = pytest.importorskip("paper_2201_12523_gb300.blco")

_SPEC = synth.small(3, 60_000, (1 << 20, 1 << 16, 1 << 12, 1 << 8))
_BUILD = dict(force_stream=True, max_nnz_per_block=3000, n_queues=3)


@pytest.fixture(autouse=True)
def _disarm():
    yield
    blco.blco_inject_fault(blco.BLCO_FAULT_ALLOC, 0)
    blco.blco_inject_fault(blco.BLCO_FAULT_COPY, 0)


def test_inject_fault_rejects_bad_arguments():
    for kind, k in [(0, 1), (3, 1), (blco.BLCO_FAULT_COPY, -1)]:
        with pytest.raises(blco.BlcoError) as ei:
            blco.blco_inject_fault(kind, k)
        assert ei.value.status == blco.BLCO_ERR_ARG


@pytest.mark.parametrize("host_reads", [False, True])
def test_allocation_failure_at_every_point_of_a_streamed_build(host_reads):
    coords, vals, A = make(_SPEC)
    torch.cuda.synchronize()
    failed = 0
    for k in range(1, 40):
        blco.blco_inject_fault(blco.BLCO_FAULT_ALLOC, k)
        try:
            t = blco.Tensor.build(coords, vals, _SPEC.dims, host_reads=host_reads, **_BUILD)
        except blco.BlcoError as e:
            assert e.status == blco.BLCO_ERR_OOM, str(e)
            assert "injected" in str(e) or "out of memory" in str(e).lower()
            failed += 1
            continue
        # past the last allocation point: the build succeeds and is correct
        blco.blco_inject_fault(blco.BLCO_FAULT_ALLOC, 0)
        assert t.info()["streamed"]
        check_mttkrp_all(t, coords, vals, A, _SPEC.dims)
        t.destroy()
        break
    else:
        pytest.fail("the build never got past its allocation points")
    assert failed >= 3, "a streamed build allocates its store, tables and scratch (and queues)"


def test_copy_failure_mid_mttkrp_leaves_the_handle_usable():
    coords, vals, A = make(_SPEC)
    t = blco.Tensor.build(coords, vals, _SPEC.dims, **_BUILD)
    assert t.info()["nblocks"] > 10
    c, v = coords.cpu().numpy(), vals.cpu().numpy().astype(np.float64)
    for n, k in [(0, 1), (1, 4), (3, 9)]:
        blco.blco_inject_fault(blco.BLCO_FAULT_COPY, k)
        with pytest.raises(blco.BlcoError) as ei:
            t.mttkrp(n, A)
        assert ei.value.status == blco.BLCO_ERR_CUDA and "injected" in str(ei.value)
        torch.cuda.synchronize()  # the work the failed call had queued drains normally
        out = t.mttkrp(n, A)      # the fault fired once; the next call is whole
        torch.cuda.synchronize()
        M, S = oracle.mttkrp(c, v, _SPEC.dims, to_np64(A), n)
        assert oracle.max_rel_err(out.cpu().numpy(), M, S) <= FP32_TOL
    t.destroy()
