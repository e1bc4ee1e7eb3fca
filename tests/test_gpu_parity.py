"""GPU parity of the BLCO library against the FP64 oracle (oracle-sized
cases: several tiles, ragged tails, blocked and streamed stores, every rank
and factor type, edge cases). Everything goes through the C ABI."""

import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2201_12523_gb300 import synth
from tests._util import BF16_TOL, CP_TOL, FP32_TOL, check_mttkrp_all, make, rounded16, to_np64

pytestmark = pytest.mark.gpu

blco = pytest.importorskip("paper_2201_12523_gb300.blco")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "blco_worked_example.txt")


def _store_equal(t, coords, vals, dims, line_bits, cap):
    ref = oracle.build_store(coords.cpu().numpy(), vals.cpu().numpy(), dims, line_bits, cap)
    keys = t.keys()
    perm = t.perm()
    svals = t.values().cpu().numpy()
    bstart, bhigh = t.blocks()
    assert np.array_equal(perm, ref.perm)
    assert np.array_equal(keys, ref.keys)
    assert np.array_equal(svals.view(np.uint32), ref.svals.view(np.uint32))
    assert np.array_equal(bstart, ref.bstart)
    assert np.array_equal(bhigh, ref.bhigh)


# ------------------------------------------------------------ construction
def test_worked_example_store_bit_exact():
    rows = []
    for line in open(GOLDEN):
        t = line.split()
        if t and not line.startswith("#") and t[0] != "store_order":
            rows.append([int(t[0]) - 1, int(t[1]) - 1, int(t[2]) - 1, float(t[3])])
    coords = torch.tensor([r[:3] for r in rows], dtype=torch.int32)
    vals = torch.tensor([r[3] for r in rows], dtype=torch.float32)
    t = blco.Tensor.build(coords.cuda(), vals.cuda(), (4, 4, 4), line_bits=5, max_nnz_per_block=6)
    _store_equal(t, coords, vals, (4, 4, 4), 5, 6)
    assert t.values().cpu().tolist() == [1.0, 2.0, 4.0, 8.0, 6.0, 9.0, 5.0, 3.0, 10.0, 11.0, 7.0, 12.0]


@pytest.mark.parametrize("dims,nnz,line,cap", [
    ((1000, 800, 600), 100_000, 64, 1 << 27),          # uniform 3-mode, one block
    ((1 << 14, 1 << 13, 1 << 7), 54_321, 64, 5000),     # split at a small cap, ragged
    ((1 << 12, 1 << 10, 1 << 8, 64, 16), 77_777, 30, 1 << 27),  # 40 index bits over a 30-bit line
    ((1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8), 200_000, 64, 3000),  # 80 bits: 16 block bits
    ((37, 5, 1, 3), 500, 4, 7),                         # a mode of length 1, tiny blocks
    ((1 << 20,), 4097, 64, 1 << 27),                    # 1 mode
])
def test_store_bit_exact(dims, nnz, line, cap):
    spec = synth.small(1, nnz, dims) if len(dims) != 5 else synth.small(3, nnz, dims)
    coords = synth.coordinates(spec, device="cuda")
    vals = synth.values(spec, device="cuda")
    t = blco.Tensor.build(coords, vals, dims, line_bits=line, max_nnz_per_block=cap)
    _store_equal(t, coords, vals, dims, line, cap)


def test_store_from_host_arrays_and_duplicates():
    rng = np.random.default_rng(0)
    dims = (50, 40, 30)
    c = rng.integers(0, 30, (3000, 3)).astype(np.uint32)  # many duplicates
    v = rng.random(3000).astype(np.float32)
    t = blco.Tensor.build(c, v, dims)
    _store_equal(t, torch.from_numpy(c.astype(np.int32)), torch.from_numpy(v), dims, 64, 1 << 27)


def test_empty_and_single():
    t = blco.Tensor.build(torch.zeros((0, 3), dtype=torch.int32, device="cuda"),
                          torch.zeros(0, device="cuda"), (5, 6, 7))
    assert t.nnz == 0
    A = [torch.randn(d, 16, device="cuda") for d in (5, 6, 7)]
    for n in range(3):
        assert torch.count_nonzero(t.mttkrp(n, A)) == 0
    c = torch.tensor([[4, 5, 6]], dtype=torch.int32, device="cuda")
    v = torch.tensor([2.0], device="cuda")
    t1 = blco.Tensor.build(c, v, (5, 6, 7))
    M = t1.mttkrp(0, A).cpu().numpy()
    ref = 2.0 * A[1][5].cpu().numpy() * A[2][6].cpu().numpy()
    np.testing.assert_allclose(M[4], ref, rtol=1e-6)
    assert np.count_nonzero(M[:4]) == 0


@pytest.mark.parametrize("R", [16, 64])
def test_empty_and_single_five_modes_one_pass(R):
    """The one-pass all-mode kernel on an empty 5-mode store (outputs zeroed,
    no launch) and on a single nonzero (every mode's row is the product of
    the other four rows, every other row zero), also with a streamed store
    and with one read in host memory."""
    dims = (5, 6, 7, 3, 1 << 20)
    A = [torch.randn(d, R, device="cuda") for d in dims]
    for kw in ({}, dict(force_stream=True, host_reads=True)):
        t = blco.Tensor.build(torch.zeros((0, 5), dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"),
                              dims, **kw)
        outs = [torch.full((d, R), 7.0, device="cuda") for d in dims]
        t.mttkrp_all(A, outs=outs)
        torch.cuda.synchronize()
        assert all(torch.count_nonzero(o) == 0 for o in outs)
    c = torch.tensor([[4, 5, 6, 2, (1 << 20) - 1]], dtype=torch.int32, device="cuda")
    v = torch.tensor([-1.5], device="cuda")
    for kw in ({}, dict(force_stream=True), dict(force_stream=True, host_reads=True)):
        t1 = blco.Tensor.build(c, v, dims, **kw)
        outs = t1.mttkrp_all(A)
        torch.cuda.synchronize()
        rows = c[0].tolist()
        for n in range(5):
            ref = torch.full((R,), -1.5, dtype=torch.float64, device="cuda")
            for k in range(5):
                if k != n:
                    ref *= A[k][rows[k]].double()
            np.testing.assert_allclose(outs[n][rows[n]].double().cpu().numpy(), ref.cpu().numpy(), rtol=1e-6)
            other = torch.ones(dims[n], dtype=torch.bool, device="cuda")
            other[rows[n]] = False
            assert torch.count_nonzero(outs[n][other]) == 0


def test_out_of_range_coordinate_is_index_error():
    c = torch.tensor([[0, 0, 0], [1, 6, 0], [2, 1, 1]], dtype=torch.int32, device="cuda")
    v = torch.ones(3, device="cuda")
    with pytest.raises(blco.BlcoError) as ei:
        blco.Tensor.build(c, v, (5, 6, 7))
    assert ei.value.status == blco.BLCO_ERR_INDEX


def _u32_coords(c64):
    """uint32 coordinates as the int32 tensor the binding passes (same bits)."""
    return torch.from_numpy(np.ascontiguousarray(c64.astype(np.uint32).view(np.int32)))


@pytest.mark.parametrize("dims,line,cap", [
    ((0xFFFFFFFF,) * 4, 64, 1 << 27),                     # 4 x 32 bits = 128 index bits, 64 block bits
    ((0xFFFFFFFF, (1 << 31) + 1, 3, 1), 64, 4099),         # two 32-bit modes, a length-1 mode, split blocks
    ((0xFFFFFFFF, 0xFFFFFFFF), 1, 1 << 27),                # 1-bit line: 63 of 64 bits above it
])
def test_store_at_maximum_mode_lengths(dims, line, cap):
    """The largest mode length the ABI takes (2^32 - 1, coordinates are
    uint32): every coordinate bit above bit 30 reaches the key, the block
    table and the re-encoded fields as the definition places it (Section 4.1,
    Section 4.2), with the first and last index of every mode present."""
    rng = np.random.default_rng(sum(int(d).bit_length() for d in dims) + line)
    nnz = 20_011
    c = np.stack([rng.integers(0, d, nnz, dtype=np.uint64) for d in dims], 1)
    c[0] = 0
    c[1] = [d - 1 for d in dims]
    c[2] = [d - 1 if k % 2 else 0 for k, d in enumerate(dims)]
    coords = _u32_coords(c)
    vals = torch.from_numpy(rng.random(nnz).astype(np.float32))
    t = blco.Tensor.build(coords.cuda(), vals.cuda(), dims, line_bits=line, max_nnz_per_block=cap)
    assert t.info()["total_bits"] == sum(max(int(d - 1).bit_length(), 0) for d in dims)
    _store_equal(t, coords, vals, dims, line, cap)
    # the one index past the end of a 2^32 - 1 mode is rejected
    bad = c[:3].copy()
    bad[2, 0] = 0xFFFFFFFF
    with pytest.raises(blco.BlcoError) as ei:
        blco.Tensor.build(_u32_coords(bad).cuda(), vals[:3].cuda(), dims)
    assert ei.value.status == blco.BLCO_ERR_INDEX


# ------------------------------------------------------------ MTTKRP
@pytest.mark.parametrize("R", [8, 16, 32, 64, 128])
def test_mttkrp_uniform_all_ranks(R):
    spec = synth.small(0, 30_011, (1000, 800, 600))
    coords, vals, _ = make(spec)
    A = synth.factors(spec, rank=R, device="cuda")
    t = blco.Tensor.build(coords, vals, spec.dims)
    check_mttkrp_all(t, coords, vals, A, spec.dims)


def test_mttkrp_uniform_100k_full():
    spec = synth.workload("uniform-3d-100k")
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims)
    check_mttkrp_all(t, coords, vals, A, spec.dims)


@pytest.mark.parametrize("idx,nnz,dims", [
    (1, 300_000, (1 << 16, 1 << 15, 1 << 11)),               # Zipf 1.2, 3 modes, one mode fits on chip
    (2, 300_000, (1 << 14, 1 << 12, 1 << 10, 1 << 8)),        # Zipf 1.1, 4 modes, lognormal values
    (3, 200_000, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8)),  # 5 modes, 80 bits -> blocks
    (4, 200_000, (1 << 14, 1 << 14, 1 << 10)),                # planted-model shape, R=64
])
def test_mttkrp_skewed_f32(idx, nnz, dims):
    spec = synth.small(idx, nnz, dims)
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims)
    check_mttkrp_all(t, coords, vals, A, spec.dims)


@pytest.mark.parametrize("dims,R", [
    ((1 << 16, 1 << 15, 1 << 14, 1 << 13, 1 << 12, 1 << 11), 16),   # 6 modes, 81 index bits
    ((1 << 16,) * 8, 8),                                            # 8 modes, 128 index bits
    ((1 << 16,) * 8, 32),
])
def test_many_modes_generic_path(dims, R):
    """6 and 8 modes take the kernel's run-time gather count (5 or 7
    gathered rows); 128 index bits fill both key words before blocking."""
    rng = np.random.default_rng(len(dims) * 100 + R)
    nnz = 30_011
    c = np.stack([rng.integers(0, d, nnz) for d in dims], 1).astype(np.int32)
    vals = rng.random(nnz).astype(np.float32)
    A = [torch.from_numpy(rng.standard_normal((d, R)).astype(np.float32)).cuda() for d in dims]
    coords = torch.from_numpy(c).cuda()
    t = blco.Tensor.build(coords, torch.from_numpy(vals).cuda(), dims, max_nnz_per_block=7000)
    assert t.info()["total_bits"] == sum(int(np.ceil(np.log2(d))) for d in dims)
    _store_equal(t, coords, torch.from_numpy(vals), dims, 64, 7000)
    check_mttkrp_all(t, coords, torch.from_numpy(vals), A, dims)


def test_mttkrp_positive_heavy_rows():
    """All terms positive on a Zipf head (the hardest case for float32 sums)."""
    spec = synth.small(1, 400_000, (1 << 12, 1 << 11, 1 << 11))
    coords, vals, _ = make(spec)
    A = synth.factors(spec, device="cuda", dist="u01")
    t = blco.Tensor.build(coords, vals, spec.dims)
    check_mttkrp_all(t, coords, vals, A, spec.dims)


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("nrows", [1, 3, 40])
def test_mttkrp_runs_across_subgroups(R, nrows):
    """Every nonzero in one of a few rows of a long mode: the warp's sorted
    runs cover whole subgroups and cross their boundaries."""
    rng = np.random.default_rng(nrows * 100 + R)
    dims = (100_000, 300, 200)
    nnz = 50_000
    rows = rng.choice(dims[0], nrows, replace=False)
    c = np.stack([rng.choice(rows, nnz), rng.integers(0, dims[1], nnz), rng.integers(0, dims[2], nnz)], 1)
    c = np.unique(c, axis=0)
    rng.shuffle(c)
    coords = torch.from_numpy(c.astype(np.int32)).cuda()
    vals = torch.from_numpy(rng.random(len(c)).astype(np.float32)).cuda()
    A = [torch.from_numpy(rng.random((d, R)).astype(np.float32)).cuda() for d in dims]  # positive terms
    t = blco.Tensor.build(coords, vals, dims)
    check_mttkrp_all(t, coords, vals, A, dims)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_mttkrp_16bit_factors(dtype):
    spec = synth.small(2, 300_000, (1 << 14, 1 << 12, 1 << 10, 1 << 8))
    coords, vals, A = make(spec)
    A16 = [blco.convert(a, dtype) for a in A]
    t = blco.Tensor.build(coords, vals, spec.dims)
    # accumulation error alone: oracle on the rounded factors
    check_mttkrp_all(t, coords, vals, A16, spec.dims, tol=FP32_TOL, factors_ref=rounded16(A, dtype))
    # total error against the unrounded float32 factors
    check_mttkrp_all(t, coords, vals, A16, spec.dims, tol=BF16_TOL, factors_ref=to_np64(A))


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("R", [32, 64, 128])
def test_16bit_run_sum_is_compensated(dtype, R):
    """Eight nonzeros of one output row, the first 1.0 and seven of 2^-25,
    all within one subgroup's run (factors of ones are exact in 16 bits).
    With compensated_sums the run sum returns the float32 nearest the exact
    1 + 1.75 * 2^-23, i.e. 1 + 2^-22; with the default plain float32 sums the
    terms are added one by one and each tiny one is lost: 1.0."""
    dims = (4, 8, 2)
    c = np.array([[1, j, 0] for j in range(8)], dtype=np.int32)  # ALTO order = j order
    v = np.array([1.0] + [2.0 ** -25] * 7, dtype=np.float32)
    A = [blco.convert(torch.ones((d, R), device="cuda"), dtype) for d in dims]
    for comp, want in [(True, 1.0 + 2.0 ** -22), (False, 1.0)]:
        t = blco.Tensor.build(torch.from_numpy(c).cuda(), torch.from_numpy(v).cuda(), dims, compensated_sums=comp)
        assert np.array_equal(t.perm(), np.arange(8))
        out = t.mttkrp(0, A).cpu().numpy()
        assert np.all(out[1] == np.float32(want)), (comp, out[1])
        assert np.all(out[[0, 2, 3]] == 0.0)


@pytest.mark.parametrize("nnz", [1, 31, 33, 1000, 4099])
def test_unreferenced_nonfinite_factor_rows_do_not_leak(nnz):
    """Ragged tails: lanes past the end of the store must not touch factor
    rows that no nonzero references. Every unreferenced row holds Inf or NaN;
    the outputs must still match the oracle (which never reads those rows)."""
    rng = np.random.default_rng(nnz)
    dims = (50, 40, 30)
    c = np.unique(np.stack([rng.integers(1, d, nnz) for d in dims], 1), axis=0)  # row 0 never used
    rng.shuffle(c)
    vals = rng.random(len(c)).astype(np.float32)
    R = 16
    A = []
    for n, d in enumerate(dims):
        a = rng.standard_normal((d, R)).astype(np.float32)
        unused = np.setdiff1d(np.arange(d), c[:, n])
        a[unused] = np.where(rng.random((len(unused), R)) < 0.5, np.inf, np.nan)
        A.append(torch.from_numpy(a).cuda())
    t = blco.Tensor.build(torch.from_numpy(c.astype(np.int32)).cuda(), torch.from_numpy(vals).cuda(), dims)
    v64 = vals.astype(np.float64)
    for n in range(3):
        out = t.mttkrp(n, A).cpu().numpy()
        used = np.unique(c[:, n])
        Af = [a.cpu().numpy().astype(np.float64) for a in A]
        M, S = oracle.mttkrp(c, v64, dims, Af, n)
        assert np.isfinite(out).all()
        assert oracle.max_rel_err(out[used], M[used], S[used]) <= FP32_TOL
        assert np.all(out[np.setdiff1d(np.arange(dims[n]), used)] == 0.0)


@pytest.mark.parametrize("nnz", [33, 1000, 4099])
def test_referenced_infinite_factor_row_in_the_ragged_tail(nnz):
    """The first nonzero of the last (ragged) tile references a factor row
    holding +Inf. The oracle's sums are then +Inf wherever that row enters
    (all factors positive, so no Inf - Inf): lanes past the end of the store
    must add nothing there, so the library gives +Inf too, not the NaN that
    0 * Inf would leave."""
    rng = np.random.default_rng(nnz + 7)
    dims = (50, 40, 30)
    c = np.unique(np.stack([rng.integers(0, d, nnz + 200) for d in dims], 1), axis=0)[:nnz]
    rng.shuffle(c)
    vals = (rng.random(len(c)) + 0.5).astype(np.float32)
    R = 16
    hostA = [(rng.random((d, R)) + 0.5).astype(np.float32) for d in dims]
    t = blco.Tensor.build(torch.from_numpy(c.astype(np.int32)).cuda(), torch.from_numpy(vals).cuda(), dims)
    last = (len(c) - 1) // 32 * 32  # store position of the last tile's first lane
    j = int(t.perm()[last])
    hostA[1][c[j, 1]] = np.inf
    A = [torch.from_numpy(a).cuda() for a in hostA]
    Af = [a.astype(np.float64) for a in hostA]
    v64 = vals.astype(np.float64)
    for n in range(3):
        out = t.mttkrp(n, A).cpu().numpy()
        M, S = oracle.mttkrp(c, v64, dims, Af, n)
        inf = np.isinf(M)
        assert not np.isnan(M).any()
        assert (n == 1) == (not inf.any())
        assert np.array_equal(np.isposinf(out), inf) and not np.isnan(out).any()
        fin = ~inf
        assert oracle.max_rel_err(out[fin], M[fin], S[fin]) <= FP32_TOL


def test_convert_matches_oracle_rounding():
    x = torch.randn(100_003, device="cuda") * 3
    # ties, subnormals, overflow and signed zeros as well as ordinary values
    special = torch.tensor([0.0, -0.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1e-40, -1e-40, 3.4e38, 65520.0,
                            6.1e-5, 5.9e-8, float("inf"), float("-inf")], device="cuda")
    x = torch.cat([x, special])
    y = blco.convert(x, torch.bfloat16)
    ref = oracle.bf16_round(x.cpu().numpy())
    assert np.array_equal(y.float().cpu().numpy().view(np.uint32), ref.view(np.uint32))
    # float16: IEEE binary16 round-to-nearest-even (numpy's cast), incl. overflow to inf
    h = blco.convert(x, torch.float16)
    with np.errstate(over="ignore"):
        ref16 = x.cpu().numpy().astype(np.float16)
    assert np.array_equal(h.cpu().numpy().view(np.uint16), ref16.view(np.uint16))


@pytest.mark.parametrize("nq", [1, 3, 8])
def test_streamed_store_matches(nq):
    spec = synth.small(3, 150_000, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims, force_stream=True, max_nnz_per_block=4000, n_queues=nq)
    info = t.info()
    assert info["streamed"] and info["nblocks"] > 30
    check_mttkrp_all(t, coords, vals, A, spec.dims)
    _store_equal(t, coords, vals, spec.dims, 64, 4000)


@pytest.mark.parametrize("order,nq", [(5, 1), (5, 3), (4, 2)])
def test_streamed_all_mode_uploads_each_batch_once(order, nq):
    """All-mode MTTKRP of a streamed store: each batch of blocks crosses the
    host link once per call (Section 4.2's queues), and every mode's kernel
    runs on it while it is resident (5 modes: one one-pass launch per batch;
    4 modes: one per-mode launch per batch and mode); the results match the
    oracle, also for a short R = 64 mode and with bf16 factors."""
    dims = (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8)[:order]
    spec = synth.small(3 if order == 5 else 2, 150_000, dims)
    coords, vals, _ = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims, force_stream=True, max_nnz_per_block=4000, n_queues=nq)
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    for R, dt in ((16, torch.float32), (64, torch.float32), (32, torch.bfloat16)):
        A = synth.factors(spec, rank=R, device="cuda", dist="normal")
        F = A if dt == torch.float32 else [blco.convert(a, dt) for a in A]
        Aref = to_np64(A) if dt == torch.float32 else rounded16(A, dt)
        blco.blco_profile_enable(t.handle, True)
        t.mttkrp(0, F)
        one = blco.blco_profile_read(t.handle)
        outs = t.mttkrp_all(F)
        torch.cuda.synchronize()
        allm = blco.blco_profile_read(t.handle)
        blco.blco_profile_enable(t.handle, False)
        batches = one["upload"][0]
        assert batches > 1
        assert allm["upload"][0] == batches
        if order == 5:
            assert allm["mttkrp_all_fused"][0] == batches
        else:
            assert allm["mttkrp"][0] == batches * order
        for n in range(order):
            M, S = oracle.mttkrp(c, v, spec.dims, Aref, n)
            assert oracle.max_rel_err(outs[n].cpu().numpy(), M, S) <= FP32_TOL, (R, dt, n)


@pytest.mark.parametrize("order", [3, 5])
def test_store_read_in_host_memory(order):
    """A streamed store whose kernels read keys and values in its pinned host
    memory (build option host_reads): no queue reservations in device memory,
    the same store bytes, and every call against the oracle -- per-mode
    MTTKRP, the all-mode call (one pass at 5 modes, per-mode kernels at 3),
    parts of the store, the CP model and its adjoint."""
    dims = (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8) if order == 5 else (1 << 14, 1 << 13, 1 << 7)
    spec = synth.small(3 if order == 5 else 1, 60_013, dims)
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims, force_stream=True, host_reads=True, max_nnz_per_block=4000)
    info = t.info()
    assert info["streamed"] and info["host_reads"] and info["n_queues"] == 0 and info["nblocks"] > 3
    # the device holds what a queue-streamed store holds, less its queue reservations
    iq = blco.Tensor.build(coords, vals, spec.dims, force_stream=True, max_nnz_per_block=4000).info()
    assert info["device_bytes"] + iq["n_queues"] * iq["queue_nnz"] * 12 == iq["device_bytes"]
    _store_equal(t, coords, vals, spec.dims, 64, 4000)
    check_mttkrp_all(t, coords, vals, A, spec.dims)
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    Af = to_np64(A)
    outs = t.mttkrp_all(A)
    torch.cuda.synchronize()
    for n in range(order):
        M, S = oracle.mttkrp(c, v, spec.dims, Af, n)
        assert oracle.max_rel_err(outs[n].cpu().numpy(), M, S) <= FP32_TOL, n
    # a part of the store (blco_mttkrp_range reads it in host memory too)
    b = blco.blco_partition(spec.nnz, 3)
    cs = c[t.perm()]
    vs = t.values().cpu().numpy().astype(np.float64)
    out = torch.empty((spec.dims[0], spec.rank), device="cuda")
    blco.blco_mttkrp_range(t.handle, 0, int(b[1]), int(b[2]), A, blco.BLCO_F32, spec.rank, out)
    M, S = oracle.mttkrp(cs[b[1]:b[2]], vs[b[1]:b[2]], spec.dims, Af, 0)
    assert oracle.max_rel_err(out.cpu().numpy(), M, S) <= FP32_TOL
    # CP model at the nonzeros (store order) and its adjoint with g in place of x
    xhat = t.cp_fwd(A).cpu().numpy()
    ref, scale = _cp_ref(t, coords, A)
    assert float(np.max(np.abs(xhat - ref) / scale)) <= CP_TOL
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(spec.nnz).astype(np.float32)).cuda()
    gb = t.cp_bwd(1, g, A)
    M, S = oracle.mttkrp(cs, g.cpu().numpy().astype(np.float64), spec.dims, Af, 1)
    assert oracle.max_rel_err(gb.cpu().numpy(), M, S) <= FP32_TOL


@pytest.mark.parametrize("streamed", ["resident", "queues", "host"])
def test_short_mode_output_copies(streamed):
    """R = 64 with 1024- and 600-row modes: those launches reduce into
    private output copies and sum the copies afterwards, also when the
    batches of a streamed store run concurrently on several queues, and on
    a store read in host memory."""
    spec = synth.small(4, 150_000, (1 << 16, 600, 1 << 10))
    coords, vals, A = make(spec)
    kw = {"queues": dict(force_stream=True, max_nnz_per_block=4000, n_queues=4),
          "host": dict(force_stream=True, host_reads=True, max_nnz_per_block=4000)}.get(streamed, {})
    t = blco.Tensor.build(coords, vals, spec.dims, **kw)
    check_mttkrp_all(t, coords, vals, A, spec.dims)
    check_mttkrp_all(t, coords, vals, A, spec.dims, modes=[2, 1])  # again: copies reused


def test_budget_forces_streaming():
    spec = synth.small(1, 200_000, (1 << 16, 1 << 15, 1 << 11))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims, device_budget_bytes=2_000_000, max_nnz_per_block=20_000,
                          n_queues=4)
    info = t.info()
    assert info["streamed"] and info["device_bytes"] <= 2_000_000
    check_mttkrp_all(t, coords, vals, A, spec.dims)


def test_host_factor_and_output_pointers():
    spec = synth.small(1, 100_000, (1 << 14, 1 << 13, 1 << 9))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords.cpu().numpy().astype(np.uint32), vals.cpu().numpy(), spec.dims)
    Ah = [a.cpu().numpy() for a in A]
    outs = [np.empty((d, spec.rank), np.float32) for d in spec.dims]
    blco.blco_mttkrp_all(t.handle, Ah, blco.BLCO_F32, spec.rank, outs)
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    for n in range(3):
        M, S = oracle.mttkrp(c, v, spec.dims, to_np64(A), n)
        assert oracle.max_rel_err(outs[n], M, S) <= FP32_TOL


@pytest.mark.parametrize("streamed", [False, True])
def test_mttkrp_all_mixed_host_and_device_arguments(streamed):
    """Pipelined host path: host and device factors mixed, host, device and
    absent outputs, a resident and a streamed store; called twice in a row
    (the staging workspace and copy streams are reused)."""
    spec = synth.small(2, 120_000, (1 << 13, 1 << 11, 1 << 9, 1 << 7))
    coords, vals, A = make(spec)
    kw = dict(force_stream=True, max_nnz_per_block=5000, n_queues=3) if streamed else {}
    t = blco.Tensor.build(coords, vals, spec.dims, **kw)
    R = spec.rank
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    ref = [oracle.mttkrp(c, v, spec.dims, to_np64(A), n) for n in range(4)]
    for rep in range(2):
        facs = [A[0].cpu().numpy(), A[1], A[2].cpu().numpy(), A[3]] if rep == 0 else \
               [A[0], A[1].cpu().numpy(), A[2], A[3].cpu().numpy()]
        outs = [np.empty((spec.dims[0], R), np.float32), torch.empty((spec.dims[1], R), device="cuda"),
                None, np.empty((spec.dims[3], R), np.float32)]
        blco.blco_mttkrp_all(t.handle, facs, blco.BLCO_F32, R, outs)
        torch.cuda.synchronize()
        for n in (0, 1, 3):
            got = outs[n].cpu().numpy() if isinstance(outs[n], torch.Tensor) else outs[n]
            M, S = ref[n]
            assert oracle.max_rel_err(got, M, S) <= FP32_TOL, (rep, n)


@pytest.mark.parametrize("parts", [2, 3, 7])
def test_partitioned_mttkrp_sums_to_the_full_result(parts):
    """The store cut into equal contiguous parts (blco_partition), each
    part's MTTKRP computed alone (blco_mttkrp_range, one after another on
    one GPU, as the ranks of a partitioned run would), and the parts summed:
    the oracle's MTTKRP of the whole tensor; every part alone matches the
    oracle on that part's nonzeros. A blocked 5-mode store, so that parts
    cut blocks."""
    spec = synth.small(3, 50_000, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims, max_nnz_per_block=3000)
    assert t.info()["nblocks"] > parts
    b = blco.blco_partition(spec.nnz, parts)
    cs = coords.cpu().numpy()[t.perm()]
    vs = t.values().cpu().numpy().astype(np.float64)
    Af = to_np64(A)
    R = spec.rank
    for mode in (0, 2, 4):
        total = torch.zeros((spec.dims[mode], R), device="cuda")
        for i in range(parts):
            out = torch.empty((spec.dims[mode], R), device="cuda")
            blco.blco_mttkrp_range(t.handle, mode, int(b[i]), int(b[i + 1]), A, blco.BLCO_F32, R, out)
            M, S = oracle.mttkrp(cs[b[i]:b[i + 1]], vs[b[i]:b[i + 1]], spec.dims, Af, mode)
            assert oracle.max_rel_err(out.cpu().numpy(), M, S) <= FP32_TOL, (mode, i)
            total += out
        M, S = oracle.mttkrp(cs, vs, spec.dims, Af, mode)
        assert oracle.max_rel_err(total.cpu().numpy(), M, S) <= 2 * FP32_TOL
    # empty range: zeros; unaligned begin and a streamed store are refused
    out = torch.full((spec.dims[0], R), 7.0, device="cuda")
    blco.blco_mttkrp_range(t.handle, 0, 64, 64, A, blco.BLCO_F32, R, out)
    assert torch.all(out == 0)
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_mttkrp_range(t.handle, 0, 33, 64, A, blco.BLCO_F32, R, out)
    assert ei.value.status == blco.BLCO_ERR_ARG
    ts = blco.Tensor.build(coords, vals, spec.dims, force_stream=True)
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_mttkrp_range(ts.handle, 0, 0, 64, A, blco.BLCO_F32, R, out)
    assert ei.value.status == blco.BLCO_ERR_STATE


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("which", ["5d", "5d-blocked", "5d-short", "5d-host"])
def test_all_mode_one_pass_matches_oracle(which, R, dtype):
    """blco_mttkrp_all on a 5-mode store gathers each nonzero's rows once for
    every mode (one kernel launch): every mode against the FP64 oracle, with
    ragged tails, a blocked store with 2^24-row modes (also read in host
    memory), modes short enough to be held on chip whole, and a mode left
    out."""
    if which == "5d":
        spec = synth.small(3, 60_013, (1 << 12, 1 << 10, 1 << 9, 1 << 6, 1 << 4))
        kw = {}
    elif which == "5d-blocked":
        spec = synth.small(3, 40_009, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8))
        kw = dict(max_nnz_per_block=5000)
    elif which == "5d-host":
        spec = synth.small(3, 40_009, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8))
        kw = dict(max_nnz_per_block=5000, force_stream=True, host_reads=True)
    else:
        spec = synth.small(3, 20_011, (400, 9, 5, 3, 2))
        kw = {}
    coords, vals, _ = make(spec)
    A = synth.factors(spec, rank=R, device="cuda", dist="normal")
    F = A if dtype == torch.float32 else [blco.convert(a, dtype) for a in A]
    Aref = to_np64(A) if dtype == torch.float32 else rounded16(A, dtype)
    t = blco.Tensor.build(coords, vals, spec.dims, **kw)
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    blco.blco_profile_enable(t.handle, True)
    outs = t.mttkrp_all(F)
    torch.cuda.synchronize()
    prof = blco.blco_profile_read(t.handle)
    blco.blco_profile_enable(t.handle, False)
    assert prof["mttkrp_all_fused"][0] == 1 and "mttkrp" not in prof
    for n in range(spec.order):
        M, S = oracle.mttkrp(c, v, spec.dims, Aref, n)
        assert oracle.max_rel_err(outs[n].cpu().numpy(), M, S) <= FP32_TOL, n
    # mode 1 left out (a NULL output): the other modes exact as before
    outs2 = [torch.empty((d, R), device="cuda") for d in spec.dims]
    outs2[1] = None
    blco.blco_mttkrp_all(t.handle, F, blco._fdt(F), R, outs2)
    torch.cuda.synchronize()
    for n in (0, spec.order - 1):
        M, S = oracle.mttkrp(c, v, spec.dims, Aref, n)
        assert oracle.max_rel_err(outs2[n].cpu().numpy(), M, S) <= FP32_TOL, n


@pytest.mark.parametrize("dims,R", [((1 << 12, 1 << 10, 1 << 9), 32), ((1 << 11, 1 << 10, 1 << 8, 1 << 5), 16),
                                    ((1 << 10, 1 << 9, 1 << 8, 1 << 6, 1 << 4), 8)])
def test_all_mode_per_mode_kernels(dims, R):
    """blco_mttkrp_all where the one-pass kernel does not apply (3 and 4
    modes; a rank it is not built for): one per-mode launch per requested
    mode, every mode against the oracle."""
    spec = synth.small(1 if len(dims) == 3 else (2 if len(dims) == 4 else 3), 50_021, dims)
    coords, vals, _ = make(spec)
    A = synth.factors(spec, rank=R, device="cuda", dist="normal")
    t = blco.Tensor.build(coords, vals, spec.dims)
    blco.blco_profile_enable(t.handle, True)
    outs = t.mttkrp_all(A)
    torch.cuda.synchronize()
    prof = blco.blco_profile_read(t.handle)
    blco.blco_profile_enable(t.handle, False)
    assert prof["mttkrp"][0] == len(dims) and "mttkrp_all_fused" not in prof
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    for n in range(len(dims)):
        M, S = oracle.mttkrp(c, v, spec.dims, to_np64(A), n)
        assert oracle.max_rel_err(outs[n].cpu().numpy(), M, S) <= FP32_TOL, n


@pytest.mark.parametrize("R", [8, 16, 32, 64])
@pytest.mark.parametrize("which", ["3d", "4d", "5d-blocked"])
def test_mttkrp_f64_matches_oracle(which, R):
    """float64 values, factors and accumulation (the paper's precision):
    every mode against the FP64 oracle to 1e-12 of sum |terms| (only the
    summation order differs), on a skewed 3-mode, a 4-mode and a blocked
    5-mode store with ragged tails."""
    if which == "3d":
        spec = synth.small(1, 60_003, (1 << 12, 1 << 11, 1 << 8))
        kw = {}
    elif which == "4d":
        spec = synth.small(2, 40_001, (1 << 10, 1 << 9, 1 << 8, 1 << 4))
        kw = {}
    else:
        spec = synth.small(3, 30_017, (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8))
        kw = dict(max_nnz_per_block=4000)
    coords, vals32, _ = make(spec)
    rng = np.random.default_rng(R)
    v = rng.standard_normal(spec.nnz)  # float64 values with full mantissas
    A = [rng.standard_normal((d, R)) for d in spec.dims]
    t = blco.Tensor.build(coords, torch.from_numpy(v).cuda(), spec.dims, **kw)
    if which == "5d-blocked":
        assert t.info()["nblocks"] > 1
    Ad = [torch.from_numpy(a).cuda() for a in A]
    c = coords.cpu().numpy()
    for n in range(spec.order):
        out = t.mttkrp_f64(n, Ad)
        M, S = oracle.mttkrp(c, v, spec.dims, A, n)
        assert oracle.max_rel_err(out.cpu().numpy(), M, S) <= 1e-12, n
    # host factors and a host result
    outh = np.empty((spec.dims[0], R))
    blco.blco_mttkrp_f64(t.handle, 0, [None] + A[1:], R, outh)
    M, S = oracle.mttkrp(c, v, spec.dims, A, 0)
    assert oracle.max_rel_err(outh, M, S) <= 1e-12


def test_f64_store_state_errors():
    spec = synth.small(0, 5000, (100, 80, 60))
    coords, vals32, A32 = make(spec)
    v = vals32.double()
    t64 = blco.Tensor.build(coords, v, spec.dims)
    t32 = blco.Tensor.build(coords, vals32, spec.dims)
    A64 = [a.double() for a in A32]
    with pytest.raises(blco.BlcoError) as ei:
        t64.mttkrp(0, A32)
    assert ei.value.status == blco.BLCO_ERR_STATE
    with pytest.raises(blco.BlcoError) as ei:
        t32.mttkrp_f64(0, A64)
    assert ei.value.status == blco.BLCO_ERR_STATE
    with pytest.raises(blco.BlcoError) as ei:
        t64.values()
    assert ei.value.status == blco.BLCO_ERR_STATE
    A128 = [torch.zeros((d, 128), dtype=torch.float64, device="cuda") for d in spec.dims]
    with pytest.raises(blco.BlcoError) as ei:
        t64.mttkrp_f64(0, A128)
    assert ei.value.status == blco.BLCO_ERR_UNSUPPORTED
    with pytest.raises(blco.BlcoError) as ei:
        blco.Tensor.build(coords, v, spec.dims, force_stream=True)
    assert ei.value.status == blco.BLCO_ERR_UNSUPPORTED
    # the float64 store has the float32 store's order and blocks
    assert np.array_equal(t64.perm(), t32.perm()) and np.array_equal(t64.keys(), t32.keys())


def test_argument_errors():
    spec = synth.small(0, 1000, (10, 20, 30))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims)
    out = torch.empty((10, 16), device="cuda")
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_mttkrp(t.handle, 0, A, blco.BLCO_F32, 24, out)
    assert ei.value.status == blco.BLCO_ERR_UNSUPPORTED
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_mttkrp(t.handle, 3, A, blco.BLCO_F32, 16, out)
    assert ei.value.status == blco.BLCO_ERR_ARG
    bad = torch.empty(10 * 16 + 1, device="cuda")[1:].view(10, 16)
    with pytest.raises(blco.BlcoError) as ei:
        blco.blco_mttkrp(t.handle, 0, A, blco.BLCO_F32, 16, bad)
    assert ei.value.status == blco.BLCO_ERR_ARG


# ------------------------------------------------------------ CP model
def _cp_ref(t, coords, A):
    c = coords.cpu().numpy()[t.perm()]
    Af = to_np64(A)
    return oracle.cp_model(c, Af), oracle.cp_model(c, [np.abs(a) for a in Af])


@pytest.mark.parametrize("R", [16, 64])
def test_cp_fwd_matches(R):
    spec = synth.small(4, 150_000, (1 << 14, 1 << 14, 1 << 10))
    coords, vals, _ = make(spec)
    A = synth.factors(spec, rank=R, device="cuda", dist="normal")
    t = blco.Tensor.build(coords, vals, spec.dims)
    xhat = t.cp_fwd(A).cpu().numpy()
    ref, scale = _cp_ref(t, coords, A)
    assert float(np.max(np.abs(xhat - ref) / scale)) <= CP_TOL


def test_cp_bwd_is_mttkrp_with_gradient_values():
    spec = synth.small(4, 150_000, (1 << 14, 1 << 14, 1 << 10))
    coords, vals, A = make(spec)
    t = blco.Tensor.build(coords, vals, spec.dims)
    g = torch.randn(spec.nnz, device="cuda")
    c = coords.cpu().numpy()[t.perm()]
    gn = g.cpu().numpy().astype(np.float64)
    for n in range(3):
        out = t.cp_bwd(n, g, A).cpu().numpy()
        M, S = oracle.mttkrp(c, gn, spec.dims, to_np64(A), n)
        assert oracle.max_rel_err(out, M, S) <= FP32_TOL


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("R", [16, 64])
def test_cp_bwd_16bit_factors(dtype, R):
    """The adjoint with 16-bit factors (float32 accumulation): against the
    FP64 oracle on the rounded factors (accumulation error only) and on the
    unrounded float32 factors (the factor rounding, bound 1e-2)."""
    spec = synth.small(4, 150_000, (1 << 14, 1 << 14, 1 << 10))
    coords, vals, _ = make(spec)
    A = synth.factors(spec, rank=R, device="cuda", dist="normal")
    A16 = [blco.convert(a, dtype) for a in A]
    t = blco.Tensor.build(coords, vals, spec.dims)
    g = torch.randn(spec.nnz, device="cuda")
    c = coords.cpu().numpy()[t.perm()]
    gn = g.cpu().numpy().astype(np.float64)
    Ar = rounded16(A, dtype)
    for n in range(3):
        out = t.cp_bwd(n, g, A16).cpu().numpy()
        M, S = oracle.mttkrp(c, gn, spec.dims, Ar, n)
        assert oracle.max_rel_err(out, M, S) <= FP32_TOL
        M, S = oracle.mttkrp(c, gn, spec.dims, to_np64(A), n)
        assert oracle.max_rel_err(out, M, S) <= BF16_TOL


def test_sparse_cp_autograd():
    spec = synth.small(4, 50_000, (1 << 12, 1 << 12, 1 << 8))
    coords, vals, _ = make(spec)
    A = [a.requires_grad_() for a in synth.factors(spec, rank=16, device="cuda", dist="normal")]
    t = blco.Tensor.build(coords, vals, spec.dims)
    sv = t.values()
    xhat = blco.SparseCP.apply(t, *A)
    loss = 0.5 * ((xhat - sv) ** 2).sum()
    loss.backward()
    resid = (xhat.detach() - sv).cpu().numpy().astype(np.float64)
    c = coords.cpu().numpy()[t.perm()]
    for n in range(3):
        M, S = oracle.mttkrp(c, resid, spec.dims, to_np64([a.detach() for a in A]), n)
        assert oracle.max_rel_err(A[n].grad.cpu().numpy(), M, S) <= FP32_TOL


# ------------------------------------------------------------ CP-ALS (FP64 pieces)
def test_gram_and_update_match_oracle():
    rng = np.random.default_rng(3)
    R = 16
    A = [torch.from_numpy(rng.standard_normal((d, R)).astype(np.float32)).cuda() for d in (300, 200, 100)]
    G = [torch.empty((R, R), dtype=torch.float64, device="cuda") for _ in A]
    for a, g in zip(A, G):
        blco.blco_gram(a, blco.BLCO_F32, a.shape[0], R, g)
    for a, g in zip(A, G):
        ref = oracle.gram(a.cpu().numpy().astype(np.float64))
        np.testing.assert_allclose(g.cpu().numpy(), ref, rtol=1e-12, atol=1e-9)
    M = torch.from_numpy(rng.standard_normal((300, R)).astype(np.float32)).cuda()
    out = torch.empty_like(M)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    Gn = torch.empty((R, R), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    blco.blco_cpals_update(G, 3, 0, R, M, 300, out, lam, Gn, info)
    V = oracle.gram(A[1].cpu().numpy().astype(np.float64)) * oracle.gram(A[2].cpu().numpy().astype(np.float64))
    ref, rinfo = oracle.cpals.solve_right(M.cpu().numpy().astype(np.float64), V)
    lref = np.linalg.norm(ref, axis=0)
    assert int(info.item()) == rinfo == 0
    np.testing.assert_allclose(lam.cpu().numpy(), lref, rtol=1e-5)
    np.testing.assert_allclose(out.cpu().numpy(), ref / lref, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("R", [1, 5, 8, 33, 64, 128])
def test_gram_float32_pairs_match_fp64(R):
    """Grams of tall factors with a wide dynamic range (entries scaled by
    10^-3..10^3 per row, signs mixed) against the FP64 oracle, normalised by
    sum_i |A[i,r] A[i,c]|: the Dot2 accumulation must stay near 2^-48."""
    rng = np.random.default_rng(R)
    I = 200_003
    A = (rng.standard_normal((I, R)) * 10.0 ** rng.uniform(-3, 3, (I, 1))).astype(np.float32)
    G = torch.empty((R, R), dtype=torch.float64, device="cuda")
    blco.blco_gram(torch.from_numpy(A).cuda(), blco.BLCO_F32, I, R, G)
    A64 = A.astype(np.float64)
    ref = oracle.gram(A64)
    scale = np.abs(A64).T @ np.abs(A64)
    err = np.max(np.abs(G.cpu().numpy() - ref) / scale)
    assert err <= 1e-12, err
    Gh = G.cpu().numpy()
    assert np.max(np.abs(Gh - Gh.T) / scale) <= 1e-13  # symmetric up to the order of the CTA sums


@pytest.mark.parametrize("R,N", [(8, 2), (16, 3), (64, 3)])
def test_update_pseudo_inverse_path(R, N):
    """Two equal columns in every other factor make V singular: the update
    must take the pseudo-inverse branch (info 1) and give the oracle's
    A = M V^+ (normalised columns) and lambda, from the same Grams."""
    rng = np.random.default_rng(4 + R)
    dims = [50 + 10 * k for k in range(N)]
    G = []
    for d in dims:
        a = rng.standard_normal((d, R)).astype(np.float32)
        a[:, 1] = a[:, 0]
        g = torch.empty((R, R), dtype=torch.float64, device="cuda")
        blco.blco_gram(torch.from_numpy(a).cuda(), blco.BLCO_F32, d, R, g)
        G.append(g)
    mode = N - 1
    I = 40
    M = torch.from_numpy(rng.standard_normal((I, R)).astype(np.float32)).cuda()
    out = torch.empty_like(M)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    blco.blco_cpals_update(G, N, mode, R, M, I, out, lam, None, info)
    assert int(info.item()) == 1
    V = np.ones((R, R))
    for k in range(N):
        if k != mode:
            V = V * G[k].cpu().numpy()
    ref, rinfo = oracle.cpals.solve_right(M.cpu().numpy().astype(np.float64), V)
    assert rinfo == 1
    lref = np.linalg.norm(ref, axis=0)
    # V^+ is applied in float32 on the GPU: relative error ~ cond(V restricted to its range) * 2^-24
    np.testing.assert_allclose(lam.cpu().numpy(), lref, rtol=1e-4)
    np.testing.assert_allclose(out.cpu().numpy(), ref / lref, rtol=0, atol=1e-4)


def test_cp_als_tracks_oracle_and_recovers_planted():
    """GPU CP-ALS (float32 MTTKRP, FP64 R x R algebra) against the FP64 oracle
    CP-ALS from the same initial factors: every factor (columns up to sign)
    and lambda after 1, 5 and 20 sweeps, and recovery of the planted model."""
    rng = np.random.default_rng(15)
    dims = (30, 25, 20)
    R = 8
    P = [rng.standard_normal((d, R)) for d in dims]
    import itertools
    c = np.array(list(itertools.product(*[range(d) for d in dims])))
    v = np.einsum("ir,jr,kr->ijk", *P)[tuple(c.T)]
    t = blco.Tensor.build(torch.from_numpy(c.astype(np.int32)).cuda(), torch.from_numpy(v.astype(np.float32)).cuda(),
                          dims)
    init = [rng.standard_normal((d, R)).astype(np.float32) for d in dims]
    v32 = v.astype(np.float32).astype(np.float64)
    for iters in (1, 5, 20):
        A = [torch.from_numpy(a.copy()).cuda() for a in init]
        _, lam, fits = blco.cp_als(t, A, iters=iters)
        rA, rlam, rfits = oracle.cp_als(c, v32, dims, [a.astype(np.float64) for a in init], iters=iters)
        lam = lam.cpu().numpy()
        np.testing.assert_allclose(lam, rlam, rtol=1e-4)
        for n in range(3):
            got = A[n].cpu().numpy().astype(np.float64)
            sign = np.sign(np.sum(got * rA[n], axis=0))
            assert np.all(sign != 0)
            np.testing.assert_allclose(got * sign, rA[n], rtol=0, atol=1e-4)
        assert abs(fits[-1] - rfits[-1]) < 1e-5
    _, _, fits = blco.cp_als(t, [torch.from_numpy(a.copy()).cuda() for a in init], iters=60)
    assert fits[-1] > 0.999
