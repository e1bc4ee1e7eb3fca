"""The compulsory-bytes counts behind bench.py's roofline fractions, pinned to
their closed forms on the benchmark workloads (CPU only).

One mode-n MTTKRP launch must read the key/value stream once (8 + 4 bytes per
nonzero), every other factor matrix once and write the float32 output once;
the one-pass all-mode launch reads the stream once, every factor once and
writes every output once."""

import bench
from paper_2201_12523_gb300 import synth


def test_per_mode_bytes_are_mode_independent_with_float32_factors():
    # 12 nnz + 4 R sum_k I_k for every mode: the output of mode n replaces
    # the factor of mode n, both float32
    for name in ("zipf1.2-3d-150M", "zipf1.1-4d-500M"):
        spec = synth.workload(name)
        R = spec.rank
        closed = 12 * spec.nnz + 4 * R * sum(spec.dims)
        for n in range(spec.order):
            assert bench.algorithmic_bytes(spec, R, 4, n) == closed


def test_per_mode_bytes_of_the_headline_workloads():
    c2 = synth.workload("zipf1.2-3d-150M")
    assert bench.algorithmic_bytes(c2, 32, 4, 0) == 12 * 150_000_000 + 4 * 32 * ((1 << 22) + (1 << 21) + (1 << 11))
    assert bench.algorithmic_bytes(c2, 32, 4, 0) == 2_605_568_512
    c3 = synth.workload("zipf1.1-4d-500M")
    assert bench.algorithmic_bytes(c3, 32, 4, 3) == 6_176_193_536


def test_16bit_factors_halve_only_the_gathered_factor_term():
    spec = synth.workload("zipf1.1-4d-500M")
    R = spec.rank
    for n in range(spec.order):
        b32 = bench.algorithmic_bytes(spec, R, 4, n)
        b16 = bench.algorithmic_bytes(spec, R, 2, n)
        gathered = sum(d for k, d in enumerate(spec.dims) if k != n) * R
        assert b32 - b16 == 2 * gathered


def test_touched_rows_count_is_the_stricter_one():
    spec = synth.workload("zipf1.2-3d-150M")
    rows = [d // 2 for d in spec.dims]
    for n in range(spec.order):
        assert bench.algorithmic_bytes(spec, 32, 4, n, rows) < bench.algorithmic_bytes(spec, 32, 4, n)
    assert bench.algorithmic_bytes(spec, 32, 4, 0, list(spec.dims)) == bench.algorithmic_bytes(spec, 32, 4, 0)


def test_one_pass_bytes_of_the_five_mode_workload():
    spec = synth.workload("zipf1.2-5d-1B")
    R = spec.rank
    assert bench.onepass_bytes(spec, R, 4) == 12 * spec.nnz + 8 * R * sum(spec.dims)
    assert bench.onepass_bytes(spec, R, 4) == 14_290_647_040
    # every factor read once and every output written once, against N
    # per-mode launches that read the stream N times
    per_mode = sum(bench.algorithmic_bytes(spec, R, 4, n) for n in range(spec.order))
    assert per_mode - bench.onepass_bytes(spec, R, 4) == (spec.order - 1) * 12 * spec.nnz + \
        (spec.order - 2) * 4 * R * sum(spec.dims)
