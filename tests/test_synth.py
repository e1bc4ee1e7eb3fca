"""The seeded input generators (CPU): exact counts, distinct in-range
coordinates, determinism, and the skew the Zipf recipe promises."""

import numpy as np
import pytest
import torch

from paper_2201_12523_gb300 import synth


@pytest.mark.parametrize("idx,nnz,dims", [(0, 20000, (100, 80, 60)), (1, 50000, (1 << 12, 1 << 11, 1 << 5)),
                                         (2, 40000, (1 << 10, 1 << 9, 1 << 8, 16)),
                                         (3, 30000, (1 << 12, 1 << 10, 1 << 8, 64, 16)),
                                         (4, 30000, (1 << 11, 1 << 11, 1 << 6))])
def test_coordinates_distinct_in_range(idx, nnz, dims):
    spec = synth.small(idx, nnz, dims)
    c = synth.coordinates(spec)
    assert c.shape == (nnz, len(dims)) and c.dtype == torch.int32
    a = c.numpy().astype(np.int64)
    for n, d in enumerate(dims):
        assert a[:, n].min() >= 0 and a[:, n].max() < d
    assert np.unique(a, axis=0).shape[0] == nnz
    c2 = synth.coordinates(spec)
    assert torch.equal(c, c2)  # seeded


def test_zipf_skew_and_label_permutation():
    spec = synth.small(1, 100000, (1 << 14, 1 << 13, 1 << 7))
    c = synth.coordinates(spec).numpy()
    counts = np.bincount(c[:, 0], minlength=1 << 14)
    top = np.sort(counts)[::-1]
    # Zipf(1.2): the heaviest index carries a large share, far above uniform
    assert top[0] > 50 * counts.mean()
    # labels are permuted: the heaviest index is not simply label 0
    assert int(np.argmax(counts)) != 0


def test_values_and_factors():
    spec = synth.small(2, 5000, (64, 32, 16, 8))
    v = synth.values(spec)
    assert v.shape == (5000,) and v.dtype == torch.float32 and bool((v > 0).all())
    f = synth.factors(spec)
    assert [tuple(x.shape) for x in f] == [(64, 32), (32, 32), (16, 32), (8, 32)]
    assert torch.equal(f[0], synth.factors(spec)[0])
    assert not torch.equal(f[0], synth.factors(spec, stream=1)[0])
