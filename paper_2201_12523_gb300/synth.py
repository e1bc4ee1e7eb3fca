"""Seeded synthetic inputs shaped like the sparse tensors of the paper's
evaluation (Section 6, Table 2: 3- to 5-mode tensors, 10^5..10^9 nonzeros,
skewed mode lengths and index frequencies, rank around 32).

This module only draws random numbers and removes duplicate coordinates. It
holds none of the method's arithmetic (no linearization, no MTTKRP, no CP
model): both the FP64 oracle and the CUDA path receive exactly the arrays it
returns. Everything is driven by ``torch.Generator`` seeds, on the device the
caller names (CPU for the small cases, the GPU for the large ones, where the
Zipf sampling and de-duplication of up to 10^9 coordinates take seconds).

Recipes (one seed per configuration, ``SEED_BASE + 100 * index``):

* indices ``uniform``: i ~ U{0..I-1};
* indices ``zipf(a)``: rank k in 1..I with P(k) proportional to k^-a (inverse
  CDF over the truncated support), mapped through a seeded random permutation
  of the labels 0..I-1 so that hot indices are scattered over the mode;
* nonzeros are drawn independently per mode, duplicates are removed, more are
  drawn until the target count of distinct coordinates is reached, and a
  seeded random subset of exactly ``nnz`` coordinates is returned in random
  order (a raw COO file has no particular order);
* values ``u01``: U(0,1) float32; ``lognormal``: exp(N(0,1)) float32;
* factor matrices ``u01`` or ``normal``: I_k x R float32, row-major.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import torch

SEED_BASE = 2201_12523


@dataclasses.dataclass(frozen=True)
class TensorSpec:
    """One synthetic workload: shape, index distributions, values, rank."""

    name: str
    dims: Tuple[int, ...]
    nnz: int
    index_dist: Tuple[str, ...]  # per mode: "uniform" or "zipf:<alpha>"
    value_dist: str  # "u01" or "lognormal"
    rank: int
    factor_dist: str  # "u01" or "normal"
    seed: int

    @property
    def order(self) -> int:
        return len(self.dims)

    def scaled(self, nnz: int, dims: Sequence[int], name: Optional[str] = None) -> "TensorSpec":
        """Same recipe at a smaller size (for oracle-sized parity cases). With
        a different number of modes, every mode takes the first mode's index
        distribution."""
        dims = tuple(int(d) for d in dims)
        dist = self.index_dist if len(dims) == len(self.index_dist) else (self.index_dist[0],) * len(dims)
        return dataclasses.replace(self, name=name or f"{self.name}-small", nnz=int(nnz), dims=dims,
                                   index_dist=dist)


def _z(alpha: float, n: int) -> Tuple[str, ...]:
    return tuple(f"zipf:{alpha}" for _ in range(n))


# The five workloads. Factor distributions that a configuration leaves open
# are N(0,1), as for the 3-mode skewed case that states it.
CONFIGS: List[TensorSpec] = [
    TensorSpec("uniform-3d-100k", (1000, 800, 600), 100_000, ("uniform",) * 3, "u01", 16, "u01",
               SEED_BASE + 0),
    TensorSpec("zipf1.2-3d-150M", (1 << 22, 1 << 21, 1 << 11), 150_000_000, _z(1.2, 3), "u01", 32,
               "normal", SEED_BASE + 100),
    TensorSpec("zipf1.1-4d-500M", (1 << 20, 1 << 18, 1 << 16, 1 << 8), 500_000_000, _z(1.1, 4),
               "lognormal", 32, "normal", SEED_BASE + 200),
    TensorSpec("zipf1.2-5d-1B", (1 << 24, 1 << 20, 1 << 16, 1 << 12, 1 << 8), 1_000_000_000,
               _z(1.2, 3) + ("uniform", "uniform"), "u01", 16, "normal", SEED_BASE + 300),
    TensorSpec("cp-planted-3d-200M", (1 << 20, 1 << 20, 1 << 10), 200_000_000, _z(1.2, 3), "u01", 64,
               "u01", SEED_BASE + 400),
]


def generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def _draw_mode(n: int, dim: int, dist: str, gen: torch.Generator, labels: Optional[torch.Tensor],
               cdf: Optional[torch.Tensor], device) -> torch.Tensor:
    """n indices of one mode, int32 (every mode length here is below 2^31)."""
    if dist == "uniform":
        return torch.randint(0, dim, (n,), generator=gen, device=device, dtype=torch.int32)
    out = torch.empty(n, dtype=torch.int32, device=device)
    chunk = 1 << 27
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = torch.rand(b - a, generator=gen, device=device, dtype=torch.float64)
        rank = torch.searchsorted(cdf, u).clamp_(max=dim - 1)
        out[a:b] = labels[rank]
        del u, rank
    return out


def _zipf_tables(dim: int, alpha: float, gen: torch.Generator, device):
    k = torch.arange(1, dim + 1, device=device, dtype=torch.float64)
    cdf = torch.cumsum(k.pow(-alpha), 0)
    cdf /= cdf[-1].clone()
    labels = torch.randperm(dim, generator=gen, device=device).to(torch.int32)
    return labels, cdf


def _dedup_key(idx: torch.Tensor, dims: Sequence[int]) -> List[torch.Tensor]:
    """Integer keys whose joint equality is coordinate equality.

    Modes are packed greedily into int64 words of at most 62 bits each (exact
    mixed-radix packing, no hashing)."""
    words, cur, cur_bits = [], None, 0
    for k, d in enumerate(dims):
        b = max(1, math.ceil(math.log2(d))) if d > 1 else 1
        col = idx[:, k].to(torch.int64)
        if cur is None:
            cur, cur_bits = col, b
        elif cur_bits + b <= 62:
            cur = cur * d + col
            cur_bits += b
        else:
            words.append(cur)
            cur, cur_bits = col, b
    words.append(cur)
    return words


def _unique_rows(idx: torch.Tensor, dims: Sequence[int]) -> torch.Tensor:
    """Rows of ``idx`` with duplicates removed (order: lexicographic by key)."""
    words = _dedup_key(idx, dims)
    order = torch.arange(idx.shape[0], device=idx.device)
    for w in reversed(words):  # LSD: stable sorts, least significant word first
        _, o = torch.sort(w[order], stable=True)
        order = order[o]
    keep = torch.ones(order.shape[0], dtype=torch.bool, device=idx.device)
    if order.shape[0] > 1:
        diff = torch.zeros(order.shape[0] - 1, dtype=torch.bool, device=idx.device)
        for w in words:
            ws = w[order]
            diff |= ws[1:] != ws[:-1]
        keep[1:] = diff
    return idx[order[keep]]


def coordinates(spec: TensorSpec, device="cpu", oversample: float = 1.15) -> torch.Tensor:
    """``spec.nnz`` distinct coordinates, int32 (nnz x N), random order."""
    device = torch.device(device)
    gen = generator(spec.seed, device)
    tables = []
    for d, dist in zip(spec.dims, spec.index_dist):
        if dist.startswith("zipf:"):
            tables.append(_zipf_tables(d, float(dist.split(":")[1]), gen, device))
        else:
            tables.append((None, None))
    total = 1
    for d in spec.dims:
        total *= d
    if spec.nnz > total:
        raise ValueError("more nonzeros requested than the tensor has cells")
    have = torch.empty((0, spec.order), dtype=torch.int32, device=device)
    want = int(spec.nnz * oversample) + 1024
    for _ in range(64):
        cols = [_draw_mode(want, d, dist, gen, lab, cdf, device)
                for d, dist, (lab, cdf) in zip(spec.dims, spec.index_dist, tables)]
        fresh = torch.stack(cols, 1)
        del cols
        before = have.shape[0]
        have = _unique_rows(torch.cat([have, fresh], 0), spec.dims)
        del fresh
        if have.shape[0] >= spec.nnz:
            break
        # draw enough for the missing count at this round's yield of new coordinates
        missing = spec.nnz - have.shape[0]
        gained = (have.shape[0] - before) / max(1, want)
        want = int(missing / max(gained, 0.01) * 1.3) + 1024
    else:  # pragma: no cover - only for absurd specs
        raise RuntimeError("could not draw enough distinct coordinates")
    pick = torch.randperm(have.shape[0], generator=gen, device=device)[: spec.nnz]
    return have[pick].to(torch.int32).contiguous()


def values(spec: TensorSpec, device="cpu") -> torch.Tensor:
    """``spec.nnz`` float32 values (stream independent of the coordinates)."""
    device = torch.device(device)
    gen = generator(spec.seed + 1, device)
    if spec.value_dist == "u01":
        return torch.rand(spec.nnz, generator=gen, device=device, dtype=torch.float32)
    if spec.value_dist == "lognormal":
        z = torch.randn(spec.nnz, generator=gen, device=device, dtype=torch.float32)
        return torch.exp(z)
    raise ValueError(spec.value_dist)


def factors(spec: TensorSpec, rank: Optional[int] = None, device="cpu", stream: int = 0,
            dist: Optional[str] = None) -> List[torch.Tensor]:
    """Random float32 factor matrices A_k (I_k x R, row-major)."""
    device = torch.device(device)
    R = int(rank or spec.rank)
    dist = dist or spec.factor_dist
    gen = generator(spec.seed + 2 + 7 * stream, device)
    out = []
    for d in spec.dims:
        if dist == "u01":
            out.append(torch.rand((d, R), generator=gen, device=device, dtype=torch.float32))
        elif dist == "normal":
            out.append(torch.randn((d, R), generator=gen, device=device, dtype=torch.float32))
        else:
            raise ValueError(dist)
    return out


def noise(n: int, sigma: float, seed: int, device="cpu") -> torch.Tensor:
    """N(0, sigma^2) float32 draws (additive noise of a planted model)."""
    gen = generator(seed, torch.device(device))
    return sigma * torch.randn(n, generator=gen, device=torch.device(device), dtype=torch.float32)


def workload(name: str) -> TensorSpec:
    """The workload of that name (e.g. "zipf1.1-4d-500M")."""
    for spec in CONFIGS:
        if spec.name == name:
            return spec
    raise KeyError(name)


def small(index: int, nnz: int, dims: Sequence[int]) -> TensorSpec:
    """Configuration ``index``'s recipe at an oracle-sized shape."""
    return CONFIGS[index].scaled(nnz, dims)
