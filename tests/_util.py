"""Shared helpers for the GPU parity tests: run the library and the FP64
oracle on the same seeded inputs and compare."""

from typing import List, Sequence

import numpy as np
import torch

import oracle
from paper_2201_12523_gb300 import synth

FP32_TOL = 1e-5       # max |M - M_ref| / S for float32 factors
BF16_TOL = 1e-2       # against the oracle on the unrounded float32 factors
CP_TOL = 1e-5         # CP model value, normalized by sum_r |prod|


def to_np64(ts: Sequence[torch.Tensor]) -> List[np.ndarray]:
    return [t.detach().cpu().float().numpy().astype(np.float64) for t in ts]


def rounded16(A: Sequence[torch.Tensor], dtype) -> List[np.ndarray]:
    """Factors as the 16-bit kernel sees them (float64 of the rounded values).
    bfloat16 uses the oracle's own rounding; float16 uses numpy's IEEE cast."""
    out = []
    for a in A:
        x = a.detach().cpu().numpy().astype(np.float32)
        if dtype == torch.bfloat16:
            out.append(oracle.bf16_round(x).astype(np.float64))
        else:
            out.append(x.astype(np.float16).astype(np.float64))
    return out


def make(spec: synth.TensorSpec, device="cuda"):
    coords = synth.coordinates(spec, device=device)
    vals = synth.values(spec, device=device)
    A = synth.factors(spec, device=device)
    return coords, vals, A


def check_mttkrp_all(t, coords, vals, A, dims, tol=FP32_TOL, factors_ref=None, modes=None):
    """Runs blco MTTKRP for every mode and compares with the oracle."""
    c = coords.cpu().numpy()
    v = vals.cpu().numpy().astype(np.float64)
    Af = factors_ref if factors_ref is not None else to_np64(A)
    errs = []
    for n in (modes if modes is not None else range(len(dims))):
        out = t.mttkrp(n, A)
        torch.cuda.synchronize()
        M, S = oracle.mttkrp(c, v, dims, Af, n)
        err = oracle.max_rel_err(out.cpu().numpy(), M, S)
        errs.append(err)
        assert err <= tol, f"mode {n}: max rel err {err:.3e} > {tol:.1e}"
    return errs
