"""FP64 CPU oracle for the BLCO sparse-MTTKRP path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package. The product
(``paper_2201_12523_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C loops, FP64),
compiled on first use with gcc into ``liboracle.so`` next to it; this module
marshals numpy arrays and adds the CP-ALS driver of Algorithm 1 in FP64
numpy (``cpals.py``). Each function cites the passage of the paper it
follows; the file header of ``oracle.c`` lists them.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against something other than itself (the worked example of Fig. 4a/6, dense
brute force of Eq. 1, closed forms, a recursive-partition comparator, torch's
bfloat16 rounding, finite differences, planted-model recovery).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no GPU involved; with
    OpenMP when the compiler has it, else single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        _lib.orc_alto_layout.restype = ctypes.c_int
        _lib.orc_alto_layout.argtypes = [ctypes.c_int, vp, vp, vp, vp]
        _lib.orc_alto_keys.restype = ctypes.c_int64
        _lib.orc_alto_keys.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, vp]
        _lib.orc_build_store.restype = ctypes.c_int64
        _lib.orc_build_store.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                         ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp, vp]
        _lib.orc_check_store.restype = ctypes.c_int64
        _lib.orc_check_store.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                         ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp]
        _lib.orc_check_store_at.restype = ctypes.c_int64
        _lib.orc_check_store_at.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, ctypes.c_int,
                                            ctypes.c_int64, vp, vp, vp, ctypes.c_int64, vp, vp,
                                            ctypes.c_int64, vp]
        _lib.orc_is_permutation.restype = ctypes.c_int
        _lib.orc_is_permutation.argtypes = [ctypes.c_int64, vp]
        _lib.orc_mttkrp.restype = None
        _lib.orc_mttkrp.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, ctypes.c_int, vp,
                                    ctypes.c_int, vp, vp]
        _lib.orc_mttkrp_rows.restype = None
        _lib.orc_mttkrp_rows.argtypes = [ctypes.c_int64, ctypes.c_int, vp, vp, vp, ctypes.c_int, vp,
                                         ctypes.c_int, vp, ctypes.c_int64, vp, vp]
        _lib.orc_cp_model.restype = None
        _lib.orc_cp_model.argtypes = [ctypes.c_int64, ctypes.c_int, vp, ctypes.c_int, vp, vp]
        _lib.orc_bf16_rne.restype = None
        _lib.orc_bf16_rne.argtypes = [ctypes.c_int64, vp, vp]
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _coords(coords) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(coords))
    if c.ndim != 2:
        raise ValueError("coords must be nnz x N")
    return np.ascontiguousarray(c.astype(np.uint32, copy=False))


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _factor_table(factors: Sequence[Optional[np.ndarray]], R: int, dims) -> Tuple[object, List[np.ndarray]]:
    keep = []
    arr = (ctypes.c_void_p * len(factors))()
    for k, f in enumerate(factors):
        if f is None:
            f = np.zeros((1, R))
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        if f.ndim != 2 or f.shape[1] != R:
            raise ValueError("factor %d must be I_k x R" % k)
        keep.append(f)
        arr[k] = f.ctypes.data
    return arr, keep


# --------------------------------------------------------------------------
# Section 4.1: linearization
# --------------------------------------------------------------------------
def alto_layout(dims) -> Tuple[List[int], List[Tuple[int, int]]]:
    """(b_n per mode, [(mode, level) for key bits 0..B-1]) -- Section 4.1, Fig. 6a."""
    d = _dims(dims)
    N = d.shape[0]
    bits = np.zeros(N, np.int32)
    km = np.zeros(128, np.int32)
    kl = np.zeros(128, np.int32)
    B = _load().orc_alto_layout(N, _p(d), _p(bits), _p(km), _p(kl))
    if B < 0:
        raise ValueError("bad dims")
    return bits.tolist(), list(zip(km[:B].tolist(), kl[:B].tolist()))


def alto_keys(coords, dims) -> Tuple[np.ndarray, np.ndarray]:
    """Linear index of every coordinate as (hi, lo) uint64 words."""
    c = _coords(coords)
    d = _dims(dims)
    hi = np.zeros(c.shape[0], np.uint64)
    lo = np.zeros(c.shape[0], np.uint64)
    rc = _load().orc_alto_keys(c.shape[0], c.shape[1], _p(c), _p(d), _p(hi), _p(lo))
    if rc != 0:
        raise ValueError("coordinate out of range or bad dims (code %d)" % rc)
    return hi, lo


def alto_keys_int(coords, dims) -> List[int]:
    hi, lo = alto_keys(coords, dims)
    return [(int(h) << 64) | int(l) for h, l in zip(hi, lo)]


# --------------------------------------------------------------------------
# Section 4.2: blocking and re-encoding
# --------------------------------------------------------------------------
class Store:
    """The BLCO store the definition gives for a COO tensor."""

    def __init__(self, keys, vals, perm, bstart, bhigh):
        self.keys, self.svals, self.perm, self.bstart, self.bhigh = keys, vals, perm, bstart, bhigh

    @property
    def nblocks(self) -> int:
        return int(self.bstart.shape[0] - 1)


def build_store(coords, vals, dims, line_bits: int = 64, max_nnz: int = 1 << 27) -> Store:
    c = _coords(coords)
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float32))
    d = _dims(dims)
    nnz, N = c.shape
    keys = np.zeros(nnz, np.uint64)
    svals = np.zeros(nnz, np.float32)
    perm = np.zeros(nnz, np.int64)
    cap = nnz + 1
    bstart = np.zeros(cap + 1, np.int64)
    bhigh = np.zeros(cap * N + 1, np.uint32)
    nb = np.zeros(1, np.int64)
    rc = _load().orc_build_store(nnz, N, _p(c), _p(v), _p(d), int(line_bits), int(max_nnz),
                                 _p(keys), _p(svals), _p(perm), cap, _p(nb), _p(bstart), _p(bhigh))
    if rc != 0:
        raise ValueError("build_store failed (code %d)" % rc)
    n = int(nb[0])
    return Store(keys, svals, perm, bstart[: n + 1].copy(), bhigh[: n * N].reshape(n, N).copy())


def check_store(coords, vals, dims, line_bits, max_nnz, keys, svals, perm, bstart, bhigh) -> int:
    """0 if the given store equals the defined one, else a nonzero code."""
    c = _coords(coords)
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float32))
    d = _dims(dims)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
    svals = np.ascontiguousarray(np.asarray(svals, dtype=np.float32))
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int64))
    bstart = np.ascontiguousarray(np.asarray(bstart, dtype=np.int64))
    bhigh = np.ascontiguousarray(np.asarray(bhigh, dtype=np.uint32))
    return int(_load().orc_check_store(c.shape[0], c.shape[1], _p(c), _p(v), _p(d), int(line_bits),
                                       int(max_nnz), _p(keys), _p(svals), _p(perm),
                                       bstart.shape[0] - 1, _p(bstart), _p(bhigh)))


def check_store_at(coords, vals, dims, line_bits, max_nnz, keys, svals, perm, bstart, bhigh, positions) -> int:
    """The checks of check_store at the given store positions only (0 = pass)."""
    c = _coords(coords)
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float32))
    d = _dims(dims)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
    svals = np.ascontiguousarray(np.asarray(svals, dtype=np.float32))
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int64))
    bstart = np.ascontiguousarray(np.asarray(bstart, dtype=np.int64))
    bhigh = np.ascontiguousarray(np.asarray(bhigh, dtype=np.uint32))
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int64))
    return int(_load().orc_check_store_at(c.shape[0], c.shape[1], _p(c), _p(v), _p(d), int(line_bits),
                                          int(max_nnz), _p(keys), _p(svals), _p(perm), bstart.shape[0] - 1,
                                          _p(bstart), _p(bhigh), pos.shape[0], _p(pos)))


def is_permutation(perm) -> bool:
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.int64))
    return _load().orc_is_permutation(p.shape[0], _p(p)) == 1


# --------------------------------------------------------------------------
# Eq. 1 / Fig. 3: MTTKRP, and the CP model
# --------------------------------------------------------------------------
def mttkrp(coords, vals, dims, factors, mode: int) -> Tuple[np.ndarray, np.ndarray]:
    """(M, S): M = X_(n) (KRP of the other factors), S = sum |terms| (FP64)."""
    c = _coords(coords)
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
    d = _dims(dims)
    R = int(np.asarray(factors[(mode + 1) % len(factors)]).shape[1])
    arr, keep = _factor_table(factors, R, d)
    M = np.zeros((int(d[mode]), R))
    S = np.zeros((int(d[mode]), R))
    _load().orc_mttkrp(c.shape[0], c.shape[1], _p(c), _p(v), _p(d), R, arr, int(mode), _p(M), _p(S))
    return M, S


def mttkrp_rows(coords, vals, dims, factors, mode: int, rows) -> Tuple[np.ndarray, np.ndarray]:
    """MTTKRP and S for the listed output rows only (returned in the order given)."""
    c = _coords(coords)
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
    d = _dims(dims)
    rows = np.asarray(rows, dtype=np.int64)
    order = np.argsort(rows, kind="stable")
    srt = np.ascontiguousarray(rows[order])
    if srt.size and np.any(srt[1:] == srt[:-1]):
        raise ValueError("rows must be distinct")
    R = int(np.asarray(factors[(mode + 1) % len(factors)]).shape[1])
    arr, keep = _factor_table(factors, R, d)
    M = np.zeros((rows.shape[0], R))
    S = np.zeros((rows.shape[0], R))
    _load().orc_mttkrp_rows(c.shape[0], c.shape[1], _p(c), _p(v), _p(d), R, arr, int(mode),
                            _p(srt), srt.shape[0], _p(M), _p(S))
    out_M = np.empty_like(M)
    out_S = np.empty_like(S)
    out_M[order] = M
    out_S[order] = S
    return out_M, out_S


def cp_model(coords, factors) -> np.ndarray:
    """xhat_j = sum_r prod_n A_n[i_n^j, r] at every listed coordinate (FP64)."""
    c = _coords(coords)
    R = int(np.asarray(factors[0]).shape[1])
    arr, keep = _factor_table(factors, R, None)
    out = np.zeros(c.shape[0])
    _load().orc_cp_model(c.shape[0], c.shape[1], _p(c), R, arr, _p(out))
    return out


def bf16_round(x) -> np.ndarray:
    """float32 array rounded to bfloat16 (nearest-even), returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.empty_like(a)
    _load().orc_bf16_rne(a.size, _p(a), _p(y))
    return y


def max_rel_err(M_test, M_ref, S_ref) -> float:
    """max |M_test - M_ref| / S over entries with S > 0; entries with S == 0
    must be exactly zero in M_test (returns inf otherwise)."""
    M_test = np.asarray(M_test, dtype=np.float64)
    diff = np.abs(M_test - M_ref)
    zero = S_ref == 0
    if np.any(M_test[zero] != 0):
        return float("inf")
    if not np.any(~zero):
        return 0.0
    return float(np.max(diff[~zero] / S_ref[~zero]))


from .cpals import cp_als, gram, fit_of, solve_right, pinv_sym, cholesky_lower, pd_tolerance  # noqa: E402,F401
