"""Python binding of libblco.so (include/blco.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels. torch is used for device memory, streams and autograd plumbing.
The ``blco_*`` functions mirror the C entry points one to one; ``Tensor``,
``SparseCP`` and ``cp_als`` are thin conveniences built on them.

Importing this module loads ``libblco.so`` from this package directory and
raises ``ImportError`` if it is missing: there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblco.so")
MAX_MODES = 8

BLCO_OK, BLCO_ERR_ARG, BLCO_ERR_INDEX, BLCO_ERR_OOM, BLCO_ERR_CUDA, BLCO_ERR_TIMEOUT, BLCO_ERR_STATE, \
    BLCO_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["BLCO_OK", "BLCO_ERR_ARG", "BLCO_ERR_INDEX", "BLCO_ERR_OOM", "BLCO_ERR_CUDA", "BLCO_ERR_TIMEOUT",
                "BLCO_ERR_STATE", "BLCO_ERR_UNSUPPORTED"]
BLCO_F32, BLCO_BF16, BLCO_F16 = 0, 1, 2
BLCO_FAULT_ALLOC, BLCO_FAULT_COPY = 1, 2
_DTYPE_CODE = {torch.float32: BLCO_F32, torch.bfloat16: BLCO_BF16, torch.float16: BLCO_F16}

# Every symbol include/blco.h declares (checked by the test suite).
EXPORTS = ["blco_default_opts", "blco_build", "blco_mttkrp", "blco_mttkrp_all", "blco_cp_fwd", "blco_cp_bwd",
           "blco_values", "blco_perm", "blco_keys", "blco_blocks", "blco_info", "blco_sync", "blco_destroy",
           "blco_last_error", "blco_convert", "blco_gram", "blco_cpals_update", "blco_cpals_fit", "blco_norm2",
           "blco_profile_enable", "blco_profile_read", "blco_cpals_update_noalloc", "blco_inject_fault",
           "blco_partition", "blco_mttkrp_range", "blco_build_f64", "blco_mttkrp_f64"]


class BuildOpts(ctypes.Structure):
    _fields_ = [("max_nnz_per_block", ctypes.c_int64), ("line_bits", ctypes.c_int32), ("n_queues", ctypes.c_int32),
                ("device_budget_bytes", ctypes.c_int64), ("force_stream", ctypes.c_int32),
                ("compensated_sums", ctypes.c_int32), ("host_reads", ctypes.c_int32)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("order", ctypes.c_int32), ("total_bits", ctypes.c_int32),
                ("dims", ctypes.c_int64 * MAX_MODES), ("mode_bits", ctypes.c_int32 * MAX_MODES),
                ("block_bits", ctypes.c_int32 * MAX_MODES), ("line_bits", ctypes.c_int32),
                ("streamed", ctypes.c_int32), ("nblocks", ctypes.c_int64), ("max_nnz_per_block", ctypes.c_int64),
                ("queue_nnz", ctypes.c_int64), ("n_queues", ctypes.c_int32),
                ("hot_rows", ctypes.c_int32 * MAX_MODES), ("device_bytes", ctypes.c_int64),
                ("host_bytes", ctypes.c_int64), ("host_reads", ctypes.c_int32)]

    def as_dict(self) -> dict:
        N = self.order
        return {"nnz": self.nnz, "order": N, "total_bits": self.total_bits, "dims": list(self.dims[:N]),
                "mode_bits": list(self.mode_bits[:N]), "block_bits": list(self.block_bits[:N]),
                "line_bits": self.line_bits, "streamed": bool(self.streamed), "nblocks": self.nblocks,
                "max_nnz_per_block": self.max_nnz_per_block, "queue_nnz": self.queue_nnz,
                "n_queues": self.n_queues, "hot_rows": list(self.hot_rows[:N]),
                "device_bytes": self.device_bytes, "host_bytes": self.host_bytes,
                "host_reads": bool(self.host_reads)}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libblco.so not built ({LIB_PATH}); run python -m paper_2201_12523_gb300.build_lib")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "blco_default_opts": [vp],
        "blco_build": [vp, vp, i64, vp, i32, vp, vp, vp],
        "blco_mttkrp": [vp, i32, vp, i32, i32, vp, vp],
        "blco_mttkrp_all": [vp, vp, i32, i32, vp, vp],
        "blco_partition": [i64, i32, vp],
        "blco_build_f64": [vp, vp, i64, vp, i32, vp, vp, vp],
        "blco_mttkrp_f64": [vp, i32, vp, i32, vp, vp],
        "blco_mttkrp_range": [vp, i32, i64, i64, vp, i32, i32, vp, vp],
        "blco_cp_fwd": [vp, vp, i32, i32, vp, vp],
        "blco_cp_bwd": [vp, i32, vp, vp, i32, i32, vp, vp],
        "blco_values": [vp, vp, vp],
        "blco_perm": [vp, vp, vp],
        "blco_keys": [vp, vp, vp],
        "blco_blocks": [vp, vp, vp],
        "blco_info": [vp, vp],
        "blco_sync": [vp],
        "blco_convert": [vp, vp, i32, i64, vp],
        "blco_gram": [vp, i32, i64, i32, vp, vp],
        "blco_cpals_update": [vp, i32, i32, i32, vp, i64, vp, vp, vp, vp, vp],
        "blco_cpals_update_noalloc": [vp, i32, i32, i32, vp, i64, vp, vp, vp, vp, vp],
        "blco_cpals_fit": [ctypes.c_double, vp, i32, i32, vp, vp, vp, i64, vp, vp],
        "blco_norm2": [vp, vp, vp],
        "blco_profile_enable": [vp, i32],
        "blco_profile_read": [vp, vp, i32, vp],
        "blco_inject_fault": [i32, i64],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.blco_destroy.argtypes = [vp]
    lib.blco_destroy.restype = None
    lib.blco_last_error.argtypes = []
    lib.blco_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


class BlcoError(RuntimeError):
    def __init__(self, call: str, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{call}: {name}: {message}")


def _check(call: str, status: int):
    if status != BLCO_OK:
        raise BlcoError(call, status, (_lib.blco_last_error() or b"").decode())


def lib():
    return _lib


# --------------------------------------------------------------- marshalling
def _ptr(x) -> Optional[int]:
    """Address of a torch tensor / numpy array (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libblco must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libblco must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported argument type {type(x)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr_array(xs: Sequence) -> ctypes.Array:
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def _fdt(factors: Sequence) -> int:
    for f in factors:
        if f is not None:
            dt = f.dtype if isinstance(f, torch.Tensor) else {np.dtype(np.float32): torch.float32,
                                                               np.dtype(np.float16): torch.float16}[f.dtype]
            return _DTYPE_CODE[dt]
    raise ValueError("no factor given")


def _rank(factors: Sequence) -> int:
    for f in factors:
        if f is not None:
            return int(f.shape[1])
    raise ValueError("no factor given")


# ------------------------------------------------------- C entry points
def blco_default_opts() -> BuildOpts:
    o = BuildOpts()
    _check("blco_default_opts", _lib.blco_default_opts(ctypes.byref(o)))
    return o


def blco_build(coords, vals, dims: Sequence[int], opts: Optional[BuildOpts] = None, stream=None) -> ctypes.c_void_p:
    nnz = int(coords.shape[0])
    N = len(dims)
    d = (ctypes.c_int64 * N)(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    st = _lib.blco_build(_ptr(coords), _ptr(vals), nnz, d, N, ctypes.byref(opts) if opts is not None else None,
                         _stream(stream), ctypes.byref(h))
    _check("blco_build", st)
    return h


def blco_build_f64(coords, vals, dims: Sequence[int], opts: Optional[BuildOpts] = None, stream=None) -> ctypes.c_void_p:
    nnz = int(coords.shape[0])
    N = len(dims)
    d = (ctypes.c_int64 * N)(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    st = _lib.blco_build_f64(_ptr(coords), _ptr(vals), nnz, d, N, ctypes.byref(opts) if opts is not None else None,
                             _stream(stream), ctypes.byref(h))
    _check("blco_build_f64", st)
    return h


def blco_mttkrp_f64(h, mode: int, factors: Sequence, R: int, out, stream=None):
    _check("blco_mttkrp_f64", _lib.blco_mttkrp_f64(h, int(mode), _ptr_array(factors), int(R), _ptr(out),
                                                   _stream(stream)))


def blco_mttkrp(h, mode: int, factors: Sequence, fdt: int, R: int, out, stream=None):
    _check("blco_mttkrp", _lib.blco_mttkrp(h, int(mode), _ptr_array(factors), int(fdt), int(R), _ptr(out),
                                           _stream(stream)))


def blco_mttkrp_all(h, factors: Sequence, fdt: int, R: int, outs: Sequence, stream=None):
    _check("blco_mttkrp_all", _lib.blco_mttkrp_all(h, _ptr_array(factors), int(fdt), int(R), _ptr_array(outs),
                                                   _stream(stream)))


def blco_partition(nnz: int, nparts: int) -> np.ndarray:
    """Bounds (nparts + 1 store positions) of equal contiguous parts of a store of nnz nonzeros."""
    b = np.zeros(int(nparts) + 1, dtype=np.int64)
    _check("blco_partition", _lib.blco_partition(int(nnz), int(nparts), b.ctypes.data))
    return b


def blco_mttkrp_range(h, mode: int, begin: int, end: int, factors: Sequence, fdt: int, R: int, out, stream=None):
    _check("blco_mttkrp_range", _lib.blco_mttkrp_range(h, int(mode), int(begin), int(end), _ptr_array(factors),
                                                       int(fdt), int(R), _ptr(out), _stream(stream)))


def blco_cp_fwd(h, factors: Sequence, fdt: int, R: int, xhat, stream=None):
    _check("blco_cp_fwd", _lib.blco_cp_fwd(h, _ptr_array(factors), int(fdt), int(R), _ptr(xhat), _stream(stream)))


def blco_cp_bwd(h, mode: int, grad, factors: Sequence, fdt: int, R: int, out, stream=None):
    _check("blco_cp_bwd", _lib.blco_cp_bwd(h, int(mode), _ptr(grad), _ptr_array(factors), int(fdt), int(R),
                                           _ptr(out), _stream(stream)))


def blco_values(h, vals, stream=None):
    _check("blco_values", _lib.blco_values(h, _ptr(vals), _stream(stream)))


def blco_perm(h, perm, stream=None):
    _check("blco_perm", _lib.blco_perm(h, _ptr(perm), _stream(stream)))


def blco_keys(h, keys, stream=None):
    _check("blco_keys", _lib.blco_keys(h, _ptr(keys), _stream(stream)))


def blco_blocks(h, bstart, bhigh):
    _check("blco_blocks", _lib.blco_blocks(h, _ptr(bstart), _ptr(bhigh)))


def blco_info(h) -> Info:
    info = Info()
    _check("blco_info", _lib.blco_info(h, ctypes.byref(info)))
    return info


def blco_sync(h):
    _check("blco_sync", _lib.blco_sync(h))


def blco_destroy(h):
    _lib.blco_destroy(h)


def blco_convert(src, dst, dt: int, n: int, stream=None):
    _check("blco_convert", _lib.blco_convert(_ptr(src), _ptr(dst), int(dt), int(n), _stream(stream)))


def blco_gram(A, fdt: int, I: int, R: int, G, stream=None):
    _check("blco_gram", _lib.blco_gram(_ptr(A), int(fdt), int(I), int(R), _ptr(G), _stream(stream)))


def blco_cpals_update(grams: Sequence, N: int, mode: int, R: int, M, I: int, A, lam, G_out, info, stream=None):
    _check("blco_cpals_update", _lib.blco_cpals_update(_ptr_array(grams), int(N), int(mode), int(R), _ptr(M),
                                                       int(I), _ptr(A), _ptr(lam), _ptr(G_out), _ptr(info),
                                                       _stream(stream)))


def blco_cpals_update_noalloc(grams: Sequence, N: int, mode: int, R: int, M, I: int, A, lam, G_out, info,
                              stream=None):
    """blco_cpals_update without any device allocation (fixed library
    scratch, R <= 64); for callers that cannot let the library allocate."""
    _check("blco_cpals_update_noalloc",
           _lib.blco_cpals_update_noalloc(_ptr_array(grams), int(N), int(mode), int(R), _ptr(M), int(I), _ptr(A),
                                          _ptr(lam), _ptr(G_out), _ptr(info), _stream(stream)))


def blco_cpals_fit(normX2: float, grams: Sequence, N: int, R: int, lam, M_last, A_last, I_last: int, fit,
                   stream=None):
    _check("blco_cpals_fit", _lib.blco_cpals_fit(float(normX2), _ptr_array(grams), int(N), int(R), _ptr(lam),
                                                 _ptr(M_last), _ptr(A_last), int(I_last), _ptr(fit),
                                                 _stream(stream)))


def blco_norm2(h, out, stream=None):
    _check("blco_norm2", _lib.blco_norm2(h, _ptr(out), _stream(stream)))


def blco_profile_enable(h, enable: bool):
    _check("blco_profile_enable", _lib.blco_profile_enable(h, 1 if enable else 0))


def blco_inject_fault(kind: int, k: int):
    """Arm the k-th next event of `kind` (BLCO_FAULT_ALLOC / BLCO_FAULT_COPY)
    to fail on the host; 0 disarms."""
    _check("blco_inject_fault", _lib.blco_inject_fault(kind, k))


def blco_profile_read(h) -> dict:
    """{kernel kind: (launches, total_ms)} recorded since the last read."""
    cap = 16
    arr = (ProfileEntry * cap)()
    n = ctypes.c_int(0)
    _check("blco_profile_read", _lib.blco_profile_read(h, arr, cap, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


# ------------------------------------------------------------ conveniences
class Tensor:
    """A BLCO store on the current CUDA device (owns one handle)."""

    def __init__(self, handle, dims: Sequence[int]):
        self._h = handle
        self.dims = tuple(int(d) for d in dims)

    @classmethod
    def build(cls, coords, vals, dims: Sequence[int], *, max_nnz_per_block: int = 0, line_bits: int = 0,
              n_queues: int = 0, device_budget_bytes: int = 0, force_stream: bool = False,
              compensated_sums: bool = False, host_reads: bool = False, stream=None) -> "Tensor":
        o = blco_default_opts()
        if max_nnz_per_block:
            o.max_nnz_per_block = int(max_nnz_per_block)
        if line_bits:
            o.line_bits = int(line_bits)
        if n_queues:
            o.n_queues = int(n_queues)
        o.device_budget_bytes = int(device_budget_bytes)
        o.force_stream = 1 if force_stream else 0
        o.compensated_sums = 1 if compensated_sums else 0
        o.host_reads = 1 if host_reads else 0
        if getattr(vals, "dtype", None) in (torch.float64, np.float64):
            return cls(blco_build_f64(coords, vals, dims, o, stream), dims)
        return cls(blco_build(coords, vals, dims, o, stream), dims)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("tensor was destroyed")
        return self._h

    @property
    def order(self) -> int:
        return len(self.dims)

    def info(self) -> dict:
        return blco_info(self.handle).as_dict()

    @property
    def nnz(self) -> int:
        return int(blco_info(self.handle).nnz)

    def mttkrp(self, mode: int, factors: Sequence, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        R = _rank(factors)
        if out is None:
            dev = next(f.device for f in factors if f is not None)
            out = torch.empty((self.dims[mode], R), dtype=torch.float32, device=dev)
        blco_mttkrp(self.handle, mode, factors, _fdt(factors), R, out, stream)
        return out

    def mttkrp_f64(self, mode: int, factors: Sequence, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Mode-`mode` MTTKRP of a store built with float64 values, float64 factors (Section 6's precision)."""
        R = int(factors[(mode + 1) % len(factors)].shape[1])
        if out is None:
            out = torch.empty((self.dims[mode], R), dtype=torch.float64, device=factors[(mode + 1) % len(factors)].device)
        blco_mttkrp_f64(self.handle, mode, factors, R, out, stream)
        return out

    def mttkrp_all(self, factors: Sequence, outs: Optional[List[torch.Tensor]] = None, stream=None):
        R = _rank(factors)
        if outs is None:
            dev = factors[0].device
            outs = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in self.dims]
        blco_mttkrp_all(self.handle, factors, _fdt(factors), R, outs, stream)
        return outs

    def cp_fwd(self, factors: Sequence, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.nnz, dtype=torch.float32, device=factors[0].device)
        blco_cp_fwd(self.handle, factors, _fdt(factors), _rank(factors), out, stream)
        return out

    def cp_bwd(self, mode: int, grad: torch.Tensor, factors: Sequence, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
        R = _rank(factors)
        if out is None:
            out = torch.empty((self.dims[mode], R), dtype=torch.float32, device=grad.device)
        blco_cp_bwd(self.handle, mode, grad, factors, _fdt(factors), R, out, stream)
        return out

    def values(self, device="cuda") -> torch.Tensor:
        out = torch.empty(self.nnz, dtype=torch.float32, device=device)
        blco_values(self.handle, out)
        return out

    def perm(self) -> np.ndarray:
        out = np.empty(self.nnz, dtype=np.int64)
        blco_perm(self.handle, out)
        return out

    def keys(self) -> np.ndarray:
        out = np.empty(self.nnz, dtype=np.uint64)
        blco_keys(self.handle, out)
        return out

    def blocks(self):
        info = blco_info(self.handle)
        nb = int(info.nblocks)
        bstart = np.empty(nb + 1, dtype=np.int64)
        bhigh = np.empty(max(nb * self.order, 1), dtype=np.uint32)
        blco_blocks(self.handle, bstart, bhigh)
        return bstart, bhigh[: nb * self.order].reshape(nb, self.order)

    def norm2(self) -> float:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        blco_norm2(self.handle, out)
        return float(out.item())

    def sync(self):
        blco_sync(self.handle)

    def destroy(self):
        if self._h is not None:
            blco_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def convert(src: torch.Tensor, dtype: torch.dtype) -> torch.Tensor:
    """float32 -> bfloat16/float16 copy (round to nearest even) on the GPU."""
    out = torch.empty(src.shape, dtype=dtype, device=src.device)
    blco_convert(src.contiguous(), out, _DTYPE_CODE[dtype], src.numel())
    return out


class SparseCP(torch.autograd.Function):
    """CP model at the stored nonzeros, differentiable in the factors.

    forward: xhat[j] = sum_r prod_n A_n[i_n^j, r] (store order), one kernel.
    backward: dL/dA_n = MTTKRP of mode n with dL/dxhat in place of the
    values (Eq. 1); the gathered row products are recomputed, not saved.
    """

    @staticmethod
    def forward(ctx, tensor: Tensor, *factors):
        ctx.tensor = tensor
        ctx.save_for_backward(*factors)
        return tensor.cp_fwd(list(factors))

    @staticmethod
    def backward(ctx, grad_xhat):
        factors = ctx.saved_tensors
        tensor = ctx.tensor
        g = grad_xhat.contiguous()
        if g.dtype != torch.float32:
            raise TypeError("the upstream gradient must be float32")
        grads = []
        for n, f in enumerate(factors):
            if not ctx.needs_input_grad[1 + n]:
                grads.append(None)
                continue
            gn = tensor.cp_bwd(n, g, list(factors))
            grads.append(gn if f.dtype == torch.float32 else convert(gn, f.dtype))
        return (None, *grads)


def sharded_sum(nnz: int, compute_part, out: torch.Tensor, group=None) -> torch.Tensor:
    """Data-parallel reduction over the ranks of a torch.distributed group:
    rank r computes `compute_part(begin, end, out)` for the r-th of `world`
    equal contiguous parts of the store order (blco_partition), then one
    all-reduce (sum) of `out` gives every rank the result over all parts.
    Correct for any function that is a sum over nonzeros, as MTTKRP is
    (Eq. 1)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    b = blco_partition(nnz, world)
    compute_part(int(b[rank]), int(b[rank + 1]), out)
    dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out


def mttkrp_sharded(tensor: Tensor, mode: int, factors: Sequence, out: Optional[torch.Tensor] = None, group=None,
                   stream=None) -> torch.Tensor:
    """Mode-`mode` MTTKRP split over the ranks of a process group, one GPU per
    rank, each holding the store: every rank runs blco_mttkrp_range on its
    part, and the I_mode x R partial results are summed by one all-reduce
    (NCCL on GPUs)."""
    R = _rank(factors)
    if out is None:
        out = torch.empty((tensor.dims[mode], R), dtype=torch.float32, device=factors[(mode + 1) % len(factors)].device)

    def part(begin, end, o):
        blco_mttkrp_range(tensor.handle, mode, begin, end, factors, _fdt(factors), R, o, stream)

    return sharded_sum(tensor.nnz, part, out, group)


def cp_als(tensor: Tensor, factors: List[torch.Tensor], iters: int, tol: float = 0.0, stream=None):
    """CP-ALS (Algorithm 1) on the GPU: MTTKRP in float32, the R x R Hadamard
    of Grams, its Cholesky/pseudo-inverse solve and the fit in float64.
    ``factors`` (float32, device) are updated in place; returns
    (factors, lambda, fits)."""
    N = tensor.order
    R = int(factors[0].shape[1])
    dev = factors[0].device
    grams = [torch.empty((R, R), dtype=torch.float64, device=dev) for _ in range(N)]
    for n in range(N):
        blco_gram(factors[n], BLCO_F32, tensor.dims[n], R, grams[n], stream)
    nx = torch.empty(1, dtype=torch.float64, device=dev)
    blco_norm2(tensor.handle, nx, stream)
    normX2 = float(nx.item())
    lam = torch.ones(R, dtype=torch.float64, device=dev)
    M = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in tensor.dims]
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    fit_t = torch.empty(1, dtype=torch.float64, device=dev)
    fits: List[float] = []
    for _ in range(int(iters)):
        for n in range(N):
            tensor.mttkrp(n, factors, out=M[n], stream=stream)
            blco_cpals_update(grams, N, n, R, M[n], tensor.dims[n], factors[n], lam, grams[n], info, stream)
        blco_cpals_fit(normX2, grams, N, R, lam, M[N - 1], factors[N - 1], tensor.dims[N - 1], fit_t, stream)
        fits.append(float(fit_t.item()))
        if tol > 0 and len(fits) > 1 and abs(fits[-1] - fits[-2]) < tol:
            break
    return factors, lam, fits
