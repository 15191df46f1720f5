"""ctypes binding of libstark.so (``include/stark.h``).

Argument marshalling only: every step of the multiplication runs in the CUDA
kernels of libstark.so.  PyTorch supplies device memory and streams.  The
library must have been built (``__graft_entry__.build()`` or
``python -m paper_1811_07325_gb300.build_lib``); importing this module fails
loudly otherwise, and there is no fallback path.
"""
from __future__ import annotations

import ctypes
import enum
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstark.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libstark.so is not built ({_LIB_PATH}); run __graft_entry__.build() first")
_lib = ctypes.CDLL(_LIB_PATH)


class DType(enum.IntEnum):
    F64 = 0
    F32_SPLIT_BF16 = 1
    F32_SPLIT_TF32 = 2
    I64 = 3
    F32_SPLIT_FP16 = 4


class Status(enum.IntEnum):
    OK = 0
    EINVAL = 1
    ENOMEM = 2
    EUNSUPPORTED = 3
    ETIMEOUT = 4
    EBUSY = 5
    ENOTFOUND = 6
    ECUDA = 7


class StarkError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = Status(status)
        msg = _lib.stark_strerror(int(status)).decode()
        super().__init__(f"{where}: {self.status.name} ({msg})" if where else f"{self.status.name} ({msg})")


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("leaf", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("dtype", ctypes.c_int32), ("leaves", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("peel", ctypes.c_int32), ("combine", ctypes.c_int32), ("shard_levels", ctypes.c_int32),
                ("shard_first", ctypes.c_int32), ("workspace_leaves", ctypes.c_int32),
                ("promotion_k", ctypes.c_int32)]


class ErrorReport(ctypes.Structure):
    _fields_ = [("norm_a", ctypes.c_double), ("norm_b", ctypes.c_double), ("max_abs_err", ctypes.c_double),
                ("sum_sq_err", ctypes.c_double), ("sum_sq_ref", ctypes.c_double),
                ("max_componentwise", ctypes.c_double), ("compared", ctypes.c_int64)]


_i64, _i32, _vp, _ci = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int
_SIGS = {
    "stark_plan": ([_i64, _ci, _ci, ctypes.POINTER(_vp)], _ci),
    "stark_plan_ex": ([_i64, _ci, _ci, ctypes.c_uint, ctypes.POINTER(_vp)], _ci),
    "stark_plan_destroy": ([_vp], _ci),
    "stark_plan_get_info": ([_vp, ctypes.POINTER(PlanInfo)], _ci),
    "stark_mul": ([_vp, _vp, _vp, _vp, _vp], _ci),
    "stark_mul_host": ([_vp, _vp, _vp, _vp, _vp], _ci),
    "stark_mul_host_async": ([_vp, _vp, _vp, _vp, _vp], _ci),
    "stark_mul_host_enqueue": ([_vp, _vp, _vp, _vp], _ci),
    "stark_plan_host_wait": ([_vp], _ci),
    "stark_mul_leaves": ([_vp, _vp, _vp, _vp, _i64, _i64, _vp], _ci),
    "stark_plan_operands": ([_vp, _vp, _vp, _vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)], _ci),
    "stark_plan_check": ([_vp, _vp], _ci),
    "stark_plan_set_combine": ([_vp, _ci], _ci),
    "stark_plan_set_pairing": ([_vp, _ci], _ci),
    "stark_plan_set_pipeline": ([_vp, _ci], _ci),
    "stark_plan_set_raster": ([_vp, _ci], _ci),
    "stark_plan_set_promotion": ([_vp, _ci], _ci),
    "stark_plan_set_tf32_layout": ([_vp, _ci], _ci),
    "stark_plan_set_input_bound": ([_vp, _i64], _ci),
    "stark_plan_set_traversal": ([_vp, _ci], _ci),
    "stark_plan_set_shard": ([_vp, _i64, _i64], _ci),
    "stark_plan_set_timing": ([_vp, _ci], _ci),
    "stark_plan_phase_ms": ([_vp, ctypes.POINTER(ctypes.c_float)], _ci),
    "stark_plan_phases": ([_vp, ctypes.POINTER(ctypes.c_float), _ci], _ci),
    "stark_quadrant_table": ([_ci, _ci, _vp, _vp, _vp], _ci),
    "stark_strerror": ([_ci], ctypes.c_char_p),
    "stark_selftest_bounded_wait": ([ctypes.c_uint64], _ci),
    "stark_launch_count": ([], _i64),
    "stark_batch_create": ([_i32, _vp, _ci, _ci, ctypes.POINTER(_vp)], _ci),
    "stark_batch_destroy": ([_vp], _ci),
    "stark_batch_mul": ([_vp, _vp, _vp, _vp, _vp], _ci),
    "stark_batch_depth": ([_vp, _i32, ctypes.POINTER(_i32)], _ci),
    "stark_batch_tile": ([_vp, _i32, ctypes.POINTER(_i32)], _ci),
    "stark_batch_info": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                          ctypes.POINTER(_i64)], _ci),
    "stark_batch_check": ([_vp, _vp], _ci),
    "stark_server_create": ([ctypes.c_size_t, _i32, ctypes.POINTER(_vp)], _ci),
    "stark_submit": ([_vp, _i64, _ci, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)], _ci),
    "stark_poll": ([_vp, ctypes.c_uint64, ctypes.POINTER(_ci), ctypes.POINTER(_ci)], _ci),
    "stark_server_drain": ([_vp], _ci),
    "stark_request_latency": ([_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)], _ci),
    "stark_server_stats": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _ci),
    "stark_server_destroy": ([_vp], _ci),
    "stark_server_load": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _ci),
    "stark_server_admission": ([ctypes.c_size_t, _i64, _ci, _ci, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                ctypes.POINTER(_i64)], _ci),
    "stark_error_norms": ([_i64, _ci, _vp, _vp, _vp, _vp, _i64, _vp, _vp, ctypes.POINTER(ErrorReport), _vp], _ci),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(status, where):
    if status != 0:
        raise StarkError(status, where)


def declared_symbols():
    """Names of the entry points this binding uses (all declared in stark.h)."""
    return sorted(_SIGS)


def library_path():
    return _LIB_PATH


_TORCH_DTYPE = {}


def _torch_dtype(dt):
    import torch
    return {DType.F64: torch.float64, DType.F32_SPLIT_BF16: torch.float32, DType.F32_SPLIT_TF32: torch.float32,
            DType.F32_SPLIT_FP16: torch.float32, DType.I64: torch.int64}[DType(dt)]


def _numpy_dtype(dt):
    return {DType.F64: np.float64, DType.F32_SPLIT_BF16: np.float32, DType.F32_SPLIT_TF32: np.float32,
            DType.F32_SPLIT_FP16: np.float32, DType.I64: np.int64}[DType(dt)]


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class _CudaBuffer:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2, "strides": None}


class Plan:
    """A plan for n x n products (``stark_plan``)."""

    PEEL = 1  # STARK_PLAN_PEEL

    def __init__(self, n: int, depth: int = -1, dtype: DType = DType.F32_SPLIT_BF16, peel: bool = False):
        """``peel``: edge peeling instead of padding (``STARK_PLAN_PEEL``)."""
        h = _vp()
        _check(_lib.stark_plan_ex(int(n), int(depth), int(dtype), self.PEEL if peel else 0, ctypes.byref(h)),
               "stark_plan_ex")
        self._h = h
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(h, ctypes.byref(info)), "stark_plan_get_info")
        self.n, self.n_pad, self.leaf, self.depth = info.n, info.n_pad, info.leaf, info.depth
        self.dtype = DType(info.dtype)
        self.leaves, self.workspace_bytes = info.leaves, info.workspace_bytes
        self.tile = (info.tile_m, info.tile_n)
        self.peel = info.peel
        self.combine = info.combine
        self.promotion_k = info.promotion_k

    def close(self):
        if getattr(self, "_h", None):
            _lib.stark_plan_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- argument checks ---------------------------------------------------
    def _check_tensor(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be on a CUDA device")
        if t.dtype != _torch_dtype(self.dtype):
            raise TypeError(f"{name} has dtype {t.dtype}, plan expects {_torch_dtype(self.dtype)}")
        if tuple(t.shape) != (self.n, self.n) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.n}x{self.n} matrix")
        return ctypes.c_void_p(t.data_ptr())

    def mul(self, A, B, C=None, stream=None):
        """C = A @ B on the device (async on ``stream``, default: torch's current)."""
        import torch
        if C is None:
            C = torch.empty((self.n, self.n), dtype=_torch_dtype(self.dtype), device=A.device)
        a, b, c = self._check_tensor(A, "A"), self._check_tensor(B, "B"), self._check_tensor(C, "C")
        _check(_lib.stark_mul(self._h, a, b, c, _stream_handle(stream)), "stark_mul")
        return C

    def mul_leaves(self, A, B, leaf_begin, leaf_end, C=None, stream=None):
        import torch
        if C is None:
            C = torch.empty((self.n, self.n), dtype=_torch_dtype(self.dtype), device=A.device)
        a, b, c = self._check_tensor(A, "A"), self._check_tensor(B, "B"), self._check_tensor(C, "C")
        _check(_lib.stark_mul_leaves(self._h, a, b, c, int(leaf_begin), int(leaf_end), _stream_handle(stream)),
               "stark_mul_leaves")
        return C

    def mul_host(self, A, B, C=None, stream=None, asynchronous=False):
        """End to end from host memory (numpy arrays or CPU tensors, pinned is
        best).  ``asynchronous=True``: pipelined form, completion on ``stream``."""
        def ptr(x, name):
            if hasattr(x, "data_ptr"):
                if x.is_cuda or tuple(x.shape) != (self.n, self.n) or not x.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous host {self.n}x{self.n} matrix")
                return ctypes.c_void_p(x.data_ptr())
            x = np.asarray(x)
            if x.dtype != _numpy_dtype(self.dtype) or x.shape != (self.n, self.n) or not x.flags.c_contiguous:
                raise ValueError(f"{name} must be a contiguous {self.n}x{self.n} {_numpy_dtype(self.dtype)} array")
            return ctypes.c_void_p(x.ctypes.data)
        if C is None:
            C = np.empty((self.n, self.n), dtype=_numpy_dtype(self.dtype))
        fn = _lib.stark_mul_host_async if asynchronous else _lib.stark_mul_host
        _check(fn(self._h, ptr(A, "A"), ptr(B, "B"), ptr(C, "C"), _stream_handle(stream)), "stark_mul_host")
        return C

    def mul_host_enqueue(self, A, B, C):
        """Pipelined product from host memory with no wait on any stream:
        returns at once; ``host_wait()`` collects every product enqueued so
        far.  A, B, C stay untouched (C unread) until then."""
        def ptr(x, name):
            if not hasattr(x, "data_ptr") or x.is_cuda or tuple(x.shape) != (self.n, self.n) \
                    or not x.is_contiguous():
                raise ValueError(f"{name} must be a contiguous host {self.n}x{self.n} tensor")
            return ctypes.c_void_p(x.data_ptr())
        _check(_lib.stark_mul_host_enqueue(self._h, ptr(A, "A"), ptr(B, "B"), ptr(C, "C")), "stark_mul_host_enqueue")
        return C

    def host_wait(self):
        """Block until every enqueued host product is in host memory; raises
        on a device error (as ``check``)."""
        _check(_lib.stark_plan_host_wait(self._h), "stark_plan_host_wait")

    def operands(self, A, B, stream=None):
        """Divide phase only; returns torch views (X, Y) of the leaf operand planes."""
        import torch
        a, b = self._check_tensor(A, "A"), self._check_tensor(B, "B")
        x, y = _vp(), _vp()
        _check(_lib.stark_plan_operands(self._h, a, b, _stream_handle(stream), ctypes.byref(x), ctypes.byref(y)),
               "stark_plan_operands")
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(self._h, ctypes.byref(info)), "stark_plan_get_info")
        P, L = info.workspace_leaves, self.leaf  # a shard's workspace holds its subtrees' leaves only
        if self.dtype == DType.F32_SPLIT_BF16:
            shape, ts, view = (2 * P, L, L), "<i2", torch.bfloat16
        elif self.dtype == DType.F32_SPLIT_FP16:
            shape, ts, view = (2 * P, L, L), "<i2", torch.float16
        elif self.dtype == DType.F32_SPLIT_TF32:
            shape, ts, view = (2 * P, L, L), "<f4", None
        elif self.dtype == DType.F64:
            shape, ts, view = (P, L, L), "<f8", None
        else:
            shape, ts, view = (P, L, L), "<i8", None
        X = torch.as_tensor(_CudaBuffer(x.value, shape, ts), device=A.device)
        Y = torch.as_tensor(_CudaBuffer(y.value, shape, ts), device=A.device)
        if view is not None:
            X, Y = X.view(view), Y.view(view)
        return X, Y

    def info(self) -> PlanInfo:
        """What the plan decided (``stark_plan_get_info``)."""
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(self._h, ctypes.byref(info)), "stark_plan_get_info")
        return info

    def set_combine(self, mode: int):
        """0: fused, TMA bulk reductions (default); 1: fused, vector atomics;
        2: deterministic (stored leaf products, ordered combine pass);
        3: sibling fold (parent products folded in L2, ordered pass one
        level up); -1: the fastest of those that apply, measured."""
        _check(_lib.stark_plan_set_combine(self._h, int(mode)), "stark_plan_set_combine")
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(self._h, ctypes.byref(info)), "stark_plan_get_info")
        self.combine, self.workspace_bytes = info.combine, info.workspace_bytes

    def set_pairing(self, mode):
        """Leaf schedule of the split-fp32 paths: 0 single CTAs; 2 (default)
        CTA pairs on one cta_group::2 MMA of 256 x 256 (mode 1 is refused
        with EUNSUPPORTED)."""
        _check(_lib.stark_plan_set_pairing(self._h, int(mode)), "stark_plan_set_pairing")

    def set_shard(self, begin: int, end: int):
        """Restrict the plan to leaves [begin, end) (``stark_plan_set_shard``):
        a rank-local workspace and divide for sharding one product."""
        _check(_lib.stark_plan_set_shard(self._h, int(begin), int(end)), "stark_plan_set_shard")
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(self._h, ctypes.byref(info)), "stark_plan_get_info")
        self.workspace_bytes = info.workspace_bytes
        self.shard = (int(begin), int(end))
        self.shard_levels, self.shard_first = info.shard_levels, info.shard_first

    def set_tf32_layout(self, mn: bool):
        """3xTF32 B operand: MN-major planes (no transpose pass) or K-major."""
        _check(_lib.stark_plan_set_tf32_layout(self._h, 1 if mn else 0), "stark_plan_set_tf32_layout")

    def set_promotion(self, k_chunk: int):
        """Accumulator promotion of the split-fp32 leaf products: every
        ``k_chunk`` of K (a multiple of 256) the tensor-core partial sum joins
        a running fp32 sum on the CUDA cores; 0 turns it off."""
        _check(_lib.stark_plan_set_promotion(self._h, int(k_chunk)), "stark_plan_set_promotion")
        self.promotion_k = int(k_chunk)

    def set_raster(self, band: int):
        """Leaf tile order: bands of ``band`` tile columns (0: row-major)."""
        _check(_lib.stark_plan_set_raster(self._h, int(band)), "stark_plan_set_raster")

    def set_pipeline(self, deep: bool):
        """3xBF16: ``deep=True`` runs the single-CTA schedule with four 48 KB
        stages of 64-byte rows (it replaces the CTA pairs); False restores the
        plan's leaf schedule."""
        _check(_lib.stark_plan_set_pipeline(self._h, 1 if deep else 0), "stark_plan_set_pipeline")

    def set_traversal(self, levels):
        """Depth first over the top ``levels`` recursion levels (0: breadth
        first; True means 1; 2 for the split dtypes): the workspace holds one
        subtree's leaves."""
        _check(_lib.stark_plan_set_traversal(self._h, int(levels)), "stark_plan_set_traversal")
        info = PlanInfo()
        _check(_lib.stark_plan_get_info(self._h, ctypes.byref(info)), "stark_plan_get_info")
        self.workspace_bytes = info.workspace_bytes

    def set_input_bound(self, max_abs: int):
        """I64 plans: inputs bounded by max_abs run as exact bf16 tensor-core products."""
        _check(_lib.stark_plan_set_input_bound(self._h, int(max_abs)), "stark_plan_set_input_bound")

    def check(self, stream=None):
        """Synchronise and raise on a device-side timeout."""
        _check(_lib.stark_plan_check(self._h, _stream_handle(stream)), "stark_plan_check")

    def set_timing(self, records=1):
        """Record per-phase events for the next ``records`` products (0: off)."""
        _check(_lib.stark_plan_set_timing(self._h, int(records)), "stark_plan_set_timing")

    def phase_ms(self):
        """Mean per-phase device time (ms) over the recorded products:
        zeroing C, the divide, the leaf products with the combine, and that
        last phase split into the leaf kernel and what follows it (the
        separate combine pass of combine modes 2 and 3, peeled edge,
        staging copy)."""
        out = (ctypes.c_float * 4)()
        _check(_lib.stark_plan_phases(self._h, out, 4), "stark_plan_phases")
        return {"zero_c": out[0], "divide": out[1], "leaf_combine": out[2] + out[3], "leaf_kernel": out[2],
                "after_leaf": out[3]}


class Batch:
    """Independent products of mixed sizes in one grouped, graph-replayed pass
    (``stark_batch_create``)."""

    def __init__(self, sizes, depth: int = -1, dtype: DType = DType.F32_SPLIT_BF16):
        self.sizes = [int(x) for x in sizes]
        arr = (ctypes.c_int64 * len(self.sizes))(*self.sizes)
        h = _vp()
        _check(_lib.stark_batch_create(len(self.sizes), ctypes.cast(arr, _vp), int(depth), int(dtype),
                                       ctypes.byref(h)), "stark_batch_create")
        self._h = h
        self.dtype = DType(dtype)

    def close(self):
        if getattr(self, "_h", None):
            _lib.stark_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def depths(self):
        out = []
        for i in range(len(self.sizes)):
            d = _i32()
            _check(_lib.stark_batch_depth(self._h, i, ctypes.byref(d)), "stark_batch_depth")
            out.append(d.value)
        return out

    def tiles(self):
        """Leaf tile width of every member (256: CTA pairs, 128: single CTAs)."""
        out = []
        for i in range(len(self.sizes)):
            t = _i32()
            _check(_lib.stark_batch_tile(self._h, i, ctypes.byref(t)), "stark_batch_tile")
            out.append(t.value)
        return out

    def info(self):
        t, w, b, r = _i32(), _i64(), _i64(), _i64()
        _check(_lib.stark_batch_info(self._h, ctypes.byref(t), ctypes.byref(w), ctypes.byref(b), ctypes.byref(r)),
               "stark_batch_info")
        return {"tile_n": t.value, "work_items": w.value, "workspace_bytes": b.value, "graph_replays": r.value}

    def mul(self, As, Bs, Cs, stream=None):
        """Cs[i] = As[i] @ Bs[i] (device fp32 tensors)."""
        import torch
        k = len(self.sizes)
        if not (len(As) == len(Bs) == len(Cs) == k):
            raise ValueError("one A, B and C per member")
        pa, pb, pc = (_vp * k)(), (_vp * k)(), (_vp * k)()
        for i, n in enumerate(self.sizes):
            for t, name in ((As[i], "A"), (Bs[i], "B"), (Cs[i], "C")):
                if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 \
                        or tuple(t.shape) != (n, n) or not t.is_contiguous():
                    raise ValueError(f"{name}[{i}] must be a contiguous fp32 CUDA {n}x{n} tensor")
            pa[i], pb[i], pc[i] = As[i].data_ptr(), Bs[i].data_ptr(), Cs[i].data_ptr()
        _check(_lib.stark_batch_mul(self._h, ctypes.cast(pa, _vp), ctypes.cast(pb, _vp), ctypes.cast(pc, _vp),
                                    _stream_handle(stream)), "stark_batch_mul")
        return Cs

    def check(self, stream=None):
        _check(_lib.stark_batch_check(self._h, _stream_handle(stream)), "stark_batch_check")


class Server:
    """Continuous-batching request server (``stark_server_create``)."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 4):
        h = _vp()
        _check(_lib.stark_server_create(int(hbm_budget_bytes), int(slots), ctypes.byref(h)), "stark_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.stark_server_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, A, B, C, dtype: DType = DType.F32_SPLIT_BF16) -> int:
        """Queue C = A @ B (device tensors kept alive by the caller); returns the id."""
        import torch
        n = A.shape[0]
        for t, name in ((A, "A"), (B, "B"), (C, "C")):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != _torch_dtype(dtype) \
                    or tuple(t.shape) != (n, n) or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {n}x{n} CUDA tensor of the dtype's type")
        rid = ctypes.c_uint64()
        _check(_lib.stark_submit(self._h, n, int(dtype), A.data_ptr(), B.data_ptr(), C.data_ptr(), ctypes.byref(rid)),
               "stark_submit")
        return rid.value

    def poll(self, rid: int):
        """(done, status) without blocking."""
        done, st = _ci(), _ci()
        _check(_lib.stark_poll(self._h, ctypes.c_uint64(rid), ctypes.byref(done), ctypes.byref(st)), "stark_poll")
        return bool(done.value), Status(st.value) if done.value else None

    def drain(self):
        _check(_lib.stark_server_drain(self._h), "stark_server_drain")

    def latency(self, rid: int) -> float:
        x = ctypes.c_double()
        _check(_lib.stark_request_latency(self._h, ctypes.c_uint64(rid), ctypes.byref(x)), "stark_request_latency")
        return x.value

    def stats(self):
        w, b, q = _i64(), _i64(), _i64()
        _check(_lib.stark_server_stats(self._h, ctypes.byref(w), ctypes.byref(b), ctypes.byref(q)),
               "stark_server_stats")
        return {"cached_workspaces": w.value, "owned_bytes": b.value, "queued": q.value}

    def load(self):
        """Most requests queued at once, requests whose admission waited for
        device memory, requests finished (``stark_server_load``)."""
        m, d, f = _i64(), _i64(), _i64()
        _check(_lib.stark_server_load(self._h, ctypes.byref(m), ctypes.byref(d), ctypes.byref(f)),
               "stark_server_load")
        return {"max_queued": m.value, "deferred": d.value, "finished": f.value}


def server_admission(hbm_budget_bytes: int, n: int, dtype: DType = DType.F32_SPLIT_BF16, staged: bool = False):
    """How a server with this budget holds a request of side n (host only):
    {"depth", "levels" (depth-first levels; 0 breadth first), "bytes"}.
    Raises StarkError (ENOMEM) when no depth fits."""
    d, l, b = _i32(), _i32(), _i64()
    _check(_lib.stark_server_admission(int(hbm_budget_bytes), int(n), int(dtype), 1 if staged else 0,
                                       ctypes.byref(d), ctypes.byref(l), ctypes.byref(b)), "stark_server_admission")
    return {"depth": d.value, "levels": l.value, "bytes": b.value}


def quadrant_table(depth: int, side: int):
    """(count[7^d], quad[7^d, 2^d], sign[7^d, 2^d]) on the host; side 0 A, 1 B, 2 C."""
    P, T = 7 ** depth, 2 ** depth
    count = np.zeros(P, np.int32)
    quad = np.zeros((P, T), np.int32)
    sign = np.zeros((P, T), np.int8)
    _check(_lib.stark_quadrant_table(int(depth), int(side), count.ctypes.data, quad.ctypes.data,
                                     sign.ctypes.data), "stark_quadrant_table")
    return count, quad, sign


def error_norms(A, B, C=None, rows=None, want=None, absprod=None, stream=None) -> dict:
    """FP64 error statistics on the device (``stark_error_norms``): the
    Frobenius norms of A and B and, when rows are given, the error of rows
    ``rows`` of C against ``want`` (nrows x n reference rows) and, with
    ``absprod`` (the rows of |A||B|), the largest componentwise ratio.
    A, B, C: square CUDA tensors of one dtype (float32, float64, int64);
    rows / want / absprod: numpy arrays or tensors (copied to the device).
    Returns the report as a dict with the derived normwise ratio and
    relative RMS."""
    import torch
    dt = {torch.float32: DType.F32_SPLIT_BF16, torch.float64: DType.F64, torch.int64: DType.I64}[A.dtype]
    n = A.shape[0]
    for t, name in ((A, "A"), (B, "B")) + (((C, "C"),) if C is not None else ()):
        if not t.is_cuda or t.dtype != A.dtype or tuple(t.shape) != (n, n) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {n}x{n} CUDA tensor of {A.dtype}")
    keep = []

    def dev(x, dtype):
        if x is None:
            return None, None
        t = torch.as_tensor(np.ascontiguousarray(x) if isinstance(x, np.ndarray) else x, dtype=dtype,
                            device=A.device).contiguous()
        keep.append(t)
        return t, ctypes.c_void_p(t.data_ptr())
    r_t, r_p = dev(rows, torch.int64)
    nrows = 0 if r_t is None else int(r_t.numel())
    w_t, w_p = dev(want, torch.float64)
    a_t, a_p = dev(absprod, torch.float64)
    if nrows and (C is None or w_t is None or w_t.numel() != nrows * n or (a_t is not None and a_t.numel() != nrows * n)):
        raise ValueError("C, rows and want (nrows x n) are needed together")
    rep = ErrorReport()
    _check(_lib.stark_error_norms(n, int(dt), ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  ctypes.c_void_p(C.data_ptr()) if C is not None else None, r_p, nrows, w_p, a_p,
                                  ctypes.byref(rep), _stream_handle(stream)), "stark_error_norms")
    out = {f: getattr(rep, f) for f, _ in ErrorReport._fields_}
    if nrows:
        out["max_abs_over_normA_normB"] = rep.max_abs_err / (rep.norm_a * rep.norm_b)
        out["rel_rms"] = float(np.sqrt(rep.sum_sq_err / rep.sum_sq_ref)) if rep.sum_sq_ref > 0 else 0.0
    return out


def selftest_bounded_wait(timeout_ns: int = 20_000_000) -> Status:
    return Status(_lib.stark_selftest_bounded_wait(int(timeout_ns)))


def launch_count() -> int:
    return int(_lib.stark_launch_count())


def strerror(status) -> str:
    return _lib.stark_strerror(int(status)).decode()
