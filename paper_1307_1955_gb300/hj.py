"""Thin Python binding of libhj (include/hj.h): argument marshalling only.

Every step of the join runs in the library's CUDA kernels; this module turns
torch tensors into ``hj_rel`` structs (device pointer, length, width), calls the C
entry point of the same name and turns the result struct back into Python values.
PyTorch provides the device memory of the inputs and the stream.  There is no CPU
fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HJ_OK, HJ_E_INVALID, HJ_E_NOMEM, HJ_E_OVERFLOW, HJ_E_CUDA, HJ_E_TIMEOUT, HJ_E_UNSUPPORTED, HJ_E_PENDING = range(8)
HJ_COUNT, HJ_COUNT_CHECKSUM, HJ_MATERIALIZE = 0, 1, 2
HJ_ALGO_AUTO, HJ_ALGO_SHJ, HJ_ALGO_PHJ = 0, 1, 2
HJ_FLAG_CHECKSUM = 1
HJ_FLAG_GRAPH = 2
HJ_SCATTER_AUTO, HJ_SCATTER_REGION, HJ_SCATTER_RING = 0, 1, 2
HJ_OUTCORE_AUTO, HJ_OUTCORE_SPLIT = 0, 1

_STATUS = {0: "HJ_OK", 1: "HJ_E_INVALID", 2: "HJ_E_NOMEM", 3: "HJ_E_OVERFLOW", 4: "HJ_E_CUDA",
           5: "HJ_E_TIMEOUT", 6: "HJ_E_UNSUPPORTED", 7: "HJ_E_PENDING"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhj.so")


class HJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class hj_rel(ctypes.Structure):
    _fields_ = [("tuples", ctypes.c_void_p), ("n", ctypes.c_uint64), ("width", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class hj_opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("mode", ctypes.c_int32), ("radix_bits", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("out_capacity", ctypes.c_uint64), ("flags", ctypes.c_uint64)]


class hj_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("checksum", ctypes.c_uint64 * 2), ("pairs", ctypes.c_void_p),
                ("pairs_cap", ctypes.c_uint64), ("width", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("radix_bits", ctypes.c_int32), ("passes", ctypes.c_int32)]


class hj_server_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("workers", ctypes.c_int32), ("max_wave", ctypes.c_int32),
                ("wave_tuples", ctypes.c_uint64), ("flags", ctypes.c_uint64)]


class hj_req_times(ctypes.Structure):
    _fields_ = [("submit", ctypes.c_double), ("admit", ctypes.c_double), ("start", ctypes.c_double),
                ("done", ctypes.c_double)]


class hj_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "waves", "wave_max", "queued", "in_use",
                                                "peak_in_use", "budget", "launches")]


class hj_plan_info(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("radix_bits", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("predicted_ms", ctypes.c_double), ("step_ms", ctypes.c_double * 4),
                ("measured_ms", ctypes.c_double)]


class hj_prof_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhj.so (build it first with paper_1307_1955_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libhj not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P, V, I32, U64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
    sig = {
        "hj_create": (I32, [P(V), ctypes.c_int, V, U64]),
        "hj_destroy": (I32, [V]),
        "hj_last_error": (ctypes.c_char_p, [V]),
        "hj_build": (I32, [V, P(hj_rel), P(hj_opts), P(V)]),
        "hj_probe": (I32, [V, V, P(hj_rel), P(hj_opts), P(hj_result)]),
        "hj_table_free": (I32, [V, V]),
        "hj_partition": (I32, [V, P(hj_rel), ctypes.c_int, ctypes.c_int, P(hj_rel), P(V)]),
        "hj_partition_free": (I32, [V, P(hj_rel), V]),
        "hj_join": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), P(hj_result)]),
        "hj_result_free": (I32, [V, P(hj_result)]),
        "hj_join_host": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), V, U64, P(hj_result)]),
        "hj_join_static": (I32, [P(hj_rel), P(hj_rel), V, V, U64, P(U64), P(U64)]),
        "hj_join_host_large": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), U64, V, U64, P(hj_result)]),
        "hj_join_batch": (I32, [V, ctypes.c_int, P(hj_rel), P(hj_rel), P(hj_opts), P(hj_result)]),
        "hj_sync": (I32, [V]),
        "hj_copy": (I32, [V, V, V, U64]),
        "hj_prof_enable": (I32, [V, ctypes.c_int]),
        "hj_prof_only": (I32, [V, ctypes.c_char_p]),
        "hj_coproc_time": (I32, [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                 ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                 P(ctypes.c_double)]),
        "hj_coproc_ratios": (I32, [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                   ctypes.c_double, ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double)]),
        "hj_prof_reset": (I32, [V]),
        "hj_prof_read": (I32, [V, P(hj_prof_entry), ctypes.c_int, P(ctypes.c_int)]),
        "hj_launch_count": (U64, [V]),
        "hj_debug_fail_alloc": (I32, [V, ctypes.c_int64]),
        "hj_debug_bytes_in_use": (U64, [V]),
        "hj_debug_wait_limit": (I32, [V, U64]),
        "hj_debug_scatter": (I32, [V, ctypes.c_int]),
        "hj_debug_outcore": (I32, [V, ctypes.c_int]),
        "hj_debug_peak_bytes": (U64, [V, ctypes.c_int]),
        "hj_split": (I32, [V, P(hj_rel), ctypes.c_int, V, P(U64)]),
        "hj_join_coproc": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), ctypes.c_double, ctypes.c_int, P(hj_result),
                                 P(ctypes.c_double)]),
        "hj_plan": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), P(hj_plan_info)]),
        "hj_tune": (I32, [V, P(hj_rel), P(hj_rel), P(hj_opts), ctypes.c_int, P(hj_plan_info)]),
        "hj_tune_clear": (I32, [V]),
        "hj_server_create": (I32, [P(V), V, P(hj_server_opts)]),
        "hj_server_submit": (I32, [V, P(hj_rel), P(hj_rel), I32, P(U64)]),
        "hj_server_poll": (I32, [V, U64, P(hj_result), P(hj_req_times)]),
        "hj_server_wait": (I32, [V, U64, ctypes.c_double, P(hj_result), P(hj_req_times)]),
        "hj_server_result_free": (I32, [V, P(hj_result)]),
        "hj_server_stats_get": (I32, [V, P(hj_server_stats)]),
        "hj_server_last_error": (ctypes.c_char_p, [V]),
        "hj_server_destroy": (I32, [V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(ctx, st: int):
    if st != HJ_OK:
        msg = load_library().hj_last_error(ctx.handle if ctx is not None else None)
        raise HJError(st, msg.decode() if msg else "")


def rel_of(t: torch.Tensor) -> hj_rel:
    """An (n, 2) int32/int64 CUDA tensor (key, rid columns) as an hj_rel."""
    if t.dim() != 2 or t.shape[1] != 2 or t.dtype not in (torch.int32, torch.int64):
        raise ValueError("relation must be an (n, 2) int32 or int64 tensor")
    if not t.is_contiguous():
        raise ValueError("relation must be contiguous")
    width = 4 if t.dtype == torch.int32 else 8
    return hj_rel(t.data_ptr() if t.numel() else None, t.shape[0], width, 0)


@dataclass
class Result:
    count: int
    checksum: tuple
    pairs_ptr: int
    pairs_cap: int
    width: int
    algo: int
    radix_bits: int
    passes: int
    _raw: hj_result
    _ctx: "Context"
    _server: "Server | None" = None

    def pairs_numpy(self):
        """Copy the pairs to host: (count, 2) uint32/uint64 array of (rid_R, rid_S)."""
        import numpy as np

        dt = np.uint32 if self.width == 4 else np.uint64
        out = np.empty((self.count, 2), dt)
        if self.count and self.pairs_ptr:
            _check(self._ctx, load_library().hj_copy(self._ctx.handle, out.ctypes.data, self.pairs_ptr,
                                                     out.nbytes))
        return out

    def free(self):
        if self._raw is not None and self._server is not None:
            self._server._free(self._raw)
        elif self._raw is not None and self._ctx.handle:
            _check(self._ctx, load_library().hj_result_free(self._ctx.handle, ctypes.byref(self._raw)))
        self._raw = None
        self.pairs_ptr = 0


def _result(ctx, r: hj_result) -> Result:
    return Result(int(r.count), (int(r.checksum[0]), int(r.checksum[1])), int(r.pairs or 0), int(r.pairs_cap),
                  int(r.width), int(r.algo), int(r.radix_bits), int(r.passes), r, ctx)


# cudaStreamLegacy: the legacy default stream, which torch uses as its default
# stream (handle 0 on the torch side; NULL means "a stream of its own" to hj_create).
_CUDA_STREAM_LEGACY = 1


def stream_handle(stream: torch.cuda.Stream) -> int:
    """The cudaStream_t to give the library for a torch stream."""
    return stream.cuda_stream or _CUDA_STREAM_LEGACY


class Context:
    """An hj_ctx bound to a CUDA device and stream.  By default the context orders
    its work on torch's current stream of the device, so that it follows the
    kernels that produced its inputs; pass `own_stream=True` for a separate stream
    (the caller then synchronises its inputs first)."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, budget: int = 0,
                 own_stream: bool = False):
        lib = load_library()
        h = ctypes.c_void_p()
        if stream is None and not own_stream:
            stream = torch.cuda.current_stream(device)
        s = stream_handle(stream) if stream is not None else None
        st = lib.hj_create(ctypes.byref(h), device, s, budget)
        if st != HJ_OK:
            raise HJError(st, "hj_create failed")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load_library().hj_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(algo=HJ_ALGO_AUTO, mode=HJ_MATERIALIZE, radix_bits=0, passes=0, out_capacity=0, checksum=False):
    return hj_opts(algo, mode, radix_bits, passes, out_capacity, HJ_FLAG_CHECKSUM if checksum else 0)


def hj_create(device: int = 0, stream=None, budget: int = 0) -> Context:
    return Context(device, stream, budget)


def hj_destroy(ctx: Context):
    ctx.close()


class Table:
    def __init__(self, ctx, handle, width, agg):
        self.ctx, self.handle, self.width, self.agg = ctx, handle, width, agg

    def free(self):
        if self.handle:
            _check(self.ctx, load_library().hj_table_free(self.ctx.handle, self.handle))
            self.handle = None


def hj_build(ctx: Context, R: torch.Tensor, mode: int = HJ_MATERIALIZE) -> Table:
    r = rel_of(R)
    h = ctypes.c_void_p()
    o = _opts(mode=mode)
    _check(ctx, load_library().hj_build(ctx.handle, ctypes.byref(r), ctypes.byref(o), ctypes.byref(h)))
    return Table(ctx, h, r.width, mode != HJ_MATERIALIZE)


def hj_probe(ctx: Context, table: Table, S: torch.Tensor, mode: int = HJ_MATERIALIZE, out_capacity: int = 0,
             checksum: bool = False) -> Result:
    s = rel_of(S)
    o = _opts(mode=mode, out_capacity=out_capacity, checksum=checksum)
    res = hj_result()
    _check(ctx, load_library().hj_probe(ctx.handle, table.handle, ctypes.byref(s), ctypes.byref(o),
                                        ctypes.byref(res)))
    return _result(ctx, res)


def hj_table_free(ctx: Context, table: Table):
    table.free()


def hj_join(ctx: Context, R: torch.Tensor, S: torch.Tensor, algo: int = HJ_ALGO_AUTO, mode: int = HJ_MATERIALIZE,
            radix_bits: int = 0, passes: int = 0, out_capacity: int = 0, checksum: bool = False) -> Result:
    r, s = rel_of(R), rel_of(S)
    o = _opts(algo, mode, radix_bits, passes, out_capacity, checksum)
    res = hj_result()
    _check(ctx, load_library().hj_join(ctx.handle, ctypes.byref(r), ctypes.byref(s), ctypes.byref(o),
                                       ctypes.byref(res)))
    return _result(ctx, res)


def _plan_dict(p: hj_plan_info) -> dict:
    return {"algo": int(p.algo), "radix_bits": int(p.radix_bits), "passes": int(p.passes),
            "predicted_ms": float(p.predicted_ms), "step_ms": [float(x) for x in p.step_ms],
            "measured_ms": float(p.measured_ms)}


def _size_rel(n: int, width: int) -> hj_rel:
    return hj_rel(None, n, width, 0)


def hj_plan(ctx: "Context | None", R, S, algo: int = HJ_ALGO_AUTO, mode: int = HJ_MATERIALIZE, radix_bits: int = 0,
            passes: int = 0) -> dict:
    """The plan hj_join would run.  R and S may be tensors or (n, width) size pairs
    (only sizes are read); with ctx None the model uses GB300's figures (no GPU)."""
    r = rel_of(R) if isinstance(R, torch.Tensor) else _size_rel(*R)
    s = rel_of(S) if isinstance(S, torch.Tensor) else _size_rel(*S)
    o = _opts(algo, mode, radix_bits, passes)
    out = hj_plan_info()
    st = load_library().hj_plan(ctx.handle if ctx is not None else None, ctypes.byref(r), ctypes.byref(s),
                                ctypes.byref(o), ctypes.byref(out))
    if st != HJ_OK:
        if ctx is not None:
            _check(ctx, st)
        raise HJError(st, "hj_plan failed")
    return _plan_dict(out)


def hj_tune(ctx: Context, R: torch.Tensor, S: torch.Tensor, mode: int = HJ_MATERIALIZE, top_k: int = 0) -> dict:
    """Time the model's cheapest plans on R and S; the fastest is cached for their
    size class and used by later hj_join calls with algo=HJ_ALGO_AUTO."""
    r, s = rel_of(R), rel_of(S)
    o = _opts(mode=mode)
    out = hj_plan_info()
    _check(ctx, load_library().hj_tune(ctx.handle, ctypes.byref(r), ctypes.byref(s), ctypes.byref(o), top_k,
                                       ctypes.byref(out)))
    return _plan_dict(out)


def hj_tune_clear(ctx: Context):
    _check(ctx, load_library().hj_tune_clear(ctx.handle))


def hj_join_host(ctx: Context, R: torch.Tensor, S: torch.Tensor, pairs_out: torch.Tensor | None = None,
                 algo: int = HJ_ALGO_AUTO, mode: int = HJ_MATERIALIZE, radix_bits: int = 0, passes: int = 0,
                 out_capacity: int = 0, checksum: bool = False) -> Result:
    """hj_join on CPU tensors (pinned for full speed): pairs land in `pairs_out`,
    an (m, 2) CPU tensor of R's dtype with m >= the pair count."""
    if R.device.type != "cpu" or S.device.type != "cpu":
        raise ValueError("hj_join_host takes CPU tensors")
    r, s = rel_of(R), rel_of(S)
    o = _opts(algo, mode, radix_bits, passes, out_capacity, checksum)
    res = hj_result()
    ptr = pairs_out.data_ptr() if pairs_out is not None and pairs_out.numel() else None
    cap = pairs_out.shape[0] if pairs_out is not None else 0
    _check(ctx, load_library().hj_join_host(ctx.handle, ctypes.byref(r), ctypes.byref(s), ctypes.byref(o), ptr,
                                            cap, ctypes.byref(res)))
    return _result(ctx, res)


def hj_join_host_large(ctx: Context, R: torch.Tensor, S: torch.Tensor, pairs_out: torch.Tensor | None = None,
                       device_bytes: int = 0, mode: int = HJ_MATERIALIZE, checksum: bool = False) -> Result:
    """The join of CPU tensors that need not fit the device (partitioned through a
    device budget of device_bytes); pairs land in `pairs_out` ((m, 2) CPU tensor of
    R's dtype, m >= the pair count)."""
    if R.device.type != "cpu" or S.device.type != "cpu":
        raise ValueError("hj_join_host_large takes CPU tensors")
    r, s = rel_of(R), rel_of(S)
    o = _opts(mode=mode, checksum=checksum)
    res = hj_result()
    ptr = pairs_out.data_ptr() if pairs_out is not None and pairs_out.numel() else None
    cap = pairs_out.shape[0] if pairs_out is not None else 0
    _check(ctx, load_library().hj_join_host_large(ctx.handle, ctypes.byref(r), ctypes.byref(s), ctypes.byref(o),
                                                  device_bytes, ptr, cap, ctypes.byref(res)))
    return _result(ctx, res)


def rel_array(tensors: list) -> ctypes.Array:
    """hj_rel structs of many relations, built once and passed to hj_join_batch."""
    return (hj_rel * len(tensors))(*[rel_of(t) for t in tensors])


def hj_join_batch(ctx: Context, Rs, Ss, mode: int = HJ_MATERIALIZE, out_capacity: int = 0,
                  checksum: bool = False, graph: bool = False, raw: bool = False):
    """Many independent joins: Rs[j] join Ss[j] for every j.  Rs and Ss are lists of
    relations or arrays from rel_array().  Returns one Result per join, or with raw=True
    the hj_result array itself (free it with hj_results_free)."""
    n = len(Rs)
    if len(Ss) != n:
        raise ValueError("Rs and Ss differ in length")
    ra = Rs if isinstance(Rs, ctypes.Array) else rel_array(Rs)
    sa = Ss if isinstance(Ss, ctypes.Array) else rel_array(Ss)
    outs = (hj_result * max(n, 1))()
    flags = (HJ_FLAG_CHECKSUM if checksum else 0) | (HJ_FLAG_GRAPH if graph else 0)
    o = hj_opts(HJ_ALGO_AUTO, mode, 0, 0, out_capacity, flags)
    _check(ctx, load_library().hj_join_batch(ctx.handle, n, ra, sa, ctypes.byref(o), outs))
    if raw:
        return outs
    res = []
    for j in range(n):
        r = hj_result()
        ctypes.pointer(r)[0] = outs[j]
        res.append(_result(ctx, r))
    return res


def hj_results_free(ctx: Context, outs: ctypes.Array, n: int | None = None):
    """Free the first n results of an hj_result array (all of them by default)."""
    lib = load_library()
    for j in range(len(outs) if n is None else n):
        _check(ctx, lib.hj_result_free(ctx.handle, ctypes.byref(outs[j])))


def check_pairs_buffer(pairs: torch.Tensor | None, R: torch.Tensor) -> int:
    """Rows of a caller-owned pair buffer: None, or a contiguous (m, 2) CUDA tensor
    of R's dtype on R's device (anything else could let the join write past its
    end).  Raises ValueError otherwise."""
    if pairs is None:
        return 0
    if not isinstance(pairs, torch.Tensor):
        raise ValueError("pairs must be a torch tensor or None")
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be an (m, 2) tensor")
    if pairs.dtype != R.dtype:
        raise ValueError(f"pairs must have the relations' dtype {R.dtype}, not {pairs.dtype}")
    if not pairs.is_contiguous():
        raise ValueError("pairs must be contiguous")
    if not pairs.is_cuda or pairs.device != R.device:
        raise ValueError(f"pairs must be a CUDA tensor on {R.device}")
    return int(pairs.shape[0])


def hj_join_static(R: torch.Tensor, S: torch.Tensor, pairs: torch.Tensor | None, stream=None):
    """The allocation-free SHJ: pairs land in the caller's (m, 2) CUDA tensor of R's
    dtype.  The work is ordered on `stream`, by default torch's current stream of R's
    device (so it follows the kernels that made R and S).  Returns (count, (c0, c1));
    raises HJError on a non-OK status (count is then in .count for HJ_E_OVERFLOW)."""
    if not R.is_cuda or S.device != R.device:
        raise ValueError("R and S must be CUDA tensors on one device")
    r, s = rel_of(R), rel_of(S)
    cap = check_pairs_buffer(pairs, R)
    cnt = ctypes.c_uint64()
    chk = (ctypes.c_uint64 * 2)()
    ptr = pairs.data_ptr() if cap else None
    if stream is None:
        stream = torch.cuda.current_stream(R.device)
    st = load_library().hj_join_static(ctypes.byref(r), ctypes.byref(s), stream_handle(stream), ptr, cap,
                                       ctypes.byref(cnt), chk)
    if st != HJ_OK:
        e = HJError(st, "hj_join_static failed")
        e.count = int(cnt.value)
        raise e
    return int(cnt.value), (int(chk[0]), int(chk[1]))


def hj_join_coproc(ctx: Context, R: torch.Tensor, S: torch.Tensor, cpu_share: float, cpu_threads: int = 0,
                   mode: int = HJ_MATERIALIZE, radix_bits: int = 0, passes: int = 0, out_capacity: int = 0,
                   checksum: bool = False):
    """PHJ with the join step divided between the GPU and the host CPU (see
    include/hj.h).  Returns (Result, times dict in seconds)."""
    r, s = rel_of(R), rel_of(S)
    o = _opts(HJ_ALGO_PHJ, mode, radix_bits, passes, out_capacity, checksum)
    out = hj_result()
    t = (ctypes.c_double * 5)()
    _check(ctx, load_library().hj_join_coproc(ctx.handle, ctypes.byref(r), ctypes.byref(s), ctypes.byref(o),
                                              float(cpu_share), int(cpu_threads), ctypes.byref(out), t))
    names = ("partition_gpu", "join_gpu", "copy_to_host", "join_cpu", "total")
    return _result(ctx, out), {k: float(v) for k, v in zip(names, t)}


def hj_split(ctx: Context, rel: torch.Tensor, nparts: int, out: torch.Tensor | None = None):
    """Group the tuples of `rel` by the sharding hash into `nparts` groups (see
    include/hj.h).  Returns (grouped (n, 2) tensor on rel's device, offsets: list of
    nparts + 1 ints); `out` (same shape and dtype as rel, on its device) is used
    when given."""
    r = rel_of(rel)
    if out is None:
        out = torch.empty_like(rel)
    elif out.shape != rel.shape or out.dtype != rel.dtype or not out.is_contiguous() or out.device != rel.device:
        raise ValueError("out must be a contiguous tensor of rel's shape, dtype and device")
    offs = (ctypes.c_uint64 * (nparts + 1))()
    _check(ctx, load_library().hj_split(ctx.handle, ctypes.byref(r), nparts, out.data_ptr() if out.numel() else None,
                                        offs))
    return out, [int(x) for x in offs]


def hj_result_free(ctx: Context, res: Result):
    res.free()


def hj_partition(ctx: Context, rel: torch.Tensor, b1: int, b2: int = 0):
    """Radix-partition a relation; returns (tuples as numpy (n, 2) array, offsets numpy)."""
    import numpy as np

    r = rel_of(rel)
    out = hj_rel()
    off = ctypes.c_void_p()
    lib = load_library()
    _check(ctx, lib.hj_partition(ctx.handle, ctypes.byref(r), b1, b2, ctypes.byref(out), ctypes.byref(off)))
    try:
        dt = np.uint32 if r.width == 4 else np.uint64
        tup = np.empty((r.n, 2), dt)
        offs = np.empty((1 << (b1 + b2)) + 1, np.uint64)
        if r.n:
            _check(ctx, lib.hj_copy(ctx.handle, tup.ctypes.data, out.tuples, tup.nbytes))
        _check(ctx, lib.hj_copy(ctx.handle, offs.ctypes.data, off, offs.nbytes))
    finally:
        lib.hj_partition_free(ctx.handle, ctypes.byref(out), off)
    return tup, offs


def hj_sync(ctx: Context):
    _check(ctx, load_library().hj_sync(ctx.handle))


def prof_enable(ctx: Context, on: bool = True):
    _check(ctx, load_library().hj_prof_enable(ctx.handle, 1 if on else 0))


def _dbl(xs):
    return (ctypes.c_double * len(xs))(*[float(v) for v in xs])


def hj_coproc_time(x, cpu_s, gpu_s, ratios, xfer_s: float = 0.0) -> tuple[float, float, float]:
    """The co-processing cost model for per-step CPU ratios (host only): (T, T_CPU, T_GPU)."""
    n = len(x)
    t, tc, tg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = load_library().hj_coproc_time(n, _dbl(x), _dbl(cpu_s), _dbl(gpu_s), xfer_s, _dbl(ratios), ctypes.byref(t),
                                       ctypes.byref(tc), ctypes.byref(tg))
    if st != HJ_OK:
        raise HJError(st, "hj_coproc_time failed")
    return t.value, tc.value, tg.value


def hj_coproc_ratios(x, cpu_s, gpu_s, xfer_s: float = 0.0, delta: float = 0.02) -> tuple[list, float]:
    """The per-step CPU ratios minimising the cost model's time, and that time (host only)."""
    n = len(x)
    r = (ctypes.c_double * n)()
    t = ctypes.c_double()
    st = load_library().hj_coproc_ratios(n, _dbl(x), _dbl(cpu_s), _dbl(gpu_s), xfer_s, delta, r, ctypes.byref(t))
    if st != HJ_OK:
        raise HJError(st, "hj_coproc_ratios failed")
    return list(r), t.value


def prof_only(ctx: Context, name: str | None = None):
    """Bracket only launches of kernel `name` with events (None: every launch)."""
    _check(ctx, load_library().hj_prof_only(ctx.handle, name.encode() if name else None))


def prof_reset(ctx: Context):
    _check(ctx, load_library().hj_prof_reset(ctx.handle))


def prof_read(ctx: Context) -> dict:
    """{kernel name: (launches, total device ms)} since the last reset."""
    lib = load_library()
    n = ctypes.c_int()
    _check(ctx, lib.hj_prof_read(ctx.handle, None, 0, ctypes.byref(n)))
    arr = (hj_prof_entry * max(n.value, 1))()
    _check(ctx, lib.hj_prof_read(ctx.handle, arr, n.value, ctypes.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(n.value)}


def launch_count(ctx: Context) -> int:
    return int(load_library().hj_launch_count(ctx.handle))


# ------------------------------------------------------------------- serving


@dataclass
class Times:
    submit: float
    admit: float
    start: float
    done: float


class Server:
    """An hj_server: submit joins from any thread, collect them with poll / wait.
    The relations of a request are kept referenced until it is collected."""

    def __init__(self, ctx: Context, budget: int = 0, workers: int = 0, max_wave: int = 0, wave_tuples: int = 0,
                 graph: bool = False):
        lib = load_library()
        h = ctypes.c_void_p()
        o = hj_server_opts(budget, workers, max_wave, wave_tuples, HJ_FLAG_GRAPH if graph else 0)
        _check(ctx, lib.hj_server_create(ctypes.byref(h), ctx.handle, ctypes.byref(o)))
        self.handle, self.ctx = h, ctx
        self._keep = {}

    def _check(self, st):
        if st != HJ_OK:
            msg = load_library().hj_server_last_error(self.handle)
            raise HJError(st, msg.decode() if msg else "")

    def submit(self, R: torch.Tensor, S: torch.Tensor, mode: int = HJ_MATERIALIZE, sync: bool = True) -> int:
        """Queue a join.  The server's workers run on streams of their own, so R and S
        must be complete: with sync (the default) torch's current stream is
        synchronised first; pass sync=False for inputs known to be ready."""
        if sync:
            torch.cuda.current_stream(R.device).synchronize()
        r, s = rel_of(R), rel_of(S)
        rid = ctypes.c_uint64()
        self._check(load_library().hj_server_submit(self.handle, ctypes.byref(r), ctypes.byref(s), mode,
                                                    ctypes.byref(rid)))
        self._keep[rid.value] = (R, S)
        return int(rid.value)

    def _collect(self, st, rid, res, t):
        if st == HJ_E_PENDING:
            return None
        self._keep.pop(rid, None)
        self._check(st)
        out = _result(self.ctx, res)
        out._server = self
        return out, Times(t.submit, t.admit, t.start, t.done)

    def poll(self, rid: int):
        """None while the request runs, else (Result, Times)."""
        res, t = hj_result(), hj_req_times()
        st = load_library().hj_server_poll(self.handle, rid, ctypes.byref(res), ctypes.byref(t))
        return self._collect(st, rid, res, t)

    def wait(self, rid: int, timeout: float = -1.0):
        """Block until the request is done (None on timeout); returns (Result, Times)."""
        res, t = hj_result(), hj_req_times()
        st = load_library().hj_server_wait(self.handle, rid, timeout, ctypes.byref(res), ctypes.byref(t))
        return self._collect(st, rid, res, t)

    def _free(self, raw: hj_result):
        self._check(load_library().hj_server_result_free(self.handle, ctypes.byref(raw)))

    def stats(self) -> dict:
        st = hj_server_stats()
        self._check(load_library().hj_server_stats_get(self.handle, ctypes.byref(st)))
        return {n: int(getattr(st, n)) for n, _ in hj_server_stats._fields_}

    def close(self):
        if self.handle:
            load_library().hj_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def hj_server_create(ctx: Context, **kw) -> Server:
    return Server(ctx, **kw)


def hj_server_submit(srv: Server, R: torch.Tensor, S: torch.Tensor, mode: int = HJ_MATERIALIZE) -> int:
    return srv.submit(R, S, mode)


def hj_server_poll(srv: Server, rid: int):
    return srv.poll(rid)


def hj_server_wait(srv: Server, rid: int, timeout: float = -1.0):
    return srv.wait(rid, timeout)


def hj_server_result_free(srv: Server, res: Result):
    res.free()


def hj_server_stats_get(srv: Server) -> dict:
    return srv.stats()


def hj_server_destroy(srv: Server):
    srv.close()
