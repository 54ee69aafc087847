"""ctypes binding of ``libmgardgb.so`` (the C ABI in ``include/mgard_gb.h``).

Argument marshalling only: every step of the transform runs in the CUDA
library.  The ``mgard_*`` functions mirror the C entry points one to one
(plain integers for device pointers and streams); the short helpers below
them take CUDA torch tensors and the current torch stream.  There is no CPU
path: a missing library, a CPU tensor or a non-zero return code raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgardgb.so")

F32, F64 = 0, 1
OK = 0
ERRORS = {
    -1: "MGARD_ERR_ARG", -2: "MGARD_ERR_SHAPE", -3: "MGARD_ERR_COORDS", -4: "MGARD_ERR_LEVEL",
    -5: "MGARD_ERR_WORKSPACE", -6: "MGARD_ERR_OVERFLOW", -7: "MGARD_ERR_NONFINITE",
    -8: "MGARD_ERR_CUDA", -9: "MGARD_ERR_TIMEOUT",
}

# Every symbol the header declares, with its ctypes signature.
_I64P = ctypes.POINTER(ctypes.c_int64)
_DPP = ctypes.POINTER(ctypes.POINTER(ctypes.c_double))
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_SIGNATURES = {
    "mgard_num_levels": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.POINTER(ctypes.c_int)]),
    "mgard_workspace_size": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "mgard_level_tolerances": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int,
                                              ctypes.c_double, _DP]),
    "mgard_decompose": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                       _VP, _VP, ctypes.c_size_t, _VP]),
    "mgard_recompose": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                       _VP, _VP, ctypes.c_size_t, _VP]),
    "mgard_level_tolerances_mode": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_double)]),
    "mgard_quantize_levels": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_double), _VP, _VP, _VP]),
    "mgard_dequantize_levels": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP,
                                               _VP, _VP]),
    "mgard_lorenzo_encode": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                            _VP, _VP]),
    "mgard_lorenzo_decode": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                            _VP, _VP]),
    "mgard_pack_bound": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "mgard_pack_labels": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t), _VP]),
    "mgard_unpack_labels": (ctypes.c_int, [_VP, ctypes.c_size_t, ctypes.c_int64, _VP, _VP]),
    "mgard_compress_host_packed": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, _VP, _VP, ctypes.c_size_t,
                                                  ctypes.POINTER(ctypes.c_size_t),
                                                  ctypes.POINTER(ctypes.c_double), _VP, _VP, _VP,
                                                  ctypes.c_size_t, _VP, ctypes.c_size_t, _VP]),
    "mgard_decompress_host_packed": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_double, _VP,
                                                    ctypes.c_size_t, _VP, _VP, _VP, _VP,
                                                    ctypes.c_size_t, _VP, ctypes.c_size_t, _VP]),
    "mgard_level_grid": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, _I64P,
                                        ctypes.POINTER(ctypes.c_double)]),
    "mgard_recompose_partial": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "mgard_iso_area": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, _VP, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double), _VP]),
    "mgard_decompose_adaptive": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int,
                                                ctypes.c_double, _VP, _VP, ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_double), _VP]),
    "mgard_quantize": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, _VP, _VP, _DP, _VP]),
    "mgard_quantize_async": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, _VP, _VP, _DP, _VP]),
    "mgard_quantize_status": (ctypes.c_int, [ctypes.c_void_p]),
    "mgard_value_range_async": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _VP, _VP, _VP]),
    "mgard_quantize_rel_async": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, _VP, _VP, _VP, _VP]),
    "mgard_dequantize_rel": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, _VP, _VP, _VP, _VP]),
    "mgard_dequantize": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _VP, _VP, _VP]),
    "mgard_value_range": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, _VP, _DP, _VP]),
    "mgard_decompose_host": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                            _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "mgard_recompose_host": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                            _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "mgard_compress_host": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, _VP, _VP, _DP, _VP, _VP, _VP,
                                           ctypes.c_size_t, _VP]),
    "mgard_decompress_host": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, _VP, _VP, _VP, _VP, _VP,
                                             ctypes.c_size_t, _VP]),
    "mgard_num_levels_4d": (ctypes.c_int, [_I64P, ctypes.POINTER(ctypes.c_int)]),
    "mgard_workspace_size_4d": (ctypes.c_int, [_I64P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "mgard_level_tolerances_4d": (ctypes.c_int, [_I64P, _DPP, ctypes.c_int, ctypes.c_double, _DP]),
    "mgard_decompose_4d": (ctypes.c_int, [_I64P, _DPP, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                          ctypes.c_size_t, _VP]),
    "mgard_recompose_4d": (ctypes.c_int, [_I64P, _DPP, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                          ctypes.c_size_t, _VP]),
    "mgard_quantize_4d": (ctypes.c_int, [_I64P, _DPP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         _VP, _VP, _DP, _VP]),
    "mgard_dequantize_4d": (ctypes.c_int, [_I64P, _DPP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           _VP, _VP, _VP]),
    "mgard_huffman_bound": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "mgard_huffman_encode": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t), _VP]),
    "mgard_huffman_decode": (ctypes.c_int, [_VP, ctypes.c_size_t, ctypes.c_int64, _VP, _VP]),
    "mgard_label_entropy": (ctypes.c_int, [ctypes.c_int64, _VP, _DP, _VP]),
    "mgard_huffman_lengths": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint8)]),
    "mgard_cost_model": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_int, _DP, ctypes.c_double, _DP]),
    "mgard_release_plans": (ctypes.c_int, []),
    "mgard_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mgard_decompose_noalloc": (ctypes.c_int, [ctypes.c_int, _I64P, _DPP, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                               ctypes.c_void_p]),
    "mgard_batch_workspace_size": (ctypes.c_int, [ctypes.c_int, _I64P,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "mgard_batch_decompose": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.POINTER(_VP), _VP,
                                             ctypes.c_size_t, _VP]),
    "mgard_batch_recompose": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.POINTER(_VP), _VP,
                                             ctypes.c_size_t, _VP]),
    "mgard_batch_autotune": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.POINTER(_VP), _VP,
                                            ctypes.c_size_t, _VP, ctypes.POINTER(ctypes.c_int)]),
    "mgard_batch_release": (ctypes.c_int, []),
    "mgard_trace_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]),
    "mgard_batch_wait_selftest": (ctypes.c_int, [ctypes.c_int64, _VP]),
    "mgard_batch_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "mgard_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_VP)]),
    "mgard_server_submit": (ctypes.c_int, [_VP, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "mgard_server_poll": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]),
    "mgard_server_drain": (ctypes.c_int, [_VP, ctypes.c_double]),
    "mgard_server_counters": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "mgard_server_destroy": (ctypes.c_int, [_VP]),
    "mgard_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "mgard_trace_select": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mgard_trace_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), _I64P, _DP, _DP,
                                        ctypes.POINTER(ctypes.c_int)]),
    "mgard_trace_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "mgard_trace_kernel_launches": (ctypes.c_int64, []),
}

_lib = None


class MgardError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        name = ERRORS.get(code, str(code))
        msg = _lib.mgard_error_string(code).decode() if _lib is not None else name
        super().__init__(f"{what}: {name} ({msg})" if what else f"{name} ({msg})")


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


# ------------------------------------------------------------ marshalling ---

class _Shape:
    """dims / coords as C arrays, kept alive for the duration of a call."""

    def __init__(self, dims, coords=None):
        dims = [int(n) for n in dims]
        self.ndim = len(dims)
        self.dims = (ctypes.c_int64 * self.ndim)(*dims)
        if coords is None:
            self.coords = None
            self._keep = []
        else:
            if len(coords) != self.ndim:
                raise ValueError("one coordinate array (or None) per axis")
            self._keep = [None if c is None else np.ascontiguousarray(c, dtype=np.float64)
                          for c in coords]
            arr = (ctypes.POINTER(ctypes.c_double) * self.ndim)()
            for d, c in enumerate(self._keep):
                arr[d] = (ctypes.cast(c.ctypes.data, ctypes.POINTER(ctypes.c_double))
                          if c is not None else ctypes.POINTER(ctypes.c_double)())
            self.coords = ctypes.cast(arr, _DPP)
            self._arr = arr


def _check(rc: int, what: str):
    if rc != OK:
        raise MgardError(rc, what)


def mgard_num_levels(dims) -> int:
    s = _Shape(dims)
    L = ctypes.c_int()
    _check(lib().mgard_num_levels(s.ndim, s.dims, ctypes.byref(L)), "mgard_num_levels")
    return L.value


def mgard_workspace_size(dims, dtype: int) -> int:
    s = _Shape(dims)
    b = ctypes.c_size_t()
    _check(lib().mgard_workspace_size(s.ndim, s.dims, dtype, ctypes.byref(b)), "mgard_workspace_size")
    return b.value


def mgard_level_tolerances(dims, coords, stop_level: int, tau: float) -> np.ndarray:
    s = _Shape(dims, coords)
    out = np.zeros(mgard_num_levels(dims) + 1)
    _check(lib().mgard_level_tolerances(s.ndim, s.dims, s.coords, stop_level, float(tau),
                                        out.ctypes.data_as(_DP)), "mgard_level_tolerances")
    return out


def mgard_decompose(dims, coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_decompose(s.ndim, s.dims, s.coords, dtype, stop_level, data_ptr, ws_ptr,
                                 ws_bytes, stream)


def mgard_decompose_adaptive(dims, coords, dtype, tau_linf, data_ptr, ws_ptr, ws_bytes, stream):
    """Adaptive decomposition.  Returns (rc, stop_level, sums) with sums an
    (L + 1) x 2 array of (E_Lorenzo, E_interp) per level (NaN: not sampled)."""
    s = _Shape(dims, coords)
    L = mgard_num_levels(dims)
    stop = ctypes.c_int(-1)
    sums = (ctypes.c_double * (2 * (L + 1)))()
    rc = lib().mgard_decompose_adaptive(s.ndim, s.dims, s.coords, dtype, float(tau_linf), data_ptr,
                                        ws_ptr, ws_bytes, ctypes.byref(stop), sums, stream)
    return rc, stop.value, np.array(sums[:], dtype=np.float64).reshape(L + 1, 2)


def mgard_decompose_noalloc(dims, coords, dtype, stop_level, data_ptr, stream,
                            wait: bool = False):
    """Allocation-free decomposition (static device scratch).  Returns
    (rc, timed_out); with wait=False timed_out is None and the call does not
    wait for the stream."""
    s = _Shape(dims, coords)
    flag = ctypes.c_int(0)
    rc = lib().mgard_decompose_noalloc(s.ndim, s.dims, s.coords, dtype, stop_level, data_ptr,
                                       ctypes.byref(flag) if wait else None, stream)
    return rc, (bool(flag.value) if wait else None)


class _Batch:
    """Marshalled arguments of the batched calls: sizes and data pointers."""

    def __init__(self, shapes, ptrs):
        self.n = len(shapes)
        flat = [int(v) for shp in shapes for v in shp]
        if any(len(shp) != 3 for shp in shapes):
            raise ValueError("batched fields are 3D")
        self.dims = (ctypes.c_int64 * max(len(flat), 1))(*flat)
        self.ptrs = (_VP * max(self.n, 1))(*[int(p) for p in ptrs])


def mgard_batch_workspace_size(shapes) -> int:
    b = _Batch(shapes, [0] * len(shapes))
    out = ctypes.c_size_t()
    _check(lib().mgard_batch_workspace_size(b.n, b.dims, ctypes.byref(out)),
           "mgard_batch_workspace_size")
    return out.value


def mgard_batch_decompose(shapes, ptrs, ws_ptr, ws_bytes, stream) -> int:
    b = _Batch(shapes, ptrs)
    return lib().mgard_batch_decompose(b.n, b.dims, b.ptrs, ws_ptr, ws_bytes, stream)


def mgard_batch_recompose(shapes, ptrs, ws_ptr, ws_bytes, stream) -> int:
    b = _Batch(shapes, ptrs)
    return lib().mgard_batch_recompose(b.n, b.dims, b.ptrs, ws_ptr, ws_bytes, stream)


def mgard_batch_autotune(shapes, ptrs, ws_ptr, ws_bytes, stream):
    b = _Batch(shapes, ptrs)
    choice = (ctypes.c_int * 4)()
    rc = lib().mgard_batch_autotune(b.n, b.dims, b.ptrs, ws_ptr, ws_bytes, stream, choice)
    return rc, tuple(choice)


BATCH_KINDS = ("load_vector_dec", "load_vector_rec", "solve_contig_bulk", "solve_contig",
               "solve_segmented", "finish")


def mgard_batch_stats():
    """Per tile kind of the last batched launch: (tiles, wait cycles, run cycles)."""
    out = (ctypes.c_uint64 * 18)()
    _check(lib().mgard_batch_stats(out, 18), "mgard_batch_stats")
    return {k: (out[3 * i], out[3 * i + 1], out[3 * i + 2]) for i, k in enumerate(BATCH_KINDS)}


def mgard_batch_release() -> int:
    return lib().mgard_batch_release()


def mgard_batch_wait_selftest(limit_ns: int, stream) -> int:
    """Run the batched kernel on a schedule whose dependency is never met,
    with a wait limit of limit_ns; the next quantize / value-range call on
    the device reports the timeout."""
    return lib().mgard_batch_wait_selftest(int(limit_ns), stream)


OP_COMPRESS, OP_DECOMPRESS = 1, 2


class MgardRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("ndim", ctypes.c_int), ("dims", ctypes.c_int64 * 3),
                ("dtype", ctypes.c_int), ("stop_level", ctypes.c_int),
                ("rel_bound", ctypes.c_double), ("tau", ctypes.c_double),
                ("host_in", ctypes.c_void_p), ("host_out", ctypes.c_void_p)]


class Server:
    """The serving loop of the library (continuous batching on one device).
    Host buffers are tensors (pinned for overlapped copies) kept alive here
    until their request completes."""

    def __init__(self, hbm_budget: int, slots: int = 8):
        self.h = _VP()
        _check(lib().mgard_server_create(int(hbm_budget), int(slots), ctypes.byref(self.h)),
               "mgard_server_create")
        self._keep = {}

    def submit(self, op, shape, host_in, host_out, rel_bound=0.0, tau=0.0, stop_level=0,
               dtype=None):
        req = MgardRequest()
        req.op = op
        req.ndim = len(shape)
        for i, n in enumerate(shape):
            req.dims[i] = int(n)
        req.dtype = F32 if dtype is None else dtype
        req.stop_level = stop_level
        req.rel_bound = rel_bound
        req.tau = tau
        req.host_in = host_in.data_ptr()
        req.host_out = host_out.data_ptr()
        rid = ctypes.c_int64()
        _check(lib().mgard_server_submit(self.h, ctypes.byref(req), ctypes.byref(rid)),
               "mgard_server_submit")
        self._keep[rid.value] = (host_in, host_out)
        return rid.value

    def poll(self, max_items: int = 4096):
        """Completed requests: list of (id, status, latency_s, tau)."""
        ids = (ctypes.c_int64 * max_items)()
        st = (ctypes.c_int * max_items)()
        lat = (ctypes.c_double * max_items)()
        tau = (ctypes.c_double * max_items)()
        n = ctypes.c_int()
        _check(lib().mgard_server_poll(self.h, max_items, ids, st, lat, tau, ctypes.byref(n)),
               "mgard_server_poll")
        out = [(ids[i], st[i], lat[i], tau[i]) for i in range(n.value)]
        for rid, *_ in out:
            self._keep.pop(rid, None)
        return out

    def drain(self, timeout_s: float = 600.0):
        _check(lib().mgard_server_drain(self.h, float(timeout_s)), "mgard_server_drain")

    def counters(self):
        out = (ctypes.c_int64 * 5)()
        _check(lib().mgard_server_counters(self.h, out), "mgard_server_counters")
        return dict(queued=out[0], running=out[1], bytes_in_use=out[2], peak_running=out[3],
                    peak_bytes=out[4])

    def close(self):
        if self.h:
            lib().mgard_server_destroy(self.h)
            self.h = _VP()


def mgard_recompose(dims, coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_recompose(s.ndim, s.dims, s.coords, dtype, stop_level, data_ptr, ws_ptr,
                                 ws_bytes, stream)


def mgard_decompose_host(dims, coords, dtype, stop_level, host_in, host_out, dev_ptr, ws_ptr,
                         ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_decompose_host(s.ndim, s.dims, s.coords, dtype, stop_level, host_in,
                                      host_out, dev_ptr, ws_ptr, ws_bytes, stream)


def mgard_recompose_host(dims, coords, dtype, stop_level, host_in, host_out, dev_ptr, ws_ptr,
                         ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_recompose_host(s.ndim, s.dims, s.coords, dtype, stop_level, host_in,
                                      host_out, dev_ptr, ws_ptr, ws_bytes, stream)


def mgard_quantize(dims, coords, dtype, stop_level, tau, coeffs_ptr, labels_ptr, stream):
    s = _Shape(dims, coords)
    taus = np.zeros(mgard_num_levels(dims) + 1)
    rc = lib().mgard_quantize(s.ndim, s.dims, s.coords, dtype, stop_level, float(tau), coeffs_ptr,
                              labels_ptr, taus.ctypes.data_as(_DP), stream)
    return rc, taus


def mgard_dequantize(dims, coords, dtype, stop_level, tau, labels_ptr, coeffs_ptr, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_dequantize(s.ndim, s.dims, s.coords, dtype, stop_level, float(tau),
                                  labels_ptr, coeffs_ptr, stream)


def mgard_value_range(count, dtype, data_ptr, stream):
    out = np.zeros(2)
    rc = lib().mgard_value_range(int(count), dtype, data_ptr, out.ctypes.data_as(_DP), stream)
    return rc, out


def mgard_compress_host(dims, coords, dtype, stop_level, rel_bound, host_field_ptr,
                        host_labels_ptr, dev_data_ptr, dev_labels_ptr, ws_ptr, ws_bytes, stream):
    s = _Shape(dims, coords)
    tau = ctypes.c_double()
    rc = lib().mgard_compress_host(s.ndim, s.dims, s.coords, dtype, stop_level, float(rel_bound),
                                   host_field_ptr, host_labels_ptr, ctypes.byref(tau),
                                   dev_data_ptr, dev_labels_ptr, ws_ptr, ws_bytes, stream)
    return rc, tau.value


def mgard_decompress_host(dims, coords, dtype, stop_level, tau, host_labels_ptr, host_field_ptr,
                          dev_data_ptr, dev_labels_ptr, ws_ptr, ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_decompress_host(s.ndim, s.dims, s.coords, dtype, stop_level, float(tau),
                                       host_labels_ptr, host_field_ptr, dev_data_ptr,
                                       dev_labels_ptr, ws_ptr, ws_bytes, stream)


def mgard_compress_host_packed(dims, coords, dtype, stop_level, rel_bound, host_field_ptr,
                               host_stream_ptr, host_capacity, dev_data_ptr, dev_labels_ptr,
                               dev_stream_ptr, dev_capacity, ws_ptr, ws_bytes, stream):
    """Returns (rc, stream_bytes, tau)."""
    s = _Shape(dims, coords)
    tau = ctypes.c_double()
    nb = ctypes.c_size_t()
    rc = lib().mgard_compress_host_packed(s.ndim, s.dims, s.coords, dtype, stop_level,
                                          float(rel_bound), host_field_ptr, host_stream_ptr,
                                          host_capacity, ctypes.byref(nb), ctypes.byref(tau),
                                          dev_data_ptr, dev_labels_ptr, dev_stream_ptr,
                                          dev_capacity, ws_ptr, ws_bytes, stream)
    return rc, nb.value, tau.value


def mgard_decompress_host_packed(dims, coords, dtype, stop_level, tau, host_stream_ptr,
                                 stream_bytes, host_field_ptr, dev_data_ptr, dev_labels_ptr,
                                 dev_stream_ptr, dev_capacity, ws_ptr, ws_bytes, stream) -> int:
    s = _Shape(dims, coords)
    return lib().mgard_decompress_host_packed(s.ndim, s.dims, s.coords, dtype, stop_level,
                                              float(tau), host_stream_ptr, stream_bytes,
                                              host_field_ptr, dev_data_ptr, dev_labels_ptr,
                                              dev_stream_ptr, dev_capacity, ws_ptr, ws_bytes,
                                              stream)


def _shape4(dims, coords):
    if len(dims) != 4:
        raise ValueError("a 4D grid needs four axes")
    return _Shape(dims, coords)


def mgard_num_levels_4d(dims) -> int:
    s = _shape4(dims, None)
    L = ctypes.c_int()
    _check(lib().mgard_num_levels_4d(s.dims, ctypes.byref(L)), "mgard_num_levels_4d")
    return L.value


def mgard_workspace_size_4d(dims, dtype: int) -> int:
    s = _shape4(dims, None)
    b = ctypes.c_size_t()
    _check(lib().mgard_workspace_size_4d(s.dims, dtype, ctypes.byref(b)), "mgard_workspace_size_4d")
    return b.value


def mgard_level_tolerances_4d(dims, coords, stop_level: int, tau: float) -> np.ndarray:
    s = _shape4(dims, coords)
    out = np.zeros(mgard_num_levels_4d(dims) + 1)
    _check(lib().mgard_level_tolerances_4d(s.dims, s.coords, stop_level, float(tau),
                                           out.ctypes.data_as(_DP)), "mgard_level_tolerances_4d")
    return out


def mgard_decompose_4d(dims, coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes, stream) -> int:
    s = _shape4(dims, coords)
    return lib().mgard_decompose_4d(s.dims, s.coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes,
                                    stream)


def mgard_recompose_4d(dims, coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes, stream) -> int:
    s = _shape4(dims, coords)
    return lib().mgard_recompose_4d(s.dims, s.coords, dtype, stop_level, data_ptr, ws_ptr, ws_bytes,
                                    stream)


def mgard_quantize_4d(dims, coords, dtype, stop_level, tau, coeffs_ptr, labels_ptr, stream):
    s = _shape4(dims, coords)
    taus = np.zeros(mgard_num_levels_4d(dims) + 1)
    rc = lib().mgard_quantize_4d(s.dims, s.coords, dtype, stop_level, float(tau), coeffs_ptr,
                                 labels_ptr, taus.ctypes.data_as(_DP), stream)
    return rc, taus


def mgard_dequantize_4d(dims, coords, dtype, stop_level, tau, labels_ptr, coeffs_ptr, stream) -> int:
    s = _shape4(dims, coords)
    return lib().mgard_dequantize_4d(s.dims, s.coords, dtype, stop_level, float(tau), labels_ptr,
                                     coeffs_ptr, stream)


def mgard_release_plans() -> int:
    return lib().mgard_release_plans()


def mgard_trace_enable(on: bool) -> int:
    return lib().mgard_trace_enable(1 if on else 0)


def mgard_trace_select(kind=-1, level=None) -> int:
    """Bracket only the launches of one kernel kind (and level, unless None)
    with events; kind < 0 brackets every launch."""
    rc = lib().mgard_trace_select(int(kind), 0 if level is None else int(level),
                                  1 if level is None else 0)
    _check(rc, "mgard_trace_select")
    return rc


def mgard_trace_fma_rate(dtype: int, stream=None) -> float:
    """Measured FMA throughput (flop/s) of the element type on this device."""
    out = ctypes.c_double()
    _check(lib().mgard_trace_fma_rate(dtype, ctypes.byref(out), _stream(stream)),
           "mgard_trace_fma_rate")
    return out.value


def mgard_trace_kernel_launches() -> int:
    """Kernels launched by the library while tracing was on."""
    return int(lib().mgard_trace_kernel_launches())


def mgard_trace_read():
    """Rows of the kernel timing trace: dicts with kernel name, kind, level,
    launches, total_ms and bytes (algorithmic)."""
    n = ctypes.c_int()
    _check(lib().mgard_trace_read(0, None, None, None, None, None, ctypes.byref(n)),
           "mgard_trace_read")
    m = n.value
    kind = (ctypes.c_int * max(m, 1))()
    level = (ctypes.c_int * max(m, 1))()
    launches = (ctypes.c_int64 * max(m, 1))()
    ms = (ctypes.c_double * max(m, 1))()
    nbytes = (ctypes.c_double * max(m, 1))()
    _check(lib().mgard_trace_read(m, kind, level, launches, ms, nbytes, ctypes.byref(n)),
           "mgard_trace_read")
    return [dict(kernel=lib().mgard_trace_kernel_name(kind[i]).decode(), kind=kind[i],
                 level=level[i], launches=launches[i], total_ms=ms[i], bytes=nbytes[i])
            for i in range(min(m, n.value))]


# ------------------------------------------------------- torch helpers ---

def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}: float32 or float64")


def _cuda_tensor(t, what="tensor"):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous (C order)")
    return t


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def workspace(shape, dtype, device=None):
    """A device workspace tensor of the size mgard_decompose needs."""
    torch = _torch()
    code = dtype if isinstance(dtype, int) else dtype_code(torch.empty(0, dtype=dtype))
    nbytes = mgard_workspace_size(shape, code)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")


def decompose(x, coords=None, stop_level: int = 0, ws=None, stream=None):
    """In-place multilevel decomposition of a CUDA tensor (returns it)."""
    _cuda_tensor(x, "x")
    if ws is None:
        ws = workspace(x.shape, x.dtype, x.device)
    rc = mgard_decompose(x.shape, coords, dtype_code(x), stop_level, x.data_ptr(), ws.data_ptr(),
                         ws.numel(), _stream(stream))
    _check(rc, "mgard_decompose")
    return x


TOL_MODES = {"geometric": 0, "linf_optimal": 1, "l2": 2}


def mgard_level_tolerances_mode(dims, coords, stop_level: int, tau: float, mode: str) -> np.ndarray:
    """Level tolerances for one of the Section 4.1 rules (see TOL_MODES)."""
    s = _Shape(dims, coords)
    L = mgard_num_levels(dims)
    out = (ctypes.c_double * (L + 1))()
    rc = lib().mgard_level_tolerances_mode(s.ndim, s.dims, s.coords, int(stop_level), float(tau),
                                           TOL_MODES[mode], out)
    _check(rc, "mgard_level_tolerances_mode")
    return np.array(out[:], dtype=np.float64)


def quantize_levels(x, taus, coords=None, stop_level: int = 0, labels=None, stream=None):
    """int64 labels of the CUDA tensor x with the given level tolerances."""
    _cuda_tensor(x, "x")
    torch = _torch()
    if labels is None:
        labels = torch.empty(x.shape, dtype=torch.int64, device=x.device)
    t = (ctypes.c_double * len(taus))(*[float(v) for v in taus])
    s = _Shape(x.shape, coords)
    rc = lib().mgard_quantize_levels(s.ndim, s.dims, s.coords, dtype_code(x), int(stop_level), t,
                                     x.data_ptr(), labels.data_ptr(), _stream(stream))
    _check(rc, "mgard_quantize_levels")
    return labels


def dequantize_levels(labels, taus, dtype, coords=None, stop_level: int = 0, out=None, stream=None):
    """Coefficients from int64 CUDA labels with the given level tolerances."""
    _cuda_tensor(labels, "labels")
    torch = _torch()
    if out is None:
        out = torch.empty(labels.shape, dtype=dtype, device=labels.device)
    t = (ctypes.c_double * len(taus))(*[float(v) for v in taus])
    s = _Shape(labels.shape, coords)
    rc = lib().mgard_dequantize_levels(s.ndim, s.dims, s.coords, dtype_code(out), int(stop_level), t,
                                       labels.data_ptr(), out.data_ptr(), _stream(stream))
    _check(rc, "mgard_dequantize_levels")
    return out


def lorenzo(labels, dtype, encode: bool, coords=None, stop_level: int = 0, stream=None):
    """In-place Lorenzo residuals (encode) or their inverse on the coarse block
    of int64 CUDA labels (finest layout); dtype is the field's torch dtype."""
    _cuda_tensor(labels, "labels")
    torch = _torch()
    s = _Shape(labels.shape, coords)
    code = dtype_code(torch.empty(0, dtype=dtype))
    fn = lib().mgard_lorenzo_encode if encode else lib().mgard_lorenzo_decode
    rc = fn(s.ndim, s.dims, s.coords, code, int(stop_level), labels.data_ptr(), _stream(stream))
    _check(rc, "mgard_lorenzo_encode" if encode else "mgard_lorenzo_decode")
    return labels


def pack_bound(count: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().mgard_pack_bound(int(count), ctypes.byref(b)), "mgard_pack_bound")
    return b.value


def pack_labels(labels, stream=None):
    """The packed stream (a CUDA uint8 tensor of its exact size) of the int64
    CUDA tensor `labels`."""
    _cuda_tensor(labels, "labels")
    torch = _torch()
    n = labels.numel()
    out = torch.empty(pack_bound(n), dtype=torch.uint8, device=labels.device)
    nb = ctypes.c_size_t()
    rc = lib().mgard_pack_labels(n, labels.data_ptr(), out.data_ptr(), out.numel(), ctypes.byref(nb),
                                 _stream(stream))
    _check(rc, "mgard_pack_labels")
    return out[:nb.value]


def unpack_labels(stream_bytes, count: int, out=None, stream=None):
    """int64 CUDA labels from a packed CUDA uint8 stream."""
    _cuda_tensor(stream_bytes, "stream")
    torch = _torch()
    if out is None:
        out = torch.empty(int(count), dtype=torch.int64, device=stream_bytes.device)
    rc = lib().mgard_unpack_labels(stream_bytes.data_ptr(), stream_bytes.numel(), int(count),
                                   out.data_ptr(), _stream(stream))
    _check(rc, "mgard_unpack_labels")
    return out


def level_grid(dims, coords, level: int):
    """(shape, coords) of the level-`level` grid of the hierarchy of `dims`:
    the shape tuple and a list of per-axis coordinate arrays."""
    s = _Shape(dims, coords)
    shape = (ctypes.c_int64 * s.ndim)()
    rc = lib().mgard_level_grid(s.ndim, s.dims, s.coords, int(level), shape, None)
    _check(rc, "mgard_level_grid")
    out = (ctypes.c_double * int(sum(shape[:])))()
    rc = lib().mgard_level_grid(s.ndim, s.dims, s.coords, int(level), shape, out)
    _check(rc, "mgard_level_grid")
    vals, o, axes = np.array(out[:], dtype=np.float64), 0, []
    for n in shape[:]:
        axes.append(vals[o:o + n].copy())
        o += n
    return tuple(int(n) for n in shape[:]), axes


def recompose_partial(x, level: int, coords=None, stop_level: int = 0, ws=None, stream=None):
    """Q_k u on the level-k grid (a new CUDA tensor) from the decomposed CUDA
    tensor x (left unchanged)."""
    _cuda_tensor(x, "x")
    torch = _torch()
    shape, _ = level_grid(x.shape, coords, level)
    out = torch.empty(shape, dtype=x.dtype, device=x.device)
    if ws is None:
        ws = workspace(shape, x.dtype, x.device)
    s = _Shape(x.shape, coords)
    rc = lib().mgard_recompose_partial(s.ndim, s.dims, s.coords, dtype_code(x), int(stop_level),
                                       int(level), x.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                       ws.numel(), _stream(stream))
    _check(rc, "mgard_recompose_partial")
    return out


def iso_area(x, iso: float, coords=None, stream=None) -> float:
    """Iso-surface area of the 3D CUDA tensor x at `iso` (marching tetrahedra)."""
    _cuda_tensor(x, "x")
    s = _Shape(x.shape, coords)
    a = ctypes.c_double()
    rc = lib().mgard_iso_area(s.ndim, s.dims, s.coords, dtype_code(x), x.data_ptr(), float(iso),
                              ctypes.byref(a), _stream(stream))
    _check(rc, "mgard_iso_area")
    return a.value


def decompose_adaptive(x, tau_linf: float, coords=None, ws=None, stream=None):
    """In-place adaptive decomposition of a 3D CUDA tensor (Algorithm 1):
    returns (stop_level, sums) with the chosen stopping level and the sampled
    (E_Lorenzo, E_interp) per level."""
    _cuda_tensor(x, "x")
    if ws is None:
        ws = workspace(x.shape, x.dtype, x.device)
    rc, stop, sums = mgard_decompose_adaptive(x.shape, coords, dtype_code(x), tau_linf, x.data_ptr(),
                                              ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "mgard_decompose_adaptive")
    return stop, sums


def decompose_noalloc(x, coords=None, stop_level: int = 0, stream=None, wait: bool = False):
    """In-place decomposition of a CUDA tensor without any allocation by the
    library (static scratch; small fields only).  Returns x."""
    _cuda_tensor(x, "x")
    rc, _ = mgard_decompose_noalloc(x.shape, coords, dtype_code(x), stop_level, x.data_ptr(),
                                    _stream(stream), wait)
    _check(rc, "mgard_decompose_noalloc")
    return x


def batch_workspace(fields):
    """A device workspace tensor for the batched calls on these fields."""
    torch = _torch()
    nbytes = mgard_batch_workspace_size([tuple(f.shape) for f in fields])
    return torch.empty(nbytes, dtype=torch.uint8, device=fields[0].device)


def _batch_args(fields):
    for f in fields:
        _cuda_tensor(f, "field")
        if f.dtype != _torch().float32 or f.dim() != 3:
            raise ValueError("batched fields are 3D float32 CUDA tensors")
    return [tuple(f.shape) for f in fields], [f.data_ptr() for f in fields]


def batch_decompose(fields, ws=None, stream=None):
    """Decompose every tensor of `fields` in place in one persistent launch."""
    shapes, ptrs = _batch_args(fields)
    if ws is None:
        ws = batch_workspace(fields)
    _check(mgard_batch_decompose(shapes, ptrs, ws.data_ptr(), ws.numel(), _stream(stream)),
           "mgard_batch_decompose")
    return fields


def batch_recompose(fields, ws=None, stream=None):
    """Recompose every tensor of `fields` in place in one persistent launch."""
    shapes, ptrs = _batch_args(fields)
    if ws is None:
        ws = batch_workspace(fields)
    _check(mgard_batch_recompose(shapes, ptrs, ws.data_ptr(), ws.numel(), _stream(stream)),
           "mgard_batch_recompose")
    return fields


def batch_autotune(fields, ws, stream=None):
    """Pick the tile shapes for these fields (their contents are kept)."""
    shapes, ptrs = _batch_args(fields)
    rc, choice = mgard_batch_autotune(shapes, ptrs, ws.data_ptr(), ws.numel(), _stream(stream))
    _check(rc, "mgard_batch_autotune")
    return choice


def recompose(x, coords=None, stop_level: int = 0, ws=None, stream=None):
    """In-place multilevel recomposition of a CUDA tensor (returns it)."""
    _cuda_tensor(x, "x")
    if ws is None:
        ws = workspace(x.shape, x.dtype, x.device)
    rc = mgard_recompose(x.shape, coords, dtype_code(x), stop_level, x.data_ptr(), ws.data_ptr(),
                         ws.numel(), _stream(stream))
    _check(rc, "mgard_recompose")
    return x


def quantize(coeffs, tau: float, coords=None, stop_level: int = 0, labels=None, stream=None):
    """Level-wise labels (int64 CUDA tensor) and the tolerances tau_0..tau_L."""
    torch = _torch()
    _cuda_tensor(coeffs, "coeffs")
    if labels is None:
        labels = torch.empty(coeffs.shape, dtype=torch.int64, device=coeffs.device)
    rc, taus = mgard_quantize(coeffs.shape, coords, dtype_code(coeffs), stop_level, tau,
                              coeffs.data_ptr(), labels.data_ptr(), _stream(stream))
    _check(rc, "mgard_quantize")
    return labels, taus


def quantize_async(coeffs, tau: float, coords=None, stop_level: int = 0, labels=None, stream=None):
    """quantize without waiting: the labels are enqueued on the stream and
    their flags gathered until quantize_status."""
    torch = _torch()
    _cuda_tensor(coeffs, "coeffs")
    if labels is None:
        labels = torch.empty(coeffs.shape, dtype=torch.int64, device=coeffs.device)
    s = _Shape(coeffs.shape, coords)
    taus = np.zeros(mgard_num_levels(coeffs.shape) + 1)
    rc = lib().mgard_quantize_async(s.ndim, s.dims, s.coords, dtype_code(coeffs), int(stop_level),
                                    float(tau), coeffs.data_ptr(), labels.data_ptr(),
                                    taus.ctypes.data_as(_DP), _stream(stream))
    _check(rc, "mgard_quantize_async")
    return labels, taus


def quantize_status(stream=None):
    """Wait for the stream and raise if any asynchronous quantization since
    the last check met a non-finite coefficient, an overflow or a timeout."""
    _check(lib().mgard_quantize_status(_stream(stream)), "mgard_quantize_status")


def value_range_async(x, range_out=None, stream=None):
    """min and max of a CUDA tensor into a device float64 tensor of 2, without waiting."""
    torch = _torch()
    _cuda_tensor(x, "x")
    if range_out is None:
        range_out = torch.empty(2, dtype=torch.float64, device=x.device)
    rc = lib().mgard_value_range_async(x.numel(), dtype_code(x), x.data_ptr(),
                                       range_out.data_ptr(), _stream(stream))
    _check(rc, "mgard_value_range_async")
    return range_out


def quantize_rel_async(coeffs, rel: float, range_dev, coords=None, stop_level: int = 0,
                       labels=None, stream=None):
    """Labels with tau = rel x (max - min) of the device range, without waiting."""
    torch = _torch()
    _cuda_tensor(coeffs, "coeffs")
    if labels is None:
        labels = torch.empty(coeffs.shape, dtype=torch.int64, device=coeffs.device)
    s = _Shape(coeffs.shape, coords)
    rc = lib().mgard_quantize_rel_async(s.ndim, s.dims, s.coords, dtype_code(coeffs),
                                        int(stop_level), float(rel), range_dev.data_ptr(),
                                        coeffs.data_ptr(), labels.data_ptr(), _stream(stream))
    _check(rc, "mgard_quantize_rel_async")
    return labels


def dequantize_rel(labels, rel: float, range_dev, dtype, coords=None, stop_level: int = 0,
                   out=None, stream=None):
    """Bin centres with tau = rel x (max - min) of the device range."""
    torch = _torch()
    _cuda_tensor(labels, "labels")
    if out is None:
        out = torch.empty(labels.shape, dtype=dtype, device=labels.device)
    s = _Shape(labels.shape, coords)
    rc = lib().mgard_dequantize_rel(s.ndim, s.dims, s.coords, dtype_code(out), int(stop_level),
                                    float(rel), range_dev.data_ptr(), labels.data_ptr(),
                                    out.data_ptr(), _stream(stream))
    _check(rc, "mgard_dequantize_rel")
    return out


def dequantize(labels, tau: float, dtype, coords=None, stop_level: int = 0, out=None, stream=None):
    torch = _torch()
    _cuda_tensor(labels, "labels")
    if out is None:
        out = torch.empty(labels.shape, dtype=dtype, device=labels.device)
    rc = mgard_dequantize(labels.shape, coords, dtype_code(out), stop_level, tau,
                          labels.data_ptr(), out.data_ptr(), _stream(stream))
    _check(rc, "mgard_dequantize")
    return out


def value_range(x, stream=None):
    """(min, max) of a CUDA tensor, computed on the device."""
    _cuda_tensor(x, "x")
    rc, out = mgard_value_range(x.numel(), dtype_code(x), x.data_ptr(), _stream(stream))
    _check(rc, "mgard_value_range")
    return float(out[0]), float(out[1])


# ---------------------------------------------------------------- 4D grids ---

def workspace_4d(shape, dtype, device=None):
    """A device workspace tensor of the size the 4D transform needs."""
    torch = _torch()
    code = dtype if isinstance(dtype, int) else dtype_code(torch.empty(0, dtype=dtype))
    nbytes = mgard_workspace_size_4d(shape, code)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")


def decompose_4d(x, coords=None, stop_level: int = 0, ws=None, stream=None):
    """In-place multilevel decomposition of a 4D CUDA tensor (returns it)."""
    _cuda_tensor(x, "x")
    if ws is None:
        ws = workspace_4d(x.shape, x.dtype, x.device)
    _check(mgard_decompose_4d(x.shape, coords, dtype_code(x), stop_level, x.data_ptr(),
                              ws.data_ptr(), ws.numel(), _stream(stream)), "mgard_decompose_4d")
    return x


def recompose_4d(x, coords=None, stop_level: int = 0, ws=None, stream=None):
    """In-place multilevel recomposition of a 4D CUDA tensor (returns it)."""
    _cuda_tensor(x, "x")
    if ws is None:
        ws = workspace_4d(x.shape, x.dtype, x.device)
    _check(mgard_recompose_4d(x.shape, coords, dtype_code(x), stop_level, x.data_ptr(),
                              ws.data_ptr(), ws.numel(), _stream(stream)), "mgard_recompose_4d")
    return x


def quantize_4d(coeffs, tau: float, coords=None, stop_level: int = 0, labels=None, stream=None):
    """Level-wise labels of a 4D u_mc and the tolerances tau_0..tau_L."""
    torch = _torch()
    _cuda_tensor(coeffs, "coeffs")
    if labels is None:
        labels = torch.empty(coeffs.shape, dtype=torch.int64, device=coeffs.device)
    rc, taus = mgard_quantize_4d(coeffs.shape, coords, dtype_code(coeffs), stop_level, tau,
                                 coeffs.data_ptr(), labels.data_ptr(), _stream(stream))
    _check(rc, "mgard_quantize_4d")
    return labels, taus


def dequantize_4d(labels, tau: float, dtype, coords=None, stop_level: int = 0, out=None,
                  stream=None):
    torch = _torch()
    _cuda_tensor(labels, "labels")
    if out is None:
        out = torch.empty(labels.shape, dtype=dtype, device=labels.device)
    _check(mgard_dequantize_4d(labels.shape, coords, dtype_code(out), stop_level, tau,
                               labels.data_ptr(), out.data_ptr(), _stream(stream)),
           "mgard_dequantize_4d")
    return out


# ------------------------------------------------- entropy stage of labels ---

def huffman_bound(count: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().mgard_huffman_bound(int(count), ctypes.byref(b)), "mgard_huffman_bound")
    return b.value


def huffman_encode(labels, stream=None):
    """The Huffman stream (a CUDA uint8 tensor of its exact size) of the int64
    CUDA tensor `labels`."""
    _cuda_tensor(labels, "labels")
    torch = _torch()
    n = labels.numel()
    out = torch.empty(huffman_bound(n), dtype=torch.uint8, device=labels.device)
    nb = ctypes.c_size_t()
    rc = lib().mgard_huffman_encode(n, labels.data_ptr(), out.data_ptr(), out.numel(),
                                    ctypes.byref(nb), _stream(stream))
    _check(rc, "mgard_huffman_encode")
    return out[:nb.value]


def huffman_decode(stream_bytes, count: int, out=None, stream=None):
    """Labels (int64 CUDA tensor of `count`) from a device Huffman stream."""
    torch = _torch()
    _cuda_tensor(stream_bytes, "stream")
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=stream_bytes.device)
    rc = lib().mgard_huffman_decode(stream_bytes.data_ptr(), stream_bytes.numel(), int(count),
                                    out.data_ptr(), _stream(stream))
    _check(rc, "mgard_huffman_decode")
    return out


def label_entropy(labels, stream=None) -> float:
    """Order-0 entropy of the labels in bits per label."""
    _cuda_tensor(labels, "labels")
    h = ctypes.c_double()
    _check(lib().mgard_label_entropy(labels.numel(), labels.data_ptr(), ctypes.byref(h),
                                     _stream(stream)), "mgard_label_entropy")
    return h.value


def huffman_lengths(counts) -> np.ndarray:
    """Code lengths for symbol counts (host only)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.zeros(c.size, dtype=np.uint8)
    _check(lib().mgard_huffman_lengths(c.size, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
           "mgard_huffman_lengths")
    return out


def cost_model(dims, stop_level: int, taus, value_range: float) -> float:
    """Section 4.1's estimated label cost in bits (host only)."""
    s = _Shape(dims)
    t = np.ascontiguousarray(taus, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib().mgard_cost_model(s.ndim, s.dims, stop_level, t.ctypes.data_as(_DP),
                                  float(value_range), ctypes.byref(out)), "mgard_cost_model")
    return out.value
