"""ctypes binding of libgscl.so (include/gscl.h): argument marshalling only.

Every sweep and reduction runs in the library's CUDA kernels; PyTorch only
supplies device memory (grid buffers, reduction workspaces) and streams.
There is no fallback: if the library is missing or a call fails, an
exception is raised.

Terms are tuples ``(dx, dy, dz, in, coef, out, w)`` (Section 3: an operator
reads fixed offsets of its input grids around the core element, writes the
core element of its outputs and may return a value); ``VALUE`` as ``in``
reads the operator's value, as ``out`` adds to it; ``NONE`` as ``coef``
means no coefficient grid.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import torch

from . import build as _build

VALUE = 254
NONE = 255
F64, F32, BF16 = 0, 1, 2
SUM, MAXABS, L2 = 0, 1, 2

_DTYPES = {
    "f64": (F64, torch.float64, 8),
    "f32": (F32, torch.float32, 4),
    "bf16": (BF16, torch.bfloat16, 2),
}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gscl.h")


class Term(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int8), ("dy", ctypes.c_int8), ("dz", ctypes.c_int8),
                ("in_", ctypes.c_uint8), ("coef", ctypes.c_uint8), ("out", ctypes.c_uint8),
                ("reserved", ctypes.c_uint16), ("w", ctypes.c_double)]


class StencilC(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("terms", ctypes.POINTER(Term))]


class RangeC(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3)]


class GridDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("halo", ctypes.c_int32 * 3), ("elem_bytes", ctypes.c_int32),
                ("pitch_elems", ctypes.c_int64), ("offset_elems", ctypes.c_int64),
                ("plane_elems", ctypes.c_int64), ("bytes", ctypes.c_int64), ("dev_buf", ctypes.c_void_p)]


class GsclError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__(f"gscl status {status}: {detail}")


_lib = None


def declared_symbols():
    """Names of the functions include/gscl.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(gscl_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Loads libgscl.so (building it first if its sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    P, i32, i64, vp = ctypes.POINTER, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    u64 = ctypes.c_uint64
    sig = {
        "gscl_grid_layout": [i32, P(i64), P(i32), i32, P(i64), P(i64), P(i64)],
        "gscl_grid_create": [i32, P(i64), P(i32), i32, vp, i64, P(u64)],
        "gscl_grid_destroy": [u64],
        "gscl_grid_info": [u64, P(GridDesc)],
        "gscl_grid_copy_from_host": [u64, vp, vp],
        "gscl_grid_copy_to_host": [u64, vp, vp],
        "gscl_swap": [P(u64), P(u64)],
        "gscl_do_all": [P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), i32, vp],
        "gscl_do_reduce": [i32, P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), P(ctypes.c_double), i32,
                           vp, i64, vp],
        "gscl_sync": [vp],
        "gscl_do_reduce_noalloc": [i32, P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), P(ctypes.c_double),
                                   i32, vp],
        "gscl_convert": [u64, u64, ctypes.c_double, i32, P(RangeC), vp],
        "gscl_tune_sweeps": [P(StencilC), P(u64), i32, P(u64), i32, i32, vp, P(i32)],
        "gscl_fma_throughput": [i32, i32, P(ctypes.c_double), vp],
        "gscl_do_ordered": [i32, P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), vp],
        "gscl_ordered_specialization": [i32, P(StencilC), P(u64), i32, P(u64), i32, P(i32)],
        "gscl_do_colored": [P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), i32, i32, vp],
        "gscl_do_diamond": [P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), vp],
        "gscl_program_create": [ctypes.c_char_p, i32, i32, i32, P(i32), P(u64)],
        "gscl_program_destroy": [u64],
        "gscl_selftest_bounded_wait": [vp],
        "gscl_do_all_program": [u64, P(u64), i32, P(u64), i32, P(RangeC), i32, vp],
        "gscl_do_reduce_program": [u64, i32, P(u64), i32, P(u64), i32, P(RangeC), P(ctypes.c_double), i32, vp,
                                   i64, vp],
        "gscl_batch_tile": [u64, P(i32), P(i32)],
        "gscl_batch_temporal": [u64, P(i32), P(i32), P(i32)],
        "gscl_batch_set_temporal": [u64, i32, i32],
        "gscl_set_fp64_arithmetic": [i32],
        "gscl_get_fp64_arithmetic": [],
        "gscl_do_reduce_within": [P(StencilC), P(u64), i32, P(u64), i32, P(RangeC), ctypes.c_double,
                                  P(ctypes.c_double), i32, vp, i64, vp],
        "gscl_batch_create": [P(StencilC), i32, P(u64), i32, P(u64), i32, P(u64)],
        "gscl_batch_destroy": [u64],
        "gscl_batch_info": [u64, P(i32), P(i32), P(i32)],
        "gscl_batch_run": [u64, i32, i32, vp],
        "gscl_batch_create_colored": [P(StencilC), i32, P(u64), i32, P(u64), i32, P(u64)],
        "gscl_batch_run_colored": [u64, i32, i32, i32, vp],
        "gscl_batch_reduce": [u64, i32, vp, vp],
        "gscl_batch_tune": [u64, i32, vp, P(i32), P(i32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.gscl_stencil_specialization.argtypes = [P(StencilC), i32, i32]
    L.gscl_stencil_specialization.restype = i32
    L.gscl_reduce_workspace_bytes.argtypes = []
    L.gscl_reduce_workspace_bytes.restype = ctypes.c_int64
    L.gscl_status_str.argtypes = [ctypes.c_int]
    L.gscl_status_str.restype = ctypes.c_char_p
    L.gscl_last_error.argtypes = []
    L.gscl_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status):
    if status != 0:
        L = lib()
        raise GsclError(status, f"{L.gscl_status_str(status).decode()}: {L.gscl_last_error().decode()}")


def stream_ptr(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Stencil:
    """A stencil operator marshalled once for repeated calls."""

    def __init__(self, terms):
        self.terms = [tuple(t) for t in terms]
        arr = (Term * max(1, len(self.terms)))()
        for i, (dx, dy, dz, a, c, m, w) in enumerate(self.terms):
            arr[i] = Term(int(dx), int(dy), int(dz), int(a), int(c), int(m), 0, float(w))
        self._arr = arr
        self.c = StencilC(len(self.terms), 0, ctypes.cast(arr, ctypes.POINTER(Term)))


def as_stencil(op):
    if op is None or isinstance(op, Stencil):
        return op
    return Stencil(op)


def specialization(op, n_in, n_out):
    """Id of the compiled operator structure the library will use, or -1 (generic kernel)."""
    st = as_stencil(op)
    return lib().gscl_stencil_specialization(ctypes.byref(st.c), n_in, n_out)


def layout(n, halo, dtype="f64", ndim=3):
    p, o, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().gscl_grid_layout(ndim, (ctypes.c_int64 * 3)(*n), (ctypes.c_int32 * 3)(*halo),
                                 _DTYPES[dtype][0], ctypes.byref(p), ctypes.byref(o), ctypes.byref(b)))
    return p.value, o.value, b.value


class Grid:
    """A device grid: a torch-allocated buffer wrapped by a library handle.

    ``n = (nx, ny, nz)`` interior points, ``halo = (hx, hy, hz)``; a 2D grid has
    ``nz = 1, hz = 0`` and ``ndim = 2``."""

    def __init__(self, n, halo, dtype="f64", ndim=None, device=None):
        n = tuple(int(v) for v in n)
        halo = tuple(int(v) for v in halo)
        if ndim is None:
            ndim = 2 if (n[2] == 1 and halo[2] == 0) else 3
        self.n, self.halo, self.dtype, self.ndim = n, halo, dtype, ndim
        self.pitch, self.off, self.bytes = layout(n, halo, dtype, ndim)
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.empty(self.bytes, dtype=torch.uint8, device=dev)
        h = ctypes.c_uint64()
        check(lib().gscl_grid_create(ndim, (ctypes.c_int64 * 3)(*n), (ctypes.c_int32 * 3)(*halo),
                                     _DTYPES[dtype][0], ctypes.c_void_p(self.buf.data_ptr()), self.bytes,
                                     ctypes.byref(h)))
        self.handle = h.value

    def __del__(self):
        h = getattr(self, "handle", 0)
        if h and _lib is not None:
            _lib.gscl_grid_destroy(h)
            self.handle = 0

    @property
    def padded_shape(self):
        nx, ny, nz = self.n
        hx, hy, hz = self.halo
        return (nz + 2 * hz, ny + 2 * hy, nx + 2 * hx)

    @property
    def torch_dtype(self):
        return _DTYPES[self.dtype][1]

    def info(self):
        d = GridDesc()
        check(lib().gscl_grid_info(self.handle, ctypes.byref(d)))
        return d

    def view(self):
        """Strided torch view (halo included) of the storage this handle names now."""
        Z, Y, X = self.padded_shape
        t = self.buf.view(self.torch_dtype)
        return t.as_strided((Z, Y, X), (self.pitch * Y, self.pitch, 1), self.off)

    def interior(self):
        nx, ny, nz = self.n
        hx, hy, hz = self.halo
        return self.view()[hz:hz + nz, hy:hy + ny, hx:hx + nx]

    def zero(self, stream=None):
        """Sets every cell (halo included) to zero on the device: a memset of
        the grid's buffer, without a host copy."""
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            self.buf.zero_()
        return self

    def upload(self, host, stream=None):
        """Copies a dense host array (halo included) through gscl_grid_copy_from_host."""
        t = host if isinstance(host, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(host))
        t = t.to(self.torch_dtype).contiguous()
        if tuple(t.shape) != self.padded_shape:
            raise ValueError(f"host array shape {tuple(t.shape)} != {self.padded_shape}")
        check(lib().gscl_grid_copy_from_host(self.handle, ctypes.c_void_p(t.data_ptr()), stream_ptr(stream)))
        (stream or torch.cuda.current_stream()).synchronize()
        return self

    def download(self, stream=None) -> torch.Tensor:
        """Dense host copy (halo included) through gscl_grid_copy_to_host."""
        t = torch.empty(self.padded_shape, dtype=self.torch_dtype)
        check(lib().gscl_grid_copy_to_host(self.handle, ctypes.c_void_p(t.data_ptr()), stream_ptr(stream)))
        (stream or torch.cuda.current_stream()).synchronize()
        return t


def _resync(grids):
    """After the library exchanged storage between handles, make each Python
    Grid hold the torch buffer its handle now names."""
    by_ptr = {g.buf.data_ptr(): g.buf for g in grids}
    want = [(g, g.info().dev_buf) for g in grids]
    for g, ptr in want:
        if ptr != g.buf.data_ptr():
            g.buf = by_ptr[ptr]


def swap(a: Grid, b: Grid):
    """Section 5.2's swap_grids: exchanges the storage the two handles name."""
    ha, hb = ctypes.c_uint64(a.handle), ctypes.c_uint64(b.handle)
    check(lib().gscl_swap(ctypes.byref(ha), ctypes.byref(hb)))
    a.buf, b.buf = b.buf, a.buf


def _range(rng):
    if rng is None:
        return None
    lo, hi = rng
    return ctypes.byref(RangeC((ctypes.c_int64 * 3)(*lo), (ctypes.c_int64 * 3)(*hi)))


def _handles(grids):
    return (ctypes.c_uint64 * max(1, len(grids)))(*[g.handle for g in grids])


def do_all(op, ins, outs, rng=None, sweeps=1, stream=None):
    """gscl_do_all: applies the operator over the range (Section 3, do_all)."""
    st = as_stencil(op)
    check(lib().gscl_do_all(ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs), len(outs),
                            _range(rng), int(sweeps), stream_ptr(stream)))
    if sweeps > 1:
        _resync([ins[0], outs[0]])


_workspaces = {}


def workspace(stream=None):
    """A zeroed reduction workspace per (device, stream)."""
    s = stream or torch.cuda.current_stream()
    key = (s.device.index, s.cuda_stream)
    ws = _workspaces.get(key)
    if ws is None:
        ws = torch.zeros(lib().gscl_reduce_workspace_bytes(), dtype=torch.uint8, device=s.device)
        _workspaces[key] = ws
    return ws


def do_reduce(reduce_op, op, ins, outs=(), rng=None, result=None, stream=None):
    """gscl_do_reduce: reduces the operator's returned value (Section 3, do_reduce).

    ``result`` None: returns the value as a Python float (the call syncs).
    ``result`` a one-element float64 CUDA tensor (or a slice of one): written
    asynchronously, and the call returns None."""
    st = as_stencil(op)
    ws = workspace(stream)
    on_host = result is None
    if on_host:
        host = ctypes.c_double(0.0)
        rptr = ctypes.pointer(host)
    else:
        if result.dtype != torch.float64 or not result.is_cuda:
            raise ValueError("result must be a float64 CUDA tensor")
        rptr = ctypes.cast(ctypes.c_void_p(result.data_ptr()), ctypes.POINTER(ctypes.c_double))
    check(lib().gscl_do_reduce(int(reduce_op), ctypes.byref(st.c) if st is not None else None, _handles(ins),
                               len(ins), _handles(outs), len(outs), _range(rng), rptr, int(on_host),
                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream_ptr(stream)))
    return host.value if on_host else None


I_INC, I_DEC, J_INC, J_DEC, K_INC, K_DEC = range(6)


def do_ordered(order, op, ins, outs, rng=None, stream=None):
    """gscl_do_ordered: ordered iteration space (Section 3), ``order`` one of
    J_INC, J_DEC, K_INC, K_DEC.  An output passed also as an input is read at
    the element visited just before (a recurrence along the column)."""
    st = as_stencil(op)
    check(lib().gscl_do_ordered(int(order), ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs), len(outs),
                                _range(rng), stream_ptr(stream)))


class Program:
    """gscl_program_create: a point operator given as CUDA C++ statements
    (reads in0(dx, dy, dz) .., the index i, j, k; assigns out0 ..), compiled at
    run time for grids of ``dtype``; ``reach`` bounds every read's offset."""

    def __init__(self, body, n_in, n_out, dtype="f64", reach=(1, 1, 1)):
        h = ctypes.c_uint64()
        r = (ctypes.c_int32 * 3)(*[int(v) for v in reach])
        check(lib().gscl_program_create(body.encode(), int(n_in), int(n_out), _DTYPES[dtype][0], r,
                                        ctypes.byref(h)))
        self.handle = h.value
        self.n_in, self.n_out, self.dtype = n_in, n_out, dtype

    def __del__(self):
        h = getattr(self, "handle", 0)
        if h and _lib is not None:
            _lib.gscl_program_destroy(h)

    def run(self, ins, outs, rng=None, sweeps=1, stream=None):
        """gscl_do_all_program."""
        check(lib().gscl_do_all_program(self.handle, _handles(ins), len(ins), _handles(outs), len(outs), _range(rng),
                                        int(sweeps), stream_ptr(stream)))

    def reduce(self, reduce_op, ins, outs=(), rng=None, result=None, stream=None):
        """gscl_do_reduce_program: reduces the body's ``value`` over the range
        (outputs written as by run).  ``result`` as in do_reduce."""
        ws = workspace(stream)
        on_host = result is None
        if on_host:
            host = ctypes.c_double(0.0)
            rptr = ctypes.pointer(host)
        else:
            rptr = ctypes.cast(ctypes.c_void_p(result.data_ptr()), ctypes.POINTER(ctypes.c_double))
        check(lib().gscl_do_reduce_program(self.handle, int(reduce_op), _handles(ins), len(ins), _handles(outs),
                                           len(outs), _range(rng), rptr, 1 if on_host else 0,
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), stream_ptr(stream)))
        return host.value if on_host else None


def do_diamond(op, ins, outs, rng=None, stream=None):
    """gscl_do_diamond: (i-1, j) and (i, j-1) processed before (i, j)
    (Section 3), plane by plane.  An output passed also as an input is read
    updated at offsets dx, dy <= 0 and not yet updated at dx, dy >= 0."""
    st = as_stencil(op)
    check(lib().gscl_do_diamond(ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs), len(outs), _range(rng),
                                stream_ptr(stream)))


def do_colored(op, ins, outs, color=0, half_sweeps=1, rng=None, stream=None):
    """gscl_do_colored: the operator at the elements whose index sum i + j + k
    has parity ``color`` (Section 3, red-black colouring), ``half_sweeps``
    times with alternating colour.  In place (an output also passed as an
    input) when it reads that grid only at offset 0 or at odd offsets."""
    st = as_stencil(op)
    check(lib().gscl_do_colored(ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs), len(outs),
                                _range(rng), int(color), int(half_sweeps), stream_ptr(stream)))


def ordered_specialization(order, op, ins, outs):
    """gscl_ordered_specialization: the compiled recurrence id (>= 0) that
    do_ordered uses for this call, -1 for the interpreted loop with look-ahead
    loads, -2 for the interpreted loop with loads per term."""
    st = as_stencil(op)
    shape = ctypes.c_int32()
    check(lib().gscl_ordered_specialization(int(order), ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs),
                                            len(outs), ctypes.byref(shape)))
    return shape.value


def do_reduce_within(eps, op, ins, outs=(), rng=None, result=None, stream=None):
    """gscl_do_reduce_within: 1.0 if every |value| <= eps over the range (the
    logical_and convergence test of Section 5.2), else 0.0.  Same ``result``
    convention as do_reduce."""
    st = as_stencil(op)
    ws = workspace(stream)
    on_host = result is None
    if on_host:
        host = ctypes.c_double(0.0)
        rptr = ctypes.pointer(host)
    else:
        if result.dtype != torch.float64 or not result.is_cuda:
            raise ValueError("result must be a float64 CUDA tensor")
        rptr = ctypes.cast(ctypes.c_void_p(result.data_ptr()), ctypes.POINTER(ctypes.c_double))
    check(lib().gscl_do_reduce_within(ctypes.byref(st.c) if st is not None else None, _handles(ins), len(ins),
                                      _handles(outs), len(outs), _range(rng), ctypes.c_double(eps), rptr,
                                      int(on_host), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      stream_ptr(stream)))
    return host.value if on_host else None


def do_reduce_noalloc(reduce_op, op, ins, outs=(), rng=None, result=None, stream=None):
    """gscl_do_reduce_noalloc: do_reduce with the library's built-in scratch
    instead of a workspace, for callers that cannot allocate device memory.
    Same ``result`` convention as do_reduce."""
    st = as_stencil(op)
    on_host = result is None
    if on_host:
        host = ctypes.c_double(0.0)
        rptr = ctypes.pointer(host)
    else:
        if result.dtype != torch.float64 or not result.is_cuda:
            raise ValueError("result must be a float64 CUDA tensor")
        rptr = ctypes.cast(ctypes.c_void_p(result.data_ptr()), ctypes.POINTER(ctypes.c_double))
    check(lib().gscl_do_reduce_noalloc(int(reduce_op), ctypes.byref(st.c) if st is not None else None,
                                       _handles(ins), len(ins), _handles(outs), len(outs), _range(rng), rptr,
                                       int(on_host), stream_ptr(stream)))
    return host.value if on_host else None


FP64_IEEE, FP64_PAIR = 0, 1


def set_fp64_arithmetic(mode):
    """gscl_set_fp64_arithmetic: "ieee" (default) or "pair" (FP64 grids
    evaluated in pairs of FP32 numbers, off the FP64 pipe)."""
    check(lib().gscl_set_fp64_arithmetic({"ieee": FP64_IEEE, "pair": FP64_PAIR}[mode]))


def get_fp64_arithmetic():
    return {FP64_IEEE: "ieee", FP64_PAIR: "pair"}[lib().gscl_get_fp64_arithmetic()]


def fma_throughput(dtype="f64", iters=2048, stream=None):
    """gscl_fma_throughput: measured FMA FLOP/s of the device for "f64" / "f32"."""
    out = ctypes.c_double()
    check(lib().gscl_fma_throughput(_DTYPES[dtype][0], int(iters), ctypes.byref(out), stream_ptr(stream)))
    return out.value


def tune_sweeps(op, ins, outs, trial_sweeps=8, stream=None):
    """gscl_tune_sweeps: picks (and remembers) the fastest temporal factor."""
    st = as_stencil(op)
    k = ctypes.c_int32()
    check(lib().gscl_tune_sweeps(ctypes.byref(st.c), _handles(ins), len(ins), _handles(outs), len(outs),
                                 int(trial_sweeps), stream_ptr(stream), ctypes.byref(k)))
    return k.value


def convert(dst, src, alpha=1.0, accumulate=False, rng=None, stream=None):
    """gscl_convert: dst = alpha * src (+ dst), across storage dtypes."""
    check(lib().gscl_convert(dst.handle, src.handle, float(alpha), int(bool(accumulate)), _range(rng),
                             stream_ptr(stream)))


class Batch:
    """A batch: one operator over many independent instances (uneven extents
    allowed), each sweep of all of them in one launch (gscl_batch_*).

    ``instances`` is a list of (ins, outs) grid lists; the batch keeps the
    Grid objects alive and destroys its handle before them."""

    def __init__(self, op, instances):
        self.op = as_stencil(op)
        self.instances = [(list(i), list(o)) for i, o in instances]
        self.n_in = len(self.instances[0][0])
        self.n_out = len(self.instances[0][1])
        ins = [g for i, _ in self.instances for g in i]
        outs = [g for _, o in self.instances for g in o]
        h = ctypes.c_uint64()
        check(lib().gscl_batch_create(ctypes.byref(self.op.c), len(self.instances), _handles(ins), self.n_in,
                                      _handles(outs), self.n_out, ctypes.byref(h)))
        self.handle = h.value
        self._k = 1  # sweeps fused per launch (gscl_batch_temporal)

    def __del__(self):
        h = getattr(self, "handle", 0)
        if h and _lib is not None:
            _lib.gscl_batch_destroy(h)
            self.handle = 0

    def info(self):
        c, s, sp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().gscl_batch_info(self.handle, ctypes.byref(c), ctypes.byref(s), ctypes.byref(sp)))
        return {"ctas": c.value, "segments": s.value, "specialization": sp.value}

    def _launches(self, sweeps):
        """Launches gscl_batch_run takes for ``sweeps`` sweeps: fused passes
        while more than K sweeps remain, single sweeps after, and one launch
        more when that count and ``sweeps`` differ in parity (the library's
        launch plan keeps them of one parity)."""
        k, n, done = self._k, 0, 0
        while done < sweeps:
            done += k if (k > 1 and sweeps - done > k) else 1
            n += 1
        return n + (n - sweeps) % 2

    def run(self, sweeps, graph=False, stream=None):
        check(lib().gscl_batch_run(self.handle, int(sweeps), int(bool(graph)), stream_ptr(stream)))
        if self._launches(int(sweeps)) % 2 == 0:  # the library exchanged in[0] / out[0] storage
            for ins, outs in self.instances:
                ins[0].buf, outs[0].buf = outs[0].buf, ins[0].buf

    def temporal(self):
        """(sweeps per launch, tile_x, tile_y) of the batch (gscl_batch_temporal)."""
        k, x, y = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().gscl_batch_temporal(self.handle, ctypes.byref(k), ctypes.byref(x), ctypes.byref(y)))
        self._k = k.value
        return k.value, x.value, y.value

    def set_temporal(self, sweeps_per_launch, tile_shape=0):
        """gscl_batch_set_temporal: fuse ``sweeps_per_launch`` sweeps per launch
        (2D batches under a 5-point operator: up to 16, tiles of shape
        ``tile_shape``, 0..3: 32 x 16, 32 x 32, 16 x 16, 64 x 32; 3D FP32 /
        BF16 batches under a 7-point star operator: 2)."""
        check(lib().gscl_batch_set_temporal(self.handle, int(sweeps_per_launch), int(tile_shape)))
        self.temporal()

    def reduce(self, reduce_op, results, stream=None):
        """Per-instance reduction into ``results`` (float64 CUDA tensor of n_inst)."""
        if results.dtype != torch.float64 or not results.is_cuda or results.numel() < len(self.instances):
            raise ValueError("results must be a float64 CUDA tensor with one entry per instance")
        check(lib().gscl_batch_reduce(self.handle, int(reduce_op), ctypes.c_void_p(results.data_ptr()),
                                      stream_ptr(stream)))

    def tile(self):
        """(tile_x, tile_y) of the batch's launches (gscl_batch_tile)."""
        x, y = ctypes.c_int32(), ctypes.c_int32()
        check(lib().gscl_batch_tile(self.handle, ctypes.byref(x), ctypes.byref(y)))
        return x.value, y.value

    def tune(self, trial_sweeps=3, stream=None):
        w, p = ctypes.c_int32(), ctypes.c_int32()
        check(lib().gscl_batch_tune(self.handle, int(trial_sweeps), stream_ptr(stream), ctypes.byref(w),
                                    ctypes.byref(p)))
        self.temporal()
        return w.value, p.value


class ColoredBatch(Batch):
    """A coloured batch (gscl_batch_create_colored): red-black sweeps of many
    instances, every half-sweep of all of them in one launch, each instance
    with its own operator (``ops[i]``: the structure of ``ops[0]``, its own
    weights) and updated in place."""

    def __init__(self, ops, instances):
        self.ops = [as_stencil(o) for o in ops]
        self.instances = [(list(i), list(o)) for i, o in instances]
        if len(self.ops) != len(self.instances):
            raise ValueError("one operator per instance")
        self.n_in = len(self.instances[0][0])
        self.n_out = len(self.instances[0][1])
        arr = (StencilC * len(self.ops))(*[o.c for o in self.ops])
        ins = [g for i, _ in self.instances for g in i]
        outs = [g for _, o in self.instances for g in o]
        h = ctypes.c_uint64()
        check(lib().gscl_batch_create_colored(arr, len(self.instances), _handles(ins), self.n_in, _handles(outs),
                                              self.n_out, ctypes.byref(h)))
        self.handle = h.value
        self._k = 1

    def run_colored(self, color=0, half_sweeps=1, graph=False, stream=None):
        """half_sweeps launches, the colour alternating from ``color``."""
        check(lib().gscl_batch_run_colored(self.handle, int(color), int(half_sweeps), int(bool(graph)),
                                           stream_ptr(stream)))


def sync(stream=None):
    """gscl_sync: waits for the stream and reports device-side timeouts."""
    check(lib().gscl_sync(stream_ptr(stream)))
